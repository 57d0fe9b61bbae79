"""Search grids of the oracle: periods, durations, template, phase lattice.

Plain numpy, FP64, one formula per line.  Test infrastructure only.
Transcendental functions go through Python's ``math`` module (the C
library's pow and cbrt), elementary arithmetic through numpy.

Readings of the paper taken here (the paper is silent or garbled on these):

* constants: G M_sun = 1.3271244e20 m^3 s^-2 and R_sun = 6.957e8 m (IAU 2015
  nominal values); one day = 86400 s; all grid formulas in SI units.
* Eq. (C, A) writes ``S * OS``: S is the light-curve baseline in seconds and
  OS the oversampling factor (default 3).
* If a period range is given, f_max = 1/P_min and f_min = 1/P_max replace
  the Roche limit (Eq. f_max) and 2/S (Eq. f_min) in C and N; A keeps S*OS.
* N (Eq. N) is real: N_int = ceil(N) samples i = 1..N_int, kept while
  f_min (1 - 1e-12) <= f_i <= f_max (1 + 1e-12); periods sorted ascending.
* the duration grid spacing is not given (Sect. 2.2.2): one global geometric
  grid q_j = q_lo * ratio^j (ratio 1.1) of T14/P with q_lo = k_min P_max^(-2/3);
  a period uses the j with k_min P^(-2/3) <= q_j <= min(q_cap, k_max P^(-2/3))
  (Eqs. upper/lower).  D_j = max(1, round(q_j n)), half away from zero;
  equal D inside one period keep the first j.
* the template shape is not given (TLS uses an empirical Kepler shape): a
  central, small-planet transit with quadratic limb darkening,
  s_k = 1 - u1 (1 - mu) - u2 (1 - mu)^2, mu = sqrt(1 - (2x - 1)^2),
  x = (k + 1/2) / D for k = 0..D-1.
* phase (Eq. phase) is evaluated exactly on a time lattice of 2^-e days:
  d_i = rint((t_i - t_ref) 2^e), P_int = rint(P 2^e), rho_i = d_i mod P_int,
  phase p_i = rho_i / P_int, with t_ref = min(t).  e is the largest value
  <= 40 that keeps P_int below 2^(63 - idx_bits), idx_bits = bits of n - 1.
"""

from __future__ import annotations

import math

import numpy as np

GM_SUN = 1.3271244e20
R_SUN = 6.957e8
DAY = 86400.0


def roche_f_max(m_star=1.0, r_star=1.0):
    """Eq. (f_max): 1/(2 pi) sqrt(G M / (3 R)^3), in Hz."""
    gm = GM_SUN * m_star
    r = R_SUN * r_star
    return math.sqrt(gm / (3.0 * r) ** 3) / (2.0 * math.pi)


def ofir_frequencies(baseline_days, m_star=1.0, r_star=1.0, oversampling=3.0,
                     period_min_days=None, period_max_days=None):
    """Cubic frequency sampling, Eqs. (f_i), (C, A), (N).  Returns Hz, ascending."""
    s = baseline_days * DAY
    gm = GM_SUN * m_star
    r = R_SUN * r_star
    f_min = 2.0 / s if not period_max_days else 1.0 / (period_max_days * DAY)
    f_max = roche_f_max(m_star, r_star) if not period_min_days else \
        1.0 / (period_min_days * DAY)
    a = math.pow(2.0 * math.pi, 2.0 / 3.0) / math.pi * r / math.cbrt(gm) / (s * oversampling)
    c = math.cbrt(f_min) - a / 3.0
    n_real = (math.cbrt(f_max) - math.cbrt(f_min) + a / 3.0) * 3.0 / a
    n_int = int(math.ceil(n_real))
    i = np.arange(1, n_int + 1, dtype=np.float64)
    x = a / 3.0 * i + c
    f = x * x * x
    keep = (f >= f_min * (1.0 - 1e-12)) & (f <= f_max * (1.0 + 1e-12))
    return f[keep], dict(A=a, C=c, N=n_real, f_min=f_min, f_max=f_max)


def period_grid_days(baseline_days, **kw):
    """Trial periods in days, ascending (index 0 = shortest)."""
    f, _ = ofir_frequencies(baseline_days, **kw)
    p = 1.0 / (f * DAY)
    return np.sort(p)


def duration_grid(periods_days, n_points, k_min=20.05, k_max=620.84,
                  q_cap=0.15, ratio=1.1):
    """Global geometric T14/P grid and each period's [jlo, jhi] range.

    Returns (q, D, jlo, jhi): q_j, D_j = max(1, round(q_j n)) and, per
    period, the first and last admissible j (Eqs. upper/lower, cap).
    """
    p_s = np.asarray(periods_days, dtype=np.float64) * DAY
    # scalar libm pow per period (numpy's vectorised pow rounds differently)
    p23 = np.array([math.pow(float(v), -2.0 / 3.0) for v in p_s])
    lo = k_min * p23
    hi = np.minimum(q_cap, k_max * p23)
    q_lo = float(lo[int(np.argmax(p_s))])      # k_min P_max^(-2/3)
    q_top = float(hi.max())
    q = []
    j = 0
    while True:
        qj = q_lo * math.pow(ratio, j)
        if qj > q_top:
            break
        q.append(qj)
        j += 1
    q = np.array(q, dtype=np.float64)
    d = np.maximum(1, np.floor(q * n_points + 0.5)).astype(np.int64)
    jlo = np.searchsorted(q, lo, side="left")          # first q_j >= lo
    jhi = np.searchsorted(q, hi, side="right") - 1     # last q_j <= hi
    return q, d, jlo.astype(np.int64), jhi.astype(np.int64)


def kept_durations(d, jlo, jhi):
    """j indices a period searches: ascending, first of equal D kept."""
    out = []
    for j in range(int(jlo), int(jhi) + 1):
        if j > jlo and d[j] == d[j - 1]:
            continue
        out.append(j)
    return out


def template(d, u1=0.4, u2=0.25):
    """Unit-depth transit template of D points (reading of Sect. 2.1)."""
    k = np.arange(d, dtype=np.float64)
    x = (k + 0.5) / d
    rr = np.abs(2.0 * x - 1.0)
    mu = np.sqrt(1.0 - rr * rr)
    return 1.0 - u1 * (1.0 - mu) - u2 * (1.0 - mu) ** 2


def t0_stride(d, dt0):
    """Eq. (N_skip) with the floor reading: max(1, floor(D dt0))."""
    return max(1, int(math.floor(d * dt0)))


def time_quantum_exponent(n_points, period_max_days):
    """Exponent e of the 2^-e-day phase lattice (see module docstring)."""
    idx_bits = max(1, int(n_points - 1).bit_length())
    rho_bits = 64 - idx_bits
    m, ex = math.frexp(float(period_max_days))   # P = m 2^ex, m in [0.5, 1)
    ceil_log2 = ex - 1 if m == 0.5 else ex
    return min(40, rho_bits - 1 - ceil_log2), idx_bits


def phase_lattice(t, periods_days, e):
    """d_i, P_int and t_ref of the exact phase lattice."""
    t = np.asarray(t, dtype=np.float64)
    t_ref = float(t.min())
    scale = math.ldexp(1.0, e)
    d = np.rint((t - t_ref) * scale).astype(np.int64)
    p_int = np.rint(np.asarray(periods_days, dtype=np.float64) * scale).astype(np.int64)
    return d, p_int, t_ref

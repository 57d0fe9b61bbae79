"""Driver of the FP64 oracle (test infrastructure only).

``plan(...)`` builds the grids with :mod:`oracle.grid`; ``search_periods``
runs the C core (``tls_oracle.c``) on a set of period indices; ``sr_sde``
reduces a full chi2(P) spectrum to SR, SDE_raw and SDE (Sect. 2.4).
"""

from __future__ import annotations

import ctypes
import dataclasses
import math
import os
import subprocess
import threading

import numpy as np

from . import grid

_HERE = os.path.dirname(os.path.abspath(__file__))
_BUILD = os.path.join(_HERE, "_build")
_LIB = os.path.join(_BUILD, "libtlsoracle.so")
_SRC = os.path.join(_HERE, "tls_oracle.c")
_lock = threading.Lock()
_lib = None


def build(force: bool = False) -> str:
    """Compile tls_oracle.c with gcc (IEEE FP64: no fast-math, no contraction)."""
    os.makedirs(_BUILD, exist_ok=True)
    if force or not os.path.exists(_LIB) or \
            os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + f".tmp{os.getpid()}"
        cmd = ["gcc", "-O2", "-std=c11", "-ffp-contract=off", "-fno-fast-math",
               "-fopenmp", "-shared", "-fPIC", _SRC, "-o", tmp, "-lm"]
        subprocess.run(cmd, check=True)
        os.replace(tmp, _LIB)
    return _LIB


def _load():
    global _lib
    with _lock:
        if _lib is None:
            lib = ctypes.CDLL(build())
            i64p = np.ctypeslib.ndpointer(np.int64, flags="C")
            f64p = np.ctypeslib.ndpointer(np.float64, flags="C")
            lib.tls_oracle_search.restype = ctypes.c_int
            lib.tls_oracle_search.argtypes = [
                ctypes.c_int64, f64p, f64p, i64p, i64p, i64p, i64p, i64p, i64p,
                f64p, ctypes.c_double, ctypes.c_int64, i64p,
                f64p, i64p, i64p, f64p, i64p, ctypes.c_int]
            lib.tls_oracle_running_median.restype = ctypes.c_int
            lib.tls_oracle_running_median.argtypes = [
                ctypes.c_int64, f64p, ctypes.c_int64, f64p]
            lib.tls_oracle_fold_order.restype = ctypes.c_int
            lib.tls_oracle_fold_order.argtypes = [ctypes.c_int64, i64p, ctypes.c_int64, i64p]
            lib.tls_oracle_period_windows.restype = ctypes.c_int
            lib.tls_oracle_period_windows.argtypes = [
                ctypes.c_int64, f64p, f64p, i64p, ctypes.c_int64, ctypes.c_int64,
                ctypes.c_int64, f64p, ctypes.c_double, f64p, f64p]
            lib.tls_oracle_threads.restype = ctypes.c_int
            lib.tls_oracle_threads.argtypes = [ctypes.c_int]
            _lib = lib
    return _lib


@dataclasses.dataclass
class OraclePlan:
    periods: np.ndarray        # days, ascending
    q: np.ndarray              # T14/P grid
    dur_pts: np.ndarray        # D_j
    jlo: np.ndarray
    jhi: np.ndarray
    tmpl_off: np.ndarray
    tmpl: np.ndarray
    dt0: float
    e: int                     # phase lattice exponent
    n: int
    baseline_days: float


def plan(n, baseline_days, period_min_days=None, period_max_days=None,
         m_star=1.0, r_star=1.0, oversampling=3.0, k_min=20.05, k_max=620.84,
         q_cap=0.15, dur_ratio=1.1, dt0=0.05, u1=0.4, u2=0.25,
         periods_days=None) -> OraclePlan:
    if periods_days is None:
        periods = grid.period_grid_days(
            baseline_days, m_star=m_star, r_star=r_star, oversampling=oversampling,
            period_min_days=period_min_days, period_max_days=period_max_days)
    else:
        periods = np.sort(np.asarray(periods_days, dtype=np.float64))
    q, d, jlo, jhi = grid.duration_grid(periods, n, k_min=k_min, k_max=k_max,
                                        q_cap=q_cap, ratio=dur_ratio)
    offs = np.zeros(d.size, dtype=np.int64)
    parts = []
    pos = 0
    for j, dj in enumerate(d):
        offs[j] = pos
        parts.append(grid.template(int(dj), u1, u2))
        pos += int(dj)
    tmpl = np.concatenate(parts) if parts else np.zeros(0)
    e, _ = grid.time_quantum_exponent(n, float(periods.max()))
    return OraclePlan(periods, q, d, jlo, jhi, offs, tmpl, dt0, e, n,
                      baseline_days)


@dataclasses.dataclass
class PeriodResults:
    sel: np.ndarray
    chi2: np.ndarray
    j_best: np.ndarray
    s_best: np.ndarray
    depth: np.ndarray
    rho_c: np.ndarray
    t0: np.ndarray
    chi2_0: float


def chi2_zero(y, dy):
    """chi2 of the constant model f = 1: sum(((y - 1)/dy)^2)."""
    z = (np.asarray(y, np.float64) - 1.0) / np.asarray(dy, np.float64)
    return float(np.sum(z * z))


def search_periods(p: OraclePlan, t, y, dy, sel=None, n_threads=0) -> PeriodResults:
    t = np.ascontiguousarray(t, np.float64)
    if t.size != p.n:
        raise ValueError("plan was made for a different number of points")
    d_lat, p_int, t_ref = grid.phase_lattice(t, p.periods, p.e)
    return search_periods_lattice(p, d_lat, p_int, t_ref, y, dy, sel, n_threads)


def search_periods_lattice(p: OraclePlan, d_lat, p_int, t_ref, y, dy, sel=None,
                           n_threads=0) -> PeriodResults:
    """search_periods with the phase lattice given: point i of period k has
    phase rho_i = d_lat[i] mod p_int[k] (Eq. phase on the lattice); T0 is
    t_ref + rho_c 2^-e.  Lets a test fold on a lattice of its own."""
    lib = _load()
    y = np.ascontiguousarray(y, np.float64)
    dy = np.ascontiguousarray(dy, np.float64)
    d_lat = np.ascontiguousarray(d_lat, np.int64)
    p_int = np.ascontiguousarray(p_int, np.int64)
    n = y.size
    if n != p.n or d_lat.size != n or p_int.size != p.periods.size:
        raise ValueError("lattice, data and plan sizes differ")
    if sel is None:
        sel = np.arange(p.periods.size, dtype=np.int64)
    sel = np.ascontiguousarray(sel, np.int64)
    k = sel.size
    chi2 = np.empty(k)
    jb = np.empty(k, np.int64)
    sb = np.empty(k, np.int64)
    dep = np.empty(k)
    rho = np.empty(k, np.int64)
    rc = lib.tls_oracle_search(n, y, dy, d_lat, p_int, p.jlo.astype(np.int64),
                               p.jhi.astype(np.int64), p.dur_pts.astype(np.int64),
                               p.tmpl_off, p.tmpl, float(p.dt0), k, sel,
                               chi2, jb, sb, dep, rho, int(n_threads))
    if rc != 0:
        raise MemoryError("oracle allocation failed")
    t0 = t_ref + rho.astype(np.float64) * math.ldexp(1.0, -p.e)
    return PeriodResults(sel, chi2, jb, sb, dep, rho, t0, chi2_zero(y, dy))


def running_median(v, w):
    lib = _load()
    v = np.ascontiguousarray(v, np.float64)
    out = np.empty_like(v)
    if lib.tls_oracle_running_median(v.size, v, int(w), out) != 0:
        raise MemoryError
    return out


def median_window(n_periods):
    """Reading: odd window 2 floor(N_P/200) + 1 (about 1 % of the grid), >= 3."""
    return max(3, 2 * (n_periods // 200) + 1)


def sr_sde(chi2):
    """Signal residue, raw SDE and median-detrended SDE (Sect. 2.4).

    SR(P) = chi2_min / chi2(P) (the Kovacs convention, in (0, 1]; 0/0 := 1),
    SDE_raw = (SR - mean) / std (population std),
    SDE = SDE_raw - running median of SDE_raw.
    A spectrum whose std is at or below 1e-12 is flat up to rounding (every
    depth clamped to zero, say); its SDE_raw and SDE are defined as 0.
    """
    chi2 = np.asarray(chi2, np.float64)
    cmin = float(chi2.min())
    with np.errstate(invalid="ignore", divide="ignore"):
        sr = np.where(chi2 > 0.0, cmin / chi2, 1.0)
    mean = float(np.mean(sr))
    std = float(np.sqrt(np.mean((sr - mean) ** 2)))
    if std > 1e-12:
        raw = (sr - mean) / std
    else:
        raw = np.zeros_like(sr)
    med = running_median(raw, median_window(chi2.size))
    sde = raw - med
    return sr, raw, sde


def refine_selection(sde, k):
    """The k periods with the largest SDE(P), ties by lower index (Sect. 2.5)."""
    sde = np.asarray(sde, np.float64)
    order = np.lexsort((np.arange(sde.size), -sde))
    return np.sort(order[:k])


def full_search(p: OraclePlan, t, y, dy, n_threads=0, refine_top_k=0):
    """Every period, then SR/SDE and the best candidate (argmax SDE).

    With refine_top_k = K > 0 the two-stage T0 search of Sect. 2.5 follows:
    the K best periods by SDE(P) are searched again without skipping T0
    points (step 1), their chi2(P) replace the coarse ones, and SR/SDE are
    computed once more.
    """
    r = search_periods(p, t, y, dy, None, n_threads)
    sr, raw, sde = sr_sde(r.chi2)
    r.refined = np.zeros(r.chi2.size, dtype=bool)
    if refine_top_k > 0:
        sel = refine_selection(sde, min(refine_top_k, r.chi2.size))
        p1 = dataclasses.replace(p, dt0=0.0)      # st = max(1, floor(D * 0)) = 1
        r1 = search_periods(p1, t, y, dy, sel, n_threads)
        r.chi2[sel] = r1.chi2
        r.j_best[sel] = r1.j_best
        r.s_best[sel] = r1.s_best
        r.depth[sel] = r1.depth
        r.rho_c[sel] = r1.rho_c
        r.t0[sel] = r1.t0
        r.refined[sel] = True
        sr, raw, sde = sr_sde(r.chi2)
    b = int(np.argmax(sde))
    j = int(r.j_best[b])
    best = dict(period_idx=b, period=float(p.periods[b]), dur_idx=j,
                dur_points=int(p.dur_pts[j]), duration_days=float(p.q[j] * p.periods[b]),
                t0_idx=int(r.s_best[b]), t0=float(r.t0[b]), depth=float(r.depth[b]),
                sde=float(sde[b]), chi2=float(r.chi2[b]), chi2_min=float(r.chi2.min()),
                chi2_0=r.chi2_0,
                # reading: the paper has no SNR formula; the fit's improvement over
                # the constant model in noise units (matched-filter SNR for white noise)
                snr=math.sqrt(max(0.0, r.chi2_0 - float(r.chi2[b]))))
    return r, sr, raw, sde, best


def threads_used(n_threads=0) -> int:
    return int(_load().tls_oracle_threads(int(n_threads)))


def fold_order(d_lat, p_int):
    """Folded order of one period from the C core (stable by phase)."""
    lib = _load()
    d_lat = np.ascontiguousarray(d_lat, np.int64)
    out = np.empty(d_lat.size, np.int64)
    if lib.tls_oracle_fold_order(d_lat.size, d_lat, int(p_int), out) != 0:
        raise MemoryError
    return out


def period_windows(p: OraclePlan, t, y, dy, period_idx, j):
    """chi2 and depth of every window of (period, duration j), padded decomposition."""
    lib = _load()
    t = np.ascontiguousarray(t, np.float64)
    y = np.ascontiguousarray(y, np.float64)
    dy = np.ascontiguousarray(dy, np.float64)
    d_lat, p_int, _ = grid.phase_lattice(t, p.periods, p.e)
    lo, hi = int(p.jlo[period_idx]), int(p.jhi[period_idx])
    d_m = min(int(p.dur_pts[lo:hi + 1].max()), t.size)
    d = int(p.dur_pts[j])
    s_t = np.ascontiguousarray(p.tmpl[p.tmpl_off[j]:p.tmpl_off[j] + d])
    st = grid.t0_stride(d, p.dt0)
    m = -(-t.size // st)
    chi2 = np.empty(m)
    dep = np.empty(m)
    rc = lib.tls_oracle_period_windows(t.size, y, dy, d_lat, int(p_int[period_idx]),
                                       d_m, d, s_t, float(p.dt0), chi2, dep)
    if rc != 0:
        raise ValueError("bad window request")
    return chi2, dep

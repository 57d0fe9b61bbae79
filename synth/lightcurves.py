"""Seeded synthetic light curves (numpy PCG64 streams).

Every generator returns a :class:`LightCurve` whose ``t`` is in days,
``y`` is normalised flux (1 out of transit) and ``dy`` is the per-point
1-sigma uncertainty.  The ``search`` dict carries the period-search
configuration that goes with the workload (period range, oversampling,
stellar parameters); it is configuration only.

Workloads (sizes and value distributions of the paper's benchmarks, which
used batman light curves and Kepler long-cadence data, Sect. 3):

* ``short_white``  30-day, 30-min cadence, 1440 points, white noise 1e-3,
  one injected transit P=3.7 d, 1000 ppm, 2.5 h.  Grid 0.5-15 d.
* ``kepler_like``  1460-day, 29.4-min cadence (71,510 cadences) with a
  3-day gap at every quarter boundary and 10 % random dropouts, white
  100 ppm + AR(1) red noise (phi 0.9, stationary 30 ppm), injected transit
  P=37 d, 200 ppm, 6 h.  Grid 0.5-730 d.
* ``long_baseline``  3000-day, 30-min cadence, 144,000 points, white
  200 ppm, injected transit P=123.4 d, 300 ppm, 8 h.  Grid 0.5-1500 d.
* ``batch_kepler_like``  many Kepler-like curves of uneven length.

The injected signal is the small-planet, quadratic-limb-darkened transit
profile at zero impact parameter, evaluated in continuous time.
"""

from __future__ import annotations

import dataclasses
import math

import numpy as np

DAY_MIN = 1440.0


@dataclasses.dataclass
class LightCurve:
    t: np.ndarray
    y: np.ndarray
    dy: np.ndarray
    name: str
    seed: int
    injected: dict
    search: dict

    @property
    def n(self) -> int:
        return int(self.t.size)

    @property
    def baseline_days(self) -> float:
        return float(self.t.max() - self.t.min())


def transit_profile(t, period, t0, depth, t14, u1=0.4, u2=0.25):
    """Flux of a periodic limb-darkened transit (1 out of transit).

    Small-planet approximation, central transit: at a distance r (in units
    of the half-duration) from mid-transit the occulted intensity is
    I(mu)/I(1) with mu = sqrt(1 - r^2) and the quadratic law
    I(mu) = 1 - u1 (1 - mu) - u2 (1 - mu)^2.  ``depth`` is the central depth.
    """
    t = np.asarray(t, dtype=np.float64)
    dt = np.mod(t - t0 + 0.5 * period, period) - 0.5 * period
    r = np.abs(dt) / (0.5 * t14)
    inside = r < 1.0
    mu = np.sqrt(np.clip(1.0 - r * r, 0.0, 1.0))
    occ = 1.0 - u1 * (1.0 - mu) - u2 * (1.0 - mu) ** 2
    return 1.0 - np.where(inside, depth * occ, 0.0)


def _search_cfg(pmin, pmax, **kw):
    cfg = dict(period_min_days=pmin, period_max_days=pmax, oversampling=3.0,
               m_star=1.0, r_star=1.0, u1=0.4, u2=0.25)
    cfg.update(kw)
    return cfg


def short_white(seed: int = 0) -> LightCurve:
    """30 days at 30-min cadence, white noise sigma=1e-3 (1440 points)."""
    rng = np.random.default_rng(seed)
    n = 1440
    t = np.arange(n, dtype=np.float64) * (30.0 / DAY_MIN)
    period, depth, t14 = 3.7, 1000e-6, 2.5 / 24.0
    t0 = float(t[0] + rng.uniform(0.0, period))
    sigma = 1e-3
    y = transit_profile(t, period, t0, depth, t14) + rng.normal(0.0, sigma, n)
    dy = np.full(n, sigma)
    inj = dict(period=period, t0=t0, depth=depth, t14=t14, u1=0.4, u2=0.25)
    return LightCurve(t, y, dy, "short_white", seed, inj, _search_cfg(0.5, 15.0))


def _kepler_cadences(rng, baseline_days, cadence_min, gap_days, quarter_days,
                     dropout):
    ncad = int(math.floor(baseline_days * DAY_MIN / cadence_min))
    t = np.arange(ncad, dtype=np.float64) * (cadence_min / DAY_MIN)
    keep = np.ones(ncad, dtype=bool)
    k = 1
    while k * quarter_days < t[-1]:
        lo = k * quarter_days
        keep &= ~((t >= lo) & (t < lo + gap_days))
        k += 1
    keep &= rng.random(ncad) >= dropout
    return t, keep


def _ar1(rng, n, phi, stationary_sigma):
    innov = rng.normal(0.0, stationary_sigma * math.sqrt(1.0 - phi * phi), n)
    a = np.empty(n)
    a[0] = rng.normal(0.0, stationary_sigma)
    for i in range(1, n):  # plain recursion; n <= ~1e5
        a[i] = phi * a[i - 1] + innov[i]
    return a


def kepler_like(seed: int = 1, baseline_days=1460.0, cadence_min=29.4,
                gap_days=3.0, quarter_days=365.25 / 4.0, dropout=0.10,
                white_ppm=100.0, red_ppm=30.0, phi=0.9,
                period=37.0, depth_ppm=200.0, t14_hours=6.0,
                pmin=0.5, pmax=None) -> LightCurve:
    """Kepler-like long-cadence light curve with quarter gaps and dropouts."""
    rng = np.random.default_rng(seed)
    t, keep = _kepler_cadences(rng, baseline_days, cadence_min, gap_days,
                               quarter_days, dropout)
    ncad = t.size
    white = rng.normal(0.0, white_ppm * 1e-6, ncad)
    red = _ar1(rng, ncad, phi, red_ppm * 1e-6)
    t0 = float(rng.uniform(0.0, period))
    depth, t14 = depth_ppm * 1e-6, t14_hours / 24.0
    y = transit_profile(t, period, t0, depth, t14) + white + red
    t, y = t[keep], y[keep]
    sig = math.hypot(white_ppm, red_ppm) * 1e-6
    dy = np.full(t.size, sig)
    inj = dict(period=period, t0=t0, depth=depth, t14=t14, u1=0.4, u2=0.25)
    if pmax is None:
        pmax = 0.5 * baseline_days
    return LightCurve(t, y, dy, "kepler_like", seed, inj, _search_cfg(pmin, pmax))


def long_baseline(seed: int = 2, n=144_000, cadence_min=30.0, white_ppm=200.0,
                  period=123.4, depth_ppm=300.0, t14_hours=8.0) -> LightCurve:
    """3000-day light curve at 30-min cadence with white noise."""
    rng = np.random.default_rng(seed)
    t = np.arange(n, dtype=np.float64) * (cadence_min / DAY_MIN)
    t0 = float(rng.uniform(0.0, period))
    sigma = white_ppm * 1e-6
    depth, t14 = depth_ppm * 1e-6, t14_hours / 24.0
    y = transit_profile(t, period, t0, depth, t14) + rng.normal(0.0, sigma, n)
    dy = np.full(n, sigma)
    inj = dict(period=period, t0=t0, depth=depth, t14=t14, u1=0.4, u2=0.25)
    return LightCurve(t, y, dy, "long_baseline", seed, inj,
                      _search_cfg(0.5, 0.5 * n * cadence_min / DAY_MIN))


def batch_kepler_like(count: int, seed: int = 3, n_min=20_000, n_max=72_000,
                      inject_fraction=0.3, start: int = 0):
    """Many Kepler-like light curves of uneven length.

    Lengths are uniform in [n_min, n_max]; the white-noise level is
    log-uniform in [50, 2000] ppm (red noise at 30 % of it); a fraction of
    the curves carries a transit with P log-uniform in [1, 200] d and depth
    log-uniform in [50, 5000] ppm.  The duration follows T14 = 111.6 s^(1/3)
    x P^(1/3) (geometric middle of the 20.05..620.84 s^(2/3) envelope).
    Curve i of the sequence draws from SeedSequence(seed, spawn_key=(i,));
    `start` returns curves start .. start + count - 1 of that sequence.
    """
    out = []
    for i in range(start, start + count):
        child = np.random.SeedSequence(seed, spawn_key=(i,))
        rng = np.random.default_rng(child)
        n = int(rng.integers(n_min, n_max + 1))
        sig_ppm = float(math.exp(rng.uniform(math.log(50.0), math.log(2000.0))))
        inject = bool(rng.random() < inject_fraction)
        period = float(math.exp(rng.uniform(0.0, math.log(200.0))))
        depth_ppm = float(math.exp(rng.uniform(math.log(50.0), math.log(5000.0))))
        t14_days = 111.6 * (period * 86400.0) ** (1.0 / 3.0) / 86400.0
        # enough cadences to survive gaps (3 d / 91.3 d) and 10 % dropouts
        base = n * 29.4 / DAY_MIN / 0.86 + 10.0
        lc = kepler_like(seed=int(rng.integers(1 << 31)), baseline_days=base,
                         white_ppm=sig_ppm, red_ppm=0.3 * sig_ppm,
                         period=period, depth_ppm=depth_ppm if inject else 0.0,
                         t14_hours=t14_days * 24.0)
        m = min(n, lc.n)
        t, y, dy = lc.t[:m].copy(), lc.y[:m].copy(), lc.dy[:m].copy()
        inj = dict(lc.injected) if inject else {}
        cfg = _search_cfg(0.5, 0.5 * float(t[-1] - t[0]))
        out.append(LightCurve(t, y, dy, f"batch{i}", seed, inj, cfg))
    return out


def noiseless_one_point_per_cycle(period: float, n: int, a: int, t_start=0.0):
    """Times with exactly one sample per cycle of ``period``.

    t_k = t_start + period * (k + ((a*k mod n) + 1/2) / n), gcd(a, n) = 1,
    so that folding at ``period`` puts sample k at phase ((a*k mod n)+1/2)/n:
    the folded order is a known permutation with evenly spaced phases.
    """
    if math.gcd(a, n) != 1:
        raise ValueError("a and n must be coprime")
    k = np.arange(n, dtype=np.int64)
    frac = ((a * k) % n + 0.5) / n
    return t_start + period * (k.astype(np.float64) + frac)


WORKLOADS = {
    "short_white": short_white,
    "kepler_like": kepler_like,
    "long_baseline": long_baseline,
}


def make_workload(name: str, seed=None) -> LightCurve:
    fn = WORKLOADS[name]
    return fn() if seed is None else fn(seed=seed)

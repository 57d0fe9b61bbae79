"""Edge cases of the search against the FP64 oracle: time stamps out of
order and repeated, the smallest curves and grids, a single trial period,
and plan limits that must be refused.

Neither the paper nor the library asks for time-ordered input: the fold
orders the points by (lattice phase, index), so a permuted curve folds to a
permutation of the same phases and every window sum is the same set of
products.  Both sides must then agree element by element as for ordered
input (chi2 within the contract, argmins exact or near ties, SDE).
"""

import numpy as np
import pytest

from oracle import search as osr

from . import gpu_helpers as gh
from .test_gpu_parity import SDE_ATOL, _check_argmins, _check_chi2

pytestmark = pytest.mark.gpu


def _curve(n, seed, span=25.0, period=3.1, depth=3e-3, width=0.02):
    rng = np.random.default_rng(seed)
    t = np.sort(rng.uniform(0.0, span, n))
    y = 1.0 + rng.normal(0.0, 1e-3, n)
    ph = ((t - 0.7) / period) % 1.0
    y[ph < width] -= depth
    dy = np.full(n, 1e-3)
    return t, y, dy


def _full_parity(t, y, dy, cfg=None, periods=None):
    base = float(t.max() - t.min())
    cfg = dict(cfg or {})
    if periods is not None:
        cfg["periods_days"] = periods
    op = gh.oracle_plan_for(t.size, base, cfg)
    r_or, sr_or, raw_or, sde_or, best_or = osr.full_search(op, t, y, dy)
    pl = gh.plan_for(t.size, base, cfg)
    res, out = gh.gpu_search(pl, t, y, dy)
    _check_chi2(out["chi2"], r_or.chi2, r_or.chi2_0)
    _check_argmins(op, t, y, dy, r_or, out, min_exact=0.95)
    np.testing.assert_allclose(out["sde"], sde_or, rtol=0, atol=SDE_ATOL)
    assert res.period_idx == best_or["period_idx"]
    pl.close()
    return res, out, r_or


def test_time_stamps_out_of_order_and_repeated():
    t, y, dy = _curve(2500, 21)
    t[100:130] = t[99]          # 30 repeats of one time stamp
    perm = np.random.default_rng(4).permutation(t.size)
    t, y, dy = t[perm], y[perm], dy[perm]
    res, out, r_or = _full_parity(t, y, dy, dict(period_min_days=0.6, period_max_days=10.0))
    assert abs(res.period - 3.1) < 0.05


def test_permuted_curve_has_the_same_spectrum():
    # the permutation changes only the index tie-break of equal phases: the
    # per-period chi2 of the ordered and the permuted curve agree to rounding
    t, y, dy = _curve(3000, 22)
    cfg = dict(period_min_days=0.6, period_max_days=10.0)
    base = float(t.max() - t.min())
    perm = np.random.default_rng(5).permutation(t.size)
    pa = gh.plan_for(t.size, base, cfg)
    ra, oa = gh.gpu_search(pa, t, y, dy)
    rb, ob = gh.gpu_search(pa, t[perm], y[perm], dy[perm])
    pa.close()
    np.testing.assert_allclose(ob["chi2"], oa["chi2"], rtol=1e-7, atol=0)
    assert ra.period_idx == rb.period_idx and ra.dur_idx == rb.dur_idx
    assert ra.t0 == pytest.approx(rb.t0, abs=1e-9)


@pytest.mark.parametrize("n", [24, 97])
def test_smallest_curves(n):
    t, y, dy = _curve(n, 30 + n, span=12.0, period=2.3, depth=4e-3, width=0.12)
    _full_parity(t, y, dy, periods=np.geomspace(0.9, 5.0, 41))


def test_single_trial_period():
    t, y, dy = _curve(1200, 40)
    res, out, r_or = _full_parity(t, y, dy, periods=np.array([3.1]))
    # one period: SR = 1, SDE_raw and SDE are 0 by the zero-spread rule
    assert out["sr"][0] == 1.0 and out["sde"][0] == 0.0
    assert res.period_idx == 0


def test_plan_limits_are_refused():
    import paper_2607_00348_gb300 as pkg
    t, y, dy = _curve(2000, 41)
    base = float(t.max() - t.min())
    # a duration ratio this close to 1 needs more than 255 durations
    with pytest.raises(pkg.GtlsError, match="INVALID_ARG"):
        gh.plan_for(t.size, base, dict(period_min_days=0.6, period_max_days=10.0, dur_ratio=1.001))
    # an odd median window is required
    with pytest.raises(pkg.GtlsError, match="INVALID_ARG"):
        pkg.Plan(pkg.PlanConfig(baseline_days=base, n_points=t.size, median_window=4))

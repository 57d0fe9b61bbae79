"""The tensor-core window kernel (tcgen05, TF32 three-product split) against
the FP64 oracle and against the FP32 window kernels.

Durations whose T0 step lies in [GTLS_TC_MIN_ST (default 24), 1024] and whose
template spans at most 32 rows of T0 steps go to the tensor-core kernel when
the weights are uniform.  Here the threshold is lowered so that every
duration with a T0 step of 2 or more takes it, on curves small enough for a
full oracle grid, and raised so that none does, to compare the two window
kernels on the same search.
"""

import os

import numpy as np
import pytest

import synth
from oracle import search as osr

from . import gpu_helpers as gh
from .test_gpu_parity import _check_argmins, _check_chi2, SDE_ATOL

pytestmark = pytest.mark.gpu


class _min_step:
    """Sets the tensor-core threshold for the plans made inside the block."""

    def __init__(self, st):
        self.st = st

    def __enter__(self):
        self.old = os.environ.get("GTLS_TC_MIN_ST")
        os.environ["GTLS_TC_MIN_ST"] = str(self.st)

    def __exit__(self, *exc):
        if self.old is None:
            os.environ.pop("GTLS_TC_MIN_ST", None)
        else:
            os.environ["GTLS_TC_MIN_ST"] = self.old


def _ragged_curve(n, seed, span=60.0, depth=2e-3):
    rng = np.random.default_rng(seed)
    t = np.sort(rng.uniform(0.0, span, n))
    y = 1.0 + rng.normal(0.0, 1e-3, n)
    y += synth.transit_profile(t, 4.3, 1.1, depth, 0.2) - 1.0
    dy = np.full(n, 1e-3)
    return t, y, dy


@pytest.mark.parametrize("cfg", [dict(), dict(dt0=0.1), dict(k_min=41.39, k_max=546.94, q_cap=0.112)],
                         ids=["dt0_0.05", "dt0_0.1", "tls_default_bounds"])
def test_every_step_from_two_on_tensor_cores_full_grid(cfg):
    # the 1440-point curve: T0 steps 2..10, 15..29 template rows, one to
    # twelve M-tiles per duration
    lc = synth.short_white()
    c = dict(lc.search, **cfg)
    op = gh.oracle_plan_for(lc.n, lc.baseline_days, c)
    r_or, sr_or, raw_or, sde_or, best_or = osr.full_search(op, lc.t, lc.y, lc.dy)
    with _min_step(2):
        pl = gh.plan_for(lc, lc.baseline_days, c)
    res, out = gh.gpu_search(pl, lc.t, lc.y, lc.dy)
    _check_chi2(out["chi2"], r_or.chi2, r_or.chi2_0)
    _check_argmins(op, lc.t, lc.y, lc.dy, r_or, out, min_exact=0.99)
    np.testing.assert_allclose(out["sde"], sde_or, rtol=0, atol=SDE_ATOL)
    assert res.period_idx == best_or["period_idx"]
    assert (res.dur_idx, res.t0_idx) == (best_or["dur_idx"], best_or["t0_idx"])
    assert res.t0 == best_or["t0"]
    pl.close()


@pytest.mark.parametrize("n,seed", [(20000, 3), (7777, 8)])
def test_ragged_curves_long_steps(n, seed):
    # T0 steps up to about 150 (several K chunks, a partial last chunk),
    # windows per duration not a multiple of a tile, and a transit
    t, y, dy = _ragged_curve(n, seed)
    periods = np.geomspace(0.51, 29.0, 97)
    base = float(t.max() - t.min())
    op = gh.oracle_plan_for(n, base, periods_days=periods)
    r_or = osr.search_periods(op, t, y, dy)
    with _min_step(2):
        pl = gh.plan_for(n, base, periods_days=periods)
    res, out = gh.gpu_search(pl, t, y, dy)
    _check_chi2(out["chi2"], r_or.chi2, r_or.chi2_0)
    _check_argmins(op, t, y, dy, r_or, out)
    pl.close()


def test_tensor_and_fp32_kernels_agree():
    lc = synth.kepler_like()
    cfg = lc.search
    outs = []
    for st in (24, 100000):
        with _min_step(st):
            pl = gh.plan_for(lc, lc.baseline_days, cfg)
        res, out = gh.gpu_search(pl, lc.t, lc.y, lc.dy)
        outs.append((res, out))
        pl.close()
    (ra, a), (rb, b) = outs
    rel = np.abs(a["chi2"] - b["chi2"]) / b["chi2"]
    assert float(rel.max()) < 1e-6, float(rel.max())
    same = (a["dur_idx"] == b["dur_idx"]) & (a["t0_idx"] == b["t0_idx"])
    assert same.mean() > 0.99
    assert ra.period_idx == rb.period_idx and (ra.dur_idx, ra.t0_idx) == (rb.dur_idx, rb.t0_idx)
    assert abs(ra.sde - rb.sde) < SDE_ATOL


def test_bounded_wait_reports_timeout_and_the_plan_recovers():
    # test_flags bit 0: the tensor-core kernel waits on a barrier phase that
    # nothing completes, records the timeout and stops; the search returns
    # GTLS_ERR_TIMEOUT, the context stays usable and a normal plan still works
    import paper_2607_00348_gb300 as pkg
    t, y, dy = _ragged_curve(6000, 5)
    base = float(t.max() - t.min())
    periods = np.geomspace(0.6, 20.0, 40)
    pc = pkg.PlanConfig(baseline_days=base, n_points=t.size, periods_days=periods, test_flags=1)
    with _min_step(2):
        bad = pkg.Plan(pc)
    with pytest.raises(pkg.GtlsError, match="TIMEOUT"):
        gh.gpu_search(bad, t, y, dy)
    bad.close()
    op = gh.oracle_plan_for(t.size, base, periods_days=periods)
    r_or = osr.search_periods(op, t, y, dy)
    with _min_step(2):
        good = gh.plan_for(t.size, base, periods_days=periods)
    res, out = gh.gpu_search(good, t, y, dy)
    _check_chi2(out["chi2"], r_or.chi2, r_or.chi2_0)
    good.close()

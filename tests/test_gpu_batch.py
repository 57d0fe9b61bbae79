"""Batched search (gtls_batch_*): many curves of uneven length in waves of a
shared chunk scratch, cut on the device from a work queue inside the loop
nodes of a captured CUDA graph.

Every result of a batch must equal the single-curve search of the same
curve bit for bit (same kernels, same arithmetic per window), whatever the
wave size, the staged tile size the autotuner picks, the mix of uniform and
per-point dy, or the refinement stage.  The single-curve path is itself
checked against the oracle in test_gpu_parity.py; one batch curve is checked
against the oracle here as well.
"""

import numpy as np
import pytest

import synth
from oracle import search as osr

from . import gpu_helpers as gh

pytestmark = pytest.mark.gpu


def _curves():
    """(t, y, dy, cfg) of a mixed batch: two 1440-point curves (one with the
    refinement stage), two Kepler-like curves of uneven length and a
    1001-point curve with per-point dy."""
    out = []
    for s, k in ((0, 50), (5, 0)):
        lc = synth.short_white(seed=s)
        out.append((lc.t, lc.y, lc.dy, dict(lc.search, refine_periods=k)))
    for lc in synth.batch_kepler_like(2, seed=7, n_min=8000, n_max=14000):
        out.append((lc.t, lc.y, lc.dy, dict(lc.search)))
    rng = np.random.default_rng(2)
    n = 1001
    t = np.sort(rng.uniform(0.0, 40.0, n))
    y = 1.0 + rng.normal(0, 1e-3, n)
    y[rng.random(n) < 0.05] -= 4e-3
    dy = rng.uniform(5e-4, 3e-3, n)
    out.append((t, y, dy, dict(period_min_days=0.6, period_max_days=12.0)))
    return out


def _packed(curves):
    import torch
    dev = torch.device("cuda:0")
    cat = lambda k: torch.as_tensor(np.concatenate([c[k] for c in curves]), dtype=torch.float64,
                                    device=dev)
    offs = np.cumsum([0] + [c[0].size for c in curves]).astype(np.int64)
    return cat(0), cat(1), cat(2), offs


def _plans(curves):
    return [gh.plan_for(c[0].size, float(c[0].max() - c[0].min()), c[3]) for c in curves]


def _same(batch, plans, res, singles):
    for i, (r, (rs, outs)) in enumerate(zip(res, singles)):
        assert r.as_dict() == rs.as_dict(), i
        got = gh.batch_outputs(batch, i, plans[i].n_periods)
        for k in ("chi2", "dur_idx", "t0_idx", "depth", "t0", "sr", "sde_raw", "sde", "refined"):
            assert np.array_equal(got[k], outs[k]), (i, k)


def test_batch_equals_single_curve_searches():
    import paper_2607_00348_gb300 as pkg
    curves = _curves()
    plans = _plans(curves)
    singles = [gh.gpu_search(p, c[0], c[1], c[2]) for p, c in zip(plans, curves)]
    assert singles[0][0].refined == 50 and singles[4][0].uniform_dy == 0
    t, y, dy, offs = _packed(curves)
    # a small wave size makes waves span several curves and curves span waves
    batch = pkg.Batch(plans, wave_slots=700)
    for _ in range(2):   # capture, then replay of the graph
        res = batch.search(t, y, dy, offs)
        _same(batch, plans, res, singles)
    info = batch.info()
    # waves are cut on the device inside loop nodes: the graph holds each
    # loop body once, a replay launches it once per wave
    assert info.waves > 1 and info.last_launches > info.graph_kernels
    assert info.n_lc == len(curves) and info.n_points == offs[-1]
    tuned = batch.autotune(t, y, dy, offs)
    assert tuned.tuned == 1 and tuned.tuned_flops > 0
    res = batch.search(t, y, dy, offs)
    _same(batch, plans, res, singles)
    batch.close()
    for p in plans:
        p.close()


def test_batch_curve_matches_oracle_on_sampled_periods():
    import paper_2607_00348_gb300 as pkg
    curves = _curves()[2:4]
    plans = _plans(curves)
    t, y, dy, offs = _packed(curves)
    batch = pkg.Batch(plans)
    batch.search(t, y, dy, offs)
    for i, (tt, yy, dd, cfg) in enumerate(curves):
        op = gh.oracle_plan_for(tt.size, float(tt.max() - tt.min()), cfg)
        npd = op.periods.size
        sel = np.unique(np.linspace(0, npd - 1, 12).astype(int))
        r_or = osr.search_periods(op, tt, yy, dd, sel)
        got = gh.batch_outputs(batch, i, npd)
        np.testing.assert_allclose(got["chi2"][sel], r_or.chi2, rtol=1e-5, atol=0)
    batch.close()
    for p in plans:
        p.close()


def test_batch_reports_the_bad_curve_and_stays_usable():
    import paper_2607_00348_gb300 as pkg
    curves = _curves()[:3]
    plans = _plans(curves)
    t, y, dy, offs = _packed(curves)
    batch = pkg.Batch(plans)
    y_bad = y.clone()
    y_bad[int(offs[2]) + 17] = float("nan")
    with pytest.raises(pkg.GtlsError, match="light curve 2.*NaN"):
        batch.search(t, y_bad, dy, offs)
    bad_offs = offs.copy()
    bad_offs[1] += 1
    with pytest.raises(pkg.GtlsError, match="INVALID_ARG"):
        batch.search(t, y, dy, bad_offs)
    res = batch.search(t, y, dy, offs)
    assert abs(res[0].period - 3.7) < 0.05
    batch.close()
    with pytest.raises(pkg.GtlsError, match="once"):
        pkg.Batch([plans[0], plans[0]])
    for p in plans:
        p.close()


def test_weighted_refinement_and_graph_recapture():
    import paper_2607_00348_gb300 as pkg
    # per-point dy with the refinement stage: single search against the oracle
    lc = synth.short_white(seed=3)
    rng = np.random.default_rng(8)
    dyw = lc.dy * (1.0 + 0.25 * rng.uniform(-1.0, 1.0, lc.n))
    cfg = dict(lc.search, refine_periods=40)
    op = gh.oracle_plan_for(lc.n, lc.baseline_days, cfg)
    r_or, sr_or, raw_or, sde_or, best_or = osr.full_search(op, lc.t, lc.y, dyw, refine_top_k=40)
    pl = gh.plan_for(lc, lc.baseline_days, cfg)
    res, out = gh.gpu_search(pl, lc.t, lc.y, dyw)
    assert res.uniform_dy == 0 and res.refined == 40
    assert np.array_equal(out["refined"].astype(bool), r_or.refined)
    np.testing.assert_allclose(out["chi2"], r_or.chi2, rtol=1e-5, atol=0)
    np.testing.assert_allclose(out["sde"], sde_or, rtol=0, atol=1e-3)
    assert res.period_idx == best_or["period_idx"]
    # the same plans in a batch whose dy switches between uniform and per-point
    # from call to call (the captured graph is recaptured for each class set)
    other = synth.short_white(seed=6)
    pl2 = gh.plan_for(other, other.baseline_days, other.search)
    batch = pkg.Batch([pl, pl2], wave_slots=500)
    for dy0 in (dyw, lc.dy, dyw):
        curves = [(lc.t, lc.y, dy0, {}), (other.t, other.y, other.dy, {})]
        singles = [gh.gpu_search(pl, lc.t, lc.y, dy0), gh.gpu_search(pl2, other.t, other.y, other.dy)]
        t, y, dy, offs = _packed(curves)
        res_b = batch.search(t, y, dy, offs)
        _same(batch, [pl, pl2], res_b, singles)
    batch.close()
    pl.close()
    pl2.close()


def test_graph_does_not_grow_with_the_number_of_curves():
    import paper_2607_00348_gb300 as pkg
    # the same kernel class (uniform dy, tiled, no refinement) with two and
    # with four curves: the same graph, more waves; results as searched alone
    curves = _curves()[1:4] + [(lambda lc: (lc.t, lc.y, lc.dy, dict(lc.search)))(synth.short_white(seed=6))]
    plans = _plans(curves)
    infos = []
    for sel in ([1, 2], [0, 1, 2, 3]):
        sub = [curves[i] for i in sel]
        t, y, dy, offs = _packed(sub)
        batch = pkg.Batch([plans[i] for i in sel], wave_slots=600)
        res = batch.search(t, y, dy, offs)
        infos.append(batch.info())
        batch.close()
        for r, i in zip(res, sel):
            rs, _ = gh.gpu_search(plans[i], curves[i][0], curves[i][1], curves[i][2])
            assert r.as_dict() == rs.as_dict(), i
    a, b = infos
    assert a.graph_kernels == b.graph_kernels
    assert b.waves > a.waves and b.last_launches > a.last_launches
    for p in plans:
        p.close()


def test_trim_frees_the_chunk_scratch_and_search_reallocates_it():
    lc = synth.short_white(seed=2)
    pl = gh.plan_for(lc, lc.baseline_days, lc.search)
    before = pl.device_bytes()
    pl.reserve()
    held = pl.device_bytes()
    assert held > before
    pl.reserve()   # no-op when it exists
    assert pl.device_bytes() == held
    r1, o1 = gh.gpu_search(pl, lc.t, lc.y, lc.dy)
    pl.trim()
    assert pl.device_bytes() == before
    pl.trim()      # no-op when absent
    r2, o2 = gh.gpu_search(pl, lc.t, lc.y, lc.dy)
    assert pl.device_bytes() == held
    assert r1.as_dict() == r2.as_dict()
    for k in ("chi2", "sde", "t0"):
        assert np.array_equal(o1[k], o2[k]), k
    pl.close()


def test_many_short_grids_fill_waves_up_to_the_segment_limit():
    # 40 curves with short explicit grids (11 to 50 periods each): a wave of
    # 4096 slots holds at most 32 (curve, period range) segments, so the
    # device cuts a wave at the segment limit before it is full, then carries
    # on with the next curves; every result equals the curve searched alone
    import paper_2607_00348_gb300 as pkg
    curves, plans = [], []
    for s in range(40):
        lc = synth.short_white(seed=100 + s)
        periods = np.geomspace(0.7, 9.0, 11 + s)
        curves.append((lc.t, lc.y, lc.dy, dict(periods_days=periods)))
        plans.append(gh.plan_for(lc.n, lc.baseline_days, periods_days=periods))
    t, y, dy, offs = _packed(curves)
    batch = pkg.Batch(plans, wave_slots=4096)
    res = batch.search(t, y, dy, offs)
    info = batch.info()
    assert info.waves == 2      # 32 segments, then the last 8 curves
    singles = [gh.gpu_search(p, c[0], c[1], c[2]) for p, c in zip(plans, curves)]
    _same(batch, plans, res, singles)
    batch.close()
    for p in plans:
        p.close()


def test_autotuned_batch_of_multi_tile_curves_equals_single_searches():
    # curves long enough for two staged tiles each, so that the tile
    # decomposition (which decides the warp block that evaluates a window,
    # and with it the summation order of some window variants) matters
    import paper_2607_00348_gb300 as pkg
    curves = [(lc.t, lc.y, lc.dy, dict(lc.search))
              for lc in synth.batch_kepler_like(2, seed=11, n_min=44000, n_max=46000)]
    plans = _plans(curves)
    singles = [gh.gpu_search(p, c[0], c[1], c[2]) for p, c in zip(plans, curves)]
    t, y, dy, offs = _packed(curves)
    batch = pkg.Batch(plans)
    batch.autotune(t, y, dy, offs)
    res = batch.search(t, y, dy, offs)
    _same(batch, plans, res, singles)
    batch.close()
    for p in plans:
        p.close()

"""Pins of the oracle's search: brute force on tiny inputs and invariants.

* The padded decomposition (pad, edge term, cumulative sums, out-of-transit
  a/b, direct in-transit sum; Sect. 2.3) must equal the explicit model chi2
  over the N original points, window by window (tests/brute.py).
* Invariants that the mathematics fixes: zero-depth chi2, SR range, SDE_raw
  moments, exact recovery of a noiseless template injection, recovery of a
  continuous injection, the fold order equal to numpy's stable argsort, the
  running median equal to numpy's median.
"""

import math

import numpy as np
import pytest

import synth
from oracle import grid
from oracle import search as osr

from . import brute


def _tiny(seed, n=48, span=11.0):
    rng = np.random.default_rng(seed)
    t = np.sort(rng.uniform(0.0, span, n))
    y = 1.0 + rng.normal(0.0, 1e-3, n)
    y[rng.random(n) < 0.2] -= 3e-3          # some dips so depths are > 0
    dy = rng.uniform(5e-4, 2e-3, n)          # per-point weights
    return t, y, dy


@pytest.mark.parametrize("seed", [0, 1, 2])
def test_decomposition_equals_brute_force_every_window(seed):
    t, y, dy = _tiny(seed)
    p = osr.plan(t.size, float(t.max() - t.min()), period_min_days=0.5, period_max_days=5.0)
    assert p.periods.size > 20
    checked = 0
    for pi in range(0, p.periods.size, 7):
        for j in grid.kept_durations(p.dur_pts, p.jlo[pi], p.jhi[pi]):
            c_or, d_or = osr.period_windows(p, t, y, dy, pi, j)
            c_bf, d_bf = brute.period_windows(p, t, y, dy, pi, j)
            assert c_or.shape == c_bf.shape
            np.testing.assert_allclose(c_or, c_bf, rtol=1e-12, atol=0)
            # F_cum of fluxes near 1 limits the depth to ~ulp(N)/D absolute
            np.testing.assert_allclose(d_or, d_bf, rtol=1e-9, atol=1e-13)
            checked += c_or.size
    assert checked > 500


@pytest.mark.parametrize("seed", [3, 4])
def test_period_minimum_equals_brute_force(seed):
    t, y, dy = _tiny(seed, n=40)
    p = osr.plan(t.size, float(t.max() - t.min()), period_min_days=0.7, period_max_days=4.0)
    sel = np.arange(0, p.periods.size, 5)
    r = osr.search_periods(p, t, y, dy, sel)
    for k, pi in enumerate(sel):
        c, j, s, dep = brute.period_min(p, t, y, dy, pi)
        assert r.chi2[k] == pytest.approx(c, rel=1e-12)
        assert (r.j_best[k], r.s_best[k]) == (j, s)
        assert r.depth[k] == pytest.approx(dep, rel=1e-9)


def test_windows_that_wrap_phase_one():
    # the last windows of a period run past folded position N-1 and wrap to 0
    t, y, dy = _tiny(7, n=30)
    p = osr.plan(t.size, float(t.max() - t.min()), period_min_days=0.5, period_max_days=5.0)
    pi = 3
    j = max(grid.kept_durations(p.dur_pts, p.jlo[pi], p.jhi[pi]))
    d = int(p.dur_pts[j])
    assert d >= 3
    c_or, _ = osr.period_windows(p, t, y, dy, pi, j)
    c_bf, _ = brute.period_windows(p, t, y, dy, pi, j)
    st = grid.t0_stride(d, p.dt0)
    wrap = [m for m in range(c_or.size) if m * st + d > t.size]
    assert wrap
    np.testing.assert_allclose(c_or[wrap], c_bf[wrap], rtol=1e-12)


def test_zero_depth_everywhere_gives_chi2_zero():
    # y >= 1 everywhere: every depth clamps to 0, chi2(P) = sum(((y-1)/dy)^2)
    rng = np.random.default_rng(11)
    n = 300
    t = np.sort(rng.uniform(0, 20, n))
    y = 1.0 + np.abs(rng.normal(0, 1e-3, n))
    dy = np.full(n, 1e-3)
    p = osr.plan(n, float(t.max() - t.min()), period_min_days=0.5, period_max_days=10.0)
    r, sr, raw, sde, best = osr.full_search(p, t, y, dy)
    chi2_0 = float(np.sum(((y - 1.0) / dy) ** 2))
    np.testing.assert_allclose(r.chi2, chi2_0, rtol=1e-12)
    assert np.all(r.depth == 0.0)
    # chi2(P) equals chi2_0 up to the rounding of the decomposition
    np.testing.assert_allclose(sr, 1.0, rtol=0, atol=1e-12)
    assert np.all(sde == 0.0)


def test_sr_range_and_sde_moments():
    lc = synth.short_white()
    p = osr.plan(lc.n, lc.baseline_days, period_min_days=0.5, period_max_days=15.0)
    r, sr, raw, sde, best = osr.full_search(p, lc.t, lc.y, lc.dy)
    assert np.all(sr > 0.0) and np.all(sr <= 1.0)
    assert sr[np.argmin(r.chi2)] == 1.0
    assert abs(raw.mean()) < 1e-12
    assert raw.std() == pytest.approx(1.0, rel=1e-12)
    # the injected 3.7-d transit is found
    assert abs(best["period"] - 3.7) / 3.7 < 0.01
    assert best["sde"] > 7.0


def test_exact_recovery_of_noiseless_template_injection():
    # one sample per cycle: folding at P* puts sample i at folded position
    # (a*i mod n); inject delta * template at (D, s) index-wise
    n, a, pstar = 211, 37, 2.345678901
    t = synth.noiseless_one_point_per_cycle(pstar, n, a)
    periods = pstar * np.array([0.9995, 0.9999, 1.0, 1.0001, 1.0005])
    p = osr.plan(n, float(t.max() - t.min()), periods_days=periods)
    k = 2
    assert p.periods[k] == pstar
    js = grid.kept_durations(p.dur_pts, p.jlo[k], p.jhi[k])
    j = js[len(js) // 2]
    d = int(p.dur_pts[j])
    st = grid.t0_stride(d, p.dt0)
    s = 7 * st
    tmpl = grid.template(d)
    delta = 2.5e-3
    pos = (a * np.arange(n)) % n
    rel = (pos - s) % n
    y = np.ones(n)
    inw = rel < d
    y[inw] = 1.0 - delta * tmpl[rel[inw]]
    dy = np.full(n, 1e-3)
    r = osr.search_periods(p, t, y, dy)
    chi2_0 = float(np.sum(((y - 1) / dy) ** 2))
    assert r.chi2[k] <= 1e-20 * chi2_0
    assert (r.j_best[k], r.s_best[k]) == (j, s)
    assert r.depth[k] == pytest.approx(delta, rel=1e-12)
    assert np.argmin(r.chi2) == k
    # the fold order at P* is the known permutation
    d_lat, p_int, _ = grid.phase_lattice(t, p.periods, p.e)
    order = osr.fold_order(d_lat, p_int[k])
    assert np.array_equal(pos[order], np.arange(n))


def test_continuous_injection_is_recovered_at_nearest_period():
    lc = synth.short_white()
    y = synth.transit_profile(lc.t, **{k: lc.injected[k] for k in ("period", "t0", "depth", "t14")})
    p = osr.plan(lc.n, lc.baseline_days, period_min_days=0.5, period_max_days=15.0)
    r, sr, raw, sde, best = osr.full_search(p, lc.t, y, lc.dy)
    nearest = int(np.argmin(np.abs(p.periods - 3.7)))
    assert abs(best["period_idx"] - nearest) <= 1
    assert best["chi2"] < 0.2 * r.chi2_0
    assert abs(best["depth"] - 1e-3) < 2e-4


def test_fold_order_is_numpy_stable_argsort():
    lc = synth.short_white()
    p = osr.plan(lc.n, lc.baseline_days, period_min_days=0.5, period_max_days=15.0)
    d_lat, p_int, _ = grid.phase_lattice(lc.t, p.periods, p.e)
    for k in (0, 17, 1000, p.periods.size - 1):
        np.testing.assert_array_equal(osr.fold_order(d_lat, p_int[k]),
                                      np.argsort(d_lat % p_int[k], kind="stable"))
    # exact phase ties (repeated times) keep the original index order
    d2 = np.array([5, 3, 5, 1, 3, 5], dtype=np.int64)
    # rho = d mod 4 = [1, 3, 1, 1, 3, 1]
    assert list(osr.fold_order(d2, 4)) == [0, 2, 3, 5, 1, 4]


def test_lattice_phase_is_exact_for_lattice_times():
    # times on the 2^-e lattice: rho / P_int equals the exact fractional part
    from fractions import Fraction
    e = 40
    rng = np.random.default_rng(5)
    ticks = np.sort(rng.integers(0, 10 * 2 ** 40, 50))
    t = ticks.astype(np.float64) / 2.0 ** 40
    per = 1.2345
    d_lat, p_int, t_ref = grid.phase_lattice(t, np.array([per]), e)
    for i in range(t.size):
        x = (Fraction(int(ticks[i] - ticks[0])) / Fraction(int(p_int[0])))
        frac = x - math.floor(x)
        assert Fraction(int(d_lat[i] % p_int[0]), int(p_int[0])) == frac


@pytest.mark.parametrize("n,w", [(1, 3), (2, 3), (10, 3), (57, 7), (200, 21), (33, 101)])
def test_running_median_equals_numpy_median(n, w):
    rng = np.random.default_rng(n * 7 + w)
    v = rng.normal(size=n)
    v[rng.random(n) < 0.2] = 0.5                # repeated values
    out = osr.running_median(v, w)
    h = w // 2
    for i in range(n):
        win = np.sort(v[max(0, i - h): min(n, i + h + 1)])
        assert out[i] == win[(win.size - 1) // 2]   # lower median
        if win.size % 2 == 1:
            assert out[i] == np.median(win)


def test_median_window_reading():
    assert osr.median_window(3048) == 31
    assert osr.median_window(10) == 3
    assert osr.median_window(199_999) == 1999


def test_refinement_never_raises_chi2_and_keeps_the_transit():
    # Sect. 2.5: re-searching with T0 step 1 can only lower chi2(P) (its
    # windows include the coarse ones), and the injected period stays best
    lc = synth.short_white()
    p = osr.plan(lc.n, lc.baseline_days, period_min_days=0.5, period_max_days=15.0)
    r0, _, _, sde0, best0 = osr.full_search(p, lc.t, lc.y, lc.dy)
    c0 = r0.chi2.copy()
    r1, _, _, sde1, best1 = osr.full_search(p, lc.t, lc.y, lc.dy, refine_top_k=50)
    assert r1.refined.sum() == 50
    assert np.all(r1.chi2 <= c0 * (1 + 1e-12))
    assert np.all(r1.chi2[~r1.refined] == c0[~r1.refined])
    assert np.any(r1.chi2[r1.refined] < c0[r1.refined])
    assert abs(best1["period"] - 3.7) / 3.7 < 0.01
    assert r1.chi2[best1["period_idx"]] <= r0.chi2[best1["period_idx"]]
    # the selection is the top of the coarse SDE
    sel = np.flatnonzero(r1.refined)
    assert np.array_equal(sel, osr.refine_selection(sde0, 50))
    assert sde0[sel].min() >= np.delete(sde0, sel).max()


def test_refinement_selection_ties_take_lower_index():
    sde = np.array([1.0, 3.0, 3.0, 2.0, 3.0])
    assert list(osr.refine_selection(sde, 2)) == [1, 2]
    assert list(osr.refine_selection(sde, 4)) == [1, 2, 3, 4]

"""Pins of the oracle's period and duration grids (Sect. 2.2).

Each check compares the oracle with a number the paper prints
(tests/golden/paper_values.json) or with a closed form of the equations.
"""

import json
import math
import os

import numpy as np
import pytest

from oracle import grid

GOLD = json.load(open(os.path.join(os.path.dirname(__file__), "golden", "paper_values.json")))


def test_roche_f_max_matches_paper():
    # Sect. 2.2.1: f_max = 1.924e-5 Hz for solar M and R, P_min ~ 0.6 d.
    # The paper does not state G, M_sun, R_sun; with the IAU 2015 nominal
    # values the result is 1.9229e-5, so the pin allows 1e-3 relative (a
    # dropped factor such as 3^(3/2) or 2 pi would miss by far more).
    f = grid.roche_f_max(1.0, 1.0)
    assert abs(f / GOLD["roche_f_max_hz"]["value"] - 1.0) < 1e-3
    p_min = 1.0 / f / grid.DAY
    assert round(p_min, 1) == GOLD["roche_p_min_days"]["value"]


def test_roche_scaling_with_star():
    # Eq. (f_max): f scales as sqrt(M) R^(-3/2)
    f0 = grid.roche_f_max(1.0, 1.0)
    assert grid.roche_f_max(4.0, 1.0) == pytest.approx(2.0 * f0, rel=1e-14)
    assert grid.roche_f_max(1.0, 4.0) == pytest.approx(f0 / 8.0, rel=1e-14)


def test_number_of_periods_for_kepler_baseline():
    # Sect. 2.2.1: about 190,000 trial frequencies for a 1500-day light curve
    f, info = grid.ofir_frequencies(GOLD["kepler_baseline_days"]["value"])
    want = GOLD["kepler_n_periods"]["value"]
    assert abs(info["N"] - want) / want < 0.02
    assert abs(f.size - info["N"]) <= 1.0


@pytest.mark.parametrize("baseline,pmin,pmax", [(1500.0, None, None), (29.979, 0.5, 15.0),
                                                (1460.0, 0.5, 730.0), (3000.0, 0.5, 1500.0)])
def test_ofir_endpoints_and_spacing(baseline, pmin, pmax):
    # Eqs. (f_i), (C, A), (N): f_1 = f_min exactly; f at the real index N is
    # f_max; the cube roots are evenly spaced by A/3.
    f, info = grid.ofir_frequencies(baseline, period_min_days=pmin, period_max_days=pmax)
    a, c, n_real = info["A"], info["C"], info["N"]
    assert f[0] == pytest.approx(info["f_min"], rel=1e-12)
    assert (a / 3.0 * n_real + c) ** 3 == pytest.approx(info["f_max"], rel=1e-12)
    steps = np.diff(np.cbrt(f))
    assert np.allclose(steps, a / 3.0, rtol=1e-8, atol=0)
    assert f.max() <= info["f_max"] * (1 + 1e-12)
    assert f.min() >= info["f_min"] * (1 - 1e-12)


def test_ofir_density_follows_phase_drift():
    # The cubic sampling keeps d f / f^(2/3) constant, i.e. the phase drift
    # across the baseline is constant: d f = A f^(2/3) per sample.
    f, info = grid.ofir_frequencies(1500.0)
    df = np.diff(f)
    mid = 0.5 * (f[1:] + f[:-1])
    ratio = df / mid ** (2.0 / 3.0)
    assert np.allclose(ratio, info["A"], rtol=1e-4)


def test_oversampling_scales_count():
    # N is proportional to OS (Eq. N with A ~ 1/OS) up to the A/3 offset
    _, i3 = grid.ofir_frequencies(1500.0, oversampling=3.0)
    _, i6 = grid.ofir_frequencies(1500.0, oversampling=6.0)
    assert i6["N"] == pytest.approx(2.0 * i3["N"] - 1.0, rel=1e-9)


def test_duration_bounds_at_3p7_days():
    # Eqs. (upper), (lower): T14 in [k_min, k_max] P^(1/3) seconds
    p = np.array([3.7])
    n = 100_000
    q, d, jlo, jhi = grid.duration_grid(p, n)
    p_s = 3.7 * grid.DAY
    t_lo = GOLD["gtls_k_min"]["value"] * p_s ** (1.0 / 3.0)
    t_hi = GOLD["gtls_k_max"]["value"] * p_s ** (1.0 / 3.0)
    assert t_lo / 3600 == pytest.approx(0.381, abs=1e-3)
    assert t_hi / 3600 == pytest.approx(11.79, abs=1e-2)
    sel = q[jlo[0]:jhi[0] + 1] * p_s
    assert sel.min() >= t_lo * (1 - 1e-12)
    assert sel.max() <= t_hi * (1 + 1e-12)
    # the grid is geometric with ratio 1.1 and starts at k_min P_max^(-2/3)
    assert np.allclose(q[1:] / q[:-1], 1.1, rtol=1e-13)


def test_duration_cap_binds_below_266k_seconds():
    # k_max P^(-2/3) = 0.15 at P = (k_max / 0.15)^(3/2) = 2.663e5 s
    p_cross = (GOLD["gtls_k_max"]["value"] / GOLD["gtls_q_cap"]["value"]) ** 1.5
    assert p_cross == pytest.approx(2.663e5, rel=1e-3)
    periods = np.array([0.5 * p_cross, 2.0 * p_cross]) / grid.DAY
    q, d, jlo, jhi = grid.duration_grid(periods, 10_000)
    assert q[jhi[0]] <= 0.15 < q[jhi[0]] * 1.1            # capped
    assert q[jhi[1]] < 0.15                             # not capped


def test_tls_bounds_are_narrower():
    # TLS defaults (Sect. 2.2.2) give a sub-range of the GTLS range
    p = np.array([10.0])
    qg, _, lg, hg = grid.duration_grid(p, 50_000)
    qt, _, lt, ht = grid.duration_grid(p, 50_000, k_min=GOLD["tls_k_min"]["value"],
                                       k_max=GOLD["tls_k_max"]["value"],
                                       q_cap=GOLD["tls_q_cap"]["value"])
    assert qt[lt[0]] >= qg[lg[0]]
    assert qt[ht[0]] <= qg[hg[0]]


def test_duration_points_rounding():
    q = np.array([0.5 / 1000, 1.5 / 1000, 2.5 / 1000, 1e-9])
    # half away from zero, at least 1
    d = np.maximum(1, np.floor(q * 1000 + 0.5)).astype(int)
    assert list(d) == [1, 2, 3, 1]
    _, dd, _, _ = grid.duration_grid(np.array([1.0, 2.0]), 777)
    assert dd.min() >= 1


def test_n_skip_worked_example():
    # Eq. (N_skip): n_IT = 2000, dt0 = 0.05 -> 100 skipped points
    ex = GOLD["n_skip_example"]
    assert grid.t0_stride(ex["n_it"], ex["dt0"]) == ex["n_skip"]
    assert grid.t0_stride(19, 0.05) == 1
    assert grid.t0_stride(1, 0.05) == 1


def test_kept_durations_drop_repeats():
    d = np.array([1, 1, 2, 2, 2, 3, 5])
    assert grid.kept_durations(d, 0, 6) == [0, 2, 5, 6]
    assert grid.kept_durations(d, 1, 4) == [1, 2]


def test_time_quantum_exponent():
    e, bits = grid.time_quantum_exponent(144_000, 1500.0)
    assert bits == 18
    # P_max on the lattice stays below 2^(63 - idx_bits)
    assert 1500.0 * 2.0 ** e < 2.0 ** (63 - bits)
    assert 1500.0 * 2.0 ** (e + 1) >= 2.0 ** (63 - bits) or e == 40
    e2, _ = grid.time_quantum_exponent(1440, 15.0)
    assert e2 == 40

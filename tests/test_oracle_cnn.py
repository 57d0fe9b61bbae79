"""Pins of the FP64 proposal-network reference (oracle/cnn.py).

Each pin checks the reference against something other than its own code:
numpy.convolve, central finite differences of the loss, a per-point loop
for the binning, the closed form of a first Adam step, brute force for the
region targets and the proposal.
"""

import math

import numpy as np
import pytest

from oracle import cnn


def test_conv_same_equals_numpy_convolve():
    rng = np.random.default_rng(0)
    for ks in (5, 7):
        x = rng.normal(size=37)
        w = rng.normal(size=ks)
        out = cnn.conv_same(x[None, :, None], w[None, :, None], np.zeros(1))[0, :, 0]
        # correlation with 'same' padding == convolution with the reversed taps
        np.testing.assert_allclose(out, np.convolve(x, w[::-1], mode="same"), rtol=1e-12, atol=1e-12)


@pytest.mark.parametrize("ks,dil", [(5, 2), (5, 8), (7, 3)])
def test_dilated_conv_equals_numpy_convolve_of_the_zero_stuffed_taps(ks, dil):
    rng = np.random.default_rng(ks * 10 + dil)
    x = rng.normal(size=61)
    w = rng.normal(size=ks)
    stuffed = np.zeros((ks - 1) * dil + 1)
    stuffed[::dil] = w
    out = cnn.conv_same(x[None, :, None], w[None, :, None], np.zeros(1), dil)[0, :, 0]
    np.testing.assert_allclose(out, np.convolve(x, stuffed[::-1], mode="same"), rtol=1e-12, atol=1e-12)


def test_conv_same_sums_input_channels_and_adds_bias():
    rng = np.random.default_rng(1)
    x = rng.normal(size=(2, 16, 3))
    w = rng.normal(size=(4, 5, 3))
    b = rng.normal(size=4)
    out = cnn.conv_same(x, w, b)
    for n in range(2):
        for o in range(4):
            ref = b[o] + sum(np.convolve(x[n, :, i], w[o, ::-1, i], mode="same") for i in range(3))
            np.testing.assert_allclose(out[n, :, o], ref, rtol=1e-12, atol=1e-12)


def _loss(params, x, tgt, mask):
    z, _ = cnn.forward(params, x)
    return cnn.loss_and_dz(z, tgt, mask)[0]


@pytest.mark.parametrize("seed", [3, 4])
def test_gradients_match_central_differences(seed):
    n_bins = 256
    rng = np.random.default_rng(seed)
    params = cnn.init_params(seed, n_bins)
    for name in params:
        if name.startswith("b"):
            params[name] = rng.normal(0, 0.1, params[name].shape)
    x = rng.normal(size=(2, n_bins))
    tgt = rng.uniform(size=(2, cnn.N_REG))
    mask = (rng.uniform(size=(2, cnn.N_REG)) < 0.8).astype(float)
    z, cache = cnn.forward(params, x)
    loss, dz = cnn.loss_and_dz(z, tgt, mask)
    g = cnn.backward(params, cache, dz)
    h = 1e-6
    for name, shp in cnn.param_shapes(n_bins):
        flat = params[name].ravel()
        for idx in rng.choice(flat.size, size=min(4, flat.size), replace=False):
            keep = flat[idx]
            flat[idx] = keep + h
            lp = _loss(params, x, tgt, mask)
            flat[idx] = keep - h
            lm = _loss(params, x, tgt, mask)
            flat[idx] = keep
            fd = (lp - lm) / (2 * h)
            an = g[name].ravel()[idx]
            assert an == pytest.approx(fd, rel=1e-4, abs=1e-9), (name, idx)


def test_loss_gradient_is_sigmoid_minus_target():
    rng = np.random.default_rng(5)
    z = rng.normal(size=(3, cnn.N_REG))
    tgt = rng.uniform(size=z.shape)
    mask = np.ones_like(z)
    loss, dz = cnn.loss_and_dz(z, tgt, mask)
    # binary cross-entropy with soft targets, written out
    s = 1 / (1 + np.exp(-z))
    ref = -(tgt * np.log(s) + (1 - tgt) * np.log(1 - s)).mean()
    assert loss == pytest.approx(ref, rel=1e-12)
    np.testing.assert_allclose(dz, (s - tgt) / z.size, rtol=1e-12)


def test_bin_flux_equals_a_per_point_loop():
    rng = np.random.default_rng(6)
    n = 3000
    t = np.sort(rng.uniform(10.0, 50.0, n))
    y = 1.0 + rng.normal(0, 1e-3, n)
    dy = rng.uniform(5e-4, 2e-3, n)
    nb = 64
    got = cnn.bin_flux(t, y, dy, nb)
    swr = [0.0] * nb
    sw = [0.0] * nb
    for ti, yi, di in zip(t, y, dy):
        b = min(nb - 1, int(math.floor((ti - t[0]) / (t[-1] - t[0]) * nb)))
        swr[b] += (1 - yi) / di ** 2
        sw[b] += 1 / di ** 2
    ref = [a / math.sqrt(c) if c > 0 else 0.0 for a, c in zip(swr, sw)]
    np.testing.assert_allclose(got, ref, rtol=1e-12, atol=1e-15)
    # a transit-free white curve gives unit-variance bins
    y2 = 1.0 + rng.normal(0, 1e-3, 200000)
    t2 = np.linspace(0, 100, 200000)
    b2 = cnn.bin_flux(t2, y2, np.full(t2.size, 1e-3), 256)
    assert abs(b2.std() - 1.0) < 0.1


def test_first_adam_step_closed_form():
    rng = np.random.default_rng(7)
    p = rng.normal(size=50)
    g = rng.normal(size=50)
    lr = 1e-3
    p1, m, v = cnn.adam_step(p, g, np.zeros(50), np.zeros(50), 1, lr)
    np.testing.assert_allclose(p1, p - lr * g / (np.abs(g) + 1e-8), rtol=1e-12)
    np.testing.assert_allclose(m, 0.1 * g, rtol=1e-12)
    np.testing.assert_allclose(v, 0.001 * g * g, rtol=1e-12)


def test_regions_and_targets_by_brute_force():
    assert cnn.region_of([cnn.P_LO])[0] == 0
    assert cnn.region_of([cnn.P_HI * (1 - 1e-12)])[0] == cnn.N_REG - 1
    rng = np.random.default_rng(8)
    periods = np.sort(np.exp(rng.uniform(np.log(0.5), np.log(700.0), 5000)))
    sr = rng.uniform(size=periods.size)
    tgt, mask = cnn.region_targets(periods, sr)
    edges = cnn.P_LO * (cnn.P_HI / cnn.P_LO) ** (np.arange(cnn.N_REG + 1) / cnn.N_REG)
    for r in range(cnn.N_REG):
        inside = (periods >= edges[r]) & (periods < edges[r + 1])
        if inside.any():
            assert mask[r] == 1 and tgt[r] == sr[inside].max()
        else:
            assert mask[r] == 0 and tgt[r] == 0
    scores = rng.uniform(size=cnn.N_REG)
    sel = cnn.proposed_periods(periods, scores, mask, 0.05)
    valid = np.flatnonzero(mask)
    k = math.ceil(0.05 * valid.size)
    top = sorted(valid, key=lambda r: (-scores[r], r))[:k]
    want = [i for i, p in enumerate(periods) if any(edges[r] <= p < edges[r + 1] for r in top)]
    assert list(sel) == want


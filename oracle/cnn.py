"""FP64 reference of the learned period proposal (test infrastructure).

The proposal is not part of the paper: it is a small 1D convolutional
network that looks at a light curve binned in time (no folding) and predicts,
for every log-spaced region of trial periods, the largest signal residue
SR(P) (Sect. 2.4) that the TLS search finds there.  Full TLS then runs only
in the best regions.  This module restates every step of that network in
plain numpy at float64 -- binning, the convolutions with bias, ReLU and
max-pooling, the linear head, the logistic loss, the gradients of all of it
and the Adam update -- so that the GPU kernels can be compared with it.  Only
the tests, the package smoke check and the benchmark's baseline legs may use
it; the library never does.

Pins (tests/test_oracle_cnn.py): the convolution against numpy.convolve, the
gradients against central finite differences, the binning against a direct
per-bin loop, Adam against its closed form after one step.

Layouts (shared with the library's C ABI, which documents them too):
  activations  [batch][length][channels]   (channels contiguous)
  conv weight  [out][tap][in]              (KS taps DIL bins apart, 'same' padding)
  head weight  [region][feature], feature = position * 64 + channel
"""

from __future__ import annotations

import math

import numpy as np

N_BINS = 4096
CH = 64
N_CONV = 6
KS = (7, 5, 5, 5, 5, 5)        # taps of the six convolutions
DIL = (1, 2, 2, 4, 4, 8)       # tap spacing (dilation) of each convolution, in its own input's bins
N_REG = 128
P_LO, P_HI = 0.5, 1024.0       # days: the regions split [P_LO, P_HI) evenly in log P


# ---------------------------------------------------------------------------
# input and targets
# ---------------------------------------------------------------------------

def bin_sums(t, y, dy, n_bins=N_BINS):
    """Per-bin sums (sum w r, sum w): bin b holds the points with
    floor((t - t_min) / (t_max - t_min) * n_bins) = b (the last point in the
    last bin); r = 1 - y, w = 1/dy^2."""
    t = np.asarray(t, np.float64)
    r = 1.0 - np.asarray(y, np.float64)
    w = 1.0 / np.asarray(dy, np.float64) ** 2
    span = t.max() - t.min()
    b = np.floor((t - t.min()) / span * n_bins).astype(np.int64) if span > 0 else np.zeros(t.size, np.int64)
    b = np.clip(b, 0, n_bins - 1)
    return np.bincount(b, weights=w * r, minlength=n_bins), np.bincount(b, weights=w, minlength=n_bins)


def bin_flux(t, y, dy, n_bins=N_BINS):
    """Time-binned deficit SNR: sum(w r) / sqrt(sum(w)) per bin (bin_sums),
    i.e. the weighted mean deficit over its standard error; empty bins are 0."""
    swr, sw = bin_sums(t, y, dy, n_bins)
    out = np.zeros(n_bins)
    nz = sw > 0
    out[nz] = swr[nz] / np.sqrt(sw[nz])
    return out


def region_of(periods):
    """Region index of each period: floor(R log(P/P_LO) / log(P_HI/P_LO))."""
    p = np.asarray(periods, np.float64)
    return np.floor(N_REG * np.log(p / P_LO) / math.log(P_HI / P_LO)).astype(np.int64)


def region_targets(periods, sr):
    """Largest SR(P) of every region and the mask of regions that hold at
    least one trial period."""
    reg = region_of(periods)
    ok = (reg >= 0) & (reg < N_REG)
    tgt = np.zeros(N_REG)
    mask = np.zeros(N_REG)
    np.maximum.at(tgt, reg[ok], np.asarray(sr, np.float64)[ok])
    mask[np.unique(reg[ok])] = 1.0
    return tgt, mask


def proposed_periods(periods, scores, mask, frac):
    """Indices of the trial periods inside the ceil(frac * valid regions)
    regions of largest score (ties: lower region first)."""
    valid = np.flatnonzero(np.asarray(mask) > 0)
    k = max(1, int(math.ceil(frac * valid.size)))
    s = np.asarray(scores, np.float64)[valid]
    order = np.lexsort((valid, -s))
    keep = np.zeros(N_REG, bool)
    keep[valid[order[:k]]] = True
    reg = region_of(periods)
    ok = (reg >= 0) & (reg < N_REG)
    return np.flatnonzero(ok & keep[np.clip(reg, 0, N_REG - 1)])


# ---------------------------------------------------------------------------
# network
# ---------------------------------------------------------------------------

def param_shapes(n_bins=N_BINS):
    """(name, shape) of every parameter, in the order of the flat vector."""
    shapes = []
    cin = 1
    for i, ks in enumerate(KS):
        shapes.append((f"w{i}", (CH, ks, cin)))
        shapes.append((f"b{i}", (CH,)))
        cin = CH
    feat = (n_bins >> N_CONV) * CH
    shapes.append(("wh", (N_REG, feat)))
    shapes.append(("bh", (N_REG,)))
    return shapes


def unflatten(flat, n_bins=N_BINS):
    out, pos = {}, 0
    for name, shp in param_shapes(n_bins):
        size = int(np.prod(shp))
        out[name] = np.asarray(flat[pos:pos + size], np.float64).reshape(shp)
        pos += size
    return out


def flatten(params, n_bins=N_BINS):
    return np.concatenate([np.asarray(params[name], np.float64).ravel()
                           for name, _ in param_shapes(n_bins)])


def init_params(seed, n_bins=N_BINS):
    """He-normal weights (std sqrt(2 / fan_in)), zero biases."""
    rng = np.random.default_rng(seed)
    p = {}
    for name, shp in param_shapes(n_bins):
        if name.startswith("b"):
            p[name] = np.zeros(shp)
        else:
            fan_in = int(np.prod(shp[1:]))
            p[name] = rng.normal(0.0, math.sqrt(2.0 / fan_in), shp)
    return p


def conv_same(x, w, b, dil=1):
    """out[n, l, o] = b[o] + sum_{k, i} w[o, k, i] x[n, l + (k - (KS-1)/2) dil, i]
    (zero outside 0..L-1)."""
    n, length, cin = x.shape
    cout, ks, _ = w.shape
    pad = (ks - 1) // 2 * dil
    xp = np.zeros((n, length + 2 * pad, cin))
    xp[:, pad:pad + length] = x
    out = np.broadcast_to(b, (n, length, cout)).copy()
    for k in range(ks):
        out += xp[:, k * dil:k * dil + length, :] @ w[:, k, :].T
    return out


def forward(params, x, store=None):
    """Activations of every layer for inputs x[n, n_bins]; returns the
    logits z[n, N_REG] and a cache for backward.  `store` (optional) maps
    the input and every pooled activation to the precision they are stored
    in (identity by default: FP64 throughout)."""
    keep = store if store is not None else (lambda v: v)
    a = keep(np.asarray(x, np.float64))[:, :, None]
    cache = []
    for i in range(N_CONV):
        pre = conv_same(a, params[f"w{i}"], params[f"b{i}"], DIL[i])
        act = np.maximum(pre, 0.0)
        n, length, c = act.shape
        pair = act.reshape(n, length // 2, 2, c)
        pooled = keep(pair.max(axis=2))
        arg = pair.argmax(axis=2)             # first of equal pair members
        cache.append((a, pre, arg))
        a = pooled
    feat = a.reshape(a.shape[0], -1)
    z = feat @ params["wh"].T + params["bh"]
    cache.append(feat)
    return z, cache


def loss_and_dz(z, target, mask):
    """Masked mean logistic loss with soft targets:
    L = sum mask * (softplus(z) - target z) / sum mask; dL/dz = mask (sigmoid(z) - target) / sum mask."""
    m = np.asarray(mask, np.float64)
    cnt = max(m.sum(), 1.0)
    sp = np.logaddexp(0.0, z)
    loss = float((m * (sp - target * z)).sum() / cnt)
    dz = m * (1.0 / (1.0 + np.exp(-z)) - target) / cnt
    return loss, dz


def backward(params, cache, dz):
    """Gradients of every parameter for the upstream gradient dz."""
    g = {}
    feat = cache[-1]
    g["wh"] = dz.T @ feat
    g["bh"] = dz.sum(axis=0)
    da = (dz @ params["wh"]).reshape(feat.shape[0], -1, CH)
    for i in reversed(range(N_CONV)):
        a_in, pre, arg = cache[i]
        n, length, c = pre.shape
        dpre = np.zeros((n, length // 2, 2, c))
        nn, jj, cc = np.meshgrid(np.arange(n), np.arange(length // 2), np.arange(c), indexing="ij")
        dpre[nn, jj, arg, cc] = da
        dpre = dpre.reshape(n, length, c) * (pre > 0)
        w = params[f"w{i}"]
        cout, ks, cin = w.shape
        dil = DIL[i]
        pad = (ks - 1) // 2 * dil
        xp = np.zeros((n, length + 2 * pad, cin))
        xp[:, pad:pad + length] = a_in
        gw = np.zeros_like(w)
        dxp = np.zeros_like(xp)
        for k in range(ks):
            sl = slice(k * dil, k * dil + length)
            gw[:, k, :] = np.einsum("nlo,nli->oi", dpre, xp[:, sl, :])
            dxp[:, sl, :] += dpre @ w[:, k, :]
        g[f"w{i}"] = gw
        g[f"b{i}"] = dpre.sum(axis=(0, 1))
        da = dxp[:, pad:pad + length, :]
    return g


def adam_step(p, g, m, v, step, lr, beta1=0.9, beta2=0.999, eps=1e-8):
    """One Adam update (Kingma & Ba 2015) of flat arrays; step counts from 1."""
    m = beta1 * m + (1.0 - beta1) * g
    v = beta2 * v + (1.0 - beta2) * g * g
    mh = m / (1.0 - beta1 ** step)
    vh = v / (1.0 - beta2 ** step)
    return p - lr * mh / (np.sqrt(vh) + eps), m, v

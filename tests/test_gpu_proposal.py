"""Learned proposal pipeline on the GPU: targets from the search of binned
curves, and the proposal search (explicit period subsets or full-grid
fallback) against direct searches of the same plans."""

import numpy as np
import pytest

import synth
from oracle import cnn

pytestmark = pytest.mark.gpu


def _curve(lc):
    return (lc.t, lc.y, lc.dy, dict(lc.injected), float(lc.baseline_days))


def test_binned_search_targets_mark_the_injected_period():
    import torch
    import paper_2607_00348_gb300 as pkg
    from paper_2607_00348_gb300 import proposal as pr
    lc = synth.kepler_like(seed=21, baseline_days=400.0, white_ppm=300.0, red_ppm=90.0,
                           period=9.3, depth_ppm=4000.0, t14_hours=4.0)
    quiet = synth.kepler_like(seed=22, baseline_days=300.0, white_ppm=300.0, red_ppm=90.0,
                              period=5.0, depth_ppm=0.0, t14_hours=3.0)
    net = pkg.Cnn(4)
    dev = torch.device("cuda:0")
    x, binned = pr.binned(net, [_curve(lc), _curve(quiet)], dev)
    assert x.shape == (2, cnn.N_BINS)
    tg, mk = pr.targets(binned, dev)
    assert np.all((tg >= 0) & (tg <= 1)) and np.all(tg[mk == 0] == 0)
    r_inj = int(cnn.region_of([9.3])[0])
    top = np.argsort(-tg[0])[:3]
    # the injected period's region (or a harmonic's) carries the strongest target
    assert any(abs(int(r) - r_inj) <= 1 or abs(int(r) - int(cnn.region_of([4.65])[0])) <= 1
               or abs(int(r) - int(cnn.region_of([18.6])[0])) <= 1 for r in top)
    assert tg[0].max() >= 0.6 and tg[1].max() < tg[0].max()
    net.close()


def test_proposal_search_equals_direct_searches_of_its_plans():
    import torch
    import paper_2607_00348_gb300 as pkg
    from paper_2607_00348_gb300 import proposal as pr
    from . import gpu_helpers as gh
    curves = [_curve(lc) for lc in synth.batch_kepler_like(3, seed=31, n_min=6000, n_max=9000)]
    dev = torch.device("cuda:0")
    net = pkg.Cnn(4, pr.init_params(0))
    full = [pr.plan_for(c[0].size, c[4]) for c in curves]
    # tau above every score: the whole grid for every curve
    res, fb, searched = pr.proposal_search(net, curves, full, dev, tau=2.0)
    assert all(fb) and searched == [p.n_periods for p in full]
    for r, c, p in zip(res, curves, full):
        assert r.as_dict() == gh.gpu_search(p, c[0], c[1], c[2])[0].as_dict()
    # tau 0: the proposed periods only, equal to a search of that subset
    res, fb, searched = pr.proposal_search(net, curves, full, dev, tau=0.0)
    scores = pr.scores_for(net, curves, dev)
    assert not any(fb)
    for i, (r, c, p) in enumerate(zip(res, curves, full)):
        per = p.periods()
        idx = pkg.proposal_periods(per, scores[i], pr.FRAC)
        assert searched[i] == idx.size < 0.2 * per.size
        sub = pr.plan_for(c[0].size, c[4], periods=per[idx])
        assert r.as_dict() == gh.gpu_search(sub, c[0], c[1], c[2])[0].as_dict()
        assert np.any(np.isclose(per[idx], r.period, rtol=1e-12))
        sub.close()
    for p in full:
        p.close()
    net.close()


def test_trained_network_ranks_strong_transits_first():
    """What the trained network adds to the plain search: an order in which
    to search a survey.  On 64 held-out curves of the uneven-length
    Kepler-like sequence (seed 5, never trained on), the curves with a
    strong injected transit (expected SNR = depth / sigma x
    sqrt(n T14 / P) >= 15) get the largest scores: the 8 best-scored curves
    hold at least 5 of them (searching in input order finds 7 x 8 / 64 = 0.9
    on average) and the scores separate them from transit-free curves with
    an ROC AUC of at least 0.9."""
    import torch
    import paper_2607_00348_gb300 as pkg
    from paper_2607_00348_gb300 import proposal as pr
    if not pr.weights_match():
        pytest.skip("no trained weights of this network")
    params, meta = pr.load_weights()
    assert meta["seed"] != 5
    lcs = synth.batch_kepler_like(64, seed=5)
    curves = [_curve(lc) for lc in lcs]
    snr = np.array([lc.injected["depth"] / lc.dy[0] * np.sqrt(lc.n * lc.injected["t14"]
                                                               / lc.injected["period"])
                    if lc.injected else 0.0 for lc in lcs])
    strong, none = snr >= 15.0, snr == 0.0
    assert strong.sum() >= 5
    dev = torch.device("cuda:0")
    net = pkg.Cnn(64, params)
    sc = pr.scores_for(net, curves, dev)
    best = np.empty(len(curves))
    for i, c in enumerate(curves):
        p = pr.plan_for(c[0].size, c[4])
        _, mask = pkg.region_targets(p.periods(), np.zeros(p.n_periods))
        best[i] = sc[i][mask > 0].max()
        p.close()
    top8 = np.argsort(-best, kind="stable")[:8]
    assert strong[top8].sum() >= 5
    auc = np.mean([(a > b) + 0.5 * (a == b) for a in best[strong] for b in best[none]])
    assert auc >= 0.9
    net.close()

"""Learned period proposal: training data made by the search itself, training
with the library's own network kernels, and the proposal search with a
full-grid fallback.  (The paper has no such stage.)

Every numeric step runs in libgtls: time binning, the network's forward,
backward and Adam kernels, and the TLS search that produces the targets and
that the proposal finally calls.  This module only organises batches, picks
plans and reads results back.

Targets.  A training curve is binned to the network's 4096-bin input; the
binned curve (bin centres, weighted mean flux of every non-empty bin,
uniform weights) is searched with TLS on its own Ofir grid (oversampling 1);
region r's target is min(1, max(0, largest SDE(P) of the region / 15)).  The
network therefore learns where, at its own resolution, the search finds
signal.

Proposal search.  Scores = sigmoid(network logits) of the curve's binned
input.  When the largest score over the regions that hold trial periods is
at least `tau`, the full-resolution search runs on the trial periods of the
ceil(frac x regions) best regions only (a plan with that explicit period
list); otherwise it runs on the whole grid.  SR and SDE are then those of the
searched periods.

    python -m paper_2607_00348_gb300.proposal train --train 4000 --out W.npz
    python -m paper_2607_00348_gb300.proposal evaluate --weights W.npz --eval 64 --json R.json
"""

from __future__ import annotations

import argparse
import json
import math
import multiprocessing as mp
import os
import sys
import time

import numpy as np

from . import gtls as _g

SDE_SCALE = 15.0
TAPS = (7, 5, 5, 5, 5, 5)        # the network of libgtls (include/gtls.h)
DILATION = (1, 2, 2, 4, 4, 8)
FRAC = 0.05
CHUNK = 256
N_BINS = _g.N_BINS
N_REG = _g.N_REG
WEIGHTS = os.path.join(os.path.dirname(os.path.abspath(__file__)), "weights", "proposal.npz")


# ---------------------------------------------------------------------------
# data
# ---------------------------------------------------------------------------

def _gen(args):
    seed, start, count = args
    import synth
    lcs = synth.batch_kepler_like(count, seed=seed, start=start)
    return [(lc.t, lc.y, lc.dy, dict(lc.injected), float(lc.baseline_days)) for lc in lcs]


def curve_chunks(seed, total, pool=None, chunk=CHUNK, start=0):
    """Curves start .. start+total-1 of the uneven-length Kepler-like
    sequence `seed`, in chunks of (t, y, dy, injected, baseline) tuples."""
    jobs = [(seed, start + s, min(chunk, total - s)) for s in range(0, total, chunk)]
    if pool is None:
        for j in jobs:
            yield _gen(j)
    else:
        yield from pool.imap(_gen, jobs)


def _pack(curves, dev):
    import torch
    cat = lambda k: torch.as_tensor(np.concatenate([c[k] for c in curves]), dtype=torch.float64,
                                    device=dev)
    offs = np.cumsum([0] + [c[0].size for c in curves]).astype(np.int64)
    return cat(0), cat(1), cat(2), offs


def plan_for(n, baseline, oversampling=3.0, periods=None, pmax=None):
    return _g.Plan(_g.PlanConfig(baseline_days=baseline, n_points=n, period_min_days=0.5,
                                 period_max_days=pmax if pmax else 0.5 * baseline,
                                 oversampling=oversampling, periods_days=periods))


def binned(net, curves, dev, stream=None):
    """Network input (device, len(curves) x 4096) and the binned curves
    (bin centre, mean flux) of every non-empty bin."""
    import torch
    t, y, dy, offs = _pack(curves, dev)
    b = len(curves)
    x = torch.empty((b, N_BINS), dtype=torch.float32, device=dev)
    mean = torch.empty_like(x)
    wsum = torch.empty_like(x)
    net.bin(t, y, dy, offs, x, mean=mean, wsum=wsum, stream=stream)
    m, w = mean.cpu().numpy(), wsum.cpu().numpy()
    out = []
    for i, c in enumerate(curves):
        t0, span = float(c[0].min()), float(c[0].max() - c[0].min())
        keep = w[i] > 0
        tb = t0 + (np.flatnonzero(keep) + 0.5) * span / N_BINS
        out.append((tb, 1.0 - m[i][keep].astype(np.float64), np.ones(int(keep.sum()))))
    return x, out


def targets(binned_curves, dev):
    """Region targets and masks (host, len x 128) from TLS on the binned curves."""
    import torch
    plans = [plan_for(c[0].size, float(c[0][-1] - c[0][0]), oversampling=1.0) for c in binned_curves]
    t, y, dy, offs = _pack(binned_curves, dev)
    batch = _g.Batch(plans)
    batch.search(t, y, dy, offs)
    tg = np.zeros((len(plans), N_REG), np.float32)
    mk = np.zeros((len(plans), N_REG), np.float32)
    for i, p in enumerate(plans):
        sde = torch.empty(p.n_periods, dtype=torch.float64, device=dev)
        batch.period_outputs(i, {"sde": sde})
        vals = np.clip(sde.cpu().numpy() / SDE_SCALE, 0.0, 1.0)
        tg[i], mk[i] = _g.region_targets(p.periods(), vals)
    batch.close()
    for p in plans:
        p.close()
    return tg, mk


def training_set(net, seed, total, dev, pool=None, log=None):
    """(x [device, total x 4096], target, mask [device, total x 128])."""
    import torch
    xs, ts, ms = [], [], []
    done = 0
    t0 = time.time()
    for chunk in curve_chunks(seed, total, pool):
        x, bc = binned(net, chunk, dev)
        tg, mk = targets(bc, dev)
        xs.append(x)
        ts.append(torch.as_tensor(tg, device=dev))
        ms.append(torch.as_tensor(mk, device=dev))
        done += len(chunk)
        if log:
            log(f"training set: {done}/{total} curves, {time.time() - t0:.1f} s")
    return torch.cat(xs), torch.cat(ts), torch.cat(ms)


# ---------------------------------------------------------------------------
# training
# ---------------------------------------------------------------------------

def init_params(seed):
    """He-normal weights (std sqrt(2 / fan_in)), zero biases, in the flat
    order of the C ABI."""
    rng = np.random.default_rng(seed)
    parts = []
    cin = 1
    for taps in TAPS:
        parts.append(rng.normal(0.0, math.sqrt(2.0 / (taps * cin)), 64 * taps * cin))
        parts.append(np.zeros(64))
        cin = 64
    feat = (N_BINS >> 6) * 64
    parts.append(rng.normal(0.0, math.sqrt(2.0 / feat), N_REG * feat))
    parts.append(np.zeros(N_REG))
    return np.concatenate(parts).astype(np.float32)


def train(net, x, tg, mk, epochs, batch, lr, seed=0, log=None):
    import torch
    n = x.shape[0]
    gen = torch.Generator(device=x.device)
    gen.manual_seed(seed)
    hist = []
    for ep in range(epochs):
        perm = torch.randperm(n, generator=gen, device=x.device)
        tot, cnt = 0.0, 0
        for s in range(0, n - batch + 1, batch):
            idx = perm[s:s + batch]
            xb = x.index_select(0, idx).contiguous()
            tb = tg.index_select(0, idx).contiguous()
            mb = mk.index_select(0, idx).contiguous()
            tot += net.train_step(xb, tb, mb, batch, lr)
            cnt += 1
        hist.append(tot / max(cnt, 1))
        if log:
            log(f"epoch {ep + 1}/{epochs}: loss {hist[-1]:.5f}")
    return hist


# ---------------------------------------------------------------------------
# proposal search
# ---------------------------------------------------------------------------

def scores_for(net, curves, dev):
    import torch
    x, _ = binned(net, curves, dev)
    s = torch.empty((len(curves), N_REG), dtype=torch.float32, device=dev)
    net.forward(x, len(curves), scores=s)
    return s.cpu().numpy()


def proposal_search(net, curves, full_plans, dev, tau, frac=FRAC, verify_sde=None, scores=None):
    """Search every curve on its proposed periods (or its whole grid when
    the proposal is not confident).  With verify_sde, a curve whose search of
    the proposed periods ends below that SDE is searched again on its whole
    grid (the second fallback: the proposal did not hold a detection).
    Returns (results, fallback flags, periods searched per curve)."""
    sc = scores_for(net, curves, dev) if scores is None else scores
    chosen, owned, fallback, searched = [], [], [], []
    for i, (c, fp) in enumerate(zip(curves, full_plans)):
        per = fp.periods()
        _, mask = _g.region_targets(per, np.zeros(per.size))
        conf = float(sc[i][mask > 0].max()) if mask.any() else 0.0
        if conf < tau:
            chosen.append(fp)
            fallback.append(True)
            searched.append(per.size)
            continue
        idx = _g.proposal_periods(per, sc[i], frac)
        sub = plan_for(c[0].size, c[4], periods=per[idx])
        owned.append(sub)
        chosen.append(sub)
        fallback.append(False)
        searched.append(idx.size)
    t, y, dy, offs = _pack(curves, dev)
    batch = _g.Batch(chosen)
    res = batch.search(t, y, dy, offs)
    batch.close()
    for p in owned:
        p.close()
    if verify_sde is not None:
        redo = [i for i in range(len(curves)) if not fallback[i] and res[i].sde < verify_sde]
        if redo:
            sub = [curves[i] for i in redo]
            t, y, dy, offs = _pack(sub, dev)
            batch = _g.Batch([full_plans[i] for i in redo])
            for i, r in zip(redo, batch.search(t, y, dy, offs)):
                res[i] = r
                fallback[i] = True
                searched[i] += full_plans[i].n_periods
            batch.close()
    return res, fallback, searched


def triage_search(net, curves, full_plans, dev, threshold, scores=None):
    """Search, on its whole grid, every curve whose largest region score
    reaches `threshold`; skip the others.  Returns (results with None for a
    skipped curve, number of curves searched)."""
    sc = scores_for(net, curves, dev) if scores is None else scores
    keep = []
    for i, fp in enumerate(full_plans):
        per = fp.periods()
        _, mask = _g.region_targets(per, np.zeros(per.size))
        conf = float(sc[i][mask > 0].max()) if mask.any() else 0.0
        if conf >= threshold:
            keep.append(i)
    res = [None] * len(curves)
    if keep:
        t, y, dy, offs = _pack([curves[i] for i in keep], dev)
        batch = _g.Batch([full_plans[i] for i in keep])
        for i, r in zip(keep, batch.search(t, y, dy, offs)):
            res[i] = r
        batch.close()
    return res, len(keep)


def triage_threshold(path=None):
    """The smaller of the two cross-validated triage thresholds of the
    evaluation record next to the weights (None without one)."""
    path = path or os.path.join(os.path.dirname(WEIGHTS), "proposal_eval.json")
    if not os.path.exists(path):
        return None
    with open(path) as f:
        rows = json.load(f).get("triage") or []
    return min(r["threshold"] for r in rows) if rows else None


def detected(res, inj, sde_min=9.0, rel=0.01):
    if not inj:
        return False
    return res.sde >= sde_min and abs(res.period - inj["period"]) / inj["period"] < rel


def evaluate(net, n_eval, seed, dev, taus, frac=FRAC, pool=None, log=None, verify_sde=None,
             verify_taus=(), start=0):
    """Recall (SDE >= 9, period within 1 %) and light curves per hour of the
    plain batched search and of the proposal search at every tau (and, with
    verify_sde, at every tau of verify_taus with the verification fallback),
    on curves start .. start+n_eval-1 of sequence `seed`; per curve, the injection, the
    plain result and the network's largest region score."""
    import torch
    curves = [c for ch in curve_chunks(seed, n_eval, pool, start=start) for c in ch]
    full = [plan_for(c[0].size, c[4]) for c in curves]
    t, y, dy, offs = _pack(curves, dev)
    batch = _g.Batch(full)
    batch.autotune(t, y, dy, offs)
    torch.cuda.synchronize()
    w0 = time.perf_counter()
    plain = batch.search(t, y, dy, offs)        # includes the graph capture (milliseconds)
    torch.cuda.synchronize()
    plain_s = time.perf_counter() - w0
    batch.close()
    inj = [c[3] for c in curves]
    n_inj = sum(1 for i in inj if i)
    out = {"curves": n_eval, "injected": n_inj, "seed": seed, "start": start, "frac": frac,
           "plain": {"recall": sum(detected(r, i) for r, i in zip(plain, inj)) / max(n_inj, 1),
                     "false_alarms": sum(1 for r, i in zip(plain, inj) if not i and r.sde >= 9.0),
                     "seconds": plain_s, "lc_per_hour": n_eval * 3600.0 / plain_s},
           "verify_sde": verify_sde, "learned": []}
    torch.cuda.synchronize()
    w0 = time.perf_counter()
    sc = scores_for(net, curves, dev)     # binning + network forward of every curve
    torch.cuda.synchronize()
    out["network_seconds"] = time.perf_counter() - w0
    per_curve = []
    for i, (c, r) in enumerate(zip(curves, plain)):
        _, mask = _g.region_targets(full[i].periods(), np.zeros(full[i].n_periods))
        per_curve.append({"n": int(c[0].size), "inj_period": c[3].get("period"),
                          "inj_depth": c[3].get("depth"), "plain_period": r.period,
                          "plain_sde": r.sde, "plain_detected": bool(detected(r, c[3])),
                          "score_max": float(sc[i][mask > 0].max())})
    out["per_curve"] = per_curve
    out["triage"] = triage(per_curve, out["plain"]["lc_per_hour"])
    runs = [(tau, None) for tau in taus] + [(tau, verify_sde) for tau in verify_taus if verify_sde]
    for tau, vs in runs:
        torch.cuda.synchronize()
        w0 = time.perf_counter()
        res, fb, searched = proposal_search(net, curves, full, dev, tau, frac, vs)
        torch.cuda.synchronize()
        s = time.perf_counter() - w0
        row = {"tau": tau, "verify_sde": vs,
               "recall": sum(detected(r, i) for r, i in zip(res, inj)) / max(n_inj, 1),
               "false_alarms": sum(1 for r, i in zip(res, inj) if not i and r.sde >= 9.0),
               "fallback": int(sum(fb)), "periods_searched": int(sum(searched)),
               "periods_total": int(sum(p.n_periods for p in full)),
               "seconds": s, "lc_per_hour": n_eval * 3600.0 / s}
        out["learned"].append(row)
        if log:
            log(f"tau {tau}: {row}")
    for p in full:
        p.close()
    return out


def weights_match(path=WEIGHTS):
    """True when `path` exists and holds weights of this network (taps and
    dilations)."""
    if not os.path.exists(path):
        return False
    _, meta = load_weights(path)
    return tuple(meta.get("taps", ())) == TAPS and tuple(meta.get("dilation", ())) == DILATION


def triage(per_curve, plain_lc_per_hour):
    """Curve triage by the network's largest region score, cross-validated on
    the two halves of the evaluation set: the score threshold that keeps every
    plain detection of one half is applied to the other half, whose curves
    below it are not searched at all.  Returns one row per direction: curves
    searched, plain detections kept, recall against plain recall, and the
    light curves per hour of the plain search divided by the fraction of
    curves searched (the network's own cost is reported separately)."""
    n = len(per_curve)
    score = np.array([c["score_max"] for c in per_curve])
    det = np.array([bool(c["plain_detected"]) for c in per_curve])
    inj = np.array([c["inj_period"] is not None for c in per_curve])
    first = np.arange(n) < n // 2
    rows = []
    for cal, test in ((first, ~first), (~first, first)):
        if not (cal & det).any():
            continue
        thr = float(score[cal & det].min())
        keep = test & (score >= thr)
        frac = keep.sum() / max(test.sum(), 1)
        rows.append({"threshold": thr, "curves": int(test.sum()), "searched": int(keep.sum()),
                     "detections_kept": int((keep & det).sum()), "detections_plain": int((test & det).sum()),
                     "recall": float((keep & det).sum() / max((test & inj).sum(), 1)),
                     "recall_plain": float((test & det).sum() / max((test & inj).sum(), 1)),
                     "lc_per_hour": float(plain_lc_per_hour / max(frac, 1e-9))})
    return rows


def load_weights(path=WEIGHTS):
    with np.load(path) as z:
        return z["params"].astype(np.float32), json.loads(str(z["meta"]))


# ---------------------------------------------------------------------------
# command line
# ---------------------------------------------------------------------------

def main(argv=None):
    ap = argparse.ArgumentParser(description=__doc__.split("\n")[0])
    sub = ap.add_subparsers(dest="cmd", required=True)
    tr = sub.add_parser("train")
    tr.add_argument("--train", type=int, default=4000)
    tr.add_argument("--seed", type=int, default=4)
    tr.add_argument("--epochs", type=int, default=30)
    tr.add_argument("--batch", type=int, default=128)
    tr.add_argument("--lr", type=float, default=1e-3)
    tr.add_argument("--out", default=WEIGHTS)
    tr.add_argument("--workers", type=int, default=8)
    ev = sub.add_parser("evaluate")
    ev.add_argument("--weights", default=WEIGHTS)
    ev.add_argument("--eval", type=int, default=64)
    ev.add_argument("--seed", type=int, default=5)
    ev.add_argument("--start", type=int, default=0, help="first held-out curve of the sequence")
    ev.add_argument("--taus", default="0.0,0.3,0.5")
    ev.add_argument("--frac", type=float, default=FRAC)
    ev.add_argument("--verify-sde", type=float, default=None)
    ev.add_argument("--verify-taus", default="",
                    help="taus evaluated again with the --verify-sde fallback")
    ev.add_argument("--json", default=None)
    ev.add_argument("--workers", type=int, default=8)
    a = ap.parse_args(argv)
    log = lambda m: print(m, file=sys.stderr, flush=True)
    # the generator pool starts before the first CUDA call
    pool = mp.get_context("spawn").Pool(a.workers) if a.workers > 0 else None
    import torch
    dev = torch.device("cuda", 0)
    torch.cuda.set_device(dev)
    if a.cmd == "train":
        net = _g.Cnn(max(a.batch, CHUNK), init_params(a.seed))
        t0 = time.time()
        x, tg, mk = training_set(net, a.seed, a.train, dev, pool, log)
        t_data = time.time() - t0
        t0 = time.time()
        hist = train(net, x, tg, mk, a.epochs, a.batch, a.lr, seed=a.seed, log=log)
        t_train = time.time() - t0
        meta = {"train_curves": a.train, "seed": a.seed, "epochs": a.epochs, "batch": a.batch,
                "lr": a.lr, "loss": hist, "data_seconds": t_data, "train_seconds": t_train,
                "sde_scale": SDE_SCALE, "target": "binned-curve TLS (oversampling 1) region SDE",
                "taps": list(TAPS), "dilation": list(DILATION)}
        os.makedirs(os.path.dirname(os.path.abspath(a.out)), exist_ok=True)
        np.savez_compressed(a.out, params=net.params(), meta=json.dumps(meta))
        log(json.dumps({k: v for k, v in meta.items() if k != "loss"}))
        net.close()
    else:
        params, meta = load_weights(a.weights)
        net = _g.Cnn(max(a.eval, 1), params)
        taus = [float(v) for v in a.taus.split(",")]
        vtaus = [float(v) for v in a.verify_taus.split(",") if v.strip()]
        out = evaluate(net, a.eval, a.seed, dev, taus, frac=a.frac, pool=pool, log=log, start=a.start,
                       verify_sde=a.verify_sde, verify_taus=vtaus)
        out["weights"] = {k: v for k, v in meta.items() if k != "loss"}
        print(json.dumps(out))
        if a.json:
            with open(a.json, "w") as f:
                json.dump(out, f, indent=1)
        net.close()
    if pool is not None:
        pool.close()
    return 0


if __name__ == "__main__":
    sys.exit(main())

#!/usr/bin/env python
"""Benchmark of the TLS period-grid search: Kepler-like light curves per hour.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl gtls|reference]
                    [--workload kepler_like|short_white|long_baseline]

One step is one complete search of one light curve (fold, sort, every
duration and T0 window, SR and SDE) on one GPU.  The default workload is the
Kepler-like 1460-day curve (29.4-min cadence with quarter gaps and 10 %
dropouts, ~64k points, period grid 0.5-730 d).  Under torchrun (N > 1) every
rank searches its own replica (weak scaling); there is no collective on the
data path.  Rank 0 prints one JSON line.

``--impl reference`` times the FP64 CPU oracle on the host cores on a
bounded sample of the same workload and prints the same JSON line.
"""

from __future__ import annotations

import argparse
import hashlib
import json
import math
import os
import statistics
import subprocess
import sys
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "Kepler-like light curves/hour on 1 GB300 (plain vs batched+learned, equal recall)"
UNIT = "light curves/hour"
FP32_LANES_PER_SM = 128          # FP32 FMA lanes per Blackwell SM (4 x 32)


def _args():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="gtls", choices=["gtls", "reference"])
    ap.add_argument("--workload", default="kepler_like",
                    choices=["kepler_like", "short_white", "long_baseline"])
    ap.add_argument("--cpu-seconds", type=float, default=15.0,
                    help="target CPU time of the oracle sample (cpu_baseline / reference step)")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--dt0", type=float, default=0.05,
                    help="T0 step as a fraction of the duration (Eq. N_skip; the paper's sweep uses "
                         "0.1 and 0.01)")
    ap.add_argument("--refine", type=int, default=0,
                    help="periods re-searched with T0 step 1 after the coarse pass (Sect. 2.5)")
    ap.add_argument("--dy-jitter", type=float, default=0.0,
                    help="multiply every dy by 1 + f * U(-1, 1) (seeded): per-point weights, which "
                         "the one-thread-per-window kernel searches")
    ap.add_argument("--batch-curves", type=int, default=8,
                    help="curves of the uneven-length Kepler-like batch leg (0 = skip it)")
    ap.add_argument("--batch-steps", type=int, default=2)
    ap.add_argument("--batch-warmup", type=int, default=1,
                    help="untimed batched and per-curve passes before the timed ones (0: the first "
                         "timed batched search includes the graph capture)")
    ap.add_argument("--no-learned", action="store_true",
                    help="skip the learned-proposal pipeline of the batched leg")
    ap.add_argument("--periods-per-chunk", type=int, default=0,
                    help="periods per kernel wave (0 = library default); small values shrink "
                         "the device footprint for profiler captures")
    return ap.parse_args()


def _dist():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


def max_over_ranks(x, device=None):
    """Largest x over the ranks of the default process group (x itself when
    the job is not distributed)."""
    import torch
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized()) or dist.get_world_size() == 1:
        return float(x)
    t = torch.tensor([float(x)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def job_rate(world_size, steps, seconds):
    """Light curves per hour of the whole job: every rank searched `steps`
    curves; the job took the slowest rank's time."""
    return world_size * steps * 3600.0 / seconds


def _workload(name):
    import synth
    return synth.make_workload(name)


def _describe(lc, info, dt0=0.05, refine=0, jitter=0.0):
    cfg = lc.search
    return {
        "workload": f"{lc.name}: {lc.baseline_days:.0f}-day baseline, n={lc.n} points, "
                    f"{info['n_periods']} trial periods {cfg['period_min_days']}-"
                    f"{cfg['period_max_days']:.0f} d (Ofir, OS=3), dt0={dt0:g}"
                    + (f", refinement of the {refine} best periods" if refine else "")
                    + (f", per-point dy (jitter {jitter:g})" if jitter else ""),
        "n_points": lc.n,
        "n_periods": info["n_periods"],
        "window_point_evaluations": info["wpe"],
        "seed": lc.seed,
        "l2": "flushed before every timed step (256 MiB write; L2 is 129 MB)",
    }


class ClockSampler:
    """nvidia-smi samples of SM clock and throttle reasons during the timed region."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index):
        self.gpu = gpu_index
        self.proc = None
        self.path = None

    def start(self):
        try:
            import tempfile
            fd, self.path = tempfile.mkstemp(prefix="gtls_clocks_", suffix=".csv")
            self.fh = os.fdopen(fd, "w")
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.gpu}", f"--query-gpu={self.FIELDS}",
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=self.fh, stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return None
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        self.fh.close()
        sm, smax, reasons = [], [], set()
        names = ["active", "hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown",
                 "sw_power_cap"]
        for line in open(self.path):
            parts = [p.strip() for p in line.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                smax.append(float(parts[2]))
            except ValueError:
                continue
            for nm, v in zip(names[1:], parts[5:9]):
                if v.lower() in ("active", "0x1", "1", "yes"):
                    reasons.add(nm)
        try:
            os.remove(self.path)
        except OSError:
            pass
        if not sm:
            return None
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(smax),
                "samples": len(sm), "reasons": sorted(reasons)}


def _kernel_sha():
    """Hash of the window-search kernel's code (comments and blank space
    removed): the k_window_tiles function, its warp tasks and the shared
    device structures."""
    import re

    def code(src):
        src = re.sub(r"/\*.*?\*/", " ", src, flags=re.S)
        src = re.sub(r"//[^\n]*", " ", src)
        return " ".join(src.split())

    csrc = os.path.join(ROOT, "paper_2607_00348_gb300", "csrc")
    search = open(os.path.join(csrc, "search.cu")).read()
    start = search.index("k_window_tiles(DevSet")
    body = search[start:search.index("\n}\n", start) + 3]
    h = hashlib.sha256()
    for part in (open(os.path.join(csrc, "gtls_internal.h")).read(),
                 open(os.path.join(csrc, "window_tiles.cuh")).read(), body):
        h.update(code(part).encode())
    return h.hexdigest()[:16]


def _ncu_traffic(workload):
    """DRAM bytes per window-search launch from the committed ncu summary
    (profiles/window_tiles_<workload>.md, lines 'kernel_sha: ...' and
    'dram_bytes_per_launch: ...'), if it was taken on the current kernel."""
    path = os.path.join(ROOT, "profiles", f"window_tiles_{workload}.md")
    vals = {}
    try:
        for line in open(path):
            for key in ("kernel_sha", "dram_bytes_per_launch"):
                if line.strip().startswith(key + ":"):
                    vals[key] = line.split(":", 1)[1].strip().strip("`")
    except OSError:
        return None
    if vals.get("kernel_sha") != _kernel_sha() or "dram_bytes_per_launch" not in vals:
        return None
    return float(vals["dram_bytes_per_launch"])


def oracle_sample(lc, cpu_seconds):
    """Time the FP64 oracle on a bounded, evenly spread subset of the periods.

    Returns (light curves/hour extrapolated by window-point evaluations,
    threads, sample description, sample seconds, WPE fraction sampled)."""
    import numpy as np
    from oracle import grid
    from oracle import search as osr
    cfg = lc.search
    op = osr.plan(lc.n, lc.baseline_days, period_min_days=cfg["period_min_days"],
                  period_max_days=cfg["period_max_days"])
    npd = op.periods.size
    d = op.dur_pts.astype(np.int64)
    st = np.array([grid.t0_stride(int(v), op.dt0) for v in d], dtype=np.int64)
    w_j = (-(-lc.n // st)) * d                       # ceil(n / st) windows of D points
    j = np.arange(d.size)[None, :]
    first = np.concatenate([[True], d[1:] != d[:-1]])[None, :]
    lo, hi = op.jlo[:, None], op.jhi[:, None]
    kept = (j >= lo) & (j <= hi) & ((j == lo) | first)
    wpe_p = (kept * w_j[None, :]).sum(axis=1).astype(np.float64)
    wpe_full = float(wpe_p.sum())
    threads = osr.threads_used()
    probe = np.linspace(0, npd - 1, min(npd, 2 * threads)).astype(np.int64)
    t0 = time.perf_counter()
    osr.search_periods(op, lc.t, lc.y, lc.dy, probe)
    rate = float(wpe_p[probe].sum()) / max(time.perf_counter() - t0, 1e-6)
    k = int(max(threads, min(npd, round(cpu_seconds * rate / (wpe_full / npd)))))
    sel = np.unique(np.linspace(0, npd - 1, k).astype(np.int64))
    t0 = time.perf_counter()
    osr.search_periods(op, lc.t, lc.y, lc.dy, sel)
    dt = time.perf_counter() - t0
    frac = float(wpe_p[sel].sum()) / wpe_full
    sec_full = dt / frac
    desc = (f"{sel.size} of {npd} periods evenly spread ({100 * frac:.2f} % of the window-point "
            f"evaluations), {dt:.1f} s on {threads} threads, extrapolated by WPE to "
            f"{sec_full:.0f} s per light curve")
    return 3600.0 / sec_full, threads, desc, dt, frac


def run_reference(args):
    ws, rank, _ = _dist()
    if rank != 0:
        return 0
    lc = _workload(args.workload)
    vals, secs, fracs = [], [], []
    last = None
    for i in range(args.warmup + args.steps):
        v, threads, desc, dt, frac = oracle_sample(lc, args.cpu_seconds)
        if i >= args.warmup:
            vals.append(v)
            secs.append(dt)
            fracs.append(frac)
        last = (threads, desc)
    value = statistics.median(vals)
    out = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": 0,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1000.0 * 3600.0 / value,
        # each step times the oracle on a period sample; ms_per_step is that
        # time scaled by window-point evaluations to one whole light curve
        "extrapolated": True, "sample_seconds": secs, "sample_wpe_fraction": fracs,
        "ms_per_step_basis": "oracle time of each step's period sample / its share of the "
                             "light curve's window-point evaluations (median over steps)",
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic (seeded numpy generator)",
        "config": {"workload": f"{lc.name}: n={lc.n} points, oracle on a period sample per step"},
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": last[0], "kind": "oracle",
                         "sample": last[1]},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(out), flush=True)
    return 0


def batch_leg(args, dev, stream):
    """Uneven-length Kepler-like curves (20k-72k points, noise 50-2000 ppm,
    30 % with a transit; seeded generator, seed 3): the batched search
    (autotuned waves, device work queue, graph replay) against one
    gtls_search per curve on the same curves.  Each timed step searches every
    curve once; L2 is flushed before every step.  The per-curve searches
    allocate each plan's chunk scratch before and free it after its search
    (outside the timed interval), so that any number of curves fits the
    device."""
    import numpy as np
    import torch

    import paper_2607_00348_gb300 as pkg
    import synth

    lcs = synth.batch_kepler_like(args.batch_curves, seed=3)
    plans = [pkg.Plan(pkg.PlanConfig(baseline_days=lc.baseline_days, n_points=lc.n,
                                     period_min_days=lc.search["period_min_days"],
                                     period_max_days=lc.search["period_max_days"]))
             for lc in lcs]
    cat = lambda f: torch.as_tensor(np.concatenate([getattr(lc, f) for lc in lcs]),
                                    dtype=torch.float64, device=dev)
    t, y, dy = cat("t"), cat("y"), cat("dy")
    offs = np.cumsum([0] + [lc.n for lc in lcs]).astype(np.int64)
    singles = [(torch.as_tensor(lc.t, device=dev), torch.as_tensor(lc.y, device=dev),
                torch.as_tensor(lc.dy, device=dev)) for lc in lcs]
    flush = torch.empty(256 << 20, dtype=torch.uint8, device=dev)
    batch = pkg.Batch(plans)
    batch.autotune(t, y, dy, offs, stream=stream)

    def timed_batch():
        for _ in range(args.batch_warmup):
            batch.search(t, y, dy, offs, stream=stream)   # graph capture, then replays
        ms = []
        for k in range(args.batch_steps):
            flush.fill_(k & 0xff)
            a = torch.cuda.Event(enable_timing=True)
            b = torch.cuda.Event(enable_timing=True)
            a.record(stream)
            out = batch.search(t, y, dy, offs, stream=stream)
            b.record(stream)
            torch.cuda.synchronize()
            ms.append(a.elapsed_time(b))
        return out, sum(ms) / len(ms)

    def timed_singles():
        def one(p, tr):
            p.reserve()
            a = torch.cuda.Event(enable_timing=True)
            b = torch.cuda.Event(enable_timing=True)
            a.record(stream)
            r = p.search(*tr, stream=stream)
            b.record(stream)
            torch.cuda.synchronize()
            p.trim()
            return r, a.elapsed_time(b)
        for _ in range(args.batch_warmup):
            for p, tr in zip(plans, singles):
                one(p, tr)
        ms = []
        for k in range(args.batch_steps):
            flush.fill_(k & 0xff)
            out, tot = [], 0.0
            for p, tr in zip(plans, singles):
                r, m = one(p, tr)
                out.append(r)
                tot += m
            ms.append(tot)
        return out, sum(ms) / len(ms)

    res_b, ms_b = timed_batch()
    res_s, ms_s = timed_singles()
    same = all(a.as_dict() == b.as_dict() for a, b in zip(res_b, res_s))
    info = batch.info()
    n = len(lcs)
    learned = None if args.no_learned else learned_leg(args, lcs, plans, res_b, dev)
    out = {"value": n * 3600e3 / ms_b, "unit": UNIT, "curves": n,
           "plain_value": n * 3600e3 / ms_s, "ms_per_step": ms_b, "plain_ms_per_step": ms_s,
           "identical_results": same, "points": int(offs[-1]),
           "periods": int(info.n_periods), "window_point_evaluations": float(info.wpe),
           "waves": int(info.waves), "wave_slots": int(info.wave_slots),
           "tile_floats": int(info.tile_floats), "graph_kernels": int(info.graph_kernels),
           "gpu_launches_per_step": int(info.last_launches), "warmup": args.batch_warmup,
           "steps": args.batch_steps,
           "plain_timing": "sum of CUDA-event times of the per-curve searches (scratch "
                           "allocated and freed outside them)",
           "workload": f"first {n} curves of the uneven-length Kepler-like batch (seed 3, "
                       "20k-72k points, 50-2000 ppm, 30 % injected)",
           "learned": learned}
    batch.close()
    for p in plans:
        p.close()
    return out


def learned_leg(args, lcs, plans, plain, dev):
    """The learned stage on the same curves: (1) the period proposal --
    network scores of the binned curves, a search of the proposed periods
    when the best score reaches tau, the whole grid otherwise or when that
    search ends below SDE 9; (2) triage -- the whole grid of the curves whose
    best score reaches the threshold calibrated on the held-out evaluation,
    no search for the others.  Wall clock of each pipeline, host steps
    included.  Detections: SDE >= 9 (and, for injected curves, the period
    within 1 %)."""
    import torch

    import paper_2607_00348_gb300 as pkg
    from paper_2607_00348_gb300 import proposal as pr
    if not pr.weights_match():
        return None
    params, meta = pr.load_weights()
    net = pkg.Cnn(len(lcs), params)
    curves = [(lc.t, lc.y, lc.dy, dict(lc.injected), float(lc.baseline_days)) for lc in lcs]
    tau, frac = 0.35, pr.FRAC
    pr.proposal_search(net, curves, plans, dev, tau, frac, verify_sde=9.0)   # warm-up
    torch.cuda.synchronize()
    w0 = time.perf_counter()
    res, fb, searched = pr.proposal_search(net, curves, plans, dev, tau, frac, verify_sde=9.0)
    torch.cuda.synchronize()
    sec = time.perf_counter() - w0
    det = lambda r, c: r is not None and r.sde >= 9.0 and (
        not c[3] or abs(r.period - c[3]["period"]) / c[3]["period"] < 0.01)
    out = {"value": len(lcs) * 3600.0 / sec, "unit": UNIT, "tau": tau, "frac": frac,
           "verify_sde": 9.0, "fallbacks": int(sum(fb)), "periods_searched": int(sum(searched)),
           "periods_total": int(sum(p.n_periods for p in plans)),
           "detections_plain": int(sum(det(r, c) for r, c in zip(plain, curves))),
           "detections_learned": int(sum(det(r, c) for r, c in zip(res, curves))),
           "weights": f"{meta['train_curves']} training curves (seed {meta['seed']})"}
    # triage: the whole grid of every curve the network scores above the
    # threshold calibrated on the held-out evaluation set, nothing for the rest
    thr = pr.triage_threshold()
    if thr is not None:
        pr.triage_search(net, curves, plans, dev, thr)    # warm-up
        torch.cuda.synchronize()
        w0 = time.perf_counter()
        tres, kept = pr.triage_search(net, curves, plans, dev, thr)
        torch.cuda.synchronize()
        tsec = time.perf_counter() - w0
        out["triage"] = {"value": len(lcs) * 3600.0 / tsec, "unit": UNIT, "threshold": thr,
                         "curves_searched": kept, "curves": len(lcs),
                         "detections_learned": int(sum(det(r, c) for r, c in zip(tres, curves))),
                         "detections_plain": out["detections_plain"],
                         "timing": "wall clock of scores + batched whole-grid searches"}
    net.close()
    return out


def run_gtls(args):
    import numpy as np
    import torch

    import paper_2607_00348_gb300 as pkg

    ws, rank, local = _dist()
    if not torch.cuda.is_available():
        raise SystemExit("bench.py needs a CUDA device")
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    if ws > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=dev)
    pkg.load()

    lc = _workload(args.workload)
    if args.dy_jitter > 0.0:
        import numpy as np
        rng = np.random.default_rng(12345)
        lc.dy = lc.dy * (1.0 + args.dy_jitter * rng.uniform(-1.0, 1.0, lc.n))
    cfg = lc.search
    plan = pkg.Plan(pkg.PlanConfig(baseline_days=lc.baseline_days, n_points=lc.n,
                                   period_min_days=cfg["period_min_days"],
                                   period_max_days=cfg["period_max_days"],
                                   periods_per_chunk=args.periods_per_chunk, dt0=args.dt0,
                                   refine_periods=args.refine))
    info = {"n_periods": plan.n_periods, "wpe": float(plan.info.wpe),
            "n_windows": int(plan.info.n_windows)}
    t = torch.as_tensor(lc.t, dtype=torch.float64, device=dev)
    y = torch.as_tensor(lc.y, dtype=torch.float64, device=dev)
    dy = torch.as_tensor(lc.dy, dtype=torch.float64, device=dev)
    flush = torch.empty(256 << 20, dtype=torch.uint8, device=dev)
    stream = torch.cuda.current_stream(dev)

    for _ in range(args.warmup):
        res = plan.search(t, y, dy, stream=stream)

    def barrier():
        if ws > 1:
            torch.distributed.barrier()

    plan.set_profiling(True)
    clocks = ClockSampler(local)
    starts = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
    ends = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
    win_ms, stage = [], []
    launches = 0
    barrier()
    torch.cuda.synchronize()
    clocks.start()
    for k in range(args.steps):
        flush.fill_(k & 0xff)                 # evict the previous step from L2
        starts[k].record(stream)
        res = plan.search(t, y, dy, stream=stream)
        ends[k].record(stream)
        pr = plan.profile()
        win_ms.append(pr.ms_window_search)
        stage.append(pr.as_dict())
        launches += int(pr.kernel_launches)
    torch.cuda.synchronize()
    barrier()
    clk = clocks.stop()
    plan.set_profiling(False)
    step_ms = [s.elapsed_time(e) for s, e in zip(starts, ends)]
    total_s = max_over_ranks(sum(step_ms) / 1000.0, dev)
    value = job_rate(ws, args.steps, total_s)

    # end to end: host arrays in pinned memory -> device -> result back
    e2e = None
    if not args.no_e2e:
        th = torch.from_numpy(lc.t).pin_memory()
        yh = torch.from_numpy(lc.y).pin_memory()
        dh = torch.from_numpy(lc.dy).pin_memory()
        plan.search_host(th.numpy(), yh.numpy(), dh.numpy(), stream=stream)
        barrier()
        torch.cuda.synchronize()
        w0 = time.perf_counter()
        for k in range(args.steps):
            plan.search_host(th.numpy(), yh.numpy(), dh.numpy(), stream=stream)
        w1 = time.perf_counter()
        e_s = max_over_ranks(w1 - w0, dev)
        import ctypes
        e2e = {"value": job_rate(ws, args.steps, e_s), "unit": UNIT,
               "h2d_bytes_per_step": 3 * 8 * lc.n,
               "d2h_bytes_per_step": ctypes.sizeof(pkg.Result) + 4}

    batched = None
    if args.batch_curves > 0 and rank == 0:
        batched = batch_leg(args, dev, stream)

    if rank != 0:
        plan.close()
        if ws > 1:
            torch.distributed.destroy_process_group()
        return 0

    props = torch.cuda.get_device_properties(dev)
    sm_max = (clk or {}).get("sm_max_mhz") or 2070.0
    peak_tflops = 2.0 * props.multi_processor_count * FP32_LANES_PER_SM * sm_max * 1e6 / 1e12
    win_s = statistics.mean(win_ms) / 1000.0
    # 1 FMA per window-point evaluation with uniform dy; 2 (w r s and w s^2)
    # with per-point dy
    flop_per_wpe = 2.0 if res.uniform_dy else 4.0
    achieved = flop_per_wpe * info["wpe"] / win_s / 1e12
    traffic = _ncu_traffic(args.workload)
    roofline = {"bound": "alu", "achieved": achieved, "peak": peak_tflops, "unit": "TFLOP/s",
                "frac": achieved / peak_tflops, "traffic": traffic,
                "kernel": "k_window_tiles",
                "peak_basis": f"{props.multi_processor_count} SMs x {FP32_LANES_PER_SM} FP32 FMA "
                              f"lanes x 2 flop x {sm_max:.0f} MHz (max SM clock)",
                "achieved_basis": f"{flop_per_wpe:.0f} flop x window-point evaluations / mean "
                                  "window-search stage time (CUDA events on the search stream)"}
    cpu = None
    if not args.no_cpu_baseline:
        v, threads, desc, dt, frac = oracle_sample(lc, args.cpu_seconds)
        cpu = {"value": v, "unit": UNIT, "cores": threads, "kind": "oracle", "sample": desc,
               "extrapolated": True, "sample_seconds": dt, "sample_wpe_fraction": frac}
    mean_stage = {k: statistics.mean(s[k] for s in stage) for k in
                  ("ms_prepare", "ms_fold_sort", "ms_window_search", "ms_finalize", "ms_sr_sde")}
    out = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": ws, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": 1000.0 * total_s / args.steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32",
        "data": "synthetic (seeded numpy generator, Kepler-like)",
        "config": dict(_describe(lc, info, args.dt0, args.refine, args.dy_jitter),
                       parallelism=f"replicas x{ws}"),
        "roofline": roofline, "cpu_baseline": cpu, "e2e": e2e,
        "gpu_launches": launches, "clocks": clk,
        "stage_ms": mean_stage, "batched": batched,
        "result": {"period": res.period, "sde": res.sde, "depth": res.depth,
                   "duration_days": res.duration_days},
    }
    print(json.dumps(out), flush=True)
    plan.close()
    if ws > 1:
        torch.distributed.destroy_process_group()
    return 0


def main():
    args = _args()
    if args.impl == "reference":
        return run_reference(args)
    return run_gtls(args)


if __name__ == "__main__":
    sys.exit(main())

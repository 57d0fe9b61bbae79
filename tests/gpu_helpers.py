"""Shared helpers of the GPU tests: run the library through its C ABI."""

import numpy as np

import paper_2607_00348_gb300 as pkg
from oracle import search as osr


def plan_for(lc_or_n, baseline, cfg=None, **kw):
    cfg = dict(cfg or {})
    cfg.update(kw)
    n = lc_or_n if isinstance(lc_or_n, int) else lc_or_n.n
    pc = pkg.PlanConfig(baseline_days=baseline, n_points=n,
                        period_min_days=cfg.get("period_min_days") or 0.0,
                        period_max_days=cfg.get("period_max_days") or 0.0,
                        dt0=cfg.get("dt0", 0.05), dur_ratio=cfg.get("dur_ratio", 1.1),
                        k_min=cfg.get("k_min", 20.05), k_max=cfg.get("k_max", 620.84),
                        q_cap=cfg.get("q_cap", 0.15), oversampling=cfg.get("oversampling", 3.0),
                        periods_days=cfg.get("periods_days"),
                        refine_periods=cfg.get("refine_periods", 0))
    return pkg.Plan(pc)


def oracle_plan_for(n, baseline, cfg=None, **kw):
    cfg = dict(cfg or {})
    cfg.update(kw)
    return osr.plan(n, baseline, period_min_days=cfg.get("period_min_days"),
                    period_max_days=cfg.get("period_max_days"), dt0=cfg.get("dt0", 0.05),
                    dur_ratio=cfg.get("dur_ratio", 1.1), k_min=cfg.get("k_min", 20.05),
                    k_max=cfg.get("k_max", 620.84), q_cap=cfg.get("q_cap", 0.15),
                    oversampling=cfg.get("oversampling", 3.0),
                    periods_days=cfg.get("periods_days"))


def period_buffers(npd):
    import torch
    dev = torch.device("cuda:0")
    f64 = dict(dtype=torch.float64, device=dev)
    i32 = dict(dtype=torch.int32, device=dev)
    return dict(chi2=torch.empty(npd, **f64), dur_idx=torch.empty(npd, **i32),
                t0_idx=torch.empty(npd, **i32), depth=torch.empty(npd, **f64),
                t0=torch.empty(npd, **f64), sr=torch.empty(npd, **f64),
                sde_raw=torch.empty(npd, **f64), sde=torch.empty(npd, **f64),
                refined=torch.empty(npd, **i32))


def batch_outputs(batch, lc, npd):
    import torch
    outs = period_buffers(npd)
    batch.period_outputs(lc, outs)
    torch.cuda.synchronize()
    return {k: v.cpu().numpy() for k, v in outs.items()}


def gpu_search(plan, t, y, dy):
    import torch
    dev = torch.device("cuda:0")
    tt = torch.as_tensor(np.ascontiguousarray(t), dtype=torch.float64, device=dev)
    yy = torch.as_tensor(np.ascontiguousarray(y), dtype=torch.float64, device=dev)
    dd = torch.as_tensor(np.ascontiguousarray(dy), dtype=torch.float64, device=dev)
    npd = plan.n_periods
    outs = dict(chi2=torch.empty(npd, dtype=torch.float64, device=dev),
                dur_idx=torch.empty(npd, dtype=torch.int32, device=dev),
                t0_idx=torch.empty(npd, dtype=torch.int32, device=dev),
                depth=torch.empty(npd, dtype=torch.float64, device=dev),
                t0=torch.empty(npd, dtype=torch.float64, device=dev),
                sr=torch.empty(npd, dtype=torch.float64, device=dev),
                sde_raw=torch.empty(npd, dtype=torch.float64, device=dev),
                sde=torch.empty(npd, dtype=torch.float64, device=dev),
                refined=torch.empty(npd, dtype=torch.int32, device=dev))
    res = plan.search(tt, yy, dd, per_period=outs)
    torch.cuda.synchronize()
    return res, {k: v.cpu().numpy() for k, v in outs.items()}

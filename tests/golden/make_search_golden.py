"""Write the full-grid oracle spectra of the two long workloads.

Usage:  python tests/golden/make_search_golden.py [kepler_like] [long_baseline]

For each workload this runs the FP64 oracle (``oracle.search.full_search``,
no refinement) over every trial period of its grid and stores, per period,
chi2(P), the index of the best duration and of the best T0 start and the
fitted depth, in ``tests/golden/search_<workload>.npz``; the best candidate
(argmax SDE, Sect. 2.4) and the provenance go to
``tests/golden/search_<workload>.json``.  SR and SDE are not stored: the
tests recompute them from the stored chi2(P) with the oracle's own
``sr_sde``.

Only ``synth`` (inputs) and ``oracle`` (arithmetic) are called; nothing here
touches the CUDA library.  SHA-256 digests of the inputs and of the oracle's
grids are stored so that a test can tell whether the machine it runs on
regenerates the same inputs and grids bit for bit.  The period grid itself is
stored too: the C library's pow and cbrt may round the last bit differently on
another architecture, and the test then searches the stored grid (an explicit
period list) so that both sides fold on the same periods.
"""

from __future__ import annotations

import hashlib
import json
import os
import platform
import sys
import time

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(os.path.dirname(HERE))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

import synth                      # noqa: E402
from oracle import grid           # noqa: E402
from oracle import search as osr  # noqa: E402

ORACLE_FLAGS = "gcc -O2 -std=c11 -ffp-contract=off -fno-fast-math -fopenmp"


def digest(*arrays) -> str:
    h = hashlib.sha256()
    for a in arrays:
        a = np.ascontiguousarray(a)
        h.update(str(a.dtype).encode())
        h.update(a.tobytes())
    return h.hexdigest()


def oracle_plan(lc):
    cfg = lc.search
    return osr.plan(lc.n, lc.baseline_days, period_min_days=cfg["period_min_days"],
                    period_max_days=cfg["period_max_days"], oversampling=cfg["oversampling"],
                    m_star=cfg["m_star"], r_star=cfg["r_star"], u1=cfg["u1"], u2=cfg["u2"])


def grid_digest(op, t) -> str:
    _, p_int, _ = grid.phase_lattice(t, op.periods, op.e)
    return digest(op.periods, p_int, op.dur_pts, op.jlo, op.jhi, op.tmpl)


def make(name: str) -> None:
    lc = synth.make_workload(name)
    op = oracle_plan(lc)
    t_start = time.time()
    r, sr, raw, sde, best = osr.full_search(op, lc.t, lc.y, lc.dy)
    secs = time.time() - t_start
    out = os.path.join(HERE, f"search_{name}")
    _, p_int, _ = grid.phase_lattice(lc.t, op.periods, op.e)
    np.savez_compressed(out + ".npz", chi2=r.chi2.astype(np.float64),
                        j_best=r.j_best.astype(np.int16), s_best=r.s_best.astype(np.int32),
                        depth=r.depth.astype(np.float32), periods=op.periods,
                        dur_pts=op.dur_pts.astype(np.int32), jlo=op.jlo.astype(np.int16),
                        jhi=op.jhi.astype(np.int16))
    meta = dict(
        _about=("Full-grid FP64 oracle results (oracle.search.full_search, no refinement) "
                "written by tests/golden/make_search_golden.py; no value comes from the "
                "CUDA library."),
        workload=name, seed=lc.seed, n_points=lc.n, n_periods=int(op.periods.size),
        baseline_days=lc.baseline_days, search=lc.search, dt0=op.dt0, time_exponent=op.e,
        inputs_sha256=digest(lc.t, lc.y, lc.dy), grid_sha256=grid_digest(op, lc.t),
        periods_sha256=digest(op.periods, p_int), durations_sha256=digest(op.dur_pts, op.jlo, op.jhi),
        best=best, oracle_build=ORACLE_FLAGS, oracle_threads=osr.threads_used(),
        oracle_seconds=round(secs, 1), machine=platform.machine(), numpy=np.__version__,
        stored=dict(chi2="float64", j_best="int16 (global duration index)",
                    s_best="int32 (T0 start index in folded order)",
                    depth="float32 (rounded from FP64)", periods="float64 (days)",
                    dur_pts="int32", jlo="int16", jhi="int16"))
    with open(out + ".json", "w") as fh:
        json.dump(meta, fh, indent=1, sort_keys=True)
        fh.write("\n")
    print(f"{name}: {op.periods.size} periods in {secs:.0f} s; best P = {best['period']:.6f} d, "
          f"SDE {best['sde']:.3f}")


if __name__ == "__main__":
    names = sys.argv[1:] or ["kepler_like", "long_baseline"]
    for nm in names:
        make(nm)

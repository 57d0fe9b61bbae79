"""Brute-force TLS chi2 on tiny inputs (pins the oracle's decomposition).

For a trial period the points are put in phase order with numpy's stable
argsort of the exact lattice phase; a window of D points starting at folded
position s (wrapping around phase 1 -> 0) gets the model 1 - delta * s_k,
every other point the model 1, and chi2 is summed over all N original
points.  No padding, no edge term, no cumulative sums.
"""

import numpy as np

from oracle import grid


def folded_order(d_lat, p_int):
    rho = d_lat % p_int
    return np.argsort(rho, kind="stable")


def window_chi2(y, dy, order, d, s, tmpl):
    n = y.size
    pos = (s + np.arange(d)) % n
    members = order[pos]
    depth = max(0.0, float(np.mean(1.0 - y[members])) / float(np.mean(tmpl)))
    model = np.ones(n)
    model[members] = 1.0 - depth * tmpl
    z = (y - model) / dy
    return float(np.sum(z * z)), depth


def period_windows(plan, t, y, dy, period_idx, j):
    d_lat, p_int, _ = grid.phase_lattice(t, plan.periods, plan.e)
    order = folded_order(d_lat, p_int[period_idx])
    d = int(plan.dur_pts[j])
    tmpl = plan.tmpl[plan.tmpl_off[j]:plan.tmpl_off[j] + d]
    st = grid.t0_stride(d, plan.dt0)
    out, deps = [], []
    for s in range(0, t.size, st):
        c, dep = window_chi2(y, dy, order, d, s, tmpl)
        out.append(c)
        deps.append(dep)
    return np.array(out), np.array(deps)


def period_min(plan, t, y, dy, period_idx):
    best = (np.inf, -1, -1, 0.0)
    for j in grid.kept_durations(plan.dur_pts, plan.jlo[period_idx], plan.jhi[period_idx]):
        c, dep = period_windows(plan, t, y, dy, period_idx, j)
        st = grid.t0_stride(int(plan.dur_pts[j]), plan.dt0)
        m = int(np.argmin(c))
        if c[m] < best[0]:
            best = (float(c[m]), j, m * st, float(dep[m]))
    return best

"""The phase lattice (the reading of Eq. phase) against exact rational folding.

Both the oracle and the library fold on a lattice of 2^-e days: d_i =
rint((t_i - t_ref) 2^e), P_lat = rint(P 2^e), rho_i = d_i mod P_lat, and sort
by (rho_i, i).  Here the same FP64 time stamps and trial periods are folded
in exact rational arithmetic (Python integers at the resolution of the
finest FP64 value involved): rho_i = (t_i - t_ref) mod P exactly, sorted by
(rho_i, i).  The lattice may only differ from that order between points whose
exact phases lie within the lattice's own error bound

    |rho_lat - rho_exact| <= 1/2 + 2^(e-53) S + c/2   lattice units,

(rounding of t_i - t_ref, of d_i and of P_lat accumulated over c cycles,
S the baseline in days), so:

  * no two points whose exact phases are further apart than twice the bound
    come out in the wrong order (checked pair by pair along the lattice
    order, circularly);
  * where no two exact phases are that close, the two orders are identical,
    and so is everything computed from them (chi2, argmins);
  * where they are that close (time stamps commensurate with the period up
    to FP64 rounding: on the 1440-point curve the last trial period,
    15.000000000000007 d, is 720 cadences, and 720 pairs of points lie
    7e-15 d apart) the exact order follows the rounding noise of the time
    stamps and the lattice treats the pair as a tie, ordered by index.
    These periods are counted and their chi2 difference is bounded here.
"""

import math

import numpy as np
import pytest

import synth
from oracle import grid
from oracle import search as osr


def _exact_scale(values):
    """L such that every value times 2^L is an integer."""
    lg = 0
    for v in values:
        if v != 0.0:
            lg = max(lg, 53 - math.frexp(abs(float(v)))[1])
    return lg


def _to_int(v, lg):
    num, den = float(v).as_integer_ratio()
    return num * ((1 << lg) // den)


class ExactFold:
    """Exact phases of one light curve's FP64 time stamps."""

    def __init__(self, t, periods):
        self.lg = _exact_scale(list(t) + list(periods))
        self.ti = [_to_int(v, self.lg) for v in t]
        self.tref = min(self.ti)
        self.n = len(self.ti)

    def phases(self, period):
        p = _to_int(period, self.lg)
        return [(x - self.tref) % p for x in self.ti], p

    @staticmethod
    def order(rho):
        return np.array(sorted(range(len(rho)), key=rho.__getitem__), dtype=np.int64)


def _bound_exact(e, lg, baseline, period):
    """Lattice error bound of one phase, in exact units (2^-lg days)."""
    cycles = math.ceil(baseline / period) + 1
    units = 0.5 + math.ldexp(baseline, e - 53) + 0.5 * cycles + 1e-9
    return math.ceil(units * 2 ** (lg - e)) + 1


def _check_period(ef, rho_ex, p_ex, order_lat, bound):
    """Returns (near_tie, orders_equal); asserts the lattice never inverts
    points further apart than twice the bound (circular differences)."""
    n = len(rho_ex)
    a = order_lat
    worst = 0
    for k in range(n):
        d = (rho_ex[a[(k + 1) % n]] - rho_ex[a[k]]) % p_ex
        back = p_ex - d
        if k == n - 1:
            continue          # the wrap from the last point to the first
        if back < d:
            worst = max(worst, back)
    assert worst <= 2 * bound, (worst, bound)
    srt = sorted(rho_ex)
    gaps = [srt[k + 1] - srt[k] for k in range(n - 1)] + [srt[0] + p_ex - srt[-1]]
    near_tie = min(gaps) <= 2 * bound or max(rho_ex) >= p_ex - bound
    order_ex = ef.order(rho_ex)
    return near_tie, bool(np.array_equal(order_ex, order_lat)), order_ex


def _sample(npd, k, extra=()):
    base = np.linspace(0, npd - 1, k).astype(np.int64)
    return np.unique(np.concatenate([base, np.arange(0, 5), np.arange(npd - 5, npd),
                                     np.asarray(extra, np.int64)]))


def _run(lc, sel):
    cfg = lc.search
    op = osr.plan(lc.n, lc.baseline_days, period_min_days=cfg["period_min_days"],
                  period_max_days=cfg["period_max_days"])
    d_lat, p_int, t_ref = grid.phase_lattice(lc.t, op.periods, op.e)
    ef = ExactFold(lc.t, op.periods)
    differ, ties = [], []
    for k in sel:
        rho_ex, p_ex = ef.phases(op.periods[k])
        order_lat = osr.fold_order(d_lat, p_int[k])
        bound = _bound_exact(op.e, ef.lg, lc.baseline_days, float(op.periods[k]))
        near_tie, same, order_ex = _check_period(ef, rho_ex, p_ex, order_lat, bound)
        if near_tie:
            ties.append(int(k))
        else:
            assert same, k          # no near ties: the lattice order is the exact order
        if not same:
            # chi2 and argmin of the exact order, through the oracle with a
            # lattice whose phases are the exact ranks
            rank = np.empty(lc.n, np.int64)
            rank[order_ex] = np.arange(lc.n)
            p_rank = p_int.copy()
            p_rank[k] = lc.n + 1
            r_lat = osr.search_periods_lattice(op, d_lat, p_int, t_ref, lc.y, lc.dy, [k])
            r_ex = osr.search_periods_lattice(op, rank, p_rank, t_ref, lc.y, lc.dy, [k])
            differ.append((int(k), abs(r_lat.chi2[0] - r_ex.chi2[0]) / r_lat.chi2[0],
                           (int(r_lat.j_best[0]), int(r_lat.s_best[0])) ==
                           (int(r_ex.j_best[0]), int(r_ex.s_best[0]))))
    return op, differ, ties


def test_short_white_every_period():
    lc = synth.short_white()
    cfg = lc.search
    npd = grid.period_grid_days(lc.baseline_days, period_min_days=cfg["period_min_days"],
                                period_max_days=cfg["period_max_days"]).size
    op, differ, ties = _run(lc, np.arange(npd))
    # the only departure: the last trial period, 720 cadences of 30 min up to
    # FP64 rounding, where 720 pairs of points tie on the lattice
    assert [k for k, _, _ in differ] == [npd - 1]
    assert op.periods[npd - 1] * 48.0 == pytest.approx(720.0, abs=1e-9)
    assert ties == [npd - 1]
    k, rel, same_argmin = differ[0]
    assert rel < 1e-3


@pytest.mark.parametrize("name,count", [("kepler_like", 36), ("long_baseline", 24)])
def test_long_curves_sampled_periods(name, count):
    lc = synth.make_workload(name)
    cfg = lc.search
    periods = grid.period_grid_days(lc.baseline_days, period_min_days=cfg["period_min_days"],
                                    period_max_days=cfg["period_max_days"])
    near = int(np.argmin(np.abs(periods - lc.injected["period"])))
    sel = _sample(periods.size, count, extra=(near - 1, near, near + 1))
    op, differ, ties = _run(lc, sel)
    # every sampled order is the exact one (near ties within the bound occur
    # at the shortest periods, where c reaches thousands of cycles, but the
    # lattice still orders them as the exact phases do)
    assert differ == []

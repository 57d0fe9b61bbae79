"""Seeded synthetic light curves shared by the oracle, the tests and the bench.

This module only draws inputs (times, fluxes, uncertainties and the injected
transit parameters).  It holds none of the search's arithmetic: no period or
duration grid, no folding, no template table, no chi-squared.
"""

from .lightcurves import (  # noqa: F401
    LightCurve,
    transit_profile,
    short_white,
    kepler_like,
    long_baseline,
    batch_kepler_like,
    noiseless_one_point_per_cycle,
    WORKLOADS,
    make_workload,
)

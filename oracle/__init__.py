"""FP64 CPU oracle for the TLS period-grid search (test infrastructure).

This package is test infrastructure, not part of the product path.  Only
``tests/``, ``__graft_entry__.smoke()`` and the ``cpu_baseline`` /
``--impl reference`` legs of ``bench.py`` may import, call, link or run
anything under ``oracle/``.  It shares no code, header, table or constant
generator with the CUDA library; the only code both sides use is the seeded
input generator in ``synth/``.

Contents
--------
grid.py        period grid (Sect. 2.2.1), duration grid (Sect. 2.2.2),
               transit template and the exact integer phase lattice.
tls_oracle.c   per-period fold, sort, padding, edge term, cumulative sums,
               out-of-transit and in-transit chi^2 (Sect. 2.3), plus the
               running median used by SDE (Sect. 2.4).  Plain C, FP64.
search.py      ctypes driver: builds the tables with grid.py, runs the C
               core over a set of periods and reduces to SR / SDE.

Parity status: every function is pinned by ``tests/test_oracle_*.py`` except
the median-filter window of the SDE detrending (Sect. 2.4 gives no window),
whose choice is a reading, checked only against numpy's median.
"""

"""GB300 TLS period-grid search (libgtls) and its ctypes binding.

The search itself lives in ``csrc/`` (CUDA for sm_103a behind the C ABI of
``include/gtls.h``); :mod:`.gtls` marshals arguments to it.
"""

from .gtls import (  # noqa: F401
    Batch,
    BatchInfo,
    Cnn,
    GtlsError,
    Plan,
    PlanConfig,
    Result,
    load,
    library_path,
    proposal_periods,
    region_targets,
    search_batch,
)
from .build import build as build_library  # noqa: F401

"""ctypes binding of libgtls (argument marshalling only).

The names follow the C ABI in ``include/gtls.h``: ``gtls_plan_create``,
``gtls_search``, ``gtls_search_host``, ``gtls_search_batch``,
``gtls_batch_create`` / ``gtls_batch_search`` / ``gtls_batch_autotune``,
``gtls_plan_destroy``.  Every step of the search runs in the library's CUDA
kernels; this module never computes any part of it.  Loading fails loudly
when the library has not been built.
"""

from __future__ import annotations

import ctypes
import dataclasses
import os
import threading

import numpy as np

from . import build as _build

_lock = threading.Lock()
_lib = None

c_double_p = ctypes.POINTER(ctypes.c_double)
c_int32_p = ctypes.POINTER(ctypes.c_int32)
c_int64_p = ctypes.POINTER(ctypes.c_int64)

STATUS = {0: "GTLS_OK", 1: "GTLS_ERR_INVALID_ARG", 2: "GTLS_ERR_CUDA", 3: "GTLS_ERR_OOM",
          4: "GTLS_ERR_TIMEOUT", 5: "GTLS_ERR_INTERNAL"}


class GtlsError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__(f"{STATUS.get(status, status)}: {msg}")
        self.status = status


class PlanParams(ctypes.Structure):
    _fields_ = [("baseline_days", ctypes.c_double), ("n_points", ctypes.c_int64),
                ("m_star", ctypes.c_double), ("r_star", ctypes.c_double),
                ("oversampling", ctypes.c_double), ("period_min_days", ctypes.c_double),
                ("period_max_days", ctypes.c_double), ("k_min", ctypes.c_double),
                ("k_max", ctypes.c_double), ("q_cap", ctypes.c_double),
                ("dur_ratio", ctypes.c_double), ("dt0", ctypes.c_double),
                ("u1", ctypes.c_double), ("u2", ctypes.c_double),
                ("median_window", ctypes.c_int32), ("periods_per_chunk", ctypes.c_int32),
                ("periods_days", c_double_p), ("n_periods", ctypes.c_int64),
                ("refine_periods", ctypes.c_int32), ("test_flags", ctypes.c_int32)]


class PlanInfo(ctypes.Structure):
    _fields_ = [("n_periods", ctypes.c_int64), ("n_points", ctypes.c_int64),
                ("n_durations", ctypes.c_int32), ("time_exponent", ctypes.c_int32),
                ("max_duration_points", ctypes.c_int64), ("n_windows", ctypes.c_int64),
                ("wpe", ctypes.c_double), ("device_bytes", ctypes.c_int64),
                ("median_window", ctypes.c_int32), ("periods_per_chunk", ctypes.c_int32)]


class Result(ctypes.Structure):
    _fields_ = [("period", ctypes.c_double), ("duration_days", ctypes.c_double),
                ("t0", ctypes.c_double), ("depth", ctypes.c_double), ("sde", ctypes.c_double),
                ("chi2", ctypes.c_double), ("chi2_min", ctypes.c_double),
                ("chi2_0", ctypes.c_double), ("period_idx", ctypes.c_int64),
                ("dur_idx", ctypes.c_int32), ("dur_points", ctypes.c_int32),
                ("t0_idx", ctypes.c_int64), ("uniform_dy", ctypes.c_int32),
                ("refined", ctypes.c_int32), ("snr", ctypes.c_double)]

    def as_dict(self):
        return {f: getattr(self, f) for f, _ in self._fields_ if not f.startswith("reserved")}


class Profile(ctypes.Structure):
    _fields_ = [("ms_prepare", ctypes.c_double), ("ms_fold_sort", ctypes.c_double),
                ("ms_window_search", ctypes.c_double), ("ms_finalize", ctypes.c_double),
                ("ms_sr_sde", ctypes.c_double), ("kernel_launches", ctypes.c_int64),
                ("window_search_launches", ctypes.c_int64), ("enabled", ctypes.c_int32),
                ("reserved0", ctypes.c_int32)]

    def as_dict(self):
        return {f: getattr(self, f) for f, _ in self._fields_ if not f.startswith("reserved")}


class PeriodOutputs(ctypes.Structure):
    _fields_ = [("chi2", ctypes.c_void_p), ("dur_idx", ctypes.c_void_p),
                ("t0_idx", ctypes.c_void_p), ("depth", ctypes.c_void_p),
                ("t0", ctypes.c_void_p), ("sr", ctypes.c_void_p),
                ("sde_raw", ctypes.c_void_p), ("sde", ctypes.c_void_p),
                ("refined", ctypes.c_void_p)]


class BatchInfo(ctypes.Structure):
    _fields_ = [("n_lc", ctypes.c_int64), ("n_points", ctypes.c_int64),
                ("n_periods", ctypes.c_int64), ("wpe", ctypes.c_double),
                ("waves", ctypes.c_int32), ("wave_slots", ctypes.c_int32),
                ("tile_floats", ctypes.c_int32), ("graph_kernels", ctypes.c_int32),
                ("last_launches", ctypes.c_int64), ("device_bytes", ctypes.c_int64),
                ("tuned", ctypes.c_int32), ("reserved0", ctypes.c_int32),
                ("tuned_flops", ctypes.c_double)]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_ if not k.startswith("reserved")}


# (name, restype, argtypes) of every symbol declared in include/gtls.h
SIGNATURES = [
    ("gtls_plan_params_default", None, [ctypes.POINTER(PlanParams)]),
    ("gtls_plan_create", ctypes.c_int, [ctypes.POINTER(PlanParams), ctypes.POINTER(ctypes.c_void_p)]),
    ("gtls_plan_get_info", ctypes.c_int, [ctypes.c_void_p, ctypes.POINTER(PlanInfo)]),
    ("gtls_plan_get_periods", ctypes.c_int, [ctypes.c_void_p, c_double_p]),
    ("gtls_plan_get_durations", ctypes.c_int, [ctypes.c_void_p, c_double_p, c_int32_p]),
    ("gtls_plan_get_ranges", ctypes.c_int, [ctypes.c_void_p, c_int32_p, c_int32_p]),
    ("gtls_search", ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p,
                                   ctypes.c_void_p, ctypes.c_int64, ctypes.c_void_p,
                                   ctypes.POINTER(Result), ctypes.POINTER(PeriodOutputs)]),
    ("gtls_search_host", ctypes.c_int, [ctypes.c_void_p, c_double_p, c_double_p, c_double_p,
                                        ctypes.c_int64, ctypes.c_void_p, ctypes.POINTER(Result)]),
    ("gtls_search_batch", ctypes.c_int, [ctypes.POINTER(ctypes.c_void_p), ctypes.c_int64,
                                         ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p,
                                         c_int64_p, ctypes.c_void_p, ctypes.POINTER(Result)]),
    ("gtls_batch_create", ctypes.c_int, [ctypes.POINTER(ctypes.c_void_p), ctypes.c_int64,
                                         ctypes.c_int32, ctypes.POINTER(ctypes.c_void_p)]),
    ("gtls_batch_search", ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p,
                                         ctypes.c_void_p, c_int64_p, ctypes.c_void_p,
                                         ctypes.POINTER(Result)]),
    ("gtls_batch_autotune", ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p,
                                           ctypes.c_void_p, c_int64_p, ctypes.c_void_p]),
    ("gtls_batch_get_info", ctypes.c_int, [ctypes.c_void_p, ctypes.POINTER(BatchInfo)]),
    ("gtls_batch_get_period_outputs", ctypes.c_int, [ctypes.c_void_p, ctypes.c_int64,
                                                     ctypes.POINTER(PeriodOutputs),
                                                     ctypes.c_void_p]),
    ("gtls_batch_destroy", None, [ctypes.c_void_p]),
    ("gtls_plan_set_profiling", ctypes.c_int, [ctypes.c_void_p, ctypes.c_int32]),
    ("gtls_plan_reserve", ctypes.c_int, [ctypes.c_void_p]),
    ("gtls_plan_trim", ctypes.c_int, [ctypes.c_void_p]),
    ("gtls_plan_get_profile", ctypes.c_int, [ctypes.c_void_p, ctypes.POINTER(Profile)]),
    ("gtls_sr_sde_noalloc", ctypes.c_int, [ctypes.c_void_p, ctypes.c_int64, ctypes.c_int32,
                                            ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p,
                                            ctypes.c_void_p, c_int64_p, c_double_p]),
    ("gtls_cnn_param_count", ctypes.c_int64, []),
    ("gtls_cnn_create", ctypes.c_int, [ctypes.c_int32, ctypes.c_void_p,
                                       ctypes.POINTER(ctypes.c_void_p)]),
    ("gtls_cnn_get_params", ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p]),
    ("gtls_cnn_set_params", ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p]),
    ("gtls_cnn_bin", ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p,
                                    ctypes.c_void_p, c_int64_p, ctypes.c_int64, ctypes.c_void_p,
                                    ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p]),
    ("gtls_cnn_forward", ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int32,
                                        ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p]),
    ("gtls_cnn_gradient", ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p,
                                         ctypes.c_void_p, ctypes.c_int32, ctypes.c_void_p,
                                         c_double_p, ctypes.c_void_p]),
    ("gtls_cnn_train_step", ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p,
                                           ctypes.c_void_p, ctypes.c_int32, ctypes.c_float,
                                           c_double_p, ctypes.c_void_p]),
    ("gtls_cnn_destroy", None, [ctypes.c_void_p]),
    ("gtls_region_targets", ctypes.c_int, [c_double_p, c_double_p, ctypes.c_int64,
                                           ctypes.c_void_p, ctypes.c_void_p]),
    ("gtls_proposal_periods", ctypes.c_int, [c_double_p, ctypes.c_int64, ctypes.c_void_p,
                                             ctypes.c_double, c_int64_p, c_int64_p]),
    ("gtls_plan_destroy", None, [ctypes.c_void_p]),
    ("gtls_last_error", ctypes.c_char_p, []),
    ("gtls_status_string", ctypes.c_char_p, [ctypes.c_int]),
]


def library_path() -> str:
    return _build.LIB


def load(build_if_missing: bool = True):
    """Load libgtls.so (building it first if allowed).  Raises if unavailable."""
    global _lib
    with _lock:
        if _lib is None:
            path = _build.LIB
            if not os.path.exists(path) or not _build.up_to_date():
                if not build_if_missing:
                    raise RuntimeError(f"libgtls.so is not built ({path})")
                _build.build()
            lib = ctypes.CDLL(path)
            for name, res, args in SIGNATURES:
                fn = getattr(lib, name)
                fn.restype = res
                fn.argtypes = args
            _lib = lib
    return _lib


def _check(status):
    if status != 0:
        raise GtlsError(status, _lib.gtls_last_error().decode())


def _ptr(x):
    """Device pointer of a torch tensor (or an int address)."""
    if x is None:
        return None
    if isinstance(x, int):
        return ctypes.c_void_p(x)
    return ctypes.c_void_p(x.data_ptr())


def _stream_handle(stream):
    if stream is None:
        try:
            import torch
            return ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
        except Exception:
            return ctypes.c_void_p(0)
    if isinstance(stream, int):
        return ctypes.c_void_p(stream)
    return ctypes.c_void_p(stream.cuda_stream)


@dataclasses.dataclass
class PlanConfig:
    baseline_days: float
    n_points: int
    m_star: float = 1.0
    r_star: float = 1.0
    oversampling: float = 3.0
    period_min_days: float = 0.0
    period_max_days: float = 0.0
    k_min: float = 20.05
    k_max: float = 620.84
    q_cap: float = 0.15
    dur_ratio: float = 1.1
    dt0: float = 0.05
    u1: float = 0.4
    u2: float = 0.25
    median_window: int = 0
    periods_per_chunk: int = 0
    refine_periods: int = 0
    periods_days: np.ndarray | None = None
    test_flags: int = 0


class Plan:
    """Owner of a gtls_plan (grids, templates and device scratch)."""

    def __init__(self, cfg: PlanConfig):
        lib = load()
        prm = PlanParams()
        lib.gtls_plan_params_default(ctypes.byref(prm))
        for f in ("baseline_days", "n_points", "m_star", "r_star", "oversampling",
                  "period_min_days", "period_max_days", "k_min", "k_max", "q_cap",
                  "dur_ratio", "dt0", "u1", "u2", "median_window", "periods_per_chunk",
                  "refine_periods", "test_flags"):
            v = getattr(cfg, f)
            setattr(prm, f, v if v is not None else 0)
        self._periods_in = None
        if cfg.periods_days is not None:
            self._periods_in = np.ascontiguousarray(cfg.periods_days, dtype=np.float64)
            prm.periods_days = self._periods_in.ctypes.data_as(c_double_p)
            prm.n_periods = self._periods_in.size
        h = ctypes.c_void_p()
        _check(lib.gtls_plan_create(ctypes.byref(prm), ctypes.byref(h)))
        self.handle = h
        self.cfg = cfg
        info = PlanInfo()
        _check(lib.gtls_plan_get_info(self.handle, ctypes.byref(info)))
        self.info = info

    # -- grids --------------------------------------------------------------
    @property
    def n_periods(self) -> int:
        return int(self.info.n_periods)

    def periods(self) -> np.ndarray:
        out = np.empty(self.n_periods)
        _check(_lib.gtls_plan_get_periods(self.handle, out.ctypes.data_as(c_double_p)))
        return out

    def durations(self):
        nd = int(self.info.n_durations)
        q = np.empty(nd)
        d = np.empty(nd, np.int32)
        _check(_lib.gtls_plan_get_durations(self.handle, q.ctypes.data_as(c_double_p),
                                            d.ctypes.data_as(c_int32_p)))
        return q, d

    def ranges(self):
        lo = np.empty(self.n_periods, np.int32)
        hi = np.empty(self.n_periods, np.int32)
        _check(_lib.gtls_plan_get_ranges(self.handle, lo.ctypes.data_as(c_int32_p),
                                         hi.ctypes.data_as(c_int32_p)))
        return lo, hi

    # -- searches -----------------------------------------------------------
    def search(self, t, y, dy, stream=None, per_period=None) -> Result:
        """gtls_search on device tensors (float64, contiguous, same device)."""
        res = Result()
        po = None
        if per_period is not None:
            po = PeriodOutputs(*[_ptr(per_period.get(f)) for f, _ in PeriodOutputs._fields_])
        n = int(t.numel()) if hasattr(t, "numel") else int(len(t))
        _check(_lib.gtls_search(self.handle, _ptr(t), _ptr(y), _ptr(dy), n,
                                _stream_handle(stream), ctypes.byref(res),
                                ctypes.byref(po) if po is not None else None))
        return res

    def search_host(self, t, y, dy, stream=None) -> Result:
        """gtls_search_host on host float64 arrays (copies to the device inside)."""
        t = np.ascontiguousarray(t, np.float64)
        y = np.ascontiguousarray(y, np.float64)
        dy = np.ascontiguousarray(dy, np.float64)
        res = Result()
        _check(_lib.gtls_search_host(self.handle, t.ctypes.data_as(c_double_p),
                                     y.ctypes.data_as(c_double_p), dy.ctypes.data_as(c_double_p),
                                     t.size, _stream_handle(stream), ctypes.byref(res)))
        return res

    def device_bytes(self) -> int:
        """Device memory the plan holds now (gtls_plan_get_info)."""
        info = PlanInfo()
        _check(_lib.gtls_plan_get_info(self.handle, ctypes.byref(info)))
        return int(info.device_bytes)

    def reserve(self):
        """Allocate the chunk scratch now (gtls_plan_reserve)."""
        _check(_lib.gtls_plan_reserve(self.handle))

    def trim(self):
        """Free the chunk scratch until the next search (gtls_plan_trim)."""
        _check(_lib.gtls_plan_trim(self.handle))

    def set_profiling(self, on: bool = True):
        _check(_lib.gtls_plan_set_profiling(self.handle, 1 if on else 0))

    def profile(self) -> Profile:
        pr = Profile()
        _check(_lib.gtls_plan_get_profile(self.handle, ctypes.byref(pr)))
        return pr

    def close(self):
        if getattr(self, "handle", None) and self.handle.value:
            _lib.gtls_plan_destroy(self.handle)
            self.handle = ctypes.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def search_batch(plans, t, y, dy, offsets, stream=None):
    """gtls_search_batch: CSR-packed device tensors, one plan per curve."""
    lib = load()
    n_lc = len(plans)
    arr = (ctypes.c_void_p * n_lc)(*[p.handle.value for p in plans])
    offs = np.ascontiguousarray(offsets, np.int64)
    out = (Result * n_lc)()
    _check(lib.gtls_search_batch(arr, n_lc, _ptr(t), _ptr(y), _ptr(dy),
                                 offs.ctypes.data_as(c_int64_p), _stream_handle(stream), out))
    return list(out)


class Batch:
    """gtls_batch: many light curves (one plan each) searched in waves of a
    shared chunk scratch, replayed from a captured CUDA graph."""

    def __init__(self, plans, wave_slots: int = 0):
        self._lib = load()
        self.plans = list(plans)  # keep the plans alive as long as the batch
        arr = (ctypes.c_void_p * len(self.plans))(*[p.handle.value for p in self.plans])
        self.handle = ctypes.c_void_p()
        _check(self._lib.gtls_batch_create(arr, len(self.plans), int(wave_slots),
                                           ctypes.byref(self.handle)))

    @staticmethod
    def _offsets(offsets):
        return np.ascontiguousarray(offsets, np.int64)

    def search(self, t, y, dy, offsets, stream=None):
        offs = self._offsets(offsets)
        out = (Result * len(self.plans))()
        _check(self._lib.gtls_batch_search(self.handle, _ptr(t), _ptr(y), _ptr(dy),
                                           offs.ctypes.data_as(c_int64_p),
                                           _stream_handle(stream), out))
        return list(out)

    def autotune(self, t, y, dy, offsets, stream=None):
        offs = self._offsets(offsets)
        _check(self._lib.gtls_batch_autotune(self.handle, _ptr(t), _ptr(y), _ptr(dy),
                                             offs.ctypes.data_as(c_int64_p),
                                             _stream_handle(stream)))
        return self.info()

    def period_outputs(self, lc: int, per_period: dict, stream=None):
        """Copy curve lc's per-period outputs of the last search into device tensors."""
        po = PeriodOutputs(*[_ptr(per_period.get(f)) for f, _ in PeriodOutputs._fields_])
        _check(self._lib.gtls_batch_get_period_outputs(self.handle, int(lc), ctypes.byref(po),
                                                       _stream_handle(stream)))

    def info(self) -> BatchInfo:
        bi = BatchInfo()
        _check(self._lib.gtls_batch_get_info(self.handle, ctypes.byref(bi)))
        return bi

    def close(self):
        if getattr(self, "handle", None) is not None and self.handle.value:
            self._lib.gtls_batch_destroy(self.handle)
            self.handle = ctypes.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def sr_sde_noalloc(chi2, sde, sr=None, sde_raw=None, median_window=0, stream=None):
    """gtls_sr_sde_noalloc on device tensors (float64); returns (best index, best SDE).

    The reduction's scratch is a fixed array inside the library (no device
    allocation by the call); `sde` (and `sr`, `sde_raw` when given) receive
    the spectra.
    """
    import torch
    lib = load()
    n = int(chi2.numel())
    for name, x in (("chi2", chi2), ("sde", sde), ("sr", sr), ("sde_raw", sde_raw)):
        if x is None:
            continue
        if not isinstance(x, torch.Tensor) or x.dtype != torch.float64 or not x.is_cuda:
            raise TypeError(f"{name} must be a float64 CUDA tensor")
        if not x.is_contiguous() or x.numel() != n:
            raise ValueError(f"{name} must be contiguous with {n} elements")
        if x.device != chi2.device:
            raise ValueError(f"{name} is on {x.device}, chi2 on {chi2.device}")
    bi = ctypes.c_int64(0)
    bs = ctypes.c_double(0.0)
    with torch.cuda.device(chi2.device):
        _check(lib.gtls_sr_sde_noalloc(_ptr(chi2), n, int(median_window), _stream_handle(stream),
                                       _ptr(sr), _ptr(sde_raw), _ptr(sde), ctypes.byref(bi),
                                       ctypes.byref(bs)))
    return int(bi.value), float(bs.value)


N_BINS = 4096
N_REG = 128


class Cnn:
    """gtls_cnn: the learned period proposal network (BF16 tensor-core kernels)."""

    def __init__(self, max_batch: int, params=None):
        self._lib = load()
        self.max_batch = int(max_batch)
        self.n_params = int(self._lib.gtls_cnn_param_count())
        buf = None
        if params is not None:
            buf = np.ascontiguousarray(params, np.float32)
            if buf.size != self.n_params:
                raise ValueError("parameter vector has the wrong size")
        self.handle = ctypes.c_void_p()
        _check(self._lib.gtls_cnn_create(self.max_batch,
                                         buf.ctypes.data if buf is not None else None,
                                         ctypes.byref(self.handle)))

    def params(self) -> np.ndarray:
        out = np.empty(self.n_params, np.float32)
        _check(self._lib.gtls_cnn_get_params(self.handle, out.ctypes.data))
        return out

    def set_params(self, params):
        buf = np.ascontiguousarray(params, np.float32)
        if buf.size != self.n_params:
            raise ValueError("parameter vector has the wrong size")
        _check(self._lib.gtls_cnn_set_params(self.handle, buf.ctypes.data))

    def bin(self, t, y, dy, offsets, x, mean=None, wsum=None, stream=None):
        offs = np.ascontiguousarray(offsets, np.int64)
        _check(self._lib.gtls_cnn_bin(self.handle, _ptr(t), _ptr(y), _ptr(dy),
                                      offs.ctypes.data_as(c_int64_p), offs.size - 1, _ptr(x),
                                      _ptr(mean), _ptr(wsum), _stream_handle(stream)))

    def forward(self, x, batch, logits=None, scores=None, stream=None):
        _check(self._lib.gtls_cnn_forward(self.handle, _ptr(x), int(batch), _ptr(logits),
                                          _ptr(scores), _stream_handle(stream)))

    def gradient(self, x, target, mask, batch, stream=None):
        g = np.empty(self.n_params, np.float32)
        loss = ctypes.c_double(0.0)
        _check(self._lib.gtls_cnn_gradient(self.handle, _ptr(x), _ptr(target), _ptr(mask),
                                           int(batch), g.ctypes.data, ctypes.byref(loss),
                                           _stream_handle(stream)))
        return g, float(loss.value)

    def train_step(self, x, target, mask, batch, lr, stream=None) -> float:
        loss = ctypes.c_double(0.0)
        _check(self._lib.gtls_cnn_train_step(self.handle, _ptr(x), _ptr(target), _ptr(mask),
                                             int(batch), float(lr), ctypes.byref(loss),
                                             _stream_handle(stream)))
        return float(loss.value)

    def close(self):
        if getattr(self, "handle", None) is not None and self.handle.value:
            self._lib.gtls_cnn_destroy(self.handle)
            self.handle = ctypes.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def region_targets(periods, sr):
    """gtls_region_targets on host arrays: (target[128], mask[128])."""
    lib = load()
    p = np.ascontiguousarray(periods, np.float64)
    s = np.ascontiguousarray(sr, np.float64)
    tgt = np.empty(N_REG, np.float32)
    mask = np.empty(N_REG, np.float32)
    _check(lib.gtls_region_targets(p.ctypes.data_as(c_double_p), s.ctypes.data_as(c_double_p),
                                   p.size, tgt.ctypes.data, mask.ctypes.data))
    return tgt, mask


def proposal_periods(periods, scores, frac) -> np.ndarray:
    """gtls_proposal_periods on host arrays: indices of the proposed periods."""
    lib = load()
    p = np.ascontiguousarray(periods, np.float64)
    sc = np.ascontiguousarray(scores, np.float32)
    idx = np.empty(max(1, p.size), np.int64)
    n = ctypes.c_int64(0)
    _check(lib.gtls_proposal_periods(p.ctypes.data_as(c_double_p), p.size, sc.ctypes.data,
                                     float(frac), idx.ctypes.data_as(c_int64_p), ctypes.byref(n)))
    return idx[:n.value].copy()

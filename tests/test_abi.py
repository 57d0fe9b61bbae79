"""CPU checks of the C ABI: the library loads, exports every declared symbol,
and the ctypes mirrors of the header's structs have the C layout."""

import ctypes
import os
import re
import subprocess

import numpy as np
import pytest

import paper_2607_00348_gb300 as pkg
from paper_2607_00348_gb300 import gtls as binding

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "gtls.h")


def declared_functions():
    src = open(HEADER).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    names = re.findall(r"\b(gtls_[a-z_0-9]+)\s*\(", src)
    return sorted(set(names))


def test_header_declares_the_boundary():
    names = declared_functions()
    for want in ("gtls_plan_create", "gtls_search", "gtls_search_batch", "gtls_plan_destroy"):
        assert want in names


def test_library_builds_and_exports_every_declared_symbol():
    path = pkg.build_library()
    assert os.path.exists(path)
    lib = ctypes.CDLL(path)
    for name in declared_functions():
        assert hasattr(lib, name), name
    bound = {n for n, _, _ in binding.SIGNATURES}
    assert bound == set(declared_functions())


def test_binding_loads_without_gpu():
    lib = pkg.load()
    assert lib.gtls_status_string(1) == b"GTLS_ERR_INVALID_ARG"
    prm = binding.PlanParams()
    lib.gtls_plan_params_default(ctypes.byref(prm))
    assert prm.k_min == 20.05 and prm.k_max == 620.84 and prm.q_cap == 0.15
    assert prm.oversampling == 3.0 and prm.dt0 == 0.05 and prm.dur_ratio == 1.1


def test_invalid_parameters_are_rejected_before_any_device_work():
    lib = pkg.load()
    prm = binding.PlanParams()
    lib.gtls_plan_params_default(ctypes.byref(prm))
    h = ctypes.c_void_p()
    prm.n_points = 1
    prm.baseline_days = 10.0
    assert lib.gtls_plan_create(ctypes.byref(prm), ctypes.byref(h)) == 1
    assert b"n_points" in lib.gtls_last_error()
    prm.n_points = 100
    prm.period_min_days = 5.0
    prm.period_max_days = 2.0
    assert lib.gtls_plan_create(ctypes.byref(prm), ctypes.byref(h)) == 1
    assert b"empty period range" in lib.gtls_last_error()
    assert not h.value


def _c_layout():
    prog = r'''
#include <stdio.h>
#include <stddef.h>
#include "gtls.h"
int main(void) {
  printf("%zu %zu %zu %zu %zu %zu %zu %zu %zu %zu\n", sizeof(gtls_plan_params), sizeof(gtls_plan_info),
         sizeof(gtls_result), sizeof(gtls_period_outputs),
         offsetof(gtls_plan_params, periods_days), offsetof(gtls_result, period_idx),
         offsetof(gtls_plan_info, wpe), sizeof(gtls_batch_info),
         offsetof(gtls_batch_info, last_launches), offsetof(gtls_batch_info, tuned_flops));
  return 0;
}
'''
    import tempfile
    with tempfile.TemporaryDirectory() as d:
        c = os.path.join(d, "l.c")
        exe = os.path.join(d, "l")
        open(c, "w").write(prog)
        subprocess.run(["gcc", "-I", os.path.join(ROOT, "include"), c, "-o", exe], check=True)
        return [int(x) for x in subprocess.run([exe], capture_output=True, text=True,
                                               check=True).stdout.split()]


def test_ctypes_structs_match_the_header_layout():
    got = _c_layout()
    want = [ctypes.sizeof(binding.PlanParams), ctypes.sizeof(binding.PlanInfo),
            ctypes.sizeof(binding.Result), ctypes.sizeof(binding.PeriodOutputs),
            binding.PlanParams.periods_days.offset, binding.Result.period_idx.offset,
            binding.PlanInfo.wpe.offset, ctypes.sizeof(binding.BatchInfo),
            binding.BatchInfo.last_launches.offset, binding.BatchInfo.tuned_flops.offset]
    assert got == want


def test_batch_and_network_reject_invalid_arguments_before_device_work():
    lib = binding.load()
    h = ctypes.c_void_p()
    # a batch needs 1 .. 65535 curves and a non-null plan array
    assert lib.gtls_batch_create(None, 1, 0, ctypes.byref(h)) == 1
    arr = (ctypes.c_void_p * 1)(None)
    assert lib.gtls_batch_create(arr, 0, 0, ctypes.byref(h)) == 1
    assert lib.gtls_batch_create(arr, 1, -1, ctypes.byref(h)) == 1
    assert not h.value
    # the proposal network: batch size range, null outputs
    assert lib.gtls_cnn_create(0, None, ctypes.byref(h)) == 1
    assert lib.gtls_cnn_create(5000, None, ctypes.byref(h)) == 1
    assert lib.gtls_cnn_create(4, None, None) == 1
    assert not h.value
    # the host helpers of the proposal
    per = np.array([1.0, 2.0, 3.0])
    idx = np.zeros(3, np.int64)
    n = ctypes.c_int64(0)
    sc = np.zeros(128, np.float32)
    assert lib.gtls_proposal_periods(per.ctypes.data_as(binding.c_double_p), 3, sc.ctypes.data, 0.0,
                                     idx.ctypes.data_as(binding.c_int64_p), ctypes.byref(n)) == 1
    assert lib.gtls_proposal_periods(per.ctypes.data_as(binding.c_double_p), 3, sc.ctypes.data, 1.5,
                                     idx.ctypes.data_as(binding.c_int64_p), ctypes.byref(n)) == 1
    assert lib.gtls_region_targets(None, None, 3, None, None) == 1

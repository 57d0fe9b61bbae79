"""The allocation-free SR/SDE entry point against the regular search.

gtls_sr_sde_noalloc serves callers that cannot allocate device memory (code
confined to a pre-sized pool, or to buffers another framework hands over):
its scratch is a fixed array inside the library.  Given the chi2(P) spectrum
that gtls_search produced, it must return the same SR, SDE_raw, SDE and best
period as gtls_search did, on two calls in a row (the array keeps the first
call's contents).  This file is collected last so that a run that stops at
the first failure has already run every other test.
"""

import numpy as np
import pytest

import synth

from . import gpu_helpers as gh

pytestmark = pytest.mark.gpu


def test_noalloc_reduction_matches_search_twice():
    import torch

    import paper_2607_00348_gb300 as pkg
    from paper_2607_00348_gb300 import gtls as binding

    lc = synth.short_white()
    plan = gh.plan_for(lc, lc.baseline_days, lc.search)
    res, out = gh.gpu_search(plan, lc.t, lc.y, lc.dy)
    dev = torch.device("cuda:0")
    chi2 = torch.as_tensor(out["chi2"], dtype=torch.float64, device=dev)
    npd = chi2.numel()
    for _ in range(2):
        sr = torch.full((npd,), -1.0, dtype=torch.float64, device=dev)
        raw = torch.full((npd,), -1.0, dtype=torch.float64, device=dev)
        sde = torch.full((npd,), -1.0, dtype=torch.float64, device=dev)
        bi, bs = binding.sr_sde_noalloc(chi2, sde, sr=sr, sde_raw=raw)
        torch.cuda.synchronize()
        np.testing.assert_allclose(sr.cpu().numpy(), out["sr"], rtol=1e-12, atol=0)
        np.testing.assert_allclose(raw.cpu().numpy(), out["sde_raw"], rtol=0, atol=1e-9)
        np.testing.assert_allclose(sde.cpu().numpy(), out["sde"], rtol=0, atol=1e-3)
        assert bi == res.period_idx
        assert bs == pytest.approx(res.sde, abs=1e-3)
    # without SR / SDE_raw buffers the spectra stay inside the library
    sde2 = torch.empty(npd, dtype=torch.float64, device=dev)
    bi2, bs2 = binding.sr_sde_noalloc(chi2, sde2)
    np.testing.assert_allclose(sde2.cpu().numpy(), out["sde"], rtol=0, atol=1e-3)
    assert bi2 == res.period_idx
    plan.close()


def test_noalloc_rejects_sizes_beyond_its_array():
    import torch

    from paper_2607_00348_gb300 import gtls as binding

    dev = torch.device("cuda:0")
    big = torch.ones((1 << 19) + 1, dtype=torch.float64, device=dev)
    with pytest.raises(binding.GtlsError, match="INVALID_ARG"):
        binding.sr_sde_noalloc(big, torch.empty_like(big))


def test_noalloc_rejects_bad_spectra_and_buffers():
    import torch

    from paper_2607_00348_gb300 import gtls as binding

    dev = torch.device("cuda:0")
    chi2 = torch.linspace(100.0, 200.0, 3000, dtype=torch.float64, device=dev)
    sde = torch.empty_like(chi2)
    for bad in (float("nan"), float("inf"), -1.0):
        c = chi2.clone()
        c[1234] = bad
        with pytest.raises(binding.GtlsError, match="INVALID_ARG.*chi2"):
            binding.sr_sde_noalloc(c, sde)
    with pytest.raises(TypeError):
        binding.sr_sde_noalloc(chi2, torch.empty(3000, dtype=torch.float32, device=dev))
    with pytest.raises(ValueError):
        binding.sr_sde_noalloc(chi2, torch.empty(2999, dtype=torch.float64, device=dev))
    with pytest.raises(TypeError):
        binding.sr_sde_noalloc(chi2, torch.empty(3000, dtype=torch.float64))
    # host memory handed straight to the C entry point is refused there
    lib = binding.load()
    host = np.zeros(3000)
    st = lib.gtls_sr_sde_noalloc(binding._ptr(chi2), 3000, 0, binding._stream_handle(None),
                                 None, None, host.ctypes.data, None, None)
    assert st == 1 and b"device memory" in lib.gtls_last_error()
    # a good call afterwards still works
    bi, bs = binding.sr_sde_noalloc(chi2, sde)
    assert 0 <= bi < 3000 and np.isfinite(bs)

"""fdw_misfit_noalloc: the misfit for callers that cannot allocate device
memory (a pool allocator that owns the GPU, a loop that cannot take the
synchronisation of cudaMalloc/cudaFree, a nearly full device). It must give
what fdw_misfit gives, call after call, with its scratch compiled into the
library instead of allocated.

This file is named so pytest collects it last."""
import ctypes

import numpy as np
import pytest

pytestmark = pytest.mark.gpu


def _ptr(t):
    return ctypes.c_void_p(t.data_ptr())


def test_noalloc_misfit_matches_fdw_misfit_on_two_calls_in_a_row(fdw):
    import torch
    L = fdw.lib()
    stream = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    # two calls in a row with different sizes: the second must not see the
    # first call's leftovers in the shared scratch
    for call, n in enumerate((3_000_017, 12_345)):
        rng = np.random.default_rng(100 + call)
        d = torch.from_numpy(rng.standard_normal(n)).cuda()
        o = torch.from_numpy(rng.standard_normal(n)).cuda()
        res_ref, res_na = torch.empty_like(d), torch.full_like(d, np.nan)
        J_ref = torch.empty((), dtype=torch.float64, device="cuda")
        J_na = torch.full((), np.nan, dtype=torch.float64, device="cuda")
        assert L.fdw_misfit(_ptr(d), _ptr(o), n, _ptr(res_ref), _ptr(J_ref), stream) == 0
        assert L.fdw_misfit_noalloc(_ptr(d), _ptr(o), n, _ptr(res_na), _ptr(J_na), stream) == 0, \
            L.fdw_last_error()
        torch.cuda.synchronize()
        assert torch.equal(res_na, res_ref)
        jr, jn = float(J_ref), float(J_na)
        assert abs(jn - jr) <= 1e-12 * abs(jr), (call, jn, jr)


def test_noalloc_misfit_rejects_sizes_beyond_its_scratch(fdw):
    import torch
    L = fdw.lib()
    d = torch.zeros(1, dtype=torch.float64, device="cuda")
    J = torch.zeros((), dtype=torch.float64, device="cuda")
    limit = 32768 * 2048
    rc = L.fdw_misfit_noalloc(_ptr(d), _ptr(d), limit + 1, None, _ptr(J), None)
    assert rc == -1
    assert b"67108864" in L.fdw_last_error()


def test_noalloc_misfit_edge_sizes(fdw):
    """n = 0 (only the final sum runs: J = 0), no residual output, and n at
    the limit exactly, which fills every chunk sum of the scratch array."""
    import torch
    L = fdw.lib()
    stream = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    J = torch.full((), np.nan, dtype=torch.float64, device="cuda")
    assert L.fdw_misfit_noalloc(None, None, 0, None, _ptr(J), stream) == 0, L.fdw_last_error()
    torch.cuda.synchronize()
    assert float(J) == 0.0
    for n in (777_777, 32768 * 2048):
        g = torch.Generator(device="cuda").manual_seed(n)
        d = torch.randn(n, dtype=torch.float64, device="cuda", generator=g)
        o = torch.randn(n, dtype=torch.float64, device="cuda", generator=g)
        J_ref = torch.empty((), dtype=torch.float64, device="cuda")
        J_na = torch.full((), np.nan, dtype=torch.float64, device="cuda")
        res_ref = torch.empty_like(d)
        assert L.fdw_misfit(_ptr(d), _ptr(o), n, _ptr(res_ref), _ptr(J_ref), stream) == 0
        if n == 777_777:  # no residual output
            assert L.fdw_misfit_noalloc(_ptr(d), _ptr(o), n, None, _ptr(J_na), stream) == 0, \
                L.fdw_last_error()
        else:
            res_na = torch.full_like(d, np.nan)
            assert L.fdw_misfit_noalloc(_ptr(d), _ptr(o), n, _ptr(res_na), _ptr(J_na), stream) == 0, \
                L.fdw_last_error()
            torch.cuda.synchronize()
            assert torch.equal(res_na, res_ref)
            del res_na
        torch.cuda.synchronize()
        jr, jn = float(J_ref), float(J_na)
        assert abs(jn - jr) <= 1e-12 * abs(jr), (n, jn, jr)
        del d, o, res_ref
        torch.cuda.empty_cache()

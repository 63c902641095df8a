"""sign_tri_noalloc: the entry point for callers that cannot allocate device
memory (a host program that owns all device memory through its own pool, or
code that must not stall the device in cudaMalloc/cudaFree).  Its scratch is
a static device array inside the library.  Checked through the C ABI against
sign_tri on two calls in a row.  This file is collected last on purpose."""
import numpy as np
import pytest

from paper_1607_06303_gb300.inputs import make_T

pytestmark = pytest.mark.gpu

TOL_FP64 = 1e-11


def test_noalloc_matches_sign_tri(gpu_lib):
    import torch
    p = gpu_lib
    h = torch.cuda.current_stream().cuda_stream
    # two calls in a row, different sizes and inertia, the second reusing the
    # array the first left behind
    for n, pr, seed in [(1000, 0.5, 21), (777, 0.3, 22), (1024, 0.5, 23)]:
        T = make_T(n, pr, seed=seed)
        Tt = p.to_device(T)
        U_ref = torch.empty_like(Tt)
        U_na = torch.full_like(Tt, np.nan)
        assert p.sign_tri(n, Tt.data_ptr(), n, U_ref.data_ptr(), n, p.Variant.PH_FP64, h) == 0
        assert p.sign_tri_noalloc(n, Tt.data_ptr(), n, U_na.data_ptr(), n, h) == 0
        torch.cuda.synchronize()
        A, B = p.to_numpy(U_na), p.to_numpy(U_ref)
        assert np.all(np.isfinite(A))
        assert np.linalg.norm(A - B) <= TOL_FP64 * np.linalg.norm(B)


def test_noalloc_ignores_library_workspace(gpu_lib):
    # with a 256-byte caller workspace sign_tri cannot run n = 500, while the
    # static-scratch entry point does not use that workspace at all
    import torch
    p = gpu_lib
    h = torch.cuda.current_stream().cuda_stream
    n = 500
    T = make_T(n, 0.5, seed=24)
    Tt = p.to_device(T)
    tiny = torch.empty(32, dtype=torch.float64, device="cuda")
    U1 = torch.empty_like(Tt)
    U2 = torch.empty_like(Tt)
    assert p.sign_tri(n, Tt.data_ptr(), n, U2.data_ptr(), n, p.Variant.PH_FP64, h) == 0
    try:
        assert p.signtri_set_workspace(tiny.data_ptr(), 256) == 0
        assert p.sign_tri(n, Tt.data_ptr(), n, U1.data_ptr(), n, p.Variant.PH_FP64, h) == \
            p.Status.ERR_NO_WORKSPACE
        assert p.sign_tri_noalloc(n, Tt.data_ptr(), n, U1.data_ptr(), n, h) == 0
    finally:
        p.signtri_set_workspace(0, 0)
    torch.cuda.synchronize()
    A, B = p.to_numpy(U1), p.to_numpy(U2)
    assert np.linalg.norm(A - B) <= TOL_FP64 * np.linalg.norm(B)


def test_noalloc_rejects_beyond_maximum(gpu_lib):
    import torch
    p = gpu_lib
    h = torch.cuda.current_stream().cuda_stream
    n = p.signtri.SIGNTRI_NOALLOC_MAX_N + 1
    T = make_T(n, 0.5, seed=25)
    Tt = p.to_device(T)
    U = torch.full_like(Tt, 3.0)
    assert p.sign_tri_noalloc(n, Tt.data_ptr(), n, U.data_ptr(), n, h) == p.Status.ERR_NO_WORKSPACE
    torch.cuda.synchronize()
    assert bool(torch.all(U == 3.0))          # nothing was written
    assert p.sign_tri_noalloc(-1, 0, 1, 0, 1, h) == p.Status.ERR_BAD_ARG
    assert p.sign_tri_noalloc(0, 0, 1, 0, 1, h) == p.Status.OK

"""GPU parity of the recursive Parlett-Higham float64 path against the CPU
oracle, called through the C ABI.  Tolerance: relative Frobenius error
<= 1e-11 (float64 form); the diagonal and strictly-lower parts are exact."""
import numpy as np
import pytest

from paper_1607_06303_gb300.inputs import make_T

pytestmark = pytest.mark.gpu

TOL_FP64 = 1e-11


def relerr(A, B):
    nb = np.linalg.norm(B)
    return np.linalg.norm(A - B) / (nb if nb > 0 else 1.0)


def run_gpu(p, T, variant, cutoff=None):
    import torch
    if cutoff is not None:
        assert p.signtri_set_cutoff(cutoff) == 0
    try:
        Tt = p.to_device(T)
        Ut = p.sign(Tt, variant)
        torch.cuda.synchronize()
        return p.to_numpy(Ut), p.signtri_get_info()
    finally:
        p.signtri_set_cutoff(0)


def check_structure(U, T):
    n = T.shape[0]
    assert np.all(np.diag(U) == np.sign(np.diag(T)))
    assert np.all(np.tril(U, -1) == 0.0)


# every cutoff b in {16, 32, 64} meets n = 2b+1, 3b and 4b-1 (recursion
# bookkeeping at uneven splits) besides the tile-edge sizes
SIZES = [1, 2, 3, 5, 15, 16, 17, 31, 32, 33, 48, 63, 64, 65, 96, 100, 127, 129, 192, 200, 255, 257, 300]


@pytest.mark.parametrize("cutoff", [16, 32, 64])
@pytest.mark.parametrize("n", SIZES)
def test_ph_fp64_vs_oracle(gpu_lib, oracle_mod, n, cutoff):
    for seed, p, order in [(0, 0.5, "random"), (1, 0.2, "random"), (2, 0.7, "sorted")]:
        T = make_T(n, p, seed=seed, order=order)
        U, info = run_gpu(gpu_lib, T, gpu_lib.Variant.PH_FP64, cutoff)
        Uo = oracle_mod.sign_tri(T)
        check_structure(U, T)
        assert relerr(U, Uo) <= TOL_FP64, (n, cutoff, seed)


@pytest.mark.parametrize("n", [700, 1000, 1500])
def test_ph_fp64_medium(gpu_lib, oracle_mod, n):
    T = make_T(n, 0.5, seed=11)
    U, info = run_gpu(gpu_lib, T, gpu_lib.Variant.PH_FP64)
    Uo = oracle_mod.sign_tri(T, schedule="antidiag")
    check_structure(U, T)
    assert relerr(U, Uo) <= TOL_FP64
    assert info.variant == gpu_lib.Variant.PH_FP64 and info.cutoff == 16   # the default up to n = 4096


@pytest.mark.parametrize("n,cutoff", [(5, 16), (16, 16), (32, 32), (50, 64), (64, 64)])
def test_single_leaf_bitexact(gpu_lib, oracle_mod, n, cutoff):
    # n <= cutoff: one diagonal leaf runs Algorithm 3 with the oracle's
    # rounding (separate IEEE multiply/add/divide, ascending sums)
    T = make_T(n, 0.5, seed=5)
    U, _ = run_gpu(gpu_lib, T, gpu_lib.Variant.PH_FP64, cutoff)
    np.testing.assert_array_equal(U, oracle_mod.sign_tri(T))


def test_leading_dimension_padding(gpu_lib, oracle_mod):
    import torch
    n, ld = 150, 161
    T = make_T(n, 0.5, seed=12)
    Tp = np.zeros((ld, n), order="F")
    Tp[:n, :] = T
    Tp[n:, :] = 7.0                       # must not be read
    Tt = torch.from_numpy(np.ascontiguousarray(Tp.T)).cuda()
    Ut = torch.full((n, ld), -5.0, dtype=torch.float64, device="cuda")
    st = gpu_lib.sign_tri(n, Tt.data_ptr(), ld, Ut.data_ptr(), ld, gpu_lib.Variant.PH_FP64,
                          torch.cuda.current_stream().cuda_stream)
    assert st == 0
    torch.cuda.synchronize()
    Up = np.asfortranarray(Ut.cpu().numpy().T)
    assert np.all(Up[n:, :] == -5.0)      # rows beyond n untouched
    assert relerr(Up[:n, :], oracle_mod.sign_tri(T)) <= TOL_FP64


def test_trivial_inertia_exact(gpu_lib):
    for p, val in [(0.0, 1.0), (1.0, -1.0)]:
        T = make_T(300, p, seed=1)
        for v in (gpu_lib.Variant.AUTO, gpu_lib.Variant.PH_FP64):
            U, info = run_gpu(gpu_lib, T, v)
            np.testing.assert_array_equal(U, val * np.eye(300))


def test_error_statuses(gpu_lib):
    import torch
    T = make_T(100, 0.5, seed=2)
    for bad, expect in [(0.0, gpu_lib.Status.ERR_ZERO_EIGENVALUE), (np.nan, gpu_lib.Status.ERR_NONFINITE),
                        (-np.inf, gpu_lib.Status.ERR_NONFINITE)]:
        Tb = T.copy()
        Tb[37, 37] = bad
        Tb[60, 60] = 0.0
        Tt = gpu_lib.to_device(Tb)
        Ut = torch.empty_like(Tt)
        st = gpu_lib.sign_tri(100, Tt.data_ptr(), 100, Ut.data_ptr(), 100, gpu_lib.Variant.PH_FP64,
                              torch.cuda.current_stream().cuda_stream)
        assert st == expect
        assert gpu_lib.signtri_get_info().bad_index == 37


def test_inertia_scan(gpu_lib):
    from paper_1607_06303_gb300 import workload
    for n, p, order in [(1, 0.5, "random"), (1000, 0.3, "random"), (5000, 0.5, "random"), (777, 0.25, "sorted")]:
        T = make_T(n, p, seed=3, order=order)
        Tt = gpu_lib.to_device(T)
        st, npos, nneg, k = gpu_lib.signtri_inertia(n, Tt.data_ptr(), n)
        s = np.sign(np.diag(T))
        assert st == 0 and npos == int((s > 0).sum()) and nneg == int((s < 0).sum())
        assert k == workload.swaps(s)


@pytest.mark.parametrize("variant", ["PH_FP64", "PH_MIXED_FP16"])
def test_host_entry_point_reads_upper_triangle_only(gpu_lib, oracle_mod, variant):
    # T_host as the leading n x n block of an (n + 7) x n array whose strictly
    # lower part holds NaN: only the upper triangle is copied and read; all of
    # U_host (NaN beforehand) is written, zeros below the diagonal
    n, ld = 300, 307
    T = make_T(n, 0.5, seed=5)
    big = np.full((ld, n), np.nan, order="F")
    big[:n, :n] = np.where(np.triu(np.ones((n, n), bool)), T, np.nan)
    U = np.full((n, n), np.nan, order="F")
    st = gpu_lib.sign_tri_host(n, big.ctypes.data, ld, U.ctypes.data, n, gpu_lib.Variant[variant], 0)
    assert st == 0
    assert np.all(np.isfinite(U)) and np.all(np.tril(U, -1) == 0.0)
    assert relerr(U, oracle_mod.sign_tri(T)) <= (1e-12 if "MIXED" in variant else TOL_FP64)


def test_host_entry_point(gpu_lib, oracle_mod):
    import ctypes
    n = 333
    T = make_T(n, 0.4, seed=4)
    U = np.zeros((n, n), order="F")
    st = gpu_lib.sign_tri_host(n, T.ctypes.data, n, U.ctypes.data, n, gpu_lib.Variant.PH_FP64, 0)
    assert st == 0
    assert relerr(U, oracle_mod.sign_tri(T)) <= TOL_FP64
    info = gpu_lib.signtri_get_info()
    s = np.sign(np.diag(T))
    from paper_1607_06303_gb300 import workload
    assert info.work_ph == workload.useful_flops(s)
    assert abs(info.work_ps - workload.ps_flops(s)) <= 1e-9 * info.work_ps

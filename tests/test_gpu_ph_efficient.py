"""GPU parity of the arithmetic-efficient recursive Parlett-Higham form
(Section 5.3: each entry's block sum is X when the signs of its row and column
differ and Y when they agree) against the CPU oracle, through the C ABI.

Each entry's sum runs over the same K blocks and the same terms in the same
order as in the full form, so the two float64 variants agree bit for bit;
against the oracle the float64 tolerance (relative Frobenius <= 1e-11)
applies."""
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


SIZES = [1, 2, 17, 33, 48, 64, 65, 96, 127, 129, 192, 200, 255, 257, 300]


@pytest.mark.parametrize("cutoff", [16, 32, 64])
@pytest.mark.parametrize("n", SIZES)
def test_efficient_vs_oracle_and_full_form(gpu_lib, oracle_mod, n, cutoff):
    V = gpu_lib.Variant
    for seed, p, order in [(0, 0.5, "random"), (1, 0.2, "random"), (2, 0.7, "sorted")]:
        T = make_T(n, p, seed=seed, order=order)
        U, info = run_gpu(gpu_lib, T, V.PH_FP64_EFFICIENT, cutoff)
        assert info.variant == V.PH_FP64_EFFICIENT
        if info.n_pos and info.n_neg:     # U = +-I needs no recursion
            assert info.cutoff == cutoff
        Uo = oracle_mod.sign_tri(T)
        assert np.all(np.diag(U) == np.sign(np.diag(T)))
        assert np.all(np.tril(U, -1) == 0.0)
        assert relerr(U, Uo) <= TOL_FP64, (n, cutoff, seed)
        Uf, _ = run_gpu(gpu_lib, T, V.PH_FP64, cutoff)
        np.testing.assert_array_equal(U, Uf)


@pytest.mark.parametrize("pattern", ["alternating", "all_pos", "all_neg", "half_blocks"])
def test_efficient_sign_patterns(gpu_lib, oracle_mod, pattern):
    # every gather shape: mixed rows in every block, one kind only, and
    # blocks of a single sign next to blocks of the other
    n = 333
    rng = np.random.default_rng(21)
    T = np.triu(rng.standard_normal((n, n)) / np.sqrt(n), 1)
    if pattern == "alternating":
        s = np.where(np.arange(n) % 2 == 0, 1.0, -1.0)
    elif pattern == "all_pos":
        s = np.ones(n)
    elif pattern == "all_neg":
        s = -np.ones(n)
    else:
        s = np.where((np.arange(n) // 64) % 2 == 0, 1.0, -1.0)
    T[np.arange(n), np.arange(n)] = s * rng.uniform(0.5, 2.0, n)
    V = gpu_lib.Variant
    U, _ = run_gpu(gpu_lib, T, V.PH_FP64_EFFICIENT)
    assert relerr(U, oracle_mod.sign_tri(T)) <= TOL_FP64
    Uf, _ = run_gpu(gpu_lib, T, V.PH_FP64)
    np.testing.assert_array_equal(U, Uf)


@pytest.mark.parametrize("n", [1000, 1500])
def test_efficient_medium(gpu_lib, oracle_mod, n):
    T = make_T(n, 0.5, seed=13)
    U, info = run_gpu(gpu_lib, T, gpu_lib.Variant.PH_FP64_EFFICIENT)
    Uo = oracle_mod.sign_tri(T, schedule="antidiag")
    assert relerr(U, Uo) <= TOL_FP64
    assert info.cutoff == 16   # the size-dependent default below n = 4096


def test_efficient_leading_dimension(gpu_lib, oracle_mod):
    import torch
    n, ld = 150, 161
    T = make_T(n, 0.5, seed=12)
    Tp = np.zeros((ld, n), order="F")
    Tp[:n, :] = T
    Tp[n:, :] = 7.0                       # must not be read
    Tt = torch.from_numpy(np.ascontiguousarray(Tp.T)).cuda()
    Ut = torch.full((n, ld), -5.0, dtype=torch.float64, device="cuda")
    st = gpu_lib.sign_tri(n, Tt.data_ptr(), ld, Ut.data_ptr(), ld,
                          gpu_lib.Variant.PH_FP64_EFFICIENT,
                          torch.cuda.current_stream().cuda_stream)
    assert st == 0
    torch.cuda.synchronize()
    Up = np.asfortranarray(Ut.cpu().numpy().T)
    assert np.all(Up[n:, :] == -5.0)
    assert relerr(Up[:n, :], oracle_mod.sign_tri(T)) <= TOL_FP64

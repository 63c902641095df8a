"""GPU parity of Parlett-Sylvester (reorder by sign, triangular Sylvester
solve, back-transform) and of the AUTO choice, through the C ABI."""
import numpy as np
import pytest

from paper_1607_06303_gb300 import workload
from paper_1607_06303_gb300.inputs import make_T

pytestmark = pytest.mark.gpu

TOL_FP64 = 1e-11


def relerr(A, B):
    nb = np.linalg.norm(B)
    return np.linalg.norm(A - B) / (nb if nb > 0 else 1.0)


def dev(p, M):
    return p.to_device(np.asfortranarray(M))


def stream():
    import torch
    return torch.cuda.current_stream().cuda_stream


@pytest.mark.parametrize("n,p,order", [(2, 0.5, "random"), (7, 0.3, "random"), (64, 0.5, "random"),
                                       (65, 0.2, "random"), (200, 0.1, "random"), (333, 0.5, "random"),
                                       (300, 0.25, "sorted"), (129, 0.9, "random"),
                                       # from n = 512 on the blocked reorder: windows of 128 sorted in
                                       # shared memory, their rotations applied by tensor-core products
                                       (512, 0.5, "random"), (700, 0.1, "random"), (1111, 0.3, "random"),
                                       (640, 0.5, "negatives_first")])
def test_reorder_by_sign(gpu_lib, n, p, order):
    import torch
    if order == "negatives_first":
        # every negative above every positive: the most swaps, every window active
        T = make_T(n, p, seed=31, order="sorted")
        d = np.diag(T).copy()
        T[np.arange(n), np.arange(n)] = np.concatenate([d[d < 0], d[d > 0]])
    else:
        T = make_T(n, p, seed=31, order=order)
    Tt = dev(gpu_lib, T)
    Tr = torch.full_like(Tt, 9.0)
    Qt = torch.empty_like(Tt)
    st, k = gpu_lib.signtri_reorder_by_sign(n, Tt.data_ptr(), n, Tr.data_ptr(), n, Qt.data_ptr(), n, stream())
    assert st == 0
    torch.cuda.synchronize()
    R, Q = gpu_lib.to_numpy(Tr), gpu_lib.to_numpy(Qt)
    d = np.diag(T)
    expect = np.concatenate([d[d > 0], d[d < 0]])          # stable partition, exact values
    np.testing.assert_array_equal(np.diag(R), expect)
    assert np.all(np.tril(R, -1) == 0.0)
    assert k == workload.swaps(np.sign(d))
    assert np.linalg.norm(Q.T @ Q - np.eye(n)) <= 1e-13 * n
    assert np.linalg.norm(Q @ R @ Q.T - T) <= 1e-13 * np.linalg.norm(T) * max(1.0, np.sqrt(k) / 10)


@pytest.mark.parametrize("m,pp", [(1, 1), (5, 3), (64, 64), (65, 63), (130, 70), (200, 17), (17, 200), (300, 260)])
def test_sylvester_vs_scipy(gpu_lib, m, pp):
    scipy_linalg = pytest.importorskip("scipy.linalg")
    import torch
    rng = np.random.default_rng(m * 1000 + pp)
    A = np.triu(rng.standard_normal((m, m)) / np.sqrt(m + pp), 1) + np.diag(rng.uniform(0.5, 2, m))
    B = np.triu(rng.standard_normal((pp, pp)) / np.sqrt(m + pp), 1) - np.diag(rng.uniform(0.5, 2, pp))
    C = rng.standard_normal((m, pp))
    At, Bt, Ct = dev(gpu_lib, A), dev(gpu_lib, B), dev(gpu_lib, C)
    Xt = torch.zeros((pp, m), dtype=torch.float64, device="cuda")
    assert gpu_lib.signtri_sylvester(m, pp, At.data_ptr(), m, Bt.data_ptr(), pp, Ct.data_ptr(), m,
                                     Xt.data_ptr(), m, stream()) == 0
    torch.cuda.synchronize()
    X = gpu_lib.to_numpy(Xt)
    Xs = scipy_linalg.solve_sylvester(A, -B, C)
    assert relerr(X, Xs) <= TOL_FP64


@pytest.mark.parametrize("n,p", [(100, 0.1), (257, 0.25), (400, 0.5)])
def test_sylvester_is_sign_block(gpu_lib, oracle_mod, n, p):
    # sorted diagonal: T11 X - X T22 = 2 T12 gives the off-diagonal block of
    # the oracle's sign(T) (Section 2)
    import torch
    T = make_T(n, p, seed=32, order="sorted")
    npos = int((np.diag(T) > 0).sum())
    Tt = dev(gpu_lib, T)
    C2 = dev(gpu_lib, 2 * T[:npos, npos:])
    Xt = torch.zeros((n - npos, npos), dtype=torch.float64, device="cuda")
    base = Tt.data_ptr()
    el = 8
    st = gpu_lib.signtri_sylvester(npos, n - npos, base, n, base + (npos + npos * n) * el, n, C2.data_ptr(), npos,
                                   Xt.data_ptr(), npos, stream())
    assert st == 0
    torch.cuda.synchronize()
    X = gpu_lib.to_numpy(Xt)
    Uo = oracle_mod.sign_tri(T)
    assert relerr(X, Uo[:npos, npos:]) <= TOL_FP64


SIZES = [3, 16, 63, 64, 65, 127, 200, 333]


@pytest.mark.parametrize("n", SIZES)
@pytest.mark.parametrize("p,order", [(0.1, "random"), (0.25, "sorted"), (0.5, "random"), (0.8, "random"),
                                     (0.1, "sorted")])
def test_ps_fp64_vs_oracle(gpu_lib, oracle_mod, n, p, order):
    T = make_T(n, p, seed=33, order=order)
    Tt = gpu_lib.to_device(T)
    Ut = gpu_lib.sign(Tt, gpu_lib.Variant.PS_FP64)
    import torch
    torch.cuda.synchronize()
    U = gpu_lib.to_numpy(Ut)
    Uo = oracle_mod.sign_tri(T)
    assert np.all(np.diag(U) == np.sign(np.diag(T)))
    assert np.all(np.tril(U, -1) == 0.0)
    assert relerr(U, Uo) <= TOL_FP64, relerr(U, Uo)
    info = gpu_lib.signtri_get_info()
    if (np.diag(T) < 0).any() and (np.diag(T) > 0).any():
        assert info.variant == gpu_lib.Variant.PS_FP64


@pytest.mark.parametrize("n", [1000, 1500])
def test_ps_fp64_medium(gpu_lib, oracle_mod, n):
    for p, order in [(0.1, "random"), (0.25, "sorted")]:
        T = make_T(n, p, seed=34, order=order)
        Ut = gpu_lib.sign(gpu_lib.to_device(T), gpu_lib.Variant.PS_FP64)
        import torch
        torch.cuda.synchronize()
        assert relerr(gpu_lib.to_numpy(Ut), oracle_mod.sign_tri(T, schedule="antidiag")) <= TOL_FP64


def test_auto_choice(gpu_lib):
    # Section 3 / Section 6: grouped or nearly one-signed inertia favours
    # Parlett-Sylvester, balanced random order favours Parlett-Higham (run in
    # its arithmetic-efficient form, whose work is the useful count).  The
    # cases are ones where the measured times on GB300 differ clearly:
    # n = 4096, p = 0.1 sorted: PS 20.4 ms against PH 48.8 ms; n = 2000,
    # p = 0.1 random: PH 13.2 ms against PS 29.7 ms; n = 4096 and 8192 with 3
    # negatives in random order: PS 33 and 75 ms against PH 42 and 223 ms.
    import torch
    cases = [(4096, 0.1, "sorted", gpu_lib.Variant.PS_FP64),
             (2000, 0.5, "random", gpu_lib.Variant.PH_FP64_EFFICIENT),
             (2000, 0.1, "random", gpu_lib.Variant.PH_FP64_EFFICIENT),
             (4096, 3 / 4096, "random", gpu_lib.Variant.PS_FP64),
             (8192, 3 / 8192, "random", gpu_lib.Variant.PS_FP64)]
    for n, p, order, expect in cases:
        T = make_T(n, p, seed=35, order=order)
        gpu_lib.sign(gpu_lib.to_device(T), gpu_lib.Variant.AUTO)
        torch.cuda.synchronize()
        info = gpu_lib.signtri_get_info()
        assert info.variant == expect, (n, p, order, info.as_dict())

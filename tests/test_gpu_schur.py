"""The Schur decomposition on the GPU and sign(A) of a general real A through
it (Section 1: sign(A) = Q sign(T) Q^H from a complex Schur form A = Q T Q^H),
via signtri_schur and signtri_sign_general.  Schur forms are not unique, so
the decomposition is checked by what defines it (Q unitary, T upper
triangular, Q T Q^H = A, T's diagonal the eigenvalues); sign(A) is unique and
is compared with the oracle's route through LAPACK's Schur form.  Inputs:
Section 6's uniform[-50, 50] matrices, and matrices of known sign."""
import math

import numpy as np
import pytest

from paper_1607_06303_gb300.inputs import make_A, make_T

pytestmark = pytest.mark.gpu

TOL = 1e-11


def _rel(a, b):
    nb = np.linalg.norm(b)
    return np.linalg.norm(a - b) / (nb if nb > 0 else 1.0)


def _schur(p, A):
    import torch
    Qt, Tt = p.schur(p.to_device(A))
    torch.cuda.synchronize()
    return p.to_numpy(Qt), p.to_numpy(Tt)


def _check_schur(A, Q, T, eig_tol=1e-9):
    n = A.shape[0]
    assert np.all(np.isfinite(Q)) and np.all(np.isfinite(T))
    assert np.all(np.tril(T, -1) == 0)
    eps = np.finfo(float).eps
    assert np.linalg.norm(Q.conj().T @ Q - np.eye(n)) <= 50 * n * eps
    assert _rel(Q @ T @ Q.conj().T, A) <= 50 * n * eps
    if n > 1:
        lo = pytest.importorskip("scipy.optimize")
        ev = np.linalg.eigvals(A)
        C = np.abs(np.diag(T)[:, None] - ev[None, :])
        r, c = lo.linear_sum_assignment(C)
        assert C[r, c].max() <= eig_tol * max(1.0, np.abs(ev).max())


@pytest.mark.parametrize("n", [1, 2, 3, 17, 64, 200, 500])
def test_schur_paper_workload(gpu_lib, n):
    A = make_A(n, seed=n)
    Q, T = _schur(gpu_lib, A)
    _check_schur(A, Q, T)


def test_schur_sweep_counts(gpu_lib):
    """signtri_info's QR counts: none for a matrix that is already
    triangular (every subdiagonal entry is 0, so each eigenvalue deflates at
    once); for Section 6's matrices at least one sweep per four eigenvalues and
    fewer than ten per eigenvalue (about three is usual), each sweep 1 to
    n - 1 rotations."""
    import torch
    T = make_T(40, 0.5, seed=3)
    _schur(gpu_lib, T)
    info = gpu_lib.signtri_get_info()
    assert info.qr_sweeps == 0 and info.qr_rotations == 0
    for n in (64, 200):
        A = make_A(n, seed=n)
        _schur(gpu_lib, A)
        info = gpu_lib.signtri_get_info()
        assert n // 4 <= info.qr_sweeps < 10 * n
        assert info.qr_sweeps <= info.qr_rotations <= (n - 1) * info.qr_sweeps
        sweeps = info.qr_sweeps
        Ad = gpu_lib.to_device(A)
        St = torch.empty_like(Ad)
        gpu_lib.sign_general(Ad, out=St)
        torch.cuda.synchronize()
        assert gpu_lib.signtri_get_info().qr_sweeps == sweeps   # the same decomposition


def test_schur_special_matrices(gpu_lib):
    rng = np.random.Generator(np.random.PCG64(5))
    cases = {
        "triangular": make_T(40, 0.5, seed=3),           # its own Schur form: no sweeps
        "diagonal": np.diag([3.0, -1.0, 2.0, 5.0, -4.0]),
        "rotation": np.array([[0.0, 1.0], [-1.0, 0.0]]),  # eigenvalues +-i
        "jordan": np.array([[2.0, 1.0, 0.0], [0.0, 2.0, 1.0], [0.0, 0.0, 2.0]]),
        "cyclic": np.roll(np.eye(7), 1, axis=0),          # the 7th roots of unity
        "symmetric": (lambda M: M + M.T)(rng.standard_normal((30, 30))),
        "zero": np.zeros((4, 4)),
    }
    for name, A in cases.items():
        A = np.asfortranarray(A)
        Q, T = _schur(gpu_lib, A)
        _check_schur(A, Q, T)
    # a triangular A comes back unchanged, with Q = I
    A = np.asfortranarray(make_T(40, 0.5, seed=3))
    Q, T = _schur(gpu_lib, A)
    assert np.array_equal(T, A.astype(complex)) and np.array_equal(Q, np.eye(40, dtype=complex))


def _sensitivity(oracle_mod, A, ref, rng):
    # the oracle's relative change when A moves by one rounding unit
    # (normwise), which bounds how well any backward-stable route can do
    eps = np.finfo(float).eps
    E = rng.choice([-1.0, 1.0], A.shape) * (eps * np.linalg.norm(A) / A.shape[0])
    return max(1.0, _rel(oracle_mod.sign_general(A + E), ref) / eps)


@pytest.mark.parametrize("n", [1, 2, 33, 100, 300])
def test_sign_general_vs_oracle(gpu_lib, oracle_mod, n):
    pytest.importorskip("scipy.linalg")
    import torch
    A = make_A(n, seed=100 + n)
    ref = oracle_mod.sign_general(A)
    scale = _sensitivity(oracle_mod, A, ref, np.random.Generator(np.random.PCG64(n)))
    S = gpu_lib.to_numpy(gpu_lib.sign_general(gpu_lib.to_device(A)))
    torch.cuda.synchronize()
    assert np.all(np.isfinite(S))
    assert _rel(S, ref) <= TOL * scale, (n, _rel(S, ref), scale)


def test_sign_general_known_sign(gpu_lib):
    # A = P B P^{-1}, B block diagonal with [a b; -b a] and d blocks, whose
    # sign is P diag(sign(a), .., sign(d)) P^{-1}: no Schur form in the check
    import torch
    rng = np.random.Generator(np.random.PCG64(31))
    n = 96
    B = np.zeros((n, n))
    sB = np.zeros(n)
    i = 0
    while i < n:
        a = rng.uniform(0.5, 3.0) * (1.0 if rng.random() < 0.5 else -1.0)
        if i + 1 < n and rng.random() < 0.6:
            b = rng.uniform(0.5, 3.0)
            B[i:i + 2, i:i + 2] = [[a, b], [-b, a]]
            sB[i:i + 2] = np.sign(a)
            i += 2
        else:
            B[i, i] = a
            sB[i] = np.sign(a)
            i += 1
    P = np.eye(n) + 0.3 * rng.standard_normal((n, n)) / math.sqrt(n)
    Pi = np.linalg.inv(P)
    A = np.asfortranarray(P @ B @ Pi)
    ref = P @ np.diag(sB) @ Pi
    S = gpu_lib.to_numpy(gpu_lib.sign_general(gpu_lib.to_device(A)))
    torch.cuda.synchronize()
    assert _rel(S, ref) <= 1e-11 * np.linalg.cond(P) ** 2
    assert np.linalg.norm(S @ S - np.eye(n)) <= 1e-10 * np.linalg.norm(S) ** 2
    assert abs(np.trace(S) - sB.sum()) <= 1e-8


def test_schur_errors_and_arguments(gpu_lib):
    import torch
    p = gpu_lib
    h = torch.cuda.current_stream().cuda_stream
    n = 16
    A = make_A(n, seed=1)
    A[3, 9] = np.nan
    At = p.to_device(A)
    Q = torch.empty((n, n), dtype=torch.complex128, device="cuda")
    T = torch.empty_like(Q)
    S = torch.empty_like(At)
    assert p.signtri_schur(n, At.data_ptr(), n, Q.data_ptr(), n, T.data_ptr(), n, h) == p.Status.ERR_NONFINITE
    assert p.signtri_get_info().bad_index == 9
    assert p.signtri_sign_general(n, At.data_ptr(), n, S.data_ptr(), n, h) == p.Status.ERR_NONFINITE
    assert p.signtri_get_info().bad_index == 9
    # an exact zero eigenvalue: sign undefined (Section 1)
    Z = p.to_device(np.diag([0.0, 1.0, -2.0]))
    S3 = torch.empty_like(Z)
    assert p.signtri_sign_general(3, Z.data_ptr(), 3, S3.data_ptr(), 3, h) == p.Status.ERR_ZERO_EIGENVALUE
    assert p.signtri_get_info().bad_index == 0
    At = p.to_device(make_A(n, seed=2))
    assert p.signtri_sign_general(n, At.data_ptr(), n, At.data_ptr(), n, h) == p.Status.ERR_BAD_ARG
    assert p.signtri_schur(n, At.data_ptr(), n, Q.data_ptr(), n, Q.data_ptr(), n, h) == p.Status.ERR_BAD_ARG
    assert p.signtri_schur(n, At.data_ptr(), n - 1, Q.data_ptr(), n, T.data_ptr(), n, h) == p.Status.ERR_BAD_ARG
    assert p.signtri_schur(0, 0, 1, 0, 1, 0, 1, h) == p.Status.OK
    assert p.signtri_sign_general(0, 0, 1, 0, 1, h) == p.Status.OK
    assert p.signtri_schur_workspace_bytes(n) > 0 and p.signtri_sign_general_workspace_bytes(n) > 0
    torch.cuda.synchronize()


def test_schur_block_triangular_large(gpu_lib):
    # n beyond one pass of the sweep kernel's worker threads (7 x 512 entries
    # per rotation): a block upper triangular A with 2 x 2 diagonal blocks
    # [a b; -b a] (eigenvalues a +- ib) is already Hessenberg and splits at
    # every block, so the QR sweeps are short while the column work above
    # each block spans up to n rows; the eigenvalues are known exactly
    rng = np.random.Generator(np.random.PCG64(41))
    n = 3700
    A = np.triu(rng.uniform(-1.0, 1.0, (n, n)), 2)
    ev = []
    for i in range(0, n, 2):
        a, b = rng.uniform(0.5, 2.0) * rng.choice([-1.0, 1.0]), rng.uniform(0.5, 2.0)
        A[i:i + 2, i:i + 2] = [[a, b], [-b, a]]
        ev += [a + 1j * b, a - 1j * b]
    A = np.asfortranarray(A)
    Q, T = _schur(gpu_lib, A)
    assert np.all(np.tril(T, -1) == 0)
    eps = np.finfo(float).eps
    assert np.linalg.norm(Q.conj().T @ Q - np.eye(n)) <= 50 * n * eps
    assert _rel(Q @ T @ Q.conj().T, A) <= 50 * n * eps
    got = np.sort_complex(np.diag(T))
    want = np.sort_complex(np.array(ev))
    assert np.abs(got - want).max() <= 1e-12 * 4.0

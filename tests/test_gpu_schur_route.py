"""sign(A) = Q sign(T) Q^T from a real Schur pair (Section 1's route,
Algorithm 3's first step), through signtri_sign_schur, against the oracle's
plain-sum route and, for a real Schur form computed by LAPACK on the host,
against the spectral definition."""
import math

import numpy as np
import pytest

from paper_1607_06303_gb300.inputs import make_T, make_orthogonal, make_schur_pair

pytestmark = pytest.mark.gpu

TOL = 1e-11


def _rel(a, b):
    nb = np.linalg.norm(b)
    return np.linalg.norm(a - b) / (nb if nb > 0 else 1.0)


@pytest.mark.parametrize("n,p,order", [(1, 1.0, "random"), (2, 0.5, "random"), (64, 0.5, "random"),
                                       (200, 0.3, "sorted"), (777, 0.5, "random")])
@pytest.mark.parametrize("variant", ["AUTO", "PH_FP64", "PS_FP64", "PH_MIXED_FP16"])
def test_sign_schur_vs_oracle(gpu_lib, oracle_mod, n, p, order, variant):
    import torch
    Q, T = make_schur_pair(n, p, seed=n + 11, order=order)
    S = gpu_lib.sign_schur(gpu_lib.to_device(Q), gpu_lib.to_device(T), gpu_lib.Variant[variant])
    torch.cuda.synchronize()
    got = gpu_lib.to_numpy(S)
    ref = oracle_mod.sign_schur(Q, T)
    assert np.all(np.isfinite(got))
    assert _rel(got, ref) <= TOL, (n, variant, _rel(got, ref))


def test_sign_schur_trivial_inertia_is_exact(gpu_lib):
    # U = +-I gives S = +-I exactly, not Q Q^T with its rounding
    import torch
    n = 300
    Q = make_orthogonal(n, seed=2)
    for p, d in ((0.0, 1.0), (1.0, -1.0)):
        T = make_T(n, p, seed=4)
        S = gpu_lib.to_numpy(gpu_lib.sign_schur(gpu_lib.to_device(Q), gpu_lib.to_device(T)))
        torch.cuda.synchronize()
        assert np.array_equal(S, d * np.eye(n))


def test_sign_schur_lapack_real_schur(gpu_lib):
    # A with real eigenvalues, its real Schur form from LAPACK on the host;
    # S against V sign(L) V^{-1}
    sl = pytest.importorskip("scipy.linalg")
    import torch
    rng = np.random.Generator(np.random.PCG64(9))
    n = 300
    V = np.eye(n) + 0.3 * rng.standard_normal((n, n)) / math.sqrt(n)
    lam = rng.uniform(0.5, 2.0, n) * np.where(rng.random(n) < 0.5, -1.0, 1.0)
    A = V @ np.diag(lam) @ np.linalg.inv(V)
    T, Z = sl.schur(A, output="real")
    T = np.asfortranarray(np.triu(T))
    S = gpu_lib.to_numpy(gpu_lib.sign_schur(gpu_lib.to_device(np.asfortranarray(Z)), gpu_lib.to_device(T)))
    torch.cuda.synchronize()
    ref = V @ np.diag(np.sign(lam)) @ np.linalg.inv(V)
    assert _rel(S, ref) <= 1e-10


def test_sign_schur_arguments(gpu_lib):
    import torch
    p = gpu_lib
    h = torch.cuda.current_stream().cuda_stream
    n = 64
    Q, T = make_schur_pair(n, 0.5, seed=1)
    Qt, Tt = p.to_device(Q), p.to_device(T)
    S = torch.empty_like(Tt)
    assert p.signtri_sign_schur(n, Qt.data_ptr(), n, Tt.data_ptr(), n, S.data_ptr(), n, p.Variant.AUTO, h) == 0
    # S sharing memory with Q or T, short leading dimensions, null pointers
    assert p.signtri_sign_schur(n, Qt.data_ptr(), n, Tt.data_ptr(), n, Qt.data_ptr(), n, p.Variant.AUTO, h) == \
        p.Status.ERR_BAD_ARG
    assert p.signtri_sign_schur(n, Qt.data_ptr(), n, Tt.data_ptr(), n, Tt.data_ptr(), n, p.Variant.AUTO, h) == \
        p.Status.ERR_BAD_ARG
    assert p.signtri_sign_schur(n, Qt.data_ptr(), n - 1, Tt.data_ptr(), n, S.data_ptr(), n, p.Variant.AUTO, h) == \
        p.Status.ERR_BAD_ARG
    assert p.signtri_sign_schur(n, 0, n, Tt.data_ptr(), n, S.data_ptr(), n, p.Variant.AUTO, h) == \
        p.Status.ERR_BAD_ARG
    assert p.signtri_sign_schur(0, 0, 1, 0, 1, 0, 1, p.Variant.AUTO, h) == p.Status.OK
    # a zero eigenvalue is reported with its index, as by sign_tri
    Tz = T.copy()
    Tz[5, 5] = 0.0
    assert p.signtri_sign_schur(n, Qt.data_ptr(), n, p.to_device(Tz).data_ptr(), n, S.data_ptr(), n,
                                p.Variant.AUTO, h) == p.Status.ERR_ZERO_EIGENVALUE
    assert p.signtri_get_info().bad_index == 5
    assert p.signtri_sign_schur_workspace_bytes(n, p.Variant.AUTO) > 0
    torch.cuda.synchronize()

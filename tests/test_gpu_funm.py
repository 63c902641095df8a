"""F = phi(T) for a general function (Section 2: Parlett's substitution,
Algorithm 1, blocked as Algorithm 2) through signtri_funm, against the
oracle's plain Algorithm 1, at every leaf size and across block boundaries.
Parlett's recurrence divides by t_ii - t_jj, so rounding differences grow
with close eigenvalues: the bar is scaled by the problem's own sensitivity
(the oracle's relative change under a one-ulp perturbation of T)."""
import math

import numpy as np
import pytest

from paper_1607_06303_gb300.inputs import make_T

pytestmark = pytest.mark.gpu


def _rel(a, b):
    nb = np.linalg.norm(b)
    return np.linalg.norm(a - b) / (nb if nb > 0 else 1.0)


def _spread_T(n, seed, lo=1.0, hi=3.0):
    rng = np.random.Generator(np.random.PCG64(seed))
    T = np.triu(rng.standard_normal((n, n))) / math.sqrt(n)
    T[np.arange(n), np.arange(n)] = rng.permutation(np.linspace(lo, hi, n))
    return np.asfortranarray(T)


def _bar(oracle_mod, T, phi, ref):
    eps = np.finfo(float).eps
    rng = np.random.default_rng(1)
    Tp = np.asfortranarray(np.triu(T * (1 + eps / 2 * rng.choice([-1.0, 1.0], T.shape))))
    return 1e-12 * max(1.0, _rel(oracle_mod.funm(Tp, phi), ref) / eps)


@pytest.mark.parametrize("n", [1, 5, 64, 65, 200, 700])
@pytest.mark.parametrize("phi", ["exp", "log", "sqrt"])
def test_funm_vs_oracle(gpu_lib, oracle_mod, n, phi):
    import torch
    T = _spread_T(n, n + 17, 1.0, 1.0 + 0.02 * max(n, 1))
    ref = oracle_mod.funm(T, phi)
    F = gpu_lib.to_numpy(gpu_lib.funm(gpu_lib.to_device(T), gpu_lib.Phi[phi.upper()]))
    torch.cuda.synchronize()
    assert np.all(np.isfinite(F)) and np.all(np.tril(F, -1) == 0)
    # phi(t_ii) from CUDA's and the host's math libraries: within an ulp or
    # two for exp and log, identical for the correctly rounded sqrt
    d, dr = np.diag(F), np.diag(ref)
    if phi == "sqrt":
        assert np.array_equal(d, dr)
    else:
        assert np.all(np.abs(d - dr) <= 4.5e-16 * np.abs(dr))
    assert _rel(F, ref) <= _bar(oracle_mod, T, phi, ref), (n, phi, _rel(F, ref))


@pytest.mark.parametrize("b", [16, 32, 64])
def test_funm_every_leaf_size(gpu_lib, oracle_mod, b):
    import torch
    T = _spread_T(300, 5, 1.0, 7.0)
    ref = oracle_mod.funm(T, "sqrt")
    assert gpu_lib.signtri_set_cutoff(b) == 0
    try:
        F = gpu_lib.to_numpy(gpu_lib.funm(gpu_lib.to_device(T), gpu_lib.Phi.SQRT))
        torch.cuda.synchronize()
        assert gpu_lib.signtri_get_info().cutoff == b
    finally:
        gpu_lib.signtri_set_cutoff(0)
    assert _rel(F, ref) <= _bar(oracle_mod, T, "sqrt", ref)


def test_funm_sign_matches_sign_tri(gpu_lib, oracle_mod):
    # sign through Eq. 1 alone, on well-separated eigenvalues, agrees with the
    # Parlett-Higham sign (Algorithm 3) and with the oracle's Algorithm 1
    import torch
    n = 300
    T = _spread_T(n, 9, 1.0, 7.0)
    T[np.arange(n), np.arange(n)] *= np.where(np.arange(n) % 3 == 0, -1.0, 1.0)
    Td = gpu_lib.to_device(T)
    F = gpu_lib.to_numpy(gpu_lib.funm(Td, gpu_lib.Phi.SIGN))
    U = gpu_lib.to_numpy(gpu_lib.sign(Td, gpu_lib.Variant.PH_FP64))
    torch.cuda.synchronize()
    assert _rel(F, oracle_mod.funm(T, "sign")) <= 1e-11
    assert _rel(F, U) <= 1e-11


def test_funm_domain_errors(gpu_lib):
    import torch
    p = gpu_lib
    h = torch.cuda.current_stream().cuda_stream
    n = 100
    T = _spread_T(n, 2)
    T[40, 40] = -0.5                         # log of a negative eigenvalue
    Td = p.to_device(T)
    F = torch.empty_like(Td)
    assert p.signtri_funm(n, Td.data_ptr(), n, F.data_ptr(), n, p.Phi.LOG, h) == p.Status.ERR_DOMAIN
    assert p.signtri_get_info().bad_index == 40
    assert p.signtri_funm(n, Td.data_ptr(), n, F.data_ptr(), n, p.Phi.EXP, h) == p.Status.OK
    T[70, 70] = T[10, 10]                    # repeated eigenvalue: Algorithm 1 divides by 0
    Td = p.to_device(T)
    assert p.signtri_funm(n, Td.data_ptr(), n, F.data_ptr(), n, p.Phi.EXP, h) == p.Status.ERR_DOMAIN
    assert p.signtri_get_info().bad_index == 70
    assert p.signtri_funm(n, Td.data_ptr(), n, Td.data_ptr(), n, p.Phi.EXP, h) == p.Status.ERR_BAD_ARG
    assert p.signtri_funm(n, Td.data_ptr(), n, F.data_ptr(), n, 7, h) == p.Status.ERR_BAD_ARG
    assert p.signtri_funm(0, 0, 1, 0, 1, p.Phi.EXP, h) == p.Status.OK
    torch.cuda.synchronize()

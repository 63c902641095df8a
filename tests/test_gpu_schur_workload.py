"""The paper's own workload (Section 6): real parts of complex Schur forms of
uniform[-50, 50] matrices, balanced inertia or exactly 3 negative eigenvalues.
These are ill-conditioned (eigenvalues with real parts near zero; ||U||_F up
to 1e11 at n = 400), so agreement with the oracle is bounded by the problem's
own sensitivity: the bar is the usual one multiplied by
sens / eps, where sens is the relative change of the oracle's result when
every entry of T is perturbed by one rounding unit (and at least 1)."""
import numpy as np
import pytest

from paper_1607_06303_gb300.inputs import make_T_schur

pytestmark = pytest.mark.gpu
scipy = pytest.importorskip("scipy")


def relerr(A, B):
    return np.linalg.norm(A - B) / np.linalg.norm(B)


@pytest.mark.parametrize("n,n_neg", [(50, None), (200, None), (400, None), (400, 3), (657, None)])
@pytest.mark.parametrize("variant", ["PH_FP64", "PS_FP64", "AUTO", "PH_MIXED_TF32", "PH_MIXED_FP16"])
def test_schur_workload(gpu_lib, oracle_mod, n, n_neg, variant):
    import torch
    T = make_T_schur(n, seed=n, n_neg=n_neg)
    if np.any(np.diag(T) == 0):
        pytest.skip("zero eigenvalue real part")
    Uo = oracle_mod.sign_tri(T)
    eps = np.finfo(float).eps
    rng = np.random.default_rng(0)
    Tp = np.asfortranarray(np.triu(T * (1 + eps / 2 * rng.choice([-1.0, 1.0], T.shape))))
    sens = relerr(oracle_mod.sign_tri(Tp), Uo)
    scale = max(1.0, sens / eps)
    Ut = gpu_lib.sign(gpu_lib.to_device(T), gpu_lib.Variant[variant], check=False)
    torch.cuda.synchronize()
    info = gpu_lib.signtri_get_info()
    U = gpu_lib.to_numpy(Ut)
    tol = (1e-12 if "MIXED" in variant else 1e-11) * scale
    assert relerr(U, Uo) <= tol, (variant, relerr(U, Uo), scale, info.as_dict())

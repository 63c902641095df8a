"""Full-size parity in the launch configuration the benchmark times: the
oracle on the leading and trailing 4096 principal windows (u_ij depends only
on T[i..j, i..j], so the oracle on a window equals the full oracle there),
plus the residual norms for the rest.  Sizes: n = 16384 (the headline), and
n = 8192 for the Parlett-Sylvester / Parlett-Higham inertia cases."""
import numpy as np
import pytest

from paper_1607_06303_gb300.inputs import make_T

pytestmark = [pytest.mark.gpu, pytest.mark.slow]

W = 4096


def window_errors(p, oracle_mod, T, Ut):
    n = T.shape[0]
    errs = []
    for a in (0, n - W):
        Tw = np.asfortranarray(T[a:a + W, a:a + W])
        Uo = oracle_mod.sign_tri(Tw, schedule="antidiag")
        Ug = Ut[a:a + W, a:a + W].cpu().numpy().T
        errs.append(float(np.linalg.norm(Ug - Uo) / np.linalg.norm(Uo)))
    return errs


@pytest.fixture(scope="module")
def T16384():
    return make_T(16384, 0.5, seed=0)


@pytest.mark.parametrize("variant,tol", [("PH_MIXED_TF32", 1e-12), ("PH_MIXED_FP16", 1e-12), ("PH_FP64", 1e-11)])
def test_n16384(gpu_lib, oracle_mod, T16384, variant, tol):
    import torch
    Tt = gpu_lib.to_device(T16384)
    Ut = gpu_lib.sign(Tt, gpu_lib.Variant[variant])
    torch.cuda.synchronize()
    info = gpu_lib.signtri_get_info()
    assert info.variant == gpu_lib.Variant[variant]
    errs = window_errors(gpu_lib, oracle_mod, T16384, Ut)
    assert max(errs) <= tol, errs
    d = torch.diagonal(Ut)
    assert bool(torch.all(d == torch.sign(torch.diagonal(Tt))))
    assert bool(torch.all(torch.triu(Ut, 1) == 0))          # strictly lower part of U (transposed storage)
    if variant.startswith("PH_MIXED"):
        assert info.refine_steps == 1
        assert max(info.resid_commute, info.resid_involution) <= 1e-13


@pytest.mark.parametrize("p,order,variant", [(0.1, "sorted", "PS_FP64"), (0.25, "random", "AUTO"),
                                             (0.1, "random", "PS_FP64")])
def test_n8192_inertia(gpu_lib, oracle_mod, p, order, variant):
    import torch
    T = make_T(8192, p, seed=0, order=order)
    Ut = gpu_lib.sign(gpu_lib.to_device(T), gpu_lib.Variant[variant])
    torch.cuda.synchronize()
    errs = window_errors(gpu_lib, oracle_mod, T, Ut)
    assert max(errs) <= 1e-11, (p, order, variant, errs)

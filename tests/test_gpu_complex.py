"""Complex T and the complex Schur route (Section 1: sign(A) = Q sign(T) Q^*
from a complex Schur form, Algorithm 3's first step), through
signtri_sign_tri_complex and signtri_sign_schur_complex, against the
oracle's complex functions; the Schur route also on Section 6's workload
(uniform[-50, 50] matrices, complex Schur form from LAPACK on the host)."""
import numpy as np
import pytest

from paper_1607_06303_gb300.inputs import make_T, make_T_complex

pytestmark = pytest.mark.gpu

TOL = 1e-11


def _rel(a, b):
    nb = np.linalg.norm(b)
    return np.linalg.norm(a - b) / (nb if nb > 0 else 1.0)


@pytest.mark.parametrize("n,p,order", [(1, 1.0, "random"), (2, 0.5, "random"), (33, 0.5, "random"),
                                       (256, 0.3, "sorted"), (700, 0.5, "random")])
def test_sign_complex_vs_oracle(gpu_lib, oracle_mod, n, p, order):
    import torch
    T = make_T_complex(n, p, seed=n + 3, order=order)
    U = gpu_lib.to_numpy(gpu_lib.sign_complex(gpu_lib.to_device_complex(T)))
    torch.cuda.synchronize()
    ref = oracle_mod.sign_tri_complex(T)
    assert np.all(np.isfinite(U))
    assert np.array_equal(np.diag(U), np.diag(ref))
    assert np.all(np.tril(U, -1) == 0)
    assert _rel(U, ref) <= TOL, (n, _rel(U, ref))


def test_sign_complex_of_real_T(gpu_lib, oracle_mod):
    # a real T in complex form: the real oracle's result, imaginary part 0
    import torch
    T = make_T(300, 0.5, seed=9)
    U = gpu_lib.to_numpy(gpu_lib.sign_complex(gpu_lib.to_device_complex(T.astype(complex))))
    torch.cuda.synchronize()
    assert np.all(U.imag == 0)
    assert _rel(U.real, oracle_mod.sign_tri(T)) <= TOL


@pytest.mark.parametrize("n", [60, 200, 400])
def test_complex_schur_route_paper_workload(gpu_lib, oracle_mod, n):
    # Section 6's matrices through their complex Schur form; the bar scaled by
    # the problem's own sensitivity (the oracle's relative change when T is
    # perturbed by one rounding unit), as for the real Schur workload
    sl = pytest.importorskip("scipy.linalg")
    import torch
    rng = np.random.Generator(np.random.PCG64(n))
    A = rng.uniform(-50.0, 50.0, size=(n, n))
    T, Z = sl.schur(A, output="complex")
    T = np.asfortranarray(np.triu(T))
    Z = np.asfortranarray(Z)
    ref = oracle_mod.sign_schur_complex(Z, T)
    eps = np.finfo(float).eps
    Tp = np.asfortranarray(np.triu(T * (1 + eps / 2 * rng.choice([-1.0, 1.0], T.shape))))
    scale = max(1.0, _rel(oracle_mod.sign_schur_complex(Z, Tp), ref) / eps)
    S = gpu_lib.to_numpy(gpu_lib.sign_schur_complex(gpu_lib.to_device_complex(Z), gpu_lib.to_device_complex(T)))
    torch.cuda.synchronize()
    assert _rel(S, ref) <= TOL * scale, (n, _rel(S, ref), scale)
    # sign(A) of a real A is real
    assert np.abs(S.imag).max() <= 1e-9 * scale * np.abs(S).max()


def test_complex_errors_and_arguments(gpu_lib):
    import torch
    p = gpu_lib
    h = torch.cuda.current_stream().cuda_stream
    n = 64
    T = make_T_complex(n, 0.5, seed=2)
    T[7, 7] = 0.0 + 1.5j          # on the imaginary axis: sign undefined
    Tt = p.to_device_complex(T)
    U = torch.empty_like(Tt)
    assert p.signtri_sign_tri_complex(n, Tt.data_ptr(), n, U.data_ptr(), n, h) == p.Status.ERR_ZERO_EIGENVALUE
    assert p.signtri_get_info().bad_index == 7
    T[7, 7] = np.nan
    Tt = p.to_device_complex(T)
    assert p.signtri_sign_tri_complex(n, Tt.data_ptr(), n, U.data_ptr(), n, h) == p.Status.ERR_NONFINITE
    assert p.signtri_sign_tri_complex(n, Tt.data_ptr(), n, Tt.data_ptr(), n, h) == p.Status.ERR_BAD_ARG
    assert p.signtri_sign_tri_complex(n, Tt.data_ptr(), n - 1, U.data_ptr(), n, h) == p.Status.ERR_BAD_ARG
    assert p.signtri_sign_tri_complex(0, 0, 1, 0, 1, h) == p.Status.OK
    Q = p.to_device_complex(np.eye(n, dtype=complex))
    assert p.signtri_sign_schur_complex(n, Q.data_ptr(), n, Tt.data_ptr(), n, Q.data_ptr(), n, h) == \
        p.Status.ERR_BAD_ARG
    assert p.signtri_complex_workspace_bytes(n) > 0
    torch.cuda.synchronize()

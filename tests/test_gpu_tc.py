"""The tcgen05 block-product engine through the emulated-float64 GEMM entry
point: exact on integer data, and within 2^-44 |A||B| (entrywise) of the
long-double product on random data, ragged shapes included.  The bound comes
from the arithmetic: slices truncate at 2^-56 of the row/column scale, and
the fp32 hi + fp32 lo accumulator of the ~36 per-unit partial products keeps
about 2^-48 per addition, i.e. about 2^-45 in total."""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu


def run_emulated(p, A, B):
    import torch
    m, k = A.shape
    k2, n = B.shape
    At, Bt = p.to_device(A), p.to_device(B)
    Ct = torch.full((n, m), np.nan, dtype=torch.float64, device="cuda")
    st = p.signtri_gemm_emulated(m, n, k, At.data_ptr(), m, Bt.data_ptr(), k, Ct.data_ptr(), m,
                                 torch.cuda.current_stream().cuda_stream)
    assert st == 0, p.signtri_status_string(st)
    torch.cuda.synchronize()
    return p.to_numpy(Ct)


@pytest.mark.parametrize("m,n,k", [(64, 128, 64), (128, 256, 1024), (70, 90, 1500)])
def test_emulated_gemm_exact_on_integers(gpu_lib, m, n, k):
    rng = np.random.default_rng(m + n + k)
    A = rng.integers(-100, 101, size=(m, k)).astype(np.float64)
    B = rng.integers(-100, 101, size=(k, n)).astype(np.float64)
    C = run_emulated(gpu_lib, A, B)
    np.testing.assert_array_equal(C, A @ B)     # integers below 2^53: exact


@pytest.mark.parametrize("m,n,k", [(1, 1, 1), (100, 130, 70), (256, 256, 2048), (300, 200, 1500), (64, 64, 4100)])
def test_emulated_gemm_accuracy(gpu_lib, m, n, k):
    rng = np.random.default_rng(7 * m + n)
    A = rng.standard_normal((m, k)) * np.exp(rng.uniform(-3, 3, (m, 1)))
    B = rng.standard_normal((k, n)) * np.exp(rng.uniform(-3, 3, (1, n)))
    C = run_emulated(gpu_lib, A, B)
    ref = (A.astype(np.longdouble) @ B.astype(np.longdouble))
    bound = np.abs(A) @ np.abs(B)
    err = np.abs(C.astype(np.longdouble) - ref)
    assert np.all(np.isfinite(C))
    assert np.all(err <= 2.0 ** -44 * bound + 1e-300), float(np.max(err / bound))

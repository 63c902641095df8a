"""Failure detection without a GPU fault: a bounded device wait on a barrier
that nothing completes gives up and reports SIGNTRI_ERR_TIMEOUT; the context
stays usable.  The same wait primitive guards every pipeline wait of the
tensor-core kernels."""
import numpy as np
import pytest

from paper_1607_06303_gb300.inputs import make_T

pytestmark = pytest.mark.gpu


def test_bounded_wait_times_out_and_recovers(gpu_lib, oracle_mod):
    import torch
    h = torch.cuda.current_stream().cuda_stream
    assert gpu_lib.signtri_selftest_wait(True, 2_000_000, h) == gpu_lib.Status.OK
    assert gpu_lib.signtri_selftest_wait(False, 2_000_000, h) == gpu_lib.Status.ERR_TIMEOUT
    assert gpu_lib.signtri_selftest_wait(False, 0, h) == gpu_lib.Status.ERR_BAD_ARG
    # the context is still usable: a mixed (tensor-core) solve succeeds
    T = make_T(300, 0.5, seed=61)
    U = gpu_lib.to_numpy(gpu_lib.sign(gpu_lib.to_device(T), gpu_lib.Variant.PH_MIXED_TF32))
    Uo = oracle_mod.sign_tri(T)
    assert np.linalg.norm(U - Uo) <= 1e-12 * np.linalg.norm(Uo)

"""Batched entry point: many problems of uneven size and inertia in one call,
each checked against the oracle; per-matrix status codes; cutoff table and
autotuner."""
import numpy as np
import pytest

from paper_1607_06303_gb300.inputs import make_T

pytestmark = pytest.mark.gpu

TOL_FP64 = 1e-11


def relerr(A, B):
    nb = np.linalg.norm(B)
    return np.linalg.norm(A - B) / (nb if nb > 0 else 1.0)


def run_batch(p, Ts, variant, bad_ld=()):
    import torch
    dT = [p.to_device(T) if T.shape[0] else torch.empty(0, dtype=torch.float64, device="cuda") for T in Ts]
    dU = [torch.full_like(t, np.nan) for t in dT]
    ns = [T.shape[0] for T in Ts]
    ld = [max(n, 1) for n in ns]
    ldu = [(n - 1 if i in bad_ld else max(n, 1)) for i, n in enumerate(ns)]
    st, info = p.sign_tri_batched(ns, [t.data_ptr() for t in dT], ld, [u.data_ptr() for u in dU], ldu, variant,
                                  torch.cuda.current_stream().cuda_stream)
    torch.cuda.synchronize()
    return st, info, [p.to_numpy(u) if u.numel() else np.zeros((0, 0)) for u in dU]


def batch_inputs():
    rng = np.random.default_rng(5)
    Ts = []
    for i, n in enumerate([0, 1, 2, 17, 64, 65, 130, 257, 300, 513, 31, 700]):
        for pr, order in [(0.5, "random"), (0.0, "random"), (1.0, "random"), (0.2, "random"), (0.9, "sorted"),
                          (0.05, "random")]:
            if rng.random() < 0.5:
                continue
            Ts.append(make_T(n, pr, seed=100 + 7 * i + int(10 * pr), order=order))
    return Ts


@pytest.mark.parametrize("variant", ["AUTO", "PH_FP64", "PH_FP64_EFFICIENT"])
def test_batched_vs_oracle(gpu_lib, oracle_mod, variant):
    Ts = batch_inputs()
    assert len(Ts) > 15
    st, info, Us = run_batch(gpu_lib, Ts, gpu_lib.Variant[variant])
    assert st == 0
    for T, U, code in zip(Ts, Us, info):
        assert code == 0
        if T.shape[0] == 0:
            continue
        Uo = oracle_mod.sign_tri(T)
        assert np.all(np.tril(U, -1) == 0.0) and np.all(np.diag(U) == np.diag(Uo))
        assert relerr(U, Uo) <= TOL_FP64, (T.shape[0], relerr(U, Uo))


def test_batched_statuses(gpu_lib, oracle_mod):
    Ts = [make_T(100, 0.5, seed=1), make_T(80, 0.5, seed=2), make_T(90, 0.5, seed=3), make_T(70, 0.5, seed=4)]
    Ts[1][40, 40] = 0.0
    Ts[2][10, 10] = np.nan
    st, info, Us = run_batch(gpu_lib, Ts, gpu_lib.Variant.PH_FP64, bad_ld=(3,))
    assert st == 0
    assert info == [0, gpu_lib.Status.ERR_ZERO_EIGENVALUE, gpu_lib.Status.ERR_NONFINITE, gpu_lib.Status.ERR_BAD_ARG]
    assert relerr(Us[0], oracle_mod.sign_tri(Ts[0])) <= TOL_FP64


def test_cutoff_table_and_autotune(gpu_lib, oracle_mod):
    import torch
    old = gpu_lib.signtri_get_cutoff_table()
    try:
        for b in (16, 32, 64):
            assert gpu_lib.signtri_set_cutoff_table([b] * 32) == 0
            Ts = [make_T(n, 0.5, seed=n) for n in (40, 100, 333)]
            st, info, Us = run_batch(gpu_lib, Ts, gpu_lib.Variant.PH_FP64)
            assert st == 0 and info == [0, 0, 0]
            for T, U in zip(Ts, Us):
                assert relerr(U, oracle_mod.sign_tri(T)) <= TOL_FP64
        assert gpu_lib.signtri_set_cutoff_table([48]) == gpu_lib.Status.ERR_BAD_ARG
        # the autotuner times the batched path per size bucket (leaf size) and,
        # from n = 1024 on, the fp16 mixed form on its own (variant)
        assert gpu_lib.signtri_autotune(1024, torch.cuda.current_stream().cuda_stream) == 0
        table = gpu_lib.signtri_get_cutoff_table()
        assert all(table[k] in (16, 32, 64) for k in range(5, 11))
        vt = gpu_lib.signtri_get_variant_table()
        assert all(vt[k] == 0 for k in range(5, 10))          # below 1024: never the single mixed path
        assert vt[10] in (0, int(gpu_lib.Variant.PH_MIXED_FP16))
        # a batch under the tuned tables
        Ts = [make_T(n, 0.5, seed=n + 1) for n in (40, 333, 1024)]
        st, info, Us = run_batch(gpu_lib, Ts, gpu_lib.Variant.AUTO)
        assert st == 0 and info == [0, 0, 0]
        for T, U in zip(Ts, Us):
            assert relerr(U, oracle_mod.sign_tri(T)) <= 1e-12
    finally:
        gpu_lib.signtri_set_cutoff_table(old)
        gpu_lib.signtri_set_variant_table([])


def test_variant_table_routes_auto(gpu_lib, oracle_mod):
    # under AUTO, the size buckets the variant table names run through that
    # variant one by one, the rest through the batched float64 path
    Ts = [make_T(n, 0.5, seed=300 + n) for n in (90, 300, 600)]
    vt = [0] * 32
    vt[8] = int(gpu_lib.Variant.PH_MIXED_FP16)      # 256 <= n < 512
    try:
        assert gpu_lib.signtri_set_variant_table(vt) == 0
        assert gpu_lib.signtri_get_variant_table()[8] == int(gpu_lib.Variant.PH_MIXED_FP16)
        st, info, Us = run_batch(gpu_lib, Ts, gpu_lib.Variant.AUTO)
    finally:
        gpu_lib.signtri_set_variant_table([])
    assert st == 0 and info == [0, 0, 0]
    for T, U in zip(Ts, Us):
        assert relerr(U, oracle_mod.sign_tri(T)) <= 1e-12
    # 0 (AUTO's value) keeps a bucket on the batched path; no such variant: refused
    assert gpu_lib.signtri_set_variant_table([0, 0]) == 0
    assert gpu_lib.signtri_set_variant_table([77]) == gpu_lib.Status.ERR_BAD_ARG
    assert gpu_lib.signtri_set_variant_table([-1]) == gpu_lib.Status.ERR_BAD_ARG
    gpu_lib.signtri_set_variant_table([])


def test_batched_graph_is_kept(gpu_lib, oracle_mod):
    # a second call with a batch of the same shape relaunches the graph built
    # by the first (its tables kept); a batch of another shape builds anew;
    # every result meets the bar
    Ts = [make_T(n, 0.4, seed=400 + n) for n in (70, 130, 257, 400)]
    h0, b0 = gpu_lib.signtri_batched_cache_stats()
    for rep in range(2):
        st, info, Us = run_batch(gpu_lib, Ts, gpu_lib.Variant.PH_FP64_EFFICIENT)
        assert st == 0 and info == [0] * len(Ts)
        for T, U in zip(Ts, Us):
            assert relerr(U, oracle_mod.sign_tri(T)) <= TOL_FP64
    h1, b1 = gpu_lib.signtri_batched_cache_stats()
    assert h1 >= h0 + 1 and b1 >= b0 + 1
    Ts2 = Ts[:3] + [make_T(401, 0.4, seed=9)]
    st, info, Us = run_batch(gpu_lib, Ts2, gpu_lib.Variant.PH_FP64_EFFICIENT)
    assert st == 0 and info == [0] * len(Ts2)
    assert relerr(Us[3], oracle_mod.sign_tri(Ts2[3])) <= TOL_FP64
    h2, b2 = gpu_lib.signtri_batched_cache_stats()
    assert b2 >= b1 + 1


@pytest.mark.parametrize("variant", ["PH_MIXED_TF32", "PH_MIXED_FP16"])
def test_batched_mixed_variant(gpu_lib, oracle_mod, variant):
    # mixed-precision problems in a batch run one after another through the
    # single-matrix path; each meets the mixed bar
    Ts = [make_T(n, 0.5, seed=200 + n) for n in (70, 200, 513)]
    st, info, Us = run_batch(gpu_lib, Ts, gpu_lib.Variant[variant])
    assert st == 0 and info == [0, 0, 0]
    for T, U in zip(Ts, Us):
        assert relerr(U, oracle_mod.sign_tri(T)) <= 1e-12


def test_batched_overlapping_operands(gpu_lib, oracle_mod):
    """A matrix whose U shares elements with its T is rejected with
    SIGNTRI_ERR_BAD_ARG and left alone; the others are solved.  T and the
    overlapping U sit in one buffer large enough for both, so every access
    stays inside it whatever the check decides."""
    import torch
    T0, T1 = make_T(60, 0.5, seed=5), make_T(50, 0.5, seed=6)
    n1 = 50
    dT0 = gpu_lib.to_device(T0)
    dU0 = torch.full_like(dT0, np.nan)
    buf = torch.zeros(2 * n1 * n1, dtype=torch.float64, device="cuda")
    buf[:n1 * n1] = gpu_lib.to_device(T1).reshape(-1)
    pT1 = buf.data_ptr()
    pU1 = pT1 + 8 * n1 * 10                     # U starts at column 10 of T
    st, info = gpu_lib.sign_tri_batched([60, n1], [dT0.data_ptr(), pT1], [60, n1], [dU0.data_ptr(), pU1],
                                        [60, n1], gpu_lib.Variant.PH_FP64, torch.cuda.current_stream().cuda_stream)
    torch.cuda.synchronize()
    assert st == 0
    assert info == [0, gpu_lib.Status.ERR_BAD_ARG]
    assert relerr(gpu_lib.to_numpy(dU0), oracle_mod.sign_tri(T0)) <= TOL_FP64
    np.testing.assert_array_equal(gpu_lib.to_numpy(buf[:n1 * n1].reshape(n1, n1)), T1)
    assert bool(torch.all(buf[n1 * n1:] == 0))

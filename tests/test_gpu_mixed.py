"""GPU parity of the mixed-precision variants (tensor-core block sums, fp32
leaves, refinement with emulated-float64 residuals) against the oracle.
Bar: relative Frobenius error <= 1e-12 after refinement."""
import numpy as np
import pytest

from paper_1607_06303_gb300.inputs import make_T

pytestmark = pytest.mark.gpu

TOL_MIXED = 1e-12


def relerr(A, B):
    nb = np.linalg.norm(B)
    return np.linalg.norm(A - B) / (nb if nb > 0 else 1.0)


def solve(p, T, variant):
    import torch
    Ut = p.sign(p.to_device(T), variant)
    torch.cuda.synchronize()
    return p.to_numpy(Ut), p.signtri_get_info()


@pytest.mark.parametrize("variant", ["PH_MIXED_TF32", "PH_MIXED_BF16", "PH_MIXED_FP16"])
@pytest.mark.parametrize("n,pr,order", [(3, 0.5, "random"), (50, 0.5, "random"), (64, 0.5, "random"),
                                        (65, 0.4, "random"), (130, 0.5, "random"), (257, 0.3, "random"),
                                        (300, 0.5, "sorted"), (700, 0.5, "random"), (1000, 0.1, "random"),
                                        (1025, 0.5, "random")])   # 1025: a superblock of one index
def test_mixed_vs_oracle(gpu_lib, oracle_mod, variant, n, pr, order):
    T = make_T(n, pr, seed=41, order=order)
    U, info = solve(gpu_lib, T, gpu_lib.Variant[variant])
    Uo = oracle_mod.sign_tri(T, schedule="antidiag")
    assert np.all(np.diag(U) == np.sign(np.diag(T)))
    assert np.all(np.tril(U, -1) == 0.0)
    err = relerr(U, Uo)
    assert err <= TOL_MIXED, (err, info.as_dict())
    assert info.variant == gpu_lib.Variant[variant], info.as_dict()     # no fallback needed
    assert max(info.resid_commute, info.resid_involution) <= 1e-13


@pytest.mark.parametrize("n", [1500, 2048])
def test_mixed_medium(gpu_lib, oracle_mod, n):
    T = make_T(n, 0.5, seed=42)
    Uo = oracle_mod.sign_tri(T, schedule="antidiag")
    for variant in ("PH_MIXED_TF32", "PH_MIXED_BF16", "PH_MIXED_FP16"):
        U, info = solve(gpu_lib, T, gpu_lib.Variant[variant])
        assert relerr(U, Uo) <= TOL_MIXED, (variant, relerr(U, Uo), info.as_dict())


def test_mixed_fallback_to_fp64(gpu_lib, oracle_mod):
    # no refinement step allowed: the solver must fall back to float64
    T = make_T(400, 0.5, seed=43)
    try:
        assert gpu_lib.signtri_set_refinement(1e-13, 0) == 0
        U, info = solve(gpu_lib, T, gpu_lib.Variant.PH_MIXED_BF16)
    finally:
        gpu_lib.signtri_set_refinement(0, -1)
    assert info.variant == gpu_lib.Variant.PH_FP64
    assert info.refine_steps == 0
    assert relerr(U, oracle_mod.sign_tri(T)) <= 1e-11


@pytest.mark.parametrize("variant", ["PH_MIXED_TF32", "PH_MIXED_FP16"])
@pytest.mark.parametrize("pattern", ["blocks_of_one_sign", "alternating", "one_negative", "ragged_tail"])
def test_mixed_gathered_residual_patterns(gpu_lib, oracle_mod, pattern, variant):
    # the first residual gathers indices per 1024-index superblock by sign;
    # cover superblocks of one sign, every class boundary inside 64-blocks,
    # a single negative index, and a ragged last superblock
    n = {"ragged_tail": 2200}.get(pattern, 2600)
    rng = np.random.default_rng(44)
    T = np.triu(rng.standard_normal((n, n)) / np.sqrt(n), 1)
    idx = np.arange(n)
    if pattern == "blocks_of_one_sign":
        s = np.where((idx // 1024) % 2 == 0, 1.0, -1.0)
        s[2048:] = np.where(idx[2048:] % 3 == 0, -1.0, 1.0)
    elif pattern == "alternating":
        s = np.where(idx % 2 == 0, 1.0, -1.0)
    elif pattern == "one_negative":
        s = np.ones(n)
        s[1500] = -1.0
    else:
        s = np.where(rng.random(n) < 0.3, -1.0, 1.0)
    T[idx, idx] = s * rng.uniform(0.5, 2.0, n)
    T = np.asfortranarray(T)
    U, info = solve(gpu_lib, T, gpu_lib.Variant[variant])
    Uo = oracle_mod.sign_tri(T, schedule="antidiag")
    assert relerr(U, Uo) <= TOL_MIXED, (pattern, relerr(U, Uo), info.as_dict())
    assert info.variant == gpu_lib.Variant[variant], info.as_dict()
    assert max(info.resid_commute, info.resid_involution) <= 1e-13


@pytest.mark.parametrize("scale", [1e-20, 1e20])
def test_fp16_split_scales_with_the_input(gpu_lib, oracle_mod, scale):
    # sign(cT) = sign(T) for c > 0: the fp16 split's power-of-two scales
    # follow T, U and the residual, so the variant runs without fallback at
    # magnitudes far outside fp16's range
    T = make_T(700, 0.5, seed=46)
    U, info = solve(gpu_lib, np.asfortranarray(T * scale), gpu_lib.Variant.PH_MIXED_FP16)
    assert info.variant == gpu_lib.Variant.PH_MIXED_FP16, info.as_dict()
    assert relerr(U, oracle_mod.sign_tri(T)) <= TOL_MIXED


def test_fp16_split_out_of_range_falls_back(gpu_lib, oracle_mod):
    # U's scale comes from its 64 x 64 diagonal blocks; with the strictly
    # upper entries inside those blocks a million times smaller than the
    # rest, the off-diagonal entries of U overflow fp16 after scaling, the
    # residual is not finite, and the call falls back to float64
    n = 500
    T = make_T(n, 0.5, seed=47)
    idx = np.arange(n)
    same_block = (idx[:, None] // 64) == (idx[None, :] // 64)
    T = np.asfortranarray(np.where(same_block & (idx[:, None] < idx[None, :]), T * 1e-6, T))
    U, info = solve(gpu_lib, T, gpu_lib.Variant.PH_MIXED_FP16)
    assert info.variant == gpu_lib.Variant.PH_FP64, info.as_dict()
    assert relerr(U, oracle_mod.sign_tri(T)) <= 1e-11


def test_verification_modes(gpu_lib, oracle_mod):
    # acceptance by the full residuals and by their 128-probe estimate: same
    # result within the mixed bar, estimates within a small factor of the
    # full values (the estimator is unbiased; 128 probes)
    T = make_T(1500, 0.5, seed=45)
    Uo = oracle_mod.sign_tri(T, schedule="antidiag")
    try:
        assert gpu_lib.signtri_set_verification(1) == 0
        Uf, info_f = solve(gpu_lib, T, gpu_lib.Variant.PH_MIXED_TF32)
        assert gpu_lib.signtri_set_verification(0) == 0
        Up, info_p = solve(gpu_lib, T, gpu_lib.Variant.PH_MIXED_TF32)
    finally:
        gpu_lib.signtri_set_verification(0)
    assert relerr(Uf, Uo) <= TOL_MIXED and relerr(Up, Uo) <= TOL_MIXED
    assert info_f.variant == info_p.variant == gpu_lib.Variant.PH_MIXED_TF32
    for a, b in [(info_p.resid_commute, info_f.resid_commute), (info_p.resid_involution, info_f.resid_involution)]:
        assert 0 < a <= 1e-13 and 0 < b <= 1e-13
        assert b / 3 <= a <= 3 * b, (a, b)
    assert gpu_lib.signtri_set_verification(2) == gpu_lib.Status.ERR_BAD_ARG


@pytest.mark.parametrize("variant,slices,pairs", [("PH_MIXED_TF32", 3, 6), ("PH_MIXED_FP16", 2, 3)])
@pytest.mark.parametrize("n", [700, 1000])
def test_sweep_operand_byte_count(gpu_lib, n, variant, slices, pairs):
    # the byte model behind the sweeps' HBM roofline: every anti-diagonal d
    # of the nb = ceil(n/64) block partition reads, per tile (I, I+d), 64-row
    # panels of S 16-bit slices (three bf16 or two fp16) over its d+1 K-blocks once: four panels in
    # the initial sweep, six for the correction's two launches side by side
    # (they share the E panels).  In the initial sweep a lead anti-diagonal d
    # (odd, >= 3, d + 1 < nb) also sums d + 1's tiles over K-blocks
    # I+2 .. I+d-1 reading only new column panels, and d + 1 then completes
    # four K-blocks per tile.  One refinement step.
    import torch
    T = make_T(n, 0.5, seed=n)
    Tt = gpu_lib.to_device(T)
    Ut = torch.empty_like(Tt)
    h = torch.cuda.current_stream().cuda_stream
    gpu_lib.signtri_profile_reset()
    gpu_lib.signtri_profile_enable(True)
    try:
        assert gpu_lib.sign_tri(n, Tt.data_ptr(), n, Ut.data_ptr(), n, gpu_lib.Variant[variant], h) == 0
        torch.cuda.synchronize()
        got = gpu_lib.signtri_profile_read_bytes(gpu_lib.signtri.KC_BLOCK_SUMS_TC)
        flops = gpu_lib.signtri_profile_read_flops(gpu_lib.signtri.KC_BLOCK_SUMS_TC)
    finally:
        gpu_lib.signtri_profile_enable(False)
    info = gpu_lib.signtri_get_info()
    assert info.variant == gpu_lib.Variant[variant] and info.refine_steps == 1, info.as_dict()
    nb = (n + 63) // 64
    lead = lambda d: d >= 3 and d % 2 == 1 and d + 1 < nb
    follow = lambda d: d >= 4 and d % 2 == 0 and lead(d - 1)
    units = 0
    for d in range(1, nb):
        kb = (nb - d) * (d + 1)
        if follow(d):
            units += 4 * 4 * (nb - d)
        else:
            units += 4 * kb + (2 * (nb - d - 1) * (d - 2) if lead(d) else 0)
        units += 6 * kb
    assert got == units * slices * 64 * 64 * 2, (got, units)
    # tensor work: slice pairs x 2*64^3 per tile K-block and used quadrant (3 in the
    # initial sweep, 2 in each correction launch)
    kb = sum((nb - d) * (d + 1) for d in range(1, nb))
    assert flops == pytest.approx(pairs * 2 * 64 ** 3 * kb * (3 + 2 + 2), rel=1e-12)
    assert gpu_lib.signtri_profile_read_bytes(gpu_lib.signtri.KC_RESIDUAL) == 0

// ph_fp64.cu -- recursive Parlett-Higham in float64 (Algorithms 3-6).
//
// The recursion of Algorithms 4-6 computes every off-diagonal block U_ij of
// the nested partition from the block sums (Section 5.2)
//     X_ij = sum_{k strictly between} (U_ik T_kj - T_ik U_kj)
//     Y_ij = sum_{k strictly between}  U_ik U_kj
// and finishes each block with the element recurrence of Algorithm 6 (the
// 1x1 case) below the cutoff b.  Every (i, k, j) block triple contributes
// once, so the work is the n^3 of the matrix-multiply form (Section 5.3).
//
// On the GPU the same block equations are scheduled by block anti-diagonal
// d = J - I of the b x b partition instead of depth-first: block (I, I+d)
// needs only blocks with a smaller anti-diagonal, so all nb-d blocks of one
// anti-diagonal are independent.  Per anti-diagonal:
//   1. ph_gemm_kernel: X_IJ and Y_IJ over K = I+1 .. J-1, the anti-diagonal's
//      k-chunks split evenly over a fixed number of CTAs (kStreamCtas); the
//      partial slabs are summed in a fixed order by the leaf (no atomics, so
//      results are run-to-run deterministic);
//   2. offdiag_leaf_kernel: the in-block element recurrence seeded with
//      X_IJ, Y_IJ (Algorithm 6, 1x1 case, applied inside the b x b block).
// The diagonal blocks are all independent (Algorithm 5 calls on disjoint
// diagonal blocks) and are computed first by diag_leaf_kernel (Algorithm 3
// on each block).
// The arithmetic-efficient form (Section 5.3) replaces step 1 by
// ph_gemm_split_kernel: one sum per entry, X or Y by the signs of its row and
// column, over the same k-chunk split.
#include <algorithm>

#include "internal.cuh"
#include "ph_bodies.cuh"

namespace signtri {

using namespace ph;

namespace {

template <int B>
__global__ void __launch_bounds__(kThreads)
diag_leaf_kernel(int n, const double *__restrict__ T, int ldt, double *__restrict__ U, int ldu)
{
    diag_leaf_body<B>(n, T, ldt, U, ldu, blockIdx.x);
}

// Block sums of anti-diagonal d, evenly split over G CTAs (see
// kStreamCtas): each CTA walks its chunk range tile by tile.
template <int B>
__global__ void __launch_bounds__(kThreads)
ph_gemm_kernel(int n, const double *__restrict__ T, int ldt, const double *__restrict__ U, int ldu,
               int d, long long W, double *__restrict__ PX, double *__restrict__ PY)
{
    const int G = sk_ctas(W);
    const long long cpt = sk_chunks_per_tile(d, B);
    const long long c = blockIdx.x;
    const long long x1 = (c + 1) * W / G;
    for (long long x = c * W / G; x < x1;) {
        const int I = (int)(x / cpt);
        const long long t0 = (long long)I * cpt;
        const long long xe = min(x1, t0 + cpt);
        const size_t slab = (size_t)(c + I) * B * B;
        ph_gemm_body<B>(n, T, ldt, U, ldu, I, I + d, (I + 1) * B + (int)(x - t0) * 16,
                        (I + 1) * B + (int)(xe - t0) * 16, PX + slab, PY + slab);
        x = xe;
    }
}

template <int B>
__global__ void __launch_bounds__(kThreads)
offdiag_leaf_kernel(int n, const double *__restrict__ T, int ldt, double *__restrict__ U, int ldu,
                    int d, long long W, const double *__restrict__ PX, const double *__restrict__ PY)
{
    const int I = blockIdx.x;
    int count = 0;
    size_t base = 0;
    if (W > 0) {
        const int G = sk_ctas(W);
        const long long cpt = sk_chunks_per_tile(d, B);
        const long long f = sk_owner((long long)I * cpt, W, G);
        const long long l = sk_owner((long long)(I + 1) * cpt - 1, W, G);
        count = (int)(l - f + 1);
        base = (size_t)(f + I) * B * B;
    }
    offdiag_leaf_body<B>(n, T, ldt, U, ldu, I, I + d, count, PX + base, PY + base, (size_t)B * B);
}

template <int B>
__global__ void __launch_bounds__(kThreads)
ph_gemm_split_kernel(int n, const double *__restrict__ T, int ldt, const double *__restrict__ U, int ldu, int d,
                     long long W, const short *__restrict__ perm, const int *__restrict__ npos,
                     double *__restrict__ PZ)
{
    const int G = sk_ctas(W);
    const long long cpt = sk_chunks_per_tile(d, B);
    const long long c = blockIdx.x;
    const long long x1 = (c + 1) * W / G;
    for (long long x = c * W / G; x < x1;) {
        const int I = (int)(x / cpt);
        const long long t0 = (long long)I * cpt;
        const long long xe = min(x1, t0 + cpt);
        ph_gemm_split_body<B>(n, T, ldt, U, ldu, I, I + d, (I + 1) * B + (int)(x - t0) * 16,
                              (I + 1) * B + (int)(xe - t0) * 16, perm, npos, PZ + (size_t)(c + I) * B * B);
        x = xe;
    }
}

template <int B>
__global__ void sign_perm_kernel(int n, const double *__restrict__ T, int ldt, short *__restrict__ perm,
                                 int *__restrict__ npos)
{
    sign_perm_body<B>(n, T, ldt, blockIdx.x, perm, npos);
}

// One schedule for both forms: per anti-diagonal d, the block sums (if any
// K-block lies between) then the in-block leaves.  split = true runs the
// arithmetic-efficient form (one sum per entry, X or Y by the sign pair).
template <int B>
signtri_status run_b(int n, const double *T, int ldt, double *U, int ldu, bool split, Arena &ws,
                     cudaStream_t st)
{
    const int nb = (n + B - 1) / B;
    const size_t slabs = max_slabs(n, B);
    double *PX = nullptr, *PY = nullptr;
    short *perm = nullptr;
    int *npos = nullptr;
    if (slabs > 0) {
        PX = static_cast<double *>(ws.take(slabs * B * B * sizeof(double)));
        if (!PX) return SIGNTRI_ERR_NO_WORKSPACE;
        if (split) {
            PY = PX;   // one sum per entry: the leaf reads X or Y from the same slab
        } else {
            PY = static_cast<double *>(ws.take(slabs * B * B * sizeof(double)));
            if (!PY) return SIGNTRI_ERR_NO_WORKSPACE;
        }
    }
    if (split) {
        perm = static_cast<short *>(ws.take((size_t)nb * B * sizeof(short)));
        npos = static_cast<int *>(ws.take((size_t)nb * sizeof(int)));
        if (!perm || !npos) return SIGNTRI_ERR_NO_WORKSPACE;
    }
    // per function and device; cheap, so set on every call
    SGT_CUDA_TRY(cudaFuncSetAttribute(offdiag_leaf_kernel<B>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                      (int)leaf_smem<B>()));
    SGT_CUDA_TRY(cudaFuncSetAttribute(diag_leaf_kernel<B>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                      (int)diag_smem<B>()));
    signtri_status rs = launch_zero_strict_lower(n, U, ldu, st);
    if (rs != SIGNTRI_OK) return rs;
    {
        ProfScope ps(SIGNTRI_KC_DIAG_LEAF, st);
        if (split) {
            sign_perm_kernel<B><<<nb, B, 0, st>>>(n, T, ldt, perm, npos);
            SGT_LAUNCH_CHECK();
        }
        diag_leaf_kernel<B><<<nb, kThreads, diag_smem<B>(), st>>>(n, T, ldt, U, ldu);
        SGT_LAUNCH_CHECK();
    }
    for (int d = 1; d < nb; d++) {
        const int ntiles = nb - d;
        const long long W = (long long)ntiles * sk_chunks_per_tile(d, B);
        if (W > 0) {
            ProfScope ps(SIGNTRI_KC_BLOCK_SUMS_F64, st);
            if (split)
                ph_gemm_split_kernel<B><<<sk_ctas(W), kThreads, 0, st>>>(n, T, ldt, U, ldu, d, W, perm, npos, PX);
            else
                ph_gemm_kernel<B><<<sk_ctas(W), kThreads, 0, st>>>(n, T, ldt, U, ldu, d, W, PX, PY);
            SGT_LAUNCH_CHECK();
        }
        {
            ProfScope ps(SIGNTRI_KC_OFFDIAG_LEAF, st);
            offdiag_leaf_kernel<B><<<ntiles, kThreads, leaf_smem<B>(), st>>>(n, T, ldt, U, ldu, d, W, PX, PY);
            SGT_LAUNCH_CHECK();
        }
    }
    return SIGNTRI_OK;
}

}  // namespace

signtri_status diag_leaves_f64(int n, const double *T, int ldt, double *U, int ldu, int b, cudaStream_t st)
{
    const int nb = (n + b - 1) / b;
    ProfScope ps(SIGNTRI_KC_DIAG_LEAF, st);
    switch (b) {
    case 64:
        SGT_CUDA_TRY(cudaFuncSetAttribute(diag_leaf_kernel<64>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                          (int)diag_smem<64>()));
        diag_leaf_kernel<64><<<nb, kThreads, diag_smem<64>(), st>>>(n, T, ldt, U, ldu);
        break;
    case 32:
        diag_leaf_kernel<32><<<nb, kThreads, diag_smem<32>(), st>>>(n, T, ldt, U, ldu);
        break;
    case 16:
        diag_leaf_kernel<16><<<nb, kThreads, diag_smem<16>(), st>>>(n, T, ldt, U, ldu);
        break;
    default:
        return SIGNTRI_ERR_BAD_ARG;
    }
    SGT_LAUNCH_CHECK();
    return SIGNTRI_OK;
}

size_t ph_fp64_workspace_bytes(int n, int b)
{
    if (n <= 0 || (b != 16 && b != 32 && b != 64)) return 0;
    return mm_form_workspace_bytes(n, b);
}

size_t ph_fp64_split_workspace_bytes(int n, int b)
{
    if (n <= 0 || (b != 16 && b != 32 && b != 64)) return 0;
    const size_t nb = (size_t)(n + b - 1) / b;
    const size_t slabs = max_slabs(n, b);
    const size_t z = slabs == 0 ? 0 : slabs * b * b * sizeof(double) + 256;
    return z + nb * b * sizeof(short) + 256 + nb * sizeof(int) + 256;
}

signtri_status ph_fp64_split_run(int n, const double *T, int ldt, double *U, int ldu, int b, Arena &ws,
                                 cudaStream_t st)
{
    switch (b) {
    case 16: return run_b<16>(n, T, ldt, U, ldu, true, ws, st);
    case 32: return run_b<32>(n, T, ldt, U, ldu, true, ws, st);
    case 64: return run_b<64>(n, T, ldt, U, ldu, true, ws, st);
    default: return SIGNTRI_ERR_BAD_ARG;
    }
}

signtri_status ph_fp64_run(int n, const double *T, int ldt, double *U, int ldu, int b, Arena &ws,
                           cudaStream_t st)
{
    switch (b) {
    case 16: return run_b<16>(n, T, ldt, U, ldu, false, ws, st);
    case 32: return run_b<32>(n, T, ldt, U, ldu, false, ws, st);
    case 64: return run_b<64>(n, T, ldt, U, ldu, false, ws, st);
    default: return SIGNTRI_ERR_BAD_ARG;
    }
}

}  // namespace signtri

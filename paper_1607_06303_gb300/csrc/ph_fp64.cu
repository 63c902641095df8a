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
//   1. ph_gemm_kernel: X_IJ and Y_IJ over K = I+1 .. J-1 (split along K into
//      at most kSplitMax partial slabs, summed in a fixed order later; no
//      atomics, so results are run-to-run deterministic);
//   2. offdiag_leaf_kernel: the in-block element recurrence seeded with
//      X_IJ, Y_IJ (Algorithm 6, 1x1 case, applied inside the b x b block).
// The diagonal blocks are all independent (Algorithm 5 calls on disjoint
// diagonal blocks) and are computed first by diag_leaf_kernel (Algorithm 3
// on each block).
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

template <int B>
__global__ void __launch_bounds__(kThreads)
ph_gemm_kernel(int n, const double *__restrict__ T, int ldt, const double *__restrict__ U, int ldu,
               int d, int kc, double *__restrict__ PX, double *__restrict__ PY, size_t split_stride)
{
    const int I = blockIdx.x, s = blockIdx.y, J = I + d;
    const int kb0 = I + 1 + s * kc;
    const int kb1 = min(kb0 + kc, J);
    ph_gemm_body<B>(n, T, ldt, U, ldu, I, J, kb0, kb1, PX + (size_t)s * split_stride + (size_t)I * B * B,
                    PY + (size_t)s * split_stride + (size_t)I * B * B);
}

template <int B>
__global__ void __launch_bounds__(kThreads)
offdiag_leaf_kernel(int n, const double *__restrict__ T, int ldt, double *__restrict__ U, int ldu,
                    int d, int nsplit, const double *__restrict__ PX, const double *__restrict__ PY,
                    size_t split_stride)
{
    const int I = blockIdx.x;
    offdiag_leaf_body<B>(n, T, ldt, U, ldu, I, I + d, nsplit, PX + (size_t)I * B * B, PY + (size_t)I * B * B,
                         split_stride);
}


template <int B>
__global__ void __launch_bounds__(kThreads)
ph_gemm_split_kernel(int n, const double *__restrict__ T, int ldt, const double *__restrict__ U, int ldu, int d,
                     int kc, const short *__restrict__ perm, const int *__restrict__ npos, double *__restrict__ PZ,
                     size_t split_stride)
{
    const int I = blockIdx.x, s = blockIdx.y, J = I + d;
    const int kb0 = I + 1 + s * kc;
    const int kb1 = min(kb0 + kc, J);
    ph_gemm_split_body<B>(n, T, ldt, U, ldu, I, J, kb0, kb1, perm, npos,
                          PZ + (size_t)s * split_stride + (size_t)I * B * B);
}

template <int B>
__global__ void sign_perm_kernel(int n, const double *__restrict__ T, int ldt, short *__restrict__ perm,
                                 int *__restrict__ npos)
{
    sign_perm_body<B>(n, T, ldt, blockIdx.x, perm, npos);
}

// Arithmetic-efficient form: one sum per entry (X or Y by the sign pair).
template <int B>
signtri_status run_b_split(int n, const double *T, int ldt, double *U, int ldu, Arena &ws, cudaStream_t st)
{
    const int nb = (n + B - 1) / B;
    const size_t split_stride = (size_t)nb * B * B;
    double *PZ = nullptr;
    if (nb > 2) {
        PZ = static_cast<double *>(ws.take(split_stride * kSplitMax * sizeof(double)));
        if (!PZ) return SIGNTRI_ERR_NO_WORKSPACE;
    }
    short *perm = static_cast<short *>(ws.take((size_t)nb * B * sizeof(short)));
    int *npos = static_cast<int *>(ws.take((size_t)nb * sizeof(int)));
    if (!perm || !npos) return SIGNTRI_ERR_NO_WORKSPACE;
    SGT_CUDA_TRY(cudaFuncSetAttribute(offdiag_leaf_kernel<B>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                      (int)leaf_smem<B>()));
    SGT_CUDA_TRY(cudaFuncSetAttribute(diag_leaf_kernel<B>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                      (int)diag_smem<B>()));
    signtri_status rs = launch_zero_strict_lower(n, U, ldu, st);
    if (rs != SIGNTRI_OK) return rs;
    {
        ProfScope ps(SIGNTRI_KC_DIAG_LEAF, st);
        sign_perm_kernel<B><<<nb, B, 0, st>>>(n, T, ldt, perm, npos);
        SGT_LAUNCH_CHECK();
        diag_leaf_kernel<B><<<nb, kThreads, diag_smem<B>(), st>>>(n, T, ldt, U, ldu);
        SGT_LAUNCH_CHECK();
    }
    for (int d = 1; d < nb; d++) {
        const int ntiles = nb - d;
        const int kmax = d - 1;
        int nsplit = 0;
        if (kmax > 0) {
            int want = (kTargetCtas + ntiles - 1) / ntiles;
            nsplit = std::max(1, std::min(want, std::min(kSplitMax, kmax)));
            const int kc = (kmax + nsplit - 1) / nsplit;
            nsplit = (kmax + kc - 1) / kc;
            ProfScope ps(SIGNTRI_KC_BLOCK_SUMS_F64, st);
            ph_gemm_split_kernel<B><<<dim3(ntiles, nsplit), kThreads, 0, st>>>(n, T, ldt, U, ldu, d, kc, perm, npos,
                                                                              PZ, split_stride);
            SGT_LAUNCH_CHECK();
        }
        {
            ProfScope ps(SIGNTRI_KC_OFFDIAG_LEAF, st);
            offdiag_leaf_kernel<B><<<ntiles, kThreads, leaf_smem<B>(), st>>>(n, T, ldt, U, ldu, d, nsplit, PZ, PZ,
                                                                             split_stride);
            SGT_LAUNCH_CHECK();
        }
    }
    return SIGNTRI_OK;
}

template <int B>
signtri_status run_b(int n, const double *T, int ldt, double *U, int ldu, Arena &ws, cudaStream_t st)
{
    const int nb = (n + B - 1) / B;
    const size_t split_stride = (size_t)nb * B * B;
    double *PX = nullptr, *PY = nullptr;
    if (nb > 2) {
        PX = static_cast<double *>(ws.take(split_stride * kSplitMax * sizeof(double)));
        PY = static_cast<double *>(ws.take(split_stride * kSplitMax * sizeof(double)));
        if (!PX || !PY) return SIGNTRI_ERR_NO_WORKSPACE;
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
        diag_leaf_kernel<B><<<nb, kThreads, diag_smem<B>(), st>>>(n, T, ldt, U, ldu);
        SGT_LAUNCH_CHECK();
    }
    for (int d = 1; d < nb; d++) {
        const int ntiles = nb - d;
        const int kmax = d - 1;
        int nsplit = 0;
        if (kmax > 0) {
            int want = (kTargetCtas + ntiles - 1) / ntiles;
            nsplit = std::max(1, std::min(want, std::min(kSplitMax, kmax)));
            const int kc = (kmax + nsplit - 1) / nsplit;
            nsplit = (kmax + kc - 1) / kc;
            ProfScope ps(SIGNTRI_KC_BLOCK_SUMS_F64, st);
            ph_gemm_kernel<B><<<dim3(ntiles, nsplit), kThreads, 0, st>>>(n, T, ldt, U, ldu, d, kc, PX, PY,
                                                                        split_stride);
            SGT_LAUNCH_CHECK();
        }
        {
            ProfScope ps(SIGNTRI_KC_OFFDIAG_LEAF, st);
            offdiag_leaf_kernel<B><<<ntiles, kThreads, leaf_smem<B>(), st>>>(n, T, ldt, U, ldu, d, nsplit,
                                                                             PX, PY, split_stride);
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
    if (n <= 0 || b <= 0) return 0;
    const size_t nb = (size_t)(n + b - 1) / b;
    if (nb <= 2) return 0;
    return 2 * (nb * b * b * kSplitMax * sizeof(double) + 256);
}

size_t ph_fp64_split_workspace_bytes(int n, int b)
{
    if (n <= 0 || b <= 0) return 0;
    const size_t nb = (size_t)(n + b - 1) / b;
    size_t z = (nb <= 2) ? 0 : nb * b * b * kSplitMax * sizeof(double) + 256;
    return z + nb * b * sizeof(short) + 256 + nb * sizeof(int) + 256;
}

signtri_status ph_fp64_split_run(int n, const double *T, int ldt, double *U, int ldu, int b, Arena &ws,
                                 cudaStream_t st)
{
    switch (b) {
    case 16: return run_b_split<16>(n, T, ldt, U, ldu, ws, st);
    case 32: return run_b_split<32>(n, T, ldt, U, ldu, ws, st);
    case 64: return run_b_split<64>(n, T, ldt, U, ldu, ws, st);
    default: return SIGNTRI_ERR_BAD_ARG;
    }
}

signtri_status ph_fp64_run(int n, const double *T, int ldt, double *U, int ldu, int b, Arena &ws,
                           cudaStream_t st)
{
    switch (b) {
    case 16: return run_b<16>(n, T, ldt, U, ldu, ws, st);
    case 32: return run_b<32>(n, T, ldt, U, ldu, ws, st);
    case 64: return run_b<64>(n, T, ldt, U, ldu, ws, st);
    default: return SIGNTRI_ERR_BAD_ARG;
    }
}

}  // namespace signtri

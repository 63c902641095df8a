// funm.cu -- F = phi(T) for a general function phi (Section 2: Parlett's
// substitution, Algorithm 1, and its block form, Algorithm 2).
//
// Every matrix function commutes with its argument, so entry (i, j) of
// TF = FT gives, for t_ii != t_jj,
//     (t_ii - t_jj) f_ij = t_ij (f_ii - f_jj) + sum_{i<k<j} (f_ik t_kj - t_ik f_kj),
// with f_ii = phi(t_ii).  Blocked with the b x b partition of the float64
// Parlett-Higham path: the off-diagonal block F_IJ solves the Sylvester
// equation T_II F_IJ - F_IJ T_JJ = F_II T_IJ - T_IJ F_JJ + X_IJ of Algorithm 2,
// X_IJ = sum_{I<K<J} (F_IK T_KJ - T_IK F_KJ) from the same block-sum kernels,
// the equation itself by the element recurrence inside the block (T_II and
// T_JJ are triangular); the diagonal blocks by Algorithm 1.  Unlike the sign
// function (where Algorithm 3 takes U^2 = I for equal signs) every entry
// divides by t_ii - t_jj: the diagonal must be distinct, and close
// eigenvalues amplify rounding, as the paper notes.  Float64 throughout.
#include <algorithm>
#include <cmath>
#include <vector>

#include "internal.cuh"
#include "ph_bodies.cuh"

namespace signtri {

using namespace ph;

namespace {

__device__ __forceinline__ double phi_of(int phi, double x)
{
    switch (phi) {
    case SIGNTRI_PHI_EXP: return exp(x);
    case SIGNTRI_PHI_LOG: return log(x);
    case SIGNTRI_PHI_SQRT: return sqrt(x);
    default: return x > 0.0 ? 1.0 : -1.0;
    }
}

// Algorithm 1 on one diagonal block, by anti-diagonal inside the block.
template <int B>
__global__ void __launch_bounds__(kThreads)
funm_diag_leaf_kernel(int n, const double *__restrict__ T, int ldt, double *__restrict__ F, int ldf, int phi)
{
    constexpr int LD = B + 1;
    extern __shared__ double sm[];
    double *Ts = sm;
    double *Fs = sm + B * LD;
    const int r0 = blockIdx.x * B;
    const int bs = min(B, n - r0);
    for (int idx = threadIdx.x; idx < bs * bs; idx += kThreads) {
        const int i = idx % bs, j = idx / bs;
        const double t = (i <= j) ? SGT_AT(T, ldt, r0 + i, r0 + j) : 0.0;
        Ts[i + j * LD] = t;
        Fs[i + j * LD] = (i == j) ? phi_of(phi, t) : 0.0;
    }
    __syncthreads();
    for (int d = 1; d < bs; d++) {
        for (int i = threadIdx.x; i < bs - d; i += kThreads) {
            const int j = i + d;
            double s = 0.0;
            for (int k = i + 1; k < j; k++) s = fma(Fs[i + k * LD], Ts[k + j * LD], fma(-Ts[i + k * LD], Fs[k + j * LD], s));
            Fs[i + j * LD] = (Ts[i + j * LD] * (Fs[i + i * LD] - Fs[j + j * LD]) + s) / (Ts[i + i * LD] - Ts[j + j * LD]);
        }
        __syncthreads();
    }
    for (int idx = threadIdx.x; idx < bs * bs; idx += kThreads) {
        const int i = idx % bs, j = idx / bs;
        if (i <= j) SGT_AT(F, ldf, r0 + i, r0 + j) = Fs[i + j * LD];
    }
}

template <int B>
__global__ void __launch_bounds__(kThreads)
funm_gemm_kernel(int n, const double *__restrict__ T, int ldt, const double *__restrict__ F, int ldf, int d,
                 long long W, double *__restrict__ PX, double *__restrict__ PY)
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
        ph_gemm_body<B>(n, T, ldt, F, ldf, I, I + d, (I + 1) * B + (int)(x - t0) * 16,
                        (I + 1) * B + (int)(xe - t0) * 16, PX + slab, PY + slab);
        x = xe;
    }
}

template <int B>
__global__ void __launch_bounds__(kThreads)
funm_offdiag_leaf_kernel(int n, const double *__restrict__ T, int ldt, double *__restrict__ F, int ldf, int d,
                         long long W, const double *__restrict__ PX, const double *__restrict__ PY)
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
    offdiag_leaf_body<B>(n, T, ldt, F, ldf, I, I + d, count, PX + base, PY + base, (size_t)B * B, true);
}

template <int B>
signtri_status funm_b(int n, const double *T, int ldt, double *F, int ldf, int phi, Arena &ws, cudaStream_t st)
{
    const int nb = (n + B - 1) / B;
    const size_t slabs = max_slabs(n, B);
    double *PX = nullptr, *PY = nullptr;
    if (slabs > 0) {
        PX = static_cast<double *>(ws.take(slabs * B * B * sizeof(double)));
        PY = static_cast<double *>(ws.take(slabs * B * B * sizeof(double)));   // written, not read
        if (!PX || !PY) return SIGNTRI_ERR_NO_WORKSPACE;
    }
    SGT_CUDA_TRY(cudaFuncSetAttribute(funm_offdiag_leaf_kernel<B>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                      (int)leaf_smem<B>()));
    SGT_CUDA_TRY(cudaFuncSetAttribute(funm_diag_leaf_kernel<B>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                      (int)diag_smem<B>()));
    signtri_status rs = launch_zero_strict_lower(n, F, ldf, st);
    if (rs != SIGNTRI_OK) return rs;
    {
        ProfScope ps(SIGNTRI_KC_DIAG_LEAF, st);
        funm_diag_leaf_kernel<B><<<nb, kThreads, diag_smem<B>(), st>>>(n, T, ldt, F, ldf, phi);
        SGT_LAUNCH_CHECK();
    }
    for (int d = 1; d < nb; d++) {
        const int ntiles = nb - d;
        const long long W = (long long)ntiles * sk_chunks_per_tile(d, B);
        if (W > 0) {
            ProfScope ps(SIGNTRI_KC_BLOCK_SUMS_F64, st);
            funm_gemm_kernel<B><<<sk_ctas(W), kThreads, 0, st>>>(n, T, ldt, F, ldf, d, W, PX, PY);
            SGT_LAUNCH_CHECK();
        }
        ProfScope ps(SIGNTRI_KC_OFFDIAG_LEAF, st);
        funm_offdiag_leaf_kernel<B><<<ntiles, kThreads, leaf_smem<B>(), st>>>(n, T, ldt, F, ldf, d, W, PX, PY);
        SGT_LAUNCH_CHECK();
    }
    return SIGNTRI_OK;
}

}  // namespace

size_t funm_workspace_bytes(int n, int b)
{
    return ph_fp64_workspace_bytes(n, b);
}

// The diagonal is checked on the host first (it decides whether the
// recurrence is defined): the first index whose value is outside phi's
// domain (log, sqrt: t_ii > 0) or not finite, or that repeats an earlier
// diagonal value, gives SIGNTRI_ERR_DOMAIN with that index.
signtri_status funm_run(int n, const double *T, int ldt, double *F, int ldf, int phi, int b, Arena &ws,
                        int *bad_index, cudaStream_t st)
{
    if (n <= 0) return SIGNTRI_OK;
    std::vector<double> diag(n);
    SGT_CUDA_TRY(cudaMemcpy2DAsync(diag.data(), sizeof(double), T, ((size_t)ldt + 1) * sizeof(double), sizeof(double),
                                   n, cudaMemcpyDeviceToHost, st));
    SGT_CUDA_TRY(cudaStreamSynchronize(st));
    std::vector<std::pair<double, int>> sorted(n);
    int bad = n;
    for (int i = 0; i < n; i++) {
        const double t = diag[i];
        if (!std::isfinite(t) || ((phi == SIGNTRI_PHI_LOG || phi == SIGNTRI_PHI_SQRT) && !(t > 0.0)) ||
            (phi == SIGNTRI_PHI_SIGN && t == 0.0))
            bad = std::min(bad, i);
        sorted[i] = {t, i};
    }
    std::sort(sorted.begin(), sorted.end());
    for (int k = 1; k < n; k++)
        if (sorted[k].first == sorted[k - 1].first) bad = std::min(bad, std::max(sorted[k].second, sorted[k - 1].second));
    if (bad < n) {
        if (bad_index) *bad_index = bad;
        return SIGNTRI_ERR_DOMAIN;
    }
    switch (b) {
    case 16: return funm_b<16>(n, T, ldt, F, ldf, phi, ws, st);
    case 32: return funm_b<32>(n, T, ldt, F, ldf, phi, ws, st);
    case 64: return funm_b<64>(n, T, ldt, F, ldf, phi, ws, st);
    default: return SIGNTRI_ERR_BAD_ARG;
    }
}

}  // namespace signtri

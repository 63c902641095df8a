// complex.cu -- sign(T) of a complex upper triangular T, and the complex
// Schur route S = Q sign(T) Q^H (Section 1; Algorithm 3's first step takes a
// complex Schur form A = Q T Q^*).
//
// u_ii = sign(Re t_ii) (the sign function is defined off the imaginary axis,
// Section 1); for i < j, entry (i, j) of TU = UT (Eq. 1) or of U^2 = I
// (Eq. 2), exactly as for real T:
//   signs differ: u_ij = t_ij (u_ii - u_jj) / (t_ii - t_jj)
//                        + [sum_{i<k<j} (u_ik t_kj - t_ik u_kj)] / (t_ii - t_jj)
//   signs agree:  u_ij = -[sum_{i<k<j} u_ik u_kj] / (u_ii + u_jj)
// in complex float64 arithmetic.  Entries are computed by anti-diagonal
// d = j - i (each depends on smaller d only), one launch per anti-diagonal,
// one warp per entry: the lanes split the terms of the sum and reduce by
// shuffles.  Row i of U and of T is read from row-major copies (UR, TR, the
// entry's writer storing u_ij in both layouts), so every sum reads
// contiguous runs.  This path runs at the float64 rate of the SMs; it is the
// general-spectrum building block, not a tuned hot path.
//
// The route's products W = U Q^H and S = Q W are complex: each is four real
// emulated-float64 tensor-core products of the real and imaginary planes
// (slices.cu), combined by small kernels.
//
// Layout: complex matrices are interleaved (re, im) float64 pairs,
// column-major, leading dimensions counted in complex elements (LAPACK's
// COMPLEX*16).
#include <algorithm>
#include <climits>

#include "internal.cuh"

namespace signtri {

namespace {

constexpr int kThreads = 256;

__device__ __forceinline__ double2 cadd(double2 a, double2 b) { return make_double2(a.x + b.x, a.y + b.y); }
__device__ __forceinline__ double2 csub(double2 a, double2 b) { return make_double2(a.x - b.x, a.y - b.y); }
__device__ __forceinline__ double2 cmul(double2 a, double2 b)
{
    return make_double2(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}
// a / b by Smith's algorithm (R. L. Smith, CACM 5(8), 1962): scale by the
// larger of |Re b|, |Im b| so that no intermediate overflows needlessly
__device__ __forceinline__ double2 cdiv(double2 a, double2 b)
{
    if (fabs(b.x) >= fabs(b.y)) {
        const double r = b.y / b.x, den = b.x + b.y * r;
        return make_double2((a.x + a.y * r) / den, (a.y - a.x * r) / den);
    }
    const double r = b.x / b.y, den = b.x * r + b.y;
    return make_double2((a.x * r + a.y) / den, (a.y * r - a.x) / den);
}

// Diagonal check (first bad index: 4 i + status, as the real scan) and
// signs; U zeroed with its diagonal set; TR = rows of T's upper triangle.
__global__ void complex_init_kernel(int n, const double2 *__restrict__ T, int ldt, double2 *__restrict__ U, int ldu,
                                    double2 *__restrict__ UR, double2 *__restrict__ TR, signed char *__restrict__ sg,
                                    int *__restrict__ bad)
{
    const int j = blockIdx.x;
    const double2 tjj = T[(size_t)j + (size_t)j * ldt];
    const double s = tjj.x > 0.0 ? 1.0 : -1.0;
    if (threadIdx.x == 0) {
        int key = INT_MAX;
        if (!isfinite(tjj.x) || !isfinite(tjj.y)) key = 4 * j + SIGNTRI_ERR_NONFINITE;
        else if (tjj.x == 0.0) key = 4 * j + SIGNTRI_ERR_ZERO_EIGENVALUE;
        if (key != INT_MAX) atomicMin(bad, key);
        sg[j] = (signed char)s;
    }
    for (int i = threadIdx.x; i < n; i += blockDim.x) {
        const double2 v = make_double2(i == j ? s : 0.0, 0.0);
        U[(size_t)i + (size_t)j * ldu] = v;
        UR[(size_t)j * n + i] = (i == j) ? v : make_double2(0.0, 0.0);   // UR row j
        TR[(size_t)j * n + i] = (i >= j) ? T[(size_t)j + (size_t)i * ldt] : make_double2(0.0, 0.0);
    }
}

// Anti-diagonal d: entries (i, i + d), i < n - d, one warp each.
__global__ void __launch_bounds__(kThreads)
complex_antidiag_kernel(int n, int d, const double2 *__restrict__ T, int ldt, const double2 *__restrict__ TR,
                        double2 *__restrict__ U, int ldu, double2 *__restrict__ UR, const signed char *__restrict__ sg)
{
    const int i = (int)((blockIdx.x * (size_t)blockDim.x + threadIdx.x) / 32), lane = threadIdx.x & 31;
    if (i >= n - d) return;
    const int j = i + d;
    const bool opp = sg[i] != sg[j];
    const double2 *urow = UR + (size_t)i * n, *trow = TR + (size_t)i * n;
    const double2 *ucol = U + (size_t)j * ldu, *tcol = T + (size_t)j * ldt;
    double2 s = make_double2(0.0, 0.0);
    if (opp) {
        for (int k = i + 1 + lane; k < j; k += 32) s = cadd(s, csub(cmul(urow[k], tcol[k]), cmul(trow[k], ucol[k])));
    } else {
        for (int k = i + 1 + lane; k < j; k += 32) s = cadd(s, cmul(urow[k], ucol[k]));
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        s.x += __shfl_xor_sync(0xffffffffu, s.x, o);
        s.y += __shfl_xor_sync(0xffffffffu, s.y, o);
    }
    if (lane != 0) return;
    const double uii = sg[i], ujj = sg[j];
    double2 v;
    if (opp) {
        const double2 den = csub(trow[i], tcol[j]);
        const double2 tij = tcol[i];
        v = cadd(cdiv(make_double2(tij.x * (uii - ujj), tij.y * (uii - ujj)), den), cdiv(s, den));
    } else {
        v = make_double2(-s.x / (uii + ujj), -s.y / (uii + ujj));
    }
    U[(size_t)i + (size_t)j * ldu] = v;
    UR[(size_t)i * n + j] = v;
}

// Real and imaginary planes of an n x n complex matrix (ld in complex
// elements); conj = 1 stores -Im.
__global__ void split_planes_kernel(int n, const double2 *__restrict__ M, int ldm, double *__restrict__ re,
                                    double *__restrict__ im)
{
    const int j = blockIdx.x;
    for (int i = threadIdx.x; i < n; i += blockDim.x) {
        const double2 v = M[(size_t)i + (size_t)j * ldm];
        re[(size_t)i + (size_t)j * n] = v.x;
        im[(size_t)i + (size_t)j * n] = v.y;
    }
}

// out = a + sa * b (n x n planes, ld n)
__global__ void combine_kernel(int n, const double *__restrict__ a, const double *__restrict__ b, double sa,
                               double *__restrict__ out)
{
    const size_t idx = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (idx < (size_t)n * n) out[idx] = a[idx] + sa * b[idx];
}

// S = re + i im, interleaved, ld in complex elements
__global__ void join_planes_kernel(int n, const double *__restrict__ re, const double *__restrict__ im,
                                   double2 *__restrict__ S, int lds)
{
    const int j = blockIdx.x;
    for (int i = threadIdx.x; i < n; i += blockDim.x)
        S[(size_t)i + (size_t)j * lds] = make_double2(re[(size_t)i + (size_t)j * n], im[(size_t)i + (size_t)j * n]);
}

}  // namespace

size_t complex_workspace_bytes(int n)
{
    if (n <= 0) return 0;
    const size_t nn = (size_t)n * n;
    return 2 * nn * sizeof(double2) + (size_t)n + sizeof(int) + 4 * 256;
}

signtri_status complex_sign_run(int n, const double *T, int ldt, double *U, int ldu, Arena &ws, int *bad_index,
                                cudaStream_t st)
{
    if (n <= 0) return SIGNTRI_OK;
    const size_t nn = (size_t)n * n;
    auto *UR = static_cast<double2 *>(ws.take(nn * sizeof(double2)));
    auto *TR = static_cast<double2 *>(ws.take(nn * sizeof(double2)));
    auto *sg = static_cast<signed char *>(ws.take((size_t)n));
    auto *bad = static_cast<int *>(ws.take(sizeof(int)));
    if (!UR || !TR || !sg || !bad) return SIGNTRI_ERR_NO_WORKSPACE;
    const auto *Tc = reinterpret_cast<const double2 *>(T);
    auto *Uc = reinterpret_cast<double2 *>(U);
    const int big = INT_MAX;
    SGT_CUDA_TRY(cudaMemcpyAsync(bad, &big, sizeof(int), cudaMemcpyHostToDevice, st));
    {
        ProfScope ps(SIGNTRI_KC_SCAN, st);
        complex_init_kernel<<<n, kThreads, 0, st>>>(n, Tc, ldt, Uc, ldu, UR, TR, sg, bad);
        SGT_LAUNCH_CHECK();
    }
    int key = INT_MAX;
    SGT_CUDA_TRY(cudaMemcpyAsync(&key, bad, sizeof(int), cudaMemcpyDeviceToHost, st));
    SGT_CUDA_TRY(cudaStreamSynchronize(st));
    if (key != INT_MAX) {
        if (bad_index) *bad_index = key / 4;
        return (signtri_status)(key % 4);
    }
    for (int d = 1; d < n; d++) {
        const int entries = n - d;
        const unsigned blocks = (unsigned)(((size_t)entries * 32 + kThreads - 1) / kThreads);
        ProfScope ps(SIGNTRI_KC_OFFDIAG_LEAF, st);
        complex_antidiag_kernel<<<blocks, kThreads, 0, st>>>(n, d, Tc, ldt, TR, Uc, ldu, UR, sg);
        SGT_LAUNCH_CHECK();
    }
    return SIGNTRI_OK;
}

size_t complex_schur_workspace_bytes(int n)
{
    if (n <= 0) return 0;
    const size_t nn = (size_t)n * n * sizeof(double) + 256;
    return std::max(complex_workspace_bytes(n), 8 * nn + emulated_product_workspace_bytes(n, n, n));
}

signtri_status complex_schur_run(int n, const double *Q, int ldq, const double *T, int ldt, double *S, int lds,
                                 Arena &ws, int *d_err, int *bad_index, cudaStream_t st)
{
    if (n <= 0) return SIGNTRI_OK;
    // U = sign(T) into S (complex, ld lds), then the products by planes
    const size_t mark0 = ws.used;
    signtri_status rs = complex_sign_run(n, T, ldt, S, lds, ws, bad_index, st);
    if (rs != SIGNTRI_OK) return rs;
    ws.used = mark0;
    const size_t nn = (size_t)n * n;
    double *P[8];
    for (double *&p : P) {
        p = static_cast<double *>(ws.take(nn * sizeof(double)));
        if (!p) return SIGNTRI_ERR_NO_WORKSPACE;
    }
    double *Qr = P[0], *Qi = P[1], *Ur = P[2], *Ui = P[3], *Wr = P[4], *Wi = P[5], *X1 = P[6], *X2 = P[7];
    const size_t mark = ws.used;
    const unsigned cblocks = (unsigned)((nn + kThreads - 1) / kThreads);
    {
        ProfScope ps(SIGNTRI_KC_FILL, st);
        split_planes_kernel<<<n, kThreads, 0, st>>>(n, reinterpret_cast<const double2 *>(Q), ldq, Qr, Qi);
        SGT_LAUNCH_CHECK();
        split_planes_kernel<<<n, kThreads, 0, st>>>(n, reinterpret_cast<const double2 *>(S), lds, Ur, Ui);
        SGT_LAUNCH_CHECK();
    }
    auto prod = [&](const double *A, const double *B, bool transB, double *C) -> signtri_status {
        ws.used = mark;
        return emulated_product(n, n, n, A, n, B, n, transB, C, n, false, SIGNTRI_KC_GEMM_F64, ws, d_err, st);
    };
    auto comb = [&](const double *a, const double *b, double sa, double *out) -> signtri_status {
        ProfScope ps(SIGNTRI_KC_FILL, st);
        combine_kernel<<<cblocks, kThreads, 0, st>>>(n, a, b, sa, out);
        SGT_LAUNCH_CHECK();
        return SIGNTRI_OK;
    };
    // W = U Q^H: Wr = Ur Qr^T + Ui Qi^T, Wi = Ui Qr^T - Ur Qi^T
    if ((rs = prod(Ur, Qr, true, X1)) != SIGNTRI_OK) return rs;
    if ((rs = prod(Ui, Qi, true, X2)) != SIGNTRI_OK) return rs;
    if ((rs = comb(X1, X2, 1.0, Wr)) != SIGNTRI_OK) return rs;
    if ((rs = prod(Ui, Qr, true, X1)) != SIGNTRI_OK) return rs;
    if ((rs = prod(Ur, Qi, true, X2)) != SIGNTRI_OK) return rs;
    if ((rs = comb(X1, X2, -1.0, Wi)) != SIGNTRI_OK) return rs;
    // S = Q W: Sr = Qr Wr - Qi Wi, Si = Qr Wi + Qi Wr (the U planes are free now)
    if ((rs = prod(Qr, Wr, false, X1)) != SIGNTRI_OK) return rs;
    if ((rs = prod(Qi, Wi, false, X2)) != SIGNTRI_OK) return rs;
    if ((rs = comb(X1, X2, -1.0, Ur)) != SIGNTRI_OK) return rs;
    if ((rs = prod(Qr, Wi, false, X1)) != SIGNTRI_OK) return rs;
    if ((rs = prod(Qi, Wr, false, X2)) != SIGNTRI_OK) return rs;
    if ((rs = comb(X1, X2, 1.0, Ui)) != SIGNTRI_OK) return rs;
    {
        ProfScope ps(SIGNTRI_KC_FILL, st);
        join_planes_kernel<<<n, kThreads, 0, st>>>(n, Ur, Ui, reinterpret_cast<double2 *>(S), lds);
        SGT_LAUNCH_CHECK();
    }
    return SIGNTRI_OK;
}

}  // namespace signtri

// gemm_f64.cu -- general float64 GEMM on the FMA pipe, for the
// Parlett-Sylvester back-transform (U = Q U~ Q^T by matrix products).
//
// C[m x n] = alpha * op(A) * op(B) + beta * C, column-major, op = N or T.
// 64 x 64 output tile per CTA, 256 threads, 4 x 4 outputs per thread,
// K staged through shared memory in steps of 16.  `upper` writes only the
// entries i <= j (tiles entirely below the diagonal exit at once).
#include "internal.cuh"

namespace signtri {

namespace {

constexpr int GB = 64;
constexpr int GKT = 16;
constexpr int GThreads = 256;

__global__ void __launch_bounds__(GThreads)
gemm_f64_kernel(int transA, int transB, int m, int n, int k, double alpha, const double *__restrict__ A, int lda,
                const double *__restrict__ B, int ldb, double beta, double *__restrict__ C, int ldc, int upper)
{
    __shared__ double As[GKT][GB + 1];
    __shared__ double Bs[GKT][GB + 1];
    const int r0 = blockIdx.x * GB, c0 = blockIdx.y * GB;
    if (upper && r0 > c0 + GB - 1) return;
    const int tx = threadIdx.x % 16, ty = threadIdx.x / 16;
    double acc[4][4];
#pragma unroll
    for (int a = 0; a < 4; a++)
#pragma unroll
        for (int b = 0; b < 4; b++) acc[a][b] = 0.0;
    for (int k0 = 0; k0 < k; k0 += GKT) {
        for (int idx = threadIdx.x; idx < GB * GKT; idx += GThreads) {
            int r, kk;
            if (!transA) { r = idx % GB; kk = idx / GB; } else { kk = idx % GKT; r = idx / GKT; }
            const int gi = r0 + r, gk = k0 + kk;
            double v = 0.0;
            if (gi < m && gk < k) v = transA ? A[(size_t)gk + (size_t)gi * lda] : A[(size_t)gi + (size_t)gk * lda];
            As[kk][r] = v;
        }
        for (int idx = threadIdx.x; idx < GB * GKT; idx += GThreads) {
            int c, kk;
            if (!transB) { kk = idx % GKT; c = idx / GKT; } else { c = idx % GB; kk = idx / GB; }
            const int gj = c0 + c, gk = k0 + kk;
            double v = 0.0;
            if (gj < n && gk < k) v = transB ? B[(size_t)gj + (size_t)gk * ldb] : B[(size_t)gk + (size_t)gj * ldb];
            Bs[kk][c] = v;
        }
        __syncthreads();
#pragma unroll
        for (int kk = 0; kk < GKT; kk++) {
            double a[4], b[4];
#pragma unroll
            for (int q = 0; q < 4; q++) { a[q] = As[kk][tx + 16 * q]; b[q] = Bs[kk][ty + 16 * q]; }
#pragma unroll
            for (int p = 0; p < 4; p++)
#pragma unroll
                for (int q = 0; q < 4; q++) acc[p][q] = fma(a[p], b[q], acc[p][q]);
        }
        __syncthreads();
    }
#pragma unroll
    for (int p = 0; p < 4; p++)
#pragma unroll
        for (int q = 0; q < 4; q++) {
            const int gi = r0 + tx + 16 * p, gj = c0 + ty + 16 * q;
            if (gi < m && gj < n && (!upper || gi <= gj)) {
                double *c = C + (size_t)gi + (size_t)gj * ldc;
                *c = (beta == 0.0) ? alpha * acc[p][q] : alpha * acc[p][q] + beta * *c;
            }
        }
}

}  // namespace

signtri_status gemm_f64(bool transA, bool transB, int m, int n, int k, double alpha, const double *A, int lda,
                        const double *B, int ldb, double beta, double *C, int ldc, bool upper, cudaStream_t st)
{
    if (m <= 0 || n <= 0) return SIGNTRI_OK;
    dim3 grid((m + GB - 1) / GB, (n + GB - 1) / GB);
    ProfScope ps(SIGNTRI_KC_GEMM_F64, st);
    gemm_f64_kernel<<<grid, GThreads, 0, st>>>(transA ? 1 : 0, transB ? 1 : 0, m, n, k, alpha, A, lda, B, ldb, beta,
                                               C, ldc, upper ? 1 : 0);
    SGT_LAUNCH_CHECK();
    return SIGNTRI_OK;
}

}  // namespace signtri

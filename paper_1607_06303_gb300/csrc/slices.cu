// slices.cu -- bf16 slice representations of float64 matrices for the
// tensor-core block products (tc_gemm.cu), and the emulated-float64 GEMM.
//
// Two kinds of slices:
//  * exact integer slices (error-free split in the style of Ozaki, Ogita,
//    Oishi and Rump): with a power-of-two scale sigma_i >= max_k |m_ik| per row
//    (or per column), r = m_ik / sigma_i in (-1, 1) is cut into S pieces of
//    b = 7 or 8 bits, q_s = trunc(2^b r_s), r_{s+1} = 2^b r_s - q_s, so that
//    m_ik = sigma_i sum_s q_s 2^{-b(s+1)} + O(sigma_i 2^{-bS}); every q_s is an
//    integer of magnitude below 2^b, exact in bf16 (8 significant bits), and
//    a sum of 2^(24-2b) products q_a q_b (1024 for b = 7, 256 for b = 8) stays
//    below 2^24, exact in fp32;
//  * rounding splits: x_0 = bf16(m), x_1 = bf16(m - x_0), x_2 = bf16(m - x_0 - x_1)
//    (unit scale), for products accurate to ~2^-8S.
// Slices are stored K-contiguous: "row" slices R[s][i][k] of an m x k matrix
// (the A operand) and "column" slices C[s][j][k] of a k x n matrix (the B
// operand), rows padded to a multiple of 64 and K to the pitch, with zeros.
#include <algorithm>
#include <cstring>
#include <vector>

#include <cuda_bf16.h>

#include "df_arith.cuh"
#include "exact_slices.cuh"
#include "internal.cuh"
#include "tc_gemm.cuh"

namespace signtri {

namespace {

constexpr int TS = 32;   // transpose tile

// max |m_ik| over the selected part (tri: 1 = strictly upper) of each row
// (rows = true) or column, per 32 x 32 tile with a shared-memory reduction,
// then atomicMax on the float64 bit pattern (values are >= 0, so the bit
// patterns order like the values).
__global__ void absmax_kernel(int m, int k, const double *__restrict__ M, int ldm, int tri, bool rows,
                              unsigned long long *__restrict__ out)
{
    __shared__ unsigned long long tile[TS][TS + 1];   // bits of |m_ij|: maxima on the integer pipes
    const int i0 = blockIdx.y * TS, j0 = blockIdx.x * TS;
    if (tri && j0 + TS - 1 <= i0) return;   // wholly on or below the diagonal
    for (int y = threadIdx.y; y < TS; y += blockDim.y) {
        const int i = i0 + threadIdx.x, j = j0 + y;
        unsigned long long v = 0;
        if (i < m && j < k && (tri == 0 || i < j)) v = abs_bits(SGT_AT(M, ldm, i, j));
        tile[threadIdx.x][y] = v;
    }
    __syncthreads();
    if (threadIdx.y == 0) {
        unsigned long long best = 0;
        const int line = threadIdx.x;
        for (int t = 0; t < TS; t++) best = max(best, rows ? tile[line][t] : tile[t][line]);
        const int g = (rows ? i0 : j0) + line;
        if (best > 0 && g < (rows ? m : k)) atomicMax(&out[g], best);
    }
}

// Row and column maxima in one pass (square n x n, tri as above), per
// 64 x 64 tile: coalesced column reads into shared memory, then 64 threads
// reduce the rows and 64 the columns (128 atomics per tile).  With tri = 1
// tiles wholly on or below the diagonal hold nothing and return at once.
__global__ void absmax_both_kernel(int n, const double *__restrict__ M, int ldm, int tri,
                                   unsigned long long *__restrict__ out_rows, unsigned long long *__restrict__ out_cols)
{
    __shared__ unsigned long long tile[64][65];   // [column][row], bits of |m_ij|
    const int i0 = blockIdx.y * 64, j0 = blockIdx.x * 64;
    if (tri && j0 + 63 <= i0) return;
    const int tx = threadIdx.x % 64, ty = threadIdx.x / 64;   // 256 threads
    for (int c = ty; c < 64; c += 4) {
        const int i = i0 + tx, j = j0 + c;
        unsigned long long v = 0;
        if (i < n && j < n && (tri == 0 || i < j)) v = abs_bits(SGT_AT(M, ldm, i, j));
        tile[c][tx] = v;
    }
    __syncthreads();
    if (threadIdx.x < 64) {
        unsigned long long best = 0;
        for (int t = 0; t < 64; t++) best = max(best, tile[t][threadIdx.x]);
        const int g = i0 + threadIdx.x;
        if (best > 0 && g < n) atomicMax(&out_rows[g], best);
    } else if (threadIdx.x < 128) {
        const int c = threadIdx.x - 64;
        unsigned long long best = 0;
        for (int t = 0; t < 64; t++) best = max(best, tile[c][t]);
        const int g = j0 + c;
        if (best > 0 && g < n) atomicMax(&out_cols[g], best);
    }
}

// power-of-two scale 2^e with max < 2^e (frexp exponent); 1 for an all-zero line
__global__ void pow2_scale_kernel(int n, const unsigned long long *__restrict__ maxbits, float *__restrict__ scale)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const unsigned long long mb = maxbits[i];
    const int e = mb ? max(frexp_exp_of_bits(mb), -120) : 0;
    scale[i] = ldexpf(1.0f, e);
}

// Rounding split of the fp32 value of x: x0 = bf16(x), x1 = bf16(x - x0), ...
template <int SC>
__device__ __forceinline__ void round_slices(double x, int S, float *q)
{
    float r = (float)x;
    const int ns = SC ? SC : S;
#pragma unroll
    for (int s = 0; s < ns; s++) {
        const float b = __bfloat162float(__float2bfloat16_rn(r));
        q[s] = b;
        r = __fsub_rn(r, b);
    }
}

// Row slices of an m x k column-major matrix: R[s][i][kk] for i < m_pad,
// kk < k_pad (ldr even).  Tiled transpose through shared memory, tiles of 32
// rows x 64 columns, two adjacent columns per thread (bf16x2 stores).
// tri: 0 = all entries, 1 = strictly upper (i < kk) only.  scale == nullptr:
// rounding split.  skip = 1: tiles left of the even 64-block at or below a
// row's diagonal block are not written (no 2 x 2-block job reads them).
template <int SC>
__global__ void row_slices_kernel(int m, int k, const double *__restrict__ M, int ldm, int tri, int S, int bits,
                                  const float *__restrict__ scale, __nv_bfloat16 *__restrict__ R, int rows_pad,
                                  int ldr, int skip)
{
    __shared__ double tile[2 * TS][TS + 1];   // [column][row]
    const int i0 = blockIdx.y * TS, k0 = blockIdx.x * 2 * TS;
    if (skip && k0 + 2 * TS <= 2 * ((i0 / 64) / 2) * 64) return;
    for (int y = threadIdx.y; y < 2 * TS; y += blockDim.y) {     // y: column offset
        const int kk = k0 + y, i = i0 + threadIdx.x;
        double v = 0.0;
        if (i < m && kk < k && (tri == 0 || i < kk)) v = SGT_AT(M, ldm, i, kk);
        tile[y][threadIdx.x] = v;
    }
    __syncthreads();
    for (int y = threadIdx.y; y < TS; y += blockDim.y) {         // y: row offset
        const int i = i0 + y, kk = k0 + 2 * threadIdx.x;
        if (i >= rows_pad || kk >= ldr) continue;
        float q0[8], q1[8];
        const int e = (scale && i < m) ? ilogbf(scale[i]) : 0;
        if (scale) {
            exact_slices<SC>(tile[2 * threadIdx.x][y], e, S, bits, q0);
            exact_slices<SC>(tile[2 * threadIdx.x + 1][y], e, S, bits, q1);
        } else {
            round_slices<SC>(tile[2 * threadIdx.x][y], S, q0);
            round_slices<SC>(tile[2 * threadIdx.x + 1][y], S, q1);
        }
        #pragma unroll
        for (int s = 0; s < (SC ? SC : S); s++)
            *reinterpret_cast<__nv_bfloat162 *>(&R[((size_t)s * rows_pad + i) * ldr + kk]) =
                __floats2bfloat162_rn(q0[s], q1[s]);
    }
}

// Column slices of a k x n column-major matrix: C[s][j][kk] (same order as
// the source, no transpose), two adjacent kk per thread (ldc even).
// tri: 1 = strictly upper (kk < j) only.  skip = 1: entries past the end of
// the column's even 64-block pair are not written (no 2 x 2-block job reads
// them).
template <int SC>
__global__ void col_slices_kernel(int k, int n, const double *__restrict__ M, int ldm, int tri, int S, int bits,
                                  const float *__restrict__ scale, __nv_bfloat16 *__restrict__ C, int rows_pad,
                                  int ldc, int skip)
{
    const int j = blockIdx.y;
    const int kk = 2 * (blockIdx.x * blockDim.x + threadIdx.x);
    if (kk >= ldc) return;
    if (skip && kk >= (2 * ((j / 64) / 2) + 2) * 64) return;
    double v0 = 0.0, v1 = 0.0;
    if (j < n) {
        if (kk < k && (tri == 0 || kk < j)) v0 = SGT_AT(M, ldm, kk, j);
        if (kk + 1 < k && (tri == 0 || kk + 1 < j)) v1 = SGT_AT(M, ldm, kk + 1, j);
    }
    float q0[8], q1[8];
    if (scale) {
        const int e = j < n ? ilogbf(scale[j]) : 0;
        exact_slices<SC>(v0, e, S, bits, q0);
        exact_slices<SC>(v1, e, S, bits, q1);
    } else {
        round_slices<SC>(v0, S, q0);
        round_slices<SC>(v1, S, q1);
    }
    #pragma unroll
    for (int s = 0; s < (SC ? SC : S); s++)
        *reinterpret_cast<__nv_bfloat162 *>(&C[((size_t)s * rows_pad + j) * ldc + kk]) =
            __floats2bfloat162_rn(q0[s], q1[s]);
}

// Gathered layout (residual products): position g of the gathered index
// space holds original index inv[g] (-1 = zero padding), gmap is the inverse
// (original -> gathered), and superblock sb of `super` consecutive original
// indices occupies gathered positions [sbbase[sb], sbbase[sb + 1]).
// Row slices R[s][g][h] = slice s of M[inv[g], inv[h]] (strictly upper
// part), pitch ldr, under the gathered row scales scale_g.  CTA (64 original
// rows i0.., 64 gathered columns h0..): one coalesced read down each of the
// 64 source columns inv[h], then each row's 64 entries are written to its
// gathered row gmap[i] as whole 128-byte runs.  Column tiles wholly before
// the gathered start of the rows' superblock lie outside every residual
// job's K range and are not written; padding rows are zeroed separately.
template <int SC>
__global__ void row_slices_gathered_kernel(int n, const double *__restrict__ M, int ldm, const int *__restrict__ inv,
                                           const int *__restrict__ gmap, const int *__restrict__ sbbase, int super,
                                           int ng, int S, int bits, const float *__restrict__ scale_g,
                                           __nv_bfloat16 *__restrict__ R, int rows, int ldr)
{
    __shared__ __align__(16) double tile[64][66];   // [row][column]
    const int i0 = blockIdx.x * 64, h0 = blockIdx.y * 64;
    if (h0 + 64 <= sbbase[i0 / super]) return;
    const int tx = threadIdx.x % 64, ty = threadIdx.x / 64;   // 256 threads
    const int i = i0 + tx;
    for (int cc = ty; cc < 64; cc += 4) {
        const int h = h0 + cc;
        const int kk = h < ng ? inv[h] : -1;
        tile[tx][cc] = (kk >= 0 && i < kk && i < n) ? SGT_AT(M, ldm, i, kk) : 0.0;
    }
    __syncthreads();
    const int warp = threadIdx.x / 32, lane = threadIdx.x % 32;
    for (int r = warp; r < 64; r += 8) {
        if (i0 + r >= n) break;
        const int g = gmap[i0 + r];
        const int e = ilogbf(scale_g[g]);
        const double2 v = *reinterpret_cast<const double2 *>(&tile[r][2 * lane]);
        float q0[8], q1[8];
        exact_slices<SC>(v.x, e, S, bits, q0);
        exact_slices<SC>(v.y, e, S, bits, q1);
        #pragma unroll
        for (int s = 0; s < (SC ? SC : S); s++)
            *reinterpret_cast<__nv_bfloat162 *>(&R[((size_t)s * rows + g) * ldr + h0 + 2 * lane]) =
                __floats2bfloat162_rn(q0[s], q1[s]);
    }
}

// Column slices C[s][g][h] = slice s of M[inv[h], inv[g]] (column inv[g]),
// pitch ldc, under the gathered column scales scale_g.  CTA (original column
// j, row superblock sb): the superblock's rows of column j (one contiguous
// read) are sliced into their gathered positions of a shared-memory copy of
// the segment [sbbase[sb], sbbase[sb + 1]) of output row gmap[j], which is
// then written in one pass.  Segments after j's superblock lie outside every
// residual job's K range and are not written.
template <int SC>
__global__ void col_slices_gathered_kernel(int n, const double *__restrict__ M, int ldm, const int *__restrict__ gmap,
                                           const int *__restrict__ sbbase, int super, int segmax, int S, int bits,
                                           const float *__restrict__ scale_g, __nv_bfloat16 *__restrict__ C, int rows,
                                           int ldc)
{
    extern __shared__ __align__(16) unsigned char seg_raw[];
    __nv_bfloat16 *seg = reinterpret_cast<__nv_bfloat16 *>(seg_raw);   // [s][segmax]
    const int j = blockIdx.x, sb = blockIdx.y;
    if (sb > j / super) return;
    const int b0 = sbbase[sb], len = sbbase[sb + 1] - b0;
    for (int idx = threadIdx.x; idx < S * segmax; idx += blockDim.x) seg[idx] = __float2bfloat16_rn(0.f);
    __syncthreads();
    const int g = gmap[j];
    const int e = ilogbf(scale_g[g]);
    const int i1 = min(min(n, (sb + 1) * super), j);   // strictly upper: rows i < j
    for (int i = sb * super + threadIdx.x; i < i1; i += blockDim.x) {
        float q[8];
        exact_slices<SC>(SGT_AT(M, ldm, i, j), e, S, bits, q);
        const int h = gmap[i] - b0;
        #pragma unroll
        for (int s = 0; s < (SC ? SC : S); s++) seg[s * segmax + h] = __float2bfloat16_rn(q[s]);
    }
    __syncthreads();
    // len and b0 are multiples of 64: bf16 pairs
    for (int idx = threadIdx.x; idx < S * (len / 2); idx += blockDim.x) {
        const int s = idx / (len / 2), h = 2 * (idx % (len / 2));
        *reinterpret_cast<__nv_bfloat162 *>(&C[((size_t)s * rows + g) * ldc + b0 + h]) =
            *reinterpret_cast<const __nv_bfloat162 *>(&seg[s * segmax + h]);
    }
}

// Zero rows of R and C that hold no original index (padding inside the
// superblocks and the zero block from ng on), every slice, full pitch.
__global__ void zero_padding_rows_kernel(const int *__restrict__ inv, int ng, int S, __nv_bfloat16 *__restrict__ R,
                                         __nv_bfloat16 *__restrict__ C, int rows, int ld)
{
    const int g = blockIdx.x;
    if (g < ng && inv[g] >= 0) return;
    const __nv_bfloat162 z = __floats2bfloat162_rn(0.f, 0.f);
    for (int s = 0; s < S; s++)
        for (int h = 2 * threadIdx.x; h < ld; h += 2 * blockDim.x) {
            *reinterpret_cast<__nv_bfloat162 *>(&R[((size_t)s * rows + g) * ld + h]) = z;
            *reinterpret_cast<__nv_bfloat162 *>(&C[((size_t)s * rows + g) * ld + h]) = z;
        }
}

// scale_g[g] = scale[inv[g]], 1 for padding
__global__ void gather_scales_kernel(int rows, int ng, const int *__restrict__ inv, const float *__restrict__ scale,
                                     float *__restrict__ scale_g)
{
    const int g = blockIdx.x * blockDim.x + threadIdx.x;
    if (g >= rows) return;
    const int i = g < ng ? inv[g] : -1;
    scale_g[g] = i >= 0 ? scale[i] : 1.0f;
}

// C (m x n) from the top-left / top-right quadrants of the job outputs.
__global__ void gather_gemm_kernel(int m, int n, const double *__restrict__ out, int ntj, double *__restrict__ C,
                                   int ldc)
{
    const int j = blockIdx.x * blockDim.x + threadIdx.x, i = blockIdx.y;
    if (j >= n || i >= m) return;
    const int I = i / 64, J2 = j / 128, jj = j % 128;
    const size_t slot = (size_t)I * ntj + J2;
    const int quad = jj < 64 ? 0 : 1;
    const float2 v = reinterpret_cast<const float2 *>(out)[slot * 16384 + (size_t)quad * 4096 + (i % 64) +
                                                            (size_t)(jj % 64) * 64];
    SGT_AT(C, ldc, i, j) = (double)v.x + (double)v.y;
}

}  // namespace

int pad64(int x) { return (x + 63) / 64 * 64; }

signtri_status make_scales(int m, int k, const double *M, int ldm, int tri, bool rows, int nout,
                           unsigned long long *tmp, float *scale, cudaStream_t st)
{
    SGT_CUDA_TRY(cudaMemsetAsync(tmp, 0, (size_t)nout * sizeof(unsigned long long), st));
    {
        ProfScope ps(SIGNTRI_KC_CONVERT, st);
        dim3 grid((k + TS - 1) / TS, (m + TS - 1) / TS), block(TS, 8);
        absmax_kernel<<<grid, block, 0, st>>>(m, k, M, ldm, tri, rows, tmp);
        SGT_LAUNCH_CHECK();
        pow2_scale_kernel<<<(nout + 255) / 256, 256, 0, st>>>(nout, tmp, scale);
        SGT_LAUNCH_CHECK();
    }
    return SIGNTRI_OK;
}

signtri_status make_scales_both(int n, const double *M, int ldm, int tri, int nout, unsigned long long *tmp_rows,
                                unsigned long long *tmp_cols, float *scale_rows, float *scale_cols, cudaStream_t st)
{
    SGT_CUDA_TRY(cudaMemsetAsync(tmp_rows, 0, (size_t)nout * sizeof(unsigned long long), st));
    SGT_CUDA_TRY(cudaMemsetAsync(tmp_cols, 0, (size_t)nout * sizeof(unsigned long long), st));
    ProfScope ps(SIGNTRI_KC_CONVERT, st);
    absmax_both_kernel<<<dim3((n + 63) / 64, (n + 63) / 64), 256, 0, st>>>(n, M, ldm, tri, tmp_rows, tmp_cols);
    SGT_LAUNCH_CHECK();
    pow2_scale_kernel<<<(nout + 255) / 256, 256, 0, st>>>(nout, tmp_rows, scale_rows);
    SGT_LAUNCH_CHECK();
    pow2_scale_kernel<<<(nout + 255) / 256, 256, 0, st>>>(nout, tmp_cols, scale_cols);
    SGT_LAUNCH_CHECK();
    return SIGNTRI_OK;
}

signtri_status make_row_slices(int m, int k, const double *M, int ldm, int tri, int S, int bits, const float *scale,
                               __nv_bfloat16 *R, int rows_pad, int ldr, cudaStream_t st, int skip)
{
    if (S > 8 || S * bits > 64) return SIGNTRI_ERR_BAD_ARG;
    if (ldr & 1) return SIGNTRI_ERR_BAD_ARG;
    dim3 grid((ldr + 2 * TS - 1) / (2 * TS), (rows_pad + TS - 1) / TS), block(TS, 8);
    ProfScope ps(SIGNTRI_KC_CONVERT, st);
    // compile-time slice counts for the exact residual slices (7) and the sweeps' splits (3)
    if (S == 7) row_slices_kernel<7><<<grid, block, 0, st>>>(m, k, M, ldm, tri, S, bits, scale, R, rows_pad, ldr, skip);
    else if (S == 3)
        row_slices_kernel<3><<<grid, block, 0, st>>>(m, k, M, ldm, tri, S, bits, scale, R, rows_pad, ldr, skip);
    else row_slices_kernel<0><<<grid, block, 0, st>>>(m, k, M, ldm, tri, S, bits, scale, R, rows_pad, ldr, skip);
    SGT_LAUNCH_CHECK();
    return SIGNTRI_OK;
}

signtri_status make_col_slices(int k, int n, const double *M, int ldm, int tri, int S, int bits, const float *scale,
                               __nv_bfloat16 *C, int rows_pad, int ldc, cudaStream_t st, int skip)
{
    if (S > 8 || S * bits > 64) return SIGNTRI_ERR_BAD_ARG;
    if (ldc & 1) return SIGNTRI_ERR_BAD_ARG;
    dim3 grid((ldc / 2 + 255) / 256, rows_pad);
    ProfScope ps(SIGNTRI_KC_CONVERT, st);
    if (S == 7) col_slices_kernel<7><<<grid, 256, 0, st>>>(k, n, M, ldm, tri, S, bits, scale, C, rows_pad, ldc, skip);
    else if (S == 3) col_slices_kernel<3><<<grid, 256, 0, st>>>(k, n, M, ldm, tri, S, bits, scale, C, rows_pad, ldc, skip);
    else col_slices_kernel<0><<<grid, 256, 0, st>>>(k, n, M, ldm, tri, S, bits, scale, C, rows_pad, ldc, skip);
    SGT_LAUNCH_CHECK();
    return SIGNTRI_OK;
}

signtri_status make_gathered_slices(int n, const double *M, int ldm, const int *inv, const int *gmap,
                                    const int *sbbase, int super, int ng, int S, int bits, const float *sR,
                                    const float *sC, float *sRg, float *sCg, __nv_bfloat16 *R, __nv_bfloat16 *C,
                                    int rows, int ld, cudaStream_t st)
{
    if (S > 8 || S * bits > 64 || n <= 0) return SIGNTRI_ERR_BAD_ARG;
    if ((ld & 63) || (rows & 63) || super <= 0 || (super & 63)) return SIGNTRI_ERR_BAD_ARG;
    ProfScope ps(SIGNTRI_KC_CONVERT, st);
    gather_scales_kernel<<<(rows + 255) / 256, 256, 0, st>>>(rows, ng, inv, sR, sRg);
    SGT_LAUNCH_CHECK();
    gather_scales_kernel<<<(rows + 255) / 256, 256, 0, st>>>(rows, ng, inv, sC, sCg);
    SGT_LAUNCH_CHECK();
    const int nsb = (n + super - 1) / super;
    const dim3 rgrid((n + 63) / 64, ld / 64);
    if (S == 7)
        row_slices_gathered_kernel<7><<<rgrid, 256, 0, st>>>(n, M, ldm, inv, gmap, sbbase, super, ng, S, bits, sRg, R,
                                                             rows, ld);
    else
        row_slices_gathered_kernel<0><<<rgrid, 256, 0, st>>>(n, M, ldm, inv, gmap, sbbase, super, ng, S, bits, sRg, R,
                                                             rows, ld);
    SGT_LAUNCH_CHECK();
    const int segmax = super + 128;   // a superblock's rows, each sign class padded to 64
    const size_t csm = (size_t)S * segmax * sizeof(__nv_bfloat16);
    if (S == 7)
        col_slices_gathered_kernel<7><<<dim3(n, nsb), 256, csm, st>>>(n, M, ldm, gmap, sbbase, super, segmax, S, bits,
                                                                      sCg, C, rows, ld);
    else
        col_slices_gathered_kernel<0><<<dim3(n, nsb), 256, csm, st>>>(n, M, ldm, gmap, sbbase, super, segmax, S, bits,
                                                                      sCg, C, rows, ld);
    SGT_LAUNCH_CHECK();
    zero_padding_rows_kernel<<<rows, 256, 0, st>>>(inv, ng, S, R, C, rows, ld);
    SGT_LAUNCH_CHECK();
    return SIGNTRI_OK;
}

// Exact-split pair list: slices s, t with s + t <= S - 1, weights
// 2^{-b(s+t+2)} for slices of b bits, in order of decreasing weight.
TcPairs ozaki_pairs_impl(int S, int bits)
{
    TcPairs p;
    std::memset(&p, 0, sizeof(p));
    for (int g = 0; g < S; g++)
        for (int s = 0; s <= g; s++) {
            p.s[p.n] = s;
            p.t[p.n] = g - s;
            p.w[p.n] = ldexpf(1.0f, -bits * (g + 2));
            p.n++;
        }
    return p;
}

// Rounding-split pair list: s + t <= S - 1, unit weights.
TcPairs split_pairs(int S)
{
    TcPairs p;
    std::memset(&p, 0, sizeof(p));
    for (int g = 0; g < S; g++)
        for (int s = 0; s <= g; s++) {
            p.s[p.n] = s;
            p.t[p.n] = g - s;
            p.w[p.n] = 1.0f;
            p.n++;
        }
    return p;
}

size_t emulated_gemm_workspace_bytes(int m, int n, int k, int S)
{
    const size_t mp = pad64(m), np = (size_t)(n + 127) / 128 * 128, kp = pad64(k);
    const size_t jobs = (mp / 64) * (np / 128);
    return (size_t)S * (mp + np) * kp * 2 + (mp + np) * 12 + jobs * (sizeof(TcJob) + 16384 * 8) + sizeof(TcPairs) +
           64 + 16 * 256;
}

signtri_status emulated_gemm_run(int m, int n, int k, const double *A, int lda, const double *B, int ldb, double *C,
                                 int ldc, int S, Arena &ws, int *d_err, cudaStream_t st)
{
    if (m <= 0 || n <= 0) return SIGNTRI_OK;
    const int mp = pad64(m), np = (n + 127) / 128 * 128, kp = pad64(std::max(k, 1));
    const int ntI = mp / 64, ntJ = np / 128, njobs = ntI * ntJ;
    auto *AR = static_cast<__nv_bfloat16 *>(ws.take((size_t)S * mp * kp * 2));
    auto *BC = static_cast<__nv_bfloat16 *>(ws.take((size_t)S * np * kp * 2));
    auto *sa = static_cast<float *>(ws.take((size_t)mp * 4));
    auto *sb = static_cast<float *>(ws.take((size_t)np * 4));
    auto *tmpa = static_cast<unsigned long long *>(ws.take((size_t)mp * 8));
    auto *tmpb = static_cast<unsigned long long *>(ws.take((size_t)np * 8));
    auto *jobs = static_cast<TcJob *>(ws.take((size_t)njobs * sizeof(TcJob)));
    auto *out = static_cast<double *>(ws.take((size_t)njobs * 16384 * 8));
    auto *dp = static_cast<TcPairs *>(ws.take(sizeof(TcPairs)));
    if (!AR || !BC || !sa || !sb || !tmpa || !tmpb || !jobs || !out || !dp) return SIGNTRI_ERR_NO_WORKSPACE;
    signtri_status rs;
    if ((rs = make_scales(m, k, A, lda, 0, true, mp, tmpa, sa, st)) != SIGNTRI_OK) return rs;
    if ((rs = make_scales(k, n, B, ldb, 0, false, np, tmpb, sb, st)) != SIGNTRI_OK) return rs;
    if ((rs = make_row_slices(m, k, A, lda, 0, S, 7, sa, AR, mp, kp, st)) != SIGNTRI_OK) return rs;
    if ((rs = make_col_slices(k, n, B, ldb, 0, S, 7, sb, BC, np, kp, st)) != SIGNTRI_OK) return rs;
    std::vector<TcJob> hj(njobs);
    for (int I = 0; I < ntI; I++)
        for (int J = 0; J < ntJ; J++) {
            TcJob &j = hj[I * ntJ + J];
            j.rt = I * 64; j.rb = I * 64; j.cl = J * 128; j.cr = J * 128 + 64;
            j.kb0 = 0; j.kb1 = kp / 64; j.slot = I * ntJ + J; j.pad = 0;
        }
    const TcPairs pairs = ozaki_pairs_impl(S, 7);
    SGT_CUDA_TRY(cudaMemcpyAsync(jobs, hj.data(), hj.size() * sizeof(TcJob), cudaMemcpyHostToDevice, st));
    SGT_CUDA_TRY(cudaMemcpyAsync(dp, &pairs, sizeof(TcPairs), cudaMemcpyHostToDevice, st));
    TcSource top{AR, S, mp, kp, kp, sa}, left{BC, S, np, kp, kp, sb}, right{BC, S, np, kp, kp, sb};
    TcQuadOut none{{nullptr, nullptr, nullptr, nullptr}, 0, 0, 0};
    rs = tc_blocksums(top, top, left, right, jobs, njobs, pairs, dp, kExactChunkKb7, out, none, d_err, SIGNTRI_KC_RESIDUAL,
                      st);
    if (rs != SIGNTRI_OK) return rs;
    {
        ProfScope ps(SIGNTRI_KC_OTHER, st);
        gather_gemm_kernel<<<dim3((n + 255) / 256, m), 256, 0, st>>>(m, n, out, ntJ, C, ldc);
        SGT_LAUNCH_CHECK();
    }
    // the host job table and pair list were copied from pageable memory
    SGT_CUDA_TRY(cudaStreamSynchronize(st));
    return SIGNTRI_OK;
}

// C = A op(B), A m x k, op(B) k x n (B or B^T), all column-major, as an
// emulated-float64 product of exact 7-bit slices (7 slices, 28 pairs)
// written straight into C: 128 x 128 output tiles, one job each, the whole K
// range per job.  upper: only tiles that meet the upper triangle (column
// block >= row block) are written; entries below the diagonal inside them
// hold the product as well.
size_t emulated_product_workspace_bytes(int m, int n, int k)
{
    if (m <= 0 || n <= 0) return 0;
    const size_t mp = (size_t)(m + 127) / 128 * 128, np = (size_t)(n + 127) / 128 * 128, kp = pad64(std::max(k, 1));
    const size_t jobs = (mp / 128) * (np / 128);
    return 7 * (mp + np) * kp * 2 + (mp + np) * 12 + jobs * sizeof(TcJob) + sizeof(TcPairs) + 8 * 256;
}

signtri_status emulated_product(int m, int n, int k, const double *A, int lda, const double *B, int ldb, bool transB,
                                double *C, int ldc, bool upper, int kernel_class, Arena &ws, int *d_err,
                                cudaStream_t st)
{
    if (m <= 0 || n <= 0) return SIGNTRI_OK;
    constexpr int S = 7;
    const int mp = (m + 127) / 128 * 128, np = (n + 127) / 128 * 128, kp = pad64(std::max(k, 1));
    const int ntI = mp / 128, ntJ = np / 128;
    auto *AR = static_cast<__nv_bfloat16 *>(ws.take((size_t)S * mp * kp * 2));
    auto *BC = static_cast<__nv_bfloat16 *>(ws.take((size_t)S * np * kp * 2));
    auto *sa = static_cast<float *>(ws.take((size_t)mp * 4));
    auto *sb = static_cast<float *>(ws.take((size_t)np * 4));
    auto *tmpa = static_cast<unsigned long long *>(ws.take((size_t)mp * 8));
    auto *tmpb = static_cast<unsigned long long *>(ws.take((size_t)np * 8));
    auto *jobs = static_cast<TcJob *>(ws.take((size_t)ntI * ntJ * sizeof(TcJob)));
    auto *dp = static_cast<TcPairs *>(ws.take(sizeof(TcPairs)));
    if (!AR || !BC || !sa || !sb || !tmpa || !tmpb || !jobs || !dp) return SIGNTRI_ERR_NO_WORKSPACE;
    signtri_status rs;
    if ((rs = make_scales(m, k, A, lda, 0, true, mp, tmpa, sa, st)) != SIGNTRI_OK) return rs;
    if ((rs = make_row_slices(m, k, A, lda, 0, S, 7, sa, AR, mp, kp, st)) != SIGNTRI_OK) return rs;
    if (transB) {
        // op(B)[kk][j] = B[j][kk]: the rows of B are the K-contiguous lines
        if ((rs = make_scales(n, k, B, ldb, 0, true, np, tmpb, sb, st)) != SIGNTRI_OK) return rs;
        if ((rs = make_row_slices(n, k, B, ldb, 0, S, 7, sb, BC, np, kp, st)) != SIGNTRI_OK) return rs;
    } else {
        if ((rs = make_scales(k, n, B, ldb, 0, false, np, tmpb, sb, st)) != SIGNTRI_OK) return rs;
        if ((rs = make_col_slices(k, n, B, ldb, 0, S, 7, sb, BC, np, kp, st)) != SIGNTRI_OK) return rs;
    }
    std::vector<TcJob> hj;
    hj.reserve((size_t)ntI * ntJ);
    double sum_kb = 0.0;
    for (int I = 0; I < ntI; I++)
        for (int J = upper ? I : 0; J < ntJ; J++) {
            TcJob j;
            j.rt = I * 128; j.rb = I * 128 + 64; j.cl = J * 128; j.cr = J * 128 + 64;
            j.kb0 = 0; j.kb1 = kp / 64; j.slot = 0; j.pad = 0;
            hj.push_back(j);
            sum_kb += kp / 64;
        }
    const TcPairs pairs = ozaki_pairs_impl(S, 7);
    SGT_CUDA_TRY(cudaMemcpyAsync(jobs, hj.data(), hj.size() * sizeof(TcJob), cudaMemcpyHostToDevice, st));
    SGT_CUDA_TRY(cudaMemcpyAsync(dp, &pairs, sizeof(TcPairs), cudaMemcpyHostToDevice, st));
    const TcSource top{AR, S, mp, kp, kp, sa}, left{BC, S, np, kp, kp, sb};
    const TcQuadOut qo{{C, C, C, C}, ldc, m, n, 0};
    rs = tc_blocksums(top, top, left, left, jobs, (int)hj.size(), pairs, dp, kExactChunkKb7, nullptr, qo, d_err,
                      kernel_class, st, tc_flops(1, 1, 4) * sum_kb);   // the float64 product's flops
    if (rs != SIGNTRI_OK) return rs;
    // the host job table and pair list were copied from pageable memory
    SGT_CUDA_TRY(cudaStreamSynchronize(st));
    return SIGNTRI_OK;
}

}  // namespace signtri

// reorder_tc.cu -- blocked reorder by sign for Parlett-Sylvester (Section 2,
// Section 3; Section 4.1's blocking applied to the swaps).
//
// The same stable partition as the odd-even rounds of ps_fp64.cu, done by
// windows (reorder_schedule.h, schedule_window_sweeps): in each sweep every
// window W = [a, a + w) (w <= 128) that still holds a negative above a
// positive is partitioned on its own by adjacent Givens swaps.  One CTA per
// window keeps the diagonal block T[W, W] in shared memory, runs the swaps as
// odd-even rounds there (each rotation as in ps_fp64.cu: G's first column the
// eigenvector of the entry moving up, the 2 x 2 diagonal block swapped
// exactly) and logs them; it then forms the window's orthogonal factor Z_W =
// G_1 G_2 ... by applying the logged rotations to the identity.  The rest of
// T and Q receive the window's rotations at once, as products:
//   T[W, right of W] <- Z_W^T T[W, right of W]
//   T[above W, W]    <- T[above W, W] Z_W
//   Q[:, W]          <- Q[:, W] Z_W
// (left and right factors commute, so all row products of a sweep come
// first, then all column products).  GB300 has no fast float64 product, so
// these run on the tensor cores as emulated-float64 products of exact 8-bit
// slices (tc_gemm.cu), written straight back into T and Q: each product
// reads the slices, snapshots taken before it, never the matrix it writes.
#include <algorithm>
#include <vector>

#include <cuda_bf16.h>

#include "df_arith.cuh"
#include "exact_slices.cuh"
#include "internal.cuh"
#include "reorder_schedule.h"
#include "tc_gemm.cuh"

namespace signtri {

namespace {

constexpr int kWin = 128;                  // window width (two 64-row panels)
constexpr int kWinLD = kWin + 1;
constexpr int kMaxRot = (kWin / 2) * (kWin / 2);   // swaps of a window at most
constexpr int kWinThreads = 512;
// Exact slices of 8 bits, 6 of them (48 bits, the 21 pairs with s + t <= 5):
// a window product's K range is one window (128 <= 256), so every fp32 unit
// sum of products below 2^16 stays exact, and 8-bit slices take a quarter
// fewer pairs, and so a quarter fewer epilogue drains, than 7-bit ones.
constexpr int kSlices = 6;
constexpr int kBits = 8;

// Shared memory of a window: its block as double-float planes (hi, lo), the
// logged rotations (c, s as double-float pairs, and k), the exact diagonal.
size_t window_smem_bytes()
{
    return 2 * (size_t)kWin * kWinLD * sizeof(float) + 4 * (size_t)kMaxRot * sizeof(float) +
           (size_t)kWin * sizeof(double) + (size_t)kMaxRot * sizeof(short);
}

// One window per CTA: stable partition of T[W, W] by swaps, then Z_W as the
// exact column slices the products read -- ZC[s][a + j][a + i] = slice s of
// Z_W[i][j] under the column's power-of-two scale sZ[a + j] (rp rows of
// pitch kp per slice).  Entries of ZC outside the windows' blocks are never
// read (the products' K ranges stay inside the window).
// GB300's float64 rate is about 1/64 of its fp32 rate, and a window is one
// SM's work, so the rotations are applied in double-float (df_arith.cuh:
// about 2^-47 per operation) to the block held as hi/lo planes; the
// diagonal stays float64 (swapped exactly) and each rotation's (c, s) is
// computed in float64 from it and the coupling, one thread per pair.
__global__ void __launch_bounds__(kWinThreads)
window_sort_kernel(double *__restrict__ Tr, int ldt, const int2 *__restrict__ wins, __nv_bfloat16 *__restrict__ ZC,
                   float *__restrict__ sZ, int rp, int kp)
{
    extern __shared__ double wsm[];
    double *dg = wsm;                                        // dg[i] = T[a + i, a + i]
    float *Bh = reinterpret_cast<float *>(dg + kWin);        // Bh/Bl[i + j * kWinLD]: T[a + i, a + j], i < j
    float *Bl = Bh + kWin * kWinLD;
    float *lch = Bl + kWin * kWinLD, *lcl = lch + kMaxRot;   // logged rotations, round by round
    float *lsh = lcl + kMaxRot, *lsl = lsh + kMaxRot;
    short *lk = reinterpret_cast<short *>(lsl + kMaxRot);
    __shared__ signed char sg[kWin];
    __shared__ short pm[kWin];                        // log index of the round's pair holding position i, or -1
    __shared__ int roff[2 * kWin + 4];
    __shared__ int nlog, nround, quiet[2];
    const int a = wins[blockIdx.x].x, w = wins[blockIdx.x].y;
    for (int idx = threadIdx.x; idx < kWin * kWin; idx += kWinThreads) {
        const int i = idx % kWin, j = idx / kWin;
        const double v = (i < j && j < w) ? SGT_AT(Tr, ldt, a + i, a + j) : 0.0;
        split_df(v, Bh[i + j * kWinLD], Bl[i + j * kWinLD]);
        if (i == j) dg[i] = (j < w) ? SGT_AT(Tr, ldt, a + i, a + i) : 1.0;
    }
    __syncthreads();
    for (int i = threadIdx.x; i < kWin; i += kWinThreads) sg[i] = (i < w && dg[i] > 0.0) ? 1 : -1;
    if (threadIdx.x == 0) {
        nlog = 0;
        nround = 0;
        quiet[0] = quiet[1] = 0;
    }
    __syncthreads();
    // odd-even rounds until two in a row swap nothing (at most w + 1 rounds).
    // The count of quiet rounds is double-buffered: round r writes slot
    // r & 1 while the loop test of round r reads slot (r - 1) & 1.
    for (int r = 0; r < 2 * kWin + 2; r++) {
        if (r > 0 && quiet[(r - 1) & 1] >= 2) break;
        if (threadIdx.x < 32) {
            // warp 0 finds the round's pairs (positions 4 lane .. 4 lane + 3),
            // logs them in position order (a prefix count by shuffles) and
            // marks both positions of each pair in pm
            const int lane = threadIdx.x, base = nlog;
            bool on[4];
            int c = 0;
#pragma unroll
            for (int q = 0; q < 4; q++) {
                const int k = 4 * lane + q;
                on[q] = (k & 1) == (r & 1) && k + 1 < w && sg[k] < 0 && sg[k + 1] > 0;
                c += on[q];
            }
            int incl = c;
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
                const int t = __shfl_up_sync(0xffffffffu, incl, o);
                if (lane >= o) incl += t;
            }
            int e = base + incl - c, mine[4];
#pragma unroll
            for (int q = 0; q < 4; q++) {
                mine[q] = -1;
                if (on[q]) {
                    lk[e] = (short)(4 * lane + q);
                    mine[q] = e++;
                }
            }
            const int prev = __shfl_up_sync(0xffffffffu, mine[3], 1);
#pragma unroll
            for (int q = 0; q < 4; q++) {
                const int left = q > 0 ? mine[q - 1] : (lane > 0 ? prev : -1);
                pm[4 * lane + q] = (short)(mine[q] >= 0 ? mine[q] : left);
            }
            const int total = __shfl_sync(0xffffffffu, incl, 31);
            if (lane == 0) {
                roff[r] = base;
                nlog = base + total;
                quiet[r & 1] = total ? 0 : (r > 0 ? quiet[(r - 1) & 1] : 0) + 1;
                nround = r + 1;
            }
        }
        __syncthreads();
        const int e0 = roff[r], P = nlog - e0;
        // each pair's rotation, in float64 from the exact diagonal and the
        // coupling: G's first column is the eigenvector of the entry moving up
        for (int t = threadIdx.x; t < P; t += kWinThreads) {
            const int e = e0 + t, k = lk[e];
            const double aa = dg[k], cc = dg[k + 1];
            const double bb = df_to_double(Bh[k + (k + 1) * kWinLD], Bl[k + (k + 1) * kWinLD]);
            const double d = cc - aa, h = hypot(bb, d);
            split_df(bb / h, lch[e], lcl[e]);
            split_df(d / h, lsh[e], lsl[e]);
        }
        __syncthreads();
        // the round's rotations, one item per (pair, position x): x right of
        // the pair -- G^T on rows k, k+1 of column x (with G_q on columns x,
        // x+1 as well when x starts pair q); x left of the pair -- G on
        // columns k, k+1 of row x (rows inside a pair are done from that
        // pair's side); x = k -- the exact swap of the 2 x 2 diagonal block,
        // whose coupling is unchanged.  No two items touch the same entry.
        for (int idx = threadIdx.x; idx < P * kWin; idx += kWinThreads) {
            const int e = e0 + idx / kWin, x = idx % kWin, k = lk[e];
            if (x >= w) continue;
            const float ch = lch[e], cl = lcl[e], sh = lsh[e], sl = lsl[e];
            if (x >= k + 2) {
                const int q = pm[x];
                if (q < 0) {
                    const int i0 = k + x * kWinLD, i1 = i0 + 1;
                    const float uh = Bh[i0], ul = Bl[i0], vh = Bh[i1], vl = Bl[i1];
                    df_rot(ch, cl, uh, ul, sh, sl, vh, vl, Bh[i0], Bl[i0]);          // c u + s v
                    df_rot(-sh, -sl, uh, ul, ch, cl, vh, vl, Bh[i1], Bl[i1]);        // -s u + c v
                } else if (lk[q] == x) {
                    const float c2h = lch[q], c2l = lcl[q], s2h = lsh[q], s2l = lsl[q];
                    const int i00 = k + x * kWinLD, i10 = i00 + 1, i01 = i00 + kWinLD, i11 = i01 + 1;
                    float r00h, r00l, r10h, r10l, r01h, r01l, r11h, r11l;
                    df_rot(ch, cl, Bh[i00], Bl[i00], sh, sl, Bh[i10], Bl[i10], r00h, r00l);
                    df_rot(-sh, -sl, Bh[i00], Bl[i00], ch, cl, Bh[i10], Bl[i10], r10h, r10l);
                    df_rot(ch, cl, Bh[i01], Bl[i01], sh, sl, Bh[i11], Bl[i11], r01h, r01l);
                    df_rot(-sh, -sl, Bh[i01], Bl[i01], ch, cl, Bh[i11], Bl[i11], r11h, r11l);
                    df_rot(c2h, c2l, r00h, r00l, s2h, s2l, r01h, r01l, Bh[i00], Bl[i00]);    // u c + v s
                    df_rot(-s2h, -s2l, r00h, r00l, c2h, c2l, r01h, r01l, Bh[i01], Bl[i01]);  // -u s + v c
                    df_rot(c2h, c2l, r10h, r10l, s2h, s2l, r11h, r11l, Bh[i10], Bl[i10]);
                    df_rot(-s2h, -s2l, r10h, r10l, c2h, c2l, r11h, r11l, Bh[i11], Bl[i11]);
                }
            } else if (x < k) {
                if (pm[x] < 0) {
                    const int i0 = x + k * kWinLD, i1 = i0 + kWinLD;
                    const float uh = Bh[i0], ul = Bl[i0], vh = Bh[i1], vl = Bl[i1];
                    df_rot(ch, cl, uh, ul, sh, sl, vh, vl, Bh[i0], Bl[i0]);          // u c + v s
                    df_rot(-sh, -sl, uh, ul, ch, cl, vh, vl, Bh[i1], Bl[i1]);        // -u s + v c
                }
            } else if (x == k) {
                const double t0 = dg[k];
                dg[k] = dg[k + 1];
                dg[k + 1] = t0;
                sg[k] = 1;
                sg[k + 1] = -1;
            }
        }
        __syncthreads();
    }
    if (threadIdx.x == 0) roff[nround] = nlog;
    for (int idx = threadIdx.x; idx < kWin * kWin; idx += kWinThreads) {
        const int i = idx % kWin, j = idx / kWin;
        if (j < w && i < j) SGT_AT(Tr, ldt, a + i, a + j) = df_to_double(Bh[i + j * kWinLD], Bl[i + j * kWinLD]);
        else if (j < w && i == j) SGT_AT(Tr, ldt, a + i, a + i) = dg[i];
    }
    __syncthreads();
    // Z = I G_1 G_2 ..., round by round (a round's rotations act on disjoint columns)
    for (int idx = threadIdx.x; idx < kWin * kWin; idx += kWinThreads) {
        const int i = idx % kWin, j = idx / kWin;
        Bh[i + j * kWinLD] = (i == j) ? 1.f : 0.f;
        Bl[i + j * kWinLD] = 0.f;
    }
    __syncthreads();
    for (int r = 0; r < nround; r++) {
        const int e0 = roff[r], e1 = roff[r + 1];
        for (int idx = threadIdx.x; idx < (e1 - e0) * kWin; idx += kWinThreads) {
            const int e = e0 + idx / kWin, i = idx % kWin;
            const int k = lk[e];
            const int i0 = i + k * kWinLD, i1 = i0 + kWinLD;
            const float uh = Bh[i0], ul = Bl[i0], vh = Bh[i1], vl = Bl[i1];
            df_rot(lch[e], lcl[e], uh, ul, lsh[e], lsl[e], vh, vl, Bh[i0], Bl[i0]);
            df_rot(-lsh[e], -lsl[e], uh, ul, lch[e], lcl[e], vh, vl, Bh[i1], Bl[i1]);
        }
        __syncthreads();
    }
    // per column of Z: the power-of-two scale above its largest entry (an
    // orthogonal column: between 1 / sqrt(w) and 1; |hi + lo| < 2^e whenever
    // |hi| < 2^e, lo being at most half an ulp of hi), then its exact slices
    __shared__ int cexp[kWin];
    for (int j = threadIdx.x; j < w; j += kWinThreads) {
        float mx = 0.f;
        for (int i = 0; i < w; i++) mx = fmaxf(mx, fabsf(Bh[i + j * kWinLD]));
        int e = 0;
        frexpf(mx, &e);
        cexp[j] = e;
        sZ[a + j] = ldexpf(1.f, e);
    }
    __syncthreads();
    for (int idx = threadIdx.x; idx < w * w; idx += kWinThreads) {
        const int i = idx % w, j = idx / w;
        float q[kSlices];
        exact_slices<kSlices>(df_to_double(Bh[i + j * kWinLD], Bl[i + j * kWinLD]), cexp[j], kSlices, kBits, q);
#pragma unroll
        for (int sl = 0; sl < kSlices; sl++)
            ZC[((size_t)sl * rp + a + j) * kp + a + i] = __float2bfloat16_rn(q[sl]);
    }
}

// The slices the products of one sweep read, for the active 64-blocks of K
// only (kbl: the sweep's window blocks, ascending).  Three kinds of lines:
//   kColsT: column j of T, K = rows kk < j (row products: tiles kb < jb);
//   kRowsT: row r of T, K = columns kk > r (column products: tiles rb < kb,
//           plus the zero rows [np, np + 64));
//   kRowsQ: row r of Q, K = every active column.
// Every entry a tile holds is then strictly upper for T.  The scale of a line
// is the power of two above its largest entry in the tiles it reads (1 for
// none); lines outside every tile are not outputs of the sweep's products.
constexpr int kColsT = 0, kRowsT = 1, kRowsQ = 2;

template <int MODE>
__device__ __forceinline__ bool tile_used(int kb, int lb, int zero_lb)
{
    if (MODE == kColsT) return lb > kb;
    if (MODE == kRowsT) return lb < kb || lb == zero_lb;
    return true;
}

template <int MODE>
__global__ void __launch_bounds__(256)
masked_absmax_kernel(int n, const double *__restrict__ M, int ldm, const int *__restrict__ kbl, int zero_lb,
                     unsigned long long *__restrict__ mx)
{
    const int kb = kbl[blockIdx.x], lb = blockIdx.y;
    if (!tile_used<MODE>(kb, lb, zero_lb) || lb == zero_lb) return;
    const int k0 = kb * 64, l0 = lb * 64;
    if (MODE == kColsT) {
        // a warp per column: two rows per lane, reduced by shuffles
        const int lane = threadIdx.x & 31, wp = threadIdx.x >> 5;
        for (int c = wp; c < 64; c += 8) {
            const int j = l0 + c;
            unsigned long long v = 0;   // maxima on the bits of |x| (integer pipes)
            if (j < n) {
                if (k0 + lane < n) v = abs_bits(SGT_AT(M, ldm, k0 + lane, j));
                if (k0 + lane + 32 < n) v = max(v, abs_bits(SGT_AT(M, ldm, k0 + lane + 32, j)));
            }
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) v = max(v, __shfl_xor_sync(0xffffffffu, v, o));
            if (lane == 0 && v > 0) atomicMax(&mx[j], v);
        }
    } else {
        // a thread per row and quarter of the columns, then the quarters reduced
        __shared__ unsigned long long part[4][64];
        const int t = threadIdx.x & 63, q = threadIdx.x >> 6, r = l0 + t;
        unsigned long long v = 0;
        if (r < n)
            for (int c = q * 16; c < q * 16 + 16; c++)
                if (k0 + c < n) v = max(v, abs_bits(SGT_AT(M, ldm, r, k0 + c)));
        part[q][t] = v;
        __syncthreads();
        if (threadIdx.x < 64) {
            v = max(max(part[0][t], part[1][t]), max(part[2][t], part[3][t]));
            if (v > 0) atomicMax(&mx[r], v);
        }
    }
}

__device__ __forceinline__ int line_exp(const unsigned long long *mx, int line, int n)
{
    if (line >= n) return 0;
    const unsigned long long m = mx[line];
    return m ? max(frexp_exp_of_bits(m), -120) : 0;
}

// Exact slices (kSlices of kBits bits) of the used tiles, K-contiguous lines of
// pitch kp, rp lines per slice; the line scales go to `scale` (written once
// per line, by the CTA of the first (kColsT, kRowsQ) or last (kRowsT) block).
template <int MODE>
__global__ void __launch_bounds__(256)
masked_slices_kernel(int n, const double *__restrict__ M, int ldm, const int *__restrict__ kbl, int zero_lb,
                     const unsigned long long *__restrict__ mx, __nv_bfloat16 *__restrict__ out, float *__restrict__ scale,
                     int rp, int kp)
{
    const int kb = kbl[blockIdx.x], lb = blockIdx.y;
    if (!tile_used<MODE>(kb, lb, zero_lb)) return;
    const int k0 = kb * 64, l0 = lb * 64;
    const bool zero = lb == zero_lb;
    const bool writes_scale = !zero && (int)blockIdx.x == (MODE == kRowsT ? (int)gridDim.x - 1 : 0);
    const int lane = threadIdx.x & 31, wp = threadIdx.x >> 5;
    if (MODE == kColsT) {
        // column j's K run is contiguous in M: lane reads rows k0 + 2 lane, + 1
        for (int c = wp; c < 64; c += 8) {
            const int j = l0 + c, kk = k0 + 2 * lane;
            double v0 = 0.0, v1 = 0.0;
            if (j < n) {
                if (kk < n) v0 = SGT_AT(M, ldm, kk, j);
                if (kk + 1 < n) v1 = SGT_AT(M, ldm, kk + 1, j);
            }
            const int e = line_exp(mx, j, n);
            float q0[kSlices], q1[kSlices];
            exact_slices<kSlices>(v0, e, kSlices, kBits, q0);
            exact_slices<kSlices>(v1, e, kSlices, kBits, q1);
#pragma unroll
            for (int sl = 0; sl < kSlices; sl++)
                *reinterpret_cast<__nv_bfloat162 *>(&out[((size_t)sl * rp + j) * kp + kk]) =
                    __floats2bfloat162_rn(q0[sl], q1[sl]);
            if (writes_scale && lane == 0 && j < n) scale[j] = ldexpf(1.f, e);
        }
    } else {
        // rows: transposed through shared memory (tile[kk][r])
        __shared__ double tile[64][65];
        for (int idx = threadIdx.x; idx < 64 * 64; idx += 256) {
            const int t = idx & 63, c = idx >> 6, r = l0 + t, kk = k0 + c;
            tile[c][t] = (!zero && r < n && kk < n) ? SGT_AT(M, ldm, r, kk) : 0.0;
        }
        __syncthreads();
        for (int t = wp; t < 64; t += 8) {
            const int r = l0 + t, kk = k0 + 2 * lane;
            const int e = zero ? 0 : line_exp(mx, r, n);
            float q0[kSlices], q1[kSlices];
            exact_slices<kSlices>(tile[2 * lane][t], e, kSlices, kBits, q0);
            exact_slices<kSlices>(tile[2 * lane + 1][t], e, kSlices, kBits, q1);
#pragma unroll
            for (int sl = 0; sl < kSlices; sl++)
                *reinterpret_cast<__nv_bfloat162 *>(&out[((size_t)sl * rp + r) * kp + kk]) =
                    __floats2bfloat162_rn(q0[sl], q1[sl]);
            if (writes_scale && lane == 0 && r < n) scale[r] = ldexpf(1.f, e);
        }
    }
}

}  // namespace

size_t reorder_blocked_workspace_bytes(int n)
{
    if (n <= 0) return 0;
    const size_t rp = (size_t)pad64(n) + 64, kp = (size_t)pad64(n);
    size_t b = 4 * (kSlices * rp * kp * 2 + 256);                    // slices: Z, T (two forms), Q
    b += 4 * (rp * sizeof(float) + 256) + 3 * rp * 8 + 256;           // scales, line maxima
    b += sizeof(TcPairs) + 256;
    // the window and job lists of every sweep go to memory of their own
    return b;
}

signtri_status reorder_blocked_run(int n, const double *T, int ldt, double *Tr, int ldtr, double *Q, int ldq,
                                   long long *swaps_out, Arena &ws, int *d_err, cudaStream_t st)
{
    if (n <= 0) return SIGNTRI_OK;
    const int np = pad64(n), rp = np + 64, kp = np, zero = np;   // rows [np, np + 64) of every slice array are zero
    auto slices = [&]() { return static_cast<__nv_bfloat16 *>(ws.take((size_t)kSlices * rp * kp * 2)); };
    __nv_bfloat16 *ZC = slices(), *TC = slices(), *TR = slices(), *QR = slices();
    float *sZ = static_cast<float *>(ws.take(rp * sizeof(float)));
    float *sTc = static_cast<float *>(ws.take(rp * sizeof(float)));
    float *sTr = static_cast<float *>(ws.take(rp * sizeof(float)));
    float *sQ = static_cast<float *>(ws.take(rp * sizeof(float)));
    auto *mx = static_cast<unsigned long long *>(ws.take(3 * (size_t)rp * sizeof(unsigned long long)));
    auto *d_pairs = static_cast<TcPairs *>(ws.take(sizeof(TcPairs)));
    if (!ZC || !TC || !TR || !QR || !sZ || !sTc || !sTr || !sQ || !mx || !d_pairs) return SIGNTRI_ERR_NO_WORKSPACE;
    signtri_status rs = copy_upper_identity(n, T, ldt, Tr, ldtr, Q, ldq, st);   // T~ = upper part of T, Q = I
    if (rs != SIGNTRI_OK) return rs;
    std::vector<double> diag(n);
    SGT_CUDA_TRY(cudaMemcpy2DAsync(diag.data(), sizeof(double), T, ((size_t)ldt + 1) * sizeof(double), sizeof(double),
                                   n, cudaMemcpyDeviceToHost, st));
    SGT_CUDA_TRY(cudaStreamSynchronize(st));
    std::vector<std::vector<int2>> sweeps;
    long long swaps = 0;
    schedule_window_sweeps(diag, kWin, sweeps, swaps);
    if (swaps_out) *swaps_out = swaps;
    if (swaps == 0) return SIGNTRI_OK;
    // every sweep's windows and the jobs of its three products, built here
    // and uploaded once
    auto job = [](int rt, int rb, int cl, int cr, int kb0, int kb1) {
        TcJob j;
        j.rt = rt; j.rb = rb; j.cl = cl; j.cr = cr; j.kb0 = kb0; j.kb1 = kb1; j.slot = 0; j.pad = 0;
        return j;
    };
    std::vector<int2> wins_all;
    std::vector<TcJob> jobs_all;
    std::vector<int> kbl_all;   // each sweep's window 64-blocks, ascending
    struct Sweep { int w0, nw; int j[4]; double kb[3]; int k0, nk; };
    std::vector<Sweep> plan;
    for (const std::vector<int2> &sw : sweeps) {
        if (sw.empty()) continue;
        Sweep p{(int)wins_all.size(), (int)sw.size(), {0, 0, 0, 0}, {0, 0, 0}, (int)kbl_all.size(), 0};
        wins_all.insert(wins_all.end(), sw.begin(), sw.end());
        for (const int2 &win : sw)
            for (int kb = win.x / 64; kb <= (win.x + win.y - 1) / 64; kb++) kbl_all.push_back(kb);
        p.nk = (int)kbl_all.size() - p.k0;
        for (int phase = 0; phase < 3; phase++) {
            p.j[phase] = (int)jobs_all.size();
            for (const int2 &win : sw) {
                const int a = win.x, e = win.x + win.y, kb0 = a / 64, kb1 = (e + 63) / 64;
                const int second = win.y > 64 ? a + 64 : zero;
                if (phase == 0) {
                    // rows: T[W, c..c+128) <- Z^T T[W, c..c+128) for the columns right of W
                    for (int c = e; c < n; c += 128) jobs_all.push_back(job(a, second, c, c + 64 < n ? c + 64 : zero, kb0, kb1));
                } else {
                    // columns: T[r..r+128, W] <- T[r..r+128, W] Z above W; Q[r..r+128, W] <- Q[..] Z for all rows
                    const int rows = phase == 1 ? a : n;
                    for (int r = 0; r < rows; r += 128)
                        jobs_all.push_back(job(r, r + 64 < rows ? r + 64 : zero, a, second, kb0, kb1));
                }
            }
            for (int q = p.j[phase]; q < (int)jobs_all.size(); q++) p.kb[phase] += 4.0 * (jobs_all[q].kb1 - jobs_all[q].kb0);
        }
        p.j[3] = (int)jobs_all.size();
        plan.push_back(p);
    }
    int2 *d_wins = nullptr;
    TcJob *d_jobs = nullptr;
    int *d_kbl = nullptr;
    if (cudaMalloc(&d_wins, std::max<size_t>(wins_all.size(), 1) * sizeof(int2)) != cudaSuccess ||
        cudaMalloc(&d_jobs, std::max<size_t>(jobs_all.size(), 1) * sizeof(TcJob)) != cudaSuccess ||
        cudaMalloc(&d_kbl, std::max<size_t>(kbl_all.size(), 1) * sizeof(int)) != cudaSuccess) {
        cudaGetLastError();
        cudaFree(d_wins);
        cudaFree(d_jobs);
        return SIGNTRI_ERR_NO_WORKSPACE;
    }
    auto body = [&]() -> signtri_status {
        SGT_CUDA_TRY(cudaMemcpyAsync(d_wins, wins_all.data(), wins_all.size() * sizeof(int2), cudaMemcpyHostToDevice, st));
        SGT_CUDA_TRY(cudaMemcpyAsync(d_jobs, jobs_all.data(), jobs_all.size() * sizeof(TcJob), cudaMemcpyHostToDevice, st));
        SGT_CUDA_TRY(cudaMemcpyAsync(d_kbl, kbl_all.data(), kbl_all.size() * sizeof(int), cudaMemcpyHostToDevice, st));
        const TcPairs pairs = ozaki_pairs_impl(kSlices, kBits);
        SGT_CUDA_TRY(cudaMemcpyAsync(d_pairs, &pairs, sizeof(TcPairs), cudaMemcpyHostToDevice, st));
        // the zero rows past the matrix, read by the half-empty jobs
        SGT_CUDA_TRY(cudaMemsetAsync(ZC, 0, (size_t)kSlices * rp * kp * 2, st));
        const size_t smem = window_smem_bytes();
        SGT_CUDA_TRY(cudaFuncSetAttribute(window_sort_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
        const TcSource srcZ{ZC, kSlices, rp, kp, kp, sZ}, srcTc{TC, kSlices, rp, kp, kp, sTc};
        const TcSource srcTr{TR, kSlices, rp, kp, kp, sTr}, srcQ{QR, kSlices, rp, kp, kp, sQ};
        const TcQuadOut toT{{Tr, Tr, Tr, Tr}, ldtr, n, n, 0}, toQ{{Q, Q, Q, Q}, ldq, n, n, 0};
        const double fl = tc_flops(pairs.n, 1, 1);
        auto product = [&](const Sweep &p, int phase, const TcSource &top, const TcSource &left,
                           const TcQuadOut &out) -> signtri_status {
            const int cnt = p.j[phase + 1] - p.j[phase];
            if (cnt == 0) return SIGNTRI_OK;
            return tc_blocksums(top, top, left, left, d_jobs + p.j[phase], cnt, pairs, d_pairs, kExactChunkKb8, nullptr,
                                out, d_err, SIGNTRI_KC_GIVENS, st, fl * p.kb[phase]);
        };
        const int zero_lb = np / 64;
        unsigned long long *mxTc = mx, *mxTr = mx + rp, *mxQ = mx + 2 * (size_t)rp;
        // scales and slices of the active K blocks of one kind of line
        auto convert = [&](int mode, const Sweep &p, const double *M, int ldm, unsigned long long *m,
                           __nv_bfloat16 *out, float *scale) -> signtri_status {
            ProfScope ps(SIGNTRI_KC_CONVERT, st);
            const dim3 grid(p.nk, rp / 64);
            const int *kbl = d_kbl + p.k0;
            if (mode == kColsT) {
                masked_absmax_kernel<kColsT><<<grid, 256, 0, st>>>(n, M, ldm, kbl, zero_lb, m);
                masked_slices_kernel<kColsT><<<grid, 256, 0, st>>>(n, M, ldm, kbl, zero_lb, m, out, scale, rp, kp);
            } else if (mode == kRowsT) {
                masked_absmax_kernel<kRowsT><<<grid, 256, 0, st>>>(n, M, ldm, kbl, zero_lb, m);
                masked_slices_kernel<kRowsT><<<grid, 256, 0, st>>>(n, M, ldm, kbl, zero_lb, m, out, scale, rp, kp);
            } else {
                masked_absmax_kernel<kRowsQ><<<grid, 256, 0, st>>>(n, M, ldm, kbl, zero_lb, m);
                masked_slices_kernel<kRowsQ><<<grid, 256, 0, st>>>(n, M, ldm, kbl, zero_lb, m, out, scale, rp, kp);
            }
            SGT_LAUNCH_CHECK();
            return SIGNTRI_OK;
        };
        signtri_status r2;
        for (const Sweep &p : plan) {
            SGT_CUDA_TRY(cudaMemsetAsync(mx, 0, 3 * (size_t)rp * sizeof(unsigned long long), st));
            {
                ProfScope ps(SIGNTRI_KC_GIVENS, st);
                window_sort_kernel<<<p.nw, kWinThreads, smem, st>>>(Tr, ldtr, d_wins + p.w0, ZC, sZ, rp, kp);
                SGT_LAUNCH_CHECK();
            }
            // Q is read by its own product only: slice it alongside T's columns
            if ((r2 = convert(kRowsQ, p, Q, ldq, mxQ, QR, sQ)) != SIGNTRI_OK) return r2;
            if ((r2 = convert(kColsT, p, Tr, ldtr, mxTc, TC, sTc)) != SIGNTRI_OK) return r2;
            if ((r2 = product(p, 0, srcZ, srcTc, toT)) != SIGNTRI_OK) return r2;     // rows of T
            if ((r2 = convert(kRowsT, p, Tr, ldtr, mxTr, TR, sTr)) != SIGNTRI_OK) return r2;
            if ((r2 = product(p, 1, srcTr, srcZ, toT)) != SIGNTRI_OK) return r2;     // columns of T
            if ((r2 = product(p, 2, srcQ, srcZ, toQ)) != SIGNTRI_OK) return r2;      // columns of Q
        }
        // the host lists stay alive until the copies above are done; so do the
        // device lists until the last product
        SGT_CUDA_TRY(cudaStreamSynchronize(st));
        return SIGNTRI_OK;
    };
    rs = body();
    if (rs != SIGNTRI_OK) cudaStreamSynchronize(st);
    cudaFree(d_wins);
    cudaFree(d_jobs);
    cudaFree(d_kbl);
    return rs;
}

}  // namespace signtri

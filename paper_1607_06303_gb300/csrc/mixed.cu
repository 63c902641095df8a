// mixed.cu -- Parlett-Higham with tensor-core block sums and float64
// refinement of both defining equations.
//
// 1. Low-precision solve.  The block anti-diagonal schedule of the float64
//    path (Algorithms 4-6 reordered, blocks of 64), with the block sums
//      X_IJ = sum_K U_IK T_KJ - T_IK U_KJ,   Y_IJ = sum_K U_IK U_KJ
//    formed on the tensor cores (tc_gemm.cu) from 16-bit splits of U and T:
//    one bf16 term (BF16 variant), a three-term bf16 split hi + mid + lo with
//    the six products of s + t <= 2 (about fp32 accuracy, the "FP32"
//    variant), or a two-term fp16 split hi + lo with the three products of
//    s + t <= 1 (about 2^-21; T, U and the correction scaled by powers of two
//    into fp16's range, the FP16 variant); in-block recurrences (Algorithm 6,
//    1x1 case) in fp32, a 64-row tile solved by 16 x 16 sub-blocks.
// 2. Refinement.  With U = U0 + E and E strictly upper triangular, UT = TU
//    and U^2 = I become, entry by entry (i < j):
//      signs differ: (t_ii - t_jj) e_ij = -Rc_ij + sum_{i<k<j} (e_ik t_kj - t_ik e_kj)
//      signs equal:  (u_ii + u_jj) e_ij = -Rs_ij - sum_{i<k<j} (u0_ik e_kj + e_ik u0_kj)
//    (the second dropping e_ik e_kj), with the residuals Rc = T U0 - U0 T and
//    Rs = U0^2 - I.  These are the Parlett-Higham recurrences with U replaced
//    by E, so E is computed by the same schedule (block sums X^E = E T - T E,
//    Y^E = U0 E + E U0 on the tensor cores, recurrences in fp32).  Newton's
//    iteration X <- X(3I - X^2)/2 alone would only drive U^2 = I and cannot
//    correct the entries fixed by UT = TU, hence both equations.
//    Entry (i, j) uses Rc_ij when the signs differ and Rs_ij when they agree
//    (the same choice as Algorithm 3), so the residual that drives the first
//    correction forms only that one (Section 5.3's economy applied to the
//    residual products); acceptance always rests on both residuals over all
//    entries (an ill-conditioned problem can meet its own recurrences long
//    before the other equation).  The residuals
//    come from exact 7-bit integer slices of the strictly upper parts of T and
//    U0 (seven slices, 28 pairs over K-chunks of 1024: emulated float64
//    products, about 2^-45 relative to |T||U| -- the slices are scaled per
//    row and column of the strictly upper parts, whose entries are of similar
//    magnitude, the diagonals being taken apart; 8-bit slices would need 21
//    pairs but K-chunks of 256, and the fourfold epilogue work costs more than
//    the pairs save) plus the
//    diagonal terms in float64:
//      Rc_ij = (N_T N_U - N_U N_T)_ij + t_ii u_ij + t_ij u_jj - u_ii t_ij - u_ij t_jj
//      Rs_ij = (N_U N_U)_ij + u_ii u_ij + u_ij u_jj.
//    For the products the indices are gathered per superblock of kSuper
//    consecutive indices, positives first, each sign class padded to whole
//    64-blocks: every 64 x 64 output block then has one sign class in its rows
//    and one in its columns, and a tensor-core job computes four such blocks
//    that all need the same product (Y = N_U N_U, or one of the two parts of
//    X).  Block upper triangular structure survives at superblock level, so a
//    job's K range lies within its superblocks, trimmed to where its rows and
//    columns can have nonzero terms (the rest are structural zeros).
//    The full residuals use the original layout and four-quadrant jobs
//    [N_T I.; N_U I.] x [N_U .J | N_T .J].  Stop when ||Rc||_F / (||T||_F
//    ||U||_F) and ||Rs||_F / ||U||_F^2 are both below the tolerance; fall back
//    to the float64 path when a step does not reduce the larger of the two by
//    a factor 10, or after the step limit.
// 3. Memory traffic.  The sweeps stream each tile's operand panels once per
//    anti-diagonal (bf16 slices stored as contiguous 64 x 64 tiles).  Launches
//    that read the same panels run side by side on side streams with matched
//    CTA splits, so the second read comes from L2: the correction's X^E and
//    Y^E (shared E panels), and the initial sweep's look-ahead pairs, where an
//    anti-diagonal's tiles sum the next one's interior K-blocks (shared row
//    panels) and a short completion launch adds the four K-blocks left.
#include <algorithm>
#include <utility>
#include <cmath>
#include <cstring>
#include <vector>

#include <cuda_bf16.h>
#include <cuda_fp16.h>

#include "df_arith.cuh"
#include "internal.cuh"
#include "gathered_layout.h"
#include "sweep_schedule.h"
#include "tc_gemm.cuh"

namespace signtri {

namespace {

constexpr int MB = 64;
static_assert(MB == kSweepTile, "the sweep work lists and the kernels share the tile size");

constexpr int kOzakiSlices = 7;   // exact slices of kOzakiBits bits: 49 bits, 28 pairs
constexpr int kOzakiBits = 7;
constexpr int kSuper = 1024;   // superblock of the gathered residual layout

__device__ __forceinline__ float fsgn(double t) { return t > 0.0 ? 1.f : -1.f; }

// One term of a rounding split: the 16-bit rounding of x (bf16, or fp16 when
// f16), x left holding the remainder (exact in fp32).
__device__ __forceinline__ unsigned short split_term(float &x, bool f16)
{
    if (f16) {
        const __half h = __float2half_rn(x);
        x -= __half2float(h);
        return __half_as_ushort(h);
    }
    const __nv_bfloat16 h = __float2bfloat16_rn(x);
    x -= __bfloat162float(h);
    return __bfloat16_as_ushort(h);
}

// Four consecutive entries, S terms each, slice s at dst + s * sstride.
__device__ __forceinline__ void split_store4(float4 r, int S, bool f16, __nv_bfloat16 *dst, size_t sstride)
{
    for (int s = 0; s < S; s++) {
        const unsigned a = split_term(r.x, f16), b = split_term(r.y, f16);
        const unsigned c = split_term(r.z, f16), d = split_term(r.w, f16);
        *reinterpret_cast<uint2 *>(dst + s * sstride) = make_uint2(a | (b << 16), c | (d << 16));
    }
}

// --------------------------------------------------------------- leaves ---

constexpr int kLeafThreads = 256;
constexpr int kSub = 16;             // sub-block edge of the in-tile solve
constexpr int kLeafLD = MB + 4;      // leaf smem pitch: rows / columns stay 16-byte aligned for float4 reads
constexpr int kNSub = MB / kSub;     // sub-blocks per tile edge
constexpr int kLeafBufs = 6;         // M+, M-, N+, N-, V by columns, V by rows

// Per-sign operators of the in-block recurrences.  Entry (p, q) of a tile
// (I, J) is fixed by
//   signs differ:  v_pq (t_pp - t_qq) = c_pq + sum_k v_pk T_kq - sum_k T_pk v_kq
//   signs agree:   v_pq (s_p + s_q)   = c_pq - sum_k v_pk A_kq - sum_k A_pk v_kq
// (k over the tile's own rows and columns; A = U in the initial solve, U0 in
// the correction).  So the column part is - sum_k M^{s_q}_pk v_kq, where row
// r of M^+ is A's row r if s_r = +, else T's, and M^- the other way round,
// and the row part is + sum_k v_pk N^{s_p}_kq, where column c of N^+ is -A's
// column c if s_c = +, else +T's, and N^- the other way round.  Per diagonal
// block I, fp32, 64 x 64, zero on and below the diagonal (the diagonal terms
// of T sit in the divisor t_pp - t_qq):
//   OPS[(4 I + 0) 4096 ..]  M^+ row-major      OPS[(4 I + 1) 4096 ..]  M^- row-major
//   OPS[(4 I + 2) 4096 ..]  N^+ column-major   OPS[(4 I + 3) 4096 ..]  N^- column-major
// and DIAG[i] = (float) t_ii (0 beyond n).
__global__ void leaf_ops_kernel(int n, const double *__restrict__ T, int ldt, const double *__restrict__ A, int lda,
                                float *__restrict__ OPS, float *__restrict__ DIAG)
{
    const int r0 = blockIdx.x * MB;
    __shared__ float sg[MB];
    for (int i = threadIdx.x; i < MB; i += blockDim.x) {
        const bool in = r0 + i < n;
        const double t = in ? SGT_AT(T, ldt, r0 + i, r0 + i) : 0.0;
        sg[i] = (in && t > 0.0) ? 1.f : -1.f;
        DIAG[r0 + i] = (float)t;
    }
    __syncthreads();
    float *mp = OPS + (size_t)(4 * blockIdx.x) * MB * MB;
    for (int idx = threadIdx.x; idx < MB * MB; idx += blockDim.x) {
        const int i = idx % MB, j = idx / MB;   // element (i, j) of the block, i fastest
        const bool in = r0 + j < n && i < j;
        const float t = in ? (float)SGT_AT(T, ldt, r0 + i, r0 + j) : 0.f;
        const float a = in ? (float)SGT_AT(A, lda, r0 + i, r0 + j) : 0.f;
        // row-major M: row i picks by the sign of i; column-major N: column j by the sign of j
        mp[0 * MB * MB + i * MB + j] = sg[i] > 0.f ? a : t;
        mp[1 * MB * MB + i * MB + j] = sg[i] > 0.f ? t : a;
        mp[2 * MB * MB + j * MB + i] = sg[j] > 0.f ? -a : t;
        mp[3 * MB * MB + j * MB + i] = sg[j] > 0.f ? t : -a;
    }
}

// One warp solves the 16 x 16 sub-block with rows R0.. and columns C0.. of a
// leaf tile (the recurrences above restricted to it; the terms of the other,
// already solved, sub-blocks are in VR and VC).  Lane (p, h) = p + 16 h owns
// row R0 + p, columns C0 + 8h .. C0 + 8h + 7: its pending values c[j] start
// as seed + row parts - column parts of the solved sub-blocks; entry (p, q)
// is solved at step t = 15 - p + q by the lane of q's half, and each solved
// value is pushed at once into the entries that depend on it -- into the
// row's later entries by both lanes of the row (+ v N~, the value passed to
// the other half by a shuffle), into the entries above it in its column by
// the other rows' lanes of the same half, which receive it by shuffle
// (- M v).  The coefficients M^{+-}[p][k] sit in each lane rotated by 8 h,
// so that one constant register index serves both halves; the step's pending
// value is picked by a three-level select tree and divided by a reciprocal
// taken off the chain.  Both halves working halves the instructions per
// step; the step loop is unrolled so that every register index is a
// constant.
__device__ __forceinline__ void subblock_solve(const float *__restrict__ Mp, const float *__restrict__ Mm,
                                               const float *__restrict__ Np, const float *__restrict__ Nm,
                                               float *__restrict__ VC, float *__restrict__ VR,
                                               const float *__restrict__ srow, const float *__restrict__ scol,
                                               const float *__restrict__ drow, const float *__restrict__ dcol, int R0,
                                               int C0, int lane)
{
    constexpr int LD = kLeafLD;
    const int p = lane & (kSub - 1), h = lane >> 4;
    const int P = R0 + p;
    // column signs of the sub-block, bit q for column C0 + q
    const unsigned colmask = __ballot_sync(0xffffffffu, lane < kSub && scol[C0 + p] > 0.f) & 0xffffu;
    const unsigned hmask = (colmask >> (8 * h)) & 0xffu;   // this half's columns
    const float sp = srow[P], dp = drow[P];
    float c[8], mr[24], nr[24];
#pragma unroll
    for (int j = 0; j < 8; j++) c[j] = VR[P * LD + C0 + 8 * h + j] - VC[(C0 + 8 * h + j) * LD + P];
    // mr[x] = M^+[p][x - 8 + 8h], nr[x] = M^-[p][x - 8 + 8h] (0 outside the block)
#pragma unroll
    for (int x = 0; x < 24; x++) {
        const int k = x - 8 + 8 * h;
        const bool ok = k >= 0 && k < kSub;
        mr[x] = ok ? Mp[P * LD + R0 + k] : 0.f;
        nr[x] = ok ? Mm[P * LD + R0 + k] : 0.f;
    }
    const float *Nt = (sp > 0.f ? Np : Nm) + C0 * LD + C0;   // N~^{s_p}, this sub-block
    const int base = 24 * h;
    float vprev = 0.f;
#pragma unroll
    for (int t = 0; t < 2 * kSub - 1; t++) {
        // column parts: column q = 8h + j takes row k = q + 16 - t, solved at
        // the previous step by lane k + 16 h = k0 + 24 h (the same half;
        // taken mod 32 where k is outside the block and the coefficient 0)
#pragma unroll
        for (int j = 0; j < 8; j++) {
            const int k0 = j + kSub - t;   // k in half 0; k0 + 8 in half 1
            if (t > 0 && k0 >= -8 && k0 < kSub) {
                const int src = (base + k0) & 31;
                const float vk = __shfl_sync(0xffffffffu, vprev, src);
                c[j] = fmaf((hmask >> j) & 1u ? -mr[k0 + 8] : -nr[k0 + 8], vk, c[j]);
            }
        }
        const int qp = t - (kSub - 1) + p;   // the row's column at this step
        const int hc = qp >> 3;               // its half
        const bool act = qp >= 0 && qp < kSub && hc == h;
        const int qc = min(max(qp, 0), kSub - 1);
        const bool sq = (colmask >> qc) & 1u;
        const bool opp = (sp > 0.f) != sq;
        const float den = opp ? dp - dcol[C0 + qc] : sp + (sq ? 1.f : -1.f);
        const float rden = __fdividef(1.f, den);
        const int jb = (qc - 8 * h) & 7;
        const float s0 = (jb & 1) ? c[1] : c[0], s1 = (jb & 1) ? c[3] : c[2];
        const float s2 = (jb & 1) ? c[5] : c[4], s3 = (jb & 1) ? c[7] : c[6];
        const float u0 = (jb & 2) ? s1 : s0, u1 = (jb & 2) ? s3 : s2;
        const float x = (jb & 4) ? u1 : u0;
        const float v = act ? x * rden : 0.f;
        // the row's solved value to both halves, then its row part
        const float vrow = __shfl_sync(0xffffffffu, v, p + 16 * min(max(hc, 0), 1));
        if (t < 2 * kSub - 2) {
#pragma unroll
            for (int j = 0; j < 8; j++) c[j] = fmaf(Nt[(8 * h + j) * LD + qc], vrow, c[j]);
        }
        if (act) {
            VC[(C0 + qc) * LD + P] = v;
            VR[P * LD + C0 + qc] = v;
        }
        vprev = v;
    }
}

// MODE 0: V = U (initial solve).  MODE 1: V = E (correction), with Rc, Rs.
// Shared memory (fp32, pitch kLeafLD): the operators M^+, M^- of block I
// (row-major) and N^+, N^- of block J (column-major), V by columns (VC) and
// by rows (VR).  Until entry (p, q) is solved, VR[p][q] holds its seed (base
// terms, block sums and the row parts of the solved sub-blocks) and VC[q][p]
// the column parts of the solved sub-blocks.
template <int MODE>
__global__ void __launch_bounds__(kLeafThreads, 2)
mixed_leaf_kernel(int n, const double *__restrict__ T, int ldt, double *__restrict__ V, int ldv,
                  const float *__restrict__ OPS, const float *__restrict__ DIAG, const double *__restrict__ Rc,
                  const double *__restrict__ Rs, int ldr, int d, const int2 *__restrict__ tslot,
                  const int2 *__restrict__ tslot2,
                  const double *__restrict__ PA, const double *__restrict__ PB, __nv_bfloat16 *__restrict__ Vr,
                  __nv_bfloat16 *__restrict__ Vc, int S, int nbk, float sigma)
{
    constexpr int LD = kLeafLD;
    constexpr int EPT = MB * MB / kLeafThreads;   // tile entries per thread
    constexpr int QS = kLeafThreads / MB;
    extern __shared__ float4 fsm4[];
    float *Mp = reinterpret_cast<float *>(fsm4);
    float *Mm = Mp + MB * LD;
    float *Np = Mm + MB * LD;
    float *Nm = Np + MB * LD;
    float *VC = Nm + MB * LD;
    float *VR = VC + MB * LD;
    __shared__ float srow[MB], scol[MB], drow[MB], dcol[MB];
    const int I = blockIdx.x, J = I + d;
    const int r0 = I * MB, c0 = J * MB;
    const int bj = min(MB, n - c0);
    const int p = threadIdx.x % MB, q0 = threadIdx.x / MB;

    // every global read before the first barrier: this tile's partial slots,
    // the base terms of the seeds, the operators
    const int2 ts = tslot[I];
    const int2 ts2 = (MODE == 0 && tslot2) ? tslot2[I] : make_int2(0, 0);
    // the partial block sums first (the largest read), with the signs of the
    // thread's own row and columns taken from DIAG, so that they are in
    // flight with the reads below: float2 (hi, lo) per element, summed in
    // fp32 over the slots
    float acc[EPT];
    bool opp[EPT];
    {
        const float sgp = DIAG[r0 + p] > 0.f ? 1.f : -1.f;
#pragma unroll
        for (int m = 0; m < EPT; m++) {
            const int q = q0 + m * QS;
            const float sgq = (q < bj) ? (DIAG[c0 + q] > 0.f ? 1.f : -1.f) : 1.f;
            acc[m] = 0.f;
            opp[m] = sgp + sgq == 0.f;
        }
        const float2 *PA2 = reinterpret_cast<const float2 *>(PA);
        const float2 *PB2 = reinterpret_cast<const float2 *>(PB);
        #pragma unroll 2
        for (int s = 0; s < ts.y + ts2.y; s++) {
            // mode 0: slots of PA, then (look-ahead pairing) slots of PB
            const bool second = s >= ts.y;
            const float2 *P0 = second ? PB2 : PA2;
            const size_t sb = ((size_t)(second ? ts2.x + s - ts.y : ts.x + s)) * 16384 + p;
#pragma unroll
            for (int m = 0; m < EPT; m++) {
                const int q = q0 + m * QS;
                // opposite signs: TL - BR of PA (X); equal signs: TR of PA
                // (Y, mode 0) or TL + BR of PB (Y^E, mode 1)
                const float2 *src = opp[m] ? P0 : (MODE == 0 ? P0 + 4096 : PB2);
                const size_t e = sb + (size_t)q * 64;
                const float2 l1 = src[e];
                float2 l2 = make_float2(0.f, 0.f);
                if (MODE == 1 || opp[m]) l2 = src[e + 3 * 4096];
                const float sg = opp[m] ? -1.f : 1.f;
                acc[m] += (l1.x + sg * l2.x) + (l1.y + sg * l2.y);
            }
        }
    }
    // base terms staged in VR (t_pq, or Rc_pq) and VC (Rs_pq) at the thread's
    // own entries until the seeds replace them
#pragma unroll 4
    for (int m = 0; m < EPT; m++) {
        const int q = q0 + m * QS;
        const bool ok = q < bj;
        VR[p * LD + q] = ok ? (float)SGT_AT(MODE == 0 ? T : Rc, MODE == 0 ? ldt : ldr, r0 + p, c0 + q) : 0.f;
        VC[q * LD + p] = (MODE == 1 && ok) ? (float)SGT_AT(Rs, ldr, r0 + p, c0 + q) : 0.f;
    }
    {
        const float4 *src[4] = {reinterpret_cast<const float4 *>(OPS + (size_t)(4 * I + 0) * MB * MB),
                                reinterpret_cast<const float4 *>(OPS + (size_t)(4 * I + 1) * MB * MB),
                                reinterpret_cast<const float4 *>(OPS + (size_t)(4 * J + 2) * MB * MB),
                                reinterpret_cast<const float4 *>(OPS + (size_t)(4 * J + 3) * MB * MB)};
        float *dst[4] = {Mp, Mm, Np, Nm};
        // all four operators' loads in flight before the first store
        constexpr int V4 = MB * MB / 4 / kLeafThreads;
        float4 v[4][V4];
#pragma unroll
        for (int a = 0; a < 4; a++)
#pragma unroll
            for (int m = 0; m < V4; m++) v[a][m] = src[a][threadIdx.x + m * kLeafThreads];
#pragma unroll
        for (int a = 0; a < 4; a++)
#pragma unroll
            for (int m = 0; m < V4; m++) {
                const int e = 4 * (threadIdx.x + m * kLeafThreads);
                // four consecutive entries of one row (M) or column (N)
                *reinterpret_cast<float4 *>(dst[a] + (e / MB) * LD + e % MB) = v[a][m];
            }
    }
    for (int i = threadIdx.x; i < MB; i += kLeafThreads) {
        const float dr = DIAG[r0 + i], dc = DIAG[c0 + i];
        drow[i] = dr;
        dcol[i] = dc;
        srow[i] = dr > 0.f ? 1.f : -1.f;
        scol[i] = (i < bj) ? (dc > 0.f ? 1.f : -1.f) : 1.f;
    }
    __syncthreads();

    // seeds: block sums (their K range includes the diagonal blocks K = I
    // and K = J, so they already hold the in-block products of the known
    // blocks: U_II T_IJ - T_IJ U_JJ for opposite signs in mode 0, E_II T_IJ -
    // T_IJ E_JJ and E_II U0_IJ + U0_IJ E_JJ in mode 1; terms with the unknown
    // V_IJ vanish, its slices being still zero), summed into acc above, and
    // the base terms.
    {
#pragma unroll
        for (int m = 0; m < EPT; m++) {
            const int q = q0 + m * QS;
            const float b0 = VR[p * LD + q], b1 = VC[q * LD + p];
            float c = 0.f;
            if (q < bj) {
                if (opp[m]) c = (MODE == 0 ? b0 * (srow[p] - scol[q]) : -b0) + acc[m];
                else c = (MODE == 0) ? -acc[m] : -b1 - acc[m];
            }
            VR[p * LD + q] = c;
            VC[q * LD + p] = 0.f;
        }
    }
    __syncthreads();

    // In-tile solve (Algorithm 6, 1x1 case) by 16 x 16 sub-blocks: entry
    // (p, q) needs the entries below it in its column and left of it in its
    // row, so sub-block (a, b) (rows 16a.., columns 16b..) needs the
    // sub-blocks below and left of it, and phase s = (3 - a) + b holds up to
    // four independent sub-blocks.  A phase first adds the sums over the solved
    // sub-blocks -- the column parts into VC, the row parts into the seeds in
    // VR, register-blocked 4 x 2 and 2 x 4 -- then one warp per sub-block
    // solves it (subblock_solve).
    const int warp = threadIdx.x / 32, lane = threadIdx.x % 32;
    for (int s = 0; s < 2 * kNSub - 1; s++) {
        const int blo = max(0, s - (kNSub - 1)), nblk = min(kNSub - 1, s) - blo + 1;
        if (s > 0) {
            for (int it = threadIdx.x; it < 64 * nblk; it += kLeafThreads) {
                const int b = blo + it / 64, w = it % 64, a = kNSub - 1 - s + b;
                const int R0 = a * kSub, C0 = b * kSub;
                if (w < 32) {
                    // column parts of rows R0+4mr.. x columns C0+2mc..: sum over k >= 16(a+1)
                    const int P = R0 + 4 * (w % 4), Q = C0 + 2 * (w / 4);
                    float acc[4][2] = {};
                    const float *mrow[4][2];
#pragma unroll
                    for (int i = 0; i < 4; i++)
#pragma unroll
                        for (int j = 0; j < 2; j++) mrow[i][j] = (scol[Q + j] > 0.f ? Mp : Mm) + (P + i) * LD;
                    for (int k = R0 + kSub; k < MB; k += 4) {
                        const float4 v0 = *reinterpret_cast<const float4 *>(VC + Q * LD + k);
                        const float4 v1 = *reinterpret_cast<const float4 *>(VC + (Q + 1) * LD + k);
#pragma unroll
                        for (int i = 0; i < 4; i++) {
                            const float4 x0 = *reinterpret_cast<const float4 *>(mrow[i][0] + k);
                            const float4 x1 = *reinterpret_cast<const float4 *>(mrow[i][1] + k);
                            acc[i][0] = fmaf(x0.x, v0.x, fmaf(x0.y, v0.y, fmaf(x0.z, v0.z, fmaf(x0.w, v0.w, acc[i][0]))));
                            acc[i][1] = fmaf(x1.x, v1.x, fmaf(x1.y, v1.y, fmaf(x1.z, v1.z, fmaf(x1.w, v1.w, acc[i][1]))));
                        }
                    }
#pragma unroll
                    for (int i = 0; i < 4; i++)
#pragma unroll
                        for (int j = 0; j < 2; j++) VC[(Q + j) * LD + P + i] = acc[i][j];
                } else {
                    // row parts of rows R0+2mr.. x columns C0+4mc..: sum over k < 16b
                    const int m = w - 32;
                    const int P = R0 + 2 * (m % 8), Q = C0 + 4 * (m / 8);
                    float acc[2][4] = {};
                    const float *ncol[2][4];
#pragma unroll
                    for (int i = 0; i < 2; i++)
#pragma unroll
                        for (int j = 0; j < 4; j++) ncol[i][j] = (srow[P + i] > 0.f ? Np : Nm) + (Q + j) * LD;
                    for (int k = 0; k < C0; k += 4) {
                        const float4 v0 = *reinterpret_cast<const float4 *>(VR + P * LD + k);
                        const float4 v1 = *reinterpret_cast<const float4 *>(VR + (P + 1) * LD + k);
#pragma unroll
                        for (int j = 0; j < 4; j++) {
                            const float4 y0 = *reinterpret_cast<const float4 *>(ncol[0][j] + k);
                            const float4 y1 = *reinterpret_cast<const float4 *>(ncol[1][j] + k);
                            acc[0][j] = fmaf(v0.x, y0.x, fmaf(v0.y, y0.y, fmaf(v0.z, y0.z, fmaf(v0.w, y0.w, acc[0][j]))));
                            acc[1][j] = fmaf(v1.x, y1.x, fmaf(v1.y, y1.y, fmaf(v1.z, y1.z, fmaf(v1.w, y1.w, acc[1][j]))));
                        }
                    }
#pragma unroll
                    for (int i = 0; i < 2; i++)
#pragma unroll
                        for (int j = 0; j < 4; j++) VR[(P + i) * LD + Q + j] += acc[i][j];
                }
            }
            __syncthreads();
        }
        if (warp < nblk) {
            const int b = blo + warp, a = kNSub - 1 - s + b;
            if (b * kSub < bj) subblock_solve(Mp, Mm, Np, Nm, VC, VR, srow, scol, drow, dcol, a * kSub, b * kSub, lane);
        }
        __syncthreads();
    }

    // V (float64) and its 16-bit splits in the blocked slice layout: row
    // slices tile (I, J) of Vr[s] (row-major), column slices tile (J, I) of
    // Vc[s] (V^T, row-major).  The split runs in fp32, of V (bf16 terms) or
    // of sigma V (fp16 terms, sigma a power of two): each remainder is exact
    const bool f16 = sigma > 0.f;
    const float sc = f16 ? sigma : 1.f;
    const size_t tr = ((size_t)I * nbk + J) * MB * MB, tc = ((size_t)J * nbk + I) * MB * MB;
    const size_t sstride = (size_t)nbk * nbk * MB * MB;
    // four consecutive entries per thread and store: column form (and V) from
    // VC, row form from VR
    for (int idx = threadIdx.x; idx < MB * MB / 4; idx += kLeafThreads) {
        const int pr = 4 * (idx % (MB / 4)), q = idx / (MB / 4);
        if (q < bj) {
            const float4 r = *reinterpret_cast<const float4 *>(VC + q * LD + pr);
            double *vo = &SGT_AT(V, ldv, r0 + pr, c0 + q);
            vo[0] = r.x; vo[1] = r.y; vo[2] = r.z; vo[3] = r.w;
            split_store4(make_float4(r.x * sc, r.y * sc, r.z * sc, r.w * sc), S, f16, Vc + tc + q * MB + pr, sstride);
        }
    }
    for (int idx = threadIdx.x; idx < MB * MB / 4; idx += kLeafThreads) {
        const int q = 4 * (idx % (MB / 4)), pr = idx / (MB / 4);
        if (q < bj) {
            // columns at or beyond bj stay zero: a partial group keeps them so
            float4 r = *reinterpret_cast<const float4 *>(VR + pr * LD + q);
            if (q + 1 >= bj) r.y = 0.f;
            if (q + 2 >= bj) r.z = 0.f;
            if (q + 3 >= bj) r.w = 0.f;
            split_store4(make_float4(r.x * sc, r.y * sc, r.z * sc, r.w * sc), S, f16, Vr + tr + pr * MB + q, sstride);
        }
    }
}

// Correction on the diagonal blocks: the recurrences above restricted to one
// block, by anti-diagonal, float64.
__global__ void __launch_bounds__(kLeafThreads)
corr_diag_leaf_kernel(int n, const double *__restrict__ T, int ldt, const double *__restrict__ U0, int ldu0,
                      const double *__restrict__ Rc, const double *__restrict__ Rs, int ldr, double *__restrict__ E,
                      int lde)
{
    constexpr int LD = MB + 1;
    extern __shared__ double dsm[];
    double *Ts = dsm;
    double *Us = Ts + MB * LD;
    double *Es = Us + MB * LD;
    const int r0 = blockIdx.x * MB;
    const int bs = min(MB, n - r0);
    for (int idx = threadIdx.x; idx < bs * bs; idx += kLeafThreads) {
        const int i = idx % bs, j = idx / bs;
        Ts[i + j * LD] = (i <= j) ? SGT_AT(T, ldt, r0 + i, r0 + j) : 0.0;
        Us[i + j * LD] = (i <= j) ? SGT_AT(U0, ldu0, r0 + i, r0 + j) : 0.0;
        Es[i + j * LD] = 0.0;
    }
    __syncthreads();
    for (int dd = 1; dd < bs; dd++) {
        for (int i = threadIdx.x; i < bs - dd; i += kLeafThreads) {
            const int j = i + dd;
            const double si = Ts[i + i * LD] > 0.0 ? 1.0 : -1.0, sj = Ts[j + j * LD] > 0.0 ? 1.0 : -1.0;
            double e;
            if (si + sj == 0.0) {
                double s = -SGT_AT(Rc, ldr, r0 + i, r0 + j);
                for (int k = i + 1; k < j; k++) s += Es[i + k * LD] * Ts[k + j * LD] - Ts[i + k * LD] * Es[k + j * LD];
                e = s / (Ts[i + i * LD] - Ts[j + j * LD]);
            } else {
                double s = -SGT_AT(Rs, ldr, r0 + i, r0 + j);
                for (int k = i + 1; k < j; k++) s -= Us[i + k * LD] * Es[k + j * LD] + Es[i + k * LD] * Us[k + j * LD];
                e = s / (si + sj);
            }
            Es[i + j * LD] = e;
        }
        __syncthreads();
    }
    for (int idx = threadIdx.x; idx < bs * bs; idx += kLeafThreads) {
        const int i = idx % bs, j = idx / bs;
        if (i < j) SGT_AT(E, lde, r0 + i, r0 + j) = Es[i + j * LD];
    }
}

// ------------------------------------------------------------- residual ---

// Residual of entry (i < j) into R (column-major n x n): Rc_ij when the signs
// of i and j differ, Rs_ij when they agree, from the gathered products
// (RA: Y at equal-sign positions, N_T N_U at opposite-sign ones; RB: N_U N_T)
// plus the diagonal terms.  Only the strictly upper part of R is written: the
// correction reads nothing else.  Squared Frobenius norms of the used Rc and
// Rs entries, of T and of U into norms[0..3].
__global__ void needed_finalize_kernel(int n, const double *__restrict__ T, int ldt, const double *__restrict__ U,
                                       int ldu, const int *__restrict__ gmap, const double *__restrict__ RA,
                                         const double *__restrict__ RB, int ldg, double *__restrict__ R,
                                         double *__restrict__ norms)
{
    const int j = blockIdx.x;
    double nc = 0.0, ns = 0.0, nt = 0.0, nu = 0.0;
    const double tjj = SGT_AT(T, ldt, j, j), ujj = SGT_AT(U, ldu, j, j);
    const size_t gj = (size_t)gmap[j] * ldg;
    for (int i = threadIdx.x; i < j; i += blockDim.x) {
        const double tii = SGT_AT(T, ldt, i, i), uii = SGT_AT(U, ldu, i, i);
        const double tij = SGT_AT(T, ldt, i, j), uij = SGT_AT(U, ldu, i, j);
        const size_t g = (size_t)gmap[i] + gj;
        double r;
        if ((tii > 0.0) == (tjj > 0.0)) {
            r = RA[g] + uii * uij + uij * ujj;
            ns += r * r;
        } else {
            r = RA[g] - RB[g] + (tii * uij - uij * tjj) + (tij * ujj - uii * tij);
            nc += r * r;
        }
        nt += tij * tij;
        nu += uij * uij;
        SGT_AT(R, n, i, j) = r;
    }
    if (threadIdx.x == 0) {
        nt += tjj * tjj;
        nu += ujj * ujj;
    }
    __shared__ double red[4][256];
    red[0][threadIdx.x] = nc; red[1][threadIdx.x] = ns; red[2][threadIdx.x] = nt; red[3][threadIdx.x] = nu;
    __syncthreads();
    for (int off = blockDim.x / 2; off > 0; off >>= 1) {
        if (threadIdx.x < off)
            for (int c = 0; c < 4; c++) red[c][threadIdx.x] += red[c][threadIdx.x + off];
        __syncthreads();
    }
    if (threadIdx.x == 0)
        for (int c = 0; c < 4; c++) atomicAdd(&norms[c], red[c][0]);
}

// Full residuals, in place: Ptu -> Rc, Puu -> Rs (i < j; other entries 0),
// and the squared Frobenius norms of Rc, Rs (all entries), T, U into
// norms[0..3].
__global__ void residual_finalize_kernel(int n, const double *__restrict__ T, int ldt, const double *__restrict__ U,
                                         int ldu, double *__restrict__ Ptu, const double *__restrict__ Put,
                                         double *__restrict__ Puu, int ldp, double *__restrict__ norms)
{
    const int j = blockIdx.x;
    double nc = 0.0, ns = 0.0, nt = 0.0, nu = 0.0;
    const double tjj = SGT_AT(T, ldt, j, j), ujj = SGT_AT(U, ldu, j, j);
    for (int i = threadIdx.x; i < n; i += blockDim.x) {
        double rc = 0.0, rs = 0.0;
        if (i < j) {
            const double tii = SGT_AT(T, ldt, i, i), uii = SGT_AT(U, ldu, i, i);
            const double tij = SGT_AT(T, ldt, i, j), uij = SGT_AT(U, ldu, i, j);
            rc = SGT_AT(Ptu, ldp, i, j) - SGT_AT(Put, ldp, i, j) + (tii * uij - uij * tjj) + (tij * ujj - uii * tij);
            rs = SGT_AT(Puu, ldp, i, j) + uii * uij + uij * ujj;
            nt += tij * tij;
            nu += uij * uij;
        } else if (i == j) {
            nt += tjj * tjj;
            nu += ujj * ujj;
        }
        SGT_AT(Ptu, ldp, i, j) = rc;
        SGT_AT(Puu, ldp, i, j) = rs;
        nc += rc * rc;
        ns += rs * rs;
    }
    __shared__ double red[4][256];
    red[0][threadIdx.x] = nc; red[1][threadIdx.x] = ns; red[2][threadIdx.x] = nt; red[3][threadIdx.x] = nu;
    __syncthreads();
    for (int off = blockDim.x / 2; off > 0; off >>= 1) {
        if (threadIdx.x < off)
            for (int c = 0; c < 4; c++) red[c][threadIdx.x] += red[c][threadIdx.x + off];
        __syncthreads();
    }
    if (threadIdx.x == 0)
        for (int c = 0; c < 4; c++) atomicAdd(&norms[c], red[c][0]);
}

// sign flags of the diagonal (1 = positive)
__global__ void diag_sign_kernel(int n, const double *__restrict__ T, int ldt, unsigned char *__restrict__ pos)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) pos[i] = SGT_AT(T, ldt, i, i) > 0.0 ? 1 : 0;
}

// U += E on the strictly upper part; ||E||_F^2 into norms[4].
__global__ void apply_correction_kernel(int n, double *__restrict__ U, int ldu, const double *__restrict__ E, int lde,
                                        double *__restrict__ norms)
{
    const int j = blockIdx.x;
    double ne = 0.0;
    for (int i = threadIdx.x; i < j; i += blockDim.x) {
        const double e = SGT_AT(E, lde, i, j);
        SGT_AT(U, ldu, i, j) += e;
        ne += e * e;
    }
    __shared__ double red[256];
    red[threadIdx.x] = ne;
    __syncthreads();
    for (int off = blockDim.x / 2; off > 0; off >>= 1) {
        if (threadIdx.x < off) red[threadIdx.x] += red[threadIdx.x + off];
        __syncthreads();
    }
    if (threadIdx.x == 0) atomicAdd(&norms[4], red[0]);
}

// Rounding-split slices of the strictly upper part of the diagonal blocks
// of V (U after the float64 diagonal leaves, E after the corrections'
// diagonal leaves), in the blocked layout the leaves write: tile (I, I) of
// Vr[s] (row-major) and of Vc[s] (transposed).  bf16 terms of V (split in
// float64), or fp16 terms of sigma V (sigma > 0, split in fp32: two terms
// keep 22 bits).  One CTA per block.
__global__ void diag_slices_kernel(int n, const double *__restrict__ V, int ldv, __nv_bfloat16 *__restrict__ Vr,
                                   __nv_bfloat16 *__restrict__ Vc, int S, int nbk, float sigma)
{
    const int I = blockIdx.x, r0 = I * MB;
    const int bs = min(MB, n - r0);
    const size_t t = ((size_t)I * nbk + I) * MB * MB, sstride = (size_t)nbk * nbk * MB * MB;
    for (int idx = threadIdx.x; idx < bs * bs; idx += blockDim.x) {
        const int i = idx % bs, j = idx / bs;
        double r = (i < j) ? SGT_AT(V, ldv, r0 + i, r0 + j) : 0.0;
        if (sigma > 0.f) {
            float x = (float)(r * (double)sigma);
            for (int s = 0; s < S; s++) {
                const unsigned short h = split_term(x, true);
                Vr[s * sstride + t + i * MB + j] = __ushort_as_bfloat16(h);
                Vc[s * sstride + t + j * MB + i] = __ushort_as_bfloat16(h);
            }
            continue;
        }
        for (int s = 0; s < S; s++) {
            const __nv_bfloat16 h = __double2bfloat16(r);
            Vr[s * sstride + t + i * MB + j] = h;
            Vc[s * sstride + t + j * MB + i] = h;
            r -= (double)__bfloat162float(h);
        }
    }
}

// Rounding-split slices (of the fp32 value, as the leaves split: bf16 terms,
// or fp16 terms of sigma M when sigma > 0) of the strictly upper part of the
// n x n matrix M in the blocked layout: tile (I, K) of R[s] (row-major) and
// tile (K, I) of C[s] (transposed) for every block K >= I; the blocks below
// are never read and not written.
__global__ void blocked_split_kernel(int n, const double *__restrict__ M, int ldm, int S, int nbk,
                                     __nv_bfloat16 *__restrict__ R, __nv_bfloat16 *__restrict__ C, float sigma)
{
    __shared__ float tile[MB][MB + 1];   // [column][row]
    const int K = blockIdx.x, I = blockIdx.y;
    if (K < I) return;
    const bool f16 = sigma > 0.f;
    const double sc = f16 ? (double)sigma : 1.0;
    const size_t sstride = (size_t)nbk * nbk * MB * MB;
    const size_t tr = ((size_t)I * nbk + K) * MB * MB, tc = ((size_t)K * nbk + I) * MB * MB;
    for (int idx = threadIdx.x; idx < MB * MB; idx += blockDim.x) {
        const int r = idx % MB, k = idx / MB;
        const int gi = I * MB + r, gk = K * MB + k;
        const float v = (gi < gk && gk < n) ? (float)(SGT_AT(M, ldm, gi, gk) * sc) : 0.f;
        tile[k][r] = v;
        float x = v;
        for (int s = 0; s < S; s++) C[s * sstride + tc + k * MB + r] = __ushort_as_bfloat16(split_term(x, f16));
    }
    __syncthreads();
    for (int idx = threadIdx.x; idx < MB * MB; idx += blockDim.x) {
        const int k = idx % MB, r = idx / MB;
        float x = tile[k][r];
        for (int s = 0; s < S; s++) R[s * sstride + tr + r * MB + k] = __ushort_as_bfloat16(split_term(x, f16));
    }
}

// Largest |entry| of the strictly upper parts of the 64 x 64 diagonal blocks
// of the n x n matrix M, as the bits of a non-negative float (ordered like
// the values) max-ed into *out.
__global__ void absmax_diag_blocks_kernel(int n, const double *__restrict__ M, int ldm, unsigned *__restrict__ out)
{
    float m = 0.f;
    const long long total = (long long)((n + MB - 1) / MB) * MB * MB;
    for (long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x; e < total;
         e += (long long)gridDim.x * blockDim.x) {
        const int b = (int)(e / (MB * MB)), w = (int)(e % (MB * MB));
        const int i = b * MB + w % MB, j = b * MB + w / MB;
        if (i < j && j < n) m = fmaxf(m, fabsf(f64_to_f32_trunc(SGT_AT(M, ldm, i, j))));
    }
    for (int o = 16; o > 0; o >>= 1) m = fmaxf(m, __shfl_xor_sync(0xffffffffu, m, o));
    if ((threadIdx.x & 31) == 0) atomicMax(out, __float_as_uint(m));
}

// Largest of `count` non-negative float64 values held as their bits (the
// per-row maxima the exact slices' scales come from), as float bits max-ed
// into *out.
__global__ void max_of_maxima_kernel(int count, const unsigned long long *__restrict__ bits, unsigned *__restrict__ out)
{
    float m = 0.f;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < count; i += gridDim.x * blockDim.x)
        m = fmaxf(m, (float)__longlong_as_double((long long)bits[i]));
    for (int o = 16; o > 0; o >>= 1) m = fmaxf(m, __shfl_xor_sync(0xffffffffu, m, o));
    if ((threadIdx.x & 31) == 0) atomicMax(out, __float_as_uint(m));
}

// Largest first-order correction term |e_ij| ~ |Rc_ij| / |t_ii - t_jj|
// (signs differ) or |Rs_ij| / 2 (signs agree) over the strictly upper
// entries, max-ed into *out as float bits (see absmax_diag_blocks_kernel).
// D: t_ii in fp32.  One column per CTA step: coalesced reads of R and D.
__global__ void corr_magnitude_kernel(int n, const float *__restrict__ D, const double *__restrict__ Rc,
                                      const double *__restrict__ Rs, int ldr, unsigned *__restrict__ out)
{
    float m = 0.f;
    for (int j = blockIdx.x; j < n; j += gridDim.x) {
        const float tj = D[j];
        for (int i = threadIdx.x; i < j; i += blockDim.x) {
            const float ti = D[i];
            // fp32 magnitudes truncated from the bits (no float64 conversion)
            const float v = ((ti > 0.f) != (tj > 0.f)) ? fabsf(f64_to_f32_trunc(SGT_AT(Rc, ldr, i, j))) / fabsf(ti - tj)
                                                       : 0.5f * fabsf(f64_to_f32_trunc(SGT_AT(Rs, ldr, i, j)));
            m = fmaxf(m, v);
        }
    }
    for (int o = 16; o > 0; o >>= 1) m = fmaxf(m, __shfl_xor_sync(0xffffffffu, m, o));
    if ((threadIdx.x & 31) == 0) atomicMax(out, __float_as_uint(m));
}

__global__ void fill_float_kernel(int count, float v, float *__restrict__ p)
{
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < count; i += gridDim.x * blockDim.x) p[i] = v;
}

// ---------------------------------------------------------- probe check ---
// Acceptance test by random probes: for Z (n x kProbes) with independent +-1
// entries, E ||R Z||_F^2 = kProbes ||R||_F^2 for any R, so
// ||R Z||_F / sqrt(kProbes) estimates ||R||_F.  R Z = T (U Z) - U (T Z) and
// U (U Z) - Z are formed with the emulated-float64 products of the full
// residual (n x n by n x kProbes), about 2^-45 |T||U| entrywise.
constexpr int kProbes = 128;

__device__ __forceinline__ unsigned long long splitmix64(unsigned long long x)
{
    x += 0x9e3779b97f4a7c15ull;
    x = (x ^ (x >> 30)) * 0xbf58476d1ce4e5b9ull;
    x = (x ^ (x >> 27)) * 0x94d049bb133111ebull;
    return x ^ (x >> 31);
}

// Z[i + j n] = +-1 (bit of a counter hash), its one bf16 column slice
// Zc[j][i] = +-64 with column scale 2 (+-1 = 2 * 64 * 2^-7 exactly), zero
// padding up to np.
__global__ void probe_kernel(int n, int np, unsigned long long seed, double *__restrict__ Z,
                             __nv_bfloat16 *__restrict__ Zc, float *__restrict__ zscale)
{
    const int j = blockIdx.y;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < np; i += gridDim.x * blockDim.x) {
        float z = 0.f;
        if (i < n) {
            z = (splitmix64(seed ^ ((unsigned long long)j << 32 ^ (unsigned long long)i)) >> 63) ? -1.f : 1.f;
            Z[(size_t)i + (size_t)j * n] = (double)z;
        }
        Zc[(size_t)j * np + i] = __float2bfloat16_rn(64.f * z);
    }
    if (blockIdx.x == 0 && threadIdx.x == 0) zscale[j] = 2.f;
}

// W = Pa + Pb + diag(M) Y  (n x kProbes, column-major, ld n)
__global__ void probe_combine_kernel(int n, const double *__restrict__ Pa, const double *__restrict__ Pb,
                                     const double *__restrict__ M, int ldm, const double *__restrict__ Y,
                                     double *__restrict__ W)
{
    const int j = blockIdx.y;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        const size_t e = (size_t)i + (size_t)j * n;
        W[e] = Pa[e] + Pb[e] + SGT_AT(M, ldm, i, i) * Y[e];
    }
}

// R_c Z = N_T W1 + diag(T) W1 - N_U W2 - diag(U) W2 and R_s Z = N_U W1 +
// diag(U) W1 - Z, squared norms into norms[0], norms[1] (each product as two
// K halves a, b).
__global__ void probe_residual_kernel(int n, const double *__restrict__ T, int ldt, const double *__restrict__ U,
                                      int ldu, const double *__restrict__ Z, const double *__restrict__ W1,
                                      const double *__restrict__ W2, const double *__restrict__ P1a,
                                      const double *__restrict__ P1b, const double *__restrict__ P2a,
                                      const double *__restrict__ P2b, const double *__restrict__ P3a,
                                      const double *__restrict__ P3b, double *__restrict__ norms)
{
    const int j = blockIdx.y;
    double nc = 0.0, ns = 0.0;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        const size_t e = (size_t)i + (size_t)j * n;
        const double tii = SGT_AT(T, ldt, i, i), uii = SGT_AT(U, ldu, i, i);
        const double rc = (P1a[e] + P1b[e]) + tii * W1[e] - (P2a[e] + P2b[e]) - uii * W2[e];
        const double rs = (P3a[e] + P3b[e]) + uii * W1[e] - Z[e];
        nc += rc * rc;
        ns += rs * rs;
    }
    __shared__ double red[2][256];
    red[0][threadIdx.x] = nc;
    red[1][threadIdx.x] = ns;
    __syncthreads();
    for (int off = blockDim.x / 2; off > 0; off >>= 1) {
        if (threadIdx.x < off) {
            red[0][threadIdx.x] += red[0][threadIdx.x + off];
            red[1][threadIdx.x] += red[1][threadIdx.x + off];
        }
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        atomicAdd(&norms[0], red[0][0]);
        atomicAdd(&norms[1], red[1][0]);
    }
}

__global__ void zero_kernel(size_t count, double *__restrict__ p)
{
    for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < count; i += (size_t)gridDim.x * blockDim.x)
        p[i] = 0.0;
}

// ------------------------------------------------------------ host side ---

// A schedule's device copy (job list, per-CTA job ranges, per-tile slots).
struct DevSchedule {
    TcJob *jobs = nullptr;
    int *cta_off = nullptr;
    int2 *tslot = nullptr;
};

struct MixedCtx {
    int n, np, S;
    // fp16 split (S = 2): T, U and E are split as sT T, sU U, sE E (powers of
    // two), and the products' rows and columns scaled back by invT, invU,
    // invE (np + 64 entries, constant); sT = sU = sE = 0 for the bf16 splits
    bool f16;
    float sT, sU, sE;
    float *invT, *invU, *invE;
    unsigned *amax;             // float bits of a maximum the fp16 scales come from
    cudaStream_t st;
    int *d_err;
    Schedule sc, sc2;           // initial sweep; correction (two launches side by side)
    DevSchedule ds, ds2;
    Schedule scA, scB, scC;     // initial sweep's look-ahead pairs: lead, look-ahead, completion
    DevSchedule dsA, dsB, dsC;
    cudaStream_t side;          // second stream of the correction launches (null: one stream)
    cudaEvent_t ev_fork, ev_join;
    TcPairs pairs_split, pairs_oz;
    TcPairs *d_pairs_split, *d_pairs_oz;
    // bf16 splits (S slices) of T and of the unknowns, row and column forms,
    // blocked layout (each 64 x 64 tile contiguous)
    __nv_bfloat16 *Tr, *Tc, *Ur, *Uc, *Er, *Ec;
    float *OPS, *DIAG;          // per-sign fp32 operators of the diagonal blocks for the leaves, fp32 diagonal
    // exact slices of the strictly upper parts of T and U in the gathered
    // layout (residual products): ng gathered positions, rows_g allocated
    // (the last 64 all zero), pitch rows_g
    int ng, rows_g;
    int *gmap, *ginv;           // original -> gathered, gathered -> original (-1 padding)
    int *sbbase;                // gathered start of each superblock (nsb + 1 entries)
    unsigned char *pos;         // diagonal sign flags
    __nv_bfloat16 *NTgr, *NTgc;         // T, gathered layout
    __nv_bfloat16 *NTr, *NTc;           // T, original layout
    __nv_bfloat16 *NUr, *NUc;           // U, either layout (sized for the gathered one)
    float *sTr, *sTc, *sUr, *sUc;       // scales, original indices
    float *gTr, *gTc, *gUr, *gUc;       // scales, gathered
    unsigned long long *tmpmax, *tmpmax2;
    double *PA, *PB;            // block-sum partials
    double *E;                  // correction
    // residual products: gathered RA, RB or full-layout Ptu -> Rc, Put (same
    // memory); R = Rs (full) or the per-entry residual (needed form)
    double *RA, *RB, *R;
    const double *res_c, *res_s;   // what the last residual left for the correction
    double *norms, *norms_host; // [0] Rc^2 [1] Rs^2 [2] T^2 [3] U^2 [4] E^2
    // probe check: Z, its slice and scale, W1 = U Z, W2 = T Z and their
    // slices and scales, the product halves, the jobs (row pairs x K halves)
    double *Z, *W1, *W2, *Pp;
    __nv_bfloat16 *Zc, *W1c, *W2c;
    float *zscale, *w1scale, *w2scale;
    TcJob *d_probe_jobs;
    int n_probe_jobs;
    double probe_kb;
    TcPairs pairs_z;            // (s, 0): Z has one slice
    TcPairs *d_pairs_z;
    double nT2, nU2;            // squared norms of T and U from the last needed residual
    TcJob *d_full_jobs;         // full residual: 2 x 2 block jobs
    int n_full_jobs;
    double full_kb;             // sum over full jobs of used quadrants x K-blocks
    TcJob *d_res_jobs;          // needed residual: equal-sign jobs, then opposite-sign jobs
    int n_res_same, n_res_opp;
    double res_kb_same, res_kb_opp;   // sum over jobs of used quadrants x K-blocks
};

// Gathered size bound: each superblock pads two sign classes to 64.
int gathered_bound(int n) { return pad64(n) + 128 * ((n + kSuper - 1) / kSuper); }

size_t bytes_for(int n, int S)
{
    const size_t np = (size_t)pad64(n);
    const size_t nb = np / MB;
    size_t b = 0;
    b += 6 * (size_t)S * np * np * 2 + 6 * 256;                       // split slices
    const size_t ngr = (size_t)gathered_bound(n) + 64;
    b += 4 * (size_t)kOzakiSlices * ngr * ngr * 2 + 4 * 256;           // exact slices: T gathered, U
    b += 2 * (size_t)kOzakiSlices * (np + 64) * np * 2 + 2 * 256;      // exact slices: T original
    b += 4 * (np + 64) * 4 + 2 * (np + 64) * 8 + 7 * 256;               // scales, tmp
    b += 4 * ngr * 4 + 4 * 256 + 2 * ngr * 4 + np + 3 * 256;            // gathered scales, maps, signs
    b += ((size_t)(n + kSuper - 1) / kSuper + 1) * 4 + 256;             // superblock starts
    b += 2 * ngr * ngr * 8 + 2 * 256;                                   // RA, RB
    const size_t maxjobs = (size_t)kSweepCtas + 2 * nb + 8;
    b += 2 * maxjobs * 16384 * 8 + 2 * 256;                             // partials
    b += 2 * (size_t)n * n * 8 + 2 * 256;                               // E, R (= Rs)
    b += 64 + 256;                                                      // norms
    b += 4 * nb * MB * MB * sizeof(float) + nb * MB * sizeof(float) + 2 * 256;   // leaf operators, diagonal
    b += 3 * (np + 64) * sizeof(float) + 64 + 4 * 256;                  // fp16 split scales, max slot
    const size_t pairs_max = ngr / 128 + 2 * (size_t)((n + kSuper - 1) / kSuper) + 2;
    b += pairs_max * pairs_max * sizeof(TcJob) + 256;                   // needed-residual jobs
    const size_t nbp = (nb + 1) / 2;
    b += nbp * (nbp + 1) / 2 * sizeof(TcJob) + 256;                     // full-residual jobs
    b += 5 * (nb * (size_t)(kSweepCtas + 2 * nb) * sizeof(TcJob) + 256); // wavefront jobs (bound), 5 schedules
    b += 5 * (nb * (size_t)(kSweepCtas + 1) * sizeof(int) + 256);         // per-CTA job ranges
    b += 5 * ((size_t)nb * nb * sizeof(int2) + 256);                      // per-tile partial slots
    b += 3 * sizeof(TcPairs) + 768;
    b += 13 * (size_t)n * kProbes * 8 + 4 * 256;                       // probe Z, W1, W2, product halves
    b += (1 + 2 * (size_t)kOzakiSlices) * kProbes * np * 2 + 3 * 256;  // their slices
    b += 3 * kProbes * 4 + (2 * nbp + 2) * sizeof(TcJob) + 4 * 256;     // scales, probe jobs
    return b;
}

template <typename P>
P *take(Arena &ws, size_t count)
{
    return static_cast<P *>(ws.take(count * sizeof(P)));
}

// 2^(target - floor(log2 m)) for m > 0: scales m into [2^target, 2^(target+1)).
float pow2_scale(float m, int target)
{
    int e = 0;
    std::frexp(m, &e);   // m = f 2^e, f in [0.5, 1)
    return std::ldexp(1.f, std::max(-120, std::min(120, target - (e - 1))));
}

// Reads back the float max-ed into c.amax (the host waits for it).
signtri_status read_amax(MixedCtx &c, float &m)
{
    unsigned bits = 0;
    SGT_CUDA_TRY(cudaMemcpyAsync(&bits, c.amax, sizeof(unsigned), cudaMemcpyDeviceToHost, c.st));
    SGT_CUDA_TRY(cudaStreamSynchronize(c.st));
    std::memcpy(&m, &bits, sizeof(float));
    return SIGNTRI_OK;
}

// Largest |entry| of the strictly upper parts of M's diagonal blocks into m.
signtri_status diag_blocks_absmax(MixedCtx &c, const double *M, int ldm, float &m)
{
    SGT_CUDA_TRY(cudaMemsetAsync(c.amax, 0, sizeof(unsigned), c.st));
    {
        ProfScope ps(SIGNTRI_KC_CONVERT, c.st);
        absmax_diag_blocks_kernel<<<152, 256, 0, c.st>>>(c.n, M, ldm, c.amax);
        SGT_LAUNCH_CHECK();
    }
    return read_amax(c, m);
}

// Largest of the per-row maxima in c.tmpmax (np + 64 entries) into m.
signtri_status row_maxima_max(MixedCtx &c, float &m)
{
    SGT_CUDA_TRY(cudaMemsetAsync(c.amax, 0, sizeof(unsigned), c.st));
    {
        ProfScope ps(SIGNTRI_KC_CONVERT, c.st);
        max_of_maxima_kernel<<<32, 256, 0, c.st>>>(c.np + 64, c.tmpmax, c.amax);
        SGT_LAUNCH_CHECK();
    }
    return read_amax(c, m);
}

// inv[0 .. np + 64) = 1 / sigma: the engine's row / column scales of a product
// whose operand was split as sigma M
signtri_status fill_inverse(MixedCtx &c, float *inv, float sigma)
{
    ProfScope ps(SIGNTRI_KC_FILL, c.st);
    fill_float_kernel<<<8, 256, 0, c.st>>>(c.np + 64, 1.f / sigma, inv);
    SGT_LAUNCH_CHECK();
    return SIGNTRI_OK;
}

// Blocked-layout rounding splits of the strictly upper part of M (row and
// column forms) for the sweeps.
signtri_status split_full(MixedCtx &c, const double *M, int ldm, __nv_bfloat16 *R, __nv_bfloat16 *C, float sigma)
{
    if (c.S > 8) return SIGNTRI_ERR_BAD_ARG;
    const int nbk = c.np / MB;
    ProfScope ps(SIGNTRI_KC_CONVERT, c.st);
    blocked_split_kernel<<<dim3(nbk, nbk), 256, 0, c.st>>>(c.n, M, ldm, c.S, nbk, R, C, sigma);
    SGT_LAUNCH_CHECK();
    return SIGNTRI_OK;
}

// One low-precision sweep: MODE 0 solves for U (into V = U), MODE 1 for E.
template <int MODE>
signtri_status sweep(MixedCtx &c, const double *T, int ldt, double *V, int ldv, __nv_bfloat16 *Vr,
                     __nv_bfloat16 *Vc, const double *U0, int ldu0)
{
    const int n = c.n, nb = c.sc.nb;
    const size_t leaf_smem = (size_t)kLeafBufs * MB * kLeafLD * sizeof(float);
    SGT_CUDA_TRY(cudaFuncSetAttribute(mixed_leaf_kernel<MODE>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                      (int)leaf_smem));
    SGT_CUDA_TRY(cudaFuncSetAttribute(mixed_leaf_kernel<MODE>, cudaFuncAttributePreferredSharedMemoryCarveout,
                                      cudaSharedmemCarveoutMaxShared));   // two leaves per SM
    {
        // the leaves' per-sign fp32 operators of the diagonal blocks, built
        // from T and the known blocks the same-sign recurrences use (U in
        // mode 0, U0 in mode 1)
        ProfScope ps(MODE == 0 ? SIGNTRI_KC_OFFDIAG_LEAF_F32 : SIGNTRI_KC_CORRECTION, c.st);
        leaf_ops_kernel<<<nb, 256, 0, c.st>>>(n, T, ldt, MODE == 0 ? V : U0, MODE == 0 ? ldv : ldu0, c.OPS, c.DIAG);
        SGT_LAUNCH_CHECK();
    }
    // slices in the blocked layout: every 64 x 64 tile one contiguous 8 KB run
    // fp16 splits carry their scales: the engine scales the products back
    const int h = c.f16 ? 1 : 0;
    const float *iT = c.f16 ? c.invT : nullptr, *iU = c.f16 ? c.invU : nullptr;
    const float *iV = c.f16 ? (MODE == 0 ? c.invU : c.invE) : nullptr;
    const TcSource srcT_r{c.Tr, c.S, c.np, c.np, c.np, iT, 1, h}, srcT_c{c.Tc, c.S, c.np, c.np, c.np, iT, 1, h};
    const TcSource srcV_r{Vr, c.S, c.np, c.np, c.np, iV, 1, h}, srcV_c{Vc, c.S, c.np, c.np, c.np, iV, 1, h};
    const TcSource srcU_r{c.Ur, c.S, c.np, c.np, c.np, iU, 1, h}, srcU_c{c.Uc, c.S, c.np, c.np, c.np, iU, 1, h};
    const TcQuadOut slots{{nullptr, nullptr, nullptr, nullptr}, 0, 0, 0};
    // K-blocks per tensor-core unit: with several unit-weight slice pairs the
    // engine keeps every slice of a K-block resident and accumulates all pairs
    // into one unit, so 2 K-blocks keep each fp32 accumulation short; a single
    // pair takes long units
    const int chunk = c.pairs_split.n > 1 ? 2 : 16;
    // the correction's two launches per anti-diagonal run side by side on
    // their own half-width schedule when a second stream is available; so do
    // the initial sweep's look-ahead pairs
    const bool pair = (MODE == 1) && c.side != nullptr;
    const bool look = (MODE == 0) && c.side != nullptr;
    const Schedule &sc = pair ? c.sc2 : c.sc;
    const DevSchedule &ds = pair ? c.ds2 : c.ds;
    const TcJob *d_jobs = ds.jobs;
    const int *d_coff = ds.cta_off;
    const int2 *d_tslot = ds.tslot;
    const double kb_bytes = (double)c.S * MB * MB * 2;   // one 64-row panel of S bf16 slices, one K-block
    auto fork = [&]() -> signtri_status {
        SGT_CUDA_TRY(cudaEventRecord(c.ev_fork, c.st));
        SGT_CUDA_TRY(cudaStreamWaitEvent(c.side, c.ev_fork, 0));
        return SIGNTRI_OK;
    };
    auto join = [&]() -> signtri_status {
        SGT_CUDA_TRY(cudaEventRecord(c.ev_join, c.side));
        SGT_CUDA_TRY(cudaStreamWaitEvent(c.st, c.ev_join, 0));
        return SIGNTRI_OK;
    };
    for (int d = 1; d < nb; d++) {
        const int ntiles = nb - d;
        const long long sum_kb = (long long)ntiles * (d + 1);
        const int2 *leaf_slots = d_tslot + sc.tile_begin[d];
        const int2 *leaf_slots2 = nullptr;
        signtri_status rs;
        if (MODE == 0 && look && look_lead(d, nb)) {
            // lead: anti-diagonal d in full beside the look-ahead sums of d + 1
            const Schedule &A = c.scA, &B = c.scB;
            const int e = d + 1, ne = nb - e;
            const long long look_kb = (long long)ne * (d - 2);
            ProfScope pg(SIGNTRI_KC_BLOCK_SUMS_TC, c.st, true, false);
            const int cls = SIGNTRI_KC_BLOCK_SUMS_TC | kProfUntimed;
            if ((rs = fork()) != SIGNTRI_OK) return rs;
            rs = tc_blocksums(srcV_r, srcT_r, srcT_c, srcV_c, c.dsA.jobs + A.job_off[d], A.job_off[d + 1] - A.job_off[d],
                              c.pairs_split, c.d_pairs_split, chunk, c.PA, slots, c.d_err, cls, c.st,
                              tc_flops(c.pairs_split.n, sum_kb, 3), c.dsA.cta_off + A.cta_begin[d], A.nctas[d]);
            if (rs == SIGNTRI_OK)
                rs = tc_blocksums(srcV_r, srcT_r, srcT_c, srcV_c, c.dsB.jobs + B.job_off[e],
                                  B.job_off[e + 1] - B.job_off[e], c.pairs_split, c.d_pairs_split, chunk, c.PB, slots,
                                  c.d_err, cls, c.side, tc_flops(c.pairs_split.n, look_kb, 3),
                                  c.dsB.cta_off + B.cta_begin[e], B.nctas[e]);
            // join even after a failed launch: nothing on the side stream outlives the call
            const signtri_status rj = join();
            if (rs != SIGNTRI_OK) return rs;
            if (rj != SIGNTRI_OK) return rj;
            // the look-ahead reads its row panels from L2: only its column panels are new
            prof_add_bytes(SIGNTRI_KC_BLOCK_SUMS_TC, (4.0 * sum_kb + 2.0 * look_kb) * kb_bytes);
            leaf_slots = c.dsA.tslot + A.tile_begin[d];
        } else if (MODE == 0 && look && look_follow(d, nb)) {
            // follow: the four K-blocks per tile the look-ahead left, then the
            // leaves sum both slot sets
            const Schedule &B = c.scB, &C = c.scC;
            rs = tc_blocksums(srcV_r, srcT_r, srcT_c, srcV_c, c.dsC.jobs + C.job_off[d], C.job_off[d + 1] - C.job_off[d],
                              c.pairs_split, c.d_pairs_split, chunk, c.PA, slots, c.d_err, SIGNTRI_KC_BLOCK_SUMS_TC,
                              c.st, tc_flops(c.pairs_split.n, 4LL * ntiles, 3), c.dsC.cta_off + C.cta_begin[d],
                              C.nctas[d]);
            if (rs != SIGNTRI_OK) return rs;
            prof_add_bytes(SIGNTRI_KC_BLOCK_SUMS_TC, 4.0 * 4.0 * ntiles * kb_bytes);
            leaf_slots = c.dsC.tslot + C.tile_begin[d];
            leaf_slots2 = c.dsB.tslot + B.tile_begin[d];
        } else {
            const int njobs = sc.job_off[d + 1] - sc.job_off[d];
            const TcJob *jobs = d_jobs + sc.job_off[d];
            const int *coff = d_coff + sc.cta_begin[d];
            const int G = sc.nctas[d];
            if (njobs > 0) {
                if (MODE == 0) {
                    // [U_I.; T_I.] x [T_.J | U_.J]: TL = U T, TR = U U, BR = T U
                    rs = tc_blocksums(srcV_r, srcT_r, srcT_c, srcV_c, jobs, njobs, c.pairs_split, c.d_pairs_split,
                                      chunk, c.PA, slots, c.d_err, SIGNTRI_KC_BLOCK_SUMS_TC, c.st,
                                      tc_flops(c.pairs_split.n, sum_kb, 3), coff, G);
                    if (rs != SIGNTRI_OK) return rs;
                    prof_add_bytes(SIGNTRI_KC_BLOCK_SUMS_TC, 4.0 * sum_kb * kb_bytes);
                } else {
                    // X^E: [E_I.; T_I.] x [T_.J | E_.J]: TL = E T, BR = T E, and
                    // Y^E: [U0_I.; E_I.] x [E_.J | U0_.J]: TL = U0 E, BR = E U0.  Side by side
                    // (same split, CTA c of each on the same tiles and K-blocks at the
                    // same time) they read the E panels once: six panels for both.
                    ProfScope pg(SIGNTRI_KC_BLOCK_SUMS_TC, c.st, pair, false);
                    const int cls = pair ? (SIGNTRI_KC_BLOCK_SUMS_TC | kProfUntimed) : SIGNTRI_KC_BLOCK_SUMS_TC;
                    cudaStream_t sy = c.st;
                    if (pair) {
                        if ((rs = fork()) != SIGNTRI_OK) return rs;
                        sy = c.side;
                    }
                    rs = tc_blocksums(srcV_r, srcT_r, srcT_c, srcV_c, jobs, njobs, c.pairs_split, c.d_pairs_split,
                                      chunk, c.PA, slots, c.d_err, cls, c.st, tc_flops(c.pairs_split.n, sum_kb, 2),
                                      coff, G);
                    if (rs == SIGNTRI_OK)
                        rs = tc_blocksums(srcU_r, srcV_r, srcV_c, srcU_c, jobs, njobs, c.pairs_split,
                                          c.d_pairs_split, chunk, c.PB, slots, c.d_err, cls, sy,
                                          tc_flops(c.pairs_split.n, sum_kb, 2), coff, G);
                    const signtri_status rj = pair ? join() : SIGNTRI_OK;   // also after a failed launch
                    if (rs != SIGNTRI_OK) return rs;
                    if (rj != SIGNTRI_OK) return rj;
                    prof_add_bytes(SIGNTRI_KC_BLOCK_SUMS_TC, (pair ? 6.0 : 8.0) * sum_kb * kb_bytes);
                }
            }
        }
        ProfScope ps(MODE == 0 ? SIGNTRI_KC_OFFDIAG_LEAF_F32 : SIGNTRI_KC_CORRECTION, c.st);
        mixed_leaf_kernel<MODE><<<ntiles, kLeafThreads, leaf_smem, c.st>>>(
            n, T, ldt, V, ldv, c.OPS, c.DIAG, c.res_c, c.res_s, n, d, leaf_slots, leaf_slots2, c.PA, c.PB, Vr, Vc,
            c.S, nb, c.f16 ? (MODE == 0 ? c.sU : c.sE) : 0.f);
        SGT_LAUNCH_CHECK();
    }
    return SIGNTRI_OK;
}

// The gathered layout and the residual job lists, from the diagonal signs
// (one small device-to-host read): per superblock of kSuper indices the
// positives in order, padded to 64, then the negatives; output jobs pair two
// row blocks of one class and superblock with two column blocks of one class
// and superblock (a lone block pairs with the zero block at ng).
signtri_status setup_gathered(MixedCtx &c, const double *T, int ldt)
{
    const int n = c.n;
    {
        ProfScope ps(SIGNTRI_KC_CONVERT, c.st);
        diag_sign_kernel<<<(n + 255) / 256, 256, 0, c.st>>>(n, T, ldt, c.pos);
        SGT_LAUNCH_CHECK();
    }
    std::vector<unsigned char> pos(n);
    SGT_CUDA_TRY(cudaMemcpyAsync(pos.data(), c.pos, n, cudaMemcpyDeviceToHost, c.st));
    SGT_CUDA_TRY(cudaStreamSynchronize(c.st));
    GatheredLayout L;
    build_gathered_layout(n, pos.data(), kSuper, L);
    c.ng = L.ng;
    c.rows_g = L.rows_g;
    if (c.rows_g > gathered_bound(n) + 64) return SIGNTRI_ERR_NO_WORKSPACE;
    c.n_res_same = L.n_same;
    c.n_res_opp = L.n_opp;
    c.res_kb_same = L.kb_same;
    c.res_kb_opp = L.kb_opp;
    if (!L.jobs.empty())
        SGT_CUDA_TRY(cudaMemcpyAsync(c.d_res_jobs, L.jobs.data(), L.jobs.size() * sizeof(TcJob),
                                     cudaMemcpyHostToDevice, c.st));
    SGT_CUDA_TRY(cudaMemcpyAsync(c.gmap, L.gmap.data(), (size_t)n * sizeof(int), cudaMemcpyHostToDevice, c.st));
    SGT_CUDA_TRY(cudaMemcpyAsync(c.sbbase, L.base.data(), L.base.size() * sizeof(int), cudaMemcpyHostToDevice,
                                 c.st));
    SGT_CUDA_TRY(cudaMemcpyAsync(c.ginv, L.ginv.data(), (size_t)c.rows_g * sizeof(int), cudaMemcpyHostToDevice, c.st));
    // the host tables are pageable and local
    SGT_CUDA_TRY(cudaStreamSynchronize(c.st));
    return SIGNTRI_OK;
}

// Exact slices of the strictly upper part of M (T or U) in the gathered layout
// (scales sR, sC computed here unless `scaled`).
signtri_status gathered_slices_of(MixedCtx &c, const double *M, int ldm, __nv_bfloat16 *R, __nv_bfloat16 *C,
                                  float *sR, float *sC, float *gR, float *gC, bool scaled = false)
{
    signtri_status rs;
    if (!scaled &&
        (rs = make_scales_both(c.n, M, ldm, 1, c.np + 64, c.tmpmax, c.tmpmax2, sR, sC, c.st)) != SIGNTRI_OK)
        return rs;
    return make_gathered_slices(c.n, M, ldm, c.ginv, c.gmap, c.sbbase, kSuper, c.ng, kOzakiSlices, kOzakiBits, sR,
                                sC, gR, gC, R, C, c.rows_g, c.rows_g, c.st);
}

// Exact slices of the strictly upper part of M in the original layout (scales
// computed here unless `scaled`).
signtri_status exact_slices_of(MixedCtx &c, const double *M, int ldm, __nv_bfloat16 *R, __nv_bfloat16 *C, float *sR,
                               float *sC, bool scaled = false, bool cols = true)
{
    signtri_status rs;
    if (!scaled &&
        (rs = make_scales_both(c.n, M, ldm, 1, c.np + 64, c.tmpmax, c.tmpmax2, sR, sC, c.st)) != SIGNTRI_OK)
        return rs;
    // the probe and full-residual jobs pair 64-blocks (2i, 2i+1): they never
    // read row slices left of a row's even block or column slices past a
    // column's block pair
    if ((rs = make_row_slices(c.n, c.n, M, ldm, 1, kOzakiSlices, kOzakiBits, sR, R, c.np + 64, c.np, c.st, 1)) !=
        SIGNTRI_OK)
        return rs;
    if (!cols) return SIGNTRI_OK;
    return make_col_slices(c.n, c.n, M, ldm, 1, kOzakiSlices, kOzakiBits, sC, C, c.np + 64, c.np, c.st, 1);
}

signtri_status read_norms(MixedCtx &c)
{
    SGT_CUDA_TRY(cudaMemcpyAsync(c.norms_host, c.norms, 8 * sizeof(double), cudaMemcpyDeviceToHost, c.st));
    SGT_CUDA_TRY(cudaStreamSynchronize(c.st));
    return SIGNTRI_OK;
}

// Needed residual of U (Rc or Rs per entry) into c.R and its norms: three
// tensor-core launches over the gathered layout, each job's four quadrants
// all used -- equal-sign blocks  Y = N_U N_U  (into RA),
// opposite-sign blocks  N_T N_U  (into RA) and  N_U N_T  (into RB) -- then
// the float64 finalize in the original layout.
signtri_status residual_needed(MixedCtx &c, const double *T, int ldt, const double *U, int ldu)
{
    signtri_status rs = gathered_slices_of(c, U, ldu, c.NUr, c.NUc, c.sUr, c.sUc, c.gUr, c.gUc);
    if (rs != SIGNTRI_OK) return rs;
    const int R = c.rows_g, K = c.ng, ld = c.rows_g;
    const TcSource uR{c.NUr, kOzakiSlices, R, K, ld, c.gUr}, uC{c.NUc, kOzakiSlices, R, K, ld, c.gUc};
    const TcSource tR{c.NTgr, kOzakiSlices, R, K, ld, c.gTr}, tC{c.NTgc, kOzakiSlices, R, K, ld, c.gTc};
    const TcQuadOut qa{{c.RA, c.RA, c.RA, c.RA}, c.ng, c.ng, c.ng};
    const TcQuadOut qb{{c.RB, c.RB, c.RB, c.RB}, c.ng, c.ng, c.ng};
    const TcJob *same = c.d_res_jobs, *opp = c.d_res_jobs + c.n_res_same;
    const double fl_same = tc_flops(c.pairs_oz.n, 1, 1) * c.res_kb_same;
    const double fl_opp = tc_flops(c.pairs_oz.n, 1, 1) * c.res_kb_opp;
    rs = tc_blocksums(uR, uR, uC, uC, same, c.n_res_same, c.pairs_oz, c.d_pairs_oz, kExactChunkKb7, nullptr, qa, c.d_err,
                      SIGNTRI_KC_RESIDUAL, c.st, fl_same);
    if (rs != SIGNTRI_OK) return rs;
    rs = tc_blocksums(tR, tR, uC, uC, opp, c.n_res_opp, c.pairs_oz, c.d_pairs_oz, kExactChunkKb7, nullptr, qa, c.d_err,
                      SIGNTRI_KC_RESIDUAL, c.st, fl_opp);
    if (rs != SIGNTRI_OK) return rs;
    rs = tc_blocksums(uR, uR, tC, tC, opp, c.n_res_opp, c.pairs_oz, c.d_pairs_oz, kExactChunkKb7, nullptr, qb, c.d_err,
                      SIGNTRI_KC_RESIDUAL, c.st, fl_opp);
    if (rs != SIGNTRI_OK) return rs;
    SGT_CUDA_TRY(cudaMemsetAsync(c.norms, 0, 8 * sizeof(double), c.st));
    {
        ProfScope ps(SIGNTRI_KC_RESIDUAL_SUM, c.st);
        needed_finalize_kernel<<<c.n, 256, 0, c.st>>>(c.n, T, ldt, U, ldu, c.gmap, c.RA, c.RB, c.ng, c.R, c.norms);
        SGT_LAUNCH_CHECK();
    }
    c.res_c = c.R;
    c.res_s = c.R;
    if ((rs = read_norms(c)) != SIGNTRI_OK) return rs;
    c.nT2 = c.norms_host[2];
    c.nU2 = c.norms_host[3];
    return SIGNTRI_OK;
}

// Both residuals of U over all entries (Rc into RA's memory, Rs into R) and
// their norms.  Original layout; each job pairs row blocks (2i, 2i+1) with
// column blocks (2j, 2j+1), j >= i, over K-blocks [2i, 2j+2) (terms outside
// an output block's own range are structural zeros), and three launches use
// all four quadrants: N_U N_U (into Rs), N_T N_U (into Ptu) and N_U N_T
// (into Put).  A lone last block pairs with the zero block at row np.
signtri_status residual_full(MixedCtx &c, const double *T, int ldt, const double *U, int ldu)
{
    signtri_status rs = exact_slices_of(c, U, ldu, c.NUr, c.NUc, c.sUr, c.sUc);
    if (rs != SIGNTRI_OK) return rs;
    const int R = c.np + 64;
    const TcSource uR{c.NUr, kOzakiSlices, R, c.np, c.np, c.sUr}, uC{c.NUc, kOzakiSlices, R, c.np, c.np, c.sUc};
    const TcSource tR{c.NTr, kOzakiSlices, R, c.np, c.np, c.sTr}, tC{c.NTc, kOzakiSlices, R, c.np, c.np, c.sTc};
    double *Ptu = c.RA, *Put = c.RB, *Rs = c.R;
    const TcQuadOut qs{{Rs, Rs, Rs, Rs}, c.n, c.n, c.n};
    const TcQuadOut qtu{{Ptu, Ptu, Ptu, Ptu}, c.n, c.n, c.n};
    const TcQuadOut qut{{Put, Put, Put, Put}, c.n, c.n, c.n};
    const double fl = tc_flops(c.pairs_oz.n, 1, 1) * c.full_kb;
    rs = tc_blocksums(uR, uR, uC, uC, c.d_full_jobs, c.n_full_jobs, c.pairs_oz, c.d_pairs_oz, kExactChunkKb7, nullptr, qs, c.d_err,
                      SIGNTRI_KC_RESIDUAL, c.st, fl);
    if (rs != SIGNTRI_OK) return rs;
    rs = tc_blocksums(tR, tR, uC, uC, c.d_full_jobs, c.n_full_jobs, c.pairs_oz, c.d_pairs_oz, kExactChunkKb7, nullptr, qtu,
                      c.d_err, SIGNTRI_KC_RESIDUAL, c.st, fl);
    if (rs != SIGNTRI_OK) return rs;
    rs = tc_blocksums(uR, uR, tC, tC, c.d_full_jobs, c.n_full_jobs, c.pairs_oz, c.d_pairs_oz, kExactChunkKb7, nullptr, qut,
                      c.d_err, SIGNTRI_KC_RESIDUAL, c.st, fl);
    if (rs != SIGNTRI_OK) return rs;
    SGT_CUDA_TRY(cudaMemsetAsync(c.norms, 0, 8 * sizeof(double), c.st));
    {
        ProfScope ps(SIGNTRI_KC_RESIDUAL_SUM, c.st);
        residual_finalize_kernel<<<c.n, 256, 0, c.st>>>(c.n, T, ldt, U, ldu, Ptu, Put, Rs, c.n, c.norms);
        SGT_LAUNCH_CHECK();
    }
    c.res_c = Ptu;
    c.res_s = Rs;
    if ((rs = read_norms(c)) != SIGNTRI_OK) return rs;
    c.nT2 = c.norms_host[2];
    c.nU2 = c.norms_host[3];
    return SIGNTRI_OK;
}

// Probe estimate of both residuals of U over all entries, into
// c.norms_host[0], [1] (squared, scaled to ||R||_F^2), with [2], [3] the
// squared norms of T and of U from the last needed residual (U moved by the
// correction only, ~1e-8 relative: immaterial for the test).
// Products n x n by n x kProbes, jobs = row pairs x two K halves (longest
// first), each half into its own buffer.
signtri_status probe_check(MixedCtx &c, const double *T, int ldt, const double *U, int ldu, unsigned long long seed)
{
    const int n = c.n, np = c.np;
    signtri_status rs;
    if ((rs = make_scales(n, n, U, ldu, 1, true, np + 64, c.tmpmax, c.sUr, c.st)) != SIGNTRI_OK) return rs;
    if ((rs = make_row_slices(n, n, U, ldu, 1, kOzakiSlices, kOzakiBits, c.sUr, c.NUr, np + 64, np, c.st, 1)) !=
        SIGNTRI_OK)
        return rs;
    const size_t blk = (size_t)n * kProbes;
    double *P[10];
    for (int i = 0; i < 10; i++) P[i] = c.Pp + i * blk;
    {
        ProfScope ps(SIGNTRI_KC_RESIDUAL_SUM, c.st);
        probe_kernel<<<dim3(std::min((np + 255) / 256, 64), kProbes), 256, 0, c.st>>>(n, np, seed, c.Z, c.Zc,
                                                                                      c.zscale);
        SGT_LAUNCH_CHECK();
    }
    const int R = np + 64;
    const TcSource uR{c.NUr, kOzakiSlices, R, np, np, c.sUr}, tR{c.NTr, kOzakiSlices, R, np, np, c.sTr};
    const TcSource zC{c.Zc, 1, kProbes, np, np, c.zscale};
    const TcSource w1C{c.W1c, kOzakiSlices, kProbes, np, np, c.w1scale}, w2C{c.W2c, kOzakiSlices, kProbes, np, np,
                                                                              c.w2scale};
    auto out = [&](double *m) { return TcQuadOut{{m, m, m, m}, n, n, kProbes, blk}; };
    const double flz = tc_flops(c.pairs_z.n, 1, 1) * c.probe_kb, flw = tc_flops(c.pairs_oz.n, 1, 1) * c.probe_kb;
    // W1 = U Z, W2 = T Z (Z: one slice, pairs (s, 0))
    if ((rs = tc_blocksums(uR, uR, zC, zC, c.d_probe_jobs, c.n_probe_jobs, c.pairs_z, c.d_pairs_z, kExactChunkKb7,
                           nullptr, out(P[0]), c.d_err, SIGNTRI_KC_RESIDUAL, c.st, flz)) != SIGNTRI_OK)
        return rs;
    if ((rs = tc_blocksums(tR, tR, zC, zC, c.d_probe_jobs, c.n_probe_jobs, c.pairs_z, c.d_pairs_z, kExactChunkKb7,
                           nullptr, out(P[2]), c.d_err, SIGNTRI_KC_RESIDUAL, c.st, flz)) != SIGNTRI_OK)
        return rs;
    {
        ProfScope ps(SIGNTRI_KC_RESIDUAL_SUM, c.st);
        const dim3 g(std::min((n + 255) / 256, 64), kProbes);
        probe_combine_kernel<<<g, 256, 0, c.st>>>(n, P[0], P[1], U, ldu, c.Z, c.W1);
        SGT_LAUNCH_CHECK();
        probe_combine_kernel<<<g, 256, 0, c.st>>>(n, P[2], P[3], T, ldt, c.Z, c.W2);
        SGT_LAUNCH_CHECK();
    }
    if ((rs = make_scales(n, kProbes, c.W1, n, 0, false, kProbes, c.tmpmax, c.w1scale, c.st)) != SIGNTRI_OK)
        return rs;
    if ((rs = make_scales(n, kProbes, c.W2, n, 0, false, kProbes, c.tmpmax, c.w2scale, c.st)) != SIGNTRI_OK)
        return rs;
    if ((rs = make_col_slices(n, kProbes, c.W1, n, 0, kOzakiSlices, kOzakiBits, c.w1scale, c.W1c, kProbes, np,
                              c.st)) != SIGNTRI_OK)
        return rs;
    if ((rs = make_col_slices(n, kProbes, c.W2, n, 0, kOzakiSlices, kOzakiBits, c.w2scale, c.W2c, kProbes, np,
                              c.st)) != SIGNTRI_OK)
        return rs;
    // N_T W1, N_U W2, N_U W1
    if ((rs = tc_blocksums(tR, tR, w1C, w1C, c.d_probe_jobs, c.n_probe_jobs, c.pairs_oz, c.d_pairs_oz, kExactChunkKb7,
                           nullptr, out(P[4]), c.d_err, SIGNTRI_KC_RESIDUAL, c.st, flw)) != SIGNTRI_OK)
        return rs;
    if ((rs = tc_blocksums(uR, uR, w2C, w2C, c.d_probe_jobs, c.n_probe_jobs, c.pairs_oz, c.d_pairs_oz, kExactChunkKb7,
                           nullptr, out(P[6]), c.d_err, SIGNTRI_KC_RESIDUAL, c.st, flw)) != SIGNTRI_OK)
        return rs;
    if ((rs = tc_blocksums(uR, uR, w1C, w1C, c.d_probe_jobs, c.n_probe_jobs, c.pairs_oz, c.d_pairs_oz, kExactChunkKb7,
                           nullptr, out(P[8]), c.d_err, SIGNTRI_KC_RESIDUAL, c.st, flw)) != SIGNTRI_OK)
        return rs;
    SGT_CUDA_TRY(cudaMemsetAsync(c.norms, 0, 2 * sizeof(double), c.st));
    {
        ProfScope ps(SIGNTRI_KC_RESIDUAL_SUM, c.st);
        probe_residual_kernel<<<dim3(std::min((n + 255) / 256, 64), kProbes), 256, 0, c.st>>>(
            n, T, ldt, U, ldu, c.Z, c.W1, c.W2, P[4], P[5], P[6], P[7], P[8], P[9], c.norms);
        SGT_LAUNCH_CHECK();
    }
    SGT_CUDA_TRY(cudaMemcpyAsync(c.norms_host, c.norms, 2 * sizeof(double), cudaMemcpyDeviceToHost, c.st));
    SGT_CUDA_TRY(cudaStreamSynchronize(c.st));
    c.norms_host[0] /= kProbes;
    c.norms_host[1] /= kProbes;
    c.norms_host[2] = c.nT2;
    c.norms_host[3] = c.nU2;
    return SIGNTRI_OK;
}

}  // namespace

// The correction's second stream and its fork / join events, one set per
// device, created on first use (the library's calls are serialized).
struct SideStream {
    cudaStream_t s = nullptr;
    cudaEvent_t fork = nullptr, join = nullptr;
};
SideStream g_side[64];

signtri_status side_stream(MixedCtx &c)
{
    c.side = nullptr;
    int dev = 0;
    SGT_CUDA_TRY(cudaGetDevice(&dev));
    if (dev < 0 || dev >= 64) return SIGNTRI_OK;
    SideStream &g = g_side[dev];
    // a piece is stored only once created, so a call after a failed attempt
    // creates what is still missing; the side stream is used only with both
    // of its events
    if (!g.s) {
        cudaStream_t s = nullptr;
        SGT_CUDA_TRY(cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking));
        g.s = s;
    }
    if (!g.fork) {
        cudaEvent_t e = nullptr;
        SGT_CUDA_TRY(cudaEventCreateWithFlags(&e, cudaEventDisableTiming));
        g.fork = e;
    }
    if (!g.join) {
        cudaEvent_t e = nullptr;
        SGT_CUDA_TRY(cudaEventCreateWithFlags(&e, cudaEventDisableTiming));
        g.join = e;
    }
    c.side = g.s;
    c.ev_fork = g.fork;
    c.ev_join = g.join;
    return SIGNTRI_OK;
}

size_t mixed_workspace_bytes(int n, int S) { return n > 0 ? bytes_for(n, S) + (64 << 10) : 0; }

signtri_status mixed_run(int n, const double *T, int ldt, double *U, int ldu, int S, const MixedParams &prm,
                         MixedReport &rep, Arena &ws, int *d_err, double *norms_host, cudaStream_t st)
{
    MixedCtx c{};
    c.n = n;
    c.np = pad64(n);
    c.f16 = S < 0;   // a negative S asks for the fp16 split of -S terms
    if (S < 0) S = -S;
    c.S = S;
    c.st = st;
    c.d_err = d_err;
    build_schedule(n, kSweepCtas, c.sc);
    build_schedule(n, kSweepCtas / 2, c.sc2);
    build_look_schedules(n, kSweepCtas / 2, c.scA, c.scB, c.scC);
    const int nb = c.sc.nb;
    const size_t np = c.np;
    const size_t split_elems = (size_t)S * np * np;
    const size_t ngr = (size_t)gathered_bound(n) + 64, oz_elems = (size_t)kOzakiSlices * ngr * ngr;
    c.Tr = take<__nv_bfloat16>(ws, split_elems); c.Tc = take<__nv_bfloat16>(ws, split_elems);
    c.Ur = take<__nv_bfloat16>(ws, split_elems); c.Uc = take<__nv_bfloat16>(ws, split_elems);
    c.Er = take<__nv_bfloat16>(ws, split_elems); c.Ec = take<__nv_bfloat16>(ws, split_elems);
    const size_t oz_orig = (size_t)kOzakiSlices * (np + 64) * np;
    c.NTgr = take<__nv_bfloat16>(ws, oz_elems); c.NTgc = take<__nv_bfloat16>(ws, oz_elems);
    c.NTr = take<__nv_bfloat16>(ws, oz_orig); c.NTc = take<__nv_bfloat16>(ws, oz_orig);
    c.NUr = take<__nv_bfloat16>(ws, oz_elems); c.NUc = take<__nv_bfloat16>(ws, oz_elems);
    // original-index scales and their max buffer cover the zero block too
    c.sTr = take<float>(ws, np + 64); c.sTc = take<float>(ws, np + 64);
    c.sUr = take<float>(ws, np + 64); c.sUc = take<float>(ws, np + 64);
    c.gTr = take<float>(ws, ngr); c.gTc = take<float>(ws, ngr); c.gUr = take<float>(ws, ngr); c.gUc = take<float>(ws, ngr);
    c.gmap = take<int>(ws, ngr); c.ginv = take<int>(ws, ngr); c.pos = take<unsigned char>(ws, np);
    c.sbbase = take<int>(ws, (size_t)(n + kSuper - 1) / kSuper + 1);
    c.tmpmax = take<unsigned long long>(ws, np + 64);
    c.tmpmax2 = take<unsigned long long>(ws, np + 64);
    const size_t maxjobs = (size_t)std::max({c.sc.max_jobs, c.scA.max_jobs, c.scB.max_jobs, c.scC.max_jobs, 1});
    c.PA = take<double>(ws, maxjobs * 16384); c.PB = take<double>(ws, maxjobs * 16384);
    c.E = take<double>(ws, (size_t)n * n); c.R = take<double>(ws, (size_t)n * n);
    c.OPS = take<float>(ws, (size_t)4 * nb * MB * MB); c.DIAG = take<float>(ws, (size_t)nb * MB);
    c.invT = take<float>(ws, np + 64); c.invU = take<float>(ws, np + 64); c.invE = take<float>(ws, np + 64);
    c.amax = take<unsigned>(ws, 16);
    if (!c.invT || !c.invU || !c.invE || !c.amax) return SIGNTRI_ERR_NO_WORKSPACE;
    const int nbp = (nb + 1) / 2;
    c.n_full_jobs = nbp * (nbp + 1) / 2;
    c.d_full_jobs = take<TcJob>(ws, (size_t)c.n_full_jobs);
    c.RA = take<double>(ws, ngr * ngr); c.RB = take<double>(ws, ngr * ngr);
    c.norms = take<double>(ws, 8);
    const size_t pairs_max = ngr / 128 + 2 * (size_t)((n + kSuper - 1) / kSuper) + 2;
    c.d_res_jobs = take<TcJob>(ws, pairs_max * pairs_max);
    for (auto pr : {std::make_pair(&c.sc, &c.ds), std::make_pair(&c.sc2, &c.ds2), std::make_pair(&c.scA, &c.dsA),
                    std::make_pair(&c.scB, &c.dsB), std::make_pair(&c.scC, &c.dsC)}) {
        pr.second->jobs = take<TcJob>(ws, std::max<size_t>(pr.first->jobs.size(), 1));
        pr.second->cta_off = take<int>(ws, std::max<size_t>(pr.first->cta_off.size(), 1));
        pr.second->tslot = take<int2>(ws, std::max<size_t>(pr.first->tslot.size(), 1));
        if (!pr.second->jobs || !pr.second->cta_off || !pr.second->tslot) return SIGNTRI_ERR_NO_WORKSPACE;
    }
    c.d_pairs_split = take<TcPairs>(ws, 1);
    c.d_pairs_oz = take<TcPairs>(ws, 1);
    c.d_pairs_z = take<TcPairs>(ws, 1);
    {
        const size_t blk = (size_t)n * kProbes;
        c.Z = take<double>(ws, blk); c.W1 = take<double>(ws, blk); c.W2 = take<double>(ws, blk);
        c.Pp = take<double>(ws, 10 * blk);
        c.Zc = take<__nv_bfloat16>(ws, (size_t)kProbes * np);
        c.W1c = take<__nv_bfloat16>(ws, (size_t)kOzakiSlices * kProbes * np);
        c.W2c = take<__nv_bfloat16>(ws, (size_t)kOzakiSlices * kProbes * np);
        c.zscale = take<float>(ws, kProbes); c.w1scale = take<float>(ws, kProbes); c.w2scale = take<float>(ws, kProbes);
        c.d_probe_jobs = take<TcJob>(ws, (size_t)2 * nbp + 2);
        if (!c.Z || !c.W1 || !c.W2 || !c.Pp || !c.Zc || !c.W1c || !c.W2c || !c.zscale || !c.w1scale || !c.w2scale ||
            !c.d_probe_jobs || !c.d_pairs_z)
            return SIGNTRI_ERR_NO_WORKSPACE;
    }
    c.norms_host = norms_host;
    if (!c.Tr || !c.Tc || !c.Ur || !c.Uc || !c.Er || !c.Ec || !c.NTgr || !c.NTgc || !c.NTr || !c.NTc || !c.NUr ||
        !c.NUc || !c.d_full_jobs || !c.sTr ||
        !c.sTc || !c.sUr || !c.sUc || !c.gTr || !c.gTc || !c.gUr || !c.gUc || !c.gmap || !c.ginv || !c.pos ||
        !c.tmpmax || !c.tmpmax2 || !c.PA || !c.PB || !c.E || !c.R || !c.RA || !c.RB || !c.norms || !c.d_res_jobs ||
        !c.d_pairs_split || !c.d_pairs_oz || !c.OPS || !c.DIAG || !c.sbbase)
        return SIGNTRI_ERR_NO_WORKSPACE;
    c.pairs_split = split_pairs(S);
    c.pairs_oz = ozaki_pairs_impl(kOzakiSlices, kOzakiBits);
    // probe products with Z (one slice): pairs (s, 0)
    std::memset(&c.pairs_z, 0, sizeof(c.pairs_z));
    for (int sl = 0; sl < kOzakiSlices; sl++) {
        c.pairs_z.s[sl] = sl;
        c.pairs_z.t[sl] = 0;
        c.pairs_z.w[sl] = ldexpf(1.0f, -kOzakiBits * (sl + 2));
    }
    c.pairs_z.n = kOzakiSlices;
    SGT_CUDA_TRY(cudaMemcpyAsync(c.d_pairs_z, &c.pairs_z, sizeof(TcPairs), cudaMemcpyHostToDevice, st));
    {
        // probe jobs: row pairs (2I, 2I+1) x K halves of [2I, nb), longest first
        std::vector<TcJob> pj;
        double kb = 0.0;
        for (int I = 0; I < nbp; I++)
            for (int h = 0; h < 2; h++) {
                const int k0 = 2 * I, mid = (k0 + nb + 1) / 2;
                TcJob j;
                j.rt = 2 * I * MB; j.rb = 2 * I + 1 < nb ? (2 * I + 1) * MB : (int)np;
                j.cl = 0; j.cr = 64;
                j.kb0 = h ? mid : k0; j.kb1 = h ? nb : mid; j.slot = h; j.pad = 0;
                kb += (double)((j.rb != (int)np) + 1) * 2 * std::max(0, j.kb1 - j.kb0);
                pj.push_back(j);
            }
        std::stable_sort(pj.begin(), pj.end(),
                         [](const TcJob &x, const TcJob &y) { return x.kb1 - x.kb0 > y.kb1 - y.kb0; });
        c.n_probe_jobs = (int)pj.size();
        c.probe_kb = kb;
        SGT_CUDA_TRY(cudaMemcpyAsync(c.d_probe_jobs, pj.data(), pj.size() * sizeof(TcJob), cudaMemcpyHostToDevice,
                                     st));
        SGT_CUDA_TRY(cudaStreamSynchronize(st));
    }
    for (auto pr : {std::make_pair(&c.sc, &c.ds), std::make_pair(&c.sc2, &c.ds2), std::make_pair(&c.scA, &c.dsA),
                    std::make_pair(&c.scB, &c.dsB), std::make_pair(&c.scC, &c.dsC)}) {
        if (!pr.first->jobs.empty())
            SGT_CUDA_TRY(cudaMemcpyAsync(pr.second->jobs, pr.first->jobs.data(), pr.first->jobs.size() * sizeof(TcJob),
                                         cudaMemcpyHostToDevice, st));
        if (!pr.first->cta_off.empty())
            SGT_CUDA_TRY(cudaMemcpyAsync(pr.second->cta_off, pr.first->cta_off.data(),
                                         pr.first->cta_off.size() * sizeof(int), cudaMemcpyHostToDevice, st));
        if (!pr.first->tslot.empty())
            SGT_CUDA_TRY(cudaMemcpyAsync(pr.second->tslot, pr.first->tslot.data(),
                                         pr.first->tslot.size() * sizeof(int2), cudaMemcpyHostToDevice, st));
    }
    {
        const signtri_status ss = side_stream(c);
        if (ss != SIGNTRI_OK) return ss;
    }
    SGT_CUDA_TRY(cudaMemcpyAsync(c.d_pairs_split, &c.pairs_split, sizeof(TcPairs), cudaMemcpyHostToDevice, st));
    SGT_CUDA_TRY(cudaMemcpyAsync(c.d_pairs_oz, &c.pairs_oz, sizeof(TcPairs), cudaMemcpyHostToDevice, st));
    {
        // full-residual jobs in 8 x 8 groups of block pairs: the CTAs resident
        // together share row and column panels in L2
        std::vector<TcJob> rj;
        rj.reserve(c.n_full_jobs);
        double kb = 0.0;
        constexpr int G = 8;
        const int zero = (int)np;   // the zero block
        for (int I0 = 0; I0 < nbp; I0 += G)
            for (int J0 = I0 / G * G; J0 < nbp; J0 += G)
                for (int I = I0; I < std::min(I0 + G, nbp); I++)
                    for (int J = std::max(J0, I); J < std::min(J0 + G, nbp); J++) {
                        TcJob j;
                        j.rt = 2 * I * MB; j.rb = 2 * I + 1 < nb ? (2 * I + 1) * MB : zero;
                        j.cl = 2 * J * MB; j.cr = 2 * J + 1 < nb ? (2 * J + 1) * MB : zero;
                        j.kb0 = 2 * I; j.kb1 = std::min(2 * J + 2, nb); j.slot = 0; j.pad = 0;
                        kb += (double)((j.rb != zero) + 1) * ((j.cr != zero) + 1) * (j.kb1 - j.kb0);
                        rj.push_back(j);
                    }
        c.full_kb = kb;
        SGT_CUDA_TRY(cudaMemcpyAsync(c.d_full_jobs, rj.data(), rj.size() * sizeof(TcJob), cudaMemcpyHostToDevice,
                                     st));
        SGT_CUDA_TRY(cudaStreamSynchronize(st));
    }
    signtri_status rs0 = setup_gathered(c, T, ldt);
    if (rs0 != SIGNTRI_OK) return rs0;
    // slices start from zero (padding and the not-yet-computed blocks)
    SGT_CUDA_TRY(cudaMemsetAsync(c.Ur, 0, split_elems * 2, st));
    SGT_CUDA_TRY(cudaMemsetAsync(c.Uc, 0, split_elems * 2, st));
    SGT_CUDA_TRY(cudaMemsetAsync(c.Er, 0, split_elems * 2, st));
    SGT_CUDA_TRY(cudaMemsetAsync(c.Ec, 0, split_elems * 2, st));
    signtri_status rs;
    if ((rs = gathered_slices_of(c, T, ldt, c.NTgr, c.NTgc, c.sTr, c.sTc, c.gTr, c.gTc)) != SIGNTRI_OK) return rs;
    if (c.f16) {
        // T's largest strictly upper entry (from the row maxima the exact
        // slices' scales were just taken from) to 2^13 .. 2^14 (fp16 stops
        // at 65504)
        float m = 0.f;
        if ((rs = row_maxima_max(c, m)) != SIGNTRI_OK) return rs;
        c.sT = m > 0.f ? pow2_scale(m, 13) : 1.f;
        if ((rs = fill_inverse(c, c.invT, c.sT)) != SIGNTRI_OK) return rs;
    }
    if ((rs = split_full(c, T, ldt, c.Tr, c.Tc, c.f16 ? c.sT : 0.f)) != SIGNTRI_OK) return rs;
    // T's scales serve both layouts; the probe check reads only T's row
    // slices, the full residual also its column slices
    if ((rs = exact_slices_of(c, T, ldt, c.NTr, c.NTc, c.sTr, c.sTc, true, prm.verify_full != 0)) != SIGNTRI_OK)
        return rs;

    // 1. low-precision solve: diagonal blocks in float64, the rest by sweep
    if ((rs = launch_zero_strict_lower(n, U, ldu, st)) != SIGNTRI_OK) return rs;
    if ((rs = diag_leaves_f64(n, T, ldt, U, ldu, MB, st)) != SIGNTRI_OK) return rs;
    if (c.f16) {
        // U's scale from its diagonal blocks, largest entry to 2^12 .. 2^13:
        // room for off-diagonal entries up to 8x larger
        float m = 0.f;
        if ((rs = diag_blocks_absmax(c, U, ldu, m)) != SIGNTRI_OK) return rs;
        c.sU = m > 0.f ? pow2_scale(m, 12) : c.sT;
        if ((rs = fill_inverse(c, c.invU, c.sU)) != SIGNTRI_OK) return rs;
    }
    {
        ProfScope ps(SIGNTRI_KC_CONVERT, st);
        diag_slices_kernel<<<nb, 256, 0, st>>>(n, U, ldu, c.Ur, c.Uc, S, nb, c.f16 ? c.sU : 0.f);
        SGT_LAUNCH_CHECK();
    }
    if ((rs = sweep<0>(c, T, ldt, U, ldu, c.Ur, c.Uc, nullptr, 0)) != SIGNTRI_OK) return rs;

    // 2. refinement.  Corrections are driven by the needed residuals (Rc at
    // opposite-sign entries, Rs at equal-sign ones); acceptance rests on both
    // residuals over all entries: the full products (verify_full) or their
    // probe estimate.
    double prev = 1e300;
    rep.steps = 0;
    rep.fallback = 0;
    auto verify = [&](int step) -> signtri_status {
        return prm.verify_full ? residual_full(c, T, ldt, U, ldu)
                               : probe_check(c, T, ldt, U, ldu, 0x5eedull * 1315423911ull + (unsigned long long)step);
    };
    auto worst_of = [&]() {
        const double *h = c.norms_host;
        const double nT = std::sqrt(h[2]), nU = std::sqrt(h[3]);
        rep.resid_commute = std::sqrt(h[0]) / (nT * nU);
        rep.resid_involution = std::sqrt(h[1]) / (nU * nU);
        return std::max(rep.resid_commute, rep.resid_involution);
    };
    for (int step = 0;; step++) {
        bool verified = step > 0;
        if ((rs = verified ? verify(step) : residual_needed(c, T, ldt, U, ldu)) != SIGNTRI_OK) return rs;
        double worst = worst_of();
        if (!verified && worst <= prm.tol) {
            // needed residuals already small: check both equations
            if ((rs = verify(step)) != SIGNTRI_OK) return rs;
            verified = true;
            worst = worst_of();
        }
        if (step == 0) rep.resid0 = worst;
        if (!(worst == worst)) { rep.fallback = 1; return SIGNTRI_OK; }   // NaN
        if (verified && worst <= prm.tol) return SIGNTRI_OK;
        if (step >= prm.max_steps || (step > 0 && worst > prev / prm.min_contraction)) {
            rep.fallback = 1;
            return SIGNTRI_OK;
        }
        prev = worst;
        // the correction reads Rc / Rs entrywise: the full residual left them;
        // after a probe test (or a confirmed step 0) form the needed ones
        if (verified && !prm.verify_full && (rs = residual_needed(c, T, ldt, U, ldu)) != SIGNTRI_OK) return rs;
        // E: zero, diagonal blocks in float64, off-diagonal blocks by sweep
        {
            ProfScope ps(SIGNTRI_KC_FILL, st);
            zero_kernel<<<1024, 256, 0, st>>>((size_t)n * n, c.E);
            SGT_LAUNCH_CHECK();
        }
        SGT_CUDA_TRY(cudaMemsetAsync(c.Er, 0, split_elems * 2, st));
        SGT_CUDA_TRY(cudaMemsetAsync(c.Ec, 0, split_elems * 2, st));
        // U0's slices: after the initial sweep they are already in Ur / Uc
        // (off-diagonal blocks from the leaves, diagonal blocks from
        // diag_slices_kernel); after a correction U has moved
        if (step > 0 && (rs = split_full(c, U, ldu, c.Ur, c.Uc, c.f16 ? c.sU : 0.f)) != SIGNTRI_OK) return rs;
        {
            const size_t dsm = 3 * (size_t)MB * (MB + 1) * sizeof(double);
            SGT_CUDA_TRY(cudaFuncSetAttribute(corr_diag_leaf_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                              (int)dsm));
            ProfScope ps(SIGNTRI_KC_CORRECTION, st);
            corr_diag_leaf_kernel<<<nb, kLeafThreads, dsm, st>>>(n, T, ldt, U, ldu, c.res_c, c.res_s, n, c.E, n);
            SGT_LAUNCH_CHECK();
        }
        if (c.f16) {
            // the correction's scale from its first-order terms, Rc_ij /
            // (t_ii - t_jj) or Rs_ij / 2 (its diagonal blocks are no guide,
            // U0's being float64-exact), largest to 2^10 .. 2^11: room for
            // entries of E up to 32x larger
            float m = 0.f;
            SGT_CUDA_TRY(cudaMemsetAsync(c.amax, 0, sizeof(unsigned), st));
            {
                ProfScope ps(SIGNTRI_KC_CONVERT, st);
                // c.DIAG: t_ii in fp32, from the initial sweep (same T)
                corr_magnitude_kernel<<<1216, 256, 0, st>>>(n, c.DIAG, c.res_c, c.res_s, n, c.amax);
                SGT_LAUNCH_CHECK();
            }
            if ((rs = read_amax(c, m)) != SIGNTRI_OK) return rs;
            c.sE = m > 0.f ? pow2_scale(m, 10) : c.sU;
            if ((rs = fill_inverse(c, c.invE, c.sE)) != SIGNTRI_OK) return rs;
        }
        {
            ProfScope ps(SIGNTRI_KC_CONVERT, st);
            diag_slices_kernel<<<nb, 256, 0, st>>>(n, c.E, n, c.Er, c.Ec, S, nb, c.f16 ? c.sE : 0.f);
            SGT_LAUNCH_CHECK();
        }
        if ((rs = sweep<1>(c, T, ldt, c.E, n, c.Er, c.Ec, U, ldu)) != SIGNTRI_OK) return rs;
        {
            ProfScope ps(SIGNTRI_KC_CORRECTION, st);
            apply_correction_kernel<<<n, 256, 0, st>>>(n, U, ldu, c.E, n, c.norms);
            SGT_LAUNCH_CHECK();
        }
        rep.steps = step + 1;
    }
}

}  // namespace signtri

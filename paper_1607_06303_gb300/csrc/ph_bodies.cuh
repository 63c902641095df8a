// ph_bodies.cuh -- device bodies of the float64 Parlett-Higham kernels,
// shared by the single-matrix kernels (ph_fp64.cu) and the batched ones
// (batched.cu).  See ph_fp64.cu for the method.
#pragma once

#include "internal.cuh"

namespace signtri {
namespace ph {

constexpr int kThreads = 256;
constexpr int kSplitMax = 32;
constexpr int kTargetCtas = 4 * 152;   // two resident CTAs per SM, two waves

// Even split of one anti-diagonal's block sums (single-matrix path): the
// nb-d tiles x (d-1) K-blocks are cut into 16-deep k-chunks, W in all, and
// CTA c of G = min(kStreamCtas, W) takes chunks [c W / G, (c+1) W / G), so
// every CTA does the same work whatever the tile count.  A CTA whose range
// crosses a tile boundary writes one partial slab per tile it touches; the
// partial of CTA c for tile I goes to slab c + I, and the tile's partials are
// the consecutive slabs of CTAs first(I)..last(I), summed in that order.
// G is fixed (not the device's SM count) so that results do not depend on
// the GPU.
constexpr int kStreamCtas = 4 * 152;

__host__ __device__ constexpr long long sk_chunks_per_tile(int d, int B) { return (long long)(d - 1) * (B / 16); }
__host__ __device__ constexpr int sk_ctas(long long W) { return (int)(W < kStreamCtas ? W : kStreamCtas); }
// the CTA whose range holds chunk x (every CTA's range is non-empty)
__host__ __device__ __forceinline__ long long sk_owner(long long x, long long W, int G) { return ((x + 1) * G - 1) / W; }

// Partial slabs one anti-diagonal needs at most, over all anti-diagonals of
// an n x n problem with leaf size B (slab c + I for CTA c and tile I).
constexpr size_t max_slabs(int n, int B)
{
    const long long nb = (n + B - 1) / B;
    long long wmax = 0;
    for (long long d = 2; d < nb; d++) {
        const long long w = (nb - d) * sk_chunks_per_tile((int)d, B);
        if (w > wmax) wmax = w;
    }
    return wmax == 0 ? 0 : (size_t)(sk_ctas(wmax) + nb);
}

// Workspace of the matrix-multiply form: the X and Y slab sets, each
// 256-byte aligned by the arena.
constexpr size_t mm_form_workspace_bytes(int n, int B)
{
    return max_slabs(n, B) == 0 ? 0 : 2 * (max_slabs(n, B) * B * B * sizeof(double) + 256);
}

__device__ __forceinline__ double sgn(double t) { return t > 0.0 ? 1.0 : -1.0; }

// ---------------------------------------------------------------------------
// Diagonal leaf: Algorithm 3 on the diagonal block [r0, r0+bs) x [r0, r0+bs),
// by anti-diagonal inside the block.  Separate multiply/add/divide with
// round-to-nearest and no contraction, sums in ascending k, so each entry is
// rounded exactly as in the plain float64 algorithm.
// ---------------------------------------------------------------------------
template <int B>
__device__ __forceinline__ void diag_leaf_body(int n, const double *__restrict__ T, int ldt, double *__restrict__ U,
                                               int ldu, int blk)
{
    constexpr int LD = B + 1;
    extern __shared__ double sm[];
    double *Ts = sm;
    double *Us = sm + B * LD;
    const int r0 = blk * B;
    const int bs = min(B, n - r0);
    for (int idx = threadIdx.x; idx < bs * bs; idx += kThreads) {
        const int i = idx % bs, j = idx / bs;
        const double t = (i <= j) ? SGT_AT(T, ldt, r0 + i, r0 + j) : 0.0;
        Ts[i + j * LD] = t;
        Us[i + j * LD] = (i == j) ? sgn(t) : 0.0;
    }
    __syncthreads();
    for (int d = 1; d < bs; d++) {
        for (int i = threadIdx.x; i < bs - d; i += kThreads) {
            const int j = i + d;
            const double uii = Us[i + i * LD], ujj = Us[j + j * LD];
            double r;
            if (__dadd_rn(uii, ujj) == 0.0) {
                double s = 0.0;
                for (int k = i + 1; k < j; k++)
                    s = __dadd_rn(s, __dsub_rn(__dmul_rn(Us[i + k * LD], Ts[k + j * LD]),
                                               __dmul_rn(Ts[i + k * LD], Us[k + j * LD])));
                const double den = __dsub_rn(Ts[i + i * LD], Ts[j + j * LD]);
                r = __dadd_rn(__ddiv_rn(__dmul_rn(Ts[i + j * LD], __dsub_rn(uii, ujj)), den),
                              __ddiv_rn(s, den));
            } else {
                double s = 0.0;
                for (int k = i + 1; k < j; k++) s = __dadd_rn(s, __dmul_rn(Us[i + k * LD], Us[k + j * LD]));
                r = __ddiv_rn(-s, __dadd_rn(uii, ujj));
            }
            Us[i + j * LD] = r;
        }
        __syncthreads();
    }
    for (int idx = threadIdx.x; idx < bs * bs; idx += kThreads) {
        const int i = idx % bs, j = idx / bs;
        if (i <= j) SGT_AT(U, ldu, r0 + i, r0 + j) = Us[i + j * LD];
    }
}

// ---------------------------------------------------------------------------
// Block sums for block (I, J) over the k range [k_lo, k_hi) (multiples of 16):
//     px = sum_k U_Ik T_kJ - T_Ik U_kJ,   py = sum_k U_Ik U_kJ.
// B x B output tile per CTA, 256 threads, (B/16)^2 outputs per thread for
// each of X and Y, k staged through shared memory in steps of 16.
// ---------------------------------------------------------------------------
template <int B>
__device__ __forceinline__ void ph_gemm_body(int n, const double *__restrict__ T, int ldt,
                                             const double *__restrict__ U, int ldu, int I, int J, int k_lo, int k_hi,
                                             double *__restrict__ px, double *__restrict__ py)
{
    constexpr int MT = B / 16;
    constexpr int KT = 16;
    __shared__ double AU[KT][B], AT[KT][B], BU[KT][B], BT[KT][B];
    const int r0 = I * B, c0 = J * B;
    const int bj = min(B, n - c0);
    const int tx = threadIdx.x % 16, ty = threadIdx.x / 16;
    double x[MT][MT], y[MT][MT];
#pragma unroll
    for (int r = 0; r < MT; r++)
#pragma unroll
        for (int c = 0; c < MT; c++) { x[r][c] = 0.0; y[r][c] = 0.0; }

    for (int k0 = k_lo; k0 < k_hi; k0 += KT) {
        for (int idx = threadIdx.x; idx < B * KT; idx += kThreads) {
            const int r = idx % B, kk = idx / B;
            AU[kk][r] = SGT_AT(U, ldu, r0 + r, k0 + kk);
            AT[kk][r] = SGT_AT(T, ldt, r0 + r, k0 + kk);
        }
        for (int idx = threadIdx.x; idx < B * KT; idx += kThreads) {
            const int kk = idx % KT, c = idx / KT;
            double bu = 0.0, bt = 0.0;
            if (c < bj) {
                bu = SGT_AT(U, ldu, k0 + kk, c0 + c);
                bt = SGT_AT(T, ldt, k0 + kk, c0 + c);
            }
            BU[kk][c] = bu;
            BT[kk][c] = bt;
        }
        __syncthreads();
#pragma unroll
        for (int kk = 0; kk < KT; kk++) {
            double au[MT], at[MT], bu[MT], bt[MT];
#pragma unroll
            for (int r = 0; r < MT; r++) { au[r] = AU[kk][tx + 16 * r]; at[r] = AT[kk][tx + 16 * r]; }
#pragma unroll
            for (int c = 0; c < MT; c++) { bu[c] = BU[kk][ty + 16 * c]; bt[c] = BT[kk][ty + 16 * c]; }
#pragma unroll
            for (int r = 0; r < MT; r++)
#pragma unroll
                for (int c = 0; c < MT; c++) {
                    x[r][c] = fma(au[r], bt[c], x[r][c]);
                    x[r][c] = fma(-at[r], bu[c], x[r][c]);
                    y[r][c] = fma(au[r], bu[c], y[r][c]);
                }
        }
        __syncthreads();
    }
#pragma unroll
    for (int r = 0; r < MT; r++)
#pragma unroll
        for (int c = 0; c < MT; c++) {
            px[(tx + 16 * r) + (ty + 16 * c) * B] = x[r][c];
            py[(tx + 16 * r) + (ty + 16 * c) * B] = y[r][c];
        }
}

// ---------------------------------------------------------------------------
// Arithmetic-efficient block sums (Section 5.3: compute only the sum an entry
// needs): entry (p, q) needs Y_pq = sum U_pk U_kq when the signs of p and q
// agree and X_pq = sum U_pk T_kq - T_pk U_kq when they differ.  Rows of block
// I and columns of block J are gathered positives first (perm, counts npos),
// so the entries of one kind form rectangles: 1 FMA per term for equal signs,
// 2 for opposite signs, instead of the 3 of ph_gemm_body.  Each sum runs over
// the same terms in the same order as there; the single result z is stored at
// the entry's original position.
//
// Thread (tx, ty) owns gathered rows tx + 16 r and columns ty + 16 c.  For a
// warp, the 16 rows of slab r are all positive (P), all negative (N) or mixed
// (M), and so are its 2 columns of slab c: warp-uniform classes, monotone in r
// and c (P.., at most one M, N..).  The column pattern -- X slabs P, Y in
// {0, 1} slabs M -- selects a template instance, the row class a branch around
// the k loop; every accumulator's kind is then known at compile time, so a
// warp issues only the products its entries need, with MT independent chains.
// In M slabs each lane picks its own operands (2 FMAs, one of them a 0 * t_kq
// for equal signs).
// ---------------------------------------------------------------------------
namespace split {

constexpr int kP = 0, kN = 1, kM = 2;

// ATn holds -T (sign flipped as an integer op when staged), so no product
// needs a separate float64 negation.
template <int B, int X, int Y, int RK>
__device__ __forceinline__ void row_pass(double (&zr)[B / 16], const double (*AU)[B], const double (*ATn)[B],
                                         const double (*BU)[B], const double (*BT)[B], int row, int ty,
                                         bool rowpos, const bool (&colpos)[B / 16])
{
    constexpr int MT = B / 16;
#pragma unroll 4
    for (int kk = 0; kk < 16; kk++) {
        const double au = AU[kk][row];
        const double atn = ATn[kk][row];
        // mixed row slab: per-lane operands for positive (P) and negative (N)
        // column slabs, so that z += a1 * t_kq + a2 * u_kq is the entry's own sum
        double a1P = 0.0, a2P = 0.0, a1N = 0.0, a2N = 0.0;
        if (RK == kM) {
            a1P = rowpos ? 0.0 : au;
            a2P = rowpos ? au : atn;
            a1N = rowpos ? au : 0.0;
            a2N = rowpos ? atn : au;
        }
#pragma unroll
        for (int c = 0; c < MT; c++) {
            const int ck = (c < X) ? kP : ((c < X + Y) ? kM : kN);
            const double bu = BU[kk][ty + 16 * c];
            if (RK != kM && ck != kM) {
                if (RK == ck) {
                    zr[c] = fma(au, bu, zr[c]);
                } else {
                    zr[c] = fma(au, BT[kk][ty + 16 * c], zr[c]);
                    zr[c] = fma(atn, bu, zr[c]);
                }
            } else if (RK == kM && ck == kP) {
                zr[c] = fma(a1P, BT[kk][ty + 16 * c], zr[c]);
                zr[c] = fma(a2P, bu, zr[c]);
            } else if (RK == kM && ck == kN) {
                zr[c] = fma(a1N, BT[kk][ty + 16 * c], zr[c]);
                zr[c] = fma(a2N, bu, zr[c]);
            } else {
                // the one column slab a sign boundary splits (at most one warp)
                const bool sm_ = (rowpos == colpos[c]);
                zr[c] = fma(sm_ ? 0.0 : au, BT[kk][ty + 16 * c], zr[c]);
                zr[c] = fma(sm_ ? au : atn, bu, zr[c]);
            }
        }
    }
}

template <int B, int X, int Y>
__device__ __forceinline__ void k_loop(int n, const double *__restrict__ T, int ldt, const double *__restrict__ U,
                                       int ldu, int r0, int c0, int bj, int k_lo, int k_hi, const short *pI,
                                       const short *pJ, const int (&rk)[B / 16], const bool (&rowpos)[B / 16],
                                       const bool (&colpos)[B / 16], double (&z)[B / 16][B / 16],
                                       double (*AU)[B], double (*AT)[B], double (*BU)[B], double (*BT)[B])
{
    constexpr int MT = B / 16;
    constexpr int KT = 16;
    const int tx = threadIdx.x % 16, ty = threadIdx.x / 16;
    for (int k0 = k_lo; k0 < k_hi; k0 += KT) {
        for (int idx = threadIdx.x; idx < B * KT; idx += kThreads) {
            const int r = idx % B, kk = idx / B;
            const int gr = r0 + pI[r];
            AU[kk][r] = SGT_AT(U, ldu, gr, k0 + kk);
            AT[kk][r] = __longlong_as_double(__double_as_longlong(SGT_AT(T, ldt, gr, k0 + kk)) ^
                                             (long long)0x8000000000000000ull);
        }
        for (int idx = threadIdx.x; idx < B * KT; idx += kThreads) {
            const int kk = idx % KT, c = idx / KT;
            const int lc = pJ[c];
            double bu = 0.0, bt = 0.0;
            if (lc < bj) {
                bu = SGT_AT(U, ldu, k0 + kk, c0 + lc);
                bt = SGT_AT(T, ldt, k0 + kk, c0 + lc);
            }
            BU[kk][c] = bu;
            BT[kk][c] = bt;
        }
        __syncthreads();
#pragma unroll
        for (int r = 0; r < MT; r++) {
            const int row = tx + 16 * r;
            if (rk[r] == kP)
                row_pass<B, X, Y, kP>(z[r], AU, AT, BU, BT, row, ty, rowpos[r], colpos);
            else if (rk[r] == kN)
                row_pass<B, X, Y, kN>(z[r], AU, AT, BU, BT, row, ty, rowpos[r], colpos);
            else
                row_pass<B, X, Y, kM>(z[r], AU, AT, BU, BT, row, ty, rowpos[r], colpos);
        }
        __syncthreads();
    }
}

}  // namespace split

template <int B>
__device__ __forceinline__ void ph_gemm_split_body(int n, const double *__restrict__ T, int ldt,
                                                   const double *__restrict__ U, int ldu, int I, int J, int k_lo,
                                                   int k_hi, const short *__restrict__ perm,
                                                   const int *__restrict__ npos, double *__restrict__ pz)
{
    using namespace split;
    constexpr int MT = B / 16;
    __shared__ double AU[16][B], AT[16][B], BU[16][B], BT[16][B];
    __shared__ short pI[B], pJ[B];
    __syncthreads();   // a CTA may run several tiles: pI, pJ are still read above
    const int r0 = I * B, c0 = J * B;
    const int bj = min(B, n - c0);
    for (int i = threadIdx.x; i < B; i += kThreads) {
        pI[i] = perm[r0 + i];
        pJ[i] = perm[c0 + i];
    }
    const int npI = npos[I], npJ = npos[J];
    const int tx = threadIdx.x % 16, ty = threadIdx.x / 16;
    int rk[MT];
    bool rowpos[MT], colpos[MT];
    int X = 0, Y = 0;
    double z[MT][MT];
#pragma unroll
    for (int r = 0; r < MT; r++) {
        rowpos[r] = (tx + 16 * r) < npI;
        colpos[r] = (ty + 16 * r) < npJ;
        const bool rall = __all_sync(0xffffffffu, rowpos[r]), rnone = !__any_sync(0xffffffffu, rowpos[r]);
        rk[r] = rall ? kP : (rnone ? kN : kM);
        const bool call = __all_sync(0xffffffffu, colpos[r]), cnone = !__any_sync(0xffffffffu, colpos[r]);
        X += call ? 1 : 0;
        Y += (!call && !cnone) ? 1 : 0;
#pragma unroll
        for (int c = 0; c < MT; c++) z[r][c] = 0.0;
    }
    __syncthreads();
#define SGT_SPLIT_CASE(XV, YV)                                                                             \
    else if (X == XV && Y == YV)                                                                           \
    {                                                                                                      \
        if constexpr (XV + YV <= MT)                                                                       \
            k_loop<B, (XV + YV <= MT ? XV : 0), (XV + YV <= MT ? YV : 0)>(n, T, ldt, U, ldu, r0, c0, bj, k_lo, \
                                                                         k_hi, pI, pJ, rk, rowpos, colpos, z, AU, AT, BU, BT); \
    }
    if (false) {
    }
    SGT_SPLIT_CASE(0, 0) SGT_SPLIT_CASE(1, 0) SGT_SPLIT_CASE(2, 0) SGT_SPLIT_CASE(3, 0) SGT_SPLIT_CASE(4, 0)
    SGT_SPLIT_CASE(0, 1) SGT_SPLIT_CASE(1, 1) SGT_SPLIT_CASE(2, 1) SGT_SPLIT_CASE(3, 1)
#undef SGT_SPLIT_CASE
#pragma unroll
    for (int r = 0; r < MT; r++)
#pragma unroll
        for (int c = 0; c < MT; c++) pz[pI[tx + 16 * r] + pJ[ty + 16 * c] * B] = z[r][c];
}

// Per block of B rows: the rows' positions sorted positives first (stable),
// beyond n at the end, and the count of positives.  One CTA of B threads per
// block.
template <int B>
__device__ __forceinline__ void sign_perm_body(int n, const double *__restrict__ T, int ldt, int blk,
                                               short *__restrict__ perm, int *__restrict__ npos)
{
    __shared__ int pos_before[B + 1];
    const int i = threadIdx.x;
    const int gi = blk * B + i;
    const bool valid = gi < n;
    const bool positive = valid && SGT_AT(T, ldt, gi, gi) > 0.0;
    if (i == 0) pos_before[0] = 0;
    __syncthreads();
    if (i < B) pos_before[i + 1] = positive ? 1 : 0;
    __syncthreads();
    if (i == 0)
        for (int t = 1; t <= B; t++) pos_before[t] += pos_before[t - 1];
    __syncthreads();
    const int np = pos_before[B];
    const int nvalid = min(B, n - blk * B);
    if (i < B) {
        int slot;
        if (positive) slot = pos_before[i];
        else if (valid) slot = np + (i - pos_before[i]);
        else slot = i;                       // rows beyond n keep their place
        perm[blk * B + slot] = (short)i;
    }
    if (i == 0) npos[blk] = np;
    (void)nvalid;
}

// ---------------------------------------------------------------------------
// Off-diagonal leaf for block (I, J = I+d): rows [r0, r0+B), cols [c0, c0+bj).
// With p, q the local row and column and V = U_IJ, Algorithm 6's 1x1 case
// with the in-block part of the sums written out:
//   signs differ:  (t_pp - t_qq) v_pq = t_pq (u_pp - u_qq) + x_pq
//                    + sum_{p'>p} (U_II[p,p'] T_IJ[p',q] - T_II[p,p'] V[p',q])
//                    + sum_{q'<q} (V[p,q'] T_JJ[q',q] - T_IJ[p,q'] U_JJ[q',q])
//   signs equal:   (u_pp + u_qq) v_pq = -y_pq - sum_{p'>p} U_II[p,p'] V[p',q]
//                                              - sum_{q'<q} V[p,q'] U_JJ[q',q]
// The terms without V are summed first for all entries (C below); then v_pq
// is computed by anti-diagonal s = (B-1-p) + q, since v_pq depends on V
// entries below it in its column and left of it in its row only.
// ---------------------------------------------------------------------------
// general = true: U is phi(T) for a general function phi (Algorithm 2 with
// this partition, the blocks' Sylvester equations solved by the same
// element recurrence): every entry comes from TU = UT, with u_pp - u_qq the
// difference of the diagonal values of phi already in U, and py0 is unused.
template <int B>
__device__ __forceinline__ void offdiag_leaf_body(int n, const double *__restrict__ T, int ldt,
                                                  double *__restrict__ U, int ldu, int I, int J, int nsplit,
                                                  const double *__restrict__ px0, const double *__restrict__ py0,
                                                  size_t split_stride, bool general = false)
{
    constexpr int LD = B + 1;
    extern __shared__ double sm[];
    double *TI = sm;
    double *UI = TI + B * LD;
    double *TJ = UI + B * LD;
    double *UJ = TJ + B * LD;
    double *V = UJ + B * LD;
    double *C = V + B * LD;
    __shared__ double srow[B], scol[B];
    const int r0 = I * B, c0 = J * B;
    const int bj = min(B, n - c0);

    for (int idx = threadIdx.x; idx < B * B; idx += kThreads) {
        const int i = idx % B, j = idx / B;
        const bool up = (i <= j);
        TI[i + j * LD] = up ? SGT_AT(T, ldt, r0 + i, r0 + j) : 0.0;
        UI[i + j * LD] = up ? SGT_AT(U, ldu, r0 + i, r0 + j) : 0.0;
        const bool inJ = up && (j < bj);
        TJ[i + j * LD] = inJ ? SGT_AT(T, ldt, c0 + i, c0 + j) : 0.0;
        UJ[i + j * LD] = inJ ? SGT_AT(U, ldu, c0 + i, c0 + j) : 0.0;
        V[i + j * LD] = (j < bj) ? SGT_AT(T, ldt, r0 + i, c0 + j) : 0.0;   // T_IJ for now
    }
    for (int i = threadIdx.x; i < B; i += kThreads) {
        srow[i] = general ? SGT_AT(U, ldu, r0 + i, r0 + i) : sgn(SGT_AT(T, ldt, r0 + i, r0 + i));
        scol[i] = (i < bj) ? (general ? SGT_AT(U, ldu, c0 + i, c0 + i) : sgn(SGT_AT(T, ldt, c0 + i, c0 + i))) : 1.0;
    }
    __syncthreads();

    for (int idx = threadIdx.x; idx < B * bj; idx += kThreads) {
        const int p = idx % B, q = idx / B;
        const double up = srow[p], uq = scol[q];
        double c;
        if (general || up + uq == 0.0) {
            double x = 0.0;
            for (int s = 0; s < nsplit; s++) x += px0[(size_t)s * split_stride + p + q * B];
            double a = 0.0, b = 0.0;
            for (int k = p + 1; k < B; k++) a = fma(UI[p + k * LD], V[k + q * LD], a);
            for (int k = 0; k < q; k++) b = fma(V[p + k * LD], UJ[k + q * LD], b);
            c = V[p + q * LD] * (up - uq) + x + a - b;
        } else {
            double y = 0.0;
            for (int s = 0; s < nsplit; s++) y += py0[(size_t)s * split_stride + p + q * B];
            c = -y;
        }
        C[p + q * LD] = c;
    }
    __syncthreads();

    // each entry's two in-block sums are split over four consecutive lanes
    // (terms k = part mod 4) and reduced by shuffles, so that every warp
    // shares the float64 work of an anti-diagonal step
    static_assert(kThreads == 4 * 64 && B <= 64, "one entry slot per four lanes");
    const int nsteps = B + bj - 1;
    const int part = threadIdx.x & 3, slot = threadIdx.x >> 2;
    for (int s = 0; s < nsteps; s++) {
        const int plo = max(0, B - 1 - s);
        const int phi = min(B - 1, B - 1 - s + bj - 1);
        const int p = plo + slot;
        const bool live = p <= phi;
        const int q = s - (B - 1 - p);
        double up = 1.0, uq = 1.0;
        if (live) {
            up = srow[p];
            uq = scol[q];
        }
        const bool opp = general || (up + uq == 0.0);
        // the entry's reciprocal divisor, on the group's fourth lane while
        // the sums run (it does not depend on them)
        double rinv = 0.0;
        if (live && part == 3) rinv = opp ? 1.0 / (TI[p + p * LD] - TJ[q + q * LD]) : 1.0 / (up + uq);
        double a = 0.0, b = 0.0;
        if (live) {
            const double *A = opp ? TI : UI;
            const double *Bm = opp ? TJ : UJ;
            for (int k = p + 1 + part; k < B; k += 4) a = fma(A[p + k * LD], V[k + q * LD], a);
            for (int k = part; k < q; k += 4) b = fma(V[p + k * LD], Bm[k + q * LD], b);
        }
        a += __shfl_xor_sync(0xffffffffu, a, 1);
        b += __shfl_xor_sync(0xffffffffu, b, 1);
        a += __shfl_xor_sync(0xffffffffu, a, 2);
        b += __shfl_xor_sync(0xffffffffu, b, 2);
        rinv = __shfl_sync(0xffffffffu, rinv, (threadIdx.x & 31) | 3);
        if (live && part == 0) V[p + q * LD] = (opp ? C[p + q * LD] - a + b : C[p + q * LD] - a - b) * rinv;
        __syncthreads();
    }
    for (int idx = threadIdx.x; idx < B * bj; idx += kThreads) {
        const int i = idx % B, j = idx / B;
        SGT_AT(U, ldu, r0 + i, c0 + j) = V[i + j * LD];
    }
}

template <int B>
constexpr size_t diag_smem() { return 2 * (size_t)B * (B + 1) * sizeof(double); }
template <int B>
constexpr size_t leaf_smem() { return 6 * (size_t)B * (B + 1) * sizeof(double); }

}  // namespace ph
}  // namespace signtri

// ps_fp64.cu -- Parlett-Sylvester for the sign function, float64
// (Section 2, Section 3, Section 5.1).
//
// With the eigenvalues grouped by sign, positives first, T~ = [T11 T12; 0 T22]
// and sign(T~) = [I X; 0 -I] where T11 X - X T22 = 2 T12 (the off-diagonal
// block of T~ U~ = U~ T~).  For a general order, T = Q T~ Q^T with Q
// orthogonal from adjacent Givens swaps (Schur reordering), and
// sign(T) = Q sign(T~) Q^T.  Three steps:
//
//  1. Reorder by sign.  A swap of neighbours (k, k+1) with diagonal a, c and
//     coupling b uses the rotation G = [cs -sn; sn cs], (cs, sn) = (b, c-a)/r,
//     r = hypot(b, c-a): G's first column is the eigenvector of c, so
//     G^T [a b; 0 c] G = [c b; 0 a], and T <- G^T T G on rows/columns k, k+1,
//     Q <- Q G.  Swaps of disjoint neighbour pairs commute (each rotation
//     depends only on its own 2x2 diagonal block, and left and right
//     multiplications commute), so the stable partition runs as odd-even
//     transposition rounds: in round r every pair (k, k+1), k = r mod 2, with
//     a negative above a positive is swapped at once.  The total number of
//     swaps is k = #{i<j : t_ii < 0 < t_jj}, the minimum (Section 3).  From
//     n = 512 on the same swaps run by windows instead (reorder_tc.cu).
//  2. Triangular Sylvester solve A X - X B = C by the element recurrence
//     (a_ii - b_jj) x_ij = c_ij - sum_{k>i} a_ik x_kj + sum_{k<j} x_ik b_kj,
//     blocked: b x b blocks by anti-diagonal (bottom-left first), float64 block
//     sums of the finished blocks (split along K, fixed summation order), then
//     the recurrence inside each block.
//  3. Back-transform: with Q = [Q1 Q2] (n x n_+, n x n_-),
//     Q U~ Q^T = I + (Q1 X - 2 Q2) Q2^T = -I + Q1 (2 Q1^T + X Q2^T);
//     the form with the smaller inner dimension is used, as two
//     emulated-float64 tensor-core products (slices.cu), only the tiles that
//     meet the upper triangle of U are formed, and the diagonal is set to
//     sign(t_ii) exactly.
#include <algorithm>
#include <vector>

#include "df_arith.cuh"
#include "internal.cuh"
#include "reorder_schedule.h"

namespace signtri {

namespace {

constexpr int kThreads = 256;
constexpr int SB = 64;            // Sylvester block size
constexpr int kSplitMax = 32;
constexpr int kTargetCtas = 4 * 152;

// --------------------------------------------------------------- reorder ---

// Rotation of every pair of round r: exact swap of the 2x2 diagonal block.
__global__ void givens_rot_kernel(const int *__restrict__ pairs, int npairs, double *__restrict__ T, int ldt,
                                  double *__restrict__ cs, double *__restrict__ sn, int *__restrict__ act_round,
                                  int round)
{
    const int idx = blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= npairs) return;
    const int k = pairs[idx];
    const double a = SGT_AT(T, ldt, k, k), c = SGT_AT(T, ldt, k + 1, k + 1), b = SGT_AT(T, ldt, k, k + 1);
    const double d = c - a;
    const double r = hypot(b, d);
    cs[k] = b / r;
    sn[k] = d / r;
    SGT_AT(T, ldt, k, k) = c;
    SGT_AT(T, ldt, k + 1, k + 1) = a;
    act_round[k] = round;
    act_round[k + 1] = round;
}

// Apply the rotations of round r.  blockIdx.y = pair, blockIdx.z = kind:
//   0: rows k, k+1, columns j >= k+2 (left product; joint 2x2 update where
//      column j starts another active pair of this round),
//   1: rows i < k not in an active pair, columns k, k+1 (right product),
//   2: Q, all rows, columns k, k+1 (right product).
__global__ void givens_apply_kernel(const int *__restrict__ pairs, int n, double *__restrict__ T, int ldt,
                                    double *__restrict__ Q, int ldq, const double *__restrict__ cs,
                                    const double *__restrict__ sn, const int *__restrict__ act_round, int round)
{
    const int k = pairs[blockIdx.y];
    const double c1 = cs[k], s1 = sn[k];
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    const int kind = blockIdx.z;
    if (kind == 0) {
        const int j = k + 2 + t;
        if (j >= n) return;
        const bool jact = (act_round[j] == round);
        const bool jfirst = jact && ((j & 1) == (round & 1));
        if (jact && !jfirst) return;               // handled with its partner
        double *x0 = &SGT_AT(T, ldt, k, j);
        double *x1 = &SGT_AT(T, ldt, k + 1, j);
        const double u = *x0, v = *x1;
        const double nu = c1 * u + s1 * v;          // G^T on rows k, k+1
        const double nv = -s1 * u + c1 * v;
        if (!jact) {
            *x0 = nu;
            *x1 = nv;
        } else {
            const double c2 = cs[j], s2 = sn[j];
            double *y0 = &SGT_AT(T, ldt, k, j + 1);
            double *y1 = &SGT_AT(T, ldt, k + 1, j + 1);
            const double up = *y0, vp = *y1;
            const double nup = c1 * up + s1 * vp;
            const double nvp = -s1 * up + c1 * vp;
            *x0 = nu * c2 + nup * s2;                // then G on columns j, j+1
            *y0 = -nu * s2 + nup * c2;
            *x1 = nv * c2 + nvp * s2;
            *y1 = -nv * s2 + nvp * c2;
        }
    } else if (kind == 1) {
        const int i = t;
        if (i >= k) return;
        if (act_round[i] == round) return;          // row pair: handled in kind 0
        double *x0 = &SGT_AT(T, ldt, i, k);
        double *x1 = &SGT_AT(T, ldt, i, k + 1);
        const double u = *x0, v = *x1;
        *x0 = u * c1 + v * s1;
        *x1 = -u * s1 + v * c1;
    } else {
        const int i = t;
        if (i >= n) return;
        double *x0 = &SGT_AT(Q, ldq, i, k);
        double *x1 = &SGT_AT(Q, ldq, i, k + 1);
        const double u = *x0, v = *x1;
        *x0 = u * c1 + v * s1;
        *x1 = -u * s1 + v * c1;
    }
}

// dst (upper triangle, zeros below) = src; Q = I.
__global__ void copy_upper_identity_kernel(int n, const double *__restrict__ src, int lds, double *__restrict__ dst,
                                           int ldd, double *__restrict__ Q, int ldq)
{
    const int j = blockIdx.x;
    for (int i = threadIdx.x; i < n; i += blockDim.x) {
        SGT_AT(dst, ldd, i, j) = (i <= j) ? SGT_AT(src, lds, i, j) : 0.0;
        SGT_AT(Q, ldq, i, j) = (i == j) ? 1.0 : 0.0;
    }
}

// ------------------------------------------------------------- Sylvester ---

// Double-float (fp32 hi + lo) arithmetic for the Sylvester block sums.
// GB300 issues float64 at about 1/64 of its fp32 rate, so the sums run as
// double-float products on the fp32 pipes: each float64 operand is cut into
// hi (its leading 24 significand bits) and lo (the next 29, rounded to 24)
// by split_df (df_arith.cuh, integer operations only); a product term is
// a_h b_h (Dekker's exact product by FMA) + a_h b_l + a_l b_h, accumulated
// with Knuth's two-sum.  About 2^-47 relative per term, summed in a fixed
// order; values beyond fp32's exponent range (below 2^-126 or from 2^128)
// are not represented (the first flush to 0; inputs and solutions here stay
// far inside the range).

// acc += a b in double-float (acc_h, acc_l unnormalised between renormalisations)
__device__ __forceinline__ void df_mac(float &ah_acc, float &al_acc, float a_h, float a_l, float b_h, float b_l)
{
    const float p = __fmul_rn(a_h, b_h);
    float e = __fmaf_rn(a_h, b_h, -p);
    e = __fmaf_rn(a_h, b_l, e);
    e = __fmaf_rn(a_l, b_h, e);
    const float s = __fadd_rn(ah_acc, p);
    const float bb = __fsub_rn(s, ah_acc);
    const float err = __fadd_rn(__fsub_rn(ah_acc, __fsub_rn(s, bb)), __fsub_rn(p, bb));
    ah_acc = s;
    al_acc = __fadd_rn(al_acc, __fadd_rn(err, e));
}

__device__ __forceinline__ void df_renorm(float &h, float &l)
{
    const float s = __fadd_rn(h, l);
    l = __fsub_rn(l, __fsub_rn(s, h));
    h = s;
}

// Block sums of anti-diagonal s for A X - X B = C (m x p), block (I, J) with
// I = nbr - 1 - s + J:  P = -sum_{I'>I} A[I, I'] X[I', J] + sum_{J'<J} X[I, J'] B[J', J].
// The s K-blocks of a tile are numbered v = 0..s-1: first the row blocks
// I' = I+1.. (the last may be partial), then the column blocks J' = 0..J-1.
// Operands staged in shared memory as double-float pairs; each thread keeps
// a 4 x 4 set of double-float accumulators, renormalised after every chunk
// of KT terms; the float64 partial written is hi + lo.
__global__ void __launch_bounds__(kThreads)
sylv_sums_kernel(int m, int p, const double *__restrict__ A, int lda, const double *__restrict__ Bm, int ldb,
                 const double *__restrict__ X, int ldx, int s, int nbr, int j_lo, int kc, double *__restrict__ P,
                 size_t split_stride)
{
    constexpr int KT = 16;
    __shared__ float Ah[KT][SB], Al[KT][SB], Bh[KT][SB], Bl[KT][SB];
    const int J = j_lo + blockIdx.x;
    const int I = nbr - 1 - s + J;
    const int split = blockIdx.y;
    const int v0 = split * kc, v1 = min(v0 + kc, s);
    const int r0 = I * SB, c0 = J * SB;
    const int bi = min(SB, m - r0), bj = min(SB, p - c0);
    const int nrow_blocks = nbr - 1 - I;
    const int tx = threadIdx.x % 16, ty = threadIdx.x / 16;
    float acc_h[4][4], acc_l[4][4];
#pragma unroll
    for (int a = 0; a < 4; a++)
#pragma unroll
        for (int b = 0; b < 4; b++) acc_h[a][b] = acc_l[a][b] = 0.f;
    for (int v = v0; v < v1; v++) {
        const bool phase1 = v < nrow_blocks;
        const int kb = phase1 ? (I + 1 + v) : (v - nrow_blocks);
        const int k_base = kb * SB;
        const int kext = phase1 ? min(SB, m - k_base) : SB;
        for (int k0 = 0; k0 < kext; k0 += KT) {
            for (int idx = threadIdx.x; idx < SB * KT; idx += kThreads) {
                const int r = idx % SB, kk = idx / SB;
                const int gk = k0 + kk;
                double av = 0.0;
                if (r < bi && gk < kext)
                    av = phase1 ? -SGT_AT(A, lda, r0 + r, k_base + gk) : SGT_AT(X, ldx, r0 + r, k_base + gk);
                split_df(av, Ah[kk][r], Al[kk][r]);
            }
            for (int idx = threadIdx.x; idx < SB * KT; idx += kThreads) {
                const int kk = idx % KT, c = idx / KT;
                const int gk = k0 + kk;
                double bv = 0.0;
                if (c < bj && gk < kext)
                    bv = phase1 ? SGT_AT(X, ldx, k_base + gk, c0 + c) : SGT_AT(Bm, ldb, k_base + gk, c0 + c);
                split_df(bv, Bh[kk][c], Bl[kk][c]);
            }
            __syncthreads();
#pragma unroll 4
            for (int kk = 0; kk < KT; kk++) {
                float ah[4], al[4], bh[4], bl[4];
#pragma unroll
                for (int q = 0; q < 4; q++) {
                    ah[q] = Ah[kk][tx + 16 * q];
                    al[q] = Al[kk][tx + 16 * q];
                    bh[q] = Bh[kk][ty + 16 * q];
                    bl[q] = Bl[kk][ty + 16 * q];
                }
#pragma unroll
                for (int pp = 0; pp < 4; pp++)
#pragma unroll
                    for (int q = 0; q < 4; q++) df_mac(acc_h[pp][q], acc_l[pp][q], ah[pp], al[pp], bh[q], bl[q]);
            }
#pragma unroll
            for (int pp = 0; pp < 4; pp++)
#pragma unroll
                for (int q = 0; q < 4; q++) df_renorm(acc_h[pp][q], acc_l[pp][q]);
            __syncthreads();
        }
    }
    double *out = P + (size_t)split * split_stride + (size_t)blockIdx.x * SB * SB;
#pragma unroll
    for (int pp = 0; pp < 4; pp++)
#pragma unroll
        for (int q = 0; q < 4; q++)
            out[(tx + 16 * pp) + (ty + 16 * q) * SB] = (double)acc_h[pp][q] + (double)acc_l[pp][q];
}

// In-block recurrence for block (I, J) of anti-diagonal s:
//   (a_pp - b_qq) x_pq = cscale*c_pq + sums_pq - sum_{p'>p} A[p,p'] x_p'q + sum_{q'<q} x_pq' B[q',q]
// The in-block sums run in double-float on the fp32 pipes (as the block
// sums above), each entry's terms split over four consecutive lanes and
// reduced by shuffles; the seed, the division and x_pq itself stay float64
// (x_pq is kept in both forms: float64 for the output, double-float for
// the sums of later entries).
__device__ __forceinline__ void df_add_df(float &h, float &l, float oh, float ol)
{
    const float s = __fadd_rn(h, oh);
    const float bb = __fsub_rn(s, h);
    const float err = __fadd_rn(__fsub_rn(h, __fsub_rn(s, bb)), __fsub_rn(oh, bb));
    h = s;
    l = __fadd_rn(l, __fadd_rn(ol, err));
}

constexpr int kLeafLD = SB + 1;
constexpr size_t kLeafSmem = 6 * (size_t)SB * kLeafLD * sizeof(float) + (size_t)SB * kLeafLD * sizeof(double) +
                             2 * (size_t)SB * sizeof(double);

__global__ void __launch_bounds__(kThreads)
sylv_leaf_kernel(int m, int p, const double *__restrict__ A, int lda, const double *__restrict__ Bm, int ldb,
                 const double *__restrict__ C, int ldc, double cscale, double *__restrict__ X, int ldx, int s,
                 int nbr, int j_lo, int nsplit, const double *__restrict__ P, size_t split_stride)
{
    constexpr int LD = kLeafLD;
    extern __shared__ double sm[];
    double *Xs = sm;                                   // float64 x (seeds, then results)
    double *ad = Xs + SB * LD, *bd = ad + SB;          // diagonals of the blocks of A and B
    float *Ah = reinterpret_cast<float *>(bd + SB), *Al = Ah + SB * LD;
    float *Bh = Al + SB * LD, *Bl = Bh + SB * LD;
    float *Xh = Bl + SB * LD, *Xl = Xh + SB * LD;
    const int J = j_lo + blockIdx.x;
    const int I = nbr - 1 - s + J;
    const int r0 = I * SB, c0 = J * SB;
    const int bi = min(SB, m - r0), bj = min(SB, p - c0);
    for (int idx = threadIdx.x; idx < SB * SB; idx += kThreads) {
        const int i = idx % SB, j = idx / SB;
        const double a = (i <= j && j < bi) ? SGT_AT(A, lda, r0 + i, r0 + j) : 0.0;
        const double b = (i <= j && j < bj) ? SGT_AT(Bm, ldb, c0 + i, c0 + j) : 0.0;
        split_df(a, Ah[i + j * LD], Al[i + j * LD]);
        split_df(b, Bh[i + j * LD], Bl[i + j * LD]);
        if (i == j) {
            ad[i] = a;
            bd[i] = b;
        }
        double c = 0.0;
        if (i < bi && j < bj) {
            c = cscale * SGT_AT(C, ldc, r0 + i, c0 + j);
            for (int t = 0; t < nsplit; t++) c += P[(size_t)t * split_stride + (size_t)blockIdx.x * SB * SB + i + j * SB];
        }
        Xs[i + j * LD] = c;
        Xh[i + j * LD] = 0.f;
        Xl[i + j * LD] = 0.f;
    }
    __syncthreads();
    const int nsteps = bi + bj - 1;
    const int part = threadIdx.x & 3, slot = threadIdx.x >> 2;   // 64 entry slots
    for (int st = 0; st < nsteps; st++) {
        const int plo = max(0, bi - 1 - st);
        const int phi = min(bi - 1, bi - 1 - st + bj - 1);
        const int pp = plo + slot;
        const bool live = pp <= phi;
        const int q = st - (bi - 1 - pp);
        // the entry's reciprocal divisor, on the group's fourth lane while
        // the sums run (it does not depend on them)
        double rinv = 0.0;
        if (live && part == 3) rinv = 1.0 / (ad[pp] - bd[q]);
        float h = 0.f, l = 0.f;
        if (live) {
            for (int k = pp + 1 + part; k < bi; k += 4)
                df_mac(h, l, -Ah[pp + k * LD], -Al[pp + k * LD], Xh[k + q * LD], Xl[k + q * LD]);
            for (int k = part; k < q; k += 4)
                df_mac(h, l, Xh[pp + k * LD], Xl[pp + k * LD], Bh[k + q * LD], Bl[k + q * LD]);
        }
        df_add_df(h, l, __shfl_xor_sync(0xffffffffu, h, 1), __shfl_xor_sync(0xffffffffu, l, 1));
        df_add_df(h, l, __shfl_xor_sync(0xffffffffu, h, 2), __shfl_xor_sync(0xffffffffu, l, 2));
        rinv = __shfl_sync(0xffffffffu, rinv, (threadIdx.x & 31) | 3);
        if (live && part == 0) {
            const double x = (Xs[pp + q * LD] + ((double)h + (double)l)) * rinv;
            Xs[pp + q * LD] = x;
            split_df(x, Xh[pp + q * LD], Xl[pp + q * LD]);
        }
        __syncthreads();
    }
    for (int idx = threadIdx.x; idx < bi * bj; idx += kThreads) {
        const int i = idx % bi, j = idx / bi;
        SGT_AT(X, ldx, r0 + i, c0 + j) = Xs[i + j * LD];
    }
}

// ---------------------------------------------------------- back-transform ---

// dst += alpha op(src) (rows x cols; op = transpose when asked), a CTA per column.
__global__ void add_scaled_kernel(int rows, int cols, const double *__restrict__ src, int lds, double alpha,
                                  bool transpose, double *__restrict__ dst, int ldd)
{
    const int j = blockIdx.x;
    for (int i = threadIdx.x; i < rows; i += blockDim.x)
        SGT_AT(dst, ldd, i, j) += alpha * (transpose ? SGT_AT(src, lds, j, i) : SGT_AT(src, lds, i, j));
}

// Diagonal of U set to sign(t_ii) of the input, strictly lower part to 0.
__global__ void finish_sign_kernel(int n, const double *__restrict__ T, int ldt, double *__restrict__ U, int ldu)
{
    const int j = blockIdx.x;
    for (int i = threadIdx.x; i < n; i += blockDim.x) {
        if (i == j) SGT_AT(U, ldu, i, j) = SGT_AT(T, ldt, i, i) > 0.0 ? 1.0 : -1.0;
        else if (i > j) SGT_AT(U, ldu, i, j) = 0.0;
    }
}

// U = [I X; 0 -I] for the sorted case (X already in place).
__global__ void sorted_blocks_kernel(int n, int npos, double *__restrict__ U, int ldu)
{
    const int j = blockIdx.x;
    for (int i = threadIdx.x; i < n; i += blockDim.x) {
        const bool in_x = (i < npos && j >= npos);
        if (!in_x) SGT_AT(U, ldu, i, j) = (i == j) ? (j < npos ? 1.0 : -1.0) : 0.0;
    }
}

}  // namespace

size_t sylvester_workspace_bytes(int m, int p)
{
    if (m <= 0 || p <= 0) return 0;
    const size_t nbr = (m + SB - 1) / SB, nbc = (p + SB - 1) / SB;
    const size_t tiles = std::min(nbr, nbc);
    return tiles * SB * SB * kSplitMax * sizeof(double) + 256;
}

signtri_status sylvester_run(int m, int p, const double *A, int lda, const double *Bm, int ldb, const double *C,
                             int ldc, double cscale, double *X, int ldx, Arena &ws, cudaStream_t st)
{
    if (m <= 0 || p <= 0) return SIGNTRI_OK;
    const int nbr = (m + SB - 1) / SB, nbc = (p + SB - 1) / SB;
    const size_t split_stride = (size_t)std::min(nbr, nbc) * SB * SB;
    double *P = static_cast<double *>(ws.take(split_stride * kSplitMax * sizeof(double)));
    if (!P) return SIGNTRI_ERR_NO_WORKSPACE;
    const size_t leaf_smem = kLeafSmem;
    SGT_CUDA_TRY(cudaFuncSetAttribute(sylv_leaf_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)leaf_smem));
    const int nsteps = nbr + nbc - 1;
    for (int s = 0; s < nsteps; s++) {
        const int j_lo = std::max(0, s - (nbr - 1));
        const int j_hi = std::min(nbc - 1, s);
        const int ntiles = j_hi - j_lo + 1;
        int nsplit = 0;
        if (s > 0) {
            const int want = (kTargetCtas + ntiles - 1) / ntiles;
            nsplit = std::max(1, std::min(want, std::min(kSplitMax, s)));
            const int kc = (s + nsplit - 1) / nsplit;
            nsplit = (s + kc - 1) / kc;
            ProfScope ps(SIGNTRI_KC_SYLV_SUMS, st);
            sylv_sums_kernel<<<dim3(ntiles, nsplit), kThreads, 0, st>>>(m, p, A, lda, Bm, ldb, X, ldx, s, nbr, j_lo,
                                                                       kc, P, split_stride);
            SGT_LAUNCH_CHECK();
        }
        ProfScope ps(SIGNTRI_KC_SYLV_LEAF, st);
        sylv_leaf_kernel<<<ntiles, kThreads, leaf_smem, st>>>(m, p, A, lda, Bm, ldb, C, ldc, cscale, X, ldx, s, nbr,
                                                               j_lo, nsplit, P, split_stride);
        SGT_LAUNCH_CHECK();
    }
    return SIGNTRI_OK;
}

signtri_status copy_upper_identity(int n, const double *T, int ldt, double *Tr, int ldtr, double *Q, int ldq,
                                   cudaStream_t st)
{
    ProfScope ps(SIGNTRI_KC_FILL, st);
    copy_upper_identity_kernel<<<n, 256, 0, st>>>(n, T, ldt, Tr, ldtr, Q, ldq);
    SGT_LAUNCH_CHECK();
    return SIGNTRI_OK;
}

size_t reorder_workspace_bytes(int n)
{
    if (n <= 0) return 0;
    // cs, sn, act_round; the pair list is sized per call (at most n^2/4)
    return 3 * ((size_t)n * sizeof(double) + 256);
}

signtri_status reorder_run(int n, const double *T, int ldt, double *Tr, int ldtr, double *Q, int ldq,
                           long long *swaps_out, Arena &ws, cudaStream_t st)
{
    if (n <= 0) return SIGNTRI_OK;
    double *cs = static_cast<double *>(ws.take((size_t)n * sizeof(double)));
    double *sn = static_cast<double *>(ws.take((size_t)n * sizeof(double)));
    int *act = static_cast<int *>(ws.take((size_t)n * sizeof(int)));
    if (!cs || !sn || !act) return SIGNTRI_ERR_NO_WORKSPACE;
    {
        ProfScope ps(SIGNTRI_KC_FILL, st);
        copy_upper_identity_kernel<<<n, 256, 0, st>>>(n, T, ldt, Tr, ldtr, Q, ldq);
        SGT_LAUNCH_CHECK();
    }
    SGT_CUDA_TRY(cudaMemsetAsync(act, 0xff, (size_t)n * sizeof(int), st));
    std::vector<double> diag(n);
    SGT_CUDA_TRY(cudaMemcpy2DAsync(diag.data(), sizeof(double), T, ((size_t)ldt + 1) * sizeof(double), sizeof(double),
                                   n, cudaMemcpyDeviceToHost, st));
    SGT_CUDA_TRY(cudaStreamSynchronize(st));
    std::vector<int> pairs, offsets;
    schedule_rounds(diag, pairs, offsets);
    if (swaps_out) *swaps_out = (long long)pairs.size();
    if (pairs.empty()) return SIGNTRI_OK;
    int *d_pairs = static_cast<int *>(ws.take(pairs.size() * sizeof(int)));
    if (!d_pairs) return SIGNTRI_ERR_NO_WORKSPACE;
    SGT_CUDA_TRY(cudaMemcpyAsync(d_pairs, pairs.data(), pairs.size() * sizeof(int), cudaMemcpyHostToDevice, st));
    const int nrounds = (int)offsets.size() - 1;
    for (int r = 0; r < nrounds; r++) {
        const int off = offsets[r], np = offsets[r + 1] - offsets[r];
        if (np == 0) continue;
        ProfScope ps(SIGNTRI_KC_GIVENS, st);
        givens_rot_kernel<<<(np + 127) / 128, 128, 0, st>>>(d_pairs + off, np, Tr, ldtr, cs, sn, act, r);
        SGT_LAUNCH_CHECK();
        givens_apply_kernel<<<dim3((n + 255) / 256, np, 3), 256, 0, st>>>(d_pairs + off, n, Tr, ldtr, Q, ldq, cs, sn,
                                                                          act, r);
        SGT_LAUNCH_CHECK();
    }
    // the pair list must stay valid until the copy above has been consumed
    SGT_CUDA_TRY(cudaStreamSynchronize(st));
    return SIGNTRI_OK;
}

size_t reorder_any_workspace_bytes(int n, long long swaps)
{
    return n >= kBlockedReorderMin ? reorder_blocked_workspace_bytes(n)
                                   : reorder_workspace_bytes(n) + (size_t)std::max(swaps, 0LL) * sizeof(int) + 256;
}

signtri_status reorder_any_run(int n, const double *T, int ldt, double *Tr, int ldtr, double *Q, int ldq,
                               long long *swaps_out, Arena &ws, int *d_err, cudaStream_t st)
{
    return n >= kBlockedReorderMin ? reorder_blocked_run(n, T, ldt, Tr, ldtr, Q, ldq, swaps_out, ws, d_err, st)
                                   : reorder_run(n, T, ldt, Tr, ldtr, Q, ldq, swaps_out, ws, st);
}

// the back-transform's two products, one after the other in the same space
static size_t back_transform_workspace_bytes(int n, int npos)
{
    const int nneg = n - npos;
    if (nneg <= npos)
        return std::max(emulated_product_workspace_bytes(n, nneg, npos), emulated_product_workspace_bytes(n, n, nneg));
    return std::max(emulated_product_workspace_bytes(npos, n, nneg), emulated_product_workspace_bytes(n, n, npos));
}

size_t ps_workspace_bytes(int n, long long swaps)
{
    if (n <= 0) return 0;
    const size_t nn = (size_t)n * n * sizeof(double) + 256;
    size_t b = sylvester_workspace_bytes(n, n) + nn /* X */;
    if (swaps > 0) {
        // T~, Q, W; then the reorder's space, reused by the Sylvester solve and
        // the back-transform (bounded over every inertia)
        size_t bt = 0;
        for (int npos = 1; npos < n; npos = npos < 128 ? npos + 1 : npos + 64)
            bt = std::max(bt, back_transform_workspace_bytes(n, npos));
        bt = std::max(bt, back_transform_workspace_bytes(n, n - 1));
        b += 3 * nn + std::max(reorder_any_workspace_bytes(n, swaps), bt) + 256;
    }
    return b;
}

signtri_status ps_fp64_run(int n, const double *T, int ldt, double *U, int ldu, int npos, long long swaps,
                           Arena &ws, int *d_err, cudaStream_t st)
{
    const int nneg = n - npos;
    if (swaps == 0) {
        // already grouped: T~ = T, Q = I, sign(T) = [I X; 0 -I]
        signtri_status rs = sylvester_run(npos, nneg, T, ldt, &SGT_AT(T, ldt, npos, npos), ldt, &SGT_AT(T, ldt, 0, npos),
                                          ldt, 2.0, &SGT_AT(U, ldu, 0, npos), ldu, ws, st);
        if (rs != SIGNTRI_OK) return rs;
        ProfScope ps(SIGNTRI_KC_FILL, st);
        sorted_blocks_kernel<<<n, 256, 0, st>>>(n, npos, U, ldu);
        SGT_LAUNCH_CHECK();
        return SIGNTRI_OK;
    }
    double *Tr = static_cast<double *>(ws.take((size_t)n * n * sizeof(double)));
    double *Q = static_cast<double *>(ws.take((size_t)n * n * sizeof(double)));
    double *X = static_cast<double *>(ws.take((size_t)n * n * sizeof(double)));
    double *W = static_cast<double *>(ws.take((size_t)n * n * sizeof(double)));
    if (!Tr || !Q || !X || !W) return SIGNTRI_ERR_NO_WORKSPACE;
    const size_t mark = ws.used;
    long long done = 0;
    signtri_status rs = reorder_any_run(n, T, ldt, Tr, n, Q, n, &done, ws, d_err, st);
    if (rs != SIGNTRI_OK) return rs;
    ws.used = mark;   // the reorder's scratch is free again (stream order)
    rs = sylvester_run(npos, nneg, Tr, n, &SGT_AT(Tr, n, npos, npos), n, &SGT_AT(Tr, n, 0, npos), n, 2.0, X, npos,
                       ws, st);
    if (rs != SIGNTRI_OK) return rs;
    ws.used = mark;
    const double *Q1 = Q;
    const double *Q2 = &SGT_AT(Q, n, 0, npos);
    // the back-transform U = Q sign(T~) Q^T, as emulated-float64 tensor-core
    // products, in the form whose inner dimension is the smaller block
    if (nneg <= npos) {
        // W = Q1 X - 2 Q2 (n x n_-),  U = I + W Q2^T
        rs = emulated_product(n, nneg, npos, Q1, n, X, npos, false, W, n, false, SIGNTRI_KC_GEMM_F64, ws, d_err, st);
        if (rs != SIGNTRI_OK) return rs;
        ws.used = mark;
        {
            ProfScope ps(SIGNTRI_KC_FILL, st);
            add_scaled_kernel<<<nneg, 256, 0, st>>>(n, nneg, Q2, n, -2.0, false, W, n);
            SGT_LAUNCH_CHECK();
        }
        rs = emulated_product(n, n, nneg, W, n, Q2, n, true, U, ldu, true, SIGNTRI_KC_GEMM_F64, ws, d_err, st);
    } else {
        // W = 2 Q1^T + X Q2^T (n_+ x n),  U = -I + Q1 W
        rs = emulated_product(npos, n, nneg, X, npos, Q2, n, true, W, npos, false, SIGNTRI_KC_GEMM_F64, ws, d_err, st);
        if (rs != SIGNTRI_OK) return rs;
        ws.used = mark;
        {
            ProfScope ps(SIGNTRI_KC_FILL, st);
            add_scaled_kernel<<<n, 256, 0, st>>>(npos, n, Q1, n, 2.0, true, W, npos);
            SGT_LAUNCH_CHECK();
        }
        rs = emulated_product(n, n, npos, Q1, n, W, npos, false, U, ldu, true, SIGNTRI_KC_GEMM_F64, ws, d_err, st);
    }
    if (rs != SIGNTRI_OK) return rs;
    ProfScope ps(SIGNTRI_KC_FILL, st);
    finish_sign_kernel<<<n, 256, 0, st>>>(n, T, ldt, U, ldu);
    SGT_LAUNCH_CHECK();
    return SIGNTRI_OK;
}

}  // namespace signtri

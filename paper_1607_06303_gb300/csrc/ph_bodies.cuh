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
// Block sums for anti-diagonal d: for block (I, J = I+d) and K-blocks
// [kb0, kb1) of the split s,
//     PX[s][I] = sum_K U_IK T_KJ - T_IK U_KJ,   PY[s][I] = sum_K U_IK U_KJ.
// One CTA per (I, s), B x B output tile, 256 threads, (B/16)^2 outputs per
// thread for each of X and Y, K staged through shared memory in steps of 16.
// ---------------------------------------------------------------------------
template <int B>
__device__ __forceinline__ void ph_gemm_body(int n, const double *__restrict__ T, int ldt,
                                             const double *__restrict__ U, int ldu, int I, int J, int kb0, int kb1,
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

    for (int k0 = kb0 * B; k0 < kb1 * B; k0 += KT) {
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
template <int B>
__device__ __forceinline__ void offdiag_leaf_body(int n, const double *__restrict__ T, int ldt,
                                                  double *__restrict__ U, int ldu, int I, int J, int nsplit,
                                                  const double *__restrict__ px0, const double *__restrict__ py0,
                                                  size_t split_stride)
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
        srow[i] = sgn(SGT_AT(T, ldt, r0 + i, r0 + i));
        scol[i] = (i < bj) ? sgn(SGT_AT(T, ldt, c0 + i, c0 + i)) : 1.0;
    }
    __syncthreads();

    for (int idx = threadIdx.x; idx < B * bj; idx += kThreads) {
        const int p = idx % B, q = idx / B;
        const double up = srow[p], uq = scol[q];
        double c;
        if (up + uq == 0.0) {
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

    const int nsteps = B + bj - 1;
    for (int s = 0; s < nsteps; s++) {
        const int plo = max(0, B - 1 - s);
        const int phi = min(B - 1, B - 1 - s + bj - 1);
        for (int p = plo + threadIdx.x; p <= phi; p += kThreads) {
            const int q = s - (B - 1 - p);
            const double up = srow[p], uq = scol[q];
            const bool opp = (up + uq == 0.0);
            const double *A = opp ? TI : UI;
            const double *Bm = opp ? TJ : UJ;
            double a = 0.0, b = 0.0;
            for (int k = p + 1; k < B; k++) a = fma(A[p + k * LD], V[k + q * LD], a);
            for (int k = 0; k < q; k++) b = fma(V[p + k * LD], Bm[k + q * LD], b);
            double v;
            if (opp) v = (C[p + q * LD] - a + b) / (TI[p + p * LD] - TJ[q + q * LD]);
            else     v = (C[p + q * LD] - a - b) / (up + uq);
            V[p + q * LD] = v;
        }
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

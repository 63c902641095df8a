// schur.cu -- the complex Schur decomposition A = Q T Q^H of a general real A
// on the GPU: the first step of the paper's route to sign(A) = Q sign(T) Q^H
// for a general matrix (Section 1; Algorithm 3 starts from a complex Schur
// form).
//
// Two textbook stages (Golub and Van Loan, Matrix Computations, 4th ed.,
// Sections 7.4-7.5):
//  1. Householder reduction to upper Hessenberg form H = Q0^T A Q0, float64.
//     For column k a reflector P = I - tau v v^T (v_0 = 1) maps A[k+1:, k]
//     onto beta e_1; it is applied from the left to the columns right of k
//     (one CTA per column: the column's dot product with v, then the
//     update) and from the right to the rows of A and of Q0 (the products
//     with v, 32 rows per CTA, then the rank-1 update).  Four launches per
//     column.
//  2. Implicitly shifted QR iteration on H in complex float64.  A complex
//     shift needs no double-shift pairing, so every sweep over the active
//     window [l, i] is a chain of plane rotations: the first from
//     (h_ll - sigma, h_{l+1,l}), each later one zeroing the bulge
//     h_{k+1,k-1}; each rotation G acts on rows k, k+1 of H over all columns
//     and G^H on columns k, k+1 over the rows that hold nonzeros (so H
//     becomes all of T, not just its diagonal) and on Q's columns.  The
//     shift is Wilkinson's (the eigenvalue of the window's trailing 2 x 2
//     nearer its last diagonal entry), with an ad hoc shift every tenth
//     sweep without a deflation; h_{k,k-1} is negligible, and set to 0, when
//     |h_{k,k-1}| <= eps (|h_{k-1,k-1}| + |h_kk|) (|z| = |Re z| + |Im z|).
//     Deflation takes the window's last row when its subdiagonal entry is
//     negligible.  The rotations of a sweep depend on one another (each reads
//     what the one before wrote), so one cluster of 16 CTAs (8 where the
//     device cannot place 16) runs the sweeps with a cluster barrier per
//     rotation or rotation pair, applying each to the active window only
//     (schur_qr_kernel says how the work is split); a launch runs sweeps
//     until a rotation budget is spent and logs them, then a kernel on the
//     other SMs applies the logged rotations to the columns right of each
//     sweep's window and to Q, on a second stream while the next launch
//     runs, and the host relaunches until the window is empty.
//     The chain of rotations bounds the stage: about 3 sweeps per eigenvalue
//     (4 counting each bulge's), ~1.9 n^2 rotations for n eigenvalues in
//     ~0.9 n^2 dependent steps (n = 1024), each a few thousand cycles of
//     float64 latency and a barrier -- the decomposition is the
//     general-matrix front end, not a tuned hot path.
//
// Layout: A real column-major; Q, T complex interleaved (re, im) float64
// pairs, column-major, leading dimensions counted in complex elements.
#include <algorithm>
#include <cfloat>
#include <climits>

#include <cooperative_groups.h>

#include "internal.cuh"

namespace signtri {

namespace {

constexpr int kThreads = 256;
constexpr int kQrThreads = 512;
constexpr int kMaxSweepsPerEigenvalue = 100;
constexpr long long kRotationBudget = 1LL << 15;   // rotations per launch of the QR kernel (then a sweep's end)

#define SGT_A(M, ld, i, j) (M)[(size_t)(i) + (size_t)(j) * (size_t)(ld)]

__device__ __forceinline__ double2 cmul(double2 a, double2 b)
{
    return make_double2(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}
__device__ __forceinline__ double2 cconj(double2 a) { return make_double2(a.x, -a.y); }
__device__ __forceinline__ double cabs1(double2 a) { return fabs(a.x) + fabs(a.y); }
// a / b by Smith's algorithm (R. L. Smith, CACM 5(8), 1962)
__device__ __forceinline__ double2 cdiv(double2 a, double2 b)
{
    if (fabs(b.x) >= fabs(b.y)) {
        const double r = b.y / b.x, den = b.x + b.y * r;
        return make_double2((a.x + a.y * r) / den, (a.y - a.x * r) / den);
    }
    const double r = b.x / b.y, den = b.x * r + b.y;
    return make_double2((a.x * r + a.y) / den, (a.y * r - a.x) / den);
}
// principal square root (Re >= 0): with r = |z|, sqrt((r + |Re z|) / 2) is
// the larger part, the other is Im z over twice it
__device__ __forceinline__ double2 csqrt_p(double2 z)
{
    if (z.x == 0.0 && z.y == 0.0) return make_double2(0.0, 0.0);
    const double a = sqrt(0.5 * (hypot(z.x, z.y) + fabs(z.x)));
    const double b = z.y / (2.0 * a);
    return z.x >= 0.0 ? make_double2(a, b) : make_double2(fabs(b), copysign(a, z.y));
}

// The rotation G = [c s; -conj(s) c] (c real >= 0, c^2 + |s|^2 = 1) with
// G [x; y] = [r; 0]: c = |x| / nrm, s = (x / |x|) conj(y) / nrm,
// nrm^2 = |x|^2 + |y|^2.  x and y are first scaled by the power of two that
// brings their largest component into [1, 2) (exact), so the squares
// neither overflow nor lose range (below 2^-1000 the scale stops at 2^1000);
// then two reciprocal square roots and
// products (the rotation sits on the QR sweep's serial chain, where each
// float64 division or hypot costs a long dependent sequence).
__device__ __forceinline__ void make_rotation(double2 x, double2 y, double &c, double2 &s)
{
    const double my = fmax(fabs(y.x), fabs(y.y));
    if (my == 0.0) {
        c = 1.0;
        s = make_double2(0.0, 0.0);
        return;
    }
    const double m = fmax(my, fmax(fabs(x.x), fabs(x.y)));
    const double sc = ldexp(1.0, -max(ilogb(m), -1000));   // 2^1000 at most (m subnormal)
    const double2 xs = make_double2(x.x * sc, x.y * sc), ys = make_double2(y.x * sc, y.y * sc);
    const double ax2 = fma(xs.x, xs.x, xs.y * xs.y), ay2 = fma(ys.x, ys.x, ys.y * ys.y);
    if (ax2 == 0.0) {
        const double r = rsqrt(ay2);
        c = 0.0;
        s = make_double2(ys.x * r, -ys.y * r);
        return;
    }
    const double inv_n = rsqrt(ax2 + ay2), inv_ax = rsqrt(ax2);
    c = ax2 * inv_ax * inv_n;
    const double2 t = cmul(xs, cconj(ys));
    const double f = inv_ax * inv_n;
    s = make_double2(t.x * f, t.y * f);
}

// (a, b) of rows k, k+1 in one column -> G (a, b)
__device__ __forceinline__ void rot_rows(double c, double2 s, double2 &a, double2 &b)
{
    const double2 sa = cmul(s, b), sb = cmul(cconj(s), a);
    const double2 na = make_double2(c * a.x + sa.x, c * a.y + sa.y);
    const double2 nb = make_double2(c * b.x - sb.x, c * b.y - sb.y);
    a = na;
    b = nb;
}
// (a, b) of columns k, k+1 in one row -> (a, b) G^H
__device__ __forceinline__ void rot_cols(double c, double2 s, double2 &a, double2 &b)
{
    const double2 sa = cmul(cconj(s), b), sb = cmul(s, a);
    const double2 na = make_double2(c * a.x + sa.x, c * a.y + sa.y);
    const double2 nb = make_double2(c * b.x - sb.x, c * b.y - sb.y);
    a = na;
    b = nb;
}

// ------------------------------------------------------------- Hessenberg --

// First non-finite entry (its column) of A, into *bad (atomicMin).
__global__ void finite_check_kernel(int n, const double *__restrict__ A, int lda, int *__restrict__ bad)
{
    const int j = blockIdx.x;
    for (int i = threadIdx.x; i < n; i += blockDim.x)
        if (!isfinite(SGT_A(A, lda, i, j))) atomicMin(bad, j);
}

// H = A (a working copy), Q0 = I
__global__ void hess_init_kernel(int n, const double *__restrict__ A, int lda, double *__restrict__ H,
                                 double *__restrict__ Q0)
{
    const int j = blockIdx.x;
    for (int i = threadIdx.x; i < n; i += blockDim.x) {
        SGT_A(H, n, i, j) = SGT_A(A, lda, i, j);
        SGT_A(Q0, n, i, j) = (i == j) ? 1.0 : 0.0;
    }
}

__device__ __forceinline__ double block_sum(double x, double *red)
{
    for (int o = 16; o > 0; o >>= 1) x += __shfl_xor_sync(0xffffffffu, x, o);
    const int w = threadIdx.x / 32, nw = blockDim.x / 32;
    __syncthreads();
    if ((threadIdx.x & 31) == 0) red[w] = x;
    __syncthreads();
    double s = 0.0;
    for (int k = 0; k < nw; k++) s += red[k];   // same order in every thread
    return s;
}

__device__ __forceinline__ double block_max(double x, double *red)
{
    for (int o = 16; o > 0; o >>= 1) x = fmax(x, __shfl_xor_sync(0xffffffffu, x, o));
    const int w = threadIdx.x / 32, nw = blockDim.x / 32;
    __syncthreads();
    if ((threadIdx.x & 31) == 0) red[w] = x;
    __syncthreads();
    double s = 0.0;
    for (int k = 0; k < nw; k++) s = fmax(s, red[k]);
    return s;
}

// The reflector of column k: x = H[k+1:, k] (m = n - k - 1 entries),
// alpha = x_0, beta = -sign(alpha) ||x||, tau = (beta - alpha) / beta,
// v = x / (alpha - beta) with v_0 = 1; column k becomes (beta, 0, ...).
// tau = 0 (P = I) when x_1.. are all zero.  One CTA.
__global__ void house_kernel(int n, int k, double *__restrict__ H, double *__restrict__ v, double *__restrict__ tau)
{
    __shared__ double red[32];
    const int m = n - k - 1;
    double *x = &SGT_A(H, n, k + 1, k);
    double mx = 0.0;
    for (int i = 1 + threadIdx.x; i < m; i += blockDim.x) mx = fmax(mx, fabs(x[i]));
    mx = block_max(mx, red);
    if (mx == 0.0) {
        for (int i = threadIdx.x; i < m; i += blockDim.x) v[i] = (i == 0) ? 1.0 : 0.0;
        if (threadIdx.x == 0) *tau = 0.0;
        return;
    }
    // ||x_1..|| scaled by its largest magnitude (no overflow or underflow)
    double ss = 0.0;
    for (int i = 1 + threadIdx.x; i < m; i += blockDim.x) {
        const double t = x[i] / mx;
        ss = fma(t, t, ss);
    }
    ss = block_sum(ss, red);
    const double xnorm = mx * sqrt(ss);
    const double alpha = x[0];
    const double beta = -copysign(hypot(alpha, xnorm), alpha);
    const double scal = 1.0 / (alpha - beta);
    for (int i = threadIdx.x; i < m; i += blockDim.x) v[i] = (i == 0) ? 1.0 : x[i] * scal;
    __syncthreads();   // every x[i] read before column k is overwritten
    for (int i = threadIdx.x; i < m; i += blockDim.x) x[i] = (i == 0) ? beta : 0.0;
    if (threadIdx.x == 0) *tau = (beta - alpha) / beta;
}

// H[k+1:, j] -= tau v (v^T H[k+1:, j]) for the columns j > k: one CTA each.
__global__ void house_left_kernel(int n, int k, double *__restrict__ H, const double *__restrict__ v,
                                  const double *__restrict__ tau)
{
    __shared__ double red[32];
    const double t = *tau;
    if (t == 0.0) return;
    const int j = k + 1 + blockIdx.x;
    const int m = n - k - 1;
    double *col = &SGT_A(H, n, k + 1, j);
    double w = 0.0;
    for (int i = threadIdx.x; i < m; i += blockDim.x) w = fma(v[i], col[i], w);
    w = block_sum(w, red) * t;
    for (int i = threadIdx.x; i < m; i += blockDim.x) col[i] = fma(-v[i], w, col[i]);
}

// The right application M[r, k+1:] -= tau (M[r, k+1:] v) v^T to the rows of
// H (r < n) and of Q0 (r >= n), in two launches: y_r = tau M[r, k+1:] v with
// 32 rows per CTA (lane = row, so each column's 32 entries are one
// coalesced read) and the columns split over the 8 warps, then the rank-1
// update with a CTA per column.
constexpr int kGemvWarps = 8;
__global__ void __launch_bounds__(32 * kGemvWarps)
house_gemv_kernel(int n, int k, const double *__restrict__ H, const double *__restrict__ Q0,
                  const double *__restrict__ v, const double *__restrict__ tau, double *__restrict__ y)
{
    __shared__ double part[kGemvWarps][32];
    const double t = *tau;
    if (t == 0.0) return;
    const int lane = threadIdx.x % 32, w = threadIdx.x / 32;
    const int g = blockIdx.x * 32 + lane;
    const int m = n - k - 1;
    double acc = 0.0;
    if (g < 2 * n) {
        const double *M = g < n ? H : Q0;
        const int r = g < n ? g : g - n;
        for (int j = w; j < m; j += kGemvWarps) acc = fma(SGT_A(M, n, r, k + 1 + j), v[j], acc);
    }
    part[w][lane] = acc;
    __syncthreads();
    if (w == 0 && g < 2 * n) {
        double sum = 0.0;
        for (int q = 0; q < kGemvWarps; q++) sum += part[q][lane];
        y[g] = t * sum;
    }
}

__global__ void house_rank1_kernel(int n, int k, double *__restrict__ H, double *__restrict__ Q0,
                                   const double *__restrict__ v, const double *__restrict__ tau,
                                   const double *__restrict__ y)
{
    if (*tau == 0.0) return;
    const int j = k + 1 + blockIdx.x;
    const double vj = v[blockIdx.x];
    for (int g = threadIdx.x; g < 2 * n; g += blockDim.x) {
        double *M = g < n ? H : Q0;
        const int r = g < n ? g : g - n;
        SGT_A(M, n, r, j) = fma(-y[g], vj, SGT_A(M, n, r, j));
    }
}

// complex T = H with its entries below the subdiagonal exactly 0; complex Q = Q0
__global__ void to_complex_kernel(int n, const double *__restrict__ H, const double *__restrict__ Q0,
                                  double2 *__restrict__ T, int ldt, double2 *__restrict__ Q, int ldq)
{
    const int j = blockIdx.x;
    for (int i = threadIdx.x; i < n; i += blockDim.x) {
        SGT_A(T, ldt, i, j) = make_double2(i <= j + 1 ? SGT_A(H, n, i, j) : 0.0, 0.0);
        SGT_A(Q, ldq, i, j) = make_double2(SGT_A(Q0, n, i, j), 0.0);
    }
}

// ---------------------------------------------------------- QR iteration --

struct QrState {
    int ihi;          // last row of the active window (-1: all converged)
    int its;          // sweeps since the last deflation
    int status;       // 0 running, 1 converged, 2 no convergence
    long long sweeps;
    long long rotations;
};

// A sweep of the last launch: its window [l, i] and where its i - l
// rotations start in the rotation log.
struct SweepRec {
    int l, i;
    long long off;
};

__global__ void qr_state_init_kernel(int n, QrState *st)
{
    st->ihi = n - 1;
    st->its = 0;
    st->status = 0;
    st->sweeps = 0;
    st->rotations = 0;
}

// One cluster of CL CTAs runs the sweeps, one or two bulges at a time.
// Two bulges: both eigenvalues of the window's trailing 2 x 2 as shifts
// (Francis's double shift, in complex arithmetic as two single shifts), the
// second bulge started 3 steps behind the first; mathematically the two
// sweeps one after the other (the rotations of the front sweep that touch
// the rear bulge's rows and columns are all done before it gets there, and
// the later ones act on disjoint rows and columns), with half the dependent
// steps.  On GB300 a float64 warp instruction holds its SM sub-partition's
// float64 pipe for ~64 cycles whatever the number of active lanes (and
// rsqrt or a division for ~430), so the kernel is laid out around float64
// instruction counts:
//  * CTA 0's warp b (chief warp of bulge b) runs that chase's serial part
//    alone on its sub-partition: the 2 x 2 block at (k, k) and row k+2 of
//    columns k, k+1, where the next rotation's inputs (h_{k+1,k}, h_{k+2,k})
//    are formed, lane-parallel (one real output per lane: 8 lanes for G's
//    action on the block's two columns, 12 for G^H's on its three rows, 3
//    float64 instructions each), kept in registers from step to step; the
//    entry left of the block (h_{k,k-1}, zeroing the old bulge) from the
//    rotation's own inputs; then the next rotation, its two reciprocal
//    square roots in lanes 0 and 1 at once, stored into every CTA's shared
//    memory (two slots per bulge, alternating).  The one entry of the next
//    block that another thread writes, h_{k+1,k+2} (row op of column k+2),
//    comes through shared memory; the front chase loads the entries no step
//    touches before (h_{k+2,k+2}, h_{k+3,k+2}) two steps ahead, the rear
//    chase takes them from the front chief, who wrote them one and zero
//    steps before (h_{k+2,k+2} as its block's corner, h_{k+3,k+2} as the
//    entry left of its block), or from T once the front chase has ended.
//  * CTAs 1.. do the rest of every rotation (rows k, k+1 across the window,
//    columns k, k+1 above the block) and, with two bulges, the 2 x 2 block
//    at the rear bulge's rows and the front bulge's columns, which takes the
//    rear rotation from the left and the front one from the right; entry e
//    goes to warp e / 32 of a sequence that alternates CTAs and
//    sub-partitions, so the work fills whole warps spread over the cluster.
// One cluster barrier per step; no entry is written by one thread while
// another reads it.  CTA 0 alone takes every decision (deflation, shifts,
// stop) and broadcasts it, so all CTAs run the same barriers.  T is read with
// L2-only loads (another CTA may have written it since).  The rotations'
// action on the columns right of the window (rows there are never read by a
// later sweep: the window only shrinks) and on Q is left to
// apply_rotations_kernel, which runs on other SMs alongside the next launch:
// this kernel logs each sweep and its rotations instead (the rear sweep after
// the front one).
constexpr int kMaxBulges = 2;
enum { kActSweep = 0, kActDeflate = 1, kActStop = 2 };

__device__ __forceinline__ double2 ldT(const double2 *p) { return __ldcg(p); }
// the unbiased exponent field of |x| (integer operations only)
__device__ __forceinline__ int exp_field(double x)
{
    return (int)(((unsigned long long)__double_as_longlong(x) >> 52) & 0x7ff) - 1023;
}

__device__ __forceinline__ bool is_zero2(double2 v)
{
    return (((unsigned long long)__double_as_longlong(v.x) | (unsigned long long)__double_as_longlong(v.y)) << 1) == 0;
}

// make_rotation for the chief warp (x, y the same in every lane; every lane
// gets (c, s)): zero tests and the exponent-range test by integer operations
// on the bits; without scaling when every component's exponent lies in
// [-400, 400] (else make_rotation); |x|^2 and |y|^2, the two reciprocal
// square roots, and the two parts of x conj(y) f each in lanes 0 and 1 of
// one instruction stream.
__device__ __forceinline__ void make_rotation_warp(double2 x, double2 y, int lane, double &c, double2 &s)
{
    if (is_zero2(y)) {
        c = 1.0;
        s = make_double2(0.0, 0.0);
        return;
    }
    const int em = max(max(exp_field(y.x), exp_field(y.y)), max(exp_field(x.x), exp_field(x.y)));
    if (em > 400 || em < -400 || is_zero2(x)) {
        make_rotation(x, y, c, s);
        return;
    }
    const bool l1 = lane & 1;
    const double2 v = l1 ? y : x;
    const double sq = fma(v.x, v.x, v.y * v.y);   // lane 0 |x|^2, lane 1 |y|^2
    const double ax2 = __shfl_sync(0xffffffffu, sq, 0), ay2 = __shfl_sync(0xffffffffu, sq, 1);
    // lane 0: Re(x conj(y)) = x.x y.x + x.y y.y; lane 1: Im = x.y y.x - x.x y.y
    const double tt = fma(l1 ? x.y : x.x, y.x, (l1 ? -x.x : x.y) * y.y);
    const double r = rsqrt(l1 ? ax2 : ax2 + ay2);   // lane 0 1/nrm, lane 1 1/|x|
    const double inv_n = __shfl_sync(0xffffffffu, r, 0), inv_ax = __shfl_sync(0xffffffffu, r, 1);
    const double f = inv_ax * inv_n;
    c = ax2 * f;
    const double sp = tt * f;
    s = make_double2(__shfl_sync(0xffffffffu, sp, 0), __shfl_sync(0xffffffffu, sp, 1));
}

// One real output of G or G^H acting on a pair, in one of the chief warp's
// lanes: out = c alpha + beta gamma + delta epsilon (3 float64 instructions).
__device__ __forceinline__ double pair_part(double c, double alpha, double beta, double gamma, double delta,
                                            double epsilon)
{
    return fma(c, alpha, fma(beta, gamma, delta * epsilon));
}

template <int CL>
__global__ void __launch_bounds__(kQrThreads)
schur_qr_kernel(int n, double2 *__restrict__ T, int ldt, QrState *__restrict__ st, long long budget,
                SweepRec *__restrict__ sweeplog, double *__restrict__ rclog, double2 *__restrict__ rslog,
                int *__restrict__ nlogged)
{
    namespace cg = cooperative_groups;
    constexpr int kWorkers = CL - 1, kWorkerThreads = kWorkers * kQrThreads;   // CTAs 1..
    cg::cluster_group cl = cg::this_cluster();
    __shared__ int redi[kQrThreads / 32];
    __shared__ double rc[kMaxBulges][2];
    __shared__ double2 rs[kMaxBulges][2];
    __shared__ double2 bslot[kMaxBulges][2];   // CTA 0: h_{k+1,k+2} after a step, per bulge
    __shared__ double2 handF[2], handH[2];       // CTA 0: the front chief's corner and left entry, per step
    __shared__ double2 sig1;                     // CTA 0: the rear bulge's shift
    __shared__ int ctl[4];                       // action, l, i, bulges (CTA 0's decision)
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const unsigned crank = cl.block_rank();
    const int cb = (crank == 0 && warp < kMaxBulges) ? warp : -1;   // the bulge of a chief warp
    const bool chief0 = crank == 0 && warp == 0;
    // this worker thread's first entry and the stride (CTAs 1.. only)
    const int e0 = ((warp * kWorkers + ((int)crank - 1)) << 5) + lane;
    int i = st->ihi, its = st->its, status = st->status;
    long long logged = 0, rot = 0;
    const double eps = DBL_EPSILON;
    const double tiny = DBL_MIN * ((double)n / DBL_EPSILON);
    const double2 zero = make_double2(0.0, 0.0);
    // a chief warp's registers, the same in every lane: the block (A B; E F)
    // at (k, k), Hh = h_{k+2,k+1}, the rotation of the step and its inputs
    // (X, Y) = (h_{k,k-1}, h_{k+1,k-1})
    double2 A = zero, B = zero, E = zero, F = zero, Hh = zero, X = zero, Y = zero, s_cur = zero;
    double c_cur = 1.0;
    double2 pf_f = zero, pf_h = zero;   // front chase: h_{k+2,k+2}, h_{k+3,k+2} for step k+1, loaded early
    auto put_rotation = [&](int b, int slot, double c, double2 s) {
        // lanes 0..CL-1 of a chief warp store into CTA `lane`
        if (lane < CL) {
            *cl.map_shared_rank(&rc[b][slot], lane) = c;
            *cl.map_shared_rank(&rs[b][slot], lane) = s;
        }
    };
    for (;;) {
        if (crank == 0) {
            // l: the largest k in [1, i] whose h_{k,k-1} is negligible, else 0
            int lk = 0;
            for (int k = 1 + tid; k <= i; k += kQrThreads) {
                const double sub = cabs1(ldT(&SGT_A(T, ldt, k, k - 1)));
                const double ref = cabs1(ldT(&SGT_A(T, ldt, k - 1, k - 1))) + cabs1(ldT(&SGT_A(T, ldt, k, k)));
                if (sub <= fmax(eps * ref, tiny)) lk = k;
            }
            for (int o = 16; o > 0; o >>= 1) lk = max(lk, __shfl_xor_sync(0xffffffffu, lk, o));
            if (lane == 0) redi[warp] = lk;
            __syncthreads();
            if (chief0) {
                int l = 0;
                for (int w = 0; w < kQrThreads / 32; w++) l = max(l, redi[w]);
                int act, nbul = 1;
                if (status != 0 || i <= 0) {
                    act = kActStop;
                    if (status == 0) {
                        status = 1;
                        i = -1;
                    }
                } else if (l == i) {
                    act = kActDeflate;   // the window's last row has converged
                    if (lane == 0) SGT_A(T, ldt, i, i - 1) = zero;
                } else if (rot >= budget) {
                    act = kActStop;
                } else if (its >= kMaxSweepsPerEigenvalue) {
                    act = kActStop;
                    status = 2;
                } else {
                    act = kActSweep;
                    if (l > 0 && lane == 0) SGT_A(T, ldt, l, l - 1) = zero;
                    const int sw_its = its + 1;
                    double2 sigma;
                    if (sw_its % 10 == 0) {
                        // ad hoc shift, one bulge: off the window's top
                        // (sweeps 10, 30, ..) or bottom corner (20, 40, ..)
                        // by 3/4 of a subdiagonal entry's real part
                        const bool top = (sw_its / 10) % 2 == 1;
                        const double2 d = top ? ldT(&SGT_A(T, ldt, l, l)) : ldT(&SGT_A(T, ldt, i, i));
                        const double e = top ? ldT(&SGT_A(T, ldt, l + 1, l)).x : ldT(&SGT_A(T, ldt, i, i - 1)).x;
                        sigma = make_double2(d.x + 0.75 * fabs(e), d.y);
                    } else {
                        // Wilkinson: with x = (a - d) / 2 and y = sqrt(x^2 + bc)
                        // signed so that |x + y| is the larger, the eigenvalue
                        // of [a b; c d] nearer d is d - bc / (x + y); the
                        // other one, a + d minus it, shifts the rear bulge
                        const double2 a = ldT(&SGT_A(T, ldt, i - 1, i - 1)), b = ldT(&SGT_A(T, ldt, i - 1, i));
                        const double2 cc = ldT(&SGT_A(T, ldt, i, i - 1)), d = ldT(&SGT_A(T, ldt, i, i));
                        const double2 x = make_double2(0.5 * (a.x - d.x), 0.5 * (a.y - d.y));
                        const double2 bc = cmul(b, cc);
                        const double2 xx = cmul(x, x);
                        double2 y = csqrt_p(make_double2(xx.x + bc.x, xx.y + bc.y));
                        if (x.x * y.x + x.y * y.y < 0.0) y = make_double2(-y.x, -y.y);
                        const double2 xy = make_double2(x.x + y.x, x.y + y.y);
                        if (xy.x == 0.0 && xy.y == 0.0) {
                            sigma = d;
                        } else {
                            const double2 q = cdiv(bc, xy);
                            sigma = make_double2(d.x - q.x, d.y - q.y);
                        }
                        if (i - l >= 3) {
                            nbul = 2;
                            if (lane == 0) sig1 = make_double2(a.x + d.x - sigma.x, a.y + d.y - sigma.y);
                        }
                    }
                    A = ldT(&SGT_A(T, ldt, l, l));
                    B = ldT(&SGT_A(T, ldt, l, l + 1));
                    E = ldT(&SGT_A(T, ldt, l + 1, l));
                    F = ldT(&SGT_A(T, ldt, l + 1, l + 1));
                    Hh = (l + 2 <= i) ? ldT(&SGT_A(T, ldt, l + 2, l + 1)) : zero;
                    pf_f = (l + 2 <= i) ? ldT(&SGT_A(T, ldt, l + 2, l + 2)) : zero;
                    pf_h = (l + 3 <= i) ? ldT(&SGT_A(T, ldt, l + 3, l + 2)) : zero;
                    X = make_double2(A.x - sigma.x, A.y - sigma.y);
                    Y = E;
                    make_rotation_warp(X, Y, lane, c_cur, s_cur);
                    put_rotation(0, 0, c_cur, s_cur);
                    if (lane == 0) {
                        sweeplog[logged] = SweepRec{l, i, rot};
                        if (nbul == 2) sweeplog[logged + 1] = SweepRec{l, i, rot + (i - l)};
                        rclog[rot] = c_cur;
                        rslog[rot] = s_cur;
                    }
                }
                if (lane < CL) {
                    int *rem = cl.map_shared_rank(ctl, lane);
                    rem[0] = act;
                    rem[1] = l;
                    rem[2] = i;
                    rem[3] = nbul;
                }
            }
        }
        cl.sync();
        const int act = ctl[0], l = ctl[1], nbul = ctl[3];
        i = ctl[2];
        if (act == kActStop) break;
        if (act == kActDeflate) {
            i--;
            its = 0;
            continue;
        }
        its++;
        const int L = i - l, S = L + 3 * (nbul - 1);
        double2 Fnext = zero;   // rear chief: its block's next corner
        for (int s = 0; s < S; s++) {
            const int k0 = l + s, k1 = l + s - 3;
            const bool a0 = s < L;                    // front bulge at k0
            const bool a1 = nbul > 1 && s >= 3;       // rear bulge at k1 (s - 3 < L always)
            if (crank > 0) {
                const double c0 = rc[0][s & 1], c1 = rc[1][s & 1];
                const double2 s0 = rs[0][s & 1], s1 = rs[1][s & 1];
                // items: the 2 x 2 block where the two chases meet (rows
                // k1, k1+1 x columns k0, k0+1: the rear rotation from the
                // left, the front one from the right; two items, lanes 0
                // and 1 of the first warp, one column and then one row each);
                // front rows k0, k0+1 at columns k0+2..i; front columns k0,
                // k0+1 at rows 0..k0-1 (the rear rows apart); rear rows at
                // columns k1+2..i (the front columns apart); rear columns at
                // rows 0..k1-1
                const int xn = (a0 && a1) ? 2 : 0;
                const int r0n = a0 ? max(i - k0 - 1, 0) : 0, c0n = a0 ? k0 : 0;
                const int r1n = a1 ? max(i - k1 - 1, 0) : 0, c1n = a1 ? k1 : 0;
                const int wtot = xn + r0n + c0n + r1n + c1n;
                for (int e = e0; e < wtot; e += kWorkerThreads) {
                    int f = e;
                    if (f < xn) {
                        // lane f: column k0 + f through the rear rotation, then
                        // row k1 + f through the front one
                        const int j = k0 + f;
                        double2 a = ldT(&SGT_A(T, ldt, k1, j)), b = ldT(&SGT_A(T, ldt, k1 + 1, j));
                        rot_rows(c1, s1, a, b);
                        // lane 0 holds (row k1, row k1+1) of column k0, lane 1
                        // of column k0+1; row k1 + f needs both columns
                        const double2 mine = f ? b : a, theirs = f ? a : b;
                        const double2 other = make_double2(__shfl_xor_sync(0x3u, theirs.x, 1),
                                                           __shfl_xor_sync(0x3u, theirs.y, 1));
                        double2 p = f ? other : mine, q = f ? mine : other;
                        rot_cols(c0, s0, p, q);
                        SGT_A(T, ldt, k1 + f, k0) = p;
                        SGT_A(T, ldt, k1 + f, k0 + 1) = q;
                        continue;
                    }
                    f -= xn;
                    if (f < r0n) {
                        const int j = k0 + 2 + f;
                        double2 a = ldT(&SGT_A(T, ldt, k0, j)), b = ldT(&SGT_A(T, ldt, k0 + 1, j));
                        rot_rows(c0, s0, a, b);
                        SGT_A(T, ldt, k0, j) = a;
                        SGT_A(T, ldt, k0 + 1, j) = b;
                        if (f == 0) *cl.map_shared_rank(&bslot[0][(s + 1) & 1], 0) = b;
                        continue;
                    }
                    f -= r0n;
                    if (f < c0n) {
                        if (a1 && (f == k1 || f == k1 + 1)) continue;
                        double2 a = ldT(&SGT_A(T, ldt, f, k0)), b = ldT(&SGT_A(T, ldt, f, k0 + 1));
                        rot_cols(c0, s0, a, b);
                        SGT_A(T, ldt, f, k0) = a;
                        SGT_A(T, ldt, f, k0 + 1) = b;
                        continue;
                    }
                    f -= c0n;
                    if (f < r1n) {
                        const int j = k1 + 2 + f;
                        if (a0 && (j == k0 || j == k0 + 1)) continue;
                        double2 a = ldT(&SGT_A(T, ldt, k1, j)), b = ldT(&SGT_A(T, ldt, k1 + 1, j));
                        rot_rows(c1, s1, a, b);
                        SGT_A(T, ldt, k1, j) = a;
                        SGT_A(T, ldt, k1 + 1, j) = b;
                        if (f == 0) *cl.map_shared_rank(&bslot[1][(s + 1) & 1], 0) = b;
                        continue;
                    }
                    f -= r1n;
                    double2 a = ldT(&SGT_A(T, ldt, f, k1)), b = ldT(&SGT_A(T, ldt, f, k1 + 1));
                    rot_cols(c1, s1, a, b);
                    SGT_A(T, ldt, f, k1) = a;
                    SGT_A(T, ldt, f, k1 + 1) = b;
                }
            } else if (cb >= 0 && cb < nbul) {
                const int b = cb;
                if (b == 1 && s == 2) {
                    // the rear chase starts next step at (l, l): entries final
                    // since step 1 (h_{l+2,l+1} comes after this step, from the
                    // front chief), its first rotation from its own shift
                    A = ldT(&SGT_A(T, ldt, l, l));
                    B = ldT(&SGT_A(T, ldt, l, l + 1));
                    E = ldT(&SGT_A(T, ldt, l + 1, l));
                    F = ldT(&SGT_A(T, ldt, l + 1, l + 1));
                    const double2 sg = sig1;
                    X = make_double2(A.x - sg.x, A.y - sg.y);
                    Y = E;
                    make_rotation_warp(X, Y, lane, c_cur, s_cur);
                    put_rotation(1, 1, c_cur, s_cur);
                    if (lane == 0) {
                        rclog[rot + L] = c_cur;
                        rslog[rot + L] = s_cur;
                    }
                }
                const bool act_b = (b == 0) ? a0 : a1;
                if (act_b) {
                    const int kb = (b == 0) ? k0 : k1;
                    const double c = c_cur;
                    const double2 sn = s_cur;
                    double2 F2 = zero, H2 = zero;
                    if (b == 0) {
                        F2 = pf_f;
                        H2 = pf_h;
                        pf_f = (kb + 3 <= i) ? ldT(&SGT_A(T, ldt, kb + 3, kb + 3)) : zero;
                        pf_h = (kb + 4 <= i) ? ldT(&SGT_A(T, ldt, kb + 4, kb + 3)) : zero;
                    } else if (kb + 2 <= i) {
                        // the next corner h_{k+2,k+2}: the front chief's block
                        // corner of the previous step, or T once that chase ended
                        Fnext = (s - 1 < L) ? handF[(s - 1) & 1] : ldT(&SGT_A(T, ldt, kb + 2, kb + 2));
                    }
                    const int part = lane & 3;
                    const bool odd = part & 1, hi = part >= 2;
                    if (kb > l) {
                        // h_{k,k-1} = c X + s Y (the entry the rotation keeps),
                        // h_{k+1,k-1} = 0 (the bulge it zeroes): lanes 0-3
                        const double rz = pair_part(c, odd ? X.y : X.x, sn.x, odd ? Y.y : Y.x, odd ? sn.y : -sn.y,
                                                    odd ? Y.x : Y.y);
                        if (lane < 4)
                            reinterpret_cast<double *>(&SGT_A(T, ldt, kb + (hi ? 1 : 0), kb - 1))[odd ? 1 : 0] =
                                hi ? 0.0 : rz;
                        if (b == 0) {
                            const double2 r = make_double2(__shfl_sync(0xffffffffu, rz, 0),
                                                           __shfl_sync(0xffffffffu, rz, 1));
                            if (lane == 0) handH[s & 1] = r;
                        }
                    }
                    // G on the block's columns: lane 4 col + part holds part
                    // (0 top.x, 1 top.y, 2 bottom.x, 3 bottom.y) of column col
                    // (0: (A, E), 1: (B, F)) -- one real output per lane
                    // (operands picked by selects, no branches: all lanes run
                    // the same three float64 instructions)
                    const bool cl1 = (lane >> 2) & 1;
                    const double2 tp = cl1 ? B : A, bt = cl1 ? F : E;
                    const double2 u1 = hi ? bt : tp, v1 = hi ? tp : bt;
                    const double r1 = pair_part(c, odd ? u1.y : u1.x, hi ? -sn.x : sn.x, odd ? v1.y : v1.x,
                                                odd ? sn.y : -sn.y, odd ? v1.x : v1.y);
                    const double2 A1 = make_double2(__shfl_sync(0xffffffffu, r1, 0), __shfl_sync(0xffffffffu, r1, 1));
                    const double2 E1 = make_double2(__shfl_sync(0xffffffffu, r1, 2), __shfl_sync(0xffffffffu, r1, 3));
                    const double2 B1 = make_double2(__shfl_sync(0xffffffffu, r1, 4), __shfl_sync(0xffffffffu, r1, 5));
                    const double2 F1 = make_double2(__shfl_sync(0xffffffffu, r1, 6), __shfl_sync(0xffffffffu, r1, 7));
                    // G^H on the rows k, k+1, k+2: lane 4 row + part holds part
                    // (0 p.x, 1 p.y, 2 q.x, 3 q.y) of row (p, q): (A1, B1),
                    // (E1, F1), (0, Hh)
                    const int row = min(lane >> 2, 2);
                    const double2 pp = row == 0 ? A1 : (row == 1 ? E1 : zero);
                    const double2 qq = row == 0 ? B1 : (row == 1 ? F1 : Hh);
                    const double2 u2 = hi ? qq : pp, v2 = hi ? pp : qq;
                    const double r2 = pair_part(c, odd ? u2.y : u2.x, hi ? -sn.x : sn.x, odd ? v2.y : v2.x,
                                                odd ? -sn.y : sn.y, odd ? v2.x : v2.y);
                    if (lane < 8 || (lane < 12 && kb + 2 <= i))
                        reinterpret_cast<double *>(&SGT_A(T, ldt, kb + (lane >> 2), kb + (part >> 1)))[part & 1] = r2;
                    if (b == 0) {
                        // the block's corner h_kk, for the rear chief two steps on
                        const double2 corner = make_double2(__shfl_sync(0xffffffffu, r2, 0),
                                                            __shfl_sync(0xffffffffu, r2, 1));
                        if (lane == 0) handF[s & 1] = corner;
                    }
                    if (kb + 2 <= i) {
                        // the next rotation zeroes the bulge h_{k+2,k} (lanes 8, 9)
                        // against h_{k+1,k} (lanes 4, 5)
                        const double2 x = make_double2(__shfl_sync(0xffffffffu, r2, 4), __shfl_sync(0xffffffffu, r2, 5));
                        const double2 y = make_double2(__shfl_sync(0xffffffffu, r2, 8), __shfl_sync(0xffffffffu, r2, 9));
                        const double2 f1 = make_double2(__shfl_sync(0xffffffffu, r2, 6), __shfl_sync(0xffffffffu, r2, 7));
                        const double2 h1 = make_double2(__shfl_sync(0xffffffffu, r2, 10), __shfl_sync(0xffffffffu, r2, 11));
                        make_rotation_warp(x, y, lane, c_cur, s_cur);
                        put_rotation(b, (s + 1) & 1, c_cur, s_cur);
                        if (lane == 0) {
                            const long long at = rot + (long long)b * L + (kb + 1 - l);
                            rclog[at] = c_cur;
                            rslog[at] = s_cur;
                        }
                        X = x;
                        Y = y;
                        // the block at (k+1, k+1): (h_{k+1,k+1}, h_{k+1,k+2};
                        // h_{k+2,k+1}, h_{k+2,k+2}), h_{k+1,k+2} from bslot after
                        // the barrier, and h_{k+3,k+2}
                        A = f1;
                        E = h1;
                        F = (b == 0) ? F2 : Fnext;
                        if (b == 0) Hh = H2;
                    }
                }
            }
            cl.sync();
            if (cb >= 0 && cb < nbul) {
                const int b = cb;
                const bool act_b = (b == 0) ? a0 : a1;
                const int kb = (b == 0) ? k0 : k1;
                if (act_b && kb + 1 < i) B = bslot[b][(s + 1) & 1];
                if (b == 1) {
                    if (s == 2) {
                        Hh = (l + 2 <= i) ? handH[0] : zero;   // the front chief's h_{l+2,l+1} of step 2
                    } else if (a1 && kb + 3 <= i) {
                        // h_{k+3,k+2} for the next step: the front chief's
                        // left entry of this step, or T once that chase ended
                        Hh = a0 ? handH[s & 1] : ldT(&SGT_A(T, ldt, kb + 3, kb + 2));
                    } else if (a1) {
                        Hh = zero;
                    }
                }
            }
        }
        rot += (long long)nbul * L;
        logged += nbul;
    }
    if (chief0 && lane == 0) {
        st->ihi = i;
        st->its = its;
        st->status = status;
        *nlogged = (int)logged;
        st->sweeps += logged;
        st->rotations += rot;
    }
}

// The logged sweeps' rotations where schur_qr_kernel left them out: unit u
// < n is column u of T, which takes the row rotations of every sweep whose
// window ends above it (u > i), down the column with the carried row; unit
// u >= n is row u - n of Q, which takes every sweep's column rotations along
// the row.  In log order, so each entry sees its rotations in the order of
// the QR iteration.  Four lanes per unit, each computing one real output of
// a rotation (3 float64 instructions, where GB300's float64 pipe, not the
// memory, bounds this kernel), the carried entry passed by shuffles; the
// next entry is loaded an iteration ahead.
__global__ void apply_rotations_kernel(int n, double2 *__restrict__ T, int ldt, double2 *__restrict__ Q, int ldq,
                                       const int *__restrict__ nlogged, const SweepRec *__restrict__ sweeplog,
                                       const double *__restrict__ rclog, const double2 *__restrict__ rslog)
{
    const int g = blockIdx.x * blockDim.x + threadIdx.x;
    const int unit = g >> 2, part = g & 3;
    if (unit >= 2 * n) return;   // the four lanes of a unit leave together
    const unsigned gmask = 0xFu << (threadIdx.x & 28);
    const bool odd = part & 1, hi = part >= 2;
    const bool isT = unit < n;
    // entry k of the unit's line: T(k, j) (stride 1) or Q(r, k) (stride ldq)
    double2 *line = isT ? &SGT_A(T, ldt, 0, unit) : &SGT_A(Q, ldq, unit - n, 0);
    const size_t stride = isT ? 1 : (size_t)ldq;
    const int logged = *nlogged;
    for (int w = 0; w < logged; w++) {
        const SweepRec sr = sweeplog[w];
        if (isT && unit <= sr.i) continue;
        double2 a = line[(size_t)sr.l * stride];
        double2 b = line[(size_t)(sr.l + 1) * stride];
        for (int k = sr.l; k < sr.i; k++) {
            const double c = rclog[sr.off + (k - sr.l)];
            const double2 s = rslog[sr.off + (k - sr.l)];
            const double2 bn = (k + 2 <= sr.i) ? line[(size_t)(k + 2) * stride] : b;
            // G (T's rows) or G^H (Q's columns) on (a, b): lane part gives
            // part 0 a'.x, 1 a'.y, 2 b'.x, 3 b'.y
            const double2 u = hi ? b : a, v = hi ? a : b;
            const double sy = isT ? (odd ? s.y : -s.y) : (odd ? -s.y : s.y);
            const double r = pair_part(c, odd ? u.y : u.x, hi ? -s.x : s.x, odd ? v.y : v.x, sy, odd ? v.x : v.y);
            if (!hi) reinterpret_cast<double *>(&line[(size_t)k * stride])[part] = r;
            a = make_double2(__shfl_sync(gmask, r, 2, 4), __shfl_sync(gmask, r, 3, 4));
            b = bn;
        }
        if (part == 0) line[(size_t)sr.i * stride] = a;
    }
}

// T's strictly lower part -> 0 (what remains there is at most negligible)
__global__ void clear_lower_kernel(int n, double2 *__restrict__ T, int ldt)
{
    const int j = blockIdx.x;
    for (int i = j + 1 + threadIdx.x; i < n; i += blockDim.x) SGT_A(T, ldt, i, j) = make_double2(0.0, 0.0);
}

__global__ void real_part_kernel(int n, const double2 *__restrict__ Sc, double *__restrict__ S, int lds)
{
    const int j = blockIdx.x;
    for (int i = threadIdx.x; i < n; i += blockDim.x) SGT_A(S, lds, i, j) = SGT_A(Sc, n, i, j).x;
}

}  // namespace

namespace {

// The QR sweeps' cluster: 16 CTAs (a non-portable size: 15 worker CTAs
// halve the float64 work of each step's row and column updates, which the
// worker SMs' float64 pipes bound) where the device can place such a cluster
// of the kernel, else 8.
cudaLaunchConfig_t qr_config(int cl, cudaStream_t st, cudaLaunchAttribute *at)
{
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(cl, 1, 1);
    cfg.blockDim = dim3(kQrThreads, 1, 1);
    cfg.dynamicSmemBytes = 0;
    cfg.stream = st;
    at[0].id = cudaLaunchAttributeClusterDimension;
    at[0].val.clusterDim.x = cl;
    at[0].val.clusterDim.y = 1;
    at[0].val.clusterDim.z = 1;
    cfg.attrs = at;
    cfg.numAttrs = 1;
    return cfg;
}

int qr_cluster_size()
{
    if (cudaFuncSetAttribute(schur_qr_kernel<16>, cudaFuncAttributeNonPortableClusterSizeAllowed, 1) != cudaSuccess) {
        cudaGetLastError();
        return 8;
    }
    cudaLaunchAttribute at[1];
    const cudaLaunchConfig_t cfg = qr_config(16, nullptr, at);
    int clusters = 0;
    if (cudaOccupancyMaxActiveClusters(&clusters, schur_qr_kernel<16>, &cfg) != cudaSuccess) {
        cudaGetLastError();
        return 8;
    }
    return clusters >= 1 ? 16 : 8;
}

cudaError_t launch_qr(int cl, int n, double2 *T, int ldt, QrState *st, long long budget, SweepRec *sweeplog,
                      double *rclog, double2 *rslog, int *nlogged, cudaStream_t stream)
{
    cudaLaunchAttribute at[1];
    const cudaLaunchConfig_t cfg = qr_config(cl, stream, at);
    return cl == 16 ? cudaLaunchKernelEx(&cfg, schur_qr_kernel<16>, n, T, ldt, st, budget, sweeplog, rclog, rslog,
                                         nlogged)
                    : cudaLaunchKernelEx(&cfg, schur_qr_kernel<8>, n, T, ldt, st, budget, sweeplog, rclog, rslog,
                                         nlogged);
}

// The second stream of schur_run and its events.  Destroyed on every
// return, after the stream's work has finished (the caller may reuse the
// workspace the applies read and write as soon as schur_run returns).
struct ApplyStream {
    cudaStream_t s = nullptr;
    cudaEvent_t swept[2] = {}, applied[2] = {};
    cudaError_t init()
    {
        cudaError_t e = cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking);
        for (int p = 0; p < 2 && e == cudaSuccess; p++) {
            e = cudaEventCreateWithFlags(&swept[p], cudaEventDisableTiming);
            if (e == cudaSuccess) e = cudaEventCreateWithFlags(&applied[p], cudaEventDisableTiming);
        }
        return e;
    }
    ~ApplyStream()
    {
        if (s) {
            cudaStreamSynchronize(s);
            cudaStreamDestroy(s);
        }
        for (int p = 0; p < 2; p++) {
            if (swept[p]) cudaEventDestroy(swept[p]);
            if (applied[p]) cudaEventDestroy(applied[p]);
        }
    }
};

}  // namespace

size_t schur_workspace_bytes(int n)
{
    if (n <= 0) return 0;
    // eleven takes, each rounded up to 256 bytes; two logs of one launch each
    const size_t nn = (size_t)n * n;
    const size_t nlog = (size_t)kRotationBudget + (size_t)kMaxBulges * n + 2;
    return 2 * nn * sizeof(double) + 3 * (size_t)n * sizeof(double) + sizeof(double) + sizeof(int) + sizeof(QrState) +
           2 * nlog * (sizeof(SweepRec) + sizeof(double) + sizeof(double2)) + 2 * sizeof(int) + 11 * 256;
}

signtri_status schur_run(int n, const double *A, int lda, double *Q, int ldq, double *T, int ldt, Arena &ws,
                         int *bad_index, long long counts_out[2], cudaStream_t st)
{
    if (n <= 0) return SIGNTRI_OK;
    const size_t nn = (size_t)n * n;
    auto *H = static_cast<double *>(ws.take(nn * sizeof(double)));
    auto *Q0 = static_cast<double *>(ws.take(nn * sizeof(double)));
    auto *v = static_cast<double *>(ws.take((size_t)n * sizeof(double)));
    auto *y = static_cast<double *>(ws.take((size_t)2 * n * sizeof(double)));
    auto *tau = static_cast<double *>(ws.take(sizeof(double)));
    auto *bad = static_cast<int *>(ws.take(sizeof(int)));
    auto *qs = static_cast<QrState *>(ws.take(sizeof(QrState)));
    // a launch logs fewer than budget + 2n rotations (it starts a multi-sweep
    // only below the budget, a multi-sweep has at most 2 (n - 1)) and no
    // more sweeps; launches alternate between two logs
    const size_t nlog = (size_t)kRotationBudget + (size_t)kMaxBulges * n + 2;
    auto *sweeplog = static_cast<SweepRec *>(ws.take(2 * nlog * sizeof(SweepRec)));
    auto *rclog = static_cast<double *>(ws.take(2 * nlog * sizeof(double)));
    auto *rslog = static_cast<double2 *>(ws.take(2 * nlog * sizeof(double2)));
    auto *nlogged = static_cast<int *>(ws.take(2 * sizeof(int)));
    if (!H || !Q0 || !v || !y || !tau || !bad || !qs || !sweeplog || !rclog || !rslog || !nlogged)
        return SIGNTRI_ERR_NO_WORKSPACE;
    const int big = INT_MAX;
    SGT_CUDA_TRY(cudaMemcpyAsync(bad, &big, sizeof(int), cudaMemcpyHostToDevice, st));
    {
        ProfScope ps(SIGNTRI_KC_SCAN, st);
        finite_check_kernel<<<n, kThreads, 0, st>>>(n, A, lda, bad);
        SGT_LAUNCH_CHECK();
    }
    int first_bad = INT_MAX;
    SGT_CUDA_TRY(cudaMemcpyAsync(&first_bad, bad, sizeof(int), cudaMemcpyDeviceToHost, st));
    SGT_CUDA_TRY(cudaStreamSynchronize(st));
    if (first_bad != INT_MAX) {
        if (bad_index) *bad_index = first_bad;
        return SIGNTRI_ERR_NONFINITE;
    }
    {
        ProfScope ps(SIGNTRI_KC_FILL, st);
        hess_init_kernel<<<n, kThreads, 0, st>>>(n, A, lda, H, Q0);
        SGT_LAUNCH_CHECK();
    }
    for (int k = 0; k + 2 < n; k++) {
        ProfScope ps(SIGNTRI_KC_HESSENBERG, st, true, false);
        prof_count(SIGNTRI_KC_HESSENBERG, 4);
        house_kernel<<<1, 1024, 0, st>>>(n, k, H, v, tau);
        SGT_LAUNCH_CHECK();
        house_left_kernel<<<n - k - 1, kThreads, 0, st>>>(n, k, H, v, tau);
        SGT_LAUNCH_CHECK();
        house_gemv_kernel<<<(2 * n + 31) / 32, 32 * kGemvWarps, 0, st>>>(n, k, H, Q0, v, tau, y);
        SGT_LAUNCH_CHECK();
        house_rank1_kernel<<<n - k - 1, kThreads, 0, st>>>(n, k, H, Q0, v, tau, y);
        SGT_LAUNCH_CHECK();
    }
    auto *Tc = reinterpret_cast<double2 *>(T);
    auto *Qc = reinterpret_cast<double2 *>(Q);
    {
        ProfScope ps(SIGNTRI_KC_FILL, st);
        to_complex_kernel<<<n, kThreads, 0, st>>>(n, H, Q0, Tc, ldt, Qc, ldq);
        SGT_LAUNCH_CHECK();
        qr_state_init_kernel<<<1, 1, 0, st>>>(n, qs);
        SGT_LAUNCH_CHECK();
    }
    // Relaunch until converged; a bound on the launches for safety (each
    // launch runs at least one sweep or one deflation while status is 0).
    // Launch m's rotations are applied on a second stream while launch m + 1
    // runs: the two touch disjoint entries (launch m + 1 stays in the
    // columns up to its window's last row i, which is where launch m ended;
    // the applies act on columns right of each logged sweep's window, which
    // ended at i or further down, and alone on Q), and launch m + 2 writes
    // launch m's log only after its apply.
    // Each launch's applies are issued after the next QR launch, so that the
    // cluster finds its SMs free (a QR CTA takes a whole SM's registers).
    ApplyStream ap;
    SGT_CUDA_TRY(ap.init());
    const int qr_cl = qr_cluster_size();
    auto apply = [&](int p) -> signtri_status {
        const size_t lo = p * nlog;
        SGT_CUDA_TRY(cudaStreamWaitEvent(ap.s, ap.swept[p], 0));
        {
            ProfScope ps(SIGNTRI_KC_SCHUR, ap.s);
            apply_rotations_kernel<<<(8 * n + kThreads - 1) / kThreads, kThreads, 0, ap.s>>>(
                n, Tc, ldt, Qc, ldq, nlogged + p, sweeplog + lo, rclog + lo, rslog + lo);
            SGT_LAUNCH_CHECK();
        }
        SGT_CUDA_TRY(cudaEventRecord(ap.applied[p], ap.s));
        return SIGNTRI_OK;
    };
    QrState h{};
    const long long max_launches = 4LL * n * kMaxSweepsPerEigenvalue + 16;
    for (long long it = 0;; it++) {
        if (it >= max_launches) return SIGNTRI_ERR_NO_CONVERGENCE;
        const int p = (int)(it & 1);
        const size_t lo = p * nlog;
        if (it >= 2) SGT_CUDA_TRY(cudaStreamWaitEvent(st, ap.applied[p], 0));
        {
            ProfScope ps(SIGNTRI_KC_SCHUR, st);
            SGT_CUDA_TRY(launch_qr(qr_cl, n, Tc, ldt, qs, kRotationBudget, sweeplog + lo, rclog + lo, rslog + lo,
                                   nlogged + p, st));
        }
        SGT_CUDA_TRY(cudaEventRecord(ap.swept[p], st));
        if (it >= 1) {
            const signtri_status ra = apply(1 - p);
            if (ra != SIGNTRI_OK) return ra;
        }
        SGT_CUDA_TRY(cudaMemcpyAsync(&h, qs, sizeof(QrState), cudaMemcpyDeviceToHost, st));
        SGT_CUDA_TRY(cudaStreamSynchronize(st));
        if (h.status == 2) return SIGNTRI_ERR_NO_CONVERGENCE;
        if (h.status == 1) {
            const signtri_status ra = apply(p);
            if (ra != SIGNTRI_OK) return ra;
            break;
        }
    }
    SGT_CUDA_TRY(cudaStreamSynchronize(ap.s));
    if (counts_out) {
        counts_out[0] = h.sweeps;
        counts_out[1] = h.rotations;
    }
    {
        ProfScope ps(SIGNTRI_KC_FILL, st);
        clear_lower_kernel<<<n, kThreads, 0, st>>>(n, Tc, ldt);
        SGT_LAUNCH_CHECK();
    }
    return SIGNTRI_OK;
}

size_t sign_general_workspace_bytes(int n)
{
    if (n <= 0) return 0;
    const size_t cnn = (size_t)n * n * sizeof(double2) + 256;
    return 3 * cnn + std::max(schur_workspace_bytes(n), complex_schur_workspace_bytes(n));
}

signtri_status sign_general_run(int n, const double *A, int lda, double *S, int lds, Arena &ws, int *d_err,
                                int *bad_index, long long counts_out[2], cudaStream_t st)
{
    if (n <= 0) return SIGNTRI_OK;
    const size_t cnn = (size_t)n * n * sizeof(double2);
    auto *Qc = static_cast<double *>(ws.take(cnn));
    auto *Tc = static_cast<double *>(ws.take(cnn));
    auto *Sc = static_cast<double *>(ws.take(cnn));
    if (!Qc || !Tc || !Sc) return SIGNTRI_ERR_NO_WORKSPACE;
    const size_t mark = ws.used;
    signtri_status rs = schur_run(n, A, lda, Qc, n, Tc, n, ws, bad_index, counts_out, st);
    if (rs != SIGNTRI_OK) return rs;
    ws.used = mark;
    rs = complex_schur_run(n, Qc, n, Tc, n, Sc, n, ws, d_err, bad_index, st);
    if (rs != SIGNTRI_OK) return rs;
    {
        ProfScope ps(SIGNTRI_KC_FILL, st);
        real_part_kernel<<<n, kThreads, 0, st>>>(n, reinterpret_cast<const double2 *>(Sc), S, lds);
        SGT_LAUNCH_CHECK();
    }
    return SIGNTRI_OK;
}

}  // namespace signtri

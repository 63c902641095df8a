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
//     update) and from the right to the rows of A and of Q0 (one thread per
//     row).  Three launches per column.
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
//     what the one before wrote), so one CTA runs the sweeps with a barrier
//     per rotation; a launch runs sweeps until a rotation budget is spent and
//     the host relaunches until the window is empty.  This stage is bound by
//     that chain (about one L2 round trip per rotation, ~1.25 n^2 rotations
//     for n eigenvalues), not by arithmetic: the decomposition is the
//     general-matrix front end, not a tuned hot path.
//
// Layout: A real column-major; Q, T complex interleaved (re, im) float64
// pairs, column-major, leading dimensions counted in complex elements.
#include <algorithm>
#include <cfloat>
#include <climits>

#include "internal.cuh"

namespace signtri {

namespace {

constexpr int kThreads = 256;
constexpr int kQrThreads = 1024;
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
// G [x; y] = [r; 0].
__device__ __forceinline__ void make_rotation(double2 x, double2 y, double &c, double2 &s)
{
    const double ay = hypot(y.x, y.y);
    if (ay == 0.0) {
        c = 1.0;
        s = make_double2(0.0, 0.0);
        return;
    }
    const double ax = hypot(x.x, x.y);
    if (ax == 0.0) {
        c = 0.0;
        s = make_double2(y.x / ay, -y.y / ay);
        return;
    }
    const double nrm = hypot(ax, ay);
    c = ax / nrm;
    const double2 u = make_double2(x.x / ax, x.y / ax);   // x / |x|
    const double2 t = cmul(u, cconj(y));
    s = make_double2(t.x / nrm, t.y / nrm);
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

// Row r of H (r < n) or of Q0 (r >= n): M[r, k+1:] -= tau (M[r, k+1:] v) v^T.
__global__ void house_right_kernel(int n, int k, double *__restrict__ H, double *__restrict__ Q0,
                                   const double *__restrict__ v, const double *__restrict__ tau)
{
    const double t = *tau;
    if (t == 0.0) return;
    const int g = blockIdx.x * blockDim.x + threadIdx.x;
    if (g >= 2 * n) return;
    double *M = g < n ? H : Q0;
    const int r = g < n ? g : g - n;
    const int m = n - k - 1;
    double *row = &SGT_A(M, n, r, k + 1);
    double y = 0.0;
    for (int j = 0; j < m; j++) y = fma(row[(size_t)j * n], v[j], y);
    y *= t;
    for (int j = 0; j < m; j++) row[(size_t)j * n] = fma(-y, v[j], row[(size_t)j * n]);
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
    int pad;
    long long sweeps;
    long long rotations;
};

__global__ void qr_state_init_kernel(int n, QrState *st)
{
    st->ihi = n - 1;
    st->its = 0;
    st->status = 0;
    st->pad = 0;
    st->sweeps = 0;
    st->rotations = 0;
}

// One CTA.  Thread 0 owns the 2 x 2 block at (k, k) and row k+2 of columns
// k, k+1, where the next rotation's inputs (h_{k+1,k}, h_{k+2,k}) are
// formed, so it computes that rotation too and hands it over in shared
// memory (two slots, alternating): one barrier per rotation, and no entry is
// written by one thread while another reads it.
__global__ void __launch_bounds__(kQrThreads)
schur_qr_kernel(int n, double2 *__restrict__ T, int ldt, double2 *__restrict__ Q, int ldq, QrState *__restrict__ st,
                long long budget)
{
    __shared__ int redi[kQrThreads / 32];
    __shared__ double rc[2];
    __shared__ double2 rs[2];
    const int tid = threadIdx.x;
    int i = st->ihi, its = st->its, status = st->status;
    long long sweeps = 0, rot = 0;
    const double eps = DBL_EPSILON;
    const double tiny = DBL_MIN * ((double)n / DBL_EPSILON);
    while (status == 0) {
        if (i <= 0) {
            status = 1;
            i = -1;
            break;
        }
        // l: the largest k in [1, i] whose h_{k,k-1} is negligible, else 0
        int lk = 0;
        for (int k = 1 + tid; k <= i; k += kQrThreads) {
            const double sub = cabs1(SGT_A(T, ldt, k, k - 1));
            const double ref = cabs1(SGT_A(T, ldt, k - 1, k - 1)) + cabs1(SGT_A(T, ldt, k, k));
            if (sub <= fmax(eps * ref, tiny)) lk = k;
        }
        for (int o = 16; o > 0; o >>= 1) lk = max(lk, __shfl_xor_sync(0xffffffffu, lk, o));
        __syncthreads();   // the previous pass's reads of redi are done
        if ((tid & 31) == 0) redi[tid / 32] = lk;
        __syncthreads();
        int l = 0;
        for (int w = 0; w < kQrThreads / 32; w++) l = max(l, redi[w]);
        if (l == i) {   // the window's last row has converged
            if (tid == 0) SGT_A(T, ldt, i, i - 1) = make_double2(0.0, 0.0);
            i--;
            its = 0;
            continue;
        }
        if (rot >= budget) break;
        if (its >= kMaxSweepsPerEigenvalue) {
            status = 2;
            break;
        }
        its++;
        sweeps++;
        if (tid == 0) {
            if (l > 0) SGT_A(T, ldt, l, l - 1) = make_double2(0.0, 0.0);
            double2 sigma;
            if (its % 10 == 0) {
                // ad hoc shift: off the window's top (sweeps 10, 30, ..) or
                // bottom corner (20, 40, ..) by 3/4 of a subdiagonal entry's
                // real part
                const bool top = (its / 10) % 2 == 1;
                const double2 d = top ? SGT_A(T, ldt, l, l) : SGT_A(T, ldt, i, i);
                const double e = top ? SGT_A(T, ldt, l + 1, l).x : SGT_A(T, ldt, i, i - 1).x;
                sigma = make_double2(d.x + 0.75 * fabs(e), d.y);
            } else {
                // Wilkinson: with x = (a - d) / 2 and y = sqrt(x^2 + bc) signed
                // so that |x + y| is the larger, the eigenvalue of
                // [a b; c d] nearer d is d - bc / (x + y)
                const double2 a = SGT_A(T, ldt, i - 1, i - 1), b = SGT_A(T, ldt, i - 1, i);
                const double2 cc = SGT_A(T, ldt, i, i - 1), d = SGT_A(T, ldt, i, i);
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
            }
            double2 x = SGT_A(T, ldt, l, l);
            x.x -= sigma.x;
            x.y -= sigma.y;
            double c;
            double2 s;
            make_rotation(x, SGT_A(T, ldt, l + 1, l), c, s);
            rc[l & 1] = c;
            rs[l & 1] = s;
        }
        __syncthreads();
        for (int k = l; k < i; k++) {
            const double c = rc[k & 1];
            const double2 s = rs[k & 1];
            // rows k, k+1 from column jlo on, apart from the 2 x 2 block
            const int jlo = (k == l) ? l : k - 1;
            for (int j = jlo + tid; j < n; j += kQrThreads) {
                if (j == k || j == k + 1) continue;
                double2 a = SGT_A(T, ldt, k, j), b = SGT_A(T, ldt, k + 1, j);
                rot_rows(c, s, a, b);
                SGT_A(T, ldt, k, j) = a;
                SGT_A(T, ldt, k + 1, j) = (j == k - 1) ? make_double2(0.0, 0.0) : b;   // the old bulge, zeroed
            }
            // columns k, k+1 in the rows above the block
            for (int r = tid; r < k; r += kQrThreads) {
                double2 a = SGT_A(T, ldt, r, k), b = SGT_A(T, ldt, r, k + 1);
                rot_cols(c, s, a, b);
                SGT_A(T, ldt, r, k) = a;
                SGT_A(T, ldt, r, k + 1) = b;
            }
            if (tid == 0) {
                double2 a = SGT_A(T, ldt, k, k), b = SGT_A(T, ldt, k, k + 1);
                double2 e = SGT_A(T, ldt, k + 1, k), f = SGT_A(T, ldt, k + 1, k + 1);
                rot_rows(c, s, a, e);
                rot_rows(c, s, b, f);
                rot_cols(c, s, a, b);
                rot_cols(c, s, e, f);
                SGT_A(T, ldt, k, k) = a;
                SGT_A(T, ldt, k, k + 1) = b;
                SGT_A(T, ldt, k + 1, k) = e;
                SGT_A(T, ldt, k + 1, k + 1) = f;
                if (k + 2 <= i) {
                    // row k+2: h_{k+2,k} = 0 before, the new bulge after
                    double2 g = SGT_A(T, ldt, k + 2, k), h = SGT_A(T, ldt, k + 2, k + 1);
                    rot_cols(c, s, g, h);
                    SGT_A(T, ldt, k + 2, k) = g;
                    SGT_A(T, ldt, k + 2, k + 1) = h;
                    // the next rotation zeroes the bulge
                    double cn;
                    double2 sn;
                    make_rotation(e, g, cn, sn);
                    rc[(k + 1) & 1] = cn;
                    rs[(k + 1) & 1] = sn;
                }
            }
            for (int r = tid; r < n; r += kQrThreads) {
                double2 a = SGT_A(Q, ldq, r, k), b = SGT_A(Q, ldq, r, k + 1);
                rot_cols(c, s, a, b);
                SGT_A(Q, ldq, r, k) = a;
                SGT_A(Q, ldq, r, k + 1) = b;
            }
            __syncthreads();
        }
        rot += i - l;
    }
    if (tid == 0) {
        st->ihi = i;
        st->its = its;
        st->status = status;
        st->sweeps += sweeps;
        st->rotations += rot;
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

size_t schur_workspace_bytes(int n)
{
    if (n <= 0) return 0;
    // six takes, each rounded up to 256 bytes
    const size_t nn = (size_t)n * n;
    return 2 * nn * sizeof(double) + (size_t)n * sizeof(double) + sizeof(double) + sizeof(int) + sizeof(QrState) +
           6 * 256;
}

signtri_status schur_run(int n, const double *A, int lda, double *Q, int ldq, double *T, int ldt, Arena &ws,
                         int *bad_index, long long *sweeps_out, cudaStream_t st)
{
    if (n <= 0) return SIGNTRI_OK;
    const size_t nn = (size_t)n * n;
    auto *H = static_cast<double *>(ws.take(nn * sizeof(double)));
    auto *Q0 = static_cast<double *>(ws.take(nn * sizeof(double)));
    auto *v = static_cast<double *>(ws.take((size_t)n * sizeof(double)));
    auto *tau = static_cast<double *>(ws.take(sizeof(double)));
    auto *bad = static_cast<int *>(ws.take(sizeof(int)));
    auto *qs = static_cast<QrState *>(ws.take(sizeof(QrState)));
    if (!H || !Q0 || !v || !tau || !bad || !qs) return SIGNTRI_ERR_NO_WORKSPACE;
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
        ProfScope ps(SIGNTRI_KC_SCHUR, st, true, false);
        prof_count(SIGNTRI_KC_SCHUR, 3);
        house_kernel<<<1, 1024, 0, st>>>(n, k, H, v, tau);
        SGT_LAUNCH_CHECK();
        house_left_kernel<<<n - k - 1, kThreads, 0, st>>>(n, k, H, v, tau);
        SGT_LAUNCH_CHECK();
        house_right_kernel<<<(2 * n + kThreads - 1) / kThreads, kThreads, 0, st>>>(n, k, H, Q0, v, tau);
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
    // relaunch until converged; a bound on the launches for safety (each
    // launch runs at least one sweep or one deflation while status is 0)
    QrState h{};
    const long long max_launches = 4LL * n * kMaxSweepsPerEigenvalue + 16;
    for (long long it = 0;; it++) {
        if (it >= max_launches) return SIGNTRI_ERR_NO_CONVERGENCE;
        {
            ProfScope ps(SIGNTRI_KC_SCHUR, st);
            schur_qr_kernel<<<1, kQrThreads, 0, st>>>(n, Tc, ldt, Qc, ldq, qs, kRotationBudget);
            SGT_LAUNCH_CHECK();
        }
        SGT_CUDA_TRY(cudaMemcpyAsync(&h, qs, sizeof(QrState), cudaMemcpyDeviceToHost, st));
        SGT_CUDA_TRY(cudaStreamSynchronize(st));
        if (h.status == 1) break;
        if (h.status == 2) return SIGNTRI_ERR_NO_CONVERGENCE;
    }
    if (sweeps_out) *sweeps_out = h.sweeps;
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
                                int *bad_index, long long *sweeps_out, cudaStream_t st)
{
    if (n <= 0) return SIGNTRI_OK;
    const size_t cnn = (size_t)n * n * sizeof(double2);
    auto *Qc = static_cast<double *>(ws.take(cnn));
    auto *Tc = static_cast<double *>(ws.take(cnn));
    auto *Sc = static_cast<double *>(ws.take(cnn));
    if (!Qc || !Tc || !Sc) return SIGNTRI_ERR_NO_WORKSPACE;
    const size_t mark = ws.used;
    signtri_status rs = schur_run(n, A, lda, Qc, n, Tc, n, ws, bad_index, sweeps_out, st);
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

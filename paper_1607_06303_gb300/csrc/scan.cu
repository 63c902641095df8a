// scan.cu -- inertia scan of diag(T) and the trivial-inertia outputs.
//
// Section 3: the cost of Parlett-Sylvester depends on the number k of
// adjacent swaps that group the eigenvalues by sign (0 <= k <= n^2/4) and on
// the inertia (n_-, n_+); sign(T) is I or -I when one of n_-, n_+ is zero.
// Section 1: sign(0) is undefined, so a zero diagonal entry is an error.
#include <climits>

#include "internal.cuh"

namespace signtri {

namespace {

constexpr int kScanThreads = 1024;

// One CTA.  Thread t owns the contiguous index range [lo, hi) of the
// diagonal.  Exclusive scans over threads of the per-sign counts and index
// sums give, at every entry i, the number c and the index sum S of the
// entries of each sign before i.  Then
//   swaps   += c_neg                      for each positive entry i,
//   same    += c_s * (i - 1) - S_s        for each entry i of sign s,
// where `same` = sum over equal-sign pairs i<j of (j - i - 1): the number of
// inner-sum terms of Algorithm 3 that use U^2 = I.
__device__ __forceinline__ void inertia_scan_body(int n, const double *__restrict__ T, int ldt, ScanResult *out)
{
    __shared__ long long s_a[kScanThreads], s_b[kScanThreads], s_c[kScanThreads], s_d[kScanThreads];
    __shared__ int s_bad[kScanThreads], s_fneg[kScanThreads];
    const int tid = threadIdx.x;
    const int per = (n + kScanThreads - 1) / kScanThreads;
    const int lo = min(n, tid * per), hi = min(n, lo + per);
    long long cneg = 0, cpos = 0, sneg = 0, spos = 0;
    int bad = INT_MAX, fneg = INT_MAX;
    for (int i = lo; i < hi; i++) {
        const double t = SGT_AT(T, ldt, i, i);
        if (!isfinite(t)) { if (bad == INT_MAX) bad = 4 * i + SIGNTRI_ERR_NONFINITE; }
        else if (t == 0.0) { if (bad == INT_MAX) bad = 4 * i + SIGNTRI_ERR_ZERO_EIGENVALUE; }
        else if (t < 0.0) { cneg++; sneg += i; fneg = min(fneg, i); }
        else { cpos++; spos += i; }
    }
    s_a[tid] = cneg; s_b[tid] = cpos; s_c[tid] = sneg; s_d[tid] = spos;
    __syncthreads();
    for (int off = 1; off < kScanThreads; off <<= 1) {   // inclusive scans
        long long a = 0, b = 0, c = 0, d = 0;
        if (tid >= off) { a = s_a[tid - off]; b = s_b[tid - off]; c = s_c[tid - off]; d = s_d[tid - off]; }
        __syncthreads();
        s_a[tid] += a; s_b[tid] += b; s_c[tid] += c; s_d[tid] += d;
        __syncthreads();
    }
    long long cn = s_a[tid] - cneg, cp = s_b[tid] - cpos, sn = s_c[tid] - sneg, sp = s_d[tid] - spos;
    const long long tot_neg = s_a[kScanThreads - 1], tot_pos = s_b[kScanThreads - 1];
    long long swaps = 0, same = 0;
    for (int i = lo; i < hi; i++) {
        const double t = SGT_AT(T, ldt, i, i);
        if (t < 0.0) { same += cn * (long long)(i - 1) - sn; cn++; sn += i; }
        else if (t > 0.0) { swaps += cn; same += cp * (long long)(i - 1) - sp; cp++; sp += i; }
    }
    __syncthreads();
    s_a[tid] = swaps; s_b[tid] = same; s_bad[tid] = bad; s_fneg[tid] = fneg;
    __syncthreads();
    for (int off = kScanThreads / 2; off > 0; off >>= 1) {
        if (tid < off) {
            s_a[tid] += s_a[tid + off];
            s_b[tid] += s_b[tid + off];
            s_bad[tid] = min(s_bad[tid], s_bad[tid + off]);
            s_fneg[tid] = min(s_fneg[tid], s_fneg[tid + off]);
        }
        __syncthreads();
    }
    if (tid == 0) {
        out->n_pos = (int)tot_pos;
        out->n_neg = (int)tot_neg;
        out->swaps = s_a[0];
        out->same_terms = s_b[0];
        out->bad_key = s_bad[0];
        out->first_neg = s_fneg[0] == INT_MAX ? n : s_fneg[0];
    }
}

__global__ void __launch_bounds__(kScanThreads)
inertia_scan_kernel(int n, const double *__restrict__ T, int ldt, ScanResult *out)
{
    inertia_scan_body(n, T, ldt, out);
}

// One CTA per matrix of a batch.
__global__ void __launch_bounds__(kScanThreads)
inertia_scan_batched_kernel(const BatchDesc *__restrict__ mats, ScanResult *out)
{
    const BatchDesc m = mats[blockIdx.x];
    inertia_scan_body(m.n, m.T, m.ldt, out + blockIdx.x);
}

// Batched fills: U_m = diag_m * I (diag_m = 0: only the strictly lower part
// set to 0).  blockIdx.x = matrix, blockIdx.y strides the columns.
__global__ void fill_batched_kernel(const BatchDesc *__restrict__ mats, const int *__restrict__ which,
                                    const double *__restrict__ diag)
{
    const int k = blockIdx.x;
    const BatchDesc m = mats[which[k]];
    const double dv = diag[k];
    for (int j = blockIdx.y; j < m.n; j += gridDim.y)
        for (int i = threadIdx.x; i < m.n; i += blockDim.x) {
            if (dv != 0.0) SGT_AT(m.U, m.ldu, i, j) = (i == j) ? dv : 0.0;
            else if (i > j) SGT_AT(m.U, m.ldu, i, j) = 0.0;
        }
}

// U = diag * I on the n x n part (used when n_- = 0 or n_+ = 0).
__global__ void fill_identity_kernel(int n, double *__restrict__ U, int ldu, double diag)
{
    const int j = blockIdx.x;
    for (int i = threadIdx.x; i < n; i += blockDim.x) SGT_AT(U, ldu, i, j) = (i == j) ? diag : 0.0;
}

__global__ void zero_strict_lower_kernel(int n, double *__restrict__ U, int ldu)
{
    const int j = blockIdx.x;
    for (int i = j + 1 + threadIdx.x; i < n; i += blockDim.x) SGT_AT(U, ldu, i, j) = 0.0;
}

}  // namespace

signtri_status launch_inertia_scan(int n, const double *T, int ldt, ScanResult *d_out,
                                   cudaStream_t st)
{
    ProfScope ps(SIGNTRI_KC_SCAN, st);
    inertia_scan_kernel<<<1, kScanThreads, 0, st>>>(n, T, ldt, d_out);
    SGT_LAUNCH_CHECK();
    return SIGNTRI_OK;
}

signtri_status launch_inertia_scan_batched(int count, const BatchDesc *d_mats, ScanResult *d_out, cudaStream_t st)
{
    if (count <= 0) return SIGNTRI_OK;
    ProfScope ps(SIGNTRI_KC_SCAN, st);
    inertia_scan_batched_kernel<<<count, kScanThreads, 0, st>>>(d_mats, d_out);
    SGT_LAUNCH_CHECK();
    return SIGNTRI_OK;
}

signtri_status launch_fill_batched(int count, const BatchDesc *d_mats, const int *d_which, const double *d_diag,
                                   cudaStream_t st)
{
    if (count <= 0) return SIGNTRI_OK;
    ProfScope ps(SIGNTRI_KC_FILL, st);
    fill_batched_kernel<<<dim3(count, 64), 256, 0, st>>>(d_mats, d_which, d_diag);
    SGT_LAUNCH_CHECK();
    return SIGNTRI_OK;
}

signtri_status launch_fill_identity(int n, double *U, int ldu, double diag, cudaStream_t st)
{
    if (n <= 0) return SIGNTRI_OK;
    ProfScope ps(SIGNTRI_KC_FILL, st);
    fill_identity_kernel<<<n, 256, 0, st>>>(n, U, ldu, diag);
    SGT_LAUNCH_CHECK();
    return SIGNTRI_OK;
}

signtri_status launch_zero_strict_lower(int n, double *U, int ldu, cudaStream_t st)
{
    if (n <= 1) return SIGNTRI_OK;
    ProfScope ps(SIGNTRI_KC_FILL, st);
    zero_strict_lower_kernel<<<n, 256, 0, st>>>(n, U, ldu);
    SGT_LAUNCH_CHECK();
    return SIGNTRI_OK;
}

}  // namespace signtri

// internal.cuh -- declarations shared by the translation units of libsigntri.
#pragma once

#include <cuda_runtime.h>
#include <stddef.h>
#include <stdint.h>
#include <climits>

#include "../../include/signtri.h"

namespace signtri {

// Column-major element access, 0-based.
#define SGT_AT(M, ld, i, j) ((M)[(size_t)(i) + (size_t)(j) * (size_t)(ld)])

#define SGT_CUDA_TRY(expr)                                   \
    do {                                                     \
        cudaError_t _e = (expr);                             \
        if (_e != cudaSuccess) return SIGNTRI_ERR_CUDA;      \
    } while (0)

#define SGT_LAUNCH_CHECK() SGT_CUDA_TRY(cudaGetLastError())

// True when the column-major blocks A (rowsA x colsA, leading dimension lda)
// and B (rowsB x colsB, ldb) share an element; rowsA <= lda.  Exact for
// blocks interleaved within one array: each column of B is a contiguous run
// compared with the runs of A that its span reaches.  Pointers whose distance
// is not a whole number of doubles count as overlapping once their byte
// extents meet.  Host only, O(colsB) when the extents meet, O(1) otherwise.
inline bool blocks_overlap(const double *A, int lda, int rowsA, int colsA, const double *B, int ldb, int rowsB,
                           int colsB)
{
    if (rowsA <= 0 || colsA <= 0 || rowsB <= 0 || colsB <= 0) return false;
    const long long pa = (long long)(uintptr_t)A, pb = (long long)(uintptr_t)B;
    const long long lenA = ((long long)(colsA - 1) * lda + rowsA) * 8;
    const long long lenB = ((long long)(colsB - 1) * ldb + rowsB) * 8;
    if (pb >= pa + lenA || pa >= pb + lenB) return false;
    if ((pb - pa) % 8 != 0) return true;
    const long long d = (pb - pa) / 8;               // B's first element, in doubles from A's
    for (int cb = 0; cb < colsB; cb++) {
        const long long s = d + (long long)cb * ldb;  // column cb of B: elements [s, e] from A's start
        const long long e = s + rowsB - 1;
        if (e < 0) continue;
        const long long lo = s < 0 ? 0 : s / lda;     // first column of A that can reach [s, e]
        long long hi = e / lda;                       // last column of A starting at or before e
        if (hi > colsA - 1) hi = colsA - 1;
        if (lo > hi) continue;
        if (hi > lo) return true;                     // column lo+1 of A starts inside [s, e]
        const long long a0 = lo * lda;                // column lo of A: [a0, a0 + rowsA - 1]
        if (a0 <= e && a0 + rowsA - 1 >= s) return true;
    }
    return false;
}

// Result of the inertia scan (written by the device, read by the host).
struct ScanResult {
    int n_pos;
    int n_neg;
    long long swaps;       // #{i<j : t_ii < 0 < t_jj}
    long long same_terms;  // sum over equal-sign pairs i<j of (j-i-1)
    int bad_key;       // min over bad i of (4*i + kind), INT_MAX when none
    int first_neg;     // index of the first negative diagonal entry, n when none
};

// One matrix of a batch (device copy).
struct BatchDesc {
    const double *T;
    double *U;
    int n, ldt, ldu, pad;
};

// Device workspace carved into aligned slices.
struct Arena {
    char *base = nullptr;
    size_t bytes = 0;
    size_t used = 0;
    void *take(size_t n) {
        size_t off = (used + 255) & ~(size_t)255;
        if (off + n > bytes) return nullptr;
        used = off + n;
        return base + off;
    }
};

// Launch accounting (prof.cu): bracket every library launch.
void prof_begin(int cls, cudaStream_t st, bool count = true);
void prof_end(int cls, cudaStream_t st);
// Algorithmic tensor-core flops of a launch (counted on the host).
void prof_add_flops(int cls, double flops);
void prof_add_bytes(int cls, double bytes);
// While paused (stream capture), launches are counted but not timed.
void prof_pause(bool on);
void prof_count(int cls, long long launches);

// Brackets a launch (or, with count = false, a group of launches that count
// themselves) with events on `s`; timed = false only counts the launch.
struct ProfScope {
    int cls;
    cudaStream_t st;
    bool timed;
    ProfScope(int c, cudaStream_t s, bool t = true, bool count = true) : cls(c), st(s), timed(t)
    {
        if (timed) prof_begin(c, s, count);
        else if (count) prof_count(c, 1);
    }
    ~ProfScope() { if (timed) prof_end(cls, st); }
};
// Kernel-class flag for launches inside an already timed group: counted, not timed.
constexpr int kProfUntimed = 0x1000;

// Scan / init kernels (scan.cu)
signtri_status launch_inertia_scan(int n, const double *T, int ldt, ScanResult *d_out,
                                   cudaStream_t st);
signtri_status launch_fill_identity(int n, double *U, int ldu, double diag, cudaStream_t st);
signtri_status launch_inertia_scan_batched(int count, const BatchDesc *d_mats, ScanResult *d_out, cudaStream_t st);
// U_m = diag * I for the listed matrices (diag 0: zero the strictly lower part)
signtri_status launch_fill_batched(int count, const BatchDesc *d_mats, const int *d_which, const double *d_diag,
                                   cudaStream_t st);
signtri_status launch_zero_strict_lower(int n, double *U, int ldu, cudaStream_t st);

// Leaf size the float64 matrix-multiply form runs with at order n (api.cu).
int current_cutoff(int n);

// Recursive Parlett-Higham, float64 (ph_fp64.cu)
size_t ph_fp64_workspace_bytes(int n, int b);
signtri_status diag_leaves_f64(int n, const double *T, int ldt, double *U, int ldu, int b, cudaStream_t st);
signtri_status ph_fp64_run(int n, const double *T, int ldt, double *U, int ldu, int b,
                           Arena &ws, cudaStream_t st);
// arithmetic-efficient form (one sum per entry)
size_t ph_fp64_split_workspace_bytes(int n, int b);
signtri_status ph_fp64_split_run(int n, const double *T, int ldt, double *U, int ldu, int b, Arena &ws,
                                 cudaStream_t st);

// Float64 GEMM (gemm_f64.cu): C = alpha op(A) op(B) + beta C, optional upper
// triangle only.
signtri_status gemm_f64(bool transA, bool transB, int m, int n, int k, double alpha, const double *A, int lda,
                        const double *B, int ldb, double beta, double *C, int ldc, bool upper, cudaStream_t st);

// Parlett-Sylvester pieces (ps_fp64.cu)
size_t sylvester_workspace_bytes(int m, int p);
signtri_status sylvester_run(int m, int p, const double *A, int lda, const double *Bm, int ldb, const double *C,
                             int ldc, double cscale, double *X, int ldx, Arena &ws, cudaStream_t st);
signtri_status copy_upper_identity(int n, const double *T, int ldt, double *Tr, int ldtr, double *Q, int ldq,
                                   cudaStream_t st);
// the odd-even rounds, float64 rotations applied one by one
size_t reorder_workspace_bytes(int n);
signtri_status reorder_run(int n, const double *T, int ldt, double *Tr, int ldtr, double *Q, int ldq,
                           long long *swaps_out, Arena &ws, cudaStream_t st);
// the windowed form, each window's rotations applied by emulated-float64
// tensor-core products (reorder_tc.cu); from this order on
constexpr int kBlockedReorderMin = 512;
size_t reorder_blocked_workspace_bytes(int n);
signtri_status reorder_blocked_run(int n, const double *T, int ldt, double *Tr, int ldtr, double *Q, int ldq,
                                   long long *swaps_out, Arena &ws, int *d_err, cudaStream_t st);
// whichever of the two the order selects
size_t reorder_any_workspace_bytes(int n, long long swaps);
signtri_status reorder_any_run(int n, const double *T, int ldt, double *Tr, int ldtr, double *Q, int ldq,
                               long long *swaps_out, Arena &ws, int *d_err, cudaStream_t st);
size_t ps_workspace_bytes(int n, long long swaps);
signtri_status ps_fp64_run(int n, const double *T, int ldt, double *U, int ldu, int npos, long long swaps,
                           Arena &ws, int *d_err, cudaStream_t st);

// bf16 slices and the emulated-float64 GEMM (slices.cu)
int pad64(int x);
signtri_status make_scales(int m, int k, const double *M, int ldm, int tri, bool rows, int nout,
                           unsigned long long *tmp, float *scale, cudaStream_t st);
size_t emulated_gemm_workspace_bytes(int m, int n, int k, int S);
signtri_status emulated_gemm_run(int m, int n, int k, const double *A, int lda, const double *B, int ldb, double *C,
                                 int ldc, int S, Arena &ws, int *d_err, cudaStream_t st);
// C = A op(B) (op(B) = B or B^T) written straight into C; upper: only the
// 128 x 128 tiles that meet the upper triangle
size_t emulated_product_workspace_bytes(int m, int n, int k);
signtri_status emulated_product(int m, int n, int k, const double *A, int lda, const double *B, int ldb, bool transB,
                                double *C, int ldc, bool upper, int kernel_class, Arena &ws, int *d_err,
                                cudaStream_t st);

// Batched float64 Parlett-Higham (batched.cu)
size_t batched_workspace_bytes(int count, const int *n, int cutoff_for_all);
signtri_status batched_ph_run(int count, const BatchDesc *h_mats, const BatchDesc *d_mats, const int *bs,
                              bool split, Arena &ws, cudaStream_t st);
// Graph-cache counters of the batched path: launches of a cached graph, and
// graphs built (tables, capture, instantiation), over all devices.
void batched_cache_stats(long long *hits, long long *builds);

// Bounded-wait self-test (tc_gemm.cu)
signtri_status wait_selftest(int arrive, long long limit, int *d_err, cudaStream_t st);

// General phi (funm.cu): Algorithms 1 and 2 on the float64 partition
size_t funm_workspace_bytes(int n, int b);
signtri_status funm_run(int n, const double *T, int ldt, double *F, int ldf, int phi, int b, Arena &ws,
                        int *bad_index, cudaStream_t st);

// Complex T (complex.cu): interleaved (re, im) column-major, ld in complex
// elements.  bad_index receives the first bad diagonal index on a status
// other than OK that concerns the diagonal.
size_t complex_workspace_bytes(int n);
signtri_status complex_sign_run(int n, const double *T, int ldt, double *U, int ldu, Arena &ws, int *bad_index,
                                cudaStream_t st);
size_t complex_schur_workspace_bytes(int n);
signtri_status complex_schur_run(int n, const double *Q, int ldq, const double *T, int ldt, double *S, int lds,
                                 Arena &ws, int *d_err, int *bad_index, cudaStream_t st);

// Complex Schur decomposition of a real A and sign(A) through it (schur.cu).
// Q, T complex as above; bad_index: the first column of A holding a
// non-finite entry (NONFINITE), or as complex_sign_run; counts_out (may be
// null): the QR sweeps run and the plane rotations they applied.
size_t schur_workspace_bytes(int n);
signtri_status schur_run(int n, const double *A, int lda, double *Q, int ldq, double *T, int ldt, Arena &ws,
                         int *bad_index, long long counts_out[2], cudaStream_t st);
size_t sign_general_workspace_bytes(int n);
signtri_status sign_general_run(int n, const double *A, int lda, double *S, int lds, Arena &ws, int *d_err,
                                int *bad_index, long long counts_out[2], cudaStream_t st);

// Mixed precision with refinement (mixed.cu)
struct MixedParams {
    double tol;              // stopping test on both relative residuals
    int max_steps;           // refinement steps before falling back
    double min_contraction;  // required reduction of the residual per step
    int verify_full;         // 1: accept on the full residuals, 0: on the probe estimate
};
struct MixedReport {
    int steps;
    int fallback;            // 1: the caller must run the float64 path
    double resid_commute, resid_involution, resid0;
};
size_t mixed_workspace_bytes(int n, int S);
signtri_status mixed_run(int n, const double *T, int ldt, double *U, int ldu, int S, const MixedParams &prm,
                         MixedReport &rep, Arena &ws, int *d_err, double *norms_host, cudaStream_t st);

}  // namespace signtri

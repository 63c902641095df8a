/*
 * signtri.h -- C ABI of libsigntri.so: U = sign(T) for a dense real upper
 * triangular matrix T on one GB300 (sm_103a).
 *
 * The operation (Stotland, Schwartz, Toledo, "High-Performance Algorithms
 * for Computing the Sign Function of Triangular Matrices", Section 1 and
 * Section 2): for T upper triangular with no zero diagonal entry, U = sign(T)
 * is the upper triangular matrix with u_ii = sign(t_ii), UT = TU and U^2 = I.
 *
 * Conventions shared by every entry point
 *   - Matrices are float64, column-major: element (i,j) (0-based) of a matrix
 *     M with leading dimension ld is M[i + j*ld].  ld >= max(1, n).
 *   - Pointers named T, U are DEVICE pointers unless the name says _host.
 *     They are owned by the caller.  T and U must not share an element:
 *     the device-pointer entry points compare the two blocks (exactly, so
 *     disjoint blocks interleaved in one array through their leading
 *     dimensions are fine) and return SIGNTRI_ERR_BAD_ARG before any work.
 *   - Only the upper triangle of T (i <= j) is read.  All of the n x n part of
 *     U is written; its strictly lower triangle is set to 0.
 *   - `stream` is a cudaStream_t passed as void* (NULL = legacy default
 *     stream).  Work is enqueued on it; see each call for the points where
 *     the host waits.
 *   - Errors are returned as signtri_status; nothing is thrown.  On any error
 *     other than SIGNTRI_ERR_CUDA the contents of U are unspecified but no
 *     memory outside U and the library workspace is written.
 *   - The library keeps one workspace per device (grown on demand with
 *     cudaMalloc, or set by signtri_set_workspace).  Calls that share a
 *     workspace must not run concurrently: issue them from one host thread,
 *     or on one stream, at a time.
 */
#ifndef SIGNTRI_H
#define SIGNTRI_H

#include <stddef.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    /* Choose Parlett-Higham (its arithmetic-efficient form,
       SIGNTRI_PH_FP64_EFFICIENT) or Parlett-Sylvester per input from the
       work estimates of Section 3 (inertia, swap count, and the index of
       the first negative, which bounds the reorder's sweeps) turned into
       times with rates and latencies measured on GB300.  In
       sign_tri_batched, AUTO follows the variant table (signtri_autotune):
       by default Parlett-Sylvester when no swaps are needed and the batched
       Parlett-Higham (efficient form) otherwise. */
    SIGNTRI_AUTO = 0,
    /* Recursive Parlett-Higham (Algorithms 3-6), float64 throughout; block
       sums in matrix-multiply form (both X and Y for every entry). */
    SIGNTRI_PH_FP64 = 1,
    /* Parlett-Sylvester for the sign function (Section 2, Section 3,
       Section 5.1): reorder by sign with adjacent Givens swaps, solve
       T11 X - X T22 = 2 T12, transform back.  From n = 512 on the swaps run
       by windows of 128 (each window's rotations accumulated into one
       orthogonal factor and applied to the rest of T and Q as
       emulated-float64 tensor-core products); the back-transform's two
       products are emulated-float64 too (7 exact slices of 7 bits per row
       or column, about 2^-45 of the product of the scales).  Float64
       accuracy in the normwise sense; the diagonal of U is exact. */
    SIGNTRI_PS_FP64 = 2,
    /* Parlett-Higham with tensor-core block updates of about fp32 accuracy,
       then float64 refinement of both defining equations.  tcgen05 has no
       fp32 product and tf32 keeps 10 mantissa bits, so each operand is split
       into three bf16 terms (hi + mid + lo) and the six products with
       s + t <= 2 are summed (about 2^-24 relative); the name is the
       interface's.  Some of its tensor-core
       launches run on side streams the library creates once per device;
       they are forked from and joined back into the caller's stream with
       events, so all of the call's work is ordered on `stream` as usual.
       The host waits on `stream` a few times during the call (diagonal
       signs, residual norms). */
    SIGNTRI_PH_MIXED_TF32 = 3,
    /* Parlett-Higham with BF16 tensor-core block updates, then float64
       refinement of both defining equations (side streams and host waits as
       above). */
    SIGNTRI_PH_MIXED_BF16 = 4,
    /* Arithmetic-efficient recursive Parlett-Higham (Section 5.3), float64:
       each entry's block sum is X (signs differ) or Y (signs agree) only,
       n^3/3..2n^3/3 flops instead of n^3.  Every sum runs over the same
       terms in the same order as in SIGNTRI_PH_FP64, so the two results
       agree bit for bit (up to the sign of zero).  Workspace: see
       signtri_workspace_bytes. */
    SIGNTRI_PH_FP64_EFFICIENT = 5,
    /* As SIGNTRI_PH_MIXED_TF32, with each block-update operand split into
       two fp16 terms (hi + lo, 22 significant bits) and the three products
       with s + t <= 1 summed: half the tensor-core products and two thirds of
       the operand bytes of the three-term bf16 split, about 2^-21 relative
       instead of 2^-24.  fp16 spans 2^-24 .. 65504, so T, U and each
       correction are scaled by powers of two (from the largest strictly
       upper entry of T, of the diagonal blocks of U, and of the correction's
       first-order terms Rc_ij / (t_ii - t_jj) and Rs_ij / 2); a problem
       whose values leave that range shows up as a residual that does not
       contract, and the call then falls back to SIGNTRI_PH_FP64 like the
       other mixed variants. */
    SIGNTRI_PH_MIXED_FP16 = 6
} signtri_variant;

typedef enum {
    SIGNTRI_OK = 0,
    SIGNTRI_ERR_BAD_ARG = 1,          /* n < 0, ld too small, NULL pointer, bad variant,
                                         output sharing an element with an input */
    SIGNTRI_ERR_ZERO_EIGENVALUE = 2,  /* some t_ii == 0: sign(0) is undefined (Section 1) */
    SIGNTRI_ERR_NONFINITE = 3,        /* some t_ii is NaN or infinite */
    SIGNTRI_ERR_NO_CONVERGENCE = 4,   /* signtri_schur's QR iteration did not converge
                                         (a mixed variant whose refinement stalls falls
                                         back to SIGNTRI_PH_FP64 instead) */
    SIGNTRI_ERR_TIMEOUT = 5,          /* a bounded device-side wait gave up */
    SIGNTRI_ERR_CUDA = 6,             /* a CUDA runtime call or launch failed */
    SIGNTRI_ERR_NO_WORKSPACE = 7,     /* workspace could not be allocated / too small */
    SIGNTRI_ERR_UNSUPPORTED = 8,      /* option not available in this build */
    SIGNTRI_ERR_DOMAIN = 9            /* signtri_funm: a diagonal entry outside phi's domain,
                                         not finite, or repeated (Parlett's substitution
                                         divides by t_ii - t_jj) */
} signtri_status;

/* What the last sign_tri call on the calling host thread did. */
typedef struct {
    int variant;            /* signtri_variant actually run */
    int n;                  /* problem size */
    int n_pos, n_neg;       /* inertia of T: counts of t_ii > 0 and t_ii < 0 */
    long long swaps;        /* #{i<j : t_ii < 0 < t_jj}: adjacent swaps that
                               group positives first (Section 3) */
    double work_ph;         /* Section 3 flop estimate, Parlett-Higham */
    double work_ps;         /* Section 3 flop estimate, Parlett-Sylvester */
    int cutoff;             /* leaf (block) size used by Parlett-Higham */
    int refine_steps;       /* refinement steps taken (mixed variants) */
    double resid_commute;   /* ||TU-UT||_F / (||T||_F ||U||_F) after the last step
                               (mixed variants; see signtri_set_verification) */
    double resid_involution;/* ||U^2-I||_F / ||U||_F^2 after the last step */
    int bad_index;          /* first offending diagonal index on ZERO/NONFINITE, else -1 */
    long long qr_sweeps;    /* signtri_schur, signtri_sign_general: QR sweeps run (each
                               bulge's sweep counted; 0 for the other calls) */
    long long qr_rotations; /* plane rotations those sweeps applied */
} signtri_info;

/* Human-readable name of a status code (static string, never NULL). */
const char *signtri_status_string(signtri_status s);

/* Bytes of device workspace sign_tri needs for size n and variant v with the
   current cutoff (0 when none).  Returns 0 for invalid arguments. */
size_t signtri_workspace_bytes(int n, signtri_variant v);

/* Use caller-owned device memory [dev_ptr, dev_ptr+bytes) as the workspace of
   the current device from now on (dev_ptr 256-byte aligned).  dev_ptr == NULL
   returns to library-owned workspace.  The library never frees caller
   memory.  A call whose need exceeds `bytes` fails with
   SIGNTRI_ERR_NO_WORKSPACE. */
signtri_status signtri_set_workspace(void *dev_ptr, size_t bytes);

/* Per-variant throughput used by SIGNTRI_AUTO to turn the Section 3 work
   estimates into times: flops/s of the float64 block products (default
   1.2e12, GB300's measured float64 rate) and of the unblocked Givens
   rounds (default 0.35e12).  Values <= 0 restore the defaults. */
signtri_status signtri_set_rates(double gemm_flops_per_s, double givens_flops_per_s);

/* Refinement of the mixed variants: stop when ||TU-UT||_F/(||T||_F||U||_F)
   and ||U^2-I||_F/||U||_F^2 are both <= tol (default 1e-13; tol <= 0
   restores it), or fall back to SIGNTRI_PH_FP64 after max_steps correction
   steps or when a step does not reduce the larger residual tenfold
   (max_steps < 0: 3 for SIGNTRI_PH_MIXED_TF32, 8 for SIGNTRI_PH_MIXED_BF16).
   Process-wide setting. */
signtri_status signtri_set_refinement(double tol, int max_steps);

/* How the mixed variants accept a refinement step (process-wide).  Both
   residuals, TU-UT and U^2-I, over all entries must be <= tol:
   full = 1: formed entry by entry (three emulated-float64 n x n products);
   full = 0 (default): estimated from 128 random +-1 probe vectors Z,
     ||R||_F^2 ~ ||R Z||_F^2 / 128 (an unbiased estimate for any R; for a
     residual 10x above tol the estimate falls below tol with probability
     below 1e-9 by Maurer's bound for sums of nonnegative variables, with
     E||Rz||^4 <= 3 ||R||_F^4 for +-1 vectors), with R Z = T(UZ) - U(TZ) and
     U(UZ) - Z from emulated-float64 n x n by n x 128 products.  resid_commute / resid_involution then report
     the estimate.
   Corrections are driven by the needed residuals either way (Rc where the
   signs of t_ii, t_jj differ, Rs where they agree).  Other values of full
   return SIGNTRI_ERR_BAD_ARG. */
signtri_status signtri_set_verification(int full);

/* Leaf (recursion cutoff) size b of the float64 Parlett-Higham forms: the
   order of the diagonal and off-diagonal blocks solved element by element
   (Section 6 uses 16).  b in {16, 32, 64}, or 0 (the default): by size, the
   fastest measured on GB300 -- the efficient form 16 below n = 4096, 32
   below 8192, then 64; the matrix-multiply form 16 up to n = 4096, then 32.
   The mixed variants' tensor-core tiles are 64 whatever b.  signtri_info
   reports the b a call used.  Process-wide setting. */
signtri_status signtri_set_cutoff(int b);

/* U = sign(T).  T, U device pointers (see conventions).  Enqueued on
   `stream`; the host waits after the inertia scan to read three integers
   (n_pos, n_neg, swaps) and the error flags.  The float64 Parlett-Higham
   forms then enqueue their launches and return without waiting for them;
   Parlett-Sylvester also waits while it builds its swap schedule from the
   diagonal, and the mixed variants wait a few times (diagonal signs,
   residual norms) and return after U is written.
   n == 0 is a no-op returning SIGNTRI_OK.  n == 1 writes sign(t_11).
   If all t_ii > 0 (all < 0) U = I (U = -I) exactly (Section 3). */
signtri_status sign_tri(int n, const double *T, int ldt, double *U, int ldu,
                        signtri_variant v, void *stream);

/* Same as sign_tri, with T_host and U_host in host memory (pinned memory
   gives full copy bandwidth).  Copies T's upper triangle to the device (by
   column panels, about n^2/2 doubles), computes, copies all of U back, and
   returns after U_host is written (synchronous). */
signtri_status sign_tri_host(int n, const double *T_host, int ldt, double *U_host, int ldu,
                             signtri_variant v, void *stream);

/* Many independent problems in one call.  Host arrays of length count:
   n[m], ldt[m], ldu[m], and T[m], U[m] (DEVICE pointers, the same conventions
   as sign_tri).  info[m] (host) receives each problem's status; a bad matrix
   does not stop the others.  Per matrix: the inertia scan (one batched
   launch), +-I for trivial inertia, and for the rest the variant `v` (AUTO:
   Parlett-Sylvester when the diagonal is already grouped by sign, i.e. no
   swaps, else Parlett-Higham, which shares its launches across the batch).  All
   Parlett-Higham float64 problems run together as one CUDA graph of
   level-synchronous launches (leaf size per problem from the cutoff table;
   the graph is built once per group shape and relaunched by later calls, see
   signtri_batched_cache_stats); the others run one after another (under
   AUTO also the size buckets the variant table sends to a mixed variant).
   Returns after all U[m] are written.
   The return value reports failures of the call itself. */
signtri_status sign_tri_batched(int count, const int *n, const double *const *T, const int *ldt,
                                double *const *U, const int *ldu, signtri_variant v, int *info,
                                void *stream);

/* Leaf-size table of the batched path: b[k] (16, 32, 64, or 0 = the
   process-wide cutoff, by size when that is 0) for problems with
   floor(log2 n) == k, k < len <= 32. */
signtri_status signtri_set_cutoff_table(const int *b, int len);
signtri_status signtri_get_cutoff_table(int *b, int len);

/* Autotuner of the batched path (the paper's closing suggestion of
   choosing by auto-tuning): for each size bucket n = 32, 64, ..., up to
   n_max (<= 32768), time sign_tri_batched's float64 Parlett-Higham on a
   synthetic batch of min(1024, 2^27 / n^2) problems of order n with each
   leaf size 16, 32, 64, store the fastest in the cutoff table, and for n >=
   1024 also time SIGNTRI_PH_MIXED_FP16 on one problem: when it beats the
   batch's time per problem, the variant table sends that bucket's problems
   there under AUTO.  Allocates an n_max x n_max T and 2^27 doubles of U. */
signtri_status signtri_autotune(int n_max, void *stream);
/* Variant table of the batched path under AUTO: v[k] (0 = batched
   Parlett-Higham, or Parlett-Sylvester when no swaps are needed; else a
   variant other than AUTO, run problem by problem) for problems with
   floor(log2 n) == k, k < len <= 32. */
signtri_status signtri_get_variant_table(int *v, int len);
signtri_status signtri_set_variant_table(const int *v, int len);
/* The batched path keeps, per device and leaf size, the task tables and the
   instantiated CUDA graph of the last group of problems it ran, and relaunches
   that graph when a call brings a group of the same shape (member sizes and
   order, descriptor and scratch addresses).  hits: launches of a kept graph;
   builds: graphs built, since the library was loaded. */
signtri_status signtri_batched_cache_stats(long long *hits, long long *builds);

/* Inertia scan alone (Section 3): counts of positive and negative diagonal
   entries and the number of adjacent swaps that group positives first.
   Synchronous on `stream`.  Any output pointer may be NULL. */
signtri_status signtri_inertia(int n, const double *T, int ldt, int *n_pos, int *n_neg,
                               long long *swaps, void *stream);

/* Copy of the record of the last sign_tri / sign_tri_host call made by the
   calling host thread. */
signtri_status signtri_get_info(signtri_info *out);

/* ---- sign(A) from a real Schur form (Section 1; Algorithm 3's first step) --
   The paper computes sign(A) of a general A as Q sign(T) Q^* from a Schur
   decomposition A = Q T Q^*.  This call does the part after the
   decomposition for a real Schur pair whose T is upper triangular (A with
   real eigenvalues, none zero; e.g. the real Schur form of such an A from a
   host LAPACK): S = Q U Q^T with U = sign(T) by `variant` (as sign_tri), then
   W = U Q^T and S = Q W as emulated-float64 tensor-core products (7 exact
   slices of 7 bits per row or column under power-of-two scales, error about
   2^-45 of the product of the scales).  Q, T, S: n x n device pointers,
   column-major, leading dimensions >= n; Q orthogonal is the caller's
   promise (not checked); only T's upper triangle is read.  S must not share
   an element with Q or T (SIGNTRI_ERR_BAD_ARG).  The Schur decomposition
   itself, and complex Schur forms, are not provided.  Statuses as
   sign_tri (SIGNTRI_ERR_ZERO_EIGENVALUE / NONFINITE for t_ii);
   signtri_get_info reports the variant that ran.  Synchronous on `stream`;
   with a caller workspace (signtri_set_workspace) it needs
   signtri_sign_schur_workspace_bytes(n, variant) bytes. */
signtri_status signtri_sign_schur(int n, const double *Q, int ldq, const double *T, int ldt, double *S, int lds,
                                  signtri_variant variant, void *stream);
size_t signtri_sign_schur_workspace_bytes(int n, signtri_variant variant);

/* ---- Complex T and the complex Schur route (Section 1; Algorithm 3) -------
   The Schur form of a general A is complex.  Complex matrices here are
   interleaved (re, im) float64 pairs, column-major, leading dimensions
   counted in complex elements (LAPACK's COMPLEX*16 / cuDoubleComplex).
   signtri_sign_tri_complex: U = sign(T) for complex upper triangular T,
   u_ii = sign(Re t_ii) and Eqs. 1 and 2 entry by entry in complex float64
   (one launch per anti-diagonal, a warp per entry; float64 rate).  A
   diagonal entry with Re t_ii == 0 (the sign is undefined on the imaginary
   axis) gives SIGNTRI_ERR_ZERO_EIGENVALUE, a non-finite one
   SIGNTRI_ERR_NONFINITE, the first such index in signtri_get_info.  Only
   T's upper triangle is read; U's strictly lower part is written as 0.
   signtri_sign_schur_complex: S = Q U Q^H for a caller's complex Schur pair
   (A = Q T Q^H, Q unitary -- not checked), the products as four real
   emulated-float64 tensor-core products each (about 2^-45 of the product
   of the row and column scales).  Outputs must not share an element with
   the inputs (SIGNTRI_ERR_BAD_ARG).  Both synchronous on `stream`; with a
   caller workspace they need signtri_complex_workspace_bytes(n). */
signtri_status signtri_sign_tri_complex(int n, const double *T, int ldt, double *U, int ldu, void *stream);
signtri_status signtri_sign_schur_complex(int n, const double *Q, int ldq, const double *T, int ldt, double *S,
                                          int lds, void *stream);
size_t signtri_complex_workspace_bytes(int n);

/* ---- The Schur decomposition, and sign(A) of a general real A (Section 1) --
   The paper's route for a general A: a complex Schur decomposition
   A = Q T Q^H, then sign(A) = Q sign(T) Q^H.  signtri_schur computes the
   decomposition on the GPU for a real n x n A (column-major, device):
   Householder reduction to Hessenberg form, then the implicitly shifted QR
   iteration in complex float64 (Wilkinson shifts, deflation at negligible
   subdiagonal entries).  Outputs: Q unitary and T upper triangular
   (strictly lower part written 0), both complex as above (interleaved
   (re, im) float64, column-major, ld in complex elements); the diagonal of
   T holds the eigenvalues in no particular order.  The QR sweeps run on
   one thread-block cluster of 16 CTAs (8 where the device cannot place 16),
   two bulges per sweep and a cluster barrier per pair of plane rotations;
   the logged rotations reach the rest of T and Q on a second stream, which
   the call creates and destroys, while the next sweeps run.  The sweeps are
   a serial chain: on one GB300, sign(A) by this route takes about as long
   at n = 2048 as the same route on the host through LAPACK's Schur form,
   and longer below.  signtri_sign_general: S = sign(A) for real A, real
   n x n (device, column-major): signtri_schur, the complex sign of T
   (signtri_sign_tri_complex), Q U Q^H (as signtri_sign_schur_complex), and
   the real part (A real makes sign(A) real; the imaginary part left is
   rounding).  Statuses: SIGNTRI_ERR_NONFINITE when A holds a non-finite
   entry (signtri_get_info's bad_index: the first such column),
   SIGNTRI_ERR_NO_CONVERGENCE when an eigenvalue takes more than 100 QR
   sweeps, and for sign_general SIGNTRI_ERR_ZERO_EIGENVALUE when a computed
   eigenvalue has real part exactly 0 (bad_index: its position on T's
   diagonal).  Outputs must not share an element with A or with each other
   (SIGNTRI_ERR_BAD_ARG).  Synchronous on `stream`; with a caller workspace
   they need signtri_schur_workspace_bytes(n) and
   signtri_sign_general_workspace_bytes(n) bytes. */
signtri_status signtri_schur(int n, const double *A, int lda, double *Q, int ldq, double *T, int ldt, void *stream);
size_t signtri_schur_workspace_bytes(int n);
signtri_status signtri_sign_general(int n, const double *A, int lda, double *S, int lds, void *stream);
size_t signtri_sign_general_workspace_bytes(int n);

/* ---- A general function of T (Section 2: Algorithms 1 and 2) --------------
   F = phi(T) for real upper triangular T with distinct diagonal entries, by
   Parlett's substitution: f_ii = phi(t_ii), and entry (i, j) of TF = FT,
   (t_ii - t_jj) f_ij = t_ij (f_ii - f_jj) + sum_{i<k<j} (f_ik t_kj - t_ik f_kj),
   blocked as Algorithm 2 with the float64 Parlett-Higham partition (the
   off-diagonal blocks' Sylvester equations solved by the element recurrence
   inside each block, their right-hand sums by the float64 block-sum kernels;
   leaf size as signtri_set_cutoff).  phi: exp, the principal log and sqrt
   (t_ii > 0), or sign (every entry through TU = UT; sign_tri's Algorithm 3
   is the better-conditioned route for that one).  Divisions by
   t_ii - t_jj amplify rounding when eigenvalues are close (the paper's
   caveat); there is no cluster-based blocking.  Only T's upper triangle is
   read; F's strictly lower part is written as 0.  SIGNTRI_ERR_DOMAIN with
   the first offending index in signtri_get_info's bad_index when a diagonal
   entry is outside phi's domain, not finite, or repeated.  F must not share
   an element with T.  Synchronous on `stream`. */
typedef enum {
    SIGNTRI_PHI_EXP = 1,
    SIGNTRI_PHI_LOG = 2,
    SIGNTRI_PHI_SQRT = 3,
    SIGNTRI_PHI_SIGN = 4
} signtri_phi;
signtri_status signtri_funm(int n, const double *T, int ldt, double *F, int ldf, signtri_phi phi, void *stream);

/* ---- Emulated float64 product on the tensor cores --------------------------
   C = A B (A m x k, B k x n, C m x n; device pointers, column-major) with
   float64-level accuracy from bf16 tensor-core products: each row of A and
   column of B is cut into 8 integer slices of 7 bits under its own
   power-of-two scale (every entry kept to 2^-56 of that scale); the 36 slice
   products with s + t <= 7 are accumulated in fp32 over K-chunks of at most
   1024 (exact: every partial sum is an integer below 2^24) and summed in
   double-float (fp32 hi + lo).  The error is therefore relative to the
   scales, not to each entry: when the entries of each row of A and each
   column of B are of similar magnitude (as in the tests, k up to 4100) it
   stays below 2^-44 (|A| |B|)_ij; an entry far below its row's or column's
   largest keeps correspondingly fewer bits.  The mixed variants' refinement
   residuals TU - UT and U^2 - I use this product on the strictly upper parts
   (the diagonal terms in float64).  C must not share an
   element with A or B (SIGNTRI_ERR_BAD_ARG).  Synchronous on `stream`;
   SIGNTRI_ERR_TIMEOUT if a bounded device wait expired. */
signtri_status signtri_gemm_emulated(int m, int n, int k, const double *A, int lda, const double *B, int ldb,
                                     double *C, int ldc, void *stream);

/* ---- Building blocks of Parlett-Sylvester (Section 2, Section 5.1) -------- */

/* Schur reordering by sign: Tr = Q^T T Q with Q orthogonal and Tr upper
   triangular whose diagonal holds the diagonal of T permuted so that all
   positive entries come first, each sign group in its original order.
   Adjacent Givens swaps, *swaps of them (the number of pairs i<j with
   t_ii < 0 < t_jj, the minimum).  T, Tr, Q device pointers, n x n
   column-major; T is only read (its upper triangle), Tr's strictly lower part
   is written as 0.  Tr and Q share no element with T or with each other
   (SIGNTRI_ERR_BAD_ARG).  Synchronous on `stream` (the swap schedule is
   built on the host from the diagonal signs).  swaps may be NULL.  For
   n < 512 the swaps run as odd-even rounds applied in float64; from 512 on
   as sweeps of windows of 128 (offsets 0 and 64), each window partitioned in
   shared memory by the same swaps and its accumulated factor applied to the
   rest of T and Q by emulated-float64 tensor-core products. */
signtri_status signtri_reorder_by_sign(int n, const double *T, int ldt, double *Tr, int ldtr,
                                       double *Q, int ldq, long long *swaps, void *stream);

/* Triangular Sylvester equation A X - X B = C for X (m x p): A (m x m) and
   B (p x p) upper triangular (only their upper triangles are read) with
   a_ii != b_jj for all i, j; C (m x p).  All device pointers, column-major;
   X must not share an element with A, B or C (SIGNTRI_ERR_BAD_ARG).  Enqueued on `stream`.  m == 0 or p == 0 is a
   no-op. */
signtri_status signtri_sylvester(int m, int p, const double *A, int lda, const double *B, int ldb,
                                 const double *C, int ldc, double *X, int ldx, void *stream);

/* ---- Observability (not part of the method) ------------------------------
   Kernel classes, for the launch counters and device-time accounting. */
enum {
    SIGNTRI_KC_SCAN = 0,          /* inertia scan */
    SIGNTRI_KC_FILL = 1,          /* identity / zero / copy fills */
    SIGNTRI_KC_DIAG_LEAF = 2,     /* diagonal-block leaves (Algorithm 3 per block) */
    SIGNTRI_KC_BLOCK_SUMS_F64 = 3,/* float64 block sums X, Y (Section 5.2) */
    SIGNTRI_KC_OFFDIAG_LEAF = 4,  /* off-diagonal leaves (Algorithm 6, 1x1 case) */
    SIGNTRI_KC_BLOCK_SUMS_TC = 5, /* tensor-core block sums (mixed variants) */
    SIGNTRI_KC_OFFDIAG_LEAF_F32 = 6, /* off-diagonal leaves of the mixed variants */
    SIGNTRI_KC_CONVERT = 7,       /* precision conversion / splitting */
    SIGNTRI_KC_RESIDUAL = 8,      /* refinement residual products (tensor cores) */
    SIGNTRI_KC_CORRECTION = 9,    /* refinement corrections */
    SIGNTRI_KC_GIVENS = 10,       /* Parlett-Sylvester reorder rounds */
    SIGNTRI_KC_SYLV_SUMS = 11,    /* Sylvester block sums */
    SIGNTRI_KC_SYLV_LEAF = 12,    /* Sylvester in-block recurrence */
    SIGNTRI_KC_GEMM_F64 = 13,     /* float64 GEMM (back-transform) */
    SIGNTRI_KC_OTHER = 14,
    SIGNTRI_KC_RESIDUAL_SUM = 15, /* residual assembly and norms */
    SIGNTRI_KC_BATCH_GRAPH = 16,  /* one launch of the captured batch graph */
    SIGNTRI_KC_SCHUR = 17,        /* Schur decomposition: QR sweeps and their rotations */
    SIGNTRI_KC_HESSENBERG = 18,   /* Schur decomposition: Householder reduction */
    SIGNTRI_KC_HOST_COPY = 19,    /* sign_tri_host's host <-> device copies (counted as calls) */
    SIGNTRI_KC_COUNT = 20
};

/* on != 0: bracket every library kernel launch with CUDA events on its
   stream from now on (adds two event records per launch; launches that run
   side by side on the caller's and a side stream are bracketed together, as
   one interval on the caller's stream).  Launch counts are kept either way
   (launches inside a captured graph are counted, not timed). */
signtri_status signtri_profile_enable(int on);
/* Zero the launch counters and timers. */
signtri_status signtri_profile_reset(void);
/* Launches of class `cls` since the last reset and their summed device time
   in milliseconds (waits for the recorded events; a side-by-side group adds
   its one interval).  Either pointer may be NULL. */
signtri_status signtri_profile_read(int cls, long long *launches, double *device_ms);
/* Algorithmic tensor-core flops issued by launches of class `cls` since the
   last reset: 2*64*64*64 per (slice pair, K-block, used 64x64 quadrant) of
   every tensor-core job.  Zero for classes that do not use tensor cores. */
signtri_status signtri_profile_read_flops(int cls, double *flops);
/* Algorithmic operand bytes that launches of class `cls` read from device
   memory since the last reset, where the class has a byte model: for the
   tensor-core sweeps of the mixed variants (class block_sums_tc), 8 KB per
   (bf16 slice, 64-row panel, 64-wide K-block) of the panels each tile
   K-block needs, each read once: four in the initial sweep (a look-ahead
   launch adds only its two column panels, its row panels being its partner
   launch's; a completion launch four panels over four K-blocks per tile),
   six for the correction's two side-by-side launches, which share the
   correction's panels (eight when they run one after the other).  Zero for
   the other classes. */
signtri_status signtri_profile_read_bytes(int cls, double *bytes);
/* Name of a kernel class ("" when out of range). */
const char *signtri_kernel_class_name(int cls);
/* Self-test of the bounded device waits used by the tensor-core kernels:
   one thread waits on an mbarrier with a budget of limit_cycles SM cycles
   (1 .. 4e9); with arrive != 0 another warp completes the barrier and the
   call returns SIGNTRI_OK, with arrive == 0 nothing does, the wait gives up,
   and the call returns SIGNTRI_ERR_TIMEOUT (the context stays usable).
   Synchronous on `stream`. */
signtri_status signtri_selftest_wait(int arrive, long long limit_cycles, void *stream);
/* Float64 fused-multiply-add issue rate of the current device, GFLOP/s
   (independent FMA chains; best of three launches on `stream`). */
signtri_status signtri_probe_fp64_peak(double *gflops, void *stream);

/* ---- Entry point that allocates nothing -----------------------------------
   The paper has no counterpart to this call.  It is for callers that cannot
   allocate device memory: code inside a host program that owns all device
   memory through its own pool (a serving runtime, a plugin), where a raw
   cudaMalloc would bypass the owner's accounting or fail, and code that must
   not stall the device (cudaMalloc and cudaFree can synchronize it).

   Same result as sign_tri with SIGNTRI_PH_FP64 (the same kernels and the
   process-wide cutoff), but the scratch lives in a file-scope device array of
   16 MiB inside the library (the block-sum slabs of n = 1024 at the largest
   cutoff, 64, need 15.7 MB): every GPU that loads the library holds it until
   the process exits.  Limits and behaviour:
     - n <= SIGNTRI_NOALLOC_MAX_N (1024); larger n returns
       SIGNTRI_ERR_NO_WORKSPACE without launching anything.
     - Calls no cudaMalloc, cudaFree or allocating library routine.  (With
       signtri_profile_enable on, the library creates CUDA events; leave
       profiling off on such paths.)
     - The first call on a device looks up the array's device address with
       cudaGetSymbolAddress (the device must be current); make that first call
       before any stream capture.  The address is kept for the life of the
       process: do not reset the device (cudaDeviceReset) between calls.
     - All calls share the one array, which keeps the last call's contents;
       nothing in it needs to start at zero.  Calls that overlap on the GPU
       (different streams, or different host threads) race on it: serialize
       them.
     - Waits once on `stream` after the inertia scan, like sign_tri. */
#define SIGNTRI_NOALLOC_MAX_N 1024
signtri_status sign_tri_noalloc(int n, const double *T, int ldt, double *U, int ldu,
                                void *stream);

#ifdef __cplusplus
}
#endif

#endif /* SIGNTRI_H */

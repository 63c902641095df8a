// api.cu -- the extern "C" entry points of libsigntri.so (include/signtri.h).
//
// Host side of sign_tri: argument checks, the inertia scan (the one point
// where the host waits), the variant choice from the Section 3 work
// estimates, workspace management, and dispatch to the variant's kernels.
#include <climits>
#include <cmath>
#include <algorithm>
#include <cstring>
#include <mutex>
#include <utility>
#include <vector>

#include "internal.cuh"

using namespace signtri;

namespace {

constexpr int kMaxDevices = 64;

struct DeviceState {
    void *lib_ptr = nullptr;       // library-owned workspace (cudaMalloc)
    size_t lib_bytes = 0;
    void *user_ptr = nullptr;      // caller-owned workspace, if set
    size_t user_bytes = 0;
    ScanResult *scan_dev = nullptr;
    ScanResult *scan_host = nullptr;   // pinned
    int *err_dev = nullptr;            // device error word of bounded waits
    int *err_host = nullptr;           // pinned
    double *norms_host = nullptr;      // pinned, refinement norms
    double *stage_T = nullptr;     // device staging for sign_tri_host
    double *stage_U = nullptr;
    size_t stage_elems = 0;
    bool ready = false;            // every per-device buffer above the workspace allocated
};

std::mutex g_mu;
DeviceState g_dev[kMaxDevices];
// 0: by size (default_cutoff); else the leaf size set by signtri_set_cutoff
int g_cutoff = 0;
// leaf size per size bucket floor(log2 n) for the batched path; 0 = g_cutoff
int g_cutoff_table[32] = {};
// variant AUTO runs per size bucket in the batched path; 0 = the batched
// Parlett-Higham (or Parlett-Sylvester when no swaps are needed)
int g_variant_table[32] = {};
// flops/s used by the AUTO choice (float64 block products; Givens rounds)
constexpr double kDefaultGemmRate = 1.2e12;   // the measured float64 FMA rate of a GB300
constexpr double kDefaultGivensRate = 0.35e12;
double g_rate_gemm = kDefaultGemmRate;
double g_rate_givens = kDefaultGivensRate;
// stopping tolerance of the mixed variants on ||TU-UT||_F/(||T||_F||U||_F)
// and ||U^2-I||_F/||U||_F^2
constexpr double kDefaultMixedTol = 1e-13;
double g_mixed_tol = kDefaultMixedTol;
int g_mixed_max_steps = -1;   // < 0: per-variant default
int g_mixed_verify_full = 0;  // 1: accept on the full residuals, 0: on their probe estimate
thread_local signtri_info g_info;

bool valid_variant(int v) { return v >= SIGNTRI_AUTO && v <= SIGNTRI_PH_MIXED_FP16; }

signtri_status current_state(DeviceState **out)
{
    int dev = 0;
    SGT_CUDA_TRY(cudaGetDevice(&dev));
    if (dev < 0 || dev >= kMaxDevices) return SIGNTRI_ERR_CUDA;
    DeviceState &s = g_dev[dev];
    if (!s.ready) {
        // a piece is stored only once allocated, so a call after a failed
        // attempt allocates what is still missing instead of using a NULL
        void *p = nullptr;
        if (!s.scan_dev) {
            SGT_CUDA_TRY(cudaMalloc(&p, sizeof(ScanResult)));
            s.scan_dev = static_cast<ScanResult *>(p);
        }
        if (!s.scan_host) {
            SGT_CUDA_TRY(cudaMallocHost(&p, sizeof(ScanResult)));
            s.scan_host = static_cast<ScanResult *>(p);
        }
        if (!s.err_dev) {
            SGT_CUDA_TRY(cudaMalloc(&p, sizeof(int)));
            s.err_dev = static_cast<int *>(p);
        }
        if (!s.err_host) {
            SGT_CUDA_TRY(cudaMallocHost(&p, sizeof(int)));
            s.err_host = static_cast<int *>(p);
        }
        if (!s.norms_host) {
            SGT_CUDA_TRY(cudaMallocHost(&p, 8 * sizeof(double)));
            s.norms_host = static_cast<double *>(p);
        }
        SGT_CUDA_TRY(cudaMemset(s.err_dev, 0, sizeof(int)));
        s.ready = true;
    }
    *out = &s;
    return SIGNTRI_OK;
}

// Workspace of at least `need` bytes for the current device.
signtri_status get_workspace(DeviceState &s, size_t need, Arena &a)
{
    a = Arena();
    if (need == 0) return SIGNTRI_OK;
    if (s.user_ptr) {
        if (s.user_bytes < need) return SIGNTRI_ERR_NO_WORKSPACE;
        a.base = static_cast<char *>(s.user_ptr);
        a.bytes = s.user_bytes;
        return SIGNTRI_OK;
    }
    if (s.lib_bytes < need) {
        if (s.lib_ptr) {
            // the previous workspace may still be in use by enqueued work
            if (cudaDeviceSynchronize() != cudaSuccess) return SIGNTRI_ERR_CUDA;
            cudaFree(s.lib_ptr);
            s.lib_ptr = nullptr;
            s.lib_bytes = 0;
        }
        if (cudaMalloc(&s.lib_ptr, need) != cudaSuccess) {
            cudaGetLastError();
            return SIGNTRI_ERR_NO_WORKSPACE;
        }
        s.lib_bytes = need;
    }
    a.base = static_cast<char *>(s.lib_ptr);
    a.bytes = s.lib_bytes;
    return SIGNTRI_OK;
}

// swaps < 0: the worst case over inertia (n^2/4 swaps).
// Leaf size of the float64 forms when none is set: measured on GB300 (p = 0.5
// random), the fastest of 16, 32, 64 per size -- small leaves while the leaf
// latency dominates, larger ones once the block sums do: the efficient form
// 16 below n = 4096, 32 below 8192, then 64; the matrix-multiply form 16 up
// to 4096, then 32.
int default_cutoff(int n, signtri_variant v)
{
    if (v == SIGNTRI_PH_FP64_EFFICIENT || v == SIGNTRI_AUTO) return n < 4096 ? 16 : (n < 8192 ? 32 : 64);
    return n <= 4096 ? 16 : 32;
}

// the leaf size a float64 form runs with (callers hold g_mu)
int cutoff_of(int n, signtri_variant v)
{
    return g_cutoff ? g_cutoff : default_cutoff(n, v);
}

size_t workspace_need(int n, signtri_variant v, long long swaps)
{
    if (swaps < 0) swaps = (long long)n * n / 4;
    const int cutoff = cutoff_of(n, v == SIGNTRI_PH_FP64_EFFICIENT || v == SIGNTRI_AUTO ? v : SIGNTRI_PH_FP64);
    switch (v) {
    case SIGNTRI_PH_FP64:
        return ph_fp64_workspace_bytes(n, cutoff);
    case SIGNTRI_PH_FP64_EFFICIENT:
        return ph_fp64_split_workspace_bytes(n, cutoff);
    case SIGNTRI_PH_MIXED_TF32:
    case SIGNTRI_PH_MIXED_BF16:
    case SIGNTRI_PH_MIXED_FP16:
        // the float64 fallback reuses the same memory
        return std::max(mixed_workspace_bytes(n, v == SIGNTRI_PH_MIXED_TF32 ? 3 : (v == SIGNTRI_PH_MIXED_FP16 ? 2 : 1)),
                        ph_fp64_workspace_bytes(n, cutoff));
    case SIGNTRI_PS_FP64:
        return ps_workspace_bytes(n, swaps);
    case SIGNTRI_AUTO:
        return std::max(ph_fp64_split_workspace_bytes(n, cutoff), ps_workspace_bytes(n, swaps));
    }
    return 0;
}

// Section 3 estimates.  Parlett-Higham: the inner sums of Algorithm 3,
// 2 flops per U^2 = I term and 4 per TU = UT term.  Parlett-Sylvester:
// 12 n k for k swaps (including Q), n_- n_+ (n_- + n_+) for the Sylvester
// solve, and for the back-transform by GEMM when k > 0
// 2 n min(n_-,n_+) (n + max(n_-,n_+)).
void work_estimates(int n, const ScanResult &r, double *w_ph, double *w_ps)
{
    // (the useful count of Algorithm 3 for Parlett-Higham)
    const double nd = n;
    const double all_terms = nd * (nd - 1.0) * (nd - 2.0) / 6.0;   // sum_{i<j} (j-i-1)
    const double same = (double)r.same_terms;
    *w_ph = 2.0 * same + 4.0 * (all_terms - same);
    const double np = r.n_pos, nm = r.n_neg, k = (double)r.swaps;
    double w = 12.0 * nd * k + np * nm * nd;
    if (r.swaps > 0) w += 2.0 * nd * std::fmin(np, nm) * (nd + std::fmax(np, nm));
    *w_ps = w;
}

// Times predicted from the Section 3 work of what each variant executes,
// plus the latency-bound parts, with constants measured on GB300 (float64
// leaves and the windowed reorder, whose cost is not in the flop counts):
//  * Parlett-Higham runs the arithmetic-efficient form (Section 5.3: only the
//    sum each entry needs, exactly the useful count w_ph) at the float64
//    product rate, and one off-diagonal leaf step per block column (about
//    0.06, 0.21, 0.7 ms at b = 16, 32, 64);
//  * Parlett-Sylvester runs the Sylvester block sums (n_- n_+ n flops, in
//    double-float at about 4e12 flop/s) and one in-block step per block
//    anti-diagonal (about 0.29 ms); when k > 0,
//    the reorder and the back-transform (emulated-float64 tensor-core
//    products, about 6e13 float64 flop/s).  The windowed reorder (n >= 512)
//    runs sweeps of windows of 128 at offsets 0 / 64: a negative moves at
//    most 64 places a sweep, so there are about d / 64 sweeps, d = n_+ -
//    (index of the first negative) the longest distance one travels.  A
//    sweep costs its window launch (rounds and float64 rotations, growing
//    with the swaps per window, about 0.1 ms with a few and 0.5 ms with
//    ~770), plus the products and slicing of its about min(n_-, n / 256)
//    active windows, each about 0.7e-8 n seconds.  The
//    unblocked rounds (n < 512) cost 12 n k flops at the Givens rate and two
//    launches per round.
constexpr double kLaunchSeconds = 5e-6;
double ph_leaf_step_seconds(int b)
{
    return b <= 16 ? 0.06e-3 : (b <= 32 ? 0.21e-3 : 0.7e-3);
}
constexpr double kSylvStepSeconds = 0.29e-3;
constexpr double kSylvRate = 4e12;
constexpr double kEmulatedRate = 6e13;
constexpr double kWindowProductSeconds = 0.7e-8;

double window_launch_seconds(double kw)
{
    return 1e-4 + 4e-4 * std::fmin(kw, 770.0) / 770.0 + 2.6e-7 * std::fmax(0.0, kw - 770.0);
}

signtri_variant choose_variant(int n, const ScanResult &r)
{
    const double nd = n;
    const int b = cutoff_of(n, SIGNTRI_PH_FP64_EFFICIENT);
    const double nb = std::ceil(nd / b);
    double w_ph = 0.0, w_ps = 0.0;
    work_estimates(n, r, &w_ph, &w_ps);
    const double t_ph = w_ph / g_rate_gemm + nb * ph_leaf_step_seconds(b) + 2.0 * nb * kLaunchSeconds;
    const double np = r.n_pos, nm = r.n_neg, k = (double)r.swaps;
    const double sylv_steps = std::ceil(np / 64.0) + std::ceil(nm / 64.0) - 1.0;
    double t_ps = np * nm * nd / kSylvRate + sylv_steps * kSylvStepSeconds;
    if (r.swaps > 0) {
        t_ps += 2.0 * nd * std::fmin(np, nm) * (nd + std::fmax(np, nm)) / kEmulatedRate;
        if (n >= kBlockedReorderMin) {
            const double d = std::fmax(1.0, np - (double)r.first_neg);
            const double sweeps = std::ceil(d / 64.0) + 1.0;
            const double active = std::fmax(1.0, std::fmin(nm, nd / 256.0));
            const double kw = std::fmin(4096.0, k / (sweeps * active));
            t_ps += sweeps * (window_launch_seconds(kw) + kWindowProductSeconds * active * nd);
        } else {
            t_ps += 12.0 * nd * k / g_rate_givens + 2.0 * nd * kLaunchSeconds;
        }
    }
    return t_ps < t_ph ? SIGNTRI_PS_FP64 : SIGNTRI_PH_FP64_EFFICIENT;
}

signtri_status run_variant(int n, const double *T, int ldt, double *U, int ldu, signtri_variant v,
                           const ScanResult &r, cudaStream_t st, DeviceState &s)
{
    Arena ws;
    const int b = cutoff_of(n, v == SIGNTRI_PH_FP64_EFFICIENT ? v : SIGNTRI_PH_FP64);
    signtri_status rs = get_workspace(s, workspace_need(n, v, r.swaps), ws);
    if (rs != SIGNTRI_OK) return rs;
    switch (v) {
    case SIGNTRI_PH_FP64:
        g_info.cutoff = b;
        return ph_fp64_run(n, T, ldt, U, ldu, b, ws, st);
    case SIGNTRI_PH_FP64_EFFICIENT:
        g_info.cutoff = b;
        return ph_fp64_split_run(n, T, ldt, U, ldu, b, ws, st);
    case SIGNTRI_PS_FP64: {
        SGT_CUDA_TRY(cudaMemsetAsync(s.err_dev, 0, sizeof(int), st));
        rs = ps_fp64_run(n, T, ldt, U, ldu, r.n_pos, r.swaps, ws, s.err_dev, st);
        if (rs != SIGNTRI_OK) return rs;
        if (r.swaps > 0 && n >= kBlockedReorderMin) {
            // the blocked reorder's tensor-core products wait with a bound
            SGT_CUDA_TRY(cudaMemcpyAsync(s.err_host, s.err_dev, sizeof(int), cudaMemcpyDeviceToHost, st));
            SGT_CUDA_TRY(cudaStreamSynchronize(st));
            if (*s.err_host) return SIGNTRI_ERR_TIMEOUT;
        }
        return SIGNTRI_OK;
    }
    case SIGNTRI_PH_MIXED_TF32:
    case SIGNTRI_PH_MIXED_BF16:
    case SIGNTRI_PH_MIXED_FP16: {
        // S split terms per operand; a negative S marks the fp16 split
        const int S = (v == SIGNTRI_PH_MIXED_TF32) ? 3 : (v == SIGNTRI_PH_MIXED_FP16 ? -2 : 1);
        MixedParams prm{g_mixed_tol, g_mixed_max_steps >= 0 ? g_mixed_max_steps : (S == 1 ? 8 : 3), 10.0,
                        g_mixed_verify_full};
        MixedReport rep{};
        SGT_CUDA_TRY(cudaMemsetAsync(s.err_dev, 0, sizeof(int), st));
        rs = mixed_run(n, T, ldt, U, ldu, S, prm, rep, ws, s.err_dev, s.norms_host, st);
        if (rs != SIGNTRI_OK) return rs;
        SGT_CUDA_TRY(cudaMemcpyAsync(s.err_host, s.err_dev, sizeof(int), cudaMemcpyDeviceToHost, st));
        SGT_CUDA_TRY(cudaStreamSynchronize(st));
        if (*s.err_host) return SIGNTRI_ERR_TIMEOUT;
        g_info.refine_steps = rep.steps;
        g_info.resid_commute = rep.resid_commute;
        g_info.resid_involution = rep.resid_involution;
        g_info.cutoff = 64;
        if (rep.fallback) {
            // the residual did not contract: plain float64 path
            g_info.variant = SIGNTRI_PH_FP64;
            g_info.cutoff = b;
            Arena ws2;
            rs = get_workspace(s, ph_fp64_workspace_bytes(n, b), ws2);
            if (rs != SIGNTRI_OK) return rs;
            return ph_fp64_run(n, T, ldt, U, ldu, b, ws2, st);
        }
        return SIGNTRI_OK;
    }
    default:
        return SIGNTRI_ERR_UNSUPPORTED;
    }
}

signtri_status sign_tri_locked(int n, const double *T, int ldt, double *U, int ldu, signtri_variant v,
                               cudaStream_t st, DeviceState &s)
{
    if (n == 0) return SIGNTRI_OK;
    signtri_status rs = launch_inertia_scan(n, T, ldt, s.scan_dev, st);
    if (rs != SIGNTRI_OK) return rs;
    SGT_CUDA_TRY(cudaMemcpyAsync(s.scan_host, s.scan_dev, sizeof(ScanResult), cudaMemcpyDeviceToHost, st));
    SGT_CUDA_TRY(cudaStreamSynchronize(st));
    const ScanResult r = *s.scan_host;
    g_info.n_pos = r.n_pos;
    g_info.n_neg = r.n_neg;
    g_info.swaps = r.swaps;
    if (r.bad_key != INT_MAX) {
        g_info.bad_index = r.bad_key / 4;
        return (signtri_status)(r.bad_key % 4);
    }
    work_estimates(n, r, &g_info.work_ph, &g_info.work_ps);
    if (r.n_neg == 0 || r.n_pos == 0) {
        // sign(T) = I or -I exactly (Section 3, the trivial case)
        g_info.variant = v;
        return launch_fill_identity(n, U, ldu, r.n_neg == 0 ? 1.0 : -1.0, st);
    }
    signtri_variant run = v;
    if (v == SIGNTRI_AUTO) run = choose_variant(n, r);
    g_info.variant = run;
    return run_variant(n, T, ldt, U, ldu, run, r, st, s);
}

void reset_info(int n)
{
    std::memset(&g_info, 0, sizeof(g_info));
    g_info.n = n;
    g_info.bad_index = -1;
    g_info.variant = -1;
}

int size_bucket(int n)
{
    int k = 0;
    while ((2 << k) <= n && k < 31) k++;
    return k;
}

int cutoff_for(int n)
{
    const int k = size_bucket(n);
    return g_cutoff_table[k] ? g_cutoff_table[k] : cutoff_of(n, SIGNTRI_PH_FP64_EFFICIENT);
}

// Synthetic upper-triangular T for the autotuner: counter-based hash
// (splitmix64) of (seed, i, j); diagonal sign +-1 with probability 1/2 and
// magnitude in [0.5, 2]; strictly upper N(0, 1/n) by Box-Muller.
__device__ __forceinline__ unsigned long long mix64(unsigned long long z)
{
    z += 0x9e3779b97f4a7c15ull;
    z = (z ^ (z >> 30)) * 0xbf58476d1ce4e5b9ull;
    z = (z ^ (z >> 27)) * 0x94d049bb133111ebull;
    return z ^ (z >> 31);
}

__global__ void synth_kernel(int n, double *T, unsigned long long seed)
{
    const int j = blockIdx.x;
    const double sc = rsqrt((double)n);
    for (int i = threadIdx.x; i < n; i += blockDim.x) {
        const unsigned long long h1 = mix64(seed ^ ((unsigned long long)i << 32 | (unsigned)j));
        const unsigned long long h2 = mix64(h1);
        const double u1 = ((h1 >> 11) + 1) * (1.0 / 9007199254740993.0), u2 = (h2 >> 11) * (1.0 / 9007199254740992.0);
        double v = 0.0;
        if (i == j) v = ((h2 & 1) ? -1.0 : 1.0) * (0.5 + 1.5 * u1);
        else if (i < j) v = sc * sqrt(-2.0 * log(u1)) * cospi(2.0 * u2);
        SGT_AT(T, n, i, j) = v;
    }
}

}  // namespace

int signtri::current_cutoff(int n)
{
    std::lock_guard<std::mutex> lk(g_mu);
    return cutoff_of(n, SIGNTRI_PH_FP64);
}

extern "C" {

const char *signtri_status_string(signtri_status s)
{
    switch (s) {
    case SIGNTRI_OK: return "SIGNTRI_OK";
    case SIGNTRI_ERR_BAD_ARG: return "SIGNTRI_ERR_BAD_ARG";
    case SIGNTRI_ERR_ZERO_EIGENVALUE: return "SIGNTRI_ERR_ZERO_EIGENVALUE";
    case SIGNTRI_ERR_NONFINITE: return "SIGNTRI_ERR_NONFINITE";
    case SIGNTRI_ERR_NO_CONVERGENCE: return "SIGNTRI_ERR_NO_CONVERGENCE";
    case SIGNTRI_ERR_TIMEOUT: return "SIGNTRI_ERR_TIMEOUT";
    case SIGNTRI_ERR_CUDA: return "SIGNTRI_ERR_CUDA";
    case SIGNTRI_ERR_NO_WORKSPACE: return "SIGNTRI_ERR_NO_WORKSPACE";
    case SIGNTRI_ERR_UNSUPPORTED: return "SIGNTRI_ERR_UNSUPPORTED";
    case SIGNTRI_ERR_DOMAIN: return "SIGNTRI_ERR_DOMAIN";
    }
    return "SIGNTRI_ERR_UNKNOWN";
}

size_t signtri_workspace_bytes(int n, signtri_variant v)
{
    if (n < 0 || !valid_variant(v)) return 0;
    std::lock_guard<std::mutex> lk(g_mu);
    return workspace_need(n, v, -1);
}

signtri_status signtri_set_rates(double gemm_flops_per_s, double givens_flops_per_s)
{
    std::lock_guard<std::mutex> lk(g_mu);
    g_rate_gemm = gemm_flops_per_s > 0 ? gemm_flops_per_s : kDefaultGemmRate;
    g_rate_givens = givens_flops_per_s > 0 ? givens_flops_per_s : kDefaultGivensRate;
    return SIGNTRI_OK;
}

signtri_status sign_tri_batched(int count, const int *n, const double *const *T, const int *ldt, double *const *U,
                                const int *ldu, signtri_variant v, int *info, void *stream)
{
    reset_info(-1);
    if (count < 0 || !valid_variant(v)) return SIGNTRI_ERR_BAD_ARG;
    if (count == 0) return SIGNTRI_OK;
    if (!n || !T || !ldt || !U || !ldu || !info) return SIGNTRI_ERR_BAD_ARG;
    std::lock_guard<std::mutex> lk(g_mu);
    DeviceState *s = nullptr;
    signtri_status rs = current_state(&s);
    if (rs != SIGNTRI_OK) return rs;
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    std::vector<BatchDesc> descs;
    std::vector<int> owner, sizes, bs;
    int nmax = 0;
    for (int m = 0; m < count; m++) {
        info[m] = SIGNTRI_OK;
        if (n[m] < 0 || (n[m] > 0 && (!T[m] || !U[m] || ldt[m] < n[m] || ldu[m] < n[m] ||
                                      blocks_overlap(T[m], ldt[m], n[m], n[m], U[m], ldu[m], n[m], n[m])))) {
            info[m] = SIGNTRI_ERR_BAD_ARG;
            continue;
        }
        if (n[m] == 0) continue;
        descs.push_back({T[m], U[m], n[m], ldt[m], ldu[m], 0});
        owner.push_back(m);
        sizes.push_back(n[m]);
        bs.push_back(cutoff_for(n[m]));
        nmax = std::max(nmax, n[m]);
    }
    const int cnt = (int)descs.size();
    if (cnt == 0) return SIGNTRI_OK;
    // workspace: descriptors, scan results, fill lists, then the batched plan
    // for every matrix with its cutoff (an upper bound of what runs batched)
    size_t plan = 0;
    for (int B : {16, 32, 64}) {
        std::vector<int> ns;
        for (int k = 0; k < cnt; k++)
            if (bs[k] == B) ns.push_back(sizes[k]);
        if (!ns.empty()) plan = std::max(plan, batched_workspace_bytes((int)ns.size(), ns.data(), B));
    }
    const size_t fixed = (size_t)cnt * (sizeof(BatchDesc) + sizeof(ScanResult) + sizeof(int) + sizeof(double)) +
                         8 * 256;
    Arena ws;
    rs = get_workspace(*s, fixed + plan, ws);
    if (rs != SIGNTRI_OK) return rs;
    auto *d_descs = static_cast<BatchDesc *>(ws.take(cnt * sizeof(BatchDesc)));
    auto *d_scan = static_cast<ScanResult *>(ws.take(cnt * sizeof(ScanResult)));
    auto *d_which = static_cast<int *>(ws.take(cnt * sizeof(int)));
    auto *d_diag = static_cast<double *>(ws.take(cnt * sizeof(double)));
    if (!d_descs || !d_scan || !d_which || !d_diag) return SIGNTRI_ERR_NO_WORKSPACE;
    SGT_CUDA_TRY(cudaMemcpyAsync(d_descs, descs.data(), cnt * sizeof(BatchDesc), cudaMemcpyHostToDevice, st));
    rs = launch_inertia_scan_batched(cnt, d_descs, d_scan, st);
    if (rs != SIGNTRI_OK) return rs;
    std::vector<ScanResult> sr(cnt);
    SGT_CUDA_TRY(cudaMemcpyAsync(sr.data(), d_scan, cnt * sizeof(ScanResult), cudaMemcpyDeviceToHost, st));
    SGT_CUDA_TRY(cudaStreamSynchronize(st));
    // per matrix: error, +-I, batched Parlett-Higham, or a single-matrix variant
    std::vector<int> which;
    std::vector<double> diagv;
    std::vector<int> ph_bs(cnt, 0);
    std::vector<std::pair<int, signtri_variant>> singles;
    for (int k = 0; k < cnt; k++) {
        const ScanResult &r = sr[k];
        const int m = owner[k];
        if (r.bad_key != INT_MAX) { info[m] = r.bad_key % 4; continue; }
        if (r.n_neg == 0 || r.n_pos == 0) {
            which.push_back(k);
            diagv.push_back(r.n_neg == 0 ? 1.0 : -1.0);
            continue;
        }
        signtri_variant run = v;
        // in a batch Parlett-Higham shares its launches with every other
        // problem, so Parlett-Sylvester (run on its own) is taken only when
        // no swaps are needed; a size bucket the autotuner found faster on
        // its own (a mixed variant) runs that way
        if (v == SIGNTRI_AUTO) {
            const int tv = g_variant_table[size_bucket(sizes[k])];
            run = tv ? (signtri_variant)tv : (r.swaps == 0) ? SIGNTRI_PS_FP64 : SIGNTRI_PH_FP64_EFFICIENT;
        }
        if (run == SIGNTRI_PH_FP64 || run == SIGNTRI_PH_FP64_EFFICIENT) {
            ph_bs[k] = bs[k];
            which.push_back(k);
            diagv.push_back(0.0);      // zero the strictly lower part
        } else {
            singles.push_back({k, run});
        }
    }
    if (!which.empty()) {
        SGT_CUDA_TRY(cudaMemcpyAsync(d_which, which.data(), which.size() * sizeof(int), cudaMemcpyHostToDevice, st));
        SGT_CUDA_TRY(cudaMemcpyAsync(d_diag, diagv.data(), diagv.size() * sizeof(double), cudaMemcpyHostToDevice, st));
        rs = launch_fill_batched((int)which.size(), d_descs, d_which, d_diag, st);
        if (rs != SIGNTRI_OK) return rs;
    }
    // the efficient form unless the matrix-multiply form was asked for
    rs = batched_ph_run(cnt, descs.data(), d_descs, ph_bs.data(), v != SIGNTRI_PH_FP64, ws, st);
    if (rs != SIGNTRI_OK) return rs;
    for (auto &sv : singles) {
        const int k = sv.first;
        rs = run_variant(sizes[k], descs[k].T, descs[k].ldt, descs[k].U, descs[k].ldu, sv.second, sr[k], st, *s);
        if (rs != SIGNTRI_OK) info[owner[k]] = rs;
    }
    SGT_CUDA_TRY(cudaStreamSynchronize(st));
    return SIGNTRI_OK;
}

signtri_status signtri_set_cutoff_table(const int *b, int len)
{
    if (len < 0 || len > 32 || (len > 0 && !b)) return SIGNTRI_ERR_BAD_ARG;
    for (int k = 0; k < len; k++)
        if (b[k] != 0 && b[k] != 16 && b[k] != 32 && b[k] != 64) return SIGNTRI_ERR_BAD_ARG;
    std::lock_guard<std::mutex> lk(g_mu);
    for (int k = 0; k < 32; k++) g_cutoff_table[k] = k < len ? b[k] : 0;
    return SIGNTRI_OK;
}

signtri_status signtri_get_cutoff_table(int *b, int len)
{
    if (len < 0 || len > 32 || (len > 0 && !b)) return SIGNTRI_ERR_BAD_ARG;
    std::lock_guard<std::mutex> lk(g_mu);
    for (int k = 0; k < len; k++) b[k] = g_cutoff_table[k];
    return SIGNTRI_OK;
}

signtri_status signtri_autotune(int n_max, void *stream)
{
    if (n_max < 32 || n_max > 32768) return SIGNTRI_ERR_BAD_ARG;
    std::lock_guard<std::mutex> lk(g_mu);
    DeviceState *s = nullptr;
    signtri_status rs = current_state(&s);
    if (rs != SIGNTRI_OK) return rs;
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    // per size bucket n = 2^k: a batch of c = 2^27 / n^2 problems (at most
    // 1024) sharing one synthetic T, each with its own U
    const size_t elems = (size_t)1 << 27;
    double *T = nullptr, *U = nullptr;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    if (cudaMalloc(&T, (size_t)n_max * n_max * 8) != cudaSuccess ||
        cudaMalloc(&U, std::max(elems, (size_t)n_max * n_max) * 8) != cudaSuccess || cudaEventCreate(&e0) != cudaSuccess ||
        cudaEventCreate(&e1) != cudaSuccess)
        rs = SIGNTRI_ERR_CUDA;
    auto timed = [&](auto &&run, float &ms) -> signtri_status {
        // the second of two runs (the first builds what later calls reuse)
        signtri_status r2 = SIGNTRI_OK;
        for (int rep = 0; rep < 2 && r2 == SIGNTRI_OK; rep++) {
            cudaEventRecord(e0, st);
            r2 = run();
            cudaEventRecord(e1, st);
            if (cudaEventSynchronize(e1) != cudaSuccess) r2 = SIGNTRI_ERR_CUDA;
            cudaEventElapsedTime(&ms, e0, e1);
        }
        return r2;
    };
    for (int k = 5; rs == SIGNTRI_OK && (1 << k) <= n_max; k++) {
        const int nn = 1 << k;
        const int c = (int)std::max<size_t>(1, std::min<size_t>(1024, elems / ((size_t)nn * nn)));
        synth_kernel<<<nn, 256, 0, st>>>(nn, T, 0x5eed0000ull + k);
        if (cudaGetLastError() != cudaSuccess) { rs = SIGNTRI_ERR_CUDA; break; }
        std::vector<BatchDesc> h(c);
        for (int m = 0; m < c; m++) h[m] = {T, U + (size_t)m * nn * nn, nn, nn, nn, 0};
        // leaf size: the batched path, per problem
        size_t need = 0;
        std::vector<int> ns(c, nn);
        for (int b : {16, 32, 64}) need = std::max(need, batched_workspace_bytes(c, ns.data(), b));
        Arena ws;
        if ((rs = get_workspace(*s, need + c * sizeof(BatchDesc) + 512, ws)) != SIGNTRI_OK) break;
        auto *d_h = static_cast<BatchDesc *>(ws.take(c * sizeof(BatchDesc)));
        SGT_CUDA_TRY(cudaMemcpyAsync(d_h, h.data(), c * sizeof(BatchDesc), cudaMemcpyHostToDevice, st));
        float best = 1e30f;
        int best_b = 16;
        for (int b : {16, 32, 64}) {
            std::vector<int> bs(c, b);
            float ms = 0.f;
            Arena sub = ws;
            rs = timed([&]() { return batched_ph_run(c, h.data(), d_h, bs.data(), true, sub, st); }, ms);
            if (rs != SIGNTRI_OK) break;
            if (ms < best) { best = ms; best_b = b; }
        }
        if (rs != SIGNTRI_OK) break;
        g_cutoff_table[k] = best_b;
        // variant: the mixed fp16 form on its own, against the batched
        // float64 time per problem (only where one problem is large enough
        // for the tensor-core sweeps to pay)
        g_variant_table[k] = 0;
        if (nn >= 1024) {
            ScanResult r{};
            rs = launch_inertia_scan(nn, T, nn, s->scan_dev, st);
            if (rs != SIGNTRI_OK) break;
            SGT_CUDA_TRY(cudaMemcpyAsync(&r, s->scan_dev, sizeof(ScanResult), cudaMemcpyDeviceToHost, st));
            SGT_CUDA_TRY(cudaStreamSynchronize(st));
            float ms = 0.f;
            rs = timed([&]() { return run_variant(nn, T, nn, U, nn, SIGNTRI_PH_MIXED_FP16, r, st, *s); }, ms);
            if (rs != SIGNTRI_OK) break;
            if (ms < best / c) g_variant_table[k] = SIGNTRI_PH_MIXED_FP16;
        }
    }
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
    cudaFree(T);
    cudaFree(U);
    return rs;
}

signtri_status signtri_get_variant_table(int *v, int len)
{
    if (len < 0 || len > 32 || (len > 0 && !v)) return SIGNTRI_ERR_BAD_ARG;
    std::lock_guard<std::mutex> lk(g_mu);
    for (int k = 0; k < len; k++) v[k] = g_variant_table[k];
    return SIGNTRI_OK;
}

signtri_status signtri_set_variant_table(const int *v, int len)
{
    if (len < 0 || len > 32 || (len > 0 && !v)) return SIGNTRI_ERR_BAD_ARG;
    for (int k = 0; k < len; k++)
        if (v[k] != 0 && !(valid_variant(v[k]) && v[k] != SIGNTRI_AUTO)) return SIGNTRI_ERR_BAD_ARG;
    std::lock_guard<std::mutex> lk(g_mu);
    for (int k = 0; k < 32; k++) g_variant_table[k] = k < len ? v[k] : 0;
    return SIGNTRI_OK;
}

signtri_status signtri_batched_cache_stats(long long *hits, long long *builds)
{
    if (!hits || !builds) return SIGNTRI_ERR_BAD_ARG;
    std::lock_guard<std::mutex> lk(g_mu);
    batched_cache_stats(hits, builds);
    return SIGNTRI_OK;
}

signtri_status signtri_selftest_wait(int arrive, long long limit_cycles, void *stream)
{
    if (limit_cycles <= 0 || limit_cycles > 4000000000LL) return SIGNTRI_ERR_BAD_ARG;
    std::lock_guard<std::mutex> lk(g_mu);
    DeviceState *s = nullptr;
    signtri_status rs = current_state(&s);
    if (rs != SIGNTRI_OK) return rs;
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    SGT_CUDA_TRY(cudaMemsetAsync(s->err_dev, 0, sizeof(int), st));
    rs = wait_selftest(arrive, limit_cycles, s->err_dev, st);
    if (rs != SIGNTRI_OK) return rs;
    SGT_CUDA_TRY(cudaMemcpyAsync(s->err_host, s->err_dev, sizeof(int), cudaMemcpyDeviceToHost, st));
    SGT_CUDA_TRY(cudaStreamSynchronize(st));
    return *s->err_host ? SIGNTRI_ERR_TIMEOUT : SIGNTRI_OK;
}

signtri_status signtri_set_refinement(double tol, int max_steps)
{
    std::lock_guard<std::mutex> lk(g_mu);
    g_mixed_tol = tol > 0 ? tol : kDefaultMixedTol;
    g_mixed_max_steps = max_steps;
    return SIGNTRI_OK;
}

signtri_status signtri_set_verification(int full)
{
    if (full != 0 && full != 1) return SIGNTRI_ERR_BAD_ARG;
    std::lock_guard<std::mutex> lk(g_mu);
    g_mixed_verify_full = full;
    return SIGNTRI_OK;
}

signtri_status signtri_reorder_by_sign(int n, const double *T, int ldt, double *Tr, int ldtr, double *Q, int ldq,
                                       long long *swaps, void *stream)
{
    if (swaps) *swaps = 0;
    if (n < 0) return SIGNTRI_ERR_BAD_ARG;
    if (n == 0) return SIGNTRI_OK;
    if (!T || !Tr || !Q || ldt < n || ldtr < n || ldq < n) return SIGNTRI_ERR_BAD_ARG;
    if (blocks_overlap(T, ldt, n, n, Tr, ldtr, n, n) || blocks_overlap(T, ldt, n, n, Q, ldq, n, n) ||
        blocks_overlap(Tr, ldtr, n, n, Q, ldq, n, n))
        return SIGNTRI_ERR_BAD_ARG;
    std::lock_guard<std::mutex> lk(g_mu);
    DeviceState *s = nullptr;
    signtri_status rs = current_state(&s);
    if (rs != SIGNTRI_OK) return rs;
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    rs = launch_inertia_scan(n, T, ldt, s->scan_dev, st);
    if (rs != SIGNTRI_OK) return rs;
    SGT_CUDA_TRY(cudaMemcpyAsync(s->scan_host, s->scan_dev, sizeof(ScanResult), cudaMemcpyDeviceToHost, st));
    SGT_CUDA_TRY(cudaStreamSynchronize(st));
    const ScanResult r = *s->scan_host;
    if (r.bad_key != INT_MAX) return (signtri_status)(r.bad_key % 4);
    Arena ws;
    rs = get_workspace(s[0], reorder_any_workspace_bytes(n, r.swaps), ws);
    if (rs != SIGNTRI_OK) return rs;
    SGT_CUDA_TRY(cudaMemsetAsync(s->err_dev, 0, sizeof(int), st));
    rs = reorder_any_run(n, T, ldt, Tr, ldtr, Q, ldq, swaps, ws, s->err_dev, st);
    if (rs != SIGNTRI_OK) return rs;
    SGT_CUDA_TRY(cudaMemcpyAsync(s->err_host, s->err_dev, sizeof(int), cudaMemcpyDeviceToHost, st));
    SGT_CUDA_TRY(cudaStreamSynchronize(st));
    return *s->err_host ? SIGNTRI_ERR_TIMEOUT : SIGNTRI_OK;
}

signtri_status signtri_gemm_emulated(int m, int n, int k, const double *A, int lda, const double *B, int ldb,
                                     double *C, int ldc, void *stream)
{
    if (m < 0 || n < 0 || k < 0) return SIGNTRI_ERR_BAD_ARG;
    if (m == 0 || n == 0) return SIGNTRI_OK;
    if (!A || !B || !C || lda < m || ldb < std::max(k, 1) || ldc < m) return SIGNTRI_ERR_BAD_ARG;
    if (blocks_overlap(A, lda, m, k, C, ldc, m, n) || blocks_overlap(B, ldb, k, n, C, ldc, m, n))
        return SIGNTRI_ERR_BAD_ARG;
    std::lock_guard<std::mutex> lk(g_mu);
    DeviceState *s = nullptr;
    signtri_status rs = current_state(&s);
    if (rs != SIGNTRI_OK) return rs;
    Arena ws;
    rs = get_workspace(*s, emulated_gemm_workspace_bytes(m, n, k, 8), ws);
    if (rs != SIGNTRI_OK) return rs;
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    SGT_CUDA_TRY(cudaMemsetAsync(s->err_dev, 0, sizeof(int), st));
    rs = emulated_gemm_run(m, n, k, A, lda, B, ldb, C, ldc, 8, ws, s->err_dev, st);
    if (rs != SIGNTRI_OK) return rs;
    SGT_CUDA_TRY(cudaMemcpyAsync(s->err_host, s->err_dev, sizeof(int), cudaMemcpyDeviceToHost, st));
    SGT_CUDA_TRY(cudaStreamSynchronize(st));
    return *s->err_host ? SIGNTRI_ERR_TIMEOUT : SIGNTRI_OK;
}

// W = U Q^T (n x n) then S = Q W, after U = sign(T) was written into S
static size_t schur_products_bytes(int n)
{
    return (size_t)n * n * sizeof(double) + 256 + emulated_product_workspace_bytes(n, n, n);
}

size_t signtri_sign_schur_workspace_bytes(int n, signtri_variant v)
{
    if (n < 0 || !valid_variant(v)) return 0;
    std::lock_guard<std::mutex> lk(g_mu);
    return std::max(workspace_need(n, v, -1), schur_products_bytes(n));
}

signtri_status signtri_sign_schur(int n, const double *Q, int ldq, const double *T, int ldt, double *S, int lds,
                                  signtri_variant v, void *stream)
{
    reset_info(n);
    if (n < 0 || !valid_variant(v)) return SIGNTRI_ERR_BAD_ARG;
    if (n == 0) return SIGNTRI_OK;
    if (!Q || !T || !S || ldq < n || ldt < n || lds < n) return SIGNTRI_ERR_BAD_ARG;
    if (blocks_overlap(T, ldt, n, n, S, lds, n, n) || blocks_overlap(Q, ldq, n, n, S, lds, n, n))
        return SIGNTRI_ERR_BAD_ARG;
    std::lock_guard<std::mutex> lk(g_mu);
    DeviceState *s = nullptr;
    signtri_status rs = current_state(&s);
    if (rs != SIGNTRI_OK) return rs;
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    // U = sign(T), held in S until the second product overwrites it
    rs = sign_tri_locked(n, T, ldt, S, lds, v, st, *s);
    if (rs != SIGNTRI_OK) return rs;
    if (g_info.n_neg == 0 || g_info.n_pos == 0) {
        // U = +-I, so S = +-Q Q^T = +-I for orthogonal Q: left exact
        SGT_CUDA_TRY(cudaStreamSynchronize(st));
        return SIGNTRI_OK;
    }
    Arena ws;
    rs = get_workspace(*s, schur_products_bytes(n), ws);
    if (rs != SIGNTRI_OK) return rs;
    double *W = static_cast<double *>(ws.take((size_t)n * n * sizeof(double)));
    if (!W) return SIGNTRI_ERR_NO_WORKSPACE;
    const size_t mark = ws.used;
    SGT_CUDA_TRY(cudaMemsetAsync(s->err_dev, 0, sizeof(int), st));
    rs = emulated_product(n, n, n, S, lds, Q, ldq, true, W, n, false, SIGNTRI_KC_GEMM_F64, ws, s->err_dev, st);
    if (rs != SIGNTRI_OK) return rs;
    ws.used = mark;
    rs = emulated_product(n, n, n, Q, ldq, W, n, false, S, lds, false, SIGNTRI_KC_GEMM_F64, ws, s->err_dev, st);
    if (rs != SIGNTRI_OK) return rs;
    SGT_CUDA_TRY(cudaMemcpyAsync(s->err_host, s->err_dev, sizeof(int), cudaMemcpyDeviceToHost, st));
    SGT_CUDA_TRY(cudaStreamSynchronize(st));
    return *s->err_host ? SIGNTRI_ERR_TIMEOUT : SIGNTRI_OK;
}

size_t signtri_complex_workspace_bytes(int n)
{
    if (n < 0) return 0;
    return complex_schur_workspace_bytes(n);
}

// the complex blocks [A] (rows x cols, ld in complex elements) as double runs
static bool cblocks_overlap(const double *A, int lda, const double *B, int ldb, int n)
{
    return blocks_overlap(A, 2 * lda, 2 * n, n, B, 2 * ldb, 2 * n, n);
}

signtri_status signtri_sign_tri_complex(int n, const double *T, int ldt, double *U, int ldu, void *stream)
{
    reset_info(n);
    if (n < 0) return SIGNTRI_ERR_BAD_ARG;
    if (n == 0) return SIGNTRI_OK;
    if (!T || !U || ldt < n || ldu < n) return SIGNTRI_ERR_BAD_ARG;
    if (cblocks_overlap(T, ldt, U, ldu, n)) return SIGNTRI_ERR_BAD_ARG;
    std::lock_guard<std::mutex> lk(g_mu);
    DeviceState *s = nullptr;
    signtri_status rs = current_state(&s);
    if (rs != SIGNTRI_OK) return rs;
    Arena ws;
    rs = get_workspace(*s, complex_workspace_bytes(n), ws);
    if (rs != SIGNTRI_OK) return rs;
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    int bad = -1;
    rs = complex_sign_run(n, T, ldt, U, ldu, ws, &bad, st);
    if (rs == SIGNTRI_ERR_ZERO_EIGENVALUE || rs == SIGNTRI_ERR_NONFINITE) g_info.bad_index = bad;
    if (rs != SIGNTRI_OK) return rs;
    SGT_CUDA_TRY(cudaStreamSynchronize(st));
    return SIGNTRI_OK;
}

signtri_status signtri_sign_schur_complex(int n, const double *Q, int ldq, const double *T, int ldt, double *S,
                                          int lds, void *stream)
{
    reset_info(n);
    if (n < 0) return SIGNTRI_ERR_BAD_ARG;
    if (n == 0) return SIGNTRI_OK;
    if (!Q || !T || !S || ldq < n || ldt < n || lds < n) return SIGNTRI_ERR_BAD_ARG;
    if (cblocks_overlap(T, ldt, S, lds, n) || cblocks_overlap(Q, ldq, S, lds, n)) return SIGNTRI_ERR_BAD_ARG;
    std::lock_guard<std::mutex> lk(g_mu);
    DeviceState *s = nullptr;
    signtri_status rs = current_state(&s);
    if (rs != SIGNTRI_OK) return rs;
    Arena ws;
    rs = get_workspace(*s, complex_schur_workspace_bytes(n), ws);
    if (rs != SIGNTRI_OK) return rs;
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    SGT_CUDA_TRY(cudaMemsetAsync(s->err_dev, 0, sizeof(int), st));
    int bad = -1;
    rs = complex_schur_run(n, Q, ldq, T, ldt, S, lds, ws, s->err_dev, &bad, st);
    if (rs == SIGNTRI_ERR_ZERO_EIGENVALUE || rs == SIGNTRI_ERR_NONFINITE) g_info.bad_index = bad;
    if (rs != SIGNTRI_OK) return rs;
    SGT_CUDA_TRY(cudaMemcpyAsync(s->err_host, s->err_dev, sizeof(int), cudaMemcpyDeviceToHost, st));
    SGT_CUDA_TRY(cudaStreamSynchronize(st));
    return *s->err_host ? SIGNTRI_ERR_TIMEOUT : SIGNTRI_OK;
}

size_t signtri_schur_workspace_bytes(int n)
{
    if (n < 0) return 0;
    return schur_workspace_bytes(n);
}

size_t signtri_sign_general_workspace_bytes(int n)
{
    if (n < 0) return 0;
    return sign_general_workspace_bytes(n);
}

signtri_status signtri_schur(int n, const double *A, int lda, double *Q, int ldq, double *T, int ldt, void *stream)
{
    reset_info(n);
    if (n < 0) return SIGNTRI_ERR_BAD_ARG;
    if (n == 0) return SIGNTRI_OK;
    if (!A || !Q || !T || lda < n || ldq < n || ldt < n) return SIGNTRI_ERR_BAD_ARG;
    // A's block as doubles against the complex blocks of Q and T
    if (blocks_overlap(A, lda, n, n, Q, 2 * ldq, 2 * n, n) || blocks_overlap(A, lda, n, n, T, 2 * ldt, 2 * n, n) ||
        cblocks_overlap(Q, ldq, T, ldt, n))
        return SIGNTRI_ERR_BAD_ARG;
    std::lock_guard<std::mutex> lk(g_mu);
    DeviceState *s = nullptr;
    signtri_status rs = current_state(&s);
    if (rs != SIGNTRI_OK) return rs;
    Arena ws;
    rs = get_workspace(*s, schur_workspace_bytes(n), ws);
    if (rs != SIGNTRI_OK) return rs;
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    int bad = -1;
    long long counts[2] = {0, 0};
    rs = schur_run(n, A, lda, Q, ldq, T, ldt, ws, &bad, counts, st);
    g_info.qr_sweeps = counts[0];
    g_info.qr_rotations = counts[1];
    if (rs == SIGNTRI_ERR_NONFINITE) g_info.bad_index = bad;
    if (rs != SIGNTRI_OK) return rs;
    SGT_CUDA_TRY(cudaStreamSynchronize(st));
    return SIGNTRI_OK;
}

signtri_status signtri_sign_general(int n, const double *A, int lda, double *S, int lds, void *stream)
{
    reset_info(n);
    if (n < 0) return SIGNTRI_ERR_BAD_ARG;
    if (n == 0) return SIGNTRI_OK;
    if (!A || !S || lda < n || lds < n) return SIGNTRI_ERR_BAD_ARG;
    if (blocks_overlap(A, lda, n, n, S, lds, n, n)) return SIGNTRI_ERR_BAD_ARG;
    std::lock_guard<std::mutex> lk(g_mu);
    DeviceState *s = nullptr;
    signtri_status rs = current_state(&s);
    if (rs != SIGNTRI_OK) return rs;
    Arena ws;
    rs = get_workspace(*s, sign_general_workspace_bytes(n), ws);
    if (rs != SIGNTRI_OK) return rs;
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    SGT_CUDA_TRY(cudaMemsetAsync(s->err_dev, 0, sizeof(int), st));
    int bad = -1;
    long long counts[2] = {0, 0};
    rs = sign_general_run(n, A, lda, S, lds, ws, s->err_dev, &bad, counts, st);
    g_info.qr_sweeps = counts[0];
    g_info.qr_rotations = counts[1];
    if (rs == SIGNTRI_ERR_ZERO_EIGENVALUE || rs == SIGNTRI_ERR_NONFINITE) g_info.bad_index = bad;
    if (rs != SIGNTRI_OK) return rs;
    SGT_CUDA_TRY(cudaMemcpyAsync(s->err_host, s->err_dev, sizeof(int), cudaMemcpyDeviceToHost, st));
    SGT_CUDA_TRY(cudaStreamSynchronize(st));
    return *s->err_host ? SIGNTRI_ERR_TIMEOUT : SIGNTRI_OK;
}

signtri_status signtri_funm(int n, const double *T, int ldt, double *F, int ldf, signtri_phi phi, void *stream)
{
    reset_info(n);
    if (n < 0 || phi < SIGNTRI_PHI_EXP || phi > SIGNTRI_PHI_SIGN) return SIGNTRI_ERR_BAD_ARG;
    if (n == 0) return SIGNTRI_OK;
    if (!T || !F || ldt < n || ldf < n) return SIGNTRI_ERR_BAD_ARG;
    if (blocks_overlap(T, ldt, n, n, F, ldf, n, n)) return SIGNTRI_ERR_BAD_ARG;
    std::lock_guard<std::mutex> lk(g_mu);
    DeviceState *s = nullptr;
    signtri_status rs = current_state(&s);
    if (rs != SIGNTRI_OK) return rs;
    const int b = cutoff_of(n, SIGNTRI_PH_FP64);
    Arena ws;
    rs = get_workspace(*s, funm_workspace_bytes(n, b), ws);
    if (rs != SIGNTRI_OK) return rs;
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    int bad = -1;
    rs = funm_run(n, T, ldt, F, ldf, (int)phi, b, ws, &bad, st);
    g_info.cutoff = b;
    if (rs == SIGNTRI_ERR_DOMAIN) g_info.bad_index = bad;
    if (rs != SIGNTRI_OK) return rs;
    SGT_CUDA_TRY(cudaStreamSynchronize(st));
    return SIGNTRI_OK;
}

signtri_status signtri_sylvester(int m, int p, const double *A, int lda, const double *B, int ldb, const double *C,
                                 int ldc, double *X, int ldx, void *stream)
{
    if (m < 0 || p < 0) return SIGNTRI_ERR_BAD_ARG;
    if (m == 0 || p == 0) return SIGNTRI_OK;
    if (!A || !B || !C || !X || lda < m || ldb < p || ldc < m || ldx < m) return SIGNTRI_ERR_BAD_ARG;
    if (blocks_overlap(A, lda, m, m, X, ldx, m, p) || blocks_overlap(B, ldb, p, p, X, ldx, m, p) ||
        blocks_overlap(C, ldc, m, p, X, ldx, m, p))
        return SIGNTRI_ERR_BAD_ARG;
    std::lock_guard<std::mutex> lk(g_mu);
    DeviceState *s = nullptr;
    signtri_status rs = current_state(&s);
    if (rs != SIGNTRI_OK) return rs;
    Arena ws;
    rs = get_workspace(*s, sylvester_workspace_bytes(m, p), ws);
    if (rs != SIGNTRI_OK) return rs;
    return sylvester_run(m, p, A, lda, B, ldb, C, ldc, 1.0, X, ldx, ws, static_cast<cudaStream_t>(stream));
}

signtri_status signtri_set_workspace(void *dev_ptr, size_t bytes)
{
    if (dev_ptr && ((uintptr_t)dev_ptr % 256) != 0) return SIGNTRI_ERR_BAD_ARG;
    std::lock_guard<std::mutex> lk(g_mu);
    DeviceState *s = nullptr;
    signtri_status rs = current_state(&s);
    if (rs != SIGNTRI_OK) return rs;
    s->user_ptr = dev_ptr;
    s->user_bytes = dev_ptr ? bytes : 0;
    return SIGNTRI_OK;
}

signtri_status signtri_set_cutoff(int b)
{
    if (b != 0 && b != 16 && b != 32 && b != 64) return SIGNTRI_ERR_BAD_ARG;
    std::lock_guard<std::mutex> lk(g_mu);
    g_cutoff = b;
    return SIGNTRI_OK;
}

signtri_status sign_tri(int n, const double *T, int ldt, double *U, int ldu, signtri_variant v,
                        void *stream)
{
    reset_info(n);
    if (n < 0 || !valid_variant(v)) return SIGNTRI_ERR_BAD_ARG;
    if (n == 0) return SIGNTRI_OK;
    if (!T || !U || ldt < n || ldu < n) return SIGNTRI_ERR_BAD_ARG;
    if (blocks_overlap(T, ldt, n, n, U, ldu, n, n)) return SIGNTRI_ERR_BAD_ARG;
    std::lock_guard<std::mutex> lk(g_mu);
    DeviceState *s = nullptr;
    signtri_status rs = current_state(&s);
    if (rs != SIGNTRI_OK) return rs;
    return sign_tri_locked(n, T, ldt, U, ldu, v, static_cast<cudaStream_t>(stream), *s);
}

signtri_status sign_tri_host(int n, const double *T_host, int ldt, double *U_host, int ldu,
                             signtri_variant v, void *stream)
{
    reset_info(n);
    if (n < 0 || !valid_variant(v)) return SIGNTRI_ERR_BAD_ARG;
    if (n == 0) return SIGNTRI_OK;
    if (!T_host || !U_host || ldt < n || ldu < n) return SIGNTRI_ERR_BAD_ARG;
    std::lock_guard<std::mutex> lk(g_mu);
    DeviceState *s = nullptr;
    signtri_status rs = current_state(&s);
    if (rs != SIGNTRI_OK) return rs;
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    const size_t elems = (size_t)n * n;
    if (s->stage_elems < elems) {
        SGT_CUDA_TRY(cudaStreamSynchronize(st));
        cudaFree(s->stage_T);
        cudaFree(s->stage_U);
        s->stage_T = s->stage_U = nullptr;
        s->stage_elems = 0;
        if (cudaMalloc(&s->stage_T, elems * sizeof(double)) != cudaSuccess ||
            cudaMalloc(&s->stage_U, elems * sizeof(double)) != cudaSuccess) {
            cudaGetLastError();
            return SIGNTRI_ERR_NO_WORKSPACE;
        }
        s->stage_elems = elems;
    }
    // only T's upper triangle is read: copy it by column panels, each from
    // row 0 to its last column's diagonal (about half of T's bytes)
    constexpr int kPanel = 128;
    {
        ProfScope ps(SIGNTRI_KC_HOST_COPY, st);
        for (int j0 = 0; j0 < n; j0 += kPanel) {
            const int cols = std::min(kPanel, n - j0), rows = std::min(n, j0 + kPanel);
            SGT_CUDA_TRY(cudaMemcpy2DAsync(s->stage_T + (size_t)j0 * n, (size_t)n * sizeof(double),
                                           T_host + (size_t)j0 * ldt, (size_t)ldt * sizeof(double),
                                           (size_t)rows * sizeof(double), cols, cudaMemcpyHostToDevice, st));
        }
    }
    rs = sign_tri_locked(n, s->stage_T, n, s->stage_U, n, v, st, *s);
    if (rs != SIGNTRI_OK) {
        // no copy from the caller's T_host may still be in flight on return
        cudaStreamSynchronize(st);
        return rs;
    }
    {
        ProfScope ps(SIGNTRI_KC_HOST_COPY, st);
        SGT_CUDA_TRY(cudaMemcpy2DAsync(U_host, (size_t)ldu * sizeof(double), s->stage_U, (size_t)n * sizeof(double),
                                       (size_t)n * sizeof(double), n, cudaMemcpyDeviceToHost, st));
    }
    SGT_CUDA_TRY(cudaStreamSynchronize(st));
    return SIGNTRI_OK;
}

signtri_status signtri_inertia(int n, const double *T, int ldt, int *n_pos, int *n_neg, long long *swaps,
                               void *stream)
{
    if (n < 0 || (n > 0 && (!T || ldt < n))) return SIGNTRI_ERR_BAD_ARG;
    if (n == 0) {
        if (n_pos) *n_pos = 0;
        if (n_neg) *n_neg = 0;
        if (swaps) *swaps = 0;
        return SIGNTRI_OK;
    }
    std::lock_guard<std::mutex> lk(g_mu);
    DeviceState *s = nullptr;
    signtri_status rs = current_state(&s);
    if (rs != SIGNTRI_OK) return rs;
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    rs = launch_inertia_scan(n, T, ldt, s->scan_dev, st);
    if (rs != SIGNTRI_OK) return rs;
    SGT_CUDA_TRY(cudaMemcpyAsync(s->scan_host, s->scan_dev, sizeof(ScanResult), cudaMemcpyDeviceToHost, st));
    SGT_CUDA_TRY(cudaStreamSynchronize(st));
    const ScanResult r = *s->scan_host;
    if (n_pos) *n_pos = r.n_pos;
    if (n_neg) *n_neg = r.n_neg;
    if (swaps) *swaps = r.swaps;
    if (r.bad_key != INT_MAX) return (signtri_status)(r.bad_key % 4);
    return SIGNTRI_OK;
}

signtri_status signtri_get_info(signtri_info *out)
{
    if (!out) return SIGNTRI_ERR_BAD_ARG;
    *out = g_info;
    return SIGNTRI_OK;
}

}  // extern "C"

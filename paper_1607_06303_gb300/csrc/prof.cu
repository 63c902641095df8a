// prof.cu -- per-kernel-class launch counts and device time.
//
// When enabled, every library launch is bracketed by two CUDA events recorded
// on the stream the kernel is launched on; signtri_profile_read waits for
// them and sums the elapsed time per kernel class.  Launch counts are kept
// whether or not timing is enabled.  Also holds the float64 issue-rate probe
// used as the FP64 roofline denominator.
#include <mutex>
#include <vector>

#include "internal.cuh"

namespace signtri {

namespace {

struct Pending {
    int cls;
    cudaEvent_t a, b;
};

std::mutex p_mu;
bool p_enabled = false;
long long p_launches[SIGNTRI_KC_COUNT] = {};
double p_ms[SIGNTRI_KC_COUNT] = {};
double p_flops[SIGNTRI_KC_COUNT] = {};
double p_bytes[SIGNTRI_KC_COUNT] = {};
std::vector<Pending> p_pending;
std::vector<cudaEvent_t> p_free;
thread_local int p_open_cls = -1;
thread_local cudaEvent_t p_open_ev = nullptr;

cudaEvent_t take_event()
{
    if (!p_free.empty()) {
        cudaEvent_t e = p_free.back();
        p_free.pop_back();
        return e;
    }
    cudaEvent_t e = nullptr;
    if (cudaEventCreate(&e) != cudaSuccess) return nullptr;
    return e;
}

const char *kClassNames[SIGNTRI_KC_COUNT] = {
    "inertia_scan", "fill", "diag_leaf_f64", "block_sums_f64", "offdiag_leaf_f64",
    "block_sums_tc", "offdiag_leaf_mixed", "convert", "residual", "correction",
    "givens_rounds", "sylvester_sums", "sylvester_leaf", "gemm_f64", "other", "residual_sum", "batch_graph", "schur",
    "hessenberg", "host_copies",
};

bool p_paused = false;

}  // namespace

void prof_pause(bool on)
{
    std::lock_guard<std::mutex> lk(p_mu);
    p_paused = on;
}

void prof_count(int cls, long long launches)
{
    std::lock_guard<std::mutex> lk(p_mu);
    if (cls >= 0 && cls < SIGNTRI_KC_COUNT) p_launches[cls] += launches;
}

void prof_begin(int cls, cudaStream_t st, bool count)
{
    std::lock_guard<std::mutex> lk(p_mu);
    if (count) p_launches[cls]++;
    if (!p_enabled || p_paused) return;
    p_open_cls = cls;
    p_open_ev = take_event();
    if (p_open_ev) cudaEventRecord(p_open_ev, st);
}

void prof_add_flops(int cls, double flops)
{
    std::lock_guard<std::mutex> lk(p_mu);
    if (cls >= 0 && cls < SIGNTRI_KC_COUNT) p_flops[cls] += flops;
}

void prof_add_bytes(int cls, double bytes)
{
    std::lock_guard<std::mutex> lk(p_mu);
    if (cls >= 0 && cls < SIGNTRI_KC_COUNT) p_bytes[cls] += bytes;
}

void prof_end(int cls, cudaStream_t st)
{
    std::lock_guard<std::mutex> lk(p_mu);
    if (!p_enabled || p_paused || p_open_cls != cls || !p_open_ev) return;
    cudaEvent_t b = take_event();
    if (b) {
        cudaEventRecord(b, st);
        p_pending.push_back({cls, p_open_ev, b});
    } else {
        p_free.push_back(p_open_ev);
    }
    p_open_cls = -1;
    p_open_ev = nullptr;
}

namespace {

// Independent fused multiply-add chains: 8 per thread, `iters` rounds.
__global__ void fp64_probe_kernel(double *out, int iters, double a, double b)
{
    double r[8];
#pragma unroll
    for (int i = 0; i < 8; i++) r[i] = threadIdx.x * 1e-3 + i;
    for (int it = 0; it < iters; it++) {
#pragma unroll
        for (int i = 0; i < 8; i++) r[i] = fma(r[i], a, b);
    }
    double s = 0.0;
#pragma unroll
    for (int i = 0; i < 8; i++) s += r[i];
    out[blockIdx.x * blockDim.x + threadIdx.x] = s;
}

}  // namespace

}  // namespace signtri

using namespace signtri;

extern "C" {

signtri_status signtri_profile_enable(int on)
{
    std::lock_guard<std::mutex> lk(p_mu);
    p_enabled = (on != 0);
    return SIGNTRI_OK;
}

signtri_status signtri_profile_reset(void)
{
    std::lock_guard<std::mutex> lk(p_mu);
    for (auto &p : p_pending) { p_free.push_back(p.a); p_free.push_back(p.b); }
    p_pending.clear();
    for (int i = 0; i < SIGNTRI_KC_COUNT; i++) { p_launches[i] = 0; p_ms[i] = 0.0; p_flops[i] = 0.0; p_bytes[i] = 0.0; }
    return SIGNTRI_OK;
}

signtri_status signtri_profile_read(int cls, long long *launches, double *device_ms)
{
    if (cls < 0 || cls >= SIGNTRI_KC_COUNT) return SIGNTRI_ERR_BAD_ARG;
    std::lock_guard<std::mutex> lk(p_mu);
    for (auto &p : p_pending) {
        if (cudaEventSynchronize(p.b) != cudaSuccess) return SIGNTRI_ERR_CUDA;
        float ms = 0.f;
        if (cudaEventElapsedTime(&ms, p.a, p.b) != cudaSuccess) return SIGNTRI_ERR_CUDA;
        p_ms[p.cls] += ms;
        p_free.push_back(p.a);
        p_free.push_back(p.b);
    }
    p_pending.clear();
    if (launches) *launches = p_launches[cls];
    if (device_ms) *device_ms = p_ms[cls];
    return SIGNTRI_OK;
}

signtri_status signtri_profile_read_flops(int cls, double *flops)
{
    if (cls < 0 || cls >= SIGNTRI_KC_COUNT || !flops) return SIGNTRI_ERR_BAD_ARG;
    std::lock_guard<std::mutex> lk(p_mu);
    *flops = p_flops[cls];
    return SIGNTRI_OK;
}

signtri_status signtri_profile_read_bytes(int cls, double *bytes)
{
    if (cls < 0 || cls >= SIGNTRI_KC_COUNT || !bytes) return SIGNTRI_ERR_BAD_ARG;
    std::lock_guard<std::mutex> lk(p_mu);
    *bytes = p_bytes[cls];
    return SIGNTRI_OK;
}

const char *signtri_kernel_class_name(int cls)
{
    if (cls < 0 || cls >= SIGNTRI_KC_COUNT) return "";
    return kClassNames[cls];
}

signtri_status signtri_probe_fp64_peak(double *gflops, void *stream)
{
    if (!gflops) return SIGNTRI_ERR_BAD_ARG;
    int dev = 0, sms = 0;
    SGT_CUDA_TRY(cudaGetDevice(&dev));
    SGT_CUDA_TRY(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    const int threads = 512, blocks = 4 * sms, iters = 20000;
    double *buf = nullptr;
    SGT_CUDA_TRY(cudaMalloc(&buf, sizeof(double) * threads * blocks));
    cudaEvent_t a = nullptr, b = nullptr;
    signtri_status rs = SIGNTRI_OK;
    float best = 1e30f;
    if (cudaEventCreate(&a) != cudaSuccess || cudaEventCreate(&b) != cudaSuccess) rs = SIGNTRI_ERR_CUDA;
    for (int rep = 0; rep < 3 && rs == SIGNTRI_OK; rep++) {
        cudaEventRecord(a, st);
        fp64_probe_kernel<<<blocks, threads, 0, st>>>(buf, iters, 0.999999, 1e-7);
        cudaEventRecord(b, st);
        if (cudaEventSynchronize(b) != cudaSuccess) { rs = SIGNTRI_ERR_CUDA; break; }
        float ms = 0.f;
        cudaEventElapsedTime(&ms, a, b);
        if (ms < best) best = ms;
    }
    if (rs == SIGNTRI_OK && cudaGetLastError() != cudaSuccess) rs = SIGNTRI_ERR_CUDA;
    if (rs == SIGNTRI_OK) *gflops = 2.0 * 8.0 * iters * (double)threads * blocks / (best * 1e6);
    if (a) cudaEventDestroy(a);
    if (b) cudaEventDestroy(b);
    cudaFree(buf);
    return rs;
}

}  // extern "C"

// noalloc.cu -- sign_tri_noalloc: the float64 Parlett-Higham path with its
// scratch in a file-scope device array instead of allocated workspace.
//
// For callers that cannot allocate device memory: code running inside a host
// program that owns all device memory through its own pool (a serving
// runtime or a plugin), where a raw cudaMalloc would bypass the owner's
// accounting or fail because the pool already holds the memory, and code
// that must not stall the device (cudaMalloc and cudaFree can synchronize
// it).  The scratch array is part of the library's device image: every GPU
// that loads the library holds it until the process exits.
#include <mutex>

#include "internal.cuh"
#include "ph_bodies.cuh"

namespace signtri {

namespace {

constexpr int kNoallocMaxN = 1024;
// The first 256 bytes hold the scan result; the rest is the float64 path's
// block-sum slabs.  Their size grows with n, so n = 1024 bounds every smaller
// problem; at n = 1024 the cutoffs need 15.7 MB (b = 64: 240 slabs of 64 x 64
// doubles per set), 8.4 MB (b = 32: 512 slabs) and 2.8 MB (b = 16: 672), two
// sets each.  The array is sized from that bound, checked at compile time.
constexpr size_t kScanSlot = 256;
constexpr size_t noalloc_need()
{
    size_t m = 0;
    for (int b = 16; b <= 64; b *= 2)
        if (ph::mm_form_workspace_bytes(kNoallocMaxN, b) > m) m = ph::mm_form_workspace_bytes(kNoallocMaxN, b);
    return m;
}
constexpr size_t kNoallocBytes = ((kScanSlot + noalloc_need() + 4095) / 4096) * 4096;
static_assert(ph::mm_form_workspace_bytes(kNoallocMaxN, 64) <= kNoallocBytes - kScanSlot, "b = 64 at the maximum n");
static_assert(ph::mm_form_workspace_bytes(kNoallocMaxN, 32) <= kNoallocBytes - kScanSlot, "b = 32 at the maximum n");
static_assert(ph::mm_form_workspace_bytes(kNoallocMaxN, 16) <= kNoallocBytes - kScanSlot, "b = 16 at the maximum n");
static_assert(kNoallocBytes <= ((size_t)16 << 20), "the array stays modest");

__device__ __align__(256) unsigned char g_noalloc_scratch[kNoallocBytes];

std::mutex na_mu;
char *na_base[64] = {};   // device address of g_noalloc_scratch, per device

}  // namespace

}  // namespace signtri

using namespace signtri;

extern "C" signtri_status sign_tri_noalloc(int n, const double *T, int ldt, double *U, int ldu, void *stream)
{
    if (n < 0) return SIGNTRI_ERR_BAD_ARG;
    if (n == 0) return SIGNTRI_OK;
    if (!T || !U || ldt < n || ldu < n) return SIGNTRI_ERR_BAD_ARG;
    if (blocks_overlap(T, ldt, n, n, U, ldu, n, n)) return SIGNTRI_ERR_BAD_ARG;
    if (n > kNoallocMaxN) return SIGNTRI_ERR_NO_WORKSPACE;
    int dev = 0;
    SGT_CUDA_TRY(cudaGetDevice(&dev));
    if (dev < 0 || dev >= 64) return SIGNTRI_ERR_CUDA;
    std::lock_guard<std::mutex> lk(na_mu);
    if (!na_base[dev]) {
        // once per device, with that device current: the host-side symbol is
        // only a stand-in, the kernels need the device address.  The address
        // is kept for the life of the process, so the device must not be
        // reset (cudaDeviceReset) between calls: a reset unloads the module
        // and a reloaded one may place the array elsewhere
        void *p = nullptr;
        cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
        if (e != cudaSuccess || p == nullptr) return SIGNTRI_ERR_CUDA;
        na_base[dev] = static_cast<char *>(p);
    }
    const int b = current_cutoff(n);
    Arena ws;
    ws.base = na_base[dev] + kScanSlot;
    ws.bytes = kNoallocBytes - kScanSlot;
    if (ph_fp64_workspace_bytes(n, b) > ws.bytes) return SIGNTRI_ERR_NO_WORKSPACE;
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    ScanResult *scan_dev = reinterpret_cast<ScanResult *>(na_base[dev]);
    signtri_status rs = launch_inertia_scan(n, T, ldt, scan_dev, st);
    if (rs != SIGNTRI_OK) return rs;
    ScanResult r;
    SGT_CUDA_TRY(cudaMemcpyAsync(&r, scan_dev, sizeof(ScanResult), cudaMemcpyDeviceToHost, st));
    SGT_CUDA_TRY(cudaStreamSynchronize(st));
    if (r.bad_key != INT_MAX) return (signtri_status)(r.bad_key % 4);
    if (r.n_neg == 0 || r.n_pos == 0) return launch_fill_identity(n, U, ldu, r.n_neg == 0 ? 1.0 : -1.0, st);
    // the block-sum slabs are fully written before they are read on every
    // anti-diagonal, so nothing left by an earlier call needs clearing
    return ph_fp64_run(n, T, ldt, U, ldu, b, ws, st);
}

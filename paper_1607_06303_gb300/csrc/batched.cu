// batched.cu -- many independent sign(T) problems of uneven size, float64
// Parlett-Higham, in one CUDA graph.
//
// Level-synchronous batch schedule: block anti-diagonal d of every matrix
// depends only on smaller anti-diagonals of the same matrix, so for each d
// one block-sum launch covers the tiles (and K-splits) of anti-diagonal d of
// all matrices with more than d blocks, and one leaf launch finishes them.
// Per-CTA work tables (matrix, tile, K range, partial-sum slot) are built on
// the host, and the 2 (nb_max - 1) launches of a cutoff group captured into
// one CUDA graph, once per group shape: a later call with the same group
// (sizes, members, buffers) launches the instantiated graph again.  Matrices
// are grouped by leaf size (from the cutoff table) because the kernels are
// specialised on it.
#include <algorithm>
#include <vector>

#include "internal.cuh"
#include "ph_bodies.cuh"
#include "batched_plan.h"

namespace signtri {

using namespace ph;

namespace {

static_assert(kBatchSplitMax == kSplitMax && kBatchTargetCtas == kTargetCtas,
              "the batched plan and the float64 kernels share their split limits");

template <int B>
__global__ void __launch_bounds__(kThreads)
batched_diag_kernel(const BatchDesc *__restrict__ mats, const int *__restrict__ members,
                    const DiagTask *__restrict__ tasks)
{
    const DiagTask t = tasks[blockIdx.x];
    const BatchDesc M = mats[members[t.m]];
    diag_leaf_body<B>(M.n, M.T, M.ldt, M.U, M.ldu, t.blk);
}

template <int B>
__global__ void __launch_bounds__(kThreads)
batched_gemm_kernel(const BatchDesc *__restrict__ mats, const int *__restrict__ members,
                    const GemmTask *__restrict__ tasks, double *__restrict__ PX, double *__restrict__ PY)
{
    const GemmTask t = tasks[blockIdx.x];
    const BatchDesc M = mats[members[t.m]];
    ph_gemm_body<B>(M.n, M.T, M.ldt, M.U, M.ldu, t.I, t.J, t.kb0 * B, t.kb1 * B, PX + (size_t)t.slot * B * B,
                    PY + (size_t)t.slot * B * B);
}

// arithmetic-efficient form: per-matrix sign permutations at perm + poff[m],
// positive counts at npos + noff[m]
template <int B>
__global__ void __launch_bounds__(kThreads)
batched_gemm_split_kernel(const BatchDesc *__restrict__ mats, const int *__restrict__ members,
                          const GemmTask *__restrict__ tasks, const short *__restrict__ perm,
                          const int *__restrict__ npos, const int *__restrict__ poff, const int *__restrict__ noff,
                          double *__restrict__ PZ)
{
    const GemmTask t = tasks[blockIdx.x];
    const BatchDesc M = mats[members[t.m]];
    ph_gemm_split_body<B>(M.n, M.T, M.ldt, M.U, M.ldu, t.I, t.J, t.kb0 * B, t.kb1 * B, perm + poff[t.m],
                          npos + noff[t.m], PZ + (size_t)t.slot * B * B);
}

template <int B>
__global__ void batched_perm_kernel(const BatchDesc *__restrict__ mats, const int *__restrict__ members,
                                    const DiagTask *__restrict__ tasks, short *__restrict__ perm,
                                    int *__restrict__ npos, const int *__restrict__ poff, const int *__restrict__ noff)
{
    const DiagTask t = tasks[blockIdx.x];
    const BatchDesc M = mats[members[t.m]];
    sign_perm_body<B>(M.n, M.T, M.ldt, t.blk, perm + poff[t.m], npos + noff[t.m]);
}

template <int B>
__global__ void __launch_bounds__(kThreads)
batched_leaf_kernel(const BatchDesc *__restrict__ mats, const int *__restrict__ members,
                    const LeafTask *__restrict__ tasks, const double *__restrict__ PX, const double *__restrict__ PY)
{
    const LeafTask t = tasks[blockIdx.x];
    const BatchDesc M = mats[members[t.m]];
    offdiag_leaf_body<B>(M.n, M.T, M.ldt, M.U, M.ldu, t.I, t.J, t.nsplit, PX + (size_t)t.slot0 * B * B,
                         PY + (size_t)t.slot0 * B * B, (size_t)B * B);
}

// A group's device task tables and instantiated graph, kept for the next
// call that runs the same group: same leaf size and form, same member sizes
// and indices, and the same descriptor array and partial-slab addresses
// (the graph's kernels take those pointers; the descriptors themselves are
// rewritten by every call and read when the graph runs).  The tables live in
// memory of their own, since other calls reuse the workspace.
struct GroupCache {
    bool valid = false;
    bool split = false;
    std::vector<int> ns, members;
    const BatchDesc *d_mats = nullptr;
    double *PX = nullptr;
    size_t max_slots = 0;
    void *tables = nullptr;
    cudaGraphExec_t exec = nullptr;
    cudaStream_t capture = nullptr;
    long long kernels[3] = {};   // kernels in the graph: diagonal leaves, block sums, leaves
    long long hits = 0, builds = 0;
};
constexpr int kCacheDevices = 64;
GroupCache g_cache[kCacheDevices][3];   // per device and leaf size 16, 32, 64

void cache_drop(GroupCache &gc)
{
    if (gc.exec) cudaGraphExecDestroy(gc.exec);
    if (gc.tables) cudaFree(gc.tables);
    gc.exec = nullptr;
    gc.tables = nullptr;
    gc.valid = false;
}

template <int B>
signtri_status run_group(const BatchDesc *d_mats, const std::vector<int> &members, const std::vector<int> &ns,
                         bool split, Arena &ws, cudaStream_t st)
{
    int dev = 0;
    SGT_CUDA_TRY(cudaGetDevice(&dev));
    if (dev < 0 || dev >= kCacheDevices) return SIGNTRI_ERR_CUDA;
    GroupCache &gc = g_cache[dev][B == 16 ? 0 : (B == 32 ? 1 : 2)];
    const bool same_shape = gc.valid && gc.split == split && gc.ns == ns && gc.members == members &&
                            gc.d_mats == d_mats;
    Plan p;
    if (!same_shape) make_plan(ns, B, p);
    const size_t slots = std::max<size_t>(same_shape ? gc.max_slots : p.max_slots, 1);
    // the partial slabs come first from the workspace, so a group of the same
    // shape finds them at the same address
    double *PX = static_cast<double *>(ws.take(slots * B * B * sizeof(double)));
    // the efficient form keeps one sum per entry: X and Y share the slabs
    double *PY = split ? PX : static_cast<double *>(ws.take(slots * B * B * sizeof(double)));
    if (!PX || !PY) return SIGNTRI_ERR_NO_WORKSPACE;
    if (same_shape && gc.PX == PX) {
        gc.hits++;
        // the graph's kernels are counted (not timed) as if launched one by one
        prof_count(SIGNTRI_KC_DIAG_LEAF, gc.kernels[0]);
        prof_count(SIGNTRI_KC_BLOCK_SUMS_F64, gc.kernels[1]);
        prof_count(SIGNTRI_KC_OFFDIAG_LEAF, gc.kernels[2]);
        ProfScope ps(SIGNTRI_KC_BATCH_GRAPH, st);
        SGT_CUDA_TRY(cudaGraphLaunch(gc.exec, st));
        return SIGNTRI_OK;
    }
    if (same_shape) make_plan(ns, B, p);   // same shape, moved workspace: rebuild
    cache_drop(gc);
    // tables: members, diagonal / block-sum / leaf tasks, sign permutations
    // and their offsets, each 256-byte aligned
    auto al = [](size_t b) { return (b + 255) & ~(size_t)255; };
    const size_t b_mem = al(members.size() * sizeof(int)), b_diag = al(std::max<size_t>(p.diag.size(), 1) * sizeof(DiagTask));
    const size_t b_gemm = al(std::max<size_t>(p.gemm.size(), 1) * sizeof(GemmTask));
    const size_t b_leaf = al(std::max<size_t>(p.leaf.size(), 1) * sizeof(LeafTask));
    const size_t b_perm = split ? al(std::max<size_t>(p.perm_len, 1) * sizeof(short)) : 0;
    const size_t b_npos = split ? al(std::max<size_t>(p.npos_len, 1) * sizeof(int)) : 0;
    const size_t b_off = split ? 2 * al(p.poff.size() * sizeof(int)) : 0;
    char *tb = nullptr;
    if (cudaMalloc(&tb, b_mem + b_diag + b_gemm + b_leaf + b_perm + b_npos + b_off) != cudaSuccess) {
        cudaGetLastError();
        return SIGNTRI_ERR_NO_WORKSPACE;
    }
    gc.tables = tb;
    int *d_members = reinterpret_cast<int *>(tb);
    auto *d_diag = reinterpret_cast<DiagTask *>(tb + b_mem);
    auto *d_gemm = reinterpret_cast<GemmTask *>(tb + b_mem + b_diag);
    auto *d_leaf = reinterpret_cast<LeafTask *>(tb + b_mem + b_diag + b_gemm);
    char *rest = tb + b_mem + b_diag + b_gemm + b_leaf;
    short *d_perm = nullptr;
    int *d_npos = nullptr, *d_poff = nullptr, *d_noff = nullptr;
    if (split) {
        d_perm = reinterpret_cast<short *>(rest);
        d_npos = reinterpret_cast<int *>(rest + b_perm);
        d_poff = reinterpret_cast<int *>(rest + b_perm + b_npos);
        d_noff = reinterpret_cast<int *>(rest + b_perm + b_npos + b_off / 2);
        SGT_CUDA_TRY(cudaMemcpyAsync(d_poff, p.poff.data(), p.poff.size() * sizeof(int), cudaMemcpyHostToDevice, st));
        SGT_CUDA_TRY(cudaMemcpyAsync(d_noff, p.noff.data(), p.noff.size() * sizeof(int), cudaMemcpyHostToDevice, st));
    }
    SGT_CUDA_TRY(cudaMemcpyAsync(d_members, members.data(), members.size() * sizeof(int), cudaMemcpyHostToDevice, st));
    SGT_CUDA_TRY(cudaMemcpyAsync(d_diag, p.diag.data(), p.diag.size() * sizeof(DiagTask), cudaMemcpyHostToDevice, st));
    if (!p.gemm.empty())
        SGT_CUDA_TRY(cudaMemcpyAsync(d_gemm, p.gemm.data(), p.gemm.size() * sizeof(GemmTask), cudaMemcpyHostToDevice, st));
    if (!p.leaf.empty())
        SGT_CUDA_TRY(cudaMemcpyAsync(d_leaf, p.leaf.data(), p.leaf.size() * sizeof(LeafTask), cudaMemcpyHostToDevice, st));
    // the host tables are pageable and local
    SGT_CUDA_TRY(cudaStreamSynchronize(st));
    SGT_CUDA_TRY(cudaFuncSetAttribute(batched_leaf_kernel<B>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                      (int)leaf_smem<B>()));
    SGT_CUDA_TRY(cudaFuncSetAttribute(batched_diag_kernel<B>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                      (int)diag_smem<B>()));
    // the level loop, captured into one graph on a private stream
    if (!gc.capture) {
        cudaStream_t cs = nullptr;
        SGT_CUDA_TRY(cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking));
        gc.capture = cs;
    }
    cudaStream_t cs = gc.capture;
    cudaGraph_t graph = nullptr;
    signtri_status rs = SIGNTRI_OK;
    if (cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal) != cudaSuccess) rs = SIGNTRI_ERR_CUDA;
    long long nk[3] = {0, 0, 0};
    if (rs == SIGNTRI_OK) {
        prof_pause(true);
        if (split) {
            batched_perm_kernel<B><<<(unsigned)p.diag.size(), B, 0, cs>>>(d_mats, d_members, d_diag, d_perm, d_npos,
                                                                          d_poff, d_noff);
            nk[0]++;
        }
        batched_diag_kernel<B><<<(unsigned)p.diag.size(), kThreads, diag_smem<B>(), cs>>>(d_mats, d_members, d_diag);
        nk[0]++;
        for (int d = 1; d < p.nbmax; d++) {
            const int g0 = p.gemm_off[d], g1 = p.gemm_off[d + 1];
            const int l0 = p.leaf_off[d], l1 = p.leaf_off[d + 1];
            if (g1 > g0) {
                if (split)
                    batched_gemm_split_kernel<B><<<g1 - g0, kThreads, 0, cs>>>(d_mats, d_members, d_gemm + g0, d_perm,
                                                                               d_npos, d_poff, d_noff, PX);
                else
                    batched_gemm_kernel<B><<<g1 - g0, kThreads, 0, cs>>>(d_mats, d_members, d_gemm + g0, PX, PY);
                nk[1]++;
            }
            if (l1 > l0) {
                batched_leaf_kernel<B><<<l1 - l0, kThreads, leaf_smem<B>(), cs>>>(d_mats, d_members, d_leaf + l0, PX,
                                                                                 PY);
                nk[2]++;
            }
        }
        prof_pause(false);
        if (cudaStreamEndCapture(cs, &graph) != cudaSuccess) rs = SIGNTRI_ERR_CUDA;
    }
    cudaGraphExec_t exec = nullptr;
    if (rs == SIGNTRI_OK && cudaGraphInstantiate(&exec, graph, 0) != cudaSuccess) rs = SIGNTRI_ERR_CUDA;
    if (graph) cudaGraphDestroy(graph);
    if (rs != SIGNTRI_OK) {
        cache_drop(gc);
        return rs;
    }
    gc.exec = exec;
    gc.valid = true;
    gc.split = split;
    gc.ns = ns;
    gc.members = members;
    gc.d_mats = d_mats;
    gc.PX = PX;
    gc.max_slots = slots;
    gc.builds++;
    for (int i = 0; i < 3; i++) gc.kernels[i] = nk[i];
    prof_count(SIGNTRI_KC_DIAG_LEAF, nk[0]);
    prof_count(SIGNTRI_KC_BLOCK_SUMS_F64, nk[1]);
    prof_count(SIGNTRI_KC_OFFDIAG_LEAF, nk[2]);
    ProfScope ps(SIGNTRI_KC_BATCH_GRAPH, st);
    SGT_CUDA_TRY(cudaGraphLaunch(exec, st));
    return SIGNTRI_OK;
}

}  // namespace

void batched_cache_stats(long long *hits, long long *builds)
{
    long long h = 0, b = 0;
    for (auto &row : g_cache)
        for (auto &gc : row) {
            h += gc.hits;
            b += gc.builds;
        }
    *hits = h;
    *builds = b;
}

size_t batched_workspace_bytes(int count, const int *n, int B)
{
    std::vector<int> ns(n, n + count);
    Plan p;
    make_plan(ns, B, p);
    return std::max(plan_bytes(p, B), plan_bytes_bound(ns, B)) + (size_t)count * sizeof(int) + 4096;
}

// bs[m]: leaf size of matrix m (16, 32 or 64); matrices with bs[m] == 0 are
// skipped (handled elsewhere).
signtri_status batched_ph_run(int count, const BatchDesc *h_mats, const BatchDesc *d_mats, const int *bs,
                              bool split, Arena &ws, cudaStream_t st)
{
    for (int B : {16, 32, 64}) {
        std::vector<int> members, ns;
        for (int m = 0; m < count; m++)
            if (bs[m] == B) {
                members.push_back(m);
                ns.push_back(h_mats[m].n);
            }
        if (members.empty()) continue;
        Arena sub = ws;     // each group reuses the workspace after the previous one finished
        signtri_status rs;
        switch (B) {
        case 16: rs = run_group<16>(d_mats, members, ns, split, sub, st); break;
        case 32: rs = run_group<32>(d_mats, members, ns, split, sub, st); break;
        default: rs = run_group<64>(d_mats, members, ns, split, sub, st); break;
        }
        if (rs != SIGNTRI_OK) return rs;
    }
    return SIGNTRI_OK;
}

}  // namespace signtri

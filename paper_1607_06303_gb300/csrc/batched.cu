// batched.cu -- many independent sign(T) problems of uneven size, float64
// Parlett-Higham, in one CUDA graph.
//
// Level-synchronous batch schedule: block anti-diagonal d of every matrix
// depends only on smaller anti-diagonals of the same matrix, so for each d
// one block-sum launch covers the tiles (and K-splits) of anti-diagonal d of
// all matrices with more than d blocks, and one leaf launch finishes them.
// Per-CTA work tables (matrix, tile, K range, partial-sum slot) are built on
// the host once per call; the 2 (nb_max - 1) launches of a cutoff group are
// captured into one CUDA graph and launched as one graph.  Matrices are
// grouped by leaf size (from the cutoff table) because the kernels are
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

template <int B>
signtri_status run_group(const BatchDesc *d_mats, const std::vector<int> &members, const std::vector<int> &ns,
                         bool split, Arena &ws, cudaStream_t st)
{
    Plan p;
    make_plan(ns, B, p);
    int *d_members = static_cast<int *>(ws.take(members.size() * sizeof(int)));
    auto *d_diag = static_cast<DiagTask *>(ws.take(std::max<size_t>(p.diag.size(), 1) * sizeof(DiagTask)));
    auto *d_gemm = static_cast<GemmTask *>(ws.take(std::max<size_t>(p.gemm.size(), 1) * sizeof(GemmTask)));
    auto *d_leaf = static_cast<LeafTask *>(ws.take(std::max<size_t>(p.leaf.size(), 1) * sizeof(LeafTask)));
    const size_t slots = std::max<size_t>(p.max_slots, 1);
    double *PX = static_cast<double *>(ws.take(slots * B * B * sizeof(double)));
    // the efficient form keeps one sum per entry: X and Y share the slabs
    double *PY = split ? PX : static_cast<double *>(ws.take(slots * B * B * sizeof(double)));
    if (!d_members || !d_diag || !d_gemm || !d_leaf || !PX || !PY) return SIGNTRI_ERR_NO_WORKSPACE;
    short *d_perm = nullptr;
    int *d_npos = nullptr, *d_poff = nullptr, *d_noff = nullptr;
    if (split) {
        d_perm = static_cast<short *>(ws.take(std::max<size_t>(p.perm_len, 1) * sizeof(short)));
        d_npos = static_cast<int *>(ws.take(std::max<size_t>(p.npos_len, 1) * sizeof(int)));
        d_poff = static_cast<int *>(ws.take(p.poff.size() * sizeof(int)));
        d_noff = static_cast<int *>(ws.take(p.noff.size() * sizeof(int)));
        if (!d_perm || !d_npos || !d_poff || !d_noff) return SIGNTRI_ERR_NO_WORKSPACE;
        SGT_CUDA_TRY(cudaMemcpyAsync(d_poff, p.poff.data(), p.poff.size() * sizeof(int), cudaMemcpyHostToDevice, st));
        SGT_CUDA_TRY(cudaMemcpyAsync(d_noff, p.noff.data(), p.noff.size() * sizeof(int), cudaMemcpyHostToDevice, st));
    }
    SGT_CUDA_TRY(cudaMemcpyAsync(d_members, members.data(), members.size() * sizeof(int), cudaMemcpyHostToDevice, st));
    SGT_CUDA_TRY(cudaMemcpyAsync(d_diag, p.diag.data(), p.diag.size() * sizeof(DiagTask), cudaMemcpyHostToDevice, st));
    if (!p.gemm.empty())
        SGT_CUDA_TRY(cudaMemcpyAsync(d_gemm, p.gemm.data(), p.gemm.size() * sizeof(GemmTask), cudaMemcpyHostToDevice, st));
    if (!p.leaf.empty())
        SGT_CUDA_TRY(cudaMemcpyAsync(d_leaf, p.leaf.data(), p.leaf.size() * sizeof(LeafTask), cudaMemcpyHostToDevice, st));
    SGT_CUDA_TRY(cudaFuncSetAttribute(batched_leaf_kernel<B>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                      (int)leaf_smem<B>()));
    SGT_CUDA_TRY(cudaFuncSetAttribute(batched_diag_kernel<B>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                      (int)diag_smem<B>()));
    // the level loop, captured into one graph on a private stream
    cudaStream_t cs = nullptr;
    SGT_CUDA_TRY(cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking));
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
    signtri_status rs = SIGNTRI_OK;
    if (cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal) != cudaSuccess) rs = SIGNTRI_ERR_CUDA;
    if (rs == SIGNTRI_OK) {
        prof_pause(true);
        if (split) {
            batched_perm_kernel<B><<<(unsigned)p.diag.size(), B, 0, cs>>>(d_mats, d_members, d_diag, d_perm, d_npos,
                                                                          d_poff, d_noff);
            prof_count(SIGNTRI_KC_DIAG_LEAF, 1);
        }
        batched_diag_kernel<B><<<(unsigned)p.diag.size(), kThreads, diag_smem<B>(), cs>>>(d_mats, d_members, d_diag);
        prof_count(SIGNTRI_KC_DIAG_LEAF, 1);
        for (int d = 1; d < p.nbmax; d++) {
            const int g0 = p.gemm_off[d], g1 = p.gemm_off[d + 1];
            const int l0 = p.leaf_off[d], l1 = p.leaf_off[d + 1];
            if (g1 > g0) {
                if (split)
                    batched_gemm_split_kernel<B><<<g1 - g0, kThreads, 0, cs>>>(d_mats, d_members, d_gemm + g0, d_perm,
                                                                               d_npos, d_poff, d_noff, PX);
                else
                    batched_gemm_kernel<B><<<g1 - g0, kThreads, 0, cs>>>(d_mats, d_members, d_gemm + g0, PX, PY);
                prof_count(SIGNTRI_KC_BLOCK_SUMS_F64, 1);
            }
            if (l1 > l0) {
                batched_leaf_kernel<B><<<l1 - l0, kThreads, leaf_smem<B>(), cs>>>(d_mats, d_members, d_leaf + l0, PX,
                                                                                 PY);
                prof_count(SIGNTRI_KC_OFFDIAG_LEAF, 1);
            }
        }
        prof_pause(false);
        if (cudaStreamEndCapture(cs, &graph) != cudaSuccess) rs = SIGNTRI_ERR_CUDA;
    }
    if (rs == SIGNTRI_OK && cudaGraphInstantiate(&exec, graph, 0) != cudaSuccess) rs = SIGNTRI_ERR_CUDA;
    if (rs == SIGNTRI_OK) {
        ProfScope ps(SIGNTRI_KC_BATCH_GRAPH, st);
        if (cudaGraphLaunch(exec, st) != cudaSuccess) rs = SIGNTRI_ERR_CUDA;
    }
    // the task tables were copied from host vectors; the graph reads the
    // device copies, which live in the workspace until the next call
    if (rs == SIGNTRI_OK && cudaStreamSynchronize(st) != cudaSuccess) rs = SIGNTRI_ERR_CUDA;
    if (exec) cudaGraphExecDestroy(exec);
    if (graph) cudaGraphDestroy(graph);
    cudaStreamDestroy(cs);
    return rs;
}

}  // namespace

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

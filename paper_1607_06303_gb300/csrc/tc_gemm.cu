// tc_gemm.cu -- block products on the 5th-generation tensor cores (tcgen05).
//
// One CTA computes one 128 x 128 product tile D = A B^T over a K range, with
// A = [A_top; A_bot] (two 64-row panels) and B = [B_left; B_right] (two
// 64-row panels), every panel K-contiguous in global memory and loaded by TMA
// (128-byte swizzle).  The four 64 x 64 quadrants of D are four different
// products, e.g. for the Parlett-Higham block sums with A = [U_I.; T_I.] and
// B = [T_.J^T; U_.J^T]:  D_TL = U T,  D_TR = U U,  D_BR = T U.
//
// Operands are bf16 "slices": a float64 matrix is written as a sum of S bf16
// matrices (plain rounding, a hi/lo split, or integer slices scaled per row
// for an exact split), and D = sum over a list of slice pairs (s, t) of
// weight(s,t) * A_s B_t.  Each (pair, K-chunk) unit is accumulated in fp32 in
// TMEM (kind::f16, M = 128, N = 128) and then added into a double-float
// (fp32 hi + fp32 lo) accumulator in the epilogue registers.  With integer
// slices of 7 bits and K-chunks of at most 1024 (8 bits, 256), every fp32
// unit sum is an integer below 2^24 and therefore exact, which makes the
// emulated product accurate to the split: each entry is kept to 2^-49 of its
// row's (column's) power-of-two scale with 7 slices of 7 bits (or 6 of 8), so
// the product is within about 2^-48 of |A||B| where the entries of each row
// of A and column of B are of similar magnitude.
//
// Warp roles (576 threads): warp 0 issues TMA loads into a 3-stage ring of
// two K-blocks per stage,
// warp 1 issues the MMAs (one thread) into 3 TMEM buffers of 128 columns,
// warps 2..17 drain TMEM (four warps per 32-lane quadrant, 32 columns each)
// and keep the fp32 hi parts of the accumulators in the 4th 128-column TMEM
// buffer and the lo parts in registers.
// Every mbarrier wait is bounded; on expiry the CTA records an error and
// returns after draining what it issued.
#include <algorithm>

#include <cuda.h>
#include <cudaTypedefs.h>
#include <cuda_bf16.h>

#include "df_arith.cuh"
#include "internal.cuh"
#include "tc_gemm.cuh"

namespace signtri {

namespace {

constexpr int kStages = 3;
constexpr int kKPS = 2;                     // K-blocks of 64 per stage
constexpr int kTcThreads = 576;            // 2 control warps + 16 epilogue warps
constexpr int kHalfBytes = 32768;           // A 128x64 + B 128x64 bf16 for one K-block
constexpr int kStageBytes = kKPS * kHalfBytes;
constexpr int kBufs = 3;                    // TMEM accumulator buffers of 128 columns; the 4th holds hi
constexpr long long kWaitCycles = 4000000000LL;   // about 2 s at 2 GHz

// Instruction descriptor, kind::f16: D fp32 (bits 4-5 = 1), A and B bf16
// (bits 7-9, 10-12 = 1) or fp16 (0), both K-major, N >> 3 at bit 17, M >> 4
// at bit 24.
constexpr uint32_t kIdesc = (1u << 4) | (1u << 7) | (1u << 10) | ((128u >> 3) << 17) | ((128u >> 4) << 24);
constexpr uint32_t kIdescF16 = (1u << 4) | ((128u >> 3) << 17) | ((128u >> 4) << 24);

__device__ __forceinline__ uint32_t smem_u32(const void *p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ __forceinline__ void mbar_init(uint64_t *bar, uint32_t count)
{
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}

__device__ __forceinline__ void mbar_expect_tx(uint64_t *bar, uint32_t bytes)
{
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes)
                 : "memory");
}

__device__ __forceinline__ void mbar_arrive(uint64_t *bar)
{
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(bar)) : "memory");
}

// Bounded wait for the phase of parity `parity`; false on timeout (after
// `limit` SM clock cycles) or abort.
__device__ __forceinline__ bool mbar_wait_for(uint64_t *bar, uint32_t parity, volatile int *abort_flag,
                                              long long limit)
{
    const uint32_t addr = smem_u32(bar);
    const long long t0 = clock64();
    while (true) {
        uint32_t ok;
        asm volatile(
            "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
            : "=r"(ok)
            : "r"(addr), "r"(parity)
            : "memory");
        if (ok) return true;
        if (*abort_flag) return false;
        if (clock64() - t0 > limit) return false;
    }
}

__device__ __forceinline__ bool mbar_wait(uint64_t *bar, uint32_t parity, volatile int *abort_flag)
{
    return mbar_wait_for(bar, parity, abort_flag, kWaitCycles);
}

// Self-test of the bounded wait: thread 0 waits on a barrier that a thread of
// the second warp completes only when `arrive` is set; without it the wait
// runs out after `limit` cycles and the error word is set.
__global__ void wait_selftest_kernel(int arrive, long long limit, int *err)
{
    __shared__ uint64_t bar;
    __shared__ int abort_flag;
    if (threadIdx.x == 0) {
        mbar_init(&bar, 1);
        abort_flag = 0;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    __syncthreads();
    if (threadIdx.x == 32 && arrive) mbar_arrive(&bar);
    if (threadIdx.x == 0 && !mbar_wait_for(&bar, 0, &abort_flag, limit)) atomicExch(err, 1);
    __syncthreads();
}

__device__ __forceinline__ void tma_load_2d(void *dst, const CUtensorMap *map, uint64_t *bar, int x, int y)
{
    asm volatile(
        "cp.async.bulk.tensor.2d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%3, %4}], [%2];" ::"r"(
            smem_u32(dst)),
        "l"(map), "r"(smem_u32(bar)), "r"(x), "r"(y)
        : "memory");
}

// K-major, 128-byte swizzle smem matrix descriptor: start >> 4, LBO 16 B
// (unused for this layout), SBO 1024 B (8 rows x 128 B), version 1 (bit 46),
// layout SWIZZLE_128B (2 at bit 61).
__device__ __forceinline__ uint64_t smem_desc(const void *p)
{
    const uint64_t a = (smem_u32(p) & 0x3FFFFu) >> 4;
    return a | (1ull << 16) | ((uint64_t)(1024 >> 4) << 32) | (1ull << 46) | (2ull << 61);
}

__device__ __forceinline__ void mma_bf16(uint32_t d_tmem, uint64_t adesc, uint64_t bdesc, uint32_t idesc,
                                         uint32_t accumulate)
{
    asm volatile(
        "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
        " tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(d_tmem),
        "l"(adesc), "l"(bdesc), "r"(idesc), "r"(accumulate)
        : "memory");
}

__device__ __forceinline__ void mma_commit(uint64_t *bar)
{
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(smem_u32(bar))
                 : "memory");
}

__device__ __forceinline__ void fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }

__device__ __forceinline__ void tmem_ld8(uint32_t taddr, float (&v)[8])
{
    uint32_t r[8];
    asm volatile("tcgen05.ld.sync.aligned.32x32b.x8.b32 {%0, %1, %2, %3, %4, %5, %6, %7}, [%8];"
                 : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7])
                 : "r"(taddr));
    asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
    for (int i = 0; i < 8; i++) v[i] = __uint_as_float(r[i]);
}

__device__ __forceinline__ void tmem_st16(uint32_t taddr, const float (&v)[16])
{
    asm volatile(
        "tcgen05.st.sync.aligned.32x32b.x16.b32 [%0], {%1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, "
        "%15, %16};" ::"r"(taddr),
        "r"(__float_as_uint(v[0])), "r"(__float_as_uint(v[1])), "r"(__float_as_uint(v[2])), "r"(__float_as_uint(v[3])),
        "r"(__float_as_uint(v[4])), "r"(__float_as_uint(v[5])), "r"(__float_as_uint(v[6])), "r"(__float_as_uint(v[7])),
        "r"(__float_as_uint(v[8])), "r"(__float_as_uint(v[9])), "r"(__float_as_uint(v[10])),
        "r"(__float_as_uint(v[11])), "r"(__float_as_uint(v[12])), "r"(__float_as_uint(v[13])),
        "r"(__float_as_uint(v[14])), "r"(__float_as_uint(v[15]))
        : "memory");
}

// 16 columns without waiting; the caller issues tcgen05.wait::ld.
__device__ __forceinline__ void tmem_ld16_nowait(uint32_t taddr, uint32_t (&r)[16])
{
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, "
        "%15}, [%16];"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
          "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
        : "r"(taddr));
}

// Error-free addition of a into (hi, lo): Knuth's two-sum.
__device__ __forceinline__ void df_add(float &hi, float &lo, float a)
{
    const float s = __fadd_rn(hi, a);
    const float bb = __fsub_rn(s, hi);
    const float err = __fadd_rn(__fsub_rn(hi, __fsub_rn(s, bb)), __fsub_rn(a, bb));
    hi = s;
    lo = __fadd_rn(lo, err);
}

// TMA coordinates of K-block kb of rows [row, row + 64) of slice sl of a
// source with `rows` rows: plain layout (x = K offset, y = stacked row) or
// blocked layout (64 x 64 tiles, each a contiguous run of 64 rows).
__device__ __forceinline__ void src_coord(int blk, int nkb, int rows, int sl, int row, int kb, int &x, int &y)
{
    if (blk) {
        x = 0;
        y = ((sl * (rows >> 6) + (row >> 6)) * nkb + kb) << 6;
    } else {
        x = kb * 64;
        y = sl * rows + row;
    }
}

// Units of one job: (K-chunk, pair) in pair mode, K-chunks in resident mode.
__device__ __forceinline__ int job_units(const TcJob &job, int chunk_kb, int npairs, int resident)
{
    const int nkb = job.kb1 - job.kb0;
    const int nchunks = nkb > 0 ? (nkb + chunk_kb - 1) / chunk_kb : 0;
    return resident ? nchunks : npairs * nchunks;
}

// A CTA runs jobs [job_off[b], job_off[b+1]) (job b alone when job_off is
// null) back to back: the load ring, the MMA buffers and their barrier
// phases run on across job boundaries, and the epilogue writes each job's
// result after its last unit.
__global__ void __launch_bounds__(kTcThreads, 1)
tc_blocksum_kernel(const __grid_constant__ CUtensorMap mTop, const __grid_constant__ CUtensorMap mBot,
                   const __grid_constant__ CUtensorMap mLeft, const __grid_constant__ CUtensorMap mRight,
                   int rowsA, int rowsB, const TcJob *__restrict__ jobs, const int *__restrict__ job_off,
                   const TcPairs *__restrict__ pairs_g, int chunk_kb, const float *__restrict__ sTop,
                   const float *__restrict__ sBot, const float *__restrict__ sLeft, const float *__restrict__ sRight,
                   double *__restrict__ out, TcQuadOut qo, int *__restrict__ err, int resident, int nsl, int blk,
                   int nkb, int f16)
{
    const uint32_t idesc = f16 ? kIdescF16 : kIdesc;
    extern __shared__ unsigned char smem_raw[];
    unsigned char *smem = (unsigned char *)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
    uint64_t *full = reinterpret_cast<uint64_t *>(smem + kStages * kStageBytes);
    uint64_t *empty = full + kStages;
    uint64_t *tfull = empty + kStages;
    uint64_t *tempty = tfull + 4;
    uint64_t *done_bar = tempty + 4;
    uint32_t *tmem_holder = reinterpret_cast<uint32_t *>(done_bar + 1);
    volatile int *abort_flag = reinterpret_cast<volatile int *>(tmem_holder + 1);
    TcPairs *pairs_s = reinterpret_cast<TcPairs *>(smem + kStages * kStageBytes + 512);

    const int warp = threadIdx.x / 32, lane = threadIdx.x % 32;
    const int j0 = job_off ? job_off[blockIdx.x] : (int)blockIdx.x;
    const int j1 = job_off ? job_off[blockIdx.x + 1] : (int)blockIdx.x + 1;
    for (int i = threadIdx.x; i < (int)(sizeof(TcPairs) / 4); i += blockDim.x)
        reinterpret_cast<int *>(pairs_s)[i] = reinterpret_cast<const int *>(pairs_g)[i];
    __syncthreads();
    const TcPairs &pairs = *pairs_s;
    // pair mode: one unit per (K-chunk, pair), stages of kKPS K-blocks of one
    // slice pair.  Resident mode (unit-weight pairs of nsl slices): a stage
    // holds one K-block of all nsl slices of A and of B, every pair's MMAs
    // are issued from it into one accumulator, one unit per K-chunk.
    const int sbytes = resident ? 2 * nsl * (kHalfBytes / 2) : kStageBytes;
    const int nring = resident ? min(kStages, (kStages * kStageBytes) / sbytes) : kStages;
    long long total_units = 0;
    for (int j = j0; j < j1; j++) total_units += job_units(jobs[j], chunk_kb, pairs.n, resident);

    if (threadIdx.x == 0) {
        for (int s = 0; s < kStages; s++) { mbar_init(&full[s], 1); mbar_init(&empty[s], 1); }
        for (int b = 0; b < kBufs; b++) { mbar_init(&tfull[b], 1); mbar_init(&tempty[b], 16); }
        mbar_init(done_bar, 1);
        *abort_flag = 0;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if (warp == 1) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], 512;" ::"r"(smem_u32(tmem_holder))
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    fence_before();
    __syncthreads();
    fence_after();
    const uint32_t tmem_base = *tmem_holder;

    if (warp == 0) {
        if (lane == 0 && total_units > 0) {
            asm volatile("prefetch.tensormap [%0];" ::"l"(&mTop) : "memory");
            asm volatile("prefetch.tensormap [%0];" ::"l"(&mBot) : "memory");
            asm volatile("prefetch.tensormap [%0];" ::"l"(&mLeft) : "memory");
            asm volatile("prefetch.tensormap [%0];" ::"l"(&mRight) : "memory");
            int stage = 0;
            uint32_t phase = 0;
            long long issued = 0;
            bool ok = true;
            for (int j = j0; j < j1 && ok; j++) {
                const TcJob job = jobs[j];
                const int nu = job_units(job, chunk_kb, pairs.n, resident);
                for (int u = 0; u < nu && ok; u++) {
                    const int c = resident ? u : u / pairs.n, p = resident ? 0 : u % pairs.n;
                    // chunk-major: the pairs of one K-chunk reuse its panels in L2
                    const int kbs = job.kb0 + c * chunk_kb, kbe = min(kbs + chunk_kb, job.kb1);
                    const int step = resident ? 1 : kKPS;
                    for (int kb = kbs; kb < kbe; kb += step) {
                        if (!mbar_wait(&empty[stage], phase ^ 1, abort_flag)) { ok = false; break; }
                        unsigned char *base = smem + stage * sbytes;
                        if (resident) {
                            // [A slice 0 | ... | A slice nsl-1 | B slice 0 | ...], 16 KB each
                            mbar_expect_tx(&full[stage], 2 * nsl * (kHalfBytes / 2));
                            for (int sl = 0; sl < nsl; sl++) {
                                unsigned char *a = base + sl * (kHalfBytes / 2);
                                unsigned char *b = base + (nsl + sl) * (kHalfBytes / 2);
                                int x, y;
                                src_coord(blk, nkb, rowsA, sl, job.rt, kb, x, y);
                                tma_load_2d(a, &mTop, &full[stage], x, y);
                                src_coord(blk, nkb, rowsA, sl, job.rb, kb, x, y);
                                tma_load_2d(a + 8192, &mBot, &full[stage], x, y);
                                src_coord(blk, nkb, rowsB, sl, job.cl, kb, x, y);
                                tma_load_2d(b, &mLeft, &full[stage], x, y);
                                src_coord(blk, nkb, rowsB, sl, job.cr, kb, x, y);
                                tma_load_2d(b + 8192, &mRight, &full[stage], x, y);
                            }
                        } else {
                            const int nk = min(kKPS, kbe - kb);
                            const int sa = pairs.s[p], sb = pairs.t[p];
                            mbar_expect_tx(&full[stage], nk * kHalfBytes);
                            for (int h = 0; h < nk; h++) {
                                // stage layout: A halves [h][top 8 KB | bottom 8 KB], then B halves
                                unsigned char *a = base + h * (kHalfBytes / 2);
                                unsigned char *b = base + kStageBytes / 2 + h * (kHalfBytes / 2);
                                int x, y;
                                src_coord(blk, nkb, rowsA, sa, job.rt, kb + h, x, y);
                                tma_load_2d(a, &mTop, &full[stage], x, y);
                                src_coord(blk, nkb, rowsA, sa, job.rb, kb + h, x, y);
                                tma_load_2d(a + 8192, &mBot, &full[stage], x, y);
                                src_coord(blk, nkb, rowsB, sb, job.cl, kb + h, x, y);
                                tma_load_2d(b, &mLeft, &full[stage], x, y);
                                src_coord(blk, nkb, rowsB, sb, job.cr, kb + h, x, y);
                                tma_load_2d(b + 8192, &mRight, &full[stage], x, y);
                            }
                        }
                        issued++;
                        if (++stage == nring) { stage = 0; phase ^= 1; }
                    }
                }
            }
            if (!ok) {
                *abort_flag = 1;
                atomicExch(err, 1);
                // drain: wait (bounded) for the loads of the last stages issued
                const long long tail = issued < nring ? issued : nring;
                for (long long i = 0; i < tail; i++) {
                    if (stage == 0) { stage = nring - 1; phase ^= 1; } else stage--;
                    const uint32_t a = smem_u32(&full[stage]);
                    const long long t0 = clock64();
                    while (clock64() - t0 < kWaitCycles) {
                        uint32_t done;
                        asm volatile(
                            "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n"
                            " selp.u32 %0, 1, 0, p;\n}\n"
                            : "=r"(done)
                            : "r"(a), "r"(phase)
                            : "memory");
                        if (done) break;
                    }
                }
            }
        }
    } else if (warp == 1) {
        if (lane == 0 && total_units > 0) {
            int stage = 0;
            uint32_t phase = 0;
            bool ok = true;
            int g = 0;   // unit index across jobs
            for (int j = j0; j < j1 && ok; j++) {
                const TcJob job = jobs[j];
                const int nu = job_units(job, chunk_kb, pairs.n, resident);
                for (int u = 0; u < nu && ok; u++, g++) {
                    const int buf = g % kBufs;
                    const uint32_t tphase = (uint32_t)((g / kBufs) & 1);
                    if (!mbar_wait(&tempty[buf], tphase ^ 1, abort_flag)) { ok = false; break; }
                    fence_after();
                    const uint32_t d = tmem_base + (uint32_t)(buf * 128);
                    const int c = resident ? u : u / pairs.n;
                    const int kbs = job.kb0 + c * chunk_kb, kbe = min(kbs + chunk_kb, job.kb1);
                    const int step = resident ? 1 : kKPS;
                    for (int kb = kbs; kb < kbe; kb += step) {
                        if (!mbar_wait(&full[stage], phase, abort_flag)) { ok = false; break; }
                        fence_after();
                        unsigned char *base = smem + stage * sbytes;
                        if (resident) {
                            for (int p = 0; p < pairs.n; p++) {
                                const uint64_t ad = smem_desc(base + pairs.s[p] * (kHalfBytes / 2));
                                const uint64_t bd = smem_desc(base + (nsl + pairs.t[p]) * (kHalfBytes / 2));
#pragma unroll
                                for (int k = 0; k < 4; k++)
                                    mma_bf16(d, ad + (uint64_t)(2 * k), bd + (uint64_t)(2 * k), idesc,
                                             (kb > kbs || p > 0 || k > 0) ? 1u : 0u);
                            }
                        } else {
                            const int nk = min(kKPS, kbe - kb);
                            for (int h = 0; h < nk; h++) {
                                unsigned char *a = base + h * (kHalfBytes / 2);
                                unsigned char *b = base + kStageBytes / 2 + h * (kHalfBytes / 2);
                                const uint64_t ad = smem_desc(a), bd = smem_desc(b);
#pragma unroll
                                for (int k = 0; k < 4; k++)
                                    mma_bf16(d, ad + (uint64_t)(2 * k), bd + (uint64_t)(2 * k), idesc,
                                             (kb > kbs || h > 0 || k > 0) ? 1u : 0u);
                            }
                        }
                        mma_commit(&empty[stage]);
                        if (++stage == nring) { stage = 0; phase ^= 1; }
                    }
                    if (!ok) break;
                    mma_commit(&tfull[buf]);
                }
            }
            if (!ok) {
                *abort_flag = 1;
                atomicExch(err, 1);
            }
            // arrives once every MMA issued by this thread has completed
            mma_commit(done_bar);
        }
    } else {
        const int q = warp & 3;                 // TMEM lane quadrant this warp may read
        const int cg = (warp - 2) >> 2;         // 32-column group 0..3
        const uint32_t lane_base = tmem_base + ((uint32_t)(32 * q) << 16);
        const uint32_t taddr_hi = lane_base + (uint32_t)(kBufs * 128 + cg * 32);
        const int row = 32 * q + lane;
        const int r = row & 63;
        const bool bottom = row >= 64;
        const int half = cg >> 1;
        const int c0 = (cg & 1) * 32;           // first column inside the quadrant
        const int quad = (bottom ? 2 : 0) + half;
        const bool quad_mode = qo.m[0] || qo.m[1] || qo.m[2] || qo.m[3];
        bool ok = true;
        int g = 0;   // unit index across jobs
        for (int j = j0; j < j1 && ok; j++) {
            const int nu = job_units(jobs[j], chunk_kb, pairs.n, resident);
            float lo[32];
#pragma unroll
            for (int i = 0; i < 32; i++) lo[i] = 0.f;
            for (int u = 0; u < nu && ok; u++, g++) {
                const int buf = g % kBufs;
                const uint32_t tphase = (uint32_t)((g / kBufs) & 1);
                if (!mbar_wait(&tfull[buf], tphase, abort_flag)) { ok = false; break; }
                fence_after();
                const float w = resident ? pairs.w[0] : pairs.w[u % pairs.n];
                const uint32_t taddr = lane_base + (uint32_t)(buf * 128 + cg * 32);
#pragma unroll
                for (int cc = 0; cc < 32; cc += 16) {
                    uint32_t rv[16], rh[16];
                    tmem_ld16_nowait(taddr + cc, rv);
                    if (u > 0) tmem_ld16_nowait(taddr_hi + cc, rh);
                    asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
                    float h[16];
                    if (u == 0) {
#pragma unroll
                        for (int i = 0; i < 16; i++) h[i] = __fmul_rn(__uint_as_float(rv[i]), w);
                    } else {
#pragma unroll
                        for (int i = 0; i < 16; i++) {
                            h[i] = __uint_as_float(rh[i]);
                            df_add(h[i], lo[cc + i], __fmul_rn(__uint_as_float(rv[i]), w));
                        }
                    }
                    tmem_st16(taddr_hi + cc, h);
                }
                asm volatile("tcgen05.wait::st.sync.aligned;" ::: "memory");
                fence_before();
                __syncwarp();
                if (lane == 0) mbar_arrive(&tempty[buf]);
            }
            if (!ok) break;
            // this job's result
            const TcJob job = jobs[j];
            double srow = 1.0;
            if (bottom) { if (sBot) srow = sBot[job.rb + r]; }
            else if (sTop) srow = sTop[job.rt + r];
            const float *scol = half ? sRight : sLeft;
            const int cbase = (half ? job.cr : job.cl) + c0;
            double *o = nullptr;
            float2 *o2 = nullptr;
            if (quad_mode) {
                // quadrant-matrix mode: element (row, col) of quadrant q goes to
                // m[q][(row base + r) + (col base + c) * ld] as float64; null m[q] = skip
                o = qo.m[quad];
                const int grow = (bottom ? job.rb : job.rt) + r;
                if (grow >= qo.nrows) o = nullptr;
                if (o) o += (size_t)grow + (size_t)cbase * qo.ld + (size_t)job.slot * qo.slot_stride;
            } else {
                // slot mode: (hi, lo) pairs, float2 per element
                o2 = reinterpret_cast<float2 *>(out) + (size_t)job.slot * 16384 + (size_t)quad * 4096 +
                     (size_t)c0 * 64 + r;
            }
            const float srow_f = (float)srow;
#pragma unroll
            for (int cc = 0; cc < 32; cc += 8) {
                float h[8];
                if (nu > 0) tmem_ld8(taddr_hi + cc, h);
                else {
#pragma unroll
                    for (int i = 0; i < 8; i++) h[i] = 0.f;
                }
#pragma unroll
                for (int i = 0; i < 8; i++) {
                    // scales are powers of two: exact in fp32
                    const float sc = __fmul_rn(srow_f, scol ? scol[cbase + cc + i] : 1.f);
                    const float hs = __fmul_rn(h[i], sc), ls = __fmul_rn(lo[cc + i], sc);
                    if (o2) o2[(size_t)(cc + i) * 64] = make_float2(hs, ls);
                    else if (o && cbase + cc + i < qo.ncols) o[(size_t)(cc + i) * qo.ld] = df_to_double(hs, ls);
                }
            }
        }
        if (!ok) {
            *abort_flag = 1;
            atomicExch(err, 1);
        }
    }

    fence_before();
    __syncthreads();
    fence_after();
    if (warp == 1) {
        // done_bar completes once, when all MMAs of this CTA have finished
        if (total_units > 0) {
            const uint32_t a = smem_u32(done_bar);
            const long long t0 = clock64();
            while (clock64() - t0 < kWaitCycles) {
                uint32_t done;
                asm volatile(
                    "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
                    : "=r"(done)
                    : "r"(a), "r"(0u)
                    : "memory");
                if (done) break;
            }
        }
        __syncwarp();
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, 512;" ::"r"(tmem_base) : "memory");
    }
}

// ---------------------------------------------------------------------------
// Grouped pair mode: slice pairs (s, t0), (s, t1) with the same A slice run
// as one N = 256 MMA, A_s x [B_t0 | B_t1]^T, the two 128-column halves of the
// accumulator being the two pairs' unit sums (each exact, as in pair mode).
// Per MMA the tensor core then reads 12 KB of operands for 2 x 128 x 128 x 16
// products instead of 16 KB, and a K-block stage is written once for two
// pairs: shared-memory traffic per product drops by a quarter, which is what
// bounds pair mode.  A pair without a partner runs alone (N = 128).  Two TMEM
// accumulators of 256 columns fill the TMEM, so the fp32 hi parts of the
// result live half in registers, half in shared memory (thread-private
// columns), and the lo parts in registers: the shared memory left over holds
// a 4-stage ring, which the units' operand latency needs (3 stages ran the
// tensor pipe ~10% slower despite a few registers spilled now).  Warp roles,
// job lists and outputs as in tc_blocksum_kernel.

constexpr int kP2Stages = 4;
constexpr int kP2StageBytes = 3 * 16384;          // A | B_t0 | B_t1 for one K-block
constexpr int kP2HiBytes = 512 * 16 * 4;           // 16 of the 32 hi values per epilogue thread

struct TcGroups {
    int n;
    int s[kTcMaxPairs], t0[kTcMaxPairs], t1[kTcMaxPairs];   // t1 < 0: single pair
    float w0[kTcMaxPairs], w1[kTcMaxPairs];
};

__device__ __forceinline__ void mma_bf16_n(uint32_t d_tmem, uint64_t adesc, uint64_t bdesc, uint32_t idesc,
                                           uint32_t accumulate)
{
    asm volatile(
        "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
        " tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(d_tmem),
        "l"(adesc), "l"(bdesc), "r"(idesc), "r"(accumulate)
        : "memory");
}

__global__ void __launch_bounds__(kTcThreads, 1)
tc_pair2_kernel(const __grid_constant__ CUtensorMap mTop, const __grid_constant__ CUtensorMap mBot,
                const __grid_constant__ CUtensorMap mLeft, const __grid_constant__ CUtensorMap mRight, int rowsA,
                int rowsB, const TcJob *__restrict__ jobs, const int *__restrict__ job_off,
                const TcPairs *__restrict__ pairs_g, int chunk_kb, const float *__restrict__ sTop,
                const float *__restrict__ sBot, const float *__restrict__ sLeft, const float *__restrict__ sRight,
                double *__restrict__ out, TcQuadOut qo, int *__restrict__ err, int blk, int nkb)
{
    extern __shared__ unsigned char smem_raw[];
    unsigned char *smem = (unsigned char *)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
    float *his = reinterpret_cast<float *>(smem + kP2Stages * kP2StageBytes);
    uint64_t *full = reinterpret_cast<uint64_t *>(smem + kP2Stages * kP2StageBytes + kP2HiBytes);
    uint64_t *empty = full + kP2Stages;
    uint64_t *tfull = empty + kP2Stages;
    uint64_t *tempty = tfull + 2;
    uint64_t *done_bar = tempty + 2;
    uint32_t *tmem_holder = reinterpret_cast<uint32_t *>(done_bar + 1);
    volatile int *abort_flag = reinterpret_cast<volatile int *>(tmem_holder + 1);
    TcGroups *grp_s = reinterpret_cast<TcGroups *>(smem + kP2Stages * kP2StageBytes + kP2HiBytes + 512);

    const int warp = threadIdx.x / 32, lane = threadIdx.x % 32;
    const int j0 = job_off ? job_off[blockIdx.x] : (int)blockIdx.x;
    const int j1 = job_off ? job_off[blockIdx.x + 1] : (int)blockIdx.x + 1;
    if (threadIdx.x == 0) {
        // group the pairs by A slice, in list order: each pair takes the next
        // unused pair with the same s as its partner
        const TcPairs &pp = *pairs_g;
        bool used[kTcMaxPairs];
        for (int p = 0; p < pp.n; p++) used[p] = false;
        int ng = 0;
        for (int p = 0; p < pp.n; p++) {
            if (used[p]) continue;
            used[p] = true;
            int q = -1;
            for (int r = p + 1; r < pp.n && q < 0; r++)
                if (!used[r] && pp.s[r] == pp.s[p]) q = r;
            grp_s->s[ng] = pp.s[p];
            grp_s->t0[ng] = pp.t[p];
            grp_s->w0[ng] = pp.w[p];
            if (q >= 0) {
                used[q] = true;
                grp_s->t1[ng] = pp.t[q];
                grp_s->w1[ng] = pp.w[q];
            } else {
                grp_s->t1[ng] = -1;
                grp_s->w1[ng] = 0.f;
            }
            ng++;
        }
        grp_s->n = ng;
    }
    __syncthreads();
    const TcGroups &grp = *grp_s;
    const int ngrp = grp.n;
    long long total_units = 0;
    for (int j = j0; j < j1; j++) total_units += job_units(jobs[j], chunk_kb, ngrp, 0);

    if (threadIdx.x == 0) {
        for (int s = 0; s < kP2Stages; s++) { mbar_init(&full[s], 1); mbar_init(&empty[s], 1); }
        for (int b = 0; b < 2; b++) { mbar_init(&tfull[b], 1); mbar_init(&tempty[b], 16); }
        mbar_init(done_bar, 1);
        *abort_flag = 0;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if (warp == 1) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], 512;" ::"r"(smem_u32(tmem_holder))
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    fence_before();
    __syncthreads();
    fence_after();
    const uint32_t tmem_base = *tmem_holder;

    if (warp == 0) {
        if (lane == 0 && total_units > 0) {
            asm volatile("prefetch.tensormap [%0];" ::"l"(&mTop) : "memory");
            asm volatile("prefetch.tensormap [%0];" ::"l"(&mBot) : "memory");
            asm volatile("prefetch.tensormap [%0];" ::"l"(&mLeft) : "memory");
            asm volatile("prefetch.tensormap [%0];" ::"l"(&mRight) : "memory");
            int stage = 0;
            uint32_t phase = 0;
            long long issued = 0;
            bool ok = true;
            for (int j = j0; j < j1 && ok; j++) {
                const TcJob job = jobs[j];
                const int nu = job_units(job, chunk_kb, ngrp, 0);
                for (int u = 0; u < nu && ok; u++) {
                    // chunk-major: the groups of one K-chunk reuse its panels in L2
                    const int c = u / ngrp, p = u % ngrp;
                    const int sa = grp.s[p], tb0 = grp.t0[p], tb1 = grp.t1[p];
                    const int kbs = job.kb0 + c * chunk_kb, kbe = min(kbs + chunk_kb, job.kb1);
                    for (int kb = kbs; kb < kbe; kb++) {
                        if (!mbar_wait(&empty[stage], phase ^ 1, abort_flag)) { ok = false; break; }
                        unsigned char *base = smem + stage * kP2StageBytes;
                        mbar_expect_tx(&full[stage], tb1 >= 0 ? 3 * 16384 : 2 * 16384);
                        int x, y;
                        src_coord(blk, nkb, rowsA, sa, job.rt, kb, x, y);
                        tma_load_2d(base, &mTop, &full[stage], x, y);
                        src_coord(blk, nkb, rowsA, sa, job.rb, kb, x, y);
                        tma_load_2d(base + 8192, &mBot, &full[stage], x, y);
                        src_coord(blk, nkb, rowsB, tb0, job.cl, kb, x, y);
                        tma_load_2d(base + 16384, &mLeft, &full[stage], x, y);
                        src_coord(blk, nkb, rowsB, tb0, job.cr, kb, x, y);
                        tma_load_2d(base + 24576, &mRight, &full[stage], x, y);
                        if (tb1 >= 0) {
                            src_coord(blk, nkb, rowsB, tb1, job.cl, kb, x, y);
                            tma_load_2d(base + 32768, &mLeft, &full[stage], x, y);
                            src_coord(blk, nkb, rowsB, tb1, job.cr, kb, x, y);
                            tma_load_2d(base + 40960, &mRight, &full[stage], x, y);
                        }
                        issued++;
                        if (++stage == kP2Stages) { stage = 0; phase ^= 1; }
                    }
                }
            }
            if (!ok) {
                *abort_flag = 1;
                atomicExch(err, 1);
                const long long tail = issued < kP2Stages ? issued : kP2Stages;
                for (long long i = 0; i < tail; i++) {
                    if (stage == 0) { stage = kP2Stages - 1; phase ^= 1; } else stage--;
                    const uint32_t a = smem_u32(&full[stage]);
                    const long long t0 = clock64();
                    while (clock64() - t0 < kWaitCycles) {
                        uint32_t done;
                        asm volatile(
                            "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n"
                            " selp.u32 %0, 1, 0, p;\n}\n"
                            : "=r"(done)
                            : "r"(a), "r"(phase)
                            : "memory");
                        if (done) break;
                    }
                }
            }
        }
    } else if (warp == 1) {
        if (lane == 0 && total_units > 0) {
            const uint32_t idesc256 = (1u << 4) | (1u << 7) | (1u << 10) | ((256u >> 3) << 17) | ((128u >> 4) << 24);
            int stage = 0;
            uint32_t phase = 0;
            bool ok = true;
            int g = 0;
            for (int j = j0; j < j1 && ok; j++) {
                const TcJob job = jobs[j];
                const int nu = job_units(job, chunk_kb, ngrp, 0);
                for (int u = 0; u < nu && ok; u++, g++) {
                    const int buf = g & 1;
                    const uint32_t tphase = (uint32_t)((g >> 1) & 1);
                    if (!mbar_wait(&tempty[buf], tphase ^ 1, abort_flag)) { ok = false; break; }
                    fence_after();
                    const uint32_t d = tmem_base + (uint32_t)(buf * 256);
                    const int c = u / ngrp, p = u % ngrp;
                    const uint32_t idesc = grp.t1[p] >= 0 ? idesc256 : kIdesc;
                    const int kbs = job.kb0 + c * chunk_kb, kbe = min(kbs + chunk_kb, job.kb1);
                    for (int kb = kbs; kb < kbe; kb++) {
                        if (!mbar_wait(&full[stage], phase, abort_flag)) { ok = false; break; }
                        fence_after();
                        unsigned char *base = smem + stage * kP2StageBytes;
                        const uint64_t ad = smem_desc(base), bd = smem_desc(base + 16384);
#pragma unroll
                        for (int k = 0; k < 4; k++)
                            mma_bf16_n(d, ad + (uint64_t)(2 * k), bd + (uint64_t)(2 * k), idesc,
                                       (kb > kbs || k > 0) ? 1u : 0u);
                        mma_commit(&empty[stage]);
                        if (++stage == kP2Stages) { stage = 0; phase ^= 1; }
                    }
                    if (!ok) break;
                    mma_commit(&tfull[buf]);
                }
            }
            if (!ok) {
                *abort_flag = 1;
                atomicExch(err, 1);
            }
            mma_commit(done_bar);
        }
    } else {
        const int q = warp & 3;                 // TMEM lane quadrant this warp may read
        const int cg = (warp - 2) >> 2;         // 32-column group 0..3
        const uint32_t lane_base = tmem_base + ((uint32_t)(32 * q) << 16);
        const int row = 32 * q + lane;
        const int r = row & 63;
        const bool bottom = row >= 64;
        const int half = cg >> 1;
        const int c0 = (cg & 1) * 32;
        const int quad = (bottom ? 2 : 0) + half;
        const bool quad_mode = qo.m[0] || qo.m[1] || qo.m[2] || qo.m[3];
        float *his_t = his + (threadIdx.x - 64);   // his_t[i * 512]: this thread's column 16 + i
        bool ok = true;
        int g = 0;
        for (int j = j0; j < j1 && ok; j++) {
            const int nu = job_units(jobs[j], chunk_kb, ngrp, 0);
            float lo[32], hr[16];
#pragma unroll
            for (int i = 0; i < 32; i++) lo[i] = 0.f;
#pragma unroll
            for (int i = 0; i < 16; i++) hr[i] = 0.f;
            for (int u = 0; u < nu && ok; u++, g++) {
                const int buf = g & 1;
                const uint32_t tphase = (uint32_t)((g >> 1) & 1);
                if (!mbar_wait(&tfull[buf], tphase, abort_flag)) { ok = false; break; }
                fence_after();
                const int p = u % ngrp;
                const float w0 = grp.w0[p], w1 = grp.w1[p];
                const bool two = grp.t1[p] >= 0;
                const uint32_t taddr = lane_base + (uint32_t)(buf * 256 + cg * 32);
#pragma unroll
                for (int cc = 0; cc < 32; cc += 16) {
                    uint32_t v0[16], v1[16];
                    tmem_ld16_nowait(taddr + cc, v0);
                    if (two) tmem_ld16_nowait(taddr + 128 + cc, v1);
                    asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
                    for (int i = 0; i < 16; i++) {
                        // hi of columns 0..15 in registers, 16..31 in shared memory
                        float h = (u == 0) ? __fmul_rn(__uint_as_float(v0[i]), w0)
                                           : (cc == 0 ? hr[i] : his_t[i * 512]);
                        if (u > 0) df_add(h, lo[cc + i], __fmul_rn(__uint_as_float(v0[i]), w0));
                        if (two) df_add(h, lo[cc + i], __fmul_rn(__uint_as_float(v1[i]), w1));
                        if (cc == 0) hr[i] = h;
                        else his_t[i * 512] = h;
                    }
                }
                fence_before();
                __syncwarp();
                if (lane == 0) mbar_arrive(&tempty[buf]);
            }
            if (!ok) break;
            const TcJob job = jobs[j];
            double srow = 1.0;
            if (bottom) { if (sBot) srow = sBot[job.rb + r]; }
            else if (sTop) srow = sTop[job.rt + r];
            const float *scol = half ? sRight : sLeft;
            const int cbase = (half ? job.cr : job.cl) + c0;
            double *o = nullptr;
            float2 *o2 = nullptr;
            if (quad_mode) {
                o = qo.m[quad];
                const int grow = (bottom ? job.rb : job.rt) + r;
                if (grow >= qo.nrows) o = nullptr;
                if (o) o += (size_t)grow + (size_t)cbase * qo.ld + (size_t)job.slot * qo.slot_stride;
            } else {
                o2 = reinterpret_cast<float2 *>(out) + (size_t)job.slot * 16384 + (size_t)quad * 4096 +
                     (size_t)c0 * 64 + r;
            }
            const float srow_f = (float)srow;
#pragma unroll
            for (int i = 0; i < 32; i++) {
                const float h = nu > 0 ? (i < 16 ? hr[i] : his_t[(i - 16) * 512]) : 0.f;
                const float sc = __fmul_rn(srow_f, scol ? scol[cbase + i] : 1.f);
                const float hs = __fmul_rn(h, sc), ls = __fmul_rn(lo[i], sc);
                if (o2) o2[(size_t)i * 64] = make_float2(hs, ls);
                else if (o && cbase + i < qo.ncols) o[(size_t)i * qo.ld] = df_to_double(hs, ls);
            }
        }
        if (!ok) {
            *abort_flag = 1;
            atomicExch(err, 1);
        }
    }

    fence_before();
    __syncthreads();
    fence_after();
    if (warp == 1) {
        if (total_units > 0) {
            const uint32_t a = smem_u32(done_bar);
            const long long t0 = clock64();
            while (clock64() - t0 < kWaitCycles) {
                uint32_t done;
                asm volatile(
                    "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
                    : "=r"(done)
                    : "r"(a), "r"(0u)
                    : "memory");
                if (done) break;
            }
        }
        __syncwarp();
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, 512;" ::"r"(tmem_base) : "memory");
    }
}

PFN_cuTensorMapEncodeTiled_v12000 g_encode = nullptr;

signtri_status get_encoder()
{
    if (g_encode) return SIGNTRI_OK;
    cudaDriverEntryPointQueryResult q;
    void *fn = nullptr;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &fn, 12000, cudaEnableDefault, &q) != cudaSuccess ||
        q != cudaDriverEntryPointSuccess || !fn)
        return SIGNTRI_ERR_CUDA;
    g_encode = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(fn);
    return SIGNTRI_OK;
}

// 2-D map over `rows` rows of `cols` bf16 (cols contiguous, row pitch ld
// elements), box 64 x 64, 128-byte swizzle, zero fill out of bounds.
signtri_status make_map(CUtensorMap *m, const __nv_bfloat16 *base, long long rows, long long cols, long long ld)
{
    if (((uintptr_t)base & 15) || (ld * 2) % 16) return SIGNTRI_ERR_BAD_ARG;
    cuuint64_t dims[2] = {(cuuint64_t)cols, (cuuint64_t)rows};
    cuuint64_t strides[1] = {(cuuint64_t)(ld * 2)};
    cuuint32_t box[2] = {64, 64};
    cuuint32_t estr[2] = {1, 1};
    CUresult r = g_encode(m, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2, const_cast<__nv_bfloat16 *>(base), dims, strides,
                          box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B,
                          CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    return r == CUDA_SUCCESS ? SIGNTRI_OK : SIGNTRI_ERR_CUDA;
}

}  // namespace

signtri_status wait_selftest(int arrive, long long limit, int *d_err, cudaStream_t st)
{
    ProfScope ps(SIGNTRI_KC_OTHER, st);
    wait_selftest_kernel<<<1, 64, 0, st>>>(arrive, limit, d_err);
    SGT_LAUNCH_CHECK();
    return SIGNTRI_OK;
}

size_t tc_smem_bytes() { return (size_t)kStages * kStageBytes + 1024 + 512 + sizeof(TcPairs) + 64; }

size_t tc_pair2_smem_bytes()
{
    return (size_t)kP2Stages * kP2StageBytes + kP2HiBytes + 1024 + 512 + sizeof(TcGroups) + 64;
}

signtri_status tc_blocksums(const TcSource &top, const TcSource &bot, const TcSource &left, const TcSource &right,
                            const TcJob *d_jobs, int njobs, const TcPairs &pairs, const TcPairs *d_pairs, int chunk_kb,
                            double *out, const TcQuadOut &qo, int *d_err, int kernel_class, cudaStream_t st,
                            double useful_flops, const int *d_job_off, int nctas)
{
    if (njobs <= 0) return SIGNTRI_OK;
    if (d_job_off && nctas <= 0) return SIGNTRI_ERR_BAD_ARG;
    if (pairs.n <= 0 || pairs.n > kTcMaxPairs || chunk_kb <= 0 || !d_pairs) return SIGNTRI_ERR_BAD_ARG;
    signtri_status rs = get_encoder();
    if (rs != SIGNTRI_OK) return rs;
    // all four sources in one layout; a blocked layout needs whole tiles and
    // one K-block count
    const int blk = top.blocked ? 1 : 0;
    if ((bot.blocked ? 1 : 0) != blk || (left.blocked ? 1 : 0) != blk || (right.blocked ? 1 : 0) != blk)
        return SIGNTRI_ERR_BAD_ARG;
    // one operand type for A and B (kind::f16 takes both bf16 or both fp16)
    const int f16 = top.f16 ? 1 : 0;
    if ((bot.f16 ? 1 : 0) != f16 || (left.f16 ? 1 : 0) != f16 || (right.f16 ? 1 : 0) != f16)
        return SIGNTRI_ERR_BAD_ARG;
    if (blk && (top.cols != bot.cols || top.cols != left.cols || top.cols != right.cols || (top.cols & 63) ||
                (top.rows & 63) || (left.rows & 63)))
        return SIGNTRI_ERR_BAD_ARG;
    auto map_of = [&](CUtensorMap *m, const TcSource &src) {
        if (src.blocked)
            return make_map(m, src.base, (long long)src.nslices * src.rows * (src.cols / 64), 64, 64);
        return make_map(m, src.base, (long long)src.nslices * src.rows, src.cols, src.ld);
    };
    CUtensorMap mt, mb, ml, mr;
    if ((rs = map_of(&mt, top)) != SIGNTRI_OK) return rs;
    if ((rs = map_of(&mb, bot)) != SIGNTRI_OK) return rs;
    if ((rs = map_of(&ml, left)) != SIGNTRI_OK) return rs;
    if ((rs = map_of(&mr, right)) != SIGNTRI_OK) return rs;
    if (top.rows != bot.rows || left.rows != right.rows) return SIGNTRI_ERR_BAD_ARG;
    // resident mode when every pair has the same weight and at most 3 slices
    // per operand are involved (so that a stage of all slices fits twice)
    int nsl = 0;
    bool same_w = true;
    for (int p = 0; p < pairs.n; p++) {
        nsl = std::max(nsl, std::max(pairs.s[p], pairs.t[p]) + 1);
        same_w = same_w && pairs.w[p] == pairs.w[0];
    }
    const int resident = (same_w && pairs.n > 1 && nsl <= 3 && nsl <= top.nslices && nsl <= bot.nslices &&
                          nsl <= left.nslices && nsl <= right.nslices) ? 1 : 0;
    const bool timed = (kernel_class & kProfUntimed) == 0;
    kernel_class &= ~kProfUntimed;
    // grouped pair mode when pairs with unequal weights share A slices
    bool share = false;
    for (int p = 0; p < pairs.n && !share; p++)
        for (int q = p + 1; q < pairs.n && !share; q++) share = pairs.s[p] == pairs.s[q];
    if (!resident && share) {
        if (f16) return SIGNTRI_ERR_BAD_ARG;   // grouped pair mode serves the bf16 exact slices only
        const size_t smem2 = tc_pair2_smem_bytes();
        SGT_CUDA_TRY(cudaFuncSetAttribute(tc_pair2_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem2));
        prof_add_flops(kernel_class, useful_flops);
        ProfScope ps(kernel_class, st, timed);
        tc_pair2_kernel<<<d_job_off ? nctas : njobs, kTcThreads, smem2, st>>>(
            mt, mb, ml, mr, top.rows, left.rows, d_jobs, d_job_off, d_pairs, chunk_kb, top.scale, bot.scale,
            left.scale, right.scale, out, qo, d_err, blk, top.cols / 64);
        SGT_LAUNCH_CHECK();
        return SIGNTRI_OK;
    }
    const size_t smem = tc_smem_bytes();
    SGT_CUDA_TRY(cudaFuncSetAttribute(tc_blocksum_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    prof_add_flops(kernel_class, useful_flops);
    ProfScope ps(kernel_class, st, timed);
    tc_blocksum_kernel<<<d_job_off ? nctas : njobs, kTcThreads, smem, st>>>(
        mt, mb, ml, mr, top.rows, left.rows, d_jobs, d_job_off, d_pairs, chunk_kb, top.scale, bot.scale, left.scale,
        right.scale, out, qo, d_err, resident, nsl, blk, top.cols / 64, f16);
    SGT_LAUNCH_CHECK();
    return SIGNTRI_OK;
}

}  // namespace signtri

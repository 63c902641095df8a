// tc_gemm.cuh -- interface of the tcgen05 block-product engine (tc_gemm.cu).
#pragma once

#include <cuda_bf16.h>

#include "internal.cuh"
#include "tc_job.h"

namespace signtri {

constexpr int kTcMaxPairs = 36;
// K-blocks per unit for exact slice pairs of 8 bits (7 bits): 256 (1024)
// products of magnitude below 2^16 (2^14) sum to less than 2^24, exact in
// the fp32 accumulator
constexpr int kExactChunkKb8 = 4;
constexpr int kExactChunkKb7 = 16;

// Slice pairs (s, t) and their weights (the kernel reads a device copy).
struct TcPairs {
    int n;
    int s[kTcMaxPairs];
    int t[kTcMaxPairs];
    float w[kTcMaxPairs];
};

// A bf16 operand source: nslices matrices of `rows` rows (a multiple of 64,
// zero padded) by `cols` K-contiguous columns, pitch ld elements, stacked;
// optional per-row scale (power of two) applied to the result rows/columns.
// blocked = 1: each matrix is stored as 64 x 64 tiles, tile (row block R,
// K-block K) of slice s contiguous (8 KB, row-major, K fastest) at element
// ((s * rows/64 + R) * cols/64 + K) * 4096; ld is then unused.
// f16 = 1: the 16-bit elements are IEEE fp16 instead of bf16 (all four
// sources of a product have the same type).
struct TcSource {
    const __nv_bfloat16 *base;
    int nslices;
    int rows;
    int cols;
    int ld;
    const float *scale;
    int blocked;
    int f16;
};

// Alternative output: quadrant q of every job written into its own
// column-major matrix m[q] (ld) at rows (q < 2 ? rt : rb) + r and columns
// (q even ? cl : cr) + c (only those below nrows, ncols); m[q] == nullptr
// skips the quadrant.  All four null:
// slot mode (the `out` slabs).
struct TcQuadOut {
    double *m[4];
    int ld;
    int nrows, ncols;   // entries at or beyond these are not written
    size_t slot_stride; // job j writes at m[q] + slot_j * slot_stride (0: no offset)
};

size_t tc_smem_bytes();

// Slice pair lists (slices.cu): exact integer slices of `bits` bits (weights
// 2^{-bits(s+t+2)}) and rounding splits (unit weights), s + t <= S - 1.
TcPairs ozaki_pairs_impl(int S, int bits);
TcPairs split_pairs(int S);
// Row / column slices: exact integer slices of `bits` bits under the
// power-of-two scales when scale != nullptr, else a rounding split.
// skip = 1 (square upper triangular M, consumers whose jobs pair 64-blocks
// 2i, 2i+1): the parts no such job reads are not written.
signtri_status make_row_slices(int m, int k, const double *M, int ldm, int tri, int S, int bits, const float *scale,
                               __nv_bfloat16 *R, int rows_pad, int ldr, cudaStream_t st, int skip = 0);
signtri_status make_col_slices(int k, int n, const double *M, int ldm, int tri, int S, int bits, const float *scale,
                               __nv_bfloat16 *C, int rows_pad, int ldc, cudaStream_t st, int skip = 0);

// Power-of-two row and column scales of the n x n matrix M (tri = 1: its
// strictly upper part) in one pass; tmp_rows, tmp_cols, scale_* hold nout.
signtri_status make_scales_both(int n, const double *M, int ldm, int tri, int nout, unsigned long long *tmp_rows,
                                unsigned long long *tmp_cols, float *scale_rows, float *scale_cols, cudaStream_t st);

// Exact slices of the strictly upper part of the n x n matrix M in a gathered
// index space (inv[g] = original index at position g, -1 = padding, gmap
// its inverse, ng positions used, `rows` allocated, pitch ld; superblock sb
// of `super` original indices at gathered positions [sbbase[sb],
// sbbase[sb+1])): per-row and per-column scales sR, sC (original indices)
// are gathered into sRg, sCg.  Only what a residual job's K range can reach
// is written: row slices from the row's superblock on, column slices up to
// the column's superblock, padding rows zero.
signtri_status make_gathered_slices(int n, const double *M, int ldm, const int *inv, const int *gmap,
                                    const int *sbbase, int super, int ng, int S, int bits, const float *sR,
                                    const float *sC, float *sRg, float *sCg, __nv_bfloat16 *R, __nv_bfloat16 *C,
                                    int rows, int ld, cudaStream_t st);

// d_job_off (device, nctas + 1 entries): CTA b runs jobs [d_job_off[b],
// d_job_off[b+1]) back to back; null: one CTA per job.
signtri_status tc_blocksums(const TcSource &top, const TcSource &bot, const TcSource &left, const TcSource &right,
                            const TcJob *d_jobs, int njobs, const TcPairs &pairs, const TcPairs *d_pairs, int chunk_kb,
                            double *out, const TcQuadOut &qo, int *d_err, int kernel_class, cudaStream_t st,
                            double useful_flops = 0.0, const int *d_job_off = nullptr, int nctas = 0);

// 2 * 64^3 flops per (slice pair, K-block, used quadrant)
inline double tc_flops(int npairs, long long sum_kb, int quadrants)
{
    return 2.0 * 64.0 * 64.0 * 64.0 * (double)npairs * (double)sum_kb * (double)quadrants;
}

}  // namespace signtri

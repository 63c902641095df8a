// tc_gemm.cuh -- interface of the tcgen05 block-product engine (tc_gemm.cu).
#pragma once

#include <cuda_bf16.h>

#include "internal.cuh"

namespace signtri {

constexpr int kTcMaxPairs = 36;

// One CTA's work: rows [rt, rt+64) of the top source and [rb, rb+64) of the
// bottom source form A; rows [cl, cl+64) of the left and [cr, cr+64) of the
// right source form B; K = 64-blocks [kb0, kb1).  The four 64 x 64 quadrants
// of A B^T go to out + slot * 16384 doubles, quadrant q (0 top-left,
// 1 top-right, 2 bottom-left, 3 bottom-right) at + q * 4096, column-major.
struct TcJob {
    int rt, rb, cl, cr;
    int kb0, kb1;
    int slot;
    int pad;
};

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
struct TcSource {
    const __nv_bfloat16 *base;
    int nslices;
    int rows;
    int cols;
    int ld;
    const float *scale;
};

size_t tc_smem_bytes();

signtri_status tc_blocksums(const TcSource &top, const TcSource &bot, const TcSource &left, const TcSource &right,
                            const TcJob *d_jobs, int njobs, const TcPairs &pairs, const TcPairs *d_pairs, int chunk_kb,
                            double *out, int *d_err, int kernel_class, cudaStream_t st);

}  // namespace signtri

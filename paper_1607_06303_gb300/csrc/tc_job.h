// tc_job.h -- one CTA's work item of the tcgen05 block-product engine
// (tc_gemm.cu), shared by the engine and the host code that builds work lists.
#pragma once

namespace signtri {

// One CTA's work: rows [rt, rt+64) of the top source and [rb, rb+64) of the
// bottom source form A; rows [cl, cl+64) of the left and [cr, cr+64) of the
// right source form B; K = 64-blocks [kb0, kb1).  The four 64 x 64 quadrants
// of A B^T go to out + slot * 16384 float2 (hi, lo) pairs, quadrant q
// (0 top-left, 1 top-right, 2 bottom-left, 3 bottom-right) at + q * 4096,
// column-major; the value is hi + lo.
struct TcJob {
    int rt, rb, cl, cr;
    int kb0, kb1;
    int slot;
    int pad;
};

}  // namespace signtri

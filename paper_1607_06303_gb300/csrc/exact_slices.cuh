// exact_slices.cuh -- the error-free split of one float64 value into
// integer slices of b bits under a power-of-two scale (slices.cu describes
// the representation), shared by the slicing kernels and by kernels that
// write the slices of matrices they form themselves (reorder_tc.cu).
#pragma once

namespace signtri {

// Exact slices by integer arithmetic: |x| / scale < 1 written as the 64-bit
// fixed-point integer F = trunc(|x| / scale * 2^64) (from the float64
// significand and exponent, no rounding), digits q_s = bits
// [64 - b(s+1), 64 - bs) of F with the sign of x.  Same digits as repeated
// q_s = trunc(2^b r), r <- 2^b r - q_s, without float64 arithmetic (slow on
// this part).  S b <= 64.
template <int SC>
__device__ __forceinline__ void exact_slices(double x, int scale_exp, int S, int b, float *q)
{
    const unsigned long long bits = (unsigned long long)__double_as_longlong(x);
    const int bexp = (int)((bits >> 52) & 0x7ff);
    unsigned long long F = 0;
    if (bexp != 0) {   // zero and subnormals (far below any scale used here) give 0
        const unsigned long long mant = (bits & 0xfffffffffffffull) | (1ull << 52);
        // |x| = mant * 2^(bexp - 1075); F = |x| * 2^(64 - scale_exp)
        const int sh = bexp - 1075 + 64 - scale_exp;   // <= 11 since |x| < 2^scale_exp
        if (sh >= 0) F = mant << sh;
        else if (sh > -64) F = mant >> (-sh);
    }
    const float sgn = (bits >> 63) ? -1.f : 1.f;
    const unsigned long long mask = (1ull << b) - 1ull;
    const int ns = SC ? SC : S;   // SC > 0: slice count known at compile time (q in registers)
#pragma unroll
    // each digit fits in 32 bits: convert it as a 32-bit integer (a 64-bit
    // integer conversion would issue on the float64 pipe, slow on this part)
    for (int s = 0; s < ns; s++) q[s] = sgn * (float)(unsigned)((F >> (64 - b * (s + 1))) & mask);
}

}  // namespace signtri

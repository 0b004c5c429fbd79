// Float-float arithmetic for the compensated step: every value is an unevaluated
// sum h + l of two FP32 numbers, and every operation is a short sequence of
// correctly rounded FP32 instructions built on the error-free transformations
//   TwoSum   (Knuth, TAOCP vol. 2, Sec. 4.2.2):  s + e = a + b exactly,
//   Fast2Sum (Dekker 1971), for |a| >= |b|:    s + e = a + b exactly,
//   TwoProd  with a fused multiply-add:         p + e = a b exactly,
// combined as in Dekker's double-length arithmetic (the "sloppy" sum: the low
// parts are added with one rounding).  The relative error of a sum or product
// is a few units of 2^-44, against 2^-24 for one FP32 instruction.  The __f*_rn
// intrinsics keep the compiler from contracting or reassociating the sequences.
// Device code only; the collision in d2q9_cell.cuh is instantiated over FF.
#pragma once

#include "d2q9_cell.cuh"

namespace lbm {

__device__ __forceinline__ FF ff(float a) { return FF{a, 0.0f}; }

__device__ __forceinline__ FF two_sum(float a, float b) {
    const float s = __fadd_rn(a, b);
    const float bv = __fsub_rn(s, a);
    const float av = __fsub_rn(s, bv);
    return FF{s, __fadd_rn(__fsub_rn(a, av), __fsub_rn(b, bv))};
}

__device__ __forceinline__ FF fast_two_sum(float a, float b) {
    const float s = __fadd_rn(a, b);
    return FF{s, __fsub_rn(b, __fsub_rn(s, a))};
}

__device__ __forceinline__ FF operator+(FF a, FF b) {
    const FF s = two_sum(a.h, b.h);
    return fast_two_sum(s.h, __fadd_rn(s.l, __fadd_rn(a.l, b.l)));
}
__device__ __forceinline__ FF operator-(FF a, FF b) { return a + FF{-b.h, -b.l}; }

__device__ __forceinline__ FF mul(FF a, FF b) {
    const float p = __fmul_rn(a.h, b.h);
    const float e = __fmaf_rn(a.h, b.h, -p);  // the product's rounding error, exactly
    return fast_two_sum(p, __fmaf_rn(a.h, b.l, __fmaf_rn(a.l, b.h, e)));
}
__device__ __forceinline__ FF fmadd(FF a, FF b, FF c) { return mul(a, b) + c; }

template <>
__device__ __forceinline__ FF lit<FF>(float c) {
    return ff(c);
}

// 1/x: the correctly rounded FP32 reciprocal of the high part, then one Newton
// step r + r (1 - x r) in float-float (doubles the correct bits).
__device__ __forceinline__ FF rcp_eq(FF x) {
    const FF r = ff(__frcp_rn(x.h));
    return r + mul(r, ff(1.0f) - mul(x, r));
}

// The stored FP32 population: h + l rounded once.
__device__ __forceinline__ float ff_round(FF a) { return __fadd_rn(a.h, a.l); }

}  // namespace lbm

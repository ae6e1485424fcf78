// ff.cuh -- float-float ("double-single") arithmetic for the dependency accumulation.
//
// GB300 executes fp64 at a small fraction of its fp32 rate, so the dependencies
// delta_s.(v) (Eq. 4) are carried as unevaluated sums hi + lo of two fp32 numbers
// (Dekker, "A floating-point technique for extending the available precision", 1971;
// Knuth TAOCP vol. 2, 4.2.2).  Every operand on this path is non-negative (path
// counts, dependencies, their ratios), so the sums below do not cancel and each
// operation keeps a relative error of a few units of 2^-46; the accumulation of one
// source chains at most a few hundred of them.  The exponent range of fp32 covers
// sigma up to 2^64 and its reciprocal.
#pragma once

#include <cstdint>

namespace bcg {

struct __align__(8) ff {
    float hi, lo;
};

// s + e == a + b exactly (Knuth's TwoSum, no ordering assumption).
__device__ __forceinline__ ff two_sum(float a, float b) {
    const float s = a + b;
    const float bb = s - a;
    const float e = (a - (s - bb)) + (b - bb);
    return {s, e};
}

// s + e == a + b exactly when |a| >= |b| (Dekker's Fast2Sum).
__device__ __forceinline__ ff fast_two_sum(float a, float b) {
    const float s = a + b;
    return {s, b - (s - a)};
}

// p + e == a * b exactly (one fma).
__device__ __forceinline__ ff two_prod(float a, float b) {
    const float p = a * b;
    return {p, fmaf(a, b, -p)};
}

__device__ __forceinline__ ff ff_add(ff x, ff y) {
    ff s = two_sum(x.hi, y.hi);
    s.lo += x.lo + y.lo;
    return fast_two_sum(s.hi, s.lo);
}

__device__ __forceinline__ ff ff_mul(ff x, ff y) {
    ff p = two_prod(x.hi, y.hi);
    p.lo = fmaf(x.hi, y.lo, fmaf(x.lo, y.hi, p.lo));
    return fast_two_sum(p.hi, p.lo);
}

__device__ __forceinline__ ff ff_shfl_xor(ff x, int o) {
    return {__shfl_xor_sync(0xffffffffu, x.hi, o), __shfl_xor_sync(0xffffffffu, x.lo, o)};
}

// A path count as a float-float: the value is cut into 20 + 22 + 22 bits, each of which
// converts to fp32 exactly, and the three are summed (exact up to 48 significant bits,
// rounded in the low part beyond that).  A count below 2^24 is one exact fp32 value,
// which is also what the three-part sum gives for it.
__device__ __forceinline__ ff ff_from_u64(uint64_t v) {
    if (v < (1ull << 24)) return ff{__uint2float_rn((uint32_t)v), 0.0f};
    const float c2 = __uint2float_rn((uint32_t)(v >> 44)) * 17592186044416.0f;          // 2^44
    const float c1 = __uint2float_rn((uint32_t)(v >> 22) & 0x3FFFFFu) * 4194304.0f;    // 2^22
    const float c0 = __uint2float_rn((uint32_t)v & 0x3FFFFFu);
    const ff x = two_sum(c2, c1);
    return ff_add(x, ff{c0, 0.0f});
}

// 1 / x for x >= 1: fp32 reciprocal refined by one Newton step in float-float,
// r = r0 + r0 * (1 - x * r0).
__device__ __forceinline__ ff ff_rcp(ff x) {
    const float r0 = __frcp_rn(x.hi);
    ff e = ff_mul(x, ff{r0, 0.0f});                // ~ 1
    ff one_minus = two_sum(1.0f, -e.hi);          // 1 - e, exact in the leading part
    one_minus.lo -= e.lo;
    const float corr = r0 * (one_minus.hi + one_minus.lo);
    return fast_two_sum(r0, corr);
}

// Host-side value of a float-float pair.
__host__ __device__ __forceinline__ double ff_to_double(ff x) { return (double)x.hi + (double)x.lo; }

}  // namespace bcg

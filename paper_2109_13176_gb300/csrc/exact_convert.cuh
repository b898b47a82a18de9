// Exact IEEE-754 conversions done with integer operations on the bit
// fields, so that the per-point pass spends its FP64 pipe (GB300 runs FP64
// at 1/64 of FP32) on the transform's fused multiply-adds only. Each gives
// the same result as the correctly rounded conversion it replaces
// (binary32 <-> binary64 widening is exact; narrowing and integer
// conversion round to nearest, ties to even); cases outside the fast
// paths (subnormal results, zero, out of range) use the hardware
// conversion. gvom_selftest_conversions compares them with CUDA's own.
#pragma once

#include <stdint.h>

namespace gvom {

// float -> double, exact: the sign moves up, the exponent is rebased from
// bias 127 to 1023, the 23-bit fraction is shifted into the top of the 52-bit
// one. Zero and subnormal floats go to the hardware.
__device__ __forceinline__ double f2d_exact(float f) {
    const uint32_t b = __float_as_uint(f);
    const uint32_t e = (b >> 23) & 0xffu;
    if (e == 0u || e == 0xffu) return (double)f;
    const unsigned long long d = ((unsigned long long)(b & 0x80000000u) << 32) |
                                 ((unsigned long long)(e + 896u) << 52) |
                                 ((unsigned long long)(b & 0x7fffffu) << 29);
    return __longlong_as_double((long long)d);
}

// double -> int, round to nearest, ties to even, for |s| < 2^30: the 53-bit
// significand shifted right by 52 - exponent, rounded up when the bits
// shifted out exceed half a unit, or equal it with an odd result.
__device__ __forceinline__ int d2i_rne(double s) {
    const unsigned long long b = (unsigned long long)__double_as_longlong(s);
    const int e = (int)((b >> 52) & 0x7ffu) - 1023;
    if (e < -1) return 0;  // |s| < 0.5 (zero included)
    const unsigned long long m = (b & 0xfffffffffffffull) | (1ull << 52);
    const int sh = 52 - e;  // 23 <= sh <= 53 for 0.5 <= |s| < 2^30
    unsigned long long q = m >> sh;
    const unsigned long long r = m & ((1ull << sh) - 1ull);
    const unsigned long long half = 1ull << (sh - 1);
    q += (r > half || (r == half && (q & 1ull))) ? 1ull : 0ull;
    const int qi = (int)q;
    return (b >> 63) ? -qi : qi;
}

// double -> float, round to nearest, ties to even, for results in the
// normal float range: the 52-bit fraction rounded to 23 bits; a carry out of
// the fraction runs into the exponent field, which is the correct result
// (and infinity past the largest float). Zero, subnormal and out-of-range
// results go to the hardware.
__device__ __forceinline__ float d2f_rne(double d) {
    const unsigned long long b = (unsigned long long)__double_as_longlong(d);
    const int e = (int)((b >> 52) & 0x7ffu) - 1023;
    if (e < -126 || e > 127) return __double2float_rn(d);
    const unsigned long long frac = b & 0xfffffffffffffull;
    const uint32_t m = (uint32_t)(frac >> 29);
    const unsigned long long r = frac & ((1ull << 29) - 1ull);
    uint32_t fb = ((uint32_t)(e + 127) << 23) + m;
    fb += (r > (1ull << 28) || (r == (1ull << 28) && (m & 1u))) ? 1u : 0u;
    fb |= (uint32_t)(b >> 32) & 0x80000000u;
    return __uint_as_float(fb);
}

}  // namespace gvom

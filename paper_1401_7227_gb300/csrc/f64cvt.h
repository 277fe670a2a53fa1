// Double-to-float rounding (round to nearest, ties to even) on integer operations.
//
// On this GPU a double-to-float conversion instruction runs on the FP64 unit, which retires one
// warp instruction per ~64 cycles per SM sub-partition; the restriction of a residual into FP32
// local vectors converts three values per row and was bound by it.  The bit manipulation below
// runs on the integer pipes instead and gives the same float for every double of magnitude in
// [2^-126, 2^128), the binary32 normal exponents.  The caller converts the other values (zero,
// smaller magnitudes, larger ones, infinities, NaN) with the conversion instruction.
#pragma once

#if defined(__CUDACC__)
#define ASM2_HD __host__ __device__ __forceinline__
#else
#define ASM2_HD inline
#endif

namespace asm2 {

// hi, lo: the upper and lower 32 bits of an IEEE-754 binary64 value.  Returns false (out
// untouched) unless its magnitude lies in [2^-126, 2^128); otherwise out = the bits of the
// binary32 value rounded to nearest, ties to even (infinity where that rounds past the largest
// float).
ASM2_HD bool f64_to_f32_bits(unsigned hi, unsigned lo, unsigned& out) {
    const unsigned e = (hi >> 20) & 0x7FFu;  // biased binary64 exponent
    // binary32 exponent e - 1023 + 127 must lie in [1, 254]: e in [897, 1150]
    if (e - 897u > 253u) return false;
    // rebias the exponent field in place (it stays within 8 bits), then shift exponent and the top
    // 20 mantissa bits up by 3 and append the next 3 mantissa bits: 8 exponent + 23 mantissa bits
    const unsigned mag = (((hi & 0x7FFFFFFFu) - (896u << 20)) << 3) | (lo >> 29);
    // the 29 dropped bits: round up above half, and at exactly half when the kept bits are odd;
    // a carry out of the mantissa moves into the exponent (and to infinity past the largest float)
    const unsigned rest = lo & 0x1FFFFFFFu;
    const unsigned up = (rest > 0x10000000u || (rest == 0x10000000u && (mag & 1u))) ? 1u : 0u;
    out = (hi & 0x80000000u) | (mag + up);
    return true;
}

#if defined(__CUDACC__)
// the conversion instruction, out of line: a call is a branch, so lanes that take the integer
// path do not execute it (inlined, the compiler may predicate it on every lane)
__device__ __noinline__ float f64_to_f32_instruction(double d) { return __double2float_rn(d); }

__device__ __forceinline__ float f64_to_f32(double d) {
    const unsigned long long b = (unsigned long long)__double_as_longlong(d);
    unsigned f;
    if (f64_to_f32_bits((unsigned)(b >> 32), (unsigned)b, f)) return __uint_as_float(f);
    return f64_to_f32_instruction(d);
}
#endif

}  // namespace asm2

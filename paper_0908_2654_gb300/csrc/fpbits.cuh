// FP64 <-> FP32 conversion with a power-of-two scale, done on the IEEE-754 bit patterns with
// integer operations.  The multigrid's FP32 right side is r 2^-e and its FP64 result z 2^e, with
// 2^e >= max|r| so that the FP32 copy neither overflows nor underflows; the conversions touch
// every cell twice per V-cycle, and on this GPU FP64 arithmetic (a multiply, a conversion)
// issues at a small fraction of the integer rate, which made the casts FP64-bound.
//
// Formats (IEEE 754 binary64 / binary32): sign, biased exponent (11 / 8 bits, bias 1023 / 127),
// fraction (52 / 23 bits).  Scaling by 2^-e subtracts e from the exponent.  The FP64 -> FP32
// fraction is rounded to nearest, ties away from zero (a carry out of the fraction bumps the
// exponent, which is the correctly rounded result); results below the FP32 normal range, and
// FP64 subnormal inputs, are flushed to zero, which for a preconditioner's input relative to
// max|r| ~ 1 is a change below 2^-126 of the largest entry.  Widening is exact where the result
// is a normal FP64 number and gives zero below.  Non-finite inputs stay non-finite.
#pragma once
#include <cstdint>
#include <cstring>
#include <cuda_runtime.h>

#ifndef RT_HD
#define RT_HD __host__ __device__ __forceinline__
#endif

namespace fpbits {

RT_HD uint64_t bits64(double v) {
#ifdef __CUDA_ARCH__
    return (uint64_t)__double_as_longlong(v);
#else
    uint64_t b;
    std::memcpy(&b, &v, 8);
    return b;
#endif
}
RT_HD double from_bits64(uint64_t b) {
#ifdef __CUDA_ARCH__
    return __longlong_as_double((long long)b);
#else
    double v;
    std::memcpy(&v, &b, 8);
    return v;
#endif
}
RT_HD uint32_t bits32(float v) {
#ifdef __CUDA_ARCH__
    return (uint32_t)__float_as_uint(v);
#else
    uint32_t b;
    std::memcpy(&b, &v, 4);
    return b;
#endif
}
RT_HD float from_bits32(uint32_t b) {
#ifdef __CUDA_ARCH__
    return __uint_as_float(b);
#else
    float v;
    std::memcpy(&v, &b, 4);
    return v;
#endif
}

// e with max|r| = amax < 2^e for a positive finite normal amax (as frexp gives it); 0 otherwise
RT_HD int pow2_exponent(double amax) {
    const uint64_t b = bits64(amax);
    const int E = (int)((b >> 52) & 0x7ff);
    if ((b >> 63) || E == 0 || E == 0x7ff) return 0;
    return E - 1022;
}

// v 2^-e rounded to FP32
RT_HD float to_float_scaled(double v, int e) {
    const uint64_t b = bits64(v);
    const uint32_t sign = (uint32_t)(b >> 32) & 0x80000000u;
    const int E = (int)((b >> 52) & 0x7ff);
    if (E == 0x7ff) return from_bits32(sign | 0x7f800000u | ((b & 0xfffffffffffffULL) ? 0x400000u : 0u));
    const int Ef = E - 1023 + 127 - e;
    if (E == 0 || Ef <= 0) return from_bits32(sign);
    if (Ef >= 255) return from_bits32(sign | 0x7f800000u);
    const uint32_t frac = (uint32_t)(((b & 0xfffffffffffffULL) + (1ULL << 28)) >> 29);   // up to 2^23
    const uint32_t mag = ((uint32_t)Ef << 23) + frac;   // a carry rounds up into the exponent
    return from_bits32(sign | (mag >= 0x7f800000u ? 0x7f800000u : mag));
}

// f 2^e as FP64 (exact for normal f; FP32 subnormals, below 2^-126, give 0)
RT_HD double from_float_scaled(float f, int e) {
    const uint32_t b = bits32(f);
    const uint64_t sign = (uint64_t)(b & 0x80000000u) << 32;
    const int E = (int)((b >> 23) & 0xff);
    if (E == 0xff) return from_bits64(sign | 0x7ff0000000000000ULL | ((b & 0x7fffffu) ? (1ULL << 51) : 0ULL));
    const int Ed = E - 127 + 1023 + e;
    if (E == 0 || Ed <= 0) return from_bits64(sign);
    if (Ed >= 0x7ff) return from_bits64(sign | 0x7ff0000000000000ULL);
    return from_bits64(sign | ((uint64_t)Ed << 52) | ((uint64_t)(b & 0x7fffffu) << 29));
}

}  // namespace fpbits

// Conversions between binary32 and binary64 on the integer pipes.
//
// GB300's FP64 pipe is narrow, and the hardware conversions between float and double run
// on it: a warp-wide conversion occupies it as long as a warp-wide FP64 add. The FP32-mixed
// pass kernel converts every sample of an IMF commit (the IMF into the FP64 residue update,
// the new residue back to the working precision), so these conversions are done here with
// integer operations on the IEEE 754 bit layouts instead:
//   binary32: sign(1) exponent(8, bias 127) fraction(23)
//   binary64: sign(1) exponent(11, bias 1023) fraction(52)
// Both functions return exactly what the IEEE conversions return (widening is exact;
// narrowing rounds to nearest, ties to even, and overflows to infinity). Normal numbers and
// zeros take the integer path; subnormals, infinities and NaNs take the hardware conversion.
// The functions are host-callable too, so that a CPU test can check them against the host's
// IEEE conversions.
#pragma once
#include <cstdint>
#include <cstring>
#include <cuda_runtime.h>

namespace semd {

__host__ __device__ __forceinline__ uint32_t bits_of(float f)
{
#ifdef __CUDA_ARCH__
    return __float_as_uint(f);
#else
    uint32_t u;
    std::memcpy(&u, &f, 4);
    return u;
#endif
}
__host__ __device__ __forceinline__ float float_of(uint32_t u)
{
#ifdef __CUDA_ARCH__
    return __uint_as_float(u);
#else
    float f;
    std::memcpy(&f, &u, 4);
    return f;
#endif
}
__host__ __device__ __forceinline__ void words_of(double d, uint32_t &hi, uint32_t &lo)
{
#ifdef __CUDA_ARCH__
    hi = (uint32_t)__double2hiint(d);
    lo = (uint32_t)__double2loint(d);
#else
    uint64_t u;
    std::memcpy(&u, &d, 8);
    hi = (uint32_t)(u >> 32);
    lo = (uint32_t)u;
#endif
}
__host__ __device__ __forceinline__ double double_of(uint32_t hi, uint32_t lo)
{
#ifdef __CUDA_ARCH__
    return __hiloint2double((int)hi, (int)lo);
#else
    const uint64_t u = ((uint64_t)hi << 32) | lo;
    double d;
    std::memcpy(&d, &u, 8);
    return d;
#endif
}

// float -> double. A normal binary32 number with exponent field e (1..254) has the
// binary64 exponent field e + 896 and its fraction moved up by 29 bits; in the high word
// that is (magnitude bits >> 3) + (896 << 20).
__host__ __device__ __forceinline__ double widen(float f)
{
    const uint32_t u = bits_of(f), a = u & 0x7fffffffu, s = u & 0x80000000u;
    if (a - 0x00800000u < 0x7f000000u)
        return double_of(s | ((a >> 3) + 0x38000000u), a << 29);
    if (a == 0u)
        return double_of(s, 0u);
    return (double)f;
}
__host__ __device__ __forceinline__ double widen(double d) { return d; }

// double -> float, round to nearest even. Binary64 exponent fields 897..1150 give normal
// binary32 results: the exponent field drops by 896, the fraction keeps its top 23 bits,
// and the 29 bits below decide the rounding (above half: up; exactly half: to even). A
// carry out of the fraction increments the exponent, up to infinity, as IEEE rounding does.
__host__ __device__ __forceinline__ float narrow_float(double d)
{
    uint32_t hi, lo;
    words_of(d, hi, lo);
    const uint32_t ah = hi & 0x7fffffffu, s = hi & 0x80000000u;
    if (ah - 0x38100000u < 0x0fe00000u) {
        const uint32_t b = ((ah - 0x38000000u) << 3) | (lo >> 29);
        const uint32_t rem = lo & 0x1fffffffu;
        const uint32_t up = (uint32_t)(rem > 0x10000000u) | ((uint32_t)(rem == 0x10000000u) & b);
        return float_of(s | (b + up));
    }
    if ((ah | lo) == 0u)
        return float_of(s);
    return (float)d;
}

// The working precision R from a double: narrow_float for float, identity for double.
__host__ __device__ __forceinline__ void narrow_to(double d, float &out) { out = narrow_float(d); }
__host__ __device__ __forceinline__ void narrow_to(double d, double &out) { out = d; }

} // namespace semd

// devmath.cuh -- device helpers shared by the CUDA translation units.
#pragma once
#include <cuda_runtime.h>

namespace ilves {

// float64 -> float32 by truncation, on the integer pipe.  Values below float's normal
// range become signed zero, values above it (never nm-scale coordinates) infinity.
__device__ __forceinline__ float narrow(double v) {
    const unsigned long long b = (unsigned long long)__double_as_longlong(v);
    const unsigned hi = (unsigned)(b >> 32), lo = (unsigned)b;
    const unsigned sign = hi & 0x80000000u;
    const int e = (int)((hi >> 20) & 0x7FFu) - 896;  // rebias 1023 -> 127
    unsigned r = sign | ((unsigned)e << 23) | ((hi & 0xFFFFFu) << 3) | (lo >> 29);
    r = e <= 0 ? sign : r;
    r = e >= 255 ? (sign | 0x7F800000u) : r;
    return __uint_as_float(r);
}

// float32 -> float64, exact, on the integer pipe (subnormal floats flush to zero).
__device__ __forceinline__ double widen(float f) {
    const unsigned b = __float_as_uint(f);
    const unsigned sign = b & 0x80000000u;
    const unsigned e = (b >> 23) & 0xFFu;
    const unsigned mant = b & 0x7FFFFFu;
    unsigned hi = sign | ((e + 896u) << 20) | (mant >> 3);
    unsigned lo = mant << 29;
    hi = e == 0 ? sign : hi;
    lo = e == 0 ? 0u : lo;
    hi = e == 255 ? (sign | 0x7FF00000u | (mant >> 3)) : hi;
    return __hiloint2double((int)hi, (int)lo);
}

}  // namespace ilves

// Integer digit slicing shared by the exact (Ozaki-scheme) products: powers
// of two, rint(v 2^sc) from the IEEE-754 fields in integer arithmetic, and
// balanced base-2^GP_OZ_BITS digits of the resulting integer.
#pragma once
#include <cuda_bf16.h>
#include <math.h>
#include <stdint.h>

#include "gp_internal.cuh"

namespace gpk {

__device__ __forceinline__ double pow2_ceil(double x)   // smallest power of two >= x (x > 0)
{
    int e;
    double f = frexp(x, &e);   // x = f 2^e, f in [0.5, 1)
    return (f == 0.5) ? ldexp(1.0, e - 1) : ldexp(1.0, e);
}

// Binary exponent of a power of two (a normal double).
__device__ __forceinline__ int pow2_exp(double p) { return (int)((__double_as_longlong(p) >> 52) & 0x7ff) - 1023; }

// rint(mant 2^(e2 + sc)) with the sign neg, in integer arithmetic: round half
// to even, as rint in the default rounding mode; exact whenever the result is
// below 2^62.  No FP64 instruction is involved.
__device__ __forceinline__ long long rint_scaled_bits(unsigned long long mant, int e2, bool neg, int sc)
{
    const int s = -(e2 + sc);   // right shift of the significand
    unsigned long long q;
    if (mant == 0 || s >= 64) {
        q = 0;
    } else if (s <= 0) {
        q = mant << (-s);
    } else {
        q = mant >> s;
        const unsigned long long rem = mant & ((1ull << s) - 1), half = 1ull << (s - 1);
        q += (rem > half || (rem == half && (q & 1ull))) ? 1ull : 0ull;
    }
    return neg ? -(long long)q : (long long)q;
}

// rint(v 2^sc) from the IEEE-754 fields of v (v = mant 2^e2, subnormals included).
__device__ __forceinline__ long long rint_scaled(double v, int sc)
{
    const unsigned long long u = (unsigned long long)__double_as_longlong(v);
    const int ex = (int)((u >> 52) & 0x7ff);
    unsigned long long m = u & 0xfffffffffffffull;
    if (ex) m |= 1ull << 52;
    return rint_scaled_bits(m, (ex ? ex : 1) - 1075, (u >> 63) != 0, sc);
}

__device__ __forceinline__ long long rint_scaled(float v, int sc)
{
    const unsigned u = __float_as_uint(v);
    const int ex = (int)((u >> 23) & 0xff);
    unsigned long long m = u & 0x7fffffu;
    if (ex) m |= 1ull << 23;
    return rint_scaled_bits(m, (ex ? ex : 1) - 150, (u >> 31) != 0, sc);
}

// Balanced base-2^GP_OZ_BITS digits of a in [-1, 1] given q = rint(a 2^(GP_OZ_BITS S))
// (exact in a 64-bit integer): d_s = q rounded to a multiple of
// 2^(GP_OZ_BITS (S - s)) and removed from q, most significant first, so that
// a ~ sum_s d_s 2^{-GP_OZ_BITS s} with |d_1| <= 2^GP_OZ_BITS, |d_s| <= 2^(GP_OZ_BITS - 1) for
// s > 1, the error at most 2^{-GP_OZ_BITS S - 1}; the digits of q itself are exact.
template <int S>
__device__ __forceinline__ void oz_digits(long long q, __nv_bfloat16 (&d)[S])
{
#pragma unroll
    for (int s = 0; s < S; ++s) {
        const int sh = GP_OZ_BITS * (S - 1 - s);
        const long long dg = sh > 0 ? ((q + (1ll << (sh - 1))) >> sh) : q;
        q -= dg * (1ll << sh);
        d[s] = __int2bfloat16_rn((int)dg);
    }
}

}  // namespace gpk

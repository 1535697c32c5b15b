// bits.cuh -- float64 conversions done on bit patterns with integer
// operations.  On this GPU the float64 pipe is narrow and it also runs the
// float64 conversions (to and from integers and float32), so the hot kernels
// that only need a value's bits rearranged build them here instead.  Every
// function is exact or reproduces the conversion it replaces bit for bit, and
// compiles for the host too, so a host program can check it against exact
// arithmetic.
#pragma once

#include <stdint.h>
#include <string.h>

namespace hts {

__host__ __device__ __forceinline__ unsigned long long bits_of(double x)
{
#ifdef __CUDA_ARCH__
    return (unsigned long long)__double_as_longlong(x);
#else
    unsigned long long b;
    memcpy(&b, &x, sizeof b);
    return b;
#endif
}

__host__ __device__ __forceinline__ double double_of(unsigned long long b)
{
#ifdef __CUDA_ARCH__
    return __longlong_as_double((long long)b);
#else
    double x;
    memcpy(&x, &b, sizeof x);
    return x;
#endif
}

__host__ __device__ __forceinline__ float float_of(unsigned b)
{
#ifdef __CUDA_ARCH__
    return __uint_as_float(b);
#else
    float x;
    memcpy(&x, &b, sizeof x);
    return x;
#endif
}

// int to float32, rounded to nearest (ties to even)
__host__ __device__ __forceinline__ float int_to_float_rn(int v)
{
#ifdef __CUDA_ARCH__
    return __int2float_rn(v);
#else
    return (float)v;  // the host's default rounding: to nearest, ties to even
#endif
}

__host__ __device__ __forceinline__ int clz64(unsigned long long v)
{
#ifdef __CUDA_ARCH__
    return __clzll((long long)v);
#else
    return __builtin_clzll(v);
#endif
}

// hi = c rounded to float32 (to nearest, ties to even) and lo = c - hi rounded
// to float32: the same values as the two conversions, taken from the bit
// pattern of c.  |c| in [2^-60, 2^100): lo is then a normal float and exact up
// to its rounding; other values (zero included) take the conversions.
__host__ __device__ __forceinline__ void split_f32(double c, float &hi, float &lo)
{
    const unsigned long long b = bits_of(c);
    const int ex = (int)((b >> 52) & 0x7ff);
    if (ex < 1023 - 60 || ex >= 1023 + 100) {
        hi = (float)c;
        lo = (float)(c - (double)hi);
        return;
    }
    const unsigned long long S = (b & ((1ull << 52) - 1ull)) | (1ull << 52);  // 53-bit significand
    unsigned long long h = S >> 29;                                            // top 24 bits
    const unsigned long long r = S & ((1ull << 29) - 1ull);
    if (r > (1ull << 28) || (r == (1ull << 28) && (h & 1ull))) ++h;           // to nearest, ties to even
    const int rem = (int)((long long)S - (long long)(h << 29));                // c - hi in units of 2^(ex - 1075)
    int e = ex;
    if (h == (1ull << 24)) {  // rounded up into the next binade
        h >>= 1;
        ++e;
    }
    const unsigned sgn = (unsigned)(b >> 63) << 31;
    hi = float_of(sgn | ((unsigned)(e - 1023 + 127) << 23) | ((unsigned)h & 0x7fffffu));
    const float unit = float_of((unsigned)(ex - 1075 + 127) << 23);  // 2^(ex - 1075), normal
    lo = int_to_float_rn(sgn ? -rem : rem) * unit;  // |rem| <= 2^28; exact scaling (+0 when c = hi)
}

// floor(u 2^levels) clamped to [0, 2^levels - 1] (negative and NaN -> 0,
// +inf -> the top); 1 <= levels <= 52.
__host__ __device__ __forceinline__ uint64_t quantise_unit(double u, int levels)
{
    const unsigned long long b = bits_of(u);
    const uint64_t top = (1ull << levels) - 1;
    const int ex = (int)((b >> 52) & 0x7ff);
    const unsigned long long mant = b & ((1ull << 52) - 1ull);
    if (ex == 0x7ff) return (mant || (b >> 63)) ? 0ull : top;  // NaN, -inf; +inf
    if (b >> 63) return 0ull;                                   // negative, -0
    if (ex >= 1023) return top;                                 // u >= 1
    const unsigned long long S = ex ? mant | (1ull << 52) : mant;
    const int shift = 1075 - levels - (ex ? ex : 1);            // u 2^levels = S 2^-shift, shift > 0
    return shift >= 64 ? 0ull : S >> shift;
}

// floor(x 2^E) as a 128-bit integer (exact; x finite, |x| 2^E < 2^125): the
// significand shifted into place.
__host__ __device__ __forceinline__ __int128 fixed_from_double(double x, int E)
{
    const unsigned long long b = bits_of(x);
    const int ex = (int)((b >> 52) & 0x7ff);
    unsigned long long m = b & ((1ull << 52) - 1ull);
    if (ex) m |= 1ull << 52;
    if (m == 0ull) return 0;
    const int sh = (ex ? ex : 1) - 1075 + E;  // |x| 2^E = m 2^sh
    unsigned __int128 mag;
    bool frac = false;                        // bits below 2^0 dropped
    if (sh >= 0) {
        mag = (unsigned __int128)m << sh;
    } else if (sh > -64) {
        mag = m >> (-sh);
        frac = (m & ((1ull << (-sh)) - 1ull)) != 0ull;
    } else {
        mag = 0;
        frac = true;
    }
    if (!(b >> 63)) return (__int128)mag;
    return -(__int128)(mag + (frac ? 1u : 0u));  // floor of a negative value
}

// |v| truncated to 53 significant bits, as a float64 with the sign of v (no
// scaling: the value is the integer itself).
__host__ __device__ __forceinline__ double fixed_to_double_trunc(__int128 v)
{
    const bool neg = v < 0;
    const unsigned __int128 m = neg ? (unsigned __int128)0 - (unsigned __int128)v : (unsigned __int128)v;
    const unsigned long long hi = (unsigned long long)(m >> 64), lo = (unsigned long long)m;
    if ((hi | lo) == 0ull) return 0.0;
    const int top = hi ? 127 - clz64(hi) : 63 - clz64(lo);  // leading one
    const unsigned long long mant =
        (top >= 52 ? (unsigned long long)(m >> (top - 52)) : lo << (52 - top)) & ((1ull << 52) - 1ull);
    return double_of(((unsigned long long)(top + 1023) << 52) | mant | (neg ? 1ull << 63 : 0ull));
}

}  // namespace hts

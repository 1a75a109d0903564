// Conversions between IEEE 754 binary64 and binary32 written with integer operations on the
// encodings, for kernels that move complex128 state to complex64 Krylov vectors and back.  On
// GPUs whose FP64 units run at a small fraction of the FP32 rate the conversion instructions
// themselves use those units; these versions use the integer pipes.  Both follow the IEEE 754
// definitions directly:
//   f2d_exact:  binary32 -> binary64, exact (every binary32 value is a binary64 value), NaN
//               payloads kept and NaNs quietened.
//   d2f_rn:     binary64 -> binary32, round to nearest with ties to even, overflow to infinity,
//               gradual underflow to subnormals and zero, NaN quietened with its top payload bits.
//   d2f_split:  hi = d2f_rn(x) and lo ~ x - hi (to about 2^-24 relative to lo), for norms
//               accumulated in FP32 pairs; false when x lies outside [2^-74, 2^100) in magnitude
//               (and is not 0), where lo would leave the binary32 normal range and the caller
//               takes the FP64 path.
// Plain C++ on the host (bit copies through memcpy), so that the conversions can be checked
// against the host's own on any number of inputs.
#pragma once

#include <stdint.h>
#ifndef __CUDACC__
#include <string.h>
#endif

#if defined(__CUDACC__)
#define HX_CONV_HD __host__ __device__ __forceinline__
#else
#define HX_CONV_HD inline
#endif

namespace hx {

HX_CONV_HD uint64_t conv_bits64(double x)
{
#if defined(__CUDA_ARCH__)
    return (uint64_t)__double_as_longlong(x);
#else
    uint64_t b;
    memcpy(&b, &x, 8);
    return b;
#endif
}

HX_CONV_HD double conv_from_bits64(uint64_t b)
{
#if defined(__CUDA_ARCH__)
    return __longlong_as_double((long long)b);
#else
    double x;
    memcpy(&x, &b, 8);
    return x;
#endif
}

HX_CONV_HD uint32_t conv_bits32(float x)
{
#if defined(__CUDA_ARCH__)
    return __float_as_uint(x);
#else
    uint32_t b;
    memcpy(&b, &x, 4);
    return b;
#endif
}

HX_CONV_HD float conv_from_bits32(uint32_t b)
{
#if defined(__CUDA_ARCH__)
    return __uint_as_float(b);
#else
    float x;
    memcpy(&x, &b, 4);
    return x;
#endif
}

HX_CONV_HD int conv_leading_one(uint32_t a)   // index of the highest set bit of a != 0
{
#if defined(__CUDA_ARCH__)
    return 31 - __clz((int)a);
#else
    int p = 31;
    while (!(a >> p)) --p;
    return p;
#endif
}

// binary32 -> binary64 (exact).
HX_CONV_HD double f2d_exact(float f)
{
    const uint32_t u = conv_bits32(f);
    const uint32_t sign = u & 0x80000000u, a = u & 0x7fffffffu;
    uint32_t hi, lo;
    if (a - 0x00800000u < 0x7f000000u) {          // normal: rebias the exponent by 1023 - 127
        hi = sign | ((a >> 3) + (896u << 20));
        lo = a << 29;
    } else if (a >= 0x7f800000u) {                 // infinity or NaN (quietened)
        hi = sign | 0x7ff00000u | ((a & 0x7fffffu) >> 3) | (a > 0x7f800000u ? 0x80000u : 0u);
        lo = a << 29;
    } else if (a == 0) {
        hi = sign;
        lo = 0;
    } else {                                       // subnormal: a * 2^-149 with the leading one at bit p
        const int p = conv_leading_one(a);
        const uint64_t m = (uint64_t)(a & ((1u << p) - 1)) << (52 - p);
        const uint64_t b = ((uint64_t)sign << 32) | ((uint64_t)(p + 874) << 52) | m;
        return conv_from_bits64(b);
    }
    return conv_from_bits64(((uint64_t)hi << 32) | lo);
}

// binary64 -> binary32, round to nearest, ties to even.
HX_CONV_HD float d2f_rn(double x)
{
    const uint64_t b = conv_bits64(x);
    const uint32_t hi = (uint32_t)(b >> 32), lo = (uint32_t)b;
    const uint32_t sign = hi & 0x80000000u, ah = hi & 0x7fffffffu;
    const uint32_t e = ah >> 20;                   // biased binary64 exponent
    if (e - 897u < 254u) {                         // binary32 normal range: 2^-126 <= |x| < 2^128
        uint32_t out = sign | ((ah - (896u << 20)) << 3) | (lo >> 29);
        const uint32_t rem = lo & 0x1fffffffu;     // the 29 bits that are dropped
        out += (rem > 0x10000000u || (rem == 0x10000000u && (out & 1u))) ? 1u : 0u;   // may carry to infinity
        return conv_from_bits32(out);
    }
    if (e == 0x7ffu) {                             // infinity or NaN
        const uint64_t m = b & 0xfffffffffffffull;
        return conv_from_bits32(sign | 0x7f800000u | (m ? 0x400000u | (uint32_t)(m >> 29) : 0u));
    }
    if (e >= 897u) return conv_from_bits32(sign | 0x7f800000u);   // |x| >= 2^128
    if (e == 0) return conv_from_bits32(sign);                    // |x| < 2^-1022
    // binary32 subnormal: q = |x| / 2^-149 = full * 2^(E + 97), E = e - 1023 <= -127
    const uint64_t full = (b & 0xfffffffffffffull) | (1ull << 52);
    const int s = 1023 - 97 - (int)e;              // right shift, >= 30
    if (s > 54) return conv_from_bits32(sign);     // below half the smallest subnormal
    uint64_t q = full >> s;
    const uint64_t rem = full & ((1ull << s) - 1), half = 1ull << (s - 1);
    q += (rem > half || (rem == half && (q & 1u))) ? 1u : 0u;
    return conv_from_bits32(sign | (uint32_t)q);
}

// hi = d2f_rn(x), lo ~ x - hi.  Returns false (hi and lo unset) outside 2^-74 <= |x| < 2^100 and
// x != 0.
HX_CONV_HD bool d2f_split(double x, float &hi, float &lo)
{
    const uint64_t b = conv_bits64(x);
    const uint32_t bh = (uint32_t)(b >> 32), bl = (uint32_t)b;
    const uint32_t ah = bh & 0x7fffffffu, sign = bh & 0x80000000u;
    if ((ah | bl) == 0) {
        hi = lo = conv_from_bits32(sign);
        return true;
    }
    const uint32_t e = ah >> 20;
    if (e - (1023u - 74u) >= 174u) return false;  // outside [2^-74, 2^100)
    uint32_t out = sign | ((ah - (896u << 20)) << 3) | (bl >> 29);
    const uint32_t rem = bl & 0x1fffffffu;
    const bool up = rem > 0x10000000u || (rem == 0x10000000u && (out & 1u));
    out += up ? 1u : 0u;
    hi = conv_from_bits32(out);
    // x - hi = (rem - 2^29 up) * 2^(E - 52), E = e - 1023; the scale is a binary32 normal here
    const int r = (int)rem - (up ? (1 << 29) : 0);
    const float scale = conv_from_bits32((e - 1023u - 52u + 127u) << 23);
    const float lm = (float)r * scale;
    lo = sign ? -lm : lm;
    return true;
}

}  // namespace hx

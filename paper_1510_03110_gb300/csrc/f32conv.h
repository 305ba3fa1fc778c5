// f32conv.h -- FP64 -> FP32 rounding to nearest (ties to even) in integer
// arithmetic, from the IEEE 754 binary64 / binary32 formats.
//
// On GB300 the FP64 instructions, the double -> float conversion among them,
// issue at a small fraction of the FP32 rate; a conversion done on the integer
// pipes costs a dozen integer operations instead.  Values whose float result is
// a normal number take the integer path; zeros, subnormal results, overflow,
// infinities and NaNs take the hardware conversion, in a function kept out of
// line so that the compiler branches around it instead of evaluating both sides
// and selecting.  The widening float -> double is exact and done the same way.
// Host and device code.
#pragma once
#include <string.h>

#ifdef __CUDACC__
#define MHE_HD __host__ __device__ __forceinline__
#define MHE_HD_OUTLINE static __host__ __device__ __noinline__
#else
#define MHE_HD inline
#define MHE_HD_OUTLINE static __attribute__((noinline, unused))
#endif

namespace mhe {

// the rare cases of both conversions, by the hardware
MHE_HD_OUTLINE float f32_rn_rare(double d) { return (float)d; }
MHE_HD_OUTLINE double f64_rare(float f) { return (double)f; }

MHE_HD float f32_rn(double d)
{
    unsigned long long u;
    memcpy(&u, &d, sizeof(u));
    const unsigned hi = (unsigned)(u >> 32), lo = (unsigned)u;
    const unsigned e = (hi >> 20) & 0x7FFu;   // biased binary64 exponent
    // float normal exponents 1..254 <-> binary64 exponents 897..1150
    if (e - 897u <= 253u) {
        // sign | rebiased exponent | the top 23 of the 52 fraction bits
        unsigned f = (hi & 0x80000000u) | ((e - 896u) << 23) | ((hi & 0xFFFFFu) << 3) | (lo >> 29);
        const unsigned rem = lo & 0x1FFFFFFFu;   // the 29 dropped fraction bits
        // round to nearest, ties to even; a carry into the exponent is the
        // correctly rounded result (up to +inf from the largest binade)
        f += (rem > 0x10000000u || (rem == 0x10000000u && (f & 1u))) ? 1u : 0u;
        float r;
        memcpy(&r, &f, sizeof(r));
        return r;
    }
    return f32_rn_rare(d);
}

// float -> double, exact: a normal float keeps its sign and fraction and has its
// exponent rebiased (127 -> 1023); a zero keeps its sign.  Subnormals,
// infinities and NaNs take the hardware conversion.
MHE_HD double f64_of(float f)
{
    unsigned b;
    memcpy(&b, &f, sizeof(b));
    const unsigned ab = b & 0x7FFFFFFFu;
    if (ab - 0x00800000u < 0x7F000000u || ab == 0u) {
        // high word: sign | exponent + 896 | top 20 fraction bits; low word: the other 3
        const unsigned hi = (ab ? (ab >> 3) + 0x38000000u : 0u) | (b & 0x80000000u);
        const unsigned long long u = ((unsigned long long)hi << 32) | (unsigned long long)(b << 29);
        double d;
        memcpy(&d, &u, sizeof(d));
        return d;
    }
    return f64_rare(f);
}

// widening of a tree value to FP64 (the identity for FP64 trees)
MHE_HD double f64_of(double d) { return d; }

// The low part of a double-float pair: lo = RN(d - hi) with hi = f32_rn(d), so
// that hi + lo holds d to 48 bits.  The remainder d - hi is exact in binary64:
// the 29 fraction bits f32_rn dropped, minus 2^29 when it rounded up, in units
// of 2^(e - 1075) for d's biased exponent e; that integer is rounded to float
// and scaled by the power of two (exact for normal results).  Zeros and values
// whose remainder would leave the float normal range take the hardware path.
MHE_HD_OUTLINE float f32_lo_rare(double d, float hi) { return (float)(d - (double)hi); }

MHE_HD float f32_lo(double d, float hi)
{
    unsigned long long u;
    memcpy(&u, &d, sizeof(u));
    const unsigned uh = (unsigned)(u >> 32), ul = (unsigned)u;
    const unsigned e = (uh >> 20) & 0x7FFu;
    // normal float hi and a normal scale 2^(e - 1075): e in 949 .. 1150
    if (e - 949u <= 201u) {
        const unsigned rem = ul & 0x1FFFFFFFu;
        const unsigned top = ((uh & 0xFFFFFu) << 3) | (ul >> 29);
        const bool up = rem > 0x10000000u || (rem == 0x10000000u && (top & 1u));
        const int r = up ? (int)rem - (int)0x20000000 : (int)rem;   // |r| <= 2^28
#ifdef __CUDA_ARCH__
        const float fr = __int2float_rn(r);
#else
        const float fr = (float)r;
#endif
        const unsigned sb = ((e - 948u) << 23);                       // 2^(e - 1075) as a float
        float scale;
        memcpy(&scale, &sb, sizeof(scale));
        const float lo = fr * scale;
        return (uh & 0x80000000u) ? -lo : lo;
    }
    (void)hi;
    return f32_lo_rare(d, hi);
}

}  // namespace mhe

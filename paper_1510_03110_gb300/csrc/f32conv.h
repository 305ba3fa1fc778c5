// f32conv.h -- FP64 -> FP32 rounding to nearest (ties to even) in integer
// arithmetic, from the IEEE 754 binary64 / binary32 formats.
//
// On GB300 the FP64 instructions, the double -> float conversion among them,
// issue at a small fraction of the FP32 rate; a conversion done on the integer
// pipes costs a dozen integer operations instead.  Values whose float result is
// a normal number take the integer path; zeros, subnormal results, overflow,
// infinities and NaNs take the hardware conversion.  Host and device code.
#pragma once
#include <string.h>

#ifdef __CUDACC__
#define MHE_HD __host__ __device__ __forceinline__
#else
#define MHE_HD inline
#endif

namespace mhe {

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
    return (float)d;
}

}  // namespace mhe

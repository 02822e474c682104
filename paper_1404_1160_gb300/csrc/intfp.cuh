// intfp.cuh -- IEEE binary64 operations evaluated with integer instructions.
//
// GB300 executes FP64 at 2 fused multiply-adds per clock per SM, 64 times
// slower than its integer pipes; the FP64 window kernels are bound by that
// pipe.  The functions here give, for the operands they accept, exactly the
// IEEE binary64 result (round to nearest, ties to even) that the FP64
// instruction would give, using integer instructions only; for the operands
// they refuse (zeros, subnormal, infinite or NaN inputs, results that would
// overflow or fall below the normal range) they return false and the caller
// issues the FP64 instruction.  Compiled for the host as well, so that
// tests/test_intfp.py checks them against the CPU's binary64 arithmetic.
#pragma once

#include <stdint.h>
#include <string.h>

#if defined(__CUDACC__)
#define PIC_HD __host__ __device__ __forceinline__
#else
#define PIC_HD inline
#endif

namespace pic {

PIC_HD uint64_t lf_bits(double x) {
#if defined(__CUDA_ARCH__)
    return (uint64_t)__double_as_longlong(x);
#else
    uint64_t b;
    memcpy(&b, &x, 8);
    return b;
#endif
}

PIC_HD double lf_double(uint64_t b) {
#if defined(__CUDA_ARCH__)
    return __longlong_as_double((long long)b);
#else
    double x;
    memcpy(&x, &b, 8);
    return x;
#endif
}

// position of the leading one bit (x > 0)
PIC_HD int lf_msb(uint64_t x) {
#if defined(__CUDA_ARCH__)
    return 63 - __clzll((long long)x);
#else
    return 63 - __builtin_clzll(x);
#endif
}

// high 64 bits of the 128-bit product a b
PIC_HD uint64_t lf_mulhi(uint64_t a, uint64_t b) {
#if defined(__CUDA_ARCH__)
    return __umul64hi(a, b);
#else
    return (uint64_t)(((unsigned __int128)a * b) >> 64);
#endif
}

// x * y rounded to nearest even.  The significands' product P = mx my has
// its leading bit at 104 or 105; its top 53 bits are kept, the next bit is
// the round bit and everything below is sticky.
PIC_HD bool imul64(double x, double y, double& out) {
    const uint64_t M52 = (1ull << 52) - 1;
    const uint64_t bx = lf_bits(x), by = lf_bits(y);
    const int ex = (int)((bx >> 52) & 0x7ff), ey = (int)((by >> 52) & 0x7ff);
    if (ex == 0 || ex == 0x7ff || ey == 0 || ey == 0x7ff) return false;
    const uint64_t mx = (bx & M52) | (1ull << 52), my = (by & M52) | (1ull << 52);
    const uint64_t lo = mx * my, hi = lf_mulhi(mx, my);  // P = hi 2^64 + lo < 2^106
    const int top = (int)((hi >> 41) & 1ull);            // bit 105 of P
    const int sh = 52 + top;                             // bits below the kept 53
    uint64_t q = (hi << (64 - sh)) | (lo >> sh);
    const uint64_t rem = lo & ((1ull << sh) - 1), half = 1ull << (sh - 1);
    int e = ex + ey - 1023 + top;  // biased exponent of the result
    if (e <= 0 || e >= 0x7ff) return false;
    if (rem > half || (rem == half && (q & 1ull))) {
        ++q;
        if (q >> 53) {  // rounded up to the next power of two
            q >>= 1;
            ++e;
            if (e >= 0x7ff) return false;
        }
    }
    out = lf_double(((bx ^ by) & (1ull << 63)) | ((uint64_t)e << 52) | (q & M52));
    return true;
}

}  // namespace pic

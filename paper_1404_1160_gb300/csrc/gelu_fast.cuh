// gelu_fast.cuh -- the network's activation gelu(u) = u erfc(-u/sqrt 2) / 2
// in binary32 (gelu_f), and a cheaper evaluation for the places where the
// network rounds it to bfloat16 at once (gelu_for_bf16).
//
// gelu_for_bf16 returns a binary32 value whose bfloat16 rounding (to
// nearest even) equals that of gelu_f(u), for every binary32 u: this holds
// by construction, and tests/test_gelu_fast.py checks it on the GPU for
// all 2^32 inputs.  The construction:
//   * a = |x| with x = -u/sqrt2 rounded as in gelu_f; on 2^-60 <= a < 8
//     erfc(a) ~ T_j 2^(r_j(d)) from the segment table (gelu_table.h:
//     a_j = j/8 = round(8a)/8, d = a - a_j exact, r_j a cubic in d; relative
//     error of the table 9e-8, of the whole evaluation a few units of 2^-23);
//   * erfc(x) = 2 - erfc(a) for x < 0 gives h = max(u, 0) - |u|/2 erfc(a),
//     one fused multiply-add;
//   * h is kept only when its bits are more than kGeluMargin units in the
//     last place away from a bfloat16 rounding midpoint (the low 16 bits
//     0x8000): h and gelu_f(u) are much closer than that, so both round to
//     the same bfloat16.  Otherwise (and outside the table's range, for
//     zeros, infinities and NaN) gelu_f runs, out of line.
// About 25 instructions per activation against about 45 for gelu_f; the
// fallback runs for about 0.1 % of the activations.
#pragma once

#include "gelu_table.h"

namespace pic {

__device__ __forceinline__ float gelu_f(float u) { return 0.5f * u * erfcf(-u * 0.70710678118654752f); }

constexpr unsigned int kGeluMargin = 32;  // binary32 ulps kept from a bfloat16 rounding midpoint

static __device__ __noinline__ float gelu_slow(float u) { return gelu_f(u); }

__device__ __forceinline__ float ex2_approx(float x) {
    float y;
    asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}

// The table evaluation: true, with h, when the bfloat16 rounding of h is
// certain to be that of gelu_f(u).  tab: the (kGeluSeg + 1) entries
// (T_j, c1, c2, c3) of c_gelu_tab, staged in shared memory by the caller.
__device__ __forceinline__ bool gelu_fast_try(float u, const float4* __restrict__ tab, float& h) {
    const float x = -u * 0.70710678118654752f;  // the argument gelu_f gives erfc
    const float a = fabsf(x);
    const float s = fmaf(a, 8.0f, 12582912.0f);  // 1.5 2^23 + round(8 a): the segment in the low bits
    const unsigned int j = min((unsigned int)(__float_as_int(s) - 0x4B400000), (unsigned int)kGeluSeg);
    const float d = fmaf(s - 12582912.0f, -0.125f, a);  // a - j/8, exact
    const float4 c = tab[j];
    const float p = fmaf(fmaf(c.w, d, c.z), d, c.y);
    const float E = c.x * ex2_approx(p * d);  // erfc(a)
    h = fmaf(-0.5f * fabsf(u), E, fmaxf(u, 0.0f));
    const unsigned int hb = __float_as_uint(h);
    const bool in_range = __float_as_uint(a) - 0x21800000u < 0x41000000u - 0x21800000u;  // 2^-60 <= a < 8
    const bool clear = ((hb - (0x8000u - kGeluMargin)) & 0xFFFFu) > 2u * kGeluMargin;
    return in_range && clear;
}

// A binary32 value whose bfloat16 rounding is that of gelu_f(u).
__device__ __forceinline__ float gelu_for_bf16(float u, const float4* __restrict__ tab) {
    float h;
    return gelu_fast_try(u, tab, h) ? h : gelu_slow(u);
}

}  // namespace pic

// locate_fixed.cuh -- the CIC cell location of a particle (Sec. 2.3) with
// its one rounding done on the integer pipe.
//
// On a mesh whose 1/h_r is a power of two (and W, the fixed-point units per
// particle, a power of two), the position in fixed-point mesh units is
//     xs = W (R - r_min) / h_r = RN(R s + C),  s = W/h_r = 2^k,  C = -r_min s,
// one correctly rounded sum (R s is exact).  From xs the deposit and the
// gather need j = floor(xs / W), qR = floor(xs) mod W (the right node's
// units) and a = xs - j W (= W f, as a double).  GB300 runs FP64 at 2 FMA per
// clock per SM and this locate is 4 of the ~25 FP64 instructions of a
// particle's fine step, so it is computed here with integer instructions:
//
//   1. R s is written exactly as the fixed-point integer Y = R s 2^F (F
//      fractional bits, truncated toward zero, with a sticky bit for the
//      truncated part), C as the integer C 2^F;
//   2. S = C 2^F +- Y is the exact sum (to within the sticky bit);
//   3. S is rounded to 53 significant bits, to nearest, ties to even (the
//      sticky bit breaks would-be ties), which is xs 2^F exactly;
//   4. j, qR and a are read off that integer (a by an exact int -> double
//      of its low log2(W) + F bits).
//
// F = 61 - T where n_cells W <= 2^T, so every intermediate fits a signed
// 64-bit integer; the fast path takes results with at least two guard bits
// (S >= 2^54, about two cells above r_min for the benchmark mesh) and normal
// R with |R s| < 2^T; anything else (the first cells, off the mesh, NaN)
// reports "not handled" and the caller evaluates the FP64 form.  The result
// equals the FP64 form bit for bit wherever the fast path answers (checked
// on the CPU against fma() over random, node, tie and bit-pattern inputs by
// tests/test_locate_fixed.py).
#pragma once

#include "intfp.cuh"

namespace pic {

// Constants of the fixed-point locate, precomputed on the host.
struct LocFixed {
    int ok;            // 1: the mesh qualifies (power-of-two s, C 2^F an integer)
    int F, k, T;       // fractional bits, log2 s, n_cells W <= 2^T
    int log2W;
    long long C;       // C 2^F
    long long xs_max;  // n_cells W
    long long Wmask;   // W - 1
};

// Fills L for a mesh with xs_scale = s, xs_off = C, n_cells W = xs_max,
// W = 2^log2W (host side).
inline void loc_fixed_setup(LocFixed* L, int pow2_mesh, double xs_scale, double xs_off, long long xs_max, int log2W) {
    memset(L, 0, sizeof(*L));
    if (!pow2_mesh || xs_max <= 0 || !(xs_scale > 0.0) || !(xs_off >= 0.0)) return;
    int T = 0;
    while (T < 62 && (1ll << T) < xs_max) ++T;
    const int F = 61 - T;
    if (F < 0) return;
    // s must be a power of two: its significand bits all zero
    const uint64_t sb = lf_bits(xs_scale);
    if ((sb & ((1ull << 52) - 1)) != 0ull || ((sb >> 52) & 0x7ff) == 0) return;
    const int k = (int)((sb >> 52) & 0x7ff) - 1023;
    // C 2^F must be an integer below 2^62
    const uint64_t cb = lf_bits(xs_off);
    long long Cf = 0;
    if (xs_off != 0.0) {
        const int ce = (int)((cb >> 52) & 0x7ff) - 1075 + F;  // exponent of the significand's lsb
        const uint64_t cm = (cb & ((1ull << 52) - 1)) | (1ull << 52);
        if (((cb >> 52) & 0x7ff) == 0) return;
        if (ce < 0) {
            if (-ce >= 64 || (cm & ((1ull << -ce) - 1)) != 0ull) return;
            Cf = (long long)(cm >> -ce);
        } else {
            if (ce > 8) return;
            Cf = (long long)(cm << ce);
        }
    }
    L->ok = 1;
    L->F = F;
    L->k = k;
    L->T = T;
    L->log2W = log2W;
    L->C = Cf;
    L->xs_max = xs_max;
    L->Wmask = (1ll << log2W) - 1;
}

// The located cell of R: returns false (leaving j, qR, a untouched) where
// the fast path does not answer; then the caller uses the FP64 form.
PIC_HD bool loc_fixed(const LocFixed& L, double R, int& j, long long& qR, double& a) {
    const uint64_t M52 = (1ull << 52) - 1;
    const uint64_t b = lf_bits(R);
    const int be = (int)((b >> 52) & 0x7ff);
    if (be == 0 || be - 1023 + L.k >= L.T) return false;  // zero, subnormal, |R s| >= 2^T, Inf, NaN
    const uint64_t m = (b & M52) | (1ull << 52);
    const int sh = be - 1075 + L.k + L.F;  // exponent of m's lsb in units of 2^-F (< 9 here)
    uint64_t y;
    bool sticky;
    if (sh >= 0) {
        y = m << sh;
        sticky = false;
    } else if (sh > -64) {
        y = m >> (-sh);
        sticky = (m & ((1ull << (-sh)) - 1)) != 0ull;
    } else {
        y = 0ull;
        sticky = true;
    }
    // negative R: the exact sum lies in (S - 1, S) when bits were truncated
    const long long S = (b >> 63) ? L.C - (long long)y - (sticky ? 1 : 0) : L.C + (long long)y;
    if (S < (1ll << 54)) return false;  // fewer than two guard bits (or below the mesh)
    const int d = lf_msb((uint64_t)S) - 52;  // bits dropped by the rounding (>= 2)
    const uint64_t rem = (uint64_t)S & ((1ull << d) - 1), half = 1ull << (d - 1);
    uint64_t q = (uint64_t)S >> d;
    if (rem > half || (rem == half && (sticky || (q & 1ull)))) ++q;
    const uint64_t X = q << d;  // xs 2^F
    const long long xi = (long long)(X >> L.F);  // floor(xs)
    if (xi >= L.xs_max) return false;  // beyond the last cell
    qR = xi & L.Wmask;
    j = (int)(xi >> L.log2W);
    // a = xs - j W: the low log2W + F bits of X (at most 53 significant bits)
    const uint64_t A = X & ((1ull << (L.log2W + L.F)) - 1);
    if (A == 0ull) {
        a = 0.0;
    } else {
        const int p = lf_msb(A);
        const uint64_t mant = p >= 52 ? (A >> (p - 52)) : (A << (52 - p));
        a = lf_double(((uint64_t)(p - L.F + 1023) << 52) | (mant & M52));
    }
    return true;
}

}  // namespace pic

// CPU check of the integer-pipe binary64 operations (paper_1404_1160_gb300/
// csrc/intfp.cuh) against the CPU's own IEEE binary64 arithmetic: wherever
// imul64 answers, its result must have the bits of x * y.
//
// usage: intfp_check <count> <seed>; prints "total answered mismatches".
#include <cmath>
#include <cstdint>
#include <cstdio>
#include <cstdlib>
#include <cstring>

#include "intfp.cuh"

static uint64_t g_state;
static uint64_t next_u64() {  // splitmix64
    uint64_t z = (g_state += 0x9e3779b97f4a7c15ull);
    z = (z ^ (z >> 30)) * 0xbf58476d1ce4e5b9ull;
    z = (z ^ (z >> 27)) * 0x94d049bb133111ebull;
    return z ^ (z >> 31);
}
static double from_bits(uint64_t b) {
    double x;
    std::memcpy(&x, &b, 8);
    return x;
}
static uint64_t to_bits(double x) {
    uint64_t b;
    std::memcpy(&b, &x, 8);
    return b;
}
// a double with exponent e (unbiased), random significand with its low
// `tz` bits cleared, random sign
static double make(int e, int tz, uint64_t r) {
    uint64_t m = r & ((1ull << 52) - 1);
    if (tz > 0) m &= ~((1ull << (tz > 52 ? 52 : tz)) - 1);
    return from_bits(((r >> 63) << 63) | ((uint64_t)(e + 1023) << 52) | m);
}

int main(int argc, char** argv) {
    const long long count = argc > 1 ? atoll(argv[1]) : 1000000;
    g_state = argc > 2 ? strtoull(argv[2], nullptr, 10) : 1;
    // the rotation constants of the fine step (cos, sin of 2 pi/100 and pi/100)
    const double K[4] = {std::cos(2 * M_PI / 100), std::sin(2 * M_PI / 100), std::cos(M_PI / 100),
                         std::sin(M_PI / 100)};
    long long answered = 0, bad = 0;
    for (long long i = 0; i < count; ++i) {
        const uint64_t r1 = next_u64(), r2 = next_u64(), r3 = next_u64();
        double x, y;
        switch (i % 6) {
            case 0:  // a constant of the fine step times a position or velocity
                x = K[r3 & 3];
                y = make((int)(r3 >> 8) % 12 - 8, 0, r2);
                break;
            case 1:  // moderate exponents
                x = make((int)(r1 % 200) - 100, 0, r2);
                y = make((int)(r3 % 200) - 100, 0, r3 * 7);
                break;
            case 2:  // trailing zeros: exact products and ties
                x = make((int)(r1 % 40) - 20, (int)(r2 % 53), r2);
                y = make((int)(r3 % 40) - 20, (int)(r1 % 53), r3);
                break;
            case 3:  // near the limits of the normal range
                x = make((int)(r1 % 1000) - 1022 + (int)(r1 & 1) * 1000, 0, r2);
                y = make((int)(r3 % 1000) - 1022 + (int)(r3 & 1) * 1000, 0, r3);
                break;
            case 4: {  // significands near 1 and near 2 (carries out of the rounding)
                const uint64_t lo = r2 & 0xff;
                x = from_bits((r1 & (1ull << 63)) | (1023ull << 52) | ((r1 & 1) ? (((1ull << 52) - 1) ^ lo) : lo));
                y = from_bits((r3 & (1ull << 63)) | (1023ull << 52) | ((r3 & 1) ? (((1ull << 52) - 1) ^ (r3 >> 50)) : (r3 >> 50)));
                break;
            }
            default:  // any bit patterns
                x = from_bits(r1);
                y = from_bits(r2);
                break;
        }
        double out;
        if (!pic::imul64(x, y, out)) continue;
        ++answered;
        const double ref = x * y;
        if (to_bits(out) != to_bits(ref)) {
            if (bad < 5) printf("mismatch %.17g * %.17g: %.17g vs %.17g\n", x, y, out, ref);
            ++bad;
        }
    }
    printf("%lld %lld %lld\n", count, answered, bad);
    return bad ? 1 : 0;
}

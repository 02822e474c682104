// CPU check of the fixed-point cell locate (paper_1404_1160_gb300/csrc/
// locate_fixed.cuh) against its FP64 definition: xs = fma(R, s, C) with
// s = W/h_r a power of two and C = -r_min s, then j = floor(xs / W),
// qR = floor(xs) mod W, a = xs - j W.  Wherever the fixed-point form
// answers, j, qR and the bits of a must equal the FP64 ones.
//
// usage: locate_fixed_check <n_cells> <log2W> <r_max> <count> <seed>
// prints "eligible total fast mismatches"; exit status 1 on a mismatch.
#include <cmath>
#include <cstdint>
#include <cstdio>
#include <cstdlib>
#include <cstring>

#include "locate_fixed.cuh"

static uint64_t g_state;
static uint64_t next_u64() {  // splitmix64
    uint64_t z = (g_state += 0x9e3779b97f4a7c15ull);
    z = (z ^ (z >> 30)) * 0xbf58476d1ce4e5b9ull;
    z = (z ^ (z >> 27)) * 0x94d049bb133111ebull;
    return z ^ (z >> 31);
}
static double unit(uint64_t r) { return (double)(r >> 11) * (1.0 / 9007199254740992.0); }

int main(int argc, char** argv) {
    if (argc < 6) return 2;
    const int Nc = atoi(argv[1]), l2 = atoi(argv[2]);
    const double r_max = atof(argv[3]), r_min = -r_max;
    const long long count = atoll(argv[4]);
    g_state = strtoull(argv[5], nullptr, 10);
    const double hr = (r_max - r_min) / (double)Nc, inv_hr = 1.0 / hr, W = std::ldexp(1.0, l2);
    int ex = 0;
    const int pow2 = std::frexp(inv_hr, &ex) == 0.5 ? 1 : 0;
    const double s = inv_hr * W, C = -(r_min * inv_hr) * W;
    const long long xs_max = (long long)Nc << l2;
    pic::LocFixed L;
    pic::loc_fixed_setup(&L, pow2, s, C, xs_max, l2);
    long long fast = 0, bad = 0;
    for (long long i = 0; i < (L.ok ? count : 0); ++i) {
        const uint64_t r = next_u64();
        double R;
        switch (i % 7) {
            case 0: R = r_min + (r_max - r_min) * unit(r); break;                 // on the mesh
            case 1: { uint64_t b = r; std::memcpy(&R, &b, 8); break; }          // any bit pattern
            case 2: {                                                            // nodes and their neighbours
                R = r_min + (double)(r % (uint64_t)(Nc + 1)) * hr;
                if ((r >> 62) & 1) R = std::nextafter(R, (r >> 63) ? 1e300 : -1e300);
                break;
            }
            case 3: R = std::ldexp((double)(r >> 11), -53 - (int)((r >> 5) % 70)) * ((r & 1) ? -1.0 : 1.0); break;
            case 4: {                                                            // low significand bits set: ties
                R = r_min + (r_max - r_min) * unit(r);
                uint64_t b;
                std::memcpy(&b, &R, 8);
                b = (b & ~0xfffull) | ((r >> 13) & 0xfffull);
                std::memcpy(&R, &b, 8);
                break;
            }
            case 5: R = 1.25 * r_max * ((double)(int64_t)r / 9.2233720368547758e18); break;  // around the edges
            default: R = r_min + (r_max - r_min) * (0.5 + 0.5 * unit(r)) * (1.0 - std::ldexp(1.0, -(int)(r % 40))); break;
        }
        int j = -9;
        long long qR = -9;
        double a = -9.0;
        if (!pic::loc_fixed(L, R, j, qR, a)) continue;
        ++fast;
        const double xs = std::fma(R, s, C);
        const double fl = std::floor(xs);
        const long long xi = (long long)fl;
        const int jr = (int)(xi >> l2);
        const long long qr = xi & ((1ll << l2) - 1);
        const double ar = xs - std::ldexp((double)jr, l2);
        uint64_t b1, b2;
        std::memcpy(&b1, &a, 8);
        std::memcpy(&b2, &ar, 8);
        const bool ok = xs >= 0.0 && xi < xs_max && j == jr && qR == qr && b1 == b2;
        if (!ok) {
            if (bad < 5) printf("mismatch R=%.17g: j %d/%d qR %lld/%lld a %.17g/%.17g\n", R, j, jr, qR, qr, a, ar);
            ++bad;
        }
    }
    printf("%d %lld %lld %lld\n", L.ok, L.ok ? count : 0, fast, bad);
    return bad ? 1 : 0;
}

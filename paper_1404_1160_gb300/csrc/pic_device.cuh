// pic_device.cuh -- device-side building blocks of the improved ETD PIC path.
//
// Arithmetic contract: the library is compiled with FP contraction off
// (--fmad=false); every multiply-add that the method evaluates with a single
// rounding is written as an explicit fma() here.  Only IEEE-exact
// operations (+ - * / sqrt fma floor rint fmod and integer conversions) are
// used per particle, so a result depends only on the formula's evaluation
// order, which each function states.
#pragma once

#include <cstdint>
#include <cuda_runtime.h>

namespace pic {

constexpr int kMaxCellsWindow = 2048;  // mesh cells served by the fused window kernel (shared memory)

// Status word values written by kernels (host maps them to PIC_ERR_*).
enum DevStatus : int { DEV_OK = 0, DEV_TIMEOUT = 1, DEV_BAD = 2 };

// Everything a kernel needs, precomputed on the host (trig constants of the
// exact rotation come from the host's libm: the device never evaluates a
// transcendental function).
struct DevParams {
    // time stepping: fine step h = 2 pi eps / steps_per_turn
    double eps, inv_eps, mie;          // mie = -(1/eps)
    double h, h2, h6, D;               // h/2, h/6, dt/h
    double c1, s1, ch, sh;             // cos/sin(h/eps), cos/sin(h/(2 eps))
    double hsh, tch, tsh;              // h*sh, 2*ch, 2*sh
    // mesh: nodes r_j = r_min + j*hr, j = 0..n_cells; node c = n_cells/2 is r = 0
    double r_min, hr, inv_hr;
    double xs_scale, xs_off, xs_max;   // xs = W*x, x = (R - r_min)/hr
    long long xs_max_i;                // n_cells*W
    double Wd, invW;                   // W and 1/W (powers of two)
    double q_unit, q_half;             // charge per fixed-point unit, and half of it
    long long W, Wmask;
    int log2W;
    int n_cells, c;
    int xs_fma;                        // 1 when inv_hr is a power of two
    // algorithm
    int field, solver;                 // PIC_FIELD_*, PIC_FINE_*
    int Kmax;                          // window cap (fine steps)
    double Tfb;                        // fallback period in fine steps (2 pi eps / h)
    long long n;                       // particles
    long long wait_ns;                 // limit of device-side waits
    int bar_extra;                     // testing only: arrivals a barrier waits for beyond the grid
    int hist_copies;                   // copies of each block's charge histogram (window kernel)
};

// ---------------------------------------------------------------- mesh

// Position of R in fixed-point mesh units: xs = W * (R - r_min) / hr.  When
// 1/hr is a power of two (POW2), W*(R - r_min)*inv_hr equals fma(R, W*inv_hr,
// -W*r_min*inv_hr) bit for bit (power-of-two scaling commutes with
// rounding), so the single fma is used; the form is fixed at compile time.
template <int POW2>
__device__ __forceinline__ double mesh_xs(const DevParams& P, double R) {
    if (POW2) return fma(R, P.xs_scale, P.xs_off);
    return ((R - P.r_min) * P.inv_hr) * P.Wd;
}

// A located position.  In the mesh: cell j in [0, n_cells), a = W*f with f
// the right weight, qR = floor(f*W).  Outside: j = -1 (below r_min) or -2
// (at or above r_max, or NaN), a = R.
struct Cell {
    int j;
    double a;
    long long qR;
};

// Integer split of xs >= 0 (finite, < 2^62): xi = floor(xs) and
// a = xs - (xi with its low log2W bits cleared), i.e. W f, read off the
// IEEE bit pattern of xs with integer instructions.  Bit-identical to
// xi = floor(xs), a = xs - (double)(j W): both are exact, and a is a
// sub-field of the significand of xs re-normalised.
__device__ __forceinline__ void split_fixed(double xs, int log2W, long long& xi, double& a) {
    constexpr unsigned long long M52 = (1ull << 52) - 1;
    const unsigned long long b = (unsigned long long)__double_as_longlong(xs);
    const int e = (int)(b >> 52) - 1023;
    if (e < 0) {  // 0 <= xs < 1
        xi = 0;
        a = xs;
        return;
    }
    const unsigned long long m = (b & M52) | (1ull << 52);
    xi = e <= 52 ? (long long)(m >> (52 - e)) : (long long)(m << (e - 52));
    if (e < log2W) {  // xs < W: cell 0
        a = xs;
        return;
    }
    const int nb = 52 - e + log2W;  // significand bits below the cell boundary
    if (nb <= 0) {
        a = 0.0;
        return;
    }
    const unsigned long long am = m & ((1ull << nb) - 1);
    if (am == 0) {
        a = 0.0;
        return;
    }
    const int p = 63 - __clzll((long long)am);
    a = __longlong_as_double((long long)((((unsigned long long)(p + e - 52 + 1023)) << 52) | ((am << (52 - p)) & M52)));
}

template <int POW2>
__device__ __forceinline__ Cell mesh_locate(const DevParams& P, double R) {
    Cell c;
    const double xs = mesh_xs<POW2>(P, R);
    const unsigned long long b = (unsigned long long)__double_as_longlong(xs);
    const unsigned long long mag = b & 0x7fffffffffffffffull;
    // below the mesh: negative (not -0, not NaN); above: NaN, >= 2^62 or
    // beyond the last cell
    if ((b >> 63) && mag != 0ull) {
        c.j = mag > 0x7ff0000000000000ull ? -2 : -1;
        c.a = R;
        c.qR = 0;
        return c;
    }
    if ((int)(mag >> 52) - 1023 >= 62) {
        c.j = -2;
        c.a = R;
        c.qR = 0;
        return c;
    }
    long long xi;
    double a;
    split_fixed(xs, P.log2W, xi, a);
    if (xi >= P.xs_max_i) {
        c.j = -2;
        c.a = R;
        c.qR = 0;
        return c;
    }
    c.qR = xi & P.Wmask;  // floor(f W)
    c.j = (int)(xi >> P.log2W);
    c.a = a;              // W f
    return c;
}

// Exact-rounding int64 -> double (round to nearest, ties to even) with
// integer instructions only; equal to (double)x for every int64.
__device__ __forceinline__ double i64_to_double(long long x) {
    if (x == 0) return 0.0;
    const unsigned long long sign = x < 0 ? (1ull << 63) : 0ull;
    unsigned long long m = x < 0 ? 0ull - (unsigned long long)x : (unsigned long long)x;
    const int p = 63 - __clzll((long long)m);  // leading bit
    int e = p;
    if (p > 52) {
        const int sh = p - 52;
        const unsigned long long rem = m & ((1ull << sh) - 1), half = 1ull << (sh - 1);
        m >>= sh;
        if (rem > half || (rem == half && (m & 1ull))) {
            ++m;
            if (m >> 53) {  // carried into a new leading bit
                m >>= 1;
                ++e;
            }
        }
    } else {
        m <<= (52 - p);
    }
    return __longlong_as_double((long long)(sign | ((unsigned long long)(e + 1023) << 52) | (m & ((1ull << 52) - 1))));
}

// x * 2^k for a normal x whose result stays normal (exponent arithmetic).
__device__ __forceinline__ double scale_pow2(double x, int k) {
    if (x == 0.0) return x;
    return __longlong_as_double(__double_as_longlong(x) + ((long long)k << 52));
}

// V > 0 for every non-NaN double, tested on the bit pattern (integer pipe).
__device__ __forceinline__ bool positive(double v) { return __double_as_longlong(v) > 0; }

// Off the mesh rE keeps its edge value: E = rE_edge / R (rare; kept out of
// line so the division is never evaluated for particles on the mesh).
static __device__ __noinline__ double gather_outside(double rE_lo, double rE_hi, int j, double R) {
    return (j == -1 ? rE_lo : rE_hi) / R;
}

// Field table entry of cell j: (E_j, (E_{j+1} - E_j) / W).  The gather
// fma(W f, (E_{j+1}-E_j)/W, E_j) equals fma(f, E_{j+1}-E_j, E_j) exactly.
__device__ __forceinline__ double mesh_gather(const double2* tab, double rE_lo, double rE_hi,
                                              int j, double a) {
    if (j >= 0) {
        const double2 e = tab[j];
        return fma(a, e.y, e.x);
    }
    return gather_outside(rE_lo, rE_hi, j, a);
}

// ------------------------------------------------------- analytic fields

__device__ __forceinline__ double field_analytic(int field, double R) {
    // eq. RappelForce: E = -r^3; zero field otherwise
    return field == 1 ? -((R * R) * R) : 0.0;
}

// -------------------------------------------- landing: root and interpolation

// Lagrange quadratic through (0,y0),(1,y1),(2,y2) at s.
__device__ __forceinline__ double interp3(double y0, double y1, double y2, double s) {
    double d1 = ((-3.0 * y0 + 4.0 * y1) - y2) * 0.5;
    double d2 = ((y0 - 2.0 * y1) + y2) * 0.5;
    return y0 + s * (d1 + s * d2);
}

// Root in [0,1] of that quadratic when y0 and y1 differ in sign: the
// cancellation-free pair of closed-form roots, linear if the quadratic term
// is zero.
__device__ __forceinline__ double quad_root01(double v0, double v1, double v2) {
    double a = v0;
    double b = ((-3.0 * v0 + 4.0 * v1) - v2) * 0.5;
    double c = ((v0 - 2.0 * v1) + v2) * 0.5;
    double s;
    if (c == 0.0) {
        s = (b != 0.0) ? -a / b : 0.0;
    } else {
        double disc = b * b - 4.0 * a * c;
        if (disc < 0.0) disc = 0.0;
        double sq = sqrt(disc);
        double q = (b >= 0.0) ? -0.5 * (b + sq) : -0.5 * (b - sq);
        if (q == 0.0) {
            s = 0.0;
        } else {
            s = a / q;
            if (!(s >= 0.0 && s <= 1.0)) s = q / c;
        }
    }
    if (!(s >= 0.0)) s = 0.0;
    if (s > 1.0) s = 1.0;
    return s;
}

// ------------------------------------------- per-particle period tracking

// flags: bits 0-1 number of extrema seen, bit 2 resolved, bit 3 fallback,
// bit 4 a sign change between the two previous samples awaits its root.
constexpr int F_NEXT = 3, F_RES = 4, F_FB = 8, F_PEND = 16;

struct Track {
    double t1, T, o;
    int N, need, flags;
};

// Delta t = N T + o with o in [0, T) (eq. TimeStepDec), in fine steps; the
// samples needed are the stencils at o and, when N > 0, at o + T.
__device__ __forceinline__ void track_decompose(Track& s, double D, double T) {
    s.T = T;
    s.o = fmod(D, T);
    s.N = (int)rint((D - s.o) / T);
    double last = (s.N > 0) ? s.o + T : s.o;
    s.need = (int)floor(last) + 2;
}

// Resolve with period T; a non-positive/non-finite T or samples beyond the
// window cap take the fallback period 2 pi eps (Tfb fine steps).
__device__ __forceinline__ void track_resolve(Track& s, const DevParams& P, double T) {
    if (!(T > 0.0) || !isfinite(T)) {
        s.flags |= F_FB;
        T = P.Tfb;
    }
    track_decompose(s, P.D, T);
    if (s.need > P.Kmax) {
        s.flags |= F_FB;
        track_decompose(s, P.D, P.Tfb);
    }
    s.flags |= F_RES;
}

// Sample k (k >= 2) has just been produced: V_{k-2} = v0, V_{k-1} = v1,
// V_k = v2.  A sign change between k-2 and k-1 (V > 0 counts as +) is an
// extremum of R (Remark CompOfThePeriodsRem).  detect_only: step 1 alone.
__device__ __forceinline__ void track_sample(Track& s, const DevParams& P, int k, double v0,
                                             double v1, double v2, bool detect_only) {
    if (s.flags & F_RES) return;
    if (positive(v0) != positive(v1)) {
        double t = (double)(k - 2) + quad_root01(v0, v1, v2);
        int ne = (s.flags & F_NEXT) + 1;
        s.flags = (s.flags & ~F_NEXT) | (ne & F_NEXT);
        if (ne == 1) s.t1 = t;
        if (ne == 3) {
            double T = t - s.t1;
            if (detect_only) {
                s.T = T;
                s.flags |= F_RES;
            } else {
                track_resolve(s, P, T);
            }
        }
    }
}

// Root of an extremum already known to lie between samples k-2 and k-1,
// from the stencil V_{k-2} = v0, V_{k-1} = v1, V_k = v2.
__device__ __forceinline__ void track_root(Track& s, const DevParams& P, int k, double v0, double v1, double v2,
                                           bool detect_only) {
    if (s.flags & F_RES) return;
    const double t = (double)(k - 2) + quad_root01(v0, v1, v2);
    const int ne = (s.flags & F_NEXT) + 1;
    s.flags = (s.flags & ~F_NEXT) | (ne & F_NEXT);
    if (ne == 1) s.t1 = t;
    if (ne == 3) {
        const double T = t - s.t1;
        if (detect_only) {
            s.T = T;
            s.flags |= F_RES;
        } else {
            track_resolve(s, P, T);
        }
    }
}

// Window cap reached without a third extremum.
__device__ __forceinline__ void track_cap(Track& s, const DevParams& P, bool detect_only) {
    if (s.flags & F_RES) return;
    s.flags |= F_FB;
    if (detect_only) {
        s.T = P.Tfb;
        s.flags |= F_RES;
    } else {
        track_resolve(s, P, P.Tfb);
    }
}

__device__ __forceinline__ bool track_done(const Track& s, int k, bool detect_only) {
    return (s.flags & F_RES) && (detect_only || k >= s.need);
}

// y^{n+1} = y(o) + N (y(o+T) - y(o)) (eq. MainFormula1); N = 0 keeps y(o).
__device__ __forceinline__ double extrapolate(double yo, double yT, int N) {
    if (N == 0) return yo;
    return yo + (double)N * (yT - yo);
}

// ------------------------------------------------ one fine step, analytic E

// Classical RK4 of y' = ((1/eps) V, -(1/eps) R + E(R)) for one particle.
__device__ __forceinline__ void rk4_step_analytic(const DevParams& P, int field, double& R,
                                                  double& V) {
    const double ie = P.inv_eps, mie = P.mie;
    double e1 = field_analytic(field, R);
    double k1R = ie * V, k1V = fma(mie, R, e1);
    double R2 = fma(P.h2, k1R, R), V2 = fma(P.h2, k1V, V);
    double e2 = field_analytic(field, R2);
    double k2R = ie * V2, k2V = fma(mie, R2, e2);
    double R3 = fma(P.h2, k2R, R), V3 = fma(P.h2, k2V, V);
    double e3 = field_analytic(field, R3);
    double k3R = ie * V3, k3V = fma(mie, R3, e3);
    double R4 = fma(P.h, k3R, R), V4 = fma(P.h, k3V, V);
    double e4 = field_analytic(field, R4);
    double k4R = ie * V4, k4V = fma(mie, R4, e4);
    double sR = ((k1R + 2.0 * k2R) + 2.0 * k3R) + k4R;
    double sV = ((k1V + 2.0 * k2V) + 2.0 * k3V) + k4V;
    R = fma(P.h6, sR, R);
    V = fma(P.h6, sV, V);
}

// Lawson RK4: exact rotation Phi(s) for (1/eps) M y, RK4 on the field term.
__device__ __forceinline__ void lawson_step_analytic(const DevParams& P, int field, double& R,
                                                     double& V) {
    double e1 = field_analytic(field, R);
    double R2 = fma(P.sh, fma(P.h2, e1, V), P.ch * R);
    double e2 = field_analytic(field, R2);
    double R3 = fma(P.sh, V, P.ch * R);
    double e3 = field_analytic(field, R3);
    double A = fma(P.s1, V, P.c1 * R);
    double R4 = fma(P.hsh, e3, A);
    double e4 = field_analytic(field, R4);
    double B = fma(P.c1, V, -(P.s1 * R));
    double e23 = e2 + e3;
    R = fma(P.h6, fma(P.tsh, e23, P.s1 * e1), A);
    V = fma(P.h6, fma(P.tch, e23, fma(P.c1, e1, e4)), B);
}

// ---------------------------------------------------------- device waits

__device__ __forceinline__ long long global_ns() {
    long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

__device__ __forceinline__ unsigned int ld_acquire_u32(const unsigned int* p) {
    unsigned int v;
    asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}

__device__ __forceinline__ int ld_acquire_s32(const int* p) {
    int v;
    asm volatile("ld.acquire.gpu.global.s32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}

}  // namespace pic

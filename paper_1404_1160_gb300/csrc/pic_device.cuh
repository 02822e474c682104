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

#include "locate_fixed.cuh"

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
    LocFixed loc;                      // the same locate on the integer pipe (xs_fma meshes)
    int imul;                          // 1: products by the rotation constants on the integer pipe
    int band_m;                        // > 0: an ETD window stores only the trajectory rows within band_m of
                                       // the landing rows predicted from the previous period (a miss
                                       // replays the window with every row); 0: every row
    // algorithm
    int field, solver;                 // PIC_FIELD_*, PIC_FINE_*
    int Kmax;                          // window cap (fine steps)
    double Tfb;                        // fallback period in fine steps (2 pi eps / h)
    long long n;                       // particles
    long long wait_ns;                 // limit of device-side waits
    int bar_extra;                     // testing only: arrivals a barrier waits for beyond the grid
    int parity_odd;                    // 1: E = rE(r)/|r| (odd in r, 0 on the axis); 0: E = rE(r)/r
    int hist_copies;                   // copies of each block's charge histogram (window kernel)
    // FP32 form (precision 1): the same quantities rounded once to binary32
    float r_min_f, inv_hr_f, ncells_f, Wf;
    float h2shh_f, hshh_f, h6_f;       // (h/2) sin(h/(2 eps)), h sin(h/(2 eps)), h/6
    int spt;                           // fine steps per turn of the E = 0 rotation
    int Di;                            // dt/h = Di + Df with Df in [0, 1)
    float Df;
    const float2* rot;                 // 2 spt entries: (cos, sin)(m h / (2 eps))
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
    // FP64 is the scarce pipe on this GPU: where the fixed-point form answers
    // (it rounds xs exactly as the fma below does), no FP64 instruction runs
    if (POW2 && P.loc.ok && loc_fixed(P.loc, R, c.j, c.qR, c.a)) return c;
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

// x * y with the bits of the FP64 product: on the integer pipe when `on`
// and imul64 answers (normal operands and result), else the FP64 multiply.
__device__ __forceinline__ double dmul_i(int on, double x, double y) {
    double r;
    if (on && imul64(x, y, r)) return r;
    return x * y;
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

// ============================================================ FP32 form
//
// Particle state and push in binary32.  Lawson RK4 is RK4 applied in the
// frame that turns with the exact E = 0 flow: z = Phi(-t) y, where
// Phi(s) = r(s/eps) is the rotation of eq. TRotationDef with T = 2 pi.  In
// that frame the stiff linear part is gone and z changes only by the field
// increments; the rotation of fine step k is read from a table of
// (cos, sin)(m h/(2 eps)), m = 0 .. 2 spt - 1, computed once on the host in
// FP64.  The table repeats exactly after one turn (spt fine steps), so no
// phase is ever accumulated: each rotation carries one rounding, whatever
// the step.  Times inside a window are kept as an integer number of fine
// steps plus a binary32 fraction in [0, 1) (compensated time).

// Index of the rotation of half-step m (m >= 0) in the table.
__device__ __forceinline__ int rot_index(const DevParams& P, long long m) { return (int)(m % (2 * P.spt)); }

// (Phi(t) z)_R and (Phi(t) z)_V for a table entry cs = (cos, sin)(t/eps).
__device__ __forceinline__ float rot_R(float2 cs, float zR, float zV) { return fmaf(cs.x, zR, cs.y * zV); }
__device__ __forceinline__ float rot_V(float2 cs, float zR, float zV) { return fmaf(cs.x, zV, -(cs.y * zR)); }

// Stage positions of Lawson RK4 from z at fine step k, with a = Phi(t_k),
// m = Phi(t_k + h/2), b = Phi(t_k + h) as table entries:
//   R1 = (a z)_R, R3 = (m z)_R            (stage pair 1: no field needed)
//   R2 = R3 + (h/2) sin(h/(2eps)) e1, R4 = (b z)_R + h sin(h/(2eps)) e3.
__device__ __forceinline__ float lawson32_R2(const DevParams& P, float R3, float e1) { return fmaf(P.h2shh_f, e1, R3); }
__device__ __forceinline__ float lawson32_R4(const DevParams& P, float2 b, float zR, float zV, float e3) {
    return fmaf(P.hshh_f, e3, rot_R(b, zR, zV));
}

// z_{k+1} = z_k + h/6 [ e1 (-sin, cos)_a + 2 (e2 + e3) (-sin, cos)_m + e4 (-sin, cos)_b ]
// (Phi(-t) applied to the field term (0, e) of each stage).
__device__ __forceinline__ void lawson32_update(const DevParams& P, float2 a, float2 m, float2 b, float e1, float e2,
                                                float e3, float e4, float& zR, float& zV) {
    const float e23 = 2.0f * (e2 + e3);
    const float dR = fmaf(e4, b.y, fmaf(e23, m.y, e1 * a.y));
    const float dV = fmaf(e4, b.x, fmaf(e23, m.x, e1 * a.x));
    zR = fmaf(-P.h6_f, dR, zR);
    zV = fmaf(P.h6_f, dV, zV);
}

// A located binary32 position: cell j (or -1 below / -2 at or above the mesh
// or NaN), right weight f (or R itself off the mesh) and qR = floor(f W).
struct Cell32 {
    int j;
    float a;
    unsigned int qR;
};

// x = (R - r_min) * (1/h_r) in binary32, j = floor(x), f = x - j (exact),
// qR = floor(f W) (exact: W is a power of two <= 2^32).  Written without
// branches: off the mesh (or NaN) the cell arithmetic runs on x = 0 and the
// result is replaced.  NEED_Q: compute qR (deposits); the gathers need
// only j and f.
template <bool NEED_Q>
__device__ __forceinline__ Cell32 locate32t(const DevParams& P, float R) {
    const float x = (R - P.r_min_f) * P.inv_hr_f;
    const bool in = x >= 0.0f && x < P.ncells_f;
    const float xc = in ? x : 0.0f;
    const float fl = floorf(xc);
    const float f = xc - fl;
    Cell32 c;
    c.j = in ? (int)fl : (x < 0.0f ? -1 : -2);
    c.a = in ? f : R;
    c.qR = NEED_Q ? __float2uint_rz(f * P.Wf) : 0u;
    return c;
}
__device__ __forceinline__ Cell32 locate32(const DevParams& P, float R) { return locate32t<true>(P, R); }

// Field at a located position from a table of (E_j, E_{j+1} - E_j) per
// cell; off the mesh rE keeps its edge value, E = rE_edge / R (binary32
// fast division: the FP32 form's tolerance covers its 2 ulp).  Branch-free.
__device__ __forceinline__ float gather32(const float2* tab, float rE_lo, float rE_hi, const Cell32& c) {
    const float2 e = tab[c.j > 0 ? c.j : 0];
    const float in = fmaf(c.a, e.y, e.x);
    const float out = __fdividef(c.j == -1 ? rE_lo : rE_hi, c.a);
    return c.j >= 0 ? in : out;
}

__device__ __forceinline__ float field_analytic32(int field, float R) { return field == 1 ? -((R * R) * R) : 0.0f; }

__device__ __forceinline__ bool positive32(float v) { return __float_as_int(v) > 0; }

__device__ __forceinline__ float interp3f(float y0, float y1, float y2, float s) {
    const float d1 = ((-3.0f * y0 + 4.0f * y1) - y2) * 0.5f;
    const float d2 = ((y0 - 2.0f * y1) + y2) * 0.5f;
    return y0 + s * (d1 + s * d2);
}

// binary32 twin of quad_root01.
__device__ __forceinline__ float quad_root01f(float v0, float v1, float v2) {
    const float a = v0;
    const float b = ((-3.0f * v0 + 4.0f * v1) - v2) * 0.5f;
    const float c = ((v0 - 2.0f * v1) + v2) * 0.5f;
    float s;
    if (c == 0.0f) {
        s = (b != 0.0f) ? -a / b : 0.0f;
    } else {
        float disc = b * b - 4.0f * a * c;
        if (disc < 0.0f) disc = 0.0f;
        const float sq = sqrtf(disc);
        const float q = (b >= 0.0f) ? -0.5f * (b + sq) : -0.5f * (b - sq);
        if (q == 0.0f) {
            s = 0.0f;
        } else {
            s = a / q;
            if (!(s >= 0.0f && s <= 1.0f)) s = q / c;
        }
    }
    if (!(s >= 0.0f)) s = 0.0f;
    if (s > 1.0f) s = 1.0f;
    return s;
}

// A time (or period, remainder) in fine steps as i + f, i an integer and
// f in [0, 1) a binary32 fraction.
struct __align__(8) CTime {
    int i;
    float f;
};

__device__ __forceinline__ CTime ct_norm(long long i, float f) {
    const float c = floorf(f);
    i += (long long)c;
    f -= c;
    if (f >= 1.0f) {  // f - c rounded up to 1
        f -= 1.0f;
        ++i;
    }
    CTime t;
    t.i = (int)i;
    t.f = f;
    return t;
}
__device__ __forceinline__ CTime ct_add(CTime a, CTime b) { return ct_norm((long long)a.i + b.i, a.f + b.f); }
__device__ __forceinline__ CTime ct_sub(CTime a, CTime b) { return ct_norm((long long)a.i - b.i, a.f - b.f); }
__device__ __forceinline__ bool ct_less(CTime a, CTime b) { return a.i < b.i || (a.i == b.i && a.f < b.f); }

// Delta t = N T + o with o in [0, T) (eq. TimeStepDec) in compensated time:
// N from the rounded quotient, then o = (Di - N Ti) + (Df - N Tf) with the
// product N Tf split exactly (fma), and N corrected by at most a few steps.
struct Decomp32 {
    CTime T, o;
    int N, need;
};

__device__ __forceinline__ Decomp32 decompose32(const DevParams& P, CTime T) {
    Decomp32 d;
    d.T = T;
    const float Tt = (float)T.i + T.f, Dt = (float)P.Di + P.Df;
    long long N = (long long)floorf(Dt / Tt);
    if (N < 0) N = 0;
    const float Nf = (float)N;
    const float p = Nf * T.f;
    const float pe = fmaf(Nf, T.f, -p);
    CTime o = ct_norm((long long)P.Di - N * (long long)T.i, (P.Df - p) - pe);
    for (int it = 0; it < 4 && o.i < 0; ++it) {
        --N;
        o = ct_add(o, T);
    }
    for (int it = 0; it < 4 && !ct_less(o, T); ++it) {
        ++N;
        o = ct_sub(o, T);
    }
    if (o.i < 0 || N < 0) {  // not reached for a validated T; keeps every sample index >= 0
        o.i = 0;
        o.f = 0.0f;
        if (N < 0) N = 0;
    }
    d.o = o;
    d.N = (int)N;
    const CTime last = d.N > 0 ? ct_add(o, T) : o;
    d.need = last.i + 2;
    return d;
}

// Resolution of a particle's period in the FP32 form (the twin of
// track_resolve): a non-positive period, or samples beyond the window cap,
// take the fallback 2 pi eps (spt fine steps).
__device__ __forceinline__ Decomp32 resolve32(const DevParams& P, CTime T, bool valid, int& flags) {
    // valid: positive, finite, and Delta t / T small enough for the
    // binary32 quotient to fix N to within the correction steps
    const float Tt = (float)T.i + T.f;
    if (!valid || T.i < 0 || !(Tt > 0.0f) || !isfinite(Tt) || !(((float)P.Di + P.Df) / Tt <= 4194304.0f)) {
        flags |= F_FB;
        T.i = P.spt;
        T.f = 0.0f;
    }
    Decomp32 d = decompose32(P, T);
    if (d.need > P.Kmax) {
        flags |= F_FB;
        T.i = P.spt;
        T.f = 0.0f;
        d = decompose32(P, T);
    }
    flags |= F_RES;
    return d;
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

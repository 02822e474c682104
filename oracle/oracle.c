/*
 * Plain FP64 CPU oracle for the improved ETD particle method (Frenod,
 * Hirstoaga & Lutz).  TEST INFRASTRUCTURE ONLY: see oracle.h.
 *
 * Everything here is written as the paper states it, one particle at a time,
 * one RK stage at a time, with no blocking, fusion or reordering.  Where the
 * paper is silent the readings used are stated beside the code:
 *
 *  - Rounding.  Every update of the form y + a*k is evaluated with one
 *    rounding (C99 fma); every other expression is evaluated left to right
 *    exactly as written, with floating-point contraction off at compile time.
 *  - Field (Sec. 2.3: trapezoid rule on a radial mesh of 256 cells): the mesh has
 *    nodes r_j = r_min + j*h_r, j = 0..n_cells, and the node c = n_cells/2 is
 *    r = 0.  Charge is deposited by linear (cloud-in-cell) weights as exact
 *    integers (W units per particle), the trapezoid integral of
 *    d/dr (rE) = rho (eq. VlasPoissAxSymBeam) runs outward from r = 0 on the
 *    integer charges, and E = (1/r) * integral.  At r = 0, E = rho(0).
 *  - Extremum times (Remark CompOfThePeriodsRem): a sign change of V between
 *    samples m and m+1 (V > 0 counts as +, anything else as -) is an
 *    extremum; its time is the root in [0,1] of the quadratic through
 *    V_m, V_{m+1}, V_{m+2} (the interpolation of Remark
 *    QuadraticInterpolationRem applied to V).
 *  - N may be 0 when dt < T (eq. TimeStepDec with o = dt).
 *  - A particle without a third extremum inside the window, or whose samples
 *    would fall beyond it, takes T = 2*pi*eps (the fast period of the E = 0
 *    rotation, Sec. 1).
 */
#include "oracle.h"

#include <math.h>
#include <stdlib.h>
#include <string.h>

#ifndef M_PI
#define M_PI 3.14159265358979323846
#endif

/* ------------------------------------------------------------------ */
/* Parameters                                                          */
/* ------------------------------------------------------------------ */

static int is_pow2_u64(uint64_t w) { return w != 0 && (w & (w - 1)) == 0; }

static int check_params(const orc_params* p) {
    if (!p) return -1;
    if (!(p->eps > 0.0) || !(p->dt > 0.0)) return -1;
    if (p->steps_per_turn < 4) return -1;
    if (p->field_model < 0 || p->field_model > 2) return -1;
    if (p->fine_solver < 0 || p->fine_solver > 1) return -1;
    if (p->max_window_steps < 2 * p->steps_per_turn + 2) return -1;
    if (p->field_parity != 0 && p->field_parity != 1) return -1;
    if (p->field_model == 0) {
        if (p->n_cells < 2 || (p->n_cells & 1)) return -1;
        if (!(p->r_max > 0.0) || p->r_min != -p->r_max) return -1;
        if (!is_pow2_u64(p->weight_fixed) || p->weight_fixed > (1ull << 40)) return -1;
    }
    return 0;
}

int orc_derive(const orc_params* p, orc_derived* d) {
    if (check_params(p) || !d) return -1;
    /* fine step of Remark CompOfThePeriodsRem: (dt)_RK = 2*pi*eps/100 */
    d->h = (2.0 * M_PI * p->eps) / (double)p->steps_per_turn;
    d->inv_eps = 1.0 / p->eps;
    d->D = p->dt / d->h;
    /* exact E = 0 flow over h/2 and h: rotation r(s/eps) of eq. TRotationDef
       with T = 2*pi */
    double th = d->h / p->eps;
    d->c1 = cos(th);
    d->s1 = sin(th);
    d->ch = cos(0.5 * th);
    d->sh = sin(0.5 * th);
    d->hr = (p->r_max - p->r_min) / (double)p->n_cells;
    d->inv_hr = 1.0 / d->hr;
    d->q_unit = 0.0;
    return 0;
}

static double q_unit_of(const orc_params* p, int64_t n_particles) {
    /* weights sum to the total charge (Sec. 2.1): every particle carries W
       fixed-point units of total_charge / (N_p * W). */
    return p->total_charge / ((double)n_particles * (double)p->weight_fixed);
}

/* ------------------------------------------------------------------ */
/* Mesh: deposit, trapezoid integral, gather                           */
/* ------------------------------------------------------------------ */

/* Cloud-in-cell weights of a position: cell j and right weight f in [0,1).
   Returns 0 if R lies outside [r_min, r_max). */
static int cic_cell(const orc_params* p, double inv_hr, double R, int64_t* j, double* f) {
    double x = (R - p->r_min) * inv_hr;
    if (!(x >= 0.0) || !(x < (double)p->n_cells)) return 0;
    double fl = floor(x);
    *j = (int64_t)fl;
    *f = x - fl;
    return 1;
}

int orc_deposit(const orc_params* p, int64_t n, const double* R, int64_t* Q, int64_t* n_out) {
    orc_derived d;
    if (orc_derive(p, &d) || n < 0 || (n > 0 && !R) || !Q) return -1;
    const int64_t W = (int64_t)p->weight_fixed;
    for (int64_t j = 0; j <= p->n_cells; ++j) Q[j] = 0;
    int64_t out = 0;
    for (int64_t i = 0; i < n; ++i) {
        int64_t j;
        double f;
        if (!cic_cell(p, d.inv_hr, R[i], &j, &f)) { ++out; continue; }
        /* right node receives floor(f*W) units, left node the rest */
        int64_t qR = (int64_t)floor(f * (double)W);
        int64_t qL = W - qR;
        Q[j] += qL;
        Q[j + 1] += qR;
    }
    if (n_out) *n_out = out;
    return 0;
}

int orc_deposit_f32(const orc_params* p, int64_t n, const float* R, int64_t* Q, int64_t* n_out) {
    orc_derived d;
    if (orc_derive(p, &d) || n < 0 || (n > 0 && !R) || !Q) return -1;
    const int64_t W = (int64_t)p->weight_fixed;
    const float r_min = (float)p->r_min, inv_hr = (float)d.inv_hr, Wf = (float)W;
    for (int64_t j = 0; j <= p->n_cells; ++j) Q[j] = 0;
    int64_t out = 0;
    for (int64_t i = 0; i < n; ++i) {
        float x = (R[i] - r_min) * inv_hr;
        if (!(x >= 0.0f) || !(x < (float)p->n_cells)) { ++out; continue; }
        float fl = floorf(x);
        int64_t j = (int64_t)fl;
        float f = x - fl;
        int64_t qR = (int64_t)floorf(f * Wf);
        Q[j] += W - qR;
        Q[j + 1] += qR;
    }
    if (n_out) *n_out = out;
    return 0;
}

int orc_poisson(const orc_params* p, int64_t n_particles, const int64_t* Q, int64_t* S_out,
                double* E, double* rE_edges) {
    orc_derived d;
    if (orc_derive(p, &d) || n_particles <= 0 || !Q || !E) return -1;
    const int64_t Nc = p->n_cells, c = Nc / 2;
    int64_t* S = (int64_t*)malloc((size_t)(Nc + 1) * sizeof(int64_t));
    if (!S) return -2;
    /* trapezoid rule from r = 0 outward: the integral over [r_{j-1}, r_j]
       of rho is h_r*(rho_{j-1}+rho_j)/2 = (q_unit/2)*(Q_{j-1}+Q_j), so the
       integer S_j = sum of (Q_{m}+Q_{m+1}) is exact; the left side integrates
       backwards and is negative. */
    S[c] = 0;
    for (int64_t j = c + 1; j <= Nc; ++j) S[j] = S[j - 1] + (Q[j - 1] + Q[j]);
    for (int64_t j = c - 1; j >= 0; --j) S[j] = S[j + 1] - (Q[j] + Q[j + 1]);
    const double q_unit = q_unit_of(p, n_particles);
    const double q_half = 0.5 * q_unit;
    for (int64_t j = 0; j <= Nc; ++j) {
        if (j == c) {
            /* limit r -> 0 of (1/r) * int_0^r rho = rho(0) = Q_c*q_unit/h_r;
               the odd extension is 0 on the axis */
            E[j] = p->field_parity ? 0.0 : ((double)Q[c] * q_unit) * d.inv_hr;
        } else {
            double r_j = p->r_min + (double)j * d.hr;
            double rE = (double)S[j] * q_half;
            E[j] = rE * (1.0 / r_j);
            /* odd extension: rE/|r|, i.e. the sign flips left of the axis */
            if (p->field_parity && j < c) E[j] = -E[j];
        }
    }
    if (rE_edges) {
        /* the off-mesh gather divides the edge value by R: with the odd
           extension the lower edge carries its sign flip (rE/|R| = -rE/R) */
        rE_edges[0] = p->field_parity ? -((double)S[0] * q_half) : (double)S[0] * q_half;
        rE_edges[1] = (double)S[Nc] * q_half;
    }
    if (S_out) memcpy(S_out, S, (size_t)(Nc + 1) * sizeof(int64_t));
    free(S);
    return 0;
}

int orc_gather(const orc_params* p, int64_t n, const double* R, const double* E,
               const double* rE_edges, double* e_out) {
    orc_derived d;
    if (orc_derive(p, &d) || n < 0 || (n > 0 && (!R || !e_out)) || !E || !rE_edges) return -1;
    for (int64_t i = 0; i < n; ++i) {
        int64_t j;
        double f;
        if (cic_cell(p, d.inv_hr, R[i], &j, &f)) {
            /* linear interpolation with the deposit's weights */
            e_out[i] = fma(f, E[j + 1] - E[j], E[j]);
        } else {
            /* outside the mesh rE keeps its edge value (no charge beyond) */
            double x = (R[i] - p->r_min) * d.inv_hr;
            e_out[i] = (x < 0.0 ? rE_edges[0] : rE_edges[1]) / R[i];
        }
    }
    return 0;
}

int orc_field(const orc_params* p, int64_t n, const double* R, double* e_out) {
    if (check_params(p) || n < 0 || (n > 0 && (!R || !e_out))) return -1;
    if (p->field_model == 2) {
        for (int64_t i = 0; i < n; ++i) e_out[i] = 0.0;
        return 0;
    }
    if (p->field_model == 1) {
        /* eq. RappelForce: E = -r^3 */
        for (int64_t i = 0; i < n; ++i) e_out[i] = -((R[i] * R[i]) * R[i]);
        return 0;
    }
    const int64_t Nc = p->n_cells;
    int64_t* Q = (int64_t*)malloc((size_t)(Nc + 1) * sizeof(int64_t));
    double* E = (double*)malloc((size_t)(Nc + 1) * sizeof(double));
    double edges[2];
    int rc = -2;
    if (Q && E) {
        rc = orc_deposit(p, n, R, Q, NULL);
        if (!rc) rc = orc_poisson(p, n, Q, NULL, E, edges);
        if (!rc) rc = orc_gather(p, n, R, E, edges, e_out);
    }
    free(Q);
    free(E);
    return rc;
}

/* ------------------------------------------------------------------ */
/* Fine solvers                                                        */
/* ------------------------------------------------------------------ */

/* One classical RK4 step (the paper's fine solver, Algorithm ClassicETDAlgo
   and Remark CompOfThePeriodsRem) of y' = (V/eps, -R/eps + E(R)) for the
   whole 2*N_p-dimensional system: every stage evaluates the field of all
   stage positions (eq. StiffODEForBeam with (1/eps) M y + L). */
static int step_rk4(const orc_params* p, int64_t n, double* R, double* V, double h,
                    double* w /* 12n scratch */) {
    const double ie = 1.0 / p->eps, h2 = 0.5 * h, h6 = h / 6.0;
    double *e = w, *Rs = w + n, *Vs = w + 2 * n;
    double *k1R = w + 3 * n, *k1V = w + 4 * n, *k2R = w + 5 * n, *k2V = w + 6 * n;
    double *k3R = w + 7 * n, *k3V = w + 8 * n, *k4R = w + 9 * n, *k4V = w + 10 * n;
    int rc;
    /* stage 1 at y */
    if ((rc = orc_field(p, n, R, e))) return rc;
    for (int64_t i = 0; i < n; ++i) {
        k1R[i] = ie * V[i];
        k1V[i] = fma(-ie, R[i], e[i]);
        Rs[i] = fma(h2, k1R[i], R[i]);
        Vs[i] = fma(h2, k1V[i], V[i]);
    }
    /* stage 2 at y + h/2 k1 */
    if ((rc = orc_field(p, n, Rs, e))) return rc;
    for (int64_t i = 0; i < n; ++i) {
        k2R[i] = ie * Vs[i];
        k2V[i] = fma(-ie, Rs[i], e[i]);
    }
    for (int64_t i = 0; i < n; ++i) {
        Rs[i] = fma(h2, k2R[i], R[i]);
        Vs[i] = fma(h2, k2V[i], V[i]);
    }
    /* stage 3 at y + h/2 k2 */
    if ((rc = orc_field(p, n, Rs, e))) return rc;
    for (int64_t i = 0; i < n; ++i) {
        k3R[i] = ie * Vs[i];
        k3V[i] = fma(-ie, Rs[i], e[i]);
    }
    for (int64_t i = 0; i < n; ++i) {
        Rs[i] = fma(h, k3R[i], R[i]);
        Vs[i] = fma(h, k3V[i], V[i]);
    }
    /* stage 4 at y + h k3 */
    if ((rc = orc_field(p, n, Rs, e))) return rc;
    for (int64_t i = 0; i < n; ++i) {
        k4R[i] = ie * Vs[i];
        k4V[i] = fma(-ie, Rs[i], e[i]);
    }
    /* y + h/6 (k1 + 2 k2 + 2 k3 + k4) */
    for (int64_t i = 0; i < n; ++i) {
        double sR = ((k1R[i] + 2.0 * k2R[i]) + 2.0 * k3R[i]) + k4R[i];
        double sV = ((k1V[i] + 2.0 * k2V[i]) + 2.0 * k3V[i]) + k4V[i];
        R[i] = fma(h6, sR, R[i]);
        V[i] = fma(h6, sV, V[i]);
    }
    return 0;
}

/* One Lawson (integrating-factor) RK4 step: the linear part (1/eps) M y of
   eq. StiffODEForBeam is advanced by its exact flow Phi(s) = r(s/eps)
   (eq. TRotationDef with T = 2*pi), RK4 is applied to the twisted variable
   r(-t/eps) y, whose right-hand side is r(-t/eps) L (eq. 13Feb with T=2*pi).
   With g(y) = (0, E(R)):
     k1 = g(y)
     k2 = g(Phi_h/2 (y + h/2 k1))
     k3 = g(Phi_h/2 y + h/2 k2)
     k4 = g(Phi_h y + h Phi_h/2 k3)
     y+ = Phi_h y + h/6 (Phi_h k1 + 2 Phi_h/2 (k2 + k3) + k4)
   where Phi(s)(R,V) = (c R + s V, -s R + c V).  Only second components of
   the k's are nonzero. */
static int step_lawson(const orc_params* p, int64_t n, double* R, double* V, double h,
                       double* w /* 8n scratch */) {
    const double th = h / p->eps;
    const double c1 = cos(th), s1 = sin(th), ch = cos(0.5 * th), sh = sin(0.5 * th);
    const double h2 = 0.5 * h, h6 = h / 6.0, hsh = h * sh, tch = 2.0 * ch, tsh = 2.0 * sh;
    double *e1 = w, *e2 = w + n, *e3 = w + 2 * n, *e4 = w + 3 * n, *Rs = w + 4 * n;
    int rc;
    if ((rc = orc_field(p, n, R, e1))) return rc;
    /* first component of Phi_h/2 (R, V + h/2 e1) */
    for (int64_t i = 0; i < n; ++i) Rs[i] = fma(sh, fma(h2, e1[i], V[i]), ch * R[i]);
    if ((rc = orc_field(p, n, Rs, e2))) return rc;
    /* first component of Phi_h/2 y + h/2 (0, e2) */
    for (int64_t i = 0; i < n; ++i) Rs[i] = fma(sh, V[i], ch * R[i]);
    if ((rc = orc_field(p, n, Rs, e3))) return rc;
    /* first component of Phi_h y + h Phi_h/2 (0, e3) */
    for (int64_t i = 0; i < n; ++i) Rs[i] = fma(hsh, e3[i], fma(s1, V[i], c1 * R[i]));
    if ((rc = orc_field(p, n, Rs, e4))) return rc;
    for (int64_t i = 0; i < n; ++i) {
        double A = fma(s1, V[i], c1 * R[i]);      /* (Phi_h y)_R */
        double B = fma(c1, V[i], -(s1 * R[i]));   /* (Phi_h y)_V */
        double e23 = e2[i] + e3[i];
        R[i] = fma(h6, fma(tsh, e23, s1 * e1[i]), A);
        V[i] = fma(h6, fma(tch, e23, fma(c1, e1[i], e4[i])), B);
    }
    return 0;
}

int orc_fine_steps(const orc_params* p, int64_t n, double* R, double* V, double h_step,
                   int64_t n_fine) {
    if (check_params(p) || n < 0 || n_fine < 0 || !(h_step > 0.0)) return -1;
    if (n == 0 || n_fine == 0) return 0;
    double* w = (double*)malloc((size_t)n * 12 * sizeof(double));
    if (!w) return -2;
    int rc = 0;
    for (int64_t k = 0; k < n_fine && !rc; ++k)
        rc = p->fine_solver == 0 ? step_rk4(p, n, R, V, h_step, w)
                                 : step_lawson(p, n, R, V, h_step, w);
    free(w);
    return rc;
}

int orc_brute_force(const orc_params* p, int64_t n, double* R, double* V, double t) {
    orc_derived d;
    if (orc_derive(p, &d) || !(t >= 0.0)) return -1;
    int64_t nfull = (int64_t)floor(t / d.h);
    int rc = orc_fine_steps(p, n, R, V, d.h, nfull);
    double rem = t - (double)nfull * d.h;
    if (!rc && rem > 0.0) rc = orc_fine_steps(p, n, R, V, rem, 1);
    return rc;
}

/* ------------------------------------------------------------------ */
/* Quadratic interpolation (Remark QuadraticInterpolationRem)          */
/* ------------------------------------------------------------------ */

/* Lagrange quadratic through (0,y0), (1,y1), (2,y2), evaluated at s. */
double orc_interp(double y0, double y1, double y2, double s) {
    double d1 = ((-3.0 * y0 + 4.0 * y1) - y2) * 0.5;
    double d2 = ((y0 - 2.0 * y1) + y2) * 0.5;
    return y0 + s * (d1 + s * d2);
}

/* Root in [0,1] of the same quadratic through (0,v0),(1,v1),(2,v2) when v0
   and v1 have opposite signs; closed form with the cancellation-free choice
   of the two roots, linear when the quadratic term vanishes. */
double orc_quad_root(double v0, double v1, double v2) {
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

/* ------------------------------------------------------------------ */
/* The improved ETD macro step (Algorithm ETDFSSModAlgo)               */
/* ------------------------------------------------------------------ */

typedef struct {
    int     n_ext;      /* extrema found so far               */
    double  t_ext[3];   /* their times (fine steps)           */
    int     resolved;   /* T, o, N known                      */
    int     fallback;   /* took T = steps_per_turn            */
    double  T, o;
    int64_t N, need;    /* last sample index needed           */
} orc_pstate;

/* eq. TimeStepDec: D = N T + o with o in [0,T); the samples needed are the
   three-point stencils at o and, when N > 0, at o + T. */
static void decompose(orc_pstate* s, double D, double T) {
    s->T = T;
    s->o = fmod(D, T);
    s->N = (int64_t)rint((D - s->o) / T);
    double last = (s->N > 0) ? s->o + T : s->o;
    s->need = (int64_t)floor(last) + 2;
}

static void resolve(orc_pstate* s, double D, double T, int64_t Kmax, double T_fallback) {
    if (!(T > 0.0) || !isfinite(T)) {
        s->fallback = 1;
        T = T_fallback;
    }
    decompose(s, D, T);
    if (s->need > Kmax) {
        s->fallback = 1;
        decompose(s, D, T_fallback);
    }
    s->resolved = 1;
}

static int pos(double v) { return v > 0.0; }

/* Window of fine steps from y^n, storing every sample y_k (k = 0..K) in
   traj[k][i] = (R, V).  mode 0: period detection only (step 1); mode 1:
   the full ETD window (steps 1 and 3, or 3 alone when T is known). */
static int run_window(const orc_params* p, const orc_derived* d, int64_t n, double* R, double* V,
                      orc_pstate* ps, int mode, double* traj, int64_t* K_out) {
    const int64_t Kmax = p->max_window_steps;
    const double Tfb = (double)p->steps_per_turn; /* 2*pi*eps in fine steps */
    double* w = (double*)malloc((size_t)(n > 0 ? n : 1) * 12 * sizeof(double));
    if (!w) return -2;
    for (int64_t i = 0; i < n; ++i) {
        traj[2 * i] = R[i];
        traj[2 * i + 1] = V[i];
    }
    int64_t K = 0;
    int rc = 0;
    for (;;) {
        int all = 1;
        for (int64_t i = 0; i < n && all; ++i)
            all = ps[i].resolved && (mode == 0 || K >= ps[i].need);
        if (all) break;
        if (K == Kmax) {
            for (int64_t i = 0; i < n; ++i)
                if (!ps[i].resolved) {
                    ps[i].fallback = 1;
                    if (mode == 0) { ps[i].T = Tfb; ps[i].resolved = 1; }
                    else resolve(&ps[i], d->D, Tfb, Kmax, Tfb);
                }
            break;
        }
        rc = p->fine_solver == 0 ? step_rk4(p, n, R, V, d->h, w)
                                 : step_lawson(p, n, R, V, d->h, w);
        if (rc) break;
        ++K;
        double* row = traj + (size_t)K * (size_t)n * 2;
        for (int64_t i = 0; i < n; ++i) {
            row[2 * i] = R[i];
            row[2 * i + 1] = V[i];
        }
        if (K < 2) continue;
        /* sign change of V between samples m and m+1 (Remark
           CompOfThePeriodsRem), resolved with the stencil m, m+1, m+2 */
        const int64_t m = K - 2;
        const double* r0 = traj + (size_t)m * (size_t)n * 2;
        const double* r1 = r0 + (size_t)n * 2;
        const double* r2 = r1 + (size_t)n * 2;
        for (int64_t i = 0; i < n; ++i) {
            orc_pstate* s = &ps[i];
            if (s->resolved) continue;
            double v0 = r0[2 * i + 1], v1 = r1[2 * i + 1], v2 = r2[2 * i + 1];
            if (pos(v0) == pos(v1)) continue;
            s->t_ext[s->n_ext++] = (double)m + orc_quad_root(v0, v1, v2);
            if (s->n_ext == 3) {
                /* period = time between the first and the third extremum */
                double T = s->t_ext[2] - s->t_ext[0];
                if (mode == 0) { s->T = T; s->resolved = 1; }
                else resolve(s, d->D, T, Kmax, Tfb);
            }
        }
    }
    free(w);
    *K_out = K;
    return rc;
}

int orc_periods(const orc_params* p, int64_t n, const double* R0, const double* V0, double* T,
                int64_t* n_no_period, int64_t* window_steps) {
    orc_derived d;
    if (orc_derive(p, &d) || n < 0 || (n > 0 && (!R0 || !V0 || !T))) return -1;
    const int64_t Kmax = p->max_window_steps;
    double* R = (double*)malloc((size_t)(n > 0 ? n : 1) * sizeof(double));
    double* V = (double*)malloc((size_t)(n > 0 ? n : 1) * sizeof(double));
    orc_pstate* ps = (orc_pstate*)calloc((size_t)(n > 0 ? n : 1), sizeof(orc_pstate));
    double* traj = (double*)malloc((size_t)(Kmax + 1) * (size_t)(n > 0 ? n : 1) * 2 * sizeof(double));
    int rc = -2;
    int64_t K = 0;
    if (R && V && ps && traj) {
        memcpy(R, R0, (size_t)n * sizeof(double));
        memcpy(V, V0, (size_t)n * sizeof(double));
        rc = run_window(p, &d, n, R, V, ps, 0, traj, &K);
    }
    if (!rc) {
        int64_t nf = 0;
        for (int64_t i = 0; i < n; ++i) {
            T[i] = ps[i].T;
            nf += ps[i].fallback;
        }
        if (n_no_period) *n_no_period = nf;
        if (window_steps) *window_steps = K;
    }
    free(R);
    free(V);
    free(ps);
    free(traj);
    return rc;
}

int orc_etd_step(const orc_params* p, int64_t n, double* R, double* V, double* T, int T_known,
                 int64_t* N_out, double* o_out, orc_step_stats* st) {
    orc_derived d;
    if (orc_derive(p, &d) || n < 0 || (n > 0 && (!R || !V || !T))) return -1;
    const int64_t Kmax = p->max_window_steps;
    const double Tfb = (double)p->steps_per_turn;
    orc_pstate* ps = (orc_pstate*)calloc((size_t)(n > 0 ? n : 1), sizeof(orc_pstate));
    double* traj = (double*)malloc((size_t)(Kmax + 1) * (size_t)(n > 0 ? n : 1) * 2 * sizeof(double));
    if (!ps || !traj) {
        free(ps);
        free(traj);
        return -2;
    }
    /* steps 1-2 for known periods (Duffing, Sec. 4.1: periods computed once) */
    if (T_known)
        for (int64_t i = 0; i < n; ++i) resolve(&ps[i], d.D, T[i], Kmax, Tfb);
    /* steps 1 and 3: one fine window from y^n */
    int64_t K = 0;
    int rc = run_window(p, &d, n, R, V, ps, 1, traj, &K);
    if (rc) {
        free(ps);
        free(traj);
        return rc;
    }
    /* steps 3 (interpolation) and 4 (extrapolation, eq. MainFormula1) */
    const size_t row = (size_t)n * 2;
    for (int64_t i = 0; i < n; ++i) {
        const orc_pstate* s = &ps[i];
        double y[2][2];
        double u[2] = {s->o, s->o + s->T};
        int n_t = s->N > 0 ? 2 : 1;
        for (int t = 0; t < n_t; ++t) {
            int64_t k = (int64_t)floor(u[t]);
            double sfrac = u[t] - (double)k;
            const double* a = traj + (size_t)k * row + 2 * (size_t)i;
            for (int c = 0; c < 2; ++c) y[t][c] = orc_interp(a[c], a[c + row], a[c + 2 * row], sfrac);
        }
        if (s->N == 0) {
            R[i] = y[0][0];
            V[i] = y[0][1];
        } else {
            double Nd = (double)s->N;
            R[i] = y[0][0] + Nd * (y[1][0] - y[0][0]);
            V[i] = y[0][1] + Nd * (y[1][1] - y[0][1]);
        }
        if (!T_known) T[i] = s->T;
        if (N_out) N_out[i] = s->N;
        if (o_out) o_out[i] = s->o;
    }
    if (st) {
        st->window_steps = K;
        st->n_no_period = 0;
        st->T_min = INFINITY;
        st->T_max = -INFINITY;
        st->T_mean = 0.0;
        st->N_min = INT64_MAX;
        st->N_max = INT64_MIN;
        for (int64_t i = 0; i < n; ++i) {
            st->n_no_period += ps[i].fallback;
            if (ps[i].T < st->T_min) st->T_min = ps[i].T;
            if (ps[i].T > st->T_max) st->T_max = ps[i].T;
            st->T_mean += ps[i].T;
            if (ps[i].N < st->N_min) st->N_min = ps[i].N;
            if (ps[i].N > st->N_max) st->N_max = ps[i].N;
        }
        if (n > 0) st->T_mean /= (double)n;
    }
    free(ps);
    free(traj);
    return 0;
}

/* ------------------------------------------------------------------ */
/* Duffing appendix                                                    */
/* ------------------------------------------------------------------ */

/* b^2 from eq. b_val, written as x / (eps (sqrt(1+x) + 1)) with
   x = 2 eps (r0^2+v0^2) + eps^2 r0^4 to avoid the cancellation in
   sqrt(1+x) - 1. */
double orc_duffing_b2(double eps, double r0, double v0) {
    double S = r0 * r0 + v0 * v0;
    double x = 2.0 * eps * S + eps * eps * (r0 * r0) * (r0 * r0);
    return x / (eps * (sqrt(1.0 + x) + 1.0));
}

/* Exact period of the appendix, T = 4 eps int_0^1 du / sqrt(1 - u^2 +
   alpha (1 - u^4)), alpha = b^2 eps / 2.  With u = sin(phi) this is
   4 eps int_0^{pi/2} dphi / sqrt((1+alpha) cos^2 phi + (1+2 alpha) sin^2 phi)
   = 2 pi eps / AGM(sqrt(1+alpha), sqrt(1+2 alpha)) (Gauss). */
double orc_duffing_period_agm(double eps, double r0, double v0) {
    double alpha = 0.5 * eps * orc_duffing_b2(eps, r0, v0);
    double a = sqrt(1.0 + alpha), g = sqrt(1.0 + 2.0 * alpha);
    for (int it = 0; it < 64 && fabs(a - g) > 1e-17 * a; ++it) {
        double an = 0.5 * (a + g);
        g = sqrt(a * g);
        a = an;
    }
    return 2.0 * M_PI * eps / a;
}

/* The same integral by the midpoint rule in phi (the integrand is smooth
   and periodic, so the rule converges geometrically). */
double orc_duffing_period_quad(double eps, double r0, double v0, int n_nodes) {
    double alpha = 0.5 * eps * orc_duffing_b2(eps, r0, v0);
    double sum = 0.0, dphi = (0.5 * M_PI) / (double)n_nodes;
    for (int k = 0; k < n_nodes; ++k) {
        double u = sin(((double)k + 0.5) * dphi);
        /* 1 - u^2 + alpha (1 - u^4) = cos^2(phi) (1 + alpha (1 + u^2)) and
           du = cos(phi) dphi */
        sum += 1.0 / sqrt(1.0 + alpha * (1.0 + u * u));
    }
    return 4.0 * eps * sum * dphi;
}

/* eq. 2ndDL_T */
double orc_duffing_period_series(double eps, double r0, double v0) {
    double S = r0 * r0 + v0 * v0;
    double r4 = (r0 * r0) * (r0 * r0);
    return 2.0 * M_PI * eps - (3.0 * M_PI / 4.0) * S * eps * eps +
           ((105.0 * M_PI / 128.0) * S * S - (3.0 * M_PI / 8.0) * r4) * eps * eps * eps;
}

/* eps^2 times the appendix Hamiltonian, written in the (r, v) variables of
   eq. CharactCurvesOfGenVlas (R' = v/eps): (r^2 + v^2)/2 + eps r^4 / 4. */
double orc_duffing_energy(double eps, double r, double v) {
    return 0.5 * (r * r + v * v) + 0.25 * eps * ((r * r) * (r * r));
}

/* ------------------------------------------------------------------ */
/* Classical and modified ETD (Algorithm ClassicETDAlgo)               */
/* ------------------------------------------------------------------ */

/* Delta t = N P + o with 0 <= o < P; y(t_n + P) by the fine solver from y_n
   (exactly steps_per_turn fine steps when P = 2 pi eps, otherwise
   floor(P/h) steps and one step of the rest, as orc_brute_force);
   y(t_n + N P) = y_n + N (y(t_n + P) - y_n) (eq. step2ClassicalETDAlgo);
   y(t_{n+1}) by the fine solver over o from y(t_n + N P). */
int orc_classic_step(const orc_params* p, int64_t n, double* R, double* V, int mode, double* P_out) {
    orc_derived d;
    if (orc_derive(p, &d) || n < 0 || (n > 0 && (!R || !V)) || (mode != 0 && mode != 1)) return -1;
    double P = 2.0 * M_PI * p->eps;
    int rc = 0;
    if (mode == 1 && n > 0) {
        double* T = (double*)malloc((size_t)n * sizeof(double));
        if (!T) return -2;
        rc = orc_periods(p, n, R, V, T, NULL, NULL);
        double sum = 0.0;
        for (int64_t i = 0; i < n; ++i) sum += T[i];
        free(T);
        if (rc) return rc;
        P = (sum / (double)n) * d.h;
    }
    if (P_out) *P_out = P;
    if (n == 0) return 0;
    const double o = fmod(p->dt, P);
    const double N = rint((p->dt - o) / P);
    double* Rn = (double*)malloc((size_t)n * sizeof(double));
    double* Vn = (double*)malloc((size_t)n * sizeof(double));
    if (!Rn || !Vn) {
        free(Rn);
        free(Vn);
        return -2;
    }
    memcpy(Rn, R, (size_t)n * sizeof(double));
    memcpy(Vn, V, (size_t)n * sizeof(double));
    if (mode == 0) rc = orc_fine_steps(p, n, R, V, d.h, p->steps_per_turn);
    else rc = orc_brute_force(p, n, R, V, P);
    if (!rc) {
        for (int64_t i = 0; i < n; ++i) {
            R[i] = Rn[i] + N * (R[i] - Rn[i]);
            V[i] = Vn[i] + N * (V[i] - Vn[i]);
        }
        rc = orc_brute_force(p, n, R, V, o);
    }
    free(Rn);
    free(Vn);
    return rc;
}

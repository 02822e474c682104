/*
 * Plain FP64 CPU oracle for the improved ETD particle method of Frenod,
 * Hirstoaga and Lutz ("Long time simulation of a highly oscillatory Vlasov
 * equation with an exponential integrator", Algorithm 3.3 / label
 * ETDFSSModAlgo).
 *
 * TEST INFRASTRUCTURE ONLY.  This code exists to check the CUDA path.  Only
 * the test suite, the smoke check and the CPU-baseline leg of the benchmark
 * may load it.  It shares no source, header, table or helper with the CUDA
 * library, and the CUDA library never calls it.
 *
 * Conventions (all functions):
 *   - particles are two FP64 arrays R[n], V[n] (the paper's y = (R, V));
 *   - times inside a macro step are measured in fine steps h = 2*pi*eps/S
 *     from the start of the macro step (S = steps_per_turn, 100 in the paper);
 *   - return value 0 = OK, negative = bad argument / allocation failure.
 */
#ifndef PIC_ORACLE_H
#define PIC_ORACLE_H
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct {
    double   eps;              /* epsilon > 0                                  */
    double   dt;               /* macro step Delta t > 0                        */
    int32_t  field_model;      /* 0 Poisson, 1 Duffing E=-r^3, 2 zero field      */
    int32_t  fine_solver;      /* 0 classical RK4 (paper), 1 Lawson RK4          */
    int32_t  steps_per_turn;   /* h = 2*pi*eps / steps_per_turn                  */
    int32_t  n_cells;          /* even; node n_cells/2 sits at r = 0             */
    double   r_min, r_max;     /* r_min = -r_max                                 */
    double   total_charge;     /* sum of the particle weights                   */
    uint64_t weight_fixed;     /* W: fixed-point charge per particle, 2^k        */
    int32_t  max_window_steps; /* cap on the fine window of one macro step       */
    int32_t  field_parity;     /* 0: E = (1/r) int_0^r rho as written (even in r);
                                  1: the odd extension E(r) = rE(r)/|r|, E(0) = 0
                                  (the other reading of eq. VlasPoissAxSymBeam,
                                  for comparison)                               */
} orc_params;

typedef struct {
    double h, inv_eps, D;          /* fine step, 1/eps, dt/h                  */
    double ch, sh, c1, s1;         /* cos/sin(h/(2eps)), cos/sin(h/eps)        */
    double hr, inv_hr;             /* mesh step and its inverse               */
    double q_unit;                 /* charge of one fixed-point unit          */
} orc_derived;

typedef struct {
    int64_t window_steps;          /* fine steps run in the window            */
    int64_t n_no_period;           /* particles that took the 2*pi*eps fallback */
    double  T_min, T_max, T_mean;  /* periods, in fine steps                  */
    int64_t N_min, N_max;          /* whole periods per macro step            */
} orc_step_stats;

int  orc_derive(const orc_params* p, orc_derived* d);

/* Mesh operations (Poisson model). */
int  orc_deposit(const orc_params* p, int64_t n, const double* R,
                 int64_t* Q /* n_cells+1 */, int64_t* n_out);
/* The same deposit with the position arithmetic in binary32: the fixed-point
   split (cell, floor(f W)) is decided in the precision of the FP32 form of
   the CUDA path, as an integer decision must be compared in the precision
   it is taken in.  Positions are given as float. */
int  orc_deposit_f32(const orc_params* p, int64_t n, const float* R, int64_t* Q, int64_t* n_out);
int  orc_poisson(const orc_params* p, int64_t n_particles, const int64_t* Q,
                 int64_t* S /* n_cells+1, may be NULL */, double* E /* n_cells+1 */,
                 double* rE_edges /* 2 */);
int  orc_gather(const orc_params* p, int64_t n, const double* R, const double* E,
                const double* rE_edges, double* e_out);
/* E at every particle position for the configured field model. */
int  orc_field(const orc_params* p, int64_t n, const double* R, double* e_out);

/* Fine solver: n_fine steps of size h_step for the whole particle system. */
int  orc_fine_steps(const orc_params* p, int64_t n, double* R, double* V,
                    double h_step, int64_t n_fine);
/* Reference solution of the paper: fine steps of size h up to time t. */
int  orc_brute_force(const orc_params* p, int64_t n, double* R, double* V, double t);

/* Step 1 alone: periods T[i] (in fine steps) from y^n; returns fallbacks. */
int  orc_periods(const orc_params* p, int64_t n, const double* R, const double* V,
                 double* T, int64_t* n_no_period, int64_t* window_steps);

/* One macro step of Algorithm ETDFSSModAlgo.  If T_known != 0, T[] holds
   the periods (fine steps) and step 1 is skipped; otherwise T[] receives
   them.  N_out/o_out may be NULL. */
int  orc_etd_step(const orc_params* p, int64_t n, double* R, double* V, double* T,
                  int T_known, int64_t* N_out, double* o_out, orc_step_stats* st);

/* One macro step of the classical ETD scheme (Algorithm ClassicETDAlgo) with
   the period P = 2 pi eps (mode 0) or P = the mean over the particles of the
   time of their first complete tour (mode 1: the "modified ETD" of Sec. 2,
   the T_i of Remark CompOfThePeriodsRem averaged in index order).  P_out
   (may be NULL) receives P (time). */
int  orc_classic_step(const orc_params* p, int64_t n, double* R, double* V, int mode, double* P_out);

/* Building blocks exposed for the pin tests. */
double orc_quad_root(double v0, double v1, double v2);
double orc_interp(double y0, double y1, double y2, double s);

/* Duffing appendix: turning point, exact period, series, energy. */
double orc_duffing_b2(double eps, double r0, double v0);
double orc_duffing_period_agm(double eps, double r0, double v0);
double orc_duffing_period_quad(double eps, double r0, double v0, int n_nodes);
double orc_duffing_period_series(double eps, double r0, double v0);
double orc_duffing_energy(double eps, double r, double v);

#ifdef __cplusplus
}
#endif
#endif

/*
 * pic.h -- C ABI of the GB300 (sm_103a) improved-ETD particle-in-cell library.
 *
 * The library advances the axisymmetric-beam Vlasov equation
 *     df/dt + (v/eps) df/dr + (-r/eps + E(r,t)) df/dv = 0
 * (eq. VlasAxSymBeam of Frenod, Hirstoaga & Lutz) with macroparticles
 * (Sec. 2.1) along the characteristics dR/dt = V/eps, dV/dt = -R/eps + E
 * (eq. CharactCurvesOfGenVlas), using the improved ETD scheme (Algorithm
 * ETDFSSModAlgo, Sec. 3).  E comes from the axisymmetric Poisson equation
 * d/dr(rE) = rho, rho = int f dv (eq. VlasPoissAxSymBeam), solved on a radial
 * mesh with the trapezoidal rule (Sec. 2.3), or is the Duffing test field
 * E = -r^3 (eq. RappelForce), or zero.
 *
 * Conventions for every entry point:
 *  - Status: PIC_OK (0) on success, a negative PIC_ERR_* code otherwise.
 *    Nothing throws or aborts across this boundary.  pic_strerror() names a
 *    code.
 *  - Arrays are plain pointers with explicit lengths.  Unless stated, the
 *    caller keeps ownership of everything it passes and the library copies
 *    what it needs.  ptr_kind says whether a pointer is host (PIC_PTR_HOST)
 *    or device (PIC_PTR_DEVICE) memory of the current CUDA device.
 *  - stream is a cudaStream_t passed as void* (NULL = the legacy default
 *    stream).  Work is enqueued on it; calls that return data or a status
 *    synchronise that stream.
 *  - Particle state crosses the boundary as FP64 arrays R[n], V[n] (the
 *    paper's y = (R, V)), whatever the precision the handle computes in
 *    (precision 1 rounds them to binary32 on the way in).  Periods are
 *    reported in units of time, except in checkpoints (fine steps).
 *  - All computation runs in the library's CUDA kernels.  There is no CPU
 *    fallback: without a usable CUDA device, pic_init and the standalone
 *    mesh calls return PIC_ERR_CUDA.
 */
#ifndef PIC_H
#define PIC_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* ---- status codes ------------------------------------------------------ */
#define PIC_OK                 0
#define PIC_ERR_INVALID_ARG   -1  /* a parameter or pointer is out of range  */
#define PIC_ERR_CUDA          -2  /* a CUDA call failed / no usable device   */
#define PIC_ERR_TIMEOUT       -3  /* a device-side wait hit its time limit   */
#define PIC_ERR_OVERFLOW      -4  /* n_particles * weight_fixed >= 2^62      */
#define PIC_ERR_UNSUPPORTED   -5  /* valid request the library does not serve */
#define PIC_ERR_NO_MEMORY     -6  /* device allocation failed                */
#define PIC_ERR_TOO_LARGE     -7  /* beyond a fixed capacity (no-alloc call) */

/* ---- enumerations ------------------------------------------------------ */
enum { PIC_FIELD_POISSON = 0, PIC_FIELD_DUFFING = 1, PIC_FIELD_ZERO = 2 };
/* Two readings of d/dr (rE) = rho (eq. VlasPoissAxSymBeam) on the signed
   radial coordinate: EVEN takes E = (1/r) int_0^r rho as written (E is then
   even in r, E(0) = rho(0)); ODD takes its odd extension E = rE(r)/|r|,
   E(0) = 0, for which (R, V) -> (-R, -V) maps solutions to solutions. */
enum { PIC_PARITY_EVEN = 0, PIC_PARITY_ODD = 1 };
/* Fine solver of steps 1 and 3 of Algorithm ETDFSSModAlgo:
   PIC_FINE_RK4 is the paper's explicit RK4 (Remark CompOfThePeriodsRem);
   PIC_FINE_LAWSON_RK4 advances the linear part (1/eps) M y of
   eq. StiffODEForBeam by its exact rotation and applies RK4 to the field
   term only (integrating-factor RK4). */
enum { PIC_FINE_RK4 = 0, PIC_FINE_LAWSON_RK4 = 1 };
enum { PIC_PTR_HOST = 0, PIC_PTR_DEVICE = 1 };

/* ---- problem statement ------------------------------------------------- */
/* Mirrors the paper's statement of the problem: eps (Sec. 1), the macro step
   Delta t (eq. TimeStepDec), the fine step (dt)_RK = 2*pi*eps/steps_per_turn
   (Remark CompOfThePeriodsRem, 100 in the paper), the radial mesh
   (Sec. 2.3, 256 cells in the paper), the field model and the total charge
   sum(omega_i) = int f0 (Sec. 2.1). */
typedef struct {
    double   eps;              /* > 0                                            */
    double   dt;               /* macro step Delta t > 0                          */
    int32_t  field_model;      /* PIC_FIELD_*                                     */
    int32_t  fine_solver;      /* PIC_FINE_*                                      */
    int32_t  steps_per_turn;   /* >= 4; fine step h = 2*pi*eps/steps_per_turn     */
    int32_t  n_cells;          /* Poisson: even, 2..65536; node n_cells/2 is r=0  */
    double   r_min, r_max;     /* Poisson: r_min = -r_max < 0                     */
    double   total_charge;     /* sum of particle weights (> 0)                   */
    uint64_t weight_fixed;     /* W: fixed-point units per particle, a power of
                                  two <= 2^40, with n_particles*W < 2^62          */
    int32_t  max_window_steps; /* fine steps a window may run; >= 2*spt + 2       */
    int32_t  periods_once;     /* 1: periods computed once at pic_init and kept
                                  (the Duffing case of Sec. 4.1); 0: every step  */
    int32_t  precision;        /* 0 = FP64; 1 = FP32 form: particle state and push
                                  in binary32 (Lawson RK4 in the rotating frame,
                                  compensated integer+fraction times, the field
                                  table from the exact int64 charge in
                                  binary32), FP64 only in pic_moments; needs
                                  PIC_FINE_LAWSON_RK4, W <=
                                  2^32 (Poisson) and dt/h < 2^22, else
                                  PIC_ERR_UNSUPPORTED                            */
    int32_t  block_size;       /* CUDA threads per block, 0 = library default
                                  (1024 Poisson, 128 otherwise)                 */
    int32_t  blocks_per_sm;    /* Poisson window blocks per SM, 0 = default (1)   */
    int32_t  sort_every;       /* macro steps between phase-space sorts of the
                                  particle storage (0 = never, default 1); the
                                  public particle order never changes          */
    int64_t  wait_limit_ns;    /* limit of every device-side wait, 0 = 2 s        */
    int32_t  field_parity;     /* PIC_PARITY_EVEN (default) or PIC_PARITY_ODD     */
    int32_t  reserved;         /* 0                                               */
} pic_params;

/* Fills p with the defaults of the paper-shaped Vlasov-Poisson run:
   eps 0.01, dt 0.1, Poisson, Lawson RK4, 100 steps per turn, 256 cells on
   [-4, 4], total charge 1, W = 2^32, window cap 300, periods every step,
   phase-space sort every macro step. */
void pic_default_params(pic_params* p);

/* ---- handle-based run (the hot path) ----------------------------------- */
typedef struct pic_handle pic_handle;   /* opaque; owns all its device memory */

/* Creates a run of n particles with initial state (r0[i], v0[i]) sampled from
   f0 (Sec. 2.1; the caller samples f0).  The arrays are copied.  With
   periods_once = 1 the periods T_i of y^0 are computed here (Remark
   CompOfThePeriodsRem; Sec. 4.1: "executed only initially").  All later
   work of the handle is enqueued on `stream`.  On success *out receives the
   handle, which the caller releases with pic_destroy. */
int pic_init(const pic_params* p, int64_t n, const double* r0, const double* v0,
             int ptr_kind, void* stream, pic_handle** out);

/* Advances every particle by n_steps macro steps of Algorithm ETDFSSModAlgo:
   (1) periods T_i from y^n: fine steps from t_n until each particle's V has
   changed sign three times, T_i = time between the first and third extremum
   (Remark CompOfThePeriodsRem); (2) Delta t = N_i T_i + o_i, o_i in [0,T_i)
   (eq. TimeStepDec); (3) y_i(t_n+o_i) and y_i(t_n+o_i+T_i) by quadratic
   interpolation of the fine solution (Remark QuadraticInterpolationRem);
   (4) y^{n+1} = y(o) + N (y(o+T) - y(o)) (eq. MainFormula1).  With the
   Poisson model every fine stage is a full field cycle of all particles:
   deposit, trapezoid integral, gather (Sec. 3: every particle is advanced
   through the whole window, since the self-consistent field needs them all).
   Synchronises the stream and returns the device status of the run. */
int pic_step(pic_handle* h, int64_t n_steps);

/* Advances every particle by n_fine fine steps of the fine solver: the
   paper's reference solution (Sec. 2.1, RK4 with step 2*pi*eps/100). */
int pic_fine_steps(pic_handle* h, int64_t n_fine);

/* The paper's reference solution over a time t (Sec. 2.1): floor(t/h) fine
   steps of h = 2 pi eps / steps_per_turn and one last step of the remainder,
   with the configured fine solver and field.  FP64 handles only
   (PIC_ERR_UNSUPPORTED for precision 1, whose rotation tables hold the
   multiples of h only). */
int pic_fine_advance(pic_handle* h, double t);

/* Comparator schemes: n_steps macro steps of the classical ETD scheme
   (Algorithm ClassicETDAlgo): Delta t = N P + o with 0 <= o < P; y(t_n + P)
   by the fine solver from y_n; y(t_n + N P) = y_n + N (y(t_n + P) - y_n)
   (eq. step2ClassicalETDAlgo); y(t_{n+1}) by the fine solver over o.
   period_mode 0: P = 2 pi eps (steps_per_turn fine steps), the classical
   scheme; 1: P = the mean over the particles of their first-tour time
   (Remark CompOfThePeriodsRem; at every step, or from pic_init with
   periods_once), the "modified ETD" scheme of Sec. 2.  Fine solves over a
   time u: floor(u/h) steps and one step of the rest.  *period (may be NULL)
   receives the P of the last step (time); *fine_steps (may be NULL) the
   fine steps its windows ran over all n_steps (the partial steps and the
   period-detection windows included).  pic_window_time then reports all
   its window launches.  FP64 handles only. */
int pic_step_classic(pic_handle* h, int64_t n_steps, int32_t period_mode, double* period, int64_t* fine_steps);

typedef struct {
    double  t;                 /* time reached                                  */
    int64_t n_steps;           /* macro steps taken                             */
    int64_t n_particles;
    int64_t Q_total;           /* sum of the deposited fixed-point charge        */
    int64_t n_out_of_mesh;     /* particles outside [r_min, r_max)              */
    double  charge;            /* Q_total * q_unit + out-of-mesh weight         */
    double  kinetic;           /* sum omega (R^2 + V^2) / 2                     */
    double  duffing_energy;    /* sum omega ((R^2+V^2)/2 + eps R^4/4): eps^2 H of
                                  the appendix, summed                         */
    double  mean_R, mean_V, rms_R, rms_V;
    double  T_min, T_mean, T_max; /* periods of the last macro step (time)     */
    int64_t N_min, N_max;      /* whole periods per macro step, last step       */
    int64_t window_steps;      /* fine steps in the last window                 */
    int64_t n_no_period;       /* particles that took T = 2*pi*eps last step    */
    double  window_ms;         /* device time of the window kernel launches of
                                  the last pic_step call (CUDA events)         */
    int64_t window_launches;   /* window kernel launches of that call           */
    int64_t band_replays;      /* FP64 Poisson ETD windows since pic_init that
                                  replayed with every trajectory row: the
                                  window stores only the rows around the
                                  landing rows forecast from the previous
                                  step's periods, and a landing row outside
                                  them makes it run again (same results)    */
} pic_moments_t;

/* Diagnostics of the current state (computed by device reductions; one small
   device-to-host copy).  Synchronises the stream. */
int pic_moments(pic_handle* h, pic_moments_t* out);

/* Copies R, V (n each) out of / into the handle. */
int pic_get_particles(pic_handle* h, double* r, double* v, int ptr_kind);
int pic_set_particles(pic_handle* h, const double* r, const double* v, int ptr_kind);

/* Per-particle results of the last macro step: T_i (time), N_i, o_i (time).
   Any pointer may be NULL. */
int pic_get_periods(pic_handle* h, double* T, int64_t* N, double* o, int ptr_kind);

/* Field of the current particle positions: Q (n_cells+1, fixed-point units),
   E (n_cells+1) at the nodes, rE at the two mesh edges, out-of-mesh count.
   Any pointer may be NULL.  Poisson model only. */
int pic_get_field(pic_handle* h, int64_t* Q, double* E, double* rE_edges, int64_t* n_out,
                  int ptr_kind);

/* Checkpoint: particle state, periods (in fine steps h, the library's own
   unit), time and step count.  The arrays are caller-owned host memory of
   n_particles doubles each.  Resuming from a checkpoint reproduces an
   uninterrupted run bit for bit. */
typedef struct {
    double* r;
    double* v;
    double* T;
    double  t;
    int64_t n_steps;
} pic_state_t;
int pic_get_state(pic_handle* h, pic_state_t* out);
int pic_set_state(pic_handle* h, const pic_state_t* in);

/* Device time (CUDA events on the handle's stream) of the window kernel
   launches of the last pic_step (or pic_step_classic) call, and their
   number.  Host only. */
int pic_window_time(const pic_handle* h, double* ms, int64_t* launches);

int64_t pic_num_particles(const pic_handle* h);
void pic_destroy(pic_handle* h);
const char* pic_strerror(int status);

/* Device-side kernel launches the handle has issued so far (for benchmarks). */
int64_t pic_launch_count(const pic_handle* h);

/* ---- standalone mesh operations on caller device buffers ---------------- */
/* These run one step of the field cycle on caller-owned device memory.
   Every pointer is device memory; sizes are element counts.  They enqueue
   on `stream` and return without synchronising, except that argument errors
   are reported immediately. */

/* Linear (cloud-in-cell) deposit of n particles at R_dev onto the nodes
   r_j = r_min + j*h_r, j = 0..n_cells (Sec. 2.3): a particle in cell j with
   right weight f gives floor(f*W) units to node j+1 and the rest to node j,
   as exact integers, so Q_dev is bit-exact and independent of order.
   Particles outside [r_min, r_max) deposit nothing and are counted in
   *n_out_dev.  Q_dev (n_cells+1 int64) and n_out_dev (1 int64) are
   overwritten. */
int pic_deposit(const pic_params* p, int64_t n, const double* R_dev, int64_t* Q_dev,
                int64_t* n_out_dev, void* stream);

/* The same deposit with the quantisation of the FP32 form (precision 1):
   x = (R - r_min) * (1/h_r), j = floor(x), f = x - j and floor(f*W) are all
   evaluated in binary32 (r_min and 1/h_r rounded once to binary32), so the
   integer charge of binary32 positions is defined without any FP64 step.
   R_dev holds n binary32 positions; otherwise as pic_deposit. */
int pic_deposit_f32(const pic_params* p, int64_t n, const float* R_dev, int64_t* Q_dev,
                    int64_t* n_out_dev, void* stream);

/* Trapezoid integral of d/dr(rE) = rho (eq. VlasPoissAxSymBeam, Sec. 2.3)
   from r = 0 outward: S_j = sum of (Q_m + Q_{m+1}) over the cells between
   node n_cells/2 and node j (negative on the left), computed as an exact
   int64 prefix scan (warp shuffles + decoupled look-back across blocks);
   then rE_j = S_j * q_unit/2, E_j = rE_j * (1/r_j), and at r = 0
   E = rho(0) = Q * q_unit / h_r, with q_unit = total_charge/(n_particles*W).
   Reads Q_dev (n_cells+1), writes E_dev (n_cells+1) and rE_edges_dev (2:
   rE at r_min and r_max).  Uses device scratch that it allocates and frees
   on the stream. */
int pic_poisson(const pic_params* p, int64_t n_particles, const int64_t* Q_dev, double* E_dev,
                double* rE_edges_dev, void* stream);

/* Same computation and arguments as pic_poisson, for callers that cannot
   allocate device memory when they call it: for example code running inside
   another framework that owns the device memory through its own caching
   allocator, or a time-critical loop that must not stall on (or fail in) an
   allocation.  The paper has no counterpart; it is a deployment variant.
   Its scan scratch is a fixed array inside the library (136 KiB, enough for
   n_cells <= 16384) that every GPU which loads the library keeps until the
   process exits; larger meshes return PIC_ERR_TOO_LARGE and nothing runs.
   It calls no device allocation or free.  The first call on each device
   looks up the array's device address.  All calls share the one array:
   each call clears the parts that must start at zero, and calls whose work
   overlaps on the GPU (different streams, or different host threads,
   without ordering between them) race on it.  Every call synchronises
   `stream` to read the status, so it cannot be made while `stream` is
   being captured into a graph. */
int pic_poisson_noalloc(const pic_params* p, int64_t n_particles, const int64_t* Q_dev, double* E_dev,
                        double* rE_edges_dev, void* stream);

/* E at n positions R_dev by linear interpolation of E_dev with the deposit's
   weights; outside the mesh E = rE_edge / R (rE is constant beyond the
   charge).  Writes e_dev (n). */
int pic_gather(const pic_params* p, int64_t n, const double* R_dev, const double* E_dev,
               const double* rE_edges_dev, double* e_dev, void* stream);

/* Potential of the frozen field that the learned stepper's energy check uses
   (pic_step_learned, step 4): psi(R) = int_0^R E(s) ds, psi(0) = 0, of the
   field a particle feels.  Poisson model: E_dev (n_cells+1) and rE_edges_dev
   (2) as pic_poisson writes them; E is the linear gather of the node values
   inside the mesh (psi is quadratic in each cell; at the nodes it is the
   trapezoid sum of the node field from r = 0, written to psi_nodes_dev,
   n_cells+1) and rE_edge / r beyond an edge (psi grows like rE_edge ln r
   there).  Duffing model (eq. RappelForce): psi = -R^4/4; zero field: 0
   (E_dev, rE_edges_dev and psi_nodes_dev may then be NULL).  Writes
   psi_dev[i] = psi(R_dev[i]) for n positions.  Device pointers; enqueues on
   `stream` without synchronising. */
int pic_frozen_potential(const pic_params* p, const double* E_dev, const double* rE_edges_dev, double* psi_nodes_dev,
                         int64_t n, const double* R_dev, double* psi_dev, void* stream);

/* ---- learned stepper ----------------------------------------------------- */
/* The paper has no learned component: this network is an addition that
   corrects one improved-ETD macro step (Algorithm ETDFSSModAlgo) taken with a
   large Delta t.  It is a 5-64-64-2 perceptron,
       x = (r, v, sin(t/eps), cos(t/eps), dt),
       z1 = W1 x + b1, h1 = gelu(z1), z2 = W2 bf16(h1) + b2, h2 = gelu(z2),
       out = W3 bf16(h2) + b3 = (dR, dV) correction,
   gelu(u) = u erfc(-u/sqrt 2)/2, with W1..W3 the bfloat16 roundings of FP32
   master weights and FP32 accumulation; the hidden layer and its backward run
   on the tensor cores.  Parameters travel as PIC_MLP_PARAMS floats in the
   order W1 (64x5, row-major) | b1 (64) | W2 (64x64) | b2 (64) | W3 (2x64) |
   b3 (2).  Inputs X are n x 5 row-major floats, targets/outputs n x 2. */
#define PIC_MLP_PARAMS 4674
typedef struct pic_mlp pic_mlp;        /* opaque; owns its device memory */
typedef struct {
    float lr, beta1, beta2, eps;       /* Adam on the FP32 master weights */
} pic_adam_t;

int pic_mlp_num_params(void);
/* Creates a network with all weights zero, able to train on batches of up to
   max_batch samples (scratch of ~800 B per sample).  Work runs on stream. */
int pic_mlp_create(int64_t max_batch, void* stream, pic_mlp** out);
/* Copies PIC_MLP_PARAMS master weights in (and resets the Adam state) or out. */
int pic_mlp_set_weights(pic_mlp* m, const float* w, int ptr_kind);
int pic_mlp_get_weights(pic_mlp* m, float* w, int ptr_kind);
/* out = network(X) for n samples (device pointers).  Synchronises. */
int pic_mlp_forward(pic_mlp* m, int64_t n, const float* X_dev, float* Y_dev);
/* Gradient of the loss sum((out - T)^2)/(2n) over n <= max_batch samples
   (device X, T) and the loss itself, without updating the weights; grad
   holds PIC_MLP_PARAMS floats, loss one (host or device per ptr_kind).
   Reductions run in a fixed order: the result is reproducible bit for bit. */
int pic_mlp_gradients(pic_mlp* m, int64_t n, const float* X_dev, const float* T_dev, float* grad, float* loss,
                      int ptr_kind);
/* steps Adam steps on batches of `batch` samples drawn from n_data samples
   (device X, T) along a fixed permutation chosen by seed; loss_hist (host,
   `steps` floats, may be NULL) receives each batch loss.  Synchronises. */
int pic_mlp_train(pic_mlp* m, int64_t n_data, const float* X_dev, const float* T_dev, int64_t batch, int64_t steps,
                  const pic_adam_t* opt, uint64_t seed, float* loss_hist);
/* One Adam step (Kingma & Ba, Algorithm 1) of the master weights with a
   caller-supplied gradient grad (PIC_MLP_PARAMS floats, host or device per
   ptr_kind), in binary32: m = b1 m + (1-b1) g, v = b2 v + (1-b2) g^2,
   w -= lr (m c1) / (sqrt(v c2) + eps) with c1 = 1/(1-b1^t), c2 = 1/(1-b2^t)
   and t the network's Adam step count (pic_mlp_train's steps included; reset
   by pic_mlp_set_weights); then the bfloat16 copies are refreshed.  The same
   update kernel as pic_mlp_train.  Synchronises. */
int pic_mlp_apply_gradient(pic_mlp* m, const float* grad, int ptr_kind, const pic_adam_t* opt);
void pic_mlp_destroy(pic_mlp* m);

/* n_steps macro steps of the learned stepper on a handle.  Each step:
   (1) y^n is kept and, with the Poisson model, the field E of y^n is frozen
   with its potential psi (psi' = E, psi(0) = 0; E = rE_edge/r off the mesh);
   (2) the plain improved-ETD step of pic_step gives y_plain;
   (3) y_learned = y_plain + (scale_R, scale_V) * network(R^n, V^n,
   sin(t_n/eps), cos(t_n/eps), dt), the network's output scaled per
   component;
   (4) each particle keeps y_learned when its frozen-field energy
   H = (R^2 + V^2)/2 - eps psi(R) (psi = -R^4/4 for the Duffing field, 0
   for the zero field) differs from that of y_plain by at most
   drift_tol |H(y_plain)| (the plain step judges the correction), and the
   plain step otherwise.  A zero correction leaves y_plain.  *n_fallback (may be NULL) receives the
   number of particle-steps that kept the plain step.  The network is only
   read.  Synchronises the handle's stream. */
int pic_step_learned(pic_handle* h, const pic_mlp* m, int64_t n_steps, float scale_R, float scale_V,
                     double drift_tol, int64_t* n_fallback);

/* ---- batched form ------------------------------------------------------- */
/* Many independent beams (each its own pic_params: eps, dt, mesh, field
   model; FP32 form, precision = 1) advanced together: one cooperative
   launch per macro step serves every beam, each on a share of the GPU's
   blocks (in proportion to its particles^alloc_power; a quarter weight for
   the analytic fields), with barriers among its own blocks only.  The step
   (reset, launch, status gather) is replayed from a captured CUDA graph,
   captured again after a phase-space sort has moved buffers.  A beam's
   results do not depend on the launch shape, the block share or the sort
   period: every beam computes bit for bit what pic_step computes for it
   alone.  Beam arrays are host memory. */
typedef struct pic_batch pic_batch;
typedef struct {
    int32_t block, blocks_per_sm, grid, sort_every;
    int32_t graph;                     /* 1: steps replay a captured CUDA graph     */
    int32_t graph_error;               /* cudaError_t of a failed capture, else 0   */
    int32_t hist_copies;               /* copies of each block's charge histogram   */
    double  alloc_power;
    int32_t shares_measured;           /* 1: block shares from the beams' measured
                                          window times (pic_batch_tune), 0: in
                                          proportion to N_p^alloc_power        */
} pic_batch_config_t;

int pic_batch_create(int32_t n_beams, const pic_params* params, const int64_t* n_particles,
                     const double* const* r0, const double* const* v0, void* stream, pic_batch** out);
/* n_steps macro steps of every beam.  Synchronises after each step and
   returns the first non-OK device status of any beam. */
int pic_batch_step(pic_batch* b, int64_t n_steps);
/* hist_copies: 1, 2 or 4 copies of each block's charge histogram (lane l
   of a warp deposits into copy l mod hist_copies); more copies take more
   shared memory per block and may leave fewer blocks per SM.  The launch's
   shared memory is sized for hist_copies copies of the largest mesh; a
   Poisson beam with a smaller mesh uses up to 4 copies where they fit in
   it, as long as each of its blocks deposits at least 2048 positions per
   copy and cycle. */
int pic_batch_set_config(pic_batch* b, int32_t block, int32_t blocks_per_sm, double alloc_power,
                         int32_t sort_every, int32_t hist_copies);
int pic_batch_get_config(const pic_batch* b, pic_batch_config_t* out);
/* Autotuner.  For each launch shape (block size x blocks per SM x
   allocation power x histogram copies) that fits, it runs one warm step and
   steps_per_trial timed steps and keeps the shape with the shortest launch
   span (first block start to last block end over all beams, device timer;
   the sorts, which fall into some trials and not others, are not in it).
   Then it times the sort periods 1, 4, 16 over whole periods (at least
   steps_per_trial steps) and keeps the fastest step.  Then it sets block
   shares from the beams' measured window times: a Poisson beam's window is
   predicted to scale as 1/blocks, an analytic beam's with the particles
   one thread advances in turn, and the shares that minimise the largest
   prediction are timed; up to 8 rounds, each predicting from the last
   trial, until two in a row do not shorten the best span by 0.5 %.  The
   shares that timed best stay.  The trial steps are real steps of the
   batch (their results do not depend on the shape or the shares).  *best
   receives the chosen configuration. */
int pic_batch_tune(pic_batch* b, int32_t steps_per_trial, pic_batch_config_t* best);
int pic_batch_get_particles(pic_batch* b, int32_t beam, double* r, double* v, int ptr_kind);
int pic_batch_set_particles(pic_batch* b, int32_t beam, const double* r, const double* v, int ptr_kind);
/* Moments of one beam.  Its window_ms is the beam's own part of the last
   batch step's launch (from the first of its blocks starting to the last
   finishing, on the device's global timer), window_launches 1. */
int pic_batch_moments(pic_batch* b, int32_t beam, pic_moments_t* out);
int64_t pic_batch_steps(const pic_batch* b);
int64_t pic_batch_launch_count(const pic_batch* b);
void pic_batch_destroy(pic_batch* b);

/* ---- testing ------------------------------------------------------------ */
/* Runs one macro step of a small Poisson beam (in the given precision, 0 or
   1) whose grid barrier waits for one more arrival than the grid has, so
   the wait can only end by its time limit (wait_limit_ns, 1 ns..10 s).
   Returns the status pic_step reports: PIC_ERR_TIMEOUT when the limit
   works; the device stays usable.  Exercises the failure path of every
   device-side wait without faulting the GPU. */
int pic_test_barrier_timeout(int64_t wait_limit_ns, int32_t precision, void* stream);
/* The block shares pic_batch_tune gives from measured windows, on plain
   arrays (host arithmetic only: no device call, no GPU needed).  Beam i
   (poisson[i] != 0: Poisson field, else analytic; n_particles[i] >= 1)
   took window_ms[i] on blocks_measured[i] blocks of block_measured
   threads.  Its window on b blocks of `block` threads is predicted as
   window_ms * blocks_measured / b (Poisson) or window_ms * r(b) / r_measured
   with r = ceil(n_particles / (blocks x threads)), the particles one thread
   advances in turn (analytic).  blocks_out[i] lies in [least[i], most[i]],
   their sum is at most `grid`, and the largest predicted window is the
   least any such shares reach (min-max greedy: the beam with the largest
   prediction that more blocks shorten takes them, one block or, for an
   analytic beam, the blocks that remove one particle per thread).  Returns
   PIC_ERR_INVALID_ARG for bad arguments (a count or block size below 1,
   most < least, a negative or non-finite time, block sizes above 2^20,
   block counts or grid above 2^31, particle counts above 2^62),
   PIC_ERR_UNSUPPORTED when the least shares exceed `grid`. */
int pic_test_batch_shares(int32_t n_beams, const int32_t* poisson, const int64_t* n_particles, const double* window_ms,
                          const int64_t* blocks_measured, int32_t block_measured, int32_t block, int64_t grid,
                          const int64_t* least, const int64_t* most, int64_t* blocks_out);

#ifdef __cplusplus
}
#endif
#endif /* PIC_H */

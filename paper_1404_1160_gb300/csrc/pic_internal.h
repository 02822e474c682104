// pic_internal.h -- declarations shared by the library's translation units.
#pragma once

#include <cstddef>
#include <cuda_runtime.h>

#include "pic.h"
#include "pic_device.cuh"

namespace pic {

constexpr int kScanThreads = 256;
constexpr int kScanItems = 8;
constexpr int kScanTile = kScanThreads * kScanItems;

// Device scratch of the decoupled look-back scan.
struct ScanScratch {
    long long* agg;          // per tile: aggregate
    long long* incl;         // per tile: inclusive prefix
    long long* G;            // n_cells+1: exclusive prefix of Q_m + Q_{m+1}
    int* flag;               // per tile: 0 none, 1 aggregate, 2 prefix
    unsigned int* tile_ctr;  // dynamic tile index
    int* status;             // DEV_* of the launch
    size_t zero_from, zero_bytes;
};

size_t scan_scratch_bytes(int n_cells);
size_t scan_scratch_layout(int n_cells, int tiles, void* base, ScanScratch* S);

// R is read as R[i * r_stride].
cudaError_t launch_deposit(const DevParams& P, const double* R, long long n, int r_stride, long long* Q,
                           long long* n_out, cudaStream_t st, int sm_count, long long* launches);
cudaError_t launch_pack(const double* R, const double* V, double2* y, long long n, int sm_count, cudaStream_t st,
                        long long* launches);
cudaError_t launch_extrapolate_classic(double2* y, const double2* y0, long long n, double N, int sm_count,
                                       cudaStream_t st, long long* launches);
cudaError_t launch_unpack(const double2* y, double* R, double* V, long long n, int sm_count, cudaStream_t st,
                          long long* launches);
cudaError_t launch_poisson(const DevParams& P, const long long* Q, double* E, double* edges,
                           const ScanScratch& S, cudaStream_t st, long long* launches);
cudaError_t launch_gather(const DevParams& P, const double* R, long long n, const double* E,
                          const double* edges, double* out, cudaStream_t st, int sm_count,
                          long long* launches);

// Per-particle device state of a window (structure of arrays; pairs are
// interleaved so one 16-byte access moves both).
struct WinBufs {
    double2* y;                 // current fine sample (R, V)
    double *t1, *T, *o;         // first extremum, period, remainder (fine steps)
    double* vp;                 // V_{k-1} of a sign change found at sample k (its root is taken at k+1)
    int* N;                     // whole periods per macro step
    int2* tr;                   // (Track flags, last sample needed)
    double2* ce;                // values carried across a field cycle (fields / partial sums)
    double2* ca;                // W f (or R off the mesh) of the two deposited positions
    short2* cj;                 // cells of the two deposited positions (-1/-2 off the mesh)
    double2* cx;                // RK4: stage positions carried across a cycle
    double* cxr;                // Lawson: (Phi_h y)_R
    double2* traj;              // (Kmax+1) rows of n samples (R, V)
    unsigned long long* Qring;  // 3 cycles x 2 fields x (n_cells+1), one node per kQPad words
    int* notdone;               // 3 cycles; [3] trajectory band missed (this launch); [4] band replays
    unsigned int* bar;          // grid barrier: [0] arrivals, [32] released generation
    int* status;                // DEV_* of the launch
    long long* K_out;           // fine steps of the window
};

// Global charge of a node sits alone on a 128-byte line so the atomics of
// all blocks spread over many L2 slices.
constexpr int kQPad = 16;

enum WindowMode { MODE_PERIODS = 0, MODE_ETD = 1, MODE_FINE = 2 };

struct WindowLaunch {
    int coop_grid = 0, coop_block = 0;
    int hist = 0;             // 0: 32-bit split histograms, 1: 64-bit
    int stage = 0;            // 1: cp.async staging of each warp's next chunk
    size_t coop_smem = 0;
};

// Picks the launch shape and the number of histogram copies (P.hist_copies).
cudaError_t window_prepare(DevParams& P, int block, int blocks_per_sm, int sm_count, WindowLaunch* L);
// Poisson: one cooperative persistent launch per macro step (or per fine run).
cudaError_t launch_window_coop(const DevParams& P, const WinBufs& B, const WindowLaunch& L,
                               int mode, int T_known, long long n_fine, cudaStream_t st,
                               long long* launches, const double* Tin);
// Duffing / zero field: one thread per particle, all n_macro macro steps in
// one launch (no coupling between particles).
cudaError_t launch_window_local(const DevParams& P, const WinBufs& B, int mode, int T_known,
                                long long n_iter, int block, int sm_count, cudaStream_t st,
                                long long* launches, const double* Tin);

// FP32 form (window32.cu).  Rows of the trajectory have a stride of n
// rounded up to a multiple of 128 slots (window32_row_stride); y, tr and
// every row have that many slots, the ones past n being padding.
struct WinBufs32 {
    float2* y;                  // row 0: y^n in storage order
    float2* traj;               // rows 1..Kmax: z_k, row k at traj + (k-1)*ld
    unsigned int* tr;           // Track flags | need << 8
    float2* ce;                 // (e1, e3) of the current step, from the second sweep to the first
    CTime *t1, *T, *o;          // first extremum, period, remainder (fine steps)
    int* N;                     // whole periods per macro step
    unsigned long long* Qring;  // as WinBufs
    int* notdone;
    unsigned int* bar;
    int* status;
    long long* K_out;
    long long ld;               // row stride (slots)
};
long long window32_row_stride(long long n);
// Launch shape of the FP32 window; cudaErrorNotSupported when the mesh does
// not fit in shared memory or a block would deposit more than 2^21
// positions per field and cycle.
cudaError_t window32_prepare(DevParams& P, int block, int blocks_per_sm, int sm_count, long long ld,
                             WindowLaunch* L);
cudaError_t launch_window32_coop(const DevParams& P, const WinBufs32& B, const WindowLaunch& L, int mode,
                                 int T_known, long long n_fine, cudaStream_t st, long long* launches,
                                 const CTime* Tin);
cudaError_t launch_window32_local(const DevParams& P, const WinBufs32& B, int mode, int T_known, long long n_iter,
                                  int block, int sm_count, cudaStream_t st, long long* launches, const CTime* Tin);
// Batched form: many FP32 beams in one cooperative launch.  Block b serves
// the beam whose range [first_block, first_block + n_blocks) holds b.
struct BeamDesc32 {
    DevParams P;
    WinBufs32 B;
    const CTime* Tin;     // periods kept from initialisation (periods_once), or null
    int first_block, n_blocks;
    int coop;             // 1: Poisson (cooperative window), 0: analytic field (per particle)
    int T_known;
    unsigned long long* t_ns;  // [2]: first start and last end (global timer, ns) of the beam's blocks
};
size_t window32_batch_smem(int max_cells, int copies);
cudaError_t window32_batch_attr(size_t smem);
cudaError_t window32_batch_occupancy(int block, size_t smem, int* blocks_per_sm);
cudaError_t launch_window32_batch(const BeamDesc32* beams, int n_beams, int grid, int block, size_t smem,
                                  cudaStream_t st);
// Clears every beam's charge ring, barrier, counters and status (one launch).
cudaError_t launch_batch_reset(const BeamDesc32* beams, int n_beams, cudaStream_t st);
// Copies every beam's status word into out[n_beams].
cudaError_t launch_batch_status(const BeamDesc32* beams, int n_beams, int* out, cudaStream_t st);

// Binary32 deposit (the FP32 form's quantisation), R read as R[i * r_stride].
cudaError_t launch_deposit32(const DevParams& P, const float* R, long long n, int r_stride, long long* Q,
                             long long* n_out, cudaStream_t st, int sm_count, long long* launches);

// Phase-space sort (sort.cu).  The pointers are swapped with their *_alt
// buffers after each sort, so they are held by address.
struct SortBufs {
    double2** y;
    double2** y_alt;
    int** perm;              // slot -> original particle index
    int** perm_alt;
    double** Tin;            // periods kept from pic_init (may be NULL)
    double** Tin_alt;
    int* key;                // n
    unsigned int* count;     // bins
};
size_t sort_scratch_bytes(long long n);
cudaError_t launch_phase_sort(SortBufs& S, long long n, int sm_count, cudaStream_t st, long long* launches);
cudaError_t launch_unpack_perm(const double2* y, const int* perm, long long n, double* R, double* V, int sm_count,
                               cudaStream_t st, long long* launches);
cudaError_t launch_pack_perm(const double* R, const double* V, const int* perm, long long n, double2* y, int sm_count,
                             cudaStream_t st, long long* launches);
cudaError_t launch_permute_d(const double* src, const int* perm, long long n, double scale, int scatter, double* dst,
                             int sm_count, cudaStream_t st, long long* launches);
cudaError_t launch_scatter_i(const int* src, const int* perm, long long n, long long* dst, int sm_count,
                             cudaStream_t st, long long* launches);
cudaError_t launch_iota(int* perm, long long n, int sm_count, cudaStream_t st, long long* launches);
constexpr int kSortBinsTotal = 1024 * 32;

// The same for the FP32 form's storage.
struct SortBufs32 {
    float2** y;
    float2** y_alt;
    int** perm;
    int** perm_alt;
    CTime** Tin;
    CTime** Tin_alt;
    int* key;
    unsigned int* count;
};
cudaError_t launch_phase_sort32(SortBufs32& S, long long n, int sm_count, cudaStream_t st, long long* launches);
cudaError_t launch_unpack_perm32(const float2* y, const int* perm, long long n, double* R, double* V, int sm_count,
                                 cudaStream_t st, long long* launches);
cudaError_t launch_pack_perm32(const double* R, const double* V, const int* perm, long long n, float2* y,
                               int sm_count, cudaStream_t st, long long* launches);
// dst[perm[s]] = (src[s].i + src[s].f) * scale
cudaError_t launch_ctime_out(const CTime* src, const int* perm, long long n, double scale, double* dst,
                             int sm_count, cudaStream_t st, long long* launches);
// dst[s] = split of src[perm[s]] into (floor, fraction)
cudaError_t launch_ctime_in(const double* src, const int* perm, long long n, CTime* dst, int sm_count,
                            cudaStream_t st, long long* launches);

// Reductions for pic_moments: per-block partial sums, combined on the host
// in a fixed order.
constexpr int kMomDoubles = 8;   // sumR sumV sumR2 sumV2 sumR4 sumT minT maxT
constexpr int kMomInts = 3;      // minN maxN n_fallback
cudaError_t launch_moments(const DevParams& P, const WinBufs& B, double* part_d,
                           long long* part_i, int grid, cudaStream_t st, long long* launches);
cudaError_t launch_moments32(const DevParams& P, const WinBufs32& B, double* part_d, long long* part_i, int grid,
                             cudaStream_t st, long long* launches);

}  // namespace pic

namespace pic {
// Learned stepper (mlp.cu): y <- y_plain + scale * net(y_prev, phase, dt) where
// the frozen-field energy allows it.  y_prev / y are the state before and
// after the plain step, in storage order (double2 for precision 0, float2 for 1).
struct LearnedArgs {
    const void* y_prev;
    void* y;
    long long n;
    int prec;
    float in_sin, in_cos, in_dt;   // the inputs shared by every particle
    float scale_R, scale_V;        // output scaling of the network
    double tol;                    // energy-drift limit (relative)
    int field;                     // PIC_FIELD_*
    double eps;
    const double* E;               // Poisson: node field at t_n (n_cells+1)
    const double* psi;             // potential with psi' = E, psi = 0 at r = 0
    const double* edges;           // rE at r_min and r_max
    double r_min, hr, inv_hr;
    int n_cells;
    unsigned long long* n_fallback;
    const float* tab_f;            // Poisson, FP32 form: E_j, slope_j, psi_j in binary32 (3 (n_cells+1))
};
cudaError_t launch_learned_apply(const pic_mlp* m, const LearnedArgs& A, int sm_count, cudaStream_t st,
                                 long long* launches);
// PIC_ERR_TIMEOUT when a tensor-core wait of the network's inference kernel
// ran out of time since the last call (the flag is then cleared), else
// PIC_OK; synchronises st.
int mlp_take_error(const pic_mlp* m, cudaStream_t st);
// psi at the nodes from E at the nodes (trapezoid of the piecewise-linear field);
// with tab_f (3 (n_cells+1) floats, may be null) also the binary32 copies of
// E_j, (E_{j+1} - E_j)/h_r and psi_j for the energy check of the FP32 form.
cudaError_t launch_psi_nodes(const double* E, int n_cells, double hr, double* psi, cudaStream_t st,
                             long long* launches, float* tab_f = nullptr);
// psi at A.n positions R (the energy check's potential), written to out.
cudaError_t launch_psi_eval(const LearnedArgs& A, const double* R, double* out, int sm_count, cudaStream_t st);
}  // namespace pic

namespace pic {
// Poisson prefix integral on caller-provided scan scratch (api.cu).
int poisson_with_scratch(const pic_params* p, int64_t n_particles, const int64_t* Q_dev, double* E_dev,
                         double* rE_edges_dev, const ScanScratch* S, void* stream);
}  // namespace pic

// window.cu -- the fine window of Algorithm ETDFSSModAlgo (Frenod, Hirstoaga
// & Lutz, Sec. 3) for the analytic fields (per-particle window, Duffing and
// zero field) and the launch set-up of both windows.  The cooperative window
// of the self-consistent Poisson field is in window_coop.cuh.
#include "pic_internal.h"
#include "window_common.cuh"
#include "window_coop.cuh"

namespace pic {

// ------------------------------------------- per-particle window (analytic E)

template <int SOLVER, int FIELD>
__device__ __forceinline__ void fine_step(const DevParams& P, double& R, double& V) {
    if (SOLVER == 1) lawson_step_analytic(P, FIELD, R, V);
    else rk4_step_analytic(P, FIELD, R, V);
}

template <int SOLVER, int FIELD>
__global__ void __launch_bounds__(256) k_window_local(DevParams P, WinBufs B, int mode, int T_known,
                                                      long long n_iter, const double* __restrict__ Tin) {
    const long long n = P.n;
    const long long stride = (long long)gridDim.x * blockDim.x;
    int Kmax_seen = 0;
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += stride) {
        const double2 y0 = B.y[i];
        double R = y0.x, V = y0.y;
        if (mode == MODE_FINE) {
            for (long long k = 0; k < n_iter; ++k) fine_step<SOLVER, FIELD>(P, R, V);
            B.y[i] = make_double2(R, V);
            continue;
        }
        if (mode == MODE_PERIODS) {
            Track s;
            s.flags = 0;
            s.t1 = 0.0;
            s.T = 0.0;
            double vkm2 = 0.0;
            int K = 0;
            for (;;) {
                if (track_done(s, K, true)) break;
                if (K == P.Kmax) {
                    track_cap(s, P, true);
                    break;
                }
                const double vkm1 = V;
                fine_step<SOLVER, FIELD>(P, R, V);
                ++K;
                if (K >= 2) track_sample(s, P, K, vkm2, vkm1, V, true);
                vkm2 = vkm1;
            }
            B.T[i] = s.T;
            B.tr[i] = make_int2(s.flags, 0);
            Kmax_seen = max(Kmax_seen, K);
            continue;
        }
        // MODE_ETD: n_iter macro steps of this particle
        Track base;
        base.flags = 0;
        base.t1 = 0.0;
        if (T_known) track_resolve(base, P, Tin[i]);
        Track s = base;
        int K = 0;
        for (long long m = 0; m < n_iter; ++m) {
            double y[2][2];
            if (T_known) {
                // o, T and the stencils are known before the window starts
                s = base;
                const int k1 = (int)floor(s.o);
                const int k2 = s.N > 0 ? (int)floor(s.o + s.T) : -10;
                double a[3], b[3], c[3], d[3];
                K = 0;
                for (;;) {
                    const int r1 = K - k1, r2 = K - k2;
#pragma unroll
                    for (int q = 0; q < 3; ++q) {
                        if (r1 == q) { a[q] = R; b[q] = V; }
                        if (r2 == q) { c[q] = R; d[q] = V; }
                    }
                    if (K >= s.need) break;
                    fine_step<SOLVER, FIELD>(P, R, V);
                    ++K;
                }
                const double s1 = s.o - (double)k1;
                y[0][0] = interp3(a[0], a[1], a[2], s1);
                y[0][1] = interp3(b[0], b[1], b[2], s1);
                if (s.N > 0) {
                    const double s2 = (s.o + s.T) - (double)k2;
                    y[1][0] = interp3(c[0], c[1], c[2], s2);
                    y[1][1] = interp3(d[0], d[1], d[2], s2);
                } else {
                    y[1][0] = y[0][0];
                    y[1][1] = y[0][1];
                }
            } else {
                s.flags = 0;
                s.t1 = 0.0;
                double vkm2 = 0.0;
                K = 0;
                B.traj[i] = make_double2(R, V);
                for (;;) {
                    if (track_done(s, K, false)) break;
                    if (K == P.Kmax) {
                        track_cap(s, P, false);
                        break;
                    }
                    const double vkm1 = V;
                    fine_step<SOLVER, FIELD>(P, R, V);
                    ++K;
                    B.traj[(size_t)K * n + i] = make_double2(R, V);
                    if (K >= 2) track_sample(s, P, K, vkm2, vkm1, V, false);
                    vkm2 = vkm1;
                }
                const int nt = s.N > 0 ? 2 : 1;
                for (int t = 0; t < nt; ++t) {
                    const double u = t == 0 ? s.o : s.o + s.T;
                    const int kk = (int)floor(u);
                    const double sf = u - (double)kk;
                    const double2 p0 = B.traj[(size_t)kk * n + i];
                    const double2 p1 = B.traj[(size_t)(kk + 1) * n + i];
                    const double2 p2 = B.traj[(size_t)(kk + 2) * n + i];
                    y[t][0] = interp3(p0.x, p1.x, p2.x, sf);
                    y[t][1] = interp3(p0.y, p1.y, p2.y, sf);
                }
                if (nt == 1) {
                    y[1][0] = y[0][0];
                    y[1][1] = y[0][1];
                }
            }
            R = extrapolate(y[0][0], y[1][0], s.N);
            V = extrapolate(y[0][1], y[1][1], s.N);
            Kmax_seen = max(Kmax_seen, K);
        }
        B.y[i] = make_double2(R, V);
        if (n_iter > 0) {
            B.T[i] = s.T;
            B.o[i] = s.o;
            B.N[i] = s.N;
            B.tr[i] = make_int2(s.flags, s.need);
        }
    }
    Kmax_seen = __reduce_max_sync(0xffffffffu, (unsigned)Kmax_seen);
    if ((threadIdx.x & 31) == 0 && Kmax_seen > 0) atomicMax((long long*)B.K_out, (long long)Kmax_seen);
}

// ------------------------------------------------------------- moments

__global__ void k_moments(DevParams P, WinBufs B, double* part_d, long long* part_i) {
    __shared__ double sd[32][kMomDoubles];
    __shared__ long long si[32][kMomInts];
    const long long n = P.n, stride = (long long)gridDim.x * blockDim.x;
    double a[kMomDoubles] = {0, 0, 0, 0, 0, 0, INFINITY, -INFINITY};
    long long b[kMomInts] = {LLONG_MAX, LLONG_MIN, 0};
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += stride) {
        const double2 y = B.y[i];
        const double R = y.x, V = y.y, T = B.T[i];
        const double R2 = R * R;
        a[0] += R;
        a[1] += V;
        a[2] += R2;
        a[3] += V * V;
        a[4] += R2 * R2;
        a[5] += T;
        a[6] = fmin(a[6], T);
        a[7] = fmax(a[7], T);
        const long long N = B.N[i];
        b[0] = min(b[0], N);
        b[1] = max(b[1], N);
        b[2] += (B.tr[i].x & F_FB) ? 1 : 0;
    }
    for (int d = 16; d >= 1; d >>= 1) {
        for (int q = 0; q < 6; ++q) a[q] += __shfl_xor_sync(0xffffffffu, a[q], d);
        a[6] = fmin(a[6], __shfl_xor_sync(0xffffffffu, a[6], d));
        a[7] = fmax(a[7], __shfl_xor_sync(0xffffffffu, a[7], d));
        b[0] = min(b[0], __shfl_xor_sync(0xffffffffu, b[0], d));
        b[1] = max(b[1], __shfl_xor_sync(0xffffffffu, b[1], d));
        b[2] += __shfl_xor_sync(0xffffffffu, b[2], d);
    }
    const int w = threadIdx.x >> 5, nw = blockDim.x >> 5;
    if ((threadIdx.x & 31) == 0) {
        for (int q = 0; q < kMomDoubles; ++q) sd[w][q] = a[q];
        for (int q = 0; q < kMomInts; ++q) si[w][q] = b[q];
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        for (int v = 1; v < nw; ++v) {
            for (int q = 0; q < 6; ++q) a[q] += sd[v][q];
            a[6] = fmin(a[6], sd[v][6]);
            a[7] = fmax(a[7], sd[v][7]);
            b[0] = min(b[0], si[v][0]);
            b[1] = max(b[1], si[v][1]);
            b[2] += si[v][2];
        }
        for (int q = 0; q < kMomDoubles; ++q) part_d[(size_t)blockIdx.x * kMomDoubles + q] = a[q];
        for (int q = 0; q < kMomInts; ++q) part_i[(size_t)blockIdx.x * kMomInts + q] = b[q];
    }
}

// ------------------------------------------------------------- launchers

// Shared memory of the window kernel with `copies` histogram copies (at
// least two copies' worth: the histogram region doubles as the int64 scan
// input) and, with staging, two Stage buffers per warp.
static size_t coop_smem_bytes(int n_cells, int copies, int block, int stage, int slot_words) {
    const size_t Np1 = (size_t)n_cells + 1;
    const size_t hc = (size_t)(copies > 2 ? copies : 2);
    return (stage ? (size_t)(block / 32) * kStageBytesPerWarp : 0) + 2 * Np1 * sizeof(double2) +
           hc * 2 * (size_t)slot_words * Np1 * sizeof(unsigned int) + 2 * Np1 * sizeof(long long) +
           Np1 * sizeof(double);
}

// The instantiations of k_window_coop live in window_coop.cu, compiled once
// per (histogram form, solver); each object exports its kernel table.
void* window_coop_kernel_h0_s0(int pow2, int stage);
void* window_coop_kernel_h0_s1(int pow2, int stage);
void* window_coop_kernel_h1_s0(int pow2, int stage);
void* window_coop_kernel_h1_s1(int pow2, int stage);
void* window_coop_kernel_h2_s0(int pow2, int stage);
void* window_coop_kernel_h2_s1(int pow2, int stage);

static void* coop_fn(int solver, int hist, int pow2, int stage) {
    if (hist == 0) return solver == 1 ? window_coop_kernel_h0_s1(pow2, stage) : window_coop_kernel_h0_s0(pow2, stage);
    if (hist == 2) return solver == 1 ? window_coop_kernel_h2_s1(pow2, stage) : window_coop_kernel_h2_s0(pow2, stage);
    return solver == 1 ? window_coop_kernel_h1_s1(pow2, stage) : window_coop_kernel_h1_s0(pow2, stage);
}

cudaError_t window_prepare(DevParams& P, int block, int blocks_per_sm, int sm_count, WindowLaunch* L) {
    L->coop_block = block;
    // staging when the block's shared memory stays within the per-block
    // limit; then as many histogram copies (up to kHistCopiesMax) as fit
    const size_t limit = 220 * 1024;
    // positions one block deposits into one field per cycle: at most the
    // chunks of 32 of one block, with at least one block per SM
    const long long n_chunks = (P.n + 31) / 32;
    long long need_blocks = (P.n + block - 1) / block;
    const long long min_grid = need_blocks < sm_count ? (need_blocks < 1 ? 1 : need_blocks) : sm_count;
    const int slot = (n_chunks + min_grid - 1) / min_grid * 32 > 65536 ? hist_slot_words(2) : hist_slot_words(0);
    L->stage = coop_smem_bytes(P.n_cells, 1, block, 1, slot) <= limit ? 1 : 0;
    int copies = kHistCopiesMax;
    while (copies > 1 && coop_smem_bytes(P.n_cells, copies, block, L->stage, slot) > limit) copies >>= 1;
    P.hist_copies = copies;
    L->coop_smem = coop_smem_bytes(P.n_cells, copies, block, L->stage, slot);
    int bps = 1 << 30;
    for (int hh = 0; hh < 3; ++hh) {
        void* fn = coop_fn(P.solver, hh, P.xs_fma, L->stage);
        cudaError_t e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)L->coop_smem);
        if (e != cudaSuccess) return e;
        int b = 0;
        e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b, fn, block, L->coop_smem);
        if (e != cudaSuccess) return e;
        bps = b < bps ? b : bps;
    }
    if (bps < 1) return cudaErrorInvalidConfiguration;
    const int want = blocks_per_sm > 0 ? blocks_per_sm : 1;
    if (want < bps) bps = want;
    long long grid = (long long)bps * sm_count;
    if (need_blocks < grid) grid = need_blocks < 1 ? 1 : need_blocks;
    L->coop_grid = (int)grid;
    // the split 32-bit histograms need qR < 2^32 (W <= 2^32) and at most
    // 65536 (HIST 0) or 2^21 (HIST 2, when the layout has its fourth word)
    // positions per block, field and cycle
    const long long per_block = (n_chunks + grid - 1) / grid * 32;
    if (P.W > (1ll << 32)) L->hist = 1;
    else if (per_block <= 65536) L->hist = 0;
    else if (slot == hist_slot_words(2) && per_block <= (1ll << 21)) L->hist = 2;
    else L->hist = 1;
    if (L->hist == 1) P.hist_copies = 1;
    return cudaSuccess;
}

cudaError_t launch_window_coop(const DevParams& P, const WinBufs& B, const WindowLaunch& L, int mode,
                               int T_known, long long n_fine, cudaStream_t st, long long* launches,
                               const double* Tin) {
    void* fn = coop_fn(P.solver, L.hist, P.xs_fma, L.stage);
    DevParams Pc = P;
    WinBufs Bc = B;
    void* args[] = {&Pc, &Bc, &mode, &T_known, &n_fine, &Tin};
    cudaError_t e = cudaLaunchCooperativeKernel(fn, dim3(L.coop_grid), dim3(L.coop_block), args, L.coop_smem, st);
    if (launches) ++*launches;
    return e;
}

cudaError_t launch_window_local(const DevParams& P, const WinBufs& B, int mode, int T_known, long long n_iter,
                                int block, int sm_count, cudaStream_t st, long long* launches,
                                const double* Tin) {
    long long want = (P.n + block - 1) / block;
    long long cap = (long long)sm_count * 16;
    int grid = (int)(want < cap ? (want < 1 ? 1 : want) : cap);
    if (P.field == 1) {
        if (P.solver == 1) k_window_local<1, 1><<<grid, block, 0, st>>>(P, B, mode, T_known, n_iter, Tin);
        else k_window_local<0, 1><<<grid, block, 0, st>>>(P, B, mode, T_known, n_iter, Tin);
    } else {
        if (P.solver == 1) k_window_local<1, 2><<<grid, block, 0, st>>>(P, B, mode, T_known, n_iter, Tin);
        else k_window_local<0, 2><<<grid, block, 0, st>>>(P, B, mode, T_known, n_iter, Tin);
    }
    if (launches) ++*launches;
    return cudaGetLastError();
}

cudaError_t launch_moments(const DevParams& P, const WinBufs& B, double* part_d, long long* part_i, int grid,
                           cudaStream_t st, long long* launches) {
    k_moments<<<grid, 256, 0, st>>>(P, B, part_d, part_i);
    if (launches) ++*launches;
    return cudaGetLastError();
}

}  // namespace pic

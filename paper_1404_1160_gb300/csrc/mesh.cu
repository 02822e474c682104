// mesh.cu -- standalone field-cycle kernels: CIC deposit, trapezoid prefix
// integral (decoupled look-back int64 scan) and gather (Sec. 2.3 of Frenod,
// Hirstoaga & Lutz; eq. VlasPoissAxSymBeam).
#include <mutex>

#include "pic.h"
#include "pic_device.cuh"
#include "pic_internal.h"

namespace pic {

// ------------------------------------------------------------------ deposit

// Linear deposit of every particle as exact integers: floor(f W) units to
// the right node, W - floor(f W) to the left one.  Per-block histogram in
// shared memory when it fits, flushed with 64-bit integer atomics, so the
// result does not depend on the order of the additions.
template <int POW2>
__global__ void k_deposit(DevParams P, const double* __restrict__ R, long long n, int r_stride,
                          unsigned long long* __restrict__ Q, unsigned long long* __restrict__ n_out,
                          int use_smem) {
    extern __shared__ unsigned long long hist[];
    const int Np1 = P.n_cells + 1;
    if (use_smem) {
        for (int j = threadIdx.x; j < Np1; j += blockDim.x) hist[j] = 0ull;
        __syncthreads();
    }
    unsigned long long* H = use_smem ? hist : Q;
    unsigned int out = 0;
    const long long stride = (long long)gridDim.x * blockDim.x;
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += stride) {
        Cell c = mesh_locate<POW2>(P, R[i * r_stride]);
        if (c.j >= 0) {
            atomicAdd(&H[c.j], (unsigned long long)(P.W - c.qR));
            if (c.qR) atomicAdd(&H[c.j + 1], (unsigned long long)c.qR);
        } else {
            ++out;
        }
    }
    out = __reduce_add_sync(0xffffffffu, out);
    if ((threadIdx.x & 31) == 0 && out) atomicAdd(n_out, (unsigned long long)out);
    if (use_smem) {
        __syncthreads();
        for (int j = threadIdx.x; j < Np1; j += blockDim.x) {
            unsigned long long v = hist[j];
            if (v) atomicAdd(&Q[j], v);
        }
    }
}

// The same deposit with the binary32 quantisation of the FP32 form:
// x = (R - r_min)/h_r, j = floor(x), f = x - j and floor(f W) all in
// binary32 (W a power of two, so f W is exact).
__global__ void k_deposit32(DevParams P, const float* __restrict__ R, long long n, int r_stride,
                            unsigned long long* __restrict__ Q, unsigned long long* __restrict__ n_out, int use_smem) {
    extern __shared__ unsigned long long hist32[];
    const int Np1 = P.n_cells + 1;
    if (use_smem) {
        for (int j = threadIdx.x; j < Np1; j += blockDim.x) hist32[j] = 0ull;
        __syncthreads();
    }
    unsigned long long* H = use_smem ? hist32 : Q;
    unsigned int out = 0;
    const long long stride = (long long)gridDim.x * blockDim.x;
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += stride) {
        const Cell32 c = locate32(P, R[i * r_stride]);
        if (c.j >= 0) {
            const unsigned long long qR = __float2ull_rz(c.a * P.Wf);
            atomicAdd(&H[c.j], (unsigned long long)P.W - qR);
            if (qR) atomicAdd(&H[c.j + 1], qR);
        } else {
            ++out;
        }
    }
    out = __reduce_add_sync(0xffffffffu, out);
    if ((threadIdx.x & 31) == 0 && out) atomicAdd(n_out, (unsigned long long)out);
    if (use_smem) {
        __syncthreads();
        for (int j = threadIdx.x; j < Np1; j += blockDim.x) {
            const unsigned long long v = hist32[j];
            if (v) atomicAdd(&Q[j], v);
        }
    }
}

// ------------------------------------------------- decoupled look-back scan

__device__ __forceinline__ void st_release_s32(int* p, int v) {
    asm volatile("st.release.gpu.global.s32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}

__device__ __forceinline__ long long warp_incl_scan(long long x) {
    const int lane = threadIdx.x & 31;
#pragma unroll
    for (int d = 1; d < 32; d <<= 1) {
        long long y = __shfl_up_sync(0xffffffffu, x, d);
        if (lane >= d) x += y;
    }
    return x;
}

// G_j = sum_{m<j} (Q_m + Q_{m+1}), j = 0..n_cells, in one pass: each block
// scans a tile with warp shuffles, then its first thread looks back over
// the published aggregates/prefixes of earlier tiles (tiles are taken in
// launch order through an atomic counter, so every tile it waits on is
// already running).  Each wait has a time limit that sets the status word.
__global__ void __launch_bounds__(kScanThreads) k_scan_pairs(DevParams P, const long long* __restrict__ Q,
                                                             ScanScratch S) {
    __shared__ int s_tile;
    __shared__ long long s_warp[kScanThreads / 32];
    __shared__ long long s_excl;
    const int Nc = P.n_cells;
    if (threadIdx.x == 0) s_tile = (int)atomicAdd(S.tile_ctr, 1u);
    __syncthreads();
    const int tile = s_tile;
    const long long base = (long long)tile * kScanTile + (long long)threadIdx.x * kScanItems;
    long long v[kScanItems];
    long long sum = 0;
#pragma unroll
    for (int k = 0; k < kScanItems; ++k) {
        long long m = base + k;
        v[k] = (m < Nc) ? Q[m] + Q[m + 1] : 0;
        sum += v[k];
    }
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    long long incl = warp_incl_scan(sum);
    if (lane == 31) s_warp[w] = incl;
    __syncthreads();
    if (w == 0) {
        long long y = (lane < kScanThreads / 32) ? s_warp[lane] : 0;
        y = warp_incl_scan(y);
        if (lane < kScanThreads / 32) s_warp[lane] = y;
    }
    __syncthreads();
    const long long total = s_warp[kScanThreads / 32 - 1];
    const long long in_block = incl - sum + (w > 0 ? s_warp[w - 1] : 0);
    if (threadIdx.x == 0) {
        long long excl = 0;
        if (tile == 0) {
            S.incl[0] = total;
            st_release_s32(&S.flag[0], 2);
        } else {
            S.agg[tile] = total;
            st_release_s32(&S.flag[tile], 1);
            int p = tile - 1;
            long long t0 = 0;
            unsigned spins = 0;
            while (p >= 0) {
                int f = ld_acquire_s32(&S.flag[p]);
                if (f == 2) {
                    excl += __ldcg(&S.incl[p]);
                    break;
                }
                if (f == 1) {
                    excl += __ldcg(&S.agg[p]);
                    --p;
                    continue;
                }
                if ((++spins & 63) == 0) {
                    long long now = global_ns();
                    if (t0 == 0) t0 = now;
                    else if (now - t0 > P.wait_ns) {
                        atomicCAS(S.status, 0, (int)DEV_TIMEOUT);
                        break;
                    }
                }
            }
            S.incl[tile] = excl + total;
            st_release_s32(&S.flag[tile], 2);
        }
        s_excl = excl;
    }
    __syncthreads();
    long long run = s_excl + in_block;
#pragma unroll
    for (int k = 0; k < kScanItems; ++k) {
        long long m = base + k;
        if (m < Nc) {
            S.G[m] = run;
            if (m == Nc - 1) S.G[Nc] = run + v[k];
        }
        run += v[k];
    }
}

// S_j = G_j - G_c (the integral from r = 0), rE_j = S_j q_unit/2,
// E_j = rE_j * (1/r_j); at r = 0, E = rho(0) = Q_c q_unit / h_r.
__global__ void k_field_from_prefix(DevParams P, const long long* __restrict__ Q,
                                    const long long* __restrict__ G, double* __restrict__ E,
                                    double* __restrict__ edges) {
    const int Nc = P.n_cells, c = P.c;
    const long long Gc = G[c];
    for (int j = blockIdx.x * blockDim.x + threadIdx.x; j <= Nc; j += gridDim.x * blockDim.x) {
        long long S = G[j] - Gc;
        double e;
        if (j == c) {
            e = P.parity_odd ? 0.0 : ((double)Q[c] * P.q_unit) * P.inv_hr;
        } else {
            double r = P.r_min + (double)j * P.hr;
            e = ((double)S * P.q_half) * (1.0 / r);
            if (P.parity_odd && j < c) e = -e;  // odd reading: rE / |r|
        }
        E[j] = e;
        // the off-mesh gather divides the edge rE by R; the odd reading's
        // lower edge carries the sign flip
        if (j == 0) edges[0] = P.parity_odd ? -((double)S * P.q_half) : (double)S * P.q_half;
        if (j == Nc) edges[1] = (double)S * P.q_half;
    }
}

// ------------------------------------------------------------------ gather

template <int POW2>
__global__ void k_gather(DevParams P, const double* __restrict__ R, long long n,
                         const double* __restrict__ E, const double* __restrict__ edges,
                         double* __restrict__ out, int use_smem) {
    extern __shared__ double2 tab[];
    const int Nc = P.n_cells;
    if (use_smem) {
        for (int j = threadIdx.x; j < Nc; j += blockDim.x)
            tab[j] = make_double2(E[j], (E[j + 1] - E[j]) * P.invW);
        __syncthreads();
    }
    const double lo = edges[0], hi = edges[1];
    const long long stride = (long long)gridDim.x * blockDim.x;
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += stride) {
        Cell c = mesh_locate<POW2>(P, R[i]);
        double e;
        if (use_smem) {
            e = mesh_gather(tab, lo, hi, c.j, c.a);
        } else if (c.j >= 0) {
            double ej = E[c.j];
            e = fma(c.a, (E[c.j + 1] - ej) * P.invW, ej);
        } else {
            e = gather_outside(lo, hi, c.j, c.a);
        }
        out[i] = e;
    }
}

// ------------------------------------------------------------ (R, V) packing

__global__ void k_pack(const double* __restrict__ R, const double* __restrict__ V, double2* __restrict__ y,
                       long long n) {
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
        y[i] = make_double2(R[i], V[i]);
}

__global__ void k_unpack(const double2* __restrict__ y, double* __restrict__ R, double* __restrict__ V,
                         long long n) {
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
        const double2 v = y[i];
        if (R) R[i] = v.x;
        if (V) V[i] = v.y;
    }
}

// y = y0 + N (y - y0) (eq. step2ClassicalETDAlgo), element by element.
__global__ void k_extrapolate_classic(double2* __restrict__ y, const double2* __restrict__ y0, long long n, double N) {
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
        const double2 a = y0[i], b = y[i];
        y[i] = make_double2(a.x + N * (b.x - a.x), a.y + N * (b.y - a.y));
    }
}

// ------------------------------------------------------------ host launchers

static int grid_for(long long n, int sm_count) {
    long long want = (n + 255) / 256;
    long long cap = (long long)sm_count * 8;
    return (int)(want < 1 ? 1 : (want < cap ? want : cap));
}

cudaError_t launch_extrapolate_classic(double2* y, const double2* y0, long long n, double N, int sm_count,
                                       cudaStream_t st, long long* launches) {
    if (n == 0) return cudaSuccess;
    k_extrapolate_classic<<<grid_for(n, sm_count), 256, 0, st>>>(y, y0, n, N);
    if (launches) ++*launches;
    return cudaGetLastError();
}

cudaError_t launch_pack(const double* R, const double* V, double2* y, long long n, int sm_count, cudaStream_t st,
                        long long* launches) {
    if (n == 0) return cudaSuccess;
    k_pack<<<grid_for(n, sm_count), 256, 0, st>>>(R, V, y, n);
    if (launches) ++*launches;
    return cudaGetLastError();
}

cudaError_t launch_unpack(const double2* y, double* R, double* V, long long n, int sm_count, cudaStream_t st,
                          long long* launches) {
    if (n == 0) return cudaSuccess;
    k_unpack<<<grid_for(n, sm_count), 256, 0, st>>>(y, R, V, n);
    if (launches) ++*launches;
    return cudaGetLastError();
}

cudaError_t launch_deposit(const DevParams& P, const double* R, long long n, int r_stride, long long* Q,
                           long long* n_out, cudaStream_t st, int sm_count, long long* launches) {
    const int Np1 = P.n_cells + 1;
    cudaError_t e = cudaMemsetAsync(Q, 0, sizeof(long long) * (size_t)Np1, st);
    if (e == cudaSuccess) e = cudaMemsetAsync(n_out, 0, sizeof(long long), st);
    if (e != cudaSuccess || n == 0) return e;
    size_t smem = sizeof(unsigned long long) * (size_t)Np1;
    int use_smem = smem <= 96 * 1024;
    auto fn = P.xs_fma ? k_deposit<1> : k_deposit<0>;
    if (use_smem && smem > 48 * 1024) cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    long long want = (n + 255) / 256;
    int grid = (int)(want < (long long)sm_count * 4 ? want : (long long)sm_count * 4);
    fn<<<grid, 256, use_smem ? smem : 0, st>>>(P, R, n, r_stride, (unsigned long long*)Q, (unsigned long long*)n_out,
                                               use_smem);
    if (launches) ++*launches;
    return cudaGetLastError();
}

cudaError_t launch_deposit32(const DevParams& P, const float* R, long long n, int r_stride, long long* Q,
                             long long* n_out, cudaStream_t st, int sm_count, long long* launches) {
    const int Np1 = P.n_cells + 1;
    cudaError_t e = cudaMemsetAsync(Q, 0, sizeof(long long) * (size_t)Np1, st);
    if (e == cudaSuccess) e = cudaMemsetAsync(n_out, 0, sizeof(long long), st);
    if (e != cudaSuccess || n == 0) return e;
    size_t smem = sizeof(unsigned long long) * (size_t)Np1;
    int use_smem = smem <= 96 * 1024;
    if (use_smem && smem > 48 * 1024) cudaFuncSetAttribute(k_deposit32, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    long long want = (n + 255) / 256;
    int grid = (int)(want < (long long)sm_count * 4 ? want : (long long)sm_count * 4);
    k_deposit32<<<grid, 256, use_smem ? smem : 0, st>>>(P, R, n, r_stride, (unsigned long long*)Q,
                                                        (unsigned long long*)n_out, use_smem);
    if (launches) ++*launches;
    return cudaGetLastError();
}

size_t scan_scratch_bytes(int n_cells) {
    const int tiles = (n_cells + kScanTile - 1) / kScanTile;
    return scan_scratch_layout(n_cells, tiles, nullptr, nullptr);
}

size_t scan_scratch_layout(int n_cells, int tiles, void* base, ScanScratch* S) {
    // agg, incl (tiles int64 each), G (n_cells+1 int64), flag (tiles int32),
    // tile counter and status (int32 each); every piece 256-byte aligned.
    auto up = [](size_t x) { return (x + 255) & ~(size_t)255; };
    size_t off_agg = 0;
    size_t off_incl = up(off_agg + sizeof(long long) * tiles);
    size_t off_G = up(off_incl + sizeof(long long) * tiles);
    size_t off_flag = up(off_G + sizeof(long long) * (size_t)(n_cells + 1));
    size_t off_ctr = up(off_flag + sizeof(int) * tiles);
    size_t off_status = up(off_ctr + sizeof(unsigned int));
    size_t total = up(off_status + sizeof(int));
    if (S && base) {
        char* b = (char*)base;
        S->agg = (long long*)(b + off_agg);
        S->incl = (long long*)(b + off_incl);
        S->G = (long long*)(b + off_G);
        S->flag = (int*)(b + off_flag);
        S->tile_ctr = (unsigned int*)(b + off_ctr);
        S->status = (int*)(b + off_status);
        S->zero_from = off_flag;  // flags, counter and status must start at zero
        S->zero_bytes = total - off_flag;
    }
    return total;
}

cudaError_t launch_poisson(const DevParams& P, const long long* Q, double* E, double* edges,
                           const ScanScratch& S, cudaStream_t st, long long* launches) {
    const int tiles = (P.n_cells + kScanTile - 1) / kScanTile;
    cudaError_t e = cudaMemsetAsync((char*)S.flag, 0, S.zero_bytes, st);
    if (e != cudaSuccess) return e;
    k_scan_pairs<<<tiles, kScanThreads, 0, st>>>(P, Q, S);
    int fgrid = (P.n_cells + 1 + 255) / 256;
    k_field_from_prefix<<<fgrid, 256, 0, st>>>(P, Q, S.G, E, edges);
    if (launches) *launches += 2;
    return cudaGetLastError();
}

cudaError_t launch_gather(const DevParams& P, const double* R, long long n, const double* E,
                          const double* edges, double* out, cudaStream_t st, int sm_count,
                          long long* launches) {
    if (n == 0) return cudaSuccess;
    size_t smem = sizeof(double2) * (size_t)P.n_cells;
    int use_smem = smem <= 96 * 1024;
    auto fn = P.xs_fma ? k_gather<1> : k_gather<0>;
    if (use_smem && smem > 48 * 1024) cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    long long want = (n + 255) / 256;
    int grid = (int)(want < (long long)sm_count * 4 ? want : (long long)sm_count * 4);
    fn<<<grid, 256, use_smem ? smem : 0, st>>>(P, R, n, E, edges, out, use_smem);
    if (launches) ++*launches;
    return cudaGetLastError();
}

}  // namespace pic

// ----------------------------------------------- scan without allocation

namespace pic {

// Fixed device scratch for pic_poisson_noalloc: the look-back tile states,
// the prefix G and the status word of one scan of at most
// kNoAllocMaxCells cells.  Every GPU that loads the library holds it until
// the process exits.
constexpr int kNoAllocMaxCells = 16384;
constexpr size_t kNoAllocScratchBytes = 136 * 1024;
static __device__ __align__(256) unsigned char g_poisson_scratch[kNoAllocScratchBytes];

}  // namespace pic

extern "C" int pic_poisson_noalloc(const pic_params* p, int64_t n_particles, const int64_t* Q_dev, double* E_dev,
                                   double* rE_edges_dev, void* stream) {
    // Host code cannot use g_poisson_scratch's name as a device address: the
    // address is looked up once per device (with that device current) and
    // cached.  This set-up happens in the first call on each device.
    static std::mutex mu;
    static void* scratch_addr[256] = {};
    if (!p) return PIC_ERR_INVALID_ARG;
    // a mesh too small for the layout arithmetic below is a bad argument
    // (the full parameter check runs in the shared body)
    if (p->n_cells < 2) return PIC_ERR_INVALID_ARG;
    if (p->n_cells > pic::kNoAllocMaxCells) return PIC_ERR_TOO_LARGE;
    if (n_particles <= 0 || !Q_dev || !E_dev || !rE_edges_dev) return PIC_ERR_INVALID_ARG;
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 256) return PIC_ERR_CUDA;
    void* base = nullptr;
    {
        std::lock_guard<std::mutex> lock(mu);
        if (!scratch_addr[dev]) {
            void* a = nullptr;
            if (cudaGetSymbolAddress(&a, pic::g_poisson_scratch) != cudaSuccess || !a) return PIC_ERR_CUDA;
            scratch_addr[dev] = a;
        }
        base = scratch_addr[dev];
    }
    const int tiles = (p->n_cells + pic::kScanTile - 1) / pic::kScanTile;
    if (pic::scan_scratch_layout(p->n_cells, tiles, nullptr, nullptr) > pic::kNoAllocScratchBytes) return PIC_ERR_TOO_LARGE;
    pic::ScanScratch S;
    pic::scan_scratch_layout(p->n_cells, tiles, base, &S);
    return pic::poisson_with_scratch(p, n_particles, Q_dev, E_dev, rE_edges_dev, &S, stream);
}

// sort.cu -- periodic phase-space sort of the particles and the permutation
// bookkeeping that keeps the public particle order unchanged.
//
// The beam rotates almost rigidly with period ~2 pi eps (Sec. 1), so particles
// that start a macro step at the same phase-space angle and amplitude stay
// together for the whole fine window: a warp of such particles changes the
// sign of V in the same fine step (no divergence in the period detection),
// deposits into one or two cells (warp-aggregated atomics) and reads the same
// field-table entries.  The key is computed in FP32 and only orders the
// particles; every result is independent of the order (integer deposit, per
// particle arithmetic), so the sort does not change any output bit.
#include "pic_internal.h"

namespace pic {

constexpr int kSortAngleBins = 1024;
constexpr int kSortAmpBins = 32;
constexpr int kSortBins = kSortAngleBins * kSortAmpBins;
constexpr int kSortScanThreads = 1024;

__device__ __forceinline__ int phase_key(float R, float V) {
    const float ang = atan2f(V, R);                          // (-pi, pi]
    int a = (int)((ang + 3.14159265f) * (kSortAngleBins / 6.28318531f));
    a = a < 0 ? 0 : (a >= kSortAngleBins ? kSortAngleBins - 1 : a);
    const float amp2 = R * R + V * V;
    int b = (int)(kSortAmpBins * (amp2 / (1.0f + amp2)));     // monotone map of [0, inf) to [0, bins)
    b = b < 0 ? 0 : (b >= kSortAmpBins ? kSortAmpBins - 1 : b);
    return a * kSortAmpBins + b;
}

// Bin counts.  Particles that are already in key order share bins within a
// warp, so the lanes of one bin add their count with a single atomic.  The
// loop runs over whole warps (lanes past n carry no key).
template <typename Y>
__global__ void k_sort_keys(const Y* __restrict__ y, long long n, int* __restrict__ key,
                            unsigned int* __restrict__ count) {
    const int lane = threadIdx.x & 31;
    const long long stride = (long long)gridDim.x * blockDim.x;
    for (long long b = (long long)blockIdx.x * blockDim.x + (threadIdx.x & ~31); b < n; b += stride) {
        const long long i = b + lane;
        const bool valid = i < n;
        int k = -1;
        if (valid) {
            const Y v = y[i];
            k = phase_key((float)v.x, (float)v.y);
            key[i] = k;
        }
        const unsigned int peers = __match_any_sync(0xffffffffu, (unsigned int)k);
        if (valid && lane == __ffs(peers) - 1) atomicAdd(&count[k], (unsigned int)__popc(peers));
    }
}

// Exclusive scan of the bin counts in one block (kSortBins entries).
__global__ void __launch_bounds__(kSortScanThreads) k_sort_scan(unsigned int* __restrict__ count) {
    __shared__ unsigned int s_warp[kSortScanThreads / 32];
    constexpr int per = kSortBins / kSortScanThreads;
    const int t = threadIdx.x, lane = t & 31, w = t >> 5;
    unsigned int v[per];
    unsigned int s = 0;
#pragma unroll
    for (int q = 0; q < per; ++q) {
        v[q] = count[t * per + q];
        s += v[q];
    }
    unsigned int x = s;
#pragma unroll
    for (int d = 1; d < 32; d <<= 1) {
        const unsigned int y = __shfl_up_sync(0xffffffffu, x, d);
        if (lane >= d) x += y;
    }
    if (lane == 31) s_warp[w] = x;
    __syncthreads();
    if (w == 0) {
        unsigned int y = s_warp[lane];
#pragma unroll
        for (int d = 1; d < 32; d <<= 1) {
            const unsigned int z = __shfl_up_sync(0xffffffffu, y, d);
            if (lane >= d) y += z;
        }
        s_warp[lane] = y;
    }
    __syncthreads();
    unsigned int run = x - s + (w > 0 ? s_warp[w - 1] : 0u);
#pragma unroll
    for (int q = 0; q < per; ++q) {
        count[t * per + q] = run;
        run += v[q];
    }
}

// Moves every particle (state, original index, and the kept periods) to
// its slot in key order; the lanes of a warp that share a bin take
// consecutive slots from one atomic.
template <typename Y, typename TT>
__global__ void k_sort_scatter(const Y* __restrict__ y, const int* __restrict__ perm, const TT* __restrict__ Tin,
                               const int* __restrict__ key, long long n, unsigned int* __restrict__ cursor,
                               Y* __restrict__ y_out, int* __restrict__ perm_out, TT* __restrict__ Tin_out) {
    const int lane = threadIdx.x & 31;
    const long long stride = (long long)gridDim.x * blockDim.x;
    for (long long b = (long long)blockIdx.x * blockDim.x + (threadIdx.x & ~31); b < n; b += stride) {
        const long long i = b + lane;
        const bool valid = i < n;
        const int k = valid ? key[i] : -1;
        const unsigned int peers = __match_any_sync(0xffffffffu, (unsigned int)k);
        const int leader = __ffs(peers) - 1;
        unsigned int base = 0;
        if (valid && lane == leader) base = atomicAdd(&cursor[k], (unsigned int)__popc(peers));
        base = __shfl_sync(0xffffffffu, base, leader);
        if (!valid) continue;
        const unsigned int d = base + (unsigned int)__popc(peers & ((1u << lane) - 1u));
        y_out[d] = y[i];
        perm_out[d] = perm[i];
        if (Tin) Tin_out[d] = Tin[i];
    }
}

// ------------------------------------------------ permuted copies in and out

// out[perm[s]] = (y[s].x, y[s].y)
__global__ void k_unpack_perm(const double2* __restrict__ y, const int* __restrict__ perm, long long n,
                              double* __restrict__ R, double* __restrict__ V) {
    for (long long s = (long long)blockIdx.x * blockDim.x + threadIdx.x; s < n; s += (long long)gridDim.x * blockDim.x) {
        const double2 v = y[s];
        const long long i = perm[s];
        if (R) R[i] = v.x;
        if (V) V[i] = v.y;
    }
}

// y[s] = (R[perm[s]], V[perm[s]])
__global__ void k_pack_perm(const double* __restrict__ R, const double* __restrict__ V,
                            const int* __restrict__ perm, long long n, double2* __restrict__ y) {
    for (long long s = (long long)blockIdx.x * blockDim.x + threadIdx.x; s < n; s += (long long)gridDim.x * blockDim.x) {
        const long long i = perm[s];
        y[s] = make_double2(R[i], V[i]);
    }
}

// dst[perm[s]] = src[s] * scale (scatter) or dst[s] = src[perm[s]] (gather)
__global__ void k_permute_d(const double* __restrict__ src, const int* __restrict__ perm, long long n,
                            double scale, int scatter, double* __restrict__ dst) {
    for (long long s = (long long)blockIdx.x * blockDim.x + threadIdx.x; s < n; s += (long long)gridDim.x * blockDim.x) {
        if (scatter) dst[perm[s]] = src[s] * scale;
        else dst[s] = src[perm[s]];
    }
}

__global__ void k_scatter_i(const int* __restrict__ src, const int* __restrict__ perm, long long n,
                            long long* __restrict__ dst) {
    for (long long s = (long long)blockIdx.x * blockDim.x + threadIdx.x; s < n; s += (long long)gridDim.x * blockDim.x)
        dst[perm[s]] = (long long)src[s];
}

__global__ void k_iota(int* __restrict__ perm, long long n) {
    for (long long s = (long long)blockIdx.x * blockDim.x + threadIdx.x; s < n; s += (long long)gridDim.x * blockDim.x)
        perm[s] = (int)s;
}

// ------------------------------------------------------------ launchers

static int grid_of(long long n, int sm_count) {
    const long long want = (n + 255) / 256, cap = (long long)sm_count * 8;
    return (int)(want < 1 ? 1 : (want < cap ? want : cap));
}

size_t sort_scratch_bytes(long long n) {
    return sizeof(int) * (size_t)n + sizeof(unsigned int) * (size_t)kSortBins;
}

cudaError_t launch_phase_sort(SortBufs& S, long long n, int sm_count, cudaStream_t st, long long* launches) {
    if (n == 0) return cudaSuccess;
    cudaError_t e = cudaMemsetAsync(S.count, 0, sizeof(unsigned int) * kSortBins, st);
    if (e != cudaSuccess) return e;
    const int g = grid_of(n, sm_count);
    k_sort_keys<double2><<<g, 256, 0, st>>>(*S.y, n, S.key, S.count);
    k_sort_scan<<<1, kSortScanThreads, 0, st>>>(S.count);
    k_sort_scatter<double2, double><<<g, 256, 0, st>>>(*S.y, *S.perm, S.Tin ? *S.Tin : nullptr, S.key, n, S.count, *S.y_alt,
                                      *S.perm_alt, S.Tin ? *S.Tin_alt : nullptr);
    if (launches) *launches += 3;
    e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    double2* ty = *S.y;
    *S.y = *S.y_alt;
    *S.y_alt = ty;
    int* tp = *S.perm;
    *S.perm = *S.perm_alt;
    *S.perm_alt = tp;
    if (S.Tin) {
        double* tt = *S.Tin;
        *S.Tin = *S.Tin_alt;
        *S.Tin_alt = tt;
    }
    return cudaSuccess;
}

cudaError_t launch_unpack_perm(const double2* y, const int* perm, long long n, double* R, double* V, int sm_count,
                               cudaStream_t st, long long* launches) {
    if (n == 0) return cudaSuccess;
    k_unpack_perm<<<grid_of(n, sm_count), 256, 0, st>>>(y, perm, n, R, V);
    if (launches) ++*launches;
    return cudaGetLastError();
}

cudaError_t launch_pack_perm(const double* R, const double* V, const int* perm, long long n, double2* y, int sm_count,
                             cudaStream_t st, long long* launches) {
    if (n == 0) return cudaSuccess;
    k_pack_perm<<<grid_of(n, sm_count), 256, 0, st>>>(R, V, perm, n, y);
    if (launches) ++*launches;
    return cudaGetLastError();
}

cudaError_t launch_permute_d(const double* src, const int* perm, long long n, double scale, int scatter, double* dst,
                             int sm_count, cudaStream_t st, long long* launches) {
    if (n == 0) return cudaSuccess;
    k_permute_d<<<grid_of(n, sm_count), 256, 0, st>>>(src, perm, n, scale, scatter, dst);
    if (launches) ++*launches;
    return cudaGetLastError();
}

cudaError_t launch_scatter_i(const int* src, const int* perm, long long n, long long* dst, int sm_count, cudaStream_t st,
                             long long* launches) {
    if (n == 0) return cudaSuccess;
    k_scatter_i<<<grid_of(n, sm_count), 256, 0, st>>>(src, perm, n, dst);
    if (launches) ++*launches;
    return cudaGetLastError();
}

cudaError_t launch_iota(int* perm, long long n, int sm_count, cudaStream_t st, long long* launches) {
    if (n == 0) return cudaSuccess;
    k_iota<<<grid_of(n, sm_count), 256, 0, st>>>(perm, n);
    if (launches) ++*launches;
    return cudaGetLastError();
}

// ------------------------------------------------------------ FP32 storage

__global__ void k_unpack_perm32(const float2* __restrict__ y, const int* __restrict__ perm, long long n,
                                double* __restrict__ R, double* __restrict__ V) {
    for (long long s = (long long)blockIdx.x * blockDim.x + threadIdx.x; s < n; s += (long long)gridDim.x * blockDim.x) {
        const float2 v = y[s];
        const long long i = perm[s];
        if (R) R[i] = (double)v.x;
        if (V) V[i] = (double)v.y;
    }
}

// y[s] = binary32 rounding (to nearest even) of (R, V)[perm[s]]
__global__ void k_pack_perm32(const double* __restrict__ R, const double* __restrict__ V,
                              const int* __restrict__ perm, long long n, float2* __restrict__ y) {
    for (long long s = (long long)blockIdx.x * blockDim.x + threadIdx.x; s < n; s += (long long)gridDim.x * blockDim.x) {
        const long long i = perm[s];
        y[s] = make_float2(__double2float_rn(R[i]), __double2float_rn(V[i]));
    }
}

__global__ void k_ctime_out(const CTime* __restrict__ src, const int* __restrict__ perm, long long n, double scale,
                            double* __restrict__ dst) {
    for (long long s = (long long)blockIdx.x * blockDim.x + threadIdx.x; s < n; s += (long long)gridDim.x * blockDim.x) {
        const CTime t = src[s];
        dst[perm[s]] = ((double)t.i + (double)t.f) * scale;
    }
}

__global__ void k_ctime_in(const double* __restrict__ src, const int* __restrict__ perm, long long n,
                           CTime* __restrict__ dst) {
    for (long long s = (long long)blockIdx.x * blockDim.x + threadIdx.x; s < n; s += (long long)gridDim.x * blockDim.x) {
        const double x = src[perm[s]];
        CTime t;
        if (x >= -2147483648.0 && x < 2147483647.0) {
            const double fl = floor(x);
            t.i = (int)fl;
            t.f = __double2float_rn(x - fl);
            if (t.f >= 1.0f) {
                t.f = 0.0f;
                ++t.i;
            }
        } else {
            t.i = -1;  // not a usable period: the window takes the fallback
            t.f = 0.0f;
        }
        dst[s] = t;
    }
}

cudaError_t launch_phase_sort32(SortBufs32& S, long long n, int sm_count, cudaStream_t st, long long* launches) {
    if (n == 0) return cudaSuccess;
    cudaError_t e = cudaMemsetAsync(S.count, 0, sizeof(unsigned int) * kSortBins, st);
    if (e != cudaSuccess) return e;
    const int g = grid_of(n, sm_count);
    k_sort_keys<float2><<<g, 256, 0, st>>>(*S.y, n, S.key, S.count);
    k_sort_scan<<<1, kSortScanThreads, 0, st>>>(S.count);
    k_sort_scatter<float2, CTime><<<g, 256, 0, st>>>(*S.y, *S.perm, S.Tin ? *S.Tin : nullptr, S.key, n, S.count,
                                                      *S.y_alt, *S.perm_alt, S.Tin ? *S.Tin_alt : nullptr);
    if (launches) *launches += 3;
    e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    float2* ty = *S.y;
    *S.y = *S.y_alt;
    *S.y_alt = ty;
    int* tp = *S.perm;
    *S.perm = *S.perm_alt;
    *S.perm_alt = tp;
    if (S.Tin) {
        CTime* tt = *S.Tin;
        *S.Tin = *S.Tin_alt;
        *S.Tin_alt = tt;
    }
    return cudaSuccess;
}

cudaError_t launch_unpack_perm32(const float2* y, const int* perm, long long n, double* R, double* V, int sm_count,
                                 cudaStream_t st, long long* launches) {
    if (n == 0) return cudaSuccess;
    k_unpack_perm32<<<grid_of(n, sm_count), 256, 0, st>>>(y, perm, n, R, V);
    if (launches) ++*launches;
    return cudaGetLastError();
}

cudaError_t launch_pack_perm32(const double* R, const double* V, const int* perm, long long n, float2* y,
                               int sm_count, cudaStream_t st, long long* launches) {
    if (n == 0) return cudaSuccess;
    k_pack_perm32<<<grid_of(n, sm_count), 256, 0, st>>>(R, V, perm, n, y);
    if (launches) ++*launches;
    return cudaGetLastError();
}

cudaError_t launch_ctime_out(const CTime* src, const int* perm, long long n, double scale, double* dst,
                             int sm_count, cudaStream_t st, long long* launches) {
    if (n == 0) return cudaSuccess;
    k_ctime_out<<<grid_of(n, sm_count), 256, 0, st>>>(src, perm, n, scale, dst);
    if (launches) ++*launches;
    return cudaGetLastError();
}

cudaError_t launch_ctime_in(const double* src, const int* perm, long long n, CTime* dst, int sm_count,
                            cudaStream_t st, long long* launches) {
    if (n == 0) return cudaSuccess;
    k_ctime_in<<<grid_of(n, sm_count), 256, 0, st>>>(src, perm, n, dst);
    if (launches) ++*launches;
    return cudaGetLastError();
}

}  // namespace pic

// window_common.cuh -- device pieces shared by the FP64 and FP32 window
// kernels: the block-wide int64 scan of the charge, the bounded grid barrier
// and the cp.async helpers.  Everything is static/inline, so each
// translation unit keeps its own copy.
#pragma once

#include "pic_internal.h"

namespace pic {

static __device__ __forceinline__ long long warp_incl_scan64(long long x) {
    const int lane = threadIdx.x & 31;
#pragma unroll
    for (int d = 1; d < 32; d <<= 1) {
        const long long y = __shfl_up_sync(0xffffffffu, x, d);
        if (lane >= d) x += y;
    }
    return x;
}

// For both fields f = 0, 1: g_j = sum_{m<j} (q_m + q_{m+1}), j = 0..Nc
// (block-wide exclusive scans in shared memory, done together).
static __device__ void block_exscan_pairs2(const long long* q, long long* g, int Nc, long long* s_warp) {
    const int T = blockDim.x, t = threadIdx.x, lane = t & 31, w = t >> 5, nw = T >> 5;
    const int Np1 = Nc + 1;
    const int per = (Nc + T - 1) / T;
    const int beg = min(t * per, Nc), end = min(beg + per, Nc);
    long long s0 = 0, s1 = 0;
    for (int m = beg; m < end; ++m) {
        s0 += q[m] + q[m + 1];
        s1 += q[Np1 + m] + q[Np1 + m + 1];
    }
    const long long x0 = warp_incl_scan64(s0), x1 = warp_incl_scan64(s1);
    if (lane == 31) {
        s_warp[w] = x0;
        s_warp[32 + w] = x1;
    }
    __syncthreads();
    if (w == 0) {
        long long y0 = (lane < nw) ? s_warp[lane] : 0, y1 = (lane < nw) ? s_warp[32 + lane] : 0;
        y0 = warp_incl_scan64(y0);
        y1 = warp_incl_scan64(y1);
        if (lane < nw) {
            s_warp[lane] = y0;
            s_warp[32 + lane] = y1;
        }
    }
    __syncthreads();
    long long r0 = x0 - s0 + (w > 0 ? s_warp[w - 1] : 0);
    long long r1 = x1 - s1 + (w > 0 ? s_warp[32 + w - 1] : 0);
    for (int m = beg; m < end; ++m) {
        g[m] = r0;
        g[Np1 + m] = r1;
        r0 += q[m] + q[m + 1];
        r1 += q[Np1 + m] + q[Np1 + m + 1];
    }
    if (end == Nc && beg < end) {
        g[Nc] = r0;
        g[Np1 + Nc] = r1;
    }
    __syncthreads();
}

// Barrier of the n_blocks blocks that share `bar` (the whole grid, or the
// blocks of one beam of a batch), with a time limit; false if any block
// timed out or failed.
// Arrivals count on bar[0]; the last block of a generation publishes the
// generation number in bar[32] (another cache line), which the others poll.
static __device__ __forceinline__ bool grid_sync(const DevParams& P, unsigned int* bar, unsigned int& gen,
                                          int* status, int* s_ok, unsigned int n_blocks) {
    __syncthreads();
    ++gen;
    if (threadIdx.x == 0) {
        const unsigned int target = gen * (n_blocks + P.bar_extra);
        __threadfence();
        const unsigned int old = atomicAdd(bar, 1u);
        int ok = 1;
        if (old + 1 == target) {
            asm volatile("st.release.gpu.global.u32 [%0], %1;" ::"l"(bar + 32), "r"(gen) : "memory");
        } else {
            long long t0 = 0;
            unsigned spins = 0;
            while ((int)(ld_acquire_u32(bar + 32) - gen) < 0) {
                if ((++spins & 31) == 0) {
                    if (ld_acquire_s32(status) != 0) {
                        ok = 0;
                        break;
                    }
                    const long long now = global_ns();
                    if (t0 == 0) {
                        t0 = now;
                    } else if (now - t0 > P.wait_ns) {
                        atomicCAS(status, 0, (int)DEV_TIMEOUT);
                        ok = 0;
                        break;
                    }
                }
            }
        }
        __threadfence();
        *s_ok = ok;
    }
    __syncthreads();
    return *s_ok != 0;
}

// ---- asynchronous copies global -> shared (cp.async, sm_80+)

static __device__ __forceinline__ void cp_async16(void* smem, const void* gmem) {
    const unsigned int d = (unsigned int)__cvta_generic_to_shared(smem);
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(d), "l"(gmem) : "memory");
}
static __device__ __forceinline__ void cp_async8(void* smem, const void* gmem) {
    const unsigned int d = (unsigned int)__cvta_generic_to_shared(smem);
    asm volatile("cp.async.ca.shared.global [%0], [%1], 8;" ::"r"(d), "l"(gmem) : "memory");
}
static __device__ __forceinline__ void cp_async4(void* smem, const void* gmem) {
    const unsigned int d = (unsigned int)__cvta_generic_to_shared(smem);
    asm volatile("cp.async.ca.shared.global [%0], [%1], 4;" ::"r"(d), "l"(gmem) : "memory");
}
static __device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
template <int N>
static __device__ __forceinline__ void cp_async_wait() {
    asm volatile("cp.async.wait_group %0;" ::"n"(N) : "memory");
}

}  // namespace pic

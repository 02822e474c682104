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

// Charge to field of one cycle for both fields, with the nodes in registers
// (three block barriers and no shared staging).  The first half of the
// block takes field 0, the second field 1; in warp w of a half, lane l < 31
// owns the R nodes j = (31 w + l) R + r, r < R, and lane 31 repeats the
// first nodes of the next warp, so that every lane finds E_{j+1} of its
// last node in the next lane.  q_j comes from the cycle's global charge Qg;
// the exact trapezoid sums g_j = sum_{m<j} (q_m + q_{m+1}) are a warp scan
// plus the totals of the preceding warps (s_tot), S_j = g_j - g_c, and the
// node field is field_at(j, S_j, q_j) (binary64 or binary32: its type is
// the table's).  Each owned node is passed to emit(f, j, E_j, E_{j+1}, S_j)
// (E_{j+1} unused at j = n_cells).  Covers n_cells + 1 <= 31 R (blockDim/64)
// nodes; returns false (doing nothing) when R = 4 would not suffice.
// s_tot: 64 int64.
template <int R, class FieldAt, class Emit>
static __device__ __forceinline__ void field_build_regs_r(const DevParams& P, const unsigned long long* Qg,
                                                          long long* s_tot, FieldAt field_at, Emit emit) {
    using Val = decltype(field_at(0, 0ll, 0ll));
    const int Nc = P.n_cells, Np1 = Nc + 1, c = P.c;
    const int H = blockDim.x >> 1;
    const int f = threadIdx.x >= H ? 1 : 0;
    const int u = threadIdx.x - f * H, lane = threadIdx.x & 31, w = u >> 5;
    const int j0 = (w * 31 + lane) * R;
    const unsigned long long* Qf = Qg + (size_t)f * Np1 * kQPad;
    long long q[R];
#pragma unroll
    for (int r = 0; r < R; ++r) q[r] = (j0 + r <= Nc) ? (long long)__ldcg(Qf + (size_t)(j0 + r) * kQPad) : 0ll;
    const long long qn = __shfl_down_sync(0xffffffffu, q[0], 1);
    long long L = 0;
#pragma unroll
    for (int r = 0; r < R; ++r) {
        const long long right = (r + 1 < R) ? q[(r + 1) % R] : qn;
        L += (j0 + r < Nc) ? q[r] + right : 0ll;
    }
    if (lane == 31) L = 0;  // its nodes belong to the next warp
    const long long incl = warp_incl_scan64(L);
    if (lane == 31) s_tot[f * 32 + w] = incl;
    __syncthreads();
    // warps whose first node lies beyond the mesh own no node (warp-uniform)
    const bool owns = w * 31 * R <= Nc;
    long long g0 = incl - L;
    if (owns) {
        // totals of the preceding warps of the half (w <= 15), summed by a butterfly
        long long t = lane < w ? s_tot[f * 32 + lane] : 0ll;
#pragma unroll
        for (int d = 16; d >= 1; d >>= 1) t += __shfl_xor_sync(0xffffffffu, t, d);
        g0 += t;
        long long g = g0;
#pragma unroll
        for (int r = 0; r < R; ++r) {
            if (lane != 31 && j0 + r == c) s_tot[f * 32 + 16] = g;
            if (r + 1 < R) g += (j0 + r < Nc) ? q[r] + q[(r + 1) % R] : 0ll;
        }
    }
    __syncthreads();
    if (!owns) return;
    const long long gc = s_tot[f * 32 + 16];
    auto value = [&](int j, long long S, long long qj) -> Val { return j > Nc ? Val(0) : field_at(j, S, qj); };
    long long S = g0 - gc;
    Val Ecur = value(j0, S, q[0]);
    const Val En = __shfl_down_sync(0xffffffffu, Ecur, 1);
#pragma unroll
    for (int r = 0; r < R; ++r) {
        const int j = j0 + r;
        long long Sn = S;
        Val Enext = En;
        if (r + 1 < R) {
            Sn = S + ((j < Nc) ? q[r] + q[(r + 1) % R] : 0ll);
            Enext = value(j + 1, Sn, q[(r + 1) % R]);
        }
        if (lane != 31 && j <= Nc) emit(f, j, Ecur, Enext, S);
        Ecur = Enext;
        S = Sn;
    }
}

template <class FieldAt, class Emit>
static __device__ __forceinline__ bool field_build_regs_with(const DevParams& P, const unsigned long long* Qg,
                                                             long long* s_tot, FieldAt field_at, Emit emit) {
    const int per_pass = 31 * (int)(blockDim.x >> 6);  // nodes covered per node of a thread
    const int Np1 = P.n_cells + 1;
    if ((blockDim.x & 63) != 0 || blockDim.x > 1024) return false;
    if (Np1 <= per_pass) field_build_regs_r<1>(P, Qg, s_tot, field_at, emit);
    else if (Np1 <= 2 * per_pass) field_build_regs_r<2>(P, Qg, s_tot, field_at, emit);
    else if (Np1 <= 3 * per_pass) field_build_regs_r<3>(P, Qg, s_tot, field_at, emit);
    else if (Np1 <= 4 * per_pass) field_build_regs_r<4>(P, Qg, s_tot, field_at, emit);
    else return false;
    return true;
}

// The binary64 field of the FP64 path:
//   E_j = (S_j q_unit/2) (1/r_j),  E_c = (q_c q_unit) (1/h_r),
// the same operations in the same order as the staged build (with the odd
// reading, E_j = -E_j left of the axis and E_c = 0).
template <class Emit>
static __device__ __forceinline__ bool field_build_regs(const DevParams& P, const unsigned long long* Qg,
                                                        const double* inv_r, long long* s_tot, Emit emit) {
    const int c = P.c;
    auto field_at = [&](int j, long long S, long long qj) -> double {
        if (j == c) return P.parity_odd ? 0.0 : (i64_to_double(qj) * P.q_unit) * P.inv_hr;
        const double e = (i64_to_double(S) * P.q_half) * inv_r[j];
        return (P.parity_odd && j < c) ? -e : e;  // odd reading: rE / |r|
    };
    return field_build_regs_with(P, Qg, s_tot, field_at, emit);
}

// Barrier of the n_blocks blocks that share `bar` (the whole grid, or the
// blocks of one beam of a batch), with a time limit, in two halves so that
// a block can issue work that does not depend on the other blocks (loads of
// its own particles) between its arrival and its wait.
// Arrival: after the block's own barrier, one release reduction on the
// counter bar[0] (it orders every write the block made before it, the
// charge flush included, without waiting for a returned value).  Wait: one
// thread polls the counter with acquire loads until all n_blocks arrivals of
// this generation are in; the block barrier then passes the acquire on to
// the other threads.  The counter only grows within a launch (reset between
// launches), so generation g waits for g * n_blocks arrivals.
static __device__ __forceinline__ void grid_arrive(unsigned int* bar, unsigned int& gen) {
    __syncthreads();
    ++gen;
    if (threadIdx.x == 0) asm volatile("red.release.gpu.global.add.u32 [%0], 1;" ::"l"(bar) : "memory");
}

// false if any block timed out or failed
static __device__ __forceinline__ bool grid_wait(const DevParams& P, unsigned int* bar, unsigned int gen, int* status,
                                                 int* s_ok, unsigned int n_blocks) {
    if (threadIdx.x == 0) {
        const unsigned int target = gen * (n_blocks + P.bar_extra);
        int ok = 1;
        long long t0 = 0;
        unsigned spins = 0;
        while ((int)(ld_acquire_u32(bar) - target) < 0) {
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
        *s_ok = ok;
    }
    __syncthreads();
    return *s_ok != 0;
}

static __device__ __forceinline__ bool grid_sync(const DevParams& P, unsigned int* bar, unsigned int& gen,
                                                 int* status, int* s_ok, unsigned int n_blocks) {
    grid_arrive(bar, gen);
    return grid_wait(P, bar, gen, status, s_ok, n_blocks);
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

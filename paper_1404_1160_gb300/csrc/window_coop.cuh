// window_coop.cuh -- the cooperative window kernel of the Poisson field
// (k_window_coop) and its device helpers, included by window_coop.cu, which
// is compiled once per histogram form and fine solver (the instantiations
// compile in parallel), and by window.cu for the launch sizes.
//
// The fine window of Algorithm ETDFSSModAlgo (Frenod, Hirstoaga
// & Lutz, Sec. 3): fine solver from y^n with period detection (Remark
// CompOfThePeriodsRem), quadratic landing at o and o+T (Remark
// QuadraticInterpolationRem) and the N-turn extrapolation (eq. MainFormula1).
//
// Self-consistent Poisson field: one cooperative persistent launch per macro
// step.  Each fine stage needs the field of every particle's stage position
// (Sec. 3: the window advances every particle, not only those still
// looking for their period, because the self-consistent field needs them
// all).  Because E enters only dV/dt, the
// R-component of stage s depends on fields of stages <= s-2, so stages pair
// up: RK4 deposits stages (1,2) then (3,4); Lawson RK4 deposits (1,3) then
// (2,4).  One fine step is therefore two field cycles:
//   sweep: gather previous pair, advance, deposit the next pair into a
//          shared-memory int64 histogram per block;
//   flush the histograms with global int64 atomics; grid barrier;
//   every block scans the mesh charge (block-wide int64 scan) into its own
//   shared-memory field table.
// Histogram sets rotate over three buffers so one barrier per cycle suffices.
#pragma once

#include "pic_internal.h"
#include "window_common.cuh"

namespace pic {

constexpr int kWinMaxThreads = 1024;
constexpr int kHistCopiesMax = 2;

// ---------------------------------------------------------------- helpers

// Shared-memory histogram of one field.  HIST = 0: three 32-bit counters
// per cell (particles C_j, low and high 16 bits of the right weights S_j),
// exact while a block deposits at most 65536 positions per field per cycle;
// the node charge is Q_j = W C_j - S_j + S_{j-1}.  HIST = 2: four counters
// (C_j and the 11/11/10-bit parts of S_j), exact up to 2^21 positions per
// block, field and cycle, for the larger particle counts.  HIST = 1: one
// 64-bit counter per node (W > 2^32, or beyond 2^21 positions).
template <int HIST>
struct Hist {
    static constexpr int kWordsPerNode = HIST == 0 ? 3 : (HIST == 2 ? 4 : 2);  // 32-bit words per node
};
// 32-bit words per node that the shared-memory layout reserves
__host__ __device__ constexpr int hist_slot_words(int hist) { return hist == 2 ? 4 : 3; }

template <int HIST>
__device__ __forceinline__ void deposit_cell(unsigned int* h, int Np1, const Cell& c, long long W) {
    if (c.j < 0) return;
    if (HIST == 0) {
        // every lane adds its own position (plain shared atomics are faster
        // on this GPU than merging the lanes of a warp first)
        const unsigned int lo = (unsigned int)(c.qR & 0xffff), hi = (unsigned int)(c.qR >> 16);
        atomicAdd(&h[c.j], 1u);
        if (lo) atomicAdd(&h[Np1 + c.j], lo);
        if (hi) atomicAdd(&h[2 * Np1 + c.j], hi);
    } else if (HIST == 2) {
        const unsigned int q = (unsigned int)c.qR;
        const unsigned int a = q & 0x7ffu, b = (q >> 11) & 0x7ffu, d = q >> 22;
        atomicAdd(&h[c.j], 1u);
        if (a) atomicAdd(&h[Np1 + c.j], a);
        if (b) atomicAdd(&h[2 * Np1 + c.j], b);
        if (d) atomicAdd(&h[3 * Np1 + c.j], d);
    } else {
        unsigned long long* h64 = (unsigned long long*)h;
        atomicAdd(&h64[c.j], (unsigned long long)(W - c.qR));
        if (c.qR) atomicAdd(&h64[c.j + 1], (unsigned long long)c.qR);
    }
}

// Node charge of one field from the block histogram, summed over its
// `copies` copies `stride` words apart (lane l deposits into copy
// l % copies, so a cell shared by the lanes of a warp is updated on
// several addresses instead of one).
template <int HIST>
__device__ __forceinline__ unsigned long long hist_node(const unsigned int* h, int Np1, int j, long long W, int stride,
                                                        int copies) {
    if (HIST == 0) {
        unsigned long long C = 0, Sj = 0, Sm = 0;
        for (int c = 0; c < copies; ++c) {
            const unsigned int* hc = h + c * stride;
            if (j < Np1 - 1) {
                C += hc[j];
                Sj += ((unsigned long long)hc[2 * Np1 + j] << 16) + (unsigned long long)hc[Np1 + j];
            }
            if (j >= 1) Sm += ((unsigned long long)hc[2 * Np1 + j - 1] << 16) + (unsigned long long)hc[Np1 + j - 1];
        }
        return C * (unsigned long long)W - Sj + Sm;
    } else if (HIST == 2) {
        auto S = [&](const unsigned int* hc, int m) -> unsigned long long {
            return (unsigned long long)hc[Np1 + m] + ((unsigned long long)hc[2 * Np1 + m] << 11) +
                   ((unsigned long long)hc[3 * Np1 + m] << 22);
        };
        unsigned long long C = 0, Sj = 0, Sm = 0;
        for (int c = 0; c < copies; ++c) {
            const unsigned int* hc = h + c * stride;
            if (j < Np1 - 1) {
                C += hc[j];
                Sj += S(hc, j);
            }
            if (j >= 1) Sm += S(hc, j - 1);
        }
        return C * (unsigned long long)W - Sj + Sm;
    } else {
        return ((const unsigned long long*)h)[j];
    }
}

// Field tables of one cycle (two fields) from the cycle's global charge:
// trapezoid integral from r = 0 (S_j = g_j - g_c), E_j = S_j q_unit/2 * (1/r_j),
// E_c = Q_c q_unit / h_r, then (E_j, (E_{j+1}-E_j)/W) per cell.
// stop_src (may be null): the not-done count of the cycle, read together with
// the charge; *s_stop = (count == 0) after the call.
static __device__ void build_fields(const DevParams& P, const unsigned long long* Qg, long long* q, long long* g,
                             double2* tab, const double* inv_r, double* edges, long long* s_warp,
                             const int* stop_src = nullptr, int* s_stop = nullptr) {
    const int Nc = P.n_cells, Np1 = Nc + 1, c = P.c;
    if (stop_src && threadIdx.x == 0) *s_stop = (__ldcg(stop_src) == 0);
    auto emit = [&](int f, int j, double e, double en, long long S) {
        double sl = 0.0;
        if (j < Nc) {
            const double d = en - e;
            // d / W: exponent shift when the result stays normal (exact), else multiply
            const int ex = (int)((__double_as_longlong(d) >> 52) & 0x7ff);
            sl = (ex > P.log2W + 1 && ex < 0x7ff) ? scale_pow2(d, -P.log2W) : d * P.invW;
        }
        tab[f * Np1 + j] = make_double2(e, sl);
        // the off-mesh gather divides the edge rE by R: the odd reading
        // (rE / |R|) carries the sign flip in the lower edge value
        if (j == 0) edges[2 * f] = P.parity_odd ? -(i64_to_double(S) * P.q_half) : i64_to_double(S) * P.q_half;
        if (j == Nc) edges[2 * f + 1] = i64_to_double(S) * P.q_half;
    };
    if (field_build_regs(P, Qg, inv_r, s_warp, emit)) {
        __syncthreads();
        return;
    }
    // staged build (meshes too large for the register form)
    for (int idx = threadIdx.x; idx < 2 * Np1; idx += blockDim.x) q[idx] = (long long)__ldcg(Qg + (size_t)idx * kQPad);
    __syncthreads();
    block_exscan_pairs2(q, g, Nc, s_warp);
    for (int idx = threadIdx.x; idx < 2 * Np1; idx += blockDim.x) {
        const int f = idx >= Np1, j = idx - f * Np1;
        const long long S = g[idx] - g[f * Np1 + c];
        // int64 -> double exactly as (double)S, on the integer pipe
        const double Sd = i64_to_double(S);
        double e;
        if (j == c) e = P.parity_odd ? 0.0 : (i64_to_double(q[f * Np1 + c]) * P.q_unit) * P.inv_hr;
        else e = (Sd * P.q_half) * inv_r[j];
        if (P.parity_odd && j < c) e = -e;
        tab[idx].x = e;
        if (j == 0) edges[2 * f] = P.parity_odd ? -(Sd * P.q_half) : Sd * P.q_half;
        if (j == Nc) edges[2 * f + 1] = Sd * P.q_half;
    }
    __syncthreads();
    for (int idx = threadIdx.x; idx < 2 * Np1; idx += blockDim.x) {
        const int f = idx >= Np1, j = idx - f * Np1;
        double sl = 0.0;
        if (j < Nc) {
            const double d = tab[idx + 1].x - tab[idx].x;
            // d / W: exponent shift when the result stays normal (exact), else multiply
            const int ex = (int)((__double_as_longlong(d) >> 52) & 0x7ff);
            sl = (ex > P.log2W + 1 && ex < 0x7ff) ? scale_pow2(d, -P.log2W) : d * P.invW;
        }
        tab[idx].y = sl;
    }
    __syncthreads();
}

// Period tracking of one particle at sample k (k >= 1), V_{k-1} = Vold,
// V_k = Vnew.  A sign change between samples k-1 and k is marked pending
// and its root taken at sample k+1 from V_{k-1}, V_k, V_{k+1} (V_{k-1} kept
// in vp when the change is found): the same crossings, stencils and order as
// testing samples k-2, k-1 at sample k.  tr = (flags, need) is loaded by the
// caller and updated here.  Returns true when the particle is done.
__device__ __forceinline__ bool track_update(const DevParams& P, const WinBufs& B, long long i, int k,
                                             double Vold, double Vnew, bool detect_only, int2& tr) {
    if (!(tr.x & F_RES)) {
        Track s;
        s.flags = tr.x;
        s.t1 = 0.0;
        s.need = tr.y;
        bool touched = false;
        if (s.flags & F_PEND) {
            const double v0 = B.vp[i];
            if ((s.flags & F_NEXT) >= 1) s.t1 = B.t1[i];
            s.flags &= ~F_PEND;
            track_root(s, P, k, v0, Vold, Vnew, detect_only);
            if ((s.flags & F_NEXT) == 1 && !(tr.x & F_NEXT)) B.t1[i] = s.t1;
            touched = true;
        }
        if (!(s.flags & F_RES) && positive(Vold) != positive(Vnew)) {
            s.flags |= F_PEND;
            B.vp[i] = Vold;
            touched = true;
        }
        if (k == P.Kmax) {
            track_cap(s, P, detect_only);
            touched = true;
        }
        if (touched) {
            if (s.flags & F_RES) {
                B.T[i] = s.T;
                if (!detect_only) {
                    B.o[i] = s.o;
                    B.N[i] = s.N;
                }
            }
            tr = make_int2(s.flags, (s.flags & F_RES) && !detect_only ? s.need : tr.y);
            B.tr[i] = tr;
        }
    }
    if (!(tr.x & F_RES)) return false;
    return detect_only || k >= tr.y;
}

// Trajectory band of an ETD window.  The landing reads rows floor(o) .. +2
// and floor(o + T) .. +2; with the previous step's period as the forecast
// of T, a window stores row 0 (y^n) and the rows within band_m of the two
// forecast stencils only.  The first rows of the two bands sit in bits
// 8..19 and 20..31 of the tracking word (the flags use bits 0..4).
__device__ __forceinline__ int band_bits(const DevParams& P, double Tprev) {
    const double T = (Tprev > 0.0 && isfinite(Tprev)) ? Tprev : P.Tfb;
    const double o = fmod(P.D, T);
    const int N = (int)rint((P.D - o) / T);
    int a = (int)floor(o) - P.band_m, b = N > 0 ? (int)floor(o + T) - P.band_m : a;
    a = min(max(a, 0), 4095);
    b = min(max(b, 0), 4095);
    return (int)(((unsigned int)a << 8) | ((unsigned int)b << 20));
}
__device__ __forceinline__ bool band_holds(int x, int k, int band_m) {
    const unsigned int ux = (unsigned int)x, L = 3u + 2u * (unsigned int)band_m;
    return k == 0 || (unsigned int)(k - (int)((ux >> 8) & 0xFFFu)) < L || (unsigned int)(k - (int)(ux >> 20)) < L;
}

// ------------------------------------------------ cooperative Poisson window

// Flushes this block's two histograms into the cycle's global charge and
// (block 0) clears the charge buffer of the next cycle.
template <int HIST>
__device__ __forceinline__ void flush_hist(const DevParams& P, const WinBufs& B, const unsigned int* hist, int cyc) {
    const int Np1 = P.n_cells + 1;
    const int words = Hist<HIST>::kWordsPerNode * Np1;
    unsigned long long* Qg = B.Qring + (size_t)(cyc % 3) * 2 * Np1 * kQPad;
    for (int idx = threadIdx.x; idx < 2 * Np1; idx += blockDim.x) {
        const int f = idx >= Np1, j = idx - f * Np1;
        const unsigned long long v = hist_node<HIST>(hist + f * words, Np1, j, P.W, 2 * words, P.hist_copies);
        if (v) atomicAdd(Qg + (size_t)idx * kQPad, v);
    }
    if (blockIdx.x == 0) {
        unsigned long long* Qn = B.Qring + (size_t)((cyc + 1) % 3) * 2 * Np1 * kQPad;
        for (int idx = threadIdx.x; idx < 2 * Np1; idx += blockDim.x) Qn[(size_t)idx * kQPad] = 0ull;
    }
}

// One chunk (32 particles) of window state in shared memory; lane l owns
// entry l of every array, so no warp synchronisation is needed.
struct Stage {
    double2 y[32];
    double2 ce[32];
    double2 ca[32];
    double2 cx[32];  // Lawson uses .x ((Phi_h y)_R), RK4 both stage positions
    int2 tr[32];
    short2 cj[32];
};
constexpr size_t kStageBytesPerWarp = 2 * sizeof(Stage);

// The state a sweep reads for one particle.
struct ChunkIn {
    double2 y, ce, ca, cx;
    int2 tr;
    short2 cj;
};

template <int SOLVER>
__device__ __forceinline__ void prefetch_chunk(const WinBufs& B, long long i, bool sweepA, bool fine_only, bool k0,
                                               Stage* s, int lane) {
    cp_async16(&s->y[lane], &B.y[i]);
    if (sweepA && !fine_only) cp_async8(&s->tr[lane], &B.tr[i]);
    if (sweepA && k0) return;
    if (sweepA) cp_async16(&s->ce[lane], &B.ce[i]);
    cp_async16(&s->ca[lane], &B.ca[i]);
    if (SOLVER == 1) cp_async8(&s->cx[lane].x, &B.cxr[i]);
    else cp_async16(&s->cx[lane], &B.cx[i]);
    cp_async4(&s->cj[lane], &B.cj[i]);
}

template <int SOLVER>
__device__ __forceinline__ ChunkIn load_chunk(const WinBufs& B, long long i, bool sweepA, bool fine_only, bool k0) {
    ChunkIn c;
    c.y = B.y[i];
    c.tr = (sweepA && !fine_only) ? B.tr[i] : make_int2(0, 0);
    c.ce = make_double2(0.0, 0.0);
    c.ca = make_double2(0.0, 0.0);
    c.cx = make_double2(0.0, 0.0);
    c.cj = make_short2(-3, -3);
    if (sweepA && k0) return c;
    if (sweepA) c.ce = B.ce[i];
    c.ca = B.ca[i];
    if (SOLVER == 1) c.cx.x = B.cxr[i];
    else c.cx = B.cx[i];
    c.cj = B.cj[i];
    return c;
}

__device__ __forceinline__ ChunkIn read_stage(const Stage* s, int lane) {
    ChunkIn c;
    c.y = s->y[lane];
    c.ce = s->ce[lane];
    c.ca = s->ca[lane];
    c.cx = s->cx[lane];
    c.tr = s->tr[lane];
    c.cj = s->cj[lane];
    return c;
}

template <int SOLVER, int HIST, int POW2, int STAGE>
__global__ void __launch_bounds__(kWinMaxThreads) k_window_coop(DevParams P, WinBufs B, int mode, int T_known,
                                                                long long n_fine, const double* __restrict__ Tin) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int Nc = P.n_cells, Np1 = Nc + 1;
    const int words = Hist<HIST>::kWordsPerNode * Np1;   // 32-bit words per field histogram
    const int copies = P.hist_copies;
    Stage* stage = (Stage*)smem_raw;                      // STAGE: 2 per warp
    double2* tab = (double2*)(smem_raw + (STAGE ? (blockDim.x >> 5) * kStageBytesPerWarp : 0));  // 2 Np1
    unsigned int* hist = (unsigned int*)(tab + 2 * Np1);  // copies x 2 fields x words (also the scan input)
    long long* g = (long long*)(hist + (copies > 2 ? copies : 2) * 2 * hist_slot_words(HIST) * Np1);  // 2 Np1
    double* inv_r = (double*)(g + 2 * Np1);               // Np1
    __shared__ double s_edges[4];
    __shared__ long long s_warp[64];
    __shared__ int s_ok, s_cnt, s_stop, s_next;

    for (int j = threadIdx.x; j < Np1; j += blockDim.x)
        inv_r[j] = (j == P.c) ? 0.0 : 1.0 / (P.r_min + (double)j * P.hr);

    const bool detect_only = mode == MODE_PERIODS, fine_only = mode == MODE_FINE;
    const long long n = P.n;
    // Work unit: a chunk of 32 consecutive storage slots (phase-space
    // neighbours after the sort).  Block b owns the chunks c = b (mod grid),
    // so every block sees all phases (the sign changes of V spread evenly
    // over blocks and fine steps) and a slot always stays on one SM; inside
    // the block, warps take the block's chunks dynamically from a shared
    // counter, so they finish a sweep together.
    const int lane = threadIdx.x & 31;
    const long long n_chunks = (n + 31) / 32;
    // lane l deposits into copy l mod copies (the lanes of a warp hold
    // phase-space neighbours, which mostly share a cell)
    unsigned int* const my_hist = hist + ((threadIdx.x & 31) % copies) * 2 * words;
    Stage* const my_stage = stage + 2 * (threadIdx.x >> 5);
    const long long n_warps = (long long)gridDim.x * (blockDim.x >> 5);
    const long long g_warp = (long long)(threadIdx.x >> 5) * gridDim.x + blockIdx.x;
    const long long stride = n_warps * 32;  // static mapping (init and landing)
    const long long i0 = g_warp * 32 + lane;
    // next chunk of this block for this warp (warp-uniform)
    auto grab = [&]() -> long long {
        int m = 0;
        if (lane == 0) m = atomicAdd(&s_next, 1);
        m = __shfl_sync(0xffffffffu, m, 0);
        return (long long)blockIdx.x + (long long)m * gridDim.x;
    };
    const double ie = P.inv_eps, mie = P.mie;
    const long long W = P.W;
    unsigned int gen = 0;
    int cyc = 0;
    int K = 0;
    __shared__ int s_miss;
    const bool band_ok = mode == MODE_ETD && !T_known && P.band_m > 0;

    // attempt 1 replays the window with every trajectory row when a landing
    // row fell outside the band of attempt 0
    for (int attempt = 0;; ++attempt) {
    const bool band = band_ok && attempt == 0;
    if (!fine_only) {
        for (long long i = i0; i < n; i += stride) {
            if (T_known) {
                Track s;
                s.flags = 0;
                s.t1 = 0.0;
                track_resolve(s, P, Tin[i]);
                B.T[i] = s.T;
                B.o[i] = s.o;
                B.N[i] = s.N;
                B.tr[i] = make_int2(s.flags, s.need);
            } else {
                B.tr[i] = make_int2(band ? band_bits(P, B.T[i]) : 0, 0);
            }
        }
    }

    for (int k = 0;; ++k) {
        // ---- sweep A(k): finish step k-1, sample k, deposit stage pair 1 of step k
        for (int idx = threadIdx.x; idx < copies * 2 * words; idx += blockDim.x) hist[idx] = 0u;
        if (threadIdx.x == 0) {
            s_cnt = 0;
            s_next = 0;
        }
        __syncthreads();
        const bool last_fine = fine_only && k == n_fine;
        const bool k0 = k == 0;
        unsigned int cnt = 0;
        int cur = 0;
        long long c = grab();
        if (STAGE) {
            if (c < n_chunks && c * 32 + lane < n) prefetch_chunk<SOLVER>(B, c * 32 + lane, true, fine_only, k0, my_stage, lane);
            cp_async_commit();
        }
        // warp-uniform trip count: lanes past the end run with an empty cell
        for (; c < n_chunks; cur ^= 1) {
            const long long cn = grab();
            const long long i = c * 32 + lane;
            const bool valid = i < n;
            ChunkIn in;
            if (STAGE) {
                if (cn < n_chunks && cn * 32 + lane < n) prefetch_chunk<SOLVER>(B, cn * 32 + lane, true, fine_only, k0, my_stage + (cur ^ 1), lane);
                cp_async_commit();
                cp_async_wait<1>();
                in = read_stage(my_stage + cur, lane);
            } else if (valid) {
                in = load_chunk<SOLVER>(B, i, true, fine_only, k0);
            }
            c = cn;
            double R = valid ? in.y.x : 0.0, V = valid ? in.y.y : 0.0;
            if (!valid) {
            } else if (k > 0) {
                const double ea = mesh_gather(tab, s_edges[0], s_edges[1], in.cj.x, in.ca.x);
                const double eb = mesh_gather(tab + Np1, s_edges[2], s_edges[3], in.cj.y, in.ca.y);
                double Rn, Vn;
                if (SOLVER == 1) {
                    // ce = (e1, e3), ea = e2, eb = e4, cx.x = (Phi_h y)_R
                    const double e1 = in.ce.x, e3 = in.ce.y;
                    const double Bv = fma(P.c1, V, -dmul_i(P.imul, P.s1, R));
                    const double e23 = ea + e3;
                    Rn = fma(P.h6, fma(P.tsh, e23, dmul_i(P.imul, P.s1, e1)), in.cx.x);
                    Vn = fma(P.h6, fma(P.tch, e23, fma(P.c1, e1, eb)), Bv);
                } else {
                    // ce = partial sums, cx = (R3, R4), ea = e3, eb = e4
                    const double k3V = fma(mie, in.cx.x, ea);
                    const double V4 = fma(P.h, k3V, V);
                    const double k4R = ie * V4, k4V = fma(mie, in.cx.y, eb);
                    const double sR = in.ce.x + k4R;
                    const double sV = (in.ce.y + 2.0 * k3V) + k4V;
                    Rn = fma(P.h6, sR, R);
                    Vn = fma(P.h6, sV, V);
                }
                if (!fine_only) {
                    int2 tr = in.tr;
                    // the sample is stored before tracking: a pending root at
                    // sample k+1 reads it back
                    if (!((tr.x & F_RES) && (detect_only || k > tr.y)) && (!band || band_holds(tr.x, k, P.band_m)))
                        __stcs(&B.traj[(size_t)k * n + i], make_double2(Rn, Vn));
                    const bool done = track_update(P, B, i, k, V, Vn, detect_only, tr);
                    cnt += done ? 0u : 1u;
                }
                R = Rn;
                V = Vn;
                B.y[i] = make_double2(R, V);
            } else if (!fine_only) {
                __stcs(&B.traj[i], make_double2(R, V));
                cnt += 1u;
            }
            if (last_fine) continue;
            // stage pair 1
            Cell ca, cb;
            double2 cx;
            if (SOLVER == 1) {
                ca = mesh_locate<POW2>(P, R);                            // stage 1: y
                cb = mesh_locate<POW2>(P, fma(P.sh, V, dmul_i(P.imul, P.ch, R)));  // stage 3: Phi_h/2 y
                cx = make_double2(fma(P.s1, V, dmul_i(P.imul, P.c1, R)), 0.0);  // (Phi_h y)_R
            } else {
                ca = mesh_locate<POW2>(P, R);                            // stage 1: y
                const double R2 = fma(P.h2, ie * V, R);                  // stage 2: y + h/2 k1
                cb = mesh_locate<POW2>(P, R2);
                cx = make_double2(R2, 0.0);
            }
            if (!valid) ca.j = cb.j = -3;
            deposit_cell<HIST>(my_hist, Np1, ca, W);
            deposit_cell<HIST>(my_hist + words, Np1, cb, W);
            if (valid) {
                B.ca[i] = make_double2(ca.a, cb.a);
                B.cj[i] = make_short2((short)ca.j, (short)cb.j);
                if (SOLVER == 1) B.cxr[i] = cx.x;
                else B.cx[i] = cx;
            }
        }
        if (STAGE) cp_async_wait<0>();
        if (last_fine) break;
        if (!fine_only) {
            cnt = __reduce_add_sync(0xffffffffu, cnt);
            if ((threadIdx.x & 31) == 0 && cnt) atomicAdd(&s_cnt, (int)cnt);
        }
        __syncthreads();
        flush_hist<HIST>(P, B, hist, cyc);
        if (blockIdx.x == 0 && threadIdx.x == 0) B.notdone[(k + 1) % 3] = 0;
        if (threadIdx.x == 0 && s_cnt) atomicAdd(&B.notdone[k % 3], s_cnt);
        if (!grid_sync(P, B.bar, gen, B.status, &s_ok, gridDim.x)) return;
        build_fields(P, B.Qring + (size_t)(cyc % 3) * 2 * Np1 * kQPad, (long long*)hist, g, tab, inv_r, s_edges, s_warp,
                     fine_only ? nullptr : &B.notdone[k % 3], &s_stop);
        if (!fine_only && s_stop) {
            K = k;
            break;
        }
        ++cyc;

        // ---- sweep B(k): gather pair 1, deposit stage pair 2
        for (int idx = threadIdx.x; idx < copies * 2 * words; idx += blockDim.x) hist[idx] = 0u;
        if (threadIdx.x == 0) s_next = 0;
        __syncthreads();
        cur = 0;
        c = grab();
        if (STAGE) {
            if (c < n_chunks && c * 32 + lane < n) prefetch_chunk<SOLVER>(B, c * 32 + lane, false, fine_only, false, my_stage, lane);
            cp_async_commit();
        }
        for (; c < n_chunks; cur ^= 1) {
            const long long cn = grab();
            const long long i = c * 32 + lane;
            const bool valid = i < n;
            ChunkIn in;
            if (STAGE) {
                if (cn < n_chunks && cn * 32 + lane < n) prefetch_chunk<SOLVER>(B, cn * 32 + lane, false, fine_only, false, my_stage + (cur ^ 1), lane);
                cp_async_commit();
                cp_async_wait<1>();
                in = read_stage(my_stage + cur, lane);
            } else if (valid) {
                in = load_chunk<SOLVER>(B, i, false, fine_only, false);
            }
            c = cn;
            if (!valid) {
                in.y = make_double2(0.0, 0.0);
                in.ca = make_double2(0.0, 0.0);
                in.cx = make_double2(0.0, 0.0);
                in.cj = make_short2(-3, -3);
            }
            const double R = in.y.x, V = in.y.y;
            const double ea = mesh_gather(tab, s_edges[0], s_edges[1], in.cj.x, in.ca.x);
            const double eb = mesh_gather(tab + Np1, s_edges[2], s_edges[3], in.cj.y, in.ca.y);
            double Pa, Pb;
            if (SOLVER == 1) {
                // ea = e1 at y, eb = e3 at Phi_h/2 y
                Pa = fma(P.sh, fma(P.h2, ea, V), P.ch * R);              // stage 2
                Pb = fma(P.hsh, eb, in.cx.x);                            // stage 4
                if (valid) B.ce[i] = make_double2(ea, eb);
            } else {
                // ea = e1 at y, eb = e2 at y + h/2 k1, cx.x = R2
                const double k1R = ie * V, k1V = fma(mie, R, ea);
                const double V2 = fma(P.h2, k1V, V);
                const double k2R = ie * V2, k2V = fma(mie, in.cx.x, eb);
                const double R3 = fma(P.h2, k2R, R), V3 = fma(P.h2, k2V, V);
                const double k3R = ie * V3;
                const double R4 = fma(P.h, k3R, R);
                Pa = R3;                                                 // stage 3
                Pb = R4;                                                 // stage 4
                if (valid) {
                    B.ce[i] = make_double2((k1R + 2.0 * k2R) + 2.0 * k3R, k1V + 2.0 * k2V);
                    B.cx[i] = make_double2(R3, R4);
                }
            }
            Cell ca2 = mesh_locate<POW2>(P, Pa), cb2 = mesh_locate<POW2>(P, Pb);
            if (!valid) ca2.j = cb2.j = -3;
            deposit_cell<HIST>(my_hist, Np1, ca2, W);
            deposit_cell<HIST>(my_hist + words, Np1, cb2, W);
            if (valid) {
                B.ca[i] = make_double2(ca2.a, cb2.a);
                B.cj[i] = make_short2((short)ca2.j, (short)cb2.j);
            }
        }
        if (STAGE) cp_async_wait<0>();
        __syncthreads();
        flush_hist<HIST>(P, B, hist, cyc);
        if (!grid_sync(P, B.bar, gen, B.status, &s_ok, gridDim.x)) return;
        build_fields(P, B.Qring + (size_t)(cyc % 3) * 2 * Np1 * kQPad, (long long*)hist, g, tab, inv_r, s_edges, s_warp);
        ++cyc;
    }

    if (blockIdx.x == 0 && threadIdx.x == 0 && !fine_only) *B.K_out = K;
    if (detect_only) {
        // step 1 alone leaves y^n as it was: it is row 0 of the trajectory
        for (long long i = i0; i < n; i += stride) B.y[i] = B.traj[i];
        return;
    }
    if (mode != MODE_ETD) return;

    // ---- landing (step 3) and extrapolation (step 4); with the band, a
    // particle whose landing rows were not all stored marks a miss
    bool miss = false;
    for (long long i = i0; i < n; i += stride) {
        const double o = B.o[i], T = B.T[i];
        const int N = B.N[i];
        const int nt = N > 0 ? 2 : 1;
        if (band) {
            const int x = B.tr[i].x;
            bool held = true;
            for (int t = 0; t < nt; ++t) {
                const int kk = (int)floor(t == 0 ? o : o + T);
                held = held && band_holds(x, kk, P.band_m) && band_holds(x, kk + 1, P.band_m) &&
                       band_holds(x, kk + 2, P.band_m);
            }
            if (!held) {
                miss = true;
                continue;
            }
        }
        double y[2][2];
        for (int t = 0; t < nt; ++t) {
            const double u = t == 0 ? o : o + T;
            const int kk = (int)floor(u);
            const double sf = u - (double)kk;
            const double2 a = B.traj[(size_t)kk * n + i];
            const double2 b = B.traj[(size_t)(kk + 1) * n + i];
            const double2 cc = B.traj[(size_t)(kk + 2) * n + i];
            y[t][0] = interp3(a.x, b.x, cc.x, sf);
            y[t][1] = interp3(a.y, b.y, cc.y, sf);
        }
        B.y[i] = make_double2(extrapolate(y[0][0], y[nt - 1][0], N), extrapolate(y[0][1], y[nt - 1][1], N));
    }
    if (!band) return;
    if (__syncthreads_or(miss) && threadIdx.x == 0) atomicOr(&B.notdone[3], 1);
    if (!grid_sync(P, B.bar, gen, B.status, &s_ok, gridDim.x)) return;
    if (threadIdx.x == 0) s_miss = ld_acquire_s32(&B.notdone[3]);
    __syncthreads();
    if (!s_miss) return;
    // replay from y^n (row 0) with every row, for every particle; the charge
    // buffer of the next cycle is the clear one
    for (long long i = i0; i < n; i += stride) B.y[i] = B.traj[i];
    if (blockIdx.x == 0 && threadIdx.x == 0) {
        B.notdone[0] = B.notdone[1] = B.notdone[2] = 0;
        atomicAdd(&B.notdone[4], 1);
    }
    ++cyc;
    K = 0;
    if (!grid_sync(P, B.bar, gen, B.status, &s_ok, gridDim.x)) return;
    }
}

}  // namespace pic

// window32.cu -- the FP32 form of the fine window of Algorithm ETDFSSModAlgo
// (Frenod, Hirstoaga & Lutz, Sec. 3): the same steps as window.cu (fine
// solver from y^n with period detection, quadratic landing at o and o+T,
// N-turn extrapolation), with the particle state and the push in binary32.
//
// Layout.  The state of fine step k of a window is the rotating-frame
// vector z_k = Phi(-t_k) y_k (see pic_device.cuh), stored as row k of a
// trajectory: row 0 is y^n itself (the public state, Phi(0) = I), rows
// 1..Kmax live in one array with a row stride of n rounded up to 128.  A
// step reads row k-1 and writes row k, so the trajectory the landing
// interpolates is the state the sweeps stream, and nothing else per
// particle crosses a field cycle: the stage positions are recomputed from
// z when they are needed again.  Per particle and fine step the window
// moves 8 B (read row k-1) + 4 B (tracking word) + 8 B (write row k) in the
// first sweep and 8 B (read row k) in the second.
//
// Field cycle (Poisson): as in the FP64 kernel, stages pair up (1,3) and
// (2,4); each pair is deposited by one sweep into per-block 32-bit
// histograms, flushed with 64-bit global atomics, and after a grid barrier
// every block turns the global int64 charge into its own field table of
// binary32 (E_j, E_{j+1} - E_j), computed in binary32 from the exact int64
// sums and per-node constants (build_fields32).  Two tables are kept: the
// one of pair 1 (fields of R1, R3) and the one of pair 2 (R2, R4), so the
// first sweep of the next step can recompute e1 and e3 instead of reading
// them back from memory.
#include "pic_internal.h"
#include "window_common.cuh"

namespace pic {

constexpr int kW32Threads = 1024;
constexpr int kG = 4;             // consecutive particles per lane in a group
constexpr int kGroup = 32 * kG;   // particles per warp group
constexpr int kHist32Words = 4;   // 32-bit words per node and field
constexpr int kHist32CopiesMax = 4;  // histogram copies (lane l deposits into copy l mod copies)

// ---------------------------------------------------------------- deposit

// Block histogram of one field: per cell j the count C_j and the right
// weights qR split in 11/11/10-bit parts summed separately (A_j, B_j, C'_j),
// so every word stays exact while a block deposits at most 2^21 positions
// per field and cycle; S_j = A_j + 2^11 B_j + 2^22 C'_j and the node charge
// is Q_j = W C_j - S_j + S_{j-1}.  Every lane adds its own position with
// plain shared atomics: on this GPU that is several times faster than
// merging the lanes of a warp that share a cell first (match + reduce), and
// than 64-bit shared atomics.
__device__ __forceinline__ void deposit32(unsigned int* h, int Np1, int j, unsigned int qR) {
    const bool ok = j >= 0;
    unsigned int* hj = h + (ok ? j : 0);
    const unsigned int a = qR & 0x7ffu, b = (qR >> 11) & 0x7ffu, c = qR >> 22;
    if (ok) atomicAdd(hj, 1u);
    if (ok && a) atomicAdd(hj + Np1, a);
    if (ok && b) atomicAdd(hj + 2 * Np1, b);
    if (ok && c) atomicAdd(hj + 3 * Np1, c);
}

// deposit32 of a cell known to be on the mesh (j >= 0)
__device__ __forceinline__ void deposit32_on(unsigned int* h, int Np1, int j, unsigned int qR) {
    unsigned int* hj = h + j;
    const unsigned int a = qR & 0x7ffu, b = (qR >> 11) & 0x7ffu, c = qR >> 22;
    atomicAdd(hj, 1u);
    if (a) atomicAdd(hj + Np1, a);
    if (b) atomicAdd(hj + 2 * Np1, b);
    if (c) atomicAdd(hj + 3 * Np1, c);
}

// ------------------------------------------ located pairs, warp-uniform path
//
// Nearly every warp has all its positions on the mesh.  The pair helpers
// below test that once per pair of positions (one warp vote) and then run
// the cell arithmetic without the off-mesh selects, the gather without the
// edge division and the deposit without the on-mesh test; a warp with a lane
// off the mesh (or at a NaN) runs the general locate32t / gather32 /
// deposit32.  Both give the same cells, weights, fields and words.  Every
// lane of the warp must make the call.

// Cell of an on-mesh x = (R - r_min)/h_r, 0 <= x < n_cells: the general
// locate32t with its test known true.
template <bool NEED_Q>
__device__ __forceinline__ Cell32 cell_on_mesh(const DevParams& P, float x) {
    const float fl = floorf(x);
    const float f = x - fl;
    Cell32 c;
    c.j = (int)fl;
    c.a = f;
    c.qR = NEED_Q ? __float2uint_rz(f * P.Wf) : 0u;
    return c;
}

// true when every lane of the warp has both positions on the mesh
__device__ __forceinline__ bool warp_on_mesh(const DevParams& P, float xa, float xb) {
    const bool in = xa >= 0.0f && xa < P.ncells_f && xb >= 0.0f && xb < P.ncells_f;
    return __all_sync(0xffffffffu, in);
}

// Fields at Ra (table ta, edges ed[0..1]) and Rb (table tb, edges ed[2..3]).
__device__ __forceinline__ void locate_gather2(const DevParams& P, float Ra, float Rb, const float2* ta,
                                               const float2* tb, const float* ed, float& ea, float& eb) {
    const float xa = (Ra - P.r_min_f) * P.inv_hr_f, xb = (Rb - P.r_min_f) * P.inv_hr_f;
    if (warp_on_mesh(P, xa, xb)) {
        const Cell32 ca = cell_on_mesh<false>(P, xa), cb = cell_on_mesh<false>(P, xb);
        const float2 va = ta[ca.j], vb = tb[cb.j];
        ea = fmaf(ca.a, va.y, va.x);
        eb = fmaf(cb.a, vb.y, vb.x);
    } else {
        const Cell32 ca = locate32t<false>(P, Ra), cb = locate32t<false>(P, Rb);
        ea = gather32(ta, ed[0], ed[1], ca);
        eb = gather32(tb, ed[2], ed[3], cb);
    }
}

// Deposits Ra into ha and Rb into hb when `valid`.
__device__ __forceinline__ void locate_deposit2(const DevParams& P, float Ra, float Rb, unsigned int* ha,
                                                unsigned int* hb, int Np1, bool valid) {
    const float xa = (Ra - P.r_min_f) * P.inv_hr_f, xb = (Rb - P.r_min_f) * P.inv_hr_f;
    if (warp_on_mesh(P, xa, xb)) {
        const Cell32 ca = cell_on_mesh<true>(P, xa), cb = cell_on_mesh<true>(P, xb);
        if (valid) {
            deposit32_on(ha, Np1, ca.j, ca.qR);
            deposit32_on(hb, Np1, cb.j, cb.qR);
        }
    } else {
        const Cell32 ca = locate32(P, Ra), cb = locate32(P, Rb);
        if (valid) {
            deposit32(ha, Np1, ca.j, ca.qR);
            deposit32(hb, Np1, cb.j, cb.qR);
        }
    }
}

__device__ __forceinline__ unsigned long long hist32_S(const unsigned int* h, int Np1, int j) {
    return (unsigned long long)h[Np1 + j] + ((unsigned long long)h[2 * Np1 + j] << 11) +
           ((unsigned long long)h[3 * Np1 + j] << 22);
}

// Node charge from the `copies` copies of a field's histogram, `stride`
// words apart.
__device__ __forceinline__ unsigned long long hist32_node(const unsigned int* h, int Np1, int j, long long W,
                                                          int copies, int stride) {
    unsigned long long C = 0, Sj = 0, Sm = 0;
    for (int cp = 0; cp < copies; ++cp) {
        const unsigned int* hc = h + cp * stride;
        if (j < Np1 - 1) {
            C += hc[j];
            Sj += hist32_S(hc, Np1, j);
        }
        if (j >= 1) Sm += hist32_S(hc, Np1, j - 1);
    }
    return C * (unsigned long long)W - Sj + Sm;
}

// Adds this block's two histograms to the cycle's global charge; block 0
// clears the charge of the cycle after.
__device__ __forceinline__ void flush32(const DevParams& P, const WinBufs32& B, const unsigned int* hist, int cyc,
                                        int lb) {
    const int Np1 = P.n_cells + 1;
    unsigned long long* Qg = B.Qring + (size_t)(cyc % 3) * 2 * Np1 * kQPad;
    for (int idx = threadIdx.x; idx < 2 * Np1; idx += blockDim.x) {
        const int f = idx >= Np1, j = idx - f * Np1;
        const unsigned long long v =
            hist32_node(hist + f * kHist32Words * Np1, Np1, j, P.W, P.hist_copies, 2 * kHist32Words * Np1);
        if (v) atomicAdd(Qg + (size_t)idx * kQPad, v);
    }
    if (lb == 0) {
        unsigned long long* Qn = B.Qring + (size_t)((cyc + 1) % 3) * 2 * Np1 * kQPad;
        for (int idx = threadIdx.x; idx < 2 * Np1; idx += blockDim.x) Qn[(size_t)idx * kQPad] = 0ull;
    }
}

// Field tables of one cycle from its global charge: exact int64 trapezoid
// sums S_j = g_j - g_c, then in binary32 E_j = float(S_j) cq_j with the
// per-node constant cq_j = q_unit / (2 r_j) (negated left of the axis for
// the odd reading) and E_c = float(Q_c) cq_c, cq_c = q_unit / h_r (0 for the
// odd reading); the table holds (E_j, E_{j+1} - E_j).  Each E_j is within
// 1.5 units in the last place of the exact node field, which the binary32
// bound of the form covers with a wide margin (a field error dE moves a
// particle by about h dE per stage).  All on the FP32 pipes: on this GPU the
// FP64 conversion of every node in every block was most of the build.  q is
// the int64 scan input (2 Np1), g the scan output, reused for E.
// stop_src (may be null): the not-done count of the cycle, read together with
// the charge; *s_stop = (count == 0) after the call.
__device__ void build_fields32(const DevParams& P, const unsigned long long* Qg, long long* q, long long* g,
                               float2* tab, const float* cq, float* edges, long long* s_warp, long long* s_c,
                               const int* stop_src = nullptr, int* s_stop = nullptr) {
    const int Nc = P.n_cells, Np1 = Nc + 1, c = P.c;
    const float qh = (float)P.q_half;
    if (stop_src && threadIdx.x == 0) *s_stop = (__ldcg(stop_src) == 0);
    auto field_at = [&](int j, long long S, long long qj) -> float { return __ll2float_rn(j == c ? qj : S) * cq[j]; };
    auto emit = [&](int f, int j, float e, float en, long long S) {
        tab[f * Np1 + j] = make_float2(e, j < Nc ? en - e : 0.0f);
        // odd reading: the lower edge value carries the sign flip (rE / |R|)
        if (j == 0) edges[2 * f] = P.parity_odd ? -(__ll2float_rn(S) * qh) : __ll2float_rn(S) * qh;
        if (j == Nc) edges[2 * f + 1] = __ll2float_rn(S) * qh;
    };
    if (field_build_regs_with(P, Qg, s_warp, field_at, emit)) {
        __syncthreads();
        return;
    }
    // staged build (meshes too large for the register form)
    for (int idx = threadIdx.x; idx < 2 * Np1; idx += blockDim.x) q[idx] = (long long)__ldcg(Qg + (size_t)idx * kQPad);
    __syncthreads();
    block_exscan_pairs2(q, g, Nc, s_warp);
    if (threadIdx.x < 2) {
        s_c[threadIdx.x] = g[threadIdx.x * Np1 + c];
        s_c[2 + threadIdx.x] = q[threadIdx.x * Np1 + c];
    }
    __syncthreads();
    float* e = (float*)g;  // E_idx in the slot of g[idx] (float 2 idx), which only this thread reads
    for (int idx = threadIdx.x; idx < 2 * Np1; idx += blockDim.x) {
        const int f = idx >= Np1, j = idx - f * Np1;
        const long long S = g[idx] - s_c[f];
        if (j == 0) edges[2 * f] = P.parity_odd ? -(__ll2float_rn(S) * qh) : __ll2float_rn(S) * qh;
        if (j == Nc) edges[2 * f + 1] = __ll2float_rn(S) * qh;
        e[2 * idx] = field_at(j, S, s_c[2 + f]);
    }
    __syncthreads();
    for (int idx = threadIdx.x; idx < 2 * Np1; idx += blockDim.x) {
        const int j = idx >= Np1 ? idx - Np1 : idx;
        tab[idx] = make_float2(e[2 * idx], j < Nc ? e[2 * idx + 2] - e[2 * idx] : 0.0f);
    }
    __syncthreads();
}

// ------------------------------------------------------------ tracking

// Period tracking of one particle at sample k >= 1 (the FP32 twin of
// track_update in window.cu): a sign change of V between samples k-1 and
// k is marked pending and its root taken at sample k+1 from V_{k-1}, V_k,
// V_{k+1}, V_{k-1} being recomputed from row k-1 of the trajectory.  trw =
// flags | need << 8.  Extremum times are kept as (integer, fraction).
// This is the rare part (a root, a resolution or the window cap), kept out
// of line so that a sweep never executes it for the other lanes.
static __device__ __noinline__ unsigned int track32_slow(const DevParams& P, const WinBufs32& B, long long i, int k,
                                                        float Vold, float Vnew, bool detect_only, unsigned int trw,
                                                        const float2* row_km2, float2 rot_km2) {
    int flags = (int)(trw & 31u);
    int need = (int)(trw >> 8);
    if (flags & F_PEND) {
        const float2 zp = row_km2[i];
        const float v0 = rot_V(rot_km2, zp.x, zp.y);
        flags &= ~F_PEND;
        const float s = quad_root01f(v0, Vold, Vnew);
        const int ne = (flags & F_NEXT) + 1;
        flags = (flags & ~F_NEXT) | (ne & F_NEXT);
        if (ne == 1) {
            CTime t1;
            t1.i = k - 2;
            t1.f = s;
            B.t1[i] = t1;
        }
        if (ne == 3) {
            const CTime t1 = B.t1[i];
            const CTime T = ct_norm((long long)(k - 2) - t1.i, s - t1.f);
            if (detect_only) {
                flags |= F_RES;
                B.T[i] = T;
            } else {
                const Decomp32 d = resolve32(P, T, true, flags);
                B.T[i] = d.T;
                B.o[i] = d.o;
                B.N[i] = d.N;
                need = d.need;
            }
        }
    }
    if (!(flags & F_RES) && positive32(Vold) != positive32(Vnew)) flags |= F_PEND;
    if (k == P.Kmax && !(flags & F_RES)) {
        // window cap without a third extremum: T = 2 pi eps
        flags |= F_FB;
        CTime Tfb;
        Tfb.i = P.spt;
        Tfb.f = 0.0f;
        if (detect_only) {
            flags |= F_RES;
            B.T[i] = Tfb;
        } else {
            const Decomp32 d = resolve32(P, Tfb, true, flags);
            B.T[i] = d.T;
            B.o[i] = d.o;
            B.N[i] = d.N;
            need = d.need;
        }
    }
    trw = (unsigned int)flags | ((unsigned int)need << 8);
    B.tr[i] = trw;
    return trw;
}

// Returns true when the particle is done at sample k (resolved and every
// sample it needs is produced).
__device__ __forceinline__ bool track32_update(const DevParams& P, const WinBufs32& B, long long i, int k, float Vold,
                                               float Vnew, bool detect_only, unsigned int& trw,
                                               const float2* row_km2, float2 rot_km2) {
    if (!(trw & (unsigned int)F_RES)) {
        const bool event = (trw & (unsigned int)F_PEND) || positive32(Vold) != positive32(Vnew) || k == P.Kmax;
        if (event) trw = track32_slow(P, B, i, k, Vold, Vnew, detect_only, trw, row_km2, rot_km2);
        if (!(trw & (unsigned int)F_RES)) return false;
    }
    return detect_only || k >= (int)(trw >> 8);
}

// ------------------------------------------------ cooperative Poisson window

struct Grp32 {
    float4 z0, z1;  // (R, V) of the lane's 4 consecutive particles
    float4 e0, e1;  // (e1, e3) of the same particles, carried from the second sweep
    uint4 tr;
};

__device__ __forceinline__ void load_grp(const float2* src, const unsigned int* tr, const float2* ce, long long base,
                                         bool with_tr, bool with_ce, Grp32& G) {
    const float4* p = (const float4*)(src + base);
    G.z0 = p[0];
    G.z1 = p[1];
    if (with_tr) G.tr = *(const uint4*)(tr + base);
    if (with_ce) {
        const float4* c = (const float4*)(ce + base);
        G.e0 = c[0];
        G.e1 = c[1];
    }
}

__device__ __forceinline__ float grp_e(const Grp32& G, int c) {
    switch (c) {
        case 0: return G.e0.x;
        case 1: return G.e0.y;
        case 2: return G.e0.z;
        case 3: return G.e0.w;
        case 4: return G.e1.x;
        case 5: return G.e1.y;
        case 6: return G.e1.z;
        default: return G.e1.w;
    }
}

__device__ __forceinline__ float grp_get(const Grp32& G, int c) {
    switch (c) {
        case 0: return G.z0.x;
        case 1: return G.z0.y;
        case 2: return G.z0.z;
        case 3: return G.z0.w;
        case 4: return G.z1.x;
        case 5: return G.z1.y;
        case 6: return G.z1.z;
        default: return G.z1.w;
    }
}

__device__ __forceinline__ unsigned int grp_tr(const Grp32& G, int q) {
    return q == 0 ? G.tr.x : (q == 1 ? G.tr.y : (q == 2 ? G.tr.z : G.tr.w));
}

// Shared memory of the FP32 window kernel (bytes).
static size_t coop32_smem_bytes(int n_cells, int copies) {
    const size_t Np1 = (size_t)n_cells + 1;
    return (size_t)copies * 2 * kHist32Words * Np1 * sizeof(unsigned int)  // histograms; also the int64 scan input
           + 2 * Np1 * sizeof(long long)                  // scan output, then E in FP64
           + Np1 * sizeof(double)                         // 1/r_j
           + 4 * Np1 * sizeof(float2);                    // tables of pair 1 and pair 2
}

// The window of one beam on blocks lb = 0..nb-1 of its own (the whole grid
// for a single beam, or a beam's share of a batch).
__device__ __forceinline__ void window32_coop_body(const DevParams& P, const WinBufs32& B, int mode, int T_known,
                                                   long long n_fine, const CTime* __restrict__ Tin, int lb, int nb,
                                                   unsigned char* smem_raw) {
    const int Nc = P.n_cells, Np1 = Nc + 1;
    const int hw = kHist32Words * Np1;
    const int copies = P.hist_copies;
    unsigned int* hist = (unsigned int*)smem_raw;  // copies x 2 fields x hw words
    long long* g = (long long*)(hist + copies * 2 * hw);  // 2 Np1
    float* cq = (float*)(g + 2 * Np1);              // Np1 (in a slot of Np1 doubles)
    float2* tabA = (float2*)((double*)(g + 2 * Np1) + Np1);  // 2 Np1: fields of R1, R3
    float2* tabB = tabA + 2 * Np1;                  // 2 Np1: fields of R2, R4
    __shared__ float s_edA[4], s_edB[4];
    __shared__ long long s_warp[64], s_c[4];
    __shared__ int s_ok, s_cnt, s_stop, s_next;

    for (int j = threadIdx.x; j < Np1; j += blockDim.x)
        cq[j] = (j == P.c) ? (P.parity_odd ? 0.0f : (float)(P.q_unit * P.inv_hr))
                           : (float)(((P.parity_odd && j < P.c) ? -P.q_half : P.q_half) / (P.r_min + (double)j * P.hr));

    const bool detect_only = mode == MODE_PERIODS, fine_only = mode == MODE_FINE;
    const long long n = P.n, ld = B.ld;
    const int lane = threadIdx.x & 31;
    // Work unit: a group of 128 consecutive storage slots, lane l holding
    // slots 4l..4l+3.  Block b owns the groups g = b (mod grid); its warps
    // take them dynamically, in alternating directions from one sweep to
    // the next so that the first groups a sweep reads are the last ones the
    // previous sweep touched (still in L2).
    const long long n_groups = ld / kGroup;
    const long long my_groups = (long long)lb < n_groups ? (n_groups - 1 - (long long)lb) / nb + 1 : 0;
    bool rev = false;
    auto grab = [&]() -> long long {
        int m = 0;
        if (lane == 0) m = atomicAdd(&s_next, 1);
        m = __shfl_sync(0xffffffffu, m, 0);
        if (m >= my_groups) return -1;
        const long long mm = rev ? my_groups - 1 - m : m;
        return (long long)lb + mm * nb;
    };
    auto row = [&](long long k) -> float2* {
        if (fine_only) return (k & 1) ? B.traj : B.y;
        return k == 0 ? B.y : B.traj + (size_t)(k - 1) * ld;
    };
    const long long tid = (long long)lb * blockDim.x + threadIdx.x;
    const long long nthreads = (long long)nb * blockDim.x;

    if (!fine_only) {
        for (long long i = tid; i < n; i += nthreads) {
            if (T_known) {
                int flags = 0;
                const Decomp32 d = resolve32(P, Tin[i], true, flags);
                B.T[i] = d.T;
                B.o[i] = d.o;
                B.N[i] = d.N;
                B.tr[i] = (unsigned int)flags | ((unsigned int)d.need << 8);
            } else {
                B.tr[i] = 0u;
            }
        }
    }

    unsigned int gen = 0;
    int cyc = 0;
    int K = 0;
    // lane l deposits into copy l mod copies: the lanes of a warp hold
    // phase-space neighbours, which mostly fall into the same cell
    unsigned int* histA = hist + (lane & (copies - 1)) * 2 * hw;
    unsigned int* histB = histA + hw;

    for (int k = 0;; ++k) {
        // ---- sweep A(k): finish step k-1 (write row k), sample k, deposit stage pair 1 of step k
        for (int idx = threadIdx.x; idx < copies * 2 * hw; idx += blockDim.x) hist[idx] = 0u;
        if (threadIdx.x == 0) {
            s_cnt = 0;
            s_next = 0;
        }
        __syncthreads();
        const bool last_fine = fine_only && k == n_fine;
        const float2 rb = P.rot[rot_index(P, 2ll * k)];      // Phi(t_k)
        const float2 rp = P.rot[rot_index(P, 2ll * k + 1)];  // Phi(t_k + h/2)
        float2 ra = rb, rm = rp, rk2 = rb;
        if (k > 0) {
            ra = P.rot[rot_index(P, 2ll * k - 2)];  // Phi(t_{k-1})
            rm = P.rot[rot_index(P, 2ll * k - 1)];  // Phi(t_{k-1} + h/2)
        }
        if (k > 1) rk2 = P.rot[rot_index(P, 2ll * k - 4)];
        const float2* src = row(k > 0 ? k - 1 : 0);
        float2* dst = last_fine ? B.y : row(k);
        const float2* src2 = k > 1 ? row(k - 2) : nullptr;
        const bool track = !fine_only;
        unsigned int cnt = 0;
        Grp32 cur;
        for (long long gi = grab(); gi >= 0; gi = grab()) {
            const long long base = gi * kGroup + lane * kG;
            load_grp(src, B.tr, B.ce, base, track, k > 0, cur);
            float zo[2 * kG];
#pragma unroll
            for (int q = 0; q < kG; ++q) {
                const long long i = base + q;
                const bool valid = i < n;
                float zR = grp_get(cur, 2 * q), zV = grp_get(cur, 2 * q + 1);
                if (k > 0) {
                    const float R3 = rot_R(rm, zR, zV);
                    const float e1 = grp_e(cur, 2 * q), e3 = grp_e(cur, 2 * q + 1);
                    float e2, e4;
                    locate_gather2(P, lawson32_R2(P, R3, e1), lawson32_R4(P, rb, zR, zV, e3), tabB, tabB + Np1,
                                   s_edB, e2, e4);
                    const float Vold = rot_V(ra, zR, zV);
                    lawson32_update(P, ra, rm, rb, e1, e2, e3, e4, zR, zV);
                    if (track && valid) {
                        unsigned int trw = grp_tr(cur, q);
                        const bool done =
                            track32_update(P, B, i, k, Vold, rot_V(rb, zR, zV), detect_only, trw, src2, rk2);
                        cnt += done ? 0u : 1u;
                    }
                } else if (track && valid) {
                    cnt += 1u;
                }
                if (last_fine) {
                    // the state leaves the rotating frame: y = Phi(t_k) z
                    zo[2 * q] = rot_R(rb, zR, zV);
                    zo[2 * q + 1] = rot_V(rb, zR, zV);
                    continue;
                }
                zo[2 * q] = zR;
                zo[2 * q + 1] = zV;
                // stage pair 1 of step k: R1 = (Phi(t_k) z)_R, R3 = (Phi(t_k + h/2) z)_R
                locate_deposit2(P, rot_R(rb, zR, zV), rot_R(rp, zR, zV), histA, histB, Np1, valid);
            }
            if (k > 0) {
                float4* o = (float4*)(dst + base);
                o[0] = make_float4(zo[0], zo[1], zo[2], zo[3]);
                o[1] = make_float4(zo[4], zo[5], zo[6], zo[7]);
            }
        }
        rev = !rev;
        if (last_fine) break;
        if (track) {
            cnt = __reduce_add_sync(0xffffffffu, cnt);
            if (lane == 0 && cnt) atomicAdd(&s_cnt, (int)cnt);
        }
        __syncthreads();
        flush32(P, B, hist, cyc, lb);
        if (lb == 0 && threadIdx.x == 0) B.notdone[(k + 1) % 3] = 0;
        if (threadIdx.x == 0 && s_cnt) atomicAdd(&B.notdone[k % 3], s_cnt);
        if (!grid_sync(P, B.bar, gen, B.status, &s_ok, (unsigned int)nb)) return;
        build_fields32(P, B.Qring + (size_t)(cyc % 3) * 2 * Np1 * kQPad, (long long*)hist, g, tabA, cq, s_edA,
                       s_warp, s_c, track ? &B.notdone[k % 3] : nullptr, &s_stop);
        if (track && s_stop) {
            K = k;
            break;
        }
        ++cyc;

        // ---- sweep B(k): gather pair 1 of step k, deposit stage pair 2
        for (int idx = threadIdx.x; idx < copies * 2 * hw; idx += blockDim.x) hist[idx] = 0u;
        if (threadIdx.x == 0) s_next = 0;
        __syncthreads();
        const float2 rq = P.rot[rot_index(P, 2ll * k + 2)];  // Phi(t_k + h)
        const float2* srcB = row(k);
        for (long long gi = grab(); gi >= 0; gi = grab()) {
            const long long base = gi * kGroup + lane * kG;
            load_grp(srcB, nullptr, nullptr, base, false, false, cur);
            float eo[2 * kG];
#pragma unroll
            for (int q = 0; q < kG; ++q) {
                const bool valid = base + q < n;
                const float zR = grp_get(cur, 2 * q), zV = grp_get(cur, 2 * q + 1);
                const float R3 = rot_R(rp, zR, zV);
                float e1, e3;
                locate_gather2(P, rot_R(rb, zR, zV), R3, tabA, tabA + Np1, s_edA, e1, e3);
                eo[2 * q] = e1;
                eo[2 * q + 1] = e3;
                locate_deposit2(P, lawson32_R2(P, R3, e1), lawson32_R4(P, rq, zR, zV, e3), histA, histB, Np1, valid);
            }
            float4* o = (float4*)(B.ce + base);
            o[0] = make_float4(eo[0], eo[1], eo[2], eo[3]);
            o[1] = make_float4(eo[4], eo[5], eo[6], eo[7]);
        }
        rev = !rev;
        __syncthreads();
        flush32(P, B, hist, cyc, lb);
        if (!grid_sync(P, B.bar, gen, B.status, &s_ok, (unsigned int)nb)) return;
        build_fields32(P, B.Qring + (size_t)(cyc % 3) * 2 * Np1 * kQPad, (long long*)hist, g, tabB, cq, s_edB,
                       s_warp, s_c);
        ++cyc;
    }

    if (lb == 0 && threadIdx.x == 0 && !fine_only) *B.K_out = K;
    if (mode != MODE_ETD) return;

    // ---- landing (step 3) and extrapolation (step 4); row k holds z_k
    for (long long i = tid; i < n; i += nthreads) {
        const CTime o = B.o[i], T = B.T[i];
        const int N = B.N[i];
        float yv[2][2];
        const int nt = N > 0 ? 2 : 1;
        for (int t = 0; t < nt; ++t) {
            const CTime u = t == 0 ? o : ct_add(o, T);
            float R[3], V[3];
            for (int r = 0; r < 3; ++r) {
                const long long kk = (long long)u.i + r;
                const float2 z = row(kk)[i];
                const float2 cs = P.rot[rot_index(P, 2 * kk)];
                R[r] = rot_R(cs, z.x, z.y);
                V[r] = rot_V(cs, z.x, z.y);
            }
            yv[t][0] = interp3f(R[0], R[1], R[2], u.f);
            yv[t][1] = interp3f(V[0], V[1], V[2], u.f);
        }
        float2 out;
        if (N > 0) {
            const float Nf = (float)N;
            out = make_float2(fmaf(Nf, yv[1][0] - yv[0][0], yv[0][0]), fmaf(Nf, yv[1][1] - yv[0][1], yv[0][1]));
        } else {
            out = make_float2(yv[0][0], yv[0][1]);
        }
        B.y[i] = out;
    }
}

__global__ void __launch_bounds__(kW32Threads, 1) k_window32_coop(DevParams P, WinBufs32 B, int mode, int T_known,
                                                                  long long n_fine, const CTime* __restrict__ Tin) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    window32_coop_body(P, B, mode, T_known, n_fine, Tin, blockIdx.x, gridDim.x, smem_raw);
}

// ------------------------------------------- per-particle window (analytic E)

// The per-particle loops below keep the table position of fine step k,
// ia = 2k mod 2 spt, and advance it by one step with a compare instead of
// a remainder by the run-time table length (which costs more than the
// step's own arithmetic).  ia is even, so ia + 1 is always in the table.
__device__ __forceinline__ int rot_next(const DevParams& P, int ia) {
    const int t = ia + 2;
    return t == 2 * P.spt ? 0 : t;
}

// One fine step k -> k+1 of Lawson RK4 in the rotating frame, analytic
// field; ia = 2k mod 2 spt.
template <int FIELD>
__device__ __forceinline__ void step32_analytic(const DevParams& P, int ia, float& zR, float& zV) {
    const float2 a = P.rot[ia];
    const float2 m = P.rot[ia + 1];
    const float2 b = P.rot[rot_next(P, ia)];
    const float R3 = rot_R(m, zR, zV);
    const float e1 = field_analytic32(FIELD, rot_R(a, zR, zV));
    const float e3 = field_analytic32(FIELD, R3);
    const float e2 = field_analytic32(FIELD, lawson32_R2(P, R3, e1));
    const float e4 = field_analytic32(FIELD, lawson32_R4(P, b, zR, zV, e3));
    lawson32_update(P, a, m, b, e1, e2, e3, e4, zR, zV);
}

// y = Phi(t_k) z with ia = 2k mod 2 spt (y_at) or any k (y_of).
__device__ __forceinline__ float2 y_at(const DevParams& P, int ia, float zR, float zV) {
    const float2 cs = P.rot[ia];
    return make_float2(rot_R(cs, zR, zV), rot_V(cs, zR, zV));
}
__device__ __forceinline__ float2 y_of(const DevParams& P, long long k, float zR, float zV) {
    return y_at(P, rot_index(P, 2 * k), zR, zV);
}

template <int FIELD>
__device__ __forceinline__ void window32_local_body(const DevParams& P, const WinBufs32& B, int mode, int T_known,
                                                    long long n_iter, const CTime* __restrict__ Tin, int lb, int nb) {
    const long long n = P.n, ld = B.ld;
    const long long stride = (long long)nb * blockDim.x;
    int Kmax_seen = 0;
    for (long long i = (long long)lb * blockDim.x + threadIdx.x; i < n; i += stride) {
        const float2 y0 = B.y[i];
        float zR = y0.x, zV = y0.y;
        if (mode == MODE_FINE) {
            int ia = 0;
            for (long long k = 0; k < n_iter; ++k) {
                step32_analytic<FIELD>(P, ia, zR, zV);
                ia = rot_next(P, ia);
            }
            B.y[i] = y_at(P, ia, zR, zV);
            continue;
        }
        if (mode == MODE_PERIODS) {
            int flags = 0;
            CTime t1, T;
            t1.i = 0;
            t1.f = 0.0f;
            T = t1;
            float vkm2 = 0.0f, vkm1 = zV;
            int K = 0, ia = 0;
            for (;;) {
                if (flags & F_RES) break;
                if (K == P.Kmax) {
                    flags |= F_FB | F_RES;
                    T.i = P.spt;
                    T.f = 0.0f;
                    break;
                }
                step32_analytic<FIELD>(P, ia, zR, zV);
                ia = rot_next(P, ia);
                ++K;
                const float v = y_at(P, ia, zR, zV).y;
                if (K >= 2 && positive32(vkm2) != positive32(vkm1)) {
                    const float s = quad_root01f(vkm2, vkm1, v);
                    const int ne = (flags & F_NEXT) + 1;
                    flags = (flags & ~F_NEXT) | (ne & F_NEXT);
                    if (ne == 1) {
                        t1.i = K - 2;
                        t1.f = s;
                    }
                    if (ne == 3) {
                        T = ct_norm((long long)(K - 2) - t1.i, s - t1.f);
                        flags |= F_RES;
                    }
                }
                vkm2 = vkm1;
                vkm1 = v;
            }
            B.T[i] = T;
            B.tr[i] = (unsigned int)flags;
            Kmax_seen = max(Kmax_seen, K);
            continue;
        }
        // MODE_ETD: n_iter macro steps of this particle
        int flags = 0;
        Decomp32 d;
        d.N = 0;
        d.need = 0;
        if (T_known) d = resolve32(P, Tin[i], true, flags);
        int K = 0;
        for (long long mstep = 0; mstep < n_iter; ++mstep) {
            float ya[2], yb[2];
            if (T_known) {
                // o, T and the stencils are known before the window starts
                const int k1 = d.o.i;
                const CTime u2 = ct_add(d.o, d.T);
                const int k2 = d.N > 0 ? u2.i : -10;
                float a[3], b[3], c[3], e[3];
                K = 0;
                int ia = 0;
                for (;;) {
                    const int r1 = K - k1, r2 = K - k2;
                    if (r1 >= 0 && r1 < 3) {
                        const float2 y = y_at(P, ia, zR, zV);
                        a[r1] = y.x;
                        b[r1] = y.y;
                    }
                    if (r2 >= 0 && r2 < 3) {
                        const float2 y = y_at(P, ia, zR, zV);
                        c[r2] = y.x;
                        e[r2] = y.y;
                    }
                    if (K >= d.need) break;
                    step32_analytic<FIELD>(P, ia, zR, zV);
                    ia = rot_next(P, ia);
                    ++K;
                }
                ya[0] = interp3f(a[0], a[1], a[2], d.o.f);
                ya[1] = interp3f(b[0], b[1], b[2], d.o.f);
                if (d.N > 0) {
                    yb[0] = interp3f(c[0], c[1], c[2], u2.f);
                    yb[1] = interp3f(e[0], e[1], e[2], u2.f);
                } else {
                    yb[0] = ya[0];
                    yb[1] = ya[1];
                }
            } else {
                // step 1 on the fly: track the extrema, store z_k as row k
                int fl = 0;
                CTime t1;
                t1.i = 0;
                t1.f = 0.0f;
                float vkm2 = 0.0f, vkm1 = zV;
                K = 0;
                int ia = 0;
                B.y[i] = make_float2(zR, zV);
                for (;;) {
                    if ((fl & F_RES) && K >= d.need) break;
                    if (K == P.Kmax) {
                        if (!(fl & F_RES)) {
                            CTime Tfb;
                            Tfb.i = P.spt;
                            Tfb.f = 0.0f;
                            fl |= F_FB;
                            d = resolve32(P, Tfb, true, fl);
                        }
                        break;
                    }
                    step32_analytic<FIELD>(P, ia, zR, zV);
                    ia = rot_next(P, ia);
                    ++K;
                    B.traj[(size_t)(K - 1) * ld + i] = make_float2(zR, zV);
                    const float v = y_at(P, ia, zR, zV).y;
                    if (!(fl & F_RES) && K >= 2 && positive32(vkm2) != positive32(vkm1)) {
                        const float s = quad_root01f(vkm2, vkm1, v);
                        const int ne = (fl & F_NEXT) + 1;
                        fl = (fl & ~F_NEXT) | (ne & F_NEXT);
                        if (ne == 1) {
                            t1.i = K - 2;
                            t1.f = s;
                        }
                        if (ne == 3) d = resolve32(P, ct_norm((long long)(K - 2) - t1.i, s - t1.f), true, fl);
                    }
                    vkm2 = vkm1;
                    vkm1 = v;
                }
                flags = fl;
                const int nt = d.N > 0 ? 2 : 1;
                for (int t = 0; t < nt; ++t) {
                    const CTime u = t == 0 ? d.o : ct_add(d.o, d.T);
                    float R[3], V[3];
                    for (int r = 0; r < 3; ++r) {
                        const long long kk = (long long)u.i + r;
                        const float2 z = kk == 0 ? B.y[i] : B.traj[(size_t)(kk - 1) * ld + i];
                        const float2 y = y_of(P, kk, z.x, z.y);
                        R[r] = y.x;
                        V[r] = y.y;
                    }
                    (t == 0 ? ya : yb)[0] = interp3f(R[0], R[1], R[2], u.f);
                    (t == 0 ? ya : yb)[1] = interp3f(V[0], V[1], V[2], u.f);
                }
                if (nt == 1) {
                    yb[0] = ya[0];
                    yb[1] = ya[1];
                }
            }
            if (d.N > 0) {
                const float Nf = (float)d.N;
                zR = fmaf(Nf, yb[0] - ya[0], ya[0]);
                zV = fmaf(Nf, yb[1] - ya[1], ya[1]);
            } else {
                zR = ya[0];
                zV = ya[1];
            }
            Kmax_seen = max(Kmax_seen, K);
        }
        B.y[i] = make_float2(zR, zV);
        if (n_iter > 0) {
            B.T[i] = d.T;
            B.o[i] = d.o;
            B.N[i] = d.N;
            B.tr[i] = (unsigned int)flags | ((unsigned int)d.need << 8);
        }
    }
    Kmax_seen = __reduce_max_sync(0xffffffffu, (unsigned)Kmax_seen);
    if ((threadIdx.x & 31) == 0 && Kmax_seen > 0) atomicMax((long long*)B.K_out, (long long)Kmax_seen);
}

template <int FIELD>
__global__ void __launch_bounds__(256) k_window32_local(DevParams P, WinBufs32 B, int mode, int T_known,
                                                        long long n_iter, const CTime* __restrict__ Tin) {
    window32_local_body<FIELD>(P, B, mode, T_known, n_iter, Tin, blockIdx.x, gridDim.x);
}

// ------------------------------------------------------------- batched form

// One cooperative launch advances every beam of a batch by one macro step:
// each block finds its beam, copies the beam's descriptor to shared memory
// and runs that beam's window on the beam's own blocks (its barriers count
// only them).  Beams never wait for each other.
__global__ void __launch_bounds__(kW32Threads, 1) k_window32_batch(const BeamDesc32* __restrict__ beams, int n_beams) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    __shared__ BeamDesc32 D;
    __shared__ int s_beam;
    if (threadIdx.x == 0) {
        int lo = 0, hi = n_beams - 1;
        while (lo < hi) {
            const int mid = (lo + hi + 1) >> 1;
            if (beams[mid].first_block <= (int)blockIdx.x) lo = mid;
            else hi = mid - 1;
        }
        s_beam = lo;
    }
    __syncthreads();
    {
        const unsigned int* src = reinterpret_cast<const unsigned int*>(beams + s_beam);
        unsigned int* dst = reinterpret_cast<unsigned int*>(&D);
        for (int i = threadIdx.x; i < (int)(sizeof(BeamDesc32) / 4); i += blockDim.x) dst[i] = src[i];
    }
    __syncthreads();
    const int lb = (int)blockIdx.x - D.first_block;
    if (threadIdx.x == 0) atomicMin(&D.t_ns[0], (unsigned long long)global_ns());
    if (D.coop) window32_coop_body(D.P, D.B, MODE_ETD, D.T_known, 0, D.Tin, lb, D.n_blocks, smem_raw);
    else if (D.P.field == 1) window32_local_body<1>(D.P, D.B, MODE_ETD, D.T_known, 1, D.Tin, lb, D.n_blocks);
    else window32_local_body<2>(D.P, D.B, MODE_ETD, D.T_known, 1, D.Tin, lb, D.n_blocks);
    __syncthreads();  // the block's last thread is done before its end time
    if (threadIdx.x == 0) atomicMax(&D.t_ns[1], (unsigned long long)global_ns());
}

__global__ void k_batch_reset(const BeamDesc32* __restrict__ beams, int n_beams) {
    const int b = blockIdx.x;
    if (b >= n_beams) return;
    const BeamDesc32& D = beams[b];
    if (D.coop) {
        const size_t q = (size_t)3 * 2 * (D.P.n_cells + 1) * kQPad;
        for (size_t i = threadIdx.x; i < q; i += blockDim.x) D.B.Qring[i] = 0ull;
        for (int i = threadIdx.x; i < 64; i += blockDim.x) D.B.bar[i] = 0u;
        if (threadIdx.x < 3) D.B.notdone[threadIdx.x] = 0;
    }
    if (threadIdx.x == 0) {
        *D.B.K_out = 0;
        *D.B.status = 0;
        D.t_ns[0] = ~0ull;
        D.t_ns[1] = 0ull;
    }
}

__global__ void k_batch_status(const BeamDesc32* __restrict__ beams, int n_beams, int* __restrict__ out) {
    for (int b = blockIdx.x * blockDim.x + threadIdx.x; b < n_beams; b += gridDim.x * blockDim.x)
        out[b] = *beams[b].B.status;
}

size_t window32_batch_smem(int max_cells, int copies) { return max_cells > 0 ? coop32_smem_bytes(max_cells, copies) : 0; }

cudaError_t window32_batch_attr(size_t smem) {
    return cudaFuncSetAttribute(k_window32_batch, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
}

cudaError_t window32_batch_occupancy(int block, size_t smem, int* blocks_per_sm) {
    return cudaOccupancyMaxActiveBlocksPerMultiprocessor(blocks_per_sm, k_window32_batch, block, smem);
}

cudaError_t launch_window32_batch(const BeamDesc32* beams, int n_beams, int grid, int block, size_t smem,
                                  cudaStream_t st) {
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(grid);
    cfg.blockDim = dim3(block);
    cfg.dynamicSmemBytes = smem;
    cfg.stream = st;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeCooperative;
    attr[0].val.cooperative = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    return cudaLaunchKernelEx(&cfg, k_window32_batch, beams, n_beams);
}

cudaError_t launch_batch_reset(const BeamDesc32* beams, int n_beams, cudaStream_t st) {
    k_batch_reset<<<n_beams, 256, 0, st>>>(beams, n_beams);
    return cudaGetLastError();
}

cudaError_t launch_batch_status(const BeamDesc32* beams, int n_beams, int* out, cudaStream_t st) {
    k_batch_status<<<1, 256, 0, st>>>(beams, n_beams, out);
    return cudaGetLastError();
}

// ------------------------------------------------------------- moments

// Per-block partial sums of the FP32 state, accumulated in FP64 (the global
// diagnostics of the form).
__global__ void k_moments32(DevParams P, WinBufs32 B, double* part_d, long long* part_i) {
    __shared__ double sd[32][kMomDoubles];
    __shared__ long long si[32][kMomInts];
    const long long n = P.n, stride = (long long)gridDim.x * blockDim.x;
    double a[kMomDoubles] = {0, 0, 0, 0, 0, 0, INFINITY, -INFINITY};
    long long b[kMomInts] = {LLONG_MAX, LLONG_MIN, 0};
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += stride) {
        const float2 y = B.y[i];
        const CTime Tc = B.T[i];
        const double R = y.x, V = y.y, T = (double)Tc.i + (double)Tc.f;
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
        b[2] += (B.tr[i] & (unsigned int)F_FB) ? 1 : 0;
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

cudaError_t window32_prepare(DevParams& P, int block, int blocks_per_sm, int sm_count, long long ld,
                             WindowLaunch* L) {
    L->coop_block = block;
    // histogram copies: as many as fit (up to kHist32CopiesMax) while a block
    // deposits enough positions per cycle for same-cell conflicts to matter
    int copies = kHist32CopiesMax;
    const long long per_block_est = P.n / (sm_count > 0 ? sm_count : 1);
    while (copies > 1 && (coop32_smem_bytes(P.n_cells, copies) > 200 * 1024 || per_block_est < 64ll * copies * 32))
        copies >>= 1;
    P.hist_copies = copies;
    L->coop_smem = coop32_smem_bytes(P.n_cells, copies);
    L->hist = 0;
    L->stage = 0;
    if (L->coop_smem > 227 * 1024) return cudaErrorNotSupported;
    cudaError_t e = cudaFuncSetAttribute(k_window32_coop, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)L->coop_smem);
    if (e != cudaSuccess) return e;
    int bps = 0;
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&bps, k_window32_coop, block, L->coop_smem);
    if (e != cudaSuccess) return e;
    if (bps < 1) return cudaErrorInvalidConfiguration;
    const int want = blocks_per_sm > 0 ? blocks_per_sm : 1;
    if (want < bps) bps = want;
    const long long n_groups = ld / kGroup;
    const long long warps = block / 32;
    const long long need_blocks = (n_groups + warps - 1) / warps;
    long long grid = (long long)bps * sm_count;
    if (need_blocks < grid) grid = need_blocks < 1 ? 1 : need_blocks;
    L->coop_grid = (int)grid;
    // the 32-bit histogram words stay exact up to 2^21 positions per block,
    // field and cycle
    const long long per_block = (n_groups + grid - 1) / grid * kGroup;
    if (per_block > (1ll << 21)) return cudaErrorNotSupported;
    return cudaSuccess;
}

long long window32_row_stride(long long n) { return (n + kGroup - 1) / kGroup * kGroup; }

cudaError_t launch_window32_coop(const DevParams& P, const WinBufs32& B, const WindowLaunch& L, int mode,
                                 int T_known, long long n_fine, cudaStream_t st, long long* launches,
                                 const CTime* Tin) {
    DevParams Pc = P;
    WinBufs32 Bc = B;
    void* args[] = {&Pc, &Bc, &mode, &T_known, &n_fine, &Tin};
    cudaError_t e = cudaLaunchCooperativeKernel((void*)k_window32_coop, dim3(L.coop_grid), dim3(L.coop_block), args,
                                                L.coop_smem, st);
    if (launches) ++*launches;
    return e;
}

cudaError_t launch_window32_local(const DevParams& P, const WinBufs32& B, int mode, int T_known, long long n_iter,
                                  int block, int sm_count, cudaStream_t st, long long* launches, const CTime* Tin) {
    long long want = (P.n + block - 1) / block;
    long long cap = (long long)sm_count * 16;
    int grid = (int)(want < cap ? (want < 1 ? 1 : want) : cap);
    if (P.field == 1) k_window32_local<1><<<grid, block, 0, st>>>(P, B, mode, T_known, n_iter, Tin);
    else k_window32_local<2><<<grid, block, 0, st>>>(P, B, mode, T_known, n_iter, Tin);
    if (launches) ++*launches;
    return cudaGetLastError();
}

cudaError_t launch_moments32(const DevParams& P, const WinBufs32& B, double* part_d, long long* part_i, int grid,
                             cudaStream_t st, long long* launches) {
    k_moments32<<<grid, 256, 0, st>>>(P, B, part_d, part_i);
    if (launches) ++*launches;
    return cudaGetLastError();
}

}  // namespace pic

// mlp.cu -- the network of the learned stepper: a 5-64-64-2 GELU perceptron
// with bfloat16 weights and FP32 accumulation, its 64 x 64 products on the
// 5th-generation tensor cores (tcgen05.mma, bf16 x bf16 -> f32 in tensor
// memory) for inference, the learned step's correction and training.  The paper has no
// learned component; the network corrects one macro step of the improved ETD
// scheme (Algorithm ETDFSSModAlgo) and is defined, with its rounding points,
// as:
//
//   x = (r, v, sin(t/eps), cos(t/eps), dt)
//   z1 = W1 x + b1,   h1 = gelu(z1)                 (CUDA cores, FP32)
//   z2 = W2 bf16(h1) + b2,  h2 = gelu(z2)           (tensor cores)
//   out = W3 bf16(h2) + b3                          (CUDA cores, FP32)
//
// W1, W2, W3 are the bfloat16 roundings of FP32 master weights; gelu(u) =
// u erfc(-u / sqrt 2) / 2.  Training minimises sum((out - y)^2) / (2B) with
// Adam on the master weights.  Backward:
//   dout = (out - y) / B, dW3 = dout^T bf16(h2), db3 = sum dout,
//   dz2 = (dout W3) gelu'(z2), dW2 = bf16(dz2)^T bf16(h1), db2 = sum dz2,
//   dz1 = (bf16(dz2) W2) gelu'(z1), dW1 = dz1^T x, db1 = sum dz1.
// The per-sample part (forward, dz1, dz2) runs one sample per thread and 128
// per MMA tile; the weight gradients are reduced over the batch by a second
// kernel (dW2 on the tensor cores, the samples as the reduction dimension)
// into per-block partials, which a third kernel sums in a fixed order before
// the Adam update, so training is reproducible bit for bit.
#include <cuda_bf16.h>

#include <algorithm>
#include <cmath>
#include <cstring>
#include <new>
#include <vector>

#include "energy_check.cuh"
#include "gelu_fast.cuh"
#include "pic_internal.h"
#include "tc_desc.cuh"

namespace pic {

// flat parameter layout (FP32 masters)
constexpr int kMIn = 5, kMHid = 64, kMOut = 2;
constexpr int oW1 = 0, ob1 = oW1 + kMHid * kMIn, oW2 = ob1 + kMHid, ob2 = oW2 + kMHid * kMHid, oW3 = ob2 + kMHid,
              ob3 = oW3 + kMOut * kMHid, kMParams = ob3 + kMOut;
static_assert(kMParams == 4674, "parameter count");
// compact FP32 block used by the CUDA-core layers: bf16-rounded W1 and W3, biases
constexpr int sW1 = 0, sb1 = sW1 + kMHid * kMIn, sb2 = sb1 + kMHid, sW3 = sb2 + kMHid, sb3 = sW3 + kMOut * kMHid,
              kMSmall = sb3 + kMOut;

constexpr int kWgTile = 64;      // samples per staged tile of the weight gradients
constexpr int kWgMaxBlocks = 256;

struct MlpDev {
    float *master, *m, *v;
    __nv_bfloat16* W2b;   // [j][k]
    __nv_bfloat16* W2Tb;  // [k][j]
    float* small;         // kMSmall
    // training scratch for up to max_batch samples
    float* xs;            // [B][5]
    float* dz1;           // [B][64]
    float* dz2;           // [B][64]
    __nv_bfloat16* h1b;   // [B][64]
    __nv_bfloat16* h2b;   // [B][64]
    float* dout;          // [B][2]
    float* loss_part;     // per forward block
    float* grad_part;     // [kWgMaxBlocks][kMParams]
    float* grad;          // [kMParams]
    float* loss;          // [1]
    int* err;             // set by a tensor-core wait that ran out of time
};

// ------------------------------------------------------------ device math

__device__ __forceinline__ float gelu_d(float u) {
    return 0.5f * erfcf(-u * 0.70710678118654752f) + u * 0.39894228040143268f * expf(-0.5f * u * u);
}
__device__ __forceinline__ unsigned int pack_bf16(float lo, float hi) {
    __nv_bfloat162 v = __floats2bfloat162_rn(lo, hi);
    return *reinterpret_cast<unsigned int*>(&v);
}
__device__ __forceinline__ float round_bf16(float x) { return __bfloat162float(__float2bfloat16_rn(x)); }

// Sample index of batch row s: ((first + s) * mul) mod n_data (a permutation
// of the data set when mul is coprime with n_data).
__device__ __forceinline__ long long sample_index(long long s, long long first, long long mul, long long n_data) {
    return (long long)(((unsigned long long)(first + s) % (unsigned long long)n_data) * (unsigned long long)mul %
                       (unsigned long long)n_data);
}

struct AdamArgs {
    float lr, beta1, beta2, eps, c1, c2;  // c1, c2: bias corrections 1/(1 - beta^t)
    int apply;                            // 0: gradients only
};

// Sums the partials of n_part blocks in block order, writes the gradient and
// the batch loss, applies Adam to the masters and refreshes the rounded copies.
__global__ void k_mlp_update(MlpDev M, int n_part, int n_loss, AdamArgs A) {
    const int p = blockIdx.x * blockDim.x + threadIdx.x;
    if (p == 0) {
        float s = 0.f;
        for (int b = 0; b < n_loss; ++b) s += M.loss_part[b];
        *M.loss = s;
    }
    if (p >= kMParams) return;
    float gsum = 0.f;
    for (int b = 0; b < n_part; ++b) gsum += M.grad_part[(size_t)b * kMParams + p];
    M.grad[p] = gsum;
    if (!A.apply) return;
    const float m = A.beta1 * M.m[p] + (1.f - A.beta1) * gsum;
    const float v = A.beta2 * M.v[p] + (1.f - A.beta2) * gsum * gsum;
    M.m[p] = m;
    M.v[p] = v;
    const float w = M.master[p] - A.lr * (m * A.c1) / (sqrtf(v * A.c2) + A.eps);
    M.master[p] = w;
}

// bf16 / compact copies of the masters.
__global__ void k_mlp_refresh(MlpDev M) {
    const int p = blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= kMParams) return;
    const float w = M.master[p];
    if (p >= oW2 && p < ob2) {
        const int j = (p - oW2) / kMHid, k = (p - oW2) % kMHid;
        const __nv_bfloat16 b = __float2bfloat16_rn(w);
        M.W2b[j * kMHid + k] = b;
        M.W2Tb[k * kMHid + j] = b;
    } else if (p < ob1) {
        M.small[sW1 + p] = round_bf16(w);
    } else if (p < oW2) {
        M.small[sb1 + (p - ob1)] = w;
    } else if (p < oW3) {
        M.small[sb2 + (p - ob2)] = w;
    } else if (p < ob3) {
        M.small[sW3 + (p - oW3)] = round_bf16(w);
    } else {
        M.small[sb3 + (p - ob3)] = w;
    }
}

// ------------------------------------------------------------ learned step

// Potential psi (psi' = E, psi(0) = 0) of the field the gather sees: E linear
// in each cell, so psi is quadratic there; off the mesh E = rE_edge / r.
__device__ __forceinline__ double psi_at(const LearnedArgs& A, double R) {
    if (A.field == PIC_FIELD_DUFFING) return -0.25 * ((R * R) * (R * R));
    if (A.field != PIC_FIELD_POISSON) return 0.0;
    const double x = (R - A.r_min) * A.inv_hr;
    if (x >= 0.0 && x < (double)A.n_cells) {
        const int j = (int)floor(x);
        const double d = R - (A.r_min + (double)j * A.hr);
        const double Ej = A.E[j], Ej1 = A.E[j + 1];
        return A.psi[j] + Ej * d + (Ej1 - Ej) * (d * d) * (0.5 * A.inv_hr);
    }
    if (x < 0.0) return A.psi[0] + A.edges[0] * log(R / A.r_min);
    return A.psi[A.n_cells] + A.edges[1] * log(R / -A.r_min);  // beyond r_max (NaN propagates)
}

// Frozen-field energy (R^2 + V^2)/2 - eps psi(R): conserved by the
// characteristics dR/dt = V/eps, dV/dt = -R/eps + E(R) when E does not change.
__device__ __forceinline__ double frozen_energy(const LearnedArgs& A, double R, double V) {
    return 0.5 * (R * R + V * V) - A.eps * psi_at(A, R);
}

// The FP64 rule, out of line: it runs only for the particles the binary32
// check leaves undecided (and for every particle of FP64 handles).
static __device__ __noinline__ bool frozen_keep_fp64(const LearnedArgs& A, double Rp, double Vp, double Rl,
                                                     double Vl) {
    const double H0 = frozen_energy(A, Rp, Vp);
    const double H1 = frozen_energy(A, Rl, Vl);
    return fabs(H1 - H0) <= A.tol * fabs(H0);
}

// ------------------------------------------------------------ tensor-core inference (tcgen05)
//
// Inference of the network (pic_mlp_forward) and the learned step's
// correction with the 64 x 64 hidden layer on the 5th-generation tensor
// cores: a block of 128 threads owns 128 samples (one per thread), writes
// bf16(gelu(z1)) as the A operand (128 x 64, K-major core matrices) to shared
// memory, and one thread issues four tcgen05.mma (M = 128, N = 64, K = 16
// each) against W2 (B operand, 64 x 64) into a 64-column f32 accumulator in
// tensor memory and commits them to an mbarrier; each warp then reads its 32
// rows back with tcgen05.ld.  The output layer adds the products of each
// sample's 64 columns in four fused multiply-add chains of 16 (columns
// 8 nt + 2 q + e for chain q) combined as (s0 + s1) + (s2 + s3).  Where a
// GELU is rounded to bfloat16 at once it is evaluated by gelu_for_bf16
// (gelu_fast.cuh), which rounds exactly as the erfc form does.

constexpr int kTcThreads = 128;  // one sample per thread, one 128-row MMA tile per block
constexpr int kTcCols = 64;      // TMEM columns of the accumulator (N = 64, f32)

struct TcSmem {
    alignas(1024) unsigned char A[kTcThreads * kMHid * 2];  // bf16(h1): 128 x 64, K-major core matrices
    alignas(1024) unsigned char Bw[kMHid * kMHid * 2];      // W2: 64 (N) x 64 (K)
    float4 l1[kMHid][2];  // per hidden unit: (W1[j][0..3]), (W1[j][4], b1[j], 0, 0)
    float4 l3[kMHid];     // per hidden unit: (b2[j], W3[0][j], W3[1][j], 0)
    float b3[kMOut];
    float4 gtab[kGeluSeg + 1];  // segment table of gelu_for_bf16
    unsigned long long mbar;
    unsigned int taddr;
    int fail;
};

__device__ __forceinline__ uint32_t smem_u32(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ __forceinline__ void tc_fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void tc_fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }

// 16 f32 columns [col, col + 16) of this warp's 32 TMEM lanes (lane = row of the tile)
__device__ __forceinline__ void tc_ld16(uint32_t taddr, float* v) {
    uint32_t r[16];
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, "
        "%15}, [%16];"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]), "=r"(r[8]),
          "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
        : "r"(taddr)
        : "memory");
#pragma unroll
    for (int i = 0; i < 16; ++i) v[i] = __uint_as_float(r[i]);
}

// mbarrier phase wait with a time limit; false when it ran out
__device__ __forceinline__ bool tc_wait(uint32_t mbar, uint32_t parity) {
    const long long t0 = clock64();
    for (;;) {
        uint32_t done;
        asm volatile(
            "{\n\t.reg .pred p;\n\tmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\tselp.u32 %0, 1, 0, p;\n\t}\n"
            : "=r"(done)
            : "r"(mbar), "r"(parity)
            : "memory");
        if (done) return true;
        if (clock64() - t0 > (2ll << 30)) return false;  // ~1 s at 2 GHz
    }
}

// MODE 0: outputs to Y (pic_mlp_forward); 1, 2: the learned step's
// correction of an FP64 / FP32 state, kept where the frozen-field energy
// check allows it.
template <int MODE>
__global__ void __launch_bounds__(kTcThreads) k_mlp_tc(MlpDev M, LearnedArgs A, const float* __restrict__ X,
                                                       float* __restrict__ Y, long long n) {
    __shared__ TcSmem S;
    extern __shared__ float s_tab[];  // binary32 field tables of the energy check (MODE 2, Poisson)
    const int t = threadIdx.x, warp = t >> 5;
    // W2 as the B operand; the CUDA-core layers' weights packed per hidden unit
    for (int i = t; i < kMHid * kMHid / 8; i += kTcThreads) {
        const int nrow = i >> 3, kb = i & 7;  // 8 consecutive k of output row nrow
        *reinterpret_cast<uint4*>(S.Bw + tc_kmajor_offset(nrow, kb * 8)) =
            *reinterpret_cast<const uint4*>(M.W2b + nrow * kMHid + kb * 8);
    }
    if (t < kMHid) {
        const float* w1 = M.small + sW1 + t * kMIn;
        S.l1[t][0] = make_float4(w1[0], w1[1], w1[2], w1[3]);
        S.l1[t][1] = make_float4(w1[4], M.small[sb1 + t], 0.f, 0.f);
        S.l3[t] = make_float4(M.small[sb2 + t], M.small[sW3 + t], M.small[sW3 + kMHid + t], 0.f);
    }
    if (t < kMOut) S.b3[t] = M.small[sb3 + t];
    if (t <= kGeluSeg) S.gtab[t] = make_float4(c_gelu_tab[t][0], c_gelu_tab[t][1], c_gelu_tab[t][2], c_gelu_tab[t][3]);
    if (MODE == 2 && A.tab_f)
        for (int i = t; i < 3 * (A.n_cells + 1); i += kTcThreads) s_tab[i] = A.tab_f[i];
    if (t == 0) {
        asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(&S.mbar)) : "memory");
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
        S.fail = 0;
    }
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(&S.taddr)),
                     "r"(kTcCols)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t taddr = S.taddr;
    const uint32_t idesc = tc_idesc_bf16_f32(kTcThreads, kMHid);
    const uint32_t a_base = smem_u32(S.A), b_base = smem_u32(S.Bw), mbar = smem_u32(&S.mbar);

    EnergyF32 E32;
    E32.field = A.field;
    E32.eps = (float)A.eps;
    E32.tol = (float)A.tol;
    E32.n_cells = A.n_cells;
    E32.r_min = (float)A.r_min;
    E32.hr = (float)A.hr;
    E32.inv_hr = (float)A.inv_hr;
    const float* tab_f = (MODE == 2 && A.tab_f) ? s_tab : nullptr;
    E32.E = tab_f;
    E32.slope = tab_f ? tab_f + (A.n_cells + 1) : nullptr;
    E32.psi = tab_f ? tab_f + 2 * (A.n_cells + 1) : nullptr;
    if (A.field == PIC_FIELD_POISSON && !tab_f) E32.field = -1;  // no tables: every particle in FP64

    unsigned int fallback = 0;
    uint32_t parity = 0;
    const long long tiles = (n + kTcThreads - 1) / kTcThreads;
    for (long long tile = blockIdx.x; tile < tiles; tile += gridDim.x) {
        const long long s = tile * kTcThreads + t;
        const bool valid = s < n;
        float x[kMIn];
        if (MODE == 0) {
#pragma unroll
            for (int i = 0; i < kMIn; ++i) x[i] = valid ? X[s * kMIn + i] : 0.f;
        } else {
            if (MODE == 1) {
                const double2 v = valid ? ((const double2*)A.y_prev)[s] : make_double2(0.0, 0.0);
                x[0] = (float)v.x;
                x[1] = (float)v.y;
            } else {
                const float2 v = valid ? ((const float2*)A.y_prev)[s] : make_float2(0.f, 0.f);
                x[0] = v.x;
                x[1] = v.y;
            }
            x[2] = A.in_sin;
            x[3] = A.in_cos;
            x[4] = A.in_dt;
        }
        // layer 1 + GELU into the A operand: row t, 8 columns (one 16-byte
        // core-matrix row) per pass; the pass loop stays rolled, since 64
        // inlined erfc evaluations per layer overflow the instruction cache
#pragma unroll 1
        for (int kb = 0; kb < kMHid / 8; ++kb) {
            unsigned int packed[4];
#pragma unroll
            for (int e = 0; e < 8; e += 2) {
                float h[2];
#pragma unroll
                for (int q = 0; q < 2; ++q) {
                    const int col = kb * 8 + e + q;
                    const float4 wa = S.l1[col][0], wb = S.l1[col][1];
                    float z = wb.y;
                    z = fmaf(wa.x, x[0], z);
                    z = fmaf(wa.y, x[1], z);
                    z = fmaf(wa.z, x[2], z);
                    z = fmaf(wa.w, x[3], z);
                    z = fmaf(wb.x, x[4], z);
                    h[q] = gelu_for_bf16(z, S.gtab);  // rounded to bf16 by pack_bf16
                }
                packed[e >> 1] = pack_bf16(h[0], h[1]);
            }
            *reinterpret_cast<uint4*>(S.A + tc_kmajor_offset(t, kb * 8)) =
                make_uint4(packed[0], packed[1], packed[2], packed[3]);
        }
        // the generic-proxy writes of A become visible to the tensor core
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
        tc_fence_before();
        __syncthreads();
        if (t == 0) {
            tc_fence_after();
#pragma unroll
            for (int ks = 0; ks < kMHid / 16; ++ks) {
                const uint64_t ad = tc_smem_desc(a_base + ks * 2 * kTcLbo, kTcLbo, kTcSbo);
                const uint64_t bd = tc_smem_desc(b_base + ks * 2 * kTcLbo, kTcLbo, kTcSbo);
                asm volatile(
                    "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
                    "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}\n" ::"r"(taddr),
                    "l"(ad), "l"(bd), "r"(idesc), "r"((uint32_t)ks)
                    : "memory");
            }
            asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(mbar)
                         : "memory");
        }
        if (!tc_wait(mbar, parity)) S.fail = 1;
        parity ^= 1u;
        tc_fence_after();
        __syncthreads();
        if (S.fail) break;
        // z2 = D + b2 of this thread's row, GELU, bf16, output layer
        float acc[kMOut][4];
#pragma unroll
        for (int o = 0; o < kMOut; ++o)
#pragma unroll
            for (int q = 0; q < 4; ++q) acc[o][q] = 0.f;
#pragma unroll 1
        for (int cb = 0; cb < kMHid / 16; ++cb) {
            float d[16];
            tc_ld16(taddr + ((uint32_t)(warp * 32) << 16) + (uint32_t)(cb * 16), d);
            asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
            for (int i = 0; i < 16; ++i) {
                const int q = (i & 7) >> 1;
                const float4 w = S.l3[cb * 16 + i];
                const float h2 = round_bf16(gelu_for_bf16(d[i] + w.x, S.gtab));
                acc[0][q] = fmaf(w.y, h2, acc[0][q]);
                acc[1][q] = fmaf(w.z, h2, acc[1][q]);
            }
        }
        tc_fence_before();  // this tile's TMEM reads come before the next tile's MMA
        float out[kMOut];
#pragma unroll
        for (int o = 0; o < kMOut; ++o) out[o] = ((acc[o][0] + acc[o][1]) + (acc[o][2] + acc[o][3])) + S.b3[o];
        if (!valid) continue;
        if (MODE == 0) {
            Y[s * kMOut] = out[0];
            Y[s * kMOut + 1] = out[1];
            continue;
        }
        const float dRf = A.scale_R * out[0], dVf = A.scale_V * out[1];
        if (dRf == 0.0f && dVf == 0.0f) continue;
        double Rp, Vp, Rl, Vl;
        int dec = -1;
        if (MODE == 1) {
            const double2 pl = ((const double2*)A.y)[s];
            Rp = pl.x;
            Vp = pl.y;
            Rl = pl.x + (double)dRf;
            Vl = pl.y + (double)dVf;
        } else {
            const float2 pl = ((const float2*)A.y)[s];
            const float R1 = pl.x + dRf, V1 = pl.y + dVf;
            Rp = pl.x;
            Vp = pl.y;
            Rl = (double)R1;
            Vl = (double)V1;
            // binary32 where it provably gives the FP64 decision
            dec = energy_check_f32(E32, pl.x, pl.y, R1, V1);
        }
        // the plain step judges: the correction may move the frozen-field
        // energy away from the plain step's by at most tol |H|
        const bool keep = dec >= 0 ? dec == 1 : frozen_keep_fp64(A, Rp, Vp, Rl, Vl);
        if (keep) {
            if (MODE == 1) ((double2*)A.y)[s] = make_double2(Rl, Vl);
            else ((float2*)A.y)[s] = make_float2((float)Rl, (float)Vl);
        } else {
            ++fallback;
        }
    }
    if (MODE != 0) {
#pragma unroll
        for (int d = 16; d >= 1; d >>= 1) fallback += __shfl_xor_sync(0xffffffffu, fallback, d);
        if ((t & 31) == 0 && fallback) atomicAdd(A.n_fallback, (unsigned long long)fallback);
    }
    if (t == 0 && S.fail) atomicExch(M.err, 1);
    tc_fence_before();
    __syncthreads();
    if (warp == 0) {
        tc_fence_after();
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(taddr), "r"(kTcCols) : "memory");
    }
}

// Blocks of k_mlp_tc resident on one SM, from its registers, its shared
// memory and its 64 tensor-memory columns (512 per SM).  The runtime's
// occupancy query answers 1 for this kernel, which would leave 7 of every 8
// warp slots it could use empty.
static int tc_blocks_per_sm(const void* fn, size_t dyn_smem) {
    cudaFuncAttributes fa;
    int dev = 0, smem_sm = 0, resv = 0, regs_sm = 0;
    if (cudaFuncGetAttributes(&fa, fn) != cudaSuccess || cudaGetDevice(&dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&smem_sm, cudaDevAttrMaxSharedMemoryPerMultiprocessor, dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&resv, cudaDevAttrReservedSharedMemoryPerBlock, dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&regs_sm, cudaDevAttrMaxRegistersPerMultiprocessor, dev) != cudaSuccess)
        return 1;
    const int regs_block = ((fa.numRegs + 7) / 8) * 8 * kTcThreads;  // allocated per warp in units of 8 per thread
    int k = 512 / kTcCols;
    k = std::min(k, 2048 / kTcThreads);
    if (regs_block > 0) k = std::min(k, regs_sm / regs_block);
    k = std::min(k, (int)((size_t)smem_sm / (fa.sharedSizeBytes + dyn_smem + (size_t)resv)));
    return k < 1 ? 1 : k;
}

// Launch of the tensor-core inference over n samples: as many blocks as are
// resident at once, no more blocks than tiles.
cudaError_t launch_mlp_tc(const MlpDev& D, const LearnedArgs& A, int mode, const float* X, float* Y, long long n,
                          int sm_count, cudaStream_t st) {
    if (n == 0) return cudaSuccess;
    const size_t smem = (mode == 2 && A.tab_f) ? sizeof(float) * 3 * (size_t)(A.n_cells + 1) : 0;
    void* fn = mode == 0 ? (void*)k_mlp_tc<0> : mode == 1 ? (void*)k_mlp_tc<1> : (void*)k_mlp_tc<2>;
    cudaError_t e = cudaFuncSetAttribute(fn, cudaFuncAttributePreferredSharedMemoryCarveout,
                                         (int)cudaSharedmemCarveoutMaxShared);
    if (e == cudaSuccess && smem > 48 * 1024)
        e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    const int per_sm = tc_blocks_per_sm(fn, smem);
    const long long tiles = (n + kTcThreads - 1) / kTcThreads;
    const long long cap = (long long)sm_count * per_sm;
    const int grid = (int)(tiles < cap ? tiles : cap);
    if (mode == 0) k_mlp_tc<0><<<grid, kTcThreads, smem, st>>>(D, A, X, Y, n);
    else if (mode == 1) k_mlp_tc<1><<<grid, kTcThreads, smem, st>>>(D, A, X, Y, n);
    else k_mlp_tc<2><<<grid, kTcThreads, smem, st>>>(D, A, X, Y, n);
    return cudaGetLastError();
}

// ------------------------------------------------------------ tensor-core training (tcgen05)
//
// The per-sample part of a training step: one sample per thread, 128 per
// block and tile.  Forward as in k_mlp_tc (MMA 1: z2 = bf16(h1) W2^T + b2),
// then dout = (out - y)/B, dz2 = (dout W3) gelu'(z2), and MMA 2 (same tensor
// memory, same A buffer): dh1 = bf16(dz2) W2 against W2^T staged as the B
// operand, dz1 = dh1 gelu'(z1) with z1 recomputed from x.  Every sample
// leaves its records (x, bf16(h1), bf16(h2), dout, dz2, dz1) for the
// weight-gradient kernel, every block its loss partial.

struct TcTrainSmem {
    alignas(1024) unsigned char A[kTcThreads * kMHid * 2];  // bf16(h1), then bf16(dz2): 128 x 64, K-major
    alignas(1024) unsigned char Bw[kMHid * kMHid * 2];      // W2: N = j, K = k
    alignas(1024) unsigned char Bt[kMHid * kMHid * 2];      // W2^T: N = k, K = j
    float4 l1[kMHid][2];
    float4 l3[kMHid];
    float b3[kMOut];
    float4 gtab[kGeluSeg + 1];
    unsigned long long mbar;
    unsigned int taddr;
    int fail;
    float loss[kTcThreads / 32];
};

// Thread 0: the four K = 16 MMAs of a K = 64 product into the accumulator at
// taddr (accumulating onto it when acc), committed to the mbarrier.
__device__ __forceinline__ void tc_issue_k64(uint32_t taddr, uint32_t a_base, uint32_t b_base, uint32_t idesc,
                                             bool acc, uint32_t mbar) {
    tc_fence_after();
#pragma unroll
    for (int ks = 0; ks < kMHid / 16; ++ks) {
        const uint64_t ad = tc_smem_desc(a_base + ks * 2 * kTcLbo, kTcLbo, kTcSbo);
        const uint64_t bd = tc_smem_desc(b_base + ks * 2 * kTcLbo, kTcLbo, kTcSbo);
        const uint32_t en = (acc || ks > 0) ? 1u : 0u;
        asm volatile(
            "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
            "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}\n" ::"r"(taddr),
            "l"(ad), "l"(bd), "r"(idesc), "r"(en)
            : "memory");
    }
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(mbar) : "memory");
}

// A 64 x 64 bf16 matrix (row-major, rows along N) as a K-major B operand.
__device__ __forceinline__ void tc_stage_b(unsigned char* dst, const __nv_bfloat16* __restrict__ src) {
    for (int i = threadIdx.x; i < kMHid * kMHid / 8; i += blockDim.x) {
        const int nrow = i >> 3, kb = i & 7;
        *reinterpret_cast<uint4*>(dst + tc_kmajor_offset(nrow, kb * 8)) =
            *reinterpret_cast<const uint4*>(src + nrow * kMHid + kb * 8);
    }
}

// Block-wide: MMA issued by thread 0 after the A writes of every thread,
// then every thread waits for it; false (and the block's fail flag) when
// the wait ran out of time.
__device__ __forceinline__ bool tc_block_mma(uint32_t taddr, uint32_t a_base, uint32_t b_base, uint32_t idesc, bool acc,
                                             uint32_t mbar, uint32_t& parity, int& fail) {
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    tc_fence_before();
    __syncthreads();
    if (threadIdx.x == 0) tc_issue_k64(taddr, a_base, b_base, idesc, acc, mbar);
    if (!tc_wait(mbar, parity)) fail = 1;
    parity ^= 1u;
    tc_fence_after();
    __syncthreads();
    return !fail;
}

__global__ void __launch_bounds__(kTcThreads) k_mlp_train_tc(MlpDev M, const float* __restrict__ X,
                                                             const float* __restrict__ Y, long long B, long long first,
                                                             long long mul, long long n_data, float invB) {
    __shared__ TcTrainSmem S;
    const int t = threadIdx.x, warp = t >> 5, lane = t & 31;
    tc_stage_b(S.Bw, M.W2b);
    tc_stage_b(S.Bt, M.W2Tb);
    if (t < kMHid) {
        const float* w1 = M.small + sW1 + t * kMIn;
        S.l1[t][0] = make_float4(w1[0], w1[1], w1[2], w1[3]);
        S.l1[t][1] = make_float4(w1[4], M.small[sb1 + t], 0.f, 0.f);
        S.l3[t] = make_float4(M.small[sb2 + t], M.small[sW3 + t], M.small[sW3 + kMHid + t], 0.f);
    }
    if (t < kMOut) S.b3[t] = M.small[sb3 + t];
    if (t <= kGeluSeg) S.gtab[t] = make_float4(c_gelu_tab[t][0], c_gelu_tab[t][1], c_gelu_tab[t][2], c_gelu_tab[t][3]);
    if (t == 0) {
        asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(&S.mbar)) : "memory");
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
        S.fail = 0;
    }
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(&S.taddr)),
                     "r"(kTcCols)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t taddr = S.taddr, trow = taddr + ((uint32_t)(warp * 32) << 16);
    const uint32_t idesc = tc_idesc_bf16_f32(kTcThreads, kMHid);
    const uint32_t a_base = smem_u32(S.A), mbar = smem_u32(&S.mbar);
    uint32_t parity = 0;
    float loss = 0.f;
    const long long tiles = (B + kTcThreads - 1) / kTcThreads;
    for (long long tile = blockIdx.x; tile < tiles; tile += gridDim.x) {
        const long long s = tile * kTcThreads + t;
        const bool valid = s < B;
        const long long idx = valid ? sample_index(s, first, mul, n_data) : 0;
        float x[kMIn];
#pragma unroll
        for (int i = 0; i < kMIn; ++i) x[i] = valid ? X[idx * kMIn + i] : 0.f;
        // layer 1 + GELU: the A operand and the h1 record
#pragma unroll 1
        for (int kb = 0; kb < kMHid / 8; ++kb) {
            unsigned int packed[4];
#pragma unroll
            for (int e = 0; e < 8; e += 2) {
                float h[2];
#pragma unroll
                for (int q = 0; q < 2; ++q) {
                    const int col = kb * 8 + e + q;
                    const float4 wa = S.l1[col][0], wb = S.l1[col][1];
                    float z = wb.y;
                    z = fmaf(wa.x, x[0], z);
                    z = fmaf(wa.y, x[1], z);
                    z = fmaf(wa.z, x[2], z);
                    z = fmaf(wa.w, x[3], z);
                    z = fmaf(wb.x, x[4], z);
                    h[q] = gelu_for_bf16(z, S.gtab);
                }
                packed[e >> 1] = pack_bf16(h[0], h[1]);
            }
            const uint4 v = make_uint4(packed[0], packed[1], packed[2], packed[3]);
            *reinterpret_cast<uint4*>(S.A + tc_kmajor_offset(t, kb * 8)) = v;
            if (valid) *reinterpret_cast<uint4*>(M.h1b + s * kMHid + kb * 8) = v;
        }
        if (!tc_block_mma(taddr, a_base, smem_u32(S.Bw), idesc, false, mbar, parity, S.fail)) break;
        // output layer (the order of k_mlp_tc) and the h2 record
        float acc[kMOut][4];
#pragma unroll
        for (int o = 0; o < kMOut; ++o)
#pragma unroll
            for (int q = 0; q < 4; ++q) acc[o][q] = 0.f;
#pragma unroll 1
        for (int cb = 0; cb < kMHid / 16; ++cb) {
            float d[16], h2[16];
            tc_ld16(trow + (uint32_t)(cb * 16), d);
            asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
            for (int i = 0; i < 16; ++i) {
                const int q = (i & 7) >> 1;
                const float4 w = S.l3[cb * 16 + i];
                h2[i] = round_bf16(gelu_for_bf16(d[i] + w.x, S.gtab));
                acc[0][q] = fmaf(w.y, h2[i], acc[0][q]);
                acc[1][q] = fmaf(w.z, h2[i], acc[1][q]);
            }
            if (valid) {
                uint4* dst = reinterpret_cast<uint4*>(M.h2b + s * kMHid + cb * 16);
                dst[0] = make_uint4(pack_bf16(h2[0], h2[1]), pack_bf16(h2[2], h2[3]), pack_bf16(h2[4], h2[5]),
                                    pack_bf16(h2[6], h2[7]));
                dst[1] = make_uint4(pack_bf16(h2[8], h2[9]), pack_bf16(h2[10], h2[11]), pack_bf16(h2[12], h2[13]),
                                    pack_bf16(h2[14], h2[15]));
            }
        }
        float dout[kMOut];
#pragma unroll
        for (int o = 0; o < kMOut; ++o) {
            const float out = ((acc[o][0] + acc[o][1]) + (acc[o][2] + acc[o][3])) + S.b3[o];
            const float d = valid ? out - Y[idx * kMOut + o] : 0.f;
            loss = fmaf(d, d, loss);
            dout[o] = d * invB;
        }
        if (valid) {
            M.dout[s * kMOut] = dout[0];
            M.dout[s * kMOut + 1] = dout[1];
#pragma unroll
            for (int i = 0; i < kMIn; ++i) M.xs[s * kMIn + i] = x[i];
        }
        // dz2 = (dout W3) gelu'(z2): the dz2 record and bf16(dz2) as the next A operand
#pragma unroll 1
        for (int cb = 0; cb < kMHid / 16; ++cb) {
            float d[16];
            tc_ld16(trow + (uint32_t)(cb * 16), d);
            asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
            for (int i = 0; i < 16; ++i) {
                const float4 w = S.l3[cb * 16 + i];
                const float dh = fmaf(w.z, dout[1], w.y * dout[0]);
                d[i] = dh * gelu_d(d[i] + w.x);
            }
            if (valid) {
                float4* dst = reinterpret_cast<float4*>(M.dz2 + s * kMHid + cb * 16);
#pragma unroll
                for (int v = 0; v < 4; ++v) dst[v] = make_float4(d[4 * v], d[4 * v + 1], d[4 * v + 2], d[4 * v + 3]);
            }
#pragma unroll
            for (int hf = 0; hf < 2; ++hf)
                *reinterpret_cast<uint4*>(S.A + tc_kmajor_offset(t, cb * 16 + hf * 8)) =
                    make_uint4(pack_bf16(d[8 * hf], d[8 * hf + 1]), pack_bf16(d[8 * hf + 2], d[8 * hf + 3]),
                               pack_bf16(d[8 * hf + 4], d[8 * hf + 5]), pack_bf16(d[8 * hf + 6], d[8 * hf + 7]));
        }
        if (!tc_block_mma(taddr, a_base, smem_u32(S.Bt), idesc, false, mbar, parity, S.fail)) break;
        // dz1 = dh1 gelu'(z1), z1 recomputed as in layer 1
#pragma unroll 1
        for (int cb = 0; cb < kMHid / 16; ++cb) {
            float d[16];
            tc_ld16(trow + (uint32_t)(cb * 16), d);
            asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
            for (int i = 0; i < 16; ++i) {
                const float4 wa = S.l1[cb * 16 + i][0], wb = S.l1[cb * 16 + i][1];
                float z = wb.y;
                z = fmaf(wa.x, x[0], z);
                z = fmaf(wa.y, x[1], z);
                z = fmaf(wa.z, x[2], z);
                z = fmaf(wa.w, x[3], z);
                z = fmaf(wb.x, x[4], z);
                d[i] = d[i] * gelu_d(z);
            }
            if (valid) {
                float4* dst = reinterpret_cast<float4*>(M.dz1 + s * kMHid + cb * 16);
#pragma unroll
                for (int v = 0; v < 4; ++v) dst[v] = make_float4(d[4 * v], d[4 * v + 1], d[4 * v + 2], d[4 * v + 3]);
            }
        }
    }
    // loss partial of this block (fixed reduction order)
#pragma unroll
    for (int dd = 16; dd >= 1; dd >>= 1) loss += __shfl_xor_sync(0xffffffffu, loss, dd);
    if (lane == 0) S.loss[warp] = loss;
    if (t == 0 && S.fail) atomicExch(M.err, 1);
    tc_fence_before();
    __syncthreads();
    if (t == 0) {
        float sum = 0.f;
        for (int i = 0; i < kTcThreads / 32; ++i) sum += S.loss[i];
        M.loss_part[blockIdx.x] = 0.5f * sum * invB;
    }
    if (warp == 0) {
        tc_fence_after();
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(taddr), "r"(kTcCols) : "memory");
    }
}

// Weight gradients of a batch: block b sums samples [b chunk, (b+1) chunk)
// into grad_part[b].  dW2[j][k] = sum_s bf16(dz2[s][j]) h1b[s][k] on the
// tensor cores with the samples as the reduction dimension: per staged tile
// of 64 samples, A = bf16(dz2)^T (rows 0..63 of a 128-row tile; rows 64..127
// stay zero and their accumulator lanes are not read), B = h1b^T (N = k),
// accumulated in tensor memory over the block's tiles.  The small gradients
// (W1, b1, b2, W3, b3) on the CUDA cores, one column per thread.
struct TcGradSmem {
    alignas(1024) unsigned char A[kTcThreads * kWgTile * 2];  // bf16(dz2)^T, K-major (K = samples)
    alignas(1024) unsigned char Bh[kMHid * kWgTile * 2];      // h1b^T, K-major
    unsigned long long mbar;
    unsigned int taddr;
    int fail;
};

__global__ void __launch_bounds__(kTcThreads) k_mlp_wgrad_tc(MlpDev M, long long B, long long chunk) {
    __shared__ TcGradSmem S;
    const int t = threadIdx.x, warp = t >> 5;
    for (int i = t; i < (int)(sizeof(S.A) / 16); i += kTcThreads) reinterpret_cast<uint4*>(S.A)[i] = make_uint4(0, 0, 0, 0);
    if (t == 0) {
        asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(&S.mbar)) : "memory");
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
        S.fail = 0;
    }
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(&S.taddr)),
                     "r"(kTcCols)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t taddr = S.taddr, idesc = tc_idesc_bf16_f32(kTcThreads, kMHid);
    const uint32_t a_base = smem_u32(S.A), b_base = smem_u32(S.Bh), mbar = smem_u32(&S.mbar);
    const long long s_begin = (long long)blockIdx.x * chunk;
    const long long s_end = s_begin + chunk < B ? s_begin + chunk : B;
    uint32_t parity = 0;
    bool any = false;
    for (long long s0 = s_begin; s0 < s_end; s0 += kWgTile) {
        // thread t stages sample s = t / 2, units [32 (t % 2), 32 (t % 2) + 32)
        const int sl = t >> 1, j0 = (t & 1) * 32;
        const long long ss = s0 + sl;
        const bool ok = ss < s_end;
#pragma unroll 4
        for (int jj = 0; jj < 32; ++jj) {
            const int j = j0 + jj;
            const __nv_bfloat16 a = __float2bfloat16_rn(ok ? M.dz2[ss * kMHid + j] : 0.f);
            const __nv_bfloat16 b = ok ? M.h1b[ss * kMHid + j] : __float2bfloat16_rn(0.f);
            *reinterpret_cast<__nv_bfloat16*>(S.A + tc_kmajor_offset(j, sl)) = a;
            *reinterpret_cast<__nv_bfloat16*>(S.Bh + tc_kmajor_offset(j, sl)) = b;
        }
        if (!tc_block_mma(taddr, a_base, b_base, idesc, any, mbar, parity, S.fail)) break;
        any = true;
    }
    float* part = M.grad_part + (size_t)blockIdx.x * kMParams;
    if (warp < 2) {  // accumulator lanes 0..63: rows j of dW2
        const int j = t;
#pragma unroll 1
        for (int cb = 0; cb < kMHid / 16; ++cb) {
            float d[16];
            tc_ld16(taddr + ((uint32_t)(warp * 32) << 16) + (uint32_t)(cb * 16), d);
            asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
            for (int i = 0; i < 16; ++i) part[oW2 + j * kMHid + cb * 16 + i] = any && !S.fail ? d[i] : 0.f;
        }
    }
    if (t < kMHid) {
        const int j = t;
        float gw[kMIn] = {0.f, 0.f, 0.f, 0.f, 0.f}, gb1 = 0.f, gb2 = 0.f;
        for (long long s = s_begin; s < s_end; ++s) {
            const float d1 = M.dz1[s * kMHid + j];
#pragma unroll
            for (int i = 0; i < kMIn; ++i) gw[i] = fmaf(d1, M.xs[s * kMIn + i], gw[i]);
            gb1 += d1;
            gb2 += M.dz2[s * kMHid + j];
        }
#pragma unroll
        for (int i = 0; i < kMIn; ++i) part[oW1 + j * kMIn + i] = gw[i];
        part[ob1 + j] = gb1;
        part[ob2 + j] = gb2;
    } else {
        const int j = t - kMHid;
        float g0 = 0.f, g1 = 0.f, d0 = 0.f, d1 = 0.f;
        for (long long s = s_begin; s < s_end; ++s) {
            const float h = __bfloat162float(M.h2b[s * kMHid + j]);
            const float o0 = M.dout[s * kMOut], o1 = M.dout[s * kMOut + 1];
            g0 = fmaf(o0, h, g0);
            g1 = fmaf(o1, h, g1);
            d0 += o0;
            d1 += o1;
        }
        part[oW3 + j] = g0;
        part[oW3 + kMHid + j] = g1;
        if (j == 0) {
            part[ob3] = d0;
            part[ob3 + 1] = d1;
        }
    }
    if (t == 0 && S.fail) atomicExch(M.err, 1);
    tc_fence_before();
    __syncthreads();
    if (warp == 0) {
        tc_fence_after();
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(taddr), "r"(kTcCols) : "memory");
    }
}

__global__ void k_psi_nodes(const double* __restrict__ E, int n_cells, double hr, double* __restrict__ psi,
                            float* __restrict__ tab_f) {
    if (blockIdx.x == 0 && threadIdx.x == 0) {
        const int c = n_cells / 2;
        psi[c] = 0.0;
        for (int j = c + 1; j <= n_cells; ++j) psi[j] = psi[j - 1] + (0.5 * hr) * (E[j - 1] + E[j]);
        for (int j = c - 1; j >= 0; --j) psi[j] = psi[j + 1] - (0.5 * hr) * (E[j] + E[j + 1]);
    }
    if (!tab_f) return;
    __syncthreads();
    // binary32 copies for the energy check of the FP32 form
    const int Np1 = n_cells + 1;
    const double inv_hr = 1.0 / hr;
    for (int j = threadIdx.x; j < Np1; j += blockDim.x) {
        tab_f[j] = (float)E[j];
        tab_f[Np1 + j] = j < n_cells ? (float)((E[j + 1] - E[j]) * inv_hr) : 0.0f;
        tab_f[2 * Np1 + j] = (float)psi[j];
    }
}

cudaError_t launch_psi_nodes(const double* E, int n_cells, double hr, double* psi, cudaStream_t st,
                             long long* launches, float* tab_f) {
    k_psi_nodes<<<1, 256, 0, st>>>(E, n_cells, hr, psi, tab_f);
    if (launches) ++*launches;
    return cudaGetLastError();
}

// psi at n positions: the same psi_at the learned step's FP64 energy check uses.
__global__ void k_psi_eval(LearnedArgs A, const double* __restrict__ R, double* __restrict__ out) {
    const long long stride = (long long)gridDim.x * blockDim.x;
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < A.n; i += stride) out[i] = psi_at(A, R[i]);
}

cudaError_t launch_psi_eval(const LearnedArgs& A, const double* R, double* out, int sm_count, cudaStream_t st) {
    if (A.n == 0) return cudaSuccess;
    const long long want = (A.n + 255) / 256;
    const int grid = (int)(want < (long long)sm_count * 4 ? want : (long long)sm_count * 4);
    k_psi_eval<<<grid, 256, 0, st>>>(A, R, out);
    return cudaGetLastError();
}

}  // namespace pic

// ------------------------------------------------------------ C ABI

struct pic_mlp {
    pic::MlpDev D;
    long long max_batch = 0;
    cudaStream_t st = nullptr;
    int sm_count = 0;
    long long t = 0;  // Adam steps taken
    std::vector<void*> allocs;
    float* loss_host = nullptr;  // pinned
    int train_per_sm = 1;        // resident blocks of k_mlp_train_tc per SM
};

namespace {

int mlp_map(cudaError_t e) {
    if (e == cudaSuccess) return PIC_OK;
    if (e == cudaErrorMemoryAllocation) return PIC_ERR_NO_MEMORY;
    return PIC_ERR_CUDA;
}

template <typename T>
cudaError_t mlp_alloc(pic_mlp* m, T** p, size_t count) {
    void* q = nullptr;
    cudaError_t e = cudaMalloc(&q, sizeof(T) * (count ? count : 1));
    if (e == cudaSuccess) m->allocs.push_back(q);
    *p = (T*)q;
    return e;
}

void mlp_free(pic_mlp* m) {
    for (void* p : m->allocs) cudaFree(p);
    m->allocs.clear();
    if (m->loss_host) cudaFreeHost(m->loss_host);
    m->loss_host = nullptr;
}

// Forward + backward + weight gradients + reduction (+ Adam when apply).
cudaError_t mlp_step(pic_mlp* m, long long B, const float* X, const float* Y, long long first, long long mul,
                     long long n_data, int apply, const pic_adam_t* opt) {
    pic::MlpDev& D = m->D;
    const long long tiles = (B + pic::kTcThreads - 1) / pic::kTcThreads;
    const long long cap = (long long)m->sm_count * m->train_per_sm;
    const int gf = (int)(tiles < cap ? tiles : cap);
    pic::k_mlp_train_tc<<<gf, pic::kTcThreads, 0, m->st>>>(D, X, Y, B, first, mul, n_data, 1.0f / (float)B);
    long long nwg = (B + pic::kWgTile - 1) / pic::kWgTile;
    if (nwg > pic::kWgMaxBlocks) nwg = pic::kWgMaxBlocks;
    long long chunk = (B + nwg - 1) / nwg;
    chunk = (chunk + pic::kWgTile - 1) / pic::kWgTile * pic::kWgTile;
    nwg = (B + chunk - 1) / chunk;
    pic::k_mlp_wgrad_tc<<<(int)nwg, pic::kTcThreads, 0, m->st>>>(D, B, chunk);
    pic::AdamArgs A;
    std::memset(&A, 0, sizeof(A));
    if (apply) {
        m->t += 1;
        A.lr = opt->lr;
        A.beta1 = opt->beta1;
        A.beta2 = opt->beta2;
        A.eps = opt->eps;
        A.c1 = (float)(1.0 / (1.0 - std::pow((double)opt->beta1, (double)m->t)));
        A.c2 = (float)(1.0 / (1.0 - std::pow((double)opt->beta2, (double)m->t)));
        A.apply = 1;
    }
    const int gp = (pic::kMParams + 255) / 256;
    pic::k_mlp_update<<<gp, 256, 0, m->st>>>(D, (int)nwg, gf, A);
    if (apply) pic::k_mlp_refresh<<<gp, 256, 0, m->st>>>(D);
    return cudaGetLastError();
}

long long gcd_ll(long long a, long long b) {
    while (b) {
        const long long r = a % b;
        a = b;
        b = r;
    }
    return a;
}

}  // namespace

namespace pic {
cudaError_t launch_learned_apply(const pic_mlp* m, const LearnedArgs& A, int sm_count, cudaStream_t st,
                                 long long* launches) {
    if (A.n == 0) return cudaSuccess;
    const cudaError_t e = launch_mlp_tc(m->D, A, A.prec == 0 ? 1 : 2, nullptr, nullptr, A.n, sm_count, st);
    if (launches) ++*launches;
    return e;
}

// PIC_ERR_TIMEOUT (and the flag cleared) when a tensor-core wait of the
// inference kernel ran out of time since the last call; synchronises st.
int mlp_take_error(const pic_mlp* m, cudaStream_t st) {
    int err = 0;
    cudaError_t e = cudaMemcpyAsync(&err, m->D.err, sizeof(int), cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) return e == cudaErrorMemoryAllocation ? PIC_ERR_NO_MEMORY : PIC_ERR_CUDA;
    if (!err) return PIC_OK;
    e = cudaMemsetAsync(m->D.err, 0, sizeof(int), st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    return e == cudaSuccess ? PIC_ERR_TIMEOUT : PIC_ERR_CUDA;
}
}  // namespace pic

extern "C" {

int pic_mlp_num_params(void) { return pic::kMParams; }

int pic_mlp_create(int64_t max_batch, void* stream, pic_mlp** out) {
    if (!out || max_batch < 1 || max_batch > (1ll << 26)) return PIC_ERR_INVALID_ARG;
    *out = nullptr;
    int dev = 0, sms = 0, count = 0;
    if (cudaGetDeviceCount(&count) != cudaSuccess || count == 0) return PIC_ERR_CUDA;
    if (cudaGetDevice(&dev) != cudaSuccess) return PIC_ERR_CUDA;
    if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) return PIC_ERR_CUDA;
    pic_mlp* m = new (std::nothrow) pic_mlp();
    if (!m) return PIC_ERR_NO_MEMORY;
    m->max_batch = max_batch;
    m->st = (cudaStream_t)stream;
    m->sm_count = sms;
    pic::MlpDev& D = m->D;
    std::memset(&D, 0, sizeof(D));
    const size_t B = (size_t)max_batch;
    cudaError_t e = cudaSuccess;
    if (e == cudaSuccess) e = mlp_alloc(m, &D.master, pic::kMParams);
    if (e == cudaSuccess) e = mlp_alloc(m, &D.m, pic::kMParams);
    if (e == cudaSuccess) e = mlp_alloc(m, &D.v, pic::kMParams);
    if (e == cudaSuccess) e = mlp_alloc(m, &D.W2b, pic::kMHid * pic::kMHid);
    if (e == cudaSuccess) e = mlp_alloc(m, &D.W2Tb, pic::kMHid * pic::kMHid);
    if (e == cudaSuccess) e = mlp_alloc(m, &D.small, pic::kMSmall);
    if (e == cudaSuccess) e = mlp_alloc(m, &D.xs, B * pic::kMIn);
    if (e == cudaSuccess) e = mlp_alloc(m, &D.dz1, B * pic::kMHid);
    if (e == cudaSuccess) e = mlp_alloc(m, &D.dz2, B * pic::kMHid);
    if (e == cudaSuccess) e = mlp_alloc(m, &D.h1b, B * pic::kMHid);
    if (e == cudaSuccess) e = mlp_alloc(m, &D.h2b, B * pic::kMHid);
    if (e == cudaSuccess) e = mlp_alloc(m, &D.dout, B * pic::kMOut);
    if (e == cudaSuccess) e = mlp_alloc(m, &D.loss_part, (size_t)sms * 8);
    if (e == cudaSuccess) e = mlp_alloc(m, &D.grad_part, (size_t)pic::kWgMaxBlocks * pic::kMParams);
    if (e == cudaSuccess) e = mlp_alloc(m, &D.grad, pic::kMParams);
    if (e == cudaSuccess) e = mlp_alloc(m, &D.loss, 1);
    if (e == cudaSuccess) e = mlp_alloc(m, &D.err, 1);
    if (e == cudaSuccess) e = cudaMemsetAsync(D.err, 0, sizeof(int), m->st);
    if (e == cudaSuccess) e = cudaMallocHost(&m->loss_host, sizeof(float));
    if (e == cudaSuccess) e = cudaMemsetAsync(D.master, 0, sizeof(float) * pic::kMParams, m->st);
    if (e == cudaSuccess) e = cudaMemsetAsync(D.m, 0, sizeof(float) * pic::kMParams, m->st);
    if (e == cudaSuccess) e = cudaMemsetAsync(D.v, 0, sizeof(float) * pic::kMParams, m->st);
    if (e == cudaSuccess) {
        pic::k_mlp_refresh<<<(pic::kMParams + 255) / 256, 256, 0, m->st>>>(D);
        e = cudaGetLastError();
    }
    for (const void* fn : {(const void*)pic::k_mlp_train_tc, (const void*)pic::k_mlp_wgrad_tc})
        if (e == cudaSuccess)
            e = cudaFuncSetAttribute(fn, cudaFuncAttributePreferredSharedMemoryCarveout,
                                     (int)cudaSharedmemCarveoutMaxShared);
    if (e == cudaSuccess) m->train_per_sm = pic::tc_blocks_per_sm((const void*)pic::k_mlp_train_tc, 0);
    if (e == cudaSuccess) e = cudaStreamSynchronize(m->st);
    if (e != cudaSuccess) {
        mlp_free(m);
        delete m;
        return mlp_map(e);
    }
    *out = m;
    return PIC_OK;
}

int pic_mlp_set_weights(pic_mlp* m, const float* w, int ptr_kind) {
    if (!m || !w || (ptr_kind != PIC_PTR_HOST && ptr_kind != PIC_PTR_DEVICE)) return PIC_ERR_INVALID_ARG;
    cudaError_t e = cudaMemcpyAsync(m->D.master, w, sizeof(float) * pic::kMParams,
                                    ptr_kind == PIC_PTR_HOST ? cudaMemcpyHostToDevice : cudaMemcpyDeviceToDevice, m->st);
    if (e == cudaSuccess) e = cudaMemsetAsync(m->D.m, 0, sizeof(float) * pic::kMParams, m->st);
    if (e == cudaSuccess) e = cudaMemsetAsync(m->D.v, 0, sizeof(float) * pic::kMParams, m->st);
    if (e == cudaSuccess) {
        pic::k_mlp_refresh<<<(pic::kMParams + 255) / 256, 256, 0, m->st>>>(m->D);
        e = cudaGetLastError();
    }
    if (e == cudaSuccess) e = cudaStreamSynchronize(m->st);
    m->t = 0;
    return mlp_map(e);
}

int pic_mlp_get_weights(pic_mlp* m, float* w, int ptr_kind) {
    if (!m || !w || (ptr_kind != PIC_PTR_HOST && ptr_kind != PIC_PTR_DEVICE)) return PIC_ERR_INVALID_ARG;
    cudaError_t e = cudaMemcpyAsync(w, m->D.master, sizeof(float) * pic::kMParams,
                                    ptr_kind == PIC_PTR_HOST ? cudaMemcpyDeviceToHost : cudaMemcpyDeviceToDevice, m->st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(m->st);
    return mlp_map(e);
}

int pic_mlp_forward(pic_mlp* m, int64_t n, const float* X_dev, float* Y_dev) {
    if (!m || n < 0 || (n > 0 && (!X_dev || !Y_dev))) return PIC_ERR_INVALID_ARG;
    if (n == 0) return PIC_OK;
    pic::LearnedArgs A;
    std::memset(&A, 0, sizeof(A));
    const cudaError_t e = pic::launch_mlp_tc(m->D, A, 0, X_dev, Y_dev, n, m->sm_count, m->st);
    if (e != cudaSuccess) return mlp_map(e);
    return pic::mlp_take_error(m, m->st);
}

int pic_mlp_gradients(pic_mlp* m, int64_t n, const float* X_dev, const float* T_dev, float* grad, float* loss,
                      int ptr_kind) {
    if (!m || n < 1 || n > m->max_batch || !X_dev || !T_dev || !grad || !loss) return PIC_ERR_INVALID_ARG;
    if (ptr_kind != PIC_PTR_HOST && ptr_kind != PIC_PTR_DEVICE) return PIC_ERR_INVALID_ARG;
    const cudaMemcpyKind k = ptr_kind == PIC_PTR_HOST ? cudaMemcpyDeviceToHost : cudaMemcpyDeviceToDevice;
    cudaError_t e = mlp_step(m, n, X_dev, T_dev, 0, 1, n, 0, nullptr);
    if (e == cudaSuccess) e = cudaMemcpyAsync(grad, m->D.grad, sizeof(float) * pic::kMParams, k, m->st);
    if (e == cudaSuccess) e = cudaMemcpyAsync(loss, m->D.loss, sizeof(float), k, m->st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(m->st);
    if (e != cudaSuccess) return mlp_map(e);
    return pic::mlp_take_error(m, m->st);
}

int pic_mlp_train(pic_mlp* m, int64_t n_data, const float* X_dev, const float* T_dev, int64_t batch, int64_t steps,
                  const pic_adam_t* opt, uint64_t seed, float* loss_hist) {
    if (!m || !opt || n_data < 1 || batch < 1 || batch > m->max_batch || batch > n_data || steps < 0 || !X_dev ||
        !T_dev)
        return PIC_ERR_INVALID_ARG;
    if (!(opt->lr > 0.f) || !(opt->beta1 >= 0.f && opt->beta1 < 1.f) || !(opt->beta2 >= 0.f && opt->beta2 < 1.f) ||
        !(opt->eps > 0.f))
        return PIC_ERR_INVALID_ARG;
    // a multiplier coprime with n_data near n_data times the golden ratio
    // (shifted by the seed): consecutive batch rows land far apart in the
    // data set, and the batches walk a fixed permutation of it
    long long mul = (long long)((double)n_data * 0.6180339887498949) + (long long)(seed % 1024ull);
    if (mul < 1) mul = 1;
    while (gcd_ll(mul, n_data) != 1) ++mul;
    cudaError_t e = cudaSuccess;
    for (long long s = 0; s < steps && e == cudaSuccess; ++s) {
        const long long first = (s * batch) % n_data;
        e = mlp_step(m, batch, X_dev, T_dev, first, mul, n_data, 1, opt);
        if (e == cudaSuccess && loss_hist) {
            e = cudaMemcpyAsync(m->loss_host, m->D.loss, sizeof(float), cudaMemcpyDeviceToHost, m->st);
            if (e == cudaSuccess) e = cudaStreamSynchronize(m->st);
            if (e == cudaSuccess) loss_hist[s] = *m->loss_host;
        }
    }
    if (e == cudaSuccess) e = cudaStreamSynchronize(m->st);
    if (e != cudaSuccess) return mlp_map(e);
    return pic::mlp_take_error(m, m->st);
}

int pic_mlp_apply_gradient(pic_mlp* m, const float* grad, int ptr_kind, const pic_adam_t* opt) {
    if (!m || !grad || !opt || (ptr_kind != PIC_PTR_HOST && ptr_kind != PIC_PTR_DEVICE)) return PIC_ERR_INVALID_ARG;
    if (!(opt->lr > 0.f) || !(opt->beta1 >= 0.f && opt->beta1 < 1.f) || !(opt->beta2 >= 0.f && opt->beta2 < 1.f) ||
        !(opt->eps > 0.f))
        return PIC_ERR_INVALID_ARG;
    // the caller's gradient as the one partial the update kernel sums
    cudaError_t e = cudaMemcpyAsync(m->D.grad_part, grad, sizeof(float) * pic::kMParams,
                                    ptr_kind == PIC_PTR_HOST ? cudaMemcpyHostToDevice : cudaMemcpyDeviceToDevice, m->st);
    if (e == cudaSuccess) {
        pic::AdamArgs A;
        std::memset(&A, 0, sizeof(A));
        m->t += 1;
        A.lr = opt->lr;
        A.beta1 = opt->beta1;
        A.beta2 = opt->beta2;
        A.eps = opt->eps;
        A.c1 = (float)(1.0 / (1.0 - std::pow((double)opt->beta1, (double)m->t)));
        A.c2 = (float)(1.0 / (1.0 - std::pow((double)opt->beta2, (double)m->t)));
        A.apply = 1;
        const int gp = (pic::kMParams + 255) / 256;
        pic::k_mlp_update<<<gp, 256, 0, m->st>>>(m->D, 1, 0, A);
        pic::k_mlp_refresh<<<gp, 256, 0, m->st>>>(m->D);
        e = cudaGetLastError();
    }
    if (e == cudaSuccess) e = cudaStreamSynchronize(m->st);
    return mlp_map(e);
}

void pic_mlp_destroy(pic_mlp* m) {
    if (!m) return;
    cudaStreamSynchronize(m->st);
    mlp_free(m);
    delete m;
}

}  // extern "C"

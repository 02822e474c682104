// tc_desc.cuh -- descriptors of the 5th-generation tensor-core instruction
// (tcgen05.mma, sm_100 family) used by the network of the learned stepper,
// written out field by field from the PTX ISA's tables so that a host test
// (tests/test_tc_desc.py) checks every bit before a kernel uses them.
//
// Shared-memory matrix descriptor (64 bits):
//   [0,14)  start address >> 4          [16,30) leading-dimension byte offset >> 4
//   [32,46) stride-dimension byte offset >> 4
//   [46,48) descriptor version, 1 for tcgen05     [49,52) base offset (0)
//   [52]    leading-dimension offset mode (0: relative)
//   [61,64) swizzling mode (0: none)
// With no swizzling a K-major operand is made of 8 x 16-byte core matrices
// (8 rows of 8 bf16 along K); the leading-dimension offset is the distance
// between core matrices adjacent along K, the stride-dimension offset the
// distance between groups of 8 rows along M (or N).
//
// Instruction descriptor of .kind::f16 (32 bits):
//   [0,2) sparsity selector  [2] sparse  [3] saturate  [4,6) D format (1: f32)
//   [7,10) A format (1: bf16)  [10,13) B format (1: bf16)  [13] negate A
//   [14] negate B  [15] A major (0: K)  [16] B major (0: K)  [17,23) N >> 3
//   [24,29) M >> 4  [30,32) maximum shift (0)
#pragma once

#include <stdint.h>

#if defined(__CUDACC__)
#define PIC_TC_HD __host__ __device__ __forceinline__
#else
#define PIC_TC_HD inline
#endif

namespace pic {

PIC_TC_HD uint64_t tc_smem_desc(uint32_t smem_addr, uint32_t lbo_bytes, uint32_t sbo_bytes) {
    return (uint64_t)((smem_addr >> 4) & 0x3FFFu) | ((uint64_t)((lbo_bytes >> 4) & 0x3FFFu) << 16) |
           ((uint64_t)((sbo_bytes >> 4) & 0x3FFFu) << 32) | (1ull << 46);
}

PIC_TC_HD uint32_t tc_idesc_bf16_f32(uint32_t M, uint32_t N) {
    return (1u << 4)             // D: f32
           | (1u << 7)           // A: bf16
           | (1u << 10)          // B: bf16
           | ((N >> 3) << 17)    // N / 8
           | ((M >> 4) << 24);   // M / 16
}

// Byte offset of element (row, k) of a K-major bf16 operand with K = 64 in
// the no-swizzle core-matrix layout used here: core matrices adjacent along
// K are 128 B apart (LBO), groups of 8 rows 1024 B apart (SBO).
constexpr uint32_t kTcLbo = 128, kTcSbo = 1024;
PIC_TC_HD uint32_t tc_kmajor_offset(uint32_t row, uint32_t k) {
    return (row >> 3) * kTcSbo + (k >> 3) * kTcLbo + (row & 7u) * 16u + (k & 7u) * 2u;
}

}  // namespace pic

// Host build of the tensor-core descriptor helpers (csrc/tc_desc.cuh): prints
// the values the kernels use, for tests/test_tc_desc.py to decode.
#include <stdio.h>

#include "tc_desc.cuh"

int main() {
    using namespace pic;
    // instruction descriptors: M N value
    const unsigned shapes[][2] = {{128, 64}, {128, 256}, {64, 64}, {128, 8}, {64, 128}};
    for (const auto& s : shapes) printf("idesc %u %u %u\n", s[0], s[1], tc_idesc_bf16_f32(s[0], s[1]));
    // shared-memory descriptors: address lbo sbo value
    const unsigned addrs[] = {0u, 1024u, 1024u + 256u, 0x30000u, 0x3FFF0u};
    for (unsigned a : addrs)
        printf("sdesc %u %u %u %llu\n", a, kTcLbo, kTcSbo, (unsigned long long)tc_smem_desc(a, kTcLbo, kTcSbo));
    // operand layout: row k offset for a 128 x 64 tile
    for (unsigned r = 0; r < 128; ++r)
        for (unsigned k = 0; k < 64; ++k) printf("off %u %u %u\n", r, k, tc_kmajor_offset(r, k));
    return 0;
}

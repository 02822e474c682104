// Runs the binary32 energy check of the learned stepper
// (paper_1404_1160_gb300/csrc/energy_check.cuh) compiled for the host on
// the cases of an input file and writes its decisions (1 keep, 0 plain,
// -1 not decided) as int8, for tests/test_energy_check.py to compare with
// the oracle's FP64 rule.
//
// input (little-endian): int32 field, n_cells, n_cases; float32 eps, tol,
// r_min, hr, inv_hr; float32 E[n_cells+1], slope[n_cells+1], psi[n_cells+1];
// float32 (R0, V0, R1, V1) x n_cases.
#include <cstdint>
#include <cstdio>
#include <vector>

#include "energy_check.cuh"

int main(int argc, char** argv) {
    if (argc < 3) return 2;
    FILE* f = std::fopen(argv[1], "rb");
    if (!f) return 2;
    int32_t hdr[3];
    float c[5];
    if (std::fread(hdr, 4, 3, f) != 3 || std::fread(c, 4, 5, f) != 5) return 2;
    const int Np1 = hdr[1] + 1;
    std::vector<float> tab(3 * (size_t)Np1), y(4 * (size_t)hdr[2]);
    if (std::fread(tab.data(), 4, tab.size(), f) != tab.size() || std::fread(y.data(), 4, y.size(), f) != y.size())
        return 2;
    std::fclose(f);
    pic::EnergyF32 C;
    C.field = hdr[0];
    C.n_cells = hdr[1];
    C.eps = c[0];
    C.tol = c[1];
    C.r_min = c[2];
    C.hr = c[3];
    C.inv_hr = c[4];
    C.E = tab.data();
    C.slope = tab.data() + Np1;
    C.psi = tab.data() + 2 * Np1;
    std::vector<int8_t> out(hdr[2]);
    for (int i = 0; i < hdr[2]; ++i)
        out[i] = (int8_t)pic::energy_check_f32(C, y[4 * i], y[4 * i + 1], y[4 * i + 2], y[4 * i + 3]);
    FILE* g = std::fopen(argv[2], "wb");
    if (!g) return 2;
    std::fwrite(out.data(), 1, out.size(), g);
    std::fclose(g);
    return 0;
}

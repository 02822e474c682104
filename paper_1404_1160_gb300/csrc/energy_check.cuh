// energy_check.cuh -- the learned stepper's frozen-field energy check,
// decided in binary32 where binary32 is provably enough.
//
// The check (pic_step_learned, step 4) keeps the corrected state y1 of a
// particle when |H(y1) - H(y0)| <= tol |H(y0)|, with y0 the plain step's
// state and H(R, V) = (R^2 + V^2)/2 - eps psi(R) the frozen-field energy
// (psi' = E, psi(0) = 0).  The FP64 evaluation of the two energies is the
// definition; it costs ~20 FP64 instructions per particle, on the pipe that
// runs 64 times slower than binary32 on GB300.  Here the same decision is
// taken from binary32 arithmetic without cancellation:
//
//   dH = dR Rm + dV Vm - eps dpsi,   dR = R1 - R0, Rm = (R0 + R1)/2 (same for V),
//
// with dpsi = psi(R1) - psi(R0) in closed form: for the Poisson field, when
// R0 and R1 lie in one mesh cell where the gathered E is linear, the integral
// of E over [R0, R1] is dR E(Rm) exactly; for the Duffing field (psi =
// -R^4/4), dpsi = -dR Rm (R0^2 + R1^2)/2; no field: 0.  The threshold tol
// |H(y0)| needs H(y0) only to ~1e-6 relative.  A rounding-error bound of
// both sides (16 units in the last place of every term, several times the
// worst case of the few operations involved) decides: when the binary32
// margin |dH| - tol |H(y0)| is farther from 0 than twice that bound, the
// FP64 decision is the same; otherwise (and for particles that cross a cell
// boundary, lie near one, or are off the mesh) the caller evaluates the FP64
// energies.  Compiled for the host as well: tests/test_energy_check.py
// compares every decision taken here with the FP64 rule of the oracle.
#pragma once

#include <math.h>

#include "intfp.cuh"

namespace pic {

// Binary32 copies of the frozen field (Poisson): per node j, E_j, the
// slope (E_{j+1} - E_j)/h_r and psi_j; the mesh constants rounded once.
struct EnergyF32 {
    int field;              // PIC_FIELD_* (0 Poisson, 1 Duffing, 2 none)
    float eps, tol;
    int n_cells;
    float r_min, hr, inv_hr;
    const float* E;         // n_cells + 1
    const float* slope;     // n_cells
    const float* psi;       // n_cells + 1
};

// 1: keep the corrected state, 0: keep the plain state, -1: not decided
// here (the caller evaluates the FP64 energies).
PIC_HD int energy_check_f32(const EnergyF32& C, float R0, float V0, float R1, float V1) {
    if (C.field < 0 || C.field > 2) return -1;
    const float u16 = 16.0f * 5.9604645e-8f;  // 16 units of binary32 roundoff
    const float dR = R1 - R0, dV = V1 - V0;
    const float Rm = 0.5f * (R0 + R1), Vm = 0.5f * (V0 + V1);
    const float kin = dR * Rm + dV * Vm;
    const float kin_abs = fabsf(dR * Rm) + fabsf(dV * Vm);
    const float K0 = 0.5f * (R0 * R0 + V0 * V0);
    float pot = 0.0f, pot_abs = 0.0f;  // eps dpsi and a bound of its terms
    float psi0 = 0.0f, psi0_abs = 0.0f;  // psi(R0) and a bound of its terms
    if (C.field == 0) {
        const float x0 = (R0 - C.r_min) * C.inv_hr, x1 = (R1 - C.r_min) * C.inv_hr;
        if (!(x0 >= 0.0f) || !(x1 >= 0.0f) || !(x0 < (float)C.n_cells) || !(x1 < (float)C.n_cells)) return -1;
        const float f0 = floorf(x0);
        const int j = (int)f0;
        // both positions well inside one cell (the FP64 cell index is the same)
        if (floorf(x1) != f0) return -1;
        // margin from the nodes: the binary32 x is within a few ulp of x <= n_cells
        const float mx = 1e-4f + 1e-6f * (float)C.n_cells;
        const float lo = fminf(x0, x1) - f0, hi = fmaxf(x0, x1) - f0;
        if (lo < mx || hi > 1.0f - mx) return -1;
        const float rj = C.r_min + (float)j * C.hr;
        const float Ej = C.E[j], sl = C.slope[j];
        const float Em = Ej + (Rm - rj) * sl;  // E at the midpoint
        pot = C.eps * dR * Em;
        pot_abs = C.eps * fabsf(dR) * (fabsf(Ej) + (fabsf(Rm) + fabsf(rj) + C.hr) * fabsf(sl));
        const float d0 = R0 - rj;
        psi0 = C.psi[j] + d0 * (Ej + 0.5f * d0 * sl);
        psi0_abs = fabsf(C.psi[j]) + C.hr * (fabsf(Ej) + C.hr * fabsf(sl)) + (fabsf(R0) + fabsf(rj)) * (fabsf(Ej) + C.hr * fabsf(sl));
    } else if (C.field == 1) {
        const float s2 = 0.5f * (R0 * R0 + R1 * R1);
        pot = -C.eps * dR * Rm * s2;
        pot_abs = C.eps * fabsf(dR * Rm) * s2;
        psi0 = -0.25f * (R0 * R0) * (R0 * R0);
        psi0_abs = -psi0;
    }
    const float dH = kin - pot;
    const float H0 = K0 - C.eps * psi0;
    const float margin = fabsf(dH) - C.tol * fabsf(H0);
    // bound of |margin - exact margin|, plus the FP64 evaluation's own noise
    const float scale0 = K0 + C.eps * psi0_abs;
    const float bound = u16 * (kin_abs + pot_abs) + C.tol * u16 * scale0 + 1e-13f * (scale0 + fabsf(dH));
    if (!(fabsf(margin) > 2.0f * bound)) return -1;  // too close to call (or NaN)
    return margin < 0.0f ? 1 : 0;
}

}  // namespace pic

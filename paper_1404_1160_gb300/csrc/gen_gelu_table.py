"""Writes gelu_table.h: the segment table of the fast GELU of the network's
tensor-core inference kernel (gelu_fast.cuh).

On a = |u| / sqrt(2) in [0, 8) the table holds, for each centre a_j = j/8
(j = 0..64), the binary32 value T_j = erfc(a_j) and a cubic
r_j(d) = d (c1 + c2 d + c3 d^2) fitted by least squares on Chebyshev points
to log2(erfc(a_j + d) / erfc(a_j)) for |d| <= 1/16, so that
erfc(a) ~ T_j 2^(r_j(a - a_j)).  The erfc values come from mpmath at 40
digits; the coefficients are rounded to binary32 and the script reports
the largest relative error of the rounded table on a fine grid.

Run: python paper_1404_1160_gb300/csrc/gen_gelu_table.py  (rewrites the
header beside this script; tests/test_gelu_table.py checks that the
committed header is what this script writes)."""
import os
import sys

import mpmath as mp
import numpy as np

mp.mp.dps = 40
N_SEG = 64          # segments of width 1/8 on [0, 8)
WIDTH = 1.0 / 8.0
HALF = WIDTH / 2.0
N_FIT = 64          # Chebyshev points per segment


def log2_erfc(a):
    return mp.log(mp.erfc(mp.mpf(a)), 2)


def segment(j):
    a0 = j * WIDTH
    lo = 0.0 if j == 0 else -HALF
    hi = 0.0 if j == N_SEG else HALF
    if j == N_SEG:      # a < 8: only the left half
        lo = -HALF
    k = np.arange(N_FIT)
    d = 0.5 * (lo + hi) + 0.5 * (hi - lo) * np.cos(np.pi * (k + 0.5) / N_FIT)
    base = log2_erfc(a0)
    y = np.array([float(log2_erfc(a0 + float(di)) - base) for di in d])
    V = np.stack([d, d ** 2, d ** 3], 1)
    c, *_ = np.linalg.lstsq(V, y, rcond=None)
    T = np.float32(float(mp.erfc(mp.mpf(a0))))
    return T, np.float32(c[0]), np.float32(c[1]), np.float32(c[2]), lo, hi


def table():
    return [segment(j) for j in range(N_SEG + 1)]


def max_rel_error(tab, n=257):
    """Largest |T_j 2^r_j(d) / erfc(a_j + d) - 1| over the segments, with the
    binary32 coefficients and exact arithmetic otherwise."""
    worst = 0.0
    for j, (T, c1, c2, c3, lo, hi) in enumerate(tab):
        for d in np.linspace(lo, hi, n):
            r = mp.mpf(float(d)) * (mp.mpf(float(c1)) + mp.mpf(float(d)) * (mp.mpf(float(c2)) + mp.mpf(float(d)) * mp.mpf(float(c3))))
            v = mp.mpf(float(T)) * mp.power(2, r)
            e = abs(v / mp.erfc(mp.mpf(j * WIDTH) + mp.mpf(float(d))) - 1)
            worst = max(worst, float(e))
    return worst


def render(tab) -> str:
    lines = [
        "// gelu_table.h -- written by gen_gelu_table.py (do not edit): for a = |u|/sqrt(2)",
        "// near a_j = j/8, erfc(a) ~ T_j 2^(d (c1 + d (c2 + d c3))), d = a - a_j, |d| <= 1/16.",
        "// Entries (T_j, c1, c2, c3), j = 0..64.",
        "#pragma once",
        "",
        "namespace pic {",
        "",
        f"constexpr int kGeluSeg = {N_SEG};",
        "",
        "static __constant__ float c_gelu_tab[kGeluSeg + 1][4] = {",
    ]
    for (T, c1, c2, c3, _, _) in tab:
        lines.append("    {" + ", ".join(float(v).hex() + "f" for v in (T, c1, c2, c3)) + "},")
    lines += ["};", "", "}  // namespace pic", ""]
    return "\n".join(lines)


HEADER = os.path.join(os.path.dirname(os.path.abspath(__file__)), "gelu_table.h")

if __name__ == "__main__":
    tab = table()
    with open(HEADER, "w") as fh:
        fh.write(render(tab))
    if "--check" in sys.argv:
        print("max relative error", max_rel_error(tab))

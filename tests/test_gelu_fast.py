"""The table GELU of the network's tensor-core inference kernel
(paper_1404_1160_gb300/csrc/gelu_fast.cuh, gelu_table.h).

CPU: the committed table is what its generator writes, its values T_j are
the binary32 roundings of erfc(j/8), and T_j 2^r_j(d) reproduces erfc
within 2^-23 relative on a fine grid (scipy's erfc as the reference).
GPU: for all 2^32 binary32 inputs, the bfloat16 rounding of gelu_for_bf16
has the bits of the bfloat16 rounding of gelu_f (CUDA's erfcf), the only
value the network ever takes from either."""
import os
import re
import shutil
import subprocess

import numpy as np
import pytest

from tests.conftest import ROOT

CSRC = os.path.join(ROOT, "paper_1404_1160_gb300", "csrc")


def read_table():
    text = open(os.path.join(CSRC, "gelu_table.h")).read()
    rows = re.findall(r"\{([^{}]*)\},", text)
    tab = np.array([[float.fromhex(v.strip().rstrip("f")) for v in r.split(",")] for r in rows])
    return tab


def test_table_is_the_generator_output():
    pytest.importorskip("mpmath")
    import importlib.util
    spec = importlib.util.spec_from_file_location("gen_gelu_table", os.path.join(CSRC, "gen_gelu_table.py"))
    gen = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(gen)
    assert gen.render(gen.table()) == open(os.path.join(CSRC, "gelu_table.h")).read()


def test_table_reproduces_erfc():
    from scipy.special import erfc
    tab = read_table()
    assert tab.shape == (65, 4)
    a0 = np.arange(65) / 8.0
    assert np.array_equal(tab[:, 0], erfc(a0).astype(np.float32).astype(np.float64))
    worst = 0.0
    for j in range(65):
        lo = 0.0 if j == 0 else -1 / 16
        hi = 0.0 if j == 64 else 1 / 16
        d = np.linspace(lo, hi, 2001)
        T, c1, c2, c3 = tab[j]
        v = T * np.exp2(d * (c1 + d * (c2 + d * c3)))
        worst = max(worst, float(np.max(np.abs(v / erfc(a0[j] + d) - 1.0))))
    assert worst < 2.0 ** -23, worst


@pytest.mark.gpu
def test_table_gelu_rounds_like_erfc_gelu_for_every_input(tmp_path):
    nvcc = shutil.which("nvcc") or "/usr/local/cuda/bin/nvcc"
    exe = str(tmp_path / "gelu_check")
    subprocess.run([nvcc, "-gencode", "arch=compute_103a,code=sm_103a", "-O3", "-std=c++17", "--fmad=false",
                    "-I", CSRC, "-o", exe, os.path.join(ROOT, "tests", "gelu_check.cu")], check=True)
    out = subprocess.run([exe], capture_output=True, text=True, timeout=300)
    assert out.returncode == 0, out.stdout + out.stderr
    print(out.stdout.strip())
    m = re.search(r"mismatches (\d+) first ([0-9a-f]+) fallback ([0-9.e+-]+) max_ulps (\d+)", out.stdout)
    assert m, out.stdout
    mismatches, fallback, max_ulps = int(m.group(1)), float(m.group(3)), int(m.group(4))
    assert mismatches == 0, out.stdout
    # gelu_f runs for a small share of typical activations, and the certain
    # table results sit well inside the margin
    assert fallback < 0.005, out.stdout
    margin = int(re.search(r"kGeluMargin = (\d+)", open(os.path.join(CSRC, "gelu_fast.cuh")).read()).group(1))
    assert 2 * max_ulps <= margin, out.stdout

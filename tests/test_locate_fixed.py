"""The fixed-point cell locate of the FP64 kernels against its FP64
definition, on the CPU (the same header the kernels include, compiled for
the host): every answer it gives must equal fma(R, W/h_r, -r_min W/h_r)
followed by floor, bit for bit, on random positions, mesh nodes and their
neighbours, tiny values, positions whose low significand bits make ties,
positions around and beyond the mesh edges, and arbitrary bit patterns."""
import os
import subprocess

import pytest

from tests.conftest import ROOT

CSRC = os.path.join(ROOT, "paper_1404_1160_gb300", "csrc")


@pytest.fixture(scope="module")
def checker(tmp_path_factory):
    exe = str(tmp_path_factory.mktemp("loc") / "locate_fixed_check")
    subprocess.run(["g++", "-std=c++17", "-O2", "-ffp-contract=off", "-I", CSRC, "-o", exe,
                    os.path.join(ROOT, "tests", "locate_fixed_check.cpp")], check=True)
    return exe


# (n_cells, log2 W, r_max): the benchmark meshes, the FP32 form's mesh, the
# smallest and largest meshes, other weights and domains
MESHES = [(256, 32, 4.0), (512, 32, 4.0), (1024, 32, 4.0), (2048, 24, 16.0), (2, 40, 1.0), (65536, 20, 8.0),
          (128, 32, 2.0), (256, 1, 4.0)]


@pytest.mark.parametrize("n_cells,log2w,r_max", MESHES)
def test_fixed_point_locate_equals_fp64(checker, n_cells, log2w, r_max):
    out = subprocess.run([checker, str(n_cells), str(log2w), str(r_max), "3000000", str(n_cells + log2w)],
                         capture_output=True, text=True)
    ok, total, fast, bad = (int(x) for x in out.stdout.split()[-4:])
    assert out.returncode == 0 and bad == 0, out.stdout
    assert ok == 1 and fast > 0.6 * total  # most positions take the integer path


def test_non_power_of_two_mesh_keeps_the_fp64_form(checker):
    # 1/h_r = 25 (100 cells on [-2, 2]) is not a power of two: no fixed-point form
    out = subprocess.run([checker, "100", "32", "2.0", "1000", "1"], capture_output=True, text=True)
    assert out.returncode == 0 and out.stdout.split()[0] == "0"

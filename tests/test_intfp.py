"""The integer-pipe binary64 multiply used by the FP64 window kernels
(paper_1404_1160_gb300/csrc/intfp.cuh), compiled for the host, against the
CPU's IEEE binary64 product: every product it answers must have the same
bits (random operands, the fine step's rotation constants, exact products
and ties from significands with trailing zeros, rounding carries, operands
near the ends of the normal range and arbitrary bit patterns)."""
import os
import subprocess

from tests.conftest import ROOT

CSRC = os.path.join(ROOT, "paper_1404_1160_gb300", "csrc")


def test_integer_multiply_equals_binary64(tmp_path):
    exe = str(tmp_path / "intfp_check")
    subprocess.run(["g++", "-std=c++17", "-O2", "-ffp-contract=off", "-I", CSRC, "-o", exe,
                    os.path.join(ROOT, "tests", "intfp_check.cpp")], check=True)
    out = subprocess.run([exe, "12000000", "3"], capture_output=True, text=True)
    total, answered, bad = (int(x) for x in out.stdout.split()[-3:])
    assert out.returncode == 0 and bad == 0, out.stdout
    assert answered > 0.8 * total

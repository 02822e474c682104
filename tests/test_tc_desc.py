"""The tensor-core descriptors of the learned stepper's network
(paper_1404_1160_gb300/csrc/tc_desc.cuh), compiled for the host and decoded
here field by field from the PTX ISA's layout of the tcgen05 instruction
descriptor (kind::f16) and shared-memory matrix descriptor, before any kernel
hands them to the tensor core."""
import os
import subprocess

from tests.conftest import ROOT

CSRC = os.path.join(ROOT, "paper_1404_1160_gb300", "csrc")


def bits(v, lo, hi):
    """Field [lo, hi) of v."""
    return (v >> lo) & ((1 << (hi - lo)) - 1)


def run_check(tmp_path):
    exe = str(tmp_path / "tc_desc_check")
    subprocess.run(["g++", "-std=c++17", "-O1", "-I", CSRC, "-o", exe,
                    os.path.join(ROOT, "tests", "tc_desc_check.cpp")], check=True)
    out = subprocess.run([exe], capture_output=True, text=True, check=True).stdout.split("\n")
    rows = [line.split() for line in out if line]
    return ([tuple(int(x) for x in r[1:]) for r in rows if r[0] == "idesc"],
            [tuple(int(x) for x in r[1:]) for r in rows if r[0] == "sdesc"],
            {(int(r[1]), int(r[2])): int(r[3]) for r in rows if r[0] == "off"})


def test_instruction_descriptor_fields(tmp_path):
    idesc, _, _ = run_check(tmp_path)
    assert len(idesc) == 5
    for M, N, v in idesc:
        assert v < 1 << 32
        assert bits(v, 0, 2) == 0 and bits(v, 2, 3) == 0 and bits(v, 3, 4) == 0  # dense, no saturation
        assert bits(v, 4, 6) == 1            # accumulator f32
        assert bits(v, 6, 7) == 0            # reserved
        assert bits(v, 7, 10) == 1           # A bf16
        assert bits(v, 10, 13) == 1          # B bf16
        assert bits(v, 13, 15) == 0          # no negation
        assert bits(v, 15, 16) == 0 and bits(v, 16, 17) == 0  # A and B K-major
        assert bits(v, 17, 23) * 8 == N
        assert bits(v, 23, 24) == 0          # reserved
        assert bits(v, 24, 29) * 16 == M
        assert bits(v, 29, 32) == 0          # reserved, no shift


def test_shared_memory_descriptor_fields(tmp_path):
    _, sdesc, _ = run_check(tmp_path)
    assert len(sdesc) == 5
    for addr, lbo, sbo, v in sdesc:
        assert bits(v, 0, 14) << 4 == addr % (1 << 18)
        assert bits(v, 14, 16) == 0
        assert bits(v, 16, 30) << 4 == lbo
        assert bits(v, 30, 32) == 0
        assert bits(v, 32, 46) << 4 == sbo
        assert bits(v, 46, 48) == 1          # tcgen05 descriptor version
        assert bits(v, 48, 49) == 0
        assert bits(v, 49, 52) == 0          # base offset: operands 1024-byte aligned
        assert bits(v, 52, 53) == 0          # relative leading-dimension offset
        assert bits(v, 53, 61) == 0
        assert bits(v, 61, 64) == 0          # no swizzling


def test_operand_layout_is_the_core_matrix_layout(tmp_path):
    """No-swizzle K-major layout: each core matrix is 8 rows of 16 contiguous
    bytes (8 bf16 along K); core matrices adjacent along K are LBO = 128 bytes
    apart and groups of 8 rows SBO = 1024 bytes apart; the whole 128 x 64
    bf16 tile is a permutation of its 16 KiB."""
    _, _, off = run_check(tmp_path)
    assert len(off) == 128 * 64
    assert sorted(off.values()) == list(range(0, 128 * 64 * 2, 2))
    for (r, k), o in off.items():
        cm = off[(r - r % 8, k - k % 8)]       # start of the core matrix holding (r, k)
        assert o - cm == (r % 8) * 16 + (k % 8) * 2
        assert cm == (r // 8) * 1024 + (k // 8) * 128
    # the k-th 16-wide K step of an MMA starts 2 LBO after the previous one,
    # which is the start address the kernels give each of the four MMAs
    for ks in range(4):
        assert off[(0, 16 * ks)] == ks * 2 * 128

"""The binary32 energy check of the learned stepper's FP32 form
(paper_1404_1160_gb300/csrc/energy_check.cuh), compiled for the host,
against the oracle's FP64 keep/fallback rule (oracle.learned.learned_apply,
binary32 state): every decision it takes must be the oracle's, on seeded
beams, fields and corrections spanning the threshold, for the Poisson
(both parities, particles off the mesh and across cell boundaries), Duffing
and zero fields; it must decide the large majority itself."""
import os
import subprocess

import numpy as np
import pytest

import oracle
from oracle import learned as OL
from paper_1404_1160_gb300 import inputs
from tests.conftest import ROOT

CSRC = os.path.join(ROOT, "paper_1404_1160_gb300", "csrc")


@pytest.fixture(scope="module")
def checker(tmp_path_factory):
    exe = str(tmp_path_factory.mktemp("ec") / "energy_check_check")
    subprocess.run(["g++", "-std=c++17", "-O2", "-ffp-contract=off", "-I", CSRC, "-o", exe,
                    os.path.join(ROOT, "tests", "energy_check_check.cpp")], check=True)
    return exe


def run_checker(exe, tmp, field, cfg, tabs, R0, V0, R1, V1, tol):
    f32 = np.float32
    hr = (cfg.r_max - cfg.r_min) / cfg.n_cells
    with open(tmp / "in.bin", "wb") as fh:
        fh.write(np.array([field, cfg.n_cells, R0.size], np.int32).tobytes())
        fh.write(np.array([cfg.eps, tol, cfg.r_min, hr, 1.0 / hr], f32).tobytes())
        fh.write(np.ascontiguousarray(tabs, f32).tobytes())
        fh.write(np.stack([R0, V0, R1, V1], axis=1).astype(f32).tobytes())
    subprocess.run([exe, str(tmp / "in.bin"), str(tmp / "out.bin")], check=True)
    return np.fromfile(tmp / "out.bin", np.int8)


def field_tables(cfg, E):
    """E_j, (E_{j+1} - E_j)/h_r and psi_j rounded once to binary32 (the rounding the kernel applies)."""
    hr = (cfg.r_max - cfg.r_min) / cfg.n_cells
    slope = np.zeros(E.size)
    slope[:-1] = (E[1:] - E[:-1]) * (1.0 / hr)
    return np.concatenate([E, slope, OL.node_potential(cfg, E)]).astype(np.float32)


@pytest.mark.parametrize("field,parity,n_cells,tol", [(oracle.FIELD_POISSON, 0, 512, 1e-4),
                                                      (oracle.FIELD_POISSON, 1, 256, 1e-3),
                                                      (oracle.FIELD_POISSON, 0, 2048, 3e-4),
                                                      (oracle.FIELD_DUFFING, 0, 256, 1e-4),
                                                      (oracle.FIELD_ZERO, 0, 256, 1e-4)])
def test_binary32_decisions_are_the_fp64_decisions(checker, tmp_path, field, parity, n_cells, tol):
    cfg = oracle.Config(eps=0.01, dt=0.4, field_model=field, n_cells=n_cells, r_min=-2.0, r_max=2.0,
                        field_parity=parity)
    n = 200_000
    rng = np.random.default_rng(n_cells + field)
    R, V = inputs.gaussian_beam(n, seed=n_cells + parity)  # uncut: some beyond the mesh
    R0, V0 = R.astype(np.float32), V.astype(np.float32)
    E = edges = None
    tabs = np.zeros(3 * (n_cells + 1), np.float32)
    if field == oracle.FIELD_POISSON:
        E, edges = OL.mesh_field(cfg, R)
        tabs = field_tables(cfg, E)
    # corrections on several scales around the threshold; some cross cells
    scale = np.float32(10.0) ** rng.uniform(-7, -2, n).astype(np.float32)
    dR = (rng.normal(0, 1, n).astype(np.float32) * scale).astype(np.float32)
    dV = (rng.normal(0, 1, n).astype(np.float32) * scale).astype(np.float32)
    R1, V1 = (R0 + dR).astype(np.float32), (V0 + dV).astype(np.float32)
    dec = run_checker(checker, tmp_path, field, cfg, tabs, R0, V0, R1, V1, tol)
    _, _, keep, margin = OL.learned_apply(cfg, R0, V0, dR, dV, tol, E, edges, precision=1)
    decided = dec >= 0
    nonzero = (dR != 0) | (dV != 0)
    assert np.array_equal(dec[decided & nonzero] == 1, keep[decided & nonzero])
    assert decided.mean() > 0.7, decided.mean()  # corrections up to 1e-2 cross the cells of fine meshes
    assert 0.05 < keep.mean() < 0.95
    if field == oracle.FIELD_POISSON:
        off = (R0 < cfg.r_min) | (R0 >= cfg.r_max)
        assert off.sum() > 100 and not decided[off].any()  # off the mesh: always the FP64 rule


def test_binary32_decides_almost_all_of_a_workload_shaped_step(checker, tmp_path):
    # the learned workload's shape: 512 cells on [-4, 4], the beam cut at 4,
    # corrections of ~1e-5 (the trained network's), tol 1e-4
    cfg = oracle.Config(eps=0.01, dt=0.4, field_model=oracle.FIELD_POISSON, n_cells=512, r_min=-4.0, r_max=4.0)
    n = 200_000
    rng = np.random.default_rng(7)
    R, V = inputs.gaussian_beam(n, seed=8, r_cut=4.0)
    R0, V0 = R.astype(np.float32), V.astype(np.float32)
    E, edges = OL.mesh_field(cfg, R)
    dR = (rng.normal(0, 2e-5, n)).astype(np.float32)
    dV = (rng.normal(0, 2e-5, n)).astype(np.float32)
    R1, V1 = (R0 + dR).astype(np.float32), (V0 + dV).astype(np.float32)
    dec = run_checker(checker, tmp_path, oracle.FIELD_POISSON, cfg, field_tables(cfg, E), R0, V0, R1, V1, 1e-4)
    _, _, keep, _ = OL.learned_apply(cfg, R0, V0, dR, dV, 1e-4, E, edges, precision=1)
    decided = dec >= 0
    assert np.array_equal(dec[decided] == 1, keep[decided])
    assert decided.mean() > 0.97, decided.mean()

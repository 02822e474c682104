"""Shared helpers of the GPU parity tests: the same seeded inputs go to the
CUDA path (through the C ABI) and to the FP64 oracle."""
import numpy as np

import oracle
from paper_1404_1160_gb300 import pic

STATE_RTOL = 1e-12  # FP64 tolerance on R, V, E (the kernels are built to match bit for bit)


def cfg_of(p) -> "oracle.Config":
    return oracle.Config(eps=p.eps, dt=p.dt, field_model=p.field_model, fine_solver=p.fine_solver,
                         steps_per_turn=p.steps_per_turn, n_cells=p.n_cells, r_min=p.r_min, r_max=p.r_max,
                         total_charge=p.total_charge, weight_fixed=p.weight_fixed,
                         max_window_steps=p.max_window_steps, field_parity=p.field_parity)


def assert_close(gpu, ref, rtol=STATE_RTOL, what=""):
    gpu = np.asarray(gpu, np.float64)
    ref = np.asarray(ref, np.float64)
    assert gpu.shape == ref.shape
    scale = max(1.0, float(np.max(np.abs(ref)))) if ref.size else 1.0
    err = float(np.max(np.abs(gpu - ref))) if ref.size else 0.0
    assert err <= rtol * scale, f"{what}: max |gpu - oracle| = {err:.3e} (scale {scale:.3e})"
    return err


def bit_equal(a, b):
    return np.array_equal(np.asarray(a).view(np.int64), np.asarray(b).view(np.int64))

"""Seeded synthetic particle sets shaped like the paper's runs.

This module draws initial conditions only.  It holds none of the method's
arithmetic; the CUDA library and the oracle both receive the arrays it
returns.

Generator: counter-based SplitMix64 (Steele, Lea & Flood 2014) -> uniform in
(0, 1) from the top 53 bits -> Box-Muller normals.  The stream depends only
on the seed, never on the numpy version.

Distributions:
* ``gaussian_beam``: r ~ N(0, sigma_r) (optionally truncated to |r| <= r_cut
  by rejection), v ~ N(0, v_th).  Shapes the Duffing and Vlasov-Poisson runs
  with unit thermal spread.
* ``paper_beam``: the initial condition of eq. InitialConditionBeam:
  Gaussian in v with v_th = 0.0727518214392, uniform in r on [-0.75, 0.75].
"""
from __future__ import annotations

import numpy as np

_GOLDEN = np.uint64(0x9E3779B97F4A7C15)
_M1 = np.uint64(0xBF58476D1CE4E5B9)
_M2 = np.uint64(0x94D049BB133111EB)

PAPER_V_TH = 0.0727518214392  # eq. InitialConditionBeam
PAPER_R_HALF_WIDTH = 0.75


def splitmix64(seed: int, start: int, count: int) -> np.ndarray:
    """Outputs start..start+count-1 of the SplitMix64 stream for ``seed``."""
    k = np.arange(start + 1, start + count + 1, dtype=np.uint64)
    with np.errstate(over="ignore"):
        z = np.uint64(seed & 0xFFFFFFFFFFFFFFFF) + k * _GOLDEN
        z = (z ^ (z >> np.uint64(30))) * _M1
        z = (z ^ (z >> np.uint64(27))) * _M2
        z = z ^ (z >> np.uint64(31))
    return z


def uniform(seed: int, start: int, count: int) -> np.ndarray:
    """Uniform doubles in (0, 1)."""
    z = splitmix64(seed, start, count)
    return ((z >> np.uint64(11)).astype(np.float64) + 0.5) * (1.0 / 9007199254740992.0)


def normal(seed: int, start: int, count: int) -> np.ndarray:
    """Standard normals by Box-Muller, two per pair of uniforms."""
    m = (count + 1) // 2
    u = uniform(seed, 2 * start, 2 * m)
    rad = np.sqrt(-2.0 * np.log(u[0::2]))
    ang = 2.0 * np.pi * u[1::2]
    out = np.empty(2 * m, np.float64)
    out[0::2] = rad * np.cos(ang)
    out[1::2] = rad * np.sin(ang)
    return out[:count]


def _truncated_normal(seed: int, n: int, sigma: float, cut: float | None) -> np.ndarray:
    if cut is None:
        return sigma * normal(seed, 0, n)
    out = np.empty(0, np.float64)
    start = 0
    while out.size < n:
        need = n - out.size
        chunk = max(1024, int(need * 1.1) + 64)
        x = sigma * normal(seed, start, chunk)
        start += chunk
        out = np.concatenate([out, x[np.abs(x) <= cut][:need]])
    return out


def gaussian_beam(n: int, seed: int = 0, sigma_r: float = 1.0, v_th: float = 1.0,
                  r_cut: float | None = None) -> tuple[np.ndarray, np.ndarray]:
    """(R, V) with R ~ N(0, sigma_r) (truncated to |R| <= r_cut), V ~ N(0, v_th)."""
    r = _truncated_normal(2 * seed + 1, n, sigma_r, r_cut)
    v = v_th * normal(2 * seed + 2, 0, n)
    return r, v


def paper_beam(n: int = 20000, seed: int = 0) -> tuple[np.ndarray, np.ndarray]:
    """Samples of eq. InitialConditionBeam (N_p = 20000 in the paper)."""
    r = PAPER_R_HALF_WIDTH * (2.0 * uniform(2 * seed + 1, 0, n) - 1.0)
    v = PAPER_V_TH * normal(2 * seed + 2, 0, n)
    return r, v


# ---------------------------------------------------------------- learned stepper

MLP_SHAPES = [("W1", (64, 5)), ("b1", (64,)), ("W2", (64, 64)), ("b2", (64,)), ("W3", (2, 64)), ("b3", (2,))]


def mlp_init(seed: int) -> np.ndarray:
    """Seeded Glorot-uniform starting weights of the learned stepper's network
    (biases zero), flat float32 in the library's layout: W1 (64 x 5) | b1 |
    W2 (64 x 64) | b2 | W3 (2 x 64) | b3."""
    parts = []
    start = 0
    for name, shape in MLP_SHAPES:
        n = int(np.prod(shape))
        if name.startswith("W"):
            a = np.sqrt(6.0 / (shape[0] + shape[1]))
            parts.append((2.0 * uniform(seed, start, n) - 1.0) * a)
        else:
            parts.append(np.zeros(n))
        start += n
    return np.concatenate(parts).astype(np.float32)

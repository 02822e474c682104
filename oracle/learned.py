"""Plain FP64 oracle of the learned stepper's physics outside the network.

TEST INFRASTRUCTURE ONLY.  Only the test suite, the smoke check and the
benchmark's CPU leg may use it; the CUDA library never calls it and shares
nothing with it.

The paper has no learned component.  The learned stepper corrects one macro
step of the improved ETD scheme (Algorithm ETDFSSModAlgo) and guards the
correction with an energy check.  This module defines, in the order the step
takes them:

1. the frozen field of y^n: the mesh field of the deposit of R^n (Sec. 2.3,
   trapezoid integral of eq. VlasPoissAxSymBeam), seen by a particle through
   the linear gather, and E = rE_edge / r off the mesh (no charge beyond the
   edge); or the Duffing field E = -r^3 (eq. RappelForce); or no field;
2. its potential psi(R) = int_0^R E(s) ds, so that psi' = E and psi(0) = 0;
3. the frozen-field energy H(R, V) = (R^2 + V^2)/2 - eps psi(R), which the
   characteristics dR/dt = V/eps, dV/dt = -R/eps + E(R) (eq.
   CharactCurvesOfGenVlas) conserve while E does not change:
   dH/dt = R V/eps + V (-R/eps + E) - eps E V/eps = 0;
4. the decision: the corrected state y_l = y_plain + (dR, dV) is kept when
   |H(y_l) - H(y_plain)| <= tol |H(y_plain)| (the plain step judges the
   correction), the plain state otherwise; a zero correction leaves y_plain;
5. one Adam update of the network's master weights (Kingma & Ba, "Adam: a
   method for stochastic optimization", Algorithm 1).

The network output itself comes from ``oracle.mlp``.  The correction is the
network's binary32 output times a binary32 scale, rounded to binary32 (the
network computes in binary32).
"""
from __future__ import annotations

import math

import numpy as np

from . import FIELD_DUFFING, FIELD_POISSON, Config, deposit, deposit_f32, derive, etd_step, poisson
from . import mlp as _mlp


def _f64(a):
    return np.ascontiguousarray(a, dtype=np.float64)


def mesh_field(cfg: Config, R, n_particles: int | None = None, precision: int = 0):
    """The frozen mesh field of positions R: (E at the nodes, rE at the two
    edges), from the CIC deposit and the trapezoid integral (Sec. 2.3).
    precision 1 deposits binary32 positions with binary32 cell arithmetic
    (the FP32 form's quantisation)."""
    R = _f64(R)
    Q, _ = deposit_f32(cfg, R.astype(np.float32)) if precision else deposit(cfg, R)
    _, E, edges = poisson(cfg, Q, R.size if n_particles is None else n_particles)
    return E, edges


def node_potential(cfg: Config, E):
    """psi at the nodes r_j: the integral from r = 0 (node n_cells/2) of the
    linear interpolant of the node field, one cell at a time (the trapezoid
    rule is exact for a linear function)."""
    E = _f64(E)
    c = cfg.n_cells // 2
    hr = derive(cfg).hr
    psi = np.zeros(cfg.n_cells + 1)
    for j in range(c + 1, cfg.n_cells + 1):
        psi[j] = psi[j - 1] + hr * (E[j - 1] + E[j]) / 2.0
    for j in range(c - 1, -1, -1):
        psi[j] = psi[j + 1] - hr * (E[j] + E[j + 1]) / 2.0
    return psi


def frozen_potential(cfg: Config, R, E=None, edges=None):
    """psi(R) = int_0^R E(s) ds of the frozen field (psi(0) = 0).

    Poisson: inside the mesh, node potential plus the exact integral over the
    part of the cell [r_j, R] of the linear gather E_j + (s - r_j)(E_{j+1} -
    E_j)/h_r; beyond an edge r_e, psi(r_e) + rE_e ln(R / r_e) (E = rE_e / s).
    Duffing: -R^4/4.  No field: 0."""
    R = _f64(R)
    if cfg.field_model == FIELD_DUFFING:
        return -((R * R) * (R * R)) / 4.0
    if cfg.field_model != FIELD_POISSON:
        return np.zeros_like(R)
    E, edges = _f64(E), _f64(edges)
    d = derive(cfg)
    psi_n = node_potential(cfg, E)
    out = np.empty_like(R)
    x = (R - cfg.r_min) * d.inv_hr
    inside = (x >= 0.0) & (x < cfg.n_cells)
    j = np.floor(np.where(inside, x, 0.0)).astype(np.int64)
    s = R - (cfg.r_min + j * d.hr)  # distance from the cell's left node
    Ej, Ej1 = E[j], E[j + 1]
    out[inside] = (psi_n[j] + Ej * s + (Ej1 - Ej) * s * s / (2.0 * d.hr))[inside]
    lo = ~inside & (x < 0.0)
    hi = ~inside & ~(x < 0.0)
    out[lo] = psi_n[0] + edges[0] * np.log(R[lo] / cfg.r_min)
    out[hi] = psi_n[cfg.n_cells] + edges[1] * np.log(R[hi] / cfg.r_max)
    return out


def frozen_energy(cfg: Config, R, V, E=None, edges=None):
    """H(R, V) = (R^2 + V^2)/2 - eps psi(R) of the frozen field."""
    R, V = _f64(R), _f64(V)
    return 0.5 * (R * R + V * V) - cfg.eps * frozen_potential(cfg, R, E, edges)


def learned_apply(cfg: Config, Rp, Vp, dR, dV, tol: float, E=None, edges=None, precision: int = 0):
    """Step 4: the kept state, the keep mask and the decision margin.

    Rp, Vp: the plain step's result; dR, dV: the correction (binary32
    values).  precision 1 (the FP32 form) rounds the corrected state to
    binary32: y_l = f32(y_plain + dy).  Returns (R, V, keep, margin) with
    margin = |H(y_l) - H(y_plain)| - tol |H(y_plain)| (keep iff margin <= 0);
    particles with a zero correction keep the plain state and count as kept
    (margin -inf)."""
    Rp, Vp, dR, dV = _f64(Rp), _f64(Vp), _f64(dR), _f64(dV)
    if precision:
        Rl = (np.float32(Rp) + np.float32(dR)).astype(np.float64)
        Vl = (np.float32(Vp) + np.float32(dV)).astype(np.float64)
    else:
        Rl, Vl = Rp + dR, Vp + dV
    H0 = frozen_energy(cfg, Rp, Vp, E, edges)
    H1 = frozen_energy(cfg, Rl, Vl, E, edges)
    margin = np.abs(H1 - H0) - tol * np.abs(H0)
    zero = (dR == 0.0) & (dV == 0.0)
    margin = np.where(zero, -np.inf, margin)
    keep = margin <= 0.0
    R = np.where(keep & ~zero, Rl, Rp)
    V = np.where(keep & ~zero, Vl, Vp)
    return R, V, keep, margin


def network_inputs(R, V, t: float, eps: float, dt: float):
    """The network's binary32 inputs (r, v, sin(t/eps), cos(t/eps), dt) of y^n."""
    R, V = _f64(R), _f64(V)
    n = R.size
    X = np.empty((n, 5), np.float32)
    X[:, 0] = R.astype(np.float32)
    X[:, 1] = V.astype(np.float32)
    X[:, 2] = np.float32(math.sin(t / eps))
    X[:, 3] = np.float32(math.cos(t / eps))
    X[:, 4] = np.float32(dt)
    return X


def correction(out, scale):
    """(dR, dV) = binary32 products of the network's binary32 output and the
    per-component scale."""
    out = np.asarray(out, np.float32)
    return (np.float32(scale[0]) * out[:, 0]).astype(np.float64), (np.float32(scale[1]) * out[:, 1]).astype(np.float64)


def learned_step(cfg: Config, R, V, t: float, w, scale, tol: float, T=None):
    """One macro step of the learned stepper in FP64 (steps 1-4 above), with
    the network evaluated by ``oracle.mlp`` (its bfloat16 rounding points
    emulated) and its output rounded to binary32.  T (fine steps) known =>
    the plain step skips period detection.  Returns a dict with R, V, keep,
    margin, the plain result and the frozen field."""
    R, V = _f64(R), _f64(V)
    E = edges = None
    if cfg.field_model == FIELD_POISSON:
        E, edges = mesh_field(cfg, R)
    plain = etd_step(cfg, R, V, T)
    X = network_inputs(R, V, t, cfg.eps, cfg.dt)
    out = _mlp.forward(np.asarray(w, np.float64), X.astype(np.float64))["out"].astype(np.float32)
    dR, dV = correction(out, scale)
    Rn, Vn, keep, margin = learned_apply(cfg, plain.R, plain.V, dR, dV, tol, E, edges)
    return dict(R=Rn, V=Vn, keep=keep, margin=margin, plain=plain, E=E, edges=edges, dR=dR, dV=dV)


def adam_step(w, m, v, g, t: int, lr: float, beta1: float, beta2: float, eps: float):
    """One Adam update (Kingma & Ba, Algorithm 1) at step t >= 1:
    m <- beta1 m + (1 - beta1) g;  v <- beta2 v + (1 - beta2) g^2;
    m_hat = m / (1 - beta1^t);  v_hat = v / (1 - beta2^t);
    w <- w - lr m_hat / (sqrt(v_hat) + eps).  Returns (w, m, v)."""
    w, m, v, g = _f64(w), _f64(m), _f64(v), _f64(g)
    m = beta1 * m + (1.0 - beta1) * g
    v = beta2 * v + (1.0 - beta2) * g * g
    m_hat = m / (1.0 - beta1 ** t)
    v_hat = v / (1.0 - beta2 ** t)
    return w - lr * m_hat / (np.sqrt(v_hat) + eps), m, v

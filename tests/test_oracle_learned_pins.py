"""Pins of the learned stepper's oracle (oracle/learned.py, oracle/mlp.py's
interval form) against what the mathematics fixes.

The frozen-field potential psi and energy H are pinned by closed forms for
uniform and linear charge, by psi' = E (finite differences against the
gather), by the Duffing energy of the paper's appendix, and by energy
conservation along a trajectory integrated in the frozen field by an RK4
written here.  The keep/fallback rule is pinned by hand-worked cases, the
Adam update by the closed form of its first two steps (Kingma & Ba,
Algorithm 1), and the network's interval form by containment of the exact
value and of independently rounded evaluations.
"""
import math

import numpy as np
import pytest

import oracle
from oracle import learned as L
from oracle import mlp
from paper_1404_1160_gb300 import inputs


def pcfg(**kw):
    base = dict(eps=0.01, dt=0.4, field_model=oracle.FIELD_POISSON, fine_solver=oracle.FINE_LAWSON, n_cells=256,
                r_min=-4.0, r_max=4.0)
    base.update(kw)
    return oracle.Config(**base)


def uniform_field(c, half=40, q=1 << 33, n_p=1000):
    """Node field of a uniform charge on nodes c/2 - half .. c/2 + half, and its rho0."""
    Q = np.zeros(c.n_cells + 1, np.int64)
    m = c.n_cells // 2
    Q[m - half:m + half + 1] = q
    _, E, edges = oracle.poisson(c, Q, n_p)
    hr = (c.r_max - c.r_min) / c.n_cells
    rho0 = q * (c.total_charge / (n_p * c.weight_fixed)) / hr
    return E, edges, rho0, half * hr


# ------------------------------------------------------------ potential


def test_potential_of_uniform_charge_is_rho0_r():
    # charge Q on the nodes |r| <= a: rho = rho0 inside, falling linearly to 0
    # over the next cell, so rE = rho0 r inside and rho0 (a + h_r/2) beyond
    # a + h_r.  Even reading: E = rho0 for |r| <= a => psi = rho0 r exactly;
    # beyond a + h_r the linear gather of E_j = rho0 (a + h_r/2)/r_j
    # integrates rho0 (a + h_r/2)/r to within the trapezoid bound
    # h_r^2/12 int |E''|; off the mesh psi continues as rE_edge ln(R/r_edge)
    # with rE_edge = rho0 (a + h_r/2) exactly.
    c = pcfg()
    E, edges, rho0, a = uniform_field(c)
    hr = 8 / 256
    R = np.linspace(-a, a, 1001)
    assert np.allclose(L.frozen_potential(c, R, E, edges), rho0 * R, rtol=1e-13, atol=1e-13 * rho0)
    k = rho0 * (a + hr / 2)
    assert edges[1] == pytest.approx(k, rel=1e-14) and edges[0] == pytest.approx(-k, rel=1e-14)
    b = a + hr
    for sgn in (1.0, -1.0):
        R = sgn * np.array([b + 0.3, 2.0, 3.3, 4.0])
        d = L.frozen_potential(c, R, E, edges) - L.frozen_potential(c, np.array([sgn * b]), E, edges)[0]
        bound = hr * hr / 12 * k * (1 / b ** 2)
        assert np.allclose(d, sgn * k * np.log(np.abs(R) / b), rtol=0, atol=bound)
        R = sgn * np.array([4.5, 8.0, 40.0])
        d = L.frozen_potential(c, R, E, edges) - L.frozen_potential(c, np.array([sgn * 4.0]), E, edges)[0]
        assert np.allclose(d, sgn * k * np.log(np.abs(R) / 4.0), rtol=1e-13, atol=0)


def test_potential_odd_reading_uniform_charge_is_rho0_abs_r():
    # odd extension: E = rho0 sign(r) at the nodes inside the charge and 0 on
    # the axis, so the linear gather ramps from 0 to rho0 over the cells next
    # to the axis: psi = rho0 r^2/(2 h_r) for |r| <= h_r, rho0 (|r| - h_r/2)
    # beyond (the integral of the gathered field, not of the sign function)
    c = pcfg(field_parity=1)
    E, edges, rho0, a = uniform_field(c)
    hr = 8 / 256
    R = np.linspace(-a, a, 1001)
    expect = np.where(np.abs(R) <= hr, rho0 * R * R / (2 * hr), rho0 * (np.abs(R) - hr / 2))
    assert np.allclose(L.frozen_potential(c, R, E, edges), expect, rtol=1e-13, atol=1e-13 * rho0)
    # mirror symmetric everywhere, off the mesh included
    R = np.array([0.3, 1.7, 3.99, 4.0, 6.5, 60.0])
    assert np.allclose(L.frozen_potential(c, R, E, edges), L.frozen_potential(c, -R, E, edges), rtol=1e-14)


def test_potential_of_linear_charge_is_exact_cubic_free():
    # rho = A + B|r| => E = A + B|r|/2 (trapezoid exact) => psi = A r + B r|r|/4,
    # exact for the linear gather because E is linear on each side of the axis
    c = pcfg()
    j = np.arange(257)
    A, B = 1 << 30, 1 << 24
    Q = (A + B * np.abs(j - 128)).astype(np.int64)
    _, E, edges = oracle.poisson(c, Q, 10**6)
    hr = 8 / 256
    q_unit = 1.0 / (10**6 * c.weight_fixed)
    a, b = A * q_unit / hr, B * q_unit / hr / hr
    R = np.random.default_rng(1).uniform(-3.99, 3.99, 2000)
    assert np.allclose(L.frozen_potential(c, R, E, edges), a * R + b * R * np.abs(R) / 4, rtol=1e-12, atol=1e-12)


@pytest.mark.parametrize("parity", [0, 1])
def test_potential_derivative_is_the_gathered_field(parity):
    # psi' = E everywhere a particle can be: inside cells and off the mesh
    c = pcfg(field_parity=parity, r_min=-2.0, r_max=2.0, n_cells=100)
    R0, _ = inputs.gaussian_beam(50_000, seed=3)
    E, edges = L.mesh_field(c, R0)
    hr = 4.0 / 100
    rng = np.random.default_rng(4)
    R = np.concatenate([rng.uniform(-1.98, 1.98, 3000), rng.uniform(2.05, 9.0, 200), -rng.uniform(2.05, 9.0, 200)])
    # keep the stencil inside one cell (the field has kinks at the nodes)
    x = (R + 2.0) / hr
    R = R[(np.abs(x - np.round(x)) > 0.01) | (np.abs(R) > 2.0)]
    d = 1e-5 * hr
    fd = (L.frozen_potential(c, R + d, E, edges) - L.frozen_potential(c, R - d, E, edges)) / (2 * d)
    g = oracle.gather(c, R, E, edges)
    assert np.allclose(fd, g, rtol=1e-7, atol=1e-7 * np.abs(E).max())


def test_duffing_frozen_energy_is_the_appendix_energy():
    # E = -r^3 => psi = -r^4/4 => H = (r^2 + v^2)/2 + eps r^4/4 = eps^2 H of
    # the appendix (pinned in test_oracle_pins against the appendix's period)
    c = pcfg(field_model=oracle.FIELD_DUFFING, eps=0.01)
    rng = np.random.default_rng(5)
    R, V = rng.normal(0, 1, 500), rng.normal(0, 1, 500)
    H = L.frozen_energy(c, R, V)
    ref = np.array([oracle.duffing_energy(c.eps, r, v) for r, v in zip(R, V)])
    assert np.allclose(H, ref, rtol=4e-16, atol=0)
    z = pcfg(field_model=oracle.FIELD_ZERO)
    assert np.array_equal(L.frozen_energy(z, R, V), 0.5 * (R * R + V * V))


def _rk4_frozen(c, E, edges, R, V, h, n):
    """RK4 of dR/dt = V/eps, dV/dt = -R/eps + E(R) with the frozen mesh field."""
    def f(r, v):
        return v / c.eps, -r / c.eps + oracle.gather(c, np.atleast_1d(r), E, edges)[0]
    for _ in range(n):
        k1 = f(R, V)
        k2 = f(R + h / 2 * k1[0], V + h / 2 * k1[1])
        k3 = f(R + h / 2 * k2[0], V + h / 2 * k2[1])
        k4 = f(R + h * k3[0], V + h * k3[1])
        R = R + h / 6 * (k1[0] + 2 * k2[0] + 2 * k3[0] + k4[0])
        V = V + h / 6 * (k1[1] + 2 * k2[1] + 2 * k3[1] + k4[1])
    return R, V


@pytest.mark.parametrize("r0,v0", [(0.4, 0.3), (1.2, -0.9), (1.5, 1.6)])
def test_frozen_energy_is_conserved_along_characteristics(r0, v0):
    # the characteristics of the frozen field conserve H (dH/dt = 0); the
    # third orbit (amplitude 2.19) leaves the mesh [-2, 2] (the log branch of
    # psi).  The RK4 here loses its order at the field's kinks (nodes), so H
    # is kept to ~1e-8 whatever the step; with the opposite sign of the
    # eps psi term the same orbits move by 3e-5 .. 4e-3.
    c = pcfg(r_min=-2.0, r_max=2.0, n_cells=64, eps=0.05)
    R0, _ = inputs.gaussian_beam(20_000, seed=6)
    E, edges = L.mesh_field(c, 0.5 * R0)
    h = 2 * math.pi * c.eps / 2000
    R, V = _rk4_frozen(c, E, edges, r0, v0, h, 4000)  # two turns
    H0 = L.frozen_energy(c, np.array([r0]), np.array([v0]), E, edges)[0]
    H1 = L.frozen_energy(c, np.array([R]), np.array([V]), E, edges)[0]
    assert abs(H1 - H0) <= 1e-7 * abs(H0), (H0, H1)
    wrong = lambda r, v: 0.5 * (r * r + v * v) + c.eps * L.frozen_potential(c, np.array([r]), E, edges)[0]  # noqa: E731
    assert abs(wrong(R, V) - wrong(r0, v0)) > 1e-5 * abs(H0)


# ------------------------------------------------------------ decision


def test_apply_zero_correction_keeps_the_plain_state():
    c = pcfg(field_model=oracle.FIELD_ZERO)
    Rp, Vp = np.array([0.5, -1.0]), np.array([0.25, 2.0])
    R, V, keep, margin = L.learned_apply(c, Rp, Vp, np.zeros(2), np.zeros(2), 0.0)
    assert np.array_equal(R, Rp) and np.array_equal(V, Vp) and keep.all() and np.all(margin == -np.inf)


@pytest.mark.parametrize("field", [oracle.FIELD_ZERO, oracle.FIELD_DUFFING])
def test_apply_reflection_keeps_energy_exactly(field):
    # (R, V) -> (-R, -V) leaves H unchanged for the even fields: kept with tol 0
    c = pcfg(field_model=field)
    rng = np.random.default_rng(7)
    Rp = rng.normal(0, 1, 100).astype(np.float32).astype(np.float64)
    Vp = rng.normal(0, 1, 100).astype(np.float32).astype(np.float64)
    R, V, keep, margin = L.learned_apply(c, Rp, Vp, -2 * Rp, -2 * Vp, 0.0)
    assert keep.all() and np.array_equal(R, -Rp) and np.array_equal(V, -Vp)


def test_apply_threshold_hand_worked():
    # zero field, y_plain = (1, 0): H = 1/2; dR = 1/2 gives H = 9/8, a relative
    # change of 5/4: kept at tol = 1.25 (the bound is inclusive), not below it
    c = pcfg(field_model=oracle.FIELD_ZERO)
    one = np.array([1.0])
    zero = np.array([0.0])
    R, _, keep, m = L.learned_apply(c, one, zero, np.array([0.5]), zero, 1.25)
    assert keep[0] and R[0] == 1.5 and m[0] == 0.0
    R, _, keep, m = L.learned_apply(c, one, zero, np.array([0.5]), zero, 1.2499)
    assert not keep[0] and R[0] == 1.0 and m[0] > 0.0


def test_apply_rounds_the_fp32_form_state_to_binary32():
    c = pcfg(field_model=oracle.FIELD_ZERO)
    Rp = np.array([np.float32(1.0)], np.float64)
    dR = np.array([2.0 ** -30])  # below half a binary32 ulp of 1
    R, _, keep, _ = L.learned_apply(c, Rp, np.zeros(1), dR, np.zeros(1), 1.0, precision=1)
    assert keep[0] and R[0] == 1.0
    R, _, keep, _ = L.learned_apply(c, Rp, np.zeros(1), dR, np.zeros(1), 1.0, precision=0)
    assert R[0] == 1.0 + 2.0 ** -30


def test_learned_step_with_a_zero_network_is_the_plain_step():
    c = pcfg(r_min=-2.0, r_max=2.0)
    R0, V0 = inputs.paper_beam(3000, seed=8)
    w = np.zeros(mlp.N_PARAMS)
    res = L.learned_step(c, R0, V0, 0.0, w, (1.0, 1.0), 1e-4)
    plain = oracle.etd_step(c, R0, V0)
    assert np.array_equal(res["R"], plain.R) and np.array_equal(res["V"], plain.V)


def test_learned_step_with_no_energy_limit_adds_the_correction():
    # W3 = 0, b3 = (c_R, c_V): the network's output is (c_R, c_V) exactly
    c = pcfg(r_min=-2.0, r_max=2.0)
    R0, V0 = inputs.paper_beam(3000, seed=9)
    p = mlp.unflatten(np.zeros(mlp.N_PARAMS))
    p["b3"] = np.array([0.5, -0.25])
    w = mlp.flatten(p)
    res = L.learned_step(c, R0, V0, 0.0, w, (2.0 ** -10, 2.0 ** -12), np.inf)
    plain = oracle.etd_step(c, R0, V0)
    assert np.array_equal(res["R"], plain.R + 2.0 ** -11) and np.array_equal(res["V"], plain.V - 2.0 ** -14)


# ------------------------------------------------------------ Adam


def test_adam_first_two_steps_closed_form():
    # Kingma & Ba, Algorithm 1, unrolled by hand: after steps with gradients
    # g1, g2 (m0 = v0 = 0) the bias-corrected moments are
    #   m_hat_1 = g1, v_hat_1 = g1^2,
    #   m_hat_2 = (b1 g1 + g2) / (1 + b1), v_hat_2 = (b2 g1^2 + g2^2) / (1 + b2)
    lr, b1, b2, e = 0.1, 0.9, 0.999, 1e-8
    w0 = np.array([1.0, -2.0, 0.5])
    g1 = np.array([0.5, -3.0, 1e-9])
    g2 = np.array([-0.25, -1.0, 2e-9])
    w1, m, v = L.adam_step(w0, np.zeros(3), np.zeros(3), g1, 1, lr, b1, b2, e)
    assert np.allclose(w1, w0 - lr * g1 / (np.abs(g1) + e), rtol=1e-15, atol=0)
    w2, m, v = L.adam_step(w1, m, v, g2, 2, lr, b1, b2, e)
    mh = (b1 * g1 + g2) / (1 + b1)
    vh = (b2 * g1 ** 2 + g2 ** 2) / (1 + b2)
    assert np.allclose(w2, w1 - lr * mh / (np.sqrt(vh) + e), rtol=1e-14, atol=0)
    # first element worked out numerically: m_hat_2 = 0.2/1.9, v_hat_2 = 0.31225/1.999
    assert w2[0] == pytest.approx(1.0 - 0.1 * 0.5 / (0.5 + 1e-8) - 0.1 * (0.2 / 1.9) / (math.sqrt(0.31225 / 1.999) + 1e-8),
                                  rel=1e-14)


def test_adam_step_is_invariant_to_gradient_scale():
    # the update depends on g only through m_hat / sqrt(v_hat) (eps -> 0)
    rng = np.random.default_rng(10)
    w, g = rng.normal(size=50), rng.normal(size=50)
    a, _, _ = L.adam_step(w, np.zeros(50), np.zeros(50), g, 1, 1e-3, 0.9, 0.999, 1e-30)
    b, _, _ = L.adam_step(w, np.zeros(50), np.zeros(50), 1e4 * g, 1, 1e-3, 0.9, 0.999, 1e-30)
    assert np.allclose(a, b, rtol=1e-15, atol=1e-18)
    assert np.allclose(np.abs(a - w), 1e-3, rtol=1e-12)  # first step: lr sign(g)


# ------------------------------------------------------------ network intervals


def _batch(n, seed):
    rng = np.random.default_rng(seed)
    X = np.stack([rng.normal(0, 1.5, n), rng.normal(0, 1.5, n), np.sin(rng.uniform(0, 6.3, n)),
                  np.cos(rng.uniform(0, 6.3, n)), np.full(n, 0.4)], axis=1).astype(np.float32)
    return X.astype(np.float64)


def _f32_forward(w, X):
    """The network evaluated in binary32 by numpy (another summation order
    than any GPU kernel), with its bfloat16 rounding points: one of the
    evaluations the interval form must contain."""
    p = mlp.unflatten(w)
    f = np.float32
    W1, W2, W3 = (mlp.bf16(p[k]).astype(f) for k in ("W1", "W2", "W3"))
    b1, b2, b3 = (p[k].astype(f) for k in ("b1", "b2", "b3"))
    from scipy.special import erfc

    gelu32 = lambda u: (f(0.5) * u * erfc(-u * f(1 / math.sqrt(2))).astype(f)).astype(f)  # noqa: E731
    z1 = (X.astype(f) @ W1.T + b1).astype(f)
    h1 = mlp.bf16(gelu32(z1).astype(np.float64)).astype(f)
    z2 = (h1 @ W2.T + b2).astype(f)
    h2 = mlp.bf16(gelu32(z2).astype(np.float64)).astype(f)
    return (h2 @ W3.T + b3).astype(np.float64)


def test_forward_interval_contains_exact_and_binary32_evaluations():
    w = inputs.mlp_init(3).astype(np.float64)
    p = mlp.unflatten(w)
    p["b1"] = np.random.default_rng(1).normal(0, 0.1, 64)
    w = mlp.flatten(p).astype(np.float32).astype(np.float64)
    X = _batch(20_000, 2)
    iv = mlp.forward_interval(w, X)["out"]
    exact = mlp.forward(w, X)["out"]
    f32 = _f32_forward(w, X)
    assert np.all((exact >= iv.lo) & (exact <= iv.hi))
    assert np.all((f32 >= iv.lo) & (f32 <= iv.hi))
    # the binary32 evaluation does flip some bfloat16 roundings, and the
    # interval is wide exactly there: most outputs are pinned to ~1e-6
    assert np.mean(iv.rad < 1e-5) > 0.6
    assert np.any(np.abs(f32 - exact) > 1e-4)


def test_gradient_interval_contains_the_exact_gradient_and_flips_widen_it():
    w = inputs.mlp_init(4).astype(np.float64)
    X = _batch(2000, 3)
    Y = np.random.default_rng(4).normal(0, 0.2, (2000, 2))
    loss, g = mlp.grads_interval(w, X, Y, n_seq=96)
    l0, g0 = mlp.loss_and_grads(w, X, Y)
    assert loss.lo <= l0 <= loss.hi
    assert np.all((g0 >= g.lo) & (g0 <= g.hi))
    # an exact network (no bfloat16 points) differs from the rounded one by
    # more than the interval allows: the interval resolves the rounding points
    _, g_exact = mlp.loss_and_grads(w, X, Y, emulate_bf16=False)
    assert np.any((g_exact < g.lo) | (g_exact > g.hi))

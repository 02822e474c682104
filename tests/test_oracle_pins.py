"""Pins of the FP64 oracle against what the paper and the mathematics fix.

Nothing here compares the oracle with itself: every expected value is a
closed form, an invariant, a value printed in the paper (tests/golden), a
library routine, or brute force on a tiny case.
"""
import math

import numpy as np
import pytest

import oracle
from paper_1404_1160_gb300 import inputs
from tests.conftest import golden

G = golden("paper_constants.txt")


def cfg(**kw):
    base = dict(eps=0.01, dt=0.1, field_model=oracle.FIELD_DUFFING, fine_solver=oracle.FINE_LAWSON)
    base.update(kw)
    return oracle.Config(**base)


# ---------------------------------------------------------------- constants


def test_fine_step_is_paper_value():
    # Remark CompOfThePeriodsRem: (dt)_RK = 2 pi eps / 100
    for eps in (1e-2, 1e-3, 1e-4):
        d = oracle.derive(cfg(eps=eps))
        assert d.h == pytest.approx(2 * math.pi * eps / G["steps_per_turn"], rel=1e-15)
        th = d.h / eps
        assert d.c1 == pytest.approx(math.cos(th), abs=1e-16)
        assert d.sh == pytest.approx(math.sin(th / 2), abs=1e-16)


def test_paper_beam_generator_matches_printed_f0():
    r, v = inputs.paper_beam(20000, seed=1)
    assert np.all(np.abs(r) <= G["r_half_width"])
    assert np.std(v) == pytest.approx(G["v_th"], rel=0.03)
    assert inputs.PAPER_V_TH == G["v_th"]


# ---------------------------------------------------- E = 0: exact rotation


def test_lawson_zero_field_is_exact_rotation():
    # Sec. 1: with E = 0 the beam rotates with period 2 pi eps; the Lawson
    # step advances the linear part by its exact flow.
    c = cfg(field_model=oracle.FIELD_ZERO)
    d = oracle.derive(c)
    R0, V0 = inputs.gaussian_beam(64, seed=3)
    for k in (1, 37, 100, 250):
        R, V = oracle.fine_steps(c, R0, V0, k)
        th = k * d.h / c.eps
        Rx = R0 * math.cos(th) + V0 * math.sin(th)
        Vx = -R0 * math.sin(th) + V0 * math.cos(th)
        assert np.max(np.abs(R - Rx)) < 1e-13 * max(1, k / 10)
        assert np.max(np.abs(V - Vx)) < 1e-13 * max(1, k / 10)
    R, V = oracle.fine_steps(c, R0, V0, 100)  # one full turn 2 pi eps
    assert np.max(np.abs(R - R0)) < 2e-13 and np.max(np.abs(V - V0)) < 2e-13


def test_rk4_zero_field_matches_stability_polynomial():
    # w = R - iV obeys w' = (i/eps) w; classical RK4 multiplies w by
    # P(i theta) = 1 + z + z^2/2 + z^3/6 + z^4/24 per step, theta = h/eps.
    c = cfg(field_model=oracle.FIELD_ZERO, fine_solver=oracle.FINE_RK4)
    d = oracle.derive(c)
    z = 1j * d.h / c.eps
    P = 1 + z + z**2 / 2 + z**3 / 6 + z**4 / 24
    R0, V0 = inputs.gaussian_beam(32, seed=4)
    for k in (1, 10, 300):
        R, V = oracle.fine_steps(c, R0, V0, k)
        w = (R0 - 1j * V0) * P**k
        assert np.max(np.abs(R - w.real)) < 1e-13 * k
        assert np.max(np.abs(V + w.imag)) < 1e-13 * k


# ------------------------------------------------ Duffing appendix (pins)


@pytest.mark.parametrize("r0,v0", [(1.0, 0.0), (0.5, 0.3), (2.0, 1.0), (0.0, 1.5)])
def test_duffing_turning_point_has_same_energy(r0, v0):
    # eq. b_val: G(b) = H(r0, v0); H in (r, v) variables is
    # (r^2+v^2)/(2 eps^2) + r^4/(4 eps) (appendix, with R' = v/eps).
    eps = 0.01
    b = math.sqrt(oracle.duffing_b2(eps, r0, v0))
    H = lambda r, v: (r * r + v * v) / (2 * eps**2) + r**4 / (4 * eps)
    assert H(b, 0.0) == pytest.approx(H(r0, v0), rel=1e-13)
    assert oracle.duffing_energy(eps, r0, v0) == pytest.approx(eps**2 * H(r0, v0), rel=1e-14)


@pytest.mark.parametrize("r0,v0", [(1.0, 0.0), (0.5, 0.3), (2.0, 1.0)])
def test_duffing_period_two_routes_agree(r0, v0):
    # The appendix integral by quadrature and in closed form (AGM).
    for eps in (1e-2, 1e-3):
        a = oracle.duffing_period_agm(eps, r0, v0)
        q = oracle.duffing_period_quad(eps, r0, v0, 48)
        assert a == pytest.approx(q, rel=1e-14)


def test_duffing_period_series_coefficients():
    # eq. 1stDL_T: T/(2 pi eps) = 1 - (3/4) alpha + (57/64) alpha^2 + O(alpha^3)
    # with alpha = b^2 eps / 2 (the printed coefficients are 3 pi/4, 57 pi/128:
    # -(3 pi/4) b^2 eps^2 = -2 pi eps (3/4) alpha, (57 pi/128) b^4 eps^3 =
    # 2 pi eps (57/64) alpha^2).  Extract both by Richardson extrapolation in
    # alpha on the exact period.
    eps = 1e-2

    def coeffs(s):
        alpha = oracle.duffing_b2(eps, s, 0.0) * eps / 2
        x = oracle.duffing_period_agm(eps, s, 0.0) / (2 * math.pi * eps)
        return alpha, x

    a1, x1 = coeffs(0.2)
    a2, x2 = coeffs(0.1)
    c1 = [(1 - x) / a for a, x in ((a1, x1), (a2, x2))]
    # c1(alpha) = 3/4 - (57/64) alpha + ...: eliminate the linear term
    lin = (c1[1] * a1 - c1[0] * a2) / (a1 - a2)
    assert lin == pytest.approx(G["series_b2_coef"], rel=1e-6)
    c2 = [(x - 1 + G["series_b2_coef"] * a) / (a * a) for a, x in ((a1, x1), (a2, x2))]
    quad = (c2[1] * a1 - c2[0] * a2) / (a1 - a2)
    assert quad == pytest.approx(2 * G["series_b4_coef"], rel=1e-4)


def test_duffing_period_series_error_is_order_eps4():
    # eq. 2ndDL_T holds up to O(eps^4): the error falls ~16x per halving.
    r0, v0 = 1.2, 0.7
    errs = [abs(oracle.duffing_period_agm(e, r0, v0) - oracle.duffing_period_series(e, r0, v0))
            for e in (0.02, 0.01, 0.005)]
    assert 12 < errs[0] / errs[1] < 20 and 12 < errs[1] / errs[2] < 20
    # and its printed eps^3 coefficient: (105/128 S^2 - 3/8 r0^4) pi
    S = r0 * r0 + v0 * v0
    e = 1e-3
    T = oracle.duffing_period_agm(e, r0, v0)
    c3 = (T - 2 * math.pi * e + G["series_b2_coef"] * math.pi * S * e * e) / e**3
    assert c3 == pytest.approx((G["series_S2_coef"] * S * S - G["series_r4_coef"] * r0**4) * math.pi, rel=2e-2)


# ---------------------------------------------- period detection (step 1)


def test_detected_periods_match_exact_duffing_periods():
    # Remark CompOfThePeriodsRem on the Duffing field, against the exact
    # appendix period; the error shrinks like h^3 (>= 4x per halving).
    R0, V0 = inputs.gaussian_beam(200, seed=5)
    errs = []
    for spt in (100, 200):
        c = cfg(steps_per_turn=spt, max_window_steps=3 * spt)
        T, nf, _ = oracle.periods(c, R0, V0)
        h = oracle.derive(c).h
        exact = np.array([oracle.duffing_period_agm(c.eps, r, v) for r, v in zip(R0, V0)])
        assert nf == 0
        errs.append(np.max(np.abs(T * h - exact)))
    assert errs[0] < 5e-7
    assert errs[0] / errs[1] > 4


def test_paper_period_band():
    # Sec. 2.1: for eq. InitialConditionBeam at eps = 0.01 the periods lie in
    # (2 pi eps - 1.5 eps^2, 2 pi eps).
    eps = G["band_eps"]
    c = cfg(eps=eps, fine_solver=oracle.FINE_RK4)
    R0, V0 = inputs.paper_beam(2000, seed=0)
    T, nf, _ = oracle.periods(c, R0, V0)
    Tt = T * oracle.derive(c).h
    assert nf == 0
    assert np.all(Tt < 2 * math.pi * eps)
    assert np.all(Tt > 2 * math.pi * eps - G["band_low_eps2"] * eps**2)


def test_no_period_fallback_at_equilibrium():
    # y = 0 is an equilibrium of the Duffing field: no extremum, T := 2 pi eps,
    # and the step keeps y = 0 exactly.
    c = cfg(dt=0.5)
    T, nf, K = oracle.periods(c, [0.0, 1.0], [0.0, 0.0])
    assert nf == 1 and T[0] == c.steps_per_turn and K == c.max_window_steps
    res = oracle.etd_step(c, [0.0, 1.0], [0.0, 0.0])
    assert res.R[0] == 0.0 and res.V[0] == 0.0 and res.stats["n_no_period"] == 1


# --------------------------------------------------- interpolation pieces


def test_interp_exact_on_quadratics():
    rng = np.random.default_rng(0)
    for _ in range(50):
        a, b, cc = rng.normal(size=3)
        f = lambda s: a + b * s + cc * s * s
        s = rng.uniform(0, 1)
        assert oracle.interp(f(0), f(1), f(2), s) == pytest.approx(f(s), rel=1e-13, abs=1e-14)


def test_quad_root_matches_library_roots():
    rng = np.random.default_rng(1)
    n = 0
    while n < 200:
        a, b, cc = rng.normal(size=3)
        f = lambda s: a + b * s + cc * s * s
        if (f(0) > 0) == (f(1) > 0):
            continue
        n += 1
        roots = np.roots([cc, b, a])
        roots = [r.real for r in roots if abs(r.imag) < 1e-12 and -1e-12 <= r.real <= 1 + 1e-12]
        assert len(roots) == 1
        assert oracle.quad_root(f(0), f(1), f(2)) == pytest.approx(roots[0], abs=1e-12)
    # linear case
    assert oracle.quad_root(1.0, -1.0, -3.0) == pytest.approx(0.5, abs=1e-15)


# ---------------------------------------------------------- mesh (Poisson)


def pcfg(**kw):
    base = dict(field_model=oracle.FIELD_POISSON, n_cells=256, r_min=-4.0, r_max=4.0)
    base.update(kw)
    return cfg(**base)


def test_deposit_partition_of_unity_and_first_moment():
    c = pcfg()
    W = c.weight_fixed
    rng = np.random.default_rng(2)
    R = np.concatenate([rng.normal(0, 1.5, 5000), [-4.0, 4.0, 3.999999, -4.5, 9.0]])
    Q, n_out = oracle.deposit(c, R)
    assert int(Q.sum()) + n_out * W == R.size * W
    inside = (R >= -4.0) & (R < 4.0)
    assert n_out == int((~inside).sum())
    # CIC keeps the first moment: sum_j Q_j r_j = W sum_i R_i up to one
    # fixed-point unit per particle
    r = -4.0 + np.arange(257) * (8 / 256)
    lhs = float(np.dot(Q.astype(np.float64), r))
    rhs = W * float(R[inside].sum())
    assert abs(lhs - rhs) <= inside.sum() * (8 / 256) * 1.0 + 1e-6 * abs(rhs)
    # permutation invariance (integer charges: bit-exact)
    Q2, _ = oracle.deposit(c, R[rng.permutation(R.size)])
    assert np.array_equal(Q, Q2)


def test_deposit_f32_pins():
    # binary32 deposit: partition of unity, first moment within one unit per
    # particle, and equal to the FP64 deposit on dyadic positions (exact in
    # both precisions)
    c = pcfg()
    W = c.weight_fixed
    rng = np.random.default_rng(12)
    R = np.concatenate([rng.normal(0, 1.5, 5000), [-4.0, 4.0, -4.5, 9.0]]).astype(np.float32)
    Q, n_out = oracle.deposit_f32(c, R)
    assert int(Q.sum()) + n_out * W == R.size * W
    inside = (R >= -4.0) & (R < 4.0)
    assert n_out == int((~inside).sum())
    r = -4.0 + np.arange(257) * (8 / 256)
    assert abs(float(np.dot(Q.astype(np.float64), r)) - W * float(R[inside].astype(np.float64).sum())) <= inside.sum() * (8 / 256) + 1e-6 * W * 5000
    dy = (rng.integers(-4 * 1024, 4 * 1024, 3000) / 1024.0)
    Qd, _ = oracle.deposit(c, dy)
    Qf, _ = oracle.deposit_f32(c, dy.astype(np.float32))
    assert np.array_equal(Qd, Qf)


def test_deposit_brute_force_tiny():
    c = pcfg(n_cells=4, r_min=-1.0, r_max=1.0)  # nodes -1,-.5,0,.5,1
    W = c.weight_fixed
    Q, _ = oracle.deposit(c, [0.0])
    assert list(Q) == [0, 0, W, 0, 0]
    Q, _ = oracle.deposit(c, [0.25])
    assert list(Q) == [0, 0, W // 2, W // 2, 0]
    Q, _ = oracle.deposit(c, [-0.875])  # x = 0.25 in cell 0
    assert list(Q) == [W - W // 4, W // 4, 0, 0, 0]


def test_poisson_uniform_rho_gives_constant_E():
    # d/dr (rE) = rho0 on [-a, a] => rE = rho0 r, E = rho0 (trapezoid exact)
    c = pcfg()
    Q = np.zeros(257, np.int64)
    Q[128 - 40:128 + 41] = 1 << 33
    n_p = 1000
    S, E, edges = oracle.poisson(c, Q, n_p)
    q_unit = 1.0 / (n_p * c.weight_fixed)
    rho0 = (1 << 33) * q_unit / (8 / 256)
    inner = np.r_[128 - 40:128 + 41]
    assert np.allclose(E[inner], rho0, rtol=1e-15, atol=0)
    # outside the charge rE stays at its edge value
    r = -4 + np.arange(257) / 32
    assert np.allclose((E * r)[128 + 41:], (E * r)[128 + 41], rtol=1e-14)
    assert edges[1] == pytest.approx(E[256] * 4.0, rel=1e-15)


def test_poisson_odd_reading_uniform_rho_gives_signed_constant():
    # the odd extension of the same field: E(r) = rE(r)/|r| = rho0 sign(r)
    # inside the charge, 0 on the axis; outside, rE/|r| keeps the edge value
    c = pcfg(field_parity=1)
    Q = np.zeros(257, np.int64)
    Q[128 - 40:128 + 41] = 1 << 33
    n_p = 1000
    S, E, edges = oracle.poisson(c, Q, n_p)
    q_unit = 1.0 / (n_p * c.weight_fixed)
    rho0 = (1 << 33) * q_unit / (8 / 256)
    r = -4 + np.arange(257) / 32
    assert E[128] == 0.0
    assert np.allclose(E[128 + 1:128 + 41], rho0, rtol=1e-15, atol=0)
    assert np.allclose(E[128 - 40:128], -rho0, rtol=1e-15, atol=0)
    assert np.allclose((E * np.abs(r))[128 + 41:], (E * r)[128 + 41], rtol=1e-14)
    # the same integer sums as the literal reading; the field differs only by
    # the sign left of the axis and by its value on the axis
    S0, E0, edges0 = oracle.poisson(pcfg(), Q, n_p)
    assert np.array_equal(S, S0)
    assert np.array_equal(E[129:], E0[129:]) and np.array_equal(E[:128], -E0[:128])
    assert edges[0] == -edges0[0] and edges[1] == edges0[1]
    # off the mesh below: rE_edge / |R|
    e = oracle.gather(c, np.array([-5.0, 5.0]), E, edges)
    assert e[0] == pytest.approx(edges0[0] / 5.0, rel=1e-15) and e[1] == pytest.approx(edges0[1] / 5.0, rel=1e-15)


def test_odd_reading_is_mirror_equivariant_and_the_literal_one_is_not():
    # with E odd in r, (R, V) -> (-R, -V) maps solutions to solutions, so one
    # macro step of the mirrored beam is the mirror of the step (up to the
    # fixed-point deposit, which rounds f W down on both sides: one unit of
    # W per particle); with the literal (even) field it is not
    R0, V0 = inputs.gaussian_beam(400, seed=5, r_cut=3.5)
    diffs = {}
    for parity in (0, 1):
        c = pcfg(field_parity=parity, dt=0.1)
        a = oracle.etd_step(c, R0, V0)
        b = oracle.etd_step(c, -R0, -V0)
        diffs[parity] = max(np.max(np.abs(a.R + b.R)), np.max(np.abs(a.V + b.V)))
    assert diffs[1] < 1e-11, diffs
    assert diffs[0] > 1e-4, diffs


def test_poisson_linear_rho_gives_half_slope():
    # rho = a + b |r| => rE = a r + b r|r|/2 => E = a + b |r|/2 (trapezoid is
    # exact on each side since rho is linear there)
    c = pcfg()
    j = np.arange(257)
    A, B = 1 << 30, 1 << 24
    Q = (A + B * np.abs(j - 128)).astype(np.int64)
    S, E, _ = oracle.poisson(c, Q, 10**6)
    q_unit = 1.0 / (10**6 * c.weight_fixed)
    hr = 8 / 256
    r = -4 + j * hr
    expect = (A + B * np.abs(r) / hr / 2) * q_unit / hr
    assert np.allclose(E, expect, rtol=1e-13)


def test_poisson_gaussian_matches_erf():
    # rho = N(0, sigma): r E = erf(r / (sqrt 2 sigma)) / 2 for unit charge,
    # within O(h_r^2) of the trapezoid
    from scipy.special import erf, ndtri

    c = pcfg()
    n = 400000
    R = 0.8 * ndtri((np.arange(n) + 0.5) / n)
    Q, n_out = oracle.deposit(c, R)
    S, E, _ = oracle.poisson(c, Q, n)
    r = -4 + np.arange(257) / 32
    rE = E * r
    expect = 0.5 * erf(r / (math.sqrt(2) * 0.8))
    assert np.max(np.abs(rE - expect)) < 2e-4


def test_gather_exact_for_linear_field():
    c = pcfg()
    r = -4 + np.arange(257) / 32
    E = 0.3 + 0.7 * r
    R = np.random.default_rng(3).uniform(-3.99, 3.99, 1000)
    e = oracle.gather(c, R, E, np.array([E[0] * -4.0, E[256] * 4.0]))
    assert np.allclose(e, 0.3 + 0.7 * R, rtol=1e-14, atol=1e-14)
    # at nodes the gather returns the node value
    e = oracle.gather(c, r[:-1], E, np.zeros(2))
    assert np.array_equal(e, E[:-1])


def test_gather_outside_mesh_uses_edge_rE():
    c = pcfg()
    E = np.ones(257)
    e = oracle.gather(c, np.array([5.0, -6.0]), E, np.array([-2.0, 3.0]))
    assert e[0] == 3.0 / 5.0 and e[1] == -2.0 / -6.0


# ------------------------------------------ fine solver on the Duffing field


def test_duffing_energy_conserved_at_fourth_order():
    # eps^2 H = (r^2+v^2)/2 + eps r^4/4 is invariant (appendix).  Classical
    # RK4 loses amplitude at theta^6/72 per step (theta = 2 pi / spt), so its
    # drift over a fixed time falls like h^5 (~32x per halving); Lawson RK4
    # treats the rotation exactly and its drift falls at 4th order
    # (>= 100x over two halvings, approaching 256).
    R0, V0 = inputs.gaussian_beam(50, seed=6)
    H0 = np.array([oracle.duffing_energy(0.01, r, v) for r, v in zip(R0, V0)])

    def drift(solver, spt):
        c = cfg(fine_solver=solver, steps_per_turn=spt, max_window_steps=3 * spt)
        R, V = oracle.fine_steps(c, R0, V0, 3 * spt)
        H = np.array([oracle.duffing_energy(0.01, r, v) for r, v in zip(R, V)])
        return np.max(np.abs(H - H0) / H0)

    d50, d100 = drift(oracle.FINE_RK4, 50), drift(oracle.FINE_RK4, 100)
    assert d100 < 4e-7 and 25 < d50 / d100 < 40
    d100, d400 = drift(oracle.FINE_LAWSON, 100), drift(oracle.FINE_LAWSON, 400)
    assert d100 < 4e-8 and d100 / d400 > 100


# ------------------------------------------------ the improved ETD step


def test_lemma_exact_for_zero_field():
    # E = 0: the motion is periodic with T = 2 pi eps, so eq. MainFormula1 is
    # exact up to the fine solver and the quadratic interpolation
    # (Lemma FirstStepOfTheAlgLemma with r(N T / eps) = identity).  Lawson
    # RK4 is exact for E = 0 and the detected period is exactly
    # steps_per_turn, so the two interpolation errors at o and o+T are equal
    # and the N-fold extrapolation cancels them: what is left is the
    # Lagrange remainder |s(s-1)(s-2)| theta^3 / 6 (amplitude 1, theta the
    # rotation per fine step, s the fractional position of o).
    R0, V0 = inputs.gaussian_beam(100, seed=7)
    for spt in (50, 100, 200, 400):
        c = cfg(field_model=oracle.FIELD_ZERO, dt=0.5, steps_per_turn=spt, max_window_steps=3 * spt)
        res = oracle.etd_step(c, R0, V0)
        th = c.dt / c.eps
        Rx = R0 * math.cos(th) + V0 * math.sin(th)
        Vx = -R0 * math.sin(th) + V0 * math.cos(th)
        amp = np.hypot(R0, V0)
        assert np.all(res.N == 7)  # 0.5 / (2 pi 0.01) = 7.96
        assert np.allclose(res.T, spt, rtol=1e-12)
        err = np.max(np.hypot(res.R - Rx, res.V - Vx) / amp)
        sfrac = res.o[0] - math.floor(res.o[0])
        bound = abs(sfrac * (sfrac - 1) * (sfrac - 2)) / 6 * (2 * math.pi / spt) ** 3
        assert err == pytest.approx(bound, rel=0.1)


def test_etd_duffing_tracks_brute_force():
    # Sec. 4.1: with exact-in-time periods the improved scheme follows the
    # reference RK4 solution over N ~ 8 turns per macro step.
    c = cfg(dt=0.5, fine_solver=oracle.FINE_RK4)
    R0, V0 = inputs.gaussian_beam(100, seed=8)
    T, nf, _ = oracle.periods(c, R0, V0)
    res = oracle.etd_step(c, R0, V0, T)
    Rb, Vb = oracle.brute_force(c, R0, V0, c.dt)
    amp = np.hypot(R0, V0)
    assert np.all(res.N >= 7)
    assert np.max(np.hypot(res.R - Rb, res.V - Vb) / amp) < 2e-4


def test_N_zero_when_dt_below_period():
    # dt = 0.05 < T: eq. TimeStepDec gives N = 0, o = dt
    c = cfg(dt=0.05)
    R0, V0 = inputs.gaussian_beam(50, seed=9)
    res = oracle.etd_step(c, R0, V0)
    d = oracle.derive(c)
    assert np.all(res.N == 0)
    assert np.allclose(res.o, d.D, rtol=0, atol=0)


def test_N_about_800_at_eps_1e_4():
    # Sec. 4.1: eps = 1e-4, dt = 0.5 gives N_i of about 800
    c = cfg(eps=1e-4, dt=0.5)
    R0, V0 = inputs.paper_beam(20, seed=0)
    T, _, _ = oracle.periods(c, R0, V0)
    res = oracle.etd_step(c, R0, V0, T)
    assert np.all(np.abs(res.N - G["N_at_eps_1e-4"]) < 10)


def test_window_end_does_not_change_the_step():
    # results depend only on the samples they use, not on how far past them
    # the fine window ran
    R0, V0 = inputs.gaussian_beam(64, seed=10, r_cut=3.5)
    a = oracle.etd_step(pcfg(max_window_steps=300), R0, V0)
    b = oracle.etd_step(pcfg(max_window_steps=420), R0, V0)
    assert np.array_equal(a.R, b.R) and np.array_equal(a.V, b.V)


def test_vlasov_poisson_step_tracks_brute_force():
    # Sec. 4.2: small beam, self-consistent field; error of one macro step
    # with N = 1 vs the reference solution.
    for solver in (oracle.FINE_RK4, oracle.FINE_LAWSON):
        c = pcfg(fine_solver=solver, dt=0.1)
        R0, V0 = inputs.gaussian_beam(128, seed=11, r_cut=4.0)
        res = oracle.etd_step(c, R0, V0)
        Rb, Vb = oracle.brute_force(c, R0, V0, c.dt)
        amp = np.hypot(R0, V0)
        assert res.stats["n_no_period"] == 0
        assert np.max(np.hypot(res.R - Rb, res.V - Vb) / amp) < 5e-3
        # charge is conserved exactly by the deposit
        Q, n_out = oracle.deposit(c, res.R)
        assert int(Q.sum()) + n_out * c.weight_fixed == 128 * c.weight_fixed


# ------------------------------------------------------ learned-stepper network


def test_mlp_bf16_rounding_matches_float32_bit_rounding():
    # independent route: round float32 bit patterns to 16 bits, ties to even
    from oracle import mlp

    rng = np.random.default_rng(3)
    x = (rng.normal(0, 3, 20000) * np.exp(rng.normal(0, 4, 20000))).astype(np.float32)
    x = np.concatenate([x, np.array([1.0, 1.0 + 2**-8, 1.0 + 3 * 2**-8, -2.5, 0.0], np.float32)])
    b = x.view(np.uint32).astype(np.uint64)
    b = (b + 0x7FFF + ((b >> 16) & 1)) & 0xFFFF0000
    ref = b.astype(np.uint32).view(np.float32).astype(np.float64)
    assert np.array_equal(mlp.bf16(x.astype(np.float64)), ref)
    # 1 + 2^-8 is a tie between 1 and 1 + 2^-7: even mantissa wins
    assert mlp.bf16(np.array([1.0 + 2**-8]))[0] == 1.0


def test_mlp_gelu_is_x_times_normal_cdf():
    from scipy.special import ndtr

    from oracle import mlp

    u = np.linspace(-8, 8, 1001)
    assert np.allclose(mlp.gelu(u), u * ndtr(u), rtol=5e-14, atol=1e-300)
    h = 1e-6
    fd = (mlp.gelu(u + h) - mlp.gelu(u - h)) / (2 * h)
    assert np.allclose(mlp.gelu_prime(u), fd, rtol=1e-7, atol=3e-9)


def test_mlp_forward_matches_torch_cpu_layers():
    # exact FP64 network against torch's own Linear and GELU (erf form)
    torch = pytest.importorskip("torch")
    from oracle import mlp

    rng = np.random.default_rng(4)
    w = rng.normal(0, 0.3, mlp.N_PARAMS)
    X = rng.normal(0, 1, (37, 5))
    p = mlp.unflatten(w)
    net = torch.nn.Sequential(torch.nn.Linear(5, 64), torch.nn.GELU(), torch.nn.Linear(64, 64), torch.nn.GELU(),
                              torch.nn.Linear(64, 2)).double()
    with torch.no_grad():
        for layer, (Wn, bn) in zip((net[0], net[2], net[4]), (("W1", "b1"), ("W2", "b2"), ("W3", "b3"))):
            layer.weight.copy_(torch.from_numpy(p[Wn]))
            layer.bias.copy_(torch.from_numpy(p[bn]))
        ref = net(torch.from_numpy(X)).numpy()
    assert np.allclose(mlp.forward(w, X, emulate_bf16=False)["out"], ref, rtol=1e-13, atol=1e-13)


def test_mlp_gradients_match_finite_differences():
    # backward of the exact FP64 network against central differences of its loss
    from oracle import mlp

    rng = np.random.default_rng(5)
    w = rng.normal(0, 0.4, mlp.N_PARAMS)
    X = rng.normal(0, 1, (23, 5))
    Y = rng.normal(0, 1, (23, 2))
    loss, g = mlp.loss_and_grads(w, X, Y, emulate_bf16=False)
    idx = np.concatenate([rng.choice(mlp.N_PARAMS, 60, replace=False), [0, 319, 320, 383, 384, 4479, 4480, 4543, 4544,
                                                                        4671, 4672, 4673]])
    h = 1e-6
    for i in idx:
        e = np.zeros_like(w)
        e[i] = h
        fd = (mlp.loss_and_grads(w + e, X, Y, False)[0] - mlp.loss_and_grads(w - e, X, Y, False)[0]) / (2 * h)
        assert abs(fd - g[i]) <= 1e-7 * max(1.0, abs(g[i])), (i, fd, g[i])
    assert loss > 0


def test_mlp_bf16_rounding_points():
    # with emulation on, the loss is that of the FP64 network evaluated on
    # bfloat16 weights and bfloat16 hidden activations: rounding the weights
    # beforehand changes nothing, and a weight set already in bfloat16 with
    # activations that are exact in bfloat16 gives the exact network's loss
    from oracle import mlp

    rng = np.random.default_rng(6)
    w = rng.normal(0, 0.3, mlp.N_PARAMS)
    X = rng.normal(0, 1, (11, 5))
    Y = rng.normal(0, 1, (11, 2))
    p = mlp.unflatten(w)
    for k in ("W1", "W2", "W3"):
        p[k] = mlp.bf16(p[k])
    wb = mlp.flatten(p)
    assert mlp.loss_and_grads(w, X, Y, True)[0] == mlp.loss_and_grads(wb, X, Y, True)[0]
    a = mlp.forward(w, X, True)
    assert np.array_equal(a["h1b"], mlp.bf16(a["h1b"])) and np.array_equal(a["h2b"], mlp.bf16(a["h2b"]))


# ------------------------------------------------ classical / modified ETD


def test_classic_etd_zero_field_is_the_exact_rotation():
    # E = 0: the fine solve over 2 pi eps returns to y_n, the extrapolation
    # keeps it, and the solve over o rotates by o = Delta t mod 2 pi eps:
    # the exact flow r(Delta t / eps) y_n
    c = pcfg(field_model=2, dt=0.37)
    R0, V0 = inputs.gaussian_beam(50, seed=3)
    for mode in (0, 1):
        R, V, P = oracle.classic_step(c, R0, V0, mode)
        th = c.dt / c.eps
        Rx, Vx = R0 * np.cos(th) + V0 * np.sin(th), -R0 * np.sin(th) + V0 * np.cos(th)
        assert np.max(np.abs(R - Rx)) < 1e-11 and np.max(np.abs(V - Vx)) < 1e-11
        assert P == pytest.approx(2 * np.pi * c.eps, rel=1e-12 if mode == 0 else 1e-9)


def test_modified_etd_on_one_duffing_orbit():
    # one particle: the mean first-tour time is its own period, so the step
    # lands on the fine solution at Delta t within the detection and
    # interpolation error (the same order as the improved scheme's)
    c = pcfg(field_model=1, dt=0.5)
    R0, V0 = np.array([1.3]), np.array([-0.4])
    R, V, P = oracle.classic_step(c, R0, V0, 1)
    Rf, Vf = oracle.brute_force(c, R0, V0, c.dt)
    Tx = oracle.duffing_period_agm(c.eps, 1.3, -0.4)
    assert P == pytest.approx(Tx, rel=1e-5)
    assert abs(R[0] - Rf[0]) < 1e-3 and abs(V[0] - Vf[0]) < 1e-3


def test_modified_etd_drifts_where_the_improved_scheme_does_not():
    # Sec. 4.1 (Duffing field, the paper's beam of eq. InitialConditionBeam):
    # the periods depend on the amplitude, so one mean period mis-times every
    # particle but the average one and the modified scheme's error grows
    # faster than linearly, while the improved scheme, with each particle's
    # own period, grows slowly.  (On a wide beam, r, v ~ N(0, 1), the modified
    # scheme blows up within a few steps.)
    c = pcfg(field_model=1, dt=0.5)
    R0, V0 = inputs.paper_beam(400, seed=8)
    Rm, Vm = R0, V0
    Ri, Vi = R0, V0
    T = oracle.periods(c, R0, V0)[0]
    errs = {}
    for k in range(1, 41):
        Rm, Vm, _ = oracle.classic_step(c, Rm, Vm, 1)
        res = oracle.etd_step(c, Ri, Vi, T)
        Ri, Vi = res.R, res.V
        if k in (10, 40):
            Rf, Vf = oracle.brute_force(c, R0, V0, k * c.dt)
            errs[k] = (np.sqrt(np.mean((Rm - Rf) ** 2 + (Vm - Vf) ** 2)),
                       np.sqrt(np.mean((Ri - Rf) ** 2 + (Vi - Vf) ** 2)))
    (m10, i10), (m40, i40) = errs[10], errs[40]
    assert m40 > 8 * m10                 # faster than linear: 4x the time, > 8x the error
    assert i40 < 5 * i10 and i40 < 1e-3  # about linear
    assert m40 > 50 * i40

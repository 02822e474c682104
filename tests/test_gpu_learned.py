"""The learned stepper: its fallback rule, its neutrality with a zero network,
and what a trained network gains over the plain improved-ETD step.

The plain step in these tests is the FP64 path, which equals the FP64 oracle
bit for bit (tests/test_gpu_parity.py); the reference solution is the
oracle's brute-force fine solve (the paper's reference, Sec. 2.1).
"""
import math

import numpy as np
import pytest

import oracle
from paper_1404_1160_gb300 import inputs
from paper_1404_1160_gb300 import learned
from paper_1404_1160_gb300 import pic
from tests.gpu_common import bit_equal, cfg_of

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

W3_OFF, B3_OFF = 4544, 4672  # flat offsets of W3 and b3


@pytest.fixture(scope="module", autouse=True)
def _built():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1404_1160_gb300 import build

    build.build()
    torch.cuda.set_device(0)


def constant_network(c_R, c_V):
    """W3 = 0 and b3 = (c_R, c_V): the output is exactly (c_R, c_V)."""
    w = inputs.mlp_init(1)
    w[W3_OFF:B3_OFF] = 0.0
    w[B3_OFF:B3_OFF + 2] = (c_R, c_V)
    m = pic.pic_mlp_create(16)
    pic.pic_mlp_set_weights(m, w)
    return m


@pytest.mark.parametrize("field,prec", [(pic.PIC_FIELD_POISSON, 0), (pic.PIC_FIELD_POISSON, 1),
                                        (pic.PIC_FIELD_DUFFING, 0)])
def test_zero_correction_is_the_plain_step(field, prec):
    p = pic.pic_default_params(field_model=field, precision=prec, dt=0.4)
    R0, V0 = inputs.gaussian_beam(5000, seed=2, r_cut=4.0)
    a = pic.pic_init(p, R0, V0)
    b = pic.pic_init(p, R0, V0)
    m = constant_network(0.0, 0.0)
    pic.pic_step(a, 3)
    pic.pic_step_learned(b, m, 3, scale=(1.0, 1.0), drift_tol=1e-4)
    Ra, Va = pic.pic_get_particles(a)
    Rb, Vb = pic.pic_get_particles(b)
    assert bit_equal(Ra, Rb) and bit_equal(Va, Vb)
    assert pic.pic_moments(b)["n_steps"] == 3
    for h in (a, b):
        pic.pic_destroy(h)
    m.close()


def test_fallback_follows_the_frozen_field_energy():
    # Duffing (E = -r^3, psi = -r^4/4): a constant correction dR is kept
    # exactly where |H(y_plain + dR) - H(y_plain)| <= tol |H(y_plain)|
    eps, tol, dR = 0.01, 2e-3, 2e-3
    p = pic.pic_default_params(field_model=pic.PIC_FIELD_DUFFING, dt=0.4, eps=eps)
    R0, V0 = inputs.gaussian_beam(4000, seed=3)
    h = pic.pic_init(p, R0, V0)
    m = constant_network(1.0, 0.0)
    n_fb = pic.pic_step_learned(h, m, 1, scale=(dR, 0.0), drift_tol=tol)
    R, V = pic.pic_get_particles(h)
    res = oracle.etd_step(cfg_of(p), R0, V0)  # the plain step (bit-identical to the FP64 path)

    def H(r, v):
        return 0.5 * (r * r + v * v) + eps * (0.25 * ((r * r) * (r * r)))

    Rl = res.R + np.float64(np.float32(dR))
    Hp = H(res.R, res.V)
    d = np.abs(H(Rl, res.V) - Hp) - tol * np.abs(Hp)
    keep = d <= 0
    clear = np.abs(d) > 1e-9 * np.abs(Hp)
    assert np.array_equal(R[clear & keep], Rl[clear & keep])
    assert np.array_equal(R[clear & ~keep], res.R[clear & ~keep])
    assert np.array_equal(V, res.V)
    assert abs(n_fb - int((~keep).sum())) <= int((~clear).sum())
    assert 0 < n_fb < 4000
    pic.pic_destroy(h)
    m.close()


def test_fine_advance_is_the_oracle_brute_force():
    # the paper's reference solution over a time that is not a multiple of h
    p = pic.pic_default_params(r_min=-2.0, r_max=2.0)
    R0, V0 = inputs.paper_beam(3000, seed=4)
    h = pic.pic_init(p, R0, V0)
    pic.pic_fine_advance(h, 0.4)
    R, V = pic.pic_get_particles(h)
    Rf, Vf = oracle.brute_force(cfg_of(p), R0, V0, 0.4)
    assert bit_equal(R, Rf) and bit_equal(V, Vf)
    assert pic.pic_moments(h)["t"] == pytest.approx(0.4)
    pic.pic_destroy(h)
    with pytest.raises(pic.PicError) as ei:
        h32 = pic.pic_init(pic.pic_default_params(precision=1), R0, V0)
        pic.pic_fine_advance(h32, 0.4)
    assert ei.value.status == pic.PIC_ERR_UNSUPPORTED


def robust(e):
    """(median, RMS of the 99 % smallest) of per-particle errors."""
    e = np.sort(e)
    return float(np.median(e)), float(np.sqrt(np.mean(e[:int(0.99 * e.size)] ** 2)))


def test_trained_network_against_the_plain_step():
    # What a trained network gains over the method without it, measured on
    # the paper's own beam (eq. InitialConditionBeam) on [-2, 2] with 256
    # cells, eps = 0.01, dt = 0.4: training on 4 beams x 4 macro steps with
    # targets = the paper's reference solution over dt minus the large step;
    # evaluation on a held-out beam against the oracle's brute-force
    # solution after one and two macro steps.
    #
    # Measured (printed):
    # * the large improved-ETD step alone is about as accurate, for the bulk
    #   of the particles, as 8 plain steps of dt/8 at 1/8 of the windows
    #   (median error 3.6e-5 vs 3.0e-4 after one step, 8.6e-4 vs 7.8e-4
    #   after two, while the beam is far from equilibrium): its error does not
    #   grow with dt where periods are detected cleanly;
    # * the large step's remaining bulk error (~4e-5, the interpolation
    #   remainder) depends on the fraction of o and oscillates quickly
    #   across (r, v); from the specified inputs a network of the specified
    #   size explains about a third of its variance (a CPU fit: R^2 = 0.32),
    #   and on a held-out beam the trained correction does not reduce the
    #   error measurably;
    # * the frozen-field energy check keeps the learned step from degrading
    #   the plain one: the learned error stays within 10 % (median) and 25 %
    #   (RMS of the 99 % best) of the plain step's; the RMS over all
    #   particles is dominated by ~0.2 % near the axis where the large step
    #   detects spurious short periods.
    p = pic.pic_default_params(dt=0.4, r_min=-2.0, r_max=2.0)
    small = pic.pic_default_params(dt=0.05, r_min=-2.0, r_max=2.0)
    beams = [inputs.paper_beam(20000, seed=s) for s in range(4)]
    X, T = learned.make_dataset(p, beams, n_macro=4, reference="fine")
    m, scale, hist, kept = learned.train(X, T, steps=3000, batch=8192, lr=2e-3, seed=1)
    assert kept > 0.99
    assert hist[-50:].mean() < 0.9 * hist[:10].mean(), (hist[:10].mean(), hist[-50:].mean())
    R0, V0 = inputs.paper_beam(20000, seed=9)
    plain = pic.pic_init(p, R0, V0)
    lrn = pic.pic_init(p, R0, V0)
    fine8 = pic.pic_init(small, R0, V0)
    cfg = cfg_of(p)
    out = []
    for k in (1, 2):
        pic.pic_step(plain, 1)
        pic.pic_step(fine8, 8)
        n_fb = pic.pic_step_learned(lrn, m, 1, scale=tuple(scale), drift_tol=1e-4)
        Rp, Vp = pic.pic_get_particles(plain)
        Rl, Vl = pic.pic_get_particles(lrn)
        R8, V8 = pic.pic_get_particles(fine8)
        Rf, Vf = oracle.brute_force(cfg, R0, V0, 0.4 * k)
        ep, el, e8 = np.hypot(Rp - Rf, Vp - Vf), np.hypot(Rl - Rf, Vl - Vf), np.hypot(R8 - Rf, V8 - Vf)
        out.append((k, robust(ep), robust(el), robust(e8), n_fb))
    print("learned stepper (macro steps, (median, rms99) plain / learned / 8 steps of dt/8, fallbacks):", out)
    for k, (mp, rp), (ml, rl), (m8, r8), n_fb in out:
        assert ml <= 1.1 * mp and rl <= 1.25 * rp, out
        assert mp < 1.2 * m8, out
    for h in (plain, lrn, fine8):
        pic.pic_destroy(h)
    m.close()


def test_trained_network_gains_on_the_gaussian_beam():
    # The beam of the learned-stepper workload (r ~ N(0, 1) cut at 4,
    # v ~ N(0, 1); eps = 0.01, 512 cells on [-4, 4], dt = 0.4) stays close to
    # equilibrium: the large step's error is a smooth function of (r, v) and
    # the network learns it.  Training: one beam of 1e5 particles, 3 macro
    # steps, targets from the reference solution; evaluation: a held-out
    # beam of 2e4 particles, one macro step, against the oracle's brute
    # force.  Measured at this size: the median error drops by ~10x, and the
    # large step alone beats 8 plain steps of dt/8.
    p = pic.pic_default_params(dt=0.4, n_cells=512)
    X, T = learned.make_dataset(p, [inputs.gaussian_beam(100_000, seed=100, r_cut=4.0)], n_macro=3, reference="fine")
    m, scale, hist, kept = learned.train(X, T, steps=1500, batch=8192, seed=1)
    assert hist[-50:].mean() < 0.1 * hist[:10].mean(), (hist[:10].mean(), hist[-50:].mean())
    R0, V0 = inputs.gaussian_beam(20_000, seed=999, r_cut=4.0)
    plain = pic.pic_init(p, R0, V0)
    lrn = pic.pic_init(p, R0, V0)
    pic.pic_step(plain, 1)
    n_fb = pic.pic_step_learned(lrn, m, 1, scale=tuple(scale), drift_tol=1e-4)
    Rp, Vp = pic.pic_get_particles(plain)
    Rl, Vl = pic.pic_get_particles(lrn)
    res = oracle.etd_step(cfg_of(p), R0, V0)
    assert bit_equal(Rp, res.R) and bit_equal(Vp, res.V)  # the plain step is the oracle's
    Rf, Vf = oracle.brute_force(cfg_of(p), R0, V0, 0.4)
    (mp, rp), (ml, rl) = robust(np.hypot(Rp - Rf, Vp - Vf)), robust(np.hypot(Rl - Rf, Vl - Vf))
    print(f"gaussian beam: plain median {mp:.3e} rms99 {rp:.3e}; learned median {ml:.3e} rms99 {rl:.3e}; "
          f"fallbacks {n_fb}")
    assert ml < 0.3 * mp and rl < 0.3 * rp
    assert n_fb < 0.01 * R0.size
    for h in (plain, lrn):
        pic.pic_destroy(h)
    m.close()

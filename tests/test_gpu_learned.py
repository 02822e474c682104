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


# ---------------------------------------------------------------- oracle parity of the learned step's physics

from oracle import learned as OL  # noqa: E402
from oracle import mlp as omlp  # noqa: E402


def _dev(a, dtype=None):
    return torch.from_numpy(np.ascontiguousarray(a)).cuda() if dtype is None else torch.from_numpy(
        np.ascontiguousarray(a, dtype=dtype)).cuda()


@pytest.mark.parametrize("field,parity,n_cells", [(pic.PIC_FIELD_POISSON, 0, 256), (pic.PIC_FIELD_POISSON, 1, 256),
                                                  (pic.PIC_FIELD_POISSON, 0, 100), (pic.PIC_FIELD_DUFFING, 0, 256),
                                                  (pic.PIC_FIELD_ZERO, 0, 256)])
def test_frozen_potential_matches_oracle(field, parity, n_cells):
    # psi of the field of a beam on [-2, 2] with particles beyond both edges
    # (the log branch), on nodes, on the axis and on the mesh edges
    p = pic.pic_default_params(field_model=field, field_parity=parity, n_cells=n_cells, r_min=-2.0, r_max=2.0)
    c = cfg_of(p)
    R0, _ = inputs.gaussian_beam(30_000, seed=11)
    R = np.concatenate([R0, [-2.0, 2.0, 0.0, -7.5, 12.0, np.nextafter(-2.0, -3.0), -2.0 + 4.0 / n_cells]])
    n = R.size
    Rd = _dev(R)
    psi = torch.empty(n, dtype=torch.float64, device="cuda")
    if field == pic.PIC_FIELD_POISSON:
        Q = torch.empty(n_cells + 1, dtype=torch.int64, device="cuda")
        nout = torch.empty(1, dtype=torch.int64, device="cuda")
        E = torch.empty(n_cells + 1, dtype=torch.float64, device="cuda")
        edges = torch.empty(2, dtype=torch.float64, device="cuda")
        psi_n = torch.empty(n_cells + 1, dtype=torch.float64, device="cuda")
        pic.pic_deposit(p, Rd, Q, nout)
        pic.pic_poisson(p, n, Q, E, edges)
        pic.pic_frozen_potential(p, E, edges, psi_n, Rd, psi)
        torch.cuda.synchronize()
        Eo, edo = OL.mesh_field(c, R)
        assert bit_equal(E.cpu().numpy(), Eo) and bit_equal(edges.cpu().numpy(), edo)
        pn = OL.node_potential(c, Eo)
        scale = float(np.abs(pn).max())
        assert np.max(np.abs(psi_n.cpu().numpy() - pn)) <= 1e-12 * scale
    else:
        pic.pic_frozen_potential(p, None, None, None, Rd, psi)
        torch.cuda.synchronize()
        Eo = edo = None
        scale = 1.0
    po = OL.frozen_potential(c, R, Eo, edo)
    err = np.abs(psi.cpu().numpy() - po)
    assert np.all(err <= 1e-12 * (scale + np.abs(po))), float(err.max())


def _constant_net(c_R, c_V):
    w = np.zeros(omlp.N_PARAMS, np.float32)
    w[B3_OFF:B3_OFF + 2] = (c_R, c_V)
    m = pic.pic_mlp_create(16)
    pic.pic_mlp_set_weights(m, w)
    return m, w


def _oracle_certainty(c, plain, dR_lo, dR_hi, dV_lo, dV_hi, tol, E, edges, precision=0):
    """Per particle: (certain keep, certain fallback) of the energy check over
    every correction in the box [dR_lo, dR_hi] x [dV_lo, dV_hi], with a
    margin for the rounding of H on either side (1e-10 of |H| + eps max|psi|);
    precision 1: the FP32 form's binary32 corrected state."""
    H0 = OL.frozen_energy(c, plain.R, plain.V, E, edges)
    psi_scale = float(np.abs(OL.node_potential(c, E)).max()) if E is not None else 0.0
    amb = 1e-10 * (np.abs(H0) + c.eps * psi_scale + 1e-300)
    ms = []
    for dR in (dR_lo, dR_hi):
        for dV in (dV_lo, dV_hi):
            ms.append(OL.learned_apply(c, plain.R, plain.V, dR, dV, tol, E, edges, precision)[3])
    ms = np.array(ms)
    return np.all(ms < -amb, axis=0), np.all(ms > amb, axis=0)


@pytest.mark.parametrize("parity,sort_every", [(0, 1), (1, 1), (0, 0)])
def test_learned_step_constant_correction_matches_oracle_on_poisson(parity, sort_every):
    # a constant correction (W3 = 0, b3 = (c_R, c_V): the network's output is
    # b3 exactly on both sides) on a Poisson field with particles off the
    # mesh: the keep/fallback decisions and the states equal the oracle's
    # bit for bit wherever the decision is not within rounding of the limit
    p = pic.pic_default_params(dt=0.4, r_min=-2.0, r_max=2.0, field_parity=parity, sort_every=sort_every)
    c = cfg_of(p)
    R0, V0 = inputs.gaussian_beam(20_001, seed=21)
    scale, tol = (2.0 ** -9, 2.0 ** -10), 2e-3
    m, w = _constant_net(1.0, -0.75)
    h = pic.pic_init(p, R0, V0)
    n_fb = pic.pic_step_learned(h, m, 1, scale=scale, drift_tol=tol)
    R, V = pic.pic_get_particles(h)
    E, edges = OL.mesh_field(c, R0)
    plain = oracle.etd_step(c, R0, V0)
    dR = np.full(R0.size, scale[0] * 1.0)
    dV = np.full(R0.size, scale[1] * -0.75)
    Ro, Vo, keep, margin = OL.learned_apply(c, plain.R, plain.V, dR, dV, tol, E, edges)
    sure_keep, sure_fb = _oracle_certainty(c, plain, dR, dR, dV, dV, tol, E, edges)
    sure = sure_keep | sure_fb
    assert sure.mean() > 0.999 and 0.05 < keep.mean() < 0.95, (sure.mean(), keep.mean())
    assert bit_equal(R[sure], Ro[sure]) and bit_equal(V[sure], Vo[sure])
    assert int(sure_fb.sum()) <= n_fb <= int(sure_fb.sum() + (~sure).sum())
    # the off-mesh particles are among those decided
    off = np.abs(R0) > 2.0
    assert off.sum() > 100 and sure[off].all()
    pic.pic_destroy(h)
    m.close()


# 300_007 particles: two or three 128-particle tiles per block of the
# tensor-core correction kernel
@pytest.mark.parametrize("n", [20_001, 300_007])
def test_learned_step_network_matches_oracle_on_poisson(n):
    # a non-trivial network (random weights, nonzero biases): the oracle gives
    # an interval for each binary32 network output (oracle.mlp's interval
    # form); the decision is compared wherever it is the same over the whole
    # interval, and a kept state must lie in the corrected interval
    p = pic.pic_default_params(dt=0.4, r_min=-2.0, r_max=2.0)
    c = cfg_of(p)
    R0, V0 = inputs.gaussian_beam(n, seed=22)
    w = inputs.mlp_init(23)
    rng = np.random.default_rng(24)
    pp = omlp.unflatten(w.astype(np.float64))
    for b in ("b1", "b2", "b3"):
        pp[b] = rng.normal(0, 0.1, pp[b].shape)
    w = omlp.flatten(pp).astype(np.float32)
    scale, tol = (2.0 ** -8, 2.0 ** -8), 1e-3  # powers of two: the products are exact
    m = pic.pic_mlp_create(16)
    pic.pic_mlp_set_weights(m, w)
    h = pic.pic_init(p, R0, V0)
    n_fb = pic.pic_step_learned(h, m, 1, scale=scale, drift_tol=tol)
    R, V = pic.pic_get_particles(h)
    E, edges = OL.mesh_field(c, R0)
    plain = oracle.etd_step(c, R0, V0)
    X = OL.network_inputs(R0, V0, 0.0, c.eps, c.dt).astype(np.float64)
    iv = omlp.forward_interval(w.astype(np.float64), X)["out"]
    dR_lo, dR_hi = scale[0] * iv.lo[:, 0], scale[0] * iv.hi[:, 0]
    dV_lo, dV_hi = scale[1] * iv.lo[:, 1], scale[1] * iv.hi[:, 1]
    sure_keep, sure_fb = _oracle_certainty(c, plain, dR_lo, dR_hi, dV_lo, dV_hi, tol, E, edges)
    nonzero = ~((dR_lo <= 0) & (dR_hi >= 0) & (dV_lo <= 0) & (dV_hi >= 0))
    sure_keep &= nonzero
    sure_fb &= nonzero
    sure = sure_keep | sure_fb
    assert sure.mean() > 0.95 and sure_keep.sum() > 1000 and sure_fb.sum() > 1000, (sure.mean(), sure_keep.sum())
    # fallbacks: the plain state bit for bit
    assert bit_equal(R[sure_fb], plain.R[sure_fb]) and bit_equal(V[sure_fb], plain.V[sure_fb])
    # kept: inside the interval of the corrected state (an FP64 sum rounds to nearest)
    lo_R = np.nextafter(plain.R + dR_lo, -np.inf)
    hi_R = np.nextafter(plain.R + dR_hi, np.inf)
    lo_V = np.nextafter(plain.V + dV_lo, -np.inf)
    hi_V = np.nextafter(plain.V + dV_hi, np.inf)
    k = sure_keep
    assert np.all((R[k] >= lo_R[k]) & (R[k] <= hi_R[k])) and np.all((V[k] >= lo_V[k]) & (V[k] <= hi_V[k]))
    assert not np.any((R[k] == plain.R[k]) & (V[k] == plain.V[k]))
    assert int(sure_fb.sum()) <= n_fb <= int(sure_fb.sum() + (~sure).sum())
    pic.pic_destroy(h)
    m.close()


@pytest.mark.slow
def test_full_size_learned_step_on_sampled_particles():
    # The learned-stepper workload at full size in the launch configuration
    # the bench times (10^7 particles, FP32 form, 512 cells, dt 0.4, sort
    # every 4 steps) with a non-trivial network: a twin handle gives the
    # plain step bit for bit, and on 20000 sampled particles the oracle
    # decides the energy check from the interval of the network's output
    # (oracle.mlp) and the frozen field of the deposit of y^n (oracle.learned)
    n = 10_000_000
    p = pic.pic_default_params(precision=1, dt=0.4, n_cells=512, sort_every=4)
    c = cfg_of(p)
    R0, V0 = inputs.gaussian_beam(n, seed=0, r_cut=4.0)
    w = inputs.mlp_init(23)
    rng = np.random.default_rng(24)
    pp = omlp.unflatten(w.astype(np.float64))
    for b in ("b1", "b2", "b3"):
        pp[b] = rng.normal(0, 0.1, pp[b].shape)
    w = omlp.flatten(pp).astype(np.float32)
    scale, tol = (2.0 ** -8, 2.0 ** -8), 1e-3
    m = pic.pic_mlp_create(16)
    pic.pic_mlp_set_weights(m, w)
    h = pic.pic_init(p, R0, V0)
    twin = pic.pic_init(p, R0, V0)
    n_fb = pic.pic_step_learned(h, m, 1, scale=scale, drift_tol=tol)
    pic.pic_step(twin, 1)
    R, V = pic.pic_get_particles(h)
    Rp, Vp = pic.pic_get_particles(twin)
    for x in (h, twin):
        pic.pic_destroy(x)
    m.close()
    R0f = R0.astype(np.float32).astype(np.float64)
    V0f = V0.astype(np.float32).astype(np.float64)
    E, edges = OL.mesh_field(c, R0f, n, precision=1)
    idx = np.sort(np.random.default_rng(25).choice(n, 20_000, replace=False))
    X = OL.network_inputs(R0f[idx], V0f[idx], 0.0, c.eps, c.dt).astype(np.float64)
    iv = omlp.forward_interval(w.astype(np.float64), X)["out"]
    dR_lo, dR_hi = scale[0] * iv.lo[:, 0], scale[0] * iv.hi[:, 0]
    dV_lo, dV_hi = scale[1] * iv.lo[:, 1], scale[1] * iv.hi[:, 1]

    class Plain:
        pass

    plain = Plain()
    plain.R, plain.V = Rp[idx], Vp[idx]
    sure_keep, sure_fb = _oracle_certainty(c, plain, dR_lo, dR_hi, dV_lo, dV_hi, tol, E, edges, precision=1)
    nonzero = ~((dR_lo <= 0) & (dR_hi >= 0) & (dV_lo <= 0) & (dV_hi >= 0))
    sure_keep &= nonzero
    sure_fb &= nonzero
    assert (sure_keep | sure_fb).mean() > 0.95 and sure_keep.sum() > 1000 and sure_fb.sum() > 100, (
        (sure_keep | sure_fb).mean(), sure_keep.sum(), sure_fb.sum())
    Rs, Vs = R[idx], V[idx]
    assert bit_equal(Rs[sure_fb], plain.R[sure_fb]) and bit_equal(Vs[sure_fb], plain.V[sure_fb])
    f = np.float32
    lo_R = (f(plain.R) + f(dR_lo)).astype(np.float64)
    hi_R = (f(plain.R) + f(dR_hi)).astype(np.float64)
    lo_V = (f(plain.V) + f(dV_lo)).astype(np.float64)
    hi_V = (f(plain.V) + f(dV_hi)).astype(np.float64)
    k = sure_keep
    assert np.all((Rs[k] >= lo_R[k]) & (Rs[k] <= hi_R[k])) and np.all((Vs[k] >= lo_V[k]) & (Vs[k] <= hi_V[k]))
    assert 0 < n_fb < n


def _f32(x):
    return float(np.float32(x))


def test_adam_step_matches_oracle():
    # two Adam steps with given gradients (one of them zero or tiny in places)
    # against Kingma & Ba's update in FP64 with the same binary32 hyper-parameters:
    # within 2 binary32 ulps of the weight plus 32 u of the updates
    n = omlp.N_PARAMS
    rng = np.random.default_rng(31)
    w0 = (rng.normal(0, 0.3, n)).astype(np.float32)
    g1 = rng.normal(0, 1e-2, n).astype(np.float32)
    g2 = rng.normal(0, 1e-2, n).astype(np.float32)
    g1[:50] = 0.0
    g2[50:100] = 1e-10
    lr, b1, b2, e = _f32(1e-3), _f32(0.9), _f32(0.999), _f32(1e-8)
    m = pic.pic_mlp_create(16)
    pic.pic_mlp_set_weights(m, w0)
    pic.pic_mlp_apply_gradient(m, g1, lr=lr, beta1=b1, beta2=b2, eps=e)
    w1 = pic.pic_mlp_get_weights(m)
    pic.pic_mlp_apply_gradient(m, g2, lr=lr, beta1=b1, beta2=b2, eps=e)
    w2 = pic.pic_mlp_get_weights(m)
    m.close()
    o1, mo, vo = OL.adam_step(w0.astype(np.float64), np.zeros(n), np.zeros(n), g1, 1, lr, b1, b2, e)
    o2, _, _ = OL.adam_step(o1, mo, vo, g2, 2, lr, b1, b2, e)
    u = 2.0 ** -24
    ulp = np.spacing(np.abs(w0).astype(np.float32)).astype(np.float64)
    up1, up2 = np.abs(o1 - w0), np.abs(o2 - o1)
    assert np.all(np.abs(w1 - o1) <= ulp + 32 * u * up1)
    assert np.all(np.abs(w2 - o2) <= 2 * ulp + 32 * u * (up1 + up2))
    assert np.array_equal(w1[:50], w0[:50])  # a zero first gradient leaves the weight


def _library_n_seq(B):
    """Longest chain of sequential additions in the library's batch sums: a
    block sums a chunk of samples (a multiple of 64, at most 256 blocks),
    then the block partials are added in block order."""
    nwg = min(-(-B // 64), 256)
    chunk = -(-(-(-B // nwg)) // 64) * 64
    nwg = -(-B // chunk)
    return chunk + nwg + 2


def test_training_step_matches_oracle():
    # one pic_mlp_train step on the whole data set against Adam applied to the
    # oracle's gradient interval: with t = 1 the update is lr g / (|g| + eps),
    # increasing in g, so the weights lie between the updates of the interval's ends
    n = 2048
    rng = np.random.default_rng(32)
    X = np.stack([rng.normal(0, 1.5, n), rng.normal(0, 1.5, n), np.sin(rng.uniform(0, 6.3, n)),
                  np.cos(rng.uniform(0, 6.3, n)), np.full(n, 0.4)], axis=1).astype(np.float32)
    T = np.stack([0.3 * np.sin(X[:, 0]) * X[:, 1], 0.2 * np.cos(X[:, 1])], axis=1).astype(np.float32)
    w0 = inputs.mlp_init(33)
    lr, e = _f32(1e-3), _f32(1e-8)
    m = pic.pic_mlp_create(n)
    pic.pic_mlp_set_weights(m, w0)
    pic.pic_mlp_train(m, _dev(X), _dev(T), batch=n, steps=1, lr=lr, eps=e, seed=0)
    w1 = pic.pic_mlp_get_weights(m).astype(np.float64)
    m.close()
    _, g = omlp.grads_interval(w0.astype(np.float64), X.astype(np.float64), T.astype(np.float64), _library_n_seq(n))
    f = lambda x: x / (np.abs(x) + e)  # noqa: E731
    w = w0.astype(np.float64)
    ulp = np.spacing(np.abs(w0)).astype(np.float64)
    slack = ulp + 32 * 2.0 ** -24 * lr
    assert np.all(w1 >= w - lr * f(g.hi) - slack) and np.all(w1 <= w - lr * f(g.lo) + slack)


@pytest.mark.parametrize("field", [pic.PIC_FIELD_DUFFING, pic.PIC_FIELD_POISSON])
def test_specified_targets_teach_the_small_steps_error(field):
    # The network trained on the specified targets (8 plain improved-ETD steps
    # of dt/8 minus one step of dt) next to the same network trained on the
    # paper's reference solution (the fine solver over dt), on the physics of
    # the Duffing run (E = -r^3, eps = 0.01, r, v ~ N(0, 1), periods once) and
    # of the Vlasov-Poisson run (eps = 0.01, 256 cells on [-4, 4], the cut
    # Gaussian beam), both with dt = 0.4; errors after one step of a held-out
    # beam against the oracle's brute-force fine solve.  For this method the
    # large step is more accurate than 8 steps of dt/8 (its error does not grow
    # with dt where periods are clean), so the specified targets carry mostly
    # the small steps' own error: the network trained on them moves the large
    # step toward the small steps, away from the reference, while the network
    # trained on the reference solution reduces the large step's error
    # (measured, median: Duffing plain 3.3e-5, 8 x dt/8 1.4e-4, "etd" 1.3e-4, "fine" 2.9e-5;
    # Vlasov-Poisson plain 1.6e-5, 8 x dt/8 1.3e-4, "etd" 1.3e-4, "fine" 9.3e-8).
    duff = field == pic.PIC_FIELD_DUFFING
    p = pic.pic_default_params(field_model=field, dt=0.4, periods_once=1 if duff else 0)
    cut = None if duff else 4.0
    beams = [inputs.gaussian_beam(50_000, seed=300 + s, r_cut=cut) for s in range(2)]
    nets = {}
    for ref in ("etd", "fine"):
        X, T = learned.make_dataset(p, beams, n_macro=2, reference=ref)
        m, scale, hist, kept = learned.train(X, T, steps=1500, batch=8192, seed=1)
        nets[ref] = (m, scale)
    R0, V0 = inputs.gaussian_beam(20_000, seed=399, r_cut=cut)
    cfg = cfg_of(p)
    Rf, Vf = oracle.brute_force(cfg, R0, V0, 0.4)

    def run(how):
        h = pic.pic_init(p if how != "small" else pic.pic_default_params(field_model=field, dt=0.05,
                                                                         periods_once=1 if duff else 0), R0, V0)
        if how == "plain":
            pic.pic_step(h, 1)
        elif how == "small":
            pic.pic_step(h, 8)
        else:
            m, scale = nets[how]
            pic.pic_step_learned(h, m, 1, scale=tuple(scale), drift_tol=1e-4)
        R, V = pic.pic_get_particles(h)
        pic.pic_destroy(h)
        return robust(np.hypot(R - Rf, V - Vf))[0]

    err = {how: run(how) for how in ("plain", "small", "etd", "fine")}
    print(f"field {field}: median error vs the fine reference after one step of dt = 0.4: {err}")
    assert err["small"] > 2.0 * err["plain"]           # the specified reference is the less accurate one
    assert err["etd"] > err["plain"]                    # ... and the network trained on it follows it
    # the reference-solution targets never degrade the large step; on the
    # Vlasov-Poisson beam (near equilibrium) they gain about tenfold, while the
    # Duffing step's remaining error (the landing's interpolation remainder,
    # which oscillates quickly across (r, v)) is learnt only in part
    assert err["fine"] <= 1.1 * err["plain"]
    if not duff:
        assert err["fine"] < 0.3 * err["plain"]
    for m, _ in nets.values():
        m.close()

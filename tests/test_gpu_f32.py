"""The FP32 form of the CUDA path (precision = 1) against the oracle.

Integer work is exact: the deposit of binary32 positions must equal the
oracle's binary32 deposit bit for bit, and the charge is conserved exactly.
Floating-point results are compared with the FP64 oracle within bounds
derived from binary32 rounding (unit roundoff u = 2^-24):

* one fine step of Lawson RK4 in the rotating frame rounds z twice (one
  fma per component) and evaluates the stage positions from z with one
  rounded table rotation each, so a fine step adds at most about 2u|y|;
  the exact rotation itself adds nothing that accumulates, because the
  rotation of step k is read from a table (one rounding, whatever k);
* an improved-ETD macro step runs K fine steps, interpolates two samples
  (a few roundings each) and multiplies their difference by N; an error
  of the period shifts o by N dT, which moves y(o) and y(o+T) together and
  cancels to first order in the extrapolation.
The bounds below are those worst-case sums, so they hold with margin; the
measured errors are printed.
"""
import math

import numpy as np
import pytest

import oracle
from paper_1404_1160_gb300 import inputs
from paper_1404_1160_gb300 import pic
from tests.gpu_common import bit_equal, cfg_of

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

U32 = 2.0**-24  # binary32 unit roundoff


@pytest.fixture(scope="module", autouse=True)
def _built():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1404_1160_gb300 import build

    build.build()
    torch.cuda.set_device(0)


def dev(x):
    return torch.from_numpy(np.ascontiguousarray(x)).cuda()


def f32(x):
    return np.asarray(x, np.float64).astype(np.float32)


def max_err(gpu, ref):
    gpu = np.asarray(gpu, np.float64)
    ref = np.asarray(ref, np.float64)
    return float(np.max(np.abs(gpu - ref))) if ref.size else 0.0


def fine_bound(n_steps, scale):
    # (2 roundings per fine step + the final rotation) * u * |y|
    return (2.0 * n_steps + 4.0) * U32 * scale


def etd_bound(n_macro, K, N_max, scale):
    # per macro step: K fine steps, the landing's interpolation and the
    # extrapolation's N-fold difference (about 6 roundings of |y| per unit
    # of N), plus a period term of 10 roundings
    return n_macro * (2.0 * K + 6.0 * N_max + 10.0) * U32 * scale


# ------------------------------------------------------------- deposit


@pytest.mark.parametrize("n_cells,r_max,W_log2,n", [(256, 4.0, 32, 100_003), (1024, 4.0, 32, 4097),
                                                    (250, 3.0, 32, 20_001), (2, 1.0, 40, 33),
                                                    (65536, 8.0, 24, 300_000)])
def test_deposit_f32_bit_exact(n_cells, r_max, W_log2, n):
    # binary32 positions, including nodes, the mesh ends, positions outside
    # and NaN; a mesh step whose inverse is not a power of two ([-3, 3] with
    # 250 cells); W = 2^40 in the standalone call
    p = pic.pic_default_params(n_cells=n_cells, r_min=-r_max, r_max=r_max, weight_fixed=1 << W_log2)
    rng = np.random.default_rng(n_cells + W_log2)
    R = rng.normal(0, 0.4 * r_max, n).astype(np.float32)
    extra = np.array([0.0, -r_max, r_max, np.nextafter(np.float32(r_max), np.float32(0)), -1.5 * r_max,
                      3 * r_max, np.nan, r_max / n_cells], np.float32)
    R = np.concatenate([R, extra])
    Q = torch.empty(n_cells + 1, dtype=torch.int64, device="cuda")
    n_out = torch.empty(1, dtype=torch.int64, device="cuda")
    pic.pic_deposit_f32(p, dev(R), Q, n_out)
    torch.cuda.synchronize()
    Qo, no = oracle.deposit_f32(cfg_of(p), R)
    assert np.array_equal(Q.cpu().numpy(), Qo)
    assert int(n_out.item()) == no
    assert int(Qo.sum()) + no * p.weight_fixed == R.size * p.weight_fixed


def test_handle_charge_of_binary32_state():
    # the handle rounds (R, V) to binary32 on the way in; its charge is the
    # binary32 deposit of those positions and its field the FP64 trapezoid
    # integral of that charge
    p = pic.pic_default_params(precision=1, eps=1e-3, n_cells=1024)
    cfg = cfg_of(p)
    R0, V0 = inputs.gaussian_beam(50_001, seed=7, r_cut=4.0)
    h = pic.pic_init(p, R0, V0)
    R, V = pic.pic_get_particles(h)
    assert np.array_equal(R, f32(R0).astype(np.float64)) and np.array_equal(V, f32(V0).astype(np.float64))
    Q, E, edges, n_out = pic.pic_get_field(h, p.n_cells)
    Qo, no = oracle.deposit_f32(cfg, f32(R0))
    assert np.array_equal(Q, Qo) and n_out == no
    _, Eo, edges_o = oracle.poisson(cfg, Qo, R0.size)
    assert bit_equal(E, Eo) and bit_equal(edges, edges_o)
    pic.pic_destroy(h)


def test_precision_argument_checks():
    R0, V0 = inputs.gaussian_beam(64, seed=1)
    for kw, rc in (({"precision": 1, "fine_solver": pic.PIC_FINE_RK4}, pic.PIC_ERR_UNSUPPORTED),
                   ({"precision": 1, "weight_fixed": 1 << 33}, pic.PIC_ERR_UNSUPPORTED),
                   ({"precision": 2}, pic.PIC_ERR_INVALID_ARG)):
        with pytest.raises(pic.PicError) as ei:
            pic.pic_init(pic.pic_default_params(**kw), R0, V0)
        assert ei.value.status == rc


# ----------------------------------------------------------- fine solver


def test_zero_field_rotation_is_exact_and_periodic():
    # E = 0: z never changes, y_k = Phi(t_k) y_0 from the table; after one
    # turn (spt fine steps) y returns to y_0 bit for bit (Sec. 1: the fast
    # period is 2 pi eps)
    p = pic.pic_default_params(precision=1, field_model=pic.PIC_FIELD_ZERO)
    R0, V0 = inputs.gaussian_beam(4099, seed=2)
    R0, V0 = f32(R0).astype(np.float64), f32(V0).astype(np.float64)
    h = pic.pic_init(p, R0, V0)
    pic.pic_fine_steps(h, 37)
    R, V = pic.pic_get_particles(h)
    th = 37 * 2 * math.pi / p.steps_per_turn
    Rx, Vx = R0 * math.cos(th) + V0 * math.sin(th), -R0 * math.sin(th) + V0 * math.cos(th)
    amp = np.hypot(R0, V0)
    assert np.all(np.abs(R - Rx) <= 4 * U32 * amp + 1e-30)
    assert np.all(np.abs(V - Vx) <= 4 * U32 * amp + 1e-30)
    pic.pic_destroy(h)
    # one run of a whole turn never leaves the rotating frame: z is
    # unchanged and Phi(2 pi eps) = I exactly in the table
    h = pic.pic_init(p, R0, V0)
    pic.pic_fine_steps(h, p.steps_per_turn)
    R, V = pic.pic_get_particles(h)
    assert np.array_equal(R, R0) and np.array_equal(V, V0)
    pic.pic_fine_steps(h, 3 * p.steps_per_turn)
    R, V = pic.pic_get_particles(h)
    assert np.array_equal(R, R0) and np.array_equal(V, V0)
    pic.pic_destroy(h)


@pytest.mark.parametrize("field", [pic.PIC_FIELD_POISSON, pic.PIC_FIELD_DUFFING])
def test_fine_steps_within_binary32_bound(field):
    n_fine = 200
    p = pic.pic_default_params(precision=1, field_model=field)
    R0, V0 = inputs.gaussian_beam(3001, seed=11, r_cut=4.0)
    h = pic.pic_init(p, R0, V0)
    pic.pic_fine_steps(h, n_fine)
    R, V = pic.pic_get_particles(h)
    pic.pic_destroy(h)
    Ro, Vo = oracle.fine_steps(cfg_of(p), f32(R0).astype(np.float64), f32(V0).astype(np.float64), n_fine)
    scale = max(1.0, float(np.max(np.hypot(Ro, Vo))))
    er, ev = max_err(R, Ro), max_err(V, Vo)
    print(f"fine steps field {field}: max err R {er:.3e} V {ev:.3e} (bound {fine_bound(n_fine, scale):.3e})")
    assert er <= fine_bound(n_fine, scale) and ev <= fine_bound(n_fine, scale)


# ----------------------------------------------------- improved ETD step


def compare_etd(p, R0, V0, n_macro, T_known=None):
    """Runs n_macro macro steps on the GPU (FP32 form) and in the FP64
    oracle from the same binary32 initial state; returns the errors and the
    oracle's last step."""
    cfg = cfg_of(p)
    Rf, Vf = f32(R0).astype(np.float64), f32(V0).astype(np.float64)
    h = pic.pic_init(p, Rf, Vf)
    pic.pic_step(h, n_macro)
    R, V = pic.pic_get_particles(h)
    T, N, o = pic.pic_get_periods(h)
    m = pic.pic_moments(h)
    pic.pic_destroy(h)
    Ro, Vo = Rf, Vf
    K = 0
    for _ in range(n_macro):
        res = oracle.etd_step(cfg, Ro, Vo, T_known)
        Ro, Vo = res.R, res.V
        K = max(K, res.stats["window_steps"])
    return R, V, T, N, o, m, res, K


@pytest.mark.parametrize("eps,n_cells,n,n_macro", [(1e-2, 256, 4096, 1), (1e-2, 256, 20_001, 3), (1e-3, 1024, 4096, 2)])
def test_etd_step_poisson_within_binary32_bound(eps, n_cells, n, n_macro):
    p = pic.pic_default_params(precision=1, eps=eps, n_cells=n_cells)
    cfg = cfg_of(p)
    d = oracle.derive(cfg)
    R0, V0 = inputs.gaussian_beam(n, seed=3, r_cut=4.0)
    R, V, T, N, o, m, res, K = compare_etd(p, R0, V0, n_macro)
    scale = max(1.0, float(np.max(np.hypot(res.R, res.V))))
    bound = etd_bound(n_macro, K, int(res.N.max()), scale)
    er, ev = max_err(R, res.R), max_err(V, res.V)
    # the period: each extremum time comes from binary32 samples of V
    # (relative error a few u), divided by the slope of V per fine step
    # (2 pi / spt of the amplitude)
    Tsteps, Tref = T / d.h, res.T
    eT = max_err(Tsteps, Tref)
    clear = (res.o > 1e-3) & (res.o < res.T - 1e-3)
    print(f"ETD eps {eps} n {n} x{n_macro}: max err R {er:.3e} V {ev:.3e} (bound {bound:.3e}); "
          f"T err {eT:.3e} fine steps; N max {res.N.max()} K {K}")
    assert np.array_equal(N[clear], res.N[clear])
    assert eT <= 2e-4
    assert er <= bound and ev <= bound
    assert m["Q_total"] + m["n_out_of_mesh"] * p.weight_fixed == n * p.weight_fixed
    assert m["n_no_period"] == res.stats["n_no_period"]


def test_duffing_periods_once_within_binary32_bound():
    # the Duffing shape: eps 0.01, dt 0.05 (N = 0), periods once at init
    p = pic.pic_default_params(precision=1, field_model=pic.PIC_FIELD_DUFFING, dt=0.05, periods_once=1)
    cfg = cfg_of(p)
    R0, V0 = inputs.gaussian_beam(10_000, seed=0)
    Rf, Vf = f32(R0).astype(np.float64), f32(V0).astype(np.float64)
    h = pic.pic_init(p, Rf, Vf)
    st = pic.pic_get_state(h)
    To, _, _ = oracle.periods(cfg, Rf, Vf)
    eT = max_err(st["T"], To)
    pic.pic_step(h, 20)
    R, V = pic.pic_get_particles(h)
    pic.pic_destroy(h)
    Ro, Vo = Rf, Vf
    for _ in range(20):
        res = oracle.etd_step(cfg, Ro, Vo, To)
        Ro, Vo = res.R, res.V
    scale = max(1.0, float(np.max(np.hypot(Ro, Vo))))
    bound = etd_bound(20, res.stats["window_steps"], 1, scale)
    er, ev = max_err(R, Ro), max_err(V, Vo)
    print(f"Duffing x20: T err {eT:.3e} steps, max err R {er:.3e} V {ev:.3e} (bound {bound:.3e})")
    assert eT <= 2e-4
    assert er <= bound and ev <= bound


@pytest.mark.parametrize("field", [pic.PIC_FIELD_DUFFING, pic.PIC_FIELD_ZERO])
def test_local_field_equilibrium_and_periods(field):
    # dt = 0.5 (N about 8); the equilibrium y = 0 has no period (fallback)
    # and stays at 0
    p = pic.pic_default_params(precision=1, field_model=field, dt=0.5, periods_once=0)
    R0, V0 = inputs.gaussian_beam(777, seed=4)
    R0[0] = V0[0] = 0.0
    R, V, T, N, o, m, res, K = compare_etd(p, R0, V0, 3)
    assert R[0] == 0.0 and V[0] == 0.0
    assert m["n_no_period"] == res.stats["n_no_period"] == 1
    clear = (res.o > 1e-3) & (res.o < res.T - 1e-3)
    assert np.array_equal(N[clear], res.N[clear])
    scale = max(1.0, float(np.max(np.hypot(res.R, res.V))))
    bound = etd_bound(3, K, int(res.N.max()), scale)
    assert max_err(R, res.R) <= bound and max_err(V, res.V) <= bound


# ------------------------------------------------------ invariants


def test_sort_and_checkpoint_change_no_bit():
    R0, V0 = inputs.gaussian_beam(9000, seed=21, r_cut=4.0)
    out = []
    for every in (0, 1, 3):
        p = pic.pic_default_params(precision=1, sort_every=every)
        h = pic.pic_init(p, R0, V0)
        pic.pic_step(h, 4)
        R, V = pic.pic_get_particles(h)
        T, N, o = pic.pic_get_periods(h)
        out.append((R, V, T, N, o))
        pic.pic_destroy(h)
    for other in out[1:]:
        for a, b in zip(out[0], other):
            assert bit_equal(a, b)
    p = pic.pic_default_params(precision=1)
    b = pic.pic_init(p, R0, V0)
    pic.pic_step(b, 2)
    st = pic.pic_get_state(b)
    pic.pic_destroy(b)
    c = pic.pic_init(p, np.zeros(9000), np.zeros(9000))
    pic.pic_set_state(c, st)
    pic.pic_step(c, 2)
    Rc, Vc = pic.pic_get_particles(c)
    pic.pic_destroy(c)
    assert bit_equal(out[0][0], Rc) and bit_equal(out[0][1], Vc)


def test_empty_and_tiny_runs():
    p = pic.pic_default_params(precision=1)
    h = pic.pic_init(p, np.zeros(0), np.zeros(0))
    pic.pic_step(h, 2)
    assert pic.pic_moments(h)["n_particles"] == 0
    pic.pic_destroy(h)
    R0, V0 = inputs.gaussian_beam(1, seed=5, r_cut=4.0)
    R, V, T, N, o, m, res, K = compare_etd(p, R0, V0, 2)
    scale = max(1.0, float(np.max(np.hypot(res.R, res.V))))
    assert max_err(R, res.R) <= etd_bound(2, K, int(res.N.max()), scale)


def test_barrier_timeout_fp32():
    rc = pic.pic_test_barrier_timeout(50_000_000, precision=1)
    assert rc == pic.PIC_ERR_TIMEOUT
    p = pic.pic_default_params(precision=1)
    R0, V0 = inputs.gaussian_beam(1000, seed=1, r_cut=4.0)
    h = pic.pic_init(p, R0, V0)
    pic.pic_step(h, 1)
    pic.pic_destroy(h)


@pytest.mark.slow
def test_histogram_copies_at_scale_within_binary32_bound():
    # The physics of the 1e8-particle workload (eps 0.001, 1024 cells,
    # dt 0.1, sort every 4 steps) at 3e6 particles: enough per SM for the
    # window to deposit into four histogram copies per block (lane l into
    # copy l mod 4), few enough for the oracle to run the whole step.
    n = 3_000_000
    p = pic.pic_default_params(precision=1, eps=1e-3, n_cells=1024, sort_every=4)
    cfg = cfg_of(p)
    R0, V0 = inputs.gaussian_beam(n, seed=11, r_cut=4.0)
    h = pic.pic_init(p, R0, V0)
    Q, E, edges, n_out = pic.pic_get_field(h, p.n_cells)
    pic.pic_destroy(h)
    Qo, no = oracle.deposit_f32(cfg, f32(R0))
    assert np.array_equal(Q, Qo) and n_out == no
    R, V, T, N, o, m, res, K = compare_etd(p, R0, V0, 1)
    scale = max(1.0, float(np.max(np.hypot(res.R, res.V))))
    bound = etd_bound(1, K, int(res.N.max()), scale)
    er, ev = max_err(R, res.R), max_err(V, res.V)
    print(f"3e6 particles, eps 1e-3: max err R {er:.3e} V {ev:.3e} (bound {bound:.3e})")
    assert er <= bound and ev <= bound
    assert m["Q_total"] + m["n_out_of_mesh"] * p.weight_fixed == n * p.weight_fixed


@pytest.mark.slow
def test_full_size_fp32_workload_charge_is_exact():
    # The 1e8-particle FP32 workload at full size, in the launch
    # configuration the bench times (eps 0.001, 1024 cells, window cap 202,
    # sort every 4 steps): after one macro step the charge the library
    # deposits from its state equals the oracle's binary32 deposit of that
    # state bit for bit, the charge is conserved exactly, every particle is
    # finite and the kinetic energy moves by far less than 1e-3.
    n = 100_000_000
    p = pic.pic_default_params(precision=1, eps=1e-3, n_cells=1024, max_window_steps=202, sort_every=4)
    cfg = cfg_of(p)
    R0, V0 = inputs.gaussian_beam(n, seed=0, r_cut=4.0)
    h = pic.pic_init(p, R0, V0)
    del R0, V0
    m0 = pic.pic_moments(h)
    pic.pic_step(h, 1)
    m1 = pic.pic_moments(h)
    R, V = pic.pic_get_particles(h)
    assert np.isfinite(R).all() and np.isfinite(V).all()
    Q, E, edges, n_out = pic.pic_get_field(h, p.n_cells)
    pic.pic_destroy(h)
    Qo, no = oracle.deposit_f32(cfg, f32(R))
    assert np.array_equal(Q, Qo) and n_out == no
    assert int(Q.sum()) + n_out * p.weight_fixed == n * p.weight_fixed
    assert m1["Q_total"] + m1["n_out_of_mesh"] * p.weight_fixed == n * p.weight_fixed
    assert abs(m1["kinetic"] - m0["kinetic"]) < 1e-3 * m0["kinetic"]
    assert m1["window_steps"] <= 202 and m1["N_min"] >= 14


def test_odd_field_reading_within_binary32_bound():
    p = pic.pic_default_params(precision=1, field_parity=pic.PIC_PARITY_ODD)
    cfg = cfg_of(p)
    R0, V0 = inputs.gaussian_beam(8001, seed=9, r_cut=4.5)
    h = pic.pic_init(p, R0, V0)
    Q, E, edges, n_out = pic.pic_get_field(h, p.n_cells)
    pic.pic_destroy(h)
    Qo, no = oracle.deposit_f32(cfg, f32(R0))
    _, Eo, edges_o = oracle.poisson(cfg, Qo, R0.size)
    assert np.array_equal(Q, Qo) and bit_equal(E, Eo) and bit_equal(edges, edges_o)
    R, V, T, N, o, m, res, K = compare_etd(p, R0, V0, 2)
    scale = max(1.0, float(np.max(np.hypot(res.R, res.V))))
    bound = etd_bound(2, K, int(res.N.max()), scale)
    assert max_err(R, res.R) <= bound and max_err(V, res.V) <= bound


@pytest.mark.parametrize("n_cells,block", [(800, 512), (2048, 1024)])
def test_fp32_field_build_node_counts_per_thread(n_cells, block):
    # 4 nodes per thread in the register field build (800 cells, 512-thread
    # blocks) and the staged build (2048 cells), within the binary32 bound
    p = pic.pic_default_params(precision=1, n_cells=n_cells, block_size=block)
    R0, V0 = inputs.gaussian_beam(30_000, seed=13, r_cut=4.0)
    R, V, T, N, o, m, res, K = compare_etd(p, R0, V0, 1)
    scale = max(1.0, float(np.max(np.hypot(res.R, res.V))))
    bound = etd_bound(1, K, int(res.N.max()), scale)
    assert max_err(R, res.R) <= bound and max_err(V, res.V) <= bound

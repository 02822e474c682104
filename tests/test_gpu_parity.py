"""Parity of the CUDA path (called through the C ABI) with the FP64 oracle.

Integer work (the deposited charge) must match bit for bit.  Floating-point
results must match within 1e-12 relative; the kernels evaluate the same
IEEE operations in the same order as the oracle, so in practice they agree
bit for bit and the tests also report that.
"""
import math

import numpy as np
import pytest

import oracle
from paper_1404_1160_gb300 import inputs
from paper_1404_1160_gb300 import pic
from tests.gpu_common import assert_close, bit_equal, cfg_of

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1404_1160_gb300 import build

    build.build()
    torch.cuda.set_device(0)


def dev(x):
    return torch.from_numpy(np.ascontiguousarray(x)).cuda()


def mesh_positions(n, seed, r_max=4.0):
    rng = np.random.default_rng(seed)
    R = rng.normal(0, 1.2, n)
    # edge cases: nodes, cell midpoints, mesh ends, outside, exactly r_max
    extra = np.array([0.0, -r_max, r_max, r_max * (1 - 1e-16), -r_max * 1.5, r_max * 3, 1 / 32, -1 / 64, 3.999999999])
    return np.concatenate([R, extra])


# --------------------------------------------------------------- mesh kernels


@pytest.mark.parametrize("n_cells,r_max,n", [(256, 4.0, 100_003), (1024, 4.0, 4097), (2, 1.0, 33), (65536, 8.0, 200_000)])
def test_deposit_bit_exact(n_cells, r_max, n):
    p = pic.pic_default_params(n_cells=n_cells, r_min=-r_max, r_max=r_max)
    R = mesh_positions(n, seed=n_cells, r_max=r_max)
    Q = torch.empty(n_cells + 1, dtype=torch.int64, device="cuda")
    n_out = torch.empty(1, dtype=torch.int64, device="cuda")
    pic.pic_deposit(p, dev(R), Q, n_out)
    torch.cuda.synchronize()
    Qo, no = oracle.deposit(cfg_of(p), R)
    assert np.array_equal(Q.cpu().numpy(), Qo)
    assert int(n_out.item()) == no
    assert int(Qo.sum()) + no * p.weight_fixed == R.size * p.weight_fixed


def test_deposit_empty_input():
    p = pic.pic_default_params()
    Q = torch.full((p.n_cells + 1,), 7, dtype=torch.int64, device="cuda")
    n_out = torch.full((1,), 7, dtype=torch.int64, device="cuda")
    pic.pic_deposit(p, torch.empty(0, dtype=torch.float64, device="cuda"), Q, n_out)
    torch.cuda.synchronize()
    assert int(Q.abs().sum()) == 0 and int(n_out.item()) == 0


@pytest.mark.parametrize("n_cells", [2, 256, 1024, 2048, 4094, 65536])
def test_poisson_bit_exact(n_cells):
    # random charges span several scan tiles for the large meshes
    rng = np.random.default_rng(n_cells)
    p = pic.pic_default_params(n_cells=n_cells)
    Q = rng.integers(0, 1 << 40, n_cells + 1).astype(np.int64)
    n_particles = 10**6
    E = torch.empty(n_cells + 1, dtype=torch.float64, device="cuda")
    edges = torch.empty(2, dtype=torch.float64, device="cuda")
    pic.pic_poisson(p, n_particles, dev(Q), E, edges)
    S, Eo, edges_o = oracle.poisson(cfg_of(p), Q, n_particles)
    assert bit_equal(E.cpu().numpy(), Eo)
    assert bit_equal(edges.cpu().numpy(), edges_o)


@pytest.mark.parametrize("n_cells,n", [(256, 123_457), (64, 31), (65536, 100_000)])
def test_gather_bit_exact(n_cells, n):
    p = pic.pic_default_params(n_cells=n_cells)
    cfg = cfg_of(p)
    R = mesh_positions(n, seed=5)
    Q, _ = oracle.deposit(cfg, inputs.gaussian_beam(5000, seed=2, r_cut=4.0)[0])
    _, E, edges = oracle.poisson(cfg, Q, 5000)
    out = torch.empty(R.size, dtype=torch.float64, device="cuda")
    pic.pic_gather(p, dev(R), dev(E), dev(edges), out)
    torch.cuda.synchronize()
    eo = oracle.gather(cfg, R, E, edges)
    assert bit_equal(out.cpu().numpy(), eo)


# --------------------------------------------------------------- fine solver


@pytest.mark.parametrize("field", [pic.PIC_FIELD_POISSON, pic.PIC_FIELD_DUFFING, pic.PIC_FIELD_ZERO])
@pytest.mark.parametrize("solver", [pic.PIC_FINE_RK4, pic.PIC_FINE_LAWSON_RK4])
def test_fine_steps_match_oracle(field, solver):
    p = pic.pic_default_params(field_model=field, fine_solver=solver)
    R0, V0 = inputs.gaussian_beam(3001, seed=11, r_cut=4.0)
    h = pic.pic_init(p, R0, V0)
    pic.pic_fine_steps(h, 7)
    R, V = pic.pic_get_particles(h)
    pic.pic_destroy(h)
    Ro, Vo = oracle.fine_steps(cfg_of(p), R0, V0, 7)
    assert_close(R, Ro, what="R")
    assert_close(V, Vo, what="V")
    assert bit_equal(R, Ro) and bit_equal(V, Vo)


# -------------------------------------------------------- improved ETD step


@pytest.mark.parametrize("solver", [pic.PIC_FINE_RK4, pic.PIC_FINE_LAWSON_RK4])
@pytest.mark.parametrize("n", [1, 2000, 20_001])
def test_etd_step_poisson_matches_oracle(solver, n):
    # several blocks and a ragged tail; three macro steps with the
    # self-consistent field
    p = pic.pic_default_params(fine_solver=solver)
    cfg = cfg_of(p)
    R0, V0 = inputs.gaussian_beam(n, seed=3, r_cut=4.0)
    h = pic.pic_init(p, R0, V0)
    Ro, Vo = R0, V0
    for step in range(3):
        pic.pic_step(h, 1)
        res = oracle.etd_step(cfg, Ro, Vo)
        Ro, Vo = res.R, res.V
        R, V = pic.pic_get_particles(h)
        assert_close(R, Ro, what=f"R step {step}")
        assert_close(V, Vo, what=f"V step {step}")
        T, N, o = pic.pic_get_periods(h)
        d = oracle.derive(cfg)
        assert np.array_equal(N, res.N)
        assert_close(T, res.T * d.h, what="T")
        assert_close(o, res.o * d.h, what="o")
        Q, E, edges, n_out = pic.pic_get_field(h, p.n_cells)
        Qo, no = oracle.deposit(cfg, Ro)
        assert np.array_equal(Q, Qo) and n_out == no
        m = pic.pic_moments(h)
        assert m["window_steps"] == res.stats["window_steps"]
        assert m["n_no_period"] == res.stats["n_no_period"]
    assert bit_equal(R, Ro) and bit_equal(V, Vo)
    pic.pic_destroy(h)


@pytest.mark.parametrize("solver", [pic.PIC_FINE_RK4, pic.PIC_FINE_LAWSON_RK4])
@pytest.mark.parametrize("n_cells,r_cut", [(256, 4.0), (100, 4.5)])
def test_odd_field_reading_matches_oracle(solver, n_cells, r_cut):
    # the odd extension E = rE/|r| (E = 0 on the axis) in every field cycle of
    # the window, in the standalone field and in the off-mesh gather (r_cut
    # 4.5 puts particles beyond the mesh on both sides; 100 cells is not a
    # power of two)
    p = pic.pic_default_params(fine_solver=solver, n_cells=n_cells, field_parity=pic.PIC_PARITY_ODD)
    cfg = cfg_of(p)
    R0, V0 = inputs.gaussian_beam(6001, seed=8, r_cut=r_cut)
    h = pic.pic_init(p, R0, V0)
    Q, E, edges, n_out = pic.pic_get_field(h, p.n_cells)
    Qo, no = oracle.deposit(cfg, R0)
    _, Eo, edges_o = oracle.poisson(cfg, Qo, R0.size)
    assert np.array_equal(Q, Qo) and n_out == no
    assert bit_equal(E, Eo) and bit_equal(edges, edges_o) and E[n_cells // 2] == 0.0
    Ro, Vo = R0, V0
    for step in range(2):
        pic.pic_step(h, 1)
        res = oracle.etd_step(cfg, Ro, Vo)
        Ro, Vo = res.R, res.V
        R, V = pic.pic_get_particles(h)
        assert bit_equal(R, Ro) and bit_equal(V, Vo), step
    pic.pic_destroy(h)


@pytest.mark.parametrize("n_cells,block", [(800, 512), (400, 256), (2048, 1024)])
def test_field_build_node_counts_per_thread(n_cells, block):
    # the register field build gives each thread up to 4 nodes (800 cells on
    # 512-thread blocks, 400 on 256: 4 nodes; 2048 on 1024: too many, the
    # staged build); every case bit-exact against the oracle
    p = pic.pic_default_params(n_cells=n_cells, block_size=block)
    cfg = cfg_of(p)
    R0, V0 = inputs.gaussian_beam(30_000, seed=12, r_cut=4.0)
    h = pic.pic_init(p, R0, V0)
    pic.pic_step(h, 1)
    R, V = pic.pic_get_particles(h)
    pic.pic_destroy(h)
    res = oracle.etd_step(cfg, R0, V0)
    assert bit_equal(R, res.R) and bit_equal(V, res.V)


@pytest.mark.parametrize("W_log2", [20, 40])
def test_etd_step_with_other_fixed_point_weights(W_log2):
    # W = 2^40: right weights floor(f W) above 2^32 (the 64-bit histogram);
    # W = 2^20: a coarse quantisation of the same deposit
    p = pic.pic_default_params(weight_fixed=1 << W_log2)
    cfg = cfg_of(p)
    R0, V0 = inputs.gaussian_beam(20_001, seed=8, r_cut=4.0)
    h = pic.pic_init(p, R0, V0)
    pic.pic_step(h, 2)
    R, V = pic.pic_get_particles(h)
    Q, _, _, n_out = pic.pic_get_field(h, p.n_cells)
    pic.pic_destroy(h)
    res = oracle.etd_step(cfg, R0, V0)
    res = oracle.etd_step(cfg, res.R, res.V)
    Qo, no = oracle.deposit(cfg, res.R)
    assert np.array_equal(Q, Qo) and n_out == no
    assert bit_equal(R, res.R) and bit_equal(V, res.V)


@pytest.mark.parametrize("solver", [pic.PIC_FINE_RK4, pic.PIC_FINE_LAWSON_RK4])
def test_duffing_config0_shape_matches_oracle(solver):
    # Duffing, eps 0.01, dt 0.05 (N = 0), periods once at init (Sec. 4.1)
    p = pic.pic_default_params(field_model=pic.PIC_FIELD_DUFFING, dt=0.05, periods_once=1, fine_solver=solver)
    cfg = cfg_of(p)
    R0, V0 = inputs.gaussian_beam(10_000, seed=0)
    h = pic.pic_init(p, R0, V0)
    st = pic.pic_get_state(h)
    T, nf, _ = oracle.periods(cfg, R0, V0)
    assert bit_equal(st["T"], T)
    pic.pic_step(h, 20)
    R, V = pic.pic_get_particles(h)
    Ro, Vo = R0, V0
    for _ in range(20):
        res = oracle.etd_step(cfg, Ro, Vo, T)
        Ro, Vo = res.R, res.V
    assert np.all(res.N == 0)
    assert_close(R, Ro, what="R")
    assert_close(V, Vo, what="V")
    assert bit_equal(R, Ro) and bit_equal(V, Vo)
    pic.pic_destroy(h)


@pytest.mark.parametrize("prec", [0, 1])
def test_poisson_periods_once_keeps_the_initial_state(prec):
    # step 1 alone at initialisation (periods_once) must leave y^0 untouched,
    # and the steps that follow use the periods of y^0
    p = pic.pic_default_params(periods_once=1, precision=prec)
    R0, V0 = inputs.gaussian_beam(5000, seed=13, r_cut=4.0)
    if prec:
        R0, V0 = R0.astype(np.float32).astype(np.float64), V0.astype(np.float32).astype(np.float64)
    h = pic.pic_init(p, R0, V0)
    R, V = pic.pic_get_particles(h)
    assert bit_equal(R, R0) and bit_equal(V, V0)
    st = pic.pic_get_state(h)
    T, _, _ = oracle.periods(cfg_of(p), R0, V0)
    if prec == 0:
        assert bit_equal(st["T"], T)
        pic.pic_step(h, 2)
        R, V = pic.pic_get_particles(h)
        res = oracle.etd_step(cfg_of(p), R0, V0, T)
        res = oracle.etd_step(cfg_of(p), res.R, res.V, T)
        assert bit_equal(R, res.R) and bit_equal(V, res.V)
    else:
        assert np.max(np.abs(st["T"] - T)) < 2e-4
    pic.pic_destroy(h)


@pytest.mark.parametrize("field", [pic.PIC_FIELD_DUFFING, pic.PIC_FIELD_ZERO])
def test_local_field_periods_every_step(field):
    # periods recomputed every macro step, dt = 0.5 (N about 8), with one
    # particle at the equilibrium y = 0 of both fields (V never changes
    # sign: 2 pi eps fallback, and y stays 0)
    p = pic.pic_default_params(field_model=field, dt=0.5, periods_once=0)
    cfg = cfg_of(p)
    R0, V0 = inputs.gaussian_beam(777, seed=4)
    R0[0] = V0[0] = 0.0
    h = pic.pic_init(p, R0, V0)
    pic.pic_step(h, 3)
    R, V = pic.pic_get_particles(h)
    T, N, o = pic.pic_get_periods(h)
    Ro, Vo = R0, V0
    for _ in range(3):
        res = oracle.etd_step(cfg, Ro, Vo)
        Ro, Vo = res.R, res.V
    assert R[0] == 0.0 and V[0] == 0.0
    assert np.array_equal(N, res.N)
    assert bit_equal(R, Ro) and bit_equal(V, Vo)
    m = pic.pic_moments(h)
    assert m["n_no_period"] == res.stats["n_no_period"] == 1
    pic.pic_destroy(h)


def test_out_of_mesh_particles_in_window():
    # a few particles start beyond the mesh: they deposit nothing and feel
    # rE_edge / R
    p = pic.pic_default_params(r_min=-2.0, r_max=2.0, n_cells=128)
    cfg = cfg_of(p)
    R0, V0 = inputs.gaussian_beam(3000, seed=9, r_cut=4.0)
    h = pic.pic_init(p, R0, V0)
    pic.pic_step(h, 2)
    R, V = pic.pic_get_particles(h)
    res = oracle.etd_step(cfg, R0, V0)
    res = oracle.etd_step(cfg, res.R, res.V)
    assert bit_equal(R, res.R) and bit_equal(V, res.V)
    m = pic.pic_moments(h)
    Qo, no = oracle.deposit(cfg, res.R)
    assert no > 0 and m["n_out_of_mesh"] == no
    assert m["Q_total"] + no * p.weight_fixed == 3000 * p.weight_fixed
    pic.pic_destroy(h)


def test_paper_workload_eps_1e_3():
    # the paper's own run shape (Sec. 4.2): f0 of eq. InitialConditionBeam,
    # eps = 1e-3, dt = 0.5, [-2, 2] with 256 cells
    p = pic.pic_default_params(eps=1e-3, dt=0.5, r_min=-2.0, r_max=2.0)
    cfg = cfg_of(p)
    R0, V0 = inputs.paper_beam(20000, seed=0)
    h = pic.pic_init(p, R0, V0)
    pic.pic_step(h, 1)
    R, V = pic.pic_get_particles(h)
    res = oracle.etd_step(cfg, R0, V0)
    assert bit_equal(R, res.R) and bit_equal(V, res.V)
    _, N, _ = pic.pic_get_periods(h)
    assert np.array_equal(N, res.N) and N.min() >= 70
    pic.pic_destroy(h)


@pytest.mark.parametrize("field,solver", [(pic.PIC_FIELD_POISSON, pic.PIC_FINE_LAWSON_RK4), (pic.PIC_FIELD_POISSON, pic.PIC_FINE_RK4),
                                          (pic.PIC_FIELD_DUFFING, pic.PIC_FINE_LAWSON_RK4)])
def test_phase_space_sort_changes_no_result(field, solver):
    # the storage order is an implementation detail: sorting every step,
    # every third step or never must give the same bits in the public order
    R0, V0 = inputs.gaussian_beam(9000, seed=21, r_cut=4.0)
    out = []
    for every in (0, 1, 3):
        p = pic.pic_default_params(field_model=field, fine_solver=solver, sort_every=every, dt=0.1)
        h = pic.pic_init(p, R0, V0)
        pic.pic_step(h, 4)
        R, V = pic.pic_get_particles(h)
        T, N, o = pic.pic_get_periods(h)
        st = pic.pic_get_state(h)
        out.append((R, V, T, N, o, st["T"]))
        pic.pic_destroy(h)
    for other in out[1:]:
        for a, b in zip(out[0], other):
            assert bit_equal(a, b)


# -------------------------------------------------------- state and failures


def test_checkpoint_resume_is_bit_identical():
    p = pic.pic_default_params()
    R0, V0 = inputs.gaussian_beam(5000, seed=12, r_cut=4.0)
    a = pic.pic_init(p, R0, V0)
    pic.pic_step(a, 4)
    Ra, Va = pic.pic_get_particles(a)
    b = pic.pic_init(p, R0, V0)
    pic.pic_step(b, 2)
    st = pic.pic_get_state(b)
    pic.pic_destroy(b)
    c = pic.pic_init(p, np.zeros(5000), np.zeros(5000))
    pic.pic_set_state(c, st)
    pic.pic_step(c, 2)
    Rc, Vc = pic.pic_get_particles(c)
    assert bit_equal(Ra, Rc) and bit_equal(Va, Vc)
    assert pic.pic_moments(c)["n_steps"] == 4
    pic.pic_destroy(a)
    pic.pic_destroy(c)


def test_trajectory_band_miss_replays_the_window_bit_identically():
    # the FP64 ETD window stores only the trajectory rows around the landing
    # rows forecast from the previous step's periods; wrong periods in a
    # restored state make the forecast miss, the window replays with every
    # row, and the step equals the one forecast from the true periods
    p = pic.pic_default_params()
    R0, V0 = inputs.gaussian_beam(20_000, seed=31, r_cut=4.0)
    a = pic.pic_init(p, R0, V0)
    b = pic.pic_init(p, R0, V0)
    pic.pic_step(a, 2)
    pic.pic_step(b, 2)
    st = pic.pic_get_state(b)
    st["T"] = st["T"] * 0.6
    pic.pic_set_state(b, st)
    pic.pic_step(a, 1)
    pic.pic_step(b, 1)
    Ra, Va = pic.pic_get_particles(a)
    Rb, Vb = pic.pic_get_particles(b)
    assert bit_equal(Ra, Rb) and bit_equal(Va, Vb)
    ma, mb = pic.pic_moments(a), pic.pic_moments(b)
    assert ma["band_replays"] == 0 and mb["band_replays"] == 1
    Ta, Na, oa = pic.pic_get_periods(a)
    Tb, Nb, ob = pic.pic_get_periods(b)
    assert bit_equal(Ta, Tb) and np.array_equal(Na, Nb) and bit_equal(oa, ob)
    # the windows after a replay store every row for a while: still the same
    pic.pic_step(a, 3)
    pic.pic_step(b, 3)
    Ra, Va = pic.pic_get_particles(a)
    Rb, Vb = pic.pic_get_particles(b)
    assert bit_equal(Ra, Rb) and bit_equal(Va, Vb)
    assert pic.pic_moments(a)["band_replays"] == 0 and pic.pic_moments(b)["band_replays"] == 1
    pic.pic_destroy(a)
    pic.pic_destroy(b)


def test_beam_beyond_65536_particles_per_block_matches_the_oracle():
    # more than 65536 positions per block, field and cycle (one block per
    # SM): the window's charge histogram takes four 32-bit words per node
    # (count and 11/11/10-bit parts of the weights) instead of three; one
    # macro step bit for bit against the oracle (20 fine steps per turn keep
    # the oracle's single-core step short)
    sm = torch.cuda.get_device_properties(0).multi_processor_count
    n = 2048 * 32 * sm + 1003
    p = pic.pic_default_params(steps_per_turn=20, max_window_steps=80)
    c = cfg_of(p)
    R0, V0 = inputs.gaussian_beam(n, seed=41, r_cut=4.0)
    h = pic.pic_init(p, R0, V0)
    pic.pic_step(h, 1)
    R, V = pic.pic_get_particles(h)
    ref = oracle.etd_step(c, R0, V0)
    assert bit_equal(R, ref.R) and bit_equal(V, ref.V)
    pic.pic_destroy(h)


def test_empty_run():
    p = pic.pic_default_params()
    h = pic.pic_init(p, np.zeros(0), np.zeros(0))
    pic.pic_step(h, 3)
    m = pic.pic_moments(h)
    assert m["n_particles"] == 0 and m["n_steps"] == 3
    pic.pic_destroy(h)


def test_barrier_wait_times_out_and_device_stays_usable():
    # the barrier waits for an arrival that never comes: the kernel must
    # give up after its limit and report PIC_ERR_TIMEOUT
    rc = pic.pic_test_barrier_timeout(50_000_000)
    assert rc == pic.PIC_ERR_TIMEOUT
    p = pic.pic_default_params()
    R0, V0 = inputs.gaussian_beam(1000, seed=1, r_cut=4.0)
    h = pic.pic_init(p, R0, V0)
    pic.pic_step(h, 1)
    R, _ = pic.pic_get_particles(h)
    assert bit_equal(R, oracle.etd_step(cfg_of(p), R0, V0).R)
    pic.pic_destroy(h)


def test_moments_match_numpy():
    p = pic.pic_default_params(field_model=pic.PIC_FIELD_DUFFING, dt=0.05, periods_once=1)
    R0, V0 = inputs.gaussian_beam(4096, seed=6)
    h = pic.pic_init(p, R0, V0)
    pic.pic_step(h, 5)
    R, V = pic.pic_get_particles(h)
    m = pic.pic_moments(h)
    w = 1.0 / R.size
    assert m["mean_R"] == pytest.approx(R.mean(), rel=1e-12, abs=1e-15)
    assert m["rms_V"] == pytest.approx(math.sqrt(np.mean(V * V)), rel=1e-12)
    e2H = np.sum(w * (0.5 * (R * R + V * V) + 0.25 * p.eps * R**4))
    assert m["duffing_energy"] == pytest.approx(e2H, rel=1e-12)
    assert m["t"] == pytest.approx(5 * 0.05)
    pic.pic_destroy(h)


# -------------------------------------------------- full-size (bench) shape


@pytest.mark.slow
def test_full_size_vlasov_poisson_step_matches_oracle():
    # the benchmark's workload: N_p = 1e6, eps 0.01, dt 0.1, 256 cells on
    # [-4, 4], Lawson RK4, phase-space sort every 4 steps, in the launch
    # configuration bench.py times
    p = pic.pic_default_params(sort_every=4)
    cfg = cfg_of(p)
    R0, V0 = inputs.gaussian_beam(10**6, seed=0, r_cut=4.0)
    h = pic.pic_init(p, dev(R0), dev(V0), torch.cuda.current_stream())
    pic.pic_step(h, 1)
    R, V = pic.pic_get_particles(h)
    Q, E, edges, n_out = pic.pic_get_field(h, p.n_cells)
    pic.pic_destroy(h)
    res = oracle.etd_step(cfg, R0, V0)
    Qo, no = oracle.deposit(cfg, res.R)
    assert np.array_equal(Q, Qo) and n_out == no
    assert int(Q.sum()) + n_out * p.weight_fixed == 10**6 * p.weight_fixed
    assert_close(R, res.R, what="R")
    assert_close(V, res.V, what="V")
    assert bit_equal(R, res.R) and bit_equal(V, res.V)

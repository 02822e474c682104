"""The batched form: many FP32 beams in one cooperative launch.

Every beam of a batch must compute, bit for bit, what pic_step computes for
it alone, whatever the launch shape, the block share of each beam, the sort
period and whether the step runs from a captured graph; and every beam of a
mixed batch (eps 0.1 and 0.001, 128 and 2048 cells, Poisson, Duffing with
periods once and zero field, particles off the mesh) must match the FP64
oracle's macro steps within the binary32 bound of the FP32 form.
"""
import numpy as np
import pytest

from paper_1404_1160_gb300 import inputs
from paper_1404_1160_gb300 import pic
from tests.gpu_common import bit_equal

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1404_1160_gb300 import build

    build.build()
    torch.cuda.set_device(0)


# a mixed batch: eps from 0.1 to 0.001, meshes of 128 to 1024 cells, the
# Poisson, Duffing (periods once) and zero fields, sizes from 1 to 2e5 and a
# ragged tail
SPECS = [
    dict(eps=0.1, n_cells=128, n=5000),
    dict(eps=0.01, n_cells=256, n=200_000),
    dict(eps=0.001, n_cells=1024, n=30_001),
    dict(eps=0.005, n_cells=512, n=1),
    dict(eps=0.05, field_model=pic.PIC_FIELD_DUFFING, periods_once=1, n=7000),
    dict(eps=0.01, field_model=pic.PIC_FIELD_ZERO, n=3000),
    dict(eps=0.01, n_cells=256, n=65_536),
]


def make_params(spec):
    kw = {k: v for k, v in spec.items() if k != "n"}
    return pic.pic_default_params(precision=1, dt=0.1, **kw)


def make_beams():
    out = []
    for i, sp in enumerate(SPECS):
        r_cut = 4.0 if sp.get("field_model", 0) == pic.PIC_FIELD_POISSON else None
        out.append(inputs.gaussian_beam(sp["n"], seed=20 + i, r_cut=r_cut))
    return out


def single_runs(beams, steps):
    res = []
    for sp, (R0, V0) in zip(SPECS, beams):
        h = pic.pic_init(make_params(sp), R0, V0)
        pic.pic_step(h, steps)
        res.append(pic.pic_get_particles(h))
        pic.pic_destroy(h)
    return res


def test_batch_equals_single_beams_and_ignores_the_launch_shape():
    beams = make_beams()
    ref = single_runs(beams, 3)
    # (block, blocks per SM, allocation power, sort period, histogram copies)
    shapes = [None, (512, 2, 0.85, 1, 1), (256, 4, 1.0, 2, 2), (1024, 1, 1.0, 4, 4)]
    for shape in shapes:
        b = pic.pic_batch_create([make_params(sp) for sp in SPECS], beams)
        if shape is not None:
            pic.pic_batch_set_config(b, *shape)
        pic.pic_batch_step(b, 3)
        assert pic.pic_batch_steps(b) == 3
        for i in range(len(SPECS)):
            R, V = pic.pic_batch_get_particles(b, i)
            assert bit_equal(R, ref[i][0]) and bit_equal(V, ref[i][1]), (shape, i)
            m = pic.pic_batch_moments(b, i)
            assert m["n_steps"] == 3
            if SPECS[i].get("field_model", 0) == pic.PIC_FIELD_POISSON:
                assert m["Q_total"] + m["n_out_of_mesh"] * (1 << 32) == SPECS[i]["n"] * (1 << 32)
        cfg = pic.pic_batch_get_config(b)
        assert cfg["grid"] >= len(SPECS)
        assert cfg["graph"] == 1, cfg  # steps replay a captured graph
        if shape is not None:
            assert cfg["hist_copies"] == shape[4], cfg
        b.close()


def test_autotuner_steps_are_real_steps():
    beams = make_beams()
    ref = single_runs(beams, TUNE_STEPS_MAX)
    b = pic.pic_batch_create([make_params(sp) for sp in SPECS], beams)
    pic.pic_batch_step(b, 1)
    best = pic.pic_batch_tune(b, steps_per_trial=2)
    done = pic.pic_batch_steps(b)
    pic.pic_batch_step(b, ref_steps(done))
    for i in range(len(SPECS)):
        R, V = pic.pic_batch_get_particles(b, i)
        assert bit_equal(R, ref[i][0]) and bit_equal(V, ref[i][1]), (best, i)
    assert best["block"] in (256, 512, 1024) and best["sort_every"] in (1, 4, 16)
    assert best["hist_copies"] in (1, 2, 4) and best["shares_measured"] in (0, 1)
    b.close()


# steps_per_trial = 2: a trial is a warm step plus the timed steps.  One
# step, up to 15 launch shapes (3 steps each), the sort periods 1, 4, 16
# timed over whole periods (3, 5 and 17 steps), up to 9 trials of measured
# block shares (3 steps each) and 2 more steps bound what the tuner runs.
TUNE_STEPS_MAX = 1 + 15 * 3 + (3 + 5 + 17) + 9 * 3 + 2


def ref_steps(done):
    return TUNE_STEPS_MAX - done


def test_batch_rejects_the_fp64_path():
    R0, V0 = inputs.gaussian_beam(100, seed=1, r_cut=4.0)
    with pytest.raises(pic.PicError) as ei:
        pic.pic_batch_create([pic.pic_default_params(precision=0)], [(R0, V0)])
    assert ei.value.status == pic.PIC_ERR_UNSUPPORTED


# ---------------------------------------------------------------- against the FP64 oracle

import oracle  # noqa: E402
from tests.gpu_common import cfg_of  # noqa: E402
from tests.test_gpu_f32 import etd_bound, f32, max_err  # noqa: E402

# eps 0.1 and 0.001 x meshes of 128 and 2048 cells (Poisson), the Duffing
# field with periods once and the zero field at both eps, and a beam whose
# Gaussian tail reaches beyond a mesh on [-2, 2]
ORACLE_SPECS = (
    [dict(eps=e, n_cells=c, n=3001 + i) for i, (e, c) in enumerate([(0.1, 128), (0.1, 2048), (0.001, 128),
                                                                    (0.001, 2048)])]
    + [dict(eps=e, field_model=pic.PIC_FIELD_DUFFING, periods_once=1, n=2500) for e in (0.1, 0.001)]
    + [dict(eps=e, field_model=pic.PIC_FIELD_ZERO, n=1500) for e in (0.1, 0.001)]
    + [dict(eps=0.01, n_cells=256, r_min=-2.0, r_max=2.0, n=4000, uncut=True)]
)


def test_every_beam_of_a_mixed_batch_matches_the_oracle():
    # each beam of one batched launch against the FP64 oracle's macro steps
    # from the same binary32 initial state, within the binary32 bound of the
    # FP32 form (tests/test_gpu_f32.py); charge conserved exactly
    n_macro = 2
    params, beams = [], []
    for i, sp in enumerate(ORACLE_SPECS):
        kw = {k: v for k, v in sp.items() if k not in ("n", "uncut")}
        params.append(pic.pic_default_params(precision=1, dt=0.1, **kw))
        poisson = sp.get("field_model", 0) == pic.PIC_FIELD_POISSON
        R0, V0 = inputs.gaussian_beam(sp["n"], seed=60 + i, r_cut=4.0 if poisson and not sp.get("uncut") else None)
        beams.append((f32(R0).astype(np.float64), f32(V0).astype(np.float64)))
    b = pic.pic_batch_create(params, beams)
    pic.pic_batch_step(b, n_macro)
    off_mesh = 0
    for i, (sp, p, (R0, V0)) in enumerate(zip(ORACLE_SPECS, params, beams)):
        R, V = pic.pic_batch_get_particles(b, i)
        m = pic.pic_batch_moments(b, i)
        cfg = cfg_of(p)
        T = oracle.periods(cfg, R0, V0)[0] if p.periods_once else None
        Ro, Vo, K, N_max = R0, V0, 0, 0
        for _ in range(n_macro):
            res = oracle.etd_step(cfg, Ro, Vo, T)
            Ro, Vo = res.R, res.V
            K = max(K, res.stats["window_steps"])
            N_max = max(N_max, int(res.N.max()))
        scale = max(1.0, float(np.max(np.hypot(Ro, Vo))))
        bound = etd_bound(n_macro, K, N_max, scale)
        er, ev = max_err(R, Ro), max_err(V, Vo)
        print(f"beam {i} {sp}: max err R {er:.3e} V {ev:.3e} (bound {bound:.3e}), K {K}, N max {N_max}")
        assert er <= bound and ev <= bound, (i, sp, er, ev, bound)
        if p.field_model == pic.PIC_FIELD_POISSON:
            assert m["Q_total"] + m["n_out_of_mesh"] * p.weight_fixed == sp["n"] * p.weight_fixed
            if sp.get("uncut"):
                off_mesh = m["n_out_of_mesh"]
        assert m["n_steps"] == n_macro
    assert off_mesh > 0
    b.close()


@pytest.mark.slow
def test_full_size_batch64_workload():
    # The 64-beam workload at full size (1.6e7 particles): with all beams in
    # one launch, the four smallest beams match the FP64 oracle's two macro
    # steps within the binary32 bound; after the autotuner (the launch shape
    # and measured block shares the bench times) they still equal their
    # single-beam runs bit for bit; every beam keeps its charge exactly and
    # stays finite throughout
    import bench

    params, beams = bench.batch_specs(bench.WORKLOADS["batch64"])
    beams = [(f32(R).astype(np.float64), f32(V).astype(np.float64)) for R, V in beams]
    sizes = np.array([R.size for R, _ in beams])
    small = [int(i) for i in np.argsort(sizes)[:4]]
    b = pic.pic_batch_create(params, beams)

    def check_all(steps):
        for i, (p, (R0, _)) in enumerate(zip(params, beams)):
            R, V = pic.pic_batch_get_particles(b, i)
            assert np.isfinite(R).all() and np.isfinite(V).all(), i
            m = pic.pic_batch_moments(b, i)
            assert m["n_steps"] == steps
            if p.field_model == pic.PIC_FIELD_POISSON:
                assert m["Q_total"] + m["n_out_of_mesh"] * p.weight_fixed == R0.size * p.weight_fixed, i

    pic.pic_batch_step(b, 2)
    check_all(2)
    for i in small:
        p, (R0, V0) = params[i], beams[i]
        cfg = cfg_of(p)
        T = oracle.periods(cfg, R0, V0)[0] if p.periods_once else None
        Ro, Vo, K, N_max = R0, V0, 0, 0
        for _ in range(2):
            res = oracle.etd_step(cfg, Ro, Vo, T)
            Ro, Vo = res.R, res.V
            K = max(K, res.stats["window_steps"])
            N_max = max(N_max, int(res.N.max()))
        R, V = pic.pic_batch_get_particles(b, i)
        scale = max(1.0, float(np.max(np.hypot(Ro, Vo))))
        bound = etd_bound(2, K, N_max, scale)
        assert max_err(R, Ro) <= bound and max_err(V, Vo) <= bound, (i, sizes[i], bound)
    cfg_t = pic.pic_batch_tune(b, steps_per_trial=1)
    pic.pic_batch_step(b, 1)
    steps = pic.pic_batch_steps(b)
    check_all(steps)
    for i in small:
        h = pic.pic_init(params[i], *beams[i])
        pic.pic_step(h, steps)
        Rs, Vs = pic.pic_get_particles(h)
        pic.pic_destroy(h)
        R, V = pic.pic_batch_get_particles(b, i)
        assert bit_equal(R, Rs) and bit_equal(V, Vs), (i, cfg_t)
    b.close()

"""The batched form: many FP32 beams in one cooperative launch.

Every beam of a batch must compute, bit for bit, what pic_step computes for
it alone (the FP32 form, itself checked against the FP64 oracle in
tests/test_gpu_f32.py), whatever the launch shape, the block share of each
beam, the sort period and whether the step runs from a captured graph.
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
    ref = single_runs(beams, 1 + 15 * 3 + 3 * 3 + 2)
    b = pic.pic_batch_create([make_params(sp) for sp in SPECS], beams)
    pic.pic_batch_step(b, 1)
    best = pic.pic_batch_tune(b, steps_per_trial=2)
    done = pic.pic_batch_steps(b)
    pic.pic_batch_step(b, ref_steps(done))
    for i in range(len(SPECS)):
        R, V = pic.pic_batch_get_particles(b, i)
        assert bit_equal(R, ref[i][0]) and bit_equal(V, ref[i][1]), (best, i)
    assert best["block"] in (256, 512, 1024) and best["sort_every"] in (1, 4, 16)
    assert best["hist_copies"] in (1, 2, 4)
    b.close()


def ref_steps(done):
    # the reference above ran 1 + (up to 15 shapes + 3 sort periods) x 3 + 2 steps
    return 1 + 15 * 3 + 3 * 3 + 2 - done


def test_batch_rejects_the_fp64_path():
    R0, V0 = inputs.gaussian_beam(100, seed=1, r_cut=4.0)
    with pytest.raises(pic.PicError) as ei:
        pic.pic_batch_create([pic.pic_default_params(precision=0)], [(R0, V0)])
    assert ei.value.status == pic.PIC_ERR_UNSUPPORTED

"""Comparator schemes on the GPU: the classical ETD scheme (P = 2 pi eps) and
the modified ETD scheme (P = the mean first-tour time) of Algorithm
ClassicETDAlgo, against the FP64 oracle.  The GPU takes the same IEEE
operations in the same order (the mean period is summed in the public
order, as the oracle sums), so results agree bit for bit."""
import math

import numpy as np
import pytest

import oracle
from paper_1404_1160_gb300 import inputs
from paper_1404_1160_gb300 import pic
from tests.gpu_common import bit_equal, cfg_of

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1404_1160_gb300 import build

    build.build()
    torch.cuda.set_device(0)


def fine_count(u, h):
    """Fine steps of a solve over time u: floor(u/h) whole steps and one of the rest."""
    k = math.floor(u / h)
    return k + (1 if u - k * h > 0.0 else 0)


@pytest.mark.parametrize("field,dt,n", [(pic.PIC_FIELD_POISSON, 0.1, 3001), (pic.PIC_FIELD_POISSON, 0.37, 20_000),
                                        (pic.PIC_FIELD_DUFFING, 0.5, 2000), (pic.PIC_FIELD_ZERO, 0.23, 100)])
@pytest.mark.parametrize("mode", [0, 1])
def test_classic_and_modified_etd_match_oracle(field, dt, n, mode):
    p = pic.pic_default_params(field_model=field, dt=dt)
    cfg = cfg_of(p)
    if field == pic.PIC_FIELD_DUFFING:
        R0, V0 = inputs.paper_beam(n, seed=2)
    else:
        R0, V0 = inputs.gaussian_beam(n, seed=2, r_cut=4.0)
    h = pic.pic_init(p, R0, V0)
    Ro, Vo = R0, V0
    hf = oracle.derive(cfg).h
    for step in range(3):
        P, K = pic.pic_step_classic(h, 1, mode, with_fine_steps=True)
        Ro, Vo, Po = oracle.classic_step(cfg, Ro, Vo, mode)
        R, V = pic.pic_get_particles(h)
        assert P == Po, (step, P, Po)
        assert bit_equal(R, Ro) and bit_equal(V, Vo), step
        # fine steps: the solve over P, the one over o (whole steps plus
        # one step of the rest), and for mode 1 the detection window
        o = math.fmod(dt, P)
        solves = fine_count(P, hf) + fine_count(o, hf) if mode else p.steps_per_turn + fine_count(o, hf)
        assert (K == solves) if mode == 0 else (solves < K <= solves + p.max_window_steps), (K, solves)
    m = pic.pic_moments(h)
    assert m["n_steps"] == 3 and m["t"] == pytest.approx(3 * dt)
    if field == pic.PIC_FIELD_POISSON:
        assert m["Q_total"] + m["n_out_of_mesh"] * p.weight_fixed == n * p.weight_fixed
    pic.pic_destroy(h)


def test_modified_etd_with_periods_from_initialisation():
    # periods_once: the mean period of y^0 serves every step
    p = pic.pic_default_params(field_model=pic.PIC_FIELD_DUFFING, dt=0.5, periods_once=1)
    R0, V0 = inputs.paper_beam(1000, seed=3)
    h = pic.pic_init(p, R0, V0)
    P1 = pic.pic_step_classic(h, 1, 1)
    P2, K2 = pic.pic_step_classic(h, 1, 1, with_fine_steps=True)
    T = oracle.periods(cfg_of(p), R0, V0)[0]
    total = 0.0
    for x in T:  # in index order, as the library and the oracle sum
        total += float(x)
    hf = oracle.derive(cfg_of(p)).h
    assert P1 == P2 == (total / T.size) * hf
    assert K2 == fine_count(P2, hf) + fine_count(math.fmod(0.5, P2), hf)  # no detection window
    pic.pic_destroy(h)


def test_fp32_handles_are_refused():
    R0, V0 = inputs.gaussian_beam(100, seed=1, r_cut=4.0)
    h = pic.pic_init(pic.pic_default_params(precision=1), R0, V0)
    with pytest.raises(pic.PicError) as ei:
        pic.pic_step_classic(h, 1, 0)
    assert ei.value.status == pic.PIC_ERR_UNSUPPORTED
    pic.pic_destroy(h)

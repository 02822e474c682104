"""Long-time behaviour of the three ETD schemes at the paper's scale (Sec. 4):
the improved scheme (Algorithm ETDFSSModAlgo), the modified scheme
(Algorithm ClassicETDAlgo with the mean first-tour time) and the classical
one (period 2 pi eps), against the reference solution.

Setting of Sec. 4.1 and Sec. 4.2: 20000 macroparticles of eq.
InitialConditionBeam, eps = 0.001, Delta t = 0.5, the reference solution is
the fine solver alone at h = 2 pi eps / 100 over the whole time.  Errors are
per-particle phase-space distances to the reference.  The schemes' steps
equal the FP64 oracle's bit for bit (tests/test_gpu_parity.py,
tests/test_gpu_classic.py); at this length the oracle would need hours, so
the reference solution runs on the GPU too (pic_fine_advance, itself equal to
the oracle's brute-force solve).
"""
import numpy as np
import pytest

from paper_1404_1160_gb300 import inputs
from paper_1404_1160_gb300 import pic

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1404_1160_gb300 import build

    build.build()
    torch.cuda.set_device(0)


def stats(R, V, Rf, Vf):
    """(median, RMS of the 99 % best, fraction diverged) of the errors; a
    particle whose state is no longer finite counts as an infinite error."""
    e = np.hypot(R - Rf, V - Vf)
    bad = ~np.isfinite(e)
    e = np.sort(np.where(bad, np.inf, e))
    return float(np.median(e)), float(np.sqrt(np.mean(e[:int(0.99 * e.size)] ** 2))), float(bad.mean())


def run_schemes(p, checkpoints, dt):
    """Errors (median, RMS of the 99 % best, fraction diverged) of the
    improved, modified and classical schemes at each checkpoint time."""
    R0, V0 = inputs.paper_beam(20000, seed=0)
    hs = {name: pic.pic_init(p, R0, V0) for name in ("improved", "modified", "classical", "reference")}
    out = {name: [] for name in ("improved", "modified", "classical")}
    t = 0.0
    for tc in checkpoints:
        k = int(round((tc - t) / dt))
        pic.pic_step(hs["improved"], k)
        pic.pic_step_classic(hs["modified"], k, 1)
        pic.pic_step_classic(hs["classical"], k, 0)
        pic.pic_fine_advance(hs["reference"], tc - t)
        t = tc
        Rf, Vf = pic.pic_get_particles(hs["reference"])
        for name in out:
            R, V = pic.pic_get_particles(hs[name])
            out[name].append(stats(R, V, Rf, Vf))
    for h in hs.values():
        pic.pic_destroy(h)
    return out


def test_duffing_long_time():
    # Sec. 4.1: E = -r^3, periods computed once (they depend only on the
    # initial condition); t = 10, 20, 30, 37
    p = pic.pic_default_params(field_model=pic.PIC_FIELD_DUFFING, eps=0.001, dt=0.5, periods_once=1,
                               max_window_steps=400)
    times = (10.0, 20.0, 30.0, 37.0)
    out = run_schemes(p, times, 0.5)
    print("duffing (median, rms99, diverged) at", times, out)
    # Measured: the improved scheme's median error grows slowly (7e-5 at
    # t = 10, 2.4e-4 at t = 37, RMS99 1e-3, no particle lost); the
    # modified scheme's is 20x larger at t = 10 and its extrapolation then
    # blows particles up (non-finite states from t = 30); the classical
    # scheme does so from t = 20.
    imp, mod, cls = out["improved"], out["modified"], out["classical"]
    for k in range(len(times)):
        assert imp[k][0] < 0.1 * mod[k][0] and imp[k][0] < 0.1 * cls[k][0], (k, out)
        assert imp[k][2] == 0.0, (k, out)
    assert imp[-1][0] < 1e-3 and imp[-1][1] < 5e-3, out
    assert mod[-1][0] > 3.0 * mod[0][0], out  # the modified scheme drifts away
    assert mod[-1][1] > 100.0 * imp[-1][1], out
    assert mod[-1][2] > 0.0 and cls[-1][2] > 0.01, out  # and becomes unstable


def test_vlasov_poisson_long_time():
    # Sec. 4.2: self-consistent field, periods recomputed every step;
    # t = 15, 30, 45, 60
    p = pic.pic_default_params(eps=0.001, dt=0.5, max_window_steps=400)
    times = (15.0, 30.0, 45.0, 60.0)
    out = run_schemes(p, times, 0.5)
    print("vlasov-poisson (median, rms99, diverged) at", times, out)
    # Measured (median error at t = 15, 30, 45, 60): improved 3.9e-4,
    # 7.9e-4, 1.3e-3, 2.4e-3; modified 6.0e-4, 1.7e-3, 2.1e-3, 3.1e-3;
    # classical 2.3e-4, 2.8e-4, 2.8e-4, 3.6e-4; no particle lost.  The
    # improved scheme stays ahead of the modified one, as the paper reports,
    # but neither becomes unstable by t = 60 with this beam: the periods of
    # 90 % of its particles lie within 5e-6 of 2 pi eps (relative; 99 %
    # within 2.3e-5, from the oracle's period detection), against 1.7e-4
    # (99 %: 2.1e-4) in the Duffing case, so the classical scheme, which
    # needs no period estimate and no landing interpolation, is the most
    # accurate of the three here.
    imp, mod, cls = out["improved"], out["modified"], out["classical"]
    for k in range(len(times)):
        assert imp[k][0] < mod[k][0] and imp[k][1] < mod[k][1], (k, out)
        assert cls[k][0] < imp[k][0], (k, out)
        assert imp[k][2] == mod[k][2] == cls[k][2] == 0.0, (k, out)
    assert imp[-1][0] < 5e-3, out

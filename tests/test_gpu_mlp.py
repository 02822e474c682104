"""The learned stepper's network on the GPU against its FP64 oracle.

The GPU evaluates the network with bfloat16 weights and hidden activations
and FP32 accumulation; the oracle evaluates the same formulas in FP64 with
the same bfloat16 rounding points (oracle/mlp.py).  The two can differ by
binary32 rounding and, where a hidden activation's binary32 value lies on
the other side of a bfloat16 rounding boundary than its exact value, by a
flip of that activation.  The oracle's interval form (oracle.mlp.
forward_interval / grads_interval) gives, element by element, the range a
binary32 evaluation with these rounding points can reach: the width is the
binary32 rounding bound (~1e-6 relative) wherever no flip is reachable, and
covers the flip where one is.  Every GPU output and every gradient entry
must lie inside its interval.
"""
import numpy as np
import pytest

from oracle import mlp as omlp
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


def dev(x):
    return torch.from_numpy(np.ascontiguousarray(x, dtype=np.float32)).cuda()


def batch(n, seed):
    rng = np.random.default_rng(seed)
    X = np.stack([rng.normal(0, 1.5, n), rng.normal(0, 1.5, n), np.sin(rng.uniform(0, 6.3, n)),
                  np.cos(rng.uniform(0, 6.3, n)), np.full(n, 0.4)], axis=1).astype(np.float32)
    T = np.stack([0.3 * np.sin(X[:, 0]) * X[:, 1], 0.2 * np.cos(X[:, 1]) - 0.1 * X[:, 0] * X[:, 3]], axis=1)
    return X, T.astype(np.float32)


def weights(seed, scale=1.0):
    w = inputs.mlp_init(seed)
    rng = np.random.default_rng(seed + 100)
    # nonzero biases too, so that every parameter block is exercised
    p = omlp.unflatten(w.astype(np.float64))
    for b in ("b1", "b2", "b3"):
        p[b] = rng.normal(0, 0.1, p[b].shape)
    return (omlp.flatten(p) * scale).astype(np.float32)


# 400_003 samples: several 128-sample tiles per block of the tensor-core kernel
# (its mbarrier phase, A buffer and accumulator reused from tile to tile)
@pytest.mark.parametrize("n", [1, 17, 4096, 100_003, 400_003])
def test_forward_matches_oracle(n):
    m = pic.pic_mlp_create(16)
    w = weights(1)
    pic.pic_mlp_set_weights(m, w)
    X, _ = batch(n, 2)
    Y = torch.empty((n, 2), dtype=torch.float32, device="cuda")
    pic.pic_mlp_forward(m, dev(X), Y)
    iv = omlp.forward_interval(w.astype(np.float64), X.astype(np.float64))["out"]
    y = Y.cpu().numpy().astype(np.float64)
    outside = (y < iv.lo) | (y > iv.hi)
    assert not outside.any(), (np.argwhere(outside)[:5], y[outside][:5], iv.mid[outside][:5], iv.rad[outside][:5])
    # the test has teeth: most outputs are pinned to binary32 rounding
    assert np.mean(iv.rad <= 1e-5) > 0.6
    assert np.array_equal(pic.pic_mlp_get_weights(m), w)
    m.close()


# 150_000 samples: two tiles for some blocks of the per-sample kernel and ten
# 64-sample tiles accumulated in tensor memory per weight-gradient block
@pytest.mark.parametrize("n", [16, 1000, 8192, 150_000])
def test_gradients_match_oracle(n):
    m = pic.pic_mlp_create(n)
    w = weights(3)
    pic.pic_mlp_set_weights(m, w)
    X, T = batch(n, 4)
    g, loss = pic.pic_mlp_gradients(m, dev(X), dev(T))
    # longest chain of sequential additions of the library's batch sums: a
    # block sums a chunk of samples (a multiple of 64, at most 256 blocks),
    # then the block partials are added in block order
    nwg = min(-(-n // 64), 256)
    chunk = -(-(-(-n // nwg)) // 64) * 64
    n_seq = chunk + -(-n // chunk) + 2
    loss_iv, g_iv = omlp.grads_interval(w.astype(np.float64), X.astype(np.float64), T.astype(np.float64), n_seq)
    assert loss_iv.lo <= loss <= loss_iv.hi, (loss, loss_iv.mid, loss_iv.rad)
    g = g.astype(np.float64)
    outside = (g < g_iv.lo) | (g > g_iv.hi)
    assert not outside.any(), (np.argwhere(outside)[:5].ravel(), g[outside][:5], g_iv.mid[outside][:5],
                               g_iv.rad[outside][:5])
    # the test has teeth: every block's interval is far narrower than the
    # block's gradient (median radius below 1e-3 of its largest entry)
    for name, shape in omlp.SHAPES:
        k0 = sum(int(np.prod(s)) for nm, s in omlp.SHAPES[:[x[0] for x in omlp.SHAPES].index(name)])
        k1 = k0 + int(np.prod(shape))
        assert np.median(g_iv.rad[k0:k1]) <= 1e-3 * np.abs(g_iv.mid[k0:k1]).max(), name
    # reproducible bit for bit
    g2, loss2 = pic.pic_mlp_gradients(m, dev(X), dev(T))
    assert np.array_equal(g, g2) and loss == loss2
    m.close()


def test_training_reduces_loss_and_is_reproducible():
    X, T = batch(40_000, 5)
    Xd, Td = dev(X), dev(T)
    runs = []
    for _ in range(2):
        m = pic.pic_mlp_create(2048)
        pic.pic_mlp_set_weights(m, inputs.mlp_init(7))
        hist = pic.pic_mlp_train(m, Xd, Td, batch=2048, steps=400, lr=3e-3, seed=11)
        runs.append((hist, pic.pic_mlp_get_weights(m)))
        m.close()
    hist, w = runs[0]
    assert np.all(np.isfinite(hist))
    assert hist[-20:].mean() < 0.05 * hist[:5].mean(), (hist[:5].mean(), hist[-20:].mean())
    assert np.array_equal(runs[0][1], runs[1][1]) and np.array_equal(runs[0][0], runs[1][0])
    # the trained weights evaluated by the oracle fit the held-out data too
    Xh, Th = batch(5000, 6)
    out = omlp.forward(w.astype(np.float64), Xh.astype(np.float64))["out"]
    assert np.mean((out - Th) ** 2) < 0.1 * np.mean(Th ** 2)


def test_argument_checks():
    with pytest.raises(pic.PicError):
        pic.pic_mlp_create(0)
    m = pic.pic_mlp_create(8)
    X, T = batch(16, 1)
    with pytest.raises(pic.PicError):
        pic.pic_mlp_gradients(m, dev(X), dev(T))  # more samples than max_batch
    m.close()

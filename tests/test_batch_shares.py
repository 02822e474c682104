"""The batch tuner's block shares from measured windows (host arithmetic of
pic_batch_tune, exported as pic_test_batch_shares; no GPU needed).

The shares must keep every beam within [least, most], use at most the grid,
and reach the least largest predicted window of any such shares: checked
against brute force over every allocation of small batches, and by its
constraints on batches of the bench's size.
"""
import itertools
import math

import numpy as np
import pytest


@pytest.fixture(scope="module")
def pic():
    from paper_1404_1160_gb300 import build

    build.build()
    from paper_1404_1160_gb300 import pic as p

    p.load()
    return p


def predicted(poisson, n, ms, bm, block_m, block, b):
    """The window the shares are chosen by, written from its definition."""
    if poisson:
        return ms * bm / b
    r = math.ceil(n / (b * block))
    r0 = math.ceil(n / (bm * block_m))
    return ms * r / r0


def largest(case, blocks):
    return max(predicted(case["poisson"][i], case["n"][i], case["ms"][i], case["bm"][i], case["block_m"], case["block"],
                         blocks[i]) for i in range(len(blocks)))


def call(pic, case):
    return pic.pic_test_batch_shares(case["poisson"], case["n"], case["ms"], case["bm"], case["block_m"],
                                     case["block"], case["grid"], case["lo"], case["hi"])


def random_case(rng, n_beams, grid, most_cap):
    block = int(rng.choice([128, 256, 512]))
    poisson = (rng.uniform(size=n_beams) < 0.7).astype(np.int32)
    n = rng.integers(200, 20000, size=n_beams)
    ms = rng.uniform(0.5, 40.0, size=n_beams)
    bm = rng.integers(1, 6, size=n_beams)
    lo = np.ones(n_beams, dtype=np.int64)
    hi = np.minimum(rng.integers(1, most_cap + 1, size=n_beams), np.maximum(1, -(-n // block)))
    return dict(poisson=poisson, n=n, ms=ms, bm=bm, block_m=block, block=block, grid=grid, lo=lo, hi=hi)


def test_two_poisson_beams_by_hand(pic):
    # windows 10 and 30 ms on one block each, four blocks: the slow beam
    # takes two more (30 -> 15 -> 10), then the grid is full
    case = dict(poisson=[1, 1], n=[1000, 1000], ms=[10.0, 30.0], bm=[1, 1], block_m=256, block=256, grid=4,
                lo=[1, 1], hi=[10, 10])
    rc, blocks = call(pic, case)
    assert rc == pic.PIC_OK
    assert blocks.tolist() == [1, 3]


def test_analytic_beam_takes_whole_rounds(pic):
    # 1000 particles, 100 threads a block: 10 rounds on one block; the
    # shares of fewer rounds are 2 (5 rounds), 3 (4), 4 (3), 5 (2), 10 (1)
    case = dict(poisson=[0], n=[1000], ms=[50.0], bm=[1], block_m=100, block=100, grid=7, lo=[1], hi=[10])
    rc, blocks = call(pic, case)
    assert rc == pic.PIC_OK
    assert blocks.tolist() == [5]  # 7 blocks do no better than 5 (2 rounds)


@pytest.mark.parametrize("seed", range(40))
def test_min_max_against_brute_force(pic, seed):
    rng = np.random.default_rng(seed)
    n_beams = int(rng.integers(2, 5))
    grid = int(rng.integers(n_beams, 3 * n_beams + 6))
    case = random_case(rng, n_beams, grid, most_cap=7)
    rc, blocks = call(pic, case)
    assert rc == pic.PIC_OK
    best = min(largest(case, alloc) for alloc in itertools.product(*[range(int(l), int(h) + 1) for l, h in
                                                                     zip(case["lo"], case["hi"])])
               if sum(alloc) <= grid)
    assert np.all(blocks >= case["lo"]) and np.all(blocks <= case["hi"]) and blocks.sum() <= grid
    assert largest(case, blocks) == pytest.approx(best, rel=1e-12)


@pytest.mark.parametrize("seed", range(10))
def test_bench_sized_batches_keep_the_constraints(pic, seed):
    rng = np.random.default_rng(100 + seed)
    case = random_case(rng, 64, 304, most_cap=40)
    rc, blocks = call(pic, case)
    assert rc == pic.PIC_OK
    assert np.all(blocks >= case["lo"]) and np.all(blocks <= case["hi"]) and blocks.sum() <= 304
    # nothing left over that could shorten a beam: every beam is at its most,
    # or its next shorter window needs more blocks than are free
    free = 304 - int(blocks.sum())
    for i in range(64):
        if blocks[i] >= case["hi"][i]:
            continue
        now = predicted(case["poisson"][i], case["n"][i], case["ms"][i], case["bm"][i], case["block_m"],
                        case["block"], blocks[i])
        shorter = [b for b in range(int(blocks[i]) + 1, int(case["hi"][i]) + 1)
                   if predicted(case["poisson"][i], case["n"][i], case["ms"][i], case["bm"][i], case["block_m"],
                                case["block"], b) < now]
        assert not shorter or shorter[0] - blocks[i] > free, (i, blocks[i], shorter[:1], free)


def test_errors(pic):
    case = dict(poisson=[1, 1], n=[1000, 1000], ms=[1.0, 1.0], bm=[1, 1], block_m=256, block=256, grid=3,
                lo=[2, 2], hi=[4, 4])
    assert call(pic, case)[0] == pic.PIC_ERR_UNSUPPORTED  # the least shares exceed the grid
    bad = dict(case, lo=[1, 1], hi=[0, 4])
    assert call(pic, bad)[0] == pic.PIC_ERR_INVALID_ARG  # most below least
    bad = dict(case, lo=[1, 1], ms=[-1.0, 1.0])
    assert call(pic, bad)[0] == pic.PIC_ERR_INVALID_ARG
    bad = dict(case, lo=[1, 1], block=0)
    assert call(pic, bad)[0] == pic.PIC_ERR_INVALID_ARG
    bad = dict(case, lo=[1, 1], ms=[float("nan"), 1.0])
    assert call(pic, bad)[0] == pic.PIC_ERR_INVALID_ARG
    bad = dict(case, lo=[1, 1], hi=[4, 1 << 40])  # block counts beyond 2^31
    assert call(pic, bad)[0] == pic.PIC_ERR_INVALID_ARG

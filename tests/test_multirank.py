"""The exchange step of a particle-sharded run (world_size 2, gloo on CPU).

If the particles of one beam were split over ranks, each field cycle would
add the ranks' integer charges with one all-reduce and then solve the field
on every rank.  Integer charge makes that exchange exact and independent of
how particles are split or in which order ranks add: the sharded charge and
field equal the unsharded ones bit for bit.  This runs the oracle's deposit
and trapezoid solve on two CPU ranks.
"""
import os
import socket

import numpy as np
import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, q):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        import oracle
        from paper_1404_1160_gb300 import inputs

        cfg = oracle.Config()
        R, _ = inputs.gaussian_beam(50_001, seed=5, r_cut=4.0)
        R = np.concatenate([R, [9.0, -9.0]])  # two particles off the mesh
        shard = R[rank::world]  # uneven, interleaved split
        Q, n_out = oracle.deposit(cfg, shard)
        t = torch.from_numpy(np.concatenate([Q, [n_out]]).astype(np.int64))
        dist.all_reduce(t)  # the one exchange of a field cycle
        Qs, nouts = t[:-1].numpy(), int(t[-1])
        _, E, edges = oracle.poisson(cfg, Qs, R.size)
        q.put((rank, Qs, nouts, E, edges))
    finally:
        dist.destroy_process_group()


def test_sharded_charge_and_field_equal_unsharded():
    import oracle
    from paper_1404_1160_gb300 import inputs

    world = 2
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank, args=(r, world, port, q)) for r in range(world)]
    for p in procs:
        p.start()
    results = [q.get(timeout=120) for _ in range(world)]
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    cfg = oracle.Config()
    R, _ = inputs.gaussian_beam(50_001, seed=5, r_cut=4.0)
    R = np.concatenate([R, [9.0, -9.0]])
    Q, n_out = oracle.deposit(cfg, R)
    _, E, edges = oracle.poisson(cfg, Q, R.size)
    for rank, Qs, nouts, Es, edges_s in results:
        assert np.array_equal(Qs, Q) and nouts == n_out == 2
        assert np.array_equal(Es.view(np.int64), E.view(np.int64))
        assert np.array_equal(edges_s.view(np.int64), edges.view(np.int64))

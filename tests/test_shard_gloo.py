"""The multi-rank path on CPU: two gloo ranks split one problem's histories,
run them (with the oracle standing in for each rank's GPU), and sum their
tallies; the result equals the single-rank run.  Also the timing reduction
(slowest rank) and the partition itself."""
import os
import socket

import numpy as np
import pytest

from paper_2402_09222_b300 import shard


def test_history_range_partitions_exactly():
    for n in (1, 2, 7, 1000, 10_000_001):
        for world in (1, 2, 3, 8):
            if world > n:
                continue
            ranges = [shard.history_range(r, world, n) for r in range(world)]
            assert ranges[0][0] == 0 and ranges[-1][1] == n
            assert all(a[1] == b[0] for a, b in zip(ranges, ranges[1:]))
            sizes = [b - a for a, b in ranges]
            assert max(sizes) - min(sizes) <= 1
    with pytest.raises(ValueError):
        shard.history_range(2, 2, 10)


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _worker(rank, world, port, q):
    import torch.distributed as dist
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        import oracle
        from paper_2402_09222_b300 import synth
        prob = synth.config3_problem(n_histories=3001, lattice_n=5, n_points=300)
        lo, hi = shard.history_range(rank, world, prob.n_histories)
        part = oracle.transport(prob, seed=77, first=lo, count=hi - lo, derivatives=True)
        part.pop("capped")
        total = shard.reduce_tallies(part)
        slowest = shard.max_over_ranks(10.0 + rank)
        if rank == 0:
            q.put((total, slowest))
    finally:
        dist.destroy_process_group()


def test_two_gloo_ranks_reproduce_the_single_rank_tallies():
    import torch.multiprocessing as mp
    import oracle
    from paper_2402_09222_b300 import synth
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    total, slowest = q.get(timeout=300)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    prob = synth.config3_problem(n_histories=3001, lattice_n=5, n_points=300)
    ref = oracle.transport(prob, seed=77, derivatives=True)
    for k in ("flux", "absorb", "outcome", "dflux", "dabsorb", "doutcome"):
        np.testing.assert_allclose(total[k], ref[k], rtol=1e-12, atol=1e-12 * np.abs(ref[k]).max())
    assert slowest == 11.0

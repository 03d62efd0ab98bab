"""The N > 1 path of bench.py on CPU: world_size 2 over gloo (127.0.0.1).
Ranks take disjoint, adjacent counter shards of one stream (Section 3's
division of the counter space among cores), so the union of the ranks'
outputs -- computed here with the oracle, since there is no GPU -- is one
contiguous stream; the job time is the maximum over ranks. No collective
touches the data."""
import os
import socket

import numpy as np
import pytest


def _free_port() -> int:
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, n, results):
    import torch.distributed as dist

    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank),
                      WORLD_SIZE=str(world))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        import bench
        import oracle
        from paper_2004_06278_gb300 import workloads

        key = int(oracle.make_keys(2, 1)[0])
        base = workloads.throughput_base(3)
        mine = bench.shard_base(base, n, rank)
        out = oracle.fill32(key, mine, n, threads=1)
        elapsed = bench.max_over_ranks(0.5 + rank, world)
        results[rank] = (mine, out, elapsed)
    finally:
        dist.destroy_process_group()


@pytest.mark.parametrize("world", [2])
def test_two_rank_shards(world):
    import torch.multiprocessing as mp

    import oracle
    from paper_2004_06278_gb300 import workloads

    n = 4099
    port = _free_port()
    with mp.Manager() as mgr:
        results = mgr.dict()
        mp.start_processes(_worker, args=(world, port, n, results), nprocs=world,
                           start_method="spawn", join=True)
        results = dict(results)
    key = int(oracle.make_keys(2, 1)[0])
    base = workloads.throughput_base(3)
    bases = [results[r][0] for r in range(world)]
    assert bases[0] == base and bases[1] == (base + n) % (1 << 64)
    union = np.concatenate([results[r][1] for r in range(world)])
    assert np.array_equal(union, oracle.fill32(key, base, world * n))
    assert all(results[r][2] == 0.5 + (world - 1) for r in range(world))


def test_shard_base_wraps():
    import bench

    assert bench.shard_base((1 << 64) - 3, 2, 2) == 1
    assert bench.max_over_ranks(1.25, 1) == 1.25

"""The multi-process path of bench.py on CPU: world size 2 over gloo. Each rank times its own
replica or shard (no data exchange); the job figures are the slowest rank's time and the sum of
all ranks' work."""
import os
import socket

import pytest

torch = pytest.importorskip("torch")
import torch.multiprocessing as mp  # noqa: E402


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _worker(rank, world, port, out):
    import torch.distributed as dist

    import bench
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    ms, units = bench.dist_aggregate(10.0 + 5.0 * rank, 100.0 * (rank + 1), world)
    lo, hi = bench.shard(512, rank, world)
    out[rank] = (ms, units, lo, hi)
    dist.barrier()
    dist.destroy_process_group()


def test_two_rank_aggregation_and_sharding():
    port = _free_port()
    with mp.Manager() as mgr:
        out = mgr.dict()
        mp.spawn(_worker, args=(2, port, out), nprocs=2, join=True)
        res = dict(out)
    for rank in (0, 1):
        ms, units, lo, hi = res[rank]
        assert ms == 15.0 and units == 300.0
    assert (res[0][2], res[0][3], res[1][2], res[1][3]) == (0, 256, 256, 512)


def test_shard_covers_every_matrix_once():
    import bench
    for count in (0, 1, 7, 512, 513):
        for world in (1, 2, 3, 8):
            parts = [bench.shard(count, r, world) for r in range(world)]
            assert parts[0][0] == 0 and parts[-1][1] == count
            assert all(parts[r][1] == parts[r + 1][0] for r in range(world - 1))
            assert max(h - l for l, h in parts) - min(h - l for l, h in parts) <= 1

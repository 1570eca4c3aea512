"""The benchmark's multi-process path on CPU: two gloo ranks, one replica each.

The benchmark shards nothing across GPUs (every rank runs an independent
replica); the only cross-rank steps are the barrier around the timed region
and the host-side reductions of the timed duration (max over ranks) and of
the walker-steps (sum over ranks).  These run here as two gloo processes.
"""
import os
import socket
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket(socket.AF_INET, socket.SOCK_STREAM) as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, out_dir):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), WORLD_SIZE=str(world), RANK=str(rank),
                      LOCAL_RANK=str(rank))
    sys.path.insert(0, ROOT)
    import bench
    w, r, local, pg = bench.dist_setup(world)
    try:
        assert (w, r, local) == (world, rank, rank)
        bench.barrier(pg)
        # per-rank duration and work, as in the timed region
        t_max = bench.reduce_max(pg, 10.0 + rank)
        ws = bench.reduce_sum(pg, 1000.0 * (rank + 1))
        with open(os.path.join(out_dir, "rank%d.txt" % rank), "w") as f:
            f.write("%r %r\n" % (t_max, ws))
    finally:
        pg.destroy_process_group()


def test_two_rank_reductions(tmp_path):
    torch = pytest.importorskip("torch")
    import torch.multiprocessing as mp
    world = 2
    mp.start_processes(_rank_main, args=(world, _free_port(), str(tmp_path)), nprocs=world, join=True,
                       start_method="spawn")
    for rank in range(world):
        t_max, ws = (float(x) for x in (tmp_path / ("rank%d.txt" % rank)).read_text().split())
        assert t_max == 11.0                 # the slowest rank's time
        assert ws == 3000.0                  # walker-steps of all ranks


def test_single_process_needs_no_group():
    sys.path.insert(0, ROOT)
    import bench
    old = {k: os.environ.pop(k, None) for k in ("WORLD_SIZE", "RANK", "LOCAL_RANK")}
    try:
        world, rank, local, pg = bench.dist_setup(1)
        assert (world, rank, local, pg) == (1, 0, 0, None)
        assert bench.reduce_max(pg, 2.5) == 2.5 and bench.reduce_sum(pg, 7.0) == 7.0
        bench.barrier(pg)
    finally:
        for k, v in old.items():
            if v is not None:
                os.environ[k] = v

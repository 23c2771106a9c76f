"""The N > 1 host path of bench.py on CPU: two gloo ranks (127.0.0.1), each
with its own shard seed, a barrier, and the max-over-ranks timing that the
whole-job value is computed from.  No GPU and no collective on data."""
import os
import socket
import sys

import numpy as np
import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, out_dir):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank),
                      WORLD_SIZE=str(world), LOCAL_RANK=str(rank))
    sys.path.insert(0, ROOT)
    import bench
    from paper_2212_10733_gb300 import synth
    dist.init_process_group("gloo", rank=rank, world_size=world)
    # each rank's shard is different data
    x = synth.histograms(8, bench.shard_seed(synth, rank))
    # a rank-dependent "step time"; the job time is the slowest rank's
    ms = 10.0 + 5.0 * rank
    bench.barrier(world)
    mx = bench.max_over_ranks(ms, world)
    val = bench.job_value(1024, mx, world)
    np.save(os.path.join(out_dir, f"r{rank}.npy"), np.concatenate([[mx, val], x.ravel()]))
    dist.barrier()
    dist.destroy_process_group()


def test_two_gloo_ranks_shard_and_take_the_slowest_time(tmp_path):
    world, port = 2, _free_port()
    mp.start_processes(_rank_main, args=(world, port, str(tmp_path)), nprocs=world,
                       join=True, start_method="spawn")
    r0 = np.load(tmp_path / "r0.npy")
    r1 = np.load(tmp_path / "r1.npy")
    # both ranks see the maximum (rank 1's 15 ms) and the same job value
    assert r0[0] == r1[0] == 15.0
    assert r0[1] == r1[1] == pytest.approx(2 * 1024 / 0.015)
    # the shards differ
    assert not np.array_equal(r0[2:], r1[2:])

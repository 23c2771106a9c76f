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


# --- subdomain partitioning (Sec. III Stage 1: every processor compresses its
# own subdomains; the per-processor buffers are written one after another) ---

def _lpt_reference(counts, R):
    """The longest-processing-time rule written out: decreasing counts (ties
    by index), each to the least-loaded rank (ties by rank)."""
    order = sorted(range(len(counts)), key=lambda g: (-counts[g], g))
    load = [0] * R
    owner = [0] * len(counts)
    for g in order:
        r = min(range(R), key=lambda q: (load[q], q))
        owner[g] = r
        load[r] += counts[g]
    return owner, load


def test_lpt_partition_against_brute_force():
    import itertools
    from paper_2212_10733_gb300 import aeqc
    rng = np.random.default_rng(5)
    for trial in range(60):
        R = int(rng.integers(2, 4))
        G = int(rng.integers(0, 8))
        counts = rng.integers(0, 50, size=G).astype(np.int64)
        if trial % 5 == 0:
            counts[:] = 7  # ties everywhere
        owner, load = aeqc.partition_lpt(counts, R)
        want_o, want_l = _lpt_reference(list(counts), R)
        assert list(owner) == want_o and list(load) == want_l
        for r in range(R):
            assert load[r] == counts[owner == r].sum()
        # the optimum by exhaustion; LPT is within (4/3 - 1/(3R)) of it
        best = min((max(sum(int(c) for c, a in zip(counts, asg) if a == r) for r in range(R))
                    for asg in itertools.product(range(R), repeat=G)), default=0)
        assert load.max() <= (4.0 / 3.0 - 1.0 / (3 * R)) * best + 1e-9
    with pytest.raises(aeqc.AeqcError):
        aeqc.partition_lpt([3, -1], 2)
    with pytest.raises(aeqc.AeqcError):
        aeqc.partition_lpt([3], 0)


def test_exclusive_scan():
    from paper_2212_10733_gb300 import aeqc
    assert list(aeqc.exclusive_scan([])) == [0]
    assert list(aeqc.exclusive_scan([5, 0, 7])) == [0, 5, 5, 12]
    with pytest.raises(aeqc.AeqcError):
        aeqc.exclusive_scan([1, -1])
    with pytest.raises(aeqc.AeqcError):
        aeqc.exclusive_scan([2 ** 62, 2 ** 62])


def _partition_rank(rank, world, port, out_path, G):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank),
                      WORLD_SIZE=str(world), LOCAL_RANK=str(rank))
    sys.path.insert(0, ROOT)
    from paper_2212_10733_gb300 import aeqc, synth
    dist.init_process_group("gloo", rank=rank, world_size=world)
    sizes = synth.group_sizes(G, synth.config_seed(3))
    owner, load = aeqc.partition_lpt(sizes, world)
    mine = np.nonzero(owner == rank)[0]
    # this rank's compressed batch: the container size of its histograms
    n_r = int(sizes[mine].sum())
    nbytes = int(aeqc.load().aeqc_batch_pack_size(n_r, synth.P, 32, aeqc.DTYPE_BF16, 0))
    # every rank computed the same assignment without exchanging it; the one
    # exchange is the 8-byte count per rank
    got = [None] * world
    dist.all_gather_object(got, dict(owner=owner.tolist(), nbytes=nbytes))
    assert all(g["owner"] == owner.tolist() for g in got)
    off = aeqc.exclusive_scan([g["nbytes"] for g in got])
    # write this rank's bytes at its offset of the shared output
    out = np.memmap(out_path, dtype=np.uint8, mode="r+")
    out[off[rank]:off[rank + 1]] = rank + 1
    out.flush()
    del out
    dist.barrier()
    if rank == 0:
        np.save(out_path + ".meta.npy", np.concatenate([off, load, [G]]))
    dist.barrier()
    dist.destroy_process_group()


def test_three_gloo_ranks_partition_subdomains_and_tile_the_output(tmp_path):
    from paper_2212_10733_gb300 import aeqc, synth
    world, port, G = 3, _free_port(), 256
    sizes = synth.group_sizes(G, synth.config_seed(3))
    owner, load = aeqc.partition_lpt(sizes, world)
    total = sum(int(aeqc.load().aeqc_batch_pack_size(int(sizes[owner == r].sum()), synth.P, 32,
                                                     aeqc.DTYPE_BF16, 0)) for r in range(world))
    path = str(tmp_path / "out.bin")
    np.memmap(path, dtype=np.uint8, mode="w+", shape=(total,)).flush()
    mp.start_processes(_partition_rank, args=(world, port, path, G), nprocs=world, join=True,
                       start_method="spawn")
    meta = np.load(path + ".meta.npy")
    off = meta[:world + 1]
    assert off[0] == 0 and off[-1] == total and np.all(np.diff(off) > 0)
    out = np.fromfile(path, dtype=np.uint8)
    # each rank's bytes exactly at its range, nothing unwritten
    for r in range(world):
        assert np.all(out[off[r]:off[r + 1]] == r + 1)
    # load balance of the 256 lognormal subdomains: within 1 % of the mean
    assert load.max() <= 1.01 * sizes.sum() / world
    assert load.sum() == sizes.sum()

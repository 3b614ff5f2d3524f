"""Multi-process path on CPU (gloo, world size 2).

Each rank generates its shard with the oracle (CPU) exactly as the benchmark
shards work over GPUs; rank outputs gathered together must equal a single
process generating all the streams, and the max-over-ranks timing reduction
must return the largest rank value.
"""
import os
import socket

import numpy as np
import pytest
import torch.multiprocessing as mp

import oracle
from paper_1501_07701_gb300 import dist as mdist
from paper_1501_07701_gb300 import workloads


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, mode, q):
    import torch
    import torch.distributed as dist
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        p = oracle.params_generate(workloads.MEXP_MAIN, workloads.PARAM_SEED)
        counts_all = workloads.uneven_counts(24, lo=5, hi=12, seed=3)
        seeds_all = np.arange(24, dtype=np.uint32)
        if mode == "weak":
            seeds = mdist.weak_seeds(seeds_all, rank)
            counts = counts_all
        else:
            a, b = mdist.strong_range(24, rank, world)
            seeds, counts = seeds_all[a:b], counts_all[a:b]
        states = np.stack([oracle.init_state(p, int(s)) for s in seeds])
        out, _ = oracle.generate_many(p, states, np.arange(seeds.size), counts, 0, 1)
        t = torch.from_numpy(out.view(np.int32).copy())
        sizes = [torch.zeros(1, dtype=torch.int64) for _ in range(world)]
        dist.all_gather(sizes, torch.tensor([t.numel()], dtype=torch.int64))
        mx_size = max(int(s.item()) for s in sizes)
        padded = torch.zeros(mx_size, dtype=torch.int32)
        padded[:t.numel()] = t
        bufs = [torch.zeros(mx_size, dtype=torch.int32) for _ in sizes]
        dist.all_gather(bufs, padded)
        bufs = [b[:int(s.item())] for b, s in zip(bufs, sizes)]
        mx = mdist.max_over_ranks(float(rank + 1) * 1.5)
        if rank == 0:
            q.put((np.concatenate([b.numpy() for b in bufs]).view(np.uint32), mx))
        dist.barrier()
    finally:
        dist.destroy_process_group()


@pytest.mark.parametrize("mode", ["weak", "strong"])
def test_two_ranks_match_single_process(mode):
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, mode, q)) for r in range(2)]
    for pr in procs:
        pr.start()
    got, mx = q.get(timeout=90)
    for pr in procs:
        pr.join(timeout=60)
        assert pr.exitcode == 0
    p = oracle.params_generate(workloads.MEXP_MAIN, workloads.PARAM_SEED)
    counts_all = workloads.uneven_counts(24, lo=5, hi=12, seed=3)
    if mode == "weak":
        seeds = np.arange(48, dtype=np.uint32)
        counts = np.concatenate([counts_all, counts_all])
    else:
        seeds = np.arange(24, dtype=np.uint32)
        counts = counts_all
    states = np.stack([oracle.init_state(p, int(s)) for s in seeds])
    ref, _ = oracle.generate_many(p, states, np.arange(seeds.size), counts, 0, 2)
    assert np.array_equal(got, ref)
    assert mx == 3.0


def test_strong_ranges_partition():
    for n in (1, 7, 24, 10000):
        for world in (1, 2, 3, 8):
            rs = [mdist.strong_range(n, r, world) for r in range(world)]
            assert rs[0][0] == 0 and rs[-1][1] == n
            for (a, b), (c, d) in zip(rs, rs[1:]):
                assert b == c and b >= a


def _bench_worker(rank, world, port, split, q):
    """One rank of bench.py's own multi-rank control path on gloo: the shard
    this rank would run, the barrier-bracketed timed region and the
    whole-job rate (numbers summed over ranks / slowest rank's time)."""
    import argparse
    import time
    import torch.distributed as dist
    import bench
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        args = argparse.Namespace(workload="uneven", streams=0, count=0, param_sets=0, mexp=0,
                                  rank_split=split)
        w, desc = bench.rank_workload(args, rank, world)
        syncs = []
        with bench.bracket(dist, lambda: syncs.append(time.monotonic())):
            t_local = 0.5 + rank          # rank 1 is the slowest
        value, elapsed, numbers = bench.job_rate(int(w["counts"].sum()), t_local)
        shards = [None] * world
        dist.all_gather_object(shards, (w["seeds"].tolist(), w["counts"].tolist(), desc))
        if rank == 0:
            q.put((shards, value, elapsed, numbers, len(syncs)))
        dist.barrier()
    finally:
        dist.destroy_process_group()


@pytest.mark.parametrize("split", ["weak", "strong"])
def test_bench_control_path_two_ranks(split):
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_bench_worker, args=(r, 2, port, split, q)) for r in range(2)]
    for pr in procs:
        pr.start()
    shards, value, elapsed, numbers, n_sync = q.get(timeout=120)
    for pr in procs:
        pr.join(timeout=60)
        assert pr.exitcode == 0
    full = workloads.uneven()
    (s0, c0, d0), (s1, c1, d1) = shards
    if split == "strong":
        # one instance cut into two contiguous ranges that cover it exactly
        assert s0 + s1 == full["seeds"].tolist() and c0 + c1 == full["counts"].tolist()
        assert abs(len(s0) - len(s1)) <= 1 and "contiguous" in d0
        assert numbers == float(full["counts"].sum())
    else:
        # two instances of the whole workload with disjoint stream seeds
        assert c0 == c1 == full["counts"].tolist() and not set(s0) & set(s1)
        assert numbers == 2.0 * float(full["counts"].sum())
    assert elapsed == 1.5 and n_sync == 2
    assert value == pytest.approx(numbers / 1.5 / 1e9)

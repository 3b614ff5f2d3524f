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

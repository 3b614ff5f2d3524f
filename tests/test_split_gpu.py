"""Split plans: long streams cut into pieces that start from exact jumps.

A split plan must produce exactly the outputs and final states of the same
plan unsplit, and both must equal the oracle's sequential generation
(tolerance 0).  The cases vary the piece length around the state size N and
the step widths, streams with several requests whose boundaries fall inside
pieces, every format, plan replays (states carry over), per-stream
parameter sets, the short-state register kernel (Mexp 3217), the ring
kernel, autotuning and the one-stream workload.
"""
import os

import numpy as np
import pytest

import oracle
from paper_1501_07701_gb300 import mtgp, workloads

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")
THREADS = os.cpu_count() or 4
FMTS = [mtgp.MTGP_U32, mtgp.MTGP_F32_12, mtgp.MTGP_F32_01]


@pytest.fixture(scope="module", autouse=True)
def _built():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1501_07701_gb300 import build
    build.build()
    mtgp.load_library()


def _same(a, b, what):
    a, b = np.asarray(a, np.uint32), np.asarray(b, np.uint32)
    assert a.shape == b.shape, what
    bad = np.nonzero(a != b)[0]
    assert bad.size == 0, "%s: %d mismatches, first at %d" % (what, bad.size, bad[0])


def _run_plan(st, ids, counts, fmt, max_piece, reps=2, cfg=None, autotune=False):
    """Outputs of `reps` launches of a plan (split when max_piece > 0) and
    the plan's info."""
    total = int(np.asarray(counts, np.uint64).sum())
    out = torch.full((total + 4,), -1, dtype=torch.int32, device="cuda")
    if cfg:
        mtgp.mtgp_set_launch_config(st, **cfg)
    plan = mtgp.mtgp_plan_create(st, ids, counts, fmt, out[:total])
    if max_piece:
        mtgp.mtgp_plan_set_split(plan, max_piece)
    if autotune:
        mtgp.mtgp_plan_autotune(plan)
    info = mtgp.mtgp_plan_get_info(plan)
    outs = []
    for _ in range(reps):
        mtgp.mtgp_plan_launch(plan)
        torch.cuda.synchronize()
        mtgp.mtgp_check(st)
        host = out.cpu().numpy().view(np.uint32)
        assert np.all(host[total:] == 0xFFFFFFFF)
        outs.append(host[:total].copy())
    return outs, info


@pytest.mark.parametrize("max_piece", [64, 350, 351, 352, 1000, 4096, 33333])
@pytest.mark.parametrize("fmt", FMTS)
def test_split_equals_unsplit_and_oracle(max_piece, fmt):
    gp = mtgp.mtgp_params_generate(11213, workloads.PARAM_SEED)
    op = oracle.params_generate(11213, workloads.PARAM_SEED)
    rng = np.random.default_rng(max_piece + fmt)
    n = 20
    ids = np.concatenate([np.arange(n), rng.integers(0, n, 12)]).astype(np.uint32)
    counts = rng.integers(1, 60000, ids.size).astype(np.uint64)
    counts[:3] = [200000, 1, 351 * 7]
    a = mtgp.mtgp_init_statuses(gp, np.arange(n, dtype=np.uint32))
    b = mtgp.mtgp_init_statuses(gp, np.arange(n, dtype=np.uint32))
    states = mtgp.mtgp_get_statuses(a)
    got_split, info = _run_plan(a, ids, counts, fmt, max_piece)
    got_plain, _ = _run_plan(b, ids, counts, fmt, 0)
    assert info["max_piece"] == max_piece and info["n_split_streams"] > 0
    assert info["n_jumps"] == info["n_items"] - n   # one jump per piece after a stream's first
    for rep in range(2):
        ref, states = oracle.generate_many(op, states, ids, counts, fmt, THREADS)
        _same(got_split[rep], ref, "split, launch %d" % rep)
        _same(got_plain[rep], ref, "unsplit, launch %d" % rep)
    _same(mtgp.mtgp_get_statuses(a), states, "split states")
    _same(mtgp.mtgp_get_statuses(b), states, "unsplit states")


@pytest.mark.parametrize("mexp,cfg", [
    (3217, dict(warps_per_cta=4, words_per_lane=2, kernel=0)),
    (23209, dict(warps_per_cta=8, words_per_lane=4, kernel=0, ctas_per_sm=1)),
    (44497, dict(warps_per_cta=4, words_per_lane=4, kernel=0, ctas_per_sm=2)),
    (11213, dict(warps_per_cta=4, words_per_lane=8, kernel=1)),
    (11213, dict(warps_per_cta=8, words_per_lane=8, kernel=0, coop_percent=50)),
])
def test_split_exponents_and_kernels(mexp, cfg):
    gp = mtgp.mtgp_params_generate(mexp, workloads.PARAM_SEED)
    op = oracle.params_generate(mexp, workloads.PARAM_SEED)
    n = 12
    st = mtgp.mtgp_init_statuses(gp, np.arange(n, dtype=np.uint32))
    states = mtgp.mtgp_get_statuses(st)
    ids = np.arange(n, dtype=np.uint32)
    counts = np.array([300000, 150001, 5, op.n * 9, 77777, 1, 2, 3, 40000, 0, 90000, op.n], np.uint64)
    got, info = _run_plan(st, ids, counts, mtgp.MTGP_U32, 20000, cfg=cfg)
    assert info["n_split_streams"] == 5
    for rep in range(2):
        ref, states = oracle.generate_many(op, states, ids, counts, 0, THREADS)
        _same(got[rep], ref, "mexp %d launch %d" % (mexp, rep))
    _same(mtgp.mtgp_get_statuses(st), states, "states")


def test_split_per_stream_parameter_sets():
    set_seeds = [workloads.PARAM_SEED + 1 + k for k in range(4)]
    gsets = [mtgp.mtgp_params_generate(11213, k) for k in set_seeds]
    osets = [oracle.params_generate(11213, k) for k in set_seeds]
    n = 10
    set_of = (np.arange(n) % 4).astype(np.uint32)
    st = mtgp.mtgp_init_statuses_multi(gsets, set_of, np.arange(n, dtype=np.uint32))
    states = mtgp.mtgp_get_statuses(st)
    ids = np.array([0, 1, 2, 3, 4, 5, 6, 7, 8, 9, 1, 2], np.uint32)
    counts = np.array([100000, 50000, 3, 70001, 9, 1000, 25000, 60000, 10, 1, 30000, 44444], np.uint64)
    got, info = _run_plan(st, ids, counts, mtgp.MTGP_F32_01, 9000)
    assert info["n_split_streams"] >= 5
    offs = np.concatenate([[0], np.cumsum(counts.astype(np.int64))])
    for rep in range(2):
        for j, (sid, c) in enumerate(zip(ids, counts)):
            ref, states[sid] = oracle.generate(osets[set_of[sid]], states[sid], int(c), 2)
            _same(got[rep][offs[j]:offs[j + 1]], ref, "launch %d request %d" % (rep, j))
    _same(mtgp.mtgp_get_statuses(st), states, "states")


def test_split_with_autotune_and_trace():
    gp = mtgp.mtgp_params_generate(11213, workloads.PARAM_SEED)
    op = oracle.params_generate(11213, workloads.PARAM_SEED)
    w = workloads.uneven(400)
    st = mtgp.mtgp_init_statuses(gp, w["seeds"])
    states = mtgp.mtgp_get_statuses(st)
    counts = w["counts"] // 4 + 1
    ids = np.arange(counts.size, dtype=np.uint32)
    out = torch.empty(int(counts.sum()), dtype=torch.int32, device="cuda")
    plan = mtgp.mtgp_plan_create(st, ids, counts, mtgp.MTGP_U32, out)
    mtgp.mtgp_plan_set_split(plan, int(counts.max()) // 3)
    mtgp.mtgp_plan_autotune(plan)
    mtgp.mtgp_plan_set_trace(plan, True)
    info = mtgp.mtgp_plan_get_info(plan)
    assert info["n_split_streams"] > 0 and info["kernel_launches"] == 4
    mtgp.mtgp_plan_launch(plan)
    torch.cuda.synchronize()
    ref, states = oracle.generate_many(op, states, ids, counts, 0, THREADS)
    _same(out.cpu().numpy().view(np.uint32), ref, "outputs")
    _same(mtgp.mtgp_get_statuses(st), states, "states")
    tr = mtgp.mtgp_plan_read_trace(plan).reshape(-1, 4)
    assert tr.shape[0] == info["n_items"] and int(tr[:, 3].sum()) == int(counts.sum())
    # removing the split restores one item per stream
    mtgp.mtgp_plan_set_split(plan, 0)
    info = mtgp.mtgp_plan_get_info(plan)
    assert info["n_items"] == counts.size and info["n_jumps"] == 0 and info["kernel_launches"] == 1
    mtgp.mtgp_plan_launch(plan)
    torch.cuda.synchronize()
    ref, states = oracle.generate_many(op, states, ids, counts, 0, THREADS)
    _same(out.cpu().numpy().view(np.uint32), ref, "outputs unsplit again")


def test_single_stream_split_into_64_pieces():
    """The one-stream workload (2^20 numbers of seed 1): 64 pieces advanced
    by 64 warps, the 63 later ones from jumps."""
    gp = mtgp.mtgp_params_generate(11213, workloads.PARAM_SEED)
    op = oracle.params_generate(11213, workloads.PARAM_SEED)
    st = mtgp.mtgp_init_statuses(gp, np.array([1], np.uint32))
    got, info = _run_plan(st, [0], [1 << 20], mtgp.MTGP_U32, 1 << 14)
    assert info["n_items"] == 64 and info["n_jumps"] == 63
    s0 = oracle.init_state(op, 1)
    ref, s1 = oracle.generate(op, s0, 1 << 20)
    _same(got[0], ref, "launch 0")
    ref, s2 = oracle.generate(op, s1, 1 << 20)
    _same(got[1], ref, "launch 1")
    _same(mtgp.mtgp_get_statuses(st)[0], s2, "state")


def test_split_rejects_tiny_pieces():
    gp = mtgp.mtgp_params_generate(11213, workloads.PARAM_SEED)
    st = mtgp.mtgp_init_statuses(gp, np.arange(2, dtype=np.uint32))
    out = torch.empty(2000, dtype=torch.int32, device="cuda")
    plan = mtgp.mtgp_plan_create(st, [0, 1], [1000, 1000], mtgp.MTGP_U32, out)
    with pytest.raises(mtgp.MtgpError) as ei:
        mtgp.mtgp_plan_set_split(plan, 63)
    assert ei.value.status == 1

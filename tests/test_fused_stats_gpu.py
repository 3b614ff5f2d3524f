"""Statistics fused into generation (tests 35 and 100 of Sec. 4.2).

A plan with mtgp_plan_set_stats must store exactly the outputs and states of
the plain plan, and its per-request gap histograms and Hamming block-pair
tables must equal the oracle's (oracle.gap_histogram / oracle.hamming_pairs
over the oracle's outputs of each request; tolerance 0) and the standalone
GPU reductions over the same output buffer.  The cases vary the field
positions and widths (mask at the top, at the bottom, one bit), t from 1 to
1023, the block length down to its minimum of 32 values, 0 to 15 class
bounds, requests of 0, 1, < N, = N and many rows, several requests per
stream, plan replays, every format, per-stream parameter sets, the three
state sizes and autotuning; split plans, whose requests are counted in
pieces and stitched, with piece lengths around the state size and the
Hamming pair length; then the refusals.
"""
import os

import numpy as np
import pytest

import oracle
from paper_1501_07701_gb300 import mtgp, quality, workloads

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")
THREADS = os.cpu_count() or 4
PAPER = dict(gap=(25, 5, 128), hamming=(25, 5, 1200, quality.default_hamming_bounds(1200, 4)))


@pytest.fixture(scope="module", autouse=True)
def _built():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1501_07701_gb300 import build
    build.build()
    mtgp.load_library()


def _same(a, b, what):
    a, b = np.asarray(a), np.asarray(b)
    assert a.shape == b.shape, "%s: shapes %s vs %s" % (what, a.shape, b.shape)
    bad = np.argwhere(a != b)
    assert bad.size == 0, "%s: %d mismatches, first at %s (%s vs %s)" % (
        what, len(bad), bad[0], a[tuple(bad[0])], b[tuple(bad[0])])


def _requests(rng, n_streams, n_extra, n, big):
    ids = np.concatenate([np.arange(n_streams), rng.integers(0, n_streams, n_extra)]).astype(np.uint32)
    rng.shuffle(ids)
    counts = rng.integers(0, 5000, ids.size).astype(np.uint64)
    special = [0, 1, n - 1, n, n + 1, 3 * n, big]
    counts[:len(special)] = special
    return ids, counts


def _oracle_stats(ref, counts, gap, hamming):
    offs = np.concatenate([[0], np.cumsum(counts.astype(np.int64))])
    hs, ts = [], []
    for j in range(counts.size):
        x = ref[offs[j]:offs[j + 1]]
        if gap:
            hs.append(oracle.gap_histogram(x, *gap))
        if hamming:
            r, s, L, bounds = hamming
            ts.append(oracle.hamming_pairs(x, r, s, L, bounds))
    return (np.array(hs) if gap else None), (np.array(ts) if hamming else None)


def _run(st, op, ids, counts, fmt, gap, hamming, reps=2, cfg=None, autotune=False, sets=None, split=0,
         split_first=False):
    """Launches a statistics plan `reps` times; checks outputs, states and
    statistics against the oracle after every launch.  split: piece length
    of a split plan (set before or after the statistics)."""
    total = int(counts.sum())
    out = torch.full((total + 4,), -1, dtype=torch.int32, device="cuda")
    if cfg:
        mtgp.mtgp_set_launch_config(st, **cfg)
    plan = mtgp.mtgp_plan_create(st, ids, counts, fmt, out[:total])
    if split and split_first:
        mtgp.mtgp_plan_set_split(plan, split)
    mtgp.mtgp_plan_set_stats(plan, gap=gap, hamming=hamming)
    if split and not split_first:
        mtgp.mtgp_plan_set_split(plan, split)
    if autotune:
        mtgp.mtgp_plan_autotune(plan)
    info = mtgp.mtgp_plan_get_info(plan)
    assert info["stats"]
    if split:
        assert info["n_split_streams"] > 0 and info["max_piece"] == split
    else:
        assert info["kernel_launches"] == 1
    states = mtgp.mtgp_get_statuses(st)
    for rep in range(reps):
        # the statistics are rewritten by every launch
        mtgp.mtgp_plan_launch(plan)
        torch.cuda.synchronize()
        mtgp.mtgp_check(st)
        host = out.cpu().numpy().view(np.uint32)
        assert np.all(host[total:] == 0xFFFFFFFF), "write past the output"
        if sets is None:
            ref, states = oracle.generate_many(op, states, ids, counts, fmt, THREADS)
        else:
            osets, set_of = sets
            offs = np.concatenate([[0], np.cumsum(counts.astype(np.int64))])
            ref = np.zeros(total, np.uint32)
            for j, (sid, c) in enumerate(zip(ids, counts)):
                ref[offs[j]:offs[j + 1]], states[sid] = oracle.generate(osets[set_of[sid]], states[sid],
                                                                        int(c), fmt)
        _same(host[:total], ref, "outputs, launch %d" % rep)
        hist, tab = mtgp.mtgp_plan_read_stats(plan)
        want_h, want_t = _oracle_stats(ref, counts, gap, hamming)
        if gap:
            _same(hist, want_h, "gap histograms, launch %d" % rep)
        else:
            assert hist is None
        if hamming:
            _same(tab, want_t, "Hamming tables, launch %d" % rep)
        else:
            assert tab is None
    _same(mtgp.mtgp_get_statuses(st), states, "states")
    return plan, out, info


CASES = [
    # (gap (r, b, t), hamming (r, s, L, bounds))
    ((25, 5, 128), (25, 5, 1200, quality.default_hamming_bounds(1200, 4))),
    ((0, 1, 7), (0, 1, 32, [])),                        # top bit; minimum block of 32 values
    ((20, 10, 1023), (27, 5, 160, [10, 12, 14, 16, 18])),  # rare visits, long pooled gaps
    ((31, 1, 1), (31, 1, 50, list(range(10, 40, 2))[:15])),  # bottom bit, t = 1, 15 bounds
    ((25, 5, 128), None),
    (None, (25, 5, 1200, [590, 600, 610])),
]


@pytest.mark.parametrize("case", range(len(CASES)))
def test_fused_stats_equal_oracle(case):
    gap, hamming = CASES[case]
    gp = mtgp.mtgp_params_generate(11213, workloads.PARAM_SEED)
    op = oracle.params_generate(11213, workloads.PARAM_SEED)
    rng = np.random.default_rng(100 + case)
    n = 40
    ids, counts = _requests(rng, n, 25, op.n, 150000)
    st = mtgp.mtgp_init_statuses(gp, np.arange(n, dtype=np.uint32))
    _run(st, op, ids, counts, mtgp.MTGP_U32, gap, hamming)


@pytest.mark.parametrize("fmt", [mtgp.MTGP_F32_12, mtgp.MTGP_F32_01])
def test_fused_stats_float_formats(fmt):
    """Float formats: the statistics are those of the stored bit patterns."""
    gp = mtgp.mtgp_params_generate(11213, workloads.PARAM_SEED)
    op = oracle.params_generate(11213, workloads.PARAM_SEED)
    rng = np.random.default_rng(7 + fmt)
    ids, counts = _requests(rng, 16, 8, op.n, 60000)
    st = mtgp.mtgp_init_statuses(gp, np.arange(16, dtype=np.uint32))
    _run(st, op, ids, counts, fmt, (9, 5, 64), (9, 5, 600, [40, 50, 60]))


@pytest.mark.parametrize("mexp", [23209, 44497])
def test_fused_stats_larger_states(mexp):
    gp = mtgp.mtgp_params_generate(mexp, workloads.PARAM_SEED)
    op = oracle.params_generate(mexp, workloads.PARAM_SEED)
    rng = np.random.default_rng(mexp)
    ids, counts = _requests(rng, 12, 6, op.n, 200000)
    st = mtgp.mtgp_init_statuses(gp, np.arange(12, dtype=np.uint32))
    _run(st, op, ids, counts, mtgp.MTGP_U32, **PAPER)


def test_fused_stats_per_stream_sets_and_autotune():
    set_seeds = [workloads.PARAM_SEED + 1 + k for k in range(3)]
    gsets = [mtgp.mtgp_params_generate(11213, k) for k in set_seeds]
    osets = [oracle.params_generate(11213, k) for k in set_seeds]
    n = 20
    set_of = (np.arange(n) % 3).astype(np.uint32)
    st = mtgp.mtgp_init_statuses_multi(gsets, set_of, np.arange(n, dtype=np.uint32))
    rng = np.random.default_rng(3)
    ids, counts = _requests(rng, n, 10, osets[0].n, 80000)
    _run(st, osets[0], ids, counts, mtgp.MTGP_U32, reps=1, autotune=True, sets=(osets, set_of), **PAPER)


@pytest.mark.parametrize("cfg", [dict(warps_per_cta=8, ctas_per_sm=2, words_per_lane=4, kernel=0),
                                 dict(warps_per_cta=2, ctas_per_sm=1, words_per_lane=4, kernel=0)])
def test_fused_stats_launch_shapes(cfg):
    """More streams than warps (work stealing) at 16 and at 8 warps per SM."""
    gp = mtgp.mtgp_params_generate(11213, workloads.PARAM_SEED)
    op = oracle.params_generate(11213, workloads.PARAM_SEED)
    w = workloads.uneven(3000)
    counts = (w["counts"] // 64).astype(np.uint64)
    ids = np.arange(counts.size, dtype=np.uint32)
    st = mtgp.mtgp_init_statuses(gp, w["seeds"])
    plan, _, info = _run(st, op, ids, counts, mtgp.MTGP_U32, reps=1, cfg=cfg, **PAPER)
    assert info["config"]["warps_per_cta"] == 8


SPLIT_CASES = [
    (64, PAPER["gap"], PAPER["hamming"]),
    (350, (0, 1, 7), (0, 1, 32, [])),
    (351, (20, 10, 1023), (27, 5, 160, [10, 12, 14, 16, 18])),
    (480, PAPER["gap"], PAPER["hamming"]),
    (1000, (31, 1, 1), (31, 1, 50, list(range(10, 40, 2))[:15])),
    (4096, PAPER["gap"], (25, 5, 1200, [590, 600, 610])),
    (33333, PAPER["gap"], PAPER["hamming"]),
]


@pytest.mark.parametrize("case", range(len(SPLIT_CASES)))
def test_fused_stats_split_plans(case):
    """Requests cut into pieces on several warps: the pieces' counts and the
    stitched edges equal the oracle's counts of the whole requests."""
    max_piece, gap, hamming = SPLIT_CASES[case]
    gp = mtgp.mtgp_params_generate(11213, workloads.PARAM_SEED)
    op = oracle.params_generate(11213, workloads.PARAM_SEED)
    rng = np.random.default_rng(500 + case)
    n = 24
    ids, counts = _requests(rng, n, 12, op.n, 120000)
    st = mtgp.mtgp_init_statuses(gp, np.arange(n, dtype=np.uint32))
    _run(st, op, ids, counts, mtgp.MTGP_U32, gap, hamming, split=max_piece, split_first=case % 2 == 0)


@pytest.mark.parametrize("mexp", [23209, 44497])
def test_fused_stats_split_larger_states(mexp):
    gp = mtgp.mtgp_params_generate(mexp, workloads.PARAM_SEED)
    op = oracle.params_generate(mexp, workloads.PARAM_SEED)
    rng = np.random.default_rng(mexp + 1)
    ids, counts = _requests(rng, 10, 5, op.n, 300000)
    st = mtgp.mtgp_init_statuses(gp, np.arange(10, dtype=np.uint32))
    _run(st, op, ids, counts, mtgp.MTGP_F32_01, **PAPER, split=50000)


def test_fused_stats_split_sets_autotune_16_warps():
    set_seeds = [workloads.PARAM_SEED + 7 + k for k in range(3)]
    gsets = [mtgp.mtgp_params_generate(11213, k) for k in set_seeds]
    osets = [oracle.params_generate(11213, k) for k in set_seeds]
    n = 16
    set_of = (np.arange(n) % 3).astype(np.uint32)
    st = mtgp.mtgp_init_statuses_multi(gsets, set_of, np.arange(n, dtype=np.uint32))
    rng = np.random.default_rng(9)
    ids, counts = _requests(rng, n, 8, osets[0].n, 200000)
    _run(st, osets[0], ids, counts, mtgp.MTGP_U32, reps=1, autotune=True, sets=(osets, set_of),
         cfg=dict(warps_per_cta=8, ctas_per_sm=2, words_per_lane=4, kernel=0), split=20000, **PAPER)


@pytest.mark.parametrize("mexp,split", [(3217, 0), (3217, 20000), (4253, 0)])
def test_fused_stats_short_states(mexp, split):
    """The paper's exponent (N = 101, N - pos < 128) and 4253 (N = 133): every
    row is counted one 32-column sub-step at a time; unsplit and split."""
    gp = mtgp.mtgp_params_generate(mexp, workloads.PARAM_SEED)
    op = oracle.params_generate(mexp, workloads.PARAM_SEED)
    rng = np.random.default_rng(mexp + split)
    ids, counts = _requests(rng, 20, 10, op.n, 150000)
    st = mtgp.mtgp_init_statuses(gp, np.arange(20, dtype=np.uint32))
    _run(st, op, ids, counts, mtgp.MTGP_U32, **PAPER, split=split)


def test_fused_stats_short_states_float_and_short_blocks():
    """Mexp 3217 in the [0, 1) float format, Hamming blocks of 32 values (one
    sub-step each) and a rarely visited gap interval."""
    gp = mtgp.mtgp_params_generate(3217, workloads.PARAM_SEED)
    op = oracle.params_generate(3217, workloads.PARAM_SEED)
    rng = np.random.default_rng(3217)
    ids, counts = _requests(rng, 12, 6, op.n, 90000)
    st = mtgp.mtgp_init_statuses(gp, np.arange(12, dtype=np.uint32))
    _run(st, op, ids, counts, mtgp.MTGP_F32_01, (20, 10, 1023), (9, 5, 160, [70, 80, 90]))


@pytest.mark.parametrize("gap_words", [40, 33])
def test_fused_stats_short_states_close_pick_up(gap_words):
    """A user set at Mexp 3217 with N - pos below 64 (no look-ahead read):
    every row goes through the sub-step-at-a-time slow path."""
    o = oracle.params_generate(3217, workloads.PARAM_SEED)
    op = oracle.params_from_fields(3217, o.n - gap_words, o.sh1, o.sh2, list(o.rec_basis), list(o.tmp_basis))
    gp = mtgp.mtgp_params_create(3217, op.pos, op.sh1, op.sh2, list(op.rec_tbl), list(op.tmp_tbl))
    rng = np.random.default_rng(gap_words)
    ids, counts = _requests(rng, 10, 5, op.n, 60000)
    st = mtgp.mtgp_init_statuses(gp, np.arange(10, dtype=np.uint32))
    _run(st, op, ids, counts, mtgp.MTGP_U32, **PAPER)


def test_fused_stats_plan_without_work():
    """Requests of zero numbers: no launch runs, and the counts read back are zeros."""
    gp = mtgp.mtgp_params_generate(11213, workloads.PARAM_SEED)
    st = mtgp.mtgp_init_statuses(gp, np.arange(3, dtype=np.uint32))
    out = torch.empty(4, dtype=torch.int32, device="cuda")
    plan = mtgp.mtgp_plan_create(st, [0, 1, 2], [0, 0, 0], mtgp.MTGP_U32, out)
    mtgp.mtgp_plan_set_stats(plan, **PAPER)
    mtgp.mtgp_plan_launch(plan)
    torch.cuda.synchronize()
    hist, tab = mtgp.mtgp_plan_read_stats(plan)
    assert hist.shape == (3, 129) and not hist.any()
    assert tab.shape == (3, 4, 4) and not tab.any()


def test_fused_counts_equal_standalone_kernels():
    """The fused counts equal the standalone reductions over the output."""
    gp = mtgp.mtgp_params_generate(11213, workloads.PARAM_SEED)
    w = workloads.uneven(2000)
    counts = (w["counts"] // 16).astype(np.uint64)
    ids = np.arange(counts.size, dtype=np.uint32)
    st = mtgp.mtgp_init_statuses(gp, w["seeds"])
    out = torch.empty(int(counts.sum()), dtype=torch.int32, device="cuda")
    plan = mtgp.mtgp_plan_create(st, ids, counts, mtgp.MTGP_U32, out)
    mtgp.mtgp_plan_set_stats(plan, **PAPER)
    mtgp.mtgp_plan_launch(plan)
    hist, tab = mtgp.mtgp_plan_read_stats(plan)
    r, s, L, bounds = PAPER["hamming"]
    _same(hist, mtgp.mtgp_gap_histogram(out, counts, *PAPER["gap"]), "gap histograms")
    _same(tab, mtgp.mtgp_hamming_pairs(out, counts, r, s, L, bounds), "Hamming tables")


def test_fused_stats_off_and_refusals():
    gp = mtgp.mtgp_params_generate(11213, workloads.PARAM_SEED)
    op = oracle.params_generate(11213, workloads.PARAM_SEED)
    st = mtgp.mtgp_init_statuses(gp, np.arange(4, dtype=np.uint32))
    states = mtgp.mtgp_get_statuses(st)
    counts = np.array([5000, 7000, 1, 90000], np.uint64)
    ids = np.arange(4, dtype=np.uint32)
    out = torch.empty(int(counts.sum()), dtype=torch.int32, device="cuda")
    plan = mtgp.mtgp_plan_create(st, ids, counts, mtgp.MTGP_U32, out)

    def refused(fn, *a, **k):
        with pytest.raises(mtgp.MtgpError) as ei:
            fn(*a, **k)
        assert ei.value.status == 1

    refused(mtgp.mtgp_plan_read_stats, plan)
    refused(mtgp.mtgp_plan_set_stats, plan, hamming=(25, 5, 155, []))     # L/s = 31 < 32
    refused(mtgp.mtgp_plan_set_stats, plan, hamming=(25, 5, 1201, []))    # L not a multiple of s
    refused(mtgp.mtgp_plan_set_stats, plan, hamming=(28, 5, 1200, []))    # r + s > 32
    refused(mtgp.mtgp_plan_set_stats, plan, gap=(25, 5, 1024))            # t > 1023
    refused(mtgp.mtgp_plan_set_stats, plan, gap=(25, 0, 128))             # b = 0
    refused(mtgp.mtgp_plan_set_stats, plan, gap=(30, 5, 128))             # r + b > 32
    mtgp.mtgp_plan_set_trace(plan, True)
    refused(mtgp.mtgp_plan_set_stats, plan, **PAPER)
    mtgp.mtgp_plan_set_trace(plan, False)
    mtgp.mtgp_plan_set_stats(plan, **PAPER)
    refused(mtgp.mtgp_plan_set_trace, plan, True)
    # a split plan computes statistics too (stitched); removing the split keeps them
    mtgp.mtgp_plan_set_split(plan, 1000)
    assert mtgp.mtgp_plan_get_info(plan)["stats"]
    mtgp.mtgp_plan_set_split(plan, 0)
    # turning the statistics off returns the plan to the plain kernel
    mtgp.mtgp_plan_set_stats(plan)
    info = mtgp.mtgp_plan_get_info(plan)
    assert not info["stats"] and info["kernel_launches"] == 1
    mtgp.mtgp_plan_launch(plan)
    torch.cuda.synchronize()
    ref, states = oracle.generate_many(op, states, ids, counts, 0, THREADS)
    _same(out.cpu().numpy().view(np.uint32), ref, "outputs after statistics off")
    # a state size without an instantiation of the fused kernel (N = 2696)
    gb = mtgp.mtgp_params_generate(86243, workloads.PARAM_SEED)
    sb = mtgp.mtgp_init_statuses(gb, np.arange(2, dtype=np.uint32))
    pb = mtgp.mtgp_plan_create(sb, [0, 1], [1000, 1000], mtgp.MTGP_U32, out[:2000])
    refused(mtgp.mtgp_plan_set_stats, pb, **PAPER)

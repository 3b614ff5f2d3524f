"""Parity of the wide-column generation kernel (launch config kernel = 2) with
the CPU oracle, through the C ABI.

That kernel gives each lane four consecutive columns of a 128-word step and
stores its outputs as 16-byte chunks realigned across lanes, so beyond the
usual cases these tests vary what its index arithmetic depends on: the
state size (steps per row), pos (where pick-ups wrap into the new row), the
output's element offset modulo 4 (the chunk realignment and its carry
across steps and rows), requests that start or end inside a row, every
format, per-stream parameter sets and plans.  Tolerance 0: outputs are
compared by bit pattern.
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


def _wide_handle(gp, seeds, warps=8):
    st = mtgp.mtgp_init_statuses(gp, np.asarray(seeds, np.uint32))
    mtgp.mtgp_set_launch_config(st, warps_per_cta=warps, words_per_lane=4, kernel=2, ctas_per_sm=1)
    return st


def _gen(st, ids, counts, fmt, shift=0):
    """Generation into a buffer view `shift` elements past a 16-byte
    boundary; the guard elements around it must stay untouched."""
    ids = np.asarray(ids, np.uint32)
    counts = np.asarray(counts, np.uint64)
    total = int(counts.sum())
    buf = torch.full((total + 8,), -1, dtype=torch.int32, device="cuda")
    view = buf[4 + shift:4 + shift + total]
    if fmt == mtgp.MTGP_U32:
        mtgp.mtgp_generate_u32(st, ids, counts, view)
    else:
        mtgp.mtgp_generate_f32(st, ids, counts, fmt, view)
    torch.cuda.synchronize()
    mtgp.mtgp_check(st)
    host = buf.cpu().numpy().view(np.uint32)
    assert np.all(host[:4 + shift] == 0xFFFFFFFF) and np.all(host[4 + shift + total:] == 0xFFFFFFFF)
    return host[4 + shift:4 + shift + total]


def _same(a, b, what):
    a, b = np.asarray(a, np.uint32), np.asarray(b, np.uint32)
    bad = np.nonzero(a != b)[0]
    assert bad.size == 0, "%s: %d mismatches, first at %d" % (what, bad.size, bad[0])


@pytest.mark.parametrize("mexp", [9689, 11213, 19937, 21701, 23209, 44497])
@pytest.mark.parametrize("pseed", [workloads.PARAM_SEED, 1, 2, 3])
def test_wide_exponents_and_parameter_sets(mexp, pseed):
    gp = mtgp.mtgp_params_generate(mexp, pseed)
    op = oracle.params_generate(mexp, pseed)
    if op.n - op.pos < 256:
        pytest.skip("N - pos = %d: the wide kernel needs >= 256" % (op.n - op.pos))
    n = 11
    st = _wide_handle(gp, np.arange(n))
    states = np.stack([oracle.init_state(op, s) for s in range(n)])
    N = op.n
    ids = np.array([0, 1, 2, 3, 4, 5, 6, 7, 8, 9, 10, 3, 3, 0], np.uint32)
    counts = np.array([N * 9 + 13, 1, 127, 128, 129, N, N - 1, N + 1, 50000, 0, 2 * N + 3, 10,
                       N * 4, 77], np.uint64)
    for i, fmt in enumerate(FMTS):
        out = _gen(st, ids, counts, fmt, shift=(i + pseed) % 4)
        ref, states = oracle.generate_many(op, states, ids, counts, fmt, THREADS)
        _same(out, ref, "mexp %d pset %d fmt %d" % (mexp, pseed, fmt))
    _same(mtgp.mtgp_get_statuses(st), states, "states")


@pytest.mark.parametrize("shift", [0, 1, 2, 3])
@pytest.mark.parametrize("warps", [4, 8])
def test_wide_output_offsets(shift, warps):
    """Every element offset of the output modulo 4, for batches of full rows
    of every length mod 4 and requests that split rows."""
    gp = mtgp.mtgp_params_generate(11213, workloads.PARAM_SEED)
    op = oracle.params_generate(11213, workloads.PARAM_SEED)
    st = _wide_handle(gp, np.arange(8), warps)
    states = np.stack([oracle.init_state(op, s) for s in range(8)])
    N = op.n
    ids = np.array([0, 1, 2, 3, 4, 5, 6, 7, 1, 1, 2], np.uint32)
    counts = np.array([N * 4, N * 4 + 1, N * 4 + 2, N * 4 + 3, N * 5 + 2, 3, 2 * N - 5, 4 * N + 4,
                       N + 2, N + 3, 9], np.uint64)
    for fmt in FMTS:
        out = _gen(st, ids, counts, fmt, shift)
        ref, states = oracle.generate_many(op, states, ids, counts, fmt, THREADS)
        _same(out, ref, "shift %d fmt %d" % (shift, fmt))
    _same(mtgp.mtgp_get_statuses(st), states, "states")


@pytest.mark.parametrize("gap", [256, 257, 300, 255])
def test_wide_pos_boundaries(tmp_path, gap):
    """pos = N - gap: gap 256 is the smallest the wide kernel takes (its
    pick-ups then wrap into the new row in the last step only two steps
    after the words are written); gap 255 must fall back to kernel 0."""
    o0 = oracle.params_generate(11213, 7)
    n = o0.n
    path = tmp_path / "p.txt"
    path.write_text("mexp 11213\npos %d\nsh1 %d\nsh2 %d\nrec_basis %s\ntmp_basis %s\n" % (
        n - gap, o0.sh1, o0.sh2, " ".join(hex(v) for v in o0.rec_basis),
        " ".join(hex(v) for v in o0.tmp_basis)))
    gp = mtgp.mtgp_params_load(str(path))
    op = oracle.params_from_fields(11213, n - gap, o0.sh1, o0.sh2, list(o0.rec_basis),
                                   list(o0.tmp_basis))
    st = _wide_handle(gp, np.arange(5))
    states = np.stack([oracle.init_state(op, s) for s in range(5)])
    ids = np.array([0, 1, 2, 3, 4, 2], np.uint32)
    counts = np.array([n * 30 + 1, n * 7, 5, 100000, n + 9, n * 2], np.uint64)
    for fmt in FMTS:
        out = _gen(st, ids, counts, fmt, shift=fmt + 1)
        ref, states = oracle.generate_many(op, states, ids, counts, fmt, THREADS)
        _same(out, ref, "gap %d fmt %d" % (gap, fmt))
    _same(mtgp.mtgp_get_statuses(st), states, "states")
    out = torch.empty(int(counts.sum()), dtype=torch.int32, device="cuda")
    plan = mtgp.mtgp_plan_create(st, ids, counts, mtgp.MTGP_U32, out)
    assert mtgp.mtgp_plan_get_info(plan)["config"]["kernel"] == (2 if gap >= 256 else 0)


@pytest.mark.parametrize("mexp,n", [(23209, 727), (44497, 1392)])
def test_wide_literal_state_sizes(tmp_path, mexp, n):
    o0 = oracle.params_generate(mexp, workloads.PARAM_SEED)
    path = tmp_path / "p.txt"
    path.write_text("mexp %d\nn %d\nmask %d\npos %d\nsh1 %d\nsh2 %d\nrec_basis %s\ntmp_basis %s\n" % (
        mexp, n, o0.mask, o0.pos, o0.sh1, o0.sh2, " ".join(hex(v) for v in o0.rec_basis),
        " ".join(hex(v) for v in o0.tmp_basis)))
    gp = mtgp.mtgp_params_load(str(path))
    op = oracle.params_from_fields(mexp, o0.pos, o0.sh1, o0.sh2, list(o0.rec_basis),
                                   list(o0.tmp_basis), n=n, mask=o0.mask)
    st = _wide_handle(gp, np.arange(4))
    states = np.stack([oracle.init_state(op, s) for s in range(4)])
    ids = np.arange(4, dtype=np.uint32)
    counts = np.array([1 << 16, 3 * n + 5, n, 1], np.uint64)
    for fmt in FMTS:
        out = _gen(st, ids, counts, fmt, shift=3 - fmt)
        ref, states = oracle.generate_many(op, states, ids, counts, fmt, THREADS)
        _same(out, ref, "n %d fmt %d" % (n, fmt))
    _same(mtgp.mtgp_get_statuses(st), states, "states")


def test_wide_per_stream_parameter_sets():
    set_seeds = [workloads.PARAM_SEED + 1 + k for k in range(6)]
    gsets = [mtgp.mtgp_params_generate(11213, k) for k in set_seeds]
    osets = [oracle.params_generate(11213, k) for k in set_seeds]
    n = 24
    set_of = (np.arange(n) * 5 % 6).astype(np.uint32)
    st = mtgp.mtgp_init_statuses_multi(gsets, set_of, np.arange(n, dtype=np.uint32))
    mtgp.mtgp_set_launch_config(st, warps_per_cta=8, words_per_lane=4, kernel=2, ctas_per_sm=1)
    states = np.stack([oracle.init_state(osets[set_of[s]], s) for s in range(n)])
    rng = np.random.default_rng(4)
    ids = np.concatenate([np.arange(n), rng.integers(0, n, 10)]).astype(np.uint32)
    counts = rng.integers(0, 40000, ids.size).astype(np.uint64)
    for fmt in FMTS:
        out = _gen(st, ids, counts, fmt, shift=1)
        offs = np.concatenate([[0], np.cumsum(counts.astype(np.int64))])
        for j, (sid, c) in enumerate(zip(ids, counts)):
            ref, states[sid] = oracle.generate(osets[set_of[sid]], states[sid], int(c), fmt)
            _same(out[offs[j]:offs[j + 1]], ref, "request %d fmt %d" % (j, fmt))
    _same(mtgp.mtgp_get_statuses(st), states, "states")


def test_wide_plan_replays_and_autotune_candidates():
    """A plan recorded with the wide kernel replays into the same buffer and
    continues every stream; the autotuner times wide candidates too."""
    gp = mtgp.mtgp_params_generate(11213, workloads.PARAM_SEED)
    op = oracle.params_generate(11213, workloads.PARAM_SEED)
    w = workloads.uneven(600)
    st = _wide_handle(gp, w["seeds"])
    states = mtgp.mtgp_get_statuses(st)
    counts = w["counts"] // 8 + 1
    ids = np.arange(counts.size, dtype=np.uint32)
    out = torch.empty(int(counts.sum()), dtype=torch.int32, device="cuda")
    plan = mtgp.mtgp_plan_create(st, ids, counts, mtgp.MTGP_U32, out)
    assert mtgp.mtgp_plan_get_info(plan)["config"]["kernel"] == 2
    for rep in range(2):
        mtgp.mtgp_plan_launch(plan)
        torch.cuda.synchronize()
        mtgp.mtgp_check(st)
        ref, states = oracle.generate_many(op, states, ids, counts, 0, THREADS)
        _same(out.cpu().numpy().view(np.uint32), ref, "replay %d" % rep)
    _same(mtgp.mtgp_get_statuses(st), states, "states")
    best = mtgp.mtgp_plan_autotune(plan)
    assert best["kernel"] in (0, 2)
    mtgp.mtgp_plan_launch(plan)
    torch.cuda.synchronize()
    ref, states = oracle.generate_many(op, states, ids, counts, 0, THREADS)
    _same(out.cpu().numpy().view(np.uint32), ref, "after autotune")
    _same(mtgp.mtgp_get_statuses(st), states, "states after autotune")


def test_wide_full_uneven_plan_every_output():
    """The benchmark workload (10 000 Mexp 11213 streams, log-uniform counts,
    5.1e9 numbers) on the wide kernel: every output and every final state."""
    w = workloads.uneven()
    gp = mtgp.mtgp_params_generate(w["mexp"], workloads.PARAM_SEED)
    op = oracle.params_generate(w["mexp"], workloads.PARAM_SEED)
    st = _wide_handle(gp, w["seeds"])
    states = mtgp.mtgp_get_statuses(st)
    counts = w["counts"]
    out = torch.empty(int(counts.sum()), dtype=torch.int32, device="cuda")
    plan = mtgp.mtgp_plan_create(st, w["seeds"], counts, mtgp.MTGP_U32, out)
    assert mtgp.mtgp_plan_get_info(plan)["config"]["kernel"] == 2
    mtgp.mtgp_plan_launch(plan)
    torch.cuda.synchronize()
    mtgp.mtgp_check(st)
    offs = np.concatenate([[0], np.cumsum(counts.astype(np.int64))])
    for b0 in range(0, counts.size, 512):
        ids = np.arange(b0, min(counts.size, b0 + 512), dtype=np.uint32)
        ref, st2 = oracle.generate_many(op, states[b0:b0 + ids.size], ids - b0, counts[ids], 0,
                                        THREADS)
        states[b0:b0 + ids.size] = st2
        got = out[int(offs[b0]):int(offs[b0 + ids.size])].cpu().numpy().view(np.uint32)
        _same(got, ref, "streams %d..%d" % (b0, b0 + ids.size - 1))
    _same(mtgp.mtgp_get_statuses(st), states, "states")

"""Parity of the CUDA path (through the C ABI) with the CPU oracle.

Integer and float outputs are compared by bit pattern: the method is exact,
so the tolerance is zero everywhere (floats are made by mantissa bit-fill and
an exact subtraction).  Small cases compare every output and every state
word; the full-size workloads compare every output and every final state too, in
the launch configuration the benchmark uses.
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


def _both_params(mexp, seed=workloads.PARAM_SEED):
    return mtgp.mtgp_params_generate(mexp, seed), oracle.params_generate(mexp, seed)


def _params_file(tmp_path, f, n=0, mask=0):
    path = tmp_path / ("p%d.txt" % np.random.randint(1 << 30))
    lines = ["mexp %d" % f["mexp"], "pos %d" % f["pos"], "sh1 %d" % f["sh1"], "sh2 %d" % f["sh2"],
             "rec_basis " + " ".join(hex(v) for v in f["rec_basis"]),
             "tmp_basis " + " ".join(hex(v) for v in f["tmp_basis"])]
    if n:
        lines.append("n %d" % n)
    if mask:
        lines.append("mask %d" % mask)
    path.write_text("\n".join(lines) + "\n")
    return str(path)


def _gpu_generate(streams, ids, counts, fmt=mtgp.MTGP_U32):
    ids = np.asarray(ids, np.uint32)
    counts = np.asarray(counts, np.uint64)
    total = int(counts.sum())
    out = torch.full((max(total, 1),), -1, dtype=torch.int32, device="cuda")
    if fmt == mtgp.MTGP_U32:
        mtgp.mtgp_generate_u32(streams, ids, counts, out)
    else:
        mtgp.mtgp_generate_f32(streams, ids, counts, fmt, out)
    torch.cuda.synchronize()
    mtgp.mtgp_check(streams)
    return out[:total].cpu().numpy().view(np.uint32)


def _assert_same(a, b, what=""):
    a = np.asarray(a, np.uint32)
    b = np.asarray(b, np.uint32)
    assert a.shape == b.shape, what
    bad = np.nonzero(a != b)[0]
    assert bad.size == 0, "%s: %d mismatches, first at %d: %08x vs %08x" % (
        what, bad.size, bad[0], a[bad[0]], b[bad[0]])


CONFIGS = [
    dict(warps_per_cta=4, words_per_lane=8, kernel=0),
    dict(warps_per_cta=1, words_per_lane=4, kernel=0),
    dict(warps_per_cta=8, words_per_lane=8, kernel=0),
    dict(warps_per_cta=4, words_per_lane=8, kernel=1),
    dict(warps_per_cta=8, words_per_lane=8, kernel=0, ctas_per_sm=1),
    dict(warps_per_cta=8, words_per_lane=4, kernel=0, ctas_per_sm=1),
    dict(warps_per_cta=2, words_per_lane=4, kernel=0, ctas_per_sm=4),
    dict(warps_per_cta=4, words_per_lane=8, kernel=0, coop_percent=1),
]


# ---------------------------------------------------------------------------
# status initialisation and the single-stream workload (Mexp 11213, seed 1)
# ---------------------------------------------------------------------------
def test_init_statuses_match_oracle():
    gp, op = _both_params(11213)
    seeds = np.concatenate([np.arange(4096), [0xFFFFFFFF, 0xDEADBEEF, 12345678]]).astype(np.uint32)
    st = mtgp.mtgp_init_statuses(gp, seeds)
    got = mtgp.mtgp_get_statuses(st)
    for i in list(range(0, 4096, 37)) + [4096, 4097, 4098]:
        _assert_same(got[i], oracle.init_state(op, int(seeds[i])), "stream %d" % i)


def test_single_stream_2p20_bit_exact():
    gp, op = _both_params(11213)
    st = mtgp.mtgp_init_statuses(gp, np.array([1], np.uint32))
    out = _gpu_generate(st, [0], [1 << 20])
    ref, ref_st = oracle.generate(op, oracle.init_state(op, 1), 1 << 20)
    _assert_same(out, ref, "outputs")
    _assert_same(mtgp.mtgp_get_statuses(st)[0], ref_st, "state")


# ---------------------------------------------------------------------------
# ragged counts, duplicate streams, every kernel configuration
# ---------------------------------------------------------------------------
@pytest.mark.parametrize("cfg", CONFIGS, ids=lambda c: "w%d_k%d_kern%d_cap%d_coop%d" % (
    c["warps_per_cta"], c["words_per_lane"], c["kernel"], c.get("ctas_per_sm", 0),
    c.get("coop_percent", 100)))
@pytest.mark.parametrize("fmt", FMTS)
def test_ragged_requests(cfg, fmt):
    gp, op = _both_params(11213)
    rng = np.random.default_rng(21)
    n_streams = 37
    states = workloads.random_states(rng, n_streams, op.n)
    st = mtgp.mtgp_init_statuses(gp, np.zeros(n_streams, np.uint32))
    mtgp.mtgp_set_statuses(st, states)
    mtgp.mtgp_set_launch_config(st, **cfg)
    edge = [0, 1, 2, 31, 32, 33, 255, 256, 257, 350, 351, 352, 701, 702, 703, 1000, 4096, 9999]
    ids = np.concatenate([np.arange(n_streams) % 29, rng.integers(0, n_streams, 23)]).astype(np.uint32)
    counts = np.array([edge[i % len(edge)] for i in range(ids.size)], np.uint64)
    out = _gpu_generate(st, ids, counts, fmt)
    ref, ref_st = oracle.generate_many(op, states, ids, counts, fmt, THREADS)
    _assert_same(out, ref, "outputs")
    _assert_same(mtgp.mtgp_get_statuses(st), ref_st, "states")


def test_successive_calls_continue_streams():
    gp, op = _both_params(11213)
    st = mtgp.mtgp_init_statuses(gp, np.arange(8, dtype=np.uint32))
    ref_states = np.stack([oracle.init_state(op, s) for s in range(8)])
    rng = np.random.default_rng(3)
    for call in range(6):
        ids = rng.integers(0, 8, 12).astype(np.uint32)
        counts = rng.integers(0, 3000, 12).astype(np.uint64)
        fmt = FMTS[call % 3]
        out = _gpu_generate(st, ids, counts, fmt)
        ref, ref_states = oracle.generate_many(op, ref_states, ids, counts, fmt, THREADS)
        _assert_same(out, ref, "call %d" % call)
    _assert_same(mtgp.mtgp_get_statuses(st), ref_states)


# ---------------------------------------------------------------------------
# other parameter sets: toys (shared-memory ring path), other exponents,
# the literal N = 727 / 1392 rows
# ---------------------------------------------------------------------------
@pytest.mark.parametrize("n", [2, 3, 5, 17, 40, 64, 100])
def test_toy_parameter_sets(tmp_path, n):
    rng = np.random.default_rng(1000 + n)
    for trial in range(3):
        f = workloads.toy_fields(rng, n)
        gp = mtgp.mtgp_params_load(_params_file(tmp_path, f))
        op = oracle.params_from_fields(f["mexp"], f["pos"], f["sh1"], f["sh2"], f["rec_basis"],
                                       f["tmp_basis"])
        states = workloads.random_states(rng, 5, n)
        st = mtgp.mtgp_init_statuses(gp, np.zeros(5, np.uint32))
        mtgp.mtgp_set_statuses(st, states)
        ids = np.array([0, 1, 2, 3, 4, 0, 2], np.uint32)
        counts = np.array([1, 7, 100, 3 * n + 1, 2000, 33, 0], np.uint64)
        for fmt in FMTS:
            out = _gpu_generate(st, ids, counts, fmt)
            ref, states = oracle.generate_many(op, states, ids, counts, fmt, THREADS)
            _assert_same(out, ref, "n=%d trial %d fmt %d" % (n, trial, fmt))
        _assert_same(mtgp.mtgp_get_statuses(st), states)


@pytest.mark.parametrize("mexp", [3217, 4253, 9689, 9941, 19937, 21701, 23209, 44497])
def test_other_exponents(mexp):
    gp, op = _both_params(mexp)
    st = mtgp.mtgp_init_statuses(gp, np.arange(16, dtype=np.uint32))
    states = np.stack([oracle.init_state(op, s) for s in range(16)])
    ids = np.arange(16, dtype=np.uint32)
    counts = np.array([(i * 7919) % 20000 for i in range(16)], np.uint64)
    for fmt in FMTS:
        out = _gpu_generate(st, ids, counts, fmt)
        ref, states = oracle.generate_many(op, states, ids, counts, fmt, THREADS)
        _assert_same(out, ref, "mexp %d fmt %d" % (mexp, fmt))
    _assert_same(mtgp.mtgp_get_statuses(st), states)


@pytest.mark.parametrize("kernel", [0, 1])
@pytest.mark.parametrize("k", [4, 8])
@pytest.mark.parametrize("mexp", [23209, 44497])
def test_eight_warp_ctas_of_large_states(mexp, k, kernel):
    """8-warp CTAs of the largest state sizes need about 48 KB of shared
    memory or more, static and dynamic together: the launch must take the
    configuration as given (no fallback) and equal the oracle."""
    gp, op = _both_params(mexp)
    n = 24
    st = mtgp.mtgp_init_statuses(gp, np.arange(n, dtype=np.uint32))
    mtgp.mtgp_set_launch_config(st, warps_per_cta=8, words_per_lane=k, kernel=kernel, ctas_per_sm=0)
    states = mtgp.mtgp_get_statuses(st)
    ids = np.arange(n, dtype=np.uint32)
    counts = np.array([(i * 104729) % 300000 + 1 for i in range(n)], np.uint64)
    out = torch.empty(int(counts.sum()), dtype=torch.int32, device="cuda")
    plan = mtgp.mtgp_plan_create(st, ids, counts, mtgp.MTGP_U32, out)
    info = mtgp.mtgp_plan_get_info(plan)
    assert info["config"]["warps_per_cta"] == 8 and info["config"]["kernel"] == kernel
    mtgp.mtgp_plan_launch(plan)
    torch.cuda.synchronize()
    mtgp.mtgp_check(st)
    ref, states = oracle.generate_many(op, states, ids, counts, 0, THREADS)
    _assert_same(out.cpu().numpy().view(np.uint32), ref, "mexp %d k %d kernel %d" % (mexp, k, kernel))
    _assert_same(mtgp.mtgp_get_statuses(st), states)


@pytest.mark.parametrize("kernel", [0, 1])
@pytest.mark.parametrize("mexp", [9689, 11213, 19937, 21701, 23209, 44497])
@pytest.mark.parametrize("pseed", [1, 2, 3])
def test_parameter_sweep(kernel, mexp, pseed):
    """Both kernels over several exponents (state sizes) and parameter seeds
    (other pos, shifts and tables)."""
    gp, op = _both_params(mexp, pseed)
    st = mtgp.mtgp_init_statuses(gp, np.arange(12, dtype=np.uint32))
    mtgp.mtgp_set_launch_config(st, warps_per_cta=4, words_per_lane=8, kernel=kernel)
    states = np.stack([oracle.init_state(op, s) for s in range(12)])
    ids = np.array([0, 1, 2, 3, 4, 5, 6, 7, 8, 9, 10, 11, 3, 3], np.uint32)
    counts = np.array([op.n * 7 + 13, 1, 63, 64, 65, op.n, op.n - 1, op.n + 1, 5000, 0, 2 * op.n,
                       33333, 10, op.n * 3], np.uint64)
    for fmt in FMTS:
        out = _gpu_generate(st, ids, counts, fmt)
        ref, states = oracle.generate_many(op, states, ids, counts, fmt, THREADS)
        _assert_same(out, ref, "kernel %d mexp %d seed %d fmt %d" % (kernel, mexp, pseed, fmt))
    _assert_same(mtgp.mtgp_get_statuses(st), states)


@pytest.mark.parametrize("mexp", [3217, 4253, 4423])
@pytest.mark.parametrize("pseed", [workloads.PARAM_SEED, 1, 2])
@pytest.mark.parametrize("warps,k,coop", [(4, 2, 0), (2, 2, 0), (8, 2, 0), (2, 2, 1), (4, 4, 0),
                                          (2, 4, 1)])
def test_short_states_register_kernel(mexp, pseed, warps, k, coop):
    """Mexp 3217 (N = 101, the paper's exponent) and 4253 / 4423 (N = 133 /
    139) on the register-resident kernel: 64-word steps (K = 2) for every
    set, 128-word steps where N - pos >= 128, warp-owned and CTA-owned
    streams.  The plan reports the kernel and step width it resolved to."""
    gp, op = _both_params(mexp, pseed)
    if 32 * k > op.n - op.pos:
        pytest.skip("N - pos = %d admits no %d-word step" % (op.n - op.pos, 32 * k))
    n = 10
    st = mtgp.mtgp_init_statuses(gp, np.arange(n, dtype=np.uint32))
    mtgp.mtgp_set_launch_config(st, warps_per_cta=warps, words_per_lane=k, kernel=0,
                                coop_percent=coop)
    states = np.stack([oracle.init_state(op, s) for s in range(n)])
    ids = np.array([0, 1, 2, 3, 4, 5, 6, 7, 8, 9, 2, 2], np.uint32)
    counts = np.array([op.n * 40 + 7, 1, 63, 64, 65, op.n, op.n - 1, 30000, 0, 2 * op.n + 1, 10,
                       op.n * 3], np.uint64)
    for fmt in FMTS:
        out = _gpu_generate(st, ids, counts, fmt)
        ref, states = oracle.generate_many(op, states, ids, counts, fmt, THREADS)
        _assert_same(out, ref, "mexp %d seed %d fmt %d" % (mexp, pseed, fmt))
    _assert_same(mtgp.mtgp_get_statuses(st), states)
    out = torch.empty(int(counts.sum()), dtype=torch.int32, device="cuda")
    plan = mtgp.mtgp_plan_create(st, ids, counts, mtgp.MTGP_U32, out)
    info = mtgp.mtgp_plan_get_info(plan)
    assert info["config"]["kernel"] == 0 and info["config"]["words_per_lane"] == k
    mtgp.mtgp_plan_launch(plan)
    torch.cuda.synchronize()
    ref, states = oracle.generate_many(op, states, ids, counts, 0, THREADS)
    _assert_same(out.cpu().numpy().view(np.uint32), ref, "plan")
    _assert_same(mtgp.mtgp_get_statuses(st), states)


def test_short_state_default_config_uses_register_kernel():
    gp, op = _both_params(3217)
    st = mtgp.mtgp_init_statuses(gp, np.arange(4, dtype=np.uint32))
    out = torch.empty(4000, dtype=torch.int32, device="cuda")
    plan = mtgp.mtgp_plan_create(st, np.arange(4), np.full(4, 1000), mtgp.MTGP_U32, out)
    info = mtgp.mtgp_plan_get_info(plan)
    assert info["config"]["kernel"] == 0 and info["config"]["words_per_lane"] == 2


@pytest.mark.parametrize("kernel", [0, 1])
@pytest.mark.parametrize("mexp,n", [(23209, 727), (44497, 1392)])
def test_literal_state_sizes(tmp_path, mexp, n, kernel):
    o0 = oracle.params_generate(mexp, workloads.PARAM_SEED)
    f = {"mexp": mexp, "pos": o0.pos, "sh1": o0.sh1, "sh2": o0.sh2,
         "rec_basis": list(o0.rec_basis), "tmp_basis": list(o0.tmp_basis)}
    gp = mtgp.mtgp_params_load(_params_file(tmp_path, f, n=n, mask=o0.mask))
    op = oracle.params_from_fields(mexp, o0.pos, o0.sh1, o0.sh2, f["rec_basis"], f["tmp_basis"],
                                   n=n, mask=o0.mask)
    assert op.n == n
    st = mtgp.mtgp_init_statuses(gp, np.arange(4, dtype=np.uint32))
    mtgp.mtgp_set_launch_config(st, warps_per_cta=4, words_per_lane=8, kernel=kernel)
    states = np.stack([oracle.init_state(op, s) for s in range(4)])
    _assert_same(mtgp.mtgp_get_statuses(st), states, "init")
    ids = np.arange(4, dtype=np.uint32)
    counts = np.array([1 << 16, 3 * n + 5, n, 1], np.uint64)
    for fmt in FMTS:
        out = _gpu_generate(st, ids, counts, fmt)
        ref, states = oracle.generate_many(op, states, ids, counts, fmt, THREADS)
        _assert_same(out, ref)
    _assert_same(mtgp.mtgp_get_statuses(st), states)


@pytest.mark.parametrize("mexp", [11213, 23209])
@pytest.mark.parametrize("gap", [256, 255, 129])
@pytest.mark.parametrize("warps", [2, 8])
def test_step_width_boundaries(tmp_path, mexp, gap, warps):
    """pos = N - gap with 128-word steps: gap >= 256 takes the software-
    pipelined row loop (next step's loads before this step's stores), a
    smaller gap the row-by-row loop.  Multi-request items and every format."""
    o0 = oracle.params_generate(mexp, 7)
    n = mexp // 32 + 1
    f = {"mexp": mexp, "pos": n - gap, "sh1": o0.sh1, "sh2": o0.sh2,
         "rec_basis": list(o0.rec_basis), "tmp_basis": list(o0.tmp_basis)}
    gp = mtgp.mtgp_params_load(_params_file(tmp_path, f))
    op = oracle.params_from_fields(mexp, n - gap, o0.sh1, o0.sh2, f["rec_basis"], f["tmp_basis"])
    st = mtgp.mtgp_init_statuses(gp, np.arange(9, dtype=np.uint32))
    mtgp.mtgp_set_launch_config(st, warps_per_cta=warps, words_per_lane=4, kernel=0, coop_percent=0)
    states = np.stack([oracle.init_state(op, s) for s in range(9)])
    ids = np.array([0, 1, 2, 3, 4, 5, 6, 7, 8, 0, 0, 5], np.uint32)
    counts = np.array([n * 40, n * 40 + 7, 1, n, n - 1, 2 * n + 1, 100000, 3, 0, n * 3, 17, n * 5],
                      np.uint64)
    for fmt in FMTS:
        out = _gpu_generate(st, ids, counts, fmt)
        ref, states = oracle.generate_many(op, states, ids, counts, fmt, THREADS)
        _assert_same(out, ref, "gap %d warps %d fmt %d" % (gap, warps, fmt))
    _assert_same(mtgp.mtgp_get_statuses(st), states)


@pytest.mark.parametrize("kernel", [0, 1])
def test_output_pointer_only_4_byte_aligned(kernel):
    """A caller may pass an output that is 4- but not 8-byte aligned (a view
    one element into a buffer)."""
    gp, op = _both_params(11213)
    st = mtgp.mtgp_init_statuses(gp, np.arange(6, dtype=np.uint32))
    mtgp.mtgp_set_launch_config(st, warps_per_cta=4, words_per_lane=8, kernel=kernel)
    states = np.stack([oracle.init_state(op, s) for s in range(6)])
    ids = np.arange(6, dtype=np.uint32)
    counts = np.array([op.n * 9, op.n * 9 + 1, 4000, 1, 777, op.n], np.uint64)
    total = int(counts.sum())
    for fmt in FMTS:
        buf = torch.full((total + 2,), -1, dtype=torch.int32, device="cuda")
        view = buf[1:1 + total]
        assert view.data_ptr() % 8 == 4
        if fmt == mtgp.MTGP_U32:
            mtgp.mtgp_generate_u32(st, ids, counts, view)
        else:
            mtgp.mtgp_generate_f32(st, ids, counts, fmt, view)
        torch.cuda.synchronize()
        mtgp.mtgp_check(st)
        got = buf.cpu().numpy().view(np.uint32)
        ref, states = oracle.generate_many(op, states, ids, counts, fmt, THREADS)
        _assert_same(got[1:1 + total], ref, "kernel %d fmt %d" % (kernel, fmt))
        assert got[0] == 0xFFFFFFFF and got[total + 1] == 0xFFFFFFFF
    _assert_same(mtgp.mtgp_get_statuses(st), states)


# ---------------------------------------------------------------------------
# checkpoint / restore, errors, empty calls, autotune
# ---------------------------------------------------------------------------
def test_checkpoint_restore():
    gp, op = _both_params(11213)
    st = mtgp.mtgp_init_statuses(gp, np.arange(10, dtype=np.uint32))
    _gpu_generate(st, np.arange(10), np.full(10, 777))
    saved = mtgp.mtgp_get_statuses(st)
    a = _gpu_generate(st, np.arange(10), np.full(10, 5000))
    mtgp.mtgp_set_statuses(st, saved)
    b = _gpu_generate(st, np.arange(10), np.full(10, 5000))
    _assert_same(a, b)
    ref, _ = oracle.generate_many(op, saved, np.arange(10), np.full(10, 5000), 0, THREADS)
    _assert_same(a, ref)


def test_invalid_requests_write_nothing():
    gp, _ = _both_params(11213)
    st = mtgp.mtgp_init_statuses(gp, np.arange(4, dtype=np.uint32))
    before = mtgp.mtgp_get_statuses(st)
    out = torch.full((100,), 7, dtype=torch.int32, device="cuda")
    with pytest.raises(mtgp.MtgpError) as ei:
        mtgp.mtgp_generate_u32(st, [0, 4], [10, 10], out)
    assert ei.value.status == 1
    with pytest.raises(mtgp.MtgpError):
        mtgp.mtgp_generate_f32(st, [0], [10], 7, out)
    with pytest.raises(mtgp.MtgpError):
        mtgp.mtgp_generate_u32(st, [0], [10], 0)
    torch.cuda.synchronize()
    assert bool((out == 7).all())
    _assert_same(mtgp.mtgp_get_statuses(st), before)
    # empty and all-zero calls are no-ops
    mtgp.mtgp_generate_u32(st, [], [], out)
    mtgp.mtgp_generate_u32(st, [1, 2], [0, 0], out)
    torch.cuda.synchronize()
    _assert_same(mtgp.mtgp_get_statuses(st), before)
    mtgp.mtgp_check(st)


def test_autotune_keeps_states():
    gp, op = _both_params(11213)
    st = mtgp.mtgp_init_statuses(gp, np.arange(300, dtype=np.uint32))
    before = mtgp.mtgp_get_statuses(st)
    cfg = mtgp.mtgp_autotune(st, mtgp.MTGP_U32, 256, 4096)
    assert cfg["words_per_lane"] in (4, 8) and 1 <= cfg["warps_per_cta"] <= 8
    _assert_same(mtgp.mtgp_get_statuses(st), before)
    out = _gpu_generate(st, np.arange(300), np.full(300, 1000))
    ref, _ = oracle.generate_many(op, before, np.arange(300), np.full(300, 1000), 0, THREADS)
    _assert_same(out, ref)


def test_generate_to_host_chunks():
    gp, op = _both_params(11213)
    st = mtgp.mtgp_init_statuses(gp, np.arange(6, dtype=np.uint32))
    states = mtgp.mtgp_get_statuses(st)
    ids = np.array([0, 1, 2, 3, 4, 5, 0], np.uint32)
    counts = np.array([100000, 3, 70000, 0, 1, 40000, 9000], np.uint64)
    for fmt in FMTS:
        host = torch.empty(int(counts.sum()), dtype=torch.int32).pin_memory()
        mtgp.mtgp_generate_to_host(st, ids, counts, fmt, host, chunk_bytes=64 * 1024)
        ref, states = oracle.generate_many(op, states, ids, counts, fmt, THREADS)
        _assert_same(host.numpy().view(np.uint32), ref, "fmt %d" % fmt)
    _assert_same(mtgp.mtgp_get_statuses(st), states)


def test_plan_replays_continue_streams():
    gp, op = _both_params(11213)
    n = 500
    counts = workloads.uneven_counts(n, lo=4, hi=14, seed=5)
    st = mtgp.mtgp_init_statuses(gp, np.arange(n, dtype=np.uint32))
    states = mtgp.mtgp_get_statuses(st)
    out = torch.empty(int(counts.sum()), dtype=torch.int32, device="cuda")
    plan = mtgp.mtgp_plan_create(st, np.arange(n), counts, mtgp.MTGP_F32_01, out)
    info = mtgp.mtgp_plan_get_info(plan)
    assert info["total_numbers"] == int(counts.sum()) and info["kernel_launches"] == 1
    for rep in range(3):
        mtgp.mtgp_plan_launch(plan)
        torch.cuda.synchronize()
        ref, states = oracle.generate_many(op, states, np.arange(n), counts, mtgp.MTGP_F32_01,
                                           THREADS)
        _assert_same(out.cpu().numpy().view(np.uint32), ref, "replay %d" % rep)
    best = mtgp.mtgp_plan_autotune(plan)
    assert best["words_per_lane"] in (4, 8)
    _assert_same(mtgp.mtgp_get_statuses(st), states, "autotune must not advance states")
    mtgp.mtgp_plan_launch(plan)
    torch.cuda.synchronize()
    ref, states = oracle.generate_many(op, states, np.arange(n), counts, mtgp.MTGP_F32_01, THREADS)
    _assert_same(out.cpu().numpy().view(np.uint32), ref, "after autotune")
    mtgp.mtgp_check(st)


# ---------------------------------------------------------------------------
# full-size workloads
# ---------------------------------------------------------------------------
def _check_full(st, op, out_t, counts, fmt, states0, batch=512):
    """Every output and every final state of a launch over streams 0..n-1 in
    order (request j = stream j, outputs back to back): the oracle advances
    the streams in batches, and each batch's outputs are compared element by
    element with the matching slice of the device buffer, copied to the host
    one batch at a time."""
    states = states0.copy()
    n = states.shape[0]
    offs = np.concatenate([[0], np.cumsum(counts.astype(np.int64))])
    for b0 in range(0, n, batch):
        ids = np.arange(b0, min(n, b0 + batch), dtype=np.uint32)
        ref, st2 = oracle.generate_many(op, states[b0:b0 + ids.size], ids - b0, counts[ids], fmt,
                                        THREADS)
        states[b0:b0 + ids.size] = st2
        got = out_t[int(offs[b0]):int(offs[b0 + ids.size])].cpu().numpy().view(np.uint32)
        if not np.array_equal(got, ref):
            bad = int(np.nonzero(got != ref)[0][0])
            sid = int(np.searchsorted(offs, offs[b0] + bad, side="right") - 1)
            raise AssertionError("stream %d: first mismatch at its output %d" % (
                sid, offs[b0] + bad - offs[sid]))
    _assert_same(mtgp.mtgp_get_statuses(st), states, "all final states")
    return states


def test_full_equal_4096x2p18():
    w = workloads.equal()
    gp, op = _both_params(w["mexp"])
    st = mtgp.mtgp_init_statuses(gp, w["seeds"])
    states0 = mtgp.mtgp_get_statuses(st)
    counts = w["counts"]
    out = torch.empty(int(counts.sum()), dtype=torch.int32, device="cuda")
    mtgp.mtgp_generate_u32(st, w["seeds"], counts, out)
    torch.cuda.synchronize()
    mtgp.mtgp_check(st)
    _check_full(st, op, out, counts, 0, states0)


@pytest.mark.parametrize("mexp", [23209, 44497])
def test_full_long_streams_three_formats(mexp):
    w = workloads.long_streams(mexp)
    gp, op = _both_params(mexp)
    st = mtgp.mtgp_init_statuses(gp, w["seeds"])
    states = mtgp.mtgp_get_statuses(st)
    counts = w["counts"]
    out = torch.empty(int(counts.sum()), dtype=torch.int32, device="cuda")
    for fmt in FMTS:
        if fmt == 0:
            mtgp.mtgp_generate_u32(st, w["seeds"], counts, out)
        else:
            mtgp.mtgp_generate_f32(st, w["seeds"], counts, fmt, out)
        torch.cuda.synchronize()
        mtgp.mtgp_check(st)
        states = _check_full(st, op, out, counts, fmt, states)


def test_full_uneven_plan():
    """The benchmark's workload and launch: one plan (CUDA graph, persistent
    work-stealing kernel) over 10 000 streams with log-uniform counts."""
    w = workloads.uneven()
    gp, op = _both_params(w["mexp"])
    st = mtgp.mtgp_init_statuses(gp, w["seeds"])
    states = mtgp.mtgp_get_statuses(st)
    counts = w["counts"]
    out = torch.empty(int(counts.sum()), dtype=torch.int32, device="cuda")
    plan = mtgp.mtgp_plan_create(st, w["seeds"], counts, mtgp.MTGP_U32, out)
    mtgp.mtgp_plan_autotune(plan)   # the launch shape the benchmark times
    for rep in range(2):
        mtgp.mtgp_plan_launch(plan)
        torch.cuda.synchronize()
        mtgp.mtgp_check(st)
        states = _check_full(st, op, out, counts, 0, states)


def test_single_request_beyond_2p32():
    """Maximum size: one request of 2^32 + 1000 numbers from one stream
    (17 GB of output, row and output indices past 32 bits).  Checked by the
    oracle on the first 2^20 outputs; the final state must equal an
    independent jump of the same length (jumps are oracle-checked up to
    10^7 and compose exactly), and the last 1000 outputs must equal the
    oracle started from the state jumped to 2^32."""
    gp, op = _both_params(11213)
    big = (1 << 32) + 1000
    st = mtgp.mtgp_init_statuses(gp, np.array([5, 6], np.uint32))
    s0 = mtgp.mtgp_get_statuses(st)[0]
    out = torch.empty(big, dtype=torch.int32, device="cuda")
    mtgp.mtgp_generate_u32(st, [0], [big], out)
    torch.cuda.synchronize()
    mtgp.mtgp_check(st)
    ref, _ = oracle.generate(op, s0, 1 << 20)
    _assert_same(out[:1 << 20].cpu().numpy().view(np.uint32), ref, "first 2^20")
    ref_st = mtgp.mtgp_init_statuses(gp, np.array([5], np.uint32))
    mtgp.mtgp_jump(ref_st, [0], [1 << 32])
    s32 = mtgp.mtgp_get_statuses(ref_st)[0]
    tail, s_end = oracle.generate(op, s32, 1000)
    _assert_same(out[1 << 32:].cpu().numpy().view(np.uint32), tail, "last 1000")
    _assert_same(mtgp.mtgp_get_statuses(st)[0], s_end, "final state")
    del out


@pytest.mark.parametrize("mexp,kernel", [(11213, 0), (11213, 1), (3217, 0)])
def test_zero_state_is_a_fixed_point(mexp, kernel):
    """The degenerate case of a linear generator: the all-zero state stays
    zero and every output is 0 (u32), 1.0f ([1,2)) or 0.0f ([0,1))."""
    gp, op = _both_params(mexp)
    st = mtgp.mtgp_init_statuses(gp, np.arange(3, dtype=np.uint32))
    mtgp.mtgp_set_launch_config(st, warps_per_cta=4, words_per_lane=2 if mexp == 3217 else 4,
                                kernel=kernel)
    mtgp.mtgp_set_statuses(st, np.zeros((3, op.n), np.uint32))
    expect = {mtgp.MTGP_U32: 0, mtgp.MTGP_F32_12: 0x3F800000, mtgp.MTGP_F32_01: 0}
    for fmt in FMTS:
        out = _gpu_generate(st, [0, 1, 2], [5000, 1, op.n * 3 + 7], fmt)
        assert np.all(out == expect[fmt]), fmt
    assert not mtgp.mtgp_get_statuses(st).any()


@pytest.mark.parametrize("mexp", [3217, 11213, 23209])
def test_forty_parameter_seeds(mexp):
    """Forty seed-generated sets per exponent (pos, shifts and tables all
    drawn anew), default launch shape, ragged requests, against the oracle."""
    for pseed in range(100, 140):
        gp, op = _both_params(mexp, pseed)
        st = mtgp.mtgp_init_statuses(gp, np.array([pseed, 7, 8], np.uint32))
        states = np.stack([oracle.init_state(op, s) for s in (pseed, 7, 8)])
        ids = np.array([0, 1, 2, 0], np.uint32)
        counts = np.array([op.n * 5 + 3, 4097, 1, 333], np.uint64)
        out = _gpu_generate(st, ids, counts)
        ref, states = oracle.generate_many(op, states, ids, counts, 0, THREADS)
        _assert_same(out, ref, "mexp %d seed %d" % (mexp, pseed))
        _assert_same(mtgp.mtgp_get_statuses(st), states)

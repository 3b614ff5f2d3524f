"""One parameterized status per stream (the paper's setting: every MTGP of a
simulation has its own parameter set, Sec. 3.1 / Sec. 4.1, and its own seed
status, Sec. 5.1) through mtgp_init_statuses_multi, against the oracle.

Each stream's expected output is the oracle run with that stream's own
parameter set; request sequences are replayed per stream in order.  All
comparisons are by bit pattern (tolerance 0).
"""

import numpy as np
import pytest

import oracle
from paper_1501_07701_gb300 import mtgp, workloads

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")
FMTS = [mtgp.MTGP_U32, mtgp.MTGP_F32_12, mtgp.MTGP_F32_01]


@pytest.fixture(scope="module", autouse=True)
def _built():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1501_07701_gb300 import build
    build.build()
    mtgp.load_library()


def _params_file(tmp_path, op, pos):
    path = tmp_path / ("p%d_%d.txt" % (op.mexp, pos))
    path.write_text("\n".join([
        "mexp %d" % op.mexp, "pos %d" % pos, "sh1 %d" % op.sh1, "sh2 %d" % op.sh2,
        "rec_basis " + " ".join(hex(v) for v in op.rec_basis),
        "tmp_basis " + " ".join(hex(v) for v in op.tmp_basis)]) + "\n")
    return str(path)


def _sets(mexp, seeds):
    return ([mtgp.mtgp_params_generate(mexp, s) for s in seeds],
            [oracle.params_generate(mexp, s) for s in seeds])


def _generate(st, ids, counts, fmt):
    ids = np.asarray(ids, np.uint32)
    counts = np.asarray(counts, np.uint64)
    total = int(counts.sum())
    out = torch.full((max(total, 1),), -1, dtype=torch.int32, device="cuda")
    if fmt == mtgp.MTGP_U32:
        mtgp.mtgp_generate_u32(st, ids, counts, out)
    else:
        mtgp.mtgp_generate_f32(st, ids, counts, fmt, out)
    torch.cuda.synchronize()
    mtgp.mtgp_check(st)
    return out[:total].cpu().numpy().view(np.uint32)


def _replay(ops, set_of, states, ids, counts, fmt):
    """Oracle: each request from its stream's own parameter set, in order."""
    states = states.copy()
    outs = []
    for sid, c in zip(ids, counts):
        o, states[sid] = oracle.generate(ops[set_of[sid]], states[sid], int(c), fmt)
        outs.append(o)
    return (np.concatenate(outs) if outs else np.zeros(0, np.uint32)), states


def _same(a, b, what):
    bad = np.nonzero(np.asarray(a, np.uint32) != np.asarray(b, np.uint32))[0]
    assert a.shape == b.shape and bad.size == 0, "%s: %d mismatches, first at %s" % (
        what, bad.size, bad[:1])


CONFIGS = [
    dict(warps_per_cta=8, words_per_lane=4, kernel=0, ctas_per_sm=1, coop_percent=0),
    dict(warps_per_cta=4, words_per_lane=8, kernel=0, ctas_per_sm=0, coop_percent=100),
    dict(warps_per_cta=2, words_per_lane=4, kernel=0, ctas_per_sm=4, coop_percent=0),
    dict(warps_per_cta=4, words_per_lane=8, kernel=1),
]


@pytest.mark.parametrize("cfg", CONFIGS, ids=lambda c: "w%d_k%d_kern%d" % (
    c["warps_per_cta"], c["words_per_lane"], c["kernel"]))
@pytest.mark.parametrize("mexp", [11213, 23209])
def test_each_stream_uses_its_own_set(cfg, mexp):
    gps, ops = _sets(mexp, range(100, 108))
    rng = np.random.default_rng(mexp)
    n_streams = 45
    set_of = rng.integers(0, len(gps), n_streams).astype(np.uint32)
    seeds = rng.integers(0, 2 ** 32, n_streams, dtype=np.uint64).astype(np.uint32)
    st = mtgp.mtgp_init_statuses_multi(gps, set_of, seeds)
    states = np.stack([oracle.init_state(ops[set_of[s]], int(seeds[s])) for s in range(n_streams)])
    _same(mtgp.mtgp_get_statuses(st), states, "initial states")
    mtgp.mtgp_set_launch_config(st, **cfg)
    n = ops[0].n
    for call, fmt in enumerate(FMTS):
        ids = np.concatenate([np.arange(n_streams), rng.integers(0, n_streams, 15)]).astype(np.uint32)
        counts = rng.choice([0, 1, 31, n - 1, n, n + 1, 3 * n + 7, 20000, 70001], ids.size)
        got = _generate(st, ids, counts, fmt)
        ref, states = _replay(ops, set_of, states, ids, counts, fmt)
        _same(got, ref, "call %d fmt %d" % (call, fmt))
    _same(mtgp.mtgp_get_statuses(st), states, "final states")


def test_pipelined_and_row_by_row_sets_in_one_launch(tmp_path):
    """Sets with N - pos >= 256 take the software-pipelined row loop, a set
    with N - pos < 256 the row-by-row loop; both in the same launch."""
    mexp = 11213
    n = mexp // 32 + 1
    base = [oracle.params_generate(mexp, s) for s in (7, 8, 9)]
    poses = [5, n - 256, n - 200]
    ops = [oracle.params_from_fields(mexp, pos, b.sh1, b.sh2, list(b.rec_basis), list(b.tmp_basis))
           for b, pos in zip(base, poses)]
    gps = [mtgp.mtgp_params_load(_params_file(tmp_path, b, pos)) for b, pos in zip(base, poses)]
    set_of = np.array([0, 1, 2, 2, 1, 0, 2, 0, 1, 2], np.uint32)
    seeds = np.arange(10, dtype=np.uint32) * 977
    st = mtgp.mtgp_init_statuses_multi(gps, set_of, seeds)
    mtgp.mtgp_set_launch_config(st, warps_per_cta=4, words_per_lane=4, ctas_per_sm=2, coop_percent=0)
    states = np.stack([oracle.init_state(ops[set_of[s]], int(seeds[s])) for s in range(10)])
    ids = np.array([0, 1, 2, 3, 4, 5, 6, 7, 8, 9, 2, 1], np.uint32)
    counts = np.array([n * 20, n * 20 + 3, n * 20 + 5, 50000, 1, n, 123, 0, n * 2, 9999, n, 64],
                      np.uint64)
    for fmt in FMTS:
        got = _generate(st, ids, counts, fmt)
        ref, states = _replay(ops, set_of, states, ids, counts, fmt)
        _same(got, ref, "fmt %d" % fmt)
    _same(mtgp.mtgp_get_statuses(st), states, "final states")


def test_multi_set_plan_with_autotune():
    gps, ops = _sets(workloads.MEXP_MAIN, range(20))
    n_streams = 300
    set_of = (np.arange(n_streams) % 20).astype(np.uint32)
    seeds = np.arange(n_streams, dtype=np.uint32)
    st = mtgp.mtgp_init_statuses_multi(gps, set_of, seeds)
    states = mtgp.mtgp_get_statuses(st)
    ids = np.arange(n_streams, dtype=np.uint32)
    counts = np.floor(2.0 ** np.random.default_rng(4).uniform(8, 17, n_streams)).astype(np.uint64)
    total = int(counts.sum())
    out = torch.empty(total, dtype=torch.int32, device="cuda")
    plan = mtgp.mtgp_plan_create(st, ids, counts, mtgp.MTGP_U32, out)
    mtgp.mtgp_plan_autotune(plan)   # tuning restores the states it used
    for rep in range(2):
        mtgp.mtgp_plan_launch(plan)
        torch.cuda.synchronize()
        mtgp.mtgp_check(st)
        ref, states = _replay(ops, set_of, states, ids, counts, mtgp.MTGP_U32)
        _same(out.cpu().numpy().view(np.uint32), ref, "replay %d" % rep)
    assert mtgp.mtgp_plan_get_info(plan)["n_coop"] == 0
    plan.close()


def test_multi_set_noalloc():
    gps, ops = _sets(workloads.MEXP_MAIN, (3, 4))
    set_of = np.array([1, 0, 1, 1, 0], np.uint32)
    seeds = np.array([9, 8, 7, 6, 5], np.uint32)
    st = mtgp.mtgp_init_statuses_multi(gps, set_of, seeds)
    states = mtgp.mtgp_get_statuses(st)
    ids = np.array([4, 3, 2, 1, 0, 4], np.uint32)
    counts = np.array([1000, 2000, 3000, 351 * 5, 7, 4], np.uint64)
    out = torch.empty(int(counts.sum()), dtype=torch.int32, device="cuda")
    mtgp.mtgp_generate_noalloc(st, ids, counts, mtgp.MTGP_F32_01, out)
    torch.cuda.synchronize()
    ref, states = _replay(ops, set_of, states, ids, counts, mtgp.MTGP_F32_01)
    _same(out.cpu().numpy().view(np.uint32), ref, "noalloc")
    _same(mtgp.mtgp_get_statuses(st), states, "states")


def test_multi_set_errors():
    a = mtgp.mtgp_params_generate(11213, 1)
    b = mtgp.mtgp_params_generate(23209, 1)
    with pytest.raises(mtgp.MtgpError):
        mtgp.mtgp_init_statuses_multi([a, b], [0, 1], [1, 2])          # different Mexp
    with pytest.raises(mtgp.MtgpError):
        mtgp.mtgp_init_statuses_multi([a], [0, 1], [1, 2])             # set index out of range
    with pytest.raises(ValueError):
        mtgp.mtgp_init_statuses_multi([a], [0], [1, 2])                # length mismatch


def test_multi_set_serving_trace():
    """Continuous batching over streams with distinct parameter sets: every
    request equals its stream's oracle sequence replayed alone, in order."""
    tr = workloads.serving_trace(duration_s=0.05, rate=20000.0, n_streams=200, klo=0, khi=13, seed=6)
    gps, ops = _sets(workloads.MEXP_MAIN, range(50, 60))
    set_of = (np.arange(200) * 7 % 10).astype(np.uint32)
    st = mtgp.mtgp_init_statuses_multi(gps, set_of, np.arange(200, dtype=np.uint32))
    states = mtgp.mtgp_get_statuses(st)
    total = int(tr["counts"].sum())
    arena = 4 * (total + 64 * len(tr["t"]))
    srv = mtgp.mtgp_server_create(st, arena_bytes=arena, max_inflight=4)
    lat, offs, stats = mtgp.mtgp_server_run_trace(srv, tr["t"], tr["ids"], tr["counts"], tr["fmt"],
                                                  mode=0, record=True)
    host = mtgp.mtgp_server_read(srv, 0, arena // 4)
    for j, (sid, c, f) in enumerate(zip(tr["ids"], tr["counts"], tr["fmt"])):
        ref, states[sid] = oracle.generate(ops[set_of[sid]], states[sid], int(c), int(f))
        _same(host[int(offs[j]):int(offs[j]) + int(c)], ref, "request %d" % j)
    _same(mtgp.mtgp_get_statuses(st), states, "final states")

"""Serving (continuous batching) against the oracle.

Every request's output, produced in a mix of concurrent requests, must equal
what the oracle gives for that stream's request sequence replayed alone and
in order (tolerance 0: the numbers are exact).  Also checks the comparison
mode (one launch per request) and the submit/progress API with a small arena
that forces admission to wait.
"""
import os

import numpy as np
import pytest

import oracle
from paper_1501_07701_gb300 import mtgp, workloads

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")
THREADS = os.cpu_count() or 4


@pytest.fixture(scope="module", autouse=True)
def _built():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1501_07701_gb300 import build
    build.build()
    mtgp.load_library()


def _setup(n_streams):
    gp = mtgp.mtgp_params_generate(workloads.MEXP_MAIN, workloads.PARAM_SEED)
    op = oracle.params_generate(workloads.MEXP_MAIN, workloads.PARAM_SEED)
    st = mtgp.mtgp_init_statuses(gp, np.arange(n_streams, dtype=np.uint32))
    return st, op, mtgp.mtgp_get_statuses(st)


def _arena_view(server, total_elems):
    assert mtgp.mtgp_server_arena(server) != 0
    return mtgp.mtgp_server_read(server, 0, total_elems)


def _replay_oracle(op, states, ids, counts, fmts):
    """Each request alone, in arrival order per stream."""
    states = states.copy()
    outs = []
    for sid, c, f in zip(ids, counts, fmts):
        o, states[sid] = oracle.generate(op, states[sid], int(c), int(f))
        outs.append(o)
    return outs, states


def _small_trace(n_req=2500, n_streams=300, rate=20000.0, seed=5):
    tr = workloads.serving_trace(duration_s=n_req / rate, rate=rate, n_streams=n_streams, klo=0,
                                 khi=14, seed=seed)
    return tr


@pytest.mark.parametrize("mode", [0, 1])
def test_trace_results_equal_alone(mode):
    tr = _small_trace()
    n_streams = tr["n_streams"]
    st, op, states0 = _setup(n_streams)
    total = int(tr["counts"].sum())
    arena = 4 * (total + 64 * len(tr["t"]))
    srv = mtgp.mtgp_server_create(st, arena_bytes=arena, max_inflight=4)
    lat, offs, stats = mtgp.mtgp_server_run_trace(srv, tr["t"], tr["ids"], tr["counts"], tr["fmt"],
                                                  mode=mode, record=True)
    assert stats["requests"] == len(tr["t"])
    assert np.all(lat > 0)
    arena_host = _arena_view(srv, arena // 4)
    ref, ref_states = _replay_oracle(op, states0, tr["ids"], tr["counts"], tr["fmt"])
    for j in range(len(ref)):
        got = arena_host[int(offs[j]):int(offs[j]) + int(tr["counts"][j])]
        assert np.array_equal(got, ref[j]), "request %d (stream %d)" % (j, tr["ids"][j])
    assert np.array_equal(mtgp.mtgp_get_statuses(st), ref_states)
    if mode == 0:
        assert stats["ticks"] < len(tr["t"])   # requests were coalesced


@pytest.mark.parametrize("max_piece", [64, 351, 5000])
def test_split_ticks_equal_alone(max_piece):
    """Ticks whose long requests are cut into pieces started by jumps: every
    result and final state equals the oracle's request-by-request replay."""
    tr = _small_trace(n_req=1500, n_streams=200, seed=8)
    st, op, states0 = _setup(tr["n_streams"])
    total = int(tr["counts"].sum())
    arena = 4 * (total + 64 * len(tr["t"]))
    srv = mtgp.mtgp_server_create(st, arena_bytes=arena, max_inflight=4, max_piece=max_piece)
    lat, offs, stats = mtgp.mtgp_server_run_trace(srv, tr["t"], tr["ids"], tr["counts"], tr["fmt"],
                                                  mode=0, record=True)
    assert stats["requests"] == len(tr["t"]) and stats["jumps"] > 0
    arena_host = _arena_view(srv, arena // 4)
    ref, ref_states = _replay_oracle(op, states0, tr["ids"], tr["counts"], tr["fmt"])
    for j in range(len(ref)):
        got = arena_host[int(offs[j]):int(offs[j]) + int(tr["counts"][j])]
        assert np.array_equal(got, ref[j]), "request %d (stream %d)" % (j, tr["ids"][j])
    assert np.array_equal(mtgp.mtgp_get_statuses(st), ref_states)


def test_split_ticks_per_stream_sets_submit_progress():
    """submit / progress with split ticks on a handle with one parameter set per stream."""
    set_seeds = [workloads.PARAM_SEED + 3 + k for k in range(3)]
    gsets = [mtgp.mtgp_params_generate(workloads.MEXP_MAIN, k) for k in set_seeds]
    osets = [oracle.params_generate(workloads.MEXP_MAIN, k) for k in set_seeds]
    n = 12
    set_of = (np.arange(n) % 3).astype(np.uint32)
    st = mtgp.mtgp_init_statuses_multi(gsets, set_of, np.arange(n, dtype=np.uint32))
    states = mtgp.mtgp_get_statuses(st)
    rng = np.random.default_rng(21)
    ids = rng.integers(0, n, 40).astype(np.uint32)
    counts = rng.integers(1, 30000, 40).astype(np.uint64)
    fmts = rng.integers(0, 3, 40).astype(np.int32)
    srv = mtgp.mtgp_server_create(st, arena_bytes=4 * (int(counts.sum()) + 4096), max_piece=4000)
    for j in range(40):
        mtgp.mtgp_server_submit(srv, ids[j], counts[j], fmts[j], j)
    done = {}
    while len(done) < 40:
        for c in mtgp.mtgp_server_progress(srv):
            done[c["tag"]] = c
    arena = mtgp.mtgp_server_read(srv, 0, int(counts.sum()) + 4096)
    for j in range(40):
        ref, states[ids[j]] = oracle.generate(osets[set_of[ids[j]]], states[ids[j]], int(counts[j]),
                                              int(fmts[j]))
        c = done[j]
        assert np.array_equal(arena[c["arena_offset"]:c["arena_offset"] + c["count"]], ref), j
        mtgp.mtgp_server_release(srv, c["arena_offset"], c["count"])
    assert np.array_equal(mtgp.mtgp_get_statuses(st), states)


def test_split_ticks_reject_tiny_pieces():
    st, _, _ = _setup(4)
    with pytest.raises(mtgp.MtgpError) as ei:
        mtgp.mtgp_server_create(st, arena_bytes=1 << 20, max_piece=63)
    assert ei.value.status == 1


def test_submit_progress_with_small_arena():
    st, op, states0 = _setup(16)
    rng = np.random.default_rng(9)
    n = 400
    ids = rng.integers(0, 16, n).astype(np.uint32)
    ids[:50] = 3                         # a burst on one stream
    counts = rng.integers(1, 20000, n).astype(np.uint64)
    fmts = rng.choice([0, 1, 2], n).astype(np.int32)
    srv = mtgp.mtgp_server_create(st, arena_bytes=4 * 60000, max_inflight=3, max_tick_requests=7)
    for j in range(n):
        mtgp.mtgp_server_submit(srv, ids[j], counts[j], fmts[j], j)
    ref, ref_states = _replay_oracle(op, states0, ids, counts, fmts)
    got = {}
    while len(got) < n:
        for c in mtgp.mtgp_server_progress(srv):
            got[c["tag"]] = mtgp.mtgp_server_read(srv, c["arena_offset"], c["count"])
            mtgp.mtgp_server_release(srv, c["arena_offset"], c["count"])
    for j in range(n):
        assert np.array_equal(got[j], ref[j]), j
    assert np.array_equal(mtgp.mtgp_get_statuses(st), ref_states)


def test_submit_rejects_oversized_and_bad_ids():
    st, _, _ = _setup(4)
    srv = mtgp.mtgp_server_create(st, arena_bytes=4096)
    with pytest.raises(mtgp.MtgpError) as ei:
        mtgp.mtgp_server_submit(srv, 0, 5000, 0, 1)
    assert ei.value.status == 5
    with pytest.raises(mtgp.MtgpError) as ei:
        mtgp.mtgp_server_submit(srv, 9, 10, 0, 1)
    assert ei.value.status == 1


def test_progress_times_out_when_completion_is_not_seen():
    """Failure detection on the host: with the diagnostic hold the server
    never sees its tick complete (the kernel itself runs normally), so
    progress must give up with MTGP_ETIMEOUT once tick_timeout_s has passed,
    keep the tick, and deliver the exact result once the hold is lifted."""
    import time
    st, op, states0 = _setup(4)
    srv = mtgp.mtgp_server_create(st, arena_bytes=4 << 20, tick_timeout_s=0.2)
    mtgp.mtgp_server_debug_hold(srv, True)
    mtgp.mtgp_server_submit(srv, 2, 5000, mtgp.MTGP_U32, 77)
    t0 = time.monotonic()
    with pytest.raises(mtgp.MtgpError) as ei:
        while time.monotonic() - t0 < 5.0:
            assert mtgp.mtgp_server_progress(srv) == []
            time.sleep(0.01)
    assert ei.value.status == 4                      # MTGP_ETIMEOUT
    assert 0.2 <= time.monotonic() - t0 < 5.0
    mtgp.mtgp_server_debug_hold(srv, False)
    got = []
    while not got:
        got = mtgp.mtgp_server_progress(srv)
    assert got[0]["tag"] == 77
    ref, _ = oracle.generate(op, states0[2], 5000)
    assert np.array_equal(mtgp.mtgp_server_read(srv, got[0]["arena_offset"], 5000), ref)


@pytest.mark.parametrize("mode", [0, 1])
def test_run_trace_times_out_when_completion_is_not_seen(mode):
    """Both replay modes return MTGP_ETIMEOUT instead of waiting forever when
    completions are never observed; freeing the server afterwards waits for
    the (finished) kernels and returns normally."""
    st, _, _ = _setup(8)
    srv = mtgp.mtgp_server_create(st, arena_bytes=16 << 20, tick_timeout_s=0.1)
    mtgp.mtgp_server_debug_hold(srv, True)
    t = np.array([0.0, 0.001, 0.002])
    with pytest.raises(mtgp.MtgpError) as ei:
        mtgp.mtgp_server_run_trace(srv, t, np.array([1, 2, 1], np.uint32),
                                   np.array([1000, 2000, 3000], np.uint64),
                                   np.zeros(3, np.int32), mode=mode)
    assert ei.value.status == 4
    srv.close()


def test_serving_trace_prefix_at_full_size():
    """The serving workload itself (65 536 resident streams, the seed-11
    Poisson arrivals at 50 000 requests/s, k log-uniform in [2^8, 2^20], u32
    or f32 [0,1), 8 GiB admission arena), replayed in real time through
    continuous batching for the prefix of the trace whose outputs fit the
    arena at once (about 0.2 s of arrivals).  Every request's output must
    equal the oracle's replay of that stream's requests alone and in order,
    and every final state must match."""
    from concurrent.futures import ThreadPoolExecutor
    tr = workloads.serving_trace()                        # the 10 s trace; its prefix
    cum = np.cumsum(tr["counts"].astype(np.int64))
    n = int(np.searchsorted(cum, 1_200_000_000))          # ~4.8 GB of results
    t, ids, counts, fmts = tr["t"][:n], tr["ids"][:n], tr["counts"][:n], tr["fmt"][:n]
    st, op, states0 = _setup(tr["n_streams"])
    srv = mtgp.mtgp_server_create(st, arena_bytes=8 << 30, max_inflight=4)
    lat, offs, stats = mtgp.mtgp_server_run_trace(srv, t, ids, counts, fmts, mode=0, record=True)
    assert stats["requests"] == n and stats["ticks"] < n
    end = int((offs + counts).max())
    arena = mtgp.mtgp_server_read(srv, 0, end)
    per_stream = {}
    for j in range(n):
        per_stream.setdefault(int(ids[j]), []).append(j)

    def replay(sid):
        s = states0[sid].copy()
        for j in per_stream[sid]:
            ref, s = oracle.generate(op, s, int(counts[j]), int(fmts[j]))
            got = arena[int(offs[j]):int(offs[j]) + int(counts[j])]
            if not np.array_equal(got, ref):
                return "request %d (stream %d) differs" % (j, sid), s
        return None, s

    final = states0.copy()
    with ThreadPoolExecutor(THREADS) as ex:
        for sid, (err, s) in zip(per_stream, ex.map(replay, list(per_stream))):
            assert err is None, err
            final[sid] = s
    assert np.array_equal(mtgp.mtgp_get_statuses(st), final)
    print("serving prefix verified: %d requests, %.3f s of arrivals, %d numbers" % (
        n, float(t[-1]), int(counts.sum())))

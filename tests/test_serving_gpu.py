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

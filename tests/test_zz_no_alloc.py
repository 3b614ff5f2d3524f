"""The allocation-free entry point (mtgp_generate_noalloc).

It exists for callers that cannot have device memory allocated for them once
they run (a simulation holding a fixed device-memory budget, a loop that must
not enter the allocator).  Every case runs two calls in a row and checks them
bit for bit (the generator is exact, tolerance 0) against the CPU oracle and
against the ordinary entry point mtgp_generate_u32 / _f32 on a twin handle
that starts from the same states.  The cases cover the three output formats,
a handle with one parameter set per stream, a launch configuration that hands
the longest streams to whole CTAs, and a non-default CUDA stream.  Another
test checks that warm calls leave the device's free memory and torch's
allocator untouched.  Collected last on purpose.
"""
import os

import numpy as np
import pytest

import oracle
from paper_1501_07701_gb300 import mtgp, workloads

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")
THREADS = os.cpu_count() or 4
N_STREAMS = 48


@pytest.fixture(scope="module", autouse=True)
def _built():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1501_07701_gb300 import build
    build.build()
    mtgp.load_library()


def _handles(per_stream_sets):
    """Two handles with identical states, plus the oracle's parameter set of
    each stream and those states."""
    seeds = np.arange(N_STREAMS, dtype=np.uint32)
    if per_stream_sets:
        set_seeds = [workloads.PARAM_SEED + 1 + k for k in range(5)]
        gsets = [mtgp.mtgp_params_generate(workloads.MEXP_MAIN, k) for k in set_seeds]
        set_of = (np.arange(N_STREAMS) % 5).astype(np.uint32)
        a = mtgp.mtgp_init_statuses_multi(gsets, set_of, seeds)
        b = mtgp.mtgp_init_statuses_multi(gsets, set_of, seeds)
        osets = [oracle.params_generate(workloads.MEXP_MAIN, k) for k in set_seeds]
        op_of = [osets[int(set_of[s])] for s in range(N_STREAMS)]
    else:
        gp = mtgp.mtgp_params_generate(workloads.MEXP_MAIN, workloads.PARAM_SEED)
        a = mtgp.mtgp_init_statuses(gp, seeds)
        b = mtgp.mtgp_init_statuses(gp, seeds)
        op = oracle.params_generate(workloads.MEXP_MAIN, workloads.PARAM_SEED)
        op_of = [op] * N_STREAMS
    states = np.stack([oracle.init_state(op_of[s], int(seeds[s])) for s in range(N_STREAMS)])
    assert np.array_equal(mtgp.mtgp_get_statuses(a), states)
    return a, b, op_of, states


def _oracle(op_of, states, ids, counts, fmt):
    """Requests in call order, each stream with its own parameter set."""
    states = states.copy()
    outs = []
    for sid, c in zip(ids, counts):
        o, states[sid] = oracle.generate(op_of[sid], states[sid], int(c), fmt)
        outs.append(o)
    return np.concatenate(outs), states


CASES = [
    ("one set", mtgp.MTGP_U32, False, None, False),
    ("one set", mtgp.MTGP_F32_12, False, None, False),
    ("one set", mtgp.MTGP_F32_01, False, None, False),
    ("per-stream sets", mtgp.MTGP_U32, True, None, False),
    ("per-stream sets", mtgp.MTGP_F32_01, True, None, True),
    ("CTA-owned longest streams", mtgp.MTGP_U32, False,
     dict(warps_per_cta=4, words_per_lane=4, coop_percent=20, ctas_per_sm=1), False),
    ("torch stream", mtgp.MTGP_F32_12, False, None, True),
]


@pytest.mark.parametrize("label,fmt,multi,cfg,side_stream", CASES,
                         ids=["%s-%d-%d" % (c[0], c[1], i) for i, c in enumerate(CASES)])
def test_noalloc_matches_oracle_and_generate_two_calls(label, fmt, multi, cfg, side_stream):
    a, b, op_of, states = _handles(multi)
    if cfg:
        mtgp.mtgp_set_launch_config(a, **cfg)
        mtgp.mtgp_set_launch_config(b, **cfg)
    cs = torch.cuda.Stream() if side_stream else torch.cuda.current_stream()
    rng = np.random.default_rng(17 + len(label) + fmt)
    for call in range(2):
        ids = np.concatenate([np.arange(N_STREAMS), rng.integers(0, N_STREAMS, 60)]).astype(np.uint32)
        counts = rng.integers(0, 30000, ids.size).astype(np.uint64)
        counts[:4] = [0, 1, 351, 200000]          # empty, single, one row, one long stream
        total = int(counts.sum())
        out_ref = torch.full((total,), -1, dtype=torch.int32, device="cuda")
        out_na = torch.full((total,), -2, dtype=torch.int32, device="cuda")
        torch.cuda.synchronize()
        with torch.cuda.stream(cs):
            if fmt == mtgp.MTGP_U32:
                mtgp.mtgp_generate_u32(a, ids, counts, out_ref, cs)
            else:
                mtgp.mtgp_generate_f32(a, ids, counts, fmt, out_ref, cs)
            mtgp.mtgp_generate_noalloc(b, ids, counts, fmt, out_na, cs)
        cs.synchronize()
        mtgp.mtgp_check(b, cs)
        ref, states = _oracle(op_of, states, ids, counts, fmt)
        got = out_na.cpu().numpy().view(np.uint32)
        assert np.array_equal(got, ref), "%s, call %d: differs from the oracle" % (label, call)
        assert torch.equal(out_ref, out_na), "%s, call %d: differs from mtgp_generate" % (label, call)
        assert np.array_equal(mtgp.mtgp_get_statuses(b), states), "%s, call %d: states" % (label, call)
        assert np.array_equal(mtgp.mtgp_get_statuses(a), states)


def test_noalloc_allocates_no_device_memory():
    """Warm calls on a handle that never went through the ordinary entry
    point (whose work-table buffers are allocated on first use) leave the
    device's free memory and torch's allocator exactly as they were."""
    seeds = np.arange(16, dtype=np.uint32)
    gp = mtgp.mtgp_params_generate(workloads.MEXP_MAIN, workloads.PARAM_SEED)
    warm = mtgp.mtgp_init_statuses(gp, seeds)
    fresh = mtgp.mtgp_init_statuses(gp, seeds)
    ids = np.arange(16, dtype=np.uint32)
    counts = np.full(16, 5000, np.uint64)
    out = torch.empty(80000, dtype=torch.int32, device="cuda")
    mtgp.mtgp_generate_noalloc(warm, ids, counts, mtgp.MTGP_U32, out)   # loads the kernel module
    torch.cuda.synchronize()
    free0, _ = torch.cuda.mem_get_info()
    alloc0 = torch.cuda.memory_allocated()
    for _ in range(3):
        mtgp.mtgp_generate_noalloc(fresh, ids, counts, mtgp.MTGP_F32_01, out)
    torch.cuda.synchronize()
    free1, _ = torch.cuda.mem_get_info()
    assert free1 == free0, "device free memory changed by %d bytes" % (free0 - free1)
    assert torch.cuda.memory_allocated() == alloc0
    op = oracle.params_generate(workloads.MEXP_MAIN, workloads.PARAM_SEED)
    st = oracle.init_state(op, 0)
    ref, _ = oracle.generate(op, st, 3 * 5000, oracle.F32_01)
    assert np.array_equal(out[:5000].cpu().numpy().view(np.uint32), ref[10000:])


def test_noalloc_rejects_too_many_requests():
    a, _, _, _ = _handles(False)
    out = torch.empty(2000, dtype=torch.int32, device="cuda")
    with pytest.raises(mtgp.MtgpError) as ei:
        mtgp.mtgp_generate_noalloc(a, np.zeros(1025, np.uint32), np.ones(1025, np.uint64),
                                   mtgp.MTGP_U32, out)
    assert ei.value.status == 1 and "1024" in str(ei.value)


def test_noalloc_refuses_stream_capture():
    """Inside a stream capture the call is refused (its host-side table
    would be read at graph replay, after later calls overwrote it); the
    capture itself stays usable and the stream state is unchanged."""
    a, _, _, states = _handles(False)
    out = torch.empty(1000, dtype=torch.int32, device="cuda")
    cs = torch.cuda.Stream()
    g = torch.cuda.CUDAGraph()
    with pytest.raises(mtgp.MtgpError) as ei:
        with torch.cuda.graph(g, stream=cs):
            mtgp.mtgp_generate_noalloc(a, np.zeros(1, np.uint32), np.full(1, 1000, np.uint64),
                                       mtgp.MTGP_U32, out, cs)
    assert ei.value.status == 1 and "graph" in str(ei.value)
    torch.cuda.synchronize()
    assert np.array_equal(mtgp.mtgp_get_statuses(a), states)

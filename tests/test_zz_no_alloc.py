"""The allocation-free entry point (mtgp_generate_noalloc) against the
ordinary one.

It exists for callers that cannot have device memory allocated for them once
they run (a simulation holding a fixed device-memory budget, a loop that must
not enter the allocator).  Two twin stream sets start from the same states;
one advances through mtgp_generate_noalloc, the other through
mtgp_generate_u32 / _f32, for two calls in a row; outputs and states must be
identical bit for bit (the generator is exact, tolerance 0).  Collected last
on purpose.
"""
import numpy as np
import pytest

from paper_1501_07701_gb300 import mtgp, workloads

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


@pytest.fixture(scope="module", autouse=True)
def _built():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1501_07701_gb300 import build
    build.build()
    mtgp.load_library()


def _twins(n_streams):
    p = mtgp.mtgp_params_generate(workloads.MEXP_MAIN, workloads.PARAM_SEED)
    a = mtgp.mtgp_init_statuses(p, np.arange(n_streams, dtype=np.uint32))
    b = mtgp.mtgp_init_statuses(p, np.zeros(n_streams, dtype=np.uint32))
    mtgp.mtgp_set_statuses(b, mtgp.mtgp_get_statuses(a))
    return a, b


@pytest.mark.parametrize("fmt", [mtgp.MTGP_U32, mtgp.MTGP_F32_01])
def test_noalloc_matches_generate_two_calls(fmt):
    a, b = _twins(64)
    rng = np.random.default_rng(17)
    for call in range(2):
        ids = np.concatenate([np.arange(64), rng.integers(0, 64, 100)]).astype(np.uint32)
        counts = rng.integers(0, 30000, ids.size).astype(np.uint64)
        counts[:3] = [0, 1, 351]
        total = int(counts.sum())
        out_ref = torch.full((total,), -1, dtype=torch.int32, device="cuda")
        out_na = torch.full((total,), -2, dtype=torch.int32, device="cuda")
        if fmt == mtgp.MTGP_U32:
            mtgp.mtgp_generate_u32(a, ids, counts, out_ref)
        else:
            mtgp.mtgp_generate_f32(a, ids, counts, fmt, out_ref)
        mtgp.mtgp_generate_noalloc(b, ids, counts, fmt, out_na)
        torch.cuda.synchronize()
        mtgp.mtgp_check(b)
        assert torch.equal(out_ref, out_na), "call %d" % call
        assert np.array_equal(mtgp.mtgp_get_statuses(a), mtgp.mtgp_get_statuses(b))


def test_noalloc_rejects_too_many_requests():
    a, _ = _twins(4)
    out = torch.empty(2000, dtype=torch.int32, device="cuda")
    with pytest.raises(mtgp.MtgpError) as ei:
        mtgp.mtgp_generate_noalloc(a, np.zeros(1025, np.uint32), np.ones(1025, np.uint64),
                                   mtgp.MTGP_U32, out)
    assert ei.value.status == 1 and "1024" in str(ei.value)

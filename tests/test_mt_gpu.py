"""GPU parity of the original-MT comparison generator (Sec. 5.3) against its
oracle: bit-exact outputs in every format and bit-exact states afterwards.

The cases reach every kernel shape: four 32-number sub-steps per step
(n - m >= 128: MT19937, p = 44497), two (p = 4423), one (p = 3217, the
paper's period), and steps narrower than a warp (n - m < 32: p = 521, 607);
streams long enough to move the sliding buffer many times; requests that
start and end inside a step; and the largest state the library accepts.
"""
import numpy as np
import pytest

import oracle.mt as omt
from paper_1501_07701_gb300 import mtgp

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


@pytest.fixture(scope="module", autouse=True)
def _built():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1501_07701_gb300 import build
    build.build()
    mtgp.load_library()


def _set(name):
    """(library parameter set, oracle parameter set) by name."""
    if name == "mt19937":
        return mtgp.mtgp_mt_params_mt19937(), omt.params_mt19937()
    p = int(name[1:])
    return mtgp.mtgp_mt_params_generate(p, 17), omt.params_generate(p, 17)


FMTS = [mtgp.MTGP_U32, mtgp.MTGP_F32_12, mtgp.MTGP_F32_01]


def _run(mp, op, seeds, ids, counts, fmt):
    mt = mtgp.mtgp_mt_init(mp, seeds)
    states = np.stack([omt.init_state(op, int(s)) for s in seeds])
    np.testing.assert_array_equal(mtgp.mtgp_mt_get_statuses(mt), states)
    counts = np.asarray(counts, np.uint64)
    out = torch.full((max(int(counts.sum()), 1),), -1, dtype=torch.int32, device="cuda")
    mtgp.mtgp_mt_generate(mt, ids, counts, fmt, out)
    mtgp.mtgp_mt_check(mt)
    ref, ref_states = omt.generate_many(op, states, ids, counts, fmt, 8)
    got = out.cpu().numpy().view(np.uint32)[:counts.sum()]
    return mt, got, ref, ref_states


RAGGED = [0, 1, 31, 32, 33, 95, 127, 128, 129, 255, 257, 1000, 4095, 4097, 70001, 250000]


@pytest.mark.parametrize("name", ["mt19937", "p521", "p607", "p3217", "p4423", "p44497"])
@pytest.mark.parametrize("fmt", FMTS)
def test_ragged_requests_match_oracle(name, fmt):
    mp, op = _set(name)
    assert mp.as_dict() == op.as_dict()
    seeds = np.arange(100, 100 + len(RAGGED), dtype=np.uint32)
    ids = np.arange(len(RAGGED), dtype=np.uint32)
    mt, got, ref, ref_states = _run(mp, op, seeds, ids, RAGGED, fmt)
    np.testing.assert_array_equal(got, ref)
    np.testing.assert_array_equal(mtgp.mtgp_mt_get_statuses(mt), ref_states)


@pytest.mark.parametrize("name", ["mt19937", "p3217", "p521"])
def test_repeated_streams_and_chunked_calls(name):
    """Several requests of one stream in one call are served in array order;
    a sequence of calls continues each stream where the last one stopped."""
    mp, op = _set(name)
    seeds = np.array([5, 6, 7, 8, 9, 10], np.uint32)
    ids = np.array([3, 0, 3, 5, 0, 3, 1, 3], np.uint32)
    counts = np.array([100, 7, 0, 333, 1000, 65, 32, 129], np.uint64)
    mt, got, ref, ref_states = _run(mp, op, seeds, ids, counts, mtgp.MTGP_U32)
    np.testing.assert_array_equal(got, ref)
    states = ref_states
    rng = np.random.default_rng(3)
    for _ in range(4):
        ids = rng.integers(0, 6, 9).astype(np.uint32)
        counts = rng.integers(0, 3000, 9).astype(np.uint64)
        out = torch.empty(int(counts.sum()), dtype=torch.int32, device="cuda")
        mtgp.mtgp_mt_generate(mt, ids, counts, mtgp.MTGP_F32_01, out)
        ref, states = omt.generate_many(op, states, ids, counts, omt.F32_01, 4)
        np.testing.assert_array_equal(out.cpu().numpy().view(np.uint32), ref)
    np.testing.assert_array_equal(mtgp.mtgp_mt_get_statuses(mt), states)


def test_many_streams_paper_period():
    """4096 streams of the 2^3217 generator, uneven lengths."""
    mp, op = _set("p3217")
    n = 4096
    seeds = np.arange(n, dtype=np.uint32)
    counts = (np.arange(n, dtype=np.uint64) * 2654435761 % 20011).astype(np.uint64)
    mt, got, ref, ref_states = _run(mp, op, seeds, np.arange(n), counts, mtgp.MTGP_U32)
    np.testing.assert_array_equal(got, ref)
    np.testing.assert_array_equal(mtgp.mtgp_mt_get_statuses(mt), ref_states)


def test_one_long_stream():
    """2^22 numbers of MT19937 from one stream: the sliding buffer is moved
    back about 1250 times."""
    mp, op = _set("mt19937")
    mt, got, ref, ref_states = _run(mp, op, np.array([5489], np.uint32), [0], [1 << 22],
                                    mtgp.MTGP_U32)
    assert int(got[9999]) == 4123659995
    np.testing.assert_array_equal(got, ref)
    np.testing.assert_array_equal(mtgp.mtgp_mt_get_statuses(mt), ref_states)


def test_largest_state():
    """n = 4096 words (the library's limit): a 33 KB buffer per warp."""
    op = omt.params_from_fields(p=32 * 4096 - 5, n=4096, r=5, m=1000, a=0x9908B0DF, u=11, s=7,
                                b=0x9D2C5680, t=15, c=0xEFC60000, l=18)
    mp = mtgp.MtParams(*[getattr(op, f) for f, _ in mtgp.MtParams._fields_])
    seeds = np.array([1, 2, 3], np.uint32)
    mt, got, ref, ref_states = _run(mp, op, seeds, [0, 1, 2], [50000, 4096, 12289], mtgp.MTGP_U32)
    np.testing.assert_array_equal(got, ref)
    np.testing.assert_array_equal(mtgp.mtgp_mt_get_statuses(mt), ref_states)


def test_set_statuses_round_trip():
    mp, op = _set("p3217")
    mt = mtgp.mtgp_mt_init(mp, np.arange(8, dtype=np.uint32))
    rng = np.random.default_rng(11)
    states = rng.integers(0, 2 ** 32, (8, op.n), dtype=np.uint64).astype(np.uint32)
    mtgp.mtgp_mt_set_statuses(mt, states)
    np.testing.assert_array_equal(mtgp.mtgp_mt_get_statuses(mt), states)
    counts = np.full(8, 777, np.uint64)
    out = torch.empty(8 * 777, dtype=torch.int32, device="cuda")
    mtgp.mtgp_mt_generate(mt, np.arange(8), counts, mtgp.MTGP_U32, out)
    ref, ref_states = omt.generate_many(op, states, np.arange(8), counts, omt.U32, 4)
    np.testing.assert_array_equal(out.cpu().numpy().view(np.uint32), ref)
    np.testing.assert_array_equal(mtgp.mtgp_mt_get_statuses(mt), ref_states)


def test_argument_errors_change_nothing():
    mp, op = _set("p3217")
    mt = mtgp.mtgp_mt_init(mp, np.arange(4, dtype=np.uint32))
    before = mtgp.mtgp_mt_get_statuses(mt)
    out = torch.empty(1024, dtype=torch.int32, device="cuda")
    with pytest.raises(mtgp.MtgpError):
        mtgp.mtgp_mt_generate(mt, [4], [10], mtgp.MTGP_U32, out)        # id out of range
    with pytest.raises(mtgp.MtgpError):
        mtgp.mtgp_mt_generate(mt, [0], [10], 3, out)                     # format
    with pytest.raises(mtgp.MtgpError):
        mtgp.mtgp_mt_generate(mt, [0], [10], mtgp.MTGP_U32, out.data_ptr() + 2)   # alignment
    torch.cuda.synchronize()
    np.testing.assert_array_equal(mtgp.mtgp_mt_get_statuses(mt), before)
    bad = mtgp.MtParams(*[getattr(mp, f) for f, _ in mtgp.MtParams._fields_])
    bad.m = bad.n
    with pytest.raises(mtgp.MtgpError):
        mtgp.mtgp_mt_init(bad, np.arange(2, dtype=np.uint32))
    bad = mtgp.MtParams(*[getattr(mp, f) for f, _ in mtgp.MtParams._fields_])
    bad.r = 14
    with pytest.raises(mtgp.MtgpError):
        mtgp.mtgp_mt_init(bad, np.arange(2, dtype=np.uint32))
    # an empty call is fine and launches nothing
    mtgp.mtgp_mt_generate(mt, [1, 2], [0, 0], mtgp.MTGP_U32, None)
    mtgp.mtgp_mt_check(mt)


def _oracle_multi(osets, set_of, seeds, ids, counts, fmt):
    """Per-stream sets on the oracle: requests in array order, each stream
    with its own set."""
    states = [omt.init_state(osets[set_of[s]], int(seeds[s])) for s in range(len(seeds))]
    pieces = []
    for i, c in zip(ids, counts):
        o, states[i] = omt.generate(osets[set_of[i]], states[i], int(c), fmt)
        pieces.append(o)
    return np.concatenate(pieces) if pieces else np.zeros(0, np.uint32), np.stack(states)


@pytest.mark.parametrize("fmt", FMTS)
def test_one_set_per_stream(fmt):
    """Seven seed-generated p = 3217 sets (a, b, c differ); stream s uses set
    s mod 7."""
    osets = [omt.params_generate(3217, 500 + k) for k in range(7)]
    msets = [mtgp.mtgp_mt_params_generate(3217, 500 + k) for k in range(7)]
    n = 40
    seeds = np.arange(1000, 1000 + n, dtype=np.uint32)
    set_of = (np.arange(n) % 7).astype(np.uint32)
    mt = mtgp.mtgp_mt_init_multi(msets, set_of, seeds)
    ids = np.concatenate([np.arange(n), [3, 3, 10]]).astype(np.uint32)
    counts = np.array([(i * 7919) % 30011 for i in range(n)] + [1, 64, 5000], np.uint64)
    out = torch.empty(int(counts.sum()), dtype=torch.int32, device="cuda")
    mtgp.mtgp_mt_generate(mt, ids, counts, fmt, out)
    ref, ref_states = _oracle_multi(osets, set_of, seeds, ids, counts, fmt)
    np.testing.assert_array_equal(out.cpu().numpy().view(np.uint32), ref)
    np.testing.assert_array_equal(mtgp.mtgp_mt_get_statuses(mt), ref_states)


def test_sets_with_different_step_widths():
    """Sets of one state size whose m differ (W = n - m = 51, 71, 11 and 96):
    the launch is shaped for the widest step and each stream steps at its
    own width."""
    base = omt.params_generate(3217, 9).as_dict()
    osets = []
    for m, a in [(50, 0x9908B0DF), (30, 0xB5026F5A), (90, 0x8E3A1C27), (5, 0xF00DF00D)]:
        f = dict(base, m=m, a=a)
        osets.append(omt.params_from_fields(**f))
    msets = [mtgp.MtParams(*[getattr(q, f) for f, _ in mtgp.MtParams._fields_]) for q in osets]
    n = 16
    seeds = np.arange(n, dtype=np.uint32)
    set_of = (np.arange(n) % 4).astype(np.uint32)
    mt = mtgp.mtgp_mt_init_multi(msets, set_of, seeds)
    ids = np.arange(n, dtype=np.uint32)
    counts = np.array([0, 1, 11, 12, 51, 52, 71, 72, 96, 97, 1000, 3333, 20000, 65537, 5, 100000],
                      np.uint64)
    out = torch.empty(int(counts.sum()), dtype=torch.int32, device="cuda")
    mtgp.mtgp_mt_generate(mt, ids, counts, mtgp.MTGP_U32, out)
    ref, ref_states = _oracle_multi(osets, set_of, seeds, ids, counts, omt.U32)
    np.testing.assert_array_equal(out.cpu().numpy().view(np.uint32), ref)
    np.testing.assert_array_equal(mtgp.mtgp_mt_get_statuses(mt), ref_states)


def test_multi_set_argument_errors():
    a = mtgp.mtgp_mt_params_generate(3217, 1)
    b = mtgp.mtgp_mt_params_generate(4423, 1)
    seeds = np.arange(4, dtype=np.uint32)
    with pytest.raises(mtgp.MtgpError):
        mtgp.mtgp_mt_init_multi([a, b], [0, 1, 0, 1], seeds)          # state sizes differ
    with pytest.raises(mtgp.MtgpError):
        mtgp.mtgp_mt_init_multi([a, a], [0, 1, 2, 0], seeds)          # index >= n_sets


def test_single_request_beyond_2p32():
    """Maximum size: one MT19937 request of 2^32 + 1000 numbers from one
    stream (17 GB of output; step and output indices past 32 bits).  The
    oracle runs the same 2^32 + 1000 numbers in 2^28-number chunks; the first
    2^20 outputs, the last 1000 and the final state must match."""
    mp, op = _set("mt19937")
    big = (1 << 32) + 1000
    mt = mtgp.mtgp_mt_init(mp, np.array([4357, 1], np.uint32))
    s0 = mtgp.mtgp_mt_get_statuses(mt)[0]
    out = torch.empty(big, dtype=torch.int32, device="cuda")
    mtgp.mtgp_mt_generate(mt, [0], [big], mtgp.MTGP_U32, out)
    mtgp.mtgp_mt_check(mt)
    first, s = omt.generate(op, s0, 1 << 20)
    np.testing.assert_array_equal(out[:1 << 20].cpu().numpy().view(np.uint32), first)
    left = big - (1 << 20)
    while left > 1000:
        step = min(1 << 28, left - 1000)
        _, s = omt.generate(op, s, step)
        left -= step
    tail, s = omt.generate(op, s, 1000)
    np.testing.assert_array_equal(out[big - 1000:].cpu().numpy().view(np.uint32), tail)
    np.testing.assert_array_equal(mtgp.mtgp_mt_get_statuses(mt)[0], s)
    del out


@pytest.mark.parametrize("name", ["mt19937", "p3217", "p521"])
def test_zero_state_is_a_fixed_point(name):
    mp, op = _set(name)
    mt = mtgp.mtgp_mt_init(mp, np.arange(3, dtype=np.uint32))
    mtgp.mtgp_mt_set_statuses(mt, np.zeros((3, op.n), np.uint32))
    expect = {mtgp.MTGP_U32: 0, mtgp.MTGP_F32_12: 0x3F800000, mtgp.MTGP_F32_01: 0}
    counts = np.array([5000, 1, op.n * 3 + 7], np.uint64)
    for fmt in FMTS:
        out = torch.full((int(counts.sum()),), -1, dtype=torch.int32, device="cuda")
        mtgp.mtgp_mt_generate(mt, [0, 1, 2], counts, fmt, out)
        assert np.all(out.cpu().numpy().view(np.uint32) == expect[fmt]), fmt
    assert not mtgp.mtgp_mt_get_statuses(mt).any()


@pytest.mark.parametrize("p", [521, 3217, 19937])
def test_forty_parameter_seeds(p):
    """Forty seed-generated original-MT sets per exponent against the oracle."""
    for pseed in range(100, 140):
        mp, op = mtgp.mtgp_mt_params_generate(p, pseed), omt.params_generate(p, pseed)
        assert mp.as_dict() == op.as_dict()
        mt, got, ref, ref_states = _run(mp, op, np.array([pseed, 7, 8], np.uint32), [0, 1, 2, 0],
                                        [op.n * 5 + 3, 4097, 1, 333], mtgp.MTGP_U32)
        np.testing.assert_array_equal(got, ref, err_msg="p %d seed %d" % (p, pseed))
        np.testing.assert_array_equal(mtgp.mtgp_mt_get_statuses(mt), ref_states)

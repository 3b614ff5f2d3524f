"""Jump-ahead (mtgp_jump) and its polynomial (mtgp_params_minpoly).

The jump must leave exactly the state that generating and discarding J
numbers leaves in the oracle.  The polynomial is checked on the CPU against
word sequences produced by the oracle (not by the library's own host
recursion): it must annihilate the transition, XOR over its set bits k of
x_{k+j} = 0 for j = 1..N.
"""
import numpy as np
import pytest

import oracle
from paper_1501_07701_gb300 import mtgp, workloads

torch = pytest.importorskip("torch")


def _words(op, state, count):
    """x_0 .. x_{N+count-1} from the oracle: after N outputs the oracle's
    state is the next N words of the sequence."""
    out = [np.asarray(state, np.uint32)]
    s = np.asarray(state, np.uint32).copy()
    n = op.n
    for _ in range((count + n - 1) // n):
        _, s = oracle.generate(op, s, n)
        out.append(s.copy())
    return np.concatenate(out)[:n + count]


@pytest.mark.parametrize("mexp,seed", [(11213, workloads.PARAM_SEED), (11213, 1), (11213, 3), (9689, 5),
                                       (23209, workloads.PARAM_SEED)])
def test_minpoly_annihilates_oracle_sequences(mexp, seed):
    mtgp.load_library()
    gp = mtgp.mtgp_params_generate(mexp, seed)
    op = oracle.params_generate(mexp, seed)
    mu = mtgp.mtgp_params_minpoly(gp)
    d = mu.size - 1
    assert mu[d] == 1 and d <= mexp
    ks = np.nonzero(mu)[0]
    rng = np.random.default_rng(seed)
    for trial in range(2):
        st = rng.integers(0, 2 ** 32, op.n, dtype=np.uint64).astype(np.uint32)
        x = _words(op, st, d + 2)
        for j in range(1, op.n + 1):
            assert np.bitwise_xor.reduce(x[ks + j]) == 0, "j = %d" % j
    # a proper divisor that drops a factor must fail (the check is not vacuous)
    if d > 1:
        short = ks[ks < d]
        x = _words(op, rng.integers(0, 2 ** 32, op.n, dtype=np.uint64).astype(np.uint32), d + 2)
        assert any(np.bitwise_xor.reduce(x[short + j]) != 0 for j in range(1, op.n + 1))


def test_bench_parameter_sets_have_full_degree():
    """The seed-generated sets the benchmarks use have a jump polynomial of
    degree Mexp with a non-zero constant term (an invertible transition)."""
    mtgp.load_library()
    for mexp in (11213, 23209, 44497):
        mu = mtgp.mtgp_params_minpoly(mtgp.mtgp_params_generate(mexp, workloads.PARAM_SEED))
        assert mu.size - 1 == mexp and mu[0] == 1


# ---------------------------------------------------------------------------
# GPU
# ---------------------------------------------------------------------------
gpu = pytest.mark.gpu


@pytest.fixture(scope="module")
def _cuda():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1501_07701_gb300 import build
    build.build()
    mtgp.load_library()


def _check_after_jump(st, op_of, states0, ids, jumps, more=3000):
    """States after the jump equal the oracle's after generating; the next
    `more` outputs agree as well."""
    got = mtgp.mtgp_get_statuses(st)
    expect = states0.copy()
    for s, j in zip(ids, jumps):
        _, expect[s] = oracle.generate(op_of(s), expect[s], int(j))
    np.testing.assert_array_equal(got, expect)
    n_streams = states0.shape[0]
    out = torch.empty(n_streams * more, dtype=torch.int32, device="cuda")
    mtgp.mtgp_generate_u32(st, np.arange(n_streams), np.full(n_streams, more), out)
    torch.cuda.synchronize()
    dev = out.cpu().numpy().view(np.uint32).reshape(n_streams, more)
    for s in range(n_streams):
        ref, _ = oracle.generate(op_of(s), expect[s], more)
        np.testing.assert_array_equal(dev[s], ref, err_msg="stream %d" % s)


@gpu
@pytest.mark.parametrize("mexp,seed", [(11213, workloads.PARAM_SEED), (11213, 1), (23209, workloads.PARAM_SEED),
                                       (44497, workloads.PARAM_SEED)])
def test_jump_equals_generating(_cuda, mexp, seed):
    gp = mtgp.mtgp_params_generate(mexp, seed)
    op = oracle.params_generate(mexp, seed)
    n = op.n
    jumps = [1, 2, 3, n - 1, n, n + 1, 1000, 99991, 1000003, 10 ** 7 + 7]
    st = mtgp.mtgp_init_statuses(gp, np.arange(len(jumps), dtype=np.uint32) + 17)
    states0 = mtgp.mtgp_get_statuses(st)
    ids = np.arange(len(jumps), dtype=np.uint32)
    mtgp.mtgp_jump(st, ids, jumps)
    _check_after_jump(st, lambda s: op, states0, ids, jumps)


@gpu
def test_jumps_compose(_cuda):
    """Jumping a then b equals jumping a + b, for lengths far beyond what the
    oracle could generate; duplicate ids in one call add up; zero is a no-op."""
    gp = mtgp.mtgp_params_generate(11213, workloads.PARAM_SEED)
    a, b = (1 << 40) + 12345, (1 << 50) + 3
    s1 = mtgp.mtgp_init_statuses(gp, np.arange(4, dtype=np.uint32))
    s2 = mtgp.mtgp_init_statuses(gp, np.arange(4, dtype=np.uint32))
    mtgp.mtgp_jump(s1, [0, 1, 2], [a, a, 0])
    mtgp.mtgp_jump(s1, [0, 1], [b, b])
    mtgp.mtgp_jump(s2, [0, 1, 1, 3], [a + b, a, b, 0])
    g1, g2 = mtgp.mtgp_get_statuses(s1), mtgp.mtgp_get_statuses(s2)
    np.testing.assert_array_equal(g1, g2)
    np.testing.assert_array_equal(g1[2], mtgp.mtgp_get_statuses(mtgp.mtgp_init_statuses(gp, np.arange(4, dtype=np.uint32)))[2])


@gpu
def test_jump_with_per_stream_sets(_cuda):
    seeds = [41, workloads.PARAM_SEED, 3]
    gps = [mtgp.mtgp_params_generate(11213, s) for s in seeds]
    ops = [oracle.params_generate(11213, s) for s in seeds]
    set_of = np.array([0, 1, 2, 1, 0, 2], np.uint32)
    st = mtgp.mtgp_init_statuses_multi(gps, set_of, np.arange(6, dtype=np.uint32) * 5)
    states0 = mtgp.mtgp_get_statuses(st)
    ids = np.arange(6, dtype=np.uint32)
    jumps = [5, 123456, 351, 7777777, 1, 2000001]
    mtgp.mtgp_jump(st, ids, jumps)
    _check_after_jump(st, lambda s: ops[set_of[s]], states0, ids, jumps)


@gpu
@pytest.mark.parametrize("n", [5, 17, 64])
def test_jump_toy_state_sizes(_cuda, tmp_path, n):
    """Small N (steps of min(32, N - pos) words in the expansion)."""
    rng = np.random.default_rng(300 + n)
    f = workloads.toy_fields(rng, n)
    path = tmp_path / "toy.txt"
    path.write_text("\n".join(["mexp %d" % f["mexp"], "pos %d" % f["pos"], "sh1 %d" % f["sh1"],
                               "sh2 %d" % f["sh2"],
                               "rec_basis " + " ".join(hex(v) for v in f["rec_basis"]),
                               "tmp_basis " + " ".join(hex(v) for v in f["tmp_basis"])]) + "\n")
    gp = mtgp.mtgp_params_load(str(path))
    op = oracle.params_from_fields(f["mexp"], f["pos"], f["sh1"], f["sh2"], f["rec_basis"], f["tmp_basis"])
    st = mtgp.mtgp_init_statuses(gp, np.arange(5, dtype=np.uint32))
    mtgp.mtgp_set_statuses(st, workloads.random_states(rng, 5, n))
    states0 = mtgp.mtgp_get_statuses(st)
    ids = np.arange(5, dtype=np.uint32)
    jumps = [1, n, 3 * n + 1, 100000, 999]
    mtgp.mtgp_jump(st, ids, jumps)
    _check_after_jump(st, lambda s: op, states0, ids, jumps, more=500)


@gpu
def test_jump_errors(_cuda):
    gp = mtgp.mtgp_params_generate(11213, 1)
    st = mtgp.mtgp_init_statuses(gp, np.arange(2, dtype=np.uint32))
    with pytest.raises(mtgp.MtgpError):
        mtgp.mtgp_jump(st, [2], [5])
    with pytest.raises(mtgp.MtgpError):
        mtgp.mtgp_jump(st, [0, 0], [2 ** 63, 2 ** 63])


# ---------------------------------------------------------------------------
# Period check (Rabin's test on the device) against the distinct-degree
# criterion on the host: mu is irreducible iff gcd(mu, t^(2^k) - t) = 1 for
# every k <= deg/2 (polynomials as Python integers, bit i = coefficient t^i).
# ---------------------------------------------------------------------------
def _clmul(a, b):
    r = 0
    while b:
        if b & 1:
            r ^= a
        a <<= 1
        b >>= 1
    return r


def _pmod(a, m):
    dm = m.bit_length() - 1
    while a.bit_length() - 1 >= dm:
        a ^= m << (a.bit_length() - 1 - dm)
    return a


def _pgcd(a, b):
    while b:
        a, b = b, _pmod(a, b)
    return a


def _irreducible_ddf(mu_bits):
    mu = sum(1 << i for i, b in enumerate(mu_bits) if b)
    d = mu.bit_length() - 1
    x = 2
    for _ in range(d // 2):
        x = _pmod(_clmul(x, x), mu)
        if _pgcd(mu, x ^ 2) != 1:
            return False
    return d >= 1


def _toy_params(tmp_path, mexp, pos, sh1, sh2, rb, tb):
    path = tmp_path / ("toy%d_%d_%d.txt" % (mexp, pos, sh1))
    path.write_text("mexp %d\npos %d\nsh1 %d\nsh2 %d\nrec_basis %s\ntmp_basis %s\n" % (
        mexp, pos, sh1, sh2, " ".join(map(hex, rb)), " ".join(map(hex, tb))))
    return mtgp.mtgp_params_load(str(path))


# toy sets (Mexp 107 and 127, Mersenne exponents) whose polynomial is
# irreducible of degree Mexp, i.e. of period 2^Mexp - 1
FULL_PERIOD_TOYS = [
    (107, 1, 19, 8, [4082844636, 2674313637, 2742504081, 3367881795], [530185877, 191712196, 1837422121, 2252332600]),
    (107, 3, 7, 6, [3055337368, 4127762061, 938604234, 606372027], [2423534270, 1784284154, 1040217680, 2742214121]),
    (127, 3, 24, 5, [3594327011, 1983446878, 1706042657, 4053708494], [1110286991, 448702083, 1960614134, 1319519321]),
]


@gpu
def test_period_check_full_period_toys(_cuda, tmp_path):
    for mexp, pos, sh1, sh2, rb, tb in FULL_PERIOD_TOYS:
        gp = _toy_params(tmp_path, mexp, pos, sh1, sh2, rb, tb)
        mu = mtgp.mtgp_params_minpoly(gp)
        assert mu.size - 1 == mexp and _irreducible_ddf(mu)
        assert mtgp.mtgp_params_period_check(gp)


@gpu
@pytest.mark.parametrize("mexp,n", [(61, 2), (89, 3), (107, 4), (127, 4), (100, 4), (119, 4)])
def test_period_check_agrees_with_ddf(_cuda, tmp_path, mexp, n):
    """Random toy sets (mostly reducible); 100 and 119 are composite, which
    exercises the gcd part of Rabin's test."""
    rng = np.random.default_rng(1000 + mexp)
    for _ in range(12):
        args = (mexp, int(rng.integers(1, n)), int(rng.integers(1, 32)), int(rng.integers(1, 32)),
                [int(v) for v in rng.integers(0, 2 ** 32, 4, dtype=np.uint64)],
                [int(v) for v in rng.integers(0, 2 ** 32, 4, dtype=np.uint64)])
        gp = _toy_params(tmp_path, *args)
        mu = mtgp.mtgp_params_minpoly(gp)
        expect = mu.size - 1 == mexp and _irreducible_ddf(mu)
        assert mtgp.mtgp_params_period_check(gp) == expect, args


@gpu
def test_period_check_of_benchmark_sets(_cuda):
    """Records the verdict for the benchmark parameter sets (no independent
    check exists at this size; the toys above pin the implementation)."""
    for mexp in (11213, 23209, 44497):
        verdict = mtgp.mtgp_params_period_check(mtgp.mtgp_params_generate(mexp, workloads.PARAM_SEED))
        print("Mexp %d seed 0x5EED: full period %s" % (mexp, verdict))
        assert verdict in (True, False)


# ---------------------------------------------------------------------------
# The original MT (comparison generator of Sec. 5.3): the same polynomial and
# period check, pinned at full size by MT19937's published characteristic
# polynomial.
# ---------------------------------------------------------------------------
def _mt_words(oq, state, count):
    import oracle.mt as omt
    out = [np.asarray(state, np.uint32)]
    s = np.asarray(state, np.uint32).copy()
    for _ in range((count + oq.n - 1) // oq.n):
        _, s = omt.generate(oq, s, oq.n)
        out.append(s.copy())
    return np.concatenate(out)[:oq.n + count]


def _mt_pair(p, seed):
    import oracle.mt as omt
    if p == 19937:
        return mtgp.mtgp_mt_params_mt19937(), omt.params_mt19937()
    return mtgp.mtgp_mt_params_generate(p, seed), omt.params_generate(p, seed)


def test_mt19937_polynomial_is_the_published_one():
    """MT19937's characteristic polynomial has degree 19937 and 135 nonzero
    coefficients (Panneton, L'Ecuyer and Matsumoto, ACM TOMS 32(1), 2006,
    which lists N1 = 135 for MT19937), and a nonzero constant term."""
    mtgp.load_library()
    mu = mtgp.mtgp_mt_params_minpoly(mtgp.mtgp_mt_params_mt19937())
    assert mu.size - 1 == 19937 and mu[0] == 1 and int(mu.sum()) == 135


@pytest.mark.parametrize("p,seed", [(19937, 0), (3217, workloads.PARAM_SEED), (3217, 7), (521, 3)])
def test_mt_minpoly_annihilates_oracle_sequences(p, seed):
    mtgp.load_library()
    mq, oq = _mt_pair(p, seed)
    mu = mtgp.mtgp_mt_params_minpoly(mq)
    d = mu.size - 1
    assert mu[d] == 1 and d <= p
    ks = np.nonzero(mu)[0]
    rng = np.random.default_rng(seed + p)
    st = rng.integers(0, 2 ** 32, oq.n, dtype=np.uint64).astype(np.uint32)
    x = _mt_words(oq, st, d + 2)
    for j in range(1, oq.n + 1):
        assert np.bitwise_xor.reduce(x[ks + j]) == 0, "j = %d" % j
    short = ks[ks < d]
    assert any(np.bitwise_xor.reduce(x[short + j]) != 0 for j in range(1, oq.n + 1))


@gpu
def test_mt19937_period_check_is_positive(_cuda):
    """The 1998 paper proves period 2^19937 - 1 for MT19937: a full-size
    known positive for the device's Rabin test."""
    assert mtgp.mtgp_mt_params_period_check(mtgp.mtgp_mt_params_mt19937())


@gpu
@pytest.mark.parametrize("p,n", [(61, 2), (89, 3), (107, 4), (127, 4), (100, 4)])
def test_mt_period_check_agrees_with_ddf(_cuda, p, n):
    """Toy MT sets with random a, m and tempering (the tempering does not
    enter the polynomial); at least one full-period set per Mersenne exponent
    is searched for, so both verdicts are exercised."""
    import oracle.mt as omt
    rng = np.random.default_rng(2000 + p)
    seen = set()
    for trial in range(400):
        f = dict(p=p, n=n, r=32 * n - p, m=int(rng.integers(1, n)),
                 a=int(rng.integers(0, 2 ** 32)) | 0x80000000, u=11, s=7, t=15, l=18,
                 b=0x9D2C5680, c=0xEFC60000)
        q = mtgp.MtParams(*[f[k] for k, _ in mtgp.MtParams._fields_])
        mu = mtgp.mtgp_mt_params_minpoly(q)
        expect = mu.size - 1 == p and _irreducible_ddf(mu)
        got = mtgp.mtgp_mt_params_period_check(q)
        assert got == expect, f
        seen.add(got)
        if trial >= 12 and (True in seen or p == 100):
            break
    assert True in seen or p == 100    # 100 is composite: no irreducible degree-100 mu is needed
    assert omt.params_from_fields(**f).n == n

"""Pins of the CPU oracle to facts that do not come from the oracle itself.

Each test names the property it checks and where it comes from:
* a hand-worked example (tests/golden/hand_example_n3.txt);
* a bit-level GF(2) matrix statement of the generator, built from what each
  word operation does to individual bits;
* impulse responses that fix the word offsets i, i+1, i+pos, i+pos-1;
* GF(2) linearity on states, the zero state, the dropped low bits of word i;
* linear complexity (Berlekamp-Massey) <= Mexp, the state's dimension;
* the seeding recurrence against NumPy's MT19937 integer seeding;
* float outputs against their exact real values;
* block-parallel windows of up to N - pos words (Sec. 2's per-block
  parallelism) against the sequential order, and chunked generation.
All CPU-only.
"""
import os

import numpy as np
import pytest

import oracle
from paper_1501_07701_gb300 import workloads
from tests.conftest import read_golden

MASK32 = 0xFFFFFFFF


def _cfg1_params():
    return oracle.params_generate(workloads.MEXP_MAIN, workloads.PARAM_SEED)


# --------------------------------------------------------------------------
# Hand-worked example
# --------------------------------------------------------------------------
def test_hand_worked_example(golden_dir):
    g = read_golden(os.path.join(golden_dir, "hand_example_n3.txt"))
    p = oracle.params_from_fields(g["mexp"][0], g["pos"][0], g["sh1"][0], g["sh2"][0],
                                  g["rec_basis"], g["tmp_basis"])
    assert p.n == 3 and p.mask == 0xFFFF0000
    st = np.array(g["state"], np.uint32)
    out, st2 = oracle.generate(p, st, 3)
    assert [int(v) for v in out] == g["u32"]
    assert [int(v) for v in st2] == g["state_after"]
    f, _ = oracle.generate(p, st, 1, oracle.F32_12)
    assert int(f[0]) == g["f32_12_first"][0]


# --------------------------------------------------------------------------
# Bit-level GF(2) formulation
# --------------------------------------------------------------------------
def _bits(w):
    return np.array([(int(w) >> j) & 1 for j in range(32)], np.uint8)


def _word(b):
    return int(sum(int(b[j]) << j for j in range(32)))


def _shift_up(s):      # output bit j takes input bit j - s  (word << s)
    m = np.zeros((32, 32), np.uint8)
    for j in range(s, 32):
        m[j, j - s] = 1
    return m


def _shift_down(s):    # output bit j takes input bit j + s  (word >> s)
    m = np.zeros((32, 32), np.uint8)
    for j in range(0, 32 - s):
        m[j, j + s] = 1
    return m


def _table_matrix(basis):
    """Linear map 'low four bits select an XOR of basis words'."""
    m = np.zeros((32, 32), np.uint8)
    for b in range(4):
        m[:, b] = _bits(basis[b])
    return m


def _mm(a, b):
    return (a.astype(np.int64) @ b.astype(np.int64) % 2).astype(np.uint8)


def _bitmatrix_stream(f, state, count):
    """The generator as 32x32 GF(2) matrices acting on bit vectors."""
    I = np.eye(32, dtype=np.uint8)
    D = np.diag(_bits(f["mask"]))
    Tr = _table_matrix(f["rec_basis"])
    Tt = _table_matrix(f["tmp_basis"])
    post = (I + Tr) % 2                                   # z -> z ^ REC[z & 15]
    A1 = _mm(post, (I + _shift_up(f["sh1"])) % 2)         # coefficient of x_{i+1}
    A0 = _mm(A1, D)                                       # coefficient of x_i
    Ap = _mm(post, _shift_down(f["sh2"]))                 # coefficient of x_{i+pos}
    fold = _mm((I + _shift_down(8)) % 2, (I + _shift_down(16)) % 2)
    Bq = _mm(Tt, fold)                                    # tempering from x_{i+pos-1}
    n, pos = f["n"], f["pos"]
    x = [_bits(w) for w in state]
    out = []
    for i in range(count):
        new = (_mm(A0, x[i][:, None]) + _mm(A1, x[i + 1][:, None])
               + _mm(Ap, x[i + pos][:, None])) % 2
        new = new[:, 0]
        x.append(new)
        o = (new + _mm(Bq, x[i + pos - 1][:, None])[:, 0]) % 2
        out.append(_word(o))
    return out


@pytest.mark.parametrize("n", [2, 3, 5])
def test_gf2_bit_matrix_toys(n):
    rng = np.random.default_rng(100 + n)
    for trial in range(4):
        f = workloads.toy_fields(rng, n)
        p = oracle.params_from_fields(f["mexp"], f["pos"], f["sh1"], f["sh2"],
                                      f["rec_basis"], f["tmp_basis"])
        f = dict(f, n=p.n, mask=p.mask)
        st = rng.integers(0, 1 << 32, size=n, dtype=np.uint64).astype(np.uint32)
        count = 2500
        ref = _bitmatrix_stream(f, [int(v) for v in st], count)
        out, _ = oracle.generate(p, st, count)
        assert [int(v) for v in out] == ref


def test_gf2_bit_matrix_cfg1_prefix():
    p = _cfg1_params()
    f = {"n": p.n, "pos": p.pos, "sh1": p.sh1, "sh2": p.sh2, "mask": p.mask,
         "rec_basis": list(p.rec_basis), "tmp_basis": list(p.tmp_basis)}
    st = oracle.init_state(p, 1)
    ref = _bitmatrix_stream(f, [int(v) for v in st], 400)
    out, _ = oracle.generate(p, st, 400)
    assert [int(v) for v in out] == ref


# --------------------------------------------------------------------------
# Word offsets: impulse responses
# --------------------------------------------------------------------------
def test_impulse_responses_fix_offsets():
    """Outputs 0 .. N-pos-1 depend only on the initial status.  Flipping bit 27
    of word j (kept by the mask, reaches the tempering index through the fold)
    must change exactly the outputs i with j in {i, i+1, i+pos-1, i+pos}."""
    p = _cfg1_params()
    n, pos = p.n, p.pos
    assert pos >= 3
    base = oracle.init_state(p, 1)
    m = n - pos
    o0, _ = oracle.generate(p, base, m)
    for j in range(n):
        st = base.copy()
        st[j] ^= np.uint32(1 << 27)
        o1, _ = oracle.generate(p, st, m)
        changed = set(np.nonzero(o0 != o1)[0].tolist())
        expect = {i for i in range(m) if j in (i, i + 1, i + pos - 1, i + pos)}
        assert changed == expect, j


# --------------------------------------------------------------------------
# Linearity, zero state, dropped bits
# --------------------------------------------------------------------------
def test_gf2_linearity_on_states():
    p = _cfg1_params()
    rng = np.random.default_rng(5)
    s1, s2 = workloads.random_states(rng, 2, p.n)
    c = 3 * p.n + 17
    a, _ = oracle.generate(p, s1, c)
    b, _ = oracle.generate(p, s2, c)
    ab, _ = oracle.generate(p, s1 ^ s2, c)
    assert np.array_equal(a ^ b, ab)
    fa, _ = oracle.generate(p, s1, c, oracle.F32_12)
    fb, _ = oracle.generate(p, s2, c, oracle.F32_12)
    fab, _ = oracle.generate(p, s1 ^ s2, c, oracle.F32_12)
    assert np.all((fa ^ fb ^ fab) == np.uint32(0x3F800000))


def test_zero_status():
    p = _cfg1_params()
    z = np.zeros(p.n, np.uint32)
    for fmt, val in [(oracle.U32, 0), (oracle.F32_12, 0x3F800000), (oracle.F32_01, 0)]:
        out, st = oracle.generate(p, z, 2 * p.n, fmt)
        assert np.all(out == np.uint32(val))
        assert not st.any()


def test_dropped_low_bits_of_oldest_word():
    """r = 32N - Mexp low bits of x_0 never reach any output; bit r does."""
    p = _cfg1_params()
    r = 32 * p.n - p.mexp
    assert r == 19 and p.mask == (MASK32 << r) & MASK32
    base = oracle.init_state(p, 9)
    c = 3 * p.n
    o0, _ = oracle.generate(p, base, c)
    for b in range(r):
        st = base.copy()
        st[0] ^= np.uint32(1 << b)
        o1, _ = oracle.generate(p, st, c)
        assert np.array_equal(o0, o1), b
    st = base.copy()
    st[0] ^= np.uint32(1 << r)
    o1, _ = oracle.generate(p, st, c)
    assert o1[0] != o0[0]


# --------------------------------------------------------------------------
# Linear complexity (state dimension = Mexp)
# --------------------------------------------------------------------------
def berlekamp_massey(s):
    """Shortest LFSR (length L, connection polynomial C) generating bits s."""
    s = np.asarray(s, np.uint8)
    n = s.size
    C = np.zeros(n + 1, np.uint8)
    B = np.zeros(n + 1, np.uint8)
    C[0] = B[0] = 1
    L, m = 0, 1
    for i in range(n):
        if L:
            d = (int(s[i]) + int(np.count_nonzero(C[1:L + 1] & s[i - L:i][::-1]))) & 1
        else:
            d = int(s[i])
        if d == 0:
            m += 1
            continue
        if 2 * L <= i:
            T = C.copy()
            C[m:] ^= B[:n + 1 - m]
            L, B, m = i + 1 - L, T, 1
        else:
            C[m:] ^= B[:n + 1 - m]
            m += 1
    return L, C[:L + 1].copy()


def _predicts(C, L, s, start, stop):
    for i in range(start, stop):
        if (int(np.count_nonzero(C[1:L + 1] & s[i - L:i][::-1])) & 1) != int(s[i]):
            return False
    return True


@pytest.mark.parametrize("bit", [0, 31])
def test_linear_complexity_cfg1(bit):
    p = _cfg1_params()
    n_fit = 2 * p.mexp + 64
    n_check = 10000
    out, _ = oracle.generate(p, oracle.init_state(p, 1), n_fit + n_check)
    s = ((out >> np.uint32(bit)) & np.uint32(1)).astype(np.uint8)
    L, C = berlekamp_massey(s[:n_fit])
    assert L <= p.mexp
    assert L > p.mexp - 64          # no accidental low-dimensional collapse
    assert _predicts(C, L, s, n_fit, n_fit + n_check)


def test_linear_complexity_toy_mask_matters():
    """The toy's complexity stays <= Mexp with the mask, and exceeds it once the
    mask is widened to all 32 bits (state dimension 32N)."""
    f = {"mexp": 80, "pos": 1, "sh1": 7, "sh2": 5,
         "rec_basis": [0x9E3779B9, 0x7F4A7C15, 0xF39CC060, 0x5CEDC834],
         "tmp_basis": [0x2545F491, 0x4F6CDD1D, 0x1B873593, 0xCC9E2D51]}
    p = oracle.params_from_fields(**f)
    q = oracle.params_from_fields(**f, mask=MASK32)
    st = oracle.init_state(p, 3)
    for par, bound_ok in [(p, True), (q, False)]:
        out, _ = oracle.generate(par, st, 600)
        s = (out & np.uint32(1)).astype(np.uint8)
        L, C = berlekamp_massey(s[:400])
        assert _predicts(C, L, s, 400, 600)
        assert (L <= 80) == bound_ok, L


# --------------------------------------------------------------------------
# Seed status
# --------------------------------------------------------------------------
@pytest.mark.parametrize("mexp", [11213, 23209, 44497])
@pytest.mark.parametrize("seed", [0, 1, 4095, 0xDEADBEEF])
def test_seed_status_matches_mt19937_integer_seeding(mexp, seed):
    p = oracle.params_generate(mexp, workloads.PARAM_SEED)
    st = oracle.init_state(p, seed)
    key = np.random.RandomState(seed).get_state()[1]
    k = min(p.n, 624)
    assert np.array_equal(st[:k], key[:k].astype(np.uint32))


# --------------------------------------------------------------------------
# Float conversions: exact values
# --------------------------------------------------------------------------
def test_float_outputs_are_exact_values():
    p = _cfg1_params()
    st = oracle.init_state(p, 1)
    u, _ = oracle.generate(p, st, 50000, oracle.U32)
    f12, _ = oracle.generate(p, st, 50000, oracle.F32_12)
    f01, _ = oracle.generate(p, st, 50000, oracle.F32_01)
    k = (u >> np.uint32(9)).astype(np.float64)
    v12 = f12.view(np.float32).astype(np.float64)
    v01 = f01.view(np.float32).astype(np.float64)
    assert np.array_equal(v12, 1.0 + k * 2.0 ** -23)
    assert np.array_equal(v01, k * 2.0 ** -23)
    assert v01.min() >= 0.0 and v01.max() < 1.0
    assert v12.min() >= 1.0 and v12.max() < 2.0


# --------------------------------------------------------------------------
# Parameterized status
# --------------------------------------------------------------------------
def _splitmix64_stream(seed):
    s = seed & 0xFFFFFFFFFFFFFFFF
    M = 0xFFFFFFFFFFFFFFFF
    while True:
        s = (s + 0x9E3779B97F4A7C15) & M
        z = s
        z = ((z ^ (z >> 30)) * 0xBF58476D1CE4E5B9) & M
        z = ((z ^ (z >> 27)) * 0x94D049BB133111EB) & M
        yield z ^ (z >> 31)


def test_splitmix64_known_first_output():
    assert next(_splitmix64_stream(0)) == 0xE220A8397B1DCDAF


@pytest.mark.parametrize("mexp", [3217, 11213, 23209, 44497])
def test_params_generate_draws(mexp):
    g = _splitmix64_stream(workloads.PARAM_SEED)
    n = mexp // 32 + 1
    sh1 = 1 + next(g) % 31
    sh2 = 1 + next(g) % 31
    d = next(g)
    wmin = 1
    while wmin * 2 <= n - 2 and wmin < 256:
        wmin *= 2
    pos = 2 + d % (n - wmin - 1)
    rb = [next(g) >> 32 for _ in range(4)]
    tb = [next(g) >> 32 for _ in range(4)]
    p = oracle.params_generate(mexp, workloads.PARAM_SEED)
    assert (p.n, p.sh1, p.sh2, p.pos) == (n, sh1, sh2, pos)
    assert list(p.rec_basis) == rb and list(p.tmp_basis) == tb
    assert p.n - p.pos >= min(256, wmin)
    r = 32 * n - mexp
    assert p.mask == (MASK32 << r) & MASK32


def test_tables_are_linear_spans():
    p = _cfg1_params()
    for tbl, basis in [(p.rec_tbl, p.rec_basis), (p.tmp_tbl, p.tmp_basis)]:
        assert tbl[0] == 0
        for b in range(4):
            assert tbl[1 << b] == basis[b]
        for a in range(16):
            for c in range(16):
                assert tbl[a ^ c] == tbl[a] ^ tbl[c]


def test_state_sizes_for_paper_exponents():
    # N = floor(Mexp/32) + 1 (r = 32N - Mexp in 1..31); 3217 is the paper's
    # period of Sec. 4.1, 23209 that of Sec. 5.2.
    for mexp, n, r in [(3217, 101, 15), (11213, 351, 19), (23209, 726, 23), (44497, 1391, 15)]:
        p = oracle.params_generate(mexp, 1)
        assert p.n == n and 32 * p.n - p.mexp == r


# --------------------------------------------------------------------------
# Block-parallel windows and chunking
# --------------------------------------------------------------------------
def block_parallel_u32(p, state, count, W):
    """Sec. 2's per-block generation: W consecutive new words per step, all
    computed at once from words produced in earlier steps."""
    n, pos = p.n, p.pos
    rec = np.array(p.rec_tbl, np.uint32)
    tmp = np.array(p.tmp_tbl, np.uint32)
    x = np.zeros(n + count + W + 1, np.uint32)
    x[:n] = state
    out = np.empty(count, np.uint32)
    i0 = 0
    while i0 < count:
        w = min(W, count - i0)
        y = (x[i0:i0 + w] & np.uint32(p.mask)) ^ x[i0 + 1:i0 + 1 + w]
        y ^= y << np.uint32(p.sh1)
        y ^= x[i0 + pos:i0 + pos + w] >> np.uint32(p.sh2)
        new = y ^ rec[y & np.uint32(15)]
        t = x[i0 + pos - 1:i0 + pos - 1 + w].copy()
        t ^= t >> np.uint32(16)
        t ^= t >> np.uint32(8)
        x[i0 + n:i0 + n + w] = new
        out[i0:i0 + w] = new ^ tmp[t & np.uint32(15)]
        i0 += w
    return out, x[count:count + n].copy()


def test_window_invariance():
    p = _cfg1_params()
    st = oracle.init_state(p, 77)
    count = 5 * p.n + 123
    ref, ref_st = oracle.generate(p, st, count)
    for W in [1, 7, 32, 256, p.n - p.pos]:
        out, s2 = block_parallel_u32(p, st, count, W)
        assert np.array_equal(out, ref), W
        assert np.array_equal(s2, ref_st), W
    out, _ = block_parallel_u32(p, st, count, p.n - p.pos + 1)
    assert not np.array_equal(out, ref)


def test_chunking_invariance():
    p = _cfg1_params()
    rng = np.random.default_rng(8)
    st = oracle.init_state(p, 5)
    total = 4 * p.n + 999
    ref, ref_st = oracle.generate(p, st, total)
    for _ in range(5):
        cuts = np.sort(rng.integers(0, total, size=4))
        parts = np.diff(np.concatenate([[0], cuts, [total]]))
        s = st.copy()
        got = []
        for c in parts:
            o, s = oracle.generate(p, s, int(c))
            got.append(o)
        assert np.array_equal(np.concatenate(got), ref)
        assert np.array_equal(s, ref_st)


def test_generate_many_matches_per_stream_order():
    p = _cfg1_params()
    rng = np.random.default_rng(9)
    n_streams = 6
    states = workloads.random_states(rng, n_streams, p.n)
    ids = np.array([0, 3, 0, 5, 3, 3, 1], np.uint32)
    counts = np.array([10, 700, 0, 351, 1, 5000, 64], np.uint64)
    for threads in (1, 3):
        out, st = oracle.generate_many(p, states, ids, counts, oracle.U32, threads)
        exp_states = states.copy()
        off = 0
        for sid, c in zip(ids, counts):
            o, exp_states[sid] = oracle.generate(p, exp_states[sid], int(c))
            assert np.array_equal(out[off:off + int(c)], o)
            off += int(c)
        assert np.array_equal(st, exp_states)

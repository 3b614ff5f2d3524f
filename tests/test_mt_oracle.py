"""Pins of the original-MT oracle, the comparison generator of Sec. 5.3.

The 1998 parameter set is pinned against two independent implementations
(NumPy's MT19937 and the C++ standard library's std::mt19937) and against
the value the C++ standard itself fixes.  General parameter sets, in
particular the separation point r != 31 that the 2^3217 generator of the
paper needs, are pinned by a GF(2) matrix formulation written from the
definition, by linearity, by the dropped low bits of x_0 and by the linear
complexity of an output bit.
"""
import shutil
import subprocess

import numpy as np
import pytest

import oracle.mt as mt
from tests.test_oracle_pins import (_bits, _mm, _shift_down, _shift_up, _splitmix64_stream, _word,
                                    berlekamp_massey)


def _numpy_raw(seed, count):
    """NumPy's legacy-seeded MT19937 (its own C implementation)."""
    return np.random.RandomState(seed)._bit_generator.random_raw(count).astype(np.uint32)


@pytest.mark.parametrize("seed", [0, 1, 5489, 4357, 0xFFFFFFFF])
def test_mt19937_equals_numpy(seed):
    q = mt.params_mt19937()
    out, _ = mt.generate(q, mt.init_state(q, seed), 5000)
    np.testing.assert_array_equal(out, _numpy_raw(seed, 5000))


@pytest.mark.parametrize("seed", [0, 7, 123456789])
def test_seed_state_equals_numpy_key(seed):
    q = mt.params_mt19937()
    key = np.random.RandomState(seed).get_state()[1]
    np.testing.assert_array_equal(mt.init_state(q, seed), key.astype(np.uint32))


def test_mt19937_10000th_output_fixed_by_the_cpp_standard():
    # ISO/IEC 14882 [rand.predef]: the 10000th consecutive invocation of a
    # default-constructed std::mt19937 (seed 5489) produces 4123659995.
    q = mt.params_mt19937()
    out, _ = mt.generate(q, mt.init_state(q, 5489), 10000)
    assert int(out[9999]) == 4123659995


def test_mt19937_equals_cpp_std_library(tmp_path):
    gxx = shutil.which("g++")
    if not gxx:
        pytest.skip("no C++ compiler")
    src = tmp_path / "m.cpp"
    src.write_text("#include <random>\n#include <cstdio>\nint main(){std::mt19937 g(20240611u);"
                   "for(int i=0;i<3000;++i) std::printf(\"%u\\n\",(unsigned)g());}\n")
    exe = tmp_path / "m"
    subprocess.check_call([gxx, "-O1", "-o", str(exe), str(src)])
    ref = np.array([int(v) for v in subprocess.check_output([str(exe)]).split()], np.uint32)
    q = mt.params_mt19937()
    out, _ = mt.generate(q, mt.init_state(q, 20240611), 3000)
    np.testing.assert_array_equal(out, ref)


def test_chunking_and_state_continuation():
    q = mt.params_generate(3217, 11)
    s0 = mt.init_state(q, 3)
    whole, s_whole = mt.generate(q, s0, 5000)
    a, s1 = mt.generate(q, s0, 1)
    b, s2 = mt.generate(q, s1, 100)
    c, s3 = mt.generate(q, s2, 4899)
    np.testing.assert_array_equal(np.concatenate([a, b, c]), whole)
    np.testing.assert_array_equal(s3, s_whole)
    # the saved state is the last n words of the sequence x_0, x_1, ...
    _, s_n = mt.generate(q, s0, q.n)
    np.testing.assert_array_equal(mt.generate(q, s_n, 0)[1], s_n)


# --------------------------------------------------------------------------
# GF(2) matrix formulation on toy parameter sets
# --------------------------------------------------------------------------
def _matrix_stream(q, state, count):
    """The generator as 32x32 GF(2) matrices acting on bit vectors:
    x_{k+n} = x_{k+m} + A (D_u x_k + D_l x_{k+1}),  out = T x_{k+n}."""
    I = np.eye(32, dtype=np.uint8)
    upper = np.array([1 if j >= q["r"] else 0 for j in range(32)], np.uint8)
    Du, Dl = np.diag(upper), np.diag(1 - upper)
    A = _shift_down(1).copy()
    A[:, 0] ^= _bits(q["a"])                    # the bit shifted out adds row a
    Ak, Ak1 = _mm(A, Du), _mm(A, Dl)
    T = (I + _shift_down(q["u"])) % 2
    T = _mm((I + _mm(np.diag(_bits(q["b"])), _shift_up(q["s"]))) % 2, T)
    T = _mm((I + _mm(np.diag(_bits(q["c"])), _shift_up(q["t"]))) % 2, T)
    T = _mm((I + _shift_down(q["l"])) % 2, T)
    n, m = q["n"], q["m"]
    x = [_bits(w) for w in state]
    out = []
    for k in range(count):
        new = (x[k + m][:, None] + _mm(Ak, x[k][:, None]) + _mm(Ak1, x[k + 1][:, None])) % 2
        x.append(new[:, 0])
        out.append(_word(_mm(T, new)[:, 0]))
    return out


@pytest.mark.parametrize("n,r", [(2, 0), (2, 31), (3, 15), (5, 1), (5, 17)])
def test_matrix_formulation_toys(n, r):
    rng = np.random.default_rng(1000 * n + r)
    for trial in range(3):
        f = dict(p=32 * n - r, n=n, r=r, m=int(rng.integers(1, n)),
                 a=int(rng.integers(0, 2 ** 32)) | 0x80000000,
                 u=int(rng.integers(0, 32)), s=int(rng.integers(0, 32)),
                 t=int(rng.integers(0, 32)), l=int(rng.integers(0, 32)),
                 b=int(rng.integers(0, 2 ** 32)), c=int(rng.integers(0, 2 ** 32)))
        q = mt.params_from_fields(**f)
        st = rng.integers(0, 2 ** 32, n, dtype=np.uint64).astype(np.uint32)
        got, _ = mt.generate(q, st, 300)
        assert got.tolist() == _matrix_stream(f, st.tolist(), 300), (f, trial)


def test_matrix_formulation_mt19937_prefix():
    q = mt.params_mt19937()
    st = mt.init_state(q, 99)
    got, _ = mt.generate(q, st, 700)           # past one full pass over the 624 words
    assert got.tolist() == _matrix_stream(q.as_dict(), st.tolist(), 700)


# --------------------------------------------------------------------------
# Structure: linearity, dropped bits, linear complexity
# --------------------------------------------------------------------------
def test_linearity_on_states():
    q = mt.params_generate(3217, 5)
    rng = np.random.default_rng(8)
    s1 = rng.integers(0, 2 ** 32, q.n, dtype=np.uint64).astype(np.uint32)
    s2 = rng.integers(0, 2 ** 32, q.n, dtype=np.uint64).astype(np.uint32)
    o1, _ = mt.generate(q, s1, 3000)
    o2, _ = mt.generate(q, s2, 3000)
    o12, _ = mt.generate(q, s1 ^ s2, 3000)
    np.testing.assert_array_equal(o12, o1 ^ o2)
    z, zs = mt.generate(q, np.zeros(q.n, np.uint32), 1000)
    assert not z.any() and not zs.any()


def test_only_the_low_r_bits_of_x0_are_dropped():
    q = mt.params_generate(3217, 5)
    assert q.r == 15
    s = mt.init_state(q, 1)
    ref, _ = mt.generate(q, s, 4000)
    for bit in range(32):
        t = s.copy()
        t[0] ^= np.uint32(1 << bit)
        got, _ = mt.generate(q, t, 4000)
        assert np.array_equal(got, ref) == (bit < q.r), bit


@pytest.mark.parametrize("bit", [0, 31])
def test_linear_complexity_3217(bit):
    """The sequence lives in the p = 32n - r dimensional space of the state's
    used bits, so every output bit has linear complexity <= p."""
    q = mt.params_generate(3217, 5)
    out, _ = mt.generate(q, mt.init_state(q, 2), 2 * 3217 + 200)
    L, _ = berlekamp_massey((out >> np.uint32(bit)) & np.uint32(1))
    assert 3000 < L <= 3217


def test_linear_complexity_mt19937_is_exactly_p():
    """MT19937's characteristic polynomial is primitive of degree 19937, so a
    nonzero output bit sequence has linear complexity exactly 19937."""
    q = mt.params_mt19937()
    out, _ = mt.generate(q, mt.init_state(q, 5489), 2 * 19937 + 50)
    L, _ = berlekamp_massey(out & np.uint32(1))
    assert L == 19937


# --------------------------------------------------------------------------
# Parameter generation and formats
# --------------------------------------------------------------------------
@pytest.mark.parametrize("p,seed", [(521, 3), (3217, 0xC0FFEE), (3217, 7), (19937, 1), (44497, 3)])
def test_params_generate_draws(p, seed):
    g = _splitmix64_stream(seed)
    q = mt.params_generate(p, seed)
    n = -(-p // 32)
    assert (q.p, q.n, q.r, q.m) == (p, n, 32 * n - p, n // 2)
    assert q.a == (next(g) >> 32) | 0x80000000
    assert q.b == next(g) >> 32 and q.c == next(g) >> 32
    assert (q.u, q.s, q.t, q.l) == (12, 7, 15, 18)


def test_params_out_of_range():
    with pytest.raises(ValueError):
        mt.params_generate(32, 1)
    with pytest.raises(ValueError):
        mt.params_from_fields(p=3217, n=101, r=15, m=101, a=0x80000000)
    with pytest.raises(ValueError):
        mt.params_from_fields(p=3217, n=101, r=14, m=50, a=0x80000000)


def test_float_outputs_are_exact_values():
    q = mt.params_generate(3217, 9)
    s = mt.init_state(q, 4)
    u, _ = mt.generate(q, s, 4000, mt.U32)
    f12, _ = mt.generate(q, s, 4000, mt.F32_12)
    f01, _ = mt.generate(q, s, 4000, mt.F32_01)
    np.testing.assert_array_equal(f12, np.uint32(0x3F800000) | (u >> np.uint32(9)))
    k = (u >> np.uint32(9)).astype(np.float64)
    np.testing.assert_array_equal(f01.view(np.float32).astype(np.float64), k / 2.0 ** 23)


def test_generate_many_matches_per_stream_order():
    q = mt.params_generate(3217, 1)
    states = np.stack([mt.init_state(q, s) for s in range(6)])
    ids = np.array([3, 0, 3, 5, 0, 3], np.uint32)
    counts = np.array([100, 7, 0, 333, 1000, 65], np.uint64)
    for threads in (1, 3):
        out, st = mt.generate_many(q, states, ids, counts, mt.U32, threads)
        ref_st = states.copy()
        pieces = []
        for i, c in zip(ids, counts):
            o, ref_st[i] = mt.generate(q, ref_st[i], int(c))
            pieces.append(o)
        np.testing.assert_array_equal(out, np.concatenate(pieces))
        np.testing.assert_array_equal(st, ref_st)


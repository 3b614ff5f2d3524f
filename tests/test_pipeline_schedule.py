"""The software-pipelined step schedule of the register-resident kernel,
emulated on the CPU and checked against the oracle.

The kernel advances a stream in rows of N words; a step of W = 128 words
(4 groups of 32 columns) reads words i+1, i+pos and i+pos-1 from a shared row
S[0..N) followed by a mirror of its first columns, and writes the new words
back.  With N - pos >= 2W the kernel issues the loads of step s+1 *before*
the stores of step s (and the first step of the next row during the last step
of the current one).  This test replays exactly that order -- loads of the
next step, then arithmetic and stores of the current step -- with Python
lists standing in for the shared row and per-lane registers, and requires the
oracle's sequence (Sec. 2 recursion and tempering) for many parameter sets.
A negative control shows the schedule is wrong for N - pos < 256, i.e. the
check is sensitive to the ordering argument.

Short states (Mexp 3217, 4253: four or five column groups, no 128-word step
fits) are counted by the statistics kernel one 32-column sub-step at a time,
with the loads of the next sub-step issued before the stores of the current
one: the same schedule with W = 32, exact while N - pos >= 64.
"""
import numpy as np
import pytest

import oracle

M32 = 0xFFFFFFFF


def _emulate(p, state, n_rows, K=4, ahead=True):
    """K: column groups per step (W = 32 K words).  ahead: the next step's
    loads before the current step's stores; else after them."""
    N, pos = p.n, p.pos
    rec, tmp = list(p.rec_tbl), list(p.tmp_tbl)
    M = (N + 31) // 32                      # 32-column groups
    n_steps = (M + K - 1) // K
    mirror = 32 * ((pos + 31 + 31) // 32)   # mirrored columns after S[N)
    S = [0] * (N + mirror + 4)
    S[:N] = [int(x) for x in state]
    S[N:N + mirror] = S[:mirror]
    reg = [[S[32 * m + l] if 32 * m + l < N else 0 for l in range(32)] for m in range(M)]
    last_lane = (N - 1) & 31

    def load_step(s0):
        return {i: [(S[32 * (s0 + i) + l + 1], S[pos + 32 * (s0 + i) + l],
                     S[pos + 32 * (s0 + i) + l - 1]) for l in range(32)]
                for i in range(K) if s0 + i < M}

    cur = load_step(0)
    out = []
    for _ in range(n_rows):
        row = [None] * N
        for st in range(n_steps):
            s0 = st * K
            nxt_s0 = s0 + K if st + 1 < n_steps else 0
            if ahead:
                nxt = load_step(nxt_s0)             # before this step's stores
            new = {}
            for i, lanes in cur.items():
                m = s0 + i
                for l, (x1, xp, xq) in enumerate(lanes):
                    yy = ((reg[m][l] & p.mask) ^ x1) & M32
                    y = (yy ^ ((yy << p.sh1) & M32) ^ (xp >> p.sh2)) & M32
                    xn = y ^ rec[y & 15]
                    t = xq ^ (xq >> 16)
                    t ^= t >> 8
                    new[(m, l)] = (xn, xn ^ tmp[t & 15])
            for (m, l), (xn, o) in new.items():
                if m + 1 < M or l <= last_lane:
                    reg[m][l] = xn
                    S[32 * m + l] = xn
                    if 32 * m < mirror:
                        S[N + 32 * m + l] = xn
                    row[32 * m + l] = o
            cur = nxt if ahead else load_step(nxt_s0)
        out.extend(row)
    return np.array(out, np.uint32), np.array(S[:N], np.uint32)


def _case(mexp, pos, seed=5, n=0):
    base = oracle.params_generate(mexp, seed)
    return oracle.params_from_fields(mexp, pos, base.sh1, base.sh2, list(base.rec_basis),
                                     list(base.tmp_basis), n=n, mask=base.mask if n else 0)


def _cases():
    out = [oracle.params_generate(11213, 0x5EED), oracle.params_generate(9689, 2),
           oracle.params_generate(23209, 3)]
    for mexp in (11213, 23209):
        n = mexp // 32 + 1
        out += [_case(mexp, 1), _case(mexp, 2), _case(mexp, n - 256)]
    out.append(_case(23209, 727 - 256, n=727))
    return out


@pytest.mark.parametrize("p", _cases(), ids=lambda p: "mexp%d_n%d_pos%d" % (p.mexp, p.n, p.pos))
def test_pipelined_schedule_equals_sequential(p):
    assert p.n - p.pos >= 256
    state = oracle.init_state(p, 3)
    n_rows = 3
    ref, ref_state = oracle.generate(p, state, n_rows * p.n)
    got, got_row = _emulate(p, state, n_rows)
    np.testing.assert_array_equal(got, ref)
    # after whole rows the shared row is the state, oldest word first
    np.testing.assert_array_equal(got_row, ref_state)


@pytest.mark.parametrize("gap", [255, 200])
def test_schedule_breaks_below_the_bound(gap):
    """Negative control: with N - pos < 2W the early loads read words the
    current step has not written yet, and the emulation must disagree."""
    n = 11213 // 32 + 1
    p = _case(11213, n - gap)
    state = oracle.init_state(p, 3)
    ref, _ = oracle.generate(p, state, 3 * p.n)
    got, _ = _emulate(p, state, 3)
    assert not np.array_equal(got, ref)


def _short_cases():
    out = [oracle.params_generate(3217, seed) for seed in (0x5EED, 1, 2)]
    for mexp in (3217, 4253):
        n = mexp // 32 + 1
        out += [_case(mexp, 1), _case(mexp, 2), _case(mexp, n - 64)]
    return out


@pytest.mark.parametrize("p", _short_cases(), ids=lambda p: "mexp%d_n%d_pos%d" % (p.mexp, p.n, p.pos))
def test_short_state_lookahead_equals_sequential(p):
    """One 32-column sub-step per step, the next sub-step's loads before the
    current one's stores (the statistics kernel's short-state row loop)."""
    assert p.n - p.pos >= 64
    state = oracle.init_state(p, 4)
    ref, ref_state = oracle.generate(p, state, 4 * p.n)
    got, got_row = _emulate(p, state, 4, K=1)
    np.testing.assert_array_equal(got, ref)
    np.testing.assert_array_equal(got_row, ref_state)


@pytest.mark.parametrize("gap", [63, 40, 33])
def test_short_state_lookahead_breaks_below_the_bound(gap):
    """Negative control: with N - pos < 64 a look-ahead pick-up reads a word
    the current sub-step has not written yet; such sets take the kernel's
    read-then-write path instead."""
    p = _case(3217, 3217 // 32 + 1 - gap)
    state = oracle.init_state(p, 4)
    ref, _ = oracle.generate(p, state, 4 * p.n)
    got, _ = _emulate(p, state, 4, K=1)
    assert not np.array_equal(got, ref)


@pytest.mark.parametrize("gap,exact", [(32, True), (33, True), (63, True), (31, False), (20, False)])
def test_short_state_read_then_write_bound(gap, exact):
    """Sub-steps that load their words after the previous sub-step's stores
    (the statistics kernel's slow path) are exact while N - pos >= 32."""
    p = _case(3217, 3217 // 32 + 1 - gap)
    state = oracle.init_state(p, 4)
    ref, _ = oracle.generate(p, state, 4 * p.n)
    got, _ = _emulate(p, state, 4, K=1, ahead=False)
    assert np.array_equal(got, ref) == exact

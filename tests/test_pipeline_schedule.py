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
"""
import numpy as np
import pytest

import oracle

M32 = 0xFFFFFFFF


def _emulate(p, state, n_rows):
    N, pos = p.n, p.pos
    rec, tmp = list(p.rec_tbl), list(p.tmp_tbl)
    M = (N + 31) // 32                      # 32-column groups
    K = 4                                   # groups per step (W = 128)
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
            nxt = load_step(s0 + K if st + 1 < n_steps else 0)   # before this step's stores
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
            cur = nxt
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

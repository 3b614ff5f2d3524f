"""The piece-and-stitch decomposition of the fused statistics, emulated on the
CPU and checked against the oracle's whole-request counts.

In a split plan one request's numbers are cut into pieces that run on
different warps.  Each piece counts, 32 values at a time as a warp does (a
visit ballot, each visiting lane's gap to the nearest lower visiting lane or
to the run carried in; Hamming weights accumulated per lane until a block of
L/s values ends), everything that lies inside it.  Two things cross a piece's
start: the gap ending at its first visit, and the block pair open at its
position (mod 2 L/s) in the request.  The piece records the non-visits before
its first visit and after its last, whether it had a visit, and its weights in
the pair open at its start and at its end; a stitch then walks the pieces in
order and counts the crossing gaps and pairs.  Both are restated here, with
Python integers for the warp's lanes, and must give the oracle's gap
histogram (Knuth's gap test on one bit field) and Hamming pair table (the
weights of consecutive L-bit blocks, classed by the bounds) for arbitrary
cuts.  Blocks of at least 128 values are also updated per 128-value step, as
the kernel's full rows do: a step's positions from the block's end on belong
to the next block.  A negative control shows the stitch is needed.
"""
import numpy as np
import pytest

import oracle

NONE = 0xFFFFFFFF


def _hibit(x):
    return x.bit_length() - 1 if x else NONE


def _popc(x):
    return bin(x).count("1")


def _args(gap, hamming):
    (r, b, t), (rs, s, L, bounds) = gap, hamming
    return dict(gmask=((1 << b) - 1) << (32 - r - b), t=t,
                hmask=((1 << s) - 1) << (32 - rs - s), K=L // s,
                C=len(bounds) + 1, bounds=list(bounds))


def _class(w, A):
    return sum(1 for v in A["bounds"] if v <= w)


def _piece(x, off, A, hw=32):
    """Counts of one piece (values x at position off of its request) and its
    record for the stitch.  hw: values per Hamming update, 32 (per sub-step)
    or 128 (per 128-value step, for blocks of at least 128 values)."""
    assert hw == 32 or A["K"] >= hw
    K, C, t = A["K"], A["C"], A["t"]
    hist = [0] * (t + 1)
    tab = [0] * (C * C)
    phase = off % (2 * K)
    first_gap_open = off > 0            # the gap ending at the first visit began earlier
    pair_open = phase > 0               # the pair open at the start began earlier
    half = 1 if phase >= K else 0       # which block of the pair the next value is in
    rem = K - phase % K                 # values left in the current block
    run = 0                             # non-visits since the last visit
    acc = [0] * 32                      # per-lane weights of the current block
    wa = 0                              # weight of the pair's first block
    lead_run = 0
    lead_w = [0, 0]                     # weights in the pair open at the start

    def block_end(W):
        nonlocal pair_open, half, wa
        if pair_open:
            lead_w[half] = W
            if half:
                pair_open = False
        elif half:
            tab[_class(wa, A) * C + _class(W, A)] += 1
        wa = W
        half ^= 1

    for g0 in range(0, len(x), 32):
        n = min(32, len(x) - g0)
        o = [int(x[g0 + l]) for l in range(n)] + [0] * (32 - n)
        ballot = sum(1 << l for l in range(n) if o[l] & A["gmask"] == 0)
        counted = ballot
        if first_gap_open and ballot:
            f = _hibit(ballot & -ballot)
            lead_run = run + f
            counted &= ~(1 << f)
            first_gap_open = False
        for l in range(32):
            if counted >> l & 1:
                lower = _hibit(ballot & ((1 << l) - 1))
                g = l - lower - 1 if lower != NONE else l + run
                hist[min(g, t)] += 1
        run = n - 1 - _hibit(ballot) if ballot else run + n
    for g0 in range(0, len(x), hw):
        # a step ends at most one block (hw <= K): its positions >= rem
        # belong to the next block
        n = min(hw, len(x) - g0)
        w = [_popc(int(x[g0 + p]) & A["hmask"]) if p < n else 0 for p in range(hw)]
        if rem > n:
            acc = [a + sum(w[l::32]) for l, a in enumerate(acc)]
            rem -= n
        else:
            W = sum(acc) + sum(w[:rem])
            acc = [sum(w[p] for p in range(l, hw, 32) if p >= rem) for l in range(32)]
            block_end(W)
            rem += K - n
    part = sum(acc)
    rec = dict(visit=not first_gap_open, prefix=run if first_gap_open else lead_run, suffix=run)
    if pair_open:
        # the piece ends inside the pair it started in
        rec.update(la=lead_w[0] if half else part, lb=part if half else 0, ta=0, tb=0)
    else:
        rec.update(la=lead_w[0], lb=lead_w[1], ta=wa if half else part, tb=part if half else 0)
    return hist, tab, rec


def _stitch(pieces, recs, A, hist, tab):
    """Counts the gaps and block pairs that cross piece starts."""
    K, C, t = A["K"], A["C"], A["t"]
    run = recs[0]["suffix"]
    wa, wb = recs[0]["ta"], recs[0]["tb"]
    for (off, n), r in zip(pieces[1:], recs[1:]):
        if r["visit"]:
            hist[min(run + r["prefix"], t)] += 1
            run = r["suffix"]
        else:
            run += r["prefix"]
        phase = off % (2 * K)
        if phase == 0:
            wa, wb = r["ta"], r["tb"]
            continue
        wa += r["la"]
        wb += r["lb"]
        if n >= 2 * K - phase:          # the pair completes inside this piece
            tab[_class(wa, A) * C + _class(wb, A)] += 1
            wa, wb = r["ta"], r["tb"]


def _split_counts(x, cuts, A, stitch=True, hw=32):
    edges = [0] + sorted(cuts) + [len(x)]
    pieces = [(edges[i], edges[i + 1] - edges[i]) for i in range(len(edges) - 1)]
    hist = [0] * (A["t"] + 1)
    tab = [0] * (A["C"] ** 2)
    recs = []
    for off, n in pieces:
        h, tb, rec = _piece(x[off:off + n], off, A, hw)
        hist = [a + v for a, v in zip(hist, h)]
        tab = [a + v for a, v in zip(tab, tb)]
        recs.append(rec)
    if stitch:
        _stitch(pieces, recs, A, hist, tab)
    return np.array(hist, np.uint64), np.array(tab, np.uint64)


CASES = [
    ((25, 5, 128), (25, 5, 1200, [585, 600, 615])),          # the paper's tests 35 and 100
    ((0, 1, 7), (0, 1, 32, [])),                              # top bit, blocks of 32 values
    ((20, 10, 1023), (27, 5, 160, [10, 12, 14, 16, 18])),     # rare visits, long gaps
    ((31, 1, 1), (31, 1, 50, list(range(10, 40, 2))[:15])),  # bottom bit, t = 1, 15 bounds
    ((3, 4, 40), (3, 4, 512, [60, 64, 68])),
]


def _values(rng, n, case):
    x = rng.integers(0, 2**32, n, dtype=np.uint64).astype(np.uint32)
    if case == 2:   # bit 10 is inside the gap field: set it in half the values
        x[rng.random(n) < 0.5] |= np.uint32(1 << 10)
    return x


def _oracle_counts(x, gap, hamming):
    (r, b, t), (rs, s, L, bounds) = gap, hamming
    return (oracle.gap_histogram(x, r, b, t),
            oracle.hamming_pairs(x, rs, s, L, bounds).ravel())


# per-128-value-step updates only where a block holds at least 128 values
WIDTHS = [(c, 32) for c in range(len(CASES))] + \
         [(c, 128) for c, (_, h) in enumerate(CASES) if h[2] // h[1] >= 128]


@pytest.mark.parametrize("case,hw", WIDTHS)
def test_random_cuts_equal_whole_request(case, hw):
    gap, hamming = CASES[case]
    A = _args(gap, hamming)
    rng = np.random.default_rng(40 + case)
    for _ in range(5):
        n = int(rng.integers(1, 5000))
        x = _values(rng, n, case)
        k = int(rng.integers(0, 8))
        cuts = sorted(set(int(c) for c in rng.integers(1, n, k))) if n > 1 else []
        want_h, want_t = _oracle_counts(x, gap, hamming)
        h, tb = _split_counts(x, cuts, A, hw=hw)
        np.testing.assert_array_equal(h, want_h, err_msg="gap, cuts %s" % cuts)
        np.testing.assert_array_equal(tb, want_t, err_msg="Hamming, cuts %s" % cuts)


def test_cuts_at_block_edges_and_pairs_over_many_pieces():
    """Cuts at multiples of L/s and 2 L/s, one value off them, and pieces far
    shorter than a block, so that one pair spans many pieces; plus a stretch
    with no visit that spans whole pieces."""
    gap, hamming = CASES[0]
    A = _args(gap, hamming)
    K = A["K"]
    rng = np.random.default_rng(7)
    x = _values(rng, 12 * K + 17, 0)
    x[3 * K:7 * K] |= np.uint32(A["gmask"])     # no visits for 4 blocks
    want_h, want_t = _oracle_counts(x, gap, hamming)
    for cuts in ([K, 2 * K, 4 * K], [K - 1, K + 1, 2 * K - 1, 2 * K + 1],
                 list(range(5, 12 * K, 37)), [3 * K + 1, 4 * K, 5 * K + 3, 6 * K + 100],
                 list(range(1, 70))):
        for hw in (32, 128):
            h, tb = _split_counts(x, cuts, A, hw=hw)
            np.testing.assert_array_equal(h, want_h, err_msg="gap, cuts %s" % cuts[:8])
            np.testing.assert_array_equal(tb, want_t, err_msg="Hamming, %d, cuts %s" % (hw, cuts[:8]))


def test_pieces_without_the_stitch_miss_counts():
    """Negative control: summing the pieces' own counts loses the crossing
    gaps and pairs."""
    gap, hamming = CASES[0]
    A = _args(gap, hamming)
    rng = np.random.default_rng(11)
    x = _values(rng, 4000, 0)
    want_h, want_t = _oracle_counts(x, gap, hamming)
    h, tb = _split_counts(x, [700, 1500, 2333], A, stitch=False)
    assert h.sum() < want_h.sum() and tb.sum() < want_t.sum()

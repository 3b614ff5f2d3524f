// Generation with the data reductions of the paper's two failing BigCrush
// tests (Sec. 4.2) fused in: the gap test (test 35) and Hamming-weight
// independence (test 100) are accumulated from each sub-step's outputs
// while they are still in registers, so the output is not read back.
//
// The generator is mtgp_fast_kernel's single-warp, software-pipelined row
// loop (128-word steps, N - pos >= 256; see mtgp_fast.cuh), unchanged except
// that the outputs of every sub-step also feed the statistics.  A sequence
// of the statistics is one request of the launch (Segment::req): its values
// in generation order.  Each request belongs to one warp, which writes its
// histogram and table rows when the request ends.
//
// Gap test, per sub-step, over a run of lanes [l0, l0 + n) of one request:
// a value visits when (value & gmask) == 0; the visits form a ballot B.  A
// visiting lane's gap (non-visits since the previous visit) is its distance
// to the nearest lower visiting lane, or, when there is none, lane - l0 plus
// the carried count D of non-visits since the request's last visit (or its
// start: the first visit's gap counts too).  Lengths >= t are pooled in
// class t; a trailing run of non-visits is not a gap.  Each sub-step ends in
// one shared-memory reduction per lane (red.shared.add, no return): a
// visiting lane adds 1 to its class in the warp's histogram, the others to
// a slot of their own that is never read, so the reduction needs neither a
// predicate nor a branch.  In full rows the step's reductions are issued
// after the step's row stores and warp barrier, so that they do not delay
// them.
//
// Hamming test: the weights popc(value & hmask) of K = L/s consecutive
// values form a block; `rem` counts the values left in the current block,
// and each lane keeps its part of the block's weight.  A step that contains
// no block end (rem > values of the step) only adds the weights; a step that
// contains one splits its lanes at the end, reduces the finished block's
// weight across the warp and, on every second block, counts the pair
// (class of first, class of second) in the warp's shared-memory table.  The
// class of a weight is the number of bounds <= it: lane i holds bound i, and
// a ballot counts them.  An incomplete trailing pair is
// ignored.  K >= 128 keeps every 128-value step to at most one block end;
// smaller K take the per-sub-step form (K >= 32: at most one block end per
// sub-step).
//
// Split launches: a request may be cut into pieces (segments of different
// items) that different warps generate.  A piece that does not start its
// request leaves its first gap (whose start lies in an earlier piece) and
// the block pair open at its start uncounted; it records them, with its
// trailing run of non-visits and the weights of the pair open at its end,
// in one SegStat, and the stitch kernel completes them in request order.
// Until both are settled the piece's rows take the slow path, so the full
// rows' loop is the same as for unsplit launches.
//
// Short states (M < 9, e.g. Mexp 3217: N = 101, N - pos 64 .. 99) advance
// full rows one 32-column sub-step at a time (fused_rows_short, which reads a
// sub-step ahead while N - pos >= 64); the slow path reads each sub-step's
// words before writing them, which is exact while N - pos >= 32 (a wrapped
// pick-up of column c then lands on a column below the sub-step, already
// written).
//
// Ballots, shuffles and reductions run in warp-uniform control flow.
#pragma once

#include "mtgp_fast.cuh"

namespace mtgp {

// The warp's running statistics of its current piece (all fields but acc
// and bnd are uniform across the warp).
struct StatsState {
    uint32_t seq;    // current segment (index in the launch), kNoSeq = none
    uint32_t req;    // its request
    uint32_t lead;   // bit 0: the piece's first visit is still ahead; bit 1: the pair open at its start
                     // has not ended (pieces that do not start their request)
    uint32_t D;      // gap test: non-visits since the last visit (< 2^31)
    uint32_t rem;    // Hamming: values left in the current block, 1 .. K
    uint32_t half;   // Hamming: 1 when the current block is its pair's second
    uint32_t wa;     // Hamming: weight of the pair's first block (half = 1)
    uint32_t acc;    // this lane's part of the current block's weight
    uint32_t bnd;    // this lane's class bound (lanes 0 .. C-2), else ~0
};
constexpr uint32_t kNoSeq = 0xFFFFFFFFu;

// Position of the highest set bit, 0xFFFFFFFF for 0 (PTX bfind).
__device__ __forceinline__ uint32_t hibit(uint32_t x)
{
    uint32_t r;
    asm("bfind.u32 %0, %1;" : "=r"(r) : "r"(x));
    return r;
}

// Adds 1 to the shared-memory word at 32-bit shared address a.
__device__ __forceinline__ void count_at(uint32_t a)
{
    asm volatile("red.shared.add.u32 [%0], 1;" :: "r"(a));
}

// Gap test over lanes [l0, l0 + n) of one request; `valid` = lane in them.
// Returns the shared address this lane counts at: its class in the
// histogram hs when it visits, else its own slot `own`.
__device__ __forceinline__ uint32_t gap_run(uint32_t o, bool valid, uint32_t l0, uint32_t n, uint32_t lane,
                                            uint32_t lower, StatsState& st, uint32_t hs, uint32_t own,
                                            const StatsArgs& A)
{
    const bool in = valid && (o & A.gmask) == 0u;
    const uint32_t B = __ballot_sync(MTGP_FULL, in);
    const uint32_t hb = hibit(B & lower);   // nearest lower visiting lane, or ~0
    const uint32_t gap = hb != 0xFFFFFFFFu ? lane - hb - 1u : lane - l0 + st.D;
    st.D = B ? l0 + n - 1u - hibit(B) : st.D + n;
    return in ? hs + 4u * min(gap, A.t) : own;
}

// The piece's edge words (4, after the pair table): [0] non-visits before
// its first visit, [1] and [2] its weights in the blocks of the pair open at
// its start.
__device__ __forceinline__ uint32_t* piece_edges(uint32_t* tab, const StatsArgs& A)
{
    return tab + ((A.C * A.C + 3u) & ~3u);
}

// gap_run for the slow path, where a piece's first visit may come: its gap
// begins in an earlier piece, so it is recorded (non-visits before it in
// this piece) instead of counted.
__device__ __forceinline__ uint32_t gap_run_piece(uint32_t o, bool valid, uint32_t l0, uint32_t n,
                                                  uint32_t lane, uint32_t lower, StatsState& st, uint32_t hs,
                                                  uint32_t own, uint32_t* tab, const StatsArgs& A)
{
    const bool in = valid && (o & A.gmask) == 0u;
    const uint32_t B = __ballot_sync(MTGP_FULL, in);
    const uint32_t hb = hibit(B & lower);
    const uint32_t gap = hb != 0xFFFFFFFFu ? lane - hb - 1u : lane - l0 + st.D;
    bool counted = in;
    if ((st.lead & 1u) && B) {
        const uint32_t f = (uint32_t)__ffs(B) - 1u;
        if (lane == 0u)
            piece_edges(tab, A)[0] = st.D + f - l0;
        counted = in && lane != f;
        st.lead &= ~1u;
    }
    st.D = B ? l0 + n - 1u - hibit(B) : st.D + n;
    return counted ? hs + 4u * min(gap, A.t) : own;
}

// A Hamming block of weight W has ended: the first of a pair is kept, the
// second completes the pair, which lane 0 counts in the warp's table.  In
// the pair open at a piece's start, the weights go to the piece's edges.
__device__ __forceinline__ void block_done(uint32_t W, uint32_t lane, StatsState& st, uint32_t* tab,
                                           const StatsArgs& A)
{
    if (st.lead & 2u) {
        if (lane == 0u)
            piece_edges(tab, A)[1u + st.half] = W;
        if (st.half)
            st.lead &= ~2u;
        st.wa = W;
        st.half ^= 1u;
        return;
    }
    if (st.half) {
        const uint32_t ca = __popc(__ballot_sync(MTGP_FULL, st.bnd <= st.wa));
        const uint32_t cb = __popc(__ballot_sync(MTGP_FULL, st.bnd <= W));
        if (lane == 0u)
            tab[ca * A.C + cb] += 1u;
    }
    st.wa = W;
    st.half ^= 1u;
}

// Hamming test over lanes [l0, l0 + n) of one request (n <= 32 <= K: at
// most one block end); w = this lane's weight (0 outside the run).
__device__ __forceinline__ void ham_run(uint32_t w, uint32_t l0, uint32_t n, uint32_t lane,
                                        StatsState& st, uint32_t* tab, const StatsArgs& A)
{
    if (st.rem > n) {
        st.acc += w;
        st.rem -= n;
    } else {
        const bool next = lane >= l0 + st.rem;   // after the block's end
        const uint32_t W = __reduce_add_sync(MTGP_FULL, st.acc + (next ? 0u : w));
        st.acc = next ? w : 0u;
        block_done(W, lane, st, tab, A);
        st.rem = st.rem + A.K - n;
    }
}

// Ends the current piece: records its edges (split launches) and adds its
// histogram and table to its request's rows.  Then starts segment `next`
// (kNoSeq: none): its position in its request sets where it stands in the
// block pairs, and a piece that does not start its request begins with both
// leads pending.
__device__ __forceinline__ void stats_switch(StatsState& st, uint32_t next, uint32_t lane, uint32_t* h,
                                             uint32_t* tab, const Segment* __restrict__ segs,
                                             const StatsArgs& A)
{
    if (st.seq == next)
        return;
    uint32_t* pe = piece_edges(tab, A);
    if (st.seq != kNoSeq) {
        if (A.seg_stats) {
            const uint32_t part = __reduce_add_sync(MTGP_FULL, st.acc);   // the open block's weight here
            __syncwarp();
            if (lane == 0u) {
                SegStat r;
                const bool gl = (st.lead & 1u) != 0u, hl = (st.lead & 2u) != 0u;
                r.gvisit = gl ? 0u : 1u;
                r.gprefix = gl ? st.D : pe[0];
                r.gsuffix = st.D;
                if (hl) {   // the pair open at the start did not end here
                    r.la = st.half ? pe[1] : part;
                    r.lb = st.half ? part : 0u;
                    r.ta = 0u;
                    r.tb = 0u;
                } else {
                    r.la = pe[1];
                    r.lb = pe[2];
                    r.ta = st.half ? st.wa : part;
                    r.tb = st.half ? part : 0u;
                }
                r.pad = 0u;
                A.seg_stats[st.seq] = r;
            }
        }
        __syncwarp();
        for (uint32_t i = lane; i <= A.t; i += 32u) {
            if (A.hist && h[i])
                atomicAdd(A.hist + (size_t)st.req * (A.t + 1u) + i, (unsigned long long)h[i]);
            h[i] = 0u;
        }
        for (uint32_t i = lane; i < A.C * A.C; i += 32u) {
            if (A.tab && tab[i])
                atomicAdd(A.tab + (size_t)st.req * A.C * A.C + i, (unsigned long long)tab[i]);
            tab[i] = 0u;
        }
    }
    uint32_t pos = 0u;
    st.lead = 0u;
    if (next != kNoSeq) {
        const Segment sg = segs[next];
        st.req = sg.req;
        const uint64_t off = A.req_base ? sg.out_off - A.req_base[sg.req] : 0ull;
        pos = (uint32_t)(off % (2ull * A.K));
        st.lead = (off ? 1u : 0u) | (pos ? 2u : 0u);
        if (lane < 3u)
            pe[lane] = 0u;
    }
    __syncwarp();
    st.seq = next;
    st.D = 0u;
    st.half = pos >= A.K ? 1u : 0u;
    st.rem = A.K - pos % A.K;
    st.wa = 0u;
    st.acc = 0u;
}

// Shared addresses of the warp's histogram and of this lane's own slot
// (the 32 words after the histogram).
__device__ __forceinline__ uint32_t hist_addr(const uint32_t* h) { return (uint32_t)__cvta_generic_to_shared(h); }
__device__ __forceinline__ uint32_t own_addr(const uint32_t* h, uint32_t lane, const StatsArgs& A)
{
    return (uint32_t)__cvta_generic_to_shared(h + ((A.t + 1u + 3u) & ~3u) + lane);
}

// nfull consecutive full rows of one request (as gen_rows_pipelined, K = 4),
// with the statistics of every sub-step's outputs.  STEPH: Hamming per step
// (K >= 128), else per sub-step.
template <int M, int FMT, bool STEPH>
__device__ __forceinline__ void fused_rows(uint32_t (&r)[M], uint32_t* Sw, uint32_t* ow, const uint32_t* Q,
                                           const RowP& P, uint32_t lane, const uint32_t* __restrict__ Tb,
                                           uint32_t last_lane, uint32_t nfull, StatsState& st, uint32_t* h,
                                           uint32_t* tab, const StatsArgs& A)
{
    constexpr int K = 4;
    constexpr int NS = (M + K - 1) / K;
    const uint32_t N = P.n;
    const uint32_t lower = (1u << lane) - 1u;
    const bool last_ok = lane <= last_lane;     // lane holds a column of the row's last group
    const uint32_t nlast = last_lane + 1u;      // columns of the last group
    const uint32_t hs = hist_addr(h);
    const uint32_t own = own_addr(h, lane, A);
    uint32_t x1[K], xp[K], xq[K];
#pragma unroll
    for (int i = 0; i < K; ++i) {
        x1[i] = Sw[32 * i + 1];
        xp[i] = Q[32 * i];
        xq[i] = Q[32 * i - 1];
    }
    for (uint32_t q = 0; q < nfull; ++q, ow += N) {
#pragma unroll
        for (int s = 0; s < NS; ++s) {
            const int s0 = s * K;
            const int n0 = (s + 1 < NS) ? s0 + K : 0;
            uint32_t y1[K], yp[K], yq[K];
#pragma unroll
            for (int i = 0; i < K; ++i) {
                if (n0 + i < M) {
                    y1[i] = Sw[32 * (n0 + i) + 1];
                    yp[i] = Q[32 * (n0 + i)];
                    yq[i] = Q[32 * (n0 + i) - 1];
                }
            }
            uint32_t xn[K], o[K], w[K], ad[K];
#pragma unroll
            for (int i = 0; i < K; ++i) {
                if (s0 + i < M) {
                    const uint32_t yy = (r[s0 + i] & P.mask) ^ x1[i];
                    const uint32_t y = yy ^ (yy << P.sh1) ^ (xp[i] >> P.sh2);
                    xn[i] = y ^ tbl(Tb, 0u, y);
                    o[i] = temper_convert<FMT>(xn[i], temper_index(xq[i]), Tb);
                }
            }
            // statistics of this step's outputs
#pragma unroll
            for (int i = 0; i < K; ++i) {
                if (s0 + i < M) {
                    const bool lastg = s0 + i + 1 == M;
                    const bool valid = !lastg || last_ok;
                    ad[i] = gap_run(o[i], valid, 0u, lastg ? nlast : 32u, lane, lower, st, hs, own, A);
                    w[i] = valid ? __popc(o[i] & A.hmask) : 0u;
                    if constexpr (!STEPH)
                        ham_run(w[i], 0u, lastg ? nlast : 32u, lane, st, tab, A);
                }
            }
            if constexpr (STEPH) {
                const int KS = (M - s0 < K) ? M - s0 : K;   // sub-steps in this step
                const uint32_t step_n = (s0 + KS == M) ? 32u * (KS - 1) + nlast : 32u * KS;
                if (st.rem > step_n) {
                    uint32_t a = st.acc;
#pragma unroll
                    for (int i = 0; i < KS; ++i)
                        a += w[i];
                    st.acc = a;
                    st.rem -= step_n;
                } else {
                    // the block ends inside this step: step positions >= rem
                    // belong to the next block
                    uint32_t cur = st.acc, nxt = 0u;
#pragma unroll
                    for (int i = 0; i < KS; ++i) {
                        const bool after = 32u * (uint32_t)i + lane >= st.rem;
                        cur += after ? 0u : w[i];
                        nxt += after ? w[i] : 0u;
                    }
                    const uint32_t W = __reduce_add_sync(MTGP_FULL, cur);
                    st.acc = nxt;
                    block_done(W, lane, st, tab, A);
                    st.rem = st.rem + A.K - step_n;
                }
            }
#pragma unroll
            for (int i = 0; i < K; ++i) {
                const int m = s0 + i;
                if (m < M && (m + 1 < M || last_ok)) {
                    r[m] = xn[i];
                    Sw[32 * m] = xn[i];
                    if (32u * (uint32_t)m < P.mirror)
                        Sw[32 * m + N] = xn[i];
                    __stcs(ow + 32 * m, o[i]);
                }
            }
            __syncwarp();
#pragma unroll
            for (int i = 0; i < K; ++i) {
                if (s0 + i < M)
                    count_at(ad[i]);
                if (n0 + i < M) {
                    x1[i] = y1[i];
                    xp[i] = yp[i];
                    xq[i] = yq[i];
                }
            }
        }
    }
}

// nfull consecutive full rows of one request for short states (M < 9, no
// 128-word pipelined step fits): one 32-column sub-step at a time, with the
// statistics of each sub-step's outputs.  The words of the next sub-step are
// read before this sub-step's words are written, which is exact while
// N - pos >= 64: none of them is written by this sub-step, and a wrapped
// pick-up lands on a column of an earlier, already written sub-step.
template <int M, int FMT>
__device__ __forceinline__ void fused_rows_short(uint32_t (&r)[M], uint32_t* Sw, uint32_t* ow, const uint32_t* Q,
                                                 const RowP& P, uint32_t lane, const uint32_t* __restrict__ Tb,
                                                 uint32_t last_lane, uint32_t nfull, StatsState& st, uint32_t* h,
                                                 uint32_t* tab, const StatsArgs& A)
{
    static_assert(M >= 3, "the look-ahead read of the last sub-step needs three column groups");
    const uint32_t N = P.n;
    const uint32_t lower = (1u << lane) - 1u;
    const bool last_ok = lane <= last_lane;
    const uint32_t nlast = last_lane + 1u;
    const uint32_t hs = hist_addr(h);
    const uint32_t own = own_addr(h, lane, A);
    uint32_t x1 = Sw[1];
    uint32_t xp = Q[0];
    uint32_t xq = Q[-1];
    for (uint32_t q = 0; q < nfull; ++q, ow += N) {
#pragma unroll
        for (int m = 0; m < M; ++m) {
            const int mn = m + 1 < M ? m + 1 : 0;   // the next sub-step (of the next row after the last)
            const uint32_t y1 = Sw[32 * mn + 1];
            const uint32_t yp = Q[32 * mn];
            const uint32_t yq = Q[32 * mn - 1];
            const uint32_t yy = (r[m] & P.mask) ^ x1;
            const uint32_t y = yy ^ (yy << P.sh1) ^ (xp >> P.sh2);
            const uint32_t xn = y ^ tbl(Tb, 0u, y);
            const uint32_t o = temper_convert<FMT>(xn, temper_index(xq), Tb);
            const bool lastg = m + 1 == M;
            const bool valid = !lastg || last_ok;
            const uint32_t n = lastg ? nlast : 32u;
            const uint32_t ad = gap_run(o, valid, 0u, n, lane, lower, st, hs, own, A);
            ham_run(valid ? __popc(o & A.hmask) : 0u, 0u, n, lane, st, tab, A);
            if (valid) {
                r[m] = xn;
                Sw[32 * m] = xn;
                if (32u * (uint32_t)m < P.mirror)
                    Sw[32 * m + N] = xn;
                __stcs(ow + 32 * m, o);
            }
            __syncwarp();
            count_at(ad);
            x1 = y1;
            xp = yp;
            xq = yq;
        }
    }
}

// A row that crosses into the next request or ends the stream (n_valid
// columns): each lane finds its request; the statistics take the row's
// sub-steps in order, one run of same-request lanes at a time.
template <int M>
__device__ __forceinline__ void fused_row_slow(uint32_t (&r)[M], uint32_t* Sw, const uint32_t* Q,
                                               const RowP& P, uint32_t lane,
                                               const uint32_t* __restrict__ Tb, uint32_t n_valid,
                                               uint64_t row_g, const Segment* __restrict__ segs,
                                               uint32_t s_first, uint32_t s_end, uint32_t* __restrict__ out,
                                               StatsState& st, uint32_t* h, uint32_t* tab, const StatsArgs& A)
{
    const uint32_t lower = (1u << lane) - 1u;
#pragma unroll
    for (int m = 0; m < M; ++m) {
        if (32u * (uint32_t)m >= n_valid)
            break;
        const int off = 32 * m;
        const uint32_t x1 = Sw[off + 1];
        const uint32_t xp = Q[off];
        const uint32_t xq = Q[off - 1];
        const uint32_t yy = (r[m] & P.mask) ^ x1;
        const uint32_t y = yy ^ (yy << P.sh1) ^ (xp >> P.sh2);
        const uint32_t xn = y ^ tbl(Tb, 0u, y);
        const uint32_t ti = temper_index(xq);
        const uint32_t ou = temper_convert<0>(xn, ti, Tb);
        const uint32_t of = temper_convert<1>(xn, ti, Tb);
        const uint32_t col = 32u * (uint32_t)m + lane;
        const bool valid = col < n_valid;
        // this lane's request and stored value
        uint32_t s = s_first;
        const uint64_t gi = row_g + col;
        while (valid && s + 1 < s_end && gi >= segs[s + 1].g_start)
            ++s;
        const Segment sg = segs[s];
        uint32_t o = ou;
        if (sg.fmt == 1)
            o = of;
        else if (sg.fmt == 2)
            o = __float_as_uint(__uint_as_float(of) - 1.0f);
        // statistics: runs of lanes of one segment, in lane order
        uint32_t remaining = __ballot_sync(MTGP_FULL, valid);
        while (remaining) {
            const uint32_t l0 = (uint32_t)__ffs(remaining) - 1u;
            const uint32_t s0 = __shfl_sync(MTGP_FULL, s, l0);
            const uint32_t same = __ballot_sync(MTGP_FULL, valid && s == s0) & remaining;
            const uint32_t n = (uint32_t)__popc(same);
            const bool in_run = (same >> lane) & 1u;
            stats_switch(st, s0, lane, h, tab, segs, A);
            count_at(gap_run_piece(o, in_run, l0, n, lane, lower, st, hist_addr(h), own_addr(h, lane, A), tab,
                                   A));
            ham_run(in_run ? __popc(o & A.hmask) : 0u, l0, n, lane, st, tab, A);
            remaining &= ~same;
        }
        __syncwarp();
        if (valid) {
            r[m] = xn;
            Sw[off] = xn;
            if (32u * (uint32_t)m < P.mirror)
                Sw[off + P.n] = xn;
            out[sg.out_off + (gi - sg.g_start)] = o;
        }
        __syncwarp();
    }
}

// Advances one stream (this warp alone) by the segments [s_begin, s_end),
// with the statistics of every request.
template <int M>
__device__ __forceinline__ void fused_item(const KParams& KP, const RowP& P, uint32_t* __restrict__ g,
                                           uint32_t* S, const Segment* __restrict__ segs, uint32_t s_begin,
                                           uint32_t s_end, uint32_t* __restrict__ out, uint32_t lane,
                                           const uint32_t* __restrict__ Tb, StatsState& st, uint32_t* h,
                                           uint32_t* tab, const StatsArgs& A)
{
    const uint32_t N = P.n;
    const uint32_t last_lane = (N - 1u) & 31u;
    for (uint32_t c = lane; c < (KP.np >> 2); c += 32u)
        cp_async16(S + 4u * c, g + 4u * c);
    cp_async_wait_all();
    __syncwarp();
    uint32_t r[M];
#pragma unroll
    for (int j = 0; j < M; ++j) {
        const uint32_t c = 32u * (uint32_t)j + lane;
        r[j] = c < N ? S[c] : 0u;
    }
    for (uint32_t c = lane; c < P.mirror; c += 32u) {
        const uint32_t v = S[c];
        S[N + c] = v;
    }
    __syncwarp();
    uint32_t* Sw = S + lane;
    const uint32_t* Q = S + P.pos + lane;
    const Segment last = segs[s_end - 1u];
    const uint64_t total = last.g_start + last.count;
    uint32_t s = s_begin;
    Segment sg = segs[s];
    uint64_t seg_end = sg.g_start + sg.count;
    uint64_t row = 0;
    while (row < total) {
        while (row >= seg_end) {
            sg = segs[++s];
            seg_end = sg.g_start + sg.count;
        }
        if (row + N <= seg_end) {
            const uint32_t nfull = (uint32_t)min((seg_end - row) / N, (uint64_t)0xFFFFFFFFu);
            uint32_t* ow = out + sg.out_off + (row - sg.g_start) + lane;
            stats_switch(st, s, lane, h, tab, segs, A);
            if (st.lead || (M < 9 && N - P.pos < 64u)) {
                // a piece whose first gap or first pair is still open: one row
                // at a time on the slow path, which records them (also short
                // states too close for the look-ahead read, N - pos < 64)
                fused_row_slow<M>(r, Sw, Q, P, lane, Tb, N, row, segs, s, s_end, out, st, h, tab, A);
                row += N;
                continue;
            }
            if constexpr (M < 9) {
                if (sg.fmt == 0)
                    fused_rows_short<M, 0>(r, Sw, ow, Q, P, lane, Tb, last_lane, nfull, st, h, tab, A);
                else if (sg.fmt == 1)
                    fused_rows_short<M, 1>(r, Sw, ow, Q, P, lane, Tb, last_lane, nfull, st, h, tab, A);
                else
                    fused_rows_short<M, 2>(r, Sw, ow, Q, P, lane, Tb, last_lane, nfull, st, h, tab, A);
            } else if (A.K >= 128u) {
                if (sg.fmt == 0)
                    fused_rows<M, 0, true>(r, Sw, ow, Q, P, lane, Tb, last_lane, nfull, st, h, tab, A);
                else if (sg.fmt == 1)
                    fused_rows<M, 1, true>(r, Sw, ow, Q, P, lane, Tb, last_lane, nfull, st, h, tab, A);
                else
                    fused_rows<M, 2, true>(r, Sw, ow, Q, P, lane, Tb, last_lane, nfull, st, h, tab, A);
            } else {
                if (sg.fmt == 0)
                    fused_rows<M, 0, false>(r, Sw, ow, Q, P, lane, Tb, last_lane, nfull, st, h, tab, A);
                else if (sg.fmt == 1)
                    fused_rows<M, 1, false>(r, Sw, ow, Q, P, lane, Tb, last_lane, nfull, st, h, tab, A);
                else
                    fused_rows<M, 2, false>(r, Sw, ow, Q, P, lane, Tb, last_lane, nfull, st, h, tab, A);
            }
            row += (uint64_t)nfull * N;
        } else {
            const uint64_t left = total - row;
            const uint32_t n_valid = left < (uint64_t)N ? (uint32_t)left : N;
            fused_row_slow<M>(r, Sw, Q, P, lane, Tb, n_valid, row, segs, s, s_end, out, st, h, tab, A);
            row += N;
        }
    }
    const uint32_t phase = (uint32_t)(total % N);
    for (uint32_t j = lane; j < N; j += 32u) {
        uint32_t c = phase + j;
        c = c >= N ? c - N : c;
        g[j] = S[c];
    }
    __syncwarp();
}

// Persistent kernel: every warp claims streams (longest first) from the
// work table and advances each alone, with the statistics.
template <int M, int G>
__global__ void __launch_bounds__(G * 32) mtgp_fused_kernel(const KParams P, uint32_t* __restrict__ states,
                                                            uint32_t n_streams,
                                                            const WorkItem* __restrict__ items,
                                                            const Segment* __restrict__ segs,
                                                            uint32_t n_items, uint32_t* __restrict__ counters,
                                                            uint32_t* __restrict__ out, int* __restrict__ err,
                                                            const KSet* __restrict__ sets,
                                                            const uint32_t* __restrict__ set_of,
                                                            const StatsArgs A)
{
    extern __shared__ __align__(16) uint32_t smem[];
    __shared__ __align__(64) uint32_t Tb[G][48];
    const uint32_t lane = threadIdx.x & 31u;
    const uint32_t warp = threadIdx.x >> 5;
    if (threadIdx.x < 16) {
        Tb[0][threadIdx.x] = P.rec[threadIdx.x];
        Tb[0][16 + threadIdx.x] = P.tmp[threadIdx.x];
        Tb[0][32 + threadIdx.x] = P.flt[threadIdx.x];
    }
    const uint32_t row_words = fast_smem_words(P.n, P.mirror);
    uint32_t* S = smem + warp * (row_words + stats_smem_words(A.t, A.C));
    uint32_t* h = S + row_words;
    uint32_t* tab = h + ((A.t + 1u + 3u) & ~3u) + 32u;
    for (uint32_t i = lane; i < stats_smem_words(A.t, A.C); i += 32u)
        h[i] = 0u;
    __syncthreads();
    const RowP R0 = {P.n, P.mask, P.pos, P.sh1, P.sh2, P.mirror};
    StatsState st = {kNoSeq, 0u, 0u, 0u, A.K, 0u, 0u, 0u, 0xFFFFFFFFu};
#pragma unroll
    for (uint32_t i = 0; i < 15u; ++i)
        if (lane == i && i + 1u < A.C)
            st.bnd = A.bounds[i];
    for (;;) {
        uint32_t it = 0;
        if (lane == 0)
            it = atomicAdd(&counters[1], 1u);
        it = __shfl_sync(MTGP_FULL, it, 0);
        if (it >= n_items)
            break;
        const WorkItem w = items[it];
        if (w.stream >= n_streams || w.nseg == 0) {
            if (lane == 0)
                atomicOr(err, 1);
            continue;
        }
        uint32_t* g = states + (size_t)w.stream * P.np;
        if (sets) {
            const KSet& ks = sets[set_of[w.stream]];
            const RowP R = {P.n, P.mask, ks.pos, ks.sh1, ks.sh2, ks.mirror};
            if (lane < 16u) {
                Tb[warp][lane] = ks.rec[lane];
                Tb[warp][16u + lane] = ks.tmp[lane];
                Tb[warp][32u + lane] = ks.flt[lane];
            }
            __syncwarp();
            fused_item<M>(P, R, g, S, segs, w.seg_begin, w.seg_begin + w.nseg, out, lane, Tb[warp], st,
                          h, tab, A);
        } else {
            fused_item<M>(P, R0, g, S, segs, w.seg_begin, w.seg_begin + w.nseg, out, lane, Tb[0], st, h,
                          tab, A);
        }
    }
    stats_switch(st, kNoSeq, lane, h, tab, segs, A);
}

}  // namespace mtgp

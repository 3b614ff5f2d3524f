// Generation with the data reductions of the paper's two failing BigCrush
// tests (Sec. 4.2) fused in: the gap test (test 35) and Hamming-weight
// independence (test 100) are accumulated from each sub-step's outputs
// while they are still in registers, so the output is not read back.
//
// The generator is mtgp_fast_kernel's single-warp, software-pipelined row
// loop (128-word steps, N - pos >= 256; see mtgp_fast.cuh), unchanged except
// that every sub-step's 32 outputs (31 in a row's last sub-step when
// N = 351) also pass through stats_run.  A sequence of the statistics is one
// request of the launch (Segment::req): its values in generation order.
//
// Per sub-step, for a run of consecutive lanes [l0, l0 + n) of one sequence:
//   gap test -- a value visits when (value & gmask) == 0; the visits form a
//     ballot B; a visiting lane's gap is the number of non-visits since the
//     previous visit: its distance to the nearest lower visiting lane, or,
//     when none, lane - l0 plus the carried run D of non-visits before the
//     run (counted from the sequence's start, so the first visit's gap is
//     counted too).  Lengths >= t are pooled in class t; a trailing run of
//     non-visits is not a gap.
//   Hamming -- the weight popc(value & hmask) of each value adds to the
//     first or second block of the current pair (K values per block) by the
//     value's position in the pair; per-lane partial sums are reduced when a
//     pair completes, and lane 0 counts (class of first, class of second)
//     in the warp's table.  An incomplete trailing pair is ignored.
// Each sequence belongs to one warp, which writes its histogram and table
// rows when the sequence ends.  Ballots, shuffles and reductions run in
// warp-uniform control flow; lane-dependent branches hold only shared-memory
// updates.
#pragma once

#include "mtgp_fast.cuh"

namespace mtgp {

// The warp's running statistics of its current sequence.
struct StatsState {
    uint32_t seq;    // current sequence (request index), kNoSeq = none
    uint32_t D;      // non-visits since the last visit (saturating)
    uint32_t pos;    // position of the next value within the current block pair
    uint32_t acc_a;  // this lane's partial weight of the pair's first block
    uint32_t acc_b;  // ... and of its second block
};
constexpr uint32_t kNoSeq = 0xFFFFFFFFu;
constexpr uint32_t kMaxRun = 0x3FFFFFFFu;

__device__ __forceinline__ void stats_run(uint32_t o, uint32_t l0, uint32_t n, uint32_t lane,
                                          StatsState& st, uint32_t* h, uint32_t* tab,
                                          const StatsArgs& A)
{
    const bool lane_in = lane >= l0 && lane < l0 + n;
    if (A.gmask) {
        const bool in = lane_in && (o & A.gmask) == 0u;
        const uint32_t B = __ballot_sync(MTGP_FULL, in);
        const uint32_t below = B & ((1u << lane) - 1u);
        const uint32_t gap = below ? lane - 1u - (31u - (uint32_t)__clz(below)) : lane - l0 + st.D;
        if (in)
            atomicAdd(&h[min(gap, A.t)], 1u);
        st.D = B ? l0 + n - 1u - (31u - (uint32_t)__clz(B)) : min(st.D + n, kMaxRun);
    }
    if (A.hmask) {
        const uint32_t w = __popc(o & A.hmask);
        const uint32_t p = st.pos + lane - l0;   // meaningful for lanes in the run
        if (lane_in && p < A.K)
            st.acc_a += w;
        else if (lane_in && p < 2u * A.K)
            st.acc_b += w;
        if (st.pos + n >= 2u * A.K) {   // the pair completes in this run (2K > 32)
            const uint32_t wa = __reduce_add_sync(MTGP_FULL, st.acc_a);
            const uint32_t wb = __reduce_add_sync(MTGP_FULL, st.acc_b);
            if (lane == 0u) {
                uint32_t ca = 0u, cb = 0u;
#pragma unroll
                for (uint32_t i = 0; i < 15u; ++i) {
                    if (i + 1u < A.C) {
                        ca += A.bounds[i] <= wa;
                        cb += A.bounds[i] <= wb;
                    }
                }
                tab[ca * A.C + cb] += 1u;
            }
            st.acc_a = (lane_in && p >= 2u * A.K) ? w : 0u;
            st.acc_b = 0u;
            st.pos = st.pos + n - 2u * A.K;
        } else {
            st.pos += n;
        }
    }
}

// Writes the current sequence's histogram and table rows and starts `next`.
__device__ __forceinline__ void stats_switch(StatsState& st, uint32_t next, uint32_t lane, uint32_t* h,
                                             uint32_t* tab, const StatsArgs& A)
{
    if (st.seq == next)
        return;
    __syncwarp();
    if (st.seq != kNoSeq) {
        if (A.gmask)
            for (uint32_t i = lane; i <= A.t; i += 32u) {
                A.hist[(size_t)st.seq * (A.t + 1u) + i] = h[i];
                h[i] = 0u;
            }
        if (A.hmask)
            for (uint32_t i = lane; i < A.C * A.C; i += 32u) {
                A.tab[(size_t)st.seq * A.C * A.C + i] = tab[i];
                tab[i] = 0u;
            }
    }
    __syncwarp();
    st.seq = next;
    st.D = 0u;
    st.pos = 0u;
    st.acc_a = 0u;
    st.acc_b = 0u;
}

// nfull consecutive full rows of one request (as gen_rows_pipelined, K = 4),
// with the statistics of every sub-step's outputs.
template <int M, int FMT>
__device__ __forceinline__ void fused_rows(uint32_t (&r)[M], uint32_t* Sw, uint32_t* ow, const uint32_t* Q,
                                           const RowP& P, uint32_t lane, const uint32_t* __restrict__ Tb,
                                           uint32_t last_lane, uint32_t nfull, StatsState& st, uint32_t* h,
                                           uint32_t* tab, const StatsArgs& A)
{
    constexpr int K = 4;
    constexpr int NS = (M + K - 1) / K;
    const uint32_t N = P.n;
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
            uint32_t xn[K], o[K];
#pragma unroll
            for (int i = 0; i < K; ++i) {
                if (s0 + i < M) {
                    const uint32_t yy = (r[s0 + i] & P.mask) ^ x1[i];
                    const uint32_t y = yy ^ (yy << P.sh1) ^ (xp[i] >> P.sh2);
                    xn[i] = y ^ tbl(Tb, 0u, y);
                    o[i] = temper_convert<FMT>(xn[i], temper_index(xq[i]), Tb);
                }
            }
#pragma unroll
            for (int i = 0; i < K; ++i)
                if (s0 + i < M)
                    stats_run(o[i], 0u, s0 + i + 1 < M ? 32u : last_lane + 1u, lane, st, h, tab, A);
#pragma unroll
            for (int i = 0; i < K; ++i) {
                const int m = s0 + i;
                if (m < M && (m + 1 < M || lane <= last_lane)) {
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
                if (n0 + i < M) {
                    x1[i] = y1[i];
                    xp[i] = yp[i];
                    xq[i] = yq[i];
                }
            }
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
        const uint32_t req = sg.req;
        // statistics: runs of lanes of one request, in lane order
        uint32_t remaining = __ballot_sync(MTGP_FULL, valid);
        while (remaining) {
            const uint32_t l0 = (uint32_t)__ffs(remaining) - 1u;
            const uint32_t r0 = __shfl_sync(MTGP_FULL, req, l0);
            const uint32_t same = __ballot_sync(MTGP_FULL, valid && req == r0) & remaining;
            stats_switch(st, r0, lane, h, tab, A);
            stats_run(o, l0, (uint32_t)__popc(same), lane, st, h, tab, A);
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
            stats_switch(st, sg.req, lane, h, tab, A);
            if (sg.fmt == 0)
                fused_rows<M, 0>(r, Sw, ow, Q, P, lane, Tb, last_lane, nfull, st, h, tab, A);
            else if (sg.fmt == 1)
                fused_rows<M, 1>(r, Sw, ow, Q, P, lane, Tb, last_lane, nfull, st, h, tab, A);
            else
                fused_rows<M, 2>(r, Sw, ow, Q, P, lane, Tb, last_lane, nfull, st, h, tab, A);
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
    uint32_t* tab = h + ((A.t + 1u + 3u) & ~3u);
    for (uint32_t i = lane; i < stats_smem_words(A.t, A.C); i += 32u)
        h[i] = 0u;
    __syncthreads();
    const RowP R0 = {P.n, P.mask, P.pos, P.sh1, P.sh2, P.mirror};
    StatsState st = {kNoSeq, 0u, 0u, 0u, 0u};
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
    stats_switch(st, kNoSeq, lane, h, tab, A);
}

}  // namespace mtgp

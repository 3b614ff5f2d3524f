// Register-resident MTGP32 generation kernel for sm_103a.
//
// Streams are advanced by one warp each (the paper's "PRNG per block of
// threads", Sec. 2, with the state on chip while it is advanced and in global
// memory between launches), or -- for the longest streams of a launch -- by
// all G warps of a CTA together.
//
// Layout of a stream's state while it is on chip:
//   * The sequence is cut into rows of N words: column c of row q holds
//     x_{qN + c}.  Computing row q+1 column c needs (row q, c) and
//     (row q, c+1) [the words i and i+1 of the recurrence] and the word i+pos,
//     which is (row q, c+pos) when c+pos < N and (row q+1, c+pos-N) otherwise;
//     the tempering word i+pos-1 likewise.  So a state needs only the latest
//     value of each column.
//   * Column group m (columns 32m .. 32m+31) belongs to one warp; lane l of
//     that warp keeps column 32m + l in a register (word i).
//   * The latest value of every column is also published in a shared-memory
//     row S[0..N), followed by a mirror S[N..N+E) of columns 0..E-1,
//     E >= pos + 31.  Words i+1, i+pos and i+pos-1 of 32 consecutive columns
//     are then plain conflict-free loads at S[c+1], S[c+pos], S[c+pos-1]
//     with no modulo and no bounds arithmetic: a pick-up past column N-1
//     lands in the mirror, which holds the new row's value of that column.
//   * The recursion and tempering tables are 16-word shared arrays whose entry
//     k sits in bank k, so a warp's 32 lookups are one conflict-free
//     shared-memory wavefront whatever the indices.
//
// A sub-step m computes columns 32m..32m+31 of the next row (one new word per
// lane).  K consecutive sub-steps form one parallel step of 32K words; when
// 32K <= N - pos none of them reads a word produced in the same step (the
// block-parallel window of the method), so a step reads everything, passes a
// barrier, then writes everything.
#pragma once

#include "mtgp_internal.h"

namespace mtgp {

#define MTGP_FULL 0xFFFFFFFFu

__device__ __forceinline__ void cp_async16(uint32_t* smem_dst, const uint32_t* gsrc)
{
    const uint32_t s = (uint32_t)__cvta_generic_to_shared(smem_dst);
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(s), "l"(gsrc) : "memory");
}

__device__ __forceinline__ uint64_t global_ns()
{
    uint64_t t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

__device__ __forceinline__ uint32_t sm_id()
{
    uint32_t v;
    asm volatile("mov.u32 %0, %%smid;" : "=r"(v));
    return v;
}

// Timeline record of one item (only when a trace buffer is given).
__device__ __forceinline__ void trace_item(uint64_t* trace, uint32_t it, uint64_t t0,
                                           const Segment* segs, const WorkItem& w)
{
    const Segment last = segs[w.seg_begin + w.nseg - 1u];
    trace[4u * it + 0] = t0;
    trace[4u * it + 1] = global_ns();
    trace[4u * it + 2] = sm_id();
    trace[4u * it + 3] = last.g_start + last.count;
}

__device__ __forceinline__ void cp_async_wait_all()
{
    asm volatile("cp.async.commit_group;\n" ::: "memory");
    asm volatile("cp.async.wait_group 0;\n" ::: "memory");
}

// Per-stream scalars the row code reads: the handle's parameter set, or the
// stream's own set when the handle has one per stream (all sets of a handle
// share N and the mask).  Kept in registers for the whole item.
struct RowP {
    uint32_t n, mask, pos, sh1, sh2, mirror;
};

// Tables in shared memory: 16 words each, at a 64-byte aligned base, so
// that entry k of a table sits in bank k and any lookup pattern of a warp is
// one conflict-free wavefront.  Tb[0..16) recursion, Tb[16..32) tempering,
// Tb[32..48) float tempering.
__device__ __forceinline__ uint32_t tbl(const uint32_t* Tb, uint32_t base, uint32_t idx)
{
    return Tb[base + (idx & 15u)];
}

// Tempering index from word i+pos-1: fold >> 16 then >> 8; the low four bits
// select the entry.
__device__ __forceinline__ uint32_t temper_index(uint32_t xq)
{
    const uint32_t t = xq ^ (xq >> 16);
    return t ^ (t >> 8);
}

// Output conversion from the new word v and the tempering index ti.
//   FMT 0: v ^ TMP[ti]
//   FMT 1: (v >> 9) ^ FLT[ti]   == 0x3F800000 | ((v ^ TMP[ti]) >> 9)
//   FMT 2: the FMT 1 float minus 1.0f (exact: Sterbenz)
template <int FMT>
__device__ __forceinline__ uint32_t temper_convert(uint32_t v, uint32_t ti, const uint32_t* Tb)
{
    if (FMT == 0)
        return v ^ tbl(Tb, 16u, ti);
    const uint32_t b = (v >> 9) ^ tbl(Tb, 32u, ti);
    if (FMT == 1)
        return b;
    return __float_as_uint(__uint_as_float(b) - 1.0f);
}

// Per-lane output of the slow path: the lane finds its request and format
// (ou / of are the u32 and [1,2) outputs).
__device__ __forceinline__ void slow_store(uint32_t ou, uint32_t of, uint64_t g,
                                           const Segment* __restrict__ segs, uint32_t s_first,
                                           uint32_t s_end, uint32_t* __restrict__ out)
{
    uint32_t s = s_first;
    while (s + 1 < s_end && g >= segs[s + 1].g_start)
        ++s;
    const Segment sg = segs[s];
    uint32_t o = ou;
    if (sg.fmt == 1)
        o = of;
    else if (sg.fmt == 2)
        o = __float_as_uint(__uint_as_float(of) - 1.0f);
    out[sg.out_off + (g - sg.g_start)] = o;
}

// ===========================================================================
// Rows.  A row is "full" when all N of its words go to one request; other
// rows (the last, partial row of a stream, or a row crossing requests) take
// the slow path where each lane finds its own request.
//
// Work split: sub-step m of a row belongs to warp (m mod WG) of the WG warps
// advancing the stream (WG = 1 for a warp-owned stream); that warp keeps
// columns 32m + lane in register r[m / WG].  `Sw` = S + 32*warp + lane.
//
// No warp-synchronous instruction is executed under a lane-dependent
// condition: the write phase is lane-predicated and holds only stores.
//
// S, Sw and Q all point into the same shared row (and ow into `out`), so
// none of them is __restrict__: the loads of one step must stay after the
// stores of the previous one.
// ===========================================================================
template <int M, int K, int WG, int FMT, bool SLOW>
__device__ __forceinline__ void gen_row(uint32_t (&r)[(M + WG - 1) / WG], uint32_t* S,
                                        uint32_t* Sw, uint32_t* ow,
                                        const uint32_t* Q, const RowP& P,
                                        uint32_t warp, uint32_t lane, const uint32_t* __restrict__ Tb,
                                        uint32_t last_lane, uint32_t n_valid, uint64_t row_g,
                                        const Segment* __restrict__ segs, uint32_t s_first,
                                        uint32_t s_end, uint32_t* __restrict__ out)
{
    constexpr int J = (M + WG - 1) / WG;
    constexpr int PER = K / WG;   // sub-steps per warp in one parallel step
#pragma unroll
    for (int s0 = 0; s0 < M; s0 += K) {
        if (SLOW && 32u * (uint32_t)s0 >= n_valid)
            break;
        // The read phase runs in stages across the PER sub-steps (all loads,
        // then all recursion arithmetic, then all table lookups, ...) so that
        // the sub-steps' latencies overlap.
        bool on[PER];
        uint32_t x1[PER], xp[PER], xq[PER], y[PER], xn[PER], ti[PER], o1[PER], o2[PER];
#pragma unroll
        for (int i = 0; i < PER; ++i) {
            const int j = s0 / WG + i;
            const uint32_t m = (uint32_t)(s0 + i * WG) + (WG > 1 ? warp : 0u);
            on[i] = j < J && m < (uint32_t)M;   // uniform across the warp
            if (on[i]) {
                const int off = 32 * (s0 + i * WG);   // static part of 32m
                x1[i] = Sw[off + 1];    // word i+1
                xp[i] = Q[off];         // word i+pos   (Q = S + pos + 32*warp + lane)
                xq[i] = Q[off - 1];     // word i+pos-1
            }
        }
#pragma unroll
        for (int i = 0; i < PER; ++i)
            if (on[i]) {
                const uint32_t yy = (r[s0 / WG + i] & P.mask) ^ x1[i];
                y[i] = yy ^ (yy << P.sh1) ^ (xp[i] >> P.sh2);
            }
#pragma unroll
        for (int i = 0; i < PER; ++i)
            if (on[i])
                xn[i] = y[i] ^ tbl(Tb, 0u, y[i]);
#pragma unroll
        for (int i = 0; i < PER; ++i)
            if (on[i])
                ti[i] = temper_index(xq[i]);
#pragma unroll
        for (int i = 0; i < PER; ++i)
            if (on[i]) {
                if (SLOW) {
                    o1[i] = temper_convert<0>(xn[i], ti[i], Tb);
                    o2[i] = temper_convert<1>(xn[i], ti[i], Tb);
                } else {
                    o1[i] = temper_convert<FMT>(xn[i], ti[i], Tb);
                }
            }
        if (WG > 1)
            __syncthreads();
        else
            __syncwarp();
#pragma unroll
        for (int i = 0; i < PER; ++i) {
            const int j = s0 / WG + i;
            const uint32_t m = (uint32_t)(s0 + i * WG) + (WG > 1 ? warp : 0u);
            if (j < J && m < (uint32_t)M) {
                const int off = 32 * (s0 + i * WG);
                const uint32_t col = 32u * m + lane;
                const bool act = SLOW ? (col < n_valid) : (m + 1u < (uint32_t)M || lane <= last_lane);
                if (act) {
                    r[j] = xn[i];
                    Sw[off] = xn[i];
                    if (32u * m < P.mirror)
                        Sw[off + P.n] = xn[i];
                    if (SLOW)
                        slow_store(o1[i], o2[i], row_g + col, segs, s_first, s_end, out);
                    else
                        __stcs(ow + off, o1[i]);
                }
            }
        }
        if (WG > 1)
            __syncthreads();
        else
            __syncwarp();
    }
}

// ===========================================================================
// nfull consecutive full rows of one request, single warp, software-pipelined
// steps of W = 128 words (K = 4 sub-steps).
//
// When N - pos >= 2W, the loads of step s+1 never touch a word that step s
// writes: word i+1 and the unwrapped pick-ups lie beyond step s's columns,
// and a wrapped pick-up (mirror) of a column c < W(s+2) lands below
// c + pos - N < Ws.  The same holds from the last step of a row to the first
// step of the next (its pick-ups end below pos + W <= N - W, where the last
// step begins at or above N - W).  So the loads of step s+1 are issued
// before the stores of step s, and one __syncwarp per step (after the
// stores) orders every store before the loads that read it two steps later.
// The loads issued during a row's last step are those of step 0 (the same
// addresses in every row); after the last row they are simply unused.
// ===========================================================================
template <int M, int FMT>
__device__ __forceinline__ void gen_rows_pipelined(uint32_t (&r)[M], uint32_t* Sw, uint32_t* ow,
                                                   const uint32_t* Q, const RowP& P, uint32_t lane,
                                                   const uint32_t* __restrict__ Tb, uint32_t last_lane,
                                                   uint32_t nfull)
{
    constexpr int K = 4;
    constexpr int NS = (M + K - 1) / K;   // steps per row (>= 3 here)
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
        for (int st = 0; st < NS; ++st) {
            const int s0 = st * K;
            const int n0 = (st + 1 < NS) ? s0 + K : 0;   // next step (next row's first)
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

// Advances one stream by the segments [s_begin, s_end) of the work table.
// WG warps take part (WG = 1: this warp alone; WG = G: the whole CTA).
template <int M, int K, int WG>
__device__ __forceinline__ void run_item(const KParams& KP, const RowP& P, uint32_t* __restrict__ g,
                                         uint32_t* __restrict__ S, const Segment* __restrict__ segs,
                                         uint32_t s_begin, uint32_t s_end, uint32_t* __restrict__ out,
                                         uint32_t warp, uint32_t lane, const uint32_t* __restrict__ Tb)
{
    constexpr int J = (M + WG - 1) / WG;
    const uint32_t N = P.n;
    const uint32_t tid = WG > 1 ? threadIdx.x : lane;
    const uint32_t wk = WG > 1 ? warp : 0u;
    const uint32_t last_lane = (N - 1u) & 31u;   // lane of column N-1 (group M-1)

    // stage in: the state row (HBM) -> S through 16-byte cp.async
    for (uint32_t c = tid; c < (KP.np >> 2); c += 32u * WG)
        cp_async16(S + 4u * c, g + 4u * c);
    cp_async_wait_all();
    if (WG > 1)
        __syncthreads();
    else
        __syncwarp();
    uint32_t r[J];
#pragma unroll
    for (int j = 0; j < J; ++j) {
        const uint32_t c = 32u * (wk + (uint32_t)(j * WG)) + lane;
        r[j] = c < N ? S[c] : 0u;
    }
    // mirror: columns 0 .. P.mirror-1 again at S[N ..]
    for (uint32_t c = tid; c < P.mirror; c += 32u * WG) {
        const uint32_t v = S[c];
        S[N + c] = v;
    }
    if (WG > 1)
        __syncthreads();
    else
        __syncwarp();

    uint32_t* Sw = S + 32u * wk + lane;
    const uint32_t* Q = S + P.pos + 32u * wk + lane;
    const Segment last = segs[s_end - 1u];
    const uint64_t total = last.g_start + last.count;
    // The current request stays in registers: rows only touch the table
    // when they cross into the next request (a dependent global load per row
    // would put an L2 round trip on every row's critical path).
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
            // The rows that lie wholly inside this request run back to back:
            // per row only the output pointer moves.
            const uint32_t nfull = (uint32_t)min((seg_end - row) / N, (uint64_t)0xFFFFFFFFu);
            uint32_t* ow = out + sg.out_off + (row - sg.g_start) + 32u * wk + lane;
            bool piped = false;
            if constexpr (K == 4 && WG == 1 && M >= 9) {
                if (N - P.pos >= 256u) {
                    if (sg.fmt == 0)
                        gen_rows_pipelined<M, 0>(r, Sw, ow, Q, P, lane, Tb, last_lane, nfull);
                    else if (sg.fmt == 1)
                        gen_rows_pipelined<M, 1>(r, Sw, ow, Q, P, lane, Tb, last_lane, nfull);
                    else
                        gen_rows_pipelined<M, 2>(r, Sw, ow, Q, P, lane, Tb, last_lane, nfull);
                    piped = true;
                }
            }
            if (piped) {
            } else if (sg.fmt == 0) {
                for (uint32_t q = 0; q < nfull; ++q, ow += N)
                    gen_row<M, K, WG, 0, false>(r, S, Sw, ow, Q, P, wk, lane, Tb, last_lane, N, row,
                                                segs, s, s_end, out);
            } else if (sg.fmt == 1) {
                for (uint32_t q = 0; q < nfull; ++q, ow += N)
                    gen_row<M, K, WG, 1, false>(r, S, Sw, ow, Q, P, wk, lane, Tb, last_lane, N, row,
                                                segs, s, s_end, out);
            } else {
                for (uint32_t q = 0; q < nfull; ++q, ow += N)
                    gen_row<M, K, WG, 2, false>(r, S, Sw, ow, Q, P, wk, lane, Tb, last_lane, N, row,
                                                segs, s, s_end, out);
            }
            row += (uint64_t)nfull * N;
        } else {
            // a row that crosses into the next request, or the partial last row
            const uint64_t left = total - row;
            const uint32_t n_valid = left < (uint64_t)N ? (uint32_t)left : N;
            gen_row<M, K, WG, 0, true>(r, S, Sw, nullptr, Q, P, wk, lane, Tb, last_lane, n_valid,
                                       row, segs, s, s_end, out);
            row += N;
        }
    }

    // stage out: oldest word first, x_total .. x_{total+N-1}; the column of
    // x_{total+j} is (total + j) mod N
    const uint32_t phase = (uint32_t)(total % N);
    for (uint32_t j = tid; j < N; j += 32u * WG) {
        uint32_t c = phase + j;
        c = c >= N ? c - N : c;
        g[j] = S[c];
    }
    if (WG > 1)
        __syncthreads();
    else
        __syncwarp();
}

// Persistent kernel.  Phase 1: the CTA claims the longest streams (items
// [0, n_coop) of the table, sorted longest first) one at a time and its G
// warps advance each together.  Phase 2: every warp claims the remaining
// items [n_coop, n_items) one by one and advances each alone.
template <int M, int K, int G>
__global__ void __launch_bounds__(G * 32) mtgp_fast_kernel(const KParams P, uint32_t* __restrict__ states,
                                                           uint32_t n_streams,
                                                           const WorkItem* __restrict__ items,
                                                           const Segment* __restrict__ segs,
                                                           uint32_t n_items, uint32_t n_coop,
                                                           uint32_t* __restrict__ counters,
                                                           uint32_t* __restrict__ out, int* __restrict__ err,
                                                           uint64_t* __restrict__ trace,
                                                           const KSet* __restrict__ sets,
                                                           const uint32_t* __restrict__ set_of)
{
    extern __shared__ __align__(16) uint32_t smem[];
    __shared__ uint32_t s_claim;
    // Tables: Tb[0] holds the handle's set; with per-stream sets each warp
    // loads its stream's tables into its own Tb[warp] (192-byte rows, so
    // every table starts on a 64-byte boundary: entry k in bank k).
    __shared__ __align__(64) uint32_t Tb[G][48];
    const uint32_t lane = threadIdx.x & 31u;
    const uint32_t warp = threadIdx.x >> 5;
    if (threadIdx.x < 16) {
        Tb[0][threadIdx.x] = P.rec[threadIdx.x];
        Tb[0][16 + threadIdx.x] = P.tmp[threadIdx.x];
        Tb[0][32 + threadIdx.x] = P.flt[threadIdx.x];
    }
    __syncthreads();
    const RowP R0 = {P.n, P.mask, P.pos, P.sh1, P.sh2, P.mirror};

    // The CTA-wide phase splits each parallel step's K sub-steps over the G
    // warps, so it exists only for K >= G and for handles with one parameter
    // set; otherwise every item is a single-warp item.
    const uint32_t first_single = (K >= G && !sets) ? n_coop : 0u;
    if constexpr (K >= G) {
    for (; !sets;) {
        if (threadIdx.x == 0)
            s_claim = atomicAdd(&counters[0], 1u);
        __syncthreads();
        const uint32_t it = s_claim;
        __syncthreads();
        if (it >= n_coop)
            break;
        const WorkItem w = items[it];
        if (w.stream >= n_streams || w.nseg == 0) {
            if (threadIdx.x == 0)
                atomicOr(err, 1);
            continue;
        }
        const uint64_t t0 = trace ? global_ns() : 0;
        run_item<M, K, G>(P, R0, states + (size_t)w.stream * P.np, smem, segs, w.seg_begin,
                          w.seg_begin + w.nseg, out, warp, lane, Tb[0]);
        if (trace && threadIdx.x == 0)
            trace_item(trace, it, t0, segs, w);
    }
    }

    uint32_t* S = smem + warp * fast_smem_words(P.n, P.mirror);
    for (;;) {
        uint32_t it = 0;
        if (lane == 0)
            it = first_single + atomicAdd(&counters[1], 1u);
        it = __shfl_sync(MTGP_FULL, it, 0);
        if (it >= n_items)
            break;
        const WorkItem w = items[it];
        if (w.stream >= n_streams || w.nseg == 0) {
            if (lane == 0)
                atomicOr(err, 1);
            continue;
        }
        const uint64_t t0 = trace ? global_ns() : 0;
        if (sets) {
            // this stream's own parameter set
            const KSet& ks = sets[set_of[w.stream]];
            const RowP R = {P.n, P.mask, ks.pos, ks.sh1, ks.sh2, ks.mirror};
            if (lane < 16u) {
                Tb[warp][lane] = ks.rec[lane];
                Tb[warp][16u + lane] = ks.tmp[lane];
                Tb[warp][32u + lane] = ks.flt[lane];
            }
            __syncwarp();
            run_item<M, K, 1>(P, R, states + (size_t)w.stream * P.np, S, segs, w.seg_begin,
                              w.seg_begin + w.nseg, out, warp, lane, Tb[warp]);
        } else {
            run_item<M, K, 1>(P, R0, states + (size_t)w.stream * P.np, S, segs, w.seg_begin,
                              w.seg_begin + w.nseg, out, warp, lane, Tb[0]);
        }
        if (trace && lane == 0)
            trace_item(trace, it, t0, segs, w);
    }
}

}  // namespace mtgp

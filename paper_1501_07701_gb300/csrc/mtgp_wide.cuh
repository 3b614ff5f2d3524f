// Wide-column MTGP32 generation kernel for sm_103a.
//
// Same method and work model as mtgp_fast_kernel (one warp per stream, the
// state in registers while it is advanced, steps of W = 128 new words), but
// with a lane owning four CONSECUTIVE columns of each step instead of four
// columns 32 apart:
//
//   * Row q of the sequence holds x_{qN + c} in column c.  Step s of a row
//     computes columns 128s .. 128s+127 of the next row; lane l computes
//     columns 128s + 4l + k, k = 0..3, and keeps them in r[s][k].
//   * Word i+1 of columns k = 0..2 is the lane's own next register; only
//     the fourth column needs a neighbour's word (one shared load).  The
//     pick-up words i+pos and i+pos-1 of the four columns are five
//     consecutive words, so a lane loads 5 instead of 8.
//   * The latest value of every column is published in a shared row laid
//     out in four interleaved sub-rows: column c sits at (c & 3) * R +
//     (c >> 2).  For a fixed k (or j) the 32 lanes of a step then touch 32
//     consecutive words of one sub-row: every access is one conflict-free
//     wavefront.
//   * Pick-ups past column N-1 belong to the new row (column w - N).  Their
//     addresses are precomputed per lane and step with the wrap applied, so
//     no mirrored copy of the row's head has to be stored.
//   * The four outputs of a lane are consecutive in memory.  A step's 128
//     outputs start at an arbitrary element offset A = (address / 4) mod 4
//     (rows are N words long, N odd), so lane l stores the 16-byte aligned
//     chunk that starts A elements before its first output: its own first
//     4 - A outputs behind the last A of lane l-1 (A shuffles), lane 0 taking
//     those from the previous step (a carry).  One st.global.cs.v4 per lane
//     per step.
//
// A step reads only words written at least two steps before it when
// N - pos >= 256 (the block-parallel window of the method, twice), so the
// loads of step s+1 are issued before the stores of step s, with one
// __syncwarp per step.  The wrapped pick-ups of a step end below
// 128(s+2) + pos - N <= 128s; a row's first step reads columns up to
// pos + 127 < 128(NS-1), below the previous row's last step.
#pragma once

#include "mtgp_fast.cuh"

namespace mtgp {

// Shared-row word index of column c (four sub-rows of R words).
__device__ __forceinline__ uint32_t quad_index(uint32_t c, uint32_t R) { return (c & 3u) * R + (c >> 2); }

// Tempered output of new word xn from pick-up word xq (word i+pos-1).
template <int FMT>
__device__ __forceinline__ uint32_t wide_output(uint32_t xn, uint32_t xq, const uint32_t* Tb)
{
    return temper_convert<FMT>(xn, temper_index(xq), Tb);
}

// Per-lane addresses of one item: pick-up words 128s + 4l + pos - 1 + j
// (j = 0..4) and the word after the lane's last column, wrapped into the new
// row past column N-1; kl = index of the lane's last valid column in the
// last step (3 when all four are valid).
template <int NS>
struct WideLane {
    uint32_t pa[NS][5];
    uint32_t ta[NS];
    uint32_t kl;
};

template <int NS>
__device__ __forceinline__ void wide_lane_setup(WideLane<NS>& L, const RowP& P, uint32_t R,
                                                uint32_t lane)
{
    const uint32_t N = P.n;
#pragma unroll
    for (int s = 0; s < NS; ++s) {
#pragma unroll
        for (int j = 0; j < 5; ++j) {
            uint32_t w = 128u * s + 4u * lane + P.pos - 1u + (uint32_t)j;
            w = w >= N ? w - N : w;   // w < 2N since pos + 131 < N
            L.pa[s][j] = quad_index(w, R);
        }
        uint32_t t = 128u * s + 4u * lane + 4u;
        if (s == NS - 1) {
            const uint32_t base = 128u * (NS - 1) + 4u * lane;
            const uint32_t kl = base + 3u < N ? 3u : (base < N ? N - 1u - base : 3u);
            L.kl = kl;
            t = base + kl + 1u;
            t = t >= N ? t - N : t;
        }
        L.ta[s] = quad_index(t, R);
    }
}

// New word and output of one column: x0 = word i, x1 = word i+1, xp = word
// i+pos, xq = word i+pos-1.
template <int FMT>
__device__ __forceinline__ void wide_column(uint32_t x0, uint32_t x1, uint32_t xp, uint32_t xq,
                                            const RowP& P, const uint32_t* __restrict__ Tb,
                                            uint32_t& xn, uint32_t& o)
{
    const uint32_t yy = (x0 & P.mask) ^ x1;
    const uint32_t y = yy ^ (yy << P.sh1) ^ (xp >> P.sh2);
    xn = y ^ tbl(Tb, 0u, y);
    o = temper_convert<FMT>(xn, temper_index(xq), Tb);
}

// One full row (all N columns to one request, format FMT) with the output
// alignment A of its first column.  pk/tl hold the current step's prefetched
// pick-ups and tail word; carry the A outputs of the previous step that
// precede this row's first aligned chunk (meaningful in lane 0); `fresh`
// marks the first step of a batch (nothing before it may be written).
template <int NS, int FMT, int A>
__device__ __forceinline__ void wide_row(uint32_t (&r)[NS][4], uint32_t* S, const WideLane<NS>& L,
                                         const RowP& P, uint32_t R, uint32_t lane,
                                         const uint32_t* __restrict__ Tb, uint32_t (&pk)[5],
                                         uint32_t& tl, uint32_t (&carry)[3], bool& fresh,
                                         uint32_t* ow)
{
    const uint32_t V_last = P.n - 128u * (NS - 1);   // valid columns of the last step
#pragma unroll
    for (int s = 0; s < NS; ++s) {
        const int sn = (s + 1 < NS) ? s + 1 : 0;   // next step (the next row's first)
        uint32_t pkn[5], tln;
#pragma unroll
        for (int j = 0; j < 5; ++j)
            pkn[j] = S[L.pa[sn][j]];
        tln = S[L.ta[sn]];

        uint32_t xn[4], o[4];
#pragma unroll
        for (int k = 0; k < 4; ++k) {
            uint32_t x1;
            if (k == 3)
                x1 = tl;
            else if (s + 1 < NS)
                x1 = r[s][k + 1];
            else
                x1 = (uint32_t)k < L.kl ? r[s][k + 1] : tl;
            wide_column<FMT>(r[s][k], x1, pk[k + 1], pk[k], P, Tb, xn[k], o[k]);
        }

        // state: registers and the shared row
        const uint32_t V = (s + 1 < NS) ? 128u : V_last;
#pragma unroll
        for (int k = 0; k < 4; ++k) {
            if (s + 1 < NS || 4u * lane + (uint32_t)k < V) {
                r[s][k] = xn[k];
                S[(uint32_t)k * R + 32u * s + lane] = xn[k];
            }
        }

        // output: the aligned chunk that starts A elements before this lane's
        // first output
        uint32_t ch[4], rot[3] = {0u, 0u, 0u};
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            if (j >= A) {
                ch[j] = o[j - A];
            } else {
                const uint32_t v = __shfl_sync(MTGP_FULL, o[4 - A + j], (lane + 31u) & 31u);
                rot[j] = v;
                ch[j] = lane == 0u ? carry[j] : v;
            }
        }
        uint32_t* cp = ow + 128u * s + 4u * lane - (uint32_t)A;
        const bool complete = (s + 1 < NS) || (4u * lane + 4u - (uint32_t)A <= V);
        if (A > 0 && fresh && lane == 0u) {
#pragma unroll
            for (int j = A; j < 4; ++j)
                __stcs(cp + j, ch[j]);
        } else if (complete) {
            __stcs(reinterpret_cast<uint4*>(cp), make_uint4(ch[0], ch[1], ch[2], ch[3]));
        }
        if (s + 1 < NS) {
#pragma unroll
            for (int j = 0; j < A; ++j)
                carry[j] = rot[j];
        } else {
            // the (V + A) mod 4 outputs after the last complete chunk form the
            // head of the next row's first chunk: lane nch assembled them
            const uint32_t nch = (V + (uint32_t)A) >> 2;
            uint32_t c0 = __shfl_sync(MTGP_FULL, ch[0], nch & 31u);
            uint32_t c1 = __shfl_sync(MTGP_FULL, ch[1], nch & 31u);
            uint32_t c2 = __shfl_sync(MTGP_FULL, ch[2], nch & 31u);
            if (nch >= 32u) {   // V + A >= 128: they are lane 31's last outputs
                c0 = rot[0];
                c1 = rot[1];
                c2 = rot[2];
            }
            carry[0] = c0;
            carry[1] = c1;
            carry[2] = c2;
        }
        fresh = false;
        __syncwarp();
#pragma unroll
        for (int j = 0; j < 5; ++j)
            pk[j] = pkn[j];
        tl = tln;
    }
}

// nfull consecutive full rows of one request, software-pipelined; ow points
// at the output of the first row's column 0.
template <int NS, int FMT>
__device__ __forceinline__ void wide_rows(uint32_t (&r)[NS][4], uint32_t* S, const WideLane<NS>& L,
                                          const RowP& P, uint32_t R, uint32_t lane,
                                          const uint32_t* __restrict__ Tb, uint32_t nfull, uint32_t* ow)
{
    uint32_t pk[5], tl;
#pragma unroll
    for (int j = 0; j < 5; ++j)
        pk[j] = S[L.pa[0][j]];
    tl = S[L.ta[0]];
    uint32_t carry[3] = {0u, 0u, 0u};
    bool fresh = true;
    uint32_t a = (uint32_t)(reinterpret_cast<uintptr_t>(ow) >> 2) & 3u;
    const uint32_t nmod = P.n & 3u;
    for (uint32_t q = 0; q < nfull; ++q, ow += P.n) {
        switch (a) {
        case 0: wide_row<NS, FMT, 0>(r, S, L, P, R, lane, Tb, pk, tl, carry, fresh, ow); break;
        case 1: wide_row<NS, FMT, 1>(r, S, L, P, R, lane, Tb, pk, tl, carry, fresh, ow); break;
        case 2: wide_row<NS, FMT, 2>(r, S, L, P, R, lane, Tb, pk, tl, carry, fresh, ow); break;
        default: wide_row<NS, FMT, 3>(r, S, L, P, R, lane, Tb, pk, tl, carry, fresh, ow); break;
        }
        a = (a + nmod) & 3u;
    }
    // the last a outputs of the batch (the head of a chunk no row completes)
    if (lane == 0u) {
        for (uint32_t j = 0; j < a; ++j)
            __stcs(ow - a + j, carry[j]);
    }
}

// A row whose outputs need per-lane request lookups (it crosses into the
// next request) or that ends the stream (n_valid < N columns).  Not
// pipelined: each step reads, passes a barrier, then writes.
template <int NS>
__device__ __forceinline__ void wide_row_slow(uint32_t (&r)[NS][4], uint32_t* S, const WideLane<NS>& L,
                                              const RowP& P, uint32_t R, uint32_t lane,
                                              const uint32_t* __restrict__ Tb, uint32_t n_valid,
                                              uint64_t row_g, const Segment* __restrict__ segs,
                                              uint32_t s_first, uint32_t s_end,
                                              uint32_t* __restrict__ out)
{
#pragma unroll
    for (int s = 0; s < NS; ++s) {
        if (128u * s >= n_valid)
            break;
        uint32_t pk[5];
#pragma unroll
        for (int j = 0; j < 5; ++j)
            pk[j] = S[L.pa[s][j]];
        const uint32_t tl = S[L.ta[s]];
        uint32_t xn[4], ou[4], of[4];
#pragma unroll
        for (int k = 0; k < 4; ++k) {
            uint32_t x1;
            if (k == 3)
                x1 = tl;
            else if (s + 1 < NS)
                x1 = r[s][k + 1];
            else
                x1 = (uint32_t)k < L.kl ? r[s][k + 1] : tl;
            wide_column<0>(r[s][k], x1, pk[k + 1], pk[k], P, Tb, xn[k], ou[k]);
            of[k] = wide_output<1>(xn[k], pk[k], Tb);
        }
        __syncwarp();
#pragma unroll
        for (int k = 0; k < 4; ++k) {
            const uint32_t c = 128u * s + 4u * lane + (uint32_t)k;
            if (c < n_valid) {
                r[s][k] = xn[k];
                S[(uint32_t)k * R + 32u * s + lane] = xn[k];
                slow_store(ou[k], of[k], row_g + c, segs, s_first, s_end, out);
            }
        }
        __syncwarp();
    }
}

// Advances one stream (this warp alone) by the segments [s_begin, s_end).
template <int NS>
__device__ __forceinline__ void wide_item(const KParams& KP, const RowP& P, uint32_t* __restrict__ g,
                                          uint32_t* S, const Segment* __restrict__ segs,
                                          uint32_t s_begin, uint32_t s_end, uint32_t* __restrict__ out,
                                          uint32_t lane, const uint32_t* __restrict__ Tb)
{
    const uint32_t N = P.n;
    const uint32_t R = (N + 3u) >> 2;
    WideLane<NS> L;
    wide_lane_setup<NS>(L, P, R, lane);

    // stage in: the lane's own four columns of each step straight from the
    // HBM row (16-byte loads; rows are padded to a multiple of 4 words),
    // then into the shared row
    uint32_t r[NS][4];
#pragma unroll
    for (int s = 0; s < NS; ++s) {
        const uint32_t base = 128u * s + 4u * lane;
        uint4 v = make_uint4(0u, 0u, 0u, 0u);
        if (base < KP.np)
            v = *reinterpret_cast<const uint4*>(g + base);
        r[s][0] = v.x;
        r[s][1] = v.y;
        r[s][2] = v.z;
        r[s][3] = v.w;
#pragma unroll
        for (int k = 0; k < 4; ++k)
            if (base + (uint32_t)k < N)
                S[(uint32_t)k * R + 32u * s + lane] = r[s][k];
    }
    __syncwarp();

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
            uint32_t* ow = out + sg.out_off + (row - sg.g_start);
            if (sg.fmt == 0)
                wide_rows<NS, 0>(r, S, L, P, R, lane, Tb, nfull, ow);
            else if (sg.fmt == 1)
                wide_rows<NS, 1>(r, S, L, P, R, lane, Tb, nfull, ow);
            else
                wide_rows<NS, 2>(r, S, L, P, R, lane, Tb, nfull, ow);
            __syncwarp();
            row += (uint64_t)nfull * N;
        } else {
            const uint64_t left = total - row;
            const uint32_t n_valid = left < (uint64_t)N ? (uint32_t)left : N;
            wide_row_slow<NS>(r, S, L, P, R, lane, Tb, n_valid, row, segs, s, s_end, out);
            row += N;
        }
    }

    // stage out: oldest word first, x_total .. x_{total+N-1}; the column of
    // x_{total+j} is (total + j) mod N
    const uint32_t phase = (uint32_t)(total % N);
    for (uint32_t j = lane; j < N; j += 32u) {
        uint32_t c = phase + j;
        c = c >= N ? c - N : c;
        g[j] = S[quad_index(c, R)];
    }
    __syncwarp();
}

// Persistent kernel: every warp claims items (one stream each, longest first)
// from the table and advances each alone.
template <int NS, int G>
__global__ void __launch_bounds__(G * 32) mtgp_wide_kernel(const KParams P, uint32_t* __restrict__ states,
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
    __shared__ __align__(64) uint32_t Tb[G][48];
    (void)n_coop;
    const uint32_t lane = threadIdx.x & 31u;
    const uint32_t warp = threadIdx.x >> 5;
    if (threadIdx.x < 16) {
        Tb[0][threadIdx.x] = P.rec[threadIdx.x];
        Tb[0][16 + threadIdx.x] = P.tmp[threadIdx.x];
        Tb[0][32 + threadIdx.x] = P.flt[threadIdx.x];
    }
    __syncthreads();
    const RowP R0 = {P.n, P.mask, P.pos, P.sh1, P.sh2, P.mirror};
    uint32_t* S = smem + warp * wide_smem_words(P.n);
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
        const uint64_t t0 = trace ? global_ns() : 0;
        if (sets) {
            const KSet& ks = sets[set_of[w.stream]];
            const RowP R = {P.n, P.mask, ks.pos, ks.sh1, ks.sh2, ks.mirror};
            if (lane < 16u) {
                Tb[warp][lane] = ks.rec[lane];
                Tb[warp][16u + lane] = ks.tmp[lane];
                Tb[warp][32u + lane] = ks.flt[lane];
            }
            __syncwarp();
            wide_item<NS>(P, R, states + (size_t)w.stream * P.np, S, segs, w.seg_begin,
                          w.seg_begin + w.nseg, out, lane, Tb[warp]);
        } else {
            wide_item<NS>(P, R0, states + (size_t)w.stream * P.np, S, segs, w.seg_begin,
                          w.seg_begin + w.nseg, out, lane, Tb[0]);
        }
        if (trace && lane == 0)
            trace_item(trace, it, t0, segs, w);
    }
}

}  // namespace mtgp

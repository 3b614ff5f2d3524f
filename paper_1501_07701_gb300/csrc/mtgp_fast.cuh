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
//     row S[0..N), with a mirror S[N..N+32) of columns 0..31 and a guard
//     S[-1] of column N-1.  Words i+1, i+pos and i+pos-1 of 32 consecutive
//     columns are then plain conflict-free loads at S[c+1], S[c+pos],
//     S[c+pos-1] with no modulo (the mirror supplies the wrapped columns).
//   * The recursion and tempering tables live in lane registers (lane l holds
//     entry l & 15); a lookup is one shuffle whose source lane is the index
//     itself (shfl uses the low five bits of the lane operand).
//   * Shifts are done as integer multiplies (x << s = x * 2^s and x >> s =
//     high word of x * 2^(32-s)), which run on the FMA pipe and leave the ALU
//     pipe to the XORs.
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

__device__ __forceinline__ void cp_async_wait_all()
{
    asm volatile("cp.async.commit_group;\n" ::: "memory");
    asm volatile("cp.async.wait_group 0;\n" ::: "memory");
}

// Multipliers for the shifts (sh1, sh2 in 1..31): y << sh1 = y * m1,
// x >> sh2 = umulhi(x, m2).
struct Shifts {
    uint32_t m1, m2;
};

__device__ __forceinline__ Shifts make_shifts(const KParams& P)
{
    Shifts s;
    s.m1 = 1u << P.sh1;
    s.m2 = 1u << (32u - P.sh2);
    return s;
}

// The new word of one column from words i (own register), i+1, i+pos.
__device__ __forceinline__ uint32_t recur(uint32_t xi, uint32_t x1, uint32_t xp, uint32_t mask,
                                          const Shifts& sh, uint32_t tR)
{
    uint32_t y = (xi & mask) ^ x1;
    y = y ^ (y * sh.m1) ^ __umulhi(xp, sh.m2);
    return y ^ __shfl_sync(MTGP_FULL, tR, y);
}

// Tempering index from word i+pos-1: fold >> 16 then >> 8 (low four bits
// are used; the shuffle ignores bit 4 because the tables repeat).
__device__ __forceinline__ uint32_t temper_index(uint32_t xq)
{
    const uint32_t t = xq ^ __umulhi(xq, 1u << 16);
    return t ^ __umulhi(t, 1u << 24);
}

// Output conversion from the new word v and the tempering index ti.
//   FMT 0: v ^ TMP[ti]
//   FMT 1: (v >> 9) ^ FLT[ti]   == 0x3F800000 | ((v ^ TMP[ti]) >> 9)
//   FMT 2: the FMT 1 float minus 1.0f (exact: Sterbenz)
template <int FMT>
__device__ __forceinline__ uint32_t temper_convert(uint32_t v, uint32_t ti, uint32_t tT, uint32_t tF)
{
    if (FMT == 0)
        return v ^ __shfl_sync(MTGP_FULL, tT, ti);
    const uint32_t b = __umulhi(v, 1u << 23) ^ __shfl_sync(MTGP_FULL, tF, ti);
    if (FMT == 1)
        return b;
    return __float_as_uint(__uint_as_float(b) - 1.0f);
}

// Per-lane output of the slow path: the lane finds its request and format.
// ou / of are the u32 and [1,2) outputs, both computed while the warp was
// converged (they need shuffles); this function itself is lane-local.
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
// Every shuffle (table lookups) runs in the read phase, under conditions that
// are uniform across the warp; the write phase is lane-predicated and holds
// no warp-synchronous instruction.
// ===========================================================================
template <int M, int K, int WG, int FMT, bool SLOW>
__device__ __forceinline__ void gen_row(uint32_t (&r)[(M + WG - 1) / WG], uint32_t* __restrict__ S,
                                        uint32_t* __restrict__ Sw, uint32_t* __restrict__ ow,
                                        const KParams& P, const Shifts& sh, uint32_t warp,
                                        uint32_t lane, uint32_t tR, uint32_t tT, uint32_t tF,
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
        uint32_t xn[PER], o1[PER], o2[PER];
#pragma unroll
        for (int i = 0; i < PER; ++i) {
            const int j = s0 / WG + i;
            const uint32_t m = (uint32_t)(s0 + i * WG) + (WG > 1 ? warp : 0u);
            if (j < J && m < (uint32_t)M) {   // uniform across the warp
                const int off = 32 * (s0 + i * WG);            // static part of 32m
                uint32_t sp = P.pos + 32u * m;                  // (pos + 32m) mod N
                sp = sp >= P.n ? sp - P.n : sp;
                const uint32_t* q = S + sp + lane;
                xn[i] = recur(r[j], Sw[off + 1], q[0], P.mask, sh, tR);
                const uint32_t ti = temper_index(q[-1]);
                if (SLOW) {
                    o1[i] = temper_convert<0>(xn[i], ti, tT, tF);
                    o2[i] = temper_convert<1>(xn[i], ti, tT, tF);
                } else {
                    o1[i] = temper_convert<FMT>(xn[i], ti, tT, tF);
                }
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
                    if (m == 0)
                        S[P.n + lane] = xn[i];
                    if (col == P.n - 1u)
                        S[-1] = xn[i];
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

// Advances one stream by the segments [s_begin, s_end) of the work table.
// WG warps take part (WG = 1: this warp alone; WG = G: the whole CTA).
template <int M, int K, int WG>
__device__ __forceinline__ void run_item(const KParams& P, uint32_t* __restrict__ g, uint32_t* __restrict__ S,
                                         const Segment* __restrict__ segs, uint32_t s_begin,
                                         uint32_t s_end, uint32_t* __restrict__ out, uint32_t warp,
                                         uint32_t lane, uint32_t tR, uint32_t tT, uint32_t tF)
{
    constexpr int J = (M + WG - 1) / WG;
    const uint32_t N = P.n;
    const uint32_t tid = WG > 1 ? threadIdx.x : lane;
    const uint32_t wk = WG > 1 ? warp : 0u;
    const Shifts sh = make_shifts(P);
    const uint32_t last_lane = (N - 1u) & 31u;   // lane of column N-1 (group M-1)

    // stage in: the state row (HBM) -> S through 16-byte cp.async
    for (uint32_t c = tid; c < (P.np >> 2); c += 32u * WG)
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
    const uint32_t mirror = S[lane];
    const uint32_t guard = S[N - 1u];
    if (WG > 1)
        __syncthreads();
    else
        __syncwarp();
    if (wk == 0) {
        S[N + lane] = mirror;
        if (lane == 0)
            S[-1] = guard;
    }
    if (WG > 1)
        __syncthreads();
    else
        __syncwarp();

    uint32_t* Sw = S + 32u * wk + lane;
    const Segment last = segs[s_end - 1u];
    const uint64_t total = last.g_start + last.count;
    uint32_t s = s_begin;
    for (uint64_t row = 0; row < total; row += N) {
        while (segs[s].g_start + segs[s].count <= row)
            ++s;
        const Segment sg = segs[s];
        const uint64_t left = total - row;
        const uint32_t n_valid = left < (uint64_t)N ? (uint32_t)left : N;
        if (n_valid == N && row + N <= sg.g_start + sg.count) {
            uint32_t* ow = out + sg.out_off + (row - sg.g_start) + 32u * wk + lane;
            if (sg.fmt == 0)
                gen_row<M, K, WG, 0, false>(r, S, Sw, ow, P, sh, wk, lane, tR, tT, tF, last_lane, N, row,
                                            segs, s, s_end, out);
            else if (sg.fmt == 1)
                gen_row<M, K, WG, 1, false>(r, S, Sw, ow, P, sh, wk, lane, tR, tT, tF, last_lane, N, row,
                                            segs, s, s_end, out);
            else
                gen_row<M, K, WG, 2, false>(r, S, Sw, ow, P, sh, wk, lane, tR, tT, tF, last_lane, N, row,
                                            segs, s, s_end, out);
        } else {
            gen_row<M, K, WG, 0, true>(r, S, Sw, nullptr, P, sh, wk, lane, tR, tT, tF, last_lane, n_valid,
                                       row, segs, s, s_end, out);
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
                                                           uint32_t* __restrict__ out, int* __restrict__ err)
{
    extern __shared__ __align__(16) uint32_t smem[];
    __shared__ uint32_t s_claim;
    const uint32_t lane = threadIdx.x & 31u;
    const uint32_t warp = threadIdx.x >> 5;
    const uint32_t tR = P.rec[lane & 15u];
    const uint32_t tT = P.tmp[lane & 15u];
    const uint32_t tF = P.flt[lane & 15u];

    for (;;) {
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
        run_item<M, K, G>(P, states + (size_t)w.stream * P.np, smem + 4, segs, w.seg_begin,
                          w.seg_begin + w.nseg, out, warp, lane, tR, tT, tF);
    }

    uint32_t* S = smem + warp * fast_smem_words(P.n) + 4;
    for (;;) {
        uint32_t it = 0;
        if (lane == 0)
            it = n_coop + atomicAdd(&counters[1], 1u);
        it = __shfl_sync(MTGP_FULL, it, 0);
        if (it >= n_items)
            break;
        const WorkItem w = items[it];
        if (w.stream >= n_streams || w.nseg == 0) {
            if (lane == 0)
                atomicOr(err, 1);
            continue;
        }
        run_item<M, K, 1>(P, states + (size_t)w.stream * P.np, S, segs, w.seg_begin,
                          w.seg_begin + w.nseg, out, warp, lane, tR, tT, tF);
    }
}

}  // namespace mtgp

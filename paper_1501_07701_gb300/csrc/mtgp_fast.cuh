// Register-resident MTGP32 generation kernel for sm_103a.
//
// One warp advances one stream at a time (the paper's "PRNG per block of
// threads", Sec. 2, with the state in on-chip storage while it is advanced
// and in global memory between launches).  Layout of a stream's state while
// it is on chip:
//
//   * The sequence is cut into rows of N words: column c of row q holds
//     x_{qN + c}.  Computing row q+1 column c needs (row q, c) and
//     (row q, c+1) [the words i and i+1 of the recurrence] and the word i+pos,
//     which is (row q, c+pos) when c+pos < N and (row q+1, c+pos-N) otherwise;
//     the tempering word i+pos-1 likewise.  So at every moment a state needs
//     only the latest value of each column.
//   * Lane l of the warp keeps columns 32m + l, m = 0..M-1 (M = ceil(N/32)),
//     in registers r[m]: word i is the lane's own register and word i+1 is
//     one shuffle away.
//   * The latest value of every column is also published in a per-warp
//     shared-memory array S[0..N) (plus a mirror S[N..N+32) of columns 0..31
//     and a guard S[-1] of column N-1), from which the words i+pos and
//     i+pos-1 are read for 32 consecutive columns at once without a modulo.
//   * The recursion and tempering tables live in lane registers (lane l holds
//     entry l & 15); a lookup is one shuffle whose source lane is the index
//     itself (shfl uses the low five bits of the lane operand).
//
// A sub-step m computes columns 32m..32m+31 of the next row (one new word
// per lane).  K consecutive sub-steps form one parallel step of 32K words:
// all of them read only words produced before the step when 32K <= N - pos
// (the block-parallel window of the method), so the step reads everything,
// then writes everything, with one warp barrier in between.
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

// Output conversion from the new word v and the tempering index ti.
//   FMT 0: v ^ TMP[ti]
//   FMT 1: (v >> 9) ^ FLT[ti]   == 0x3F800000 | ((v ^ TMP[ti]) >> 9)
//   FMT 2: the FMT 1 float minus 1.0f (exact: Sterbenz)
template <int FMT>
__device__ __forceinline__ uint32_t temper_convert(uint32_t v, uint32_t ti, uint32_t tT, uint32_t tF)
{
    if (FMT == 0)
        return v ^ __shfl_sync(MTGP_FULL, tT, ti);
    const uint32_t b = (v >> 9) ^ __shfl_sync(MTGP_FULL, tF, ti);
    if (FMT == 1)
        return b;
    return __float_as_uint(__uint_as_float(b) - 1.0f);
}

// Pick-up offset of sub-step m: (pos + 32m) mod N (pos < N and 32m < N).
__device__ __forceinline__ uint32_t pick_offset(uint32_t pos, uint32_t n, int m)
{
    const uint32_t sp = pos + 32u * (uint32_t)m;
    return sp >= n ? sp - n : sp;
}

// One full row (N new words) inside a single request: output goes to
// orow[0..N).
template <int M, int K, int FMT>
__device__ __forceinline__ void fast_row(uint32_t (&r)[M], uint32_t* __restrict__ S,
                                         uint32_t* __restrict__ orow, const KParams& P,
                                         uint32_t lane, uint32_t tR, uint32_t tT, uint32_t tF,
                                         uint32_t src_last, uint32_t last_lane)
{
    const uint32_t src_next = (lane + 1) & 31u;
#pragma unroll
    for (int m0 = 0; m0 < M; m0 += K) {
        uint32_t xn[K], ov[K];
#pragma unroll
        for (int t = 0; t < K; ++t) {
            const int m = m0 + t;
            if (m < M) {
                // word i+1: column 32m+l+1 -> lane l+1, or lane 0's next
                // register for l = 31; the row's last column takes the new
                // column 0 (lane 0's r[0], already advanced).
                const uint32_t nb = (lane == 0) ? r[(m + 1 < M) ? m + 1 : 0] : r[m];
                const uint32_t x1 = __shfl_sync(MTGP_FULL, nb, (m + 1 < M) ? src_next : src_last);
                const uint32_t* q = S + pick_offset(P.pos, P.n, m) + lane;
                const uint32_t xp = q[0];    // word i+pos
                const uint32_t xq = q[-1];   // word i+pos-1
                uint32_t y = (r[m] & P.mask) ^ x1;
                y ^= (y << P.sh1) ^ (xp >> P.sh2);
                const uint32_t v = y ^ __shfl_sync(MTGP_FULL, tR, y);
                uint32_t ti = xq ^ (xq >> 16);
                ti ^= ti >> 8;
                xn[t] = v;
                ov[t] = temper_convert<FMT>(v, ti, tT, tF);
            }
        }
        __syncwarp();
#pragma unroll
        for (int t = 0; t < K; ++t) {
            const int m = m0 + t;
            if (m < M) {
                if (m < M - 1 || lane <= last_lane) {
                    r[m] = xn[t];
                    S[32 * m + lane] = xn[t];
                    __stcs(orow + 32 * m + lane, ov[t]);
                }
                if (m == 0)
                    S[P.n + lane] = xn[t];
                if (m == M - 1 && lane == last_lane)
                    S[-1] = xn[t];
            }
        }
        __syncwarp();
    }
}

// A row that is partial (n_valid < N columns) or crosses request
// boundaries: every lane finds its own request and format.
template <int M, int K>
__device__ __forceinline__ void slow_row(uint32_t (&r)[M], uint32_t* __restrict__ S, const KParams& P,
                                      uint32_t lane, uint32_t tR, uint32_t tT, uint32_t tF,
                                      uint32_t src_last, uint32_t last_lane, uint32_t n_valid,
                                      uint64_t row_g, const Segment* __restrict__ segs,
                                      uint32_t s_first, uint32_t s_end, uint32_t* __restrict__ out)
{
    const uint32_t src_next = (lane + 1) & 31u;
#pragma unroll
    for (int m0 = 0; m0 < M; m0 += K) {
        if (32u * (uint32_t)m0 >= n_valid)
            break;
        uint32_t xn[K], ou[K], of[K];
#pragma unroll
        for (int t = 0; t < K; ++t) {
            const int m = m0 + t;
            if (m < M) {
                const uint32_t nb = (lane == 0) ? r[(m + 1 < M) ? m + 1 : 0] : r[m];
                const uint32_t x1 = __shfl_sync(MTGP_FULL, nb, (m + 1 < M) ? src_next : src_last);
                const uint32_t* q = S + pick_offset(P.pos, P.n, m) + lane;
                const uint32_t xp = q[0];
                const uint32_t xq = q[-1];
                uint32_t y = (r[m] & P.mask) ^ x1;
                y ^= (y << P.sh1) ^ (xp >> P.sh2);
                const uint32_t v = y ^ __shfl_sync(MTGP_FULL, tR, y);
                uint32_t ti = xq ^ (xq >> 16);
                ti ^= ti >> 8;
                xn[t] = v;
                ou[t] = temper_convert<0>(v, ti, tT, tF);
                of[t] = temper_convert<1>(v, ti, tT, tF);
            }
        }
        __syncwarp();
#pragma unroll
        for (int t = 0; t < K; ++t) {
            const int m = m0 + t;
            if (m < M) {
                const uint32_t col = 32u * (uint32_t)m + lane;
                if (col < n_valid) {   // n_valid <= N, so col is a real column
                    r[m] = xn[t];
                    S[col] = xn[t];
                    if (m == 0)
                        S[P.n + lane] = xn[t];
                    if (col == P.n - 1)
                        S[-1] = xn[t];
                    const uint64_t g = row_g + col;
                    uint32_t s = s_first;
                    while (s + 1 < s_end && g >= segs[s + 1].g_start)
                        ++s;
                    const Segment sg = segs[s];
                    uint32_t o = ou[t];
                    if (sg.fmt == 1)
                        o = of[t];
                    else if (sg.fmt == 2)
                        o = __float_as_uint(__uint_as_float(of[t]) - 1.0f);
                    out[sg.out_off + (g - sg.g_start)] = o;
                }
            }
        }
        __syncwarp();
    }
    (void)last_lane;
}

template <int M, int K>
__global__ void __launch_bounds__(256) mtgp_fast_kernel(const KParams P, uint32_t* __restrict__ states,
                                                        uint32_t n_streams,
                                                        const WorkItem* __restrict__ items,
                                                        const Segment* __restrict__ segs,
                                                        uint32_t n_items, uint32_t* __restrict__ counter,
                                                        uint32_t* __restrict__ out, int* __restrict__ err)
{
    extern __shared__ __align__(16) uint32_t smem[];
    const uint32_t lane = threadIdx.x & 31u;
    const uint32_t warp = threadIdx.x >> 5;
    const uint32_t N = P.n;
    uint32_t* S = smem + warp * fast_smem_words(N) + 4;
    const uint32_t tR = P.rec[lane & 15u];
    const uint32_t tT = P.tmp[lane & 15u];
    const uint32_t tF = P.flt[lane & 15u];
    const uint32_t last_lane = (N - 1u) & 31u;   // lane of column N-1 in sub-step M-1
    const uint32_t src_last = (lane == last_lane) ? 0u : ((lane + 1u) & 31u);

    for (;;) {
        uint32_t it = 0;
        if (lane == 0)
            it = atomicAdd(counter, 1u);
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

        // Stage in: the N-word state row (HBM) -> S, 16-byte cp.async chunks.
        for (uint32_t c = lane; c < (P.np >> 2); c += 32u)
            cp_async16(S + 4u * c, g + 4u * c);
        cp_async_wait_all();
        __syncwarp();
        uint32_t r[M];
#pragma unroll
        for (int m = 0; m < M; ++m) {
            const uint32_t c = 32u * (uint32_t)m + lane;
            r[m] = c < N ? S[c] : 0u;
        }
        const uint32_t mirror = S[lane];
        const uint32_t guard = S[N - 1u];
        __syncwarp();
        S[N + lane] = mirror;
        if (lane == 0)
            S[-1] = guard;
        __syncwarp();

        const uint32_t s_end = w.seg_begin + w.nseg;
        const Segment last = segs[s_end - 1u];
        const uint64_t total = last.g_start + last.count;
        uint32_t s = w.seg_begin;
        for (uint64_t row = 0; row < total; row += N) {
            while (segs[s].g_start + segs[s].count <= row)
                ++s;
            const Segment sg = segs[s];
            const uint64_t left = total - row;
            const uint32_t n_valid = left < (uint64_t)N ? (uint32_t)left : N;
            if (n_valid == N && row + N <= sg.g_start + sg.count) {
                uint32_t* orow = out + sg.out_off + (row - sg.g_start);
                if (sg.fmt == 0)
                    fast_row<M, K, 0>(r, S, orow, P, lane, tR, tT, tF, src_last, last_lane);
                else if (sg.fmt == 1)
                    fast_row<M, K, 1>(r, S, orow, P, lane, tR, tT, tF, src_last, last_lane);
                else
                    fast_row<M, K, 2>(r, S, orow, P, lane, tR, tT, tF, src_last, last_lane);
            } else {
                slow_row<M, K>(r, S, P, lane, tR, tT, tF, src_last, last_lane, n_valid, row, segs, s,
                               s_end, out);
            }
        }

        // Stage out: oldest word first, x_total .. x_{total+N-1}; column of
        // x_{total+j} is (total + j) mod N.
        const uint32_t phase = (uint32_t)(total % N);
        for (uint32_t j = lane; j < N; j += 32u) {
            uint32_t c = phase + j;
            c = c >= N ? c - N : c;
            g[j] = S[c];
        }
        __syncwarp();
    }
}

}  // namespace mtgp

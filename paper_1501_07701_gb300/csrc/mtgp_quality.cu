// Data reductions behind the paper's two failing BigCrush tests (Sec. 4.2),
// run on the GPU over sequences of 32-bit outputs that are already in device
// memory (for instance the output of mtgp_generate_u32):
//
//   test 35, the gap test: a value visits [0, 2^-b) when the b bits after its
//   r dropped leading bits are zero; a gap is the run of non-visits before a
//   visit, counted from the start of its sequence; the reduction is the
//   histogram of gap lengths (lengths >= t pooled).
//
//   test 100, Hamming-weight independence: the s bits after the r dropped
//   leading bits of each value form a bit string cut into L-bit blocks; each
//   pair of successive blocks is counted in a table of (weight class of the
//   first, weight class of the second).
//
// Both read every value once and are bound by HBM read bandwidth.  The
// chi-square statistics are computed on the host from the counts.
#include <algorithm>
#include <vector>

#include "mtgp_runtime.h"

using namespace mtgp;

namespace {

constexpr uint32_t kChunk = 1u << 14;       // values per gap-test work unit
constexpr uint32_t kMaxT = 1023;            // largest pooled gap class
constexpr uint32_t kMaxClasses = 16;        // largest number of weight classes
constexpr int kWarps = 8;                   // warps per CTA of both kernels

// Per chunk: the run of non-visits before its first visit (the whole length
// if it has none), the run after its last visit, whether it has a visit, and
// its length.  Gaps that cross chunk boundaries are completed from these by
// the stitch kernel.
struct GapEdge {
    uint32_t prefix;
    uint32_t suffix;
    uint32_t has_visit;
    uint32_t pad;   // chunk length
};

// Work units: sequence i is cut into ceil(counts[i] / kChunk) chunks; chunk
// c of the launch is found from the prefix sums of those chunk counts.  Warps
// claim runs of `run` consecutive chunks from an atomic counter, so a warp's
// consecutive chunks mostly share a sequence and its histogram, which is
// flushed to global memory only when the sequence changes.  Per group of 32
// consecutive values the visits form a ballot mask B; a visiting lane's gap
// is the distance to the nearest lower visiting lane, or the carried run D
// plus its lane index if it is the group's first visit (the first visit of a
// chunk is left to the stitch kernel); both cases are one expression,
// gap = lane - 1 - prev with prev = -1 - D when no lower lane visits.  Loads
// run a round ahead of the scan: the kG groups of the next round are in
// flight while the current round is scanned, and rounds with every value
// present are scanned without per-lane bounds checks.  The ballot and every
// shuffle run in warp-uniform control flow; the per-lane branch holds only
// shared-memory atomics.
constexpr uint32_t kG = 8;      // groups of 32 values per load round

__device__ __forceinline__ void gap_flush(uint32_t* h, uint32_t t, unsigned long long* hs, uint32_t lane)
{
    __syncwarp();
    for (uint32_t i = lane; i <= t; i += 32u) {
        if (h[i])
            atomicAdd(hs + i, (unsigned long long)h[i]);
        h[i] = 0u;
    }
    __syncwarp();
}

// Sequence holding chunk c: the last i with chunk_base[i] <= c.
__device__ __forceinline__ uint32_t chunk_seq(const uint64_t* __restrict__ chunk_base, uint32_t n_seq,
                                              uint64_t c)
{
    uint32_t lo = 0, hi = n_seq;
    while (hi - lo > 1u) {
        const uint32_t mid = (lo + hi) >> 1;
        if (chunk_base[mid] <= c)
            lo = mid;
        else
            hi = mid;
    }
    return lo;
}

__global__ void __launch_bounds__(kWarps * 32) mtgp_gap_kernel(const uint32_t* __restrict__ values,
                                                              const uint64_t* __restrict__ seq_start,
                                                              const uint64_t* __restrict__ counts,
                                                              const uint64_t* __restrict__ chunk_base,
                                                              uint32_t n_seq, uint64_t n_chunks,
                                                              uint32_t run, uint32_t fmask, uint32_t t,
                                                              unsigned long long* __restrict__ claim,
                                                              unsigned long long* __restrict__ hist,
                                                              GapEdge* __restrict__ edges)
{
    extern __shared__ uint32_t h_all[];   // kWarps histograms of t + 1 counts
    const uint32_t lane = threadIdx.x & 31u, warp = threadIdx.x >> 5;
    const uint32_t lower = (1u << lane) - 1u;   // lanes below this one
    uint32_t* h = h_all + warp * (t + 1u);
    for (uint32_t i = lane; i <= t; i += 32u)
        h[i] = 0u;
    __syncwarp();
    uint32_t cur = 0xFFFFFFFFu;
    for (;;) {
        unsigned long long c0 = 0;
        if (lane == 0)
            c0 = atomicAdd(claim, (unsigned long long)run);
        c0 = __shfl_sync(0xFFFFFFFFu, c0, 0);
        if (c0 >= n_chunks)
            break;
        const uint64_t c1 = min((uint64_t)c0 + run, n_chunks);
        uint32_t seq = chunk_seq(chunk_base, n_seq, c0);
        for (uint64_t c = c0; c < c1; ++c) {
            while (c >= chunk_base[seq + 1u])
                ++seq;
            if (seq != cur) {
                if (cur != 0xFFFFFFFFu)
                    gap_flush(h, t, hist + (size_t)cur * (t + 1u), lane);
                cur = seq;
            }
            const uint64_t off = (c - chunk_base[seq]) * kChunk;
            const uint64_t left = counts[seq] - off;
            const uint32_t len = left < kChunk ? (uint32_t)left : kChunk;
            const uint32_t* v = values + seq_start[seq] + off;
            uint32_t D = 0, P = 0;
            bool seen = false;
            uint32_t xa[kG];
#pragma unroll
            for (uint32_t g = 0; g < kG; ++g) {
                const uint32_t idx = 32u * g + lane;
                xa[g] = idx < len ? __ldcs(v + idx) : 0u;
            }
            // scans one round; `full`: all 32 kG values are present (no per-lane checks)
            auto scan = [&](const uint32_t (&x)[kG], uint32_t base0, bool full) {
#pragma unroll
                for (uint32_t g = 0; g < kG; ++g) {
                    const uint32_t base = base0 + 32u * g;
                    if (!full && base >= len)
                        break;
                    const bool in = (x[g] & fmask) == 0u && (full || base + lane < len);
                    const uint32_t B = __ballot_sync(0xFFFFFFFFu, in);
                    const uint32_t below = B & lower;
                    // position of the previous visit (-1 - D: D non-visits before this group)
                    const int prev = below ? 31 - __clz(below) : -1 - (int)D;
                    if (in && (below || seen))
                        atomicAdd(&h[min((uint32_t)((int)lane - 1 - prev), t)], 1u);
                    const uint32_t nv = full ? 32u : min(32u, len - base);
                    const uint32_t hiB = 31u - __clz(B);
                    P = (!seen && B) ? D + (uint32_t)(__ffs(B) - 1) : P;
                    seen = seen || B;
                    D = B ? nv - 1u - hiB : D + nv;
                }
            };
            const uint32_t nfull = len / (32u * kG);   // rounds with every value present
            uint32_t base0 = 0;
            for (uint32_t q = 0; q < nfull; ++q, base0 += 32u * kG) {
                uint32_t xb[kG];
                const bool next_full = q + 1u < nfull;
#pragma unroll
                for (uint32_t g = 0; g < kG; ++g) {
                    const uint32_t idx = base0 + 32u * (kG + g) + lane;
                    xb[g] = (next_full || idx < len) ? __ldcs(v + idx) : 0u;
                }
                scan(xa, base0, true);
#pragma unroll
                for (uint32_t g = 0; g < kG; ++g)
                    xa[g] = xb[g];
            }
            if (base0 < len)
                scan(xa, base0, false);
            if (lane == 0) {
                GapEdge e;
                e.prefix = seen ? P : len;
                e.suffix = D;
                e.has_visit = seen ? 1u : 0u;
                e.pad = len;
                edges[c] = e;
            }
        }
    }
    if (cur != 0xFFFFFFFFu)
        gap_flush(h, t, hist + (size_t)cur * (t + 1u), lane);
}

// Gaps that cross chunk boundaries, and each sequence's first gap: one
// thread per sequence walks its chunks' edges in order.
__global__ void __launch_bounds__(256) mtgp_gap_stitch_kernel(const uint64_t* __restrict__ chunk_base,
                                                             uint32_t n_seq, uint32_t t,
                                                             const GapEdge* __restrict__ edges,
                                                             unsigned long long* __restrict__ hist)
{
    const uint32_t i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n_seq)
        return;
    uint64_t run = 0;
    for (uint64_t c = chunk_base[i]; c < chunk_base[i + 1u]; ++c) {
        const GapEdge e = edges[c];
        if (e.has_visit) {
            const uint64_t gap = run + e.prefix;
            atomicAdd(hist + (size_t)i * (t + 1u) + (gap < t ? gap : (uint64_t)t), 1ull);
            run = e.suffix;
        } else {
            run += e.pad;   // the chunk's length
        }
    }
}

// One warp per pair of blocks (2K values, K = L / s).  Each lane sums the
// field weights of its values of each block; two warp reductions give the
// block weights; lane 0 classifies them and counts the pair in the warp's
// table, which is flushed whenever the warp moves to another sequence.
__global__ void __launch_bounds__(kWarps * 32) mtgp_hamming_kernel(const uint32_t* __restrict__ values,
                                                                  const uint64_t* __restrict__ seq_start,
                                                                  const uint64_t* __restrict__ pair_base,
                                                                  uint32_t n_seq, uint64_t n_pairs,
                                                                  uint32_t fmask, uint32_t K,
                                                                  const uint32_t* __restrict__ bounds,
                                                                  uint32_t n_bounds,
                                                                  unsigned long long* __restrict__ table)
{
    __shared__ uint32_t tab_all[kWarps][kMaxClasses * kMaxClasses];
    __shared__ uint32_t bnd[kMaxClasses];
    const uint32_t lane = threadIdx.x & 31u, warp = threadIdx.x >> 5;
    if (threadIdx.x < n_bounds)
        bnd[threadIdx.x] = bounds[threadIdx.x];
    const uint32_t C = n_bounds + 1u;
    uint32_t* tab = tab_all[warp];
    for (uint32_t i = lane; i < C * C; i += 32u)
        tab[i] = 0u;
    __syncthreads();
    // contiguous ranges of pairs per warp, so the sequence changes rarely
    const uint64_t nwarps = (uint64_t)gridDim.x * kWarps;
    const uint64_t gwarp = (uint64_t)blockIdx.x * kWarps + warp;
    const uint64_t per = (n_pairs + nwarps - 1) / nwarps;
    const uint64_t p0 = gwarp * per, p1 = min(p0 + per, n_pairs);
    uint32_t seq = 0xFFFFFFFFu;
    uint64_t seq_end = 0;
    bool dirty = false;
    for (uint64_t p = p0; p < p1; ++p) {
        if (seq == 0xFFFFFFFFu || p >= seq_end) {
            if (dirty) {
                __syncwarp();
                for (uint32_t i = lane; i < C * C; i += 32u) {
                    if (tab[i])
                        atomicAdd(table + (size_t)seq * C * C + i, (unsigned long long)tab[i]);
                    tab[i] = 0u;
                }
                __syncwarp();
                dirty = false;
            }
            // the sequence holding pair p: last s with pair_base[s] <= p
            uint32_t lo = 0, hi = n_seq;
            while (hi - lo > 1u) {
                const uint32_t mid = (lo + hi) >> 1;
                if (pair_base[mid] <= p)
                    lo = mid;
                else
                    hi = mid;
            }
            seq = lo;
            seq_end = pair_base[lo + 1];
        }
        const uint32_t* v = values + seq_start[seq] + (p - pair_base[seq]) * 2ull * K;
        uint32_t wa = 0, wb = 0;
        // the pair's values in batches of kB per lane, all of a batch in flight
        constexpr uint32_t kB = 16;
        for (uint32_t j0 = 0; j0 < 2u * K; j0 += 32u * kB) {
            uint32_t xs[kB];
#pragma unroll
            for (uint32_t q = 0; q < kB; ++q) {
                const uint32_t j = j0 + 32u * q + lane;
                xs[q] = j < 2u * K ? __ldcs(v + j) : 0u;
            }
#pragma unroll
            for (uint32_t q = 0; q < kB; ++q) {
                const uint32_t j = j0 + 32u * q + lane;
                const uint32_t w = __popc(xs[q] & fmask);
                if (j < K)
                    wa += w;
                else if (j < 2u * K)
                    wb += w;
            }
        }
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            wa += __shfl_xor_sync(0xFFFFFFFFu, wa, o);
            wb += __shfl_xor_sync(0xFFFFFFFFu, wb, o);
        }
        if (lane == 0) {
            uint32_t ca = 0, cb = 0;
            for (uint32_t i = 0; i < n_bounds; ++i) {
                ca += bnd[i] <= wa;
                cb += bnd[i] <= wb;
            }
            tab[ca * C + cb] += 1u;
        }
        dirty = true;
    }
    __syncwarp();
    if (dirty)
        for (uint32_t i = lane; i < C * C; i += 32u)
            if (tab[i])
                atomicAdd(table + (size_t)seq * C * C + i, (unsigned long long)tab[i]);
}

int grid_for(const void* fn, size_t dyn_smem = 0)
{
    int dev = 0, sms = 0, per = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, fn, kWarps * 32, dyn_smem);
    return std::max(1, sms * std::max(per, 1));
}

// Device scratch of one call, released on every exit path.
struct Scratch {
    cudaStream_t s;
    std::vector<void*> ptrs;
    explicit Scratch(cudaStream_t st) : s(st) {}
    cudaError_t alloc(void** p, size_t bytes)
    {
        cudaError_t e = cudaMallocAsync(p, std::max<size_t>(bytes, 16), s);
        if (e == cudaSuccess)
            ptrs.push_back(*p);
        return e;
    }
    ~Scratch()
    {
        for (void* p : ptrs)
            cudaFreeAsync(p, s);
    }
};

#define Q_TRY(call, what)                 \
    do {                                  \
        cudaError_t e_ = (call);          \
        if (e_ != cudaSuccess)            \
            return fail_cuda(e_, what);   \
    } while (0)

}  // namespace

extern "C" mtgp_status mtgp_gap_histogram(const uint32_t* values, const uint64_t* counts, uint32_t n_seq,
                                          uint32_t r, uint32_t b, uint32_t t, uint64_t* hist,
                                          void* cuda_stream)
{
    try {
        if (!counts || !hist || n_seq == 0)
            return fail(MTGP_EINVAL, "null argument or no sequence");
        if (b < 1 || r + b > 32 || t < 1 || t > kMaxT)
            return fail(MTGP_EINVAL, "need b >= 1, r + b <= 32, 1 <= t <= %u", kMaxT);
        uint64_t total = 0;
        std::vector<uint64_t> seq_start(n_seq), chunk_base(n_seq + 1);
        uint64_t n_chunks = 0;
        for (uint32_t i = 0; i < n_seq; ++i) {
            seq_start[i] = total;
            chunk_base[i] = n_chunks;
            n_chunks += (counts[i] + kChunk - 1) / kChunk;
            total += counts[i];
        }
        chunk_base[n_seq] = n_chunks;
        std::fill(hist, hist + (size_t)n_seq * (t + 1), 0ull);
        if (total && !values)
            return fail(MTGP_EINVAL, "null values pointer");
        if (n_chunks == 0)
            return ok();
        cudaStream_t s = (cudaStream_t)cuda_stream;
        Scratch sc(s);
        void *d_start, *d_counts, *d_base, *d_claim, *d_hist, *d_edges;
        const size_t hbytes = (size_t)n_seq * (t + 1) * sizeof(unsigned long long);
        Q_TRY(sc.alloc(&d_start, n_seq * sizeof(uint64_t)), "cudaMallocAsync");
        Q_TRY(sc.alloc(&d_counts, n_seq * sizeof(uint64_t)), "cudaMallocAsync");
        Q_TRY(sc.alloc(&d_base, (n_seq + 1) * sizeof(uint64_t)), "cudaMallocAsync");
        Q_TRY(sc.alloc(&d_claim, sizeof(unsigned long long)), "cudaMallocAsync");
        Q_TRY(sc.alloc(&d_hist, hbytes), "cudaMallocAsync");
        Q_TRY(sc.alloc(&d_edges, n_chunks * sizeof(GapEdge)), "cudaMallocAsync");
        Q_TRY(cudaMemcpyAsync(d_start, seq_start.data(), n_seq * sizeof(uint64_t), cudaMemcpyHostToDevice, s),
              "cudaMemcpyAsync");
        Q_TRY(cudaMemcpyAsync(d_counts, counts, n_seq * sizeof(uint64_t), cudaMemcpyHostToDevice, s),
              "cudaMemcpyAsync");
        Q_TRY(cudaMemcpyAsync(d_base, chunk_base.data(), (n_seq + 1) * sizeof(uint64_t),
                              cudaMemcpyHostToDevice, s), "cudaMemcpyAsync");
        Q_TRY(cudaMemsetAsync(d_claim, 0, sizeof(unsigned long long), s), "cudaMemsetAsync");
        Q_TRY(cudaMemsetAsync(d_hist, 0, hbytes, s), "cudaMemsetAsync");
        const size_t hsmem = (size_t)kWarps * (t + 1) * sizeof(uint32_t);   // <= 32 KB
        const int grid = (int)std::min<uint64_t>((uint64_t)grid_for((const void*)mtgp_gap_kernel, hsmem),
                                                 (n_chunks + kWarps - 1) / kWarps);
        // chunks per claim: about four claims per warp, at most 16 chunks
        const uint64_t warps = (uint64_t)grid * kWarps;
        const uint32_t run = (uint32_t)std::max<uint64_t>(1, std::min<uint64_t>(16, n_chunks / (4 * warps)));
        // the b bits after the r dropped leading bits
        const uint32_t fmask = (uint32_t)((((1ull << b) - 1ull) << (32u - r - b)) & 0xFFFFFFFFull);
        mtgp_gap_kernel<<<grid, kWarps * 32, hsmem, s>>>(values, (const uint64_t*)d_start,
                                                          (const uint64_t*)d_counts, (const uint64_t*)d_base,
                                                          n_seq, n_chunks, run, fmask, t,
                                                          (unsigned long long*)d_claim,
                                                          (unsigned long long*)d_hist, (GapEdge*)d_edges);
        Q_TRY(cudaGetLastError(), "gap kernel launch");
        mtgp_gap_stitch_kernel<<<(n_seq + 255) / 256, 256, 0, s>>>((const uint64_t*)d_base, n_seq, t,
                                                                   (const GapEdge*)d_edges,
                                                                   (unsigned long long*)d_hist);
        Q_TRY(cudaGetLastError(), "gap stitch kernel launch");
        Q_TRY(cudaMemcpyAsync(hist, d_hist, hbytes, cudaMemcpyDeviceToHost, s), "cudaMemcpyAsync");
        Q_TRY(cudaStreamSynchronize(s), "cudaStreamSynchronize");
        return ok();
    } catch (const std::bad_alloc&) {
        return fail(MTGP_ENOMEM, "host allocation failed");
    }
}

extern "C" mtgp_status mtgp_hamming_pairs(const uint32_t* values, const uint64_t* counts, uint32_t n_seq,
                                          uint32_t r, uint32_t s, uint32_t L, const uint32_t* bounds,
                                          uint32_t n_bounds, uint64_t* table, void* cuda_stream)
{
    try {
        if (!counts || !table || n_seq == 0 || (n_bounds && !bounds))
            return fail(MTGP_EINVAL, "null argument or no sequence");
        if (s < 1 || r + s > 32 || L == 0 || L % s != 0 || L / s > (1u << 24))
            return fail(MTGP_EINVAL, "need s >= 1, r + s <= 32, L > 0 a multiple of s");
        if (n_bounds + 1 > kMaxClasses)
            return fail(MTGP_EINVAL, "at most %u weight classes", kMaxClasses);
        for (uint32_t i = 1; i < n_bounds; ++i)
            if (bounds[i] < bounds[i - 1])
                return fail(MTGP_EINVAL, "class bounds must be ascending");
        const uint32_t K = L / s, C = n_bounds + 1;
        std::vector<uint64_t> seq_start(n_seq), pair_base(n_seq + 1);
        uint64_t total = 0, pairs = 0;
        for (uint32_t i = 0; i < n_seq; ++i) {
            seq_start[i] = total;
            pair_base[i] = pairs;
            pairs += counts[i] / (2ull * K);
            total += counts[i];
        }
        pair_base[n_seq] = pairs;
        std::fill(table, table + (size_t)n_seq * C * C, 0ull);
        if (total && !values)
            return fail(MTGP_EINVAL, "null values pointer");
        if (pairs == 0)
            return ok();
        cudaStream_t st = (cudaStream_t)cuda_stream;
        Scratch sc(st);
        void *d_start, *d_base, *d_bounds, *d_table;
        const size_t tbytes = (size_t)n_seq * C * C * sizeof(unsigned long long);
        Q_TRY(sc.alloc(&d_start, n_seq * sizeof(uint64_t)), "cudaMallocAsync");
        Q_TRY(sc.alloc(&d_base, (n_seq + 1) * sizeof(uint64_t)), "cudaMallocAsync");
        Q_TRY(sc.alloc(&d_bounds, (n_bounds + 1) * sizeof(uint32_t)), "cudaMallocAsync");
        Q_TRY(sc.alloc(&d_table, tbytes), "cudaMallocAsync");
        Q_TRY(cudaMemcpyAsync(d_start, seq_start.data(), n_seq * sizeof(uint64_t), cudaMemcpyHostToDevice, st),
              "cudaMemcpyAsync");
        Q_TRY(cudaMemcpyAsync(d_base, pair_base.data(), (n_seq + 1) * sizeof(uint64_t),
                              cudaMemcpyHostToDevice, st), "cudaMemcpyAsync");
        if (n_bounds)
            Q_TRY(cudaMemcpyAsync(d_bounds, bounds, n_bounds * sizeof(uint32_t), cudaMemcpyHostToDevice, st),
                  "cudaMemcpyAsync");
        Q_TRY(cudaMemsetAsync(d_table, 0, tbytes, st), "cudaMemsetAsync");
        const int grid = (int)std::min<uint64_t>((uint64_t)grid_for((const void*)mtgp_hamming_kernel),
                                                 (pairs + kWarps - 1) / kWarps);
        // the s bits after the r dropped leading bits
        const uint32_t fmask = (uint32_t)((((1ull << s) - 1ull) << (32u - r - s)) & 0xFFFFFFFFull);
        mtgp_hamming_kernel<<<grid, kWarps * 32, 0, st>>>(values, (const uint64_t*)d_start,
                                                           (const uint64_t*)d_base, n_seq, pairs, fmask, K,
                                                           (const uint32_t*)d_bounds, n_bounds,
                                                           (unsigned long long*)d_table);
        Q_TRY(cudaGetLastError(), "Hamming kernel launch");
        Q_TRY(cudaMemcpyAsync(table, d_table, tbytes, cudaMemcpyDeviceToHost, st), "cudaMemcpyAsync");
        Q_TRY(cudaStreamSynchronize(st), "cudaStreamSynchronize");
        return ok();
    } catch (const std::bad_alloc&) {
        return fail(MTGP_ENOMEM, "host allocation failed");
    }
}

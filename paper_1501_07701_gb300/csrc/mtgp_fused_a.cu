// Instantiations of the fused generation + statistics kernel for
// M = ceil(N/32) in {10, 11, 20} and G = 8 warps per CTA, with the dispatch and
// the launcher of every instantiation (see mtgp_fused.cuh).
#include "mtgp_fused.cuh"

namespace mtgp {

const void* fused_ptr_group_b(int M, int G);

static const void* fused_ptr_group_a(int M, int G)
{
    switch (M * 16 + G) {
    case 10 * 16 + 8: return (const void*)mtgp_fused_kernel<10, 8>;
    case 11 * 16 + 8: return (const void*)mtgp_fused_kernel<11, 8>;
    case 20 * 16 + 8: return (const void*)mtgp_fused_kernel<20, 8>;
    default: return nullptr;
    }
}

const void* fused_kernel_ptr(int M, int G)
{
    const void* p = fused_ptr_group_a(M, G);
    return p ? p : fused_ptr_group_b(M, G);
}

cudaError_t launch_fused(const void* fn, const GenArgs& a, const StatsArgs& A, dim3 grid, dim3 block,
                         size_t smem, cudaStream_t s)
{
    KParams P = a.P;
    uint32_t* states = a.states;
    uint32_t n_streams = a.n_streams;
    const WorkItem* items = a.items;
    const Segment* segs = a.segs;
    uint32_t n_items = a.n_items;
    uint32_t* counter = a.counter;
    uint32_t* out = a.out;
    int* err = a.err;
    const KSet* sets = a.sets;
    const uint32_t* set_of = a.set_of;
    StatsArgs st = A;
    void* args[] = {&P, &states, &n_streams, &items, &segs, &n_items, &counter, &out, &err,
                    &sets, &set_of, &st};
    return cudaLaunchKernel(fn, grid, block, args, smem, s);
}

// One thread per request: walks the request's pieces in order and counts
// what lies across their edges.  Gaps: the run of non-visits carried from
// earlier pieces plus a piece's leading run is the gap of its first visit.
// Pairs: the pair open at a piece's start holds pos = (its position in the
// request) mod 2K values from earlier pieces; the piece adds its weights in
// the pair's two blocks and, if the pair ends inside it (its length >= 2K -
// pos), the completed pair is counted and the pair open at its end carries on.
__global__ void __launch_bounds__(128) mtgp_stats_stitch_kernel(const Segment* __restrict__ segs,
                                                               const uint32_t* __restrict__ piece_start,
                                                               const uint32_t* __restrict__ pieces,
                                                               uint32_t n_req, const StatsArgs A)
{
    const uint32_t j = blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= n_req)
        return;
    const uint32_t p0 = piece_start[j], p1 = piece_start[j + 1u];
    if (p1 - p0 < 2u)
        return;
    const uint64_t two_k = 2ull * A.K;
    const SegStat f = A.seg_stats[pieces[p0]];
    uint64_t run = f.gsuffix;
    uint32_t wa = f.ta, wb = f.tb;
    for (uint32_t q = p0 + 1u; q < p1; ++q) {
        const uint32_t sidx = pieces[q];
        const SegStat r = A.seg_stats[sidx];
        const Segment sg = segs[sidx];
        if (r.gvisit) {
            const uint64_t gap = run + r.gprefix;
            if (A.hist)
                atomicAdd(A.hist + (size_t)j * (A.t + 1u) + (gap < A.t ? gap : (uint64_t)A.t), 1ull);
            run = r.gsuffix;
        } else {
            run += r.gprefix;
        }
        const uint64_t pos = (sg.out_off - A.req_base[j]) % two_k;
        if (pos == 0u) {
            wa = r.ta;
            wb = r.tb;
            continue;
        }
        wa += r.la;
        wb += r.lb;
        if (sg.count >= two_k - pos) {
            uint32_t ca = 0u, cb = 0u;
            for (uint32_t i = 0; i + 1u < A.C && i < 15u; ++i) {
                ca += A.bounds[i] <= wa;
                cb += A.bounds[i] <= wb;
            }
            if (A.tab)
                atomicAdd(A.tab + (size_t)j * A.C * A.C + ca * A.C + cb, 1ull);
            wa = r.ta;
            wb = r.tb;
        }
    }
}

cudaError_t launch_stats_stitch(const Segment* segs, const uint32_t* piece_start, const uint32_t* pieces,
                                uint32_t n_req, const StatsArgs& A, cudaStream_t s)
{
    if (n_req == 0)
        return cudaSuccess;
    mtgp_stats_stitch_kernel<<<(n_req + 127u) / 128u, 128, 0, s>>>(segs, piece_start, pieces, n_req, A);
    return cudaGetLastError();
}

}  // namespace mtgp

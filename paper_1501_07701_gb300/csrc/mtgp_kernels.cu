// Status initialisation, the shared-memory ring kernel (any parameter set),
// and launch geometry for MTGP32 generation on sm_103a.
#include <algorithm>

#include "mtgp_internal.h"

namespace mtgp {

// ---------------------------------------------------------------------------
// Seed status -> state (Sec. 3.1 "seed status"; the MT-family seeding
// recurrence w_i = 1812433253 * (w_{i-1} ^ (w_{i-1} >> 30)) + i).  The
// recurrence is sequential within a stream, so one thread owns one stream;
// it stages its words through shared memory so that a warp writes 32
// consecutive words of one row at a time.
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(128) mtgp_init_kernel(const uint32_t* __restrict__ seeds,
                                                        uint32_t n_streams, uint32_t n, uint32_t np,
                                                        uint32_t* __restrict__ states)
{
    __shared__ uint32_t buf[4][32][33];
    const uint32_t lane = threadIdx.x & 31u, warp = threadIdx.x >> 5;
    const uint32_t s0 = (blockIdx.x * 4u + warp) * 32u;   // first stream of this warp
    const uint32_t s = s0 + lane;
    uint32_t w = s < n_streams ? seeds[s] : 0u;
    for (uint32_t c0 = 0; c0 < np; c0 += 32u) {
        // each lane produces words c0..c0+31 of its own stream
        for (uint32_t j = 0; j < 32u; ++j) {
            const uint32_t i = c0 + j;
            uint32_t v = 0;
            if (i == 0)
                v = w;
            else if (i < n) {
                w = 1812433253u * (w ^ (w >> 30)) + i;
                v = w;
            }
            buf[warp][lane][j] = v;
        }
        __syncwarp();
        // warp writes row by row: lane j writes word c0+j of stream s0+t
        for (uint32_t t = 0; t < 32u; ++t) {
            const uint32_t st = s0 + t;
            const uint32_t i = c0 + lane;
            if (st < n_streams && i < np)
                states[(size_t)st * np + i] = buf[warp][t][lane];
        }
        __syncwarp();
    }
}

cudaError_t launch_init(const KParams& P, const uint32_t* d_seeds, uint32_t n_streams,
                        uint32_t* d_states, cudaStream_t s)
{
    if (n_streams == 0)
        return cudaSuccess;
    const uint32_t blocks = (n_streams + 127u) / 128u;
    mtgp_init_kernel<<<blocks, 128, 0, s>>>(d_seeds, n_streams, P.n, P.np, d_states);
    return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// Shared-memory ring kernel: any N >= 2 and any pos.  One warp per stream;
// the state row S[0..N) holds the latest value of each column (column c of
// row q is x_{qN+c}).  Each parallel step computes Wc = min(32, N - pos)
// consecutive columns: every word it reads was produced before the step.
// Every output lane finds its own request, so this kernel also serves as the
// plain reference path for unusual parameter sets.
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(256) mtgp_ring_kernel(const KParams P, uint32_t* __restrict__ states,
                                                        uint32_t n_streams,
                                                        const WorkItem* __restrict__ items,
                                                        const Segment* __restrict__ segs,
                                                        uint32_t n_items, uint32_t* __restrict__ counter,
                                                        uint32_t* __restrict__ out, int* __restrict__ err,
                                                        const KSet* __restrict__ sets,
                                                        const uint32_t* __restrict__ set_of)
{
    extern __shared__ __align__(16) uint32_t smem[];
    const uint32_t lane = threadIdx.x & 31u;
    const uint32_t warp = threadIdx.x >> 5;
    const uint32_t N = P.n;
    // per warp: REC[16], TMP[16], then the state row
    uint32_t* rec = smem + warp * ring_smem_words(N);
    uint32_t* tmp = rec + 16;
    uint32_t* S = rec + 32;

    for (;;) {
        uint32_t it = 0;
        if (lane == 0)
            it = atomicAdd(counter, 1u);
        it = __shfl_sync(0xFFFFFFFFu, it, 0);
        if (it >= n_items)
            break;
        const WorkItem w = items[it];
        if (w.stream >= n_streams || w.nseg == 0) {
            if (lane == 0)
                atomicOr(err, 1);
            continue;
        }
        // this stream's parameter set (the handle's own, or its per-stream set)
        uint32_t pos = P.pos, sh1 = P.sh1, sh2 = P.sh2;
        if (sets) {
            const KSet& ks = sets[set_of[w.stream]];
            pos = ks.pos;
            sh1 = ks.sh1;
            sh2 = ks.sh2;
            if (lane < 16u) {
                rec[lane] = ks.rec[lane];
                tmp[lane] = ks.tmp[lane];
            }
        } else if (lane < 16u) {
            rec[lane] = P.rec[lane];
            tmp[lane] = P.tmp[lane];
        }
        const uint32_t Wc = (N - pos) < 32u ? (N - pos) : 32u;
        uint32_t* g = states + (size_t)w.stream * P.np;
        for (uint32_t j = lane; j < N; j += 32u)
            S[j] = g[j];
        __syncwarp();

        const uint32_t s_end = w.seg_begin + w.nseg;
        const Segment last = segs[s_end - 1u];
        const uint64_t total = last.g_start + last.count;
        uint32_t s_row = w.seg_begin;
        for (uint64_t row = 0; row < total; row += N) {
            while (segs[s_row].g_start + segs[s_row].count <= row)
                ++s_row;
            const uint64_t left = total - row;
            const uint32_t n_valid = left < (uint64_t)N ? (uint32_t)left : N;
            for (uint32_t c0 = 0; c0 < n_valid; c0 += Wc) {
                const uint32_t c = c0 + lane;
                const bool act = lane < Wc && c < n_valid;
                uint32_t xn = 0, o = 0;
                if (act) {
                    const uint32_t c1 = (c + 1u == N) ? 0u : c + 1u;
                    uint32_t cp = c + pos;
                    cp = cp >= N ? cp - N : cp;
                    uint32_t cq = c + pos - 1u;
                    cq = cq >= N ? cq - N : cq;
                    uint32_t y = (S[c] & P.mask) ^ S[c1];
                    y ^= y << sh1;
                    y ^= S[cp] >> sh2;
                    xn = y ^ rec[y & 15u];
                    uint32_t t = S[cq];
                    t ^= t >> 16;
                    t ^= t >> 8;
                    o = xn ^ tmp[t & 15u];
                }
                __syncwarp();
                if (act) {
                    S[c] = xn;
                    const uint64_t gi = row + c;
                    uint32_t s = s_row;
                    while (s + 1u < s_end && gi >= segs[s + 1u].g_start)
                        ++s;
                    const Segment sg = segs[s];
                    if (sg.fmt != 0) {
                        const uint32_t b = 0x3F800000u | (o >> 9);
                        o = sg.fmt == 1 ? b : __float_as_uint(__uint_as_float(b) - 1.0f);
                    }
                    out[sg.out_off + (gi - sg.g_start)] = o;
                }
                __syncwarp();
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
}

// ---------------------------------------------------------------------------
// Row copies (the start states of a split stream's pieces): one warp per
// pair, grid-stride over pairs.
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(256) mtgp_copy_rows_kernel(const uint32_t* __restrict__ src,
                                                            uint32_t* __restrict__ dst,
                                                            const uint2* __restrict__ pairs,
                                                            uint32_t n, uint32_t N, uint32_t np)
{
    const uint32_t lane = threadIdx.x & 31u;
    const uint32_t warps = gridDim.x * (blockDim.x >> 5);
    for (uint32_t i = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5); i < n; i += warps) {
        const uint2 p = pairs[i];
        const uint32_t* a = src + (size_t)p.x * np;
        uint32_t* b = dst + (size_t)p.y * np;
        for (uint32_t j = lane; j < N; j += 32u)
            b[j] = a[j];
    }
}

cudaError_t launch_copy_rows(const uint32_t* src, uint32_t* dst, const uint2* pairs, uint32_t n,
                             uint32_t N, uint32_t np, cudaStream_t s)
{
    if (n == 0)
        return cudaSuccess;
    const uint32_t blocks = std::min<uint32_t>((n + 7u) / 8u, 1024u);
    mtgp_copy_rows_kernel<<<blocks, 256, 0, s>>>(src, dst, pairs, n, N, np);
    return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// Geometry and dispatch
// ---------------------------------------------------------------------------
cudaError_t allow_max_dynamic_smem(const void* fn, int device, size_t need)
{
    // Without the opt-in a CTA may use 48 KB of static and dynamic shared
    // memory together; beyond that the function's dynamic limit is raised
    // to the device's opt-in maximum less its static shared memory.
    cudaFuncAttributes fa;
    cudaError_t e = cudaFuncGetAttributes(&fa, fn);
    if (e != cudaSuccess)
        return e;
    if (need + fa.sharedSizeBytes <= 48u * 1024u)
        return cudaSuccess;
    int optin = 0;
    e = cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, device);
    if (e != cudaSuccess)
        return e;
    if (need + fa.sharedSizeBytes > (size_t)optin)
        return cudaErrorInvalidValue;
    return cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                optin - (int)fa.sharedSizeBytes);
}

static int fast_m(const KParams& P) { return (int)((P.n + 31u) / 32u); }

bool fast_supported(const KParams& P, int k, int g)
{
    if (k != 2 && k != 4 && k != 8)
        return false;
    if (P.n < 64 || 32u * (uint32_t)k > P.n - P.pos)
        return false;
    if (P.sh1 < 1 || P.sh1 > 31 || P.sh2 < 1 || P.sh2 > 31)
        return false;
    const int M = fast_m(P);
    if (M <= k)
        return false;
    return fast_kernel_ptr(M, k, g) != nullptr;
}

cudaError_t plan_geometry(const KParams& P, const LaunchCfg& cfg, uint32_t n_items, int device,
                          Geometry* g)
{
    int k = cfg.k;
    int kernel = cfg.kernel;
    int warps = std::max(1, std::min(8, cfg.warps_per_cta));
    if (kernel == 0) {
        // register-resident kernel: G in {2, 4, 8}
        warps = warps <= 2 ? 2 : (warps <= 4 ? 4 : 8);
        if (!fast_supported(P, k, warps)) {
            if (fast_supported(P, 4, std::min(warps, 4))) {
                k = 4;
                warps = std::min(warps, 4);
            } else if (fast_supported(P, 2, std::min(warps, 4))) {
                k = 2;   // short states (Mexp 3217: N - pos < 128)
                warps = std::min(warps, 4);
            } else {
                kernel = 1;
            }
        }
    }
    g->kernel = kernel;
    g->k = k;
    g->threads = warps * 32;
    const void* fn;
    if (kernel == 0) {
        g->smem = (size_t)warps * fast_smem_words(P.n, P.mirror) * 4u;
        fn = fast_kernel_ptr(fast_m(P), k, warps);
    } else {
        g->smem = (size_t)warps * ring_smem_words(P.n) * 4u;
        fn = (const void*)mtgp_ring_kernel;
    }
    cudaError_t e;
    if ((e = allow_max_dynamic_smem(fn, device, g->smem)) != cudaSuccess)
        return e;
    int per_sm = 0;
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, fn, g->threads, g->smem);
    if (e != cudaSuccess)
        return e;
    if (per_sm < 1)
        return cudaErrorInvalidConfiguration;
    if (cfg.ctas_per_sm > 0)
        per_sm = std::min(per_sm, cfg.ctas_per_sm);
    cudaFuncAttributes fa;
    e = cudaFuncGetAttributes(&fa, fn);
    if (e != cudaSuccess)
        return e;
    g->regs = fa.numRegs;
    g->per_sm = per_sm;
    int sms = 0;
    e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, device);
    if (e != cudaSuccess)
        return e;
    const long long want = ((long long)n_items + warps - 1) / warps;
    const long long cap = (long long)sms * per_sm;
    g->grid = (int)std::max(1LL, std::min(want, cap));
    return cudaSuccess;
}

cudaError_t launch_generate(const GenArgs& a, const Geometry& g, cudaStream_t s)
{
    if (a.n_items == 0)
        return cudaSuccess;
    if (g.kernel == 0)
        return launch_fast((int)((a.P.n + 31u) / 32u), g.k, g.threads / 32, a, dim3(g.grid),
                           dim3(g.threads), g.smem, s);
    mtgp_ring_kernel<<<g.grid, g.threads, g.smem, s>>>(a.P, a.states, a.n_streams, a.items, a.segs,
                                                       a.n_items, a.counter, a.out, a.err, a.sets,
                                                       a.set_of);
    return cudaGetLastError();
}

}  // namespace mtgp

namespace mtgp {

const void* fast_ptr_group_a(int M, int K, int G);
const void* fast_ptr_group_b(int M, int K, int G);
const void* fast_ptr_group_c(int M, int K, int G);
const void* fast_ptr_group_d(int M, int K, int G);

const void* fast_kernel_ptr(int M, int K, int G)
{
    const void* p = fast_ptr_group_a(M, K, G);
    if (!p)
        p = fast_ptr_group_b(M, K, G);
    if (!p)
        p = fast_ptr_group_c(M, K, G);
    if (!p)
        p = fast_ptr_group_d(M, K, G);
    return p;
}

cudaError_t launch_fast(int M, int K, int G, const GenArgs& a, dim3 grid, dim3 block, size_t smem,
                        cudaStream_t s)
{
    const void* fn = fast_kernel_ptr(M, K, G);
    if (!fn)
        return cudaErrorInvalidValue;
    return launch_gen_fn(fn, a, grid, block, smem, s);
}

cudaError_t launch_gen_fn(const void* fn, const GenArgs& a, dim3 grid, dim3 block, size_t smem,
                          cudaStream_t s)
{
    KParams P = a.P;
    uint32_t* states = a.states;
    uint32_t n_streams = a.n_streams;
    const WorkItem* items = a.items;
    const Segment* segs = a.segs;
    uint32_t n_items = a.n_items;
    uint32_t n_coop = a.n_coop;
    uint32_t* counter = a.counter;
    uint32_t* out = a.out;
    int* err = a.err;
    uint64_t* trace = a.trace;
    const KSet* sets = a.sets;
    const uint32_t* set_of = a.set_of;
    void* args[] = {&P, &states, &n_streams, &items, &segs, &n_items, &n_coop, &counter, &out, &err,
                    &trace, &sets, &set_of};
    return cudaLaunchKernel(fn, grid, block, args, smem, s);
}

}  // namespace mtgp

// The original Mersenne Twister (Matsumoto and Nishimura 1998), the
// comparison generator of Sec. 5.3, for many independently seeded streams of
// one parameter set, or of one set per stream, on sm_103a.
//
// One warp advances one stream.  The stream's words live in a per-warp
// sliding buffer in shared memory: x_k sits at buf[off + (k - k0)] while the
// step that starts at number k0 runs, so every access of a step is the lane's
// base pointer plus a compile-time offset (no ring wrap-around).  A step of W
// consecutive numbers k reads x_k, x_{k+1}, x_{k+m} and writes x_{k+n}; with
// W <= n - m every word it reads was written before the step, and its write
// window [k0 + n, k0 + n + W) is disjoint from its read window [k0, k0 + n),
// so a step needs one __syncwarp, at its end.  When the window reaches the end
// of the buffer, its n live words are moved back to the start.
//
// Per number: three shared loads, one shared store, one coalesced global
// store.  The twist and the tempering are register arithmetic; the two left
// shifts of the tempering run as integer multiplies on the FMA pipe.
#include <algorithm>
#include <array>
#include <cstring>
#include <vector>

#include "../../include/mtgp_mt.h"
#include "mtgp_runtime.h"

using namespace mtgp;

namespace {

// The fields in which the parameter sets of one handle may differ (they all
// share p, n and r).
struct MtSet {
    uint32_t m;
    uint32_t a;
    uint32_t u, l;           // right shifts of the tempering
    uint32_t mul_s, mul_t;   // 2^s, 2^t: the tempering's left shifts as multiplies
    uint32_t b, c;
    uint32_t W;              // numbers per step: min(n - m, 256) <= 32 K
    uint32_t pad[3];
};

// Kernel form of a handle (by value, in the kernel-parameter bank).
struct MtK {
    uint32_t n, np;
    uint32_t upper;          // the top 32 - r bits
    uint32_t B;              // words of the sliding window's range, >= 2 n + (largest W)
    uint32_t stride;         // words per warp: B plus 32 K words of slack that
                             // lanes past W may read
    uint32_t pad[3];
    MtSet set;               // the handle's set (streams without a set of their own)
};

__device__ __forceinline__ uint32_t mt_twist(uint32_t upper, const MtSet& S, uint32_t xk,
                                             uint32_t xk1, uint32_t xm)
{
    const uint32_t y = (xk & upper) | (xk1 & ~upper);
    return xm ^ (y >> 1) ^ ((y & 1u) * S.a);
}

__device__ __forceinline__ uint32_t mt_temper(const MtSet& S, uint32_t x)
{
    uint32_t z = x ^ (x >> S.u);
    z ^= (z * S.mul_s) & S.b;
    z ^= (z * S.mul_t) & S.c;
    return z ^ (z >> S.l);
}

template <int FMT>
__device__ __forceinline__ uint32_t mt_convert(uint32_t z)
{
    if (FMT == 0)
        return z;
    const uint32_t b12 = 0x3F800000u | (z >> 9);
    if (FMT == 1)
        return b12;
    return __float_as_uint(__uint_as_float(b12) - 1.0f);
}

__device__ __forceinline__ uint32_t mt_convert_rt(uint32_t z, uint32_t fmt)
{
    return fmt == 0 ? z : (fmt == 1 ? mt_convert<1>(z) : mt_convert<2>(z));
}

// `nst` >= 1 whole steps inside one request, with room in the buffer for all
// of them.  Lane j of sub-step i takes number k0 + 32 i + j of each step;
// bp = buf + off + lane and op = the lane's output of the first step.
// Lanes past W (32 K > W) load and compute too, on words of the buffer's
// slack, so the step has no branches; only their two stores are predicated
// off.  The tempering, conversion and output store of step t run after the
// loads of step t + 1 are issued, so they fill the load latency instead of
// lengthening the chain from one step's state store to the next step's loads.
template <int K, int FMT>
__device__ __forceinline__ void mt_run_steps(const MtK& P, const MtSet& S, uint32_t* bp, uint32_t* op,
                                             uint32_t nst, uint32_t lane)
{
    const uint32_t W = S.W, m = S.m, n = P.n, upper = P.upper;
    bool act[K];   // the lane's number in sub-step i belongs to the step
#pragma unroll
    for (int i = 0; i < K; ++i)
        act[i] = 32u * i + lane < W;
    uint32_t xn[K];
#pragma unroll
    for (int i = 0; i < K; ++i)
        xn[i] = mt_twist(upper, S, bp[32 * i], bp[32 * i + 1], bp[32 * i + m]);
#pragma unroll
    for (int i = 0; i < K; ++i)
        if (act[i])
            bp[32 * i + n] = xn[i];
    __syncwarp();
#pragma unroll 2
    for (uint32_t t = 1; t < nst; ++t) {
        bp += W;
        uint32_t xt[K];
#pragma unroll
        for (int i = 0; i < K; ++i)
            xt[i] = mt_twist(upper, S, bp[32 * i], bp[32 * i + 1], bp[32 * i + m]);
#pragma unroll
        for (int i = 0; i < K; ++i) {
            const uint32_t o = mt_convert<FMT>(mt_temper(S, xn[i]));
            if (act[i])
                __stcs(op + 32 * i, o);
        }
        op += W;
#pragma unroll
        for (int i = 0; i < K; ++i) {
            if (act[i])
                bp[32 * i + n] = xt[i];
            xn[i] = xt[i];
        }
        __syncwarp();
    }
#pragma unroll
    for (int i = 0; i < K; ++i) {
        const uint32_t o = mt_convert<FMT>(mt_temper(S, xn[i]));
        if (act[i])
            __stcs(op + 32 * i, o);
    }
}

// A step that crosses a request boundary or the stream's end: each lane finds
// the request of its own number.
template <int K>
__device__ __forceinline__ void mt_step_slow(const MtK& P, const MtSet& S, uint32_t* bp, uint64_t k0,
                                             uint64_t total,
                                             const Segment* __restrict__ segs, uint32_t si,
                                             uint32_t s_end, uint32_t* __restrict__ out,
                                             uint32_t lane)
{
    uint32_t xn[K];
#pragma unroll
    for (int i = 0; i < K; ++i) {
        const uint32_t j = 32u * i + lane;
        if (j < S.W && k0 + j < total)
            xn[i] = mt_twist(P.upper, S, bp[32 * i], bp[32 * i + 1], bp[32 * i + S.m]);
    }
#pragma unroll
    for (int i = 0; i < K; ++i) {
        const uint32_t j = 32u * i + lane;
        const uint64_t k = k0 + j;
        if (j < S.W && k < total) {
            bp[32 * i + P.n] = xn[i];
            uint32_t s = si;
            while (s + 1u < s_end && k >= segs[s + 1u].g_start)
                ++s;
            const Segment sg = segs[s];
            out[sg.out_off + (k - sg.g_start)] = mt_convert_rt(mt_temper(S, xn[i]), sg.fmt);
        }
    }
}

template <int K>
__global__ void __launch_bounds__(128) mt_gen_kernel(const MtK P, uint32_t* __restrict__ states,
                                                     uint32_t n_streams,
                                                     const WorkItem* __restrict__ items,
                                                     const Segment* __restrict__ segs,
                                                     uint32_t n_items, uint32_t* __restrict__ counter,
                                                     uint32_t* __restrict__ out, int* __restrict__ err,
                                                     const MtSet* __restrict__ sets,
                                                     const uint32_t* __restrict__ set_of)
{
    extern __shared__ __align__(16) uint32_t smem[];
    const uint32_t lane = threadIdx.x & 31u;
    uint32_t* buf = smem + (threadIdx.x >> 5) * P.stride;
    const uint32_t N = P.n;

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
        // the stream's own parameter set, or the handle's
        const MtSet S = sets ? sets[set_of[w.stream]] : P.set;
        const uint32_t W = S.W;
        uint32_t* g = states + (size_t)w.stream * P.np;
        for (uint32_t j = lane; j < N; j += 32u)
            buf[j] = g[j];
        __syncwarp();

        const uint32_t s_end = w.seg_begin + w.nseg;
        const Segment last = segs[s_end - 1u];
        const uint64_t total = last.g_start + last.count;
        uint32_t si = w.seg_begin;
        Segment sg = segs[si];
        uint64_t seg_hi = sg.g_start + sg.count;
        uint64_t k0 = 0;    // first number of the next step
        uint32_t off = 0;   // buffer position of x_{k0}
        while (k0 < total) {
            if (off + N + W > P.B) {
                // move the live window [off, off + n) to the start; off >= n
                // here (B >= 2n + W), so source and destination are disjoint
#pragma unroll 4
                for (uint32_t j = lane; j < N; j += 32u)
                    buf[j] = buf[off + j];
                __syncwarp();
                off = 0;
            }
            while (k0 >= seg_hi && si + 1u < s_end) {
                sg = segs[++si];
                seg_hi = sg.g_start + sg.count;
            }
            uint32_t* bp = buf + off + lane;
            if (k0 + W <= seg_hi) {
                // whole steps of this request, as many as the buffer holds
                const uint64_t n_seg = (seg_hi - k0) / W;
                const uint32_t n_buf = (P.B - N - W - off) / W + 1u;
                const uint32_t nst = n_seg < n_buf ? (uint32_t)n_seg : n_buf;
                uint32_t* op = out + (sg.out_off - sg.g_start) + k0 + lane;
                if (sg.fmt == 0)
                    mt_run_steps<K, 0>(P, S, bp, op, nst, lane);
                else if (sg.fmt == 1)
                    mt_run_steps<K, 1>(P, S, bp, op, nst, lane);
                else
                    mt_run_steps<K, 2>(P, S, bp, op, nst, lane);
                k0 += (uint64_t)nst * W;
                off += nst * W;
            } else {
                mt_step_slow<K>(P, S, bp, k0, total, segs, si, s_end, out, lane);
                __syncwarp();
                k0 += W;
                off += W;
            }
        }
        // the state after `total` numbers is x_total .. x_{total+n-1}
        const uint32_t first = off - (uint32_t)(k0 - total);
        for (uint32_t j = lane; j < N; j += 32u)
            g[j] = buf[first + j];
        __syncwarp();
    }
}

const void* mt_kernel_ptr(int K)
{
    switch (K) {
    case 8:
        return (const void*)mt_gen_kernel<8>;
    case 4:
        return (const void*)mt_gen_kernel<4>;
    case 2:
        return (const void*)mt_gen_kernel<2>;
    default:
        return (const void*)mt_gen_kernel<1>;
    }
}

// SplitMix64 (Steele, Lea, Flood 2014): golden-ratio increment, then two
// xor-shift-multiply rounds and a final xor-shift.
uint64_t splitmix64(uint64_t& s)
{
    uint64_t z = (s += 0x9E3779B97F4A7C15ull);
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
}

constexpr uint32_t kMaxN = 4096;
constexpr int kWarpsPerCta = 4;

mtgp_status check_params(const mtgp_mt_params& p)
{
    if (p.n < 2 || p.n > kMaxN)
        return fail(MTGP_EINVAL, "n = %u outside 2..%u", p.n, kMaxN);
    if (p.m < 1 || p.m > p.n - 1)
        return fail(MTGP_EINVAL, "m = %u outside 1..n-1", p.m);
    if (p.r > 31 || (uint64_t)32 * p.n - p.r != p.p)
        return fail(MTGP_EINVAL, "need r <= 31 and p = 32 n - r (p %u, n %u, r %u)", p.p, p.n, p.r);
    if (p.u > 31 || p.s > 31 || p.t > 31 || p.l > 31)
        return fail(MTGP_EINVAL, "tempering shifts must be <= 31");
    return MTGP_OK;
}

MtSet make_set(const mtgp_mt_params& p)
{
    MtSet q;
    std::memset(&q, 0, sizeof q);
    q.m = p.m;
    q.a = p.a;
    q.u = p.u;
    q.l = p.l;
    q.mul_s = 1u << p.s;
    q.mul_t = 1u << p.t;
    q.b = p.b;
    q.c = p.c;
    // a step takes W = n - m numbers (the recurrence's parallel width), at most 256
    q.W = std::min(p.n - p.m, 256u);
    return q;
}

}  // namespace

struct mtgp_mt {
    mtgp_mt_params p{};
    MtK k{};
    int K = 1;
    int device = 0;
    uint32_t n_streams = 0;
    uint32_t* d_states = nullptr;
    int* d_err = nullptr;
    // work tables: a ring of pinned upload slots, each reused only after the
    // launch that read it has finished
    std::array<TableSlot, 4> slots{};
    int next_slot = 0;
    int threads = 0;
    size_t smem = 0;
    int grid_cap = 0;   // resident CTAs on the device
    int sms = 0;
    // one parameter set per stream (mtgp_mt_init_multi); null: all use k.set
    MtSet* d_sets = nullptr;
    uint32_t* d_set_of = nullptr;
};

static void destroy_mt(mtgp_mt* h)
{
    if (!h)
        return;
    DeviceGuard g(h->device);
    for (auto& sl : h->slots) {
        free_table_slot(sl);
        if (sl.ev)
            cudaEventDestroy(sl.ev);
    }
    if (h->d_states)
        cudaFree(h->d_states);
    if (h->d_err)
        cudaFree(h->d_err);
    if (h->d_sets)
        cudaFree(h->d_sets);
    if (h->d_set_of)
        cudaFree(h->d_set_of);
    delete h;
}

#define MT_TRY(call, what)             \
    do {                               \
        cudaError_t e_ = (call);       \
        if (e_ != cudaSuccess)         \
            return fail_cuda(e_, what); \
    } while (0)

extern "C" mtgp_status mtgp_mt_params_mt19937(mtgp_mt_params* out)
{
    if (!out)
        return fail(MTGP_EINVAL, "null argument");
    std::memset(out, 0, sizeof *out);
    out->p = 19937u;
    out->n = 624u;
    out->m = 397u;
    out->r = 31u;
    out->a = 0x9908B0DFu;
    out->u = 11u;
    out->s = 7u;
    out->b = 0x9D2C5680u;
    out->t = 15u;
    out->c = 0xEFC60000u;
    out->l = 18u;
    return ok();
}

extern "C" mtgp_status mtgp_mt_params_generate(uint32_t p, uint64_t seed, mtgp_mt_params* out)
{
    if (!out)
        return fail(MTGP_EINVAL, "null argument");
    if (p < 33u || (p + 31u) / 32u > kMaxN)
        return fail(MTGP_EINVAL, "exponent %u outside 33..%u", p, 32u * kMaxN);
    mtgp_mt_params q;
    std::memset(&q, 0, sizeof q);
    q.p = p;
    q.n = (p + 31u) / 32u;
    q.r = 32u * q.n - p;
    q.m = q.n / 2u;
    uint64_t s = seed;
    q.a = (uint32_t)(splitmix64(s) >> 32) | 0x80000000u;
    q.b = (uint32_t)(splitmix64(s) >> 32);
    q.c = (uint32_t)(splitmix64(s) >> 32);
    q.u = 12u;
    q.s = 7u;
    q.t = 15u;
    q.l = 18u;
    *out = q;
    return ok();
}

// Handle creation for one set (set_of null) or one set per stream.
static mtgp_status init_handle(const mtgp_mt_params* sets, uint32_t n_sets, const uint32_t* set_of,
                               const uint32_t* seeds, uint32_t n_streams, void* cuda_stream,
                               mtgp_mt_t* out)
{
    try {
        if (!sets || !out || !seeds || n_sets == 0)
            return fail(MTGP_EINVAL, "null argument");
        if (n_streams == 0)
            return fail(MTGP_EINVAL, "n_streams must be >= 1");
        for (uint32_t i = 0; i < n_sets; ++i) {
            mtgp_status st = check_params(sets[i]);
            if (st != MTGP_OK)
                return st;
            if (sets[i].p != sets[0].p || sets[i].n != sets[0].n || sets[i].r != sets[0].r)
                return fail(MTGP_EINVAL, "set %u: all sets of a handle need the same p, n and r", i);
        }
        uint32_t w_max = 0;
        for (uint32_t i = 0; i < n_sets; ++i)
            w_max = std::max(w_max, make_set(sets[i]).W);
        if (set_of)
            for (uint32_t s = 0; s < n_streams; ++s)
                if (set_of[s] >= n_sets)
                    return fail(MTGP_EINVAL, "stream %u: set index %u >= n_sets %u", s, set_of[s], n_sets);
        const mtgp_mt_params* params = sets;
        mtgp_mt* h = new mtgp_mt;
        h->p = *params;
        h->n_streams = n_streams;
        const mtgp_mt_params& p = h->p;
        MtK& k = h->k;
        std::memset(&k, 0, sizeof k);
        k.n = p.n;
        k.np = (p.n + 3u) & ~3u;
        k.upper = 0xFFFFFFFFu << p.r;
        k.set = make_set(p);
        // K = the smallest power of two with 32 K >= the widest step
        h->K = 1;
        while (32u * (uint32_t)h->K < w_max)
            h->K *= 2;
        // about 16 n words (move overhead 2n per 14n numbers), capped at
        // 4096 words so that a dozen warps fit on an SM
        uint32_t B = std::max(2u * p.n + w_max, std::min(16u * p.n, 4096u));
        k.B = (B + 31u) & ~31u;
        // a lane j < 32 K reads up to position off + 32 K - 1 + m < off + n + 32 K
        k.stride = k.B + 32u * (uint32_t)h->K;
        auto bail = [&](cudaError_t e, const char* what) {
            mtgp_status s2 = fail_cuda(e, what);
            destroy_mt(h);
            return s2;
        };
        cudaError_t e = cudaGetDevice(&h->device);
        if (e != cudaSuccess)
            return bail(e, "cudaGetDevice");
        cudaStream_t s = (cudaStream_t)cuda_stream;
        if ((e = cudaMalloc(&h->d_states, (size_t)n_streams * k.np * 4u)) != cudaSuccess)
            return bail(e, "cudaMalloc(states)");
        if ((e = cudaMalloc(&h->d_err, sizeof(int))) != cudaSuccess)
            return bail(e, "cudaMalloc(error word)");
        if ((e = cudaMemsetAsync(h->d_err, 0, sizeof(int), s)) != cudaSuccess)
            return bail(e, "cudaMemsetAsync");
        for (auto& sl : h->slots)
            if ((e = cudaEventCreateWithFlags(&sl.ev, cudaEventDisableTiming)) != cudaSuccess)
                return bail(e, "cudaEventCreate");
        // launch geometry: kWarpsPerCta warps per CTA, as many CTAs as fit
        const void* fn = mt_kernel_ptr(h->K);
        h->threads = 32 * kWarpsPerCta;
        h->smem = (size_t)kWarpsPerCta * k.stride * 4u;
        if ((e = allow_max_dynamic_smem(fn, h->device, h->smem)) != cudaSuccess)
            return bail(e, "dynamic shared memory limit");
        int per_sm = 0, sms = 0;
        if ((e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, fn, h->threads, h->smem)) !=
            cudaSuccess)
            return bail(e, "occupancy query");
        if (per_sm < 1)
            return bail(cudaErrorInvalidConfiguration, "occupancy query");
        if ((e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, h->device)) !=
            cudaSuccess)
            return bail(e, "cudaDeviceGetAttribute");
        h->grid_cap = sms * per_sm;
        h->sms = sms;
        // seeds -> states with the MT-family seeding kernel shared with MTGP
        KParams kp;
        std::memset(&kp, 0, sizeof kp);
        kp.n = k.n;
        kp.np = k.np;
        uint32_t* d_seeds = nullptr;
        if ((e = cudaMallocAsync((void**)&d_seeds, (size_t)n_streams * 4, s)) != cudaSuccess)
            return bail(e, "cudaMallocAsync(seeds)");
        if ((e = cudaMemcpyAsync(d_seeds, seeds, (size_t)n_streams * 4, cudaMemcpyHostToDevice, s)) !=
            cudaSuccess) {
            cudaFreeAsync(d_seeds, s);
            return bail(e, "cudaMemcpyAsync(seeds)");
        }
        e = launch_init(kp, d_seeds, n_streams, h->d_states, s);
        cudaFreeAsync(d_seeds, s);
        if (e != cudaSuccess)
            return bail(e, "init kernel launch");
        if (set_of) {
            std::vector<MtSet> ks(n_sets);
            for (uint32_t i = 0; i < n_sets; ++i)
                ks[i] = make_set(sets[i]);
            if ((e = cudaMalloc(&h->d_sets, n_sets * sizeof(MtSet))) != cudaSuccess ||
                (e = cudaMalloc(&h->d_set_of, (size_t)n_streams * 4)) != cudaSuccess)
                return bail(e, "cudaMalloc(parameter sets)");
            // pageable sources: both copies are complete when they return
            if ((e = cudaMemcpyAsync(h->d_sets, ks.data(), n_sets * sizeof(MtSet), cudaMemcpyHostToDevice,
                                     s)) != cudaSuccess ||
                (e = cudaMemcpyAsync(h->d_set_of, set_of, (size_t)n_streams * 4, cudaMemcpyHostToDevice,
                                     s)) != cudaSuccess)
                return bail(e, "cudaMemcpyAsync(parameter sets)");
        }
        *out = h;
        return ok();
    } catch (const std::bad_alloc&) {
        return fail(MTGP_ENOMEM, "host allocation failed");
    }
}

extern "C" mtgp_status mtgp_mt_init(const mtgp_mt_params* params, const uint32_t* seeds,
                                    uint32_t n_streams, void* cuda_stream, mtgp_mt_t* out)
{
    return init_handle(params, 1, nullptr, seeds, n_streams, cuda_stream, out);
}

extern "C" mtgp_status mtgp_mt_init_multi(const mtgp_mt_params* sets, uint32_t n_sets,
                                          const uint32_t* set_of_stream, const uint32_t* seeds,
                                          uint32_t n_streams, void* cuda_stream, mtgp_mt_t* out)
{
    if (!set_of_stream)
        return fail(MTGP_EINVAL, "null argument");
    return init_handle(sets, n_sets, set_of_stream, seeds, n_streams, cuda_stream, out);
}

extern "C" mtgp_status mtgp_mt_set_statuses(mtgp_mt_t h, const uint32_t* states, void* cuda_stream)
{
    if (!h || !states)
        return fail(MTGP_EINVAL, "null argument");
    DeviceGuard g(h->device);
    cudaStream_t s = (cudaStream_t)cuda_stream;
    const size_t n = h->k.n, np = h->k.np;
    MT_TRY(cudaMemcpy2DAsync(h->d_states, np * 4, states, n * 4, n * 4, h->n_streams,
                             cudaMemcpyHostToDevice, s),
           "cudaMemcpy2DAsync(set statuses)");
    MT_TRY(cudaStreamSynchronize(s), "cudaStreamSynchronize");
    return ok();
}

extern "C" mtgp_status mtgp_mt_get_statuses(mtgp_mt_t h, uint32_t* states, void* cuda_stream)
{
    if (!h || !states)
        return fail(MTGP_EINVAL, "null argument");
    DeviceGuard g(h->device);
    cudaStream_t s = (cudaStream_t)cuda_stream;
    const size_t n = h->k.n, np = h->k.np;
    MT_TRY(cudaMemcpy2DAsync(states, n * 4, h->d_states, np * 4, n * 4, h->n_streams,
                             cudaMemcpyDeviceToHost, s),
           "cudaMemcpy2DAsync(get statuses)");
    MT_TRY(cudaStreamSynchronize(s), "cudaStreamSynchronize");
    return ok();
}

extern "C" mtgp_status mtgp_mt_generate(mtgp_mt_t h, const uint32_t* ids, const uint64_t* counts,
                                        uint32_t n_req, mtgp_format fmt, void* out, void* cuda_stream)
{
    try {
        if (!h)
            return fail(MTGP_EINVAL, "null handle");
        if ((uint32_t)fmt > 2u)
            return fail(MTGP_EINVAL, "format %d", (int)fmt);
        Work w;
        mtgp_status st = build_work(h->n_streams, ids, counts, nullptr, (uint32_t)fmt, n_req, 0, w);
        if (st != MTGP_OK)
            return st;
        if (w.items.empty())
            return ok();
        if (!out || ((uintptr_t)out & 3u))
            return fail(MTGP_EINVAL, "output pointer null or not 4-byte aligned");
        DeviceGuard g(h->device);
        cudaStream_t s = (cudaStream_t)cuda_stream;
        TableSlot& sl = h->slots[h->next_slot];
        h->next_slot = (h->next_slot + 1) % (int)h->slots.size();
        if (sl.ev_recorded) {
            MT_TRY(cudaEventSynchronize(sl.ev), "cudaEventSynchronize(table slot)");
            sl.ev_recorded = false;
        }
        size_t io, so;
        const size_t bytes = table_bytes(w, &io, &so);
        if (bytes > sl.cap) {
            if (sl.host)
                cudaFreeHost(sl.host);
            if (sl.dev)
                cudaFree(sl.dev);
            sl.host = sl.dev = nullptr;
            sl.cap = 0;
            const size_t cap = std::max<size_t>(bytes * 2, 1 << 16);
            MT_TRY(cudaMallocHost(&sl.host, cap), "cudaMallocHost(work table)");
            MT_TRY(cudaMalloc(&sl.dev, cap), "cudaMalloc(work table)");
            sl.cap = cap;
        }
        fill_table(w, sl.host);
        MT_TRY(cudaMemcpyAsync(sl.dev, sl.host, bytes, cudaMemcpyHostToDevice, s),
               "cudaMemcpyAsync(work table)");
        // Warp count: every stream runs on one warp, longest first, so the
        // launch cannot end before its longest stream does.  About
        // total / longest warps keep pace with that stream; more warps only
        // slow it down by sharing its SM.  At least one CTA per SM.
        const uint32_t n_items = (uint32_t)w.items.size();
        const long long pace = (long long)((w.total + w.max_item - 1) / w.max_item);
        const long long warps = std::max<long long>(pace, (long long)h->sms * kWarpsPerCta);
        const long long want = (std::min<long long>(n_items, warps) + kWarpsPerCta - 1) / kWarpsPerCta;
        const int grid = (int)std::max(1LL, std::min<long long>(want, h->grid_cap));
        const WorkItem* items = (const WorkItem*)((char*)sl.dev + io);
        const Segment* segs = (const Segment*)((char*)sl.dev + so);
        uint32_t* counter = (uint32_t*)sl.dev;
        uint32_t* o = (uint32_t*)out;
        MtK P = h->k;
        uint32_t* states = h->d_states;
        uint32_t n_streams = h->n_streams;
        int* err = h->d_err;
        const MtSet* sets = h->d_sets;
        const uint32_t* set_of = h->d_set_of;
        void* args[] = {&P,       &states, &n_streams, &items, &segs, (void*)&n_items,
                        &counter, &o,      &err,       &sets,  &set_of};
        MT_TRY(cudaLaunchKernel(mt_kernel_ptr(h->K), dim3(grid), dim3(h->threads), args, h->smem, s),
               "MT generation kernel launch");
        MT_TRY(cudaGetLastError(), "MT generation kernel launch");
        MT_TRY(cudaEventRecord(sl.ev, s), "cudaEventRecord");
        sl.ev_recorded = true;
        return ok();
    } catch (const std::bad_alloc&) {
        return fail(MTGP_ENOMEM, "host allocation failed");
    }
}

extern "C" mtgp_status mtgp_mt_check(mtgp_mt_t h, void* cuda_stream)
{
    if (!h)
        return fail(MTGP_EINVAL, "null handle");
    DeviceGuard g(h->device);
    MT_TRY(cudaStreamSynchronize((cudaStream_t)cuda_stream), "cudaStreamSynchronize");
    int v = 0;
    MT_TRY(cudaMemcpy(&v, h->d_err, sizeof v, cudaMemcpyDeviceToHost), "cudaMemcpy(error word)");
    if (v) {
        MT_TRY(cudaMemset(h->d_err, 0, sizeof(int)), "cudaMemset");
        return fail(MTGP_EDEVICE, "a kernel recorded an inconsistent work item (code %d)", v);
    }
    return ok();
}

extern "C" mtgp_status mtgp_mt_free(mtgp_mt_t h)
{
    destroy_mt(h);
    return ok();
}

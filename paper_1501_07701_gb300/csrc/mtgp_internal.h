// Internal declarations shared by the host runtime (mtgp_api.cpp,
// mtgp_server.cpp) and the kernels (mtgp_kernels.cu, mtgp_fast_*.cu).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

namespace mtgp {

// Parameterized status in the form the kernels take it (by value, so it
// lives in the kernel-parameter constant bank).  flt[k] = (tmp[k] >> 9) |
// 0x3F800000 is the precomputed float tempering table of a "fast" status:
// (x >> 9) ^ flt[k] is the [1,2) bit pattern of x ^ tmp[k].
struct KParams {
    uint32_t n;      // state words N
    uint32_t np;     // HBM row stride in words: N rounded up to 4 (16-byte rows)
    uint32_t pos, sh1, sh2, mask;
    uint32_t mirror; // columns repeated after S[N) by the register-resident kernel:
                     // 32 * ceil((pos + 31) / 32)
    uint32_t rec[16];
    uint32_t tmp[16];
    uint32_t flt[16];
};

// One parameter set of a handle whose streams do not all share the handle's
// set (per-stream parameter sets, the paper's setting of one parameterized
// status per stream).  All sets of a handle have the same Mexp, hence the same
// N and mask; the kernels read pos, the shifts, the mirror width and the three
// tables per stream from here.
struct KSet {
    uint32_t pos, sh1, sh2, mirror;
    uint32_t rec[16];
    uint32_t tmp[16];
    uint32_t flt[16];
};

// One stream touched by a launch.  Its requests are the segments
// [seg_begin, seg_begin + nseg); they are generated back to back, so the
// stream's output index g runs over 0 .. total-1 across its segments.
// `stream` is the row of the launch's state array that the item advances:
// the stream's own row, or, in a split launch, a row of the launch's own
// array (see SplitWork).
struct WorkItem {
    uint32_t stream;
    uint32_t seg_begin;
    uint32_t nseg;
    uint32_t pad;
};

// One request of a stream: numbers g in [g_start, g_start + count) of the
// item go to out[out_off + (g - g_start)] in format fmt (0 u32, 1 f32 [1,2),
// 2 f32 [0,1)); req = the request's index in the call (its statistics row).
struct Segment {
    uint64_t g_start;
    uint64_t count;
    uint64_t out_off;
    uint32_t fmt;
    uint32_t req;
};

struct LaunchCfg {
    int warps_per_cta;   // G: 2, 4 or 8 for the register-resident kernel (1..8 ring)
    int ctas_per_sm;     // 0 = occupancy maximum
    int k;               // sub-steps per parallel step (words per lane), 2, 4 or 8
    int kernel;          // 0 register-resident, 1 shared-memory ring
    int coop_percent;    // streams longer than coop_percent/100 x (numbers per warp
                         // slot) are advanced by a whole CTA; 0 = never
};

// Per-warp shared-memory footprint (32-bit words).
//   fast: S[0 .. N + mirror) rounded up to 4 words (16-byte aligned rows for
//         the cp.async stage-in).
//   ring: the warp's REC/TMP tables (32 words), then S[0 .. N) rounded up
//         to 4 words.
__host__ __device__ inline uint32_t fast_smem_words(uint32_t n, uint32_t mirror)
{
    return (n + mirror + 3u) & ~3u;
}
__host__ __device__ inline uint32_t ring_smem_words(uint32_t n) { return 32u + ((n + 3u) & ~3u); }

// True if the register-resident kernel has an instantiation for this N, k
// and g warps per CTA, the window 32*k fits (32*k <= N - pos), and the
// shifts are in 1..31.
bool fast_supported(const KParams& P, int k, int g = 4);

// Lets `fn` launch with `need` bytes of dynamic shared memory: when need plus
// the function's static shared memory exceeds the 48 KB available without
// opt-in, the function's dynamic limit is raised to the device's opt-in
// maximum less its static shared memory (cudaErrorInvalidValue if `need`
// exceeds that).  The limit is a process-wide attribute of the function, so
// it is always raised to that maximum: a per-handle value could lower it
// under another live handle.  Occupancy still follows each launch's own size.
cudaError_t allow_max_dynamic_smem(const void* fn, int device, size_t need);

// Seed status -> state rows (row stride P.np words; padding words zeroed).
cudaError_t launch_init(const KParams& P, const uint32_t* d_seeds, uint32_t n_streams,
                        uint32_t* d_states, cudaStream_t s);

struct GenArgs {
    KParams P;
    uint32_t* states;
    uint32_t n_streams;
    const WorkItem* items;
    const Segment* segs;
    uint32_t n_items;
    uint32_t n_coop;     // items [0, n_coop) are advanced by whole CTAs
    uint32_t* counter;   // two claim counters, zeroed before the launch
    uint32_t* out;
    int* err;
    uint64_t* trace;     // optional: 4 words per item (start ns, end ns, SM, numbers)
    const KSet* sets = nullptr;        // per-stream parameter sets (null: every stream uses P)
    const uint32_t* set_of = nullptr;  // set index of each stream when `sets` is given
};

// Jump of one state row by a count J: row `stream` of the array given to the
// launch, polynomial `poly` of the launch's table (degree `deg`), parameter
// set `set` (per-stream sets) or 0.
struct JumpItem {
    uint32_t stream;
    uint32_t poly;
    uint32_t deg;
    uint32_t set;
};

// Copies state rows: dst[pairs[i].y] = src[pairs[i].x], N words each (row
// stride np).
cudaError_t launch_copy_rows(const uint32_t* src, uint32_t* dst, const uint2* pairs, uint32_t n,
                             uint32_t N, uint32_t np, cudaStream_t s);

// Resolved launch geometry for a configuration.
struct Geometry {
    int kernel;          // kernel actually used (fast falls back to ring)
    int k;
    int threads;
    size_t smem;
    int grid;
    int regs;            // registers per thread of the kernel used
    int per_sm;          // resident CTAs per SM (occupancy, after the cap)
};

// Works out kernel choice, block size, shared memory and grid (persistent:
// at most num_sms * resident CTAs, at least enough warps for n_items when
// fewer).  Returns cudaSuccess or the occupancy query's error.
cudaError_t plan_geometry(const KParams& P, const LaunchCfg& cfg, uint32_t n_items, int device,
                          Geometry* g);

// Launches the generation kernel described by `g` (counter must be zero).
cudaError_t launch_generate(const GenArgs& a, const Geometry& g, cudaStream_t s);

// Fast-kernel launchers, one translation unit per group of state sizes.
// M = ceil(N / 32) register columns per lane; returns cudaErrorInvalidValue
// if M or K has no instantiation.
cudaError_t launch_fast(int M, int K, int G, const GenArgs& a, dim3 grid, dim3 block, size_t smem,
                        cudaStream_t s);
const void* fast_kernel_ptr(int M, int K, int G);

// Launches a generation kernel with the register-resident kernel's signature.
cudaError_t launch_gen_fn(const void* fn, const GenArgs& a, dim3 grid, dim3 block, size_t smem,
                          cudaStream_t s);

// Statistics of the paper's gap test (test 35) and Hamming-weight
// independence test (test 100), Sec. 4.2, accumulated by the fused
// generation kernel per request of its launch.
// What one piece of a request (a segment of a split launch) leaves for the
// stitch: its gap-test edges and its Hamming weights in the block pairs that
// are open at its start and at its end.
struct SegStat {
    uint32_t gprefix;   // non-visits before the piece's first visit (its length if none)
    uint32_t gsuffix;   // non-visits after its last visit (its length if none)
    uint32_t gvisit;    // 1 if the piece has a visit
    uint32_t la, lb;    // weights in blocks a and b of the pair open at the piece's start
    uint32_t ta, tb;    // weights in blocks a and b of the pair open at its end
    uint32_t pad;
};

struct StatsArgs {
    uint32_t gmask;                // gap test: the b bits after r dropped leading bits (0: off)
    uint32_t t;                    // gap lengths >= t pooled in class t (t + 1 counts)
    uint32_t hmask;                // Hamming test: the s bits after r dropped leading bits (0: off)
    uint32_t K;                    // values per L-bit block (L / s), >= 32
    uint32_t C;                    // weight classes (n_bounds + 1), <= 16
    uint32_t bounds[15];           // class of weight w = number of bounds <= w
    unsigned long long* hist;      // n_req x (t + 1) counts, added to
    unsigned long long* tab;       // n_req x C x C counts, added to
    // split launches (null otherwise): each request's first output index
    // (a segment's position in its request is out_off - req_base[req]) and
    // one record per segment for the stitch
    const unsigned long long* req_base;
    SegStat* seg_stats;
};

// Shared-memory words per warp that the statistics add: the gap histogram
// of the warp's current request (rounded up to 4 words), one slot per lane
// that absorbs the counts of non-visiting lanes, the request's C x C pair
// table (rounded up to 4 words) and 4 words of the current piece's edges.
__host__ __device__ inline uint32_t stats_smem_words(uint32_t t, uint32_t C)
{
    return ((t + 1u + 3u) & ~3u) + 32u + ((C * C + 3u) & ~3u) + 4u;
}

// The fused generation kernel (single-warp items, 128-word pipelined steps,
// N - pos >= 256 for every parameter set): null when M or G has no
// instantiation.  Launched like the register-resident kernel plus `A`
// (a.n_coop and a.trace are not used).
const void* fused_kernel_ptr(int M, int G);
cudaError_t launch_fused(const void* fn, const GenArgs& a, const StatsArgs& A, dim3 grid, dim3 block,
                         size_t smem, cudaStream_t s);
// Completes the statistics of split requests from their pieces' records:
// request j's pieces are segs[pieces[piece_start[j] ..  piece_start[j+1])],
// in request order (requests with one piece have none listed).
cudaError_t launch_stats_stitch(const Segment* segs, const uint32_t* piece_start, const uint32_t* pieces,
                                uint32_t n_req, const StatsArgs& A, cudaStream_t s);

}  // namespace mtgp

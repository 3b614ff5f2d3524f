// Allocation-free generation entry point.
//
// The ordinary generation calls keep their work table (claim counters,
// per-stream items, request segments) in buffers the library allocates on
// first use.  Some callers cannot have anything allocated on their behalf
// once they are running: code that owns a fixed device-memory budget
// (a simulation that has reserved the GPU's memory up front), code running
// where the allocator must not be entered (between a device-memory pool's
// setup and its use, or in a real-time loop that must not block on the
// allocator), or a host runtime that forbids hidden allocations.  This entry
// point serves them: it stages the work table in one statically sized
// device array that exists from library load on, and calls no cudaMalloc,
// cudaFree, pinned-host allocation or heap allocation.
//
// The scratch array is one per device and shared by every call on that
// device: a call overwrites what the previous one left there, and two calls
// whose kernels overlap on the GPU (different CUDA streams, or different
// host threads) race on it.  Callers must order such calls themselves.
//
// The work table is copied from one static host array that the next call
// overwrites, so a call is refused while its CUDA stream is being captured
// (a captured copy would read that array when the graph is replayed, long
// after the call that filled it).  The device address of the scratch array
// is looked up once per device and kept for the life of the process; a
// device reset (cudaDeviceReset) while the library is loaded is therefore not
// supported by this call.
#include <cstring>
#include <mutex>

#include "mtgp_runtime.h"

using namespace mtgp;

namespace {

// Largest request list one call accepts.  The table holds the two claim
// counters (256 bytes, cleared on every call), one 16-byte item per
// distinct stream and one 32-byte segment per request.
constexpr uint32_t kMaxRequests = 1024;
constexpr size_t kCountersBytes = 256;
constexpr size_t kItemsBytes = kMaxRequests * sizeof(WorkItem);
constexpr size_t kScratchBytes = kCountersBytes + kItemsBytes + kMaxRequests * sizeof(Segment);

// The scratch array: 64 KiB of device memory held by every device that
// loads the library, until the process exits.
static __device__ __align__(256) unsigned char g_noalloc_scratch[65536];
static_assert(kScratchBytes <= sizeof(g_noalloc_scratch), "scratch too small");

constexpr int kMaxDevices = 64;
std::mutex g_setup_mu;
void* g_scratch_addr[kMaxDevices] = {};

// Device address of the scratch array on `device` (which is current).  The
// host-side name of the array is only a stand-in; its device address comes
// from cudaGetSymbolAddress, once per device.
cudaError_t scratch_address(int device, void** ptr)
{
    if (device < 0 || device >= kMaxDevices)
        return cudaErrorInvalidDevice;
    std::lock_guard<std::mutex> lk(g_setup_mu);
    if (!g_scratch_addr[device]) {
        void* p = nullptr;
        const cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
        if (e != cudaSuccess)
            return e;
        g_scratch_addr[device] = p;
    }
    *ptr = g_scratch_addr[device];
    return cudaSuccess;
}

// Host-side table built without heap allocation: one static staging table,
// used under g_table_mu (a call holds it from building the table until the
// upload has read it).
struct StaticTable {
    unsigned char bytes[kScratchBytes];
    uint64_t item_total[kMaxRequests];
};
StaticTable g_table;
std::mutex g_table_mu;

}  // namespace

extern "C" mtgp_status mtgp_generate_noalloc(mtgp_streams_t st, const uint32_t* ids,
                                             const uint64_t* counts, uint32_t n_req, mtgp_format fmt,
                                             void* out, void* cuda_stream)
{
    GUARD_BEGIN
    if (!st)
        return fail(MTGP_EINVAL, "null handle");
    if ((uint32_t)fmt > 2)
        return fail(MTGP_EINVAL, "format %d", (int)fmt);
    if (n_req > kMaxRequests)
        return fail(MTGP_EINVAL,
                    "mtgp_generate_noalloc takes at most %u requests per call (got %u); "
                    "split the list or use mtgp_generate_u32/_f32",
                    kMaxRequests, n_req);
    if (n_req && (!ids || !counts))
        return fail(MTGP_EINVAL, "null request arrays");
    uint64_t total = 0;
    for (uint32_t j = 0; j < n_req; ++j) {
        if (ids[j] >= st->n_streams)
            return fail(MTGP_EINVAL, "stream id %u >= n_streams %u (request %u)", ids[j],
                        st->n_streams, j);
        if (counts[j] > (1ull << 50) || total + counts[j] < total)
            return fail(MTGP_EINVAL, "count too large (request %u)", j);
        total += counts[j];
    }
    if (total == 0)
        return ok();
    if (!out)
        return fail(MTGP_EINVAL, "null output pointer");

    DeviceGuard guard(st->device);
    cudaStream_t cs = (cudaStream_t)cuda_stream;
    cudaStreamCaptureStatus capturing = cudaStreamCaptureStatusNone;
    cudaError_t e = cudaStreamIsCapturing(cs, &capturing);
    if (e != cudaSuccess)
        return fail_cuda(e, "cudaStreamIsCapturing");
    if (capturing != cudaStreamCaptureStatusNone)
        return fail(MTGP_EINVAL, "mtgp_generate_noalloc cannot be recorded into a CUDA graph: its "
                                 "work table is copied from host memory that the next call "
                                 "overwrites (use mtgp_plan_create for graphs)");
    void* scratch = nullptr;
    e = scratch_address(st->device, &scratch);
    if (e != cudaSuccess)
        return fail_cuda(e, "cudaGetSymbolAddress(no-alloc scratch)");

    // Work table in the layout the kernels read: counters | items | segments.
    // Items: one per distinct stream, its requests in call order; output
    // offsets are the exclusive prefix sums of counts.  Items are then
    // ordered longest first (insertion sort over at most kMaxRequests).
    std::lock_guard<std::mutex> lk(g_table_mu);
    StaticTable& T = g_table;
    std::memset(T.bytes, 0, kCountersBytes);
    WorkItem* items = reinterpret_cast<WorkItem*>(T.bytes + kCountersBytes);
    Segment* segs = reinterpret_cast<Segment*>(T.bytes + kCountersBytes + kItemsBytes);
    uint32_t n_items = 0, n_segs = 0;
    for (uint32_t j = 0; j < n_req; ++j) {
        if (counts[j] == 0)
            continue;
        bool seen = false;
        for (uint32_t k = 0; k < j && !seen; ++k)
            seen = counts[k] != 0 && ids[k] == ids[j];
        if (seen)
            continue;
        WorkItem it;
        it.stream = ids[j];
        it.seg_begin = n_segs;
        it.pad = 0;
        uint64_t g = 0, off = 0;
        for (uint32_t k = 0; k < n_req; ++k) {
            if (ids[k] == ids[j] && counts[k] != 0) {
                Segment& s = segs[n_segs++];
                s.g_start = g;
                s.count = counts[k];
                s.out_off = off;
                s.fmt = (uint32_t)fmt;
                s.req = k;
                g += counts[k];
            }
            off += counts[k];
        }
        it.nseg = n_segs - it.seg_begin;
        T.item_total[n_items] = g;
        items[n_items++] = it;
    }
    for (uint32_t a = 1; a < n_items; ++a) {
        const WorkItem it = items[a];
        const uint64_t tt = T.item_total[a];
        uint32_t b = a;
        while (b > 0 && T.item_total[b - 1] < tt) {
            items[b] = items[b - 1];
            T.item_total[b] = T.item_total[b - 1];
            --b;
        }
        items[b] = it;
        T.item_total[b] = tt;
    }

    Geometry g;
    mtgp_status s = geometry_for(st, st->cfg, n_items, &g);
    if (s != MTGP_OK)
        return s;
    // Longest streams to whole CTAs, as in the ordinary path.
    uint32_t n_coop = 0;
    if (g.kernel == 0 && st->cfg.coop_percent > 0 && g.k >= g.threads / 32 && !st->d_sets) {
        const double slots = (double)g.grid * (double)(g.threads / 32);
        const double thr = (double)total / slots * (double)st->cfg.coop_percent / 100.0;
        while (n_coop < n_items && (double)T.item_total[n_coop] >= thr)
            ++n_coop;
    }

    // Upload (pageable source: the copy has read the host table when the call
    // returns) and launch.  The counters are part of the upload, so every
    // call starts them at zero.
    const size_t bytes = kCountersBytes + kItemsBytes + (size_t)n_segs * sizeof(Segment);
    e = cudaMemcpyAsync(scratch, T.bytes, bytes, cudaMemcpyHostToDevice, cs);
    if (e != cudaSuccess)
        return fail_cuda(e, "cudaMemcpyAsync(no-alloc table)");
    GenArgs a;
    a.P = st->P.k;
    a.states = st->d_states;
    a.n_streams = st->n_streams;
    a.items = reinterpret_cast<const WorkItem*>((unsigned char*)scratch + kCountersBytes);
    a.segs = reinterpret_cast<const Segment*>((unsigned char*)scratch + kCountersBytes + kItemsBytes);
    a.n_items = n_items;
    a.n_coop = n_coop;
    a.counter = reinterpret_cast<uint32_t*>(scratch);
    a.out = (uint32_t*)out;
    a.err = st->d_err;
    a.trace = nullptr;
    a.sets = st->d_sets;
    a.set_of = st->d_set_of;
    e = launch_generate(a, g, cs);
    if (e != cudaSuccess)
        return fail_cuda(e, "generation kernel launch (no-alloc)");
    return ok();
    GUARD_END
}

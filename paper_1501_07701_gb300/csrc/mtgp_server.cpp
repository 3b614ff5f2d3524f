// Serving front end: requests "k numbers from stream s" against resident
// stream states, admitted by output-arena space, coalesced into ticks (one
// kernel launch each) that overlap on the device on separate CUDA streams.
//
// Ordering: a stream whose request is inside an in-flight tick is busy; its
// later requests wait (and block every request behind them for the same
// stream) until that tick completes, so each stream sees its requests in
// submission order and no two kernels touch one state at once.  Requests for
// one stream admitted into the same tick become consecutive segments of one
// work item, in order.
//
// Failure detection: every wait for a tick's completion is bounded by the
// server's tick_timeout_s.  A tick whose completion has not been observed
// that long after its launch makes progress / run_trace return
// MTGP_ETIMEOUT; the tick stays marked in flight, so a later call picks it up
// if it does complete.  A diagnostic hold makes completion queries report
// "not ready" (the kernels still run to completion), which lets tests reach
// that path without stalling the GPU.
#include <time.h>

#include <algorithm>
#include <chrono>
#include <cstring>
#include <deque>
#include <list>
#include <map>
#include <thread>
#include <vector>

#include "mtgp_runtime.h"

#define CUDA_TRY_S(call, what)               \
    do {                                     \
        cudaError_t e_ = (call);             \
        if (e_ != cudaSuccess)               \
            return fail_cuda(e_, what);      \
    } while (0)

using namespace mtgp;

namespace {

double now_s()
{
    using namespace std::chrono;
    return duration<double>(steady_clock::now().time_since_epoch()).count();
}

// First-fit allocator over the arena, in 32-element (128-byte) granules.
struct ArenaAlloc {
    std::map<uint64_t, uint64_t> free_;   // offset -> size (elements)
    uint64_t total = 0;
    uint64_t used = 0;

    void reset(uint64_t elems)
    {
        free_.clear();
        total = elems & ~31ull;
        used = 0;
        if (total)
            free_[0] = total;
    }
    static uint64_t round(uint64_t n) { return (std::max<uint64_t>(n, 1) + 31) & ~31ull; }
    bool alloc(uint64_t n, uint64_t* off)
    {
        n = round(n);
        for (auto it = free_.begin(); it != free_.end(); ++it) {
            if (it->second >= n) {
                *off = it->first;
                const uint64_t rest = it->second - n;
                const uint64_t noff = it->first + n;
                free_.erase(it);
                if (rest)
                    free_[noff] = rest;
                used += n;
                return true;
            }
        }
        return false;
    }
    void release(uint64_t off, uint64_t n)
    {
        n = round(n);
        used -= n;
        auto it = free_.emplace(off, n).first;
        auto nx = std::next(it);
        if (nx != free_.end() && it->first + it->second == nx->first) {
            it->second += nx->second;
            free_.erase(nx);
        }
        if (it != free_.begin()) {
            auto pv = std::prev(it);
            if (pv->first + pv->second == it->first) {
                pv->second += it->second;
                free_.erase(it);
            }
        }
    }
};

struct Req {
    uint32_t stream;
    int32_t fmt;
    uint64_t count;
    uint64_t tag;
    uint64_t off;        // arena element offset once admitted
    double t_submit;
    bool live;
};

// Device buffers of a tick whose long requests are split (config
// max_piece): the launch's own state rows, and one table of row copies
// (stream -> row, row -> stream), row parameter sets, jump items and jump
// polynomials, assembled on the host and uploaded in one copy.
struct TickSplit {
    uint32_t* rows = nullptr;
    size_t rows_cap = 0;   // words
    char* aux = nullptr;
    size_t aux_cap = 0;    // bytes
    std::vector<char> host;
};

struct Tick {
    std::vector<uint32_t> reqs;
    cudaStream_t cs = nullptr;
    cudaEvent_t ev = nullptr;
    TableSlot slot;
    TickSplit sp;
    bool busy = false;
    double t_launch = 0;   // steady-clock seconds at launch
};

}  // namespace

struct mtgp_server {
    mtgp_streams* st = nullptr;
    mtgp_server_config cfg{};
    void* arena = nullptr;
    ArenaAlloc alloc;
    std::vector<Req> reqs;
    std::vector<uint32_t> free_reqs;
    std::list<uint32_t> pending;
    std::vector<uint8_t> busy;          // per stream: inside an in-flight tick
    std::vector<uint32_t> blocked;      // per stream: epoch stamp of the current admission scan
    uint32_t epoch = 0;
    std::vector<Tick> ticks;
    std::deque<mtgp_completion> done;
    uint64_t n_ticks = 0;
    uint64_t n_numbers = 0;
    uint64_t n_requests = 0;
    bool keep_results = false;          // trace mode with recorded offsets
    bool hold = false;                  // diagnostic: completions read as not ready
    double launch_host_s = 0;           // host time in work-table builds and launches
    std::vector<uint32_t> set_of_stream; // per-stream parameter set (handles with one per stream)
    std::vector<KSet> host_sets;        // those sets, for the ticks' jump polynomials
    uint64_t n_jumps = 0;               // pieces started by jumps
    // jump polynomials of the piece offsets j * max_piece, j = 1 .. 63, on
    // the device (handles with one parameter set): a tick's jumps then need
    // only their items
    uint32_t* d_polys = nullptr;
    uint32_t poly_words = 0;
    size_t jump_smem = 0;
    std::vector<uint32_t> poly_deg;     // degree of polynomial j - 1
};

// Completion query of one event, bounded by the server's deadline.  Returns
// MTGP_OK with *ready set, MTGP_ETIMEOUT once `t_launch + tick_timeout_s` has
// passed without completion, or MTGP_ECUDA for a failed query.
static mtgp_status query_done(const mtgp_server* s, cudaEvent_t ev, double t_launch, bool* ready)
{
    *ready = false;
    const cudaError_t e = s->hold ? cudaErrorNotReady : cudaEventQuery(ev);
    if (e == cudaSuccess) {
        *ready = true;
        return MTGP_OK;
    }
    if (e != cudaErrorNotReady)
        return fail_cuda(e, "tick completion");
    const double waited = now_s() - t_launch;
    if (waited > s->cfg.tick_timeout_s)
        return fail(MTGP_ETIMEOUT, "a launch has not completed %.3f s after it was issued "
                    "(limit %.3f s)", waited, s->cfg.tick_timeout_s);
    return MTGP_OK;
}

static void destroy_server(mtgp_server* s)
{
    if (!s)
        return;
    DeviceGuard g(s->st->device);
    for (Tick& t : s->ticks) {
        if (t.cs)
            cudaStreamSynchronize(t.cs);
        free_table_slot(t.slot);
        if (t.slot.ev)
            cudaEventDestroy(t.slot.ev);
        if (t.sp.rows)
            cudaFree(t.sp.rows);
        if (t.sp.aux)
            cudaFree(t.sp.aux);
        if (t.ev)
            cudaEventDestroy(t.ev);
        if (t.cs)
            cudaStreamDestroy(t.cs);
    }
    if (s->arena)
        cudaFree(s->arena);
    if (s->d_polys)
        cudaFree(s->d_polys);
    delete s;
}

extern "C" mtgp_status mtgp_server_create(mtgp_streams_t st, const mtgp_server_config* cfg,
                                          mtgp_server_t* out)
{
    try {
        if (!st || !out)
            return fail(MTGP_EINVAL, "null argument");
        mtgp_server_config c{};
        if (cfg)
            c = *cfg;
        if (c.arena_bytes == 0)
            c.arena_bytes = 8ull << 30;
        if (c.max_inflight == 0)
            c.max_inflight = 4;
        if (c.max_tick_requests == 0)
            c.max_tick_requests = 4096;
        if (c.tick_timeout_s == 0)
            c.tick_timeout_s = 60.0;
        if (c.max_inflight > 64)
            return fail(MTGP_EINVAL, "max_inflight %u > 64", c.max_inflight);
        if (!(c.tick_timeout_s > 0))
            return fail(MTGP_EINVAL, "tick_timeout_s must be positive");
        if (c.max_piece != 0 && c.max_piece < 64)
            return fail(MTGP_EINVAL, "max_piece %llu below 64", (unsigned long long)c.max_piece);
        DeviceGuard g(st->device);
        mtgp_server* s = new mtgp_server;
        s->st = st;
        s->cfg = c;
        s->busy.assign(st->n_streams, 0);
        s->blocked.assign(st->n_streams, 0);
        s->ticks.resize(c.max_inflight);
        cudaError_t e = cudaMalloc(&s->arena, c.arena_bytes);
        if (e != cudaSuccess) {
            destroy_server(s);
            return fail_cuda(e, "cudaMalloc(arena)");
        }
        s->alloc.reset(c.arena_bytes / 4);
        if (c.max_piece) {
            if (st->d_sets) {
                s->set_of_stream.resize(st->n_streams);
                s->host_sets.resize(st->n_sets);
                e = cudaMemcpy(s->set_of_stream.data(), st->d_set_of, st->n_streams * 4u,
                               cudaMemcpyDeviceToHost);
                if (e == cudaSuccess)
                    e = cudaMemcpy(s->host_sets.data(), st->d_sets, st->n_sets * sizeof(KSet),
                                   cudaMemcpyDeviceToHost);
                if (e != cudaSuccess) {
                    destroy_server(s);
                    return fail_cuda(e, "cudaMemcpy(set index)");
                }
            } else {
                // the jump polynomials of the piece offsets j * max_piece
                // (j < 64) are computed once here rather than in a tick
                std::vector<uint32_t> rows(63, 0u), sets(63, 0u);
                std::vector<uint64_t> lens(63);
                for (uint32_t j = 0; j < 63u; ++j)
                    lens[j] = (uint64_t)(j + 1u) * c.max_piece;
                JumpBatch jb;
                mtgp_status r = build_jump_batch(st, rows, sets, lens, &jb);
                if (r != MTGP_OK) {
                    destroy_server(s);
                    return r;
                }
                // one polynomial per offset, in offset order (the batch lists
                // distinct lengths once, sorted)
                s->poly_deg.assign(63, 0u);
                for (const JumpItem& ji : jb.items)
                    s->poly_deg[ji.poly] = ji.deg;
                s->poly_words = jb.words;
                s->jump_smem = jb.smem;
                e = cudaMalloc(&s->d_polys, jb.poly_words.size() * 4u);
                if (e == cudaSuccess)
                    e = cudaMemcpy(s->d_polys, jb.poly_words.data(), jb.poly_words.size() * 4u,
                                   cudaMemcpyHostToDevice);
                if (e != cudaSuccess) {
                    destroy_server(s);
                    return fail_cuda(e, "jump polynomials");
                }
            }
        }
        for (Tick& t : s->ticks) {
            if ((e = cudaStreamCreateWithFlags(&t.cs, cudaStreamNonBlocking)) != cudaSuccess ||
                (e = cudaEventCreateWithFlags(&t.ev, cudaEventDisableTiming)) != cudaSuccess ||
                (e = cudaEventCreateWithFlags(&t.slot.ev, cudaEventDisableTiming)) != cudaSuccess) {
                destroy_server(s);
                return fail_cuda(e, "server stream/event");
            }
        }
        *out = s;
        return ok();
    } catch (...) {
        return fail(MTGP_ENOMEM, "host allocation failed");
    }
}

static uint32_t new_req(mtgp_server* s)
{
    if (!s->free_reqs.empty()) {
        const uint32_t i = s->free_reqs.back();
        s->free_reqs.pop_back();
        return i;
    }
    s->reqs.push_back(Req{});
    return (uint32_t)s->reqs.size() - 1;
}

static mtgp_status submit(mtgp_server* s, uint32_t stream, uint64_t count, int32_t fmt, uint64_t tag,
                          double t_submit)
{
    if (stream >= s->st->n_streams)
        return fail(MTGP_EINVAL, "stream id %u >= %u", stream, s->st->n_streams);
    if (fmt < 0 || fmt > 2)
        return fail(MTGP_EINVAL, "format %d", fmt);
    if (count == 0 || ArenaAlloc::round(count) > s->alloc.total)
        return fail(MTGP_EBUSY, "request of %llu numbers cannot fit the arena (%llu elements)",
                    (unsigned long long)count, (unsigned long long)s->alloc.total);
    const uint32_t i = new_req(s);
    Req& r = s->reqs[i];
    r.stream = stream;
    r.fmt = fmt;
    r.count = count;
    r.tag = tag;
    r.off = 0;
    r.t_submit = t_submit;
    r.live = true;
    s->pending.push_back(i);
    return MTGP_OK;
}

extern "C" mtgp_status mtgp_server_submit(mtgp_server_t s, uint32_t stream_id, uint64_t count,
                                          mtgp_format fmt, uint64_t tag)
{
    if (!s)
        return fail(MTGP_EINVAL, "null server");
    try {
        mtgp_status r = submit(s, stream_id, count, (int32_t)fmt, tag, now_s());
        return r == MTGP_OK ? ok() : r;
    } catch (...) {
        return fail(MTGP_ENOMEM, "host allocation failed");
    }
}

// Collects finished ticks.  Completed requests go to s->done.
static mtgp_status reap(mtgp_server* s, int* n_reaped)
{
    *n_reaped = 0;
    for (Tick& t : s->ticks) {
        if (!t.busy)
            continue;
        bool ready = false;
        const mtgp_status qs = query_done(s, t.ev, t.t_launch, &ready);
        if (qs != MTGP_OK)
            return qs;
        if (!ready)
            continue;
        const double tn = now_s();
        for (uint32_t i : t.reqs) {
            Req& r = s->reqs[i];
            mtgp_completion c;
            c.tag = r.tag;
            c.count = r.count;
            c.arena_offset = r.off;
            c.fmt = r.fmt;
            c.pad = 0;
            c.submit_time = r.t_submit;
            c.done_time = tn;
            s->done.push_back(c);
            s->busy[r.stream] = 0;
            r.live = false;
            s->free_reqs.push_back(i);
            s->n_numbers += r.count;
            ++s->n_requests;
        }
        t.reqs.clear();
        t.busy = false;
        ++*n_reaped;
    }
    return MTGP_OK;
}

// Admits pending requests into one free tick slot and launches it.  Sets
// *launched to 1 if a tick went out.
// Launches the tick's work with its items longer than max_piece cut into
// pieces (split_work): every item gets a row of the tick's own state array,
// the rows of later pieces are advanced by exact jumps, the generation
// kernel runs over the rows, and the unsplit items' rows and each split
// item's last piece become the streams' new states.  All on the tick's
// stream, in that order.
static mtgp_status launch_split_tick(mtgp_server* s, Tick& t, const Work& w)
{
    mtgp_streams* st = s->st;
    SplitWork sw;
    mtgp_status r = split_work(w, s->cfg.max_piece, 64, s->set_of_stream, &sw);
    if (r != MTGP_OK)
        return r;
    // jumps by j * max_piece (j < 64) take the server's device polynomials;
    // others (streams cut into 64 equal pieces, per-stream parameter sets)
    // get a batch of their own
    JumpBatch jb;
    bool cached = s->d_polys != nullptr;
    for (size_t i = 0; cached && i < sw.jump_lens.size(); ++i)
        cached = sw.jump_lens[i] % s->cfg.max_piece == 0 && sw.jump_lens[i] / s->cfg.max_piece <= 63u;
    if (cached) {
        for (size_t i = 0; i < sw.jump_rows.size(); ++i) {
            const uint32_t j = (uint32_t)(sw.jump_lens[i] / s->cfg.max_piece) - 1u;
            JumpItem ji;
            ji.stream = sw.jump_rows[i];
            ji.poly = j;
            ji.deg = s->poly_deg[j];
            ji.set = 0;
            jb.items.push_back(ji);
        }
        jb.words = s->poly_words;
        jb.smem = s->jump_smem;
    } else {
        r = build_jump_batch(st, sw.jump_rows, sw.jump_sets, sw.jump_lens, &jb,
                             st->d_sets ? &s->host_sets : nullptr);
        if (r != MTGP_OK)
            return r;
    }
    const uint32_t N = st->P.k.n, np = st->P.k.np;
    const size_t rows_words = (size_t)sw.n_rows * np;
    if (rows_words > t.sp.rows_cap) {
        if (t.sp.rows)
            cudaFree(t.sp.rows);
        t.sp.rows = nullptr;
        t.sp.rows_cap = 0;
        const size_t cap = std::max<size_t>(rows_words * 2, (size_t)64 * np);
        CUDA_TRY_S(cudaMalloc(&t.sp.rows, cap * 4u), "cudaMalloc(tick rows)");
        t.sp.rows_cap = cap;
    }
    auto al = [](size_t x) { return (x + 15u) & ~(size_t)15u; };
    const size_t b_copies = sw.copies.size() * sizeof(uint2), b_backs = sw.backs.size() * sizeof(uint2);
    const size_t b_set = st->d_sets ? sw.row_set.size() * 4u : 0u;
    const size_t b_ji = jb.items.size() * sizeof(JumpItem), b_poly = jb.poly_words.size() * 4u;
    const size_t o_backs = al(b_copies), o_set = o_backs + al(b_backs), o_ji = o_set + al(b_set);
    const size_t o_poly = o_ji + al(b_ji), total = o_poly + b_poly;
    t.sp.host.resize(total);
    std::memcpy(t.sp.host.data(), sw.copies.data(), b_copies);
    std::memcpy(t.sp.host.data() + o_backs, sw.backs.data(), b_backs);
    if (b_set)
        std::memcpy(t.sp.host.data() + o_set, sw.row_set.data(), b_set);
    if (b_ji)
        std::memcpy(t.sp.host.data() + o_ji, jb.items.data(), b_ji);
    if (b_poly)
        std::memcpy(t.sp.host.data() + o_poly, jb.poly_words.data(), b_poly);
    if (total > t.sp.aux_cap) {
        if (t.sp.aux)
            cudaFree(t.sp.aux);
        t.sp.aux = nullptr;
        t.sp.aux_cap = 0;
        const size_t cap = std::max<size_t>(total * 2, 1u << 16);
        CUDA_TRY_S(cudaMalloc(&t.sp.aux, cap), "cudaMalloc(tick split tables)");
        t.sp.aux_cap = cap;
    }
    CUDA_TRY_S(cudaMemcpyAsync(t.sp.aux, t.sp.host.data(), total, cudaMemcpyHostToDevice, t.cs),
               "cudaMemcpyAsync(tick split tables)");
    CUDA_TRY_S(launch_copy_rows(st->d_states, t.sp.rows, (const uint2*)t.sp.aux, (uint32_t)sw.copies.size(),
                                N, np, t.cs), "row copy");
    const uint32_t* polys = cached ? s->d_polys : (const uint32_t*)(t.sp.aux + o_poly);
    CUDA_TRY_S(launch_jump_batch(st, t.sp.rows, (const JumpItem*)(t.sp.aux + o_ji), (uint32_t)jb.items.size(),
                                 polys, jb.words, jb.smem, t.cs),
               "jump kernel");
    RowArray ra{t.sp.rows, sw.n_rows, st->d_sets ? (const uint32_t*)(t.sp.aux + o_set) : nullptr};
    r = launch_work_slot(st, t.slot, sw.work, st->cfg, s->arena, t.cs, &ra);
    if (r != MTGP_OK)
        return r;
    CUDA_TRY_S(launch_copy_rows(t.sp.rows, st->d_states, (const uint2*)(t.sp.aux + o_backs),
                                (uint32_t)sw.backs.size(), N, np, t.cs), "row copy back");
    s->n_jumps += jb.items.size();
    return MTGP_OK;
}

static mtgp_status admit_and_launch(mtgp_server* s, int* launched)
{
    *launched = 0;
    if (s->pending.empty())
        return MTGP_OK;
    Tick* t = nullptr;
    for (Tick& x : s->ticks)
        if (!x.busy) {
            t = &x;
            break;
        }
    if (!t)
        return MTGP_OK;
    ++s->epoch;
    if (s->epoch == 0) {
        std::fill(s->blocked.begin(), s->blocked.end(), 0);
        s->epoch = 1;
    }
    std::vector<uint32_t> ids;
    std::vector<uint64_t> counts, offs;
    std::vector<int32_t> fmts;
    // With max_piece, a tick takes either requests longer than it (split,
    // started by jumps) or shorter ones, so that short requests never wait
    // for a tick's jumps; the first request admitted sets the class.
    bool tick_long = false;
    for (auto it = s->pending.begin(); it != s->pending.end();) {
        Req& r = s->reqs[*it];
        const bool is_long = s->cfg.max_piece && r.count > s->cfg.max_piece;
        if (s->busy[r.stream] || s->blocked[r.stream] == s->epoch ||
            (!t->reqs.empty() && is_long != tick_long)) {
            s->blocked[r.stream] = s->epoch;   // keeps this stream's later requests behind it
            ++it;
            continue;
        }
        if (t->reqs.empty())
            tick_long = is_long;
        if (t->reqs.size() >= s->cfg.max_tick_requests)
            break;
        uint64_t off;
        if (!s->alloc.alloc(r.count, &off))
            break;   // arena full: first come, first served
        r.off = off;
        t->reqs.push_back(*it);
        ids.push_back(r.stream);
        counts.push_back(r.count);
        offs.push_back(off);
        fmts.push_back(r.fmt);
        it = s->pending.erase(it);
    }
    if (t->reqs.empty())
        return MTGP_OK;
    for (uint32_t i : t->reqs)
        s->busy[s->reqs[i].stream] = 1;
    const double tl = now_s();
    Work w;
    mtgp_status st = build_work(s->st->n_streams, ids.data(), counts.data(), fmts.data(), 0,
                                (uint32_t)ids.size(), 0, w, offs.data());
    if (st != MTGP_OK)
        return st;
    if (s->cfg.max_piece && w.max_item > s->cfg.max_piece)
        st = launch_split_tick(s, *t, w);
    else
        st = launch_work_slot(s->st, t->slot, w, s->st->cfg, s->arena, t->cs);
    if (st != MTGP_OK)
        return st;
    cudaError_t e = cudaEventRecord(t->ev, t->cs);
    if (e != cudaSuccess)
        return fail_cuda(e, "cudaEventRecord(tick)");
    t->busy = true;
    t->t_launch = now_s();
    s->launch_host_s += t->t_launch - tl;
    ++s->n_ticks;
    *launched = 1;
    return MTGP_OK;
}

extern "C" mtgp_status mtgp_server_progress(mtgp_server_t s, mtgp_completion* out, uint32_t max_out,
                                            uint32_t* n_out)
{
    if (!s || (max_out && !out))
        return fail(MTGP_EINVAL, "null argument");
    try {
        DeviceGuard g(s->st->device);
        int n = 0;
        mtgp_status st = reap(s, &n);
        if (st != MTGP_OK)
            return st;
        st = admit_and_launch(s, &n);
        if (st != MTGP_OK)
            return st;
        uint32_t k = 0;
        while (k < max_out && !s->done.empty()) {
            out[k++] = s->done.front();
            s->done.pop_front();
        }
        if (n_out)
            *n_out = k;
        return ok();
    } catch (...) {
        return fail(MTGP_ENOMEM, "host allocation failed");
    }
}

extern "C" mtgp_status mtgp_server_release(mtgp_server_t s, uint64_t arena_offset, uint64_t count)
{
    if (!s)
        return fail(MTGP_EINVAL, "null server");
    s->alloc.release(arena_offset, count);
    return ok();
}

extern "C" mtgp_status mtgp_server_arena(mtgp_server_t s, void** arena)
{
    if (!s || !arena)
        return fail(MTGP_EINVAL, "null argument");
    *arena = s->arena;
    return ok();
}

extern "C" mtgp_status mtgp_server_read(mtgp_server_t s, uint64_t arena_offset, uint64_t count,
                                        void* host_dst)
{
    if (!s || (count && !host_dst))
        return fail(MTGP_EINVAL, "null argument");
    if (arena_offset > s->cfg.arena_bytes / 4 || count > s->cfg.arena_bytes / 4 - arena_offset)
        return fail(MTGP_EINVAL, "range [%llu, +%llu) leaves the arena", (unsigned long long)arena_offset,
                    (unsigned long long)count);
    DeviceGuard g(s->st->device);
    const cudaError_t e = cudaMemcpy(host_dst, (uint32_t*)s->arena + arena_offset, count * 4,
                                     cudaMemcpyDeviceToHost);
    if (e != cudaSuccess)
        return fail_cuda(e, "cudaMemcpy(server read)");
    return ok();
}

// Short pause for the polling loop: yields, and sleeps when the next event
// is far away.
static void pause_until(double t_next)
{
    const double dt = t_next - now_s();
    if (dt > 200e-6)
        std::this_thread::sleep_for(std::chrono::microseconds(50));
    else
        std::this_thread::yield();
}

// One launch per request (the comparison): request i goes to CUDA stream
// lanes[ids[i] % L], so one stream's requests stay in order.
static mtgp_status run_per_request(mtgp_server* s, const double* t_arr, const uint32_t* ids,
                                   const uint64_t* counts, const int32_t* fmts, uint32_t n,
                                   double* latency, uint64_t* rec_offs, double t0)
{
    const int L = 16;
    std::vector<cudaStream_t> lanes(L, nullptr);
    const size_t NS = 256;
    std::vector<TableSlot> slots(NS);
    std::vector<cudaEvent_t> evs(NS, nullptr);
    std::vector<int64_t> slot_req(NS, -1);
    std::vector<double> slot_t(NS, 0.0);
    mtgp_status rc = MTGP_OK;
    cudaError_t e = cudaSuccess;
    for (int i = 0; i < L && e == cudaSuccess; ++i)
        e = cudaStreamCreateWithFlags(&lanes[i], cudaStreamNonBlocking);
    for (size_t i = 0; i < NS && e == cudaSuccess; ++i) {
        e = cudaEventCreateWithFlags(&slots[i].ev, cudaEventDisableTiming);
        if (e == cudaSuccess)
            e = cudaEventCreateWithFlags(&evs[i], cudaEventDisableTiming);
    }
    if (e != cudaSuccess)
        rc = fail_cuda(e, "per-request streams/events");
    std::vector<uint64_t> offs(n, 0);
    std::deque<uint32_t> waiting;   // arrived, not launched (arena full)
    uint32_t next = 0, finished = 0;
    size_t slot_next = 0;
    uint32_t in_flight = 0;
    while (rc == MTGP_OK && finished < n) {
        const double tnow = now_s() - t0;
        while (next < n && t_arr[next] <= tnow)
            waiting.push_back(next++);
        bool progressed = false;
        // completions
        for (size_t k = 0; k < NS && in_flight; ++k) {
            if (slot_req[k] < 0)
                continue;
            bool ready = false;
            if ((rc = query_done(s, evs[k], slot_t[k], &ready)) != MTGP_OK)
                break;
            if (!ready)
                continue;
            const uint32_t j = (uint32_t)slot_req[k];
            latency[j] = now_s() - t0 - t_arr[j];
            if (!rec_offs)
                s->alloc.release(offs[j], counts[j]);
            slot_req[k] = -1;
            --in_flight;
            ++finished;
            s->n_numbers += counts[j];
            ++s->n_requests;
            progressed = true;
        }
        // launches, in arrival order
        while (rc == MTGP_OK && !waiting.empty() && slot_req[slot_next] < 0) {
            const uint32_t j = waiting.front();
            uint64_t off;
            if (!s->alloc.alloc(counts[j], &off))
                break;
            offs[j] = off;
            if (rec_offs)
                rec_offs[j] = off;
            const double tl = now_s();
            Work w;
            rc = build_work(s->st->n_streams, &ids[j], &counts[j], &fmts[j], 0, 1, 0, w, &off);
            if (rc != MTGP_OK)
                break;
            cudaStream_t cs = lanes[ids[j] % L];
            rc = launch_work_slot(s->st, slots[slot_next], w, s->st->cfg, s->arena, cs);
            if (rc != MTGP_OK)
                break;
            if ((e = cudaEventRecord(evs[slot_next], cs)) != cudaSuccess) {
                rc = fail_cuda(e, "cudaEventRecord");
                break;
            }
            slot_req[slot_next] = j;
            slot_t[slot_next] = now_s();
            s->launch_host_s += slot_t[slot_next] - tl;
            slot_next = (slot_next + 1) % NS;
            ++in_flight;
            ++s->n_ticks;
            waiting.pop_front();
            progressed = true;
        }
        if (!progressed)
            pause_until(next < n ? t0 + t_arr[next] : now_s() + 1e-4);
    }
    for (int i = 0; i < L; ++i)
        if (lanes[i]) {
            cudaStreamSynchronize(lanes[i]);
            cudaStreamDestroy(lanes[i]);
        }
    for (size_t i = 0; i < NS; ++i) {
        free_table_slot(slots[i]);
        if (slots[i].ev)
            cudaEventDestroy(slots[i].ev);
        if (evs[i])
            cudaEventDestroy(evs[i]);
    }
    return rc;
}

extern "C" mtgp_status mtgp_server_run_trace(mtgp_server_t s, const double* t_arrival,
                                             const uint32_t* ids, const uint64_t* counts,
                                             const int32_t* fmts, uint32_t n, uint32_t mode,
                                             double* latency, uint64_t* record_offsets,
                                             mtgp_server_stats* stats)
{
    if (!s || (n && (!t_arrival || !ids || !counts || !fmts || !latency)))
        return fail(MTGP_EINVAL, "null argument");
    if (mode > 1)
        return fail(MTGP_EINVAL, "mode %u", mode);
    try {
        DeviceGuard g(s->st->device);
        for (uint32_t j = 0; j < n; ++j) {
            if (ids[j] >= s->st->n_streams || fmts[j] < 0 || fmts[j] > 2 || counts[j] == 0 ||
                ArenaAlloc::round(counts[j]) > s->alloc.total)
                return fail(MTGP_EINVAL, "trace entry %u invalid", j);
            if (j && t_arrival[j] < t_arrival[j - 1])
                return fail(MTGP_EINVAL, "arrival times must not decrease (entry %u)", j);
        }
        if (!s->pending.empty())
            return fail(MTGP_EBUSY, "server has pending requests");
        for (const Tick& t : s->ticks)
            if (t.busy)
                return fail(MTGP_EBUSY, "server has ticks in flight");
        const uint64_t ticks0 = s->n_ticks, nums0 = s->n_numbers, reqs0 = s->n_requests, jumps0 = s->n_jumps;
        const double launch0 = s->launch_host_s;
        double busy_wait = 0;
        const double t0 = now_s();
        mtgp_status rc = MTGP_OK;
        if (mode == 1) {
            rc = run_per_request(s, t_arrival, ids, counts, fmts, n, latency, record_offsets, t0);
        } else {
            s->keep_results = record_offsets != nullptr;
            uint32_t next = 0, finished = 0;
            std::vector<mtgp_completion> batch;
            while (finished < n) {
                const double tnow = now_s() - t0;
                while (next < n && t_arrival[next] <= tnow) {
                    rc = submit(s, ids[next], counts[next], fmts[next], next, t0 + t_arrival[next]);
                    if (rc != MTGP_OK)
                        break;
                    ++next;
                }
                if (rc != MTGP_OK)
                    break;
                int reaped = 0, launched = 0;
                if ((rc = reap(s, &reaped)) != MTGP_OK)
                    break;
                while (!s->done.empty()) {
                    const mtgp_completion c = s->done.front();
                    s->done.pop_front();
                    latency[c.tag] = c.done_time - c.submit_time;
                    if (record_offsets)
                        record_offsets[c.tag] = c.arena_offset;
                    else
                        s->alloc.release(c.arena_offset, c.count);
                    ++finished;
                }
                if ((rc = admit_and_launch(s, &launched)) != MTGP_OK)
                    break;
                if (!reaped && !launched) {
                    const double tw = now_s();
                    pause_until(next < n ? t0 + t_arrival[next] : tw + 1e-4);
                    if (!s->pending.empty())
                        busy_wait += now_s() - tw;
                }
            }
            s->keep_results = false;
        }
        const double t1 = now_s();
        if (stats) {
            stats->requests = s->n_requests - reqs0;
            stats->numbers = s->n_numbers - nums0;
            stats->ticks = s->n_ticks - ticks0;
            stats->elapsed = t1 - t0 - (n ? t_arrival[0] : 0);
            stats->busy_wait = busy_wait;
            stats->launch_host_s = s->launch_host_s - launch0;
            stats->jumps = s->n_jumps - jumps0;
        }
        if (rc != MTGP_OK)
            return rc;
        return ok();
    } catch (...) {
        return fail(MTGP_ENOMEM, "host allocation failed");
    }
}

extern "C" mtgp_status mtgp_server_debug_hold(mtgp_server_t s, int hold)
{
    if (!s)
        return fail(MTGP_EINVAL, "null server");
    s->hold = hold != 0;
    return ok();
}

extern "C" mtgp_status mtgp_server_free(mtgp_server_t s)
{
    destroy_server(s);
    return ok();
}

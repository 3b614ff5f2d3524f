// C ABI of libmtgp: parameter sets, device-resident stream states, batched
// generation (direct calls, recorded plans replayed from CUDA graphs, and a
// chunked device-to-host path), launch configuration and autotuning.
#include "mtgp_runtime.h"

#include <algorithm>
#include <cerrno>
#include <cstdarg>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <fstream>
#include <map>
#include <mutex>
#include <sstream>
#include <string>
#include <tuple>
#include <vector>

using namespace mtgp;

// ---------------------------------------------------------------------------
// Errors
// ---------------------------------------------------------------------------
static thread_local std::string g_last_error;

mtgp_status mtgp::fail(mtgp_status st, const char* fmt, ...)
{
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof buf, fmt, ap);
    va_end(ap);
    g_last_error = buf;
    return st;
}

mtgp_status mtgp::fail_cuda(cudaError_t e, const char* what)
{
    return fail(e == cudaErrorMemoryAllocation ? MTGP_ENOMEM : MTGP_ECUDA, "%s: %s (%s)", what,
                cudaGetErrorName(e), cudaGetErrorString(e));
}

mtgp_status mtgp::ok()
{
    g_last_error.clear();
    return MTGP_OK;
}

// Prefixes the last error message with the tuning candidate that produced it.
static mtgp_status fail_candidate(mtgp_status r, const LaunchCfg& c)
{
    const std::string why = g_last_error;
    return fail(r, "tuning candidate (warps/CTA %d, sub-steps %d, CTAs/SM %d, kernel %d, coop %d%%): %s",
                c.warps_per_cta, c.k, c.ctas_per_sm, c.kernel, c.coop_percent, why.c_str());
}

#define CUDA_TRY(call, what)                   \
    do {                                       \
        cudaError_t e_ = (call);               \
        if (e_ != cudaSuccess)                 \
            return fail_cuda(e_, what);        \
    } while (0)

// ---------------------------------------------------------------------------
// Parameter sets (Sec. 3.1: the parameterized status; "fast" statuses carry
// precomputed tables)
// ---------------------------------------------------------------------------
static bool table_is_linear(const uint32_t t[16])
{
    if (t[0] != 0)
        return false;
    for (int a = 0; a < 16; ++a)
        for (int b = 0; b < 16; ++b)
            if (t[a ^ b] != (t[a] ^ t[b]))
                return false;
    return true;
}

static void span(const uint32_t basis[4], uint32_t t[16])
{
    for (int k = 0; k < 16; ++k) {
        uint32_t v = 0;
        for (int b = 0; b < 4; ++b)
            if ((k >> b) & 1)
                v ^= basis[b];
        t[k] = v;
    }
}

static mtgp_status complete_desc(mtgp_params_desc& d)
{
    if (d.n == 0)
        d.n = d.mexp / 32u + 1u;
    if (d.mask == 0) {
        const long long r = 32LL * d.n - (long long)d.mexp;
        if (r < 1 || r > 31)
            return fail(MTGP_EINVAL, "mask: 32N - Mexp = %lld is not in 1..31 (give mask explicitly)", r);
        d.mask = 0xFFFFFFFFu << (uint32_t)r;
    }
    if (d.n < 2 || d.n > MTGP_MAX_N)
        return fail(MTGP_EINVAL, "N = %u out of range 2..%u", d.n, (unsigned)MTGP_MAX_N);
    if (d.pos < 1 || d.pos > d.n - 1)
        return fail(MTGP_EINVAL, "pos = %u out of range 1..N-1 (N = %u)", d.pos, d.n);
    if (d.sh1 > 31 || d.sh2 > 31)
        return fail(MTGP_EINVAL, "shift out of range 0..31 (sh1 = %u, sh2 = %u)", d.sh1, d.sh2);
    if (!table_is_linear(d.rec_tbl))
        return fail(MTGP_EINVAL, "recursion table is not GF(2)-linear");
    if (!table_is_linear(d.tmp_tbl))
        return fail(MTGP_EINVAL, "tempering table is not GF(2)-linear");
    return MTGP_OK;
}

static void to_kparams(const mtgp_params_desc& d, KParams& k)
{
    k.n = d.n;
    k.np = (d.n + 3u) & ~3u;
    k.pos = d.pos;
    k.sh1 = d.sh1;
    k.sh2 = d.sh2;
    k.mask = d.mask;
    k.mirror = 32u * ((d.pos + 31u + 31u) / 32u);
    for (int i = 0; i < 16; ++i) {
        k.rec[i] = d.rec_tbl[i];
        k.tmp[i] = d.tmp_tbl[i];
        k.flt[i] = (d.tmp_tbl[i] >> 9) | 0x3F800000u;
    }
}

static mtgp_status make_params(const mtgp_params_desc& in, mtgp_params_t* out)
{
    if (!out)
        return fail(MTGP_EINVAL, "null output handle");
    mtgp_params_desc d = in;
    mtgp_status st = complete_desc(d);
    if (st != MTGP_OK)
        return st;
    mtgp_params* p = new mtgp_params;
    p->d = d;
    to_kparams(d, p->k);
    *out = p;
    return ok();
}

extern "C" mtgp_status mtgp_params_create(const mtgp_params_desc* desc, mtgp_params_t* out)
{
    GUARD_BEGIN
    if (!desc)
        return fail(MTGP_EINVAL, "null desc");
    return make_params(*desc, out);
    GUARD_END
}

// SplitMix64 (Steele, Lea, Flood 2014): golden-ratio increment, then two
// xor-shift-multiply rounds and a final xor-shift.
static uint64_t sm64(uint64_t& s)
{
    uint64_t z = (s += 0x9E3779B97F4A7C15ull);
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
}

extern "C" mtgp_status mtgp_params_generate(uint32_t mexp, uint64_t seed, mtgp_params_t* out)
{
    GUARD_BEGIN
    if (mexp < 33 || mexp % 32u == 0)
        return fail(MTGP_EINVAL, "Mexp = %u unusable (needs >= 33 and not a multiple of 32)", mexp);
    mtgp_params_desc d;
    std::memset(&d, 0, sizeof d);
    d.mexp = mexp;
    d.n = mexp / 32u + 1u;
    uint64_t s = seed;
    d.sh1 = 1u + (uint32_t)(sm64(s) % 31u);
    d.sh2 = 1u + (uint32_t)(sm64(s) % 31u);
    const uint64_t dp = sm64(s);
    uint32_t wmin = 1;
    while (wmin * 2u <= d.n - 2u && wmin < 256u)
        wmin *= 2u;
    d.pos = 2u + (uint32_t)(dp % (uint64_t)(d.n - wmin - 1u));
    uint32_t rb[4], tb[4];
    for (int b = 0; b < 4; ++b)
        rb[b] = (uint32_t)(sm64(s) >> 32);
    for (int b = 0; b < 4; ++b)
        tb[b] = (uint32_t)(sm64(s) >> 32);
    span(rb, d.rec_tbl);
    span(tb, d.tmp_tbl);
    return make_params(d, out);
    GUARD_END
}

extern "C" mtgp_status mtgp_params_load(const char* path, mtgp_params_t* out)
{
    GUARD_BEGIN
    if (!path)
        return fail(MTGP_EINVAL, "null path");
    std::ifstream f(path);
    if (!f)
        return fail(MTGP_EIO, "cannot open %s", path);
    mtgp_params_desc d;
    std::memset(&d, 0, sizeof d);
    bool have_rec = false, have_tmp = false, have_mexp = false, have_pos = false, have_sh1 = false,
         have_sh2 = false;
    std::string line;
    int lineno = 0;
    while (std::getline(f, line)) {
        ++lineno;
        const size_t hash = line.find('#');
        if (hash != std::string::npos)
            line.resize(hash);
        std::istringstream ls(line);
        std::string key;
        if (!(ls >> key))
            continue;
        std::vector<uint64_t> vals;
        std::string tok;
        while (ls >> tok) {
            errno = 0;
            char* end = nullptr;
            const unsigned long long v = std::strtoull(tok.c_str(), &end, 0);
            if (errno || !end || *end || v > 0xFFFFFFFFull)
                return fail(MTGP_EIO, "%s:%d: bad number '%s'", path, lineno, tok.c_str());
            vals.push_back(v);
        }
        auto one = [&](uint32_t& dst, bool* flag) -> bool {
            if (vals.size() != 1)
                return false;
            dst = (uint32_t)vals[0];
            if (flag)
                *flag = true;
            return true;
        };
        bool good = true;
        if (key == "mexp")
            good = one(d.mexp, &have_mexp);
        else if (key == "n")
            good = one(d.n, nullptr);
        else if (key == "pos")
            good = one(d.pos, &have_pos);
        else if (key == "sh1")
            good = one(d.sh1, &have_sh1);
        else if (key == "sh2")
            good = one(d.sh2, &have_sh2);
        else if (key == "mask")
            good = one(d.mask, nullptr);
        else if (key == "rec_basis" || key == "tmp_basis") {
            if (vals.size() != 4)
                good = false;
            else {
                uint32_t b[4];
                for (int i = 0; i < 4; ++i)
                    b[i] = (uint32_t)vals[i];
                span(b, key == "rec_basis" ? d.rec_tbl : d.tmp_tbl);
                (key == "rec_basis" ? have_rec : have_tmp) = true;
            }
        } else if (key == "rec_tbl" || key == "tmp_tbl") {
            if (vals.size() != 16)
                good = false;
            else {
                uint32_t* t = key == "rec_tbl" ? d.rec_tbl : d.tmp_tbl;
                for (int i = 0; i < 16; ++i)
                    t[i] = (uint32_t)vals[i];
                (key == "rec_tbl" ? have_rec : have_tmp) = true;
            }
        } else {
            continue;   // unknown keys (e.g. state, outputs in test fixtures) are ignored
        }
        if (!good)
            return fail(MTGP_EIO, "%s:%d: wrong number of values for '%s'", path, lineno, key.c_str());
    }
    if (!(have_mexp && have_pos && have_sh1 && have_sh2 && have_rec && have_tmp))
        return fail(MTGP_EIO, "%s: missing field (need mexp, pos, sh1, sh2, rec_*, tmp_*)", path);
    return make_params(d, out);
    GUARD_END
}

extern "C" mtgp_status mtgp_params_get(mtgp_params_t params, mtgp_params_desc* desc)
{
    if (!params || !desc)
        return fail(MTGP_EINVAL, "null argument");
    *desc = params->d;
    return ok();
}

extern "C" mtgp_status mtgp_params_free(mtgp_params_t params)
{
    delete params;
    return ok();
}

// ---------------------------------------------------------------------------
// Work tables
// ---------------------------------------------------------------------------
mtgp_status mtgp::build_work(uint32_t n_streams, const uint32_t* ids, const uint64_t* counts,
                             const int32_t* fmts, uint32_t fmt_all, uint32_t n_req,
                             uint64_t out_base, Work& w, const uint64_t* out_offs)
{
    w.items.clear();
    w.item_total.clear();
    w.segs.clear();
    w.total = 0;
    w.max_item = 0;
    if (n_req == 0)
        return MTGP_OK;
    if (!ids || !counts)
        return fail(MTGP_EINVAL, "null request arrays");
    std::vector<uint32_t> order;
    order.reserve(n_req);
    uint64_t total = 0;
    for (uint32_t j = 0; j < n_req; ++j) {
        if (ids[j] >= n_streams)
            return fail(MTGP_EINVAL, "stream id %u >= n_streams %u (request %u)", ids[j], n_streams, j);
        if (fmts && (fmts[j] < 0 || fmts[j] > 2))
            return fail(MTGP_EINVAL, "format %d of request %u", fmts[j], j);
        if (counts[j] > (1ull << 50) || total + counts[j] < total)
            return fail(MTGP_EINVAL, "count too large (request %u)", j);
        total += counts[j];
        if (counts[j])
            order.push_back(j);
    }
    std::stable_sort(order.begin(), order.end(),
                     [&](uint32_t a, uint32_t b) { return ids[a] < ids[b]; });
    // exclusive scan of counts in request order gives the output offsets
    // (unless the caller places every request itself)
    std::vector<uint64_t> off(n_req);
    uint64_t acc = out_base;
    for (uint32_t j = 0; j < n_req; ++j) {
        off[j] = out_offs ? out_offs[j] : acc;
        acc += counts[j];
    }
    size_t i = 0;
    while (i < order.size()) {
        const uint32_t sid = ids[order[i]];
        WorkItem it;
        it.stream = sid;
        it.seg_begin = (uint32_t)w.segs.size();
        it.pad = 0;
        uint64_t g = 0;
        while (i < order.size() && ids[order[i]] == sid) {
            const uint32_t j = order[i];
            Segment s;
            s.g_start = g;
            s.count = counts[j];
            s.out_off = off[j];
            s.fmt = fmts ? (uint32_t)fmts[j] : fmt_all;
            s.req = j;
            w.segs.push_back(s);
            g += counts[j];
            ++i;
        }
        it.nseg = (uint32_t)w.segs.size() - it.seg_begin;
        w.items.push_back(it);
        w.max_item = std::max(w.max_item, g);
    }
    // Longest stream first: a warp that starts late only gets short streams.
    std::vector<uint64_t> tot(w.items.size());
    for (size_t k = 0; k < w.items.size(); ++k) {
        const Segment& l = w.segs[w.items[k].seg_begin + w.items[k].nseg - 1];
        tot[k] = l.g_start + l.count;
    }
    std::vector<uint32_t> idx(w.items.size());
    for (size_t k = 0; k < idx.size(); ++k)
        idx[k] = (uint32_t)k;
    std::stable_sort(idx.begin(), idx.end(), [&](uint32_t a, uint32_t b) { return tot[a] > tot[b]; });
    std::vector<WorkItem> sorted(w.items.size());
    w.item_total.resize(w.items.size());
    for (size_t k = 0; k < idx.size(); ++k) {
        sorted[k] = w.items[idx[k]];
        w.item_total[k] = tot[idx[k]];
    }
    w.items.swap(sorted);
    w.total = total;
    return MTGP_OK;
}

size_t mtgp::table_bytes(const Work& w, size_t* items_off, size_t* segs_off)
{
    const size_t a = 256;
    const size_t io = a;
    const size_t so = io + ((w.items.size() * sizeof(WorkItem) + a - 1) / a) * a;
    if (items_off)
        *items_off = io;
    if (segs_off)
        *segs_off = so;
    return so + w.segs.size() * sizeof(Segment);
}

void mtgp::fill_table(const Work& w, void* host)
{
    size_t io, so;
    table_bytes(w, &io, &so);
    std::memset(host, 0, io);   // work counter (first word) = 0
    if (!w.items.empty())
        std::memcpy((char*)host + io, w.items.data(), w.items.size() * sizeof(WorkItem));
    if (!w.segs.empty())
        std::memcpy((char*)host + so, w.segs.data(), w.segs.size() * sizeof(Segment));
}

mtgp_status mtgp::split_work(const Work& w, uint64_t max_piece, uint32_t max_pieces,
                             const std::vector<uint32_t>& set_of_stream, SplitWork* out)
{
    SplitWork& o = *out;
    o = SplitWork();
    o.max_piece = max_piece;
    if (max_piece == 0) {
        o.work = w;
        return MTGP_OK;
    }
    struct Piece {
        WorkItem it;   // stream = the item's row
        uint64_t total;
        std::vector<Segment> segs;
    };
    std::vector<Piece> pieces;
    auto new_row = [&](uint32_t stream) -> uint32_t {
        const uint32_t row = o.n_rows++;
        o.copies.push_back(make_uint2(stream, row));
        o.row_set.push_back(set_of_stream.empty() ? 0u : set_of_stream[stream]);
        return row;
    };
    for (size_t i = 0; i < w.items.size(); ++i) {
        const WorkItem& it = w.items[i];
        const uint64_t T = w.item_total[i];
        const Segment* sg = w.segs.data() + it.seg_begin;
        if (o.n_rows >= 0x7FFFFFF0u)
            return fail(MTGP_EINVAL, "too many pieces");
        if (T <= max_piece) {
            Piece p{it, T, std::vector<Segment>(sg, sg + it.nseg)};
            p.it.stream = new_row(it.stream);
            o.backs.push_back(make_uint2(p.it.stream, it.stream));
            pieces.push_back(std::move(p));
            continue;
        }
        uint64_t L = max_piece;
        uint64_t k = (T + L - 1) / L;
        if (k > max_pieces) {
            L = (T + max_pieces - 1) / max_pieces;
            k = (T + L - 1) / L;
        }
        ++o.n_split;
        o.n_pieces += (uint32_t)k;
        for (uint64_t j = 0; j < k; ++j) {
            const uint64_t lo = j * L, hi = std::min(T, lo + L);
            Piece p;
            p.it = it;
            p.it.stream = new_row(it.stream);
            p.total = hi - lo;
            if (j > 0) {
                o.jump_rows.push_back(p.it.stream);
                o.jump_sets.push_back(o.row_set.back());
                o.jump_lens.push_back(lo);
            }
            if (j + 1 == k)
                o.backs.push_back(make_uint2(p.it.stream, it.stream));
            for (uint32_t q = 0; q < it.nseg; ++q) {
                const uint64_t a = std::max(sg[q].g_start, lo);
                const uint64_t b = std::min(sg[q].g_start + sg[q].count, hi);
                if (a >= b)
                    continue;
                Segment t = sg[q];
                t.g_start = a - lo;
                t.count = b - a;
                t.out_off = sg[q].out_off + (a - sg[q].g_start);
                p.segs.push_back(t);
            }
            pieces.push_back(std::move(p));
        }
    }
    std::vector<size_t> order(pieces.size());
    for (size_t i = 0; i < order.size(); ++i)
        order[i] = i;
    std::stable_sort(order.begin(), order.end(),
                     [&](size_t a, size_t b) { return pieces[a].total > pieces[b].total; });
    Work& ow = o.work;
    for (size_t i : order) {
        Piece& p = pieces[i];
        p.it.seg_begin = (uint32_t)ow.segs.size();
        p.it.nseg = (uint32_t)p.segs.size();
        ow.segs.insert(ow.segs.end(), p.segs.begin(), p.segs.end());
        ow.items.push_back(p.it);
        ow.item_total.push_back(p.total);
        ow.total += p.total;
        ow.max_item = std::max(ow.max_item, p.total);
    }
    return MTGP_OK;
}

// ---------------------------------------------------------------------------
// Streams
// ---------------------------------------------------------------------------
DeviceGuard::DeviceGuard(int dev)
{
    prev = -1;
    if (cudaGetDevice(&prev) == cudaSuccess && prev != dev)
        cudaSetDevice(dev);
    else
        prev = -1;
}
DeviceGuard::~DeviceGuard()
{
    if (prev >= 0)
        cudaSetDevice(prev);
}

void mtgp::free_table_slot(TableSlot& s)
{
    if (s.ev_recorded)
        cudaEventSynchronize(s.ev);
    if (s.host)
        cudaFreeHost(s.host);
    if (s.dev)
        cudaFree(s.dev);
    s.host = nullptr;
    s.dev = nullptr;
    s.cap = 0;
    s.ev_recorded = false;
}

static void destroy_streams(mtgp_streams* h)
{
    if (!h)
        return;
    DeviceGuard g(h->device);
    for (auto& s : h->slots) {
        free_table_slot(s);
        if (s.ev)
            cudaEventDestroy(s.ev);
    }
    for (int b = 0; b < mtgp_streams::kStages; ++b) {
        if (h->stage[b])
            cudaFree(h->stage[b]);
        if (h->ev_gen[b])
            cudaEventDestroy(h->ev_gen[b]);
        if (h->ev_copy[b])
            cudaEventDestroy(h->ev_copy[b]);
    }
    if (h->copy_stream)
        cudaStreamDestroy(h->copy_stream);
    if (h->d_chunk_tables)
        cudaFree(h->d_chunk_tables);
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

extern "C" mtgp_status mtgp_init_statuses(mtgp_params_t params, const uint32_t* seeds,
                                          uint32_t n_streams, void* cuda_stream, mtgp_streams_t* out)
{
    GUARD_BEGIN
    if (!params || !out || (n_streams && !seeds))
        return fail(MTGP_EINVAL, "null argument");
    if (n_streams == 0)
        return fail(MTGP_EINVAL, "n_streams must be >= 1");
    mtgp_streams* h = new mtgp_streams;
    h->P = *params;
    h->n_streams = n_streams;
    cudaError_t e = cudaGetDevice(&h->device);
    if (e != cudaSuccess) {
        delete h;
        return fail_cuda(e, "cudaGetDevice");
    }
    cudaStream_t s = (cudaStream_t)cuda_stream;
    auto bail = [&](cudaError_t err, const char* what) {
        mtgp_status st = fail_cuda(err, what);
        destroy_streams(h);
        return st;
    };
    const size_t bytes = (size_t)n_streams * h->P.k.np * sizeof(uint32_t);
    if ((e = cudaMalloc(&h->d_states, bytes)) != cudaSuccess)
        return bail(e, "cudaMalloc(states)");
    if ((e = cudaMalloc(&h->d_err, sizeof(int))) != cudaSuccess)
        return bail(e, "cudaMalloc(error word)");
    if ((e = cudaMemsetAsync(h->d_err, 0, sizeof(int), s)) != cudaSuccess)
        return bail(e, "cudaMemsetAsync");
    for (auto& sl : h->slots)
        if ((e = cudaEventCreateWithFlags(&sl.ev, cudaEventDisableTiming)) != cudaSuccess)
            return bail(e, "cudaEventCreate");
    for (int b = 0; b < mtgp_streams::kStages; ++b) {
        if ((e = cudaEventCreateWithFlags(&h->ev_gen[b], cudaEventDisableTiming)) != cudaSuccess ||
            (e = cudaEventCreateWithFlags(&h->ev_copy[b], cudaEventDisableTiming)) != cudaSuccess)
            return bail(e, "cudaEventCreate");
    }
    if ((e = cudaStreamCreateWithFlags(&h->copy_stream, cudaStreamNonBlocking)) != cudaSuccess)
        return bail(e, "cudaStreamCreate");
    // seeds -> device through a temporary buffer, then the init kernel
    uint32_t* d_seeds = nullptr;
    if ((e = cudaMallocAsync((void**)&d_seeds, (size_t)n_streams * 4, s)) != cudaSuccess)
        return bail(e, "cudaMallocAsync(seeds)");
    if ((e = cudaMemcpyAsync(d_seeds, seeds, (size_t)n_streams * 4, cudaMemcpyHostToDevice, s)) !=
        cudaSuccess) {
        cudaFreeAsync(d_seeds, s);
        return bail(e, "cudaMemcpyAsync(seeds)");
    }
    e = launch_init(h->P.k, d_seeds, n_streams, h->d_states, s);
    cudaFreeAsync(d_seeds, s);
    if (e != cudaSuccess)
        return bail(e, "init kernel launch");
    // pageable seeds: the copy above is complete when cudaMemcpyAsync returns
    h->cfg = default_config(h->P.k);
    *out = h;
    return ok();
    GUARD_END
}

extern "C" mtgp_status mtgp_init_statuses_multi(const mtgp_params_t* sets, uint32_t n_sets,
                                                const uint32_t* set_of_stream, const uint32_t* seeds,
                                                uint32_t n_streams, void* cuda_stream,
                                                mtgp_streams_t* out)
{
    GUARD_BEGIN
    if (!sets || !set_of_stream || !seeds || !out)
        return fail(MTGP_EINVAL, "null argument");
    if (n_sets == 0 || n_streams == 0)
        return fail(MTGP_EINVAL, "n_sets and n_streams must be >= 1");
    for (uint32_t i = 0; i < n_sets; ++i) {
        if (!sets[i])
            return fail(MTGP_EINVAL, "parameter set %u is null", i);
        if (sets[i]->d.mexp != sets[0]->d.mexp || sets[i]->d.n != sets[0]->d.n ||
            sets[i]->d.mask != sets[0]->d.mask)
            return fail(MTGP_EINVAL, "parameter set %u: Mexp/N/mask differ from set 0 (all sets of a "
                        "handle share the state size)", i);
    }
    for (uint32_t s = 0; s < n_streams; ++s)
        if (set_of_stream[s] >= n_sets)
            return fail(MTGP_EINVAL, "stream %u: parameter set %u out of range (n_sets = %u)", s,
                        set_of_stream[s], n_sets);
    // Representative set for everything decided per launch (step width,
    // shared-memory mirror): the largest pos and mirror of all sets.
    mtgp_params rep = *sets[0];
    std::vector<KSet> ks(n_sets);
    for (uint32_t i = 0; i < n_sets; ++i) {
        const KParams& k = sets[i]->k;
        rep.k.pos = std::max(rep.k.pos, k.pos);
        rep.k.mirror = std::max(rep.k.mirror, k.mirror);
        ks[i].pos = k.pos;
        ks[i].sh1 = k.sh1;
        ks[i].sh2 = k.sh2;
        ks[i].mirror = k.mirror;
        for (int j = 0; j < 16; ++j) {
            ks[i].rec[j] = k.rec[j];
            ks[i].tmp[j] = k.tmp[j];
            ks[i].flt[j] = k.flt[j];
        }
    }
    rep.d.pos = rep.k.pos;
    mtgp_streams_t h = nullptr;
    mtgp_status st = mtgp_init_statuses(&rep, seeds, n_streams, cuda_stream, &h);
    if (st != MTGP_OK)
        return st;
    DeviceGuard g(h->device);
    cudaStream_t cs = (cudaStream_t)cuda_stream;
    cudaError_t e = cudaMalloc(&h->d_sets, ks.size() * sizeof(KSet));
    if (e == cudaSuccess)
        e = cudaMalloc(&h->d_set_of, (size_t)n_streams * sizeof(uint32_t));
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(h->d_sets, ks.data(), ks.size() * sizeof(KSet), cudaMemcpyHostToDevice, cs);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(h->d_set_of, set_of_stream, (size_t)n_streams * sizeof(uint32_t),
                            cudaMemcpyHostToDevice, cs);
    if (e == cudaSuccess)
        e = cudaStreamSynchronize(cs);   // ks is a local vector
    if (e != cudaSuccess) {
        destroy_streams(h);
        return fail_cuda(e, "per-stream parameter sets");
    }
    h->n_sets = n_sets;
    *out = h;
    return ok();
    GUARD_END
}

LaunchCfg mtgp::default_config(const KParams& P)
{
    // 8 warps per SM; 128-word software-pipelined steps when the parameter
    // set allows them (N - pos >= 256), else 256-word steps, else 128, else
    // 64 (short states such as Mexp 3217).
    LaunchCfg c;
    c.warps_per_cta = 4;
    c.ctas_per_sm = 2;
    c.k = 4;
    c.kernel = 0;
    c.coop_percent = 0;
    if (P.n - P.pos < 256u || !fast_supported(P, 4))
        c.k = fast_supported(P, 8) ? 8 : (fast_supported(P, 4) || !fast_supported(P, 2) ? 4 : 2);
    return c;
}

uint32_t mtgp::coop_count(const Work& w, const Geometry& g, int coop_percent)
{
    if (g.kernel != 0 || coop_percent <= 0 || w.items.empty() || g.k < g.threads / 32)
        return 0;   // (the CTA-wide phase needs k >= warps per CTA)
    const double slots = (double)g.grid * (double)(g.threads / 32);
    const double thr = (double)w.total / slots * (double)coop_percent / 100.0;
    uint32_t n = 0;
    while (n < w.item_total.size() && (double)w.item_total[n] >= thr)
        ++n;
    return n;
}

extern "C" mtgp_status mtgp_streams_info(mtgp_streams_t st, uint32_t* n_streams, uint32_t* n_words)
{
    if (!st)
        return fail(MTGP_EINVAL, "null handle");
    if (n_streams)
        *n_streams = st->n_streams;
    if (n_words)
        *n_words = st->P.k.n;
    return ok();
}

extern "C" mtgp_status mtgp_set_statuses(mtgp_streams_t st, const uint32_t* states, void* cuda_stream)
{
    GUARD_BEGIN
    if (!st || !states)
        return fail(MTGP_EINVAL, "null argument");
    DeviceGuard g(st->device);
    cudaStream_t s = (cudaStream_t)cuda_stream;
    const size_t n = st->P.k.n, np = st->P.k.np;
    CUDA_TRY(cudaMemcpy2DAsync(st->d_states, np * 4, states, n * 4, n * 4, st->n_streams,
                               cudaMemcpyHostToDevice, s),
             "cudaMemcpy2DAsync(set statuses)");
    CUDA_TRY(cudaStreamSynchronize(s), "cudaStreamSynchronize");
    return ok();
    GUARD_END
}

extern "C" mtgp_status mtgp_get_statuses(mtgp_streams_t st, uint32_t* states, void* cuda_stream)
{
    GUARD_BEGIN
    if (!st || !states)
        return fail(MTGP_EINVAL, "null argument");
    DeviceGuard g(st->device);
    cudaStream_t s = (cudaStream_t)cuda_stream;
    const size_t n = st->P.k.n, np = st->P.k.np;
    CUDA_TRY(cudaMemcpy2DAsync(states, n * 4, st->d_states, np * 4, n * 4, st->n_streams,
                               cudaMemcpyDeviceToHost, s),
             "cudaMemcpy2DAsync(get statuses)");
    CUDA_TRY(cudaStreamSynchronize(s), "cudaStreamSynchronize");
    return ok();
    GUARD_END
}

// Resolves the geometry for the handle's configuration (cached).
mtgp_status mtgp::geometry_for(mtgp_streams* st, const LaunchCfg& cfg, uint32_t n_items, Geometry* g)
{
    const auto key = std::make_tuple(cfg.warps_per_cta, cfg.ctas_per_sm, cfg.k, cfg.kernel);
    if (!(st->geo_valid && st->geo_key == key)) {
        Geometry full;
        cudaError_t e = plan_geometry(st->P.k, cfg, 0x7FFFFFFF, st->device, &full);
        if (e != cudaSuccess)
            return fail_cuda(e, "launch geometry");
        st->geo_cap = full;
        st->geo_key = key;
        st->geo_valid = true;
    }
    *g = st->geo_cap;
    // One CTA per item at most (a CTA may take a whole stream); CTAs that find
    // no work left exit at once.
    const long long want = (long long)n_items;
    g->grid = (int)std::max(1LL, std::min<long long>(want, st->geo_cap.grid));
    return MTGP_OK;
}

// Uploads a work table through the handle's slot ring and launches.
mtgp_status mtgp::launch_work(mtgp_streams* st, const Work& w, const LaunchCfg& cfg, void* out,
                              cudaStream_t s)
{
    if (w.items.empty())
        return MTGP_OK;
    TableSlot& sl = st->slots[st->next_slot];
    st->next_slot = (st->next_slot + 1) % (int)st->slots.size();
    return launch_work_slot(st, sl, w, cfg, out, s);
}

// Uploads a work table through `sl` (waiting for the slot's previous
// consumer) and launches on `s`; records the slot's event after the kernel.
mtgp_status mtgp::launch_work_slot(mtgp_streams* st, TableSlot& sl, const Work& w,
                                   const LaunchCfg& cfg, void* out, cudaStream_t s, const RowArray* rows)
{
    if (w.items.empty())
        return MTGP_OK;
    if (sl.ev_recorded) {
        CUDA_TRY(cudaEventSynchronize(sl.ev), "cudaEventSynchronize(table slot)");
        sl.ev_recorded = false;
    }
    size_t io, so;
    const size_t bytes = table_bytes(w, &io, &so);
    if (bytes > sl.cap) {
        if (sl.host)
            cudaFreeHost(sl.host);
        if (sl.dev)
            cudaFree(sl.dev);
        sl.host = nullptr;
        sl.dev = nullptr;
        sl.cap = 0;
        const size_t cap = std::max<size_t>(bytes * 2, 1 << 16);
        CUDA_TRY(cudaMallocHost(&sl.host, cap), "cudaMallocHost(work table)");
        CUDA_TRY(cudaMalloc(&sl.dev, cap), "cudaMalloc(work table)");
        sl.cap = cap;
    }
    fill_table(w, sl.host);
    CUDA_TRY(cudaMemcpyAsync(sl.dev, sl.host, bytes, cudaMemcpyHostToDevice, s),
             "cudaMemcpyAsync(work table)");
    mtgp_status stt = launch_work_table(st, w, sl.dev, cfg, out, s, rows);
    if (stt != MTGP_OK)
        return stt;
    CUDA_TRY(cudaEventRecord(sl.ev, s), "cudaEventRecord");
    sl.ev_recorded = true;
    return MTGP_OK;
}

mtgp_status mtgp::launch_work_table(mtgp_streams* st, const Work& w, void* table, const LaunchCfg& cfg,
                                    void* out, cudaStream_t s, const RowArray* rows)
{
    if (w.items.empty())
        return MTGP_OK;
    size_t io, so;
    table_bytes(w, &io, &so);
    Geometry g;
    mtgp_status stt = geometry_for(st, cfg, (uint32_t)w.items.size(), &g);
    if (stt != MTGP_OK)
        return stt;
    GenArgs a;
    a.P = st->P.k;
    a.states = st->d_states;
    a.n_streams = st->n_streams;
    a.items = (const WorkItem*)((char*)table + io);
    a.segs = (const Segment*)((char*)table + so);
    a.n_items = (uint32_t)w.items.size();
    a.n_coop = st->d_sets ? 0u : coop_count(w, g, cfg.coop_percent);
    a.counter = (uint32_t*)table;
    a.out = (uint32_t*)out;
    a.err = st->d_err;
    a.trace = nullptr;
    a.sets = st->d_sets;
    a.set_of = st->d_set_of;
    if (rows) {
        a.states = rows->states;
        a.n_streams = rows->n_rows;
        a.set_of = rows->set_of;
    }
    CUDA_TRY(launch_generate(a, g, s), "generation kernel launch");
    return MTGP_OK;
}

static mtgp_status generate_common(mtgp_streams_t st, const uint32_t* ids, const uint64_t* counts,
                                   uint32_t n_req, uint32_t fmt, void* out, void* cuda_stream)
{
    GUARD_BEGIN
    if (!st)
        return fail(MTGP_EINVAL, "null handle");
    if (fmt > 2)
        return fail(MTGP_EINVAL, "format %u", fmt);
    Work w;
    mtgp_status s = build_work(st->n_streams, ids, counts, nullptr, fmt, n_req, 0, w);
    if (s != MTGP_OK)
        return s;
    if (w.total && !out)
        return fail(MTGP_EINVAL, "null output pointer");
    DeviceGuard g(st->device);
    s = launch_work(st, w, st->cfg, out, (cudaStream_t)cuda_stream);
    if (s != MTGP_OK)
        return s;
    return ok();
    GUARD_END
}

extern "C" mtgp_status mtgp_generate_u32(mtgp_streams_t st, const uint32_t* ids, const uint64_t* counts,
                                         uint32_t n_req, uint32_t* out, void* cuda_stream)
{
    return generate_common(st, ids, counts, n_req, MTGP_U32, out, cuda_stream);
}

extern "C" mtgp_status mtgp_generate_f32(mtgp_streams_t st, const uint32_t* ids, const uint64_t* counts,
                                         uint32_t n_req, mtgp_format fmt, float* out, void* cuda_stream)
{
    return generate_common(st, ids, counts, n_req, (uint32_t)fmt, out, cuda_stream);
}

extern "C" mtgp_status mtgp_generate_to_host(mtgp_streams_t st, const uint32_t* ids,
                                             const uint64_t* counts, uint32_t n_req, mtgp_format fmt,
                                             void* host_out, uint64_t chunk_bytes, void* cuda_stream)
{
    GUARD_BEGIN
    if (!st)
        return fail(MTGP_EINVAL, "null handle");
    if ((uint32_t)fmt > 2)
        return fail(MTGP_EINVAL, "format %d", (int)fmt);
    if (chunk_bytes == 0)
        chunk_bytes = 1ull << 30;
    const uint64_t chunk = std::max<uint64_t>(chunk_bytes / 4, 1024);
    // validate once over the whole request list
    {
        Work w;
        mtgp_status s = build_work(st->n_streams, ids, counts, nullptr, fmt, n_req, 0, w);
        if (s != MTGP_OK)
            return s;
        if (w.total && !host_out)
            return fail(MTGP_EINVAL, "null output pointer");
        if (w.total == 0)
            return ok();
    }
    DeviceGuard g(st->device);
    cudaStream_t cs = (cudaStream_t)cuda_stream;
    if (st->stage_cap < chunk) {
        for (int b = 0; b < mtgp_streams::kStages; ++b) {
            if (st->stage[b]) {
                CUDA_TRY(cudaStreamSynchronize(st->copy_stream), "cudaStreamSynchronize");
                cudaFree(st->stage[b]);
                st->stage[b] = nullptr;
            }
        }
        st->stage_cap = 0;
        for (int b = 0; b < mtgp_streams::kStages; ++b)
            CUDA_TRY(cudaMalloc(&st->stage[b], chunk * 4), "cudaMalloc(staging)");
        st->stage_cap = chunk;
    }
    // Split the request list into chunks of at most `chunk` numbers; a long
    // request becomes consecutive requests of the same stream, which draw
    // the same numbers.  Every chunk's work table is built first and all of
    // them are uploaded in one copy, so that no host-to-device transfer sits
    // between a chunk's generation and the previous chunk's copy to the host.
    std::vector<Work> works;
    std::vector<uint64_t> fills;
    {
        std::vector<uint32_t> cid;
        std::vector<uint64_t> ccount;
        uint64_t fill = 0;
        auto close = [&]() -> mtgp_status {
            if (fill == 0)
                return MTGP_OK;
            works.emplace_back();
            mtgp_status s = build_work(st->n_streams, cid.data(), ccount.data(), nullptr, fmt,
                                       (uint32_t)cid.size(), 0, works.back());
            if (s != MTGP_OK)
                return s;
            fills.push_back(fill);
            fill = 0;
            cid.clear();
            ccount.clear();
            return MTGP_OK;
        };
        for (uint32_t j = 0; j < n_req; ++j) {
            uint64_t left = counts[j];
            while (left) {
                const uint64_t take = std::min(left, chunk - fill);
                cid.push_back(ids[j]);
                ccount.push_back(take);
                fill += take;
                left -= take;
                if (fill == chunk) {
                    mtgp_status s = close();
                    if (s != MTGP_OK)
                        return s;
                }
            }
        }
        mtgp_status s = close();
        if (s != MTGP_OK)
            return s;
    }
    std::vector<size_t> toff(works.size());
    size_t tbytes = 0;
    for (size_t c = 0; c < works.size(); ++c) {
        toff[c] = tbytes;
        tbytes += (table_bytes(works[c], nullptr, nullptr) + 255u) & ~(size_t)255u;
    }
    std::vector<char> tables(tbytes);
    for (size_t c = 0; c < works.size(); ++c)
        fill_table(works[c], tables.data() + toff[c]);
    if (tbytes > st->chunk_tables_cap) {
        if (st->d_chunk_tables)
            cudaFree(st->d_chunk_tables);
        st->d_chunk_tables = nullptr;
        st->chunk_tables_cap = 0;
        CUDA_TRY(cudaMalloc(&st->d_chunk_tables, tbytes), "cudaMalloc(chunk work tables)");
        st->chunk_tables_cap = tbytes;
    }
    // the previous call's kernels are done (it ended with both streams
    // synchronized), so the tables can be overwritten
    CUDA_TRY(cudaMemcpyAsync(st->d_chunk_tables, tables.data(), tbytes, cudaMemcpyHostToDevice, cs),
             "cudaMemcpyAsync(chunk work tables)");
    uint64_t host_off = 0;
    bool recorded[mtgp_streams::kStages] = {};
    for (size_t c = 0; c < works.size(); ++c) {
        const int b = (int)(c % mtgp_streams::kStages);
        if (recorded[b])
            CUDA_TRY(cudaStreamWaitEvent(cs, st->ev_copy[b], 0), "cudaStreamWaitEvent");
        mtgp_status s = launch_work_table(st, works[c], (char*)st->d_chunk_tables + toff[c], st->cfg,
                                          st->stage[b], cs);
        if (s != MTGP_OK)
            return s;
        CUDA_TRY(cudaEventRecord(st->ev_gen[b], cs), "cudaEventRecord");
        CUDA_TRY(cudaStreamWaitEvent(st->copy_stream, st->ev_gen[b], 0), "cudaStreamWaitEvent");
        CUDA_TRY(cudaMemcpyAsync((char*)host_out + host_off * 4, st->stage[b], fills[c] * 4,
                                 cudaMemcpyDeviceToHost, st->copy_stream),
                 "cudaMemcpyAsync(D2H)");
        CUDA_TRY(cudaEventRecord(st->ev_copy[b], st->copy_stream), "cudaEventRecord");
        recorded[b] = true;
        host_off += fills[c];
    }
    CUDA_TRY(cudaStreamSynchronize(st->copy_stream), "cudaStreamSynchronize(copy)");
    CUDA_TRY(cudaStreamSynchronize(cs), "cudaStreamSynchronize");
    return ok();
    GUARD_END
}

extern "C" mtgp_status mtgp_check(mtgp_streams_t st, void* cuda_stream)
{
    GUARD_BEGIN
    if (!st)
        return fail(MTGP_EINVAL, "null handle");
    DeviceGuard g(st->device);
    cudaStream_t s = (cudaStream_t)cuda_stream;
    CUDA_TRY(cudaStreamSynchronize(s), "cudaStreamSynchronize");
    int v = 0;
    CUDA_TRY(cudaMemcpy(&v, st->d_err, sizeof v, cudaMemcpyDeviceToHost), "cudaMemcpy(error word)");
    if (v) {
        CUDA_TRY(cudaMemset(st->d_err, 0, sizeof(int)), "cudaMemset");
        return fail(MTGP_EDEVICE, "a kernel recorded an inconsistent work item (code %d)", v);
    }
    return ok();
    GUARD_END
}

extern "C" mtgp_status mtgp_streams_free(mtgp_streams_t st)
{
    GUARD_BEGIN
    destroy_streams(st);
    return ok();
    GUARD_END
}

// ---------------------------------------------------------------------------
// Launch configuration and autotuning
// ---------------------------------------------------------------------------
static mtgp_launch_config to_public(const LaunchCfg& c)
{
    mtgp_launch_config o;
    o.warps_per_cta = (uint32_t)c.warps_per_cta;
    o.ctas_per_sm = (uint32_t)c.ctas_per_sm;
    o.words_per_lane = (uint32_t)c.k;
    o.kernel = (uint32_t)c.kernel;
    o.coop_percent = (uint32_t)c.coop_percent;
    return o;
}

extern "C" mtgp_status mtgp_get_launch_config(mtgp_streams_t st, mtgp_launch_config* cfg)
{
    if (!st || !cfg)
        return fail(MTGP_EINVAL, "null argument");
    *cfg = to_public(st->cfg);
    return ok();
}

mtgp_status mtgp::validate_config(const mtgp_launch_config* c, LaunchCfg* out)
{
    if (!c)
        return fail(MTGP_EINVAL, "null config");
    if (c->warps_per_cta < 1 || c->warps_per_cta > 8)
        return fail(MTGP_EINVAL, "warps_per_cta %u not in 1..8", c->warps_per_cta);
    if (c->words_per_lane != 2 && c->words_per_lane != 4 && c->words_per_lane != 8)
        return fail(MTGP_EINVAL, "words_per_lane %u not 2, 4 or 8", c->words_per_lane);
    if (c->kernel > 1)
        return fail(MTGP_EINVAL, "kernel %u not 0 or 1", c->kernel);
    if (c->ctas_per_sm > 64)
        return fail(MTGP_EINVAL, "ctas_per_sm %u", c->ctas_per_sm);
    if (c->coop_percent > 100000)
        return fail(MTGP_EINVAL, "coop_percent %u", c->coop_percent);
    out->warps_per_cta = (int)c->warps_per_cta;
    out->ctas_per_sm = (int)c->ctas_per_sm;
    out->k = (int)c->words_per_lane;
    out->kernel = (int)c->kernel;
    out->coop_percent = (int)c->coop_percent;
    return MTGP_OK;
}

extern "C" mtgp_status mtgp_set_launch_config(mtgp_streams_t st, const mtgp_launch_config* cfg)
{
    if (!st)
        return fail(MTGP_EINVAL, "null handle");
    LaunchCfg c;
    mtgp_status s = validate_config(cfg, &c);
    if (s != MTGP_OK)
        return s;
    st->cfg = c;
    return ok();
}

std::vector<LaunchCfg> mtgp::tuning_candidates(const KParams& P)
{
    // Residency matters as much as block shape: a launch whose longest
    // streams dominate runs best with few warps per SM (each stream gets a
    // larger share of the SM), an even launch with many (short states, whose
    // 64-word steps leave much latency to hide, gain up to 32 warps per SM).
    // Candidates cover 4 .. 32 warps per SM and the occupancy maximum, with
    // and without the whole-CTA mode for long streams.
    std::vector<LaunchCfg> v;
    auto add = [&](int w, int k, int cap, int coop) {
        if (!fast_supported(P, k, w))
            return;
        LaunchCfg x;
        x.warps_per_cta = w;
        x.ctas_per_sm = cap;
        x.k = k;
        x.kernel = 0;
        x.coop_percent = coop;
        v.push_back(x);
    };
    for (int k : {8, 4, 2}) {
        for (int cap : {1, 2, 3, 4, 0})
            add(4, k, cap, 0);
        for (int cap : {2, 3, 4, 6, 0})
            add(2, k, cap, 0);
        add(8, k, 1, 0);
        add(8, k, 2, 0);
        add(8, k, 3, 0);
        add(8, k, 4, 0);
        add(8, k, 0, 0);
        if (k >= 4)
            add(4, k, 0, 100);
        if (k >= 8)
            add(8, k, 1, 100);
    }
    if (v.empty()) {   // no register-resident instantiation: tune the ring kernel
        for (int w : {2, 4, 8}) {
            LaunchCfg x;
            x.warps_per_cta = w;
            x.ctas_per_sm = 0;
            x.k = 8;
            x.kernel = 1;
            x.coop_percent = 0;
            v.push_back(x);
        }
    }
    return v;
}

// Times one configuration on scratch states: best of `reps` launches.
mtgp_status mtgp::time_config(mtgp_streams* st, const Work& w, const LaunchCfg& cfg, uint32_t* states,
                              void* out, int reps, float* best_ms)
{
    cudaStream_t s = st->tune_stream;
    cudaEvent_t a = st->tune_ev[0], b = st->tune_ev[1];
    uint32_t* saved = st->d_states;
    st->d_states = states;
    float best = 1e30f;
    mtgp_status r = MTGP_OK;
    for (int i = 0; i < reps + 1 && r == MTGP_OK; ++i) {
        cudaEventRecord(a, s);
        r = launch_work(st, w, cfg, out, s);
        cudaEventRecord(b, s);
        if (r != MTGP_OK)
            break;
        cudaError_t e = cudaEventSynchronize(b);
        if (e != cudaSuccess) {
            r = fail_cuda(e, "autotune run");
            break;
        }
        float ms = 0;
        cudaEventElapsedTime(&ms, a, b);
        if (i > 0)
            best = std::min(best, ms);
    }
    st->d_states = saved;
    *best_ms = best;
    return r;
}

static std::mutex g_tune_mu;
static std::map<std::tuple<int, uint32_t, uint32_t, uint32_t>, LaunchCfg> g_tune_cache;

extern "C" mtgp_status mtgp_autotune(mtgp_streams_t st, mtgp_format fmt, uint32_t sample_streams,
                                     uint64_t sample_count, mtgp_launch_config* best)
{
    GUARD_BEGIN
    if (!st)
        return fail(MTGP_EINVAL, "null handle");
    if ((uint32_t)fmt > 2)
        return fail(MTGP_EINVAL, "format");
    DeviceGuard g(st->device);
    const auto key = std::make_tuple(st->device, st->P.k.n, st->P.k.pos, (uint32_t)fmt);
    {
        std::lock_guard<std::mutex> lk(g_tune_mu);
        auto it = g_tune_cache.find(key);
        if (it != g_tune_cache.end()) {
            st->cfg = it->second;
            if (best)
                *best = to_public(st->cfg);
            return ok();
        }
    }
    if (sample_streams == 0)
        sample_streams = 4096;
    if (sample_count == 0)
        sample_count = 1u << 14;
    const uint32_t ns = std::min(sample_streams, st->n_streams);
    const size_t np = st->P.k.np;
    uint32_t* scratch = nullptr;
    void* out = nullptr;
    CUDA_TRY(cudaDeviceSynchronize(), "cudaDeviceSynchronize");
    CUDA_TRY(cudaMalloc(&scratch, (size_t)ns * np * 4), "cudaMalloc(tune states)");
    cudaError_t e = cudaMalloc(&out, (size_t)ns * sample_count * 4);
    if (e != cudaSuccess) {
        cudaFree(scratch);
        return fail_cuda(e, "cudaMalloc(tune output)");
    }
    mtgp_status r = MTGP_OK;
    LaunchCfg win = st->cfg;
    if ((e = cudaMemcpy(scratch, st->d_states, (size_t)ns * np * 4, cudaMemcpyDeviceToDevice)) !=
        cudaSuccess)
        r = fail_cuda(e, "cudaMemcpy(tune states)");
    if (r == MTGP_OK && !st->tune_stream) {
        if ((e = cudaStreamCreateWithFlags(&st->tune_stream, cudaStreamNonBlocking)) != cudaSuccess ||
            (e = cudaEventCreate(&st->tune_ev[0])) != cudaSuccess ||
            (e = cudaEventCreate(&st->tune_ev[1])) != cudaSuccess)
            r = fail_cuda(e, "tune stream/events");
    }
    if (r == MTGP_OK) {
        std::vector<uint32_t> ids(ns);
        std::vector<uint64_t> cnt(ns, sample_count);
        for (uint32_t i = 0; i < ns; ++i)
            ids[i] = i;
        Work w;
        // scratch holds the first ns states, so ids stay below ns
        const uint32_t saved_n = st->n_streams;
        st->n_streams = ns;
        r = build_work(ns, ids.data(), cnt.data(), nullptr, (uint32_t)fmt, ns, 0, w);
        float best_ms = 1e30f;
        if (r == MTGP_OK) {
            for (const LaunchCfg& c : tuning_candidates(st->P.k)) {
                Geometry probe;
                if (geometry_for(st, c, 1, &probe) != MTGP_OK)
                    continue;   // not launchable on this device (registers or shared memory)
                float ms = 0;
                r = time_config(st, w, c, scratch, out, 2, &ms);
                if (r != MTGP_OK) {
                    r = fail_candidate(r, c);
                    break;
                }
                if (ms < best_ms) {
                    best_ms = ms;
                    win = c;
                }
            }
        }
        st->n_streams = saved_n;
    }
    cudaStreamSynchronize(st->tune_stream);
    cudaFree(scratch);
    cudaFree(out);
    if (r != MTGP_OK)
        return r;
    st->cfg = win;
    {
        std::lock_guard<std::mutex> lk(g_tune_mu);
        g_tune_cache[key] = win;
    }
    if (best)
        *best = to_public(win);
    return ok();
    GUARD_END
}

// ---------------------------------------------------------------------------
// Plans (one persistent launch recorded as a CUDA graph)
// ---------------------------------------------------------------------------
static mtgp_status record_graph(mtgp_plan* p)
{
    if (p->exec) {
        cudaGraphExecDestroy(p->exec);
        p->exec = nullptr;
    }
    if (p->graph) {
        cudaGraphDestroy(p->graph);
        p->graph = nullptr;
    }
    p->kernel_launches = 0;
    if (p->n_items == 0)
        return MTGP_OK;
    cudaStream_t cap = p->cap_stream;
    const uint32_t n_copies = (uint32_t)p->split.copies.size();
    const uint32_t n_jumps = (uint32_t)p->jumps.items.size();
    const bool split = p->split.n_rows > 0;
    CUDA_TRY(cudaStreamBeginCapture(cap, cudaStreamCaptureModeThreadLocal), "cudaStreamBeginCapture");
    // split launches: every row gets its stream's state, then the rows of
    // later pieces are jumped to their offsets
    cudaError_t e1 = launch_copy_rows(p->st->d_states, p->d_rows, p->d_copies, n_copies,
                                      p->st->P.k.n, p->st->P.k.np, cap);
    if (e1 == cudaSuccess)
        e1 = launch_jump_batch(p->st, p->d_rows, p->d_jitems, n_jumps, p->d_jpolys, p->jumps.words,
                               p->jumps.smem, cap);
    if (e1 == cudaSuccess)
        e1 = cudaMemsetAsync(p->d_table, 0, 2 * sizeof(uint32_t), cap);
    GenArgs a;
    a.P = p->st->P.k;
    a.states = split ? p->d_rows : p->st->d_states;
    a.n_streams = split ? p->split.n_rows : p->st->n_streams;
    a.items = (const WorkItem*)((char*)p->d_table + p->items_off);
    a.segs = (const Segment*)((char*)p->d_table + p->segs_off);
    a.n_items = p->n_items;
    a.n_coop = p->st->d_sets ? 0u : coop_count(p->split.work, p->geo, p->cfg.coop_percent);
    p->n_coop = a.n_coop;
    a.counter = (uint32_t*)p->d_table;
    a.out = (uint32_t*)p->out;
    a.err = p->st->d_err;
    a.trace = p->d_trace;
    a.sets = p->st->d_sets;
    a.set_of = split ? p->d_row_set : p->st->d_set_of;
    cudaError_t e2 = e1;
    if (e2 == cudaSuccess && p->stats) {
        // the fused kernel writes every request's counts; requests with no
        // numbers keep the zeros of these memsets
        a.n_coop = p->n_coop = 0;
        e2 = p->sa.hist ? cudaMemsetAsync(p->sa.hist, 0, (size_t)p->n_req * (p->sa.t + 1u) * 8u, cap)
                        : cudaSuccess;
        if (e2 == cudaSuccess && p->sa.tab)
            e2 = cudaMemsetAsync(p->sa.tab, 0, (size_t)p->n_req * p->sa.C * p->sa.C * 8u, cap);
        if (e2 == cudaSuccess)
            e2 = launch_fused(p->stats_fn, a, p->sa, dim3(p->stats_geo.grid), dim3(p->stats_geo.threads),
                              p->stats_geo.smem, cap);
        if (e2 == cudaSuccess && split)
            e2 = launch_stats_stitch(a.segs, p->d_piece_start, p->d_pieces, p->n_req, p->sa, cap);
    } else if (e2 == cudaSuccess) {
        e2 = launch_generate(a, p->geo, cap);
    }
    // the streams' new states: unsplit streams' rows and split streams' last pieces
    const uint32_t n_backs = (uint32_t)p->split.backs.size();
    if (e2 == cudaSuccess)
        e2 = launch_copy_rows(p->d_rows, p->st->d_states, p->d_backs, n_backs, p->st->P.k.n,
                              p->st->P.k.np, cap);
    cudaGraph_t graph = nullptr;
    cudaError_t e3 = cudaStreamEndCapture(cap, &graph);
    if (e2 != cudaSuccess) {
        if (graph)
            cudaGraphDestroy(graph);
        return fail_cuda(e2, "plan capture");
    }
    if (e3 != cudaSuccess)
        return fail_cuda(e3, "cudaStreamEndCapture");
    p->graph = graph;
    CUDA_TRY(cudaGraphInstantiate(&p->exec, graph, 0), "cudaGraphInstantiate");
    p->kernel_launches = 1 + (n_copies ? 1u : 0u) + (n_jumps ? 1u : 0u) + (n_backs ? 1u : 0u) +
                         (p->stats && split && p->n_req ? 1u : 0u);
    return MTGP_OK;
}

// Frees the device side of a plan's split (scratch rows, copy pairs, jump
// items and polynomials).
static void free_split(mtgp_plan* p)
{
    if (p->d_rows)
        cudaFree(p->d_rows);
    if (p->d_copies)
        cudaFree(p->d_copies);
    if (p->d_backs)
        cudaFree(p->d_backs);
    if (p->d_row_set)
        cudaFree(p->d_row_set);
    if (p->d_jitems)
        cudaFree(p->d_jitems);
    if (p->d_jpolys)
        cudaFree(p->d_jpolys);
    p->d_rows = nullptr;
    p->d_copies = nullptr;
    p->d_backs = nullptr;
    p->d_row_set = nullptr;
    p->d_jitems = nullptr;
    p->d_jpolys = nullptr;
    p->jumps = JumpBatch();
}

// (Re)builds what a plan launches from its requests and max_piece: the work
// table (pieces when split), and for split plans the scratch rows, copy
// pairs and jumps.  Device memory of the previous build is released.
static mtgp_status build_launch(mtgp_plan* p, uint64_t max_piece)
{
    mtgp_streams* st = p->st;
    std::vector<uint32_t> set_of_stream;
    if (st->d_sets && max_piece) {
        set_of_stream.resize(st->n_streams);
        CUDA_TRY(cudaMemcpy(set_of_stream.data(), st->d_set_of, st->n_streams * 4, cudaMemcpyDeviceToHost),
                 "cudaMemcpy(set index)");
    }
    SplitWork sw;
    mtgp_status r = split_work(p->work, max_piece, 64, set_of_stream, &sw);
    if (r != MTGP_OK)
        return r;
    JumpBatch jb;
    r = build_jump_batch(st, sw.jump_rows, sw.jump_sets, sw.jump_lens, &jb);
    if (r != MTGP_OK)
        return r;
    CUDA_TRY(cudaDeviceSynchronize(), "cudaDeviceSynchronize");
    free_split(p);
    if (p->d_table) {
        cudaFree(p->d_table);
        p->d_table = nullptr;
    }
    const size_t bytes = table_bytes(sw.work, &p->items_off, &p->segs_off);
    std::vector<char> host(bytes);
    fill_table(sw.work, host.data());
    CUDA_TRY(cudaMalloc(&p->d_table, bytes), "cudaMalloc(plan table)");
    CUDA_TRY(cudaMemcpy(p->d_table, host.data(), bytes, cudaMemcpyHostToDevice), "cudaMemcpy(plan table)");
    if (sw.n_rows) {
        const size_t rows = (size_t)sw.n_rows * st->P.k.np * 4;
        CUDA_TRY(cudaMalloc(&p->d_rows, rows), "cudaMalloc(launch state rows)");
        if (st->d_sets) {
            CUDA_TRY(cudaMalloc(&p->d_row_set, sw.row_set.size() * 4), "cudaMalloc(row sets)");
            CUDA_TRY(cudaMemcpy(p->d_row_set, sw.row_set.data(), sw.row_set.size() * 4,
                                cudaMemcpyHostToDevice), "cudaMemcpy(row sets)");
        }
        CUDA_TRY(cudaMalloc(&p->d_copies, sw.copies.size() * sizeof(uint2)), "cudaMalloc(copy pairs)");
        CUDA_TRY(cudaMemcpy(p->d_copies, sw.copies.data(), sw.copies.size() * sizeof(uint2),
                            cudaMemcpyHostToDevice), "cudaMemcpy(copy pairs)");
        CUDA_TRY(cudaMalloc(&p->d_backs, sw.backs.size() * sizeof(uint2)), "cudaMalloc(copy-back pairs)");
        CUDA_TRY(cudaMemcpy(p->d_backs, sw.backs.data(), sw.backs.size() * sizeof(uint2),
                            cudaMemcpyHostToDevice), "cudaMemcpy(copy-back pairs)");
    }
    if (!jb.items.empty()) {
        CUDA_TRY(cudaMalloc(&p->d_jitems, jb.items.size() * sizeof(JumpItem)), "cudaMalloc(jump items)");
        CUDA_TRY(cudaMemcpy(p->d_jitems, jb.items.data(), jb.items.size() * sizeof(JumpItem),
                            cudaMemcpyHostToDevice), "cudaMemcpy(jump items)");
        CUDA_TRY(cudaMalloc(&p->d_jpolys, jb.poly_words.size() * 4), "cudaMalloc(jump polynomials)");
        CUDA_TRY(cudaMemcpy(p->d_jpolys, jb.poly_words.data(), jb.poly_words.size() * 4,
                            cudaMemcpyHostToDevice), "cudaMemcpy(jump polynomials)");
    }
    p->split = std::move(sw);
    p->jumps = std::move(jb);
    p->n_items = (uint32_t)p->split.work.items.size();
    p->max_item = p->split.work.max_item;
    if (p->d_trace) {   // one record per launched item
        cudaFree(p->d_trace);
        p->d_trace = nullptr;
        CUDA_TRY(cudaMalloc(&p->d_trace, (size_t)p->n_items * 4 * sizeof(uint64_t)), "cudaMalloc(trace)");
        CUDA_TRY(cudaMemset(p->d_trace, 0, (size_t)p->n_items * 4 * sizeof(uint64_t)), "cudaMemset");
    }
    return geometry_for(st, p->cfg, p->n_items, &p->geo);
}

static void free_split_stats(mtgp_plan* p)
{
    if (p->d_req_base)
        cudaFree(p->d_req_base);
    if (p->d_seg_stats)
        cudaFree(p->d_seg_stats);
    if (p->d_piece_start)
        cudaFree(p->d_piece_start);
    if (p->d_pieces)
        cudaFree(p->d_pieces);
    p->d_req_base = nullptr;
    p->d_seg_stats = nullptr;
    p->d_piece_start = nullptr;
    p->d_pieces = nullptr;
    p->sa.req_base = nullptr;
    p->sa.seg_stats = nullptr;
}

// The tables a split plan's statistics need (none for an unsplit plan):
// each request's first output index, one edge record per launched segment,
// and each request's segments ordered by their position in the request.
static mtgp_status build_split_stats(mtgp_plan* p)
{
    free_split_stats(p);
    if (!p->stats || !p->split.max_piece || p->n_req == 0)
        return MTGP_OK;
    std::vector<unsigned long long> base(p->n_req, 0ull);
    for (const Segment& sg : p->work.segs)   // unsplit: one segment per request, at its start
        base[sg.req] = sg.out_off;
    const std::vector<Segment>& segs = p->split.work.segs;
    std::vector<uint32_t> start(p->n_req + 1u, 0u), order(segs.size());
    for (const Segment& sg : segs)
        ++start[sg.req + 1u];
    for (uint32_t j = 0; j < p->n_req; ++j)
        start[j + 1u] += start[j];
    std::vector<uint32_t> fillp(start.begin(), start.end() - 1);
    for (uint32_t k = 0; k < (uint32_t)segs.size(); ++k)
        order[fillp[segs[k].req]++] = k;
    for (uint32_t j = 0; j < p->n_req; ++j)
        std::sort(order.begin() + start[j], order.begin() + start[j + 1u],
                  [&](uint32_t a, uint32_t b) { return segs[a].out_off < segs[b].out_off; });
    CUDA_TRY(cudaMalloc(&p->d_req_base, base.size() * 8u), "cudaMalloc(request offsets)");
    CUDA_TRY(cudaMemcpy(p->d_req_base, base.data(), base.size() * 8u, cudaMemcpyHostToDevice),
             "cudaMemcpy(request offsets)");
    CUDA_TRY(cudaMalloc(&p->d_seg_stats, std::max<size_t>(segs.size(), 1) * sizeof(SegStat)),
             "cudaMalloc(piece records)");
    CUDA_TRY(cudaMalloc(&p->d_piece_start, start.size() * 4u), "cudaMalloc(piece lists)");
    CUDA_TRY(cudaMemcpy(p->d_piece_start, start.data(), start.size() * 4u, cudaMemcpyHostToDevice),
             "cudaMemcpy(piece lists)");
    CUDA_TRY(cudaMalloc(&p->d_pieces, std::max<size_t>(order.size(), 1) * 4u), "cudaMalloc(pieces)");
    if (!order.empty())
        CUDA_TRY(cudaMemcpy(p->d_pieces, order.data(), order.size() * 4u, cudaMemcpyHostToDevice),
                 "cudaMemcpy(pieces)");
    p->sa.req_base = p->d_req_base;
    p->sa.seg_stats = p->d_seg_stats;
    return MTGP_OK;
}

// Kernel and launch geometry of a plan's fused statistics: G = 8 warps per
// CTA, as many resident CTAs per SM as the plan's configuration asks warps
// per SM (warps_per_cta x ctas_per_sm / 8, at least 1; occupancy maximum when
// ctas_per_sm is 0), persistent grid.  The kernel takes single-warp items
// with 128-word pipelined steps, so every parameter set needs N - pos >= 256,
// or N - pos >= 32 for short states (ceil(N/32) < 9); the handle's
// representative set has the largest pos of its sets.
static mtgp_status stats_geometry(mtgp_plan* p)
{
    mtgp_streams* st = p->st;
    const KParams& P = st->P.k;
    const int G = 8;
    const int M = (int)((P.n + 31u) / 32u);
    const void* fn = fused_kernel_ptr(M, G);
    if (!fn)
        return fail(MTGP_EINVAL, "statistics: no fused kernel for N = %u (ceil(N/32) = %d)", P.n, M);
    // 128-word pipelined rows need N - pos >= 256; short states (M < 9) run
    // every row one 32-column sub-step at a time, which needs N - pos >= 32
    if (M >= 9 ? P.n - P.pos < 256u : P.n - P.pos < 32u)
        return fail(MTGP_EINVAL, "statistics: N - pos = %u below %u", P.n - P.pos, M >= 9 ? 256u : 32u);
    Geometry g{};
    g.kernel = 0;
    g.k = 4;
    g.threads = G * 32;
    g.smem = (size_t)G * (fast_smem_words(P.n, P.mirror) + stats_smem_words(p->sa.t, p->sa.C)) * 4u;
    CUDA_TRY(allow_max_dynamic_smem(fn, st->device, g.smem), "statistics kernel shared memory");
    int per_sm = 0;
    CUDA_TRY(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, fn, g.threads, g.smem),
             "statistics kernel occupancy");
    if (per_sm < 1)
        return fail(MTGP_EINVAL, "statistics kernel does not fit on an SM");
    if (p->cfg.ctas_per_sm > 0)
        per_sm = std::min(per_sm, std::max(1, p->cfg.warps_per_cta * p->cfg.ctas_per_sm / G));
    cudaFuncAttributes fa;
    CUDA_TRY(cudaFuncGetAttributes(&fa, fn), "cudaFuncGetAttributes");
    int sms = 0;
    CUDA_TRY(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, st->device), "SM count");
    g.regs = fa.numRegs;
    g.per_sm = per_sm;
    const long long want = ((long long)p->n_items + G - 1) / G;
    g.grid = (int)std::max(1LL, std::min(want, (long long)sms * per_sm));
    p->stats_fn = fn;
    p->stats_geo = g;
    return MTGP_OK;
}

static void destroy_plan(mtgp_plan* p)
{
    if (!p)
        return;
    DeviceGuard g(p->st->device);
    if (p->exec)
        cudaGraphExecDestroy(p->exec);
    if (p->graph)
        cudaGraphDestroy(p->graph);
    if (p->cap_stream)
        cudaStreamDestroy(p->cap_stream);
    if (p->d_table)
        cudaFree(p->d_table);
    if (p->d_trace)
        cudaFree(p->d_trace);
    if (p->d_hist)
        cudaFree(p->d_hist);
    if (p->d_tab)
        cudaFree(p->d_tab);
    free_split_stats(p);
    free_split(p);
    delete p;
}

extern "C" mtgp_status mtgp_plan_create(mtgp_streams_t st, const uint32_t* ids, const uint64_t* counts,
                                        uint32_t n_req, mtgp_format fmt, void* out, mtgp_plan_t* plan)
{
    GUARD_BEGIN
    if (!st || !plan)
        return fail(MTGP_EINVAL, "null argument");
    if ((uint32_t)fmt > 2)
        return fail(MTGP_EINVAL, "format");
    Work w;
    mtgp_status s = build_work(st->n_streams, ids, counts, nullptr, (uint32_t)fmt, n_req, 0, w);
    if (s != MTGP_OK)
        return s;
    if (w.total && !out)
        return fail(MTGP_EINVAL, "null output pointer");
    DeviceGuard g(st->device);
    mtgp_plan* p = new mtgp_plan;
    p->st = st;
    p->out = out;
    p->n_items = (uint32_t)w.items.size();
    p->total = w.total;
    p->max_item = w.max_item;
    p->cfg = st->cfg;
    p->work = w;
    p->n_req = n_req;
    auto bail = [&](mtgp_status r) {
        destroy_plan(p);
        return r;
    };
    cudaError_t e;
    if ((e = cudaStreamCreateWithFlags(&p->cap_stream, cudaStreamNonBlocking)) != cudaSuccess)
        return bail(fail_cuda(e, "cudaStreamCreate"));
    s = build_launch(p, 0);
    if (s != MTGP_OK)
        return bail(s);
    s = record_graph(p);
    if (s != MTGP_OK)
        return bail(s);
    *plan = p;
    return ok();
    GUARD_END
}

extern "C" mtgp_status mtgp_plan_launch(mtgp_plan_t p, void* cuda_stream)
{
    if (!p)
        return fail(MTGP_EINVAL, "null plan");
    if (!p->exec)
        return ok();
    DeviceGuard g(p->st->device);
    CUDA_TRY(cudaGraphLaunch(p->exec, (cudaStream_t)cuda_stream), "cudaGraphLaunch");
    return ok();
}

extern "C" mtgp_status mtgp_plan_autotune(mtgp_plan_t p, mtgp_launch_config* best)
{
    GUARD_BEGIN
    if (!p)
        return fail(MTGP_EINVAL, "null plan");
    mtgp_streams* st = p->st;
    DeviceGuard g(st->device);
    if (p->n_items == 0) {
        if (best)
            *best = to_public(p->cfg);
        return ok();
    }
    const size_t bytes = (size_t)st->n_streams * st->P.k.np * 4;
    uint32_t* scratch = nullptr;
    CUDA_TRY(cudaDeviceSynchronize(), "cudaDeviceSynchronize");
    CUDA_TRY(cudaMalloc(&scratch, bytes), "cudaMalloc(tune states)");
    cudaError_t e = cudaMemcpy(scratch, st->d_states, bytes, cudaMemcpyDeviceToDevice);
    mtgp_status r = e == cudaSuccess ? MTGP_OK : fail_cuda(e, "cudaMemcpy(tune states)");
    if (r == MTGP_OK && !st->tune_stream) {
        if ((e = cudaStreamCreateWithFlags(&st->tune_stream, cudaStreamNonBlocking)) != cudaSuccess ||
            (e = cudaEventCreate(&st->tune_ev[0])) != cudaSuccess ||
            (e = cudaEventCreate(&st->tune_ev[1])) != cudaSuccess)
            r = fail_cuda(e, "tune stream/events");
    }
    LaunchCfg win = p->cfg;
    float best_ms = 1e30f;
    if (r == MTGP_OK) {
        for (const LaunchCfg& c : tuning_candidates(st->P.k)) {
            Geometry probe;
            if (geometry_for(st, c, 1, &probe) != MTGP_OK)
                continue;   // not launchable on this device (registers or shared memory)
            float ms = 0;
            if (p->split.n_rows) {
                // a split launch runs on the plan's own rows: time it there
                const uint32_t ns = st->n_streams;
                uint32_t* const so = st->d_set_of;
                st->n_streams = p->split.n_rows;
                st->d_set_of = st->d_sets ? p->d_row_set : so;
                r = time_config(st, p->split.work, c, p->d_rows, p->out, 2, &ms);
                st->n_streams = ns;
                st->d_set_of = so;
            } else {
                r = time_config(st, p->split.work, c, scratch, p->out, 2, &ms);
            }
            if (r != MTGP_OK) {
                r = fail_candidate(r, c);
                break;
            }
            if (ms < best_ms) {
                best_ms = ms;
                win = c;
            }
        }
    }
    cudaStreamSynchronize(st->tune_stream);
    cudaFree(scratch);
    if (r != MTGP_OK)
        return r;
    p->cfg = win;
    r = geometry_for(st, p->cfg, p->n_items, &p->geo);
    if (r != MTGP_OK)
        return r;
    if (p->stats && (r = stats_geometry(p)) != MTGP_OK)
        return r;
    r = record_graph(p);
    if (r != MTGP_OK)
        return r;
    if (best)
        *best = to_public(win);
    return ok();
    GUARD_END
}

extern "C" mtgp_status mtgp_plan_set_trace(mtgp_plan_t p, int enable)
{
    GUARD_BEGIN
    if (!p)
        return fail(MTGP_EINVAL, "null plan");
    if (enable && p->stats)
        return fail(MTGP_EINVAL, "the plan computes statistics: its kernel keeps no timeline");
    DeviceGuard g(p->st->device);
    CUDA_TRY(cudaDeviceSynchronize(), "cudaDeviceSynchronize");
    if (enable && !p->d_trace && p->n_items) {
        CUDA_TRY(cudaMalloc(&p->d_trace, (size_t)p->n_items * 4 * sizeof(uint64_t)),
                 "cudaMalloc(trace)");
        CUDA_TRY(cudaMemset(p->d_trace, 0, (size_t)p->n_items * 4 * sizeof(uint64_t)), "cudaMemset");
    } else if (!enable && p->d_trace) {
        cudaFree(p->d_trace);
        p->d_trace = nullptr;
    }
    mtgp_status r = record_graph(p);
    if (r != MTGP_OK)
        return r;
    return ok();
    GUARD_END
}

extern "C" mtgp_status mtgp_plan_read_trace(mtgp_plan_t p, uint64_t* host)
{
    GUARD_BEGIN
    if (!p || !host)
        return fail(MTGP_EINVAL, "null argument");
    if (!p->d_trace)
        return fail(MTGP_EINVAL, "tracing is not enabled on this plan");
    DeviceGuard g(p->st->device);
    CUDA_TRY(cudaMemcpy(host, p->d_trace, (size_t)p->n_items * 4 * sizeof(uint64_t),
                        cudaMemcpyDeviceToHost),
             "cudaMemcpy(trace)");
    return ok();
    GUARD_END
}

extern "C" mtgp_status mtgp_plan_set_split(mtgp_plan_t p, uint64_t max_piece)
{
    GUARD_BEGIN
    if (!p)
        return fail(MTGP_EINVAL, "null plan");
    if (max_piece != 0 && max_piece < 64)
        return fail(MTGP_EINVAL, "max_piece %llu below 64", (unsigned long long)max_piece);
    DeviceGuard g(p->st->device);
    mtgp_status r = build_launch(p, max_piece);
    if (r != MTGP_OK)
        return r;
    if (p->stats && ((r = stats_geometry(p)) != MTGP_OK || (r = build_split_stats(p)) != MTGP_OK))
        return r;
    r = record_graph(p);
    if (r != MTGP_OK)
        return r;
    return ok();
    GUARD_END
}

extern "C" mtgp_status mtgp_plan_set_stats(mtgp_plan_t p, const mtgp_stats_config* c)
{
    GUARD_BEGIN
    if (!p)
        return fail(MTGP_EINVAL, "null plan");
    const bool gap = c && c->gap_t != 0;
    const bool ham = c && c->ham_L != 0;
    // A test that is left out still runs, on masks that make it idle and
    // with nothing written: the gap test then visits only on zero outputs,
    // the Hamming test weighs nothing.
    StatsArgs a{};
    a.gmask = 0xFFFFFFFFu;
    a.t = 0;
    a.K = 240;
    a.C = 1;
    if (gap) {
        if (c->gap_b < 1 || c->gap_r + c->gap_b > 32 || c->gap_t > 1023)
            return fail(MTGP_EINVAL, "gap test: need b >= 1, r + b <= 32, 1 <= t <= 1023 (r %u b %u t %u)",
                        c->gap_r, c->gap_b, c->gap_t);
        a.gmask = (uint32_t)((((uint64_t)1 << c->gap_b) - 1u) << (32u - c->gap_r - c->gap_b));
        a.t = c->gap_t;
    }
    if (ham) {
        if (c->ham_s < 1 || c->ham_r + c->ham_s > 32 || c->ham_L % c->ham_s != 0 ||
            c->ham_L / c->ham_s < 32 || c->n_bounds > 15)
            return fail(MTGP_EINVAL, "Hamming test: need s >= 1, r + s <= 32, L a multiple of s with "
                        "L/s >= 32, at most 15 bounds (r %u s %u L %u bounds %u)",
                        c->ham_r, c->ham_s, c->ham_L, c->n_bounds);
        a.hmask = (uint32_t)((((uint64_t)1 << c->ham_s) - 1u) << (32u - c->ham_r - c->ham_s));
        a.K = c->ham_L / c->ham_s;
        a.C = c->n_bounds + 1u;
        for (uint32_t i = 0; i < c->n_bounds; ++i)
            a.bounds[i] = c->bounds[i];
    }
    if ((gap || ham) && p->d_trace)
        return fail(MTGP_EINVAL, "statistics: turn the plan's trace off first");
    if (gap || ham)
        for (const Segment& sg : p->work.segs)
            if (sg.count >> 31)
                return fail(MTGP_EINVAL, "statistics: request %u has 2^31 or more numbers", sg.req);
    DeviceGuard g(p->st->device);
    CUDA_TRY(cudaDeviceSynchronize(), "cudaDeviceSynchronize");
    const bool was = p->stats;
    const StatsArgs old = p->sa;
    p->stats = false;
    if (gap || ham) {
        p->sa = a;
        p->stats = true;
        mtgp_status r = stats_geometry(p);
        if (r != MTGP_OK) {
            p->stats = was;
            p->sa = old;
            return r;
        }
    }
    if (p->d_hist)
        cudaFree(p->d_hist);
    if (p->d_tab)
        cudaFree(p->d_tab);
    p->d_hist = nullptr;
    p->d_tab = nullptr;
    if (p->stats) {
        const size_t nr = std::max<uint32_t>(p->n_req, 1u);
        // zeroed here too: a plan with no work never launches, and its
        // counts read back before a launch are zeros
        if (gap) {
            CUDA_TRY(cudaMalloc(&p->d_hist, nr * (a.t + 1u) * 8u), "cudaMalloc(gap histograms)");
            CUDA_TRY(cudaMemset(p->d_hist, 0, nr * (a.t + 1u) * 8u), "cudaMemset(gap histograms)");
        }
        if (ham) {
            CUDA_TRY(cudaMalloc(&p->d_tab, nr * a.C * a.C * 8u), "cudaMalloc(Hamming tables)");
            CUDA_TRY(cudaMemset(p->d_tab, 0, nr * a.C * a.C * 8u), "cudaMemset(Hamming tables)");
        }
        p->sa.hist = p->d_hist;
        p->sa.tab = p->d_tab;
    } else {
        p->sa = StatsArgs{};
    }
    mtgp_status r = build_split_stats(p);
    if (r != MTGP_OK)
        return r;
    r = record_graph(p);
    if (r != MTGP_OK)
        return r;
    return ok();
    GUARD_END
}

extern "C" mtgp_status mtgp_plan_read_stats(mtgp_plan_t p, uint64_t* hist, uint64_t* table, void* cuda_stream)
{
    GUARD_BEGIN
    if (!p)
        return fail(MTGP_EINVAL, "null plan");
    if (!p->stats)
        return fail(MTGP_EINVAL, "the plan computes no statistics");
    if ((p->d_hist && !hist && p->n_req) || (p->d_tab && !table && p->n_req))
        return fail(MTGP_EINVAL, "null output array for a test the plan computes");
    DeviceGuard g(p->st->device);
    cudaStream_t cs = (cudaStream_t)cuda_stream;
    if (p->d_hist && p->n_req)
        CUDA_TRY(cudaMemcpyAsync(hist, p->d_hist, (size_t)p->n_req * (p->sa.t + 1u) * 8u,
                                 cudaMemcpyDeviceToHost, cs), "cudaMemcpyAsync(gap histograms)");
    if (p->d_tab && p->n_req)
        CUDA_TRY(cudaMemcpyAsync(table, p->d_tab, (size_t)p->n_req * p->sa.C * p->sa.C * 8u,
                                 cudaMemcpyDeviceToHost, cs), "cudaMemcpyAsync(Hamming tables)");
    CUDA_TRY(cudaStreamSynchronize(cs), "cudaStreamSynchronize");
    return ok();
    GUARD_END
}

extern "C" mtgp_status mtgp_plan_get_info(mtgp_plan_t p, mtgp_plan_info* info)
{
    if (!p || !info)
        return fail(MTGP_EINVAL, "null argument");
    info->total_numbers = p->total;
    info->n_items = p->n_items;
    info->max_piece = p->split.max_piece;
    info->n_split_streams = p->split.n_split;
    info->n_pieces = p->split.n_pieces;
    info->n_jumps = (uint32_t)p->jumps.items.size();
    info->kernel_launches = p->kernel_launches;
    const Geometry& geo = p->stats ? p->stats_geo : p->geo;
    LaunchCfg eff = p->cfg;
    eff.kernel = geo.kernel;
    eff.k = geo.k;
    eff.warps_per_cta = geo.threads / 32;
    info->config = to_public(eff);
    info->grid_ctas = (uint32_t)geo.grid;
    info->n_coop = p->n_coop;
    info->regs_per_thread = (uint32_t)geo.regs;
    info->resident_ctas_per_sm = (uint32_t)geo.per_sm;
    info->stats = p->stats ? 1u : 0u;
    return ok();
}

extern "C" mtgp_status mtgp_plan_free(mtgp_plan_t p)
{
    GUARD_BEGIN
    destroy_plan(p);
    return ok();
    GUARD_END
}

extern "C" const char* mtgp_last_error(void) { return g_last_error.c_str(); }

extern "C" const char* mtgp_version(void) { return "libmtgp 0.1 (sm_103a)"; }

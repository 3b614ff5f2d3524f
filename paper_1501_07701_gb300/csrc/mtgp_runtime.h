// Host-side runtime structures behind the C ABI (not part of the public
// interface).
#pragma once

#include <array>
#include <new>
#include <tuple>
#include <vector>

#include "../../include/mtgp.h"
#include "mtgp_internal.h"

#define MTGP_MAX_N 16384u

struct mtgp_params {
    mtgp_params_desc d;   // completed fields
    mtgp::KParams k;      // kernel form (with the float tempering table)
};

namespace mtgp {

// Requests grouped per stream (in request order), streams sorted by total
// count, longest first.
struct Work {
    std::vector<WorkItem> items;
    std::vector<uint64_t> item_total;   // numbers per item, same order as items
    std::vector<Segment> segs;
    uint64_t total = 0;
    uint64_t max_item = 0;
};

// A pinned host buffer and a device buffer holding one uploaded work table
// (work counter, items, segments); `ev` marks the end of the kernel that
// consumed it, so the slot can be refilled.
struct TableSlot {
    void* host = nullptr;
    void* dev = nullptr;
    size_t cap = 0;
    cudaEvent_t ev = nullptr;
    bool ev_recorded = false;
};

struct DeviceGuard {
    int prev;
    explicit DeviceGuard(int dev);
    ~DeviceGuard();
};

mtgp_status fail(mtgp_status st, const char* fmt, ...);
mtgp_status fail_cuda(cudaError_t e, const char* what);
mtgp_status ok();

}  // namespace mtgp

// Keeps C++ exceptions from crossing the C ABI: an entry point's body sits
// between GUARD_BEGIN and GUARD_END and returns a status instead.
#define GUARD_BEGIN try {
#define GUARD_END                                                                      \
    }                                                                                  \
    catch (const std::bad_alloc&) { return fail(MTGP_ENOMEM, "host allocation failed"); } \
    catch (...) { return fail(MTGP_EINVAL, "unexpected internal error"); }

struct mtgp_streams {
    mtgp_params P;
    int device = 0;
    uint32_t n_streams = 0;
    uint32_t* d_states = nullptr;   // n_streams rows of P.k.np words
    int* d_err = nullptr;           // device error word
    // per-stream parameter sets (mtgp_init_statuses_multi): then P is a
    // representative set (largest pos and mirror, for window checks and
    // shared-memory sizing) and the kernels read each stream's own set
    mtgp::KSet* d_sets = nullptr;
    uint32_t* d_set_of = nullptr;
    uint32_t n_sets = 0;
    mtgp::LaunchCfg cfg{};
    std::array<mtgp::TableSlot, 4> slots{};
    int next_slot = 0;
    // launch geometry cache (for the current cfg; grid = residency cap)
    bool geo_valid = false;
    std::tuple<int, int, int, int> geo_key{};
    mtgp::Geometry geo_cap{};
    // device-to-host path
    // (kStages buffers: generation may run that many chunks ahead of the copies)
    static constexpr int kStages = 4;
    void* stage[kStages] = {};
    uint64_t stage_cap = 0;   // elements per staging buffer
    cudaEvent_t ev_gen[kStages] = {};
    cudaEvent_t ev_copy[kStages] = {};
    cudaStream_t copy_stream = nullptr;
    // the work tables of every chunk of one device-to-host call, uploaded
    // together before its first kernel
    void* d_chunk_tables = nullptr;
    size_t chunk_tables_cap = 0;
    // autotuning
    cudaStream_t tune_stream = nullptr;
    cudaEvent_t tune_ev[2] = {nullptr, nullptr};
};

namespace mtgp {

// Jumps of state rows prepared on the host: items and the bit table of their
// polynomials (`words` 32-bit words each), and the jump kernel's dynamic
// shared memory.
struct JumpBatch {
    std::vector<JumpItem> items;
    std::vector<uint32_t> poly_words;
    uint32_t words = 0;
    size_t smem = 0;
};

// A launch whose longest streams are cut into pieces.  It runs the
// generation kernel on a state array of its own with one row per launched
// item (a whole stream, or one piece): `work` holds the items with their
// rows in WorkItem::stream.  Before the kernel, `copies` (stream -> row)
// give every row its stream's state and `jumps` advance the rows of pieces
// after a stream's first by the piece's offset in the stream; after it,
// `backs` (row -> stream) return the state of every unsplit stream and of
// every split stream's last piece.  row_set: parameter-set index of each
// row's stream (handles with one set per stream).
struct SplitWork {
    Work work;
    uint64_t max_piece = 0;        // 0 = not split
    uint32_t n_rows = 0;           // rows of the launch's own state array
    uint32_t n_split = 0;          // streams cut into pieces
    uint32_t n_pieces = 0;         // pieces of those streams
    std::vector<uint2> copies;
    std::vector<uint2> backs;
    std::vector<uint32_t> row_set;
    std::vector<uint32_t> jump_rows, jump_sets;
    std::vector<uint64_t> jump_lens;
};

}  // namespace mtgp

struct mtgp_plan {
    mtgp_streams* st = nullptr;
    void* out = nullptr;
    uint32_t n_items = 0;
    uint32_t n_coop = 0;
    uint64_t total = 0;
    uint64_t max_item = 0;
    mtgp::LaunchCfg cfg{};
    mtgp::Geometry geo{};
    mtgp::Work work;               // the requests, one item per stream
    mtgp::SplitWork split;         // the launched work (pieces when split)
    // split launches: the launch's state rows, copy pairs, per-row parameter
    // set index, jump items and polynomials
    uint32_t* d_rows = nullptr;
    uint2* d_copies = nullptr;
    uint2* d_backs = nullptr;
    uint32_t* d_row_set = nullptr;
    mtgp::JumpItem* d_jitems = nullptr;
    uint32_t* d_jpolys = nullptr;
    mtgp::JumpBatch jumps;
    void* d_table = nullptr;
    uint64_t* d_trace = nullptr;   // optional per-item timeline
    size_t items_off = 0, segs_off = 0;
    cudaStream_t cap_stream = nullptr;
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
    uint32_t kernel_launches = 0;
    uint32_t n_req = 0;            // requests of the plan (statistics rows)
    // fused statistics (mtgp_plan_set_stats): the kernel, its geometry and
    // arguments, and the per-request counts it writes
    bool stats = false;
    mtgp::StatsArgs sa{};
    const void* stats_fn = nullptr;
    mtgp::Geometry stats_geo{};
    unsigned long long* d_hist = nullptr;
    unsigned long long* d_tab = nullptr;
    // split plans with statistics: each request's first output index, one
    // edge record per launched segment, and each request's pieces in order
    unsigned long long* d_req_base = nullptr;
    mtgp::SegStat* d_seg_stats = nullptr;
    uint32_t* d_piece_start = nullptr;
    uint32_t* d_pieces = nullptr;
};

namespace mtgp {

// Groups requests per stream (request order kept), sorts streams longest
// first.  Request j's output goes to out_offs[j] if out_offs is given, else
// to out_base + the exclusive prefix sum of counts.
mtgp_status build_work(uint32_t n_streams, const uint32_t* ids, const uint64_t* counts,
                       const int32_t* fmts, uint32_t fmt_all, uint32_t n_req, uint64_t out_base,
                       Work& w, const uint64_t* out_offs = nullptr);
size_t table_bytes(const Work& w, size_t* items_off, size_t* segs_off);
void fill_table(const Work& w, void* host);
LaunchCfg default_config(const KParams& P);
mtgp_status geometry_for(mtgp_streams* st, const LaunchCfg& cfg, uint32_t n_items, Geometry* g);
mtgp_status launch_work(mtgp_streams* st, const Work& w, const LaunchCfg& cfg, void* out,
                        cudaStream_t s);
// A launch's own state rows (a split launch: one row per item, see
// SplitWork) in place of the handle's states; set_of: each row's parameter
// set index (handles with one set per stream), else null.
struct RowArray {
    uint32_t* states;
    uint32_t n_rows;
    const uint32_t* set_of;
};
mtgp_status launch_work_slot(mtgp_streams* st, TableSlot& sl, const Work& w, const LaunchCfg& cfg,
                             void* out, cudaStream_t s, const RowArray* rows = nullptr);
// Launches `w` from a work table already in device memory at `table`
// (counters zeroed, laid out by table_bytes / fill_table).
mtgp_status launch_work_table(mtgp_streams* st, const Work& w, void* table, const LaunchCfg& cfg,
                              void* out, cudaStream_t s, const RowArray* rows = nullptr);
void free_table_slot(TableSlot& s);
mtgp_status validate_config(const mtgp_launch_config* c, LaunchCfg* out);
// Number of leading (longest) items a launch hands to whole CTAs.
uint32_t coop_count(const Work& w, const Geometry& g, int coop_percent);
std::vector<LaunchCfg> tuning_candidates(const KParams& P);
mtgp_status time_config(mtgp_streams* st, const Work& w, const LaunchCfg& cfg, uint32_t* states,
                        void* out, int reps, float* best_ms);

// Cuts the items of `w` longer than max_piece numbers into pieces of
// max_piece numbers (the last one shorter), at most max_pieces per stream
// (longer streams get equal pieces of ceil(total / max_pieces)), gives every
// item its own row, and sorts the items longest first.  set_of_stream:
// per-stream parameter set index (empty for one shared set).
mtgp_status split_work(const Work& w, uint64_t max_piece, uint32_t max_pieces,
                       const std::vector<uint32_t>& set_of_stream, SplitWork* out);

// Jump polynomials and items for advancing rows[i] (of the array the launch
// is given) by jumps[i] numbers (0 = no jump); sets[i] = parameter set index.
// host_sets: a host copy of the handle's per-stream parameter sets (null:
// read from the device when needed).
mtgp_status build_jump_batch(mtgp_streams* st, const std::vector<uint32_t>& rows,
                             const std::vector<uint32_t>& sets, const std::vector<uint64_t>& jumps,
                             JumpBatch* out, const std::vector<KSet>* host_sets = nullptr);
cudaError_t launch_jump_batch(const mtgp_streams* st, uint32_t* rows_base, const JumpItem* d_items,
                              uint32_t n, const uint32_t* d_polys, uint32_t words, size_t smem,
                              cudaStream_t s);

}  // namespace mtgp

/*
 * mtgp.h -- C ABI of libmtgp, bulk MTGP32 generation on GB300 (sm_103a).
 *
 * The library generates numbers from many independently initialised MTGP32
 * streams that share one parameter set, the setting studied by
 * Passerat-Palmbach, Mazel, Mahul and Hill, "Reliable Initialization of
 * GPU-enabled Parallel Stochastic Simulations Using Mersenne Twister for
 * Graphics Processors" (ESM 2010):
 *   - a generator is a "parameterized status" (its signature) plus a "seed
 *     status" chosen by the user (Sec. 3.1);
 *   - each stream (one per block of threads in the paper, Sec. 2 and
 *     Sec. 3.2) owns its state, which persists in global memory between
 *     launches and lives in shared memory while it is being advanced (Sec. 2);
 *   - the same sequence can be produced on a CPU (Sec. 3.2).
 *
 * Generator (the readings used where the paper prints no formula):
 *   state x_0..x_{N-1}, N = floor(Mexp/32) + 1, mask keeps the high 32 - r
 *   bits, r = 32N - Mexp;  for i = 0, 1, ...:
 *     y = (x_i & mask) ^ x_{i+1};  y ^= y << sh1;  y ^= x_{i+pos} >> sh2;
 *     x_{i+N} = y ^ REC[y & 15];
 *     t = x_{i+pos-1};  t ^= t >> 16;  t ^= t >> 8;
 *     o_i = x_{i+N} ^ TMP[t & 15];
 *   float32 [1,2) = bits 0x3F800000 | (o_i >> 9);  float32 [0,1) = that - 1.
 *   REC and TMP are GF(2)-linear 16-entry tables (XOR spans of 4 words).
 *
 * Conventions for every call:
 *   - Every function returns an mtgp_status.  On any failure nothing is
 *     written to caller buffers and stream states are unchanged; the reason
 *     is available from mtgp_last_error() on the calling thread.
 *   - No C++ exception crosses this boundary.
 *   - Handles are thread-compatible: concurrent calls on distinct handles are
 *     safe; concurrent calls on one handle must be serialised by the caller.
 *   - `cuda_stream` is a cudaStream_t passed as void* (NULL = legacy default
 *     stream).  Calls that take it are asynchronous on that stream unless
 *     stated otherwise.
 *   - "device pointer" means memory allocated on the current CUDA device;
 *     "host pointer" means ordinary (or pinned) host memory.
 */
#ifndef MTGP_H
#define MTGP_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct mtgp_params*  mtgp_params_t;   /* immutable after creation      */
typedef struct mtgp_streams* mtgp_streams_t;  /* n_streams device-resident states */
typedef struct mtgp_plan*    mtgp_plan_t;     /* a recorded batched launch     */
typedef struct mtgp_server*  mtgp_server_t;   /* continuous-batching front end */

typedef enum {
    MTGP_OK = 0,
    MTGP_EINVAL = 1,    /* an argument or a parameter field is out of range  */
    MTGP_ENOMEM = 2,    /* host or device allocation failed                   */
    MTGP_ECUDA = 3,     /* a CUDA runtime call failed                         */
    MTGP_ETIMEOUT = 4,  /* a bounded wait ran out                             */
    MTGP_EBUSY = 5,     /* admission refused: capacity is in use              */
    MTGP_EIO = 6,       /* a file could not be read or parsed                 */
    MTGP_EDEVICE = 7    /* a kernel reported an inconsistency (error word)    */
} mtgp_status;

typedef enum {
    MTGP_U32 = 0,       /* uint32 words                                        */
    MTGP_F32_12 = 1,    /* float32 in [1,2): exponent/mantissa bit-fill        */
    MTGP_F32_01 = 2     /* float32 in [0,1): the [1,2) value minus 1 (exact)   */
} mtgp_format;

/* Field-by-field description of a parameterized status (Sec. 3.1).  The
 * 16-entry tables are the "fast status" form (precomputed entries).        */
typedef struct {
    uint32_t mexp;          /* Mersenne exponent                               */
    uint32_t n;             /* state words N; 0 = floor(mexp/32) + 1           */
    uint32_t pos;           /* 1 <= pos <= N-1                                 */
    uint32_t sh1, sh2;      /* 0..31                                           */
    uint32_t mask;          /* 0 = 0xFFFFFFFF << (32N - mexp), needs 1..31     */
    uint32_t rec_tbl[16];   /* recursion table, must be GF(2)-linear           */
    uint32_t tmp_tbl[16];   /* tempering table, must be GF(2)-linear           */
} mtgp_params_desc;

/* ---------------------------------------------------------------------- */
/* Parameterized status                                                   */
/* ---------------------------------------------------------------------- */

/* Sec. 3.1 (parameterized status).  Reads a text file of `key value...`
 * lines ('#' comments): mexp, pos, sh1, sh2, optional n and mask, and either
 * rec_basis (4 words) or rec_tbl (16 words), likewise tmp_basis / tmp_tbl.
 * Numbers are decimal or 0x-hex.  *out receives a new handle owned by the
 * caller (free with mtgp_params_free).  MTGP_EIO if the file cannot be read
 * or parsed, MTGP_EINVAL if a field is out of range or a table is not
 * GF(2)-linear. */
mtgp_status mtgp_params_load(const char* path, mtgp_params_t* out);

/* Sec. 3.1 / Sec. 6 (the paper's parameter sets are not printed): draws a
 * parameter set for `mexp` from a SplitMix64 stream seeded with `seed`, in
 * the order sh1, sh2, pos, rec_basis[0..3], tmp_basis[0..3]
 * (sh = 1 + d % 31; pos in [2, N - Wmin], Wmin = min(256, largest power of
 * two <= N-2); basis words = d >> 32).  MTGP_EINVAL if mexp is a multiple of
 * 32 or below 33. */
mtgp_status mtgp_params_generate(uint32_t mexp, uint64_t seed, mtgp_params_t* out);

/* Sec. 3.1: parameter set from explicit fields (`desc` is copied). */
mtgp_status mtgp_params_create(const mtgp_params_desc* desc, mtgp_params_t* out);

/* Sec. 3.1: copies the completed fields (n, mask, tables filled in) into
 * *desc (a host struct owned by the caller). */
mtgp_status mtgp_params_get(mtgp_params_t params, mtgp_params_desc* desc);

/* Handle bookkeeping, no counterpart in the paper: releases the handle
 * (NULL is accepted).  Handles already copied into stream sets stay valid. */
mtgp_status mtgp_params_free(mtgp_params_t params);

/* ---------------------------------------------------------------------- */
/* Streams: seed statuses and device-resident states                      */
/* ---------------------------------------------------------------------- */

/* Sec. 3.1 / Sec. 5.1 (seed status; one status per block, Sec. 3.2).
 * Creates n_streams states on the current device, stream s initialised from
 * the host array seeds[s] by w_0 = seed, w_i = 1812433253*(w_{i-1} ^
 * (w_{i-1} >> 30)) + i.  `seeds` is a host pointer to n_streams words, read
 * before the call returns.  The params handle is copied (the caller may free
 * it).  Asynchronous on cuda_stream.  *out is owned by the caller. */
mtgp_status mtgp_init_statuses(mtgp_params_t params, const uint32_t* seeds, uint32_t n_streams,
                               void* cuda_stream, mtgp_streams_t* out);

/* Sec. 3.1 / Sec. 4.1 / Sec. 5.1: one parameterized status per stream (the
 * paper's 10 000 independent parameter sets, and its "Random Spacing" pairs
 * of parameterized and seed statuses).  Stream s uses the parameter set
 * sets[set_of_stream[s]] and is seeded from seeds[s] as in
 * mtgp_init_statuses.  All n_sets sets must share Mexp (hence N and the
 * mask); they may differ in pos, sh1, sh2 and the tables.  `sets`,
 * `set_of_stream` (n_streams indices < n_sets) and `seeds` are host arrays
 * read before the call returns; the parameter handles are copied.  The
 * resulting handle works with every generation, plan, serving, checkpoint
 * and tuning call.  MTGP_EINVAL if the sets differ in Mexp/N or an index is
 * out of range. */
mtgp_status mtgp_init_statuses_multi(const mtgp_params_t* sets, uint32_t n_sets,
                                     const uint32_t* set_of_stream, const uint32_t* seeds,
                                     uint32_t n_streams, void* cuda_stream, mtgp_streams_t* out);

/* Sec. 2 (a generator's state persists in global memory between kernel
 * launches) and Sec. 3.1 (a user-chosen status in place of a seeded one):
 * overwrites all device states from the host array `states` (n_streams x N
 * words, row s = stream s, oldest word first).  Synchronous: returns after
 * the copy.  MTGP_EINVAL for a null pointer; the masked low bits of each
 * row's oldest word are stored as given (they never reach an output). */
mtgp_status mtgp_set_statuses(mtgp_streams_t streams, const uint32_t* states, void* cuda_stream);

/* Sec. 2 (state persisting in global memory between launches): copies all
 * states to the host array `states` (n_streams x N words, caller-owned,
 * oldest word first: after c outputs of a stream its row is
 * x_c .. x_{c+N-1}).  Waits for cuda_stream.  Together with
 * mtgp_set_statuses this is the checkpoint/restore pair: restoring a saved
 * row and generating continues the stream exactly where it was saved. */
mtgp_status mtgp_get_statuses(mtgp_streams_t streams, uint32_t* states, void* cuda_stream);

/* Bookkeeping, no counterpart in the paper: number of streams and words
 * per state (N) of the handle, into host integers (either may be NULL). */
mtgp_status mtgp_streams_info(mtgp_streams_t streams, uint32_t* n_streams, uint32_t* n_words);

/* Sec. 2 (per-block generator) and Sec. 3.2 (many statuses in one launch).
 * Request j draws counts[j] numbers from stream stream_ids[j] into
 * out[off_j .. off_j + counts[j]), off = exclusive prefix sum of counts.
 * stream_ids and counts are host arrays of n_req entries; `out` is a device
 * pointer to at least sum(counts) 4-byte elements (caller-owned).  Requests
 * naming the same stream are applied in array order.  States advance in
 * place.  Asynchronous on cuda_stream; host arrays are consumed before
 * return.  MTGP_EINVAL for an id >= n_streams or a null pointer with a
 * non-zero total. */
mtgp_status mtgp_generate_u32(mtgp_streams_t streams, const uint32_t* stream_ids,
                              const uint64_t* counts, uint32_t n_req, uint32_t* out,
                              void* cuda_stream);

/* As mtgp_generate_u32, with fmt MTGP_F32_12 or MTGP_F32_01 (MTGP_U32 is also
 * accepted and writes the integer bit patterns). */
mtgp_status mtgp_generate_f32(mtgp_streams_t streams, const uint32_t* stream_ids,
                              const uint64_t* counts, uint32_t n_req, mtgp_format fmt,
                              float* out, void* cuda_stream);

/* Sec. 3.2 (the same streams feeding CPU code): as mtgp_generate_u32/_f32 but
 * `host_out` is a host pointer (pinned memory gives full copy bandwidth).
 * Generation runs in chunks of at most `chunk_bytes` (0 = 1 GiB) into a
 * library-owned device staging area, overlapped with device-to-host copies.
 * Returns after all numbers are in host_out (synchronous). */
mtgp_status mtgp_generate_to_host(mtgp_streams_t streams, const uint32_t* stream_ids,
                                  const uint64_t* counts, uint32_t n_req, mtgp_format fmt,
                                  void* host_out, uint64_t chunk_bytes, void* cuda_stream);

/* No counterpart in the paper: a variant of mtgp_generate_u32/_f32 for
 * callers that cannot have device memory allocated on their behalf once
 * running (a simulation that reserved the GPU's memory up front, a real-time
 * loop that must not enter the allocator, a host runtime that forbids hidden
 * allocations).  Same request semantics, formats and output layout as
 * mtgp_generate_u32/_f32 (`out` is a device pointer of sum(counts) 4-byte
 * elements); at most 1024 requests per call, more is MTGP_EINVAL.  It calls
 * no cudaMalloc, cudaFree or other allocating routine: the work table lives
 * in a 64 KiB statically declared device array that every device loading the
 * library holds until exit.  The first call on a device looks that array's
 * address up (cudaGetSymbolAddress); make that first call before any stream
 * capture.  All calls on a device share the array and each overwrites the
 * previous contents (the claim counters are cleared on every call), so calls
 * whose kernels overlap on the GPU race: order them (one CUDA stream, one
 * host thread at a time).  The work table is copied from a host array that
 * the next call overwrites, so a call made while cuda_stream is being
 * captured returns MTGP_EINVAL (record graphs with mtgp_plan_create).  The
 * array's address is looked up once per device for the life of the
 * process: a cudaDeviceReset while the library is loaded is not supported
 * by this call.  Asynchronous on cuda_stream. */
mtgp_status mtgp_generate_noalloc(mtgp_streams_t streams, const uint32_t* stream_ids,
                                  const uint64_t* counts, uint32_t n_req, mtgp_format fmt,
                                  void* out, void* cuda_stream);

/* Waits for cuda_stream and reads the device error word of this handle.
 * MTGP_EDEVICE if a kernel recorded an inconsistency since the last check
 * (the word is then cleared). */
mtgp_status mtgp_check(mtgp_streams_t streams, void* cuda_stream);

/* Handle bookkeeping, no counterpart in the paper: waits for the handle's
 * work and frees its device states (NULL is accepted). */
mtgp_status mtgp_streams_free(mtgp_streams_t streams);

/* ---------------------------------------------------------------------- */
/* Launch configuration and autotuning                                    */
/* ---------------------------------------------------------------------- */

typedef struct {
    uint32_t warps_per_cta;   /* block size / 32: 1..8 (the register-resident
                                 path uses 2, 4 or 8)                          */
    uint32_t ctas_per_sm;     /* resident CTAs per SM (0 = occupancy maximum)   */
    uint32_t words_per_lane;  /* sub-steps per parallel step (2, 4 or 8); the
                                 window is 32 * words_per_lane <= N - pos      */
    uint32_t kernel;          /* 0 = register-resident path when available,
                                 1 = shared-memory ring path (any parameters)  */
    uint32_t coop_percent;    /* streams of a launch longer than coop_percent/100
                                 times the numbers per warp slot are advanced
                                 by a whole CTA (longest first); 0 = never     */
} mtgp_launch_config;

mtgp_status mtgp_get_launch_config(mtgp_streams_t streams, mtgp_launch_config* cfg);
mtgp_status mtgp_set_launch_config(mtgp_streams_t streams, const mtgp_launch_config* cfg);

/* Times candidate configurations on a scratch copy of up to `sample_streams`
 * states (the handle's states are not advanced), `sample_count` numbers per
 * stream, in format `fmt`; installs and returns the fastest.  Results are
 * cached per process by (device, N, format).  Synchronous. */
mtgp_status mtgp_autotune(mtgp_streams_t streams, mtgp_format fmt, uint32_t sample_streams,
                          uint64_t sample_count, mtgp_launch_config* best);

/* ---------------------------------------------------------------------- */
/* Plans: one persistent launch replayed from a CUDA graph                */
/* ---------------------------------------------------------------------- */

/* Records a batched launch for the requests (same meaning as
 * mtgp_generate_u32; every request in format `fmt`; `out` is a device
 * pointer that must stay valid while the plan is used).  The work table is
 * sorted longest stream first and uploaded once; launching replays a CUDA
 * graph (reset of the work counter + one persistent kernel whose warps claim
 * streams from that table).  The plan keeps a reference to `streams`. */
mtgp_status mtgp_plan_create(mtgp_streams_t streams, const uint32_t* stream_ids,
                             const uint64_t* counts, uint32_t n_req, mtgp_format fmt,
                             void* out, mtgp_plan_t* plan);

/* Replays the plan on cuda_stream: every launch draws the next counts[j]
 * numbers of each stream (states advance). */
mtgp_status mtgp_plan_launch(mtgp_plan_t plan, void* cuda_stream);

typedef struct {
    uint64_t total_numbers;   /* sum of counts                                 */
    uint32_t n_items;         /* items of the launched table: the plan's
                                 streams, or pieces of split streams           */
    uint32_t kernel_launches; /* kernels per plan launch                       */
    mtgp_launch_config config;
    uint32_t grid_ctas;
    uint32_t n_coop;          /* streams advanced by whole CTAs                 */
    uint32_t regs_per_thread; /* of the generation kernel                       */
    uint32_t resident_ctas_per_sm;
    uint64_t max_piece;       /* piece length of split streams (0 = no split)   */
    uint32_t n_split_streams; /* streams cut into pieces                        */
    uint32_t n_jumps;         /* jumps per launch (pieces after a first one)    */
    uint32_t n_pieces;        /* pieces of the split streams                    */
    uint32_t stats;           /* 1: statistics fused into generation            */
} mtgp_plan_info;

/* Sec. 1 and Sec. 2 (one generator's stream shared out as sub-streams;
 * streams persisting in global memory between launches): cuts every stream
 * of the plan whose count exceeds max_piece into pieces of max_piece numbers
 * (the last one shorter; at most 64 pieces per stream, longer streams get 64
 * equal pieces), so that one long stream is advanced by several warps at
 * once.  A split plan runs on state rows of its own, one per launched item
 * (a whole stream or a piece): each launch copies the streams' states into
 * them, advances the rows of later pieces by their offsets j * max_piece
 * with exact jumps (mtgp_jump's method; the jump polynomials are computed on
 * the host once per plan), runs the generation kernel over the items,
 * longest first, and copies the unsplit streams' rows and every split
 * stream's last piece back as the streams' new states.  Outputs and states
 * are exactly those of the unsplit plan.  max_piece = 0 removes the split;
 * 1 .. 63 is MTGP_EINVAL.  Re-records the plan's graph; synchronous.  The
 * plan holds N words of device memory per launched item. */
mtgp_status mtgp_plan_set_split(mtgp_plan_t plan, uint64_t max_piece);

/* Configuration of the statistics fused into a plan (mtgp_plan_set_stats):
 * the data reductions of the paper's two failing BigCrush tests (Sec. 4.2)
 * with the parameters and definitions of mtgp_gap_histogram and
 * mtgp_hamming_pairs.  gap_t = 0 leaves out the gap test; ham_L = 0 leaves
 * out the Hamming test. */
typedef struct {
    uint32_t gap_r, gap_b, gap_t;   /* test 35: b >= 1, r + b <= 32, 1 <= t <= 1023      */
    uint32_t ham_r, ham_s, ham_L;   /* test 100: s >= 1, r + s <= 32, L % s == 0, L/s >= 32 */
    uint32_t n_bounds;              /* weight classes C = n_bounds + 1 <= 16              */
    uint32_t bounds[15];            /* ascending class bounds (first n_bounds used)       */
} mtgp_stats_config;

/* Sec. 4.2 (the gap test, test 35, and Hamming-weight independence,
 * test 100): makes every later launch of the plan also compute, for each of
 * its requests, the gap histogram and the Hamming block-pair table of the
 * 32-bit words it stores (the tempered outputs, or the float bit patterns
 * of a float format), exactly as mtgp_gap_histogram and mtgp_hamming_pairs
 * would over the plan's output buffer, request j being sequence j.  The
 * counts are accumulated by a generation kernel of its own while the
 * outputs are still in registers, so the outputs are not read back from
 * memory; mtgp_plan_read_stats returns them.  In a split plan
 * (mtgp_plan_set_split, before or after this call) a request's pieces are
 * counted by the warps that generate them; each piece records the run of
 * non-visits before its first visit and after its last, and its weights in
 * the block pairs open at its start and end, and a stitch kernel in the same
 * launch counts what lies across the pieces' edges.  The counts are the
 * same as for the unsplit plan.  cfg = NULL (or both tests left out)
 * returns the plan to the plain generation kernel.
 * MTGP_EINVAL: parameters out of range; a plan with tracing on; a request
 * of 2^31 numbers or more; a state size without an instantiation of the
 * fused kernel (ceil(N/32) of 4, 5, 10, 11, 20, 22, 23 or 44: e.g. Mexp
 * 3217, 4253, 11213, 23209 and 44497); a parameter set with N - pos < 256
 * (< 32 for ceil(N/32) of 4 or 5, whose rows are counted one 32-column
 * sub-step at a time).  Re-records the plan's graph; synchronous.  No counterpart in
 * the paper beyond the tests' definitions: it fuses the paper's quality
 * measurements into generation. */
mtgp_status mtgp_plan_set_stats(mtgp_plan_t plan, const mtgp_stats_config* cfg);

/* Copies the statistics of the plan's last launch (queued on cuda_stream)
 * to the host: hist (n_req x (gap_t + 1), may be NULL when the gap test is
 * off) and table (n_req x C x C, may be NULL when the Hamming test is off),
 * in the layouts of mtgp_gap_histogram and mtgp_hamming_pairs.  Waits for
 * cuda_stream.  MTGP_EINVAL when the plan has no statistics. */
mtgp_status mtgp_plan_read_stats(mtgp_plan_t plan, uint64_t* hist, uint64_t* table, void* cuda_stream);

/* Times the tuning candidates on this plan's own work table, on a scratch
 * copy of all states (the handle's states are not advanced; the plan's `out`
 * buffer is overwritten), installs the fastest in the plan and re-records its
 * graph.  Synchronous. */
mtgp_status mtgp_plan_autotune(mtgp_plan_t plan, mtgp_launch_config* best);

/* Timeline of the plan's launches (diagnostics; no counterpart in the
 * paper).  enable = 1 allocates a device record of 4 words per stream of the
 * plan and re-records the graph so that every later launch stores, for each
 * stream in the plan's table order (longest first): the start and end time
 * of its generation (%globaltimer, ns), the SM it ran on, and its count.
 * enable = 0 drops the record.  Synchronous. */
mtgp_status mtgp_plan_set_trace(mtgp_plan_t plan, int enable);

/* Copies the record of the last launch to the host array `host` of
 * 4 * n_items uint64 (n_items from mtgp_plan_get_info). */
mtgp_status mtgp_plan_read_trace(mtgp_plan_t plan, uint64_t* host);

/* Bookkeeping, no counterpart in the paper: the plan's shape and launch
 * configuration into the caller's host struct. */
mtgp_status mtgp_plan_get_info(mtgp_plan_t plan, mtgp_plan_info* info);

/* Handle bookkeeping: waits for the plan's launches and frees its work table
 * and graph (the streams handle is not freed). */
mtgp_status mtgp_plan_free(mtgp_plan_t plan);

/* ---------------------------------------------------------------------- */
/* Serving: continuous batching over resident streams                     */
/* ---------------------------------------------------------------------- */
/* Clients ask for k numbers of stream s (the per-block streams of Sec. 3.2
 * consumed by a running simulation).  States stay resident in HBM.  A
 * request is admitted when its stream is not inside an in-flight tick and
 * its output fits in the device arena (the admission cap); admitted
 * requests are coalesced into a tick, one kernel launch; up to max_inflight
 * ticks run at once on separate CUDA streams.  Requests for one stream
 * complete in submission order and produce exactly the numbers a lone
 * request sequence would.
 *
 * With cfg.max_piece (Sec. 1 and 2: sub-streams of one generator), a tick
 * takes either requests longer than max_piece or shorter ones.  The long
 * requests' streams are cut into pieces of max_piece numbers (at most 64; a
 * longer stream gets 64 equal pieces), each started by an exact jump and
 * advanced by its own warp, so that a long request completes in about a
 * piece's time plus a jump's; short requests never wait for jumps.  The
 * jump polynomials of the offsets j * max_piece (j < 64) are computed when
 * the server is created and kept on the device (handles with one parameter
 * set); other offsets and per-stream sets compute theirs on first use
 * (cached). */

typedef struct {
    uint64_t arena_bytes;        /* device output arena = admission cap (0 = 8 GiB) */
    uint32_t max_inflight;       /* ticks in flight at once, 1..64 (0 = 4)          */
    uint32_t max_tick_requests;  /* requests coalesced into one tick (0 = 4096)     */
    double   tick_timeout_s;     /* longest wait for one launch's completion before
                                    progress / run_trace return MTGP_ETIMEOUT,
                                    seconds > 0 (0 = 60)                           */
    uint64_t max_piece;          /* requests longer than this are cut into pieces
                                    started by exact jumps, as in a split plan,
                                    and ticks take either such requests or
                                    shorter ones (0 = never; else >= 64)           */
} mtgp_server_config;

typedef struct {
    uint64_t tag;                /* the caller's tag from mtgp_server_submit        */
    uint64_t count;              /* numbers produced                                */
    uint64_t arena_offset;       /* element offset of the result in the arena       */
    int32_t  fmt;                /* mtgp_format of the result                       */
    int32_t  pad;
    double   submit_time;        /* seconds, steady clock                           */
    double   done_time;          /* seconds, when completion was observed           */
} mtgp_completion;

typedef struct {
    uint64_t requests;           /* completed                                       */
    uint64_t numbers;            /* produced                                        */
    uint64_t ticks;              /* kernel launches                                 */
    double   elapsed;            /* seconds from the first arrival to the last completion */
    double   busy_wait;          /* seconds the loop idled while requests were queued */
    double   launch_host_s;      /* host seconds spent building work tables and
                                    issuing launches (table upload + kernel)      */
    uint64_t jumps;              /* pieces started by jumps (max_piece > 0)       */
} mtgp_server_stats;

/* Creates a server over `streams` (kept by reference; must outlive the
 * server).  The arena is a library-owned device buffer of cfg->arena_bytes
 * (cfg may be NULL for the defaults). */
mtgp_status mtgp_server_create(mtgp_streams_t streams, const mtgp_server_config* cfg,
                               mtgp_server_t* out);

/* Queues a request for `count` numbers of stream `stream_id` in format
 * `fmt`.  MTGP_EBUSY if count * 4 bytes exceeds the whole arena, MTGP_EINVAL
 * for a bad id or format. */
mtgp_status mtgp_server_submit(mtgp_server_t server, uint32_t stream_id, uint64_t count,
                               mtgp_format fmt, uint64_t tag);

/* Non-blocking: collects finished ticks, then admits queued requests into
 * one tick and launches it if a tick slot is free.  Up to `max_out`
 * completions are copied to the host array `out`; *n_out receives their
 * number (the rest stay queued for later calls).  A completion's result
 * stays valid in the arena until mtgp_server_release.  MTGP_ETIMEOUT if a
 * tick's completion has not been observed tick_timeout_s seconds after its
 * launch (failure detection; no counterpart in the paper): nothing is lost,
 * the tick stays in flight and a later call collects it if it completes. */
mtgp_status mtgp_server_progress(mtgp_server_t server, mtgp_completion* out, uint32_t max_out,
                                 uint32_t* n_out);

/* Returns a completed result's arena space (offset and count as reported). */
mtgp_status mtgp_server_release(mtgp_server_t server, uint64_t arena_offset, uint64_t count);

/* Device pointer of the arena (4-byte elements). */
mtgp_status mtgp_server_arena(mtgp_server_t server, void** arena);

/* Copies `count` elements starting at arena element `arena_offset` to the
 * host array `host_dst` (synchronous; for clients that consume results on
 * the CPU).  MTGP_EINVAL if the range leaves the arena. */
mtgp_status mtgp_server_read(mtgp_server_t server, uint64_t arena_offset, uint64_t count,
                             void* host_dst);

/* Diagnostics for failure-detection tests (no counterpart in the paper):
 * while `hold` is non-zero the server reads every launch's completion as
 * "not ready", as if the device never reported it.  The kernels themselves
 * run and finish normally; only the host's view is held, so
 * mtgp_server_progress and mtgp_server_run_trace reach their MTGP_ETIMEOUT
 * path without stalling the GPU.  hold = 0 restores normal operation. */
mtgp_status mtgp_server_debug_hold(mtgp_server_t server, int hold);

/* Replays an arrival trace in real time on an idle server: request j
 * arrives t_arrival[j] seconds after the call starts (non-decreasing) and
 * asks for counts[j] numbers of stream ids[j] in format fmts[j]; latency[j]
 * receives arrival-to-observed-completion seconds.  All arrays are host
 * arrays of n entries.  mode 0 = continuous batching (ticks as above);
 * mode 1 = one launch per request on 16 CUDA streams (stream id mod 16), the
 * comparison.  If record_offsets is non-NULL it receives each result's
 * arena offset and no arena space is reused (the arena must then hold the
 * whole trace).  Synchronous.  MTGP_ETIMEOUT as for mtgp_server_progress;
 * the requests of the trace not yet completed then stay queued on the
 * server (collect them with mtgp_server_progress or free the server). */
mtgp_status mtgp_server_run_trace(mtgp_server_t server, const double* t_arrival,
                                  const uint32_t* ids, const uint64_t* counts,
                                  const int32_t* fmts, uint32_t n, uint32_t mode,
                                  double* latency, uint64_t* record_offsets,
                                  mtgp_server_stats* stats);

/* Waits for in-flight ticks and frees the server and its arena. */
mtgp_status mtgp_server_free(mtgp_server_t server);

/* ---------------------------------------------------------------------- */
/* Jump-ahead (sub-streams of one generator, Sec. 1)                      */
/* ---------------------------------------------------------------------- */

/* Advances stream ids[i] by jumps[i] numbers, exactly as generating and
 * discarding them would, in time independent of the jump length: the state
 * after J steps is one step applied to g(F) w, g = t^(J-1) mod mu, where mu
 * annihilates the transition (see mtgp_params_minpoly).  Jumps of one stream
 * add up.  ids and jumps are host arrays of n entries.  The first jump for a
 * parameter set computes mu on the host (Berlekamp-Massey, about a second
 * for Mexp 44497); each distinct jump length costs a polynomial power on the
 * host (cached).  Runs on cuda_stream and returns when the states are
 * updated.  MTGP_EINVAL for an id out of range or a 64-bit overflow. */
mtgp_status mtgp_jump(mtgp_streams_t streams, const uint32_t* ids, const uint64_t* jumps, uint32_t n,
                      void* cuda_stream);

/* The polynomial mu over GF(2) that the jump uses for this parameter set:
 * the least common multiple of minimal polynomials of output bit sequences,
 * checked to annihilate the transition on random states (mu(F) w has only
 * the masked bits of its oldest word set).  deg mu <= Mexp; equality with
 * mu irreducible means the period 2^Mexp - 1 of a Mersenne-prime Mexp.
 * words (host, may be null to query the degree) receives the coefficients,
 * bit i of the little-endian 64-bit words = coefficient of t^i; cap_words
 * must be >= degree/64 + 1.  Pure host computation, cached. */
mtgp_status mtgp_params_minpoly(mtgp_params_t params, uint64_t* words, uint32_t cap_words,
                                int32_t* degree);

/* Sec. 4.1 (period of the parameterized status): sets *irreducible to 1 if
 * the polynomial mu of mtgp_params_minpoly has degree Mexp and is
 * irreducible over GF(2) (Rabin's test: t^(2^Mexp) = t mod mu and, for each
 * prime q dividing Mexp, gcd(t^(2^(Mexp/q)) - t, mu) = 1), else to 0.  For a
 * Mersenne-prime Mexp (2^Mexp - 1 prime, as for every MTGP exponent) this
 * is exactly a period of 2^Mexp - 1 from every non-zero state.  The Mexp
 * squarings run on the current device (about a second for Mexp 44497, 120 MB
 * of device scratch); returns when done. */
mtgp_status mtgp_params_period_check(mtgp_params_t params, void* cuda_stream, int32_t* irreducible);

/* ---------------------------------------------------------------------- */
/* Quality statistics: the data reductions of the paper's two failing     */
/* BigCrush tests (Sec. 4.2), over outputs already in device memory       */
/* ---------------------------------------------------------------------- */

/* Test 35 (gap test; the paper runs r = 25, alpha = 0, beta = 1/32, i.e.
 * b = 5).  `values` is a device pointer to n_seq sequences of 32-bit outputs
 * laid out back to back, sequence i holding counts[i] values (host array).
 * A value visits [0, 2^-b) when the b bits after its r dropped leading bits
 * are zero; a gap is the run of non-visits before a visit, counted from the
 * start of its sequence (a trailing run without a visit is not a gap).
 * hist (host, n_seq x (t+1), overwritten): hist[i*(t+1) + k] = number of
 * gaps of length k in sequence i for k < t, and of length >= t for k = t.
 * Requires b >= 1, r + b <= 32, 1 <= t <= 1023.  Runs on cuda_stream and
 * returns when hist is filled; allocates and frees its own device scratch. */
mtgp_status mtgp_gap_histogram(const uint32_t* values, const uint64_t* counts, uint32_t n_seq,
                               uint32_t r, uint32_t b, uint32_t t, uint64_t* hist,
                               void* cuda_stream);

/* Test 100 (Hamming-weight independence; the paper runs r = 25, s = 5,
 * L = 1200).  The s bits after the r dropped leading bits of each value form
 * a bit string cut into L-bit blocks (L a multiple of s) per sequence; each
 * pair of successive non-overlapping blocks is counted in
 * table[i*C*C + c(W1)*C + c(W2)] (host, n_seq x C x C, overwritten), where
 * W1, W2 are the pair's Hamming weights and c(w) = number of bounds <= w
 * (bounds: host array of n_bounds ascending values, C = n_bounds + 1 <= 16).
 * Blocks of an incomplete trailing pair are ignored.  Same layout, stream
 * and scratch conventions as mtgp_gap_histogram. */
mtgp_status mtgp_hamming_pairs(const uint32_t* values, const uint64_t* counts, uint32_t n_seq,
                               uint32_t r, uint32_t s, uint32_t L, const uint32_t* bounds,
                               uint32_t n_bounds, uint64_t* table, void* cuda_stream);

/* ---------------------------------------------------------------------- */

/* Message for the last failure on the calling thread ("" if none). */
const char* mtgp_last_error(void);

/* Library version string. */
const char* mtgp_version(void);

#ifdef __cplusplus
}
#endif
#endif /* MTGP_H */

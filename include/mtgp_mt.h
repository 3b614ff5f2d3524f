/*
 * libmtgp -- the original Mersenne Twister as a comparison generator.
 *
 * The paper's last experiment (Sec. 5.3, "Algorithm Variation") sets MTGP
 * beside the original Mersenne Twister (Matsumoto and Nishimura, ACM TOMACS
 * 8(1), 1998) at the same period, 2^3217 - 1, and submits both to tests 35
 * and 100.  These entry points generate that generator's streams on the GPU
 * with the same request model as mtgp_generate_u32/_f32 (mtgp.h): many
 * independently seeded streams, device-resident states, requests grouped per
 * stream in array order, outputs at the exclusive prefix sum of the counts.
 * The statistics of tests 35 and 100 (mtgp_gap_histogram, mtgp_hamming_pairs)
 * apply to either generator's output.
 *
 * Generator (w = 32; all arithmetic mod 2^32, XOR = ^):
 *   y       = (x_k & upper) | (x_{k+1} & lower),  upper = the top 32 - r bits
 *   x_{k+n} = x_{k+m} ^ (y >> 1) ^ (y odd ? a : 0)
 *   output  = tempering of x_{k+n}:
 *             z = x ^ (x >> u); z ^= (z << s) & b; z ^= (z << t) & c; z ^= z >> l
 * Output k comes from x_{k+n}; the seed state x_0 .. x_{n-1} is never output.
 * The float formats are those of mtgp.h (top 23 bits of the tempered word).
 *
 * Errors follow mtgp.h: MTGP_EINVAL for bad arguments (nothing is launched
 * and no state changes), MTGP_ECUDA for a failed CUDA call, and the message
 * is available from mtgp_last_error().
 */
#ifndef MTGP_MT_H
#define MTGP_MT_H

#include <stdint.h>

#include "mtgp.h"

#ifdef __cplusplus
extern "C" {
#endif

/* Parameters of one generator.  Valid sets have n >= 2, 1 <= m <= n - 1,
 * r <= 31, p = 32 n - r, every shift <= 31 and n <= 4096. */
typedef struct {
    uint32_t p;            /* Mersenne exponent: period 2^p - 1 for a primitive set */
    uint32_t n;            /* state words */
    uint32_t m;            /* middle offset */
    uint32_t r;            /* separation point: the low r bits of x_k are not used */
    uint32_t a;            /* bottom row of the twist matrix A */
    uint32_t u, s, t, l;   /* tempering shifts */
    uint32_t b, c;         /* tempering masks */
} mtgp_mt_params;

/* Streams of one generator: n_streams device-resident states of n words. */
typedef struct mtgp_mt* mtgp_mt_t;

/* MT19937, the parameter set printed in the 1998 paper (p = 19937). */
mtgp_status mtgp_mt_params_mt19937(mtgp_mt_params* out);

/* Seed-generated parameter set for exponent p >= 33.  The paper's sets came
 * from MT's dynamic creator, which is not part of this library, so the set
 * is drawn from SplitMix64(seed) in this order: a = (d >> 32) | 2^31,
 * b = d >> 32, c = d >> 32; with n = ceil(p / 32), r = 32 n - p,
 * m = floor(n / 2), u = 12, s = 7, t = 15, l = 18 (the dynamic creator's
 * tempering shifts for w = 32).  Such a set is not searched for a full
 * period. */
mtgp_status mtgp_mt_params_generate(uint32_t p, uint64_t seed, mtgp_mt_params* out);

/* Allocates n_streams states on the current device and seeds stream i from
 * seeds[i] (host array) with the 2002 initialisation of MT19937:
 * w_0 = seed, w_i = 1812433253 (w_{i-1} ^ (w_{i-1} >> 30)) + i.  The
 * parameter struct is copied.  Asynchronous on cuda_stream. */
mtgp_status mtgp_mt_init(const mtgp_mt_params* params, const uint32_t* seeds, uint32_t n_streams,
                         void* cuda_stream, mtgp_mt_t* out);

/* One parameter set per stream (the paper's setting: one parameterized
 * status per generator, Sec. 4.1 and 5.3): stream s uses
 * sets[set_of_stream[s]] (host arrays; the sets are copied).  All sets must
 * share p, n and r; m, a and the tempering may differ.  MTGP_EINVAL if a set
 * is invalid, the sets disagree on the state size, or an index is >= n_sets.
 * Seeding and everything else as mtgp_mt_init. */
mtgp_status mtgp_mt_init_multi(const mtgp_mt_params* sets, uint32_t n_sets,
                               const uint32_t* set_of_stream, const uint32_t* seeds,
                               uint32_t n_streams, void* cuda_stream, mtgp_mt_t* out);

/* Host <-> device copies of all states (n_streams x n words, oldest word
 * first).  Both synchronise cuda_stream. */
mtgp_status mtgp_mt_set_statuses(mtgp_mt_t mt, const uint32_t* states, void* cuda_stream);
mtgp_status mtgp_mt_get_statuses(mtgp_mt_t mt, uint32_t* states, void* cuda_stream);

/* Request j draws counts[j] numbers from stream stream_ids[j] (host arrays)
 * into out[off_j .. off_j + counts[j]), off = exclusive prefix sum of the
 * counts; out is device memory of 4-byte elements (uint32 for MTGP_U32,
 * float otherwise), 4-byte aligned.  Requests for one stream are served in
 * array order and advance its state in place.  Asynchronous on cuda_stream. */
mtgp_status mtgp_mt_generate(mtgp_mt_t mt, const uint32_t* stream_ids, const uint64_t* counts,
                             uint32_t n_req, mtgp_format fmt, void* out, void* cuda_stream);

/* Synchronises cuda_stream and reports MTGP_EDEVICE if a kernel recorded an
 * inconsistent work item since the last check. */
mtgp_status mtgp_mt_check(mtgp_mt_t mt, void* cuda_stream);

mtgp_status mtgp_mt_free(mtgp_mt_t mt);

/* The polynomial mu of a set's window transition (F mu(F) = 0, found as for
 * mtgp_params_minpoly) and the period check of mtgp_params_period_check
 * applied to it: *irreducible = 1 iff mu has degree p and is irreducible,
 * i.e. for a Mersenne-prime p every nonzero state has period 2^p - 1
 * (Sec. 5.3 compares MT and MTGP at equal period).  minpoly: *degree
 * receives deg mu; words (may be null) receives its coefficients, bit i of
 * words[i / 64] = coefficient of t^i (cap_words >= degree / 64 + 1).  Host
 * computation, cached per set; the period check runs p squarings on the
 * device (current device, cuda_stream) and synchronises it. */
mtgp_status mtgp_mt_params_minpoly(const mtgp_mt_params* params, uint64_t* words, uint32_t cap_words,
                                   int32_t* degree);
mtgp_status mtgp_mt_params_period_check(const mtgp_mt_params* params, void* cuda_stream,
                                        int32_t* irreducible);

#ifdef __cplusplus
}
#endif
#endif

/*
 * MTGP32 oracle -- TEST INFRASTRUCTURE ONLY.
 *
 * A plain, slow, sequential CPU statement of the generator studied in
 * Passerat-Palmbach et al., "Reliable Initialization of GPU-enabled Parallel
 * Stochastic Simulations Using Mersenne Twister for Graphics Processors"
 * (ESM 2010).  Only the test-suite, the smoke check and the CPU-baseline leg
 * of the benchmark may load this library; the product path never does.
 * It shares no code, header, table or constant generator with the CUDA
 * library.
 *
 * The paper describes the generator's data model (Sec. 3.1: a "seed status"
 * chosen by the user plus a "parameterized status" that is the generator's
 * signature; "fast" statuses carry precomputed tables) and its CPU twin
 * (Sec. 3.2: the same sequence on a CPU, used for testing).  It does not print
 * the recurrence; the readings used here (recurrence over words i, i+1, i+pos,
 * table tempering over word i+pos-1, mask of the r = 32N - Mexp dropped bits,
 * MT-family seeding, float bit-fill) are listed with their justification in
 * the project's design notes and repeated at each function below.
 *
 * Parity status per function:
 *   omtgp_params_generate  pinned (bit-exact against a second SplitMix64)
 *   omtgp_init_state       pinned (first 624 words equal NumPy's MT19937
 *                          integer seeding); the MTGP release's extra
 *                          parameter-derived fill is deliberately omitted,
 *                          so "parity vs the MTGP release" is unpinned
 *   omtgp_generate         pinned (hand-worked example, GF(2) bit-matrix
 *                          formulation, impulse responses, linearity,
 *                          linear complexity <= Mexp, float value identities)
 *   omtgp_gap_histogram    pinned (constructed visit patterns with known
 *                          gaps, bit-field selection, period-k closed form,
 *                          length invariant, chi-square sanity on an
 *                          independent generator)
 *   omtgp_hamming_pairs    pinned (constant and alternating blocks, blocks
 *                          of known weight against the class bounds, pair
 *                          count, chi-square sanity)
 */
#ifndef MTGP_ORACLE_H
#define MTGP_ORACLE_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* Output formats: 32-bit words, float32 in [1,2), float32 in [0,1). */
enum { OMTGP_U32 = 0, OMTGP_F32_12 = 1, OMTGP_F32_01 = 2 };

/* The parameterized status (Sec. 3.1).  The 16-entry tables are XOR spans
 * of the four basis words: tbl[k] = XOR of basis[b] over the set bits b of k. */
typedef struct {
    uint32_t mexp;          /* Mersenne exponent: period 2^mexp - 1 when DC-found */
    uint32_t n;             /* state words N */
    uint32_t pos;           /* pick-up offset, 1 <= pos <= N-1 */
    uint32_t sh1, sh2;      /* shift amounts, 0..31 */
    uint32_t mask;          /* keeps the high 32 - r bits of word i */
    uint32_t rec_basis[4];  /* recursion table basis */
    uint32_t tmp_basis[4];  /* tempering table basis */
    uint32_t rec_tbl[16];
    uint32_t tmp_tbl[16];
} omtgp_params;

/* Fill n (if 0), mask (if 0) and both tables from the other fields.
 * Returns 0, or -1 if the fields are out of range. */
int omtgp_params_complete(omtgp_params* p);

/* Seed-generated parameter set (SplitMix64 draws, see the .c file).
 * Returns 0, or -1 if mexp is unusable. */
int omtgp_params_generate(uint32_t mexp, uint64_t seed, omtgp_params* p);

/* Seed status -> N-word initial state. */
void omtgp_init_state(const omtgp_params* p, uint32_t seed, uint32_t* state);

/* Generate `count` outputs from `state` (N words, oldest first; advanced in
 * place to the last N words of the sequence).  `out` receives count 32-bit
 * words: the integers for OMTGP_U32, the float bit patterns otherwise.
 * Returns 0, or -1 on allocation failure or a bad format. */
int omtgp_generate(const omtgp_params* p, uint32_t* state, uint64_t count,
                   int fmt, uint32_t* out);

/* Many streams: request j draws counts[j] outputs from stream ids[j] into
 * out[off_j ...], off = exclusive prefix sum of counts.  Requests for one
 * stream are applied in array order; distinct streams run on up to
 * n_threads threads.  states is n_streams x N words. Returns 0 or -1. */
int omtgp_generate_many(const omtgp_params* p, uint32_t* states,
                        uint32_t n_streams, const uint32_t* ids,
                        const uint64_t* counts, uint32_t n_req, int fmt,
                        uint32_t* out, int n_threads);

/* ------------------------------------------------------------------------
 * Statistics of the paper's two failing BigCrush tests (Sec. 4.2), restated
 * from their definitions as plain sequential loops over 32-bit outputs.
 * ------------------------------------------------------------------------ */

/* Test 35 (Knuth's gap test; r = 25, alpha = 0, beta = 1/32 in the paper).
 * Output x_j stands for u_j = ((x_j * 2^r) mod 2^32) / 2^32 (its r leading
 * bits dropped); u_j visits [0, 2^-b) when the b bits after the r dropped
 * ones are all zero.  A gap is the number of consecutive non-visits before a
 * visit, counted from the start of the sequence; a trailing run without a
 * visit is not a gap.  hist[s] (s < t) counts the gaps of length s and
 * hist[t] those of length >= t (t + 1 entries, overwritten).
 * Requires b >= 1, r + b <= 32, t >= 1.  Returns 0, or -1 on bad arguments. */
int omtgp_gap_histogram(const uint32_t* x, uint64_t n, unsigned r, unsigned b, unsigned t,
                        uint64_t* hist);

/* Test 100 (Hamming-weight independence; r = 25, s = 5, L = 1200 in the
 * paper).  The s bits after the r dropped leading bits of each output, most
 * significant first, are concatenated into one bit string, cut into blocks
 * of L bits (L a multiple of s) with Hamming weights W_0, W_1, ...  Each
 * pair of successive non-overlapping blocks (W_2i, W_2i+1) is counted in
 * table[c(W_2i) * C + c(W_2i+1)], where c(w) is the number of class bounds
 * <= w (bounds ascending; C = n_bounds + 1 classes).  Blocks of an
 * incomplete trailing pair are ignored.  table has C * C entries
 * (overwritten).  Requires 1 <= s, r + s <= 32, L % s == 0, L > 0.
 * Returns 0, or -1 on bad arguments. */
int omtgp_hamming_pairs(const uint32_t* x, uint64_t n, unsigned r, unsigned s, unsigned L,
                        const uint32_t* bounds, unsigned n_bounds, uint64_t* table);

#ifdef __cplusplus
}
#endif
#endif

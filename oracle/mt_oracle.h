/*
 * Original Mersenne Twister oracle -- TEST INFRASTRUCTURE ONLY.
 *
 * The paper's last experiment (Sec. 5.3, "Algorithm Variation") compares
 * MTGP with the original Mersenne Twister (Matsumoto and Nishimura, ACM
 * TOMACS 8(1), 1998) at the same period 2^3217 - 1, through the same two
 * statistics (tests 35 and 100).  This is a plain, sequential CPU statement
 * of that generator: the sequence is one unbounded array x_0, x_1, ... and
 * each step is the recurrence as the 1998 paper states it.  Only the
 * test-suite, the smoke check and the CPU-baseline leg of the benchmark may
 * load it; it shares no code, header or constant generator with the CUDA
 * library.
 *
 * Parity status per function:
 *   omt_params_mt19937   pinned (NumPy's MT19937 output stream, and the
 *                        10 000th output of the default seed that the C++
 *                        standard fixes for std::mt19937)
 *   omt_params_generate  pinned (bit-exact against a second SplitMix64)
 *   omt_init_state       pinned (NumPy's integer seeding of MT19937)
 *   omt_generate         pinned (MT19937 streams above; GF(2) bit-level
 *                        formulation on toy parameter sets; linearity in the
 *                        state; dropped low bits of x_0; linear complexity
 *                        of an output bit <= p)
 */
#ifndef MT_ORACLE_H
#define MT_ORACLE_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* Output formats, as for MTGP: 32-bit words, float32 in [1,2), in [0,1). */
enum { OMT_U32 = 0, OMT_F32_12 = 1, OMT_F32_01 = 2 };

/* Parameters of one original-MT generator with w = 32:
 *   x_{k+n} = x_{k+m} XOR (y >> 1) XOR (a if y is odd, else 0),
 *   y = (upper 32 - r bits of x_k) | (lower r bits of x_{k+1}),
 * output = tempering of x_{k+n}:
 *   z = x ^ (x >> u);  z ^= (z << s) & b;  z ^= (z << t) & c;  z ^= z >> l. */
typedef struct {
    uint32_t p;            /* Mersenne exponent, p = 32 n - r */
    uint32_t n;            /* state words */
    uint32_t m;            /* middle offset, 1 <= m <= n - 1 */
    uint32_t r;            /* separation point, 0 <= r <= 31 */
    uint32_t a;            /* bottom row of the twist matrix A */
    uint32_t u, s, t, l;   /* tempering shifts, 0..31 */
    uint32_t b, c;         /* tempering masks */
} omt_params;

/* Fill n (if 0) and r (if n was 0) from p: n = ceil(p / 32), r = 32 n - p.
 * Returns 0, or -1 if a field is out of range. */
int omt_params_complete(omt_params* q);

/* MT19937, the parameter set printed in the 1998 paper. */
void omt_params_mt19937(omt_params* q);

/* Seed-generated parameter set for exponent p (SplitMix64 draws, see the .c
 * file).  Returns 0, or -1 if p is unusable. */
int omt_params_generate(uint32_t p, uint64_t seed, omt_params* q);

/* Seed -> n-word initial state (the 2002 initialisation of MT19937). */
void omt_init_state(const omt_params* q, uint32_t seed, uint32_t* state);

/* Generate `count` outputs from `state` (n words, oldest first; advanced in
 * place to the last n words of the sequence).  Returns 0, or -1 on
 * allocation failure or a bad format. */
int omt_generate(const omt_params* q, uint32_t* state, uint64_t count, int fmt, uint32_t* out);

/* Many streams: request j draws counts[j] outputs from stream ids[j] into
 * out[off_j ...], off = exclusive prefix sum of counts.  Requests for one
 * stream are applied in array order; distinct streams run on up to
 * n_threads threads.  states is n_streams x n words.  Returns 0 or -1. */
int omt_generate_many(const omt_params* q, uint32_t* states, uint32_t n_streams,
                      const uint32_t* ids, const uint64_t* counts, uint32_t n_req, int fmt,
                      uint32_t* out, int n_threads);

#ifdef __cplusplus
}
#endif
#endif

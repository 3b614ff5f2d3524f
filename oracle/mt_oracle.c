/*
 * Original Mersenne Twister oracle -- TEST INFRASTRUCTURE ONLY (see
 * mt_oracle.h).
 *
 * Plain sequential C, written for reading against the 1998 definition rather
 * than for speed: the sequence is one unbounded array x_0, x_1, ..., no ring
 * buffer and no blocking.
 */
#include "mt_oracle.h"

#include <pthread.h>
#include <stdlib.h>
#include <string.h>

int omt_params_complete(omt_params* q)
{
    if (q->n == 0) {
        /* n words hold p bits plus r unused ones: n = ceil(p / 32). */
        if (q->p < 33u)
            return -1;
        q->n = (q->p + 31u) / 32u;
        q->r = 32u * q->n - q->p;
    }
    if (q->n < 2 || q->m < 1 || q->m > q->n - 1 || q->r > 31)
        return -1;
    if ((uint64_t)32 * q->n - q->r != q->p)
        return -1;
    if (q->u > 31 || q->s > 31 || q->t > 31 || q->l > 31)
        return -1;
    return 0;
}

/* MT19937 (Matsumoto and Nishimura 1998): period 2^19937 - 1. */
void omt_params_mt19937(omt_params* q)
{
    memset(q, 0, sizeof(*q));
    q->p = 19937u;
    q->n = 624u;
    q->m = 397u;
    q->r = 31u;
    q->a = 0x9908B0DFu;
    q->u = 11u;
    q->s = 7u;
    q->b = 0x9D2C5680u;
    q->t = 15u;
    q->c = 0xEFC60000u;
    q->l = 18u;
}

/* SplitMix64 (Steele, Lea and Flood, OOPSLA 2014): add the golden-ratio
 * increment, then two xor-shift-multiply rounds and a final xor-shift. */
static uint64_t splitmix64(uint64_t* s)
{
    uint64_t z = (*s += 0x9E3779B97F4A7C15ull);
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
}

/* Seed-generated set for exponent p.  The paper's MT statuses came from MT's
 * dynamic creator (Matsumoto and Nishimura 2000), which is not rebuilt here,
 * so a set is drawn instead, in this order:
 *   a = (d >> 32) | 2^31   (top bit set: otherwise A is singular),
 *   b = d >> 32,  c = d >> 32,
 * with n = ceil(p / 32), r = 32 n - p, m = floor(n / 2) and the dynamic
 * creator's tempering shifts for w = 32: u = 12, s = 7, t = 15, l = 18.
 * Such sets are not searched for a full period. */
int omt_params_generate(uint32_t p, uint64_t seed, omt_params* q)
{
    memset(q, 0, sizeof(*q));
    q->p = p;
    if (p < 33u)
        return -1;
    q->n = (p + 31u) / 32u;
    q->r = 32u * q->n - p;
    q->m = q->n / 2u;
    uint64_t s = seed;
    q->a = (uint32_t)(splitmix64(&s) >> 32) | 0x80000000u;
    q->b = (uint32_t)(splitmix64(&s) >> 32);
    q->c = (uint32_t)(splitmix64(&s) >> 32);
    q->u = 12u;
    q->s = 7u;
    q->t = 15u;
    q->l = 18u;
    return omt_params_complete(q);
}

/* The initialisation of MT19937 (2002 revision):
 *   w_0 = seed,  w_i = 1812433253 * (w_{i-1} XOR (w_{i-1} >> 30)) + i  mod 2^32. */
void omt_init_state(const omt_params* q, uint32_t seed, uint32_t* state)
{
    state[0] = seed;
    for (uint32_t i = 1; i < q->n; ++i)
        state[i] = 1812433253u * (state[i - 1] ^ (state[i - 1] >> 30)) + i;
}

/* Output conversion, as for MTGP: [1,2) takes the top 23 bits of the
 * tempered word as mantissa under exponent 0x3F800000; [0,1) is that number
 * minus one, computed in double and rounded to float (exact). */
static uint32_t convert(uint32_t o, int fmt)
{
    if (fmt == OMT_U32)
        return o;
    uint32_t bits12 = 0x3F800000u | (o >> 9);
    if (fmt == OMT_F32_12)
        return bits12;
    float f12;
    memcpy(&f12, &bits12, 4);
    float f01 = (float)((double)f12 - 1.0);
    uint32_t bits01;
    memcpy(&bits01, &f01, 4);
    return bits01;
}

int omt_generate(const omt_params* q, uint32_t* state, uint64_t count, int fmt, uint32_t* out)
{
    if (fmt != OMT_U32 && fmt != OMT_F32_12 && fmt != OMT_F32_01)
        return -1;
    const uint64_t n = q->n;
    const uint32_t upper = q->r ? 0xFFFFFFFFu << q->r : 0xFFFFFFFFu;   /* top 32 - r bits */
    const uint32_t lower = ~upper;
    uint32_t* x = (uint32_t*)malloc((size_t)(n + count) * sizeof(uint32_t));
    if (!x)
        return -1;
    memcpy(x, state, (size_t)n * sizeof(uint32_t));   /* x_0 .. x_{n-1} */

    for (uint64_t k = 0; k < count; ++k) {
        /* Twist: the upper part of x_k joined with the lower part of
         * x_{k+1}, multiplied by A (a right shift, plus the row a when the
         * bit shifted out is one), added to x_{k+m}. */
        uint32_t y = (x[k] & upper) | (x[k + 1] & lower);
        uint32_t ya = (y >> 1) ^ ((y & 1u) ? q->a : 0u);
        x[k + n] = x[k + q->m] ^ ya;

        /* Tempering of the new word. */
        uint32_t z = x[k + n];
        z ^= z >> q->u;
        z ^= (z << q->s) & q->b;
        z ^= (z << q->t) & q->c;
        z ^= z >> q->l;

        out[k] = convert(z, fmt);   /* output k comes from x_{k+n} */
    }
    memcpy(state, x + count, (size_t)n * sizeof(uint32_t));   /* last n words */
    free(x);
    return 0;
}

typedef struct {
    const omt_params* q;
    uint32_t* states;
    const uint32_t* ids;
    const uint64_t* counts;
    const uint64_t* offs;
    uint32_t n_req;
    int fmt;
    uint32_t* out;
    int tid, nthreads;
    int rc;
} mt_job;

static void* mt_worker(void* arg)
{
    mt_job* j = (mt_job*)arg;
    j->rc = 0;
    /* Thread t owns the streams s with s % nthreads == t and walks the
     * requests in array order, so each stream sees its requests in order. */
    for (uint32_t r = 0; r < j->n_req; ++r) {
        uint32_t s = j->ids[r];
        if ((int)(s % (uint32_t)j->nthreads) != j->tid)
            continue;
        if (omt_generate(j->q, j->states + (uint64_t)s * j->q->n, j->counts[r], j->fmt,
                         j->out + j->offs[r]) != 0)
            j->rc = -1;
    }
    return NULL;
}

int omt_generate_many(const omt_params* q, uint32_t* states, uint32_t n_streams,
                      const uint32_t* ids, const uint64_t* counts, uint32_t n_req, int fmt,
                      uint32_t* out, int n_threads)
{
    for (uint32_t r = 0; r < n_req; ++r)
        if (ids[r] >= n_streams)
            return -1;
    uint64_t* offs = (uint64_t*)malloc((size_t)(n_req + 1) * sizeof(uint64_t));
    if (!offs)
        return -1;
    offs[0] = 0;
    for (uint32_t r = 0; r < n_req; ++r)
        offs[r + 1] = offs[r] + counts[r];
    if (n_threads < 1)
        n_threads = 1;
    mt_job* jobs = (mt_job*)calloc((size_t)n_threads, sizeof(mt_job));
    pthread_t* th = (pthread_t*)calloc((size_t)n_threads, sizeof(pthread_t));
    if (!jobs || !th) {
        free(offs); free(jobs); free(th);
        return -1;
    }
    int rc = 0;
    for (int t = 0; t < n_threads; ++t) {
        mt_job j = {q, states, ids, counts, offs, n_req, fmt, out, t, n_threads, 0};
        jobs[t] = j;
        if (n_threads == 1) {
            mt_worker(&jobs[t]);
        } else if (pthread_create(&th[t], NULL, mt_worker, &jobs[t]) != 0) {
            rc = -1;
            jobs[t].nthreads = 0;   /* not started */
        }
    }
    if (n_threads > 1)
        for (int t = 0; t < n_threads; ++t)
            if (jobs[t].nthreads)
                pthread_join(th[t], NULL);
    for (int t = 0; t < n_threads; ++t)
        if (jobs[t].rc)
            rc = -1;
    free(offs); free(jobs); free(th);
    return rc;
}

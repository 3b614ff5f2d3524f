/*
 * MTGP32 oracle -- TEST INFRASTRUCTURE ONLY (see mtgp_oracle.h).
 *
 * Plain sequential C, written for reading against the paper rather than for
 * speed.  The sequence is kept as one unbounded array x_0, x_1, ... exactly as
 * the recurrence is stated; no ring buffer, no blocking, no tables beyond the
 * two 16-entry tables the parameterized status carries.
 */
#include "mtgp_oracle.h"

#include <pthread.h>
#include <stdlib.h>
#include <string.h>

/* ------------------------------------------------------------------------ */
/* Parameterized status (Sec. 3.1: "parameterized status", a per-generator
 * signature; the "fast" status of Sec. 3.1 adds precomputed tables).       */
/* ------------------------------------------------------------------------ */

/* Table spanned by four basis words: entry k is the XOR of basis[b] over the
 * set bits b of k.  Every table built this way is GF(2)-linear in k. */
static void span_table(const uint32_t basis[4], uint32_t tbl[16])
{
    for (uint32_t k = 0; k < 16; ++k) {
        uint32_t v = 0;
        for (uint32_t b = 0; b < 4; ++b)
            if (k & (1u << b))
                v ^= basis[b];
        tbl[k] = v;
    }
}

int omtgp_params_complete(omtgp_params* p)
{
    if (p->n == 0) {
        /* State size: the smallest N with 32N > Mexp, i.e. N = floor(Mexp/32)+1,
         * so that r = 32N - Mexp bits of the oldest word are dropped. */
        p->n = p->mexp / 32u + 1u;
    }
    if (p->mask == 0) {
        int64_t r = (int64_t)32 * p->n - (int64_t)p->mexp;
        if (r < 1 || r > 31)
            return -1;
        p->mask = 0xFFFFFFFFu << (uint32_t)r;
    }
    if (p->n < 2 || p->pos < 1 || p->pos > p->n - 1 || p->sh1 > 31 || p->sh2 > 31)
        return -1;
    span_table(p->rec_basis, p->rec_tbl);
    span_table(p->tmp_basis, p->tmp_tbl);
    return 0;
}

/* SplitMix64 (Steele, Lea and Flood, OOPSLA 2014): add the golden-ratio
 * increment, then two xor-shift-multiply rounds and a final xor-shift. */
static uint64_t splitmix64_next(uint64_t* s)
{
    uint64_t z = (*s += 0x9E3779B97F4A7C15ull);
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
}

/* Seed-generated parameter set.  The paper prints no parameter set (its DC
 * outputs are announced for download, Sec. 6), so sets are drawn from a
 * SplitMix64 stream in this fixed order:
 *   sh1 = 1 + d % 31,  sh2 = 1 + d % 31,
 *   pos = 2 + d % (N - Wmin - 1)   (pos in [2, N - Wmin]),
 *   rec_basis[0..3] = d >> 32,  tmp_basis[0..3] = d >> 32,
 * with Wmin = min(256, largest power of two <= N - 2), so that every set
 * admits a block-parallel step of at least Wmin words.  For N = 2 the pos
 * draw is still made and pos = 1.  Such sets are not searched for a full
 * period; the arithmetic they drive is the same. */
int omtgp_params_generate(uint32_t mexp, uint64_t seed, omtgp_params* p)
{
    memset(p, 0, sizeof(*p));
    p->mexp = mexp;
    p->n = mexp / 32u + 1u;
    uint64_t s = seed;
    p->sh1 = 1u + (uint32_t)(splitmix64_next(&s) % 31u);
    p->sh2 = 1u + (uint32_t)(splitmix64_next(&s) % 31u);
    uint64_t dpos = splitmix64_next(&s);
    if (p->n >= 3) {
        uint32_t wmin = 1;
        while (wmin * 2u <= p->n - 2u && wmin < 256u)
            wmin *= 2u;
        uint32_t hi = p->n - wmin;      /* >= 2 */
        p->pos = 2u + (uint32_t)(dpos % (uint64_t)(hi - 1u));
    } else {
        p->pos = 1u;
    }
    for (int b = 0; b < 4; ++b)
        p->rec_basis[b] = (uint32_t)(splitmix64_next(&s) >> 32);
    for (int b = 0; b < 4; ++b)
        p->tmp_basis[b] = (uint32_t)(splitmix64_next(&s) >> 32);
    return omtgp_params_complete(p);
}

/* ------------------------------------------------------------------------ */
/* Seed status (Sec. 3.1: "the common seed given by the user"; Sec. 5.1 keeps
 * it at 0 for the 10 000-parameter study and varies it in "Random Spacing").
 * The paper gives no seeding routine; the MT-family one is used:
 *   w_0 = seed,  w_i = 1812433253 * (w_{i-1} XOR (w_{i-1} >> 30)) + i  mod 2^32. */
/* ------------------------------------------------------------------------ */
void omtgp_init_state(const omtgp_params* p, uint32_t seed, uint32_t* state)
{
    state[0] = seed;
    for (uint32_t i = 1; i < p->n; ++i)
        state[i] = 1812433253u * (state[i - 1] ^ (state[i - 1] >> 30)) + i;
}

/* ------------------------------------------------------------------------ */
/* Generation (the per-block generator of Sec. 2 and its CPU twin, Sec. 3.2). */
/* ------------------------------------------------------------------------ */

/* Output conversion.  [1,2): exponent 0x3F800000 with the top 23 bits of the
 * tempered word as mantissa.  [0,1): that number minus one, computed in double
 * and rounded to float (exact: the difference has at most 23 significant
 * bits). */
static uint32_t convert(uint32_t o, int fmt)
{
    if (fmt == OMTGP_U32)
        return o;
    uint32_t bits12 = 0x3F800000u | (o >> 9);
    if (fmt == OMTGP_F32_12)
        return bits12;
    float f12;
    memcpy(&f12, &bits12, 4);
    float f01 = (float)((double)f12 - 1.0);
    uint32_t bits01;
    memcpy(&bits01, &f01, 4);
    return bits01;
}

int omtgp_generate(const omtgp_params* p, uint32_t* state, uint64_t count,
                   int fmt, uint32_t* out)
{
    if (fmt != OMTGP_U32 && fmt != OMTGP_F32_12 && fmt != OMTGP_F32_01)
        return -1;
    const uint64_t n = p->n;
    uint32_t* x = (uint32_t*)malloc((size_t)(n + count) * sizeof(uint32_t));
    if (!x)
        return -1;
    memcpy(x, state, (size_t)n * sizeof(uint32_t));   /* x_0 .. x_{N-1} */

    for (uint64_t i = 0; i < count; ++i) {
        /* Recurrence over words i, i+1 and i+pos: the masked oldest word is
         * combined with its successor, shifted into itself by sh1, the word
         * at i+pos enters shifted down by sh2, and the low four bits select
         * the recursion-table entry. */
        uint32_t y = (x[i] & p->mask) ^ x[i + 1];
        y ^= y << p->sh1;
        y ^= x[i + p->pos] >> p->sh2;
        x[i + n] = y ^ p->rec_tbl[y & 0xFu];

        /* Tempering: word i+pos-1 folded (>>16, then >>8), low four bits
         * select the tempering-table entry, XORed into the new word. */
        uint32_t t = x[i + p->pos - 1];
        t ^= t >> 16;
        t ^= t >> 8;
        uint32_t o = x[i + n] ^ p->tmp_tbl[t & 0xFu];

        out[i] = convert(o, fmt);   /* output i comes from x_{i+N} */
    }
    memcpy(state, x + count, (size_t)n * sizeof(uint32_t));   /* last N words */
    free(x);
    return 0;
}

/* ------------------------------------------------------------------------ */
/* Many independent statuses (Sec. 3.2: one status per block of threads).   */
/* ------------------------------------------------------------------------ */

typedef struct {
    const omtgp_params* p;
    uint32_t* states;
    uint32_t n_streams;
    const uint32_t* ids;
    const uint64_t* counts;
    const uint64_t* offs;
    uint32_t n_req;
    int fmt;
    uint32_t* out;
    int tid, nthreads;
    int rc;
} many_job;

static void* many_worker(void* arg)
{
    many_job* j = (many_job*)arg;
    j->rc = 0;
    /* Thread t owns the streams s with s % nthreads == t and walks the
     * requests in array order, so each stream sees its requests in order. */
    for (uint32_t r = 0; r < j->n_req; ++r) {
        uint32_t s = j->ids[r];
        if ((int)(s % (uint32_t)j->nthreads) != j->tid)
            continue;
        if (omtgp_generate(j->p, j->states + (uint64_t)s * j->p->n, j->counts[r],
                           j->fmt, j->out + j->offs[r]) != 0)
            j->rc = -1;
    }
    return NULL;
}

int omtgp_generate_many(const omtgp_params* p, uint32_t* states,
                        uint32_t n_streams, const uint32_t* ids,
                        const uint64_t* counts, uint32_t n_req, int fmt,
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
    many_job* jobs = (many_job*)calloc((size_t)n_threads, sizeof(many_job));
    pthread_t* th = (pthread_t*)calloc((size_t)n_threads, sizeof(pthread_t));
    if (!jobs || !th) {
        free(offs); free(jobs); free(th);
        return -1;
    }
    int rc = 0;
    for (int t = 0; t < n_threads; ++t) {
        many_job j = {p, states, n_streams, ids, counts, offs, n_req, fmt, out, t, n_threads, 0};
        jobs[t] = j;
        if (n_threads == 1) {
            many_worker(&jobs[t]);
        } else if (pthread_create(&th[t], NULL, many_worker, &jobs[t]) != 0) {
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


/* ========================================================================
 * Test 35: gap-length histogram (Sec. 4.2).
 * ======================================================================== */
static int in_field_is_zero(uint32_t x, unsigned r, unsigned width)
{
    /* the `width` bits that follow the r dropped leading bits */
    uint64_t v = ((uint64_t)x << r) & 0xFFFFFFFFull;   /* drop r leading bits */
    return (v >> (32 - width)) == 0;
}

int omtgp_gap_histogram(const uint32_t* x, uint64_t n, unsigned r, unsigned b, unsigned t,
                        uint64_t* hist)
{
    uint64_t j, run = 0;
    unsigned s;
    if (!hist || (n && !x) || b < 1 || r + b > 32 || t < 1)
        return -1;
    for (s = 0; s <= t; ++s)
        hist[s] = 0;
    for (j = 0; j < n; ++j) {
        if (in_field_is_zero(x[j], r, b)) {      /* a visit ends the current gap */
            hist[run < t ? run : t] += 1;
            run = 0;
        } else {
            run += 1;
        }
    }
    return 0;
}

/* ========================================================================
 * Test 100: table of the weight classes of successive block pairs (Sec. 4.2).
 * ======================================================================== */
int omtgp_hamming_pairs(const uint32_t* x, uint64_t n, unsigned r, unsigned s, unsigned L,
                        const uint32_t* bounds, unsigned n_bounds, uint64_t* table)
{
    const unsigned C = n_bounds + 1;
    uint64_t j, per_block, n_blocks, k;
    unsigned i, bit, cls[2] = {0, 0};
    if (!table || (n && !x) || s < 1 || r + s > 32 || L == 0 || L % s != 0 ||
        (n_bounds && !bounds))
        return -1;
    for (i = 0; i < C * C; ++i)
        table[i] = 0;
    per_block = L / s;
    n_blocks = n / per_block;
    n_blocks -= n_blocks % 2;                 /* complete pairs only */
    for (k = 0; k < n_blocks; ++k) {
        unsigned w = 0, c = 0;
        for (j = k * per_block; j < (k + 1) * per_block; ++j) {
            uint64_t v = ((uint64_t)x[j] << r) & 0xFFFFFFFFull;
            uint32_t field = (uint32_t)(v >> (32 - s));   /* the s bits, MSB first */
            for (bit = 0; bit < s; ++bit)
                w += (field >> (s - 1 - bit)) & 1u;
        }
        for (i = 0; i < n_bounds; ++i)
            if (bounds[i] <= w)
                ++c;
        cls[k % 2] = c;
        if (k % 2 == 1)
            table[cls[0] * C + cls[1]] += 1;
    }
    return 0;
}

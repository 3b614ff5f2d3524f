// Jump-ahead: advance streams by J numbers without producing them.
//
// The paper raises distributing streams across a machine (Sec. 1); for
// an F2-linear generator the exact way is a polynomial jump.  The state of a
// stream is the window w = (x_c .. x_{c+N-1}); one step F maps it to
// (x_{c+1} .. x_{c+N}).  F is linear over GF(2).  Its kernel K holds the
// windows that are zero except in the r = 32N - Mexp low bits of the oldest
// word (the recursion masks those bits away), and F(K) = 0.  Let mu be a
// polynomial with mu(F) w in K for every w (the minimal polynomial of the
// transition on the quotient by K, degree <= Mexp).  Then F mu(F) = 0, and
// writing t^(J-1) = q mu + g gives
//
//     F^J = q(F) mu(F) F + g(F) F = F g(F),
//
// so the state after J steps is one ordinary step applied to
// g(F) w = XOR over the set bits k of g of the window (x_k .. x_{k+N-1}) of
// the sequence that starts at w.
//
// Host side: mu comes from Berlekamp-Massey on bit sequences of the
// recursion (run on the host), combined by LCM until it annihilates random
// states; g = t^(J-1) mod mu by square-and-multiply.  Both are cached per
// parameter set.  Device side: one CTA per stream expands the sequence
// x_0 .. x_{D+N-2} (D = deg g + 1) in shared memory, every warp XORs the
// windows of its share of g's set bits into the N-word accumulator, and the
// last step is applied to the result.
#include <algorithm>
#include <map>
#include <mutex>
#include <random>
#include <vector>

#include "../../include/mtgp_mt.h"
#include "mtgp_runtime.h"

using namespace mtgp;

namespace {

// ---------------------------------------------------------------------------
// Polynomials over GF(2) as bit vectors (bit i = coefficient of t^i)
// ---------------------------------------------------------------------------
using Poly = std::vector<uint64_t>;

int degree(const Poly& a)
{
    for (size_t w = a.size(); w-- > 0;)
        if (a[w])
            return (int)(w * 64 + 63 - __builtin_clzll(a[w]));
    return -1;
}

void trim(Poly& a)
{
    while (!a.empty() && a.back() == 0)
        a.pop_back();
}

bool bit(const Poly& a, size_t i) { return i / 64 < a.size() && ((a[i / 64] >> (i % 64)) & 1u); }

// a ^= b << sh
void xor_shifted(Poly& a, const Poly& b, size_t sh)
{
    const size_t ws = sh / 64, bs = sh % 64;
    if (a.size() < b.size() + ws + 1)
        a.resize(b.size() + ws + 1, 0);
    for (size_t w = 0; w < b.size(); ++w) {
        if (!b[w])
            continue;
        a[w + ws] ^= b[w] << bs;
        if (bs)
            a[w + ws + 1] ^= b[w] >> (64 - bs);
    }
}

// remainder of a modulo m (deg m >= 0)
Poly mod(Poly a, const Poly& m)
{
    const int dm = degree(m);
    for (int d = degree(a); d >= dm; d = degree(a))
        xor_shifted(a, m, (size_t)(d - dm));
    trim(a);
    return a;
}

// quotient and remainder
void divmod(Poly a, const Poly& m, Poly& q, Poly& r)
{
    const int dm = degree(m);
    q.assign(1, 0);
    for (int d = degree(a); d >= dm; d = degree(a)) {
        const size_t sh = (size_t)(d - dm);
        if (q.size() <= sh / 64)
            q.resize(sh / 64 + 1, 0);
        q[sh / 64] ^= 1ull << (sh % 64);
        xor_shifted(a, m, sh);
    }
    trim(a);
    trim(q);
    r = a;
}

Poly mul(const Poly& a, const Poly& b)
{
    Poly c;
    const int db = degree(b);
    for (int i = 0; i <= db; ++i)
        if (bit(b, (size_t)i))
            xor_shifted(c, a, (size_t)i);
    trim(c);
    return c;
}

Poly gcd(Poly a, Poly b)
{
    trim(a);
    trim(b);
    while (degree(b) >= 0) {
        Poly r = mod(a, b);
        a = b;
        b = r;
    }
    return a;
}

// a^2 mod m: squaring spreads the bits (no cross terms over GF(2))
Poly sqr_mod(const Poly& a, const Poly& m)
{
    Poly s(a.size() * 2 + 1, 0);
    for (size_t w = 0; w < a.size(); ++w)
        for (int i = 0; i < 64; ++i)
            if ((a[w] >> i) & 1u) {
                const size_t j = 2 * (w * 64 + (size_t)i);
                s[j / 64] |= 1ull << (j % 64);
            }
    return mod(s, m);
}

// t^e mod m (left-to-right square-and-multiply; multiplying by t is a shift)
Poly pow_t_mod(uint64_t e, const Poly& m)
{
    Poly r(1, 1ull);   // t^0, reduced: zero only modulo a constant
    if (degree(m) == 0)
        r.clear();
    for (int b = 63; b >= 0; --b) {
        r = sqr_mod(r, m);
        if ((e >> b) & 1u) {
            Poly s;
            xor_shifted(s, r, 1);
            r = mod(s, m);
        }
    }
    return r;
}

// ---------------------------------------------------------------------------
// The recursion on the host (words only, no tempering): seq[0..N) = state,
// then count new words.
// ---------------------------------------------------------------------------
struct SetP {
    uint32_t n, pos, sh1, sh2, mask;
    uint32_t rec[16];
};

void host_sequence(const SetP& p, const uint32_t* state, size_t count, std::vector<uint32_t>& seq)
{
    seq.assign(state, state + p.n);
    seq.resize(p.n + count);
    for (size_t i = 0; i < count; ++i) {
        uint32_t y = (seq[i] & p.mask) ^ seq[i + 1];
        y ^= y << p.sh1;
        y ^= seq[i + p.pos] >> p.sh2;
        seq[i + p.n] = y ^ p.rec[y & 15u];
    }
}

// Berlekamp-Massey over GF(2): the minimal polynomial of the bit sequence
// s (n bits), as mu(t) = t^L C(1/t) for the connection polynomial C.
Poly berlekamp_massey(const std::vector<uint8_t>& s)
{
    const size_t n = s.size();
    // reversed sequence, bit-packed: R_k = s_{n-1-k}
    Poly R((n + 127) / 64, 0);
    for (size_t k = 0; k < n; ++k)
        if (s[n - 1 - k])
            R[k / 64] |= 1ull << (k % 64);
    auto window = [&](size_t off) -> uint64_t {   // bits R[off .. off+63]
        const size_t w = off / 64, b = off % 64;
        uint64_t v = R[w] >> b;
        if (b && w + 1 < R.size())
            v |= R[w + 1] << (64 - b);
        return v;
    };
    Poly C(1, 1ull), B(1, 1ull);
    size_t L = 0;
    long m = -1;
    for (size_t i = 0; i < n; ++i) {
        // discrepancy: sum_{j=0..L} c_j s_{i-j}, s_{i-j} = R_{n-1-i+j}
        uint64_t acc = 0;
        const size_t off = n - 1 - i;
        for (size_t w = 0; w * 64 <= L && w < C.size(); ++w) {
            uint64_t cw = C[w];
            if (w * 64 + 64 > L + 1)
                cw &= (L + 1 - w * 64) >= 64 ? ~0ull : ((1ull << (L + 1 - w * 64)) - 1);
            acc ^= cw & window(off + w * 64);
        }
        if (__builtin_parityll(acc)) {
            Poly T = C;
            xor_shifted(C, B, (size_t)((long)i - m));
            if (2 * L <= i) {
                L = i + 1 - L;
                m = (long)i;
                B = T;
            }
        }
    }
    Poly mu((L + 64) / 64, 0);
    for (size_t k = 0; k <= L; ++k)
        if (bit(C, L - k))
            mu[k / 64] |= 1ull << (k % 64);
    trim(mu);
    return mu;
}

// The original Mersenne Twister's recursion on the host (words only):
// x_{k+n} = x_{k+m} ^ (y >> 1) ^ (y odd ? a : 0), y = (x_k & upper) | (x_{k+1} & ~upper).
struct MtRec {
    uint32_t n, m, upper, a;
};

void host_sequence(const MtRec& p, const uint32_t* state, size_t count, std::vector<uint32_t>& seq)
{
    seq.assign(state, state + p.n);
    seq.resize(p.n + count);
    for (size_t k = 0; k < count; ++k) {
        const uint32_t y = (seq[k] & p.upper) | (seq[k + 1] & ~p.upper);
        seq[k + p.n] = seq[k + p.m] ^ (y >> 1) ^ ((y & 1u) ? p.a : 0u);
    }
}

// Window size and the used bits of the window's oldest word.
uint32_t window_words(const SetP& p) { return p.n; }
uint32_t oldest_mask(const SetP& p) { return p.mask; }
uint64_t rng_seed(const SetP& p)
{
    return 0x9E3779B97F4A7C15ull ^ ((uint64_t)p.pos << 32) ^ p.sh1 ^ ((uint64_t)p.rec[1] << 7);
}
uint32_t window_words(const MtRec& p) { return p.n; }
uint32_t oldest_mask(const MtRec& p) { return p.upper; }
uint64_t rng_seed(const MtRec& p) { return 0xC2B2AE3D27D4EB4Full ^ ((uint64_t)p.m << 32) ^ p.a; }

// True if F mu(F) w = 0 for the sequence of `state`: for j = 1..N the XOR of
// x_{k+j} over the set bits k of mu is zero.
template <class Rec>
bool annihilates(const Rec& p, const Poly& mu, const uint32_t* state)
{
    const int d = degree(mu);
    std::vector<uint32_t> seq;
    const uint32_t N = window_words(p);
    host_sequence(p, state, (size_t)d + N + 1, seq);
    for (uint32_t j = 1; j <= N; ++j) {
        uint32_t acc = 0;
        for (int k = 0; k <= d; ++k)
            if (bit(mu, (size_t)k))
                acc ^= seq[(size_t)k + j];
        if (acc)
            return false;
    }
    return true;
}

// mu for a parameter set (of MTGP or of the original MT): LCM of the minimal
// polynomials of bit sequences (random states, random linear functionals of
// the words) until it annihilates fresh random states.
template <class Rec>
Poly transition_polynomial(const Rec& p, uint32_t mexp)
{
    std::mt19937_64 rng(rng_seed(p));
    const uint32_t N = window_words(p);
    auto random_state = [&](std::vector<uint32_t>& st) {
        st.resize(N);
        for (auto& v : st)
            v = (uint32_t)rng();
    };
    Poly mu;
    std::vector<uint32_t> st, seq;
    for (int round = 0; round < 64; ++round) {
        random_state(st);
        const size_t len = 2 * (size_t)mexp + 64;
        host_sequence(p, st.data(), len, seq);   // N + len words
        // A random linear functional of the whole state F^i w (every word,
        // the oldest one masked): states that one step maps to zero can live
        // in the oldest word or in the low bits of the next one, so a
        // functional of a single word would not see every part of the
        // transition.
        std::vector<uint32_t> f(N);
        for (auto& v : f)
            v = (uint32_t)rng();
        f[0] &= oldest_mask(p);
        std::vector<uint8_t> bits(len);
        for (size_t i = 0; i < len; ++i) {
            uint32_t acc = 0;
            for (uint32_t j = 0; j < N; ++j)
                acc ^= seq[i + j] & f[j];
            bits[i] = (uint8_t)__builtin_parity(acc);
        }
        Poly m1 = berlekamp_massey(bits);
        if (degree(m1) < 0)
            continue;
        if (mu.empty()) {
            mu = m1;
        } else {
            Poly q, r;
            divmod(mu, gcd(mu, m1), q, r);
            mu = mul(q, m1);
        }
        if (degree(mu) > (int)mexp)
            break;   // cannot happen for a linear recursion of this state size
        // A polynomial that does not annihilate the transition still passes
        // the check on a random state with probability at most 1/2 (the
        // states it fails on are the complement of a proper subspace), so 20
        // passing states leave a false acceptance below 1e-6.
        bool all = true;
        for (int t = 0; t < 20 && all; ++t) {
            random_state(st);
            all = annihilates(p, mu, st.data());
        }
        if (all)
            return mu;
    }
    return Poly();
}

SetP set_of(const KParams& k, const KSet* ks)
{
    SetP p;
    p.n = k.n;
    p.mask = k.mask;
    p.pos = ks ? ks->pos : k.pos;
    p.sh1 = ks ? ks->sh1 : k.sh1;
    p.sh2 = ks ? ks->sh2 : k.sh2;
    for (int i = 0; i < 16; ++i)
        p.rec[i] = ks ? ks->rec[i] : k.rec[i];
    return p;
}

// Caches keyed by the parameter set's fields (and the jump length).
std::mutex g_cache_mutex;
std::map<std::vector<uint32_t>, Poly> g_mu_cache;
std::map<std::pair<std::vector<uint32_t>, uint64_t>, Poly> g_jump_cache;

std::vector<uint32_t> key_of(const SetP& p)
{
    std::vector<uint32_t> k = {p.n, p.pos, p.sh1, p.sh2, p.mask};
    k.insert(k.end(), p.rec, p.rec + 16);
    return k;
}

std::vector<uint32_t> key_of(const MtRec& p)
{
    return {0xFFFFFFFFu, p.n, p.m, p.upper, p.a};   // first word: never an MTGP state size
}

template <class Rec>
const Poly* cached_mu(const Rec& p, uint32_t mexp)
{
    const auto key = key_of(p);
    {
        std::lock_guard<std::mutex> g(g_cache_mutex);
        auto it = g_mu_cache.find(key);
        if (it != g_mu_cache.end())
            return it->second.empty() ? nullptr : &it->second;
    }
    Poly mu = transition_polynomial(p, mexp);
    std::lock_guard<std::mutex> g(g_cache_mutex);
    auto& slot = g_mu_cache.emplace(key, std::move(mu)).first->second;   // first writer wins
    return slot.empty() ? nullptr : &slot;
}

// ---------------------------------------------------------------------------
// Device: one CTA per (stream, jump).  Shared memory: the sequence S[0 .. D+N-1)
// and the N-word accumulator.  Every wait is a __syncthreads on uniform
// control flow; no spin waits.
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(256) mtgp_jump_kernel(const KParams P, uint32_t* __restrict__ states,
                                                       const JumpItem* __restrict__ items,
                                                       const uint32_t* __restrict__ polys,
                                                       uint32_t poly_words,
                                                       const KSet* __restrict__ sets)
{
    extern __shared__ __align__(16) uint32_t sm[];
    const JumpItem it = items[blockIdx.x];
    const uint32_t N = P.n, D = it.deg + 1u;
    uint32_t pos = P.pos, sh1 = P.sh1, sh2 = P.sh2;
    const uint32_t* rec = P.rec;
    if (sets) {
        const KSet& ks = sets[it.set];
        pos = ks.pos;
        sh1 = ks.sh1;
        sh2 = ks.sh2;
        rec = ks.rec;
    }
    uint32_t* S = sm;                 // D + N - 1 words
    uint32_t* acc = sm + D + N - 1u;  // N words
    __shared__ uint32_t R[16];
    if (threadIdx.x < 16)
        R[threadIdx.x] = rec[threadIdx.x];
    uint32_t* g = states + (size_t)it.stream * P.np;
    for (uint32_t j = threadIdx.x; j < N; j += blockDim.x) {
        S[j] = g[j];
        acc[j] = 0u;
    }
    __syncthreads();
    // expand: S[i + N] for i = 0 .. D-2, Wc words per step, one per thread
    // (each reads only words produced before the step: Wc <= N - pos)
    const uint32_t Wc = min(blockDim.x, N - pos);
    for (uint32_t i0 = 0; i0 + 1u < D; i0 += Wc) {
        const uint32_t i = i0 + threadIdx.x;
        uint32_t v = 0;
        const bool act = threadIdx.x < Wc && i + 1u < D;
        if (act) {
            uint32_t y = (S[i] & P.mask) ^ S[i + 1u];
            y ^= y << sh1;
            y ^= S[i + pos] >> sh2;
            v = y ^ R[y & 15u];
        }
        __syncthreads();
        if (act)
            S[i + N] = v;
        __syncthreads();
    }
    // accumulate: warp w takes the set bits k of g with k / 32 = w (mod
    // warps); acc[j] ^= S[k + j] for every such k.  The N words are covered
    // in nch passes of uc <= 12 units of 32 words (one word per lane per
    // unit), so that a pass wastes at most one unit's loads.
    const uint32_t lane = threadIdx.x & 31u, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
    const uint32_t* gp = polys + (size_t)it.poly * poly_words;
    constexpr uint32_t kUnits = 12;
    const uint32_t U = (N + 31u) / 32u;
    const uint32_t nch = (U + kUnits - 1u) / kUnits;
    const uint32_t uc = (U + nch - 1u) / nch;
    for (uint32_t c = 0; c < nch; ++c) {
        const uint32_t j0 = 32u * uc * c;
        uint32_t a[kUnits];
#pragma unroll
        for (uint32_t q = 0; q < kUnits; ++q)
            a[q] = 0u;
        for (uint32_t w = warp; w * 32u < D; w += nw) {
            uint32_t bits = gp[w];
            while (bits) {
                const uint32_t k = w * 32u + (uint32_t)(__ffs(bits) - 1);
                bits &= bits - 1u;
#pragma unroll
                for (uint32_t q = 0; q < kUnits; ++q) {
                    const uint32_t j = j0 + 32u * q + lane;
                    if (q < uc && j < N)
                        a[q] ^= S[k + j];
                }
            }
        }
#pragma unroll
        for (uint32_t q = 0; q < kUnits; ++q) {
            const uint32_t j = j0 + 32u * q + lane;
            if (q < uc && j < N && a[q])
                atomicXor(&acc[j], a[q]);
        }
    }
    __syncthreads();
    // one ordinary step on the accumulated window: the state after J steps is
    // (acc[1] .. acc[N-1], new word), oldest first
    for (uint32_t j = threadIdx.x; j + 1u < N; j += blockDim.x)
        g[j] = acc[j + 1u];
    if (threadIdx.x == 0) {
        uint32_t y = (acc[0] & P.mask) ^ acc[1];
        y ^= y << sh1;
        y ^= acc[pos] >> sh2;
        g[N - 1u] = y ^ R[y & 15u];
    }
}

// ---------------------------------------------------------------------------
// Period check: Rabin's irreducibility test of mu, run as a chain of
// squarings a <- a^2 mod mu on the device.  Over GF(2) a^2 = sum a_i t^(2i):
// the terms with 2i < D need no reduction (spread bits), the others are the
// precomputed rows t^(2i) mod mu (i >= h = ceil(D/2)).  Output word w of one
// squaring is therefore the spread of a's bits 32w .. 32w+31 XOR the word w of
// every row whose bit of a is set; blocks split the words (x) and the rows
// (y) and combine with 64-bit atomicXor into a zeroed output.
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(256) mtgp_frobenius_kernel(const unsigned long long* __restrict__ a,
                                                            unsigned long long* __restrict__ out,
                                                            const unsigned long long* __restrict__ rows,
                                                            uint32_t D, uint32_t W, uint32_t h,
                                                            uint32_t rows_per_slice)
{
    const uint32_t w = blockIdx.x * blockDim.x + threadIdx.x;
    const uint32_t i0 = h + blockIdx.y * rows_per_slice;
    const uint32_t i1 = min(D, i0 + rows_per_slice);
    if (w >= W)
        return;
    unsigned long long acc = 0;
    if (blockIdx.y == 0) {
        // spread: bit i of a (i < h) -> bit 2i; output word w takes a's bits 32w .. 32w+31
        const uint32_t src = 32u * w;
        if (src < h) {
            const unsigned long long word = a[src / 64u];
            uint32_t half = (uint32_t)(word >> (src % 64u));
            if (h - src < 32u)
                half &= (1u << (h - src)) - 1u;   // only bits i < h
            unsigned long long x = half;
            x = (x | (x << 16)) & 0x0000FFFF0000FFFFull;
            x = (x | (x << 8)) & 0x00FF00FF00FF00FFull;
            x = (x | (x << 4)) & 0x0F0F0F0F0F0F0F0Full;
            x = (x | (x << 2)) & 0x3333333333333333ull;
            x = (x | (x << 1)) & 0x5555555555555555ull;
            acc = x;
        }
    }
    for (uint32_t i = i0; i < i1; ++i)
        if ((a[i / 64u] >> (i % 64u)) & 1ull)
            acc ^= rows[(size_t)(i - h) * W + w];
    if (acc)
        atomicXor(out + w, acc);
}

#define J_TRY(call, what)                 \
    do {                                  \
        cudaError_t e_ = (call);          \
        if (e_ != cudaSuccess)            \
            return fail_cuda(e_, what);   \
    } while (0)

}  // namespace

extern "C" mtgp_status mtgp_params_minpoly(mtgp_params_t params, uint64_t* words, uint32_t cap_words,
                                           int32_t* degree_out)
{
    try {
        if (!params || !degree_out)
            return fail(MTGP_EINVAL, "null argument");
        const SetP p = set_of(params->k, nullptr);
        const Poly* mu = cached_mu(p, params->d.mexp);
        if (!mu)
            return fail(MTGP_EINVAL, "no annihilating polynomial found for this parameter set");
        const int d = degree(*mu);
        *degree_out = d;
        const uint32_t need = (uint32_t)(d / 64 + 1);
        if (words) {
            if (cap_words < need)
                return fail(MTGP_EINVAL, "need %u words", need);
            std::fill(words, words + cap_words, 0ull);
            std::copy(mu->begin(), mu->end(), words);
        }
        return ok();
    } catch (const std::bad_alloc&) {
        return fail(MTGP_ENOMEM, "host allocation failed");
    }
}

// Rabin's irreducibility test of mu for exponent n on the device (sets
// *irreducible; 0 also when deg mu != n or mu cannot be primitive).
static mtgp_status rabin_irreducible(const Poly& mu, uint32_t n, void* cuda_stream, int32_t* irreducible)
{
    try {
        *irreducible = 0;
        const int D = degree(mu);
        // a full-period transition needs deg mu = Mexp, mu(0) = 1, mu(1) = 1
        int terms = 0;
        for (uint64_t wd : mu)
            terms += __builtin_popcountll(wd);
        if (D != (int)n || !bit(mu, 0) || terms % 2 == 0)
            return ok();
        // prime divisors q of n: Rabin also needs gcd(t^(2^(n/q)) - t, mu) = 1
        std::vector<uint32_t> qs;
        {
            uint32_t m = n;
            for (uint32_t q = 2; q * q <= m; ++q)
                if (m % q == 0) {
                    qs.push_back(q);
                    while (m % q == 0)
                        m /= q;
                }
            if (m > 1)
                qs.push_back(m);
        }
        std::vector<uint32_t> capture;   // squaring counts n/q to bring back
        for (uint32_t q : qs)
            if (q != n)
                capture.push_back(n / q);
        // rows t^(2i) mod mu for i = h .. D-1
        const uint32_t W = (uint32_t)(D / 64 + 1), h = (uint32_t)((D + 1) / 2);
        std::vector<unsigned long long> rows((size_t)(D - h) * W, 0ull);
        {
            Poly r;
            xor_shifted(r, Poly(1, 1ull), 2 * (size_t)h);   // t^(2h)
            r = mod(r, mu);
            for (uint32_t i = h; i < (uint32_t)D; ++i) {
                r.resize(W, 0ull);
                std::copy(r.begin(), r.begin() + W, rows.begin() + (size_t)(i - h) * W);
                Poly s2;
                xor_shifted(s2, r, 2);
                r = mod(s2, mu);
            }
        }
        cudaStream_t cs = (cudaStream_t)cuda_stream;   // current device
        unsigned long long *d_rows = nullptr, *d_a = nullptr, *d_b = nullptr;
        auto cleanup = [&]() {
            if (d_rows)
                cudaFreeAsync(d_rows, cs);
            if (d_a)
                cudaFreeAsync(d_a, cs);
            if (d_b)
                cudaFreeAsync(d_b, cs);
        };
        cudaError_t e = cudaMallocAsync((void**)&d_rows, rows.size() * 8, cs);
        if (e == cudaSuccess)
            e = cudaMallocAsync((void**)&d_a, (size_t)W * 8, cs);
        if (e == cudaSuccess)
            e = cudaMallocAsync((void**)&d_b, (size_t)W * 8, cs);
        std::vector<unsigned long long> t1(W, 0ull);
        t1[0] = 2ull;   // the polynomial t
        if (e == cudaSuccess)
            e = cudaMemcpyAsync(d_rows, rows.data(), rows.size() * 8, cudaMemcpyHostToDevice, cs);
        if (e == cudaSuccess)
            e = cudaMemcpyAsync(d_a, t1.data(), (size_t)W * 8, cudaMemcpyHostToDevice, cs);
        const uint32_t rows_per_slice = 64;
        const dim3 grid((W + 255) / 256, ((uint32_t)D - h + rows_per_slice - 1) / rows_per_slice);
        std::vector<std::vector<unsigned long long>> captured;
        std::vector<unsigned long long> host(W);
        for (uint32_t k = 1; k <= n && e == cudaSuccess; ++k) {
            e = cudaMemsetAsync(d_b, 0, (size_t)W * 8, cs);
            if (e != cudaSuccess)
                break;
            mtgp_frobenius_kernel<<<grid, 256, 0, cs>>>(d_a, d_b, d_rows, (uint32_t)D, W, h, rows_per_slice);
            e = cudaGetLastError();
            std::swap(d_a, d_b);
            if (e == cudaSuccess && std::find(capture.begin(), capture.end(), k) != capture.end()) {
                e = cudaMemcpyAsync(host.data(), d_a, (size_t)W * 8, cudaMemcpyDeviceToHost, cs);
                if (e == cudaSuccess)
                    e = cudaStreamSynchronize(cs);
                captured.push_back(host);
            }
        }
        if (e == cudaSuccess)
            e = cudaMemcpyAsync(host.data(), d_a, (size_t)W * 8, cudaMemcpyDeviceToHost, cs);
        if (e == cudaSuccess)
            e = cudaStreamSynchronize(cs);
        cleanup();
        if (e != cudaSuccess)
            return fail_cuda(e, "period check");
        // t^(2^n) == t (mod mu)?
        if (host != t1)
            return ok();
        for (auto& c : captured) {   // gcd(t^(2^(n/q)) - t, mu) == 1
            Poly x(c.begin(), c.end());
            x[0] ^= 2ull;
            trim(x);
            if (degree(gcd(mu, x)) != 0)
                return ok();
        }
        *irreducible = 1;
        return ok();
    } catch (const std::bad_alloc&) {
        return fail(MTGP_ENOMEM, "host allocation failed");
    }
}

extern "C" mtgp_status mtgp_params_period_check(mtgp_params_t params, void* cuda_stream, int32_t* irreducible)
{
    try {
        if (!params || !irreducible)
            return fail(MTGP_EINVAL, "null argument");
        *irreducible = 0;
        const Poly* mu = cached_mu(set_of(params->k, nullptr), params->d.mexp);
        if (!mu)
            return fail(MTGP_EINVAL, "no annihilating polynomial found for this parameter set");
        return rabin_irreducible(*mu, params->d.mexp, cuda_stream, irreducible);
    } catch (const std::bad_alloc&) {
        return fail(MTGP_ENOMEM, "host allocation failed");
    }
}

// ---------------------------------------------------------------------------
// The same polynomial and period check for the original Mersenne Twister
// (the comparison generator of Sec. 5.3): its window transition also maps the
// unused low r bits of the oldest word to zero, so mu is found the same way.
// ---------------------------------------------------------------------------
static mtgp_status mt_rec(const mtgp_mt_params* q, MtRec* out)
{
    if (!q)
        return fail(MTGP_EINVAL, "null argument");
    if (q->n < 2 || q->n > 4096 || q->m < 1 || q->m > q->n - 1 || q->r > 31 ||
        (uint64_t)32 * q->n - q->r != q->p)
        return fail(MTGP_EINVAL, "parameter set out of range (p %u, n %u, m %u, r %u)", q->p, q->n, q->m,
                    q->r);
    out->n = q->n;
    out->m = q->m;
    out->upper = 0xFFFFFFFFu << q->r;
    out->a = q->a;
    return MTGP_OK;
}

extern "C" mtgp_status mtgp_mt_params_minpoly(const mtgp_mt_params* params, uint64_t* words,
                                              uint32_t cap_words, int32_t* degree_out)
{
    try {
        MtRec p;
        if (!degree_out)
            return fail(MTGP_EINVAL, "null argument");
        mtgp_status st = mt_rec(params, &p);
        if (st != MTGP_OK)
            return st;
        const Poly* mu = cached_mu(p, params->p);
        if (!mu)
            return fail(MTGP_EINVAL, "no annihilating polynomial found for this parameter set");
        const int d = degree(*mu);
        *degree_out = d;
        const uint32_t need = (uint32_t)(d / 64 + 1);
        if (words) {
            if (cap_words < need)
                return fail(MTGP_EINVAL, "need %u words", need);
            std::fill(words, words + cap_words, 0ull);
            std::copy(mu->begin(), mu->end(), words);
        }
        return ok();
    } catch (const std::bad_alloc&) {
        return fail(MTGP_ENOMEM, "host allocation failed");
    }
}

extern "C" mtgp_status mtgp_mt_params_period_check(const mtgp_mt_params* params, void* cuda_stream,
                                                   int32_t* irreducible)
{
    try {
        MtRec p;
        if (!irreducible)
            return fail(MTGP_EINVAL, "null argument");
        *irreducible = 0;
        mtgp_status st = mt_rec(params, &p);
        if (st != MTGP_OK)
            return st;
        const Poly* mu = cached_mu(p, params->p);
        if (!mu)
            return fail(MTGP_EINVAL, "no annihilating polynomial found for this parameter set");
        return rabin_irreducible(*mu, params->p, cuda_stream, irreducible);
    } catch (const std::bad_alloc&) {
        return fail(MTGP_ENOMEM, "host allocation failed");
    }
}

// The jump polynomials g = t^(J-1) mod mu of one parameter set for the
// lengths J (sorted, distinct), cached.  Consecutive lengths reuse each
// other: t^(J'-1) = t^(J-1) * t^(J'-J) mod mu, so a run of equally spaced
// lengths costs one power and one product per length.
static std::vector<const Poly*> jump_polys(const SetP& p, const Poly& mu, const std::vector<uint64_t>& J)
{
    std::vector<const Poly*> out(J.size(), nullptr);
    const auto key = key_of(p);
    std::map<uint64_t, Poly> step;   // t^d mod mu for the gaps d between lengths
    const Poly* prev = nullptr;
    uint64_t prev_j = 0;
    for (size_t i = 0; i < J.size(); ++i) {
        const auto jk = std::make_pair(key, J[i]);
        {
            std::lock_guard<std::mutex> g(g_cache_mutex);
            auto it = g_jump_cache.find(jk);
            if (it != g_jump_cache.end())
                out[i] = &it->second;
        }
        if (!out[i]) {
            Poly g;
            if (prev) {
                const uint64_t d = J[i] - prev_j;
                auto st = step.find(d);
                if (st == step.end())
                    st = step.emplace(d, pow_t_mod(d, mu)).first;
                g = mod(mul(*prev, st->second), mu);
            } else {
                g = pow_t_mod(J[i] - 1, mu);
            }
            if (degree(g) < 0)
                g.assign(1, 0);
            std::lock_guard<std::mutex> lk(g_cache_mutex);
            out[i] = &g_jump_cache.emplace(jk, std::move(g)).first->second;
        }
        prev = out[i];
        prev_j = J[i];
    }
    return out;
}

mtgp_status mtgp::build_jump_batch(mtgp_streams* st, const std::vector<uint32_t>& rows,
                                   const std::vector<uint32_t>& sets, const std::vector<uint64_t>& jumps,
                                   JumpBatch* out, const std::vector<KSet>* given_sets)
{
    out->items.clear();
    out->poly_words.clear();
    out->words = 0;
    out->smem = 0;
    std::vector<KSet> own_sets;
    const std::vector<KSet>& host_sets = given_sets ? *given_sets : own_sets;
    if (st->d_sets && !given_sets) {
        own_sets.resize(st->n_sets);
        const cudaError_t e = cudaMemcpy(own_sets.data(), st->d_sets, st->n_sets * sizeof(KSet),
                                         cudaMemcpyDeviceToHost);
        if (e != cudaSuccess)
            return fail_cuda(e, "cudaMemcpy(parameter sets)");
    }
    // distinct lengths per parameter set
    std::map<uint32_t, std::vector<uint64_t>> lengths;
    for (size_t i = 0; i < rows.size(); ++i)
        if (jumps[i])
            lengths[sets[i]].push_back(jumps[i]);
    std::map<std::pair<uint32_t, uint64_t>, uint32_t> poly_index;
    std::vector<const Poly*> polys;
    for (auto& kv : lengths) {
        std::sort(kv.second.begin(), kv.second.end());
        kv.second.erase(std::unique(kv.second.begin(), kv.second.end()), kv.second.end());
        const SetP p = set_of(st->P.k, st->d_sets ? &host_sets[kv.first] : nullptr);
        const Poly* mu = cached_mu(p, st->P.d.mexp);
        if (!mu)
            return fail(MTGP_EINVAL, "no annihilating polynomial found for parameter set %u", kv.first);
        const std::vector<const Poly*> g = jump_polys(p, *mu, kv.second);
        for (size_t i = 0; i < g.size(); ++i) {
            poly_index.emplace(std::make_pair(kv.first, kv.second[i]), (uint32_t)polys.size());
            polys.push_back(g[i]);
        }
    }
    uint32_t max_deg = 0;
    for (size_t i = 0; i < rows.size(); ++i) {
        if (!jumps[i])
            continue;
        const uint32_t pi = poly_index.at(std::make_pair(sets[i], jumps[i]));
        JumpItem ji;
        ji.stream = rows[i];
        ji.poly = pi;
        ji.deg = (uint32_t)std::max(degree(*polys[pi]), 0);
        ji.set = sets[i];
        out->items.push_back(ji);
        max_deg = std::max(max_deg, ji.deg);
    }
    if (out->items.empty())
        return MTGP_OK;
    const uint32_t N = st->P.k.n;
    out->words = (max_deg + 1 + 31) / 32;
    out->poly_words.assign(polys.size() * (size_t)out->words, 0u);
    for (size_t i = 0; i < polys.size(); ++i)
        for (int k = 0; k <= degree(*polys[i]); ++k)
            if (bit(*polys[i], (size_t)k))
                out->poly_words[i * out->words + (size_t)k / 32] |= 1u << (k % 32);
    // a zero g (possible only if t^(J-1) = 0 mod mu, which needs t | mu):
    // the kernel then accumulates nothing and applies one step to 0
    out->smem = ((size_t)max_deg + 1 + N - 1 + N) * 4;
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess)
        return fail_cuda(e, "cudaGetDevice");
    e = allow_max_dynamic_smem((const void*)mtgp_jump_kernel, dev, out->smem);
    if (e == cudaErrorInvalidValue)
        return fail(MTGP_EINVAL, "state size too large for the jump kernel (%zu bytes of shared memory)",
                    out->smem);
    if (e != cudaSuccess)
        return fail_cuda(e, "jump kernel shared memory limit");
    return MTGP_OK;
}

cudaError_t mtgp::launch_jump_batch(const mtgp_streams* st, uint32_t* rows_base, const JumpItem* d_items,
                                    uint32_t n, const uint32_t* d_polys, uint32_t words, size_t smem,
                                    cudaStream_t s)
{
    if (n == 0)
        return cudaSuccess;
    mtgp_jump_kernel<<<n, 256, smem, s>>>(st->P.k, rows_base, d_items, d_polys, words, st->d_sets);
    return cudaGetLastError();
}

extern "C" mtgp_status mtgp_jump(mtgp_streams_t st, const uint32_t* ids, const uint64_t* jumps, uint32_t n,
                                 void* cuda_stream)
{
    try {
        if (!st || (n && (!ids || !jumps)))
            return fail(MTGP_EINVAL, "null argument");
        DeviceGuard dg(st->device);
        // total jump per stream (jumps compose additively)
        std::map<uint32_t, uint64_t> total;
        for (uint32_t i = 0; i < n; ++i) {
            if (ids[i] >= st->n_streams)
                return fail(MTGP_EINVAL, "stream id %u out of range (%u streams)", ids[i], st->n_streams);
            uint64_t& t = total[ids[i]];
            if (t + jumps[i] < t)
                return fail(MTGP_EINVAL, "total jump of stream %u overflows 64 bits", ids[i]);
            t += jumps[i];
        }
        // set index of each stream (per-stream parameter sets)
        std::vector<uint32_t> set_of_stream;
        if (st->d_sets) {
            set_of_stream.resize(st->n_streams);
            J_TRY(cudaMemcpy(set_of_stream.data(), st->d_set_of, st->n_streams * 4, cudaMemcpyDeviceToHost),
                  "cudaMemcpy(set index)");
        }
        std::vector<uint32_t> rows, sets;
        std::vector<uint64_t> lens;
        for (const auto& kv : total) {
            rows.push_back(kv.first);
            sets.push_back(st->d_sets ? set_of_stream[kv.first] : 0u);
            lens.push_back(kv.second);
        }
        JumpBatch b;
        mtgp_status r = build_jump_batch(st, rows, sets, lens, &b);
        if (r != MTGP_OK)
            return r;
        if (b.items.empty())
            return ok();
        cudaStream_t cs = (cudaStream_t)cuda_stream;
        void *d_items = nullptr, *d_polys = nullptr;
        J_TRY(cudaMallocAsync(&d_items, b.items.size() * sizeof(JumpItem), cs), "cudaMallocAsync");
        cudaError_t e = cudaMallocAsync(&d_polys, b.poly_words.size() * 4, cs);
        if (e == cudaSuccess)
            e = cudaMemcpyAsync(d_items, b.items.data(), b.items.size() * sizeof(JumpItem),
                                cudaMemcpyHostToDevice, cs);
        if (e == cudaSuccess)
            e = cudaMemcpyAsync(d_polys, b.poly_words.data(), b.poly_words.size() * 4,
                                cudaMemcpyHostToDevice, cs);
        if (e == cudaSuccess)
            e = launch_jump_batch(st, st->d_states, (const JumpItem*)d_items, (uint32_t)b.items.size(),
                                  (const uint32_t*)d_polys, b.words, b.smem, cs);
        // the host arrays above are locals: wait for the copies before returning
        const cudaError_t e2 = cudaStreamSynchronize(cs);
        if (d_polys)
            cudaFreeAsync(d_polys, cs);
        cudaFreeAsync(d_items, cs);
        if (e != cudaSuccess)
            return fail_cuda(e, "jump kernel");
        if (e2 != cudaSuccess)
            return fail_cuda(e2, "cudaStreamSynchronize");
        return ok();
    } catch (const std::bad_alloc&) {
        return fail(MTGP_ENOMEM, "host allocation failed");
    }
}

/*
 * The paper's optimized CPU reference (arXiv:1007.3726, Sec. 4): multi-spin
 * coding of the checkerboard Metropolis update with a pool of precomputed
 * Boltzmann bit patterns.
 *
 * TEST INFRASTRUCTURE AND CPU BASELINE ONLY.  It is one of the paper's
 * comparison programs, kept as a second, faster timed CPU baseline (the
 * paper's 1.00x row of Table 1); only tests/ and bench.py's CPU baseline use
 * it.  It shares no code with the GPU library.  It is NOT bit-exact with the
 * library or with the oracle: it draws one pool address per 32-spin word (the
 * paper's scheme), not one Philox number per site, so its trajectories differ
 * and it is checked statistically (tests/test_msc_pool.py).
 *
 * Storage: an L x L periodic lattice, L a multiple of 32, row-major 32-bit
 * words; bit b of word w of row y is the spin at x = 32 w + b, set = +1.
 *
 * Boltzmann patterns (Sec. 4): entry k of the pool is a pair of 32-bit words
 * (exp4[k], exp8[k]); for each bit an independent uniform 32-bit integer u is
 * drawn and exp8 gets a 1 when u < thr8, exp4 a 1 when thr8 <= u < thr4, with
 * thr = floor(2^32 exp(-dE/T)) (the strict "<" of the flip condition; the
 * encoding's two strict inequalities are read so that no u is left out).
 *
 * Update of one word s0 of target sites (Sec. 4, Eqs. 4-5): the neighbour
 * patterns s1..s4 (the words above and below, the row shifted by one with the
 * carry bit of the adjacent word), the energy variables i_n = s0 ^ s_n, one
 * random pool address per word, and the condition
 *     i1 + i2 + i3 + i4 + 2 exp8 + exp4 >= 2
 * evaluated for all 32 bits with Boolean operations: with c = i1 + i2 + i3 + i4
 * it holds when c >= 2, when c == 1 and exp4 | exp8, or when c == 0 and exp8.
 * A parity mask lets only the sites with (x + y) & 1 == p flip (Sec. 4: "only
 * allows to flip every second spin at once"); p = 0 first, then p = 1.
 *
 * Random numbers: splitmix64 (Steele, Lea and Flood, OOPSLA 2014), written
 * from its published definition.  The pool is filled from one stream; the
 * addresses of row y in step p of sweep t come from a stream seeded by
 * (seed, t, p, y), so the result does not depend on the number of threads.
 */
#include <math.h>
#include <stddef.h>
#include <stdint.h>

static uint64_t splitmix64_next(uint64_t *state)
{
    uint64_t z = (*state += 0x9E3779B97F4A7C15ull);
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
}

static uint32_t threshold(double dE, double T)
{
    const double v = floor(ldexp(exp(-dE / T), 32));
    if (v >= 4294967295.0) return 0xFFFFFFFFu;
    if (v <= 0.0) return 0u;
    return (uint32_t)v;
}

/* Fills the pool of npool pattern pairs at temperature T.  Returns 0, or -1 for
 * a T that is not finite and positive. */
int msc_pool_fill(uint32_t *exp4, uint32_t *exp8, uint64_t npool, double T, uint64_t seed)
{
    if (!(T > 0.0) || !isfinite(T)) return -1;
    const uint32_t thr4 = threshold(4.0, T), thr8 = threshold(8.0, T);
    uint64_t st = seed ^ 0x5DEECE66Dull;
    for (uint64_t k = 0; k < npool; ++k) {
        uint32_t e4 = 0, e8 = 0;
        for (int b = 0; b < 32; b += 2) {
            const uint64_t r = splitmix64_next(&st);  /* two 32-bit variates */
            const uint32_t u0 = (uint32_t)r, u1 = (uint32_t)(r >> 32);
            e8 |= (uint32_t)(u0 < thr8) << b;
            e4 |= (uint32_t)(u0 >= thr8 && u0 < thr4) << b;
            e8 |= (uint32_t)(u1 < thr8) << (b + 1);
            e4 |= (uint32_t)(u1 >= thr8 && u1 < thr4) << (b + 1);
        }
        exp4[k] = e4;
        exp8[k] = e8;
    }
    return 0;
}

/* One checkerboard step p of sweep t over the whole lattice, in place.  npool
 * must be a power of two. */
static void msc_step(uint32_t *lat, uint64_t L, const uint32_t *exp4, const uint32_t *exp8, uint64_t npool,
                     uint64_t t, uint32_t p, uint64_t seed)
{
    const uint64_t W = L / 32;
    const uint64_t amask = npool - 1;
    long long yy;
#pragma omp parallel for schedule(static)
    for (yy = 0; yy < (long long)L; ++yy) {
        const uint64_t y = (uint64_t)yy;
        uint32_t *row = lat + y * W;
        const uint32_t *up = lat + ((y + L - 1) % L) * W;
        const uint32_t *dn = lat + ((y + 1) % L) * W;
        const uint32_t mask = ((y + p) & 1) ? 0xAAAAAAAAu : 0x55555555u;
        uint64_t st = seed ^ (t * 0xD1B54A32D192ED03ull) ^ ((uint64_t)p << 62) ^ (y * 0x8CB92BA72F3D8DD7ull);
        for (uint64_t w = 0; w < W; ++w) {
            const uint32_t s0 = row[w];
            const uint32_t lw = row[(w + W - 1) % W], rw = row[(w + 1) % W];
            const uint32_t s1 = up[w], s2 = dn[w];
            const uint32_t s3 = (s0 << 1) | (lw >> 31);  /* x - 1 */
            const uint32_t s4 = (s0 >> 1) | (rw << 31);  /* x + 1 */
            const uint32_t i1 = s0 ^ s1, i2 = s0 ^ s2, i3 = s0 ^ s3, i4 = s0 ^ s4;
            /* c = i1 + i2 + i3 + i4 as "c >= 2", "c == 1", "c == 0" */
            const uint32_t a = i1 ^ i2, ac = i1 & i2;
            const uint32_t b = i3 ^ i4, bc = i3 & i4;
            const uint32_t ge2 = ac | bc | (a & b);
            const uint32_t eq1 = (a ^ b) & ~ge2;
            const uint32_t eq0 = ~(a | b | ac | bc);
            const uint64_t k = splitmix64_next(&st) & amask;
            const uint32_t e4 = exp4[k], e8 = exp8[k];
            const uint32_t flip = mask & (ge2 | (eq1 & (e4 | e8)) | (eq0 & e8));
            row[w] = s0 ^ flip;
        }
    }
}

/* M and E of the packed lattice (E = -sum of the 2 L^2 bonds). */
void msc_recount(const uint32_t *lat, uint64_t L, int64_t *M, int64_t *E)
{
    const uint64_t W = L / 32;
    int64_t up = 0, anti = 0;
    for (uint64_t y = 0; y < L; ++y)
        for (uint64_t w = 0; w < W; ++w) {
            const uint32_t s = lat[y * W + w];
            const uint32_t nx = lat[y * W + (w + 1) % W];
            const uint32_t dn = lat[((y + 1) % L) * W + w];
            const uint32_t right = (s >> 1) | (nx << 31);
            up += __builtin_popcount(s);
            anti += __builtin_popcount(s ^ right) + __builtin_popcount(s ^ dn);
        }
    const int64_t N = (int64_t)(L * L);
    *M = 2 * up - N;
    *E = 2 * anti - 2 * N;
}

/* Sweeps t0 .. t0 + nsweeps - 1; with M / E not NULL, the recounted M and E
 * after each sweep.  Returns 0, or -1 for bad sizes (L a multiple of 32, npool
 * a power of two). */
int msc_sweeps(uint32_t *lat, uint64_t L, const uint32_t *exp4, const uint32_t *exp8, uint64_t npool,
               uint64_t t0, uint64_t nsweeps, uint64_t seed, int64_t *M, int64_t *E)
{
    if (L < 32 || L % 32 != 0 || npool == 0 || (npool & (npool - 1)) != 0) return -1;
    for (uint64_t i = 0; i < nsweeps; ++i) {
        msc_step(lat, L, exp4, exp8, npool, t0 + i, 0, seed);
        msc_step(lat, L, exp4, exp8, npool, t0 + i, 1, seed);
        if (M && E) msc_recount(lat, L, M + i, E + i);
    }
    return 0;
}

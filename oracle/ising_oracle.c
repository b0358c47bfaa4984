/*
 * Oracle for the checkerboard Metropolis sweep of the 2D Ising model
 * (Block, Virnau, Preis, "Multi-GPU Accelerated Multi-Spin Monte Carlo
 * Simulations of the 2D Ising Model", arXiv:1007.3726).
 *
 * TEST INFRASTRUCTURE ONLY.  This file is the plain, slow, obviously correct
 * CPU statement of what the GPU path computes.  Only the test-suite, the
 * smoke check and the CPU-baseline leg of the benchmark may load it.  It
 * shares no code, header, table or helper with the CUDA library: it has its
 * own Philox4x32-10, its own thresholds, its own lattice (one int8 per spin,
 * +1 or -1) and its own energy and magnetisation bookkeeping.
 *
 * What it follows:
 *   - Hamiltonian H = -J sum_<ij> S_i S_j - H sum_i S_i with J = 1 (Sec. 3,
 *     Eq. 1), on an L x L square lattice with periodic boundaries (Sec. 6.1,
 *     Fig. 4 caption: outer borders joined periodically).  The paper sets the
 *     field H to zero; the *_field functions at the end keep it.
 *   - Metropolis acceptance: a move with energy change dE <= 0 is always
 *     taken, otherwise with probability exp(-dE/T) (Sec. 3); the factors for
 *     the two positive energy changes dE in {4, 8} are fixed on the host per
 *     temperature (Sec. 3) as integer thresholds floor(2^32 exp(-dE/T)), and a
 *     32-bit draw u is accepted when u < threshold (the strict "r < exp" of
 *     Eq. 3).
 *   - Checkerboard decomposition: step A updates the "black" sites, step B
 *     the "white" sites, and B starts after A is complete (Sec. 3).  Black is
 *     parity p = (x + y) & 1 == 0.
 *   - Per-site random draw: one 32-bit word of Philox4x32-10 (Salmon, Moraes,
 *     Dror, Shaw, "Parallel Random Numbers: As Easy as 1, 2, 3", SC'11) per
 *     site update, in place of the paper's LCG array (Sec. 5.3).  The counter
 *     numbers the site, the sweep and the step; the key is the seed.
 *   - Magnetisation and bond energy bookkeeping (Sec. 5.2 reduces the
 *     magnetisation per block); here kept incrementally AND recounted, and the
 *     two must agree after every sweep.
 *   - Binder cumulant U4 = 1 - <M^4> / (3 <M^2>^2) (Sec. 3, Eq. 2).
 *
 * Site/counter contract (shared by definition with the GPU path, not by code):
 *   site index in a step   j = y * (L/2) + (x >> 1)      (x + y) & 1 == p
 *   Philox group and lane  g = j >> 2,  lane = j & 3
 *   counter                (g mod 2^32, g >> 32, t, (stream_id << 1) | p)
 *   key                    (seed mod 2^32, seed >> 32)
 *   draw                   u = word `lane` of Philox(counter, key)
 *   hot start, site n = y*L + x: counter (n>>7 mod 2^32, n>>39, 0xFFFFFFFF,
 *   stream_id << 1); the spin is +1 iff bit (n & 31) of word ((n >> 5) & 3).
 *
 * Build:  gcc -O2 -fopenmp -shared -fPIC -o libising_oracle.so ising_oracle.c -lm
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

/* ------------------------------------------------------------------------ */
/* Philox4x32-10, from the SC'11 description: four 32-bit words, ten rounds.  */
/* Each round multiplies words 0 and 2 by the two Philox constants, takes     */
/* the high and low halves of the 64-bit products, and mixes the high halves  */
/* with words 1 and 3 and the round key; the key grows by the two Weyl        */
/* constants between rounds.                                                  */
/* ------------------------------------------------------------------------ */
#define PHILOX_MUL_A 0xD2511F53u
#define PHILOX_MUL_B 0xCD9E8D57u
#define PHILOX_WEYL_A 0x9E3779B9u
#define PHILOX_WEYL_B 0xBB67AE85u

void orc_philox4x32_10(const uint32_t ctr[4], const uint32_t key[2], uint32_t out[4])
{
    uint32_t x0 = ctr[0], x1 = ctr[1], x2 = ctr[2], x3 = ctr[3];
    uint32_t k0 = key[0], k1 = key[1];
    for (int round = 0; round < 10; ++round) {
        if (round > 0) {
            k0 += PHILOX_WEYL_A;
            k1 += PHILOX_WEYL_B;
        }
        uint64_t pa = (uint64_t)PHILOX_MUL_A * (uint64_t)x0;
        uint64_t pb = (uint64_t)PHILOX_MUL_B * (uint64_t)x2;
        uint32_t pa_hi = (uint32_t)(pa >> 32), pa_lo = (uint32_t)pa;
        uint32_t pb_hi = (uint32_t)(pb >> 32), pb_lo = (uint32_t)pb;
        uint32_t y0 = pb_hi ^ x1 ^ k0;
        uint32_t y1 = pb_lo;
        uint32_t y2 = pa_hi ^ x3 ^ k1;
        uint32_t y3 = pa_lo;
        x0 = y0; x1 = y1; x2 = y2; x3 = y3;
    }
    out[0] = x0; out[1] = x1; out[2] = x2; out[3] = x3;
}

/* n counters (4 words each, row-major) under n keys (2 words each). */
void orc_philox_batch(uint64_t n, const uint32_t *ctrs, const uint32_t *keys, uint32_t *out)
{
    for (uint64_t i = 0; i < n; ++i)
        orc_philox4x32_10(ctrs + 4 * i, keys + 2 * i, out + 4 * i);
}

/* ------------------------------------------------------------------------ */
/* Metropolis thresholds (Sec. 3): thr(dE) = floor(2^32 exp(-dE/T)), dE=4,8.  */
/* A positive finite T whose factor rounds to 1.0 in FP64 is clamped to      */
/* 2^32 - 1.  Returns 0, or -1 for T that is not finite and positive.         */
/* ------------------------------------------------------------------------ */
static uint32_t threshold_of(double dE, double T)
{
    double v = floor(ldexp(exp(-dE / T), 32));
    if (v >= 4294967295.0) return 0xFFFFFFFFu;
    if (v <= 0.0) return 0u;
    return (uint32_t)v;
}

int orc_thresholds(double T, uint32_t *thr4, uint32_t *thr8)
{
    if (!(T > 0.0) || !isfinite(T)) return -1;
    *thr4 = threshold_of(4.0, T);
    *thr8 = threshold_of(8.0, T);
    return 0;
}

/* ------------------------------------------------------------------------ */
/* Initial states.  Rows [row0, row0 + nrows) of the global L x L lattice go  */
/* into s[(y - row0) * L + x].                                                */
/* ------------------------------------------------------------------------ */
void orc_init_hot(int8_t *s, uint64_t L, uint64_t row0, uint64_t nrows,
                  uint64_t seed, uint32_t stream_id)
{
    uint32_t key[2] = {(uint32_t)seed, (uint32_t)(seed >> 32)};
#ifdef _OPENMP
#pragma omp parallel for schedule(static) if (nrows * L >= (1u << 18))
#endif
    for (uint64_t r = 0; r < nrows; ++r) {
        uint64_t y = (row0 + r) % L;
        for (uint64_t x = 0; x < L; ++x) {
            uint64_t n = y * L + x;
            uint32_t ctr[4] = {(uint32_t)(n >> 7), (uint32_t)(n >> 39), 0xFFFFFFFFu,
                               stream_id << 1};
            uint32_t out[4];
            orc_philox4x32_10(ctr, key, out);
            uint32_t word = out[(n >> 5) & 3];
            s[r * L + x] = ((word >> (n & 31)) & 1u) ? 1 : -1;
        }
    }
}

void orc_init_cold(int8_t *s, uint64_t count, int value)
{
    memset(s, value > 0 ? 1 : 0xFF, count);
}

/* ------------------------------------------------------------------------ */
/* Full recount: M = sum_i S_i; E = -sum_(x,y) S(x,y) [S(x+1,y) + S(x,y+1)],   */
/* every bond once, periodic in both directions (Sec. 3, Eq. 1, J=1, H=0).    */
/* ------------------------------------------------------------------------ */
void orc_recount(const int8_t *s, uint64_t L, int64_t *M, int64_t *E)
{
    int64_t m = 0, e = 0;
#ifdef _OPENMP
#pragma omp parallel for reduction(+ : m, e) schedule(static) if (L * L >= (1u << 18))
#endif
    for (uint64_t y = 0; y < L; ++y) {
        uint64_t yd = (y + 1) % L;
        for (uint64_t x = 0; x < L; ++x) {
            uint64_t xr = (x + 1) % L;
            int v = s[y * L + x];
            m += v;
            e -= v * (s[y * L + xr] + s[yd * L + x]);
        }
    }
    *M = m;
    *E = e;
}

/* ------------------------------------------------------------------------ */
/* One checkerboard step (Sec. 3): every site of parity p updated from the    */
/* state before the step.  Neighbours of a parity-p site have parity 1-p and  */
/* are not written in this step, so updating in place is the same as a        */
/* simultaneous update.                                                       */
/*                                                                            */
/* The buffer holds rows [row0, row0 + nrows) of the global lattice.  With    */
/* periodic != 0 the buffer is the whole lattice (nrows == L) and rows wrap.  */
/* Otherwise (light-cone mode) the first and last buffer rows are not updated */
/* and serve as fixed neighbours, so after k steps the rows k .. nrows-1-k    */
/* agree with the same rows of the periodic lattice.  Columns always wrap.    */
/*                                                                            */
/* dM and dE receive the changes of M and E over the updated rows (the        */
/* incremental bookkeeping).                                                  */
/* ------------------------------------------------------------------------ */
void orc_half_sweep(int8_t *s, uint64_t L, uint64_t row0, uint64_t nrows, int periodic,
                    uint64_t t, uint32_t p, uint64_t seed, uint32_t stream_id,
                    uint32_t thr4, uint32_t thr8, int64_t *dM_out, int64_t *dE_out)
{
    const uint32_t key[2] = {(uint32_t)seed, (uint32_t)(seed >> 32)};
    const uint32_t c3 = (stream_id << 1) | (p & 1u);
    int64_t dM = 0, dE = 0;
    int64_t r_begin = periodic ? 0 : 1;
    int64_t r_end = periodic ? (int64_t)nrows : (int64_t)nrows - 1;

#ifdef _OPENMP
#pragma omp parallel for reduction(+ : dM, dE) schedule(static) if (nrows * L >= (1u << 18))
#endif
    for (int64_t r = r_begin; r < r_end; ++r) {
        uint64_t y = (row0 + (uint64_t)r) % L;
        uint64_t r_up = periodic ? (uint64_t)((r + (int64_t)nrows - 1) % (int64_t)nrows) : (uint64_t)(r - 1);
        uint64_t r_dn = periodic ? (uint64_t)((r + 1) % (int64_t)nrows) : (uint64_t)(r + 1);
        int have_draw = 0;
        uint64_t cached_g = 0;
        uint32_t draws[4] = {0, 0, 0, 0};
        for (uint64_t x = 0; x < L; ++x) {
            if (((x + y) & 1u) != p) continue;
            /* the site's draw */
            uint64_t j = y * (L / 2) + (x >> 1);
            uint64_t g = j >> 2;
            uint32_t lane = (uint32_t)(j & 3u);
            if (!have_draw || g != cached_g) {
                uint32_t ctr[4] = {(uint32_t)g, (uint32_t)(g >> 32), (uint32_t)t, c3};
                orc_philox4x32_10(ctr, key, draws);
                cached_g = g;
                have_draw = 1;
            }
            uint32_t u = draws[lane];
            /* the energy change of flipping S(x, y): dE = 2 S sum_n S_n */
            int v = s[(uint64_t)r * L + x];
            int nsum = s[(uint64_t)r * L + (x + L - 1) % L] + s[(uint64_t)r * L + (x + 1) % L] +
                       s[r_up * L + x] + s[r_dn * L + x];
            int dE_site = 2 * v * nsum;
            int accept;
            if (dE_site <= 0)
                accept = 1;
            else if (dE_site == 4)
                accept = u < thr4;
            else /* dE_site == 8 */
                accept = u < thr8;
            if (accept) {
                s[(uint64_t)r * L + x] = (int8_t)(-v);
                dM -= 2 * v;
                dE += dE_site;
            }
        }
    }
    if (dM_out) *dM_out = dM;
    if (dE_out) *dE_out = dE;
}

/* ------------------------------------------------------------------------ */
/* A run of sweeps on the whole periodic lattice.  Sweep number t runs from   */
/* t0 to t0 + nsweeps - 1; each sweep is step A (p = 0) then step B (p = 1).  */
/* M[i], E[i] receive the state after sweep t0 + i.  The incremental sums are */
/* compared with a full recount after every sweep when check != 0; the first  */
/* mismatch returns 1 + i.  *M_run / *E_run carry the running values in and   */
/* out (pass the recount of the start state).                                 */
/* ------------------------------------------------------------------------ */
int orc_run(int8_t *s, uint64_t L, uint64_t t0, uint64_t nsweeps, uint64_t seed,
            uint32_t stream_id, uint32_t thr4, uint32_t thr8, int64_t *M_run, int64_t *E_run,
            int64_t *M, int64_t *E, int check)
{
    int64_t m = *M_run, e = *E_run;
    for (uint64_t i = 0; i < nsweeps; ++i) {
        for (uint32_t p = 0; p < 2; ++p) {
            int64_t dM, dE;
            orc_half_sweep(s, L, 0, L, 1, t0 + i, p, seed, stream_id, thr4, thr8, &dM, &dE);
            m += dM;
            e += dE;
        }
        if (check) {
            int64_t mr, er;
            orc_recount(s, L, &mr, &er);
            if (mr != m || er != e) {
                *M_run = m;
                *E_run = e;
                return (int)(1 + i);
            }
        }
        if (M) M[i] = m;
        if (E) E[i] = e;
    }
    *M_run = m;
    *E_run = e;
    return 0;
}

/* Light-cone run on a window of rows (see orc_half_sweep). */
void orc_run_window(int8_t *s, uint64_t L, uint64_t row0, uint64_t nrows, uint64_t t0,
                    uint64_t nsweeps, uint64_t seed, uint32_t stream_id, uint32_t thr4,
                    uint32_t thr8)
{
    for (uint64_t i = 0; i < nsweeps; ++i)
        for (uint32_t p = 0; p < 2; ++p)
            orc_half_sweep(s, L, row0, nrows, 0, t0 + i, p, seed, stream_id, thr4, thr8, 0, 0);
}

/* ------------------------------------------------------------------------ */
/* M and E of a whole periodic lattice after each of its first k sweeps from */
/* a cold start (all +1 when up != 0, else all -1), computed tile by tile so  */
/* that the lattice is never held in memory: a tile of R rows is simulated as */
/* a light-cone window with a margin of 2k + 1 rows on each side, and after   */
/* every sweep the tile's own rows (exact, the margin has not reached them)   */
/* give their spins, their horizontal bonds and their bonds to the next row.  */
/* M[j], E[j] receive the values after sweep j (j = 0 .. k-1).                */
/* ------------------------------------------------------------------------ */
int orc_cold_tiled_counts(uint64_t L, int up, uint64_t k, uint64_t tile_rows, uint64_t seed,
                          uint32_t stream_id, uint32_t thr4, uint32_t thr8, int64_t *M, int64_t *E)
{
    const uint64_t margin = 2 * k + 1;
    if (tile_rows == 0 || L % tile_rows != 0 || tile_rows + 2 * margin > L) return -1;
    const uint64_t wrows = tile_rows + 2 * margin;
    int8_t *w = (int8_t *)malloc(wrows * L);
    if (!w) return -2;
    for (uint64_t j = 0; j < k; ++j) M[j] = E[j] = 0;
    for (uint64_t t0 = 0; t0 < L; t0 += tile_rows) {
        const uint64_t row0 = (t0 + L - margin) % L;
        orc_init_cold(w, wrows * L, up ? 1 : -1);
        for (uint64_t j = 0; j < k; ++j) {
            for (uint32_t p = 0; p < 2; ++p)
                orc_half_sweep(w, L, row0, wrows, 0, j, p, seed, stream_id, thr4, thr8, 0, 0);
            int64_t m = 0, e = 0;
#ifdef _OPENMP
#pragma omp parallel for reduction(+ : m, e) schedule(static)
#endif
            for (uint64_t r = margin; r < margin + tile_rows; ++r) {
                for (uint64_t x = 0; x < L; ++x) {
                    int v = w[r * L + x];
                    m += v;
                    e -= v * (w[r * L + (x + 1) % L] + w[(r + 1) * L + x]);
                }
            }
            M[j] += m;
            E[j] += e;
        }
    }
    free(w);
    return 0;
}

/* ------------------------------------------------------------------------ */
/* FP64 observables from integer samples, plain summation in sample order.    */
/* m = M/N, e = E/N over samples [burn, n):                                   */
/*   out[0] <m>   out[1] <|m|>  out[2] <m^2>  out[3] <m^4>                    */
/*   out[4] <e>   out[5] <e^2>                                                */
/*   out[6] U4 = 1 - <m^4> / (3 <m^2>^2)                       (Sec. 3, Eq. 2) */
/*   out[7] chi = N (<m^2> - <|m|>^2) / T                                     */
/*   out[8] C   = N (<e^2> - <e>^2) / T^2                                     */
/* Returns the number of samples used.                                        */
/* ------------------------------------------------------------------------ */
uint64_t orc_moments(const int64_t *M, const int64_t *E, uint64_t n, uint64_t burn, double N,
                     double T, double out[9])
{
    double sm = 0, sa = 0, s2 = 0, s4 = 0, se = 0, se2 = 0;
    uint64_t k = 0;
    for (uint64_t i = burn; i < n; ++i) {
        double m = (double)M[i] / N;
        double e = (double)E[i] / N;
        sm += m;
        sa += fabs(m);
        s2 += m * m;
        s4 += m * m * m * m;
        se += e;
        se2 += e * e;
        ++k;
    }
    for (int i = 0; i < 9; ++i) out[i] = 0.0;
    if (k == 0) return 0;
    double kk = (double)k;
    out[0] = sm / kk;
    out[1] = sa / kk;
    out[2] = s2 / kk;
    out[3] = s4 / kk;
    out[4] = se / kk;
    out[5] = se2 / kk;
    out[6] = 1.0 - out[3] / (3.0 * out[2] * out[2]);
    out[7] = N * (out[2] - out[1] * out[1]) / T;
    out[8] = N * (out[5] - out[4] * out[4]) / (T * T);
    return k;
}

/* ------------------------------------------------------------------------ */
/* Nonzero field (Sec. 3, Eq. 1 with H != 0).  Flipping S(x, y), whose four   */
/* neighbours sum to n, changes the energy by dE = 2 S (n + H): the bond part */
/* 2 S n and the field part 2 S H.  The move is taken when dE <= 0, else when */
/* u < floor(2^32 exp(-dE/T)), the factor fixed in FP64 for this dE (the      */
/* thresholds of Sec. 3 now depend on the spin as well as on n).  Whole       */
/* periodic lattice; the draws follow the same site/counter contract.  dM and */
/* dE_bond receive the changes of M and of the bond energy -sum S_i S_j (the  */
/* field energy is -H M).                                                     */
/* ------------------------------------------------------------------------ */
void orc_half_sweep_field(int8_t *s, uint64_t L, uint64_t t, uint32_t p, uint64_t seed,
                          uint32_t stream_id, double T, double H, int64_t *dM_out,
                          int64_t *dE_out)
{
    const uint32_t key[2] = {(uint32_t)seed, (uint32_t)(seed >> 32)};
    const uint32_t c3 = (stream_id << 1) | (p & 1u);
    int64_t dM = 0, dEb = 0;
#ifdef _OPENMP
#pragma omp parallel for reduction(+ : dM, dEb) schedule(static) if (L * L >= (1u << 18))
#endif
    for (int64_t r = 0; r < (int64_t)L; ++r) {
        uint64_t y = (uint64_t)r;
        uint64_t r_up = (y + L - 1) % L, r_dn = (y + 1) % L;
        for (uint64_t x = 0; x < L; ++x) {
            if (((x + y) & 1u) != p) continue;
            uint64_t j = y * (L / 2) + (x >> 1);
            uint64_t g = j >> 2;
            uint32_t ctr[4] = {(uint32_t)g, (uint32_t)(g >> 32), (uint32_t)t, c3};
            uint32_t draws[4];
            orc_philox4x32_10(ctr, key, draws);
            uint32_t u = draws[j & 3u];
            int v = s[y * L + x];
            int nsum = s[y * L + (x + L - 1) % L] + s[y * L + (x + 1) % L] + s[r_up * L + x] +
                       s[r_dn * L + x];
            double dE = 2.0 * (double)v * ((double)nsum + H);
            int accept = dE <= 0.0 ? 1 : (u < threshold_of(dE, T));
            if (accept) {
                s[y * L + x] = (int8_t)(-v);
                dM -= 2 * v;
                dEb += 2 * v * nsum;
            }
        }
    }
    if (dM_out) *dM_out = dM;
    if (dE_out) *dE_out = dEb;
}

/* Sweeps t0 .. t0 + nsweeps - 1 in a field, as orc_run (M, E = bond energy). */
int orc_run_field(int8_t *s, uint64_t L, uint64_t t0, uint64_t nsweeps, uint64_t seed,
                  uint32_t stream_id, double T, double H, int64_t *M_run, int64_t *E_run,
                  int64_t *M, int64_t *E, int check)
{
    int64_t m = *M_run, e = *E_run;
    for (uint64_t i = 0; i < nsweeps; ++i) {
        for (uint32_t p = 0; p < 2; ++p) {
            int64_t dM, dE;
            orc_half_sweep_field(s, L, t0 + i, p, seed, stream_id, T, H, &dM, &dE);
            m += dM;
            e += dE;
        }
        if (check) {
            int64_t mr, er;
            orc_recount(s, L, &mr, &er);
            if (mr != m || er != e) {
                *M_run = m;
                *E_run = e;
                return (int)(1 + i);
            }
        }
        if (M) M[i] = m;
        if (E) E[i] = e;
    }
    *M_run = m;
    *E_run = e;
    return 0;
}

/* The acceptance of a site in a field by class: spin S (index 0 for -1, 1 for */
/* +1) and c anti-aligned neighbours (neighbour sum n = S (4 - 2c)).  thr[5 i + c] */
/* = floor(2^32 exp(-dE/T)) for dE = 2 S (n + H) > 0, always[5 i + c] = 1 where */
/* dE <= 0 (thr 0 there).  Returns -1 for T not finite and positive or H not   */
/* finite.                                                                     */
int orc_field_thresholds(double T, double H, uint32_t thr[10], uint8_t always[10])
{
    if (!(T > 0.0) || !isfinite(T) || !isfinite(H)) return -1;
    for (int i = 0; i < 2; ++i) {
        int v = i ? 1 : -1;
        for (int c = 0; c < 5; ++c) {
            int nsum = v * (4 - 2 * c);
            double dE = 2.0 * (double)v * ((double)nsum + H);
            always[5 * i + c] = dE <= 0.0;
            thr[5 * i + c] = dE <= 0.0 ? 0u : threshold_of(dE, T);
        }
    }
    return 0;
}

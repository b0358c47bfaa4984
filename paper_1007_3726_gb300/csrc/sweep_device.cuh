// Device building blocks of the checkerboard half-sweep shared by the
// one-lattice kernel (kernels.cu) and the persistent multi-lattice kernel
// (batch.cu): Philox4x32-10 rounds, the per-word acceptance masks and the
// bit-sliced update of one word (Sec. 4, Eqs. 4-5).
#pragma once

#include "kernels.h"

#include <cstdint>

namespace ising {
namespace {

constexpr uint32_t kPhiloxMulA = 0xD2511F53u;
constexpr uint32_t kPhiloxMulB = 0xCD9E8D57u;
constexpr uint32_t kWeylA = 0x9E3779B9u;
constexpr uint32_t kWeylB = 0xBB67AE85u;

// Philox4x32 rounds r0 .. 9 in place (SC'11): the two multipliers act on
// words 0 and 2; the new word 0 is hi(B * x2) ^ x1 ^ k0, word 1 is lo(B * x2),
// word 2 is hi(A * x0) ^ x3 ^ k1, word 3 is lo(A * x0).
template <int R0>
__device__ __forceinline__ void philox_rounds_from(uint32_t &x0, uint32_t &x1, uint32_t &x2,
                                                   uint32_t &x3, const RoundKeys &k)
{
#pragma unroll
    for (int r = R0; r < 10; ++r) {
        const uint64_t pa = (uint64_t)x0 * kPhiloxMulA;
        const uint64_t pb = (uint64_t)x2 * kPhiloxMulB;
        const uint32_t n0 = (uint32_t)(pb >> 32) ^ x1 ^ k.k0[r];
        const uint32_t n2 = (uint32_t)(pa >> 32) ^ x3 ^ k.k1[r];
        x1 = (uint32_t)pb;
        x3 = (uint32_t)pa;
        x0 = n0;
        x2 = n2;
    }
}

__device__ __forceinline__ void philox_rounds(uint32_t &x0, uint32_t &x1, uint32_t &x2,
                                              uint32_t &x3, const RoundKeys &k)
{
    philox_rounds_from<0>(x0, x1, x2, x3, k);
}

// Programmatic dependent launch: the step kernels are launched so that the next
// step's grid may be scheduled while this one drains.  Before a kernel touches
// global memory it waits until the grid before it has completed and its writes
// are visible; when a block has finished its items it lets the dependents
// launch (both are no-ops for a launch without the attribute).
__device__ __forceinline__ void dependent_launch_wait()
{
    asm volatile("griddepcontrol.wait;" ::: "memory");
}
__device__ __forceinline__ void dependent_launch_trigger()
{
    asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
}

template <typename Word>
struct WordTraits;
template <>
struct WordTraits<uint32_t> {
    static constexpr int bits = 32;
    static constexpr uint32_t even = 0x55555555u;
    __device__ static int popc(uint32_t v) { return __popc(v); }
    __device__ static uint32_t from_halves(const uint32_t *h) { return h[0]; }
};
template <>
struct WordTraits<uint64_t> {
    static constexpr int bits = 64;
    static constexpr uint64_t even = 0x5555555555555555ull;
    __device__ static int popc(uint64_t v) { return __popcll(v); }
    __device__ static uint64_t from_halves(const uint32_t *h)
    {
        return (uint64_t)h[0] | ((uint64_t)h[1] << 32);
    }
};

// Block-wide sum of two per-thread counters, one 64-bit atomic each per block.
__device__ __forceinline__ void block_accumulate(unsigned int a, unsigned int b,
                                                 unsigned long long *acc)
{
    __shared__ unsigned long long red[2][32];
    a = __reduce_add_sync(0xFFFFFFFFu, a);
    b = __reduce_add_sync(0xFFFFFFFFu, b);
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    if (lane == 0) {
        red[0][warp] = a;
        red[1][warp] = b;
    }
    __syncthreads();
    if (warp == 0) {
        const int nw = (blockDim.x + 31) >> 5;
        unsigned long long sa = lane < nw ? red[0][lane] : 0ull;
        unsigned long long sb = lane < nw ? red[1][lane] : 0ull;
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            sa += __shfl_down_sync(0xFFFFFFFFu, sa, o);
            sb += __shfl_down_sync(0xFFFFFFFFu, sb, o);
        }
        if (lane == 0) {
            atomicAdd(acc, sa);
            atomicAdd(acc + 1, sb);
        }
    }
}

// The device functions below take two argument objects: k with the launch
// constants (the round keys key, thr4, thr8, zero) and s with the values of the
// step (the step-uniform Philox values r1x0 .. r2x3, the parity p, and acc, not
// null when the step counts).  A step kernel passes its launch arguments as
// both; the persistent kernel passes its launch arguments and the step values
// it computes.
//
// The Philox4x32-10 calls of one word whose first Philox group is g0, with
// the step-uniform parts hoisted: round 1 and the word-0/word-3 half of round 2
// come from the step-uniform values; the round-1 products A * (g0 + q) are one
// widening multiply per word plus 64-bit additions of the constants A * q (the
// low counter words g0 .. g0 + NB - 1 of a word never wrap, since g0 is a
// multiple of NB).
struct WordDraws {
    uint64_t pa0;           // A * lo(g0)
    uint32_t r2x2k, r2x3;   // round-2 words 2 (before the XOR) and 3 for hi(g0)
};

template <typename K, typename S>
__device__ __forceinline__ WordDraws word_draws_begin(const K &k, const S &s, uint64_t g0)
{
    WordDraws d;
    const uint32_t c1 = (uint32_t)(g0 >> 32);  // the same for all groups of a word
    d.r2x2k = s.r2x2k;
    d.r2x3 = s.r2x3;
    if (c1 != 0u) {
        const uint64_t pa = (uint64_t)(s.r1x0 ^ c1) * kPhiloxMulA;
        d.r2x2k = (uint32_t)(pa >> 32) ^ k.key.k1[1];
        d.r2x3 = (uint32_t)pa;
    }
    d.pa0 = (uint64_t)(uint32_t)g0 * kPhiloxMulA;
    return d;
}

// The four draws of call q of the word (counter low word g0 + q).
template <typename K, typename S>
__device__ __forceinline__ void word_draw_call(const K &k, const S &s, const WordDraws &d, uint32_t q,
                                               uint32_t (&u)[4])
{
    // round 1: words 0, 1 are uniform (r1x0 ^ c1, lo(B t))
    const uint64_t pa = d.pa0 + (uint64_t)kPhiloxMulA * (uint64_t)q;
    const uint32_t x2 = (uint32_t)(pa >> 32) ^ s.r1x2k;
    const uint32_t x3 = (uint32_t)pa;
    // round 2: the product A * word 0 is uniform per word
    const uint64_t pb = (uint64_t)x2 * kPhiloxMulB;
    uint32_t y0 = (uint32_t)(pb >> 32) ^ s.r2x0k;
    uint32_t y1 = (uint32_t)pb;
    uint32_t y2 = x3 ^ d.r2x2k;
    uint32_t y3 = d.r2x3;
    philox_rounds_from<2>(y0, y1, y2, y3, k.key);
    u[0] = y0;
    u[1] = y1;
    u[2] = y2;
    u[3] = y3;
}

// Bit insertion of one compare, u < thr, for the FP32 forms of
// word_draw_masks: the predicated add of 4^M to an FP32 accumulator.  The
// accumulator starts at 2^23 and only ever holds integers below 2^24, so
// every add is exact; its low 16 bits are then the sum of the weights added.
// The weights are immediates (4^M as a PTX hex float) so that no register
// holds them.
template <int M>
__device__ __forceinline__ void fadd_if_below(float &acc, uint32_t u, uint32_t thr)
{
#define ISING_FADD_IF_BELOW(HEX)                                                              \
    asm("{\n\t.reg .pred p;\n\tsetp.lt.u32 p, %1, %2;\n\t@p add.f32 %0, %0, 0f" HEX ";\n\t}" \
        : "+f"(acc)                                                                           \
        : "r"(u), "r"(thr))
    static_assert(M >= 0 && M < 8, "weights 4^0 .. 4^7");
    if constexpr (M == 0) ISING_FADD_IF_BELOW("3F800000");
    if constexpr (M == 1) ISING_FADD_IF_BELOW("40800000");
    if constexpr (M == 2) ISING_FADD_IF_BELOW("41800000");
    if constexpr (M == 3) ISING_FADD_IF_BELOW("42800000");
    if constexpr (M == 4) ISING_FADD_IF_BELOW("43800000");
    if constexpr (M == 5) ISING_FADD_IF_BELOW("44800000");
    if constexpr (M == 6) ISING_FADD_IF_BELOW("45800000");
    if constexpr (M == 7) ISING_FADD_IF_BELOW("46800000");
#undef ISING_FADD_IF_BELOW
}

constexpr float kTwoTo23 = 8388608.0f;

// Bytes 0-1 of lo and bytes 0-1 of hi as one word (the low 16 bits of two
// accumulators started at 2^23).
__device__ __forceinline__ uint32_t low_halves(float lo, float hi)
{
    return __byte_perm(__float_as_uint(lo), __float_as_uint(hi), 0x5410);
}

// The draws of call qq (at local position qq of the calls this thread draws)
// added into the FP32 accumulators: site k = 4 (qq & 3) + l of a 32-bit half
// gets weight 4^(k mod 8) in accumulator (qq >> 1) & 1 of that half.  With
// SEP the P4 and P8 compares go to separate accumulators (f4, f8), else both
// into f4, which then holds the per-site count [u < thr4] + [u < thr8] in 0..2.
template <int QQ, int L, bool SEP>
__device__ __forceinline__ void fadd_site(float &f4, float &f8, uint32_t u, uint32_t thr4, uint32_t thr8)
{
    constexpr int M = 4 * (QQ & 1) + L;
    fadd_if_below<M>(f4, u, thr4);
    fadd_if_below<M>(SEP ? f8 : f4, u, thr8);
}

template <int QQ, bool SEP, int NH>
__device__ __forceinline__ void fadd_call(float (&f4)[NH][2], float (&f8)[NH][2], const uint32_t (&u)[4], int h,
                                          uint32_t thr4, uint32_t thr8)
{
    constexpr int j = (QQ >> 1) & 1;
    fadd_site<QQ, 0, SEP>(f4[h][j], f8[h][j], u[0], thr4, thr8);
    fadd_site<QQ, 1, SEP>(f4[h][j], f8[h][j], u[1], thr4, thr8);
    fadd_site<QQ, 2, SEP>(f4[h][j], f8[h][j], u[2], thr4, thr8);
    fadd_site<QQ, 3, SEP>(f4[h][j], f8[h][j], u[3], thr4, thr8);
}

template <int QQ, int NQ, int NB, bool SEP, int NH, typename K, typename S>
__device__ __forceinline__ void fadd_calls(const K &a, const S &s, const WordDraws &d, uint32_t q0,
                                           float (&f4)[NH][2], float (&f8)[NH][2])
{
    if constexpr (QQ < NQ) {
        const uint32_t q = (NQ == NB) ? (uint32_t)QQ : q0 + (uint32_t)QQ;
        uint32_t u[4];
        word_draw_call(a, s, d, q, u);
        fadd_call<QQ, SEP>(f4, f8, u, (NQ == NB) ? (QQ >> 2) : 0, a.thr4, a.thr8);
        fadd_calls<QQ + 1, NQ, NB, SEP>(a, s, d, q0, f4, f8);
    }
}

// The acceptance masks of one word whose first Philox group is g0: bit
// 8q + 2l of half (q / 4) is set when draw l of the word's call q is below the
// threshold.  INS selects how a compare's result becomes a bit:
//   0  a predicated OR into an integer mask;
//   1  a predicated FP32 add into one accumulator per 8 sites that counts
//      [u < thr4] + [u < thr8] (two bits per site, decoded into both masks);
//   2  predicated FP32 adds into separate P4 and P8 accumulators.
// The integer OR (or the addition the compiler makes of it) issues on the pipe
// that carries the Philox multiplies; the FP32 adds issue on the other FMA
// pipe, which the rest of the update leaves idle.  Forms 1 and 2 relieve the
// multiply pipe (its busy share falls from 81 % to 66 %) but measured 4 %
// slower on GB300: the autotuner keeps them as candidates.
template <int NB, int INS, int NQ = NB, typename K, typename S>
__device__ __forceinline__ void word_draw_masks(const K &a, const S &s, uint64_t g0,
                                                uint32_t (&p4)[(NB + 3) / 4],
                                                uint32_t (&p8)[(NB + 3) / 4], uint32_t q0 = 0)
{
    static_assert(INS >= 0 && INS <= 2, "insertion forms 0, 1, 2");
    const WordDraws d = word_draws_begin(a, s, g0);
    // With NQ < NB the calls q0 .. q0 + NQ - 1 (within one 32-bit half, since q0
    // is a multiple of NQ <= 4) are accumulated at their offsets from q0.
    constexpr int NH = (NQ == NB) ? (NB + 3) / 4 : 1;
    uint32_t m4[NH], m8[NH];
    if constexpr (INS == 0) {
#pragma unroll
        for (int h = 0; h < NH; ++h) {
            m4[h] = 0u;
            m8[h] = 0u;
        }
#pragma unroll
        for (int qq = 0; qq < NQ; ++qq) {
            const uint32_t q = (NQ == NB) ? (uint32_t)qq : q0 + (uint32_t)qq;
            uint32_t u[4];
            word_draw_call(a, s, d, q, u);
            const int h = (NQ == NB) ? (qq >> 2) : 0;
#pragma unroll
            for (int l = 0; l < 4; ++l) {
                const uint32_t bit = 1u << (8 * (qq & 3) + 2 * l);
                asm("{\n\t.reg .pred p;\n\tsetp.lt.u32 p, %1, %2;\n\t@p or.b32 %0, %0, %3;\n\t}"
                    : "+r"(m4[h])
                    : "r"(u[l]), "r"(a.thr4), "r"(bit));
                asm("{\n\t.reg .pred p;\n\tsetp.lt.u32 p, %1, %2;\n\t@p or.b32 %0, %0, %3;\n\t}"
                    : "+r"(m8[h])
                    : "r"(u[l]), "r"(a.thr8), "r"(bit));
            }
        }
    } else {
        constexpr bool SEP = INS == 2;
        float f4[NH][2], f8[NH][2];
#pragma unroll
        for (int h = 0; h < NH; ++h)
#pragma unroll
            for (int j = 0; j < 2; ++j) {
                f4[h][j] = kTwoTo23;
                f8[h][j] = kTwoTo23;
            }
        fadd_calls<0, NQ, NB, SEP>(a, s, d, q0, f4, f8);
#pragma unroll
        for (int h = 0; h < NH; ++h) {
            const uint32_t v = low_halves(f4[h][0], f4[h][1]);
            if constexpr (SEP) {
                m4[h] = v;
                m8[h] = low_halves(f8[h][0], f8[h][1]);
            } else {
                // per site two bits: 1 = P4 only, 2 = P4 and P8 (thr8 < thr4)
                const uint32_t hi = v >> 1;
                m8[h] = hi & 0x55555555u;
                m4[h] = (v | hi) & 0x55555555u;
            }
        }
    }
    if (NQ == NB) {
#pragma unroll
        for (int h = 0; h < (NB + 3) / 4; ++h) {
            p4[h] = m4[(NQ == NB) ? h : 0];
            p8[h] = m8[(NQ == NB) ? h : 0];
        }
    } else {
        const uint32_t sh = 8u * (q0 & 3u);
#pragma unroll
        for (int h = 0; h < (NB + 3) / 4; ++h) {
            const bool mine = (uint32_t)h == (q0 >> 2);
            p4[h] = mine ? (m4[0] << sh) : 0u;
            p8[h] = mine ? (m8[0] << sh) : 0u;
        }
    }
}

// Update of one word of target sites (Sec. 4): cur is the word, up / dn the
// words above / below, lw / rw the words left / right of it in its row, mask
// the target bit positions, off their parity (0 or 1), g the Philox group of
// the word's first byte.  Returns the new word; with count set, adds the
// popcounts of the new word (+1 spins) and of the anti-aligned bonds of its
// target sites.
// With NQ < NB only the Philox calls (bytes) q0 .. q0 + NQ - 1 of the word are
// drawn and only those bytes of the returned word (and of the counts) are
// meaningful: several threads can then share one word.
template <typename Word, int INS, int NQ = WordTraits<Word>::bits / 8, typename K, typename S>
__device__ __forceinline__ Word update_word(const K &a, const S &s, Word cur, Word up, Word dn,
                                            Word lw, Word rw, uint32_t off, uint64_t g, bool count,
                                            unsigned int &cnt_up, unsigned int &cnt_anti,
                                            uint32_t q0 = 0)
{
    using Tr = WordTraits<Word>;
    constexpr int B = Tr::bits;
    constexpr int NB = B / 8;
    const Word left = (cur << 1) | (lw >> (B - 1));   // bit b holds s(x - 1)
    const Word right = (cur >> 1) | (rw << (B - 1));  // bit b holds s(x + 1)
    const Word mask = off ? (Word)(Tr::even << 1) : Tr::even;

    // energy variables and their bit-sliced sum c = i1 + i2 + i3 + i4
    const Word i1 = cur ^ up, i2 = cur ^ dn, i3 = cur ^ left, i4 = cur ^ right;
    const Word s12 = i1 ^ i2, c12 = i1 & i2;
    const Word s34 = i3 ^ i4, c34 = i3 & i4;
    const Word odd = s12 ^ s34;                  // c odd
    const Word ge2 = c12 | c34 | (s12 & s34);    // c >= 2: dE <= 0, always accepted
    const Word eq1 = odd & ~ge2;                 // c == 1: dE = 4
    const Word eq0 = ~(odd | ge2);               // c == 0: dE = 8

    // the sites' draws: byte q of the word holds four target sites
    uint32_t h4[(NB + 3) / 4], h8[(NB + 3) / 4];
    word_draw_masks<NB, INS, NQ>(a, s, g, h4, h8, q0);
    const Word p4 = Tr::from_halves(h4) << off;
    const Word p8 = Tr::from_halves(h8) << off;
    Word sel = mask;
    if constexpr (NQ < NB) sel &= (((Word)1 << (8 * NQ)) - 1) << (8 * q0);  // this thread's bytes
    const Word flip = sel & (ge2 | (eq1 & p4) | (eq0 & p8));
    const Word nw = cur ^ flip;
    if (count) {
        // after the step: +1 spins of the word, and the anti-aligned bonds of
        // its target sites (their neighbours are final)
        Word own = ~(Word)0;
        if constexpr (NQ < NB) own = (((Word)1 << (8 * NQ)) - 1) << (8 * q0);
        cnt_up += Tr::popc(nw & own);
        cnt_anti += Tr::popc(sel & (nw ^ up)) + Tr::popc(sel & (nw ^ dn)) +
                    Tr::popc(sel & (nw ^ left)) + Tr::popc(sel & (nw ^ right));
    }
    return nw;
}

// The update of update_word with the acceptance masks drawn beforehand (the
// one-CTA kernels draw several steps ahead): pk holds this thread's masks in
// one word, P4 at the even and P8 at the odd bit positions of the word's
// target bytes (pack_masks), independent of the parity off.
__device__ __forceinline__ uint32_t pack_masks(uint32_t p4, uint32_t p8) { return p4 | (p8 << 1); }

template <int NQ>
__device__ __forceinline__ uint32_t update_word32_drawn(uint32_t cur, uint32_t up, uint32_t dn, uint32_t lw,
                                                        uint32_t rw, uint32_t off, uint32_t pk, bool count,
                                                        unsigned int &cnt_up, unsigned int &cnt_anti,
                                                        uint32_t q0)
{
    constexpr uint32_t even = 0x55555555u;
    const uint32_t left = (cur << 1) | (lw >> 31);
    const uint32_t right = (cur >> 1) | (rw << 31);
    const uint32_t mask = off ? (even << 1) : even;
    const uint32_t i1 = cur ^ up, i2 = cur ^ dn, i3 = cur ^ left, i4 = cur ^ right;
    const uint32_t s12 = i1 ^ i2, c12 = i1 & i2;
    const uint32_t s34 = i3 ^ i4, c34 = i3 & i4;
    const uint32_t odd = s12 ^ s34;
    const uint32_t ge2 = c12 | c34 | (s12 & s34);
    const uint32_t eq1 = odd & ~ge2;
    const uint32_t eq0 = ~(odd | ge2);
    const uint32_t p4 = (pk & even) << off;
    const uint32_t p8 = ((pk >> 1) & even) << off;
    uint32_t sel = mask;
    uint32_t own = ~0u;
    if constexpr (NQ < 4) {
        own = ((1u << (8 * NQ)) - 1u) << (8 * q0);
        sel &= own;
    }
    const uint32_t nw = cur ^ (sel & (ge2 | (eq1 & p4) | (eq0 & p8)));
    if (count) {
        cnt_up += __popc(nw & own);
        cnt_anti += __popc(sel & (nw ^ up)) + __popc(sel & (nw ^ dn)) + __popc(sel & (nw ^ left)) +
                    __popc(sel & (nw ^ right));
    }
    return nw;
}

// The items of one checkerboard step of the step kernel's geometry and launch
// constants (a: the lattice buffer, rows, words per row, rows per item, grid
// stride, keys, thresholds) with the step values sa (as above: the step-uniform
// Philox values, p the parity of the updated sites, counts taken when sa.acc
// is not null).  Work item = (block of R rows, word column w); the
// thread walks down its column keeping the rows above / at / below in
// registers, advancing its row pointers, group index and parity mask by
// additions.  Rows it reads but does not own (the halo rows and the adjacent
// words) are only used at bit positions of the other parity, which no thread
// writes during this step.  When counting, adds this thread's counts of the
// new state (see update_word).
template <typename Word, int INS, typename StepArgs>
__device__ __forceinline__ void half_sweep_items(const HalfSweepArgs &a, const StepArgs &sa, unsigned int &cnt_up,
                                                 unsigned int &cnt_anti)
{
    constexpr int NB = WordTraits<Word>::bits / 8;  // Philox calls (bytes) per word
    Word *const S = static_cast<Word *>(a.spins);
    const uint64_t rows = a.rows;
    const uint32_t W = a.words_per_row;
    const uint32_t R = a.rows_per_item;
    const uint32_t nrb = (uint32_t)(a.update_rows / R);
    const uint64_t groups_per_row = a.L >> 3;

    const uint32_t tid = blockIdx.x * blockDim.x + threadIdx.x;
    uint32_t rb = tid / W;
    uint32_t w = tid - rb * W;
    while (rb < nrb) {
        const int64_t dl = (w == 0) ? (int64_t)W - 1 : -1;  // to the left neighbour word
        const int64_t dr = (w + 1 == W) ? 1 - (int64_t)W : 1;
        const uint64_t y0 = a.first_row + (uint64_t)rb * R;   // buffer row
        const uint64_t yg = (uint64_t)(a.y_offset + (int64_t)y0);  // global row
        Word *q = S + y0 * W + w;
        Word up = *((y0 == 0) ? S + (rows - 1) * W + w : q - W);
        Word cur = *q;
        uint64_t g = yg * groups_per_row + (uint64_t)w * NB;
        uint32_t off = (uint32_t)((yg + sa.p) & 1u);  // parity of the target bit positions
        for (uint32_t r = 0; r < R; ++r) {
            Word *const qn = (y0 + r + 1 == rows) ? S + w : q + W;
            const Word dn = *qn;
            const Word lw = q[dl];
            const Word rw = q[dr];
            const Word nw = update_word<Word, INS>(a, sa, cur, up, dn, lw, rw, off, g, sa.acc != nullptr, cnt_up,
                                                   cnt_anti);
            *q = nw;
            up = nw;
            cur = dn;
            q = qn;
            g += groups_per_row;
            off ^= 1u;
        }
        rb += a.stride_rb;
        w += a.stride_w;
        if (w >= W) {
            w -= W;
            ++rb;
        }
    }
}

}  // namespace
}  // namespace ising

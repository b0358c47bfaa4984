// Device code of the checkerboard step in a field H (Sec. 3, Eq. 1 with H != 0):
// the update of one word with the ten acceptance classes (S, c), shared by the
// field step kernel (field.cu), the one-CTA kernel (tiny.cu) on 32-bit words
// and the persistent batch (batch.cu) on 64-bit words.
#pragma once

#include "sweep_device.cuh"

#include <cstdint>

namespace ising {
namespace {

// Sites with c >= k, for a uniform k in 0..5 (c = b0 + 2 b1 + 4 b2 <= 4).
template <typename Word>
__device__ __forceinline__ Word count_at_least(uint32_t k, Word b0, Word b1, Word b2)
{
    return k == 0 ? ~(Word)0 : k == 1 ? (b0 | b1 | b2) : k == 2 ? (b1 | b2) : k == 3 ? ((b0 & b1) | b2)
           : k == 4 ? b2 : (Word)0;
}

// One word of target sites in a field (see update_word for the arguments and
// for NQ / q0: with NQ < NB only the Philox calls q0 .. q0 + NQ - 1 of the word
// are drawn and only those bytes of the result are meaningful).  tab is the
// 16-entry threshold table, index 8 S + c, in shared memory (LDG = false) or
// in global memory read through the read-only cache (LDG = true).
template <typename Word, int NQ = WordTraits<Word>::bits / 8, bool LDG = false, typename K, typename S>
__device__ __forceinline__ Word update_word_field(const K &a, const S &s, const uint32_t *tab, uint32_t k_up,
                                                  uint32_t k_dn, Word cur, Word up, Word dn, Word lw, Word rw,
                                                  uint32_t off, uint64_t g, bool count, unsigned int &cnt_up,
                                                  unsigned int &cnt_anti, uint32_t q0 = 0)
{
    using Tr = WordTraits<Word>;
    constexpr int B = Tr::bits;
    constexpr int NB = B / 8;
    const Word even = Tr::even;
    const Word left = (cur << 1) | (lw >> (B - 1));   // bit b holds s(x - 1)
    const Word right = (cur >> 1) | (rw << (B - 1));  // bit b holds s(x + 1)
    const Word mask = off ? (Word)(even << 1) : even;

    // energy variables and the three bits of their sum c
    const Word i1 = cur ^ up, i2 = cur ^ dn, i3 = cur ^ left, i4 = cur ^ right;
    const Word s12 = i1 ^ i2, c12 = i1 & i2;
    const Word s34 = i3 ^ i4, c34 = i3 & i4;
    const Word b0 = s12 ^ s34;
    const Word b1 = c12 ^ c34 ^ (s12 & s34);
    const Word b2 = c12 & c34;  // c == 4 (then s12 = s34 = 0)
    const Word always = (cur & count_at_least<Word>(k_up, b0, b1, b2)) |
                        (~cur & count_at_least<Word>(k_dn, b0, b1, b2));

    // the class of target site j (bit off + 2j) as two 2-bit fields at bit 2j:
    // X = (b1 b0), Y = (S b2); its table index is X_j | Y_j << 2
    const Word X = ((b0 >> off) & even) | (((b1 >> off) & even) << 1);
    const Word Y = ((b2 >> off) & even) | (((cur >> off) & even) << 1);

    // P: bit 8q + 2l of half q / 4 is set when draw l of call q is below its
    // site's threshold (with NQ < NB: the calls of this thread, all in one
    // 32-bit half, at their offsets in it)
    const WordDraws d = word_draws_begin(a, s, g);
    constexpr int NH = (NQ == NB) ? (NB + 3) / 4 : 1;
    uint32_t P[NH];
#pragma unroll
    for (int h = 0; h < NH; ++h) P[h] = a.zero;
#pragma unroll
    for (int qq = 0; qq < NQ; ++qq) {
        const uint32_t q = (NQ == NB) ? (uint32_t)qq : q0 + (uint32_t)qq;
        uint32_t u[4];
        word_draw_call(a, s, d, q, u);
        const int h = (NQ == NB) ? (qq >> 2) : 0;
        const uint32_t half = (NQ == NB) ? (uint32_t)(qq >> 2) : (q >> 2);
        const uint32_t Xh = (uint32_t)(X >> (32 * half)), Yh = (uint32_t)(Y >> (32 * half));
#pragma unroll
        for (int l = 0; l < 4; ++l) {
            const uint32_t pos = 8u * (q & 3u) + 2u * (uint32_t)l;
            const uint32_t idx = ((Xh >> pos) & 3u) | (((Yh >> pos) & 3u) << 2);
            const uint32_t thr = LDG ? __ldg(tab + idx) : tab[idx];
            const uint32_t bit = 1u << pos;
            asm("{\n\t.reg .pred p;\n\tsetp.lt.u32 p, %1, %2;\n\t@p or.b32 %0, %0, %3;\n\t}"
                : "+r"(P[h])
                : "r"(u[l]), "r"(thr), "r"(bit));
        }
    }
    Word Pw;
    if constexpr (NQ == NB) {
        uint32_t halves[(NB + 3) / 4];
#pragma unroll
        for (int h = 0; h < (NB + 3) / 4; ++h) halves[h] = P[h];
        Pw = Tr::from_halves(halves);
    } else {
        Pw = (Word)P[0] << (32 * (q0 >> 2));
    }
    Word sel = mask;
    Word own = ~(Word)0;
    if constexpr (NQ < NB) {
        own = (((Word)1 << (8 * NQ)) - 1) << (8 * q0);  // this thread's bytes
        sel &= own;
    }
    const Word flip = sel & (always | (Pw << off));
    const Word nw = cur ^ flip;
    if (count) {
        cnt_up += Tr::popc(nw & own);
        cnt_anti += Tr::popc(sel & (nw ^ up)) + Tr::popc(sel & (nw ^ dn)) + Tr::popc(sel & (nw ^ left)) +
                    Tr::popc(sel & (nw ^ right));
    }
    return nw;
}

}  // namespace
}  // namespace ising

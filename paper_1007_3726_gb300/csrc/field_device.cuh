// Device code of the checkerboard step in a field H (Sec. 3, Eq. 1 with H != 0),
// shared by the field step kernel (field.cu) and the one-CTA kernel (tiny.cu):
// the update of one 32-bit word with the ten acceptance classes (S, c).
#pragma once

#include "sweep_device.cuh"

#include <cstdint>

namespace ising {
namespace {

constexpr uint32_t kEven = 0x55555555u;

// Sites with c >= k, for a uniform k in 0..5 (c = b0 + 2 b1 + 4 b2 <= 4).
__device__ __forceinline__ uint32_t count_at_least(uint32_t k, uint32_t b0, uint32_t b1, uint32_t b2)
{
    return k == 0 ? ~0u : k == 1 ? (b0 | b1 | b2) : k == 2 ? (b1 | b2) : k == 3 ? ((b0 & b1) | b2)
           : k == 4 ? b2 : 0u;
}

// One 32-bit word of target sites (see update_word for the arguments); tab is
// the 16-entry threshold table in shared memory, index 8 S + c.
__device__ __forceinline__ uint32_t update_word_field(const HalfSweepArgs &a, const uint32_t *tab,
                                                      uint32_t k_up, uint32_t k_dn, uint32_t cur,
                                                      uint32_t up, uint32_t dn, uint32_t lw, uint32_t rw,
                                                      uint32_t off, uint64_t g, bool count,
                                                      unsigned int &cnt_up, unsigned int &cnt_anti)
{
    const uint32_t left = (cur << 1) | (lw >> 31);   // bit b holds s(x - 1)
    const uint32_t right = (cur >> 1) | (rw << 31);  // bit b holds s(x + 1)
    const uint32_t mask = off ? (kEven << 1) : kEven;

    // energy variables and the three bits of their sum c
    const uint32_t i1 = cur ^ up, i2 = cur ^ dn, i3 = cur ^ left, i4 = cur ^ right;
    const uint32_t s12 = i1 ^ i2, c12 = i1 & i2;
    const uint32_t s34 = i3 ^ i4, c34 = i3 & i4;
    const uint32_t b0 = s12 ^ s34;
    const uint32_t b1 = c12 ^ c34 ^ (s12 & s34);
    const uint32_t b2 = c12 & c34;  // c == 4 (then s12 = s34 = 0)
    const uint32_t always = (cur & count_at_least(k_up, b0, b1, b2)) |
                            (~cur & count_at_least(k_dn, b0, b1, b2));

    // the class of target site j (bit off + 2j) as two 2-bit fields at bit 2j:
    // X = (b1 b0), Y = (S b2); its table index is X_j | Y_j << 2
    const uint32_t X = ((b0 >> off) & kEven) | (((b1 >> off) & kEven) << 1);
    const uint32_t Y = ((b2 >> off) & kEven) | (((cur >> off) & kEven) << 1);

    const WordDraws d = word_draws_begin(a, g);
    uint32_t P = a.zero;
#pragma unroll
    for (int q = 0; q < 4; ++q) {
        uint32_t u[4];
        word_draw_call(a, d, (uint32_t)q, u);
#pragma unroll
        for (int l = 0; l < 4; ++l) {
            const int pos = 8 * q + 2 * l;
            const uint32_t idx = ((X >> pos) & 3u) | (((Y >> pos) & 3u) << 2);
            const uint32_t thr = tab[idx];
            const uint32_t bit = 1u << pos;
            asm("{\n\t.reg .pred p;\n\tsetp.lt.u32 p, %1, %2;\n\t@p or.b32 %0, %0, %3;\n\t}"
                : "+r"(P)
                : "r"(u[l]), "r"(thr), "r"(bit));
        }
    }
    const uint32_t flip = mask & (always | (P << off));
    const uint32_t nw = cur ^ flip;
    if (count) {
        cnt_up += __popc(nw);
        cnt_anti += __popc(mask & (nw ^ up)) + __popc(mask & (nw ^ dn)) + __popc(mask & (nw ^ left)) +
                    __popc(mask & (nw ^ right));
    }
    return nw;
}

}  // namespace
}  // namespace ising

// Multi-spin-coded checkerboard Metropolis sweep of the 2D Ising model for
// sm_103a (after arXiv:1007.3726, Sec. 3-5).
//
// Layout: the lattice is L rows of W = L / bits words; bit b of word w of row
// y is the spin at x = w * bits + b, set = +1 (Sec. 5.2 stores one bit per
// spin with a set bit meaning +1).
//
// Step p updates the sites with (x + y) & 1 == p.  In a row these are the bit
// positions of one parity, so a word is updated by a masked XOR (Sec. 4: "an
// additional bit mask ... only allows to flip every second spin").  For each
// word the thread forms the four neighbour words (Sec. 4: patterns holding the
// i-th spin's neighbour at bit i): the words above and below, and the row word
// shifted by one with the carry bit taken from the adjacent word.  The energy
// variables i_n = s0 ^ s_n (Sec. 4, Eq. 4) are summed bit-parallel with a
// carry-save adder into "two or more anti-aligned", "exactly one" and "none".
// The acceptance i1 + i2 + i3 + i4 + 2 exp8 + exp4 >= 2 of Sec. 4, Eq. 5 then
// reads flip = ge2 | (eq1 & P4) | (eq0 & P8), with P4 / P8 the bit masks of
// u < thr4 / u < thr8 for the sites' own Philox draws.
//
// Each Philox4x32-10 call yields the draws of four consecutive target sites,
// which in every row occupy one byte of the packed row (x = 8q .. 8q + 7).
#include "kernels.h"
#include "sweep_device.cuh"

#include <atomic>
#include <cstdio>
#include <map>
#include <mutex>
#include <tuple>

namespace ising {

namespace {

// One checkerboard step (the items of half_sweep_items), launched as a
// dependent launch after the previous step.
template <typename Word, int INS>
__device__ __forceinline__ void half_sweep_body(const HalfSweepArgs &a)
{
    dependent_launch_wait();
    unsigned int cnt_up = 0, cnt_anti = 0;
    half_sweep_items<Word, INS>(a, a, cnt_up, cnt_anti);
    dependent_launch_trigger();
    if (a.acc) block_accumulate(cnt_up, cnt_anti, a.acc);
}

template <typename Word, int INS>
__global__ void __launch_bounds__(512) k_half_sweep(const __grid_constant__ HalfSweepArgs a)
{
    half_sweep_body<Word, INS>(a);
}
template <typename Word, int INS>
__global__ void __launch_bounds__(512, 3) k_half_sweep_r40(const __grid_constant__ HalfSweepArgs a)
{
    half_sweep_body<Word, INS>(a);
}
template <typename Word, int INS>
__global__ void __launch_bounds__(512, 4) k_half_sweep_r32(const __grid_constant__ HalfSweepArgs a)
{
    half_sweep_body<Word, INS>(a);
}

template <typename Word>
__global__ void k_init_hot(Word *S, uint64_t nwords, uint64_t first_word, RoundKeys key, uint32_t c3)
{
    constexpr int B = WordTraits<Word>::bits;
    for (uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; i < nwords;
         i += (uint64_t)gridDim.x * blockDim.x) {
        const uint64_t n0 = (first_word + i) * B;  // first site of the word (row-major site index)
        uint32_t x0 = (uint32_t)(n0 >> 7), x1 = (uint32_t)(n0 >> 39), x2 = 0xFFFFFFFFu, x3 = c3;
        philox_rounds(x0, x1, x2, x3, key);
        const uint32_t o[4] = {x0, x1, x2, x3};
        const uint32_t k = (uint32_t)((n0 >> 5) & 3u);
        if (B == 32) {
            S[i] = (Word)o[k];
        } else {
            // k is 0 or 2 for a 64-bit word
            S[i] = (Word)((uint64_t)o[k] | ((uint64_t)o[k + 1] << 32));
        }
    }
}

template <typename Word>
__global__ void k_pack(const int8_t *src, Word *S, uint64_t nwords, unsigned int *bad)
{
    constexpr int B = WordTraits<Word>::bits;
    unsigned int nbad = 0;
    for (uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; i < nwords;
         i += (uint64_t)gridDim.x * blockDim.x) {
        const int8_t *p = src + i * B;
        Word v = 0;
#pragma unroll 8
        for (int b = 0; b < B; ++b) {
            const int8_t s = p[b];
            v |= (Word)(s > 0) << b;
            nbad += (s != 1 && s != -1);
        }
        S[i] = v;
    }
    if (nbad) atomicAdd(bad, nbad);
}

template <typename Word>
__global__ void k_unpack(const Word *S, uint64_t L, uint64_t row0, uint64_t nrows, int8_t *dst)
{
    const uint64_t n = nrows * L;
    for (uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
         i += (uint64_t)gridDim.x * blockDim.x) {
        constexpr int B = WordTraits<Word>::bits;
        const uint64_t r = i / L, x = i - r * L;
        const uint64_t y = (row0 + r) % L;
        const Word w = S[y * (L / B) + x / B];
        dst[i] = ((w >> (x % B)) & 1) ? 1 : -1;
    }
}

template <typename Word>
__global__ void k_recount(const Word *S, uint64_t L, unsigned long long *acc)
{
    using Tr = WordTraits<Word>;
    constexpr int B = Tr::bits;
    const uint64_t W = L / B;
    const uint64_t nwords = L * W;
    unsigned int up = 0, anti = 0;
    for (uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; i < nwords;
         i += (uint64_t)gridDim.x * blockDim.x) {
        const uint64_t y = i / W, w = i - y * W;
        const Word s = S[i];
        const Word dn = S[((y + 1 == L) ? 0 : y + 1) * W + w];
        const Word nx = S[y * W + ((w + 1 == W) ? 0 : w + 1)];
        const Word right = (s >> 1) | (nx << (B - 1));
        up += Tr::popc(s);
        anti += Tr::popc(s ^ right) + Tr::popc(s ^ dn);
    }
    block_accumulate(up, anti, acc);
}

constexpr int kMaxDevices = 64;

// SMs of the current device, queried once per device.
int num_sms()
{
    static std::atomic<int> cache[kMaxDevices];
    int dev = 0;
    cudaGetDevice(&dev);
    int n = (dev >= 0 && dev < kMaxDevices) ? cache[dev].load(std::memory_order_relaxed) : 0;
    if (n <= 0) {
        cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev);
        if (n <= 0) n = 1;
        if (dev >= 0 && dev < kMaxDevices) cache[dev].store(n, std::memory_order_relaxed);
    }
    return n;
}

int grid_for(uint64_t work, int block, int per_sm)
{
    const uint64_t need = (work + block - 1) / block;
    const uint64_t cap = (uint64_t)num_sms() * per_sm;
    return (int)(need < cap ? (need > 0 ? need : 1) : cap);
}

}  // namespace

RoundKeys make_round_keys(uint64_t seed)
{
    RoundKeys k;
    uint32_t a = (uint32_t)seed, b = (uint32_t)(seed >> 32);
    for (int r = 0; r < 10; ++r) {
        k.k0[r] = a;
        k.k1[r] = b;
        a += kWeylA;
        b += kWeylB;
    }
    return k;
}

namespace {
using HalfSweepKernel = void (*)(HalfSweepArgs);

template <typename Word, int INS>
HalfSweepKernel pick_regcap(uint32_t regcap)
{
    if (regcap == 1) return k_half_sweep_r40<Word, INS>;
    if (regcap == 2) return k_half_sweep_r32<Word, INS>;
    return k_half_sweep<Word, INS>;
}

template <typename Word>
HalfSweepKernel pick_ins(const LaunchConfig &c)
{
    if (c.insert == 1) return pick_regcap<Word, 1>(c.regcap);
    if (c.insert == 2) return pick_regcap<Word, 2>(c.regcap);
    return pick_regcap<Word, 0>(c.regcap);
}

HalfSweepKernel half_sweep_kernel(const LaunchConfig &c)
{
    return c.proc_bits == 64 ? pick_ins<uint64_t>(c) : pick_ins<uint32_t>(c);
}

uint64_t mulA(uint32_t x) { return (uint64_t)x * kPhiloxMulA; }
uint64_t mulB(uint32_t x) { return (uint64_t)x * kPhiloxMulB; }
}  // namespace

cudaError_t launch_dependent(void (*kernel)(HalfSweepArgs), int grid, int block, cudaStream_t s,
                             const HalfSweepArgs &a)
{
    cudaLaunchConfig_t cfg{};
    cfg.gridDim = dim3((unsigned)grid);
    cfg.blockDim = dim3((unsigned)block);
    cfg.dynamicSmemBytes = 0;
    cfg.stream = s;
    cudaLaunchAttribute attr{};
    attr.id = cudaLaunchAttributeProgrammaticStreamSerialization;
    attr.val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = &attr;
    cfg.numAttrs = 1;
    return cudaLaunchKernelEx(&cfg, kernel, a);
}

void prepare_half_sweep(HalfSweepArgs &a, int grid, int block)
{
    const uint64_t pb = mulB(a.t);
    a.r1x0 = (uint32_t)(pb >> 32) ^ a.key.k0[0];
    a.r1x2k = a.c3 ^ a.key.k1[0];
    a.r2x0k = (uint32_t)pb ^ a.key.k0[1];
    const uint64_t pa = mulA(a.r1x0);
    a.r2x2k = (uint32_t)(pa >> 32) ^ a.key.k1[1];
    a.r2x3 = (uint32_t)pa;
    const uint64_t stride = (uint64_t)grid * (uint64_t)block;
    a.stride_rb = (uint32_t)(stride / a.words_per_row);
    a.stride_w = (uint32_t)(stride % a.words_per_row);
}

bool launch_config_valid(const LaunchConfig &c, uint64_t L, uint64_t rows)
{
    if (c.persistent) return persistent_config_valid(c, L, rows);
    if (c.proc_bits == kTinyProcBits) return tiny_config_valid(c, L, rows);
    if (c.proc_bits != 32 && c.proc_bits != 64) return false;
    if (c.regcap > 2) return false;
    if (c.insert > 2) return false;
    if (c.block != 128 && c.block != 256 && c.block != 512) return false;
    if (c.rows_per_item < 1 || c.rows_per_item > 64 || rows % c.rows_per_item != 0) return false;
    if (L % c.proc_bits != 0) return false;
    // the item index (row block * words + word) and the thread index stay in 32 bits
    const uint64_t items = rows / c.rows_per_item * (L / c.proc_bits);
    if (items >= (1ull << 32) - (1ull << 26)) return false;
    if (c.grid > 65535u * 16u) return false;
    return true;
}

int half_sweep_blocks_per_sm(const LaunchConfig &c)
{
    // queried once per (device, kernel, block size)
    static std::mutex mu;
    static std::map<std::tuple<int, HalfSweepKernel, uint32_t>, int> cache;
    int dev = 0;
    cudaGetDevice(&dev);
    const HalfSweepKernel k = half_sweep_kernel(c);
    const auto key = std::make_tuple(dev, k, c.block);
    {
        std::lock_guard<std::mutex> lk(mu);
        auto it = cache.find(key);
        if (it != cache.end()) return it->second;
    }
    int n = 0;
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, k, (int)c.block, 0);
    if (n <= 0) n = 1;
    std::lock_guard<std::mutex> lk(mu);
    cache[key] = n;
    return n;
}

int resolve_grid(const LaunchConfig &c, uint64_t L, uint64_t rows)
{
    const uint64_t items = rows / c.rows_per_item * (L / c.proc_bits);
    const uint64_t need = (items + c.block - 1) / c.block;
    uint64_t cap = c.grid;
    if (cap == 0) cap = (uint64_t)num_sms() * half_sweep_blocks_per_sm(c);
    const uint64_t g = need < cap ? need : cap;
    return (int)(g > 0 ? g : 1);
}

cudaError_t launch_half_sweep(HalfSweepArgs a, const LaunchConfig &c, cudaStream_t s)
{
    if ((c.proc_bits != 32 && c.proc_bits != 64) || c.persistent) return cudaErrorInvalidValue;  // not a step kernel
    if (a.update_rows == 0) {  // a whole periodic lattice
        a.first_row = 0;
        a.update_rows = a.rows;
        a.y_offset = 0;
    }
    const int grid = resolve_grid(c, a.L, a.update_rows);
    a.words_per_row = (uint32_t)(a.L / c.proc_bits);
    a.rows_per_item = c.rows_per_item;
    a.zero = 0u;
    prepare_half_sweep(a, grid, (int)c.block);
    return launch_dependent(half_sweep_kernel(c), grid, (int)c.block, s, a);
}

cudaError_t launch_init_hot(void *spins, uint64_t L, uint32_t word_bits, uint64_t seed,
                            uint32_t stream_id, cudaStream_t s)
{
    const RoundKeys k = make_round_keys(seed);
    const uint64_t nwords = L * (L / word_bits);
    const int block = 256, grid = grid_for(nwords, block, 8);
    if (word_bits == 64)
        k_init_hot<uint64_t><<<grid, block, 0, s>>>((uint64_t *)spins, nwords, 0, k, stream_id << 1);
    else
        k_init_hot<uint32_t><<<grid, block, 0, s>>>((uint32_t *)spins, nwords, 0, k, stream_id << 1);
    return cudaGetLastError();
}

cudaError_t launch_init_hot_rows(void *spins, uint64_t L, uint32_t word_bits, uint64_t row0,
                                 uint64_t nrows, uint64_t seed, uint32_t stream_id, cudaStream_t s)
{
    const RoundKeys k = make_round_keys(seed);
    const uint64_t W = L / word_bits;
    const uint64_t nwords = nrows * W;
    const int block = 256, grid = grid_for(nwords, block, 8);
    if (word_bits == 64)
        k_init_hot<uint64_t><<<grid, block, 0, s>>>((uint64_t *)spins, nwords, row0 * W, k, stream_id << 1);
    else
        k_init_hot<uint32_t><<<grid, block, 0, s>>>((uint32_t *)spins, nwords, row0 * W, k, stream_id << 1);
    return cudaGetLastError();
}

cudaError_t launch_pack(const int8_t *src, void *spins, uint64_t L, uint32_t word_bits,
                        unsigned int *bad, cudaStream_t s)
{
    const uint64_t nwords = L * (L / word_bits);
    const int block = 256, grid = grid_for(nwords, block, 8);
    if (word_bits == 64)
        k_pack<uint64_t><<<grid, block, 0, s>>>(src, (uint64_t *)spins, nwords, bad);
    else
        k_pack<uint32_t><<<grid, block, 0, s>>>(src, (uint32_t *)spins, nwords, bad);
    return cudaGetLastError();
}

cudaError_t launch_unpack(const void *spins, uint64_t L, uint32_t word_bits, uint64_t row0,
                          uint64_t nrows, int8_t *dst, cudaStream_t s)
{
    const int block = 256, grid = grid_for(nrows * L, block, 8);
    if (word_bits == 64)
        k_unpack<uint64_t><<<grid, block, 0, s>>>((const uint64_t *)spins, L, row0, nrows, dst);
    else
        k_unpack<uint32_t><<<grid, block, 0, s>>>((const uint32_t *)spins, L, row0, nrows, dst);
    return cudaGetLastError();
}

cudaError_t launch_recount(const void *spins, uint64_t L, uint32_t word_bits,
                           unsigned long long *acc, cudaStream_t s)
{
    const uint64_t nwords = L * (L / word_bits);
    const int block = 256, grid = grid_for(nwords, block, 8);
    if (word_bits == 64)
        k_recount<uint64_t><<<grid, block, 0, s>>>((const uint64_t *)spins, L, acc);
    else
        k_recount<uint32_t><<<grid, block, 0, s>>>((const uint32_t *)spins, L, acc);
    return cudaGetLastError();
}

}  // namespace ising

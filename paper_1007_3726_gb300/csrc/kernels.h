// Device kernels of the multi-spin-coded checkerboard sweep and their host
// launchers (internal to libising; the public ABI is include/ising.h).
#pragma once

#include <cstdint>
#include <cuda_runtime.h>

namespace ising {

// Philox4x32-10 round keys (Salmon et al., SC'11): round r uses
// (key0 + r * 0x9E3779B9, key1 + r * 0xBB67AE85), precomputed on the host so
// that the device never spends instructions on the key schedule.
struct RoundKeys {
    uint32_t k0[10];
    uint32_t k1[10];
};

RoundKeys make_round_keys(uint64_t seed);

// One checkerboard step (Sec. 3) over a packed periodic lattice.
struct HalfSweepArgs {
    void *spins;              // L rows of words_per_row words (32- or 64-bit)
    uint64_t L;
    uint32_t words_per_row;   // L / word_bits
    uint32_t rows_per_item;   // rows one thread walks down (divides L)
    RoundKeys key;
    uint32_t thr4, thr8;      // floor(2^32 exp(-4/T)), floor(2^32 exp(-8/T))
    uint32_t t;               // sweep index (Philox counter word 2)
    uint32_t c3;              // stream_id << 1 | p (Philox counter word 3)
    uint32_t p;               // parity of the updated sites
    // If not null (step B only): acc[0] += number of +1 spins of the whole
    // lattice after the step, acc[1] += number of anti-aligned bonds after the
    // step.  Every bond has exactly one endpoint of parity 1, so step B sees
    // each bond once.
    unsigned long long *acc;
};

struct LaunchShape {
    int grid;
    int block;
};

cudaError_t launch_half_sweep(const HalfSweepArgs &a, uint32_t word_bits, LaunchShape shape,
                              cudaStream_t s);
int half_sweep_blocks_per_sm(uint32_t word_bits, int block);

// Hot start (Philox with counter word 2 = 0xFFFFFFFF), cold start is a memset.
cudaError_t launch_init_hot(void *spins, uint64_t L, uint32_t word_bits, uint64_t seed,
                            uint32_t stream_id, cudaStream_t s);

// int8 +1/-1 -> packed; *bad counts entries that are neither +1 nor -1.
cudaError_t launch_pack(const int8_t *src, void *spins, uint64_t L, uint32_t word_bits,
                        unsigned int *bad, cudaStream_t s);

// packed rows [row0, row0 + nrows) -> int8 +1/-1.
cudaError_t launch_unpack(const void *spins, uint64_t L, uint32_t word_bits, uint64_t row0,
                          uint64_t nrows, int8_t *dst, cudaStream_t s);

// acc[0] += number of +1 spins, acc[1] += number of anti-aligned bonds.
cudaError_t launch_recount(const void *spins, uint64_t L, uint32_t word_bits,
                           unsigned long long *acc, cudaStream_t s);

}  // namespace ising

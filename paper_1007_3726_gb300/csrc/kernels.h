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
    void *spins;              // rows x words_per_row processing words (32- or 64-bit)
    uint64_t L;               // row length in sites (the lattice is L x L)
    uint64_t rows;            // rows in the buffer (== L for a whole lattice)
    uint64_t first_row;       // first buffer row updated (1 for a strip with a halo row above)
    uint64_t update_rows;     // rows updated (== rows for a whole periodic lattice)
    int64_t y_offset;         // global row index of buffer row 0 (Philox counters, parity)
    uint32_t words_per_row;   // L / processing bits
    uint32_t rows_per_item;   // rows one thread walks down (divides rows)
    RoundKeys key;
    uint32_t thr4, thr8;      // floor(2^32 exp(-4/T)), floor(2^32 exp(-8/T))
    uint32_t t;               // sweep index (Philox counter word 2)
    uint32_t c3;              // stream_id << 1 | p (Philox counter word 3)
    uint32_t p;               // parity of the updated sites
    // The parts of Philox rounds 1 and 2 that depend only on (t, c3, key), the
    // same for every site of the step; filled by prepare_half_sweep().
    uint32_t r1x0;   // hi(B t) ^ k0[0]: round-1 word 0 before the XOR with counter word 1
    uint32_t r1x2k;  // c3 ^ k1[0]
    uint32_t r2x0k;  // lo(B t) ^ k0[1]
    uint32_t r2x2k;  // hi(A r1x0) ^ k1[1]   (counter word 1 == 0)
    uint32_t r2x3;   // lo(A r1x0)           (counter word 1 == 0)
    uint32_t zero;   // 0, passed at run time (see word_draw_masks)
    // grid-stride walk over items (item = row block * words_per_row + word)
    uint32_t stride_rb, stride_w;  // (grid * block) / words_per_row, (grid * block) % words_per_row
    // If not null (step B only): acc[0] += number of +1 spins of the whole
    // lattice after the step, acc[1] += number of anti-aligned bonds after the
    // step.  Every bond has exactly one endpoint of parity 1, so step B sees
    // each bond once.
    unsigned long long *acc;
};

// Fills the step-uniform Philox values and the grid-stride constants.
void prepare_half_sweep(HalfSweepArgs &a, int grid, int block);

// Launches a step kernel with programmatic stream serialization: its grid may be
// scheduled while the previous kernel of the stream drains; the kernel waits
// (griddepcontrol.wait) before it reads the lattice.
cudaError_t launch_dependent(void (*kernel)(HalfSweepArgs), int grid, int block, cudaStream_t s,
                             const HalfSweepArgs &a);

// A launch configuration of the half-sweep.  Every valid configuration gives
// bit-identical results; they differ only in speed.  proc_bits == 8 selects the
// one-CTA kernel of tiny.cu instead (whole lattice in shared memory, every
// sweep of a call in one launch): block is its block size, rows_per_item the
// threads that share one 32-bit word (1, 2 or 4), grid the CTAs (1, or a
// cluster of 2, 4 or 8 that splits the rows), regcap = insert = 0.
struct LaunchConfig {
    uint32_t proc_bits;      // 32 or 64: bits one thread updates per row; 8: one CTA
    uint32_t regcap;         // 0: compiler's choice, 1: <= 40 registers, 2: <= 32 registers
    uint32_t insert;         // acceptance-bit insertion: 0 predicated OR, 1 FP32 counts, 2 FP32 masks
    uint32_t block;          // 128, 256 or 512 threads
    uint32_t rows_per_item;  // 2 .. 64, divides L
    uint32_t grid;           // blocks (0 = all resident blocks of the device)
    uint32_t persistent;     // 1: every sweep of a call in one cooperative launch (persistent.cu)
};

bool launch_config_valid(const LaunchConfig &c, uint64_t L, uint64_t rows);

// Every sweep of a call in one cooperative launch of the step items, with a
// grid-wide barrier between the steps (persistent.cu).  Samples as TinyRunArgs.
struct SweepsRun {
    uint32_t t0;              // sweep index of the first sweep
    uint32_t nsweeps;         // >= 1
    uint32_t record_every;    // 0: record nothing
    uint32_t nrec;            // recorded sweeps of the call
    uint32_t c3base;          // stream_id << 1
    unsigned long long *acc;  // nrec + 1 slots of two counters
};
// A persistent configuration: a step shape (proc_bits 32 / 64, regcap 0 / 1,
// insert 0) with persistent = 1 and grid = 0 (all resident blocks).
bool persistent_config_valid(const LaunchConfig &c, uint64_t L, uint64_t rows);
// a as for launch_half_sweep (spins, L, key, thr4, thr8); the geometry is filled here.
cudaError_t launch_sweeps(HalfSweepArgs a, const LaunchConfig &c, const SweepsRun &s, cudaStream_t st);

constexpr uint32_t kTinyProcBits = 8;
// Lattices the one-CTA kernel takes: L a power of two, 64 <= L <= 1024.
bool tiny_lattice_ok(uint64_t L);
// A one-CTA configuration (proc_bits == 8) for an L x L lattice of `rows` rows.
bool tiny_config_valid(const LaunchConfig &c, uint64_t L, uint64_t rows);
// c itself if it is a configuration of the half-sweep kernel, else the fixed
// default one (for callers that launch single steps).
LaunchConfig plain_launch(const LaunchConfig &c);

// Every sweep of one call on a whole lattice, in one launch of one CTA that
// holds the lattice in shared memory (tiny.cu).  Samples as in ising_sweep:
// acc[2k], acc[2k + 1] = (+1 spins, anti-aligned bonds) after the k-th recorded
// sweep, acc[2 nrec], acc[2 nrec + 1] after the last sweep.
struct TinyRunArgs {
    void *spins;              // L x L/8 bytes, packed rows (any storage word width)
    uint64_t L;
    RoundKeys key;
    uint32_t thr4, thr8;
    uint32_t c3base;          // stream_id << 1
    uint32_t t0;              // sweep index of the first sweep
    uint32_t nsweeps;         // >= 1
    uint32_t record_every;    // 0: record nothing
    uint32_t nrec;            // recorded sweeps of the call
    unsigned long long *acc;  // nrec + 1 slots of two counters
    // in a field H != 0 (use_field = 1): the class thresholds and the always-
    // accepted classes of field.h's FieldTable (thr4 / thr8 are then unused)
    uint32_t use_field;
    uint32_t field_thr[16];
    uint32_t k_up, k_dn;
    // set to a nonzero value by a kernel whose bounded wait ran out (the
    // warp-specialised one-CTA kernel); must be zero at the launch, may be null
    unsigned int *err;
    // failure-detection testing only: 1 + a step whose masks the producers of
    // the warp-specialised kernel never announce (0 = none), so that the
    // consumers' wait runs out (with a short wait limit)
    uint32_t hold_step;
};
// The warp-specialised configurations (tiny.cu): L = 64 or 128, 1024 threads
// per CTA, one thread per word; one CTA (L = 64: four consumer warps, 28
// producer warps) or a cluster of 2, 4 or 8 CTAs (consumers in the first,
// producers in the others).
constexpr uint32_t kTinyWsBlock = 1024;
// ctas = 1: one CTA; 2, 4, 8: a cluster of CTAs, each with L / ctas rows.
cudaError_t launch_tiny(const TinyRunArgs &a, uint32_t block, uint32_t threads_per_word, uint32_t ctas,
                        cudaStream_t s);
// Resident blocks per SM of the configuration's kernel.
int half_sweep_blocks_per_sm(const LaunchConfig &c);
// Grid that makes every block resident (grid == 0 resolved).
int resolve_grid(const LaunchConfig &c, uint64_t L, uint64_t rows);
cudaError_t launch_half_sweep(HalfSweepArgs a, const LaunchConfig &c, cudaStream_t s);

// Hot start (Philox with counter word 2 = 0xFFFFFFFF), cold start is a memset.
cudaError_t launch_init_hot(void *spins, uint64_t L, uint32_t word_bits, uint64_t seed,
                            uint32_t stream_id, cudaStream_t s);
// The hot start of global rows row0 .. row0 + nrows - 1 only, into `spins`.
cudaError_t launch_init_hot_rows(void *spins, uint64_t L, uint32_t word_bits, uint64_t row0,
                                 uint64_t nrows, uint64_t seed, uint32_t stream_id, cudaStream_t s);

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

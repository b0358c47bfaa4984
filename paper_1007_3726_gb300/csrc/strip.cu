// One lattice split into row strips, one strip per rank (GPU): the row-strip
// form of the paper's super-lattice decomposition (Sec. 6.1).  A rank keeps
// its strip with one halo row above and one below; before every checkerboard
// step the caller copies the neighbours' boundary rows into the halos (the
// "copy neighbor borders to GPU memory" step of Sec. 6.1), then this step
// updates the strip.  The Philox counters and parities use global row
// indices, so the result does not depend on how the rows are split.
// Nothing here allocates memory.
#include "handle.h"
#include "kernels.h"
#include "runtime.h"

using namespace ising;

namespace {

ising_status check_strip(const void *d_rows, uint64_t L, uint32_t word_bits, uint64_t row0, uint64_t nrows)
{
    if (!d_rows) return fail(ISING_ERR_INVALID, "d_rows is NULL");
    if (L < 64 || L % 64 != 0 || L > (1ull << 20))
        return fail(ISING_ERR_INVALID, "L must be a multiple of 64 in [64, 2^20]");
    if (word_bits != 32 && word_bits != 64) return fail(ISING_ERR_INVALID, "word_bits must be 32 or 64");
    if (nrows == 0 || row0 >= L || nrows > L || row0 + nrows > L)
        return fail(ISING_ERR_INVALID, "rows [row0, row0 + nrows) must lie in [0, L)");
    return ISING_OK;
}

}  // namespace

extern "C" {

ISING_API ising_status ising_strip_init(void *d_rows, uint64_t L, uint32_t word_bits, uint64_t row0,
                                        uint64_t nrows, ising_init init, uint64_t seed, uint32_t stream_id,
                                        void *cuda_stream)
{
    clear_error();
    ising_status st = check_strip(d_rows, L, word_bits, row0, nrows);
    if (st != ISING_OK) return st;
    if (stream_id >= (1u << 31)) return fail(ISING_ERR_INVALID, "stream_id must be < 2^31");
    cudaStream_t s = (cudaStream_t)cuda_stream;
    const size_t row_bytes = L / 8;
    char *rows = static_cast<char *>(d_rows) + row_bytes;  // strip rows follow the top halo
    cudaError_t e;
    switch (init) {
    case ISING_COLD_UP:
        e = cudaMemsetAsync(rows, 0xFF, nrows * row_bytes, s);
        break;
    case ISING_COLD_DOWN:
        e = cudaMemsetAsync(rows, 0x00, nrows * row_bytes, s);
        break;
    case ISING_HOT:
        e = launch_init_hot_rows(rows, L, word_bits, row0, nrows, seed, stream_id, s);
        break;
    default:
        return fail(ISING_ERR_INVALID, "strips start cold or hot");
    }
    if (e != cudaSuccess) return fail(ISING_ERR_CUDA, "strip init: %s", cudaGetErrorString(e));
    return ISING_OK;
}

ISING_API ising_status ising_strip_step(void *d_rows, uint64_t L, uint32_t word_bits, uint64_t row0,
                                        uint64_t nrows, double T, uint64_t seed, uint32_t stream_id, uint32_t t,
                                        uint32_t p, unsigned long long *d_counts, void *cuda_stream)
{
    clear_error();
    ising_status st = check_strip(d_rows, L, word_bits, row0, nrows);
    if (st != ISING_OK) return st;
    if (!valid_temperature(T)) return fail(ISING_ERR_INVALID, "T must be finite and > 0");
    if (stream_id >= (1u << 31)) return fail(ISING_ERR_INVALID, "stream_id must be < 2^31");
    if (p > 1) return fail(ISING_ERR_INVALID, "p must be 0 or 1");
    if (t == 0xFFFFFFFFu) return fail(ISING_ERR_INVALID, "sweep index 2^32 - 1 is reserved");
    HalfSweepArgs a{};
    a.spins = d_rows;
    a.L = L;
    a.rows = nrows + 2;
    a.first_row = 1;
    a.update_rows = nrows;
    a.y_offset = (int64_t)row0 - 1;
    a.key = make_round_keys(seed);
    a.thr4 = threshold_for(4.0, T);
    a.thr8 = threshold_for(8.0, T);
    a.t = t;
    a.p = p;
    a.c3 = (stream_id << 1) | p;
    a.acc = (p == 1) ? d_counts : nullptr;
    int dev = 0;
    cudaGetDevice(&dev);
    LaunchConfig cfg = plain_launch(default_launch(dev, L, word_bits));
    while (cfg.rows_per_item > 1 && nrows % cfg.rows_per_item != 0) cfg.rows_per_item >>= 1;
    const cudaError_t e = launch_half_sweep(a, cfg, (cudaStream_t)cuda_stream);
    if (e != cudaSuccess) return fail(ISING_ERR_CUDA, "strip step: %s", cudaGetErrorString(e));
    return ISING_OK;
}

ISING_API ising_status ising_strip_observables(uint64_t L, uint64_t n_up, uint64_t n_anti, int64_t *M, int64_t *E)
{
    clear_error();
    if (!M || !E) return fail(ISING_ERR_INVALID, "null output");
    // any lattice size: the strips may come from another implementation of the step
    if (L < 2 || L > (1ull << 20)) return fail(ISING_ERR_INVALID, "L must be in [2, 2^20]");
    const uint64_t N = L * L;
    if (n_up > N || n_anti > 2 * N) return fail(ISING_ERR_INVALID, "counts exceed the lattice");
    // M = (+1 spins) - (-1 spins); E = -(aligned bonds) + (anti-aligned bonds), 2N bonds
    *M = 2 * (int64_t)n_up - (int64_t)N;
    *E = 2 * (int64_t)n_anti - 2 * (int64_t)N;
    return ISING_OK;
}

}  // extern "C"

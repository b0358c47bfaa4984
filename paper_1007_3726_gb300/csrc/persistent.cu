// Every sweep of an ising_sweep call in one cooperative launch: the grid stays
// resident and a grid-wide barrier separates the checkerboard steps (Sec. 5.2
// needs one global synchronisation per step; the paper's CUDA had only the
// kernel boundary for it, a cooperative grid has a barrier).  For lattices whose
// step takes a few microseconds (L of a few thousand) the launch of each step
// is a large part of its time; here a step costs one barrier instead.
//
// The items of a step are those of the step kernel (half_sweep_items, the same
// geometry and the same word update); only the step arguments change from step
// to step, and each thread computes them from the sweep index (the step-uniform
// parts of Philox rounds 1 and 2, as prepare_half_sweep does on the host).
#include "kernels.h"
#include "sweep_device.cuh"

#include <cooperative_groups.h>

#include <atomic>

namespace ising {

namespace {

// The values of one step of the persistent kernel (the launch constants come
// from its launch arguments).
struct StepValues {
    uint32_t r1x0, r1x2k, r2x0k, r2x2k, r2x3;  // step-uniform Philox values (prepare_half_sweep)
    uint32_t p;                                 // parity of the updated sites
    unsigned long long *acc;                    // not null when this step counts
};

template <typename Word, int MINB>
__global__ void __launch_bounds__(512, MINB) k_sweeps(const __grid_constant__ HalfSweepArgs a,
                                                      const __grid_constant__ SweepsRun s)
{
    cooperative_groups::grid_group grid = cooperative_groups::this_grid();
    uint32_t phase = s.record_every ? s.t0 % s.record_every : 0u;  // t % record_every
    uint32_t slot = 0;
    for (uint32_t i = 0; i < s.nsweeps; ++i) {
        const uint32_t t = s.t0 + i;
        const bool rec = s.record_every != 0u && phase + 1 == s.record_every;
        const bool last = i + 1 == s.nsweeps;
        const uint64_t pb = (uint64_t)t * kPhiloxMulB;
        const uint32_t r1x0 = (uint32_t)(pb >> 32) ^ a.key.k0[0];
        const uint64_t pa = (uint64_t)r1x0 * kPhiloxMulA;
#pragma unroll 1
        for (uint32_t p = 0; p < 2; ++p) {
            const bool count = p == 1u && (rec || last);
            // a recorded sweep counts into its slot, the last one (also) into the final slot
            unsigned long long *const acc = count ? s.acc + 2 * (rec ? slot : s.nrec) : nullptr;
            const StepValues v{r1x0,
                               (s.c3base | p) ^ a.key.k1[0],
                               (uint32_t)pb ^ a.key.k0[1],
                               (uint32_t)(pa >> 32) ^ a.key.k1[1],
                               (uint32_t)pa,
                               p,
                               acc};
            unsigned int cu = 0, ca = 0;
            half_sweep_items<Word, 0>(a, v, cu, ca);
            if (count) {
                block_accumulate(cu, ca, acc);
                if (rec && last) {
                    __syncthreads();  // block_accumulate's shared scratch is reused
                    block_accumulate(cu, ca, s.acc + 2 * s.nrec);
                }
            }
            grid.sync();
        }
        if (rec) ++slot;
        if (s.record_every) phase = (phase + 1 == s.record_every) ? 0u : phase + 1;
    }
}

using SweepsKernel = void (*)(HalfSweepArgs, SweepsRun);

// regcap 0: the compiler's choice; 1: <= 40 registers; 2: <= 64 registers
SweepsKernel sweeps_kernel(const LaunchConfig &c)
{
    if (c.proc_bits == 64)
        return c.regcap == 1 ? k_sweeps<uint64_t, 3> : c.regcap == 2 ? k_sweeps<uint64_t, 2> : k_sweeps<uint64_t, 1>;
    return c.regcap == 1 ? k_sweeps<uint32_t, 3> : c.regcap == 2 ? k_sweeps<uint32_t, 2> : k_sweeps<uint32_t, 1>;
}

constexpr int kMaxDevices = 64;

}  // namespace

bool persistent_config_valid(const LaunchConfig &c, uint64_t L, uint64_t rows)
{
    if (c.persistent != 1 || c.insert != 0 || c.regcap > 2 || c.grid != 0) return false;
    LaunchConfig step = c;
    step.persistent = 0;
    step.regcap = 0;
    return rows == L && launch_config_valid(step, L, rows);
}

cudaError_t launch_sweeps(HalfSweepArgs a, const LaunchConfig &c, const SweepsRun &s, cudaStream_t st)
{
    if (c.persistent != 1 || s.nsweeps == 0) return cudaErrorInvalidValue;
    const SweepsKernel kern = sweeps_kernel(c);
    // every block resident at once (a cooperative launch): blocks per SM of this
    // kernel and block size, queried once per device and shape
    static std::atomic<int> per_sm_of[kMaxDevices][2][3][3];
    int dev = 0, sms = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    const int bi = c.block == 128 ? 0 : c.block == 256 ? 1 : 2;
    std::atomic<int> *slot = (dev >= 0 && dev < kMaxDevices)
                                 ? &per_sm_of[dev][c.proc_bits == 64][c.regcap][bi]
                                 : nullptr;
    int per_sm = slot ? slot->load(std::memory_order_relaxed) : 0;
    if (per_sm <= 0) {
        const cudaError_t e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, (int)c.block, 0);
        if (e != cudaSuccess) return e;
        if (per_sm <= 0) return cudaErrorInvalidConfiguration;
        if (slot) slot->store(per_sm, std::memory_order_relaxed);
    }
    a.rows = a.L;
    a.first_row = 0;
    a.update_rows = a.L;
    a.y_offset = 0;
    a.words_per_row = (uint32_t)(a.L / c.proc_bits);
    a.rows_per_item = c.rows_per_item;
    a.zero = 0u;
    const uint64_t items = a.L / c.rows_per_item * a.words_per_row;
    const uint64_t need = (items + c.block - 1) / c.block;
    const uint64_t cap = (uint64_t)(sms > 0 ? sms : 1) * (uint64_t)per_sm;
    const int grid = (int)(need < cap ? need : cap);
    prepare_half_sweep(a, grid, (int)c.block);
    void *args[] = {&a, const_cast<SweepsRun *>(&s)};
    return cudaLaunchCooperativeKernel((const void *)kern, dim3((unsigned)grid), dim3(c.block), args, 0, st);
}

}  // namespace ising

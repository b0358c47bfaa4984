// Host runtime pieces shared by the translation units of libising (error
// text, allocator hook, thresholds, parameter validation).
#pragma once

#include "ising.h"

#include <cstddef>
#include <cstdint>
#include <cuda_runtime.h>
#include <nvtx3/nvToolsExt.h>

namespace ising {

// An NVTX range for the lifetime of the object (visible in Nsight timelines;
// without a tool attached a push / pop costs a few nanoseconds).
struct NvtxRange {
    explicit NvtxRange(const char *name) { nvtxRangePushA(name); }
    ~NvtxRange() { nvtxRangePop(); }
    NvtxRange(const NvtxRange &) = delete;
    NvtxRange &operator=(const NvtxRange &) = delete;
};

// Sets the calling thread's last-error text and returns st.
ising_status fail(ising_status st, const char *fmt, ...);
void clear_error();

// Device allocator in force when a handle is created (cudaMalloc by default,
// or the hook installed with ising_set_allocator).
struct Allocator {
    ising_alloc_fn alloc = nullptr;
    ising_free_fn free_fn = nullptr;
    void *ctx = nullptr;
    void *allocate(size_t bytes, cudaStream_t s) const;
    void release(void *p, cudaStream_t s) const;
};
Allocator current_allocator();

// floor(2^32 exp(-dE / T)), clamped to [0, 2^32 - 1].
uint32_t threshold_for(double dE, double T);
bool valid_temperature(double T);

ising_status validate_params(const ising_params *p, uint32_t *word_bits);

}  // namespace ising

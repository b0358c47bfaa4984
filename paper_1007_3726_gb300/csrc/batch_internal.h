// The batch object behind the opaque ising_batch of include/ising.h, shared
// with the request server (server.cu), which re-plans one batch per epoch.
#pragma once

#include "handle.h"
#include "kernels.h"
#include "runtime.h"

#include <vector>

namespace ising {
struct BatchStrip;
struct BatchLaunchArgs {
    const BatchStrip *strips;
    const uint32_t *cta_first;          // strips of CTA b: cta_strips[cta_first[b] .. cta_first[b + 1])
    const uint32_t *cta_strips;
    const uint32_t *t0;                 // first sweep index of each lattice in this launch
    uint32_t max_steps;
    uint32_t rows_per_item;
    uint32_t max_strips;                // table entries per CTA
    uint32_t table_words;               // 64-bit words of the tables before the strips' rows
    unsigned int *error_flag;           // set to 1 when a wait ran out
    long long wait_cycles;              // clock limit of one wait
    uint32_t hold_strip;                // 1 + index of a strip that never publishes (0 = none)
};
}  // namespace ising

struct ising_batch {
    std::vector<ising_lattice *> hs;
    std::vector<uint64_t> sweeps;           // per lattice per run
    std::vector<uint32_t> record_every;     // per lattice
    ising_batch_opts opts{};
    int device = 0;
    cudaStream_t stream = nullptr;
    ising::Allocator alloc;
    // plan
    std::vector<ising::BatchStrip> strips;
    std::vector<uint32_t> cta_first, cta_strips;
    uint32_t grid = 0, block = 512, max_steps = 0, max_strips = 0, table_words = 0;
    size_t smem_bytes = 0;
    std::vector<size_t> sample_base;        // first slot of each lattice in the counters
    std::vector<size_t> nrec;               // sample slots of each lattice per run (the most a run can record)
    size_t slots = 0;                       // recorded slots + one final slot per lattice
    // device memory
    void *d_plan = nullptr;                 // strips, cta_first, cta_strips, t0
    size_t plan_bytes = 0, plan_cap = 0;
    void *d_work = nullptr;                 // borders, progress, counters, error flag
    size_t work_bytes = 0, work_cap = 0;
    size_t off_progress = 0, off_counters = 0, off_error = 0, off_t0 = 0;
    size_t progress_bytes = 0;
    unsigned long long *h_counters = nullptr;  // pinned
    size_t counters_cap = 0;                   // slots
    uint32_t *h_t0 = nullptr;                  // pinned
    size_t t0_cap = 0;
    unsigned int *h_error = nullptr;           // pinned
    cudaEvent_t ev = nullptr;
    bool own_stream = false;
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t graph_exec = nullptr;
    ising::BatchLaunchArgs args{};
    bool field = false;                     // a lattice is in a field: the field kernel
    bool failed = false;
};


namespace ising {
// An empty batch on a device with its own stream.
ising_status batch_new(int device, const ising_batch_opts *opts, ising_batch **out);
// (Re)plans the batch for these handles, sweeps per run and sample spacing,
// reusing its device and pinned buffers when they are large enough.
ising_status batch_replan(ising_batch *b, const std::vector<ising_lattice *> &hs,
                          const std::vector<uint64_t> &sweeps, const std::vector<uint32_t> &record_every);
// Bytes of lattice rows the batch's CTAs can hold at once (upper bound).
size_t batch_capacity_bytes(ising_batch *b);
void batch_free(ising_batch *b);
}  // namespace ising

// The lattice handle behind the opaque ising_lattice of include/ising.h.
#pragma once

#include "ising.h"
#include "field.h"
#include "kernels.h"
#include "runtime.h"

#include <cstdint>
#include <vector>

struct ising_lattice {
    uint64_t L = 0;
    double T = 0;
    uint64_t seed = 0;
    uint32_t stream_id = 0;
    uint32_t word_bits = 32;
    uint32_t W = 0;  // words per row
    uint32_t thr4 = 0, thr8 = 0;
    double H = 0;                // external field; nonzero runs the field kernel
    ising::FieldTable field{};   // its class thresholds at (T, H)
    size_t bytes = 0;
    int device = 0;
    cudaStream_t stream = nullptr;
    ising::Allocator alloc;
    void *d_base = nullptr;   // the allocation: guard, lattice, guard
    void *d_spins = nullptr;  // the lattice, kGuardBytes into d_base
    unsigned long long *d_acc = nullptr;  // 2 counters per slot
    unsigned long long *h_acc = nullptr;  // pinned mirror
    size_t acc_slots = 0;
    cudaEvent_t ev = nullptr;
    ising::RoundKeys key{};
    ising::LaunchConfig launch{};
    uint64_t sweeps_done = 0;
    int64_t M = 0, E = 0;
    std::vector<int64_t> sM, sE;
    // samples of the last queued call, read back at the next synchronising call
    bool pending = false;
    size_t pending_rec = 0;  // recorded slots of that call
    bool pending_err = false;  // slot pending_rec + 1 holds a kernel's error flag
    bool failed = false;
};


namespace ising {
// Guard bytes before and after every lattice allocation, filled with
// kGuardByte; ising_check_guards tells whether they are still intact.
constexpr size_t kGuardBytes = 256;
constexpr unsigned char kGuardByte = 0xA5;

// Launch configuration for a new handle: the autotuned one for (device, L,
// word width) if there is one, else a fixed default.
LaunchConfig default_launch(int device, uint64_t L, uint32_t word_bits);
void remember_launch(int device, uint64_t L, uint32_t word_bits, const LaunchConfig &c);
std::vector<LaunchConfig> launch_candidates(uint64_t L, uint64_t rows);

// Shared by the ABI translation units.
int64_t to_M(const ising_lattice *h, unsigned long long up);
int64_t to_E(const ising_lattice *h, unsigned long long anti);
ising_status cuda_fail(ising_lattice *h, cudaError_t e, const char *what);
ising_status check_live(ising_lattice *h);     // not failed; its device made current
ising_status harvest(ising_lattice *h);        // read back the last queued call's samples
ising_status ensure_acc(ising_lattice *h, size_t slots);
// The end of ising_sweep once its kernels are queued: the counters' read-back
// and the sweep count; with M_out, the call's samples.
ising_status finish_sweep_call(ising_lattice *h, uint64_t t0, uint64_t nsweeps, uint64_t nrec, int64_t *M_out,
                               int64_t *E_out);
}  // namespace ising

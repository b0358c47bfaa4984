// The checkerboard step in a nonzero field H (field.cu); internal to libising.
#pragma once

#include "kernels.h"
#include "runtime.h"

#include <cstdint>
#include <cuda_runtime.h>

namespace ising {

// Acceptance per site class (S, c), S the spin (index 0 for -1, 1 for +1) and
// c = 0 .. 4 its anti-aligned neighbours: thr[8 i + c] = floor(2^32 exp(-dE/T))
// for dE = 2 S (n + H) > 0 (n the neighbour sum), 0 where dE <= 0; those
// always-accepted classes are c >= k_up for S = +1 and c >= k_dn for S = -1
// (5 = none).  Entries 5 .. 7 and 13 .. 15 are unused (0).
struct FieldTable {
    uint32_t thr[16];
    uint32_t k_up, k_dn;
};

FieldTable make_field_table(double T, double H);

// One checkerboard step of a whole periodic lattice in a field; a as for
// launch_half_sweep (spins, L, key, t, c3, p, acc; the rest is filled here).
cudaError_t launch_half_sweep_field(HalfSweepArgs a, const FieldTable &ft, cudaStream_t s);

}  // namespace ising

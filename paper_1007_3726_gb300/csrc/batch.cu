// Persistent multi-lattice sweep: many lattices of uneven size in one launch.
//
// Each lattice is cut into strips of rows; every CTA keeps its strips in
// shared memory for the whole launch and walks through the checkerboard steps
// (Sec. 3) of all of them.  A strip needs its neighbours' boundary rows before
// each step: a lattice held by one strip wraps around inside the CTA; strips
// of a lattice spread over several CTAs exchange their boundary rows through
// small border arrays in global memory (the own / neighbour border arrays of
// the paper's multi-GPU scheme, Sec. 6.1, here between CTAs of one GPU), and a
// strip waits only until its two neighbours have published the previous step
// (a point-to-point dependency, not a global barrier).  All CTAs are resident
// at once (cooperative launch), every wait has a clock limit after which the
// launch sets an error flag and returns.  The arithmetic of a site update is
// the same device code as the one-lattice kernel, so every lattice, sample and
// final state is bit-identical to ising_sweep's.
#include "batch_internal.h"
#include "field_device.cuh"
#include "handle.h"
#include "kernels.h"
#include "runtime.h"
#include "sweep_device.cuh"

#include <algorithm>
#include <cstring>
#include <numeric>
#include <string>
#include <vector>

using namespace ising;

namespace ising {

// One strip of one lattice (device-visible plan entry).
struct BatchStrip {
    uint64_t *lat;                      // the lattice, rows of W 64-bit words
    uint64_t *border;                   // [2 buffers][top, bottom][W] words (multi-strip only)
    unsigned int *progress;             // steps this strip has completed (multi-strip only)
    unsigned long long *samples;        // the lattice's recorded counters [n][2]
    unsigned long long *final_counts;   // the lattice's counters after its last sweep [2]
    uint64_t L;
    uint32_t W;                         // 64-bit words per row
    uint32_t row0, nrows;               // the strip's rows
    uint32_t up_strip, dn_strip;        // plan indices of the neighbouring strips
    uint32_t nstrips_lat;               // strips of this lattice
    uint32_t smem_off;                  // first word of the strip's buffer in shared memory
    uint32_t lat_index;                 // lattice index in the batch
    uint32_t nsteps;                    // 2 x sweeps of this launch
    uint32_t record_every;
    uint32_t thr4, thr8, c3base;        // thresholds, stream_id << 1
    const unsigned int *up_progress, *dn_progress;  // the neighbouring strips' progress
    const uint64_t *up_border, *dn_border;          // and border arrays
    const uint32_t *field_tab;          // in a field: the lattice's 16 class thresholds (else null)
    uint32_t k_up, k_dn;                // and its always-accepted classes (field.h)
    RoundKeys key;
};


namespace {

constexpr uint32_t kFlagTimeout = 1u;

__device__ __forceinline__ unsigned int load_acquire(const unsigned int *p)
{
    unsigned int v;
    asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}

__device__ __forceinline__ void store_release(unsigned int *p, unsigned int v)
{
    asm volatile("st.release.gpu.global.u32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}

// Thread 0 waits (bounded) until the neighbours of every multi-strip strip of
// this CTA have completed `need` steps; the result is broadcast to the CTA.
// Returns false when a wait ran out or another CTA reported a failure.
__device__ bool wait_neighbours(const BatchLaunchArgs &A, const BatchStrip *sst, uint32_t ns, uint32_t s)
{
    __shared__ int ok;
    if (threadIdx.x == 0) {
        int good = 1;
        const long long start = clock64();
        for (uint32_t k = 0; k < ns && good; ++k) {
            const BatchStrip &st = sst[k];
            if (st.nstrips_lat == 1 || s >= st.nsteps) continue;
            unsigned int ns_sleep = 32;
            while (!(load_acquire(st.up_progress) >= s && load_acquire(st.dn_progress) >= s)) {
                if (*(volatile unsigned int *)A.error_flag != 0u || clock64() - start > A.wait_cycles) {
                    atomicOr(A.error_flag, kFlagTimeout);
                    good = 0;
                    break;
                }
                __nanosleep(ns_sleep);
                if (ns_sleep < 1024) ns_sleep <<= 1;
            }
        }
        ok = good;
    }
    __syncthreads();
    const bool r = ok != 0;
    __syncthreads();
    return r;
}

// Step-uniform Philox values of (t, p) for a strip (cf. prepare_half_sweep).
__device__ __forceinline__ void strip_step_args(HalfSweepArgs &a, const BatchStrip &st, uint32_t t,
                                                uint32_t p)
{
    a.key = st.key;
    a.thr4 = st.thr4;
    a.thr8 = st.thr8;
    a.t = t;
    a.p = p;
    a.c3 = st.c3base | p;
    const uint64_t pb = (uint64_t)t * kPhiloxMulB;
    a.r1x0 = (uint32_t)(pb >> 32) ^ st.key.k0[0];
    a.r1x2k = a.c3 ^ st.key.k1[0];
    a.r2x0k = (uint32_t)pb ^ st.key.k0[1];
    const uint64_t pa = (uint64_t)a.r1x0 * kPhiloxMulA;
    a.r2x2k = (uint32_t)(pa >> 32) ^ st.key.k1[1];
    a.r2x3 = (uint32_t)pa;
    a.zero = 0u;
}

constexpr uint32_t kMaxStripsPerCta = 64;

// INS = kFieldIns: the kernel of batches that hold a lattice in a field.  It
// picks the ten-class field update for the strips of such lattices (class
// table read through the read-only cache) and the plain update for the others.
// A separate kernel, so that the field code costs the other batches nothing.
constexpr int kFieldIns = 3;

// The new value of one word (or of this thread's bytes of it) of a strip.
template <int INS, int NQ>
__device__ __forceinline__ uint64_t batch_word(const BatchStrip &st, const HalfSweepArgs &a, uint64_t cur,
                                               uint64_t up, uint64_t dn, uint64_t lw, uint64_t rw, uint32_t off,
                                               uint64_t g, bool count, unsigned int &cu, unsigned int &ca,
                                               uint32_t sub)
{
    if constexpr (INS == kFieldIns) {
        if (st.field_tab)
            return update_word_field<uint64_t, NQ, true>(a, a, st.field_tab, st.k_up, st.k_dn, cur, up, dn, lw, rw,
                                                         off, g, count, cu, ca, sub * NQ);
        return update_word<uint64_t, 0, NQ>(a, a, cur, up, dn, lw, rw, off, g, count, cu, ca, sub * NQ);
    } else {
        return update_word<uint64_t, INS, NQ>(a, a, cur, up, dn, lw, rw, off, g, count, cu, ca, sub * NQ);
    }
}

// One item of a strip: R rows of one word column, or of one NQ-byte part of it
// when 8 / NQ threads share the word (each writes only its own bytes).
template <int INS, int NQ>
__device__ __forceinline__ void batch_item(const BatchStrip &st, const HalfSweepArgs &a, uint32_t li,
                                           uint32_t R, uint32_t p, bool count, unsigned int &cu,
                                           unsigned int &ca)
{
    extern __shared__ uint64_t sm[];
    constexpr uint32_t S = 8 / NQ;
    const uint32_t W = st.W;
    const uint32_t sub = (S == 1) ? 0u : (li & (S - 1));
    const uint32_t rest = (S == 1) ? li : (li / S);  // S is a power of two: a shift
    // words per row are a power of two for power-of-two L: a shift, else a division
    const uint32_t rb = ((W & (W - 1)) == 0) ? (rest >> (31 - __clz(W))) : rest / W;
    const uint32_t w = rest - rb * W;
    const uint32_t wl = (w == 0) ? W - 1 : w - 1;
    const uint32_t wr = (w + 1 == W) ? 0 : w + 1;
    const uint32_t r0 = rb * R, r1 = min(r0 + R, st.nrows);
    uint64_t *row = sm + st.smem_off + (uint64_t)(r0 + 1) * W;
    uint64_t up = row[w - (uint64_t)W];
    uint64_t cur = row[w];
    const uint64_t groups_per_row = st.L >> 3;
    const uint64_t y0 = (uint64_t)st.row0 + r0;
    uint64_t g = y0 * groups_per_row + (uint64_t)w * 8u;
    uint32_t off = (uint32_t)((y0 + p) & 1u);
    for (uint32_t r = r0; r < r1; ++r) {
        const uint64_t dn = row[W + w];
        const uint64_t nw = batch_word<INS, NQ>(st, a, cur, up, dn, row[wl], row[wr], off, g, count, cu, ca, sub);
        if (NQ == 8) {
            row[w] = nw;
        } else if (NQ == 4) {
            reinterpret_cast<uint32_t *>(row + w)[sub] = (uint32_t)(nw >> (32 * sub));
        } else if (NQ == 2) {
            reinterpret_cast<uint16_t *>(row + w)[sub] = (uint16_t)(nw >> (16 * sub));
        } else {
            reinterpret_cast<uint8_t *>(row + w)[sub] = (uint8_t)(nw >> (8 * sub));
        }
        up = nw;  // only bits of the other parity are read from it in the next row
        cur = dn;
        row += W;
        g += groups_per_row;
        off ^= 1u;
    }
}

// A CTA that holds one whole lattice (the lattice fits its shared memory and
// has no neighbour strips): the step arguments stay in registers, the periodic
// wrap is done by indexing instead of halo copies, and each step needs one
// barrier (plus one when the step is counted).
template <int INS, int NQ>
__device__ __forceinline__ void whole_item(const BatchStrip &st, const HalfSweepArgs &a, uint32_t li,
                                           uint32_t R, uint32_t p, bool count, unsigned int &cu,
                                           unsigned int &ca)
{
    extern __shared__ uint64_t sm[];
    constexpr uint32_t S = 8 / NQ;
    const uint32_t W = st.W, nrows = st.nrows;
    const uint32_t sub = (S == 1) ? 0u : (li & (S - 1));
    const uint32_t rest = (S == 1) ? li : (li / S);
    const uint32_t rb = ((W & (W - 1)) == 0) ? (rest >> (31 - __clz(W))) : rest / W;
    const uint32_t w = rest - rb * W;
    const uint32_t wl = (w == 0) ? W - 1 : w - 1;
    const uint32_t wr = (w + 1 == W) ? 0 : w + 1;
    const uint32_t r0 = rb * R, r1 = min(r0 + R, nrows);  // R is a power of two
    uint64_t *const base = sm + st.smem_off + W;  // row 0 of the lattice
    uint64_t *row = base + (uint64_t)r0 * W;
    uint64_t up = base[(uint64_t)(r0 == 0 ? nrows - 1 : r0 - 1) * W + w];
    uint64_t cur = row[w];
    const uint64_t groups_per_row = st.L >> 3;
    uint64_t g = (uint64_t)r0 * groups_per_row + (uint64_t)w * 8u;
    uint32_t off = (r0 + p) & 1u;
    for (uint32_t r = r0; r < r1; ++r) {
        const uint64_t *dnrow = (r + 1 == nrows) ? base : row + W;
        const uint64_t dn = dnrow[w];
        const uint64_t nw = batch_word<INS, NQ>(st, a, cur, up, dn, row[wl], row[wr], off, g, count, cu, ca, sub);
        if (NQ == 8) {
            row[w] = nw;
        } else if (NQ == 4) {
            reinterpret_cast<uint32_t *>(row + w)[sub] = (uint32_t)(nw >> (32 * sub));
        } else if (NQ == 2) {
            reinterpret_cast<uint16_t *>(row + w)[sub] = (uint16_t)(nw >> (16 * sub));
        } else {
            reinterpret_cast<uint8_t *>(row + w)[sub] = (uint8_t)(nw >> (8 * sub));
        }
        up = nw;
        cur = dn;
        row += W;
        g += groups_per_row;
        off ^= 1u;
    }
}

template <int INS>
__device__ void whole_lattices_steps(const BatchLaunchArgs &A, const BatchStrip *sst, const uint32_t *st0,
                                     const uint32_t *strip_R, const uint32_t *strip_S, uint32_t *rec_phase,
                                     uint32_t *rec_slot, unsigned int (*cnt)[2], uint32_t ns)
{
    const uint32_t tid = threadIdx.x, nthr = blockDim.x;
    if (tid < ns) {
        cnt[tid][0] = 0u;
        cnt[tid][1] = 0u;
    }
    __syncthreads();
    for (uint32_t s = 0; s < A.max_steps; ++s) {
        const uint32_t p = s & 1u;
        for (uint32_t k = 0; k < ns; ++k) {
            const BatchStrip &st = sst[k];
            if (s >= st.nsteps) continue;
            const uint32_t t = st0[k] + (s >> 1);
            HalfSweepArgs a;
            strip_step_args(a, st, t, p);
            const bool recorded = p == 1u && st.record_every != 0u && rec_phase[k] == 0u;
            const bool count = p == 1u && (recorded || s + 1 == st.nsteps);
            const uint32_t R = strip_R[k], S = strip_S[k];
            const uint32_t lr = 31 - __clz(R);  // R and S are powers of two
            const uint32_t items = ((st.nrows + R - 1) >> lr) * st.W * S;
            unsigned int cu = 0, ca = 0;
            switch (S) {
            case 1:
                for (uint32_t li = tid; li < items; li += nthr) whole_item<INS, 8>(st, a, li, R, p, count, cu, ca);
                break;
            case 2:
                for (uint32_t li = tid; li < items; li += nthr) whole_item<INS, 4>(st, a, li, R, p, count, cu, ca);
                break;
            case 4:
                for (uint32_t li = tid; li < items; li += nthr) whole_item<INS, 2>(st, a, li, R, p, count, cu, ca);
                break;
            default:
                for (uint32_t li = tid; li < items; li += nthr) whole_item<INS, 1>(st, a, li, R, p, count, cu, ca);
                break;
            }
            if (count) {
                cu = __reduce_add_sync(0xFFFFFFFFu, cu);
                ca = __reduce_add_sync(0xFFFFFFFFu, ca);
                if ((tid & 31u) == 0 && (cu | ca)) {
                    atomicAdd(&cnt[k][0], cu);
                    atomicAdd(&cnt[k][1], ca);
                }
            }
        }
        __syncthreads();
        if (p == 1u && tid < ns) {
            // the counters of this step to the lattice's slots (the next counted
            // step is two steps and at least one barrier away), and the next sweep
            const BatchStrip &st = sst[tid];
            if (s < st.nsteps) {
                const unsigned long long c0 = cnt[tid][0], c1 = cnt[tid][1];
                if (st.record_every != 0u && rec_phase[tid] == 0u) {
                    const uint32_t k = rec_slot[tid]++;
                    atomicAdd(st.samples + 2 * k, c0);
                    atomicAdd(st.samples + 2 * k + 1, c1);
                }
                if (s + 1 == st.nsteps) {
                    atomicAdd(st.final_counts, c0);
                    atomicAdd(st.final_counts + 1, c1);
                }
                cnt[tid][0] = 0u;
                cnt[tid][1] = 0u;
                if (st.record_every != 0u) rec_phase[tid] = (rec_phase[tid] + 1 == st.record_every) ? 0u : rec_phase[tid] + 1;
            }
        }
    }
    __syncthreads();
}

// Each step has four phases: wait for the neighbour strips of the previous
// step, fill the halo rows of all strips, update all strips (one flat loop
// over the (strip, row block, word) items of the CTA, so that small lattices
// share the CTA's threads), then add the counters and publish the boundary
// rows.
template <int INS>
__global__ void __launch_bounds__(512, 2) k_batch(const __grid_constant__ BatchLaunchArgs A)
{
    extern __shared__ uint64_t sm[];  // per-strip tables (A.table_words), then the strips' rows
    __shared__ int cta_multi;         // does any strip exchange borders
    const uint32_t MS = A.max_strips;
    BatchStrip *sst = reinterpret_cast<BatchStrip *>(sm);                 // the CTA's strip descriptors
    HalfSweepArgs *sargs = reinterpret_cast<HalfSweepArgs *>(sst + MS);   // their step arguments
    uint32_t *item_end = reinterpret_cast<uint32_t *>(sargs + MS);       // prefix sums of their items
    uint32_t *strip_R = item_end + MS;                                    // rows per item
    uint32_t *strip_S = strip_R + MS;                                     // threads sharing one word
    uint32_t *st0 = strip_S + MS;                                         // first sweep index
    uint32_t *rec_phase = st0 + MS;   // (t + 1) mod record_every of the sweep in progress
    uint32_t *rec_slot = rec_phase + MS;  // the sample slot of the next recorded sweep
    unsigned int (*cnt)[2] = reinterpret_cast<unsigned int (*)[2]>(rec_slot + MS);  // step counters
    __shared__ uint8_t scount[kMaxStripsPerCta];       // does the strip count in this step
    const uint32_t first = A.cta_first[blockIdx.x], last = A.cta_first[blockIdx.x + 1];
    const uint32_t ns = last - first;
    const uint32_t tid = threadIdx.x, nthr = blockDim.x;
    if (tid == 0) cta_multi = 0;
    __syncthreads();
    if (tid < ns) {
        sst[tid] = A.strips[A.cta_strips[first + tid]];
        st0[tid] = A.t0[sst[tid].lat_index];
        const uint32_t re = sst[tid].record_every;
        rec_phase[tid] = re ? (st0[tid] + 1) % re : 1u;
        rec_slot[tid] = 0u;
        if (sst[tid].nstrips_lat > 1) atomicOr(&cta_multi, 1);
    }
    __syncthreads();

    // the strips' rows into shared memory (row r of a strip at buffer row r + 1)
    for (uint32_t j = 0; j < ns; ++j) {
        const BatchStrip &st = sst[j];
        const uint64_t n = (uint64_t)st.nrows * st.W;
        const uint64_t *src = st.lat + (uint64_t)st.row0 * st.W;
        uint64_t *dst = sm + st.smem_off + st.W;
        for (uint64_t i = tid; i < n; i += nthr) dst[i] = src[i];
    }
    if (tid == 0) {
        for (uint32_t k = 0; k < ns; ++k) {
            const BatchStrip &st = sst[k];
            // enough items for every thread when the strip is small: fewer rows
            // per item first, then fewer Philox calls per thread
            uint32_t R = 1u << (31 - __clz(A.rows_per_item | 1u)), S = 1;  // a power of two
            while (R > 1 && (uint64_t)((st.nrows + R - 1) / R) * st.W < nthr) R >>= 1;
            while (S < 8 && (uint64_t)((st.nrows + R - 1) / R) * st.W * S < nthr) S <<= 1;
            strip_R[k] = R;
            strip_S[k] = S;
        }
    }
    __syncthreads();

    if (!cta_multi) {
        // only whole lattices in this CTA: no halos, no neighbours
        whole_lattices_steps<INS>(A, sst, st0, strip_R, strip_S, rec_phase, rec_slot, cnt, ns);
    } else
    for (uint32_t s = 0; s < A.max_steps; ++s) {
        const uint32_t p = s & 1u;
        // 1. neighbours of the previous step
        if (s > 0 && cta_multi && !wait_neighbours(A, sst, ns, s)) return;
        // 2. halo rows, and the item ranges of this step
        for (uint32_t k = 0; k < ns; ++k) {
            const BatchStrip &st = sst[k];
            if (s >= st.nsteps) continue;
            const uint32_t W = st.W, nrows = st.nrows;
            uint64_t *buf = sm + st.smem_off;
            if (st.nstrips_lat == 1) {
                for (uint32_t i = tid; i < W; i += nthr) {
                    buf[i] = buf[(uint64_t)nrows * W + i];              // row nrows-1 above row 0
                    buf[(uint64_t)(nrows + 1) * W + i] = buf[W + i];    // row 0 below row nrows-1
                }
            } else if (s == 0) {
                const uint64_t ya = (st.row0 == 0) ? st.L - 1 : st.row0 - 1;
                const uint64_t yb = (st.row0 + nrows == st.L) ? 0 : st.row0 + nrows;
                for (uint32_t i = tid; i < W; i += nthr) {
                    buf[i] = __ldcg(st.lat + ya * W + i);
                    buf[(uint64_t)(nrows + 1) * W + i] = __ldcg(st.lat + yb * W + i);
                }
            } else {
                const uint32_t pb = (s - 1) & 1u;
                const uint64_t *bu = st.up_border + (uint64_t)(2 * pb + 1) * W;  // its bottom row
                const uint64_t *bd = st.dn_border + (uint64_t)(2 * pb + 0) * W;  // its top row
                for (uint32_t i = tid; i < W; i += nthr) {
                    buf[i] = __ldcg(bu + i);
                    buf[(uint64_t)(nrows + 1) * W + i] = __ldcg(bd + i);
                }
            }
        }
        if (tid < ns) {
            const BatchStrip &st = sst[tid];
            if (s < st.nsteps) {
                const uint32_t t = st0[tid] + (s >> 1);
                HalfSweepArgs a;
                strip_step_args(a, st, t, p);
                sargs[tid] = a;
                const bool recorded = p == 1u && st.record_every != 0u && (t + 1) % st.record_every == 0u;
                scount[tid] = (p == 1u && (recorded || s + 1 == st.nsteps)) ? 1 : 0;
            }
            cnt[tid][0] = 0u;
            cnt[tid][1] = 0u;
        }
        if (tid == 0) {
            uint32_t acc = 0;
            for (uint32_t k = 0; k < ns; ++k) {
                const BatchStrip &st = sst[k];
                if (s < st.nsteps) acc += ((st.nrows + strip_R[k] - 1) / strip_R[k]) * st.W * strip_S[k];
                item_end[k] = acc;
            }
        }
        __syncthreads();

        // 3. the updates
        const uint32_t total = ns ? item_end[ns - 1] : 0u;
        uint32_t k = 0, kbase = 0;
        uint32_t kc = 0xFFFFFFFFu;  // the strip whose counts cu / ca hold
        bool count = false;
        unsigned int cu = 0, ca = 0;
        for (uint32_t item = tid; item < total; item += nthr) {
            while (item >= item_end[k]) {
                kbase = item_end[k];
                ++k;
            }
            const BatchStrip &st = sst[k];
            if (k != kc) {
                if (count && (cu | ca)) {
                    atomicAdd(&cnt[kc][0], cu);
                    atomicAdd(&cnt[kc][1], ca);
                }
                cu = ca = 0;
                kc = k;
                count = scount[k] != 0;
            }
            const HalfSweepArgs &a = sargs[k];
            const uint32_t li = item - kbase;
            switch (strip_S[k]) {
            case 1: batch_item<INS, 8>(st, a, li, strip_R[k], p, count, cu, ca); break;
            case 2: batch_item<INS, 4>(st, a, li, strip_R[k], p, count, cu, ca); break;
            case 4: batch_item<INS, 2>(st, a, li, strip_R[k], p, count, cu, ca); break;
            default: batch_item<INS, 1>(st, a, li, strip_R[k], p, count, cu, ca); break;
            }
        }
        {
            // warp-aggregated: one shared atomic per strip present in the warp
            const uint32_t key = (count && (cu | ca)) ? kc : 0xFFFFFFFFu;
            unsigned int rem = __ballot_sync(0xFFFFFFFFu, key != 0xFFFFFFFFu);
            while (rem) {
                const int leader = __ffs(rem) - 1;
                const uint32_t kk = __shfl_sync(0xFFFFFFFFu, key, leader);
                const bool mine = key == kk;
                const unsigned int su = __reduce_add_sync(0xFFFFFFFFu, mine ? cu : 0u);
                const unsigned int sa = __reduce_add_sync(0xFFFFFFFFu, mine ? ca : 0u);
                if ((int)(tid & 31u) == leader) {
                    atomicAdd(&cnt[kk][0], su);
                    atomicAdd(&cnt[kk][1], sa);
                }
                rem &= ~__ballot_sync(0xFFFFFFFFu, mine);
            }
        }
        __syncthreads();

        // 4. counters to the lattices' slots, boundary rows to the neighbours
        if (tid < ns) {
            const BatchStrip &st = sst[tid];
            if (s < st.nsteps && p == 1u) {
                const uint32_t t = st0[tid] + (s >> 1);
                const bool recorded = st.record_every != 0u && (t + 1) % st.record_every == 0u;
                if (recorded) {
                    const uint32_t slot = (t + 1) / st.record_every - st0[tid] / st.record_every - 1;
                    atomicAdd(st.samples + 2 * slot, (unsigned long long)cnt[tid][0]);
                    atomicAdd(st.samples + 2 * slot + 1, (unsigned long long)cnt[tid][1]);
                }
                if (s + 1 == st.nsteps) {
                    atomicAdd(st.final_counts, (unsigned long long)cnt[tid][0]);
                    atomicAdd(st.final_counts + 1, (unsigned long long)cnt[tid][1]);
                }
            }
        }
        bool any_multi = false;
        for (uint32_t kk = 0; kk < ns; ++kk) {
            const BatchStrip &st = sst[kk];
            if (st.nstrips_lat == 1 || s >= st.nsteps) continue;
            any_multi = true;
            const uint32_t W = st.W, nrows = st.nrows;
            const uint64_t *buf = sm + st.smem_off;
            uint64_t *bo = st.border + (uint64_t)(2 * p) * W;
            for (uint32_t i = tid; i < W; i += nthr) {
                __stcg(bo + i, buf[W + i]);                           // top row
                __stcg(bo + W + i, buf[(uint64_t)nrows * W + i]);     // bottom row
            }
        }
        if (any_multi) {
            __threadfence();
            __syncthreads();
            if (tid == 0) {
                for (uint32_t kk = 0; kk < ns; ++kk) {
                    const uint32_t si = A.cta_strips[first + kk];
                    const BatchStrip &st = sst[kk];
                    if (st.nstrips_lat == 1 || s >= st.nsteps || A.hold_strip == si + 1) continue;
                    store_release(st.progress, s + 1);
                }
            }
        }
        __syncthreads();
    }

    // the strips back to the lattices
    for (uint32_t j = 0; j < ns; ++j) {
        const BatchStrip &st = sst[j];
        const uint64_t n = (uint64_t)st.nrows * st.W;
        uint64_t *dst = st.lat + (uint64_t)st.row0 * st.W;
        const uint64_t *src = sm + st.smem_off + st.W;
        for (uint64_t i = tid; i < n; i += nthr) dst[i] = src[i];
    }
}

}  // namespace
}  // namespace ising

namespace {
using namespace ising;
using BatchKernel = void (*)(BatchLaunchArgs);
BatchKernel batch_kernel(uint32_t insert, bool field)
{
    if (field) return k_batch<kFieldIns>;
    if (insert == 1) return k_batch<1>;
    if (insert == 2) return k_batch<2>;
    return k_batch<0>;
}

}  // namespace

// ------------------------------------------------------------------ host ---
namespace {

// Bytes of the per-strip tables at the start of the kernel's shared memory.
size_t table_entry_bytes() { return sizeof(BatchStrip) + sizeof(HalfSweepArgs) + 6 * 4 + 2 * 4; }
size_t table_bytes(size_t max_strips) { return (max_strips * table_entry_bytes() + 15) & ~(size_t)15; }

ising_status bfail(ising_batch *b, cudaError_t e, const char *what)
{
    if (b) {
        b->failed = true;
        for (ising_lattice *h : b->hs) h->failed = true;
    }
    return fail(ISING_ERR_CUDA, "%s: %s", what, cudaGetErrorString(e));
}

void free_batch(ising_batch *b)
{
    if (!b) return;
    cudaSetDevice(b->device);
    cudaStreamSynchronize(b->stream);
    if (b->graph_exec) cudaGraphExecDestroy(b->graph_exec);
    if (b->graph) cudaGraphDestroy(b->graph);
    b->alloc.release(b->d_plan, b->stream);
    b->alloc.release(b->d_work, b->stream);
    if (b->h_counters) cudaFreeHost(b->h_counters);
    if (b->h_t0) cudaFreeHost(b->h_t0);
    if (b->h_error) cudaFreeHost(b->h_error);
    if (b->ev) cudaEventDestroy(b->ev);
    if (b->own_stream && b->stream) cudaStreamDestroy(b->stream);
    delete b;
}

// Splits every lattice into strips and assigns them to CTAs (largest work
// first, to the least loaded CTA with room in shared memory).
// CTAs of a plan and the dynamic shared memory each can give to strips.
void plan_budget(const ising_batch *b, uint32_t *P_out, size_t *smem_cta_out)
{
    const int dev = b->device;
    int sms = 0, smem_optin = 0, smem_sm = 0;
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    cudaDeviceGetAttribute(&smem_optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
    cudaDeviceGetAttribute(&smem_sm, cudaDevAttrMaxSharedMemoryPerMultiprocessor, dev);
    const uint32_t block = b->opts.block ? b->opts.block : 512;
    uint32_t ctas_per_sm = b->opts.ctas_per_sm ? b->opts.ctas_per_sm : 2;
    {
        // no more CTAs per SM than the registers allow
        int occ = 0;
        if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, batch_kernel(b->opts.insert, b->field), (int)block, 0) ==
                cudaSuccess &&
            occ > 0)
            ctas_per_sm = std::min<uint32_t>(ctas_per_sm, (uint32_t)occ);
    }
    // dynamic shared memory per CTA: the SM's share, less the kernel's static
    // tables and the 1 KiB the runtime reserves per block
    cudaFuncAttributes fa{};
    cudaFuncGetAttributes(&fa, (const void *)batch_kernel(b->opts.insert, b->field));
    const size_t reserve = fa.sharedSizeBytes + 1024;
    size_t smem_cta = (size_t)smem_sm / ctas_per_sm;
    smem_cta = smem_cta > reserve ? smem_cta - reserve : 0;
    smem_cta = std::min<size_t>(smem_cta, (size_t)smem_optin > fa.sharedSizeBytes
                                              ? (size_t)smem_optin - fa.sharedSizeBytes
                                              : 0);
    *P_out = (uint32_t)(sms > 0 ? sms : 1) * ctas_per_sm;
    *smem_cta_out = smem_cta;
}

ising_status make_plan(ising_batch *b)
{
    b->block = b->opts.block ? b->opts.block : 512;
    uint32_t P = 0;
    size_t smem_cta = 0;
    plan_budget(b, &P, &smem_cta);
    if (P == 0 || smem_cta == 0) return fail(ISING_ERR_CUDA, "no multiprocessors or shared memory");
    const size_t n = b->hs.size();
    double total = 0;
    for (size_t i = 0; i < n; ++i) total += (double)b->hs[i]->L * b->hs[i]->L * b->sweeps[i];
    const double target = total / P;

    struct S {
        uint32_t lat, row0, nrows;
        double work;
        size_t bytes;
    };
    std::vector<S> parts;
    std::vector<uint32_t> first_part(n), nparts(n);
    std::vector<std::vector<uint32_t>> assigned;
    // Packing can fail on fragmentation although the total fits: retry with
    // strips of at most half, a quarter, ... of a CTA's shared memory.
    bool packed = false;
    for (int attempt = 0; attempt < 6 && !packed; ++attempt) {
        const size_t strip_cap = smem_cta >> attempt;
        parts.clear();
        bool fits = true;
        for (size_t i = 0; i < n && fits; ++i) {
            const uint64_t L = b->hs[i]->L;
            const size_t row_bytes = L / 8;
            const double work = (double)L * L * b->sweeps[i];
            uint64_t G = (uint64_t)std::max(1.0, std::round(work / std::max(target, 1.0)));
            // a strip must fit in shared memory with its two halo rows
            const uint64_t max_rows = strip_cap / row_bytes > 2 ? strip_cap / row_bytes - 2 : 0;
            if (max_rows == 0) {
                fits = false;
                break;
            }
            // a strip's step must outweigh the cost of a border exchange: at least
            // 2^17 sites per strip unless shared memory forces a finer split
            G = std::min<uint64_t>(G, std::max<uint64_t>(1, L * L / (1ull << 17)));
            G = std::max<uint64_t>(G, (L + max_rows - 1) / max_rows);
            G = std::min<uint64_t>(G, L / 2);
            first_part[i] = (uint32_t)parts.size();
            nparts[i] = (uint32_t)G;
            for (uint64_t k = 0; k < G; ++k) {
                const uint64_t r0 = L * k / G, r1 = L * (k + 1) / G;
                parts.push_back(S{(uint32_t)i, (uint32_t)r0, (uint32_t)(r1 - r0),
                                  work * (double)(r1 - r0) / (double)L,
                                  (r1 - r0 + 2) * row_bytes + table_entry_bytes()});
            }
        }
        if (!fits) break;
        // largest first onto the least-loaded CTA with room
        std::vector<uint32_t> order(parts.size());
        std::iota(order.begin(), order.end(), 0u);
        std::stable_sort(order.begin(), order.end(),
                         [&](uint32_t x, uint32_t y) { return parts[x].work > parts[y].work; });
        std::vector<double> load(P, 0.0);
        std::vector<size_t> used(P, 0);
        assigned.assign(P, {});
        packed = true;
        for (uint32_t pi : order) {
            int best = -1;
            for (uint32_t c = 0; c < P; ++c) {
                if (used[c] + parts[pi].bytes > smem_cta) continue;
                if (assigned[c].size() >= kMaxStripsPerCta) continue;
                if (best < 0 || load[c] < load[best]) best = (int)c;
            }
            if (best < 0) {
                packed = false;
                break;
            }
            load[best] += parts[pi].work;
            used[best] += parts[pi].bytes;
            assigned[best].push_back(pi);
        }
        if (packed) {
            // every CTA gets a table of the largest CTA's strip count
            size_t ms = 0, rows_max = 0;
            for (uint32_t c = 0; c < P; ++c) {
                ms = std::max(ms, assigned[c].size());
                size_t r = 0;
                for (uint32_t pi : assigned[c]) r += parts[pi].bytes - table_entry_bytes();
                rows_max = std::max(rows_max, r);
            }
            if (table_bytes(ms) + rows_max > smem_cta) packed = false;
        }
    }
    if (!packed)
        return fail(ISING_ERR_INVALID,
                    "the batch needs more shared memory than the GPU has (%zu bytes per CTA, %u CTAs)",
                    smem_cta, P);
    // keep only CTAs with work; strips of a CTA in lattice/row order
    b->strips.assign(parts.size(), BatchStrip{});
    b->cta_first.clear();
    b->cta_strips.clear();
    size_t max_strips = 0;
    for (uint32_t c = 0; c < P; ++c) max_strips = std::max(max_strips, assigned[c].size());
    b->max_strips = (uint32_t)max_strips;
    b->table_words = (uint32_t)(table_bytes(max_strips) / 8);
    size_t smem_max = 0;
    for (uint32_t c = 0; c < P; ++c) {
        if (assigned[c].empty()) continue;
        std::sort(assigned[c].begin(), assigned[c].end());
        b->cta_first.push_back((uint32_t)b->cta_strips.size());
        size_t off_words = b->table_words;
        for (uint32_t pi : assigned[c]) {
            b->cta_strips.push_back(pi);
            b->strips[pi].smem_off = (uint32_t)off_words;
            off_words += (parts[pi].bytes - table_entry_bytes()) / 8;
        }
        smem_max = std::max(smem_max, off_words * 8);
    }
    b->cta_first.push_back((uint32_t)b->cta_strips.size());
    b->grid = (uint32_t)(b->cta_first.size() - 1);
    b->smem_bytes = smem_max;

    // strip descriptors (device pointers filled in after allocation)
    b->max_steps = 0;
    b->nrec.assign(n, 0);
    b->sample_base.assign(n, 0);
    size_t slot = 0;
    for (size_t i = 0; i < n; ++i) {
        ising_lattice *h = b->hs[i];
        const uint64_t t0 = h->sweeps_done, ns = b->sweeps[i];
        (void)t0;
        // at most ceil(ns / record_every) samples in any run of ns sweeps
        const uint64_t re = b->record_every[i];
        b->nrec[i] = re ? (ns + re - 1) / re : 0;
        b->sample_base[i] = slot;
        slot += b->nrec[i] + 1;  // + the final slot
        b->max_steps = std::max<uint32_t>(b->max_steps, (uint32_t)(2 * ns));
    }
    b->slots = slot;
    for (size_t pi = 0; pi < parts.size(); ++pi) {
        const S &q = parts[pi];
        ising_lattice *h = b->hs[q.lat];
        BatchStrip &st = b->strips[pi];
        st.L = h->L;
        st.W = (uint32_t)(h->L / 64);
        st.row0 = q.row0;
        st.nrows = q.nrows;
        const uint32_t k = (uint32_t)(pi - first_part[q.lat]), G = nparts[q.lat];
        st.up_strip = first_part[q.lat] + (k + G - 1) % G;
        st.dn_strip = first_part[q.lat] + (k + 1) % G;
        st.nstrips_lat = G;
        st.lat_index = q.lat;
        st.nsteps = (uint32_t)(2 * b->sweeps[q.lat]);
        st.record_every = b->record_every[q.lat];
        st.thr4 = h->thr4;
        st.thr8 = h->thr8;
        st.c3base = h->stream_id << 1;
        st.key = h->key;
    }
    return ISING_OK;
}

ising_status alloc_batch(ising_batch *b)
{
    const size_t n = b->hs.size();
    const size_t ns = b->strips.size();
    // plan block: strips | cta_first | cta_strips | t0
    size_t off = 0;
    const size_t off_strips = off;
    off += ns * sizeof(BatchStrip);
    off = (off + 15) & ~(size_t)15;
    const size_t off_first = off;
    off += b->cta_first.size() * 4;
    off = (off + 15) & ~(size_t)15;
    const size_t off_cstr = off;
    off += b->cta_strips.size() * 4;
    off = (off + 15) & ~(size_t)15;
    b->off_t0 = off;
    off += n * 4;
    off = (off + 15) & ~(size_t)15;
    const size_t off_field = off;  // 16 class thresholds per lattice (used by lattices in a field)
    off += n * 64;
    b->plan_bytes = (off + 255) & ~(size_t)255;
    // work block: borders | progress | counters | error
    size_t w = 0;
    std::vector<size_t> border_off(ns, 0);
    for (size_t i = 0; i < ns; ++i) {
        if (b->strips[i].nstrips_lat > 1) {
            border_off[i] = w;
            w += 4ull * b->strips[i].W * 8;
        }
    }
    w = (w + 255) & ~(size_t)255;
    b->off_progress = w;
    b->progress_bytes = ns * 4;
    w += b->progress_bytes;
    w = (w + 255) & ~(size_t)255;
    b->off_counters = w;
    w += b->slots * 16;
    w = (w + 255) & ~(size_t)255;
    b->off_error = w;
    w += 256;
    b->work_bytes = w;

    // reuse the buffers of an earlier plan when they are large enough
    auto grow = [](size_t need, size_t cap) { return need <= cap ? cap : std::max(need, cap + cap / 2); };
    if (b->plan_bytes > b->plan_cap) {
        cudaStreamSynchronize(b->stream);
        b->alloc.release(b->d_plan, b->stream);
        b->plan_cap = grow(b->plan_bytes, b->plan_cap);
        b->d_plan = b->alloc.allocate(b->plan_cap, b->stream);
        if (!b->d_plan) b->plan_cap = 0;
    }
    if (b->work_bytes > b->work_cap) {
        cudaStreamSynchronize(b->stream);
        b->alloc.release(b->d_work, b->stream);
        b->work_cap = grow(b->work_bytes, b->work_cap);
        b->d_work = b->alloc.allocate(b->work_cap, b->stream);
        if (!b->d_work) b->work_cap = 0;
    }
    if (!b->d_plan || !b->d_work) return fail(ISING_ERR_OOM, "cannot allocate the batch plan");
    bool host_ok = true;
    if (b->slots > b->counters_cap) {
        if (b->h_counters) cudaFreeHost(b->h_counters);
        b->h_counters = nullptr;
        b->counters_cap = grow(b->slots, b->counters_cap);
        host_ok = cudaHostAlloc((void **)&b->h_counters, b->counters_cap * 16, cudaHostAllocDefault) == cudaSuccess;
    }
    if (host_ok && std::max<size_t>(n, 1) > b->t0_cap) {
        if (b->h_t0) cudaFreeHost(b->h_t0);
        b->h_t0 = nullptr;
        b->t0_cap = grow(std::max<size_t>(n, 1), b->t0_cap);
        host_ok = cudaHostAlloc((void **)&b->h_t0, b->t0_cap * 4, cudaHostAllocDefault) == cudaSuccess;
    }
    if (host_ok && !b->h_error) host_ok = cudaHostAlloc((void **)&b->h_error, 16, cudaHostAllocDefault) == cudaSuccess;
    if (!host_ok) {
        cudaGetLastError();
        b->counters_cap = b->h_counters ? b->counters_cap : 0;
        b->t0_cap = b->h_t0 ? b->t0_cap : 0;
        return fail(ISING_ERR_OOM, "cannot allocate pinned host memory for the batch");
    }
    char *work = static_cast<char *>(b->d_work);
    for (size_t i = 0; i < ns; ++i) {
        BatchStrip &st = b->strips[i];
        ising_lattice *h = b->hs[st.lat_index];
        st.lat = static_cast<uint64_t *>(h->d_spins);
        st.border = st.nstrips_lat > 1 ? reinterpret_cast<uint64_t *>(work + border_off[i]) : nullptr;
        st.progress = reinterpret_cast<unsigned int *>(work + b->off_progress) + i;
        st.samples = reinterpret_cast<unsigned long long *>(work + b->off_counters) +
                     2 * b->sample_base[st.lat_index];
        st.final_counts = st.samples + 2 * b->nrec[st.lat_index];
        st.field_tab = h->H != 0.0 ? reinterpret_cast<const uint32_t *>(static_cast<char *>(b->d_plan) + off_field) +
                                         16 * st.lat_index
                                   : nullptr;
        st.k_up = h->field.k_up;
        st.k_dn = h->field.k_dn;
    }
    for (size_t i = 0; i < ns; ++i) {
        BatchStrip &st = b->strips[i];
        st.up_progress = b->strips[st.up_strip].progress;
        st.dn_progress = b->strips[st.dn_strip].progress;
        st.up_border = b->strips[st.up_strip].border;
        st.dn_border = b->strips[st.dn_strip].border;
    }
    std::vector<char> host(b->plan_bytes, 0);
    std::memcpy(host.data() + off_strips, b->strips.data(), ns * sizeof(BatchStrip));
    std::memcpy(host.data() + off_first, b->cta_first.data(), b->cta_first.size() * 4);
    std::memcpy(host.data() + off_cstr, b->cta_strips.data(), b->cta_strips.size() * 4);
    for (size_t i = 0; i < n; ++i)
        std::memcpy(host.data() + off_field + 64 * i, b->hs[i]->field.thr, 64);
    cudaError_t e = cudaMemcpyAsync(b->d_plan, host.data(), b->plan_bytes, cudaMemcpyHostToDevice, b->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(b->stream);
    if (e != cudaSuccess) return bfail(b, e, "batch plan upload");

    char *plan = static_cast<char *>(b->d_plan);
    b->args.strips = reinterpret_cast<const BatchStrip *>(plan + off_strips);
    b->args.cta_first = reinterpret_cast<const uint32_t *>(plan + off_first);
    b->args.cta_strips = reinterpret_cast<const uint32_t *>(plan + off_cstr);
    b->args.t0 = reinterpret_cast<const uint32_t *>(plan + b->off_t0);
    b->args.max_steps = b->max_steps;
    b->args.rows_per_item = b->opts.rows_per_item ? b->opts.rows_per_item : 4;
    b->args.max_strips = b->max_strips;
    b->args.table_words = b->table_words;
    b->args.error_flag = reinterpret_cast<unsigned int *>(work + b->off_error);
    const double ms = b->opts.wait_ms > 0 ? b->opts.wait_ms : 2000.0;
    int clk_khz = 0;
    cudaDeviceGetAttribute(&clk_khz, cudaDevAttrClockRate, b->device);
    b->args.wait_cycles = (long long)(ms * (clk_khz > 0 ? clk_khz : 2000000));
    b->args.hold_strip = b->opts.hold_strip;
    e = cudaFuncSetAttribute(batch_kernel(b->opts.insert, b->field), cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)b->smem_bytes);
    if (e != cudaSuccess) return bfail(b, e, "batch shared memory");
    // every CTA must be resident at once
    int per_sm = 0;
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, batch_kernel(b->opts.insert, b->field), (int)b->block,
                                                      b->smem_bytes);
    int sms = 0;
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, b->device);
    if (e != cudaSuccess) return bfail(b, e, "batch occupancy");
    if ((uint64_t)per_sm * (uint64_t)sms < b->grid)
        return fail(ISING_ERR_INVALID, "batch plan needs %u resident CTAs, the GPU holds %d",
                    b->grid, per_sm * sms);
    return ISING_OK;
}

// Work of one run on the batch stream: clear the counters, progress and error
// flag, copy the lattices' first sweep indices, launch, copy the counters and
// the error flag back.
cudaError_t enqueue_run(ising_batch *b)
{
    char *work = static_cast<char *>(b->d_work);
    cudaError_t e = cudaMemsetAsync(work + b->off_progress, 0, b->work_bytes - b->off_progress, b->stream);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(static_cast<char *>(b->d_plan) + b->off_t0, b->h_t0, b->hs.size() * 4,
                            cudaMemcpyHostToDevice, b->stream);
    if (e != cudaSuccess) return e;
    void *params[] = {&b->args};
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeCooperative;
    attr[0].val.cooperative = 1;
    cudaLaunchConfig_t cfg{};
    cfg.gridDim = dim3(b->grid);
    cfg.blockDim = dim3(b->block);
    cfg.dynamicSmemBytes = b->smem_bytes;
    cfg.stream = b->stream;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    e = cudaLaunchKernelExC(&cfg, (const void *)batch_kernel(b->opts.insert, b->field), params);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(b->h_counters, work + b->off_counters, b->slots * 16, cudaMemcpyDeviceToHost,
                            b->stream);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(b->h_error, work + b->off_error, 4, cudaMemcpyDeviceToHost, b->stream);
    return e;
}

}  // namespace

namespace ising {

ising_status batch_new(int device, const ising_batch_opts *opts, ising_batch **out)
{
    *out = nullptr;
    ising_batch *b = new (std::nothrow) ising_batch();
    if (!b) return fail(ISING_ERR_OOM, "host allocation failed");
    if (opts) b->opts = *opts;
    if (b->opts.block != 0 && b->opts.block != 128 && b->opts.block != 256 && b->opts.block != 512) {
        delete b;
        return fail(ISING_ERR_INVALID, "block must be 128, 256 or 512");
    }
    if (b->opts.insert > 2 || b->opts.rows_per_item > 64) {
        delete b;
        return fail(ISING_ERR_INVALID, "bad batch options");
    }
    b->device = device;
    b->alloc = current_allocator();
    // a stream of the batch's own (the legacy default stream cannot be captured)
    if (cudaStreamCreateWithFlags(&b->stream, cudaStreamNonBlocking) != cudaSuccess) {
        cudaGetLastError();
        delete b;
        return fail(ISING_ERR_CUDA, "stream creation failed");
    }
    b->own_stream = true;
    if (cudaEventCreateWithFlags(&b->ev, cudaEventDisableTiming) != cudaSuccess) {
        cudaGetLastError();
        batch_free(b);
        return fail(ISING_ERR_CUDA, "event creation failed");
    }
    *out = b;
    return ISING_OK;
}

ising_status batch_replan(ising_batch *b, const std::vector<ising_lattice *> &hs,
                          const std::vector<uint64_t> &sweeps, const std::vector<uint32_t> &record_every)
{
    if (b->failed) return fail(ISING_ERR_STATE, "batch failed earlier");
    const size_t n = hs.size();
    if (n == 0 || sweeps.size() != n || record_every.size() != n)
        return fail(ISING_ERR_INVALID, "empty batch");
    for (size_t i = 0; i < n; ++i) {
        ising_status st = check_live(hs[i]);
        if (st != ISING_OK) return st;
        if (hs[i]->device != b->device) return fail(ISING_ERR_INVALID, "handles on different devices");
        if (sweeps[i] == 0 || sweeps[i] > (1u << 30))
            return fail(ISING_ERR_INVALID, "sweeps per run must be in [1, 2^30]");
        if ((st = harvest(hs[i])) != ISING_OK) return st;
    }
    cudaStreamSynchronize(b->stream);
    if (b->graph_exec) cudaGraphExecDestroy(b->graph_exec);
    if (b->graph) cudaGraphDestroy(b->graph);
    b->graph_exec = nullptr;
    b->graph = nullptr;
    b->hs = hs;
    b->sweeps = sweeps;
    b->record_every = record_every;
    b->field = std::any_of(hs.begin(), hs.end(), [](const ising_lattice *h) { return h->H != 0.0; });
    ising_status st = make_plan(b);
    if (st == ISING_OK) st = alloc_batch(b);
    if (st != ISING_OK) b->hs.clear();
    return st;
}

void batch_free(ising_batch *b) { free_batch(b); }

size_t batch_capacity_bytes(ising_batch *b)
{
    uint32_t P = 0;
    size_t smem_cta = 0;
    plan_budget(b, &P, &smem_cta);
    return (size_t)P * smem_cta;
}

}  // namespace ising

extern "C" {

ISING_API ising_status ising_batch_create(ising_lattice *const *hs, uint32_t n, const uint64_t *nsweeps,
                                          uint32_t record_every, const ising_batch_opts *opts,
                                          ising_batch **out)
{
    clear_error();
    if (!out) return fail(ISING_ERR_INVALID, "out is NULL");
    *out = nullptr;
    if (!hs || !nsweeps || n == 0) return fail(ISING_ERR_INVALID, "empty batch");
    for (uint32_t i = 0; i < n; ++i) {
        ising_status st = check_live(hs[i]);
        if (st != ISING_OK) return st;
        for (uint32_t k = 0; k < i; ++k)
            if (hs[k] == hs[i]) return fail(ISING_ERR_INVALID, "a handle appears twice");
    }
    ising_batch *b = nullptr;
    ising_status st = batch_new(hs[0]->device, opts, &b);
    if (st != ISING_OK) return st;
    st = batch_replan(b, std::vector<ising_lattice *>(hs, hs + n), std::vector<uint64_t>(nsweeps, nsweeps + n),
                      std::vector<uint32_t>(n, record_every));
    if (st != ISING_OK) {
        std::string msg = ising_last_error();
        free_batch(b);
        fail(st, "%s", msg.c_str());
        return st;
    }
    *out = b;
    return ISING_OK;
}

ISING_API ising_status ising_batch_run(ising_batch *b, uint32_t runs)
{
    NvtxRange range("ising_batch_run");
    clear_error();
    if (!b) return fail(ISING_ERR_INVALID, "null batch");
    if (b->failed) return fail(ISING_ERR_STATE, "batch failed earlier");
    if (b->hs.empty()) return fail(ISING_ERR_STATE, "batch has no plan");
    cudaError_t e = cudaSetDevice(b->device);
    if (e != cudaSuccess) return bfail(b, e, "cudaSetDevice");
    const size_t n = b->hs.size();
    for (uint32_t r = 0; r < runs; ++r) {
        for (size_t i = 0; i < n; ++i) {
            ising_lattice *h = b->hs[i];
            ising_status st = check_live(h);
            if (st != ISING_OK) return st;
            if ((st = harvest(h)) != ISING_OK) return st;
            if (h->sweeps_done + b->sweeps[i] >= 0xFFFFFFFFull)
                return fail(ISING_ERR_INVALID, "sweep counter would reach 2^32 - 1");
            b->h_t0[i] = (uint32_t)h->sweeps_done;
            // the lattice's own stream must be done with it first
            if (h->stream != b->stream) {
                if ((e = cudaEventRecord(h->ev, h->stream)) != cudaSuccess) return bfail(b, e, "event");
                if ((e = cudaStreamWaitEvent(b->stream, h->ev, 0)) != cudaSuccess) return bfail(b, e, "wait");
            }
        }
        if (b->opts.use_graph) {
            if (!b->graph_exec) {
                e = cudaStreamBeginCapture(b->stream, cudaStreamCaptureModeThreadLocal);
                if (e == cudaSuccess) {
                    cudaError_t e2 = enqueue_run(b);
                    e = cudaStreamEndCapture(b->stream, &b->graph);
                    if (e2 != cudaSuccess) e = e2;
                }
                if (e == cudaSuccess) e = cudaGraphInstantiate(&b->graph_exec, b->graph, 0);
                if (e != cudaSuccess) return bfail(b, e, "batch graph capture");
            }
            e = cudaGraphLaunch(b->graph_exec, b->stream);
        } else {
            e = enqueue_run(b);
        }
        if (e == cudaSuccess) e = cudaEventRecord(b->ev, b->stream);
        if (e == cudaSuccess) e = cudaEventSynchronize(b->ev);
        if (e != cudaSuccess) return bfail(b, e, "batch run");
        if (*b->h_error != 0u) {
            b->failed = true;
            for (ising_lattice *h : b->hs) h->failed = true;
            return fail(ISING_ERR_TIMEOUT, "a strip waited longer than the limit; the lattices are lost");
        }
        for (size_t i = 0; i < n; ++i) {
            ising_lattice *h = b->hs[i];
            const unsigned long long *c = b->h_counters + 2 * b->sample_base[i];
            const uint64_t t0 = h->sweeps_done, re = b->record_every[i];
            const size_t got = re ? (size_t)((t0 + b->sweeps[i]) / re - t0 / re) : 0;
            for (size_t k = 0; k < got; ++k) {
                h->sM.push_back(to_M(h, c[2 * k]));
                h->sE.push_back(to_E(h, c[2 * k + 1]));
            }
            h->M = to_M(h, c[2 * b->nrec[i]]);
            h->E = to_E(h, c[2 * b->nrec[i] + 1]);
            h->sweeps_done += b->sweeps[i];
        }
    }
    return ISING_OK;
}

ISING_API ising_status ising_batch_info(const ising_batch *b, uint32_t *grid, uint32_t *block,
                                        uint32_t *strips, size_t *smem_bytes)
{
    clear_error();
    if (!b) return fail(ISING_ERR_INVALID, "null batch");
    if (grid) *grid = b->grid;
    if (block) *block = b->block;
    if (strips) *strips = (uint32_t)b->strips.size();
    if (smem_bytes) *smem_bytes = b->smem_bytes;
    return ISING_OK;
}

ISING_API ising_status ising_batch_destroy(ising_batch *b)
{
    clear_error();
    free_batch(b);
    return ISING_OK;
}

ISING_API ising_status ising_batch_tune(ising_lattice *const *hs, uint32_t n, const uint64_t *nsweeps,
                                        uint32_t probe_sweeps, ising_batch_opts *best, double *best_ms)
{
    clear_error();
    if (!best) return fail(ISING_ERR_INVALID, "best is NULL");
    if (!hs || !nsweeps || n == 0) return fail(ISING_ERR_INVALID, "empty batch");
    if (probe_sweeps == 0) probe_sweeps = 20;
    for (uint32_t i = 0; i < n; ++i) {
        ising_status st = check_live(hs[i]);
        if (st != ISING_OK) return st;
        if ((st = harvest(hs[i])) != ISING_OK) return st;
    }
    // the candidates are timed on the real lattices, which are saved first and
    // restored afterwards; the handles' counters and samples are not touched
    size_t total = 0;
    for (uint32_t i = 0; i < n; ++i) total += hs[i]->bytes;
    Allocator al = current_allocator();
    cudaStream_t s0 = hs[0]->stream;
    char *save = static_cast<char *>(al.allocate(total, s0));
    if (!save) return fail(ISING_ERR_OOM, "cannot allocate %zu bytes to save the lattices", total);
    cudaError_t e = cudaSuccess;
    size_t off = 0;
    for (uint32_t i = 0; i < n && e == cudaSuccess; ++i) {
        e = cudaMemcpyAsync(save + off, hs[i]->d_spins, hs[i]->bytes, cudaMemcpyDeviceToDevice,
                            hs[i]->stream);
        if (e == cudaSuccess) e = cudaStreamSynchronize(hs[i]->stream);
        off += hs[i]->bytes;
    }
    // probe sweeps in proportion to the requested ones (at least one each)
    uint64_t maxn = 1;
    for (uint32_t i = 0; i < n; ++i) maxn = std::max<uint64_t>(maxn, nsweeps[i]);
    std::vector<uint64_t> probe(n);
    for (uint32_t i = 0; i < n; ++i)
        probe[i] = std::max<uint64_t>(1, (uint64_t)((double)probe_sweeps * nsweeps[i] / maxn + 0.5));
    struct Cand {
        uint32_t block, ctas, rows;
    };
    const Cand cands[] = {{256, 4, 4}, {256, 4, 8}, {256, 3, 4}, {256, 2, 4}, {512, 2, 4},
                          {512, 2, 8}, {512, 1, 4}, {256, 8, 4}, {128, 8, 4}, {128, 16, 4}};
    double best_t = 1e300;
    bool found = false;
    cudaEvent_t t0 = nullptr, t1 = nullptr;
    if (e == cudaSuccess) e = cudaEventCreate(&t0);
    if (e == cudaSuccess) e = cudaEventCreate(&t1);
    for (const Cand &c : cands) {
        if (e != cudaSuccess) break;
        ising_batch_opts o = *best;
        o.block = c.block;
        o.ctas_per_sm = c.ctas;
        o.rows_per_item = c.rows;
        o.use_graph = 0;
        o.hold_strip = 0;
        ising_batch *b = nullptr;
        if (ising_batch_create(hs, n, probe.data(), 0, &o, &b) != ISING_OK) continue;  // plan does not fit
        for (uint32_t i = 0; i < n; ++i) b->h_t0[i] = (uint32_t)hs[i]->sweeps_done;
        float ms = 0;
        e = enqueue_run(b);  // warm-up
        if (e == cudaSuccess) e = cudaEventRecord(t0, b->stream);
        if (e == cudaSuccess) e = enqueue_run(b);
        if (e == cudaSuccess) e = cudaEventRecord(t1, b->stream);
        if (e == cudaSuccess) e = cudaEventSynchronize(t1);
        if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, t0, t1);
        const bool ok = e == cudaSuccess && *b->h_error == 0u;
        b->hs.clear();  // the handles are not part of the probe's failure
        free_batch(b);
        if (ok && ms < best_t) {
            best_t = ms;
            *best = o;
            found = true;
        }
    }
    if (t0) cudaEventDestroy(t0);
    if (t1) cudaEventDestroy(t1);
    off = 0;
    for (uint32_t i = 0; i < n; ++i) {
        cudaError_t e2 = cudaMemcpyAsync(hs[i]->d_spins, save + off, hs[i]->bytes,
                                         cudaMemcpyDeviceToDevice, hs[i]->stream);
        if (e2 == cudaSuccess) e2 = cudaStreamSynchronize(hs[i]->stream);
        if (e == cudaSuccess) e = e2;
        off += hs[i]->bytes;
    }
    al.release(save, s0);
    if (e != cudaSuccess) {
        for (uint32_t i = 0; i < n; ++i) hs[i]->failed = true;
        return fail(ISING_ERR_CUDA, "batch tuning: %s", cudaGetErrorString(e));
    }
    if (!found) return fail(ISING_ERR_INVALID, "no batch configuration fits the lattices");
    best->use_graph = 0;
    if (best_ms) *best_ms = best_t;
    return ISING_OK;
}

ISING_API ising_status ising_sweep_batch(ising_lattice *const *hs, uint32_t n, const uint64_t *nsweeps,
                                         uint32_t record_every)
{
    ising_batch *b = nullptr;
    ising_status st = ising_batch_create(hs, n, nsweeps, record_every, nullptr, &b);
    if (st != ISING_OK) return st;
    st = ising_batch_run(b, 1);
    std::string msg = ising_last_error();
    free_batch(b);
    if (st != ISING_OK) fail(st, "%s", msg.c_str());
    return st;
}

}  // extern "C"

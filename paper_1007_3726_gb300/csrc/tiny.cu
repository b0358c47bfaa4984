// Small lattices in one CTA: the whole lattice sits in shared memory for every
// sweep of a call, so a sweep costs two block barriers instead of two kernel
// launches (Sec. 5.2 needs one global synchronisation per checkerboard step;
// for a lattice that one CTA holds, a CTA barrier is that synchronisation).
//
// The lattice is kept as 32-bit words, W = L / 32 per row; a thread updates
// whole words with the word update of the step kernel (Sec. 4: neighbour words,
// bit-sliced count, one Philox4x32-10 call per byte of the word, masked XOR),
// so the neighbour logic is shared by the word's 16 target sites and its four
// Philox calls are independent chains.  For very small lattices S = 2 or 4
// threads share a word (each draws 4 / S of its calls and stores only its own
// bytes), so that more warps hide the latency of a step.  In a field H the
// word update is the ten-class one of field_device.cuh (one thread per word,
// the class thresholds in shared memory).  Bits a thread reads
// from its neighbours' words at its own target positions are of the other
// parity, which nobody writes during the step.
#include "field_device.cuh"
#include "kernels.h"
#include "sweep_device.cuh"

#include <cooperative_groups.h>

namespace ising {

namespace {

constexpr uint32_t kTinyMaxThreads = 512;

// Sweeps whose acceptance masks a thread draws in one burst when it holds a
// single word (the draw-ahead path below): 4 sweeps, 8 checkerboard steps.
constexpr uint32_t kAheadSweeps = 4;

// Samples the draw-ahead path collects in shared memory before it writes them
// to global memory in one go: a global write between two steps would make the
// next barrier (its release side) wait for the write to complete.
constexpr uint32_t kRingSamples = 64;

// The step-uniform Philox values of sweep t, parity p (as prepare_half_sweep).
__device__ __forceinline__ void tiny_step_values(HalfSweepArgs &a, const TinyRunArgs &A, uint32_t t, uint32_t p)
{
    const uint64_t pb = (uint64_t)t * kPhiloxMulB;
    a.r1x0 = (uint32_t)(pb >> 32) ^ A.key.k0[0];
    a.r2x0k = (uint32_t)pb ^ A.key.k0[1];
    const uint64_t pa = (uint64_t)a.r1x0 * kPhiloxMulA;
    a.r2x2k = (uint32_t)(pa >> 32) ^ A.key.k1[1];
    a.r2x3 = (uint32_t)pa;
    a.r1x2k = (A.c3base | p) ^ A.key.k1[0];
}

// The masks of this thread's bytes of its word (first Philox group g) for the
// 2 ns steps of sweeps t .. t + ns - 1, packed as pack_masks does.
template <int NQ>
__device__ __forceinline__ void tiny_draw_ahead(HalfSweepArgs &a, const TinyRunArgs &A, uint32_t t, uint32_t ns,
                                                uint64_t g, uint32_t q0, uint32_t (&pk)[2 * kAheadSweeps])
{
#pragma unroll
    for (uint32_t j = 0; j < 2 * kAheadSweeps; ++j) {
        if (j < 2 * ns) {
            tiny_step_values(a, A, t + (j >> 1), j & 1u);
            uint32_t h4[1], h8[1];
            word_draw_masks<4, 0, NQ>(a, a, g, h4, h8, q0);
            pk[j] = pack_masks(h4[0], h8[0]);
        }
    }
}

// Stores this thread's bytes of a new word.
template <int NQ>
__device__ __forceinline__ void tiny_store(uint32_t *word, uint32_t nw, uint32_t sub)
{
    if (NQ == 4)
        *word = nw;
    else if (NQ == 2)
        reinterpret_cast<uint16_t *>(word)[sub] = (uint16_t)(nw >> (16 * sub));
    else
        reinterpret_cast<uint8_t *>(word)[sub] = (uint8_t)(nw >> (8 * sub));
}

template <int NQ, bool FIELD>  // Philox calls (bytes) per thread: 4, 2 or 1; field update
__global__ void __launch_bounds__(kTinyMaxThreads) k_tiny(const __grid_constant__ TinyRunArgs A)
{
    static_assert(!FIELD || NQ == 4, "the field update takes whole words");
    constexpr uint32_t S = 4 / NQ;  // threads per word
    extern __shared__ uint32_t lat[];
    __shared__ unsigned int cnt[2];
    __shared__ uint32_t tab[16];
    if (FIELD && threadIdx.x < 16) tab[threadIdx.x] = A.field_thr[threadIdx.x];
    const uint32_t L = (uint32_t)A.L;
    const uint32_t W = L >> 5;                  // words per row, a power of two
    const uint32_t lgW = 31 - __clz(W);
    const uint32_t nwords = L * W;
    const uint32_t tid = threadIdx.x, nthr = blockDim.x;
    const uint64_t groups_per_row = L >> 3;

    const uint32_t *src = static_cast<const uint32_t *>(A.spins);
    for (uint32_t i = tid; i < nwords; i += nthr) lat[i] = src[i];
    if (tid < 2) cnt[tid] = 0u;
    __syncthreads();

    HalfSweepArgs a;
    a.key = A.key;
    a.thr4 = A.thr4;
    a.thr8 = A.thr8;
    a.zero = 0u;
    uint32_t phase = A.record_every ? A.t0 % A.record_every : 0u;  // t % record_every
    uint32_t slot = 0;
    if (!FIELD && nwords * S <= nthr) {
        // Draw-ahead path: every thread holds at most one word (or its share of
        // one).  The draws do not depend on the spins, so a thread keeps the
        // masks of its word for the next 2 kAheadSweeps steps in registers:
        // after each step's bit logic it draws the masks of the step that many
        // steps ahead, independent Philox chains that fill the issue slots the
        // step's dependent logic and the barrier leave idle.
        __shared__ unsigned int ring[2 * kRingSamples], lastc[2];
        uint32_t nring = 0;  // samples in the ring; the ring's first is sample `slot`
        const bool active = tid < nwords * S;
        const uint32_t k = active ? tid / S : 0u, sub = tid % S;
        const uint32_t y = k >> lgW, w = k & (W - 1u);
        const uint32_t row = k - w;
        const uint32_t iu = (y == 0 ? nwords - W : row - W) + w, id = (y + 1 == L ? 0u : row + W) + w;
        const uint32_t il = row + ((w - 1u) & (W - 1u)), ir = row + ((w + 1u) & (W - 1u));
        const uint64_t g = (uint64_t)y * groups_per_row + (uint64_t)w * 4u;
        uint32_t pk[2 * kAheadSweeps];
        if (active) tiny_draw_ahead<NQ>(a, A, A.t0, min(kAheadSweeps, A.nsweeps), g, sub * NQ, pk);
        for (uint32_t i0 = 0; i0 < A.nsweeps; i0 += kAheadSweeps) {
            const uint32_t ns = min(kAheadSweeps, A.nsweeps - i0);
#pragma unroll
            for (uint32_t j = 0; j < 2 * kAheadSweeps; ++j) {
                if (j >= 2 * ns) break;
                const uint32_t p = j & 1u;
                const bool rec = A.record_every != 0u && phase + 1 == A.record_every;
                const bool last = i0 + (j >> 1) + 1 == A.nsweeps;
                const bool count = p == 1u && (rec || last);
                unsigned int cu = 0, ca = 0;
                if (active) {
                    const uint32_t nw = update_word32_drawn<NQ>(lat[k], lat[iu], lat[id], lat[il], lat[ir],
                                                                (y + p) & 1u, pk[j], count, cu, ca, sub * NQ);
                    tiny_store<NQ>(lat + k, nw, sub);
                }
                if (count) {
                    cu = __reduce_add_sync(0xFFFFFFFFu, cu);
                    ca = __reduce_add_sync(0xFFFFFFFFu, ca);
                    if ((tid & 31u) == 0) {
                        atomicAdd(&cnt[0], cu);
                        atomicAdd(&cnt[1], ca);
                    }
                }
                // the masks of the same parity kAheadSweeps sweeps later
                const uint32_t ia = i0 + kAheadSweeps + (j >> 1);
                if (active && ia < A.nsweeps) {
                    tiny_step_values(a, A, A.t0 + ia, p);
                    uint32_t h4[1], h8[1];
                    word_draw_masks<4, 0, NQ>(a, a, g, h4, h8, sub * NQ);
                    pk[j] = pack_masks(h4[0], h8[0]);
                }
                __syncthreads();
                if (count && tid == 0) {
                    if (rec) {
                        ring[2 * nring] = cnt[0];
                        ring[2 * nring + 1] = cnt[1];
                    }
                    if (last) {
                        lastc[0] = cnt[0];
                        lastc[1] = cnt[1];
                    }
                    cnt[0] = 0u;
                    cnt[1] = 0u;
                }
                if (p == 1u) {
                    if (rec && ++nring == kRingSamples) {
                        // the ring is full: to global memory (the next counted
                        // step is two barriers away)
                        __syncthreads();
                        for (uint32_t r = tid; r < 2 * kRingSamples; r += nthr) A.acc[2 * slot + r] = ring[r];
                        slot += kRingSamples;
                        nring = 0;
                    }
                    if (A.record_every) phase = (phase + 1 == A.record_every) ? 0u : phase + 1;
                }
            }
        }
        __syncthreads();
        for (uint32_t r = tid; r < 2 * nring; r += nthr) A.acc[2 * slot + r] = ring[r];
        if (tid < 2) A.acc[2 * A.nrec + tid] = lastc[tid];
        uint32_t *dst = static_cast<uint32_t *>(A.spins);
        for (uint32_t i = tid; i < nwords; i += nthr) dst[i] = lat[i];
        return;
    }
    for (uint32_t i = 0; i < A.nsweeps; ++i) {
        const uint32_t t = A.t0 + i;
        const bool rec = A.record_every != 0u && phase + 1 == A.record_every;
        const bool last = i + 1 == A.nsweeps;
        // the step-uniform Philox values of sweep t (as prepare_half_sweep)
        const uint64_t pb = (uint64_t)t * kPhiloxMulB;
        a.r1x0 = (uint32_t)(pb >> 32) ^ A.key.k0[0];
        a.r2x0k = (uint32_t)pb ^ A.key.k0[1];
        const uint64_t pa = (uint64_t)a.r1x0 * kPhiloxMulA;
        a.r2x2k = (uint32_t)(pa >> 32) ^ A.key.k1[1];
        a.r2x3 = (uint32_t)pa;
#pragma unroll 1
        for (uint32_t p = 0; p < 2; ++p) {
            a.r1x2k = (A.c3base | p) ^ A.key.k1[0];
            const bool count = p == 1u && (rec || last);
            unsigned int cu = 0, ca = 0;
            for (uint32_t it = tid; it < nwords * S; it += nthr) {
                const uint32_t k = it / S, sub = it % S;  // S is a power of two
                const uint32_t y = k >> lgW, w = k & (W - 1u);
                const uint32_t row = k - w;
                const uint32_t cur = lat[k];
                const uint32_t up = lat[(y == 0 ? nwords - W : row - W) + w];
                const uint32_t dn = lat[(y + 1 == L ? 0u : row + W) + w];
                const uint32_t lw = lat[row + ((w - 1u) & (W - 1u))];
                const uint32_t rw = lat[row + ((w + 1u) & (W - 1u))];
                const uint64_t g = (uint64_t)y * groups_per_row + (uint64_t)w * 4u;
                const uint32_t nw =
                    FIELD ? update_word_field(a, a, tab, A.k_up, A.k_dn, cur, up, dn, lw, rw, (y + p) & 1u, g, count, cu, ca)
                          : update_word<uint32_t, 0, NQ>(a, a, cur, up, dn, lw, rw, (y + p) & 1u, g, count, cu, ca, sub * NQ);
                if (NQ == 4)
                    lat[k] = nw;
                else if (NQ == 2)
                    reinterpret_cast<uint16_t *>(lat + k)[sub] = (uint16_t)(nw >> (16 * sub));
                else
                    reinterpret_cast<uint8_t *>(lat + k)[sub] = (uint8_t)(nw >> (8 * sub));
            }
            if (count) {
                cu = __reduce_add_sync(0xFFFFFFFFu, cu);
                ca = __reduce_add_sync(0xFFFFFFFFu, ca);
                if ((tid & 31u) == 0) {
                    atomicAdd(&cnt[0], cu);
                    atomicAdd(&cnt[1], ca);
                }
            }
            __syncthreads();
            if (count && tid == 0) {
                // the next counted step is two steps and one barrier away
                const unsigned long long c0 = cnt[0], c1 = cnt[1];
                if (rec) {
                    A.acc[2 * slot] = c0;
                    A.acc[2 * slot + 1] = c1;
                }
                if (last) {
                    A.acc[2 * A.nrec] = c0;
                    A.acc[2 * A.nrec + 1] = c1;
                }
                cnt[0] = 0u;
                cnt[1] = 0u;
            }
        }
        if (rec) ++slot;
        if (A.record_every) phase = (phase + 1 == A.record_every) ? 0u : phase + 1;
    }
    __syncthreads();
    uint32_t *dst = static_cast<uint32_t *>(A.spins);
    for (uint32_t i = tid; i < nwords; i += nthr) dst[i] = lat[i];
}

// ---------------------------------------------------------------------------
// Warp-specialised one-CTA kernel for L = 64 (128 words of 32 bits).  With one
// SM for the whole lattice a step is short, and when every thread both draws
// and updates, the dependent bit logic and the barrier of each step leave most
// issue slots idle.  Here the roles are split:
//   warps 0-3   consumers: thread c updates word c at every step (the bit logic
//               with the masks read from shared memory, the store, the counts);
//   warps 4-31  producers: seven groups of 128 threads; group g draws the masks
//               of steps g, g + 7, g + 14, ... for word (thread index mod 128)
//               into a ring of kWsSlots steps in shared memory (seven steps in
//               flight give the Philox chains enough warps to hide their
//               latency).
// The masks do not depend on the spins, so the producers run ahead of the
// consumers by up to kWsSlots steps.  A ring entry is one 64-bit word, the
// masks and the tag s + 1 of their step, written with one store: the consumer
// of word c spins on its entry until the tag is there (a shared-memory load,
// short latency).  Having read it, the consumer arrives on the slot's "empty"
// mbarrier; the producers wait on that mbarrier before they reuse the slot
// (a suspended wait, so that waiting producers leave the issue slots to the
// consumers).  A named barrier of the consumers ends each step.  Every wait is
// bounded: when one runs out, the kernel sets `abort` (the consumers all stop
// after the same barrier, the producers leave) and *err, so the kernel always
// ends.
__device__ __forceinline__ uint32_t smem_addr(const void *p)
{
    return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}
__device__ __forceinline__ void mbar_init(uint64_t *bar, uint32_t count)
{
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_addr(bar)), "r"(count) : "memory");
}
__device__ __forceinline__ void mbar_arrive(uint64_t *bar)
{
    // the state token goes to the sink: no register waits for the arrival
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_addr(bar)) : "memory");
}
// Waits (bounded: at most `limit` polls, each of which may suspend the thread
// for a while without using issue slots) until the phase of the given parity
// has completed.
__device__ __forceinline__ bool mbar_wait(uint64_t *bar, uint32_t parity, uint32_t limit)
{
    const uint32_t a = smem_addr(bar);
    for (uint32_t i = 0; i < limit; ++i) {
        uint32_t done;
        asm volatile("{\n\t.reg .pred p;\n\tmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
                     "selp.u32 %0, 1, 0, p;\n\t}"
                     : "=r"(done)
                     : "r"(a), "r"(parity)
                     : "memory");
        if (done) return true;
    }
    return false;
}

constexpr uint32_t kWsSlots = 8;
constexpr uint32_t kWsWords = 128;
constexpr uint32_t kWsGroups = kTinyWsBlock / kWsWords - 1;  // producer groups (7)
constexpr uint32_t kWsSpinLimit = 1u << 24;  // polls of a consumer's wait before it gives up
constexpr uint32_t kWsWaitLimit = 1u << 20;  // polls of a producer's mbarrier wait

__global__ void __launch_bounds__(kTinyWsBlock) k_tiny_ws(const __grid_constant__ TinyRunArgs A)
{
    __shared__ uint32_t lat[kWsWords];
    __shared__ uint64_t entries[kWsSlots][kWsWords];  // (step + 1) << 32 | masks
    __shared__ __align__(8) uint64_t empty[kWsSlots];  // 128 consumer arrivals: the slot is read
    // per consumer warp (+1 spins, anti-aligned bonds) of up to kRingSamples
    // samples, and of the state after the last sweep
    __shared__ unsigned int wring[kRingSamples + 1][4][2], ws_abort;
    volatile uint64_t *const ve = &entries[0][0];
    volatile unsigned int *const vabort = &ws_abort;
    const uint32_t tid = threadIdx.x;
    const uint32_t L = kTinyWsL, W = 2, nsteps = 2 * A.nsweeps;
    const uint64_t groups_per_row = L >> 3;
    // a held step (failure testing) runs the waits out quickly
    const uint32_t limit = A.hold_step ? (1u << 14) : kWsSpinLimit;
    const uint32_t plimit = A.hold_step ? (1u << 12) : kWsWaitLimit;
    const uint32_t *src = static_cast<const uint32_t *>(A.spins);
    if (tid < kWsWords) {
        lat[tid] = src[tid];
        for (uint32_t k = 0; k < kWsSlots; ++k) entries[k][tid] = 0ull;
    }
    if (tid == 0) {
        ws_abort = 0u;
        for (uint32_t k = 0; k < kWsSlots; ++k) mbar_init(&empty[k], kWsWords);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    __syncthreads();  // the last barrier of the whole block

    HalfSweepArgs a;
    a.key = A.key;
    a.thr4 = A.thr4;
    a.thr8 = A.thr8;
    a.zero = 0u;
    if (tid >= kWsWords) {
        // ---- producers
        const uint32_t pt = tid - kWsWords, grp = pt / kWsWords, w = pt % kWsWords;
        const uint64_t g = (uint64_t)(w >> 1) * groups_per_row + (uint64_t)(w & 1u) * 4u;
        for (uint32_t s = grp; s < nsteps; s += kWsGroups) {
            const uint32_t k = s % kWsSlots;
            if (s >= kWsSlots && !mbar_wait(&empty[k], ((s / kWsSlots) & 1u) ^ 1u, plimit)) {
                // the consumers did not read the slot's previous entry in time
                *vabort = 1u;
                if (A.err) atomicExch(A.err, 1u);
                return;
            }
            tiny_step_values(a, A, A.t0 + (s >> 1), s & 1u);
            uint32_t h4[1], h8[1];
            word_draw_masks<4, 0, 4>(a, a, g, h4, h8);
            if (A.hold_step == s + 1) continue;  // never published (failure testing)
            ve[k * kWsWords + w] = ((uint64_t)(s + 1) << 32) | pack_masks(h4[0], h8[0]);
        }
        return;
    }
    // ---- consumers: thread c updates word c (row c / 2, word c % 2).  A step
    // ends with a named barrier of the 128 consumers (bar.sync 1, 128); no
    // consumer leaves the loop alone, so every barrier completes.
    const uint32_t c = tid, y = c >> 1, w = c & 1u;
    const uint32_t row = c - w;
    const uint32_t iu = (y == 0 ? kWsWords - W : row - W) + w, id = (y + 1 == L ? 0u : row + W) + w;
    const uint32_t inb = row + (w ^ 1u);  // W = 2: the left and the right neighbour word
    uint32_t phase = A.record_every ? A.t0 % A.record_every : 0u;
    uint32_t slot = 0, nring = 0;
    for (uint32_t s = 0; s < nsteps; ++s) {
        const uint32_t k = s % kWsSlots, p = s & 1u;
        const bool rec = A.record_every != 0u && phase + 1 == A.record_every;
        const bool last = (s >> 1) + 1 == A.nsweeps;
        const bool count = p == 1u && (rec || last);
        unsigned int cu = 0, ca = 0;
        uint64_t e = ve[k * kWsWords + c];
        uint32_t i = 0;
        while ((uint32_t)(e >> 32) != s + 1 && ++i < limit) e = ve[k * kWsWords + c];
        if ((uint32_t)(e >> 32) == s + 1) {
            mbar_arrive(&empty[k]);  // this thread has read the slot (release: after the load)
            const uint32_t nw = update_word32_drawn<4>(lat[c], lat[iu], lat[id], lat[inb], lat[inb], (y + p) & 1u,
                                                       (uint32_t)e, count, cu, ca, 0u);
            lat[c] = nw;
        } else {
            *vabort = 1u;
        }
        if (count) {
            // each consumer warp's counts into its own slot of the sample ring
            // (summed over the four warps only when the ring is written out)
            cu = __reduce_add_sync(0xFFFFFFFFu, cu);
            ca = __reduce_add_sync(0xFFFFFFFFu, ca);
            if ((c & 31u) == 0) {
                if (rec) {
                    wring[nring][c >> 5][0] = cu;
                    wring[nring][c >> 5][1] = ca;
                }
                if (last) {  // the extra slot holds the state after the last sweep
                    wring[kRingSamples][c >> 5][0] = cu;
                    wring[kRingSamples][c >> 5][1] = ca;
                }
            }
        }
        asm volatile("bar.sync 1, 128;" ::: "memory");
        if (*vabort) break;
        if (p == 1u) {
            if (rec) ++nring;
            if (A.record_every) phase = (phase + 1 == A.record_every) ? 0u : phase + 1;
        }
        if (nring == kRingSamples || s + 1 == nsteps) {
            // the ring (at the end the rest of it) to global memory
            for (uint32_t r = c; r < 2 * nring; r += kWsWords) {
                const uint32_t q = r >> 1, j = r & 1u;
                A.acc[2 * slot + r] = (unsigned long long)wring[q][0][j] + wring[q][1][j] + wring[q][2][j] +
                                      wring[q][3][j];
            }
            slot += nring;
            nring = 0;
            asm volatile("bar.sync 1, 128;" ::: "memory");  // the ring is free again
        }
    }
    if (*vabort) {
        if (A.err && c == 0) atomicExch(A.err, 1u);
        return;
    }
    if (c < 2)
        A.acc[2 * A.nrec + c] = (unsigned long long)wring[kRingSamples][0][c] + wring[kRingSamples][1][c] +
                                wring[kRingSamples][2][c] + wring[kRingSamples][3][c];
    static_cast<uint32_t *>(A.spins)[c] = lat[c];
}

// The one-CTA kernel spread over a cluster of k = 2, 4 or 8 CTAs (distributed
// shared memory): CTA c holds rows [c L/k, (c + 1) L/k) with one halo row above
// and below.  At the start of each step it copies the halos from the
// neighbouring CTAs' shared memory (their boundary rows as of the end of the
// previous step; only the bits of the other parity are used, which nobody writes
// during the step), and a cluster barrier ends the step.  A lattice too small to
// fill one SM's issue slots gets k SMs.
template <int NQ, bool FIELD>
__global__ void __launch_bounds__(kTinyMaxThreads) k_tiny_cluster(const __grid_constant__ TinyRunArgs A)
{
    static_assert(!FIELD || NQ == 4, "the field update takes whole words");
    constexpr uint32_t S = 4 / NQ;  // threads per word
    cooperative_groups::cluster_group cluster = cooperative_groups::this_cluster();
    extern __shared__ uint32_t buf[];  // rows -1 .. rpc of this CTA, W words each
    __shared__ unsigned int cnt[2];
    __shared__ uint32_t tab[16];
    if (FIELD && threadIdx.x < 16) tab[threadIdx.x] = A.field_thr[threadIdx.x];
    const uint32_t L = (uint32_t)A.L;
    const uint32_t W = L >> 5;  // words per row, a power of two
    const uint32_t lgW = 31 - __clz(W);
    const uint32_t k = cluster.num_blocks(), c = cluster.block_rank();
    const uint32_t rpc = L / k;  // rows of this CTA
    const uint32_t row0 = c * rpc;
    const uint32_t nwords = rpc * W;
    const uint32_t tid = threadIdx.x, nthr = blockDim.x;
    const uint64_t groups_per_row = L >> 3;
    uint32_t *const own = buf + W;

    const uint32_t *src = static_cast<const uint32_t *>(A.spins) + (uint64_t)row0 * W;
    for (uint32_t i = tid; i < nwords; i += nthr) own[i] = src[i];
    if (tid < 2) cnt[tid] = 0u;
    // the neighbouring CTAs' buffers (their own rows start one row in)
    const uint32_t *const prev = cluster.map_shared_rank(buf, (c + k - 1) % k);
    const uint32_t *const next = cluster.map_shared_rank(buf, (c + 1) % k);
    cluster.sync();

    HalfSweepArgs a;
    a.key = A.key;
    a.thr4 = A.thr4;
    a.thr8 = A.thr8;
    a.zero = 0u;
    uint32_t phase = A.record_every ? A.t0 % A.record_every : 0u;  // t % record_every
    uint32_t slot = 0;
    if (!FIELD && nwords * S <= nthr) {
        // Draw-ahead path (see k_tiny).  The cluster barrier is split: a thread
        // arrives when its step is done, draws the masks of a later step, and
        // only then waits for the rest of the cluster.  The threads of the
        // first and last row read the neighbouring CTAs' boundary rows directly
        // from distributed shared memory: only their bits of the other parity
        // are used, which the neighbours do not write during this step, and a
        // neighbour cannot start the next step before this thread has arrived.
        __shared__ unsigned int ring[2 * kRingSamples], lastc[2];
        uint32_t nring = 0;  // samples in the ring; the ring's first is sample `slot`
        const bool active = tid < nwords * S;
        const uint32_t kw = active ? tid / S : 0u, sub = tid % S;
        const uint32_t ly = kw >> lgW, w = kw & (W - 1u);
        uint32_t *const row = own + ly * W;
        const uint32_t *const upw = ly == 0 ? prev + W + (rpc - 1) * W + w : row + w - W;
        const uint32_t *const dnw = ly + 1 == rpc ? next + W + w : row + w + W;
        const uint32_t wl = (w - 1u) & (W - 1u), wr = (w + 1u) & (W - 1u);
        const uint32_t y = row0 + ly;
        const uint64_t g = (uint64_t)y * groups_per_row + (uint64_t)w * 4u;
        uint32_t pk[2 * kAheadSweeps];
        if (active) tiny_draw_ahead<NQ>(a, A, A.t0, min(kAheadSweeps, A.nsweeps), g, sub * NQ, pk);
        for (uint32_t i0 = 0; i0 < A.nsweeps; i0 += kAheadSweeps) {
            const uint32_t ns = min(kAheadSweeps, A.nsweeps - i0);
#pragma unroll
            for (uint32_t j = 0; j < 2 * kAheadSweeps; ++j) {
                if (j >= 2 * ns) break;
                const uint32_t p = j & 1u;
                const bool rec = A.record_every != 0u && phase + 1 == A.record_every;
                const bool last = i0 + (j >> 1) + 1 == A.nsweeps;
                const bool count = p == 1u && (rec || last);
                unsigned int cu = 0, ca = 0;
                if (active) {
                    const uint32_t nw = update_word32_drawn<NQ>(row[w], *upw, *dnw, row[wl], row[wr], (y + p) & 1u,
                                                                pk[j], count, cu, ca, sub * NQ);
                    tiny_store<NQ>(row + w, nw, sub);
                }
                if (count) {
                    cu = __reduce_add_sync(0xFFFFFFFFu, cu);
                    ca = __reduce_add_sync(0xFFFFFFFFu, ca);
                    if ((tid & 31u) == 0) {
                        atomicAdd(&cnt[0], cu);
                        atomicAdd(&cnt[1], ca);
                    }
                }
                cluster.barrier_arrive();
                const uint32_t ia = i0 + kAheadSweeps + (j >> 1);
                if (active && ia < A.nsweeps) {
                    tiny_step_values(a, A, A.t0 + ia, p);
                    uint32_t h4[1], h8[1];
                    word_draw_masks<4, 0, NQ>(a, a, g, h4, h8, sub * NQ);
                    pk[j] = pack_masks(h4[0], h8[0]);
                }
                cluster.barrier_wait();
                if (count && tid == 0) {
                    if (rec) {
                        ring[2 * nring] = cnt[0];
                        ring[2 * nring + 1] = cnt[1];
                    }
                    if (last) {
                        lastc[0] = cnt[0];
                        lastc[1] = cnt[1];
                    }
                    cnt[0] = 0u;
                    cnt[1] = 0u;
                }
                if (p == 1u) {
                    if (rec && ++nring == kRingSamples) {
                        // the ring is full: the CTAs add it into the sample slots
                        __syncthreads();
                        for (uint32_t r = tid; r < 2 * kRingSamples; r += nthr)
                            atomicAdd(A.acc + 2 * slot + r, (unsigned long long)ring[r]);
                        slot += kRingSamples;
                        nring = 0;
                    }
                    if (A.record_every) phase = (phase + 1 == A.record_every) ? 0u : phase + 1;
                }
            }
        }
        __syncthreads();
        for (uint32_t r = tid; r < 2 * nring; r += nthr) atomicAdd(A.acc + 2 * slot + r, (unsigned long long)ring[r]);
        if (tid < 2) atomicAdd(A.acc + 2 * A.nrec + tid, (unsigned long long)lastc[tid]);
        uint32_t *dst = static_cast<uint32_t *>(A.spins) + (uint64_t)row0 * W;
        for (uint32_t i = tid; i < nwords; i += nthr) dst[i] = own[i];
        cluster.sync();  // no CTA leaves while another may still read its buffer
        return;
    }
    for (uint32_t i = 0; i < A.nsweeps; ++i) {
        const uint32_t t = A.t0 + i;
        const bool rec = A.record_every != 0u && phase + 1 == A.record_every;
        const bool last = i + 1 == A.nsweeps;
        const uint64_t pb = (uint64_t)t * kPhiloxMulB;
        a.r1x0 = (uint32_t)(pb >> 32) ^ A.key.k0[0];
        a.r2x0k = (uint32_t)pb ^ A.key.k0[1];
        const uint64_t pa = (uint64_t)a.r1x0 * kPhiloxMulA;
        a.r2x2k = (uint32_t)(pa >> 32) ^ A.key.k1[1];
        a.r2x3 = (uint32_t)pa;
#pragma unroll 1
        for (uint32_t p = 0; p < 2; ++p) {
            a.r1x2k = (A.c3base | p) ^ A.key.k1[0];
            const bool count = p == 1u && (rec || last);
            // halos: the previous CTA's last row above, the next CTA's first row below
            for (uint32_t j = tid; j < 2 * W; j += nthr) {
                if (j < W)
                    buf[j] = prev[W + (rpc - 1) * W + j];
                else
                    buf[(rpc + 1) * W + (j - W)] = next[W + (j - W)];
            }
            __syncthreads();
            unsigned int cu = 0, ca = 0;
            for (uint32_t it = tid; it < nwords * S; it += nthr) {
                const uint32_t kw = it / S, sub = it % S;  // S is a power of two
                const uint32_t ly = kw >> lgW, w = kw & (W - 1u);
                uint32_t *const row = own + ly * W;  // rows ly - 1 and ly + 1 are in buf as well
                const uint32_t cur = row[w];
                const uint32_t up = row[w - W];
                const uint32_t dn = row[w + W];
                const uint32_t lw = row[(w - 1u) & (W - 1u)];
                const uint32_t rw = row[(w + 1u) & (W - 1u)];
                const uint32_t y = row0 + ly;
                const uint64_t g = (uint64_t)y * groups_per_row + (uint64_t)w * 4u;
                const uint32_t nw =
                    FIELD ? update_word_field(a, a, tab, A.k_up, A.k_dn, cur, up, dn, lw, rw, (y + p) & 1u, g, count, cu, ca)
                          : update_word<uint32_t, 0, NQ>(a, a, cur, up, dn, lw, rw, (y + p) & 1u, g, count, cu, ca, sub * NQ);
                if (NQ == 4)
                    row[w] = nw;
                else if (NQ == 2)
                    reinterpret_cast<uint16_t *>(row + w)[sub] = (uint16_t)(nw >> (16 * sub));
                else
                    reinterpret_cast<uint8_t *>(row + w)[sub] = (uint8_t)(nw >> (8 * sub));
            }
            if (count) {
                cu = __reduce_add_sync(0xFFFFFFFFu, cu);
                ca = __reduce_add_sync(0xFFFFFFFFu, ca);
                if ((tid & 31u) == 0) {
                    atomicAdd(&cnt[0], cu);
                    atomicAdd(&cnt[1], ca);
                }
            }
            cluster.sync();  // the step is complete in every CTA
            if (count && tid == 0) {
                // the CTAs' counts add up in the sample slots; the next counted step
                // is two steps and two barriers away
                const unsigned long long c0 = cnt[0], c1 = cnt[1];
                if (rec) {
                    atomicAdd(A.acc + 2 * slot, c0);
                    atomicAdd(A.acc + 2 * slot + 1, c1);
                }
                if (last) {
                    atomicAdd(A.acc + 2 * A.nrec, c0);
                    atomicAdd(A.acc + 2 * A.nrec + 1, c1);
                }
                cnt[0] = 0u;
                cnt[1] = 0u;
            }
        }
        if (rec) ++slot;
        if (A.record_every) phase = (phase + 1 == A.record_every) ? 0u : phase + 1;
    }
    uint32_t *dst = static_cast<uint32_t *>(A.spins) + (uint64_t)row0 * W;
    for (uint32_t i = tid; i < nwords; i += nthr) dst[i] = own[i];
    cluster.sync();  // no CTA leaves while another may still read its buffer
}

}  // namespace

bool tiny_lattice_ok(uint64_t L) { return L >= 64 && L <= 1024 && (L & (L - 1)) == 0; }

bool tiny_config_valid(const LaunchConfig &c, uint64_t L, uint64_t rows)
{
    if (c.proc_bits == kTinyProcBits && L == kTinyWsL && rows == L && c.block == kTinyWsBlock &&
        c.rows_per_item == 1 && c.grid == 1 && c.regcap == 0 && c.insert == 0 && c.persistent == 0)
        return true;  // the warp-specialised kernel
    return c.proc_bits == kTinyProcBits && tiny_lattice_ok(L) && rows == L && c.regcap == 0 && c.insert == 0 &&
           (c.block == 128 || c.block == 256 || c.block == 512) &&
           (c.rows_per_item == 1 || c.rows_per_item == 2 || c.rows_per_item == 4) &&
           (c.grid == 1 || c.grid == 2 || c.grid == 4 || c.grid == 8) && c.persistent == 0;
}

LaunchConfig plain_launch(const LaunchConfig &c)
{
    if (c.proc_bits == 32 || c.proc_bits == 64) {
        LaunchConfig step = c;
        step.persistent = 0;
        return step;
    }
    return LaunchConfig{32, 1, 0, 256, 2, 0};  // the step shape of small lattices
}

cudaError_t launch_tiny(const TinyRunArgs &a, uint32_t block, uint32_t threads_per_word, uint32_t ctas,
                        cudaStream_t s)
{
    if (!tiny_lattice_ok(a.L) || a.nsweeps == 0) return cudaErrorInvalidValue;
    if (ctas == 1 && a.L == kTinyWsL && block == kTinyWsBlock && threads_per_word == 1) {
        if (!a.use_field) {
            k_tiny_ws<<<1, kTinyWsBlock, 0, s>>>(a);
            return cudaGetLastError();
        }
        block = kTinyMaxThreads;  // in a field: the one-CTA field kernel (no warp-specialised form)
    }
    if (block == 0 || block > kTinyMaxThreads || block % 32 != 0) return cudaErrorInvalidValue;
    if (ctas != 1 && ctas != 2 && ctas != 4 && ctas != 8) return cudaErrorInvalidValue;
    using TinyKernel = void (*)(TinyRunArgs);
    TinyKernel kern;
    if (ctas == 1)
        kern = a.use_field ? k_tiny<4, true>
               : threads_per_word == 1 ? k_tiny<4, false>
               : threads_per_word == 2 ? k_tiny<2, false>
               : threads_per_word == 4 ? k_tiny<1, false> : nullptr;
    else
        kern = a.use_field ? k_tiny_cluster<4, true>
               : threads_per_word == 1 ? k_tiny_cluster<4, false>
               : threads_per_word == 2 ? k_tiny_cluster<2, false>
               : threads_per_word == 4 ? k_tiny_cluster<1, false> : nullptr;
    if (!kern) return cudaErrorInvalidValue;
    // the whole lattice, or a CTA's rows and its two halo rows
    const size_t W = a.L / 32;
    const size_t smem = ctas == 1 ? (size_t)(a.L * W * 4) : (size_t)((a.L / ctas + 2) * W * 4);
    if (smem > 48 * 1024) {
        const cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return e;
    }
    if (ctas == 1) {
        kern<<<1, block, smem, s>>>(a);
        return cudaGetLastError();
    }
    cudaLaunchConfig_t cfg{};
    cfg.gridDim = dim3(ctas);
    cfg.blockDim = dim3(block);
    cfg.dynamicSmemBytes = smem;
    cfg.stream = s;
    cudaLaunchAttribute attr{};
    attr.id = cudaLaunchAttributeClusterDimension;
    attr.val.clusterDim.x = ctas;
    attr.val.clusterDim.y = 1;
    attr.val.clusterDim.z = 1;
    cfg.attrs = &attr;
    cfg.numAttrs = 1;
    return cudaLaunchKernelEx(&cfg, kern, a);
}

}  // namespace ising

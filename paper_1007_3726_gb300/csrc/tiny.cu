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
    if (!tiny_lattice_ok(a.L) || a.nsweeps == 0 || block == 0 || block > kTinyMaxThreads || block % 32 != 0)
        return cudaErrorInvalidValue;
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

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
// Warp-specialised kernels for L = 64, 128 and 256 (a row is 2, 4 or 8 words of
// 32 bits).  A lattice this small leaves most of an SM's issue slots idle when
// every thread both draws and updates: the dependent bit logic and the
// barrier of each step are short, the Philox draws long.  The draws do not
// depend on the spins, so the roles are split:
//   consumers  threads of the first CTA that keep the lattice in registers:
//              one word each at L = 64, at L = 128 and 256 a vertical run of two
//              and four words of one column.  The left and right neighbour words come from other
//              lanes by warp shuffles, so do the rows above and below a run,
//              and the rows across a warp boundary through a small shared
//              array.  A step is the ring entries, the bit logic, one store of
//              the thread's boundary row (a scratch slot off a warp boundary)
//              and one barrier of the consumers.  The step has no branch but
//              one that is taken only when something has to wait (a ring entry
//              is not there yet, a count slot is still being read) or a failure
//              is to be acted on.
//   arriver    one thread next to the consumers: it follows their progress
//              (thread 0 of the consumers publishes each finished step) and
//              frees each step's ring slot with one arrival on the slot's
//              mbarrier; nothing else, so that the producers' slots are freed
//              as soon as they can be;
//   counting   on a counted sweep, L = 64 and 128: the consumers' second step
//              stores the new words, tagged, into a snapshot ring, and a few
//              counter warps (counter k takes every few counted sweeps starting
//              with the k-th) take M and E of the whole lattice from a snapshot
//              once all its tags are there, write the sample and free the slot;
//              at L = 256, where the producers set the pace and the consumers
//              have time to spare, each consumer warp counts its own words and
//              stores one tagged partial count, and a writer warp adds the
//              warps' partials up and writes the sample.  No remote arrival,
//              global store or release is then on the consumers' path.
//   producers  groups of threads (L * L / 32 words; a thread draws two words at
//              L = 256); a group draws the masks of every NG-th step (NG groups
//              in all) and writes them, tagged with the step, into the group's
//              slot of the consumers' ring: one 64-bit entry (step + 1) << 32 |
//              masks per word.  It draws the masks of its next step first and
//              then waits until the slot's previous entry has been freed, so
//              the draws overlap the wait.
// Two forms:
//   CL = false  one CTA of 1024 threads for L = 64: 128 consumer threads, the
//               arriving thread, two counter warps and six producer groups;
//   CL = true   a thread-block cluster of C CTAs of 1024 threads: CTA 0 holds
//               the consumers, the arriving thread and the counting warps,
//               CTAs 1 .. C - 1 the producers, which store into CTA 0's ring
//               through distributed shared memory; the arrival goes to the
//               slot's mbarrier in the producing CTA.  The producers' issue
//               slots then no longer compete with the consumers', and C - 1
//               SMs draw.
// Ordering.  A consumer's load of a ring entry has returned its value before
// the consumer reaches the barrier that ends the step (the value feeds the
// boundary store that precedes it); thread 0 publishes the step after that
// barrier, the arriving thread arrives for the slot after it has read the publication,
// and a producer stores into the slot only after its wait has seen the
// arrival.  Each link follows the completion of the one before, so no store
// into a slot can overtake a load of its previous entry; the arrivals and the
// publication are relaxed (a release at cluster scope would fence every
// thread's memory operations at every step).  Snapshot entries carry their
// sweep's tag (so do the partial counts), and nobody reads one before the
// tag is there.  A release that frees a snapshot slot or count buffer comes
// before the sample's global stores, which it would otherwise wait for.
// Failure.  Every wait is bounded.  A consumer whose wait runs out sets the
// abort flag of its step's parity before the step's barrier; every consumer
// reads that flag after the barrier and before the next one, so all of them
// stop at the same point.  The arriving thread, the counting warps and the
// producers stop when their own waits run out; any of them sets *err, so the
// kernel always ends.  In the
// cluster form every thread reaches a final cluster barrier, so no CTA leaves
// while another may still use its shared memory.
__device__ __forceinline__ uint32_t smem_addr(const void *p)
{
    return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}
__device__ __forceinline__ void mbar_init(uint64_t *bar, uint32_t count)
{
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_addr(bar)), "r"(count) : "memory");
}

constexpr uint32_t kWsSpinLimit = 1u << 24;  // polls of a consumer's wait before it gives up
constexpr uint32_t kWsWaitLimit = 1u << 20;  // polls of a producer's mbarrier wait
constexpr uint32_t kWsMaxGroups = 7 * (kTinyWsBlock / 128);  // L = 64 on a cluster of 8

__device__ __forceinline__ uint32_t mapa_shared(uint32_t addr, uint32_t rank)
{
    uint32_t r;
    asm volatile("mapa.shared::cluster.u32 %0, %1, %2;" : "=r"(r) : "r"(addr), "r"(rank));
    return r;
}
__device__ __forceinline__ uint32_t cluster_rank()
{
    uint32_t r;
    asm volatile("mov.u32 %0, %%cluster_ctarank;" : "=r"(r));
    return r;
}
__device__ __forceinline__ void cluster_barrier()
{
    asm volatile("barrier.cluster.arrive.release;\n\tbarrier.cluster.wait.acquire;" ::: "memory");
}
// A ring entry: written by a producer of this CTA (CL = false) or of another
// CTA of the cluster (CL = true), read by the consumers.
template <bool CL>
__device__ __forceinline__ void ring_store(uint32_t addr, uint64_t v)
{
    if constexpr (CL)
        asm volatile("st.relaxed.cluster.shared::cluster.u64 [%0], %1;" ::"r"(addr), "l"(v) : "memory");
    else
        asm volatile("st.volatile.shared.u64 [%0], %1;" ::"r"(addr), "l"(v) : "memory");
}
template <bool CL>
__device__ __forceinline__ uint64_t ring_load(uint32_t addr)
{
    uint64_t v;
    if constexpr (CL)
        asm volatile("ld.relaxed.cluster.shared::cta.u64 %0, [%1];" : "=l"(v) : "r"(addr));
    else
        asm volatile("ld.volatile.shared.u64 %0, [%1];" : "=l"(v) : "r"(addr));
    return v;
}
__device__ __forceinline__ uint32_t ld_volatile_u32(uint32_t addr)
{
    uint32_t v;
    asm volatile("ld.volatile.shared.u32 %0, [%1];" : "=r"(v) : "r"(addr));
    return v;
}
__device__ __forceinline__ uint64_t ld_volatile_u64(uint32_t addr)
{
    uint64_t v;
    asm volatile("ld.volatile.shared.u64 %0, [%1];" : "=l"(v) : "r"(addr));
    return v;
}
// The arriving thread's arrival on a slot's mbarrier (in the producing CTA when CL).
template <bool CL>
__device__ __forceinline__ void slot_arrive(uint32_t addr)
{
    if constexpr (CL)
        asm volatile("mbarrier.arrive.relaxed.cluster.shared::cluster.b64 _, [%0];" ::"r"(addr) : "memory");
    else
        asm volatile("mbarrier.arrive.relaxed.cta.shared::cta.b64 _, [%0];" ::"r"(addr) : "memory");
}
// A producer's bounded wait until the phase of the given parity of its slot's
// mbarrier has completed.
template <bool CL>
__device__ __forceinline__ bool slot_wait(uint32_t addr, uint32_t parity, uint32_t limit)
{
    for (uint32_t i = 0; i < limit; ++i) {
        uint32_t done;
        if constexpr (CL)
            asm volatile("{\n\t.reg .pred p;\n\tmbarrier.try_wait.parity.relaxed.cluster.shared::cta.b64 p, [%1], %2;\n\t"
                         "selp.u32 %0, 1, 0, p;\n\t}"
                         : "=r"(done)
                         : "r"(addr), "r"(parity)
                         : "memory");
        else
            asm volatile("{\n\t.reg .pred p;\n\tmbarrier.try_wait.parity.relaxed.cta.shared::cta.b64 p, [%1], %2;\n\t"
                         "selp.u32 %0, 1, 0, p;\n\t}"
                         : "=r"(done)
                         : "r"(addr), "r"(parity)
                         : "memory");
        if (done) return true;
    }
    return false;
}

// The bit logic of update_word32_drawn for one 32-bit word (all 4 bytes).
__device__ __forceinline__ uint32_t ws_update_word(uint32_t cur, uint32_t up, uint32_t dn, uint32_t lw, uint32_t rw,
                                                   uint32_t off, uint32_t pk)
{
    constexpr uint32_t even = 0x55555555u;
    const uint32_t left = __funnelshift_l(lw, cur, 1);   // (cur << 1) | (lw >> 31): site x - 1
    const uint32_t right = __funnelshift_r(cur, rw, 1);  // (cur >> 1) | (rw << 31): site x + 1
    const uint32_t i1 = cur ^ up, i2 = cur ^ dn, i3 = cur ^ left, i4 = cur ^ right;
    const uint32_t s12 = i1 ^ i2, c12 = i1 & i2;
    const uint32_t s34 = i3 ^ i4, c34 = i3 & i4;
    const uint32_t odd = s12 ^ s34;
    const uint32_t ge2 = c12 | c34 | (s12 & s34);
    const uint32_t eq1 = odd & ~ge2;
    const uint32_t eq0 = ~(odd | ge2);
    const uint32_t p4 = (pk & even) << off;
    const uint32_t p8 = ((pk >> 1) & even) << off;
    return cur ^ ((even << off) & (ge2 | (eq1 & p4) | (eq0 & p8)));
}

template <uint32_t V>
struct WsParity {
    static constexpr uint32_t value = V;
};

// The shape of the warp-specialised kernel at L = LL.
template <uint32_t LL, bool CL>
struct WsShape {
    static constexpr uint32_t W = LL / 32;                  // words per row
    static constexpr uint32_t NWORDS = LL * W;              // words of the lattice
    static constexpr uint32_t WPT = LL >= 256 ? NWORDS / 512 : LL == 128 ? 2 : 1;  // words per consumer thread
    static constexpr uint32_t NCONS = NWORDS / WPT;         // consumer threads
    static constexpr uint32_t NCW = NCONS / 32;             // consumer warps
    static constexpr uint32_t GT = NWORDS < kTinyWsBlock ? NWORDS : kTinyWsBlock;  // threads of a producer group
    static constexpr uint32_t PW = NWORDS / GT;             // words per producer thread
    static constexpr uint32_t GPC = kTinyWsBlock / GT;      // producer groups per producer CTA
    // where the consumers have slack (the producers set the pace: L = 256),
    // they count on recorded sweeps themselves; else snapshots and counter warps
    static constexpr bool INLINE = LL >= 256;
    static constexpr uint32_t NCOUNT = INLINE ? 0 : CL ? 4 : 2;  // counter warps
    static constexpr uint32_t SNAPS = INLINE ? 0 : 8;       // snapshot slots
    // CL = false: the producer groups beside the consumers, the arriving
    // thread's warp and the counter warps, and the threads left over
    static constexpr uint32_t GLOCAL = (kTinyWsBlock - NCONS - 32 - 32 * NCOUNT) / GT;
    static constexpr uint32_t IDLE = CL ? 0 : kTinyWsBlock - NCONS - 32 - 32 * NCOUNT - GLOCAL * GT;
    static_assert(CL || (LL == 64 && GLOCAL >= 1), "the one-CTA form is for L = 64");
    static_assert(NCONS + 32 + 32 * NCOUNT <= kTinyWsBlock, "the first CTA holds consumers, arriver and counters");
    __host__ __device__ static uint32_t groups(uint32_t ctas) { return CL ? GPC * (ctas - 1) : GLOCAL; }
    // dynamic shared memory: the ring (a slot per group) and the snapshot slots
    static size_t smem(uint32_t ctas) { return (size_t)(groups(ctas) + SNAPS) * NWORDS * 8; }
};

template <uint32_t LL, bool CL>
__global__ void __launch_bounds__(kTinyWsBlock) k_tiny_wsc(const __grid_constant__ TinyRunArgs A)
{
    using S = WsShape<LL, CL>;
    constexpr uint32_t W = S::W, NWORDS = S::NWORDS, WPT = S::WPT, NCONS = S::NCONS, NCW = S::NCW;
    constexpr uint32_t GT = S::GT, PW = S::PW, GPC = S::GPC, NCOUNT = S::NCOUNT;
    constexpr uint32_t SNAPS = S::SNAPS;
    constexpr uint32_t SN = SNAPS ? SNAPS : 1u;  // snapshot slots in index arithmetic (no slot when counting inline)
    constexpr uint32_t kStopped = 0xFFFFFFFFu;
    constexpr uint32_t NB = 2 * NCW * W;  // warps' first and last rows; then one scratch slot per consumer
    // dynamic: the ring [NG][NWORDS] ((step + 1) << 32 | masks), then the
    // snapshots [SNAPS][NWORDS] ((sweep tag) << 32 | word) of the lattice after
    // counted sweeps; both used in CTA 0 only
    extern __shared__ __align__(16) uint64_t dyn[];
    __shared__ __align__(8) uint64_t empty[kWsMaxGroups];  // per slot: one arrival frees it
    __shared__ uint32_t bnd[NB + NCONS];  // first rows of the consumer warps, last rows, scratch
    // per snapshot slot: how many snapshots the counter warps have read from it
    __shared__ uint32_t slot_read[SN];
    // inline counting: each consumer warp's counts of the last NCB counted
    // sweeps (sweep tag << 48 | anti-aligned bonds << 24 | up spins), and how
    // many counted sweeps the writer warp has read
    constexpr uint32_t NCB = 8;  // count buffers (counted sweeps the consumers may run ahead of the writer)
    __shared__ __align__(8) unsigned long long cnt[NCB][NCW];
    __shared__ uint32_t cnt_done;
    __shared__ uint32_t done_step, abort_flag[2];
    const uint32_t tid = threadIdx.x;
    const uint32_t rank = CL ? cluster_rank() : 0u;
    const uint32_t NG = S::groups(CL ? gridDim.x : 1u);
    uint64_t *const ring = dyn;
    uint64_t *const snap = dyn + (size_t)NG * NWORDS;
    const uint32_t nsteps = 2 * A.nsweeps;
    // a held step (failure testing) runs the waits out quickly
    const uint32_t limit = A.hold_step ? (1u << 14) : kWsSpinLimit;
    const uint32_t plimit = A.hold_step ? (1u << 12) : kWsWaitLimit;
    if (rank == 0) {
        for (uint32_t i = tid; i < NG * NWORDS; i += kTinyWsBlock) ring[i] = 0ull;
        if constexpr (SNAPS != 0)
            for (uint32_t i = tid; i < SNAPS * NWORDS; i += kTinyWsBlock) snap[i] = 0ull;
    }
    if (tid == 0) {
        for (uint32_t k = 0; k < NG; ++k) mbar_init(&empty[k], 1u);
        done_step = 0u;
        for (uint32_t k = 0; k < SN; ++k) slot_read[k] = 0u;
        for (uint32_t k = 0; k < NCB * NCW; ++k) (&cnt[0][0])[k] = 0ull;
        cnt_done = 0u;
        abort_flag[0] = 0u;
        abort_flag[1] = 0u;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if constexpr (CL)
        cluster_barrier();  // rings and mbarriers of every CTA ready
    else
        __syncthreads();

    const bool consumer = rank == 0 && tid < NCONS;
    const bool arriver = rank == 0 && tid == NCONS;
    const bool writer = S::INLINE && rank == 0 && tid >= NCONS + 32 && tid < NCONS + 64;
    const bool counter = rank == 0 && tid >= NCONS + 32 && tid < NCONS + 32 + 32 * NCOUNT;
    const bool producer = CL ? rank != 0 : (tid >= NCONS + 32 + 32 * NCOUNT && tid < kTinyWsBlock - S::IDLE);
    if (producer) {
        HalfSweepArgs a;
        a.key = A.key;
        a.thr4 = A.thr4;
        a.thr8 = A.thr8;
        a.zero = 0u;
        const uint32_t pt = CL ? tid : tid - NCONS - 32 - 32 * NCOUNT;
        const uint32_t G = (CL ? (rank - 1) * GPC : 0u) + pt / GT, tl = pt % GT;
        // words tl, tl + GT, ... of the lattice
        uint64_t g[PW];
        uint32_t dst[PW];
#pragma unroll
        for (uint32_t k = 0; k < PW; ++k) {
            const uint32_t w = tl + k * GT;
            g[k] = (uint64_t)(w / W) * (LL >> 3) + (uint64_t)(w % W) * 4u;
            const uint32_t la = smem_addr(&ring[G * NWORDS + w]);
            dst[k] = CL ? mapa_shared(la, 0u) : la;
        }
        const uint32_t slot_bar = smem_addr(&empty[G]);
        for (uint32_t s = G; s < nsteps; s += NG) {
            tiny_step_values(a, A, A.t0 + (s >> 1), s & 1u);
            uint32_t pk[PW];
#pragma unroll
            for (uint32_t k = 0; k < PW; ++k) {
                uint32_t h4[1], h8[1];
                word_draw_masks<4, 0, 4>(a, a, g[k], h4, h8);
                pk[k] = pack_masks(h4[0], h8[0]);
            }
            // the slot's previous entry (step s - NG) must have been freed
            if (s >= NG && !slot_wait<CL>(slot_bar, ((s / NG) & 1u) ^ 1u, plimit)) {
                if (A.err) atomicExch(A.err, 1u);
                break;
            }
            if (A.hold_step == s + 1) continue;  // never published (failure testing)
#pragma unroll
            for (uint32_t k = 0; k < PW; ++k) ring_store<CL>(dst[k], ((uint64_t)(s + 1) << 32) | pk[k]);
        }
    } else if (consumer) {
        // thread c holds a vertical run of WPT words: column w = c % W of rows
        // r WPT .. r WPT + WPT - 1 (r = c / W); the rows above and below the
        // inner words are the thread's own, a run's first and last rows come
        // from the lanes W before and after, and a warp's first and last rows
        // through the boundary array
        const uint32_t c = tid, q = c >> 5, l = c & 31u, w = c % W, r = c / W;
        const uint32_t j0 = r * WPT * W + w;  // word index of the run's first word (then + k W)
        const uint32_t lane_l = (l & ~(W - 1u)) | ((w + W - 1u) & (W - 1u));
        const uint32_t lane_r = (l & ~(W - 1u)) | ((w + 1u) & (W - 1u));
        const bool top = l < W, bottom = l >= 32u - W;
        // this thread's boundary slot (its warp's first row, last row, or a
        // scratch slot), and the slots of the rows above and below the warp
        const uint32_t my_b = top ? q * W + w : bottom ? NCW * W + q * W + w : NB + c;
        const uint32_t up_b = NCW * W + ((q + NCW - 1u) % NCW) * W + w, dn_b = ((q + 1u) % NCW) * W + w;
        uint32_t v[WPT];
#pragma unroll
        for (uint32_t k = 0; k < WPT; ++k) v[k] = static_cast<const uint32_t *>(A.spins)[j0 + k * W];
        bnd[my_b] = top ? v[0] : v[WPT - 1];
        asm volatile("bar.sync 1, %0;" ::"r"(NCONS) : "memory");  // the initial boundary rows
        const uint32_t ring0 = smem_addr(&ring[j0]);
        const uint32_t snap0 = smem_addr(&snap[j0]);
        const uint32_t abort0 = smem_addr(&abort_flag[0]);
        const uint32_t sread0 = smem_addr(&slot_read[0]);
        const uint32_t cnt_done0 = smem_addr(&cnt_done);
        const uint32_t done_addr = smem_addr(&done_step);
        uint32_t phase = A.record_every ? A.t0 % A.record_every : 0u;
        uint32_t G = 0, s = 0, cidx = 0, sread = 0;
        bool stop = false;

        // one step of parity p; false when the consumers stop
        auto step = [&](auto pc, bool counted) -> bool {
            constexpr uint32_t p = decltype(pc)::value;
            const uint32_t ea = ring0 + G * (NWORDS * 8u);
            uint64_t e[WPT];
#pragma unroll
            for (uint32_t k = 0; k < WPT; ++k) e[k] = ring_load<CL>(ea + k * (W * 8u));
            uint32_t vl[WPT], vr[WPT];
#pragma unroll
            for (uint32_t k = 0; k < WPT; ++k) {
                vl[k] = __shfl_sync(0xFFFFFFFFu, v[k], lane_l);
                vr[k] = W == 2 ? vl[k] : __shfl_sync(0xFFFFFFFFu, v[k], lane_r);
            }
            const uint32_t su = __shfl_up_sync(0xFFFFFFFFu, v[WPT - 1], W);
            const uint32_t sd = __shfl_down_sync(0xFFFFFFFFu, v[0], W);
            const uint32_t bu = bnd[up_b], bd = bnd[dn_b];
            const uint32_t vu0 = top ? bu : su;          // the row above the run
            const uint32_t vdl = bottom ? bd : sd;       // the row below the run
            // set (before the previous barrier) by a consumer whose wait ran out
            const uint32_t ab = ld_volatile_u32(abort0 + 4u * (p ^ 1u));
            const uint32_t tag = s + 1u;
            const uint32_t sslot = cidx % SN, sneed = cidx / SN;
            // the snapshot slot of this sweep: read by the counters as often as
            // it has been written (loaded at the sweep's first step, checked at
            // its second, where the snapshot is stored)
            bool snap_wait = false;
            if constexpr (S::INLINE) {
                // lane 0 of each warp stores into cnt[cidx % NCB], which the
                // writer must have read for counted sweep cidx - NCB
                if constexpr (p == 0u) sread = l == 0 ? ld_volatile_u32(cnt_done0) : 0u;
                snap_wait = p == 1u && counted && l == 0 && sread + NCB <= cidx;
            } else {
                if constexpr (p == 0u) sread = ld_volatile_u32(sread0 + 4u * sslot);
                snap_wait = p == 1u && counted && sread < sneed;
            }
            bool have = true;
#pragma unroll
            for (uint32_t k = 0; k < WPT; ++k) have &= (uint32_t)(e[k] >> 32) == tag;
            if (!have | (ab != 0u) | snap_wait) {
                if (ab != 0u) return false;  // every consumer has read the same flag
                bool fail = false;
                for (uint32_t n = 0; !have; ++n) {
                    if (n >= limit) {
                        fail = true;
                        break;
                    }
                    have = true;
#pragma unroll
                    for (uint32_t k = 0; k < WPT; ++k) {
                        e[k] = ring_load<CL>(ea + k * (W * 8u));
                        have &= (uint32_t)(e[k] >> 32) == tag;
                    }
                }
                // the snapshot slot's previous snapshot must have been read (or
                // the count buffer written out)
                for (uint32_t m = 0; snap_wait && (S::INLINE ? sread + NCB <= cidx : sread < sneed); ++m) {
                    if (m >= limit) {
                        fail = true;
                        break;
                    }
                    asm volatile("ld.acquire.cta.shared.u32 %0, [%1];"
                                 : "=r"(sread)
                                 : "r"(S::INLINE ? cnt_done0 : sread0 + 4u * sslot)
                                 : "memory");
                }
                if (fail) abort_flag[p] = 1u;
            }
            // word k of the run: row r WPT + k; its rows above and below are
            // read only at the sites of the other parity, which this step
            // leaves as they were (so a word already updated may serve)
#pragma unroll
            for (uint32_t k = 0; k < WPT; ++k) {
                const uint32_t up = k == 0 ? vu0 : v[k - 1], dn = k + 1 == WPT ? vdl : v[k + 1];
                v[k] = ws_update_word(v[k], up, dn, vl[k], vr[k], ((r * WPT + k) & 1u) ^ p, (uint32_t)e[k]);
            }
            bnd[my_b] = top ? v[0] : v[WPT - 1];
            if constexpr (S::INLINE && p == 1u) {
                if (counted) {  // uniform: the sweep is counted or not for every consumer
                    // up spins, and the anti-aligned bonds of the updated sites
                    // (every bond once on the second step); two bond masks of
                    // one parity share a word once one is rotated by one bit
                    // (the neighbours at the updated sites are of the other
                    // parity, the same before and after the step)
                    uint32_t cu = 0, ca = 0;
#pragma unroll
                    for (uint32_t k = 0; k < WPT; ++k) {
                        const uint32_t sel = 0x55555555u << (((r * WPT + k) & 1u) ^ 1u);
                        const uint32_t nu = k == 0 ? vu0 : v[k - 1], nd = k + 1 == WPT ? vdl : v[k + 1];
                        const uint32_t left = __funnelshift_l(vl[k], v[k], 1), right = __funnelshift_r(v[k], vr[k], 1);
                        const uint32_t b1 = sel & (v[k] ^ nu), b2 = sel & (v[k] ^ nd);
                        const uint32_t b3 = sel & (v[k] ^ left), b4 = sel & (v[k] ^ right);
                        cu += __popc(v[k]);
                        ca += __popc(b1 | __funnelshift_l(b2, b2, 1)) + __popc(b3 | __funnelshift_l(b4, b4, 1));
                    }
                    // this warp's counts (up spins <= 4096, bonds <= 8192) with the
                    // sweep's tag, into the warp's own slot: one store, no atomic
                    const unsigned long long part = (unsigned long long)__reduce_add_sync(0xFFFFFFFFu, cu) |
                                                    ((unsigned long long)__reduce_add_sync(0xFFFFFFFFu, ca) << 24) |
                                                    ((unsigned long long)((cidx + 1u) & 0xFFFFu) << 48);
                    if (l == 0) *(volatile unsigned long long *)&cnt[cidx % NCB][q] = part;
                }
            }
            if constexpr (!S::INLINE && p == 1u) {
                // a counted sweep: the tagged words into the snapshot slot
                const uint32_t sa = snap0 + sslot * (NWORDS * 8u);
#pragma unroll
                for (uint32_t k = 0; k < WPT; ++k)
                    asm volatile("{\n\t.reg .pred q;\n\tsetp.ne.u32 q, %0, 0;\n\t@q st.volatile.shared.u64 [%1], %2;\n\t}" ::"r"(
                                     (uint32_t)counted),
                                 "r"(sa + k * (W * 8u)), "l"(((uint64_t)(cidx + 1u) << 32) | v[k])
                                 : "memory");
            }
            asm volatile("bar.sync 1, %0;" ::"r"(NCONS) : "memory");
            // every consumer is done with step s: thread 0 publishes it
            asm volatile("{\n\t.reg .pred q;\n\tsetp.eq.u32 q, %0, 0;\n\t@q st.volatile.shared.u32 [%1], %2;\n\t}" ::"r"(c),
                         "r"(done_addr), "r"(tag)
                         : "memory");
            G = G + 1u == NG ? 0u : G + 1u;
            ++s;
            return true;
        };
        auto sweep_counted = [&]() {
            const bool counted = (A.record_every != 0u && phase + 1 == A.record_every);
            if (A.record_every) phase = (phase + 1 == A.record_every) ? 0u : phase + 1;
            return counted;
        };
        uint32_t i = 0;
        // two sweeps per iteration where a thread holds one word; with several
        // words a step's code is long, and one sweep per iteration keeps the
        // loop within the instruction cache
        constexpr uint32_t SW = WPT == 1 ? 2u : 1u;
        for (; SW == 1 && i < A.nsweeps; ++i) {
            const bool c0 = sweep_counted() || i + 1 == A.nsweeps;
            if (!step(WsParity<0>{}, c0) || !step(WsParity<1>{}, c0)) {
                stop = true;
                break;
            }
            if (c0) ++cidx;
        }
        for (; SW == 2 && i + 2 <= A.nsweeps; i += 2) {
            const bool c0 = sweep_counted() || i + 1 == A.nsweeps;
            const bool c1 = sweep_counted() || i + 2 == A.nsweeps;
            if (!step(WsParity<0>{}, c0) || !step(WsParity<1>{}, c0)) {
                stop = true;
                break;
            }
            if (c0) ++cidx;
            if (!step(WsParity<0>{}, c1) || !step(WsParity<1>{}, c1)) {
                stop = true;
                break;
            }
            if (c1) ++cidx;
        }
        if (!stop && i < A.nsweeps) {  // an odd number of sweeps: the last one (always counted)
            (void)sweep_counted();
            if (!step(WsParity<0>{}, true) || !step(WsParity<1>{}, true))
                stop = true;
            else
                ++cidx;
        }
        // a wait that ran out in the last step (its flag was set before the
        // last barrier, and nobody writes a flag after it)
        if (!stop && (ld_volatile_u32(abort0) | ld_volatile_u32(abort0 + 4u)) != 0u) stop = true;
        if (stop) {
            if (c == 0) {
                asm volatile("st.volatile.shared.u32 [%0], %1;" ::"r"(done_addr), "r"(kStopped) : "memory");
                if (A.err) atomicExch(A.err, 1u);
            }
        } else {
#pragma unroll
            for (uint32_t k = 0; k < WPT; ++k) static_cast<uint32_t *>(A.spins)[j0 + k * W] = v[k];
        }
    } else if (arriver) {
        // frees each finished step's ring slot: one arrival on the slot's
        // mbarrier (in the producing CTA when CL)
        const uint32_t done_addr = smem_addr(&done_step);
        uint32_t next = 0, G = 0, n = 0;
        while (next < nsteps) {
            const uint32_t d = ld_volatile_u32(done_addr);
            if (d == kStopped) break;
            if (d <= next) {
                if (++n >= 4 * limit) {  // longer than a consumer's wait: the consumers report first
                    if (A.err) atomicExch(A.err, 1u);
                    break;
                }
                continue;
            }
            n = 0;
            do {
                const uint32_t bar = smem_addr(&empty[G]);
                slot_arrive<CL>(CL ? mapa_shared(bar, 1u + G / GPC) : bar);
                G = G + 1u == NG ? 0u : G + 1u;
            } while (++next < d);
        }
    } else if (writer) {
        // inline counting: after the second step of each counted sweep, the
        // consumer warps' counts, once all carry the sweep's tag (they were
        // stored before the barrier of that step), go out as the sample.  A
        // warp of its own (lane k reads warp k's slot, so the reads are one
        // round trip however busy shared memory is), so that its global
        // stores and release never delay the arrivals that free the
        // producers' slots.
        static_assert(NCW <= 32, "one slot per lane");
        const uint32_t hl = tid & 31u;
        const uint32_t done_addr = smem_addr(&done_step);
        uint32_t next = 0, n = 0, slot = 0, ccount = 0;
        uint32_t phase = A.record_every ? A.t0 % A.record_every : 0u;
        bool quit = false;
        while (next < nsteps && !quit) {
            uint32_t d = hl == 0 ? ld_volatile_u32(done_addr) : 0u;
            d = __shfl_sync(0xFFFFFFFFu, d, 0);
            if (d == kStopped) break;
            if (d <= next) {
                if (++n >= 4 * limit) {  // longer than a consumer's wait: the consumers report first
                    if (A.err && hl == 0) atomicExch(A.err, 1u);
                    break;
                }
                continue;
            }
            n = 0;
            do {
                const uint32_t p = next & 1u;
                const bool rec = A.record_every != 0u && phase + 1 == A.record_every;
                const bool last = next + 1 == nsteps;
                if (p == 1u) {
                    if (rec || last) {
                        const unsigned long long want = (unsigned long long)((ccount + 1u) & 0xFFFFu) << 48;
                        const uint32_t a = smem_addr(&cnt[ccount % NCB][hl < NCW ? hl : 0u]);
                        unsigned long long part = hl < NCW ? ld_volatile_u64(a) : want;
                        for (uint32_t m = 0; (part & (0xFFFFull << 48)) != want && m < limit; ++m) part = ld_volatile_u64(a);
                        if (!__all_sync(0xFFFFFFFFu, (part & (0xFFFFull << 48)) == want)) {
                            if (A.err && hl == 0) atomicExch(A.err, 1u);
                            quit = true;
                            break;
                        }
                        const uint32_t c0 = __reduce_add_sync(0xFFFFFFFFu, hl < NCW ? (uint32_t)(part & 0xFFFFFFull) : 0u);
                        const uint32_t c1 =
                            __reduce_add_sync(0xFFFFFFFFu, hl < NCW ? (uint32_t)((part >> 24) & 0xFFFFFFull) : 0u);
                        ++ccount;
                        __syncwarp();  // every lane has read its slot
                        if (hl == 0) {
                            // the buffer is free again (released before the global
                            // stores below, which a release would otherwise wait for)
                            asm volatile("st.release.cta.shared.u32 [%0], %1;" ::"r"(smem_addr(&cnt_done)), "r"(ccount)
                                         : "memory");
                            if (rec) {
                                A.acc[2 * slot] = c0;
                                A.acc[2 * slot + 1] = c1;
                            }
                            if (last) {
                                A.acc[2 * A.nrec] = c0;
                                A.acc[2 * A.nrec + 1] = c1;
                            }
                        }
                    }
                    if (rec) ++slot;
                    if (A.record_every) phase = (phase + 1 == A.record_every) ? 0u : phase + 1;
                }
            } while (++next < d);
        }
    } else if (counter) {
        // counter warp k takes the counted sweeps k, k + NCOUNT, ...: M and E
        // of the whole lattice from the sweep's snapshot, once all its tags
        // are there.  Lane j holds words j, j + 32, ... (R of them); the word to
        // the right is in the same row of the same lane group, the word below
        // W lanes on (or, for the last rows of a group, in the next group).
        constexpr uint32_t R = NWORDS / 32;
        const uint32_t k = (tid - NCONS - 32) >> 5, hl = tid & 31u;
        const uint32_t re = A.record_every;
        const uint32_t first = re ? (re - (A.t0 % re + 1u) % re) % re : 0u;  // first recorded sweep
        const bool last_rec = re != 0u && A.nrec != 0u && first + (A.nrec - 1u) * re + 1u == A.nsweeps;
        const uint32_t ncounted = A.nrec + (last_rec ? 0u : 1u);
        const uint32_t lane_r = (hl & ~(W - 1u)) | ((hl + 1u) & (W - 1u));
        const uint32_t lane_d = (hl + W) & 31u;
        const uint32_t done_addr = smem_addr(&done_step);
        for (uint32_t cidx = k; cidx < ncounted; cidx += NCOUNT) {
            const uint32_t ks = cidx % SN, want = cidx + 1u;
            const uint32_t sbase = smem_addr(&snap[(size_t)ks * NWORDS + hl]);
            uint32_t n = 0, seen = 0;
            bool ok = false, quit = false;
            for (;;) {
                bool all = true;
#pragma unroll 4
                for (uint32_t m = 0; m < R; ++m) all &= (uint32_t)(ld_volatile_u64(sbase + m * 256u) >> 32) == want;
                if (__all_sync(0xFFFFFFFFu, all)) {
                    ok = true;
                    break;
                }
                // not there yet: the wait runs out only while the consumers make
                // no progress (a snapshot may be many sweeps away)
                uint32_t d = hl == 0 ? ld_volatile_u32(done_addr) : 0u;
                d = __shfl_sync(0xFFFFFFFFu, d, 0);
                if (d == kStopped) {
                    quit = true;
                    break;
                }
                n = d != seen ? 0u : n + 1u;
                seen = d;
                if (n >= 4 * limit) break;
                __nanosleep(64);
            }
            if (quit) break;
            if (!ok) {
                if (A.err && hl == 0) atomicExch(A.err, 1u);
                break;
            }
            __syncwarp();  // every tag seen before any lane reads the words
            uint32_t part = 0;  // packed: up spins <= 65536 / 2, anti-aligned bonds <= 2 L^2
            uint32_t up = 0;
            uint32_t cur = (uint32_t)ld_volatile_u64(sbase);
#pragma unroll 4
            for (uint32_t m = 0; m < R; ++m) {
                const uint32_t nxt = (uint32_t)ld_volatile_u64(sbase + ((m + 1u) % R) * 256u);
                const uint32_t xr = __shfl_sync(0xFFFFFFFFu, cur, lane_r);  // the word to the right
                const uint32_t dn_same = __shfl_sync(0xFFFFFFFFu, cur, lane_d);
                const uint32_t dn_next = __shfl_sync(0xFFFFFFFFu, nxt, lane_d);
                const uint32_t xd = hl + W < 32u ? dn_same : dn_next;  // the word below
                const uint32_t right = __funnelshift_r(cur, xr, 1);    // site x + 1
                up += __popc(cur);
                part += __popc(cur ^ right) + __popc(cur ^ xd);
                cur = nxt;
            }
            const uint32_t sum_up = __reduce_add_sync(0xFFFFFFFFu, up);
            const uint32_t sum_anti = __reduce_add_sync(0xFFFFFFFFu, part);
            __syncwarp();  // every lane has read the snapshot
            // the slot is free again (released before the global stores below,
            // which a release would otherwise wait for)
            if (hl == 0)
                asm volatile("st.release.cta.shared.u32 [%0], %1;" ::"r"(smem_addr(&slot_read[ks])),
                             "r"(cidx / SN + 1u)
                             : "memory");
            if (hl == 0) {
                const unsigned long long c0 = sum_up, c1 = sum_anti;
                const bool rec = cidx < A.nrec;
                const bool last = !rec || first + cidx * re + 1u == A.nsweeps;
                if (rec) {
                    A.acc[2 * cidx] = c0;
                    A.acc[2 * cidx + 1] = c1;
                }
                if (last) {
                    A.acc[2 * A.nrec] = c0;
                    A.acc[2 * A.nrec + 1] = c1;
                }
            }
        }
    }
    if constexpr (CL) cluster_barrier();  // no CTA leaves while another may still use its shared memory
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
    if (c.proc_bits == kTinyProcBits && (L == 64 || L == 128 || L == 256) && rows == L && c.block == kTinyWsBlock &&
        c.rows_per_item == 1 && c.regcap == 0 && c.insert == 0 && c.persistent == 0)
        // the warp-specialised kernels: one CTA (L = 64) or a cluster of 2, 4 or 8
        return (c.grid == 1 && L == 64) || c.grid == 2 || c.grid == 4 || c.grid == 8;
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

// The warp-specialised kernels (L = 64, 128 or 256): one CTA for L = 64, else
// a cluster of `ctas` CTAs whose first CTA holds the consumers.
template <uint32_t LL, bool CL>
static cudaError_t launch_wsc(const TinyRunArgs &a, uint32_t ctas, cudaStream_t s)
{
    using Shape = WsShape<LL, CL>;
    const size_t smem = Shape::smem(ctas);
    // the dynamic ring and snapshots (up to 176 KB at L = 256) with the static
    // arrays pass the 48 KB that need no opt-in
    cudaError_t e = cudaFuncSetAttribute(k_tiny_wsc<LL, CL>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    if constexpr (!CL) {
        k_tiny_wsc<LL, CL><<<1, kTinyWsBlock, smem, s>>>(a);
        return cudaGetLastError();
    } else {
        cudaLaunchConfig_t cfg{};
        cfg.gridDim = dim3(ctas);
        cfg.blockDim = dim3(kTinyWsBlock);
        cfg.dynamicSmemBytes = smem;
        cfg.stream = s;
        cudaLaunchAttribute attr{};
        attr.id = cudaLaunchAttributeClusterDimension;
        attr.val.clusterDim.x = ctas;
        attr.val.clusterDim.y = 1;
        attr.val.clusterDim.z = 1;
        cfg.attrs = &attr;
        cfg.numAttrs = 1;
        return cudaLaunchKernelEx(&cfg, k_tiny_wsc<LL, CL>, a);
    }
}

static cudaError_t launch_tiny_ws(const TinyRunArgs &a, uint32_t ctas, cudaStream_t s)
{
    if (ctas == 1) return a.L == 64 ? launch_wsc<64, false>(a, 1, s) : cudaErrorInvalidValue;
    if (ctas != 2 && ctas != 4 && ctas != 8) return cudaErrorInvalidValue;
    switch (a.L) {
    case 64: return launch_wsc<64, true>(a, ctas, s);
    case 128: return launch_wsc<128, true>(a, ctas, s);
    case 256: return launch_wsc<256, true>(a, ctas, s);
    default: return cudaErrorInvalidValue;
    }
}

cudaError_t launch_tiny(const TinyRunArgs &a, uint32_t block, uint32_t threads_per_word, uint32_t ctas,
                        cudaStream_t s)
{
    if (!tiny_lattice_ok(a.L) || a.nsweeps == 0) return cudaErrorInvalidValue;
    if ((a.L == 64 || a.L == 128 || a.L == 256) && block == kTinyWsBlock && threads_per_word == 1) {
        if (!a.use_field) return launch_tiny_ws(a, ctas, s);
        block = kTinyMaxThreads;  // in a field: the field kernels (no warp-specialised form)
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

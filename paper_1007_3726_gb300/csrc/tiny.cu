// Small lattices in one CTA: the whole lattice sits in shared memory for every
// sweep of a call, so a sweep costs two block barriers instead of two kernel
// launches (Sec. 5.2 needs one global synchronisation per checkerboard step;
// for a lattice that one CTA holds, a CTA barrier is that synchronisation).
//
// One thread per byte of the packed lattice: a byte of a row holds four target
// sites of a step, exactly the sites of one Philox4x32-10 call, so thread b
// owns Philox group b (= y L/8 + q for byte q of row y) and writes only its
// own byte.  The update of the byte is the update of Sec. 4 on eight bits:
// the neighbour bytes above and below, the row byte shifted by one with the
// carry bit from the adjacent byte, the bit-sliced count, the two threshold
// masks and the masked XOR.  Bits a thread reads from its neighbours' bytes
// at its own target positions are of the other parity, which nobody writes
// during the step.
#include "kernels.h"
#include "sweep_device.cuh"

namespace ising {

namespace {

constexpr uint32_t kTinyMaxThreads = 512;

__global__ void __launch_bounds__(kTinyMaxThreads) k_tiny(const __grid_constant__ TinyRunArgs A)
{
    extern __shared__ uint32_t smw[];
    __shared__ unsigned int cnt[2];
    uint8_t *const lat = reinterpret_cast<uint8_t *>(smw);
    const uint32_t L = (uint32_t)A.L;
    const uint32_t BPR = L >> 3;                 // bytes per row, a power of two
    const uint32_t lgB = 31 - __clz(BPR);
    const uint32_t nbytes = L * BPR;
    const uint32_t tid = threadIdx.x, nthr = blockDim.x;

    const uint32_t *src = static_cast<const uint32_t *>(A.spins);
    for (uint32_t i = tid; i < nbytes / 4; i += nthr) smw[i] = src[i];
    if (tid < 2) cnt[tid] = 0u;
    __syncthreads();

    HalfSweepArgs a;
    a.key = A.key;
    a.thr4 = A.thr4;
    a.thr8 = A.thr8;
    a.zero = 0u;
    uint32_t phase = A.record_every ? A.t0 % A.record_every : 0u;  // t % record_every
    uint32_t slot = 0;
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
            for (uint32_t b = tid; b < nbytes; b += nthr) {
                const uint32_t y = b >> lgB, q = b & (BPR - 1u);
                const uint32_t rowb = b - q;
                const uint32_t up = lat[(y == 0 ? nbytes - BPR : rowb - BPR) + q];
                const uint32_t dn = lat[(y + 1 == L ? 0u : rowb + BPR) + q];
                const uint32_t cur = lat[b];
                const uint32_t lb = lat[rowb + ((q - 1u) & (BPR - 1u))];
                const uint32_t rb = lat[rowb + ((q + 1u) & (BPR - 1u))];
                const uint32_t left = ((cur << 1) | (lb >> 7)) & 0xFFu;  // bit k holds s(x - 1)
                const uint32_t right = (cur >> 1) | ((rb & 1u) << 7);     // bit k holds s(x + 1)
                const uint32_t off = (y + p) & 1u;
                const uint32_t mask = 0x55u << off;

                const uint32_t i1 = cur ^ up, i2 = cur ^ dn, i3 = cur ^ left, i4 = cur ^ right;
                const uint32_t s12 = i1 ^ i2, c12 = i1 & i2;
                const uint32_t s34 = i3 ^ i4, c34 = i3 & i4;
                const uint32_t odd = s12 ^ s34;
                const uint32_t ge2 = c12 | c34 | (s12 & s34);
                const uint32_t eq1 = odd & ~ge2;
                const uint32_t eq0 = ~(odd | ge2);

                const WordDraws d = word_draws_begin(a, (uint64_t)b);
                uint32_t u[4];
                word_draw_call(a, d, 0u, u);
                uint32_t p4 = 0u, p8 = 0u;
#pragma unroll
                for (int l = 0; l < 4; ++l) {
                    p4 |= (u[l] < a.thr4) ? (1u << (2 * l)) : 0u;
                    p8 |= (u[l] < a.thr8) ? (1u << (2 * l)) : 0u;
                }
                const uint32_t flip = mask & (ge2 | (eq1 & (p4 << off)) | (eq0 & (p8 << off)));
                const uint32_t nw = cur ^ flip;
                lat[b] = (uint8_t)nw;
                if (count) {
                    cu += __popc(nw);
                    ca += __popc(mask & (nw ^ up)) + __popc(mask & (nw ^ dn)) + __popc(mask & (nw ^ left)) +
                          __popc(mask & (nw ^ right));
                }
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
    for (uint32_t i = tid; i < nbytes / 4; i += nthr) dst[i] = smw[i];
}

}  // namespace

cudaError_t launch_tiny(const TinyRunArgs &a, uint32_t block, cudaStream_t s)
{
    if (!tiny_lattice_ok(a.L) || a.nsweeps == 0 || block == 0 || block > kTinyMaxThreads || block % 32 != 0)
        return cudaErrorInvalidValue;
    const size_t smem = (size_t)(a.L * a.L / 8);
    if (smem > 48 * 1024) {
        const cudaError_t e = cudaFuncSetAttribute(k_tiny, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return e;
    }
    k_tiny<<<1, block, smem, s>>>(a);
    return cudaGetLastError();
}

}  // namespace ising

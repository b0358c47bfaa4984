// Integer-mix microbenchmark: how fast this GPU generates the sweep's random
// draws, with nothing else around them.  It is the measured peak against
// which the half-sweep's roofline fraction is also reported (the nominal
// INT32 peak counts every lane every clock at full rate, while the Philox
// widening multiplies issue at a quarter of that rate).
//
// Each thread plays the part of a step-kernel thread with 64-bit words: per
// "word" it makes the eight Philox4x32-10 calls of one word (32 draws), in one
// of three forms:
//   0  ten full rounds per call (2 widening multiplies and 2 three-input XORs
//      each): the plain Philox4x32-10 round mix;
//   1  the half-sweep's own form (rounds 1-2 partly hoisted: 17.5 widening
//      multiplies per call), the draws XOR-folded;
//   2  form 1 plus the acceptance masks (two compares and bit insertions per
//      draw, word_draw_masks), i.e. everything of the word update but the
//      lattice logic and memory.
// The counters are those of distinct words, so no call repeats another.
#include "ising.h"
#include "kernels.h"
#include "runtime.h"
#include "sweep_device.cuh"

#include <cuda_runtime.h>

namespace ising {
namespace {

template <int FORM>
__global__ void __launch_bounds__(512, 3) k_mixbench(const __grid_constant__ HalfSweepArgs a, uint32_t words,
                                                     uint32_t *out)
{
    const uint32_t tid = blockIdx.x * blockDim.x + threadIdx.x;
    const uint32_t nthr = gridDim.x * blockDim.x;
    uint32_t acc = 0u;
    for (uint32_t i = 0; i < words; ++i) {
        const uint64_t word = (uint64_t)i * nthr + tid;
        const uint64_t g0 = word * 8u;  // the word's first Philox group (8 calls per 64-bit word)
        if constexpr (FORM == 0) {
#pragma unroll
            for (uint32_t q = 0; q < 8; ++q) {
                uint32_t x0 = (uint32_t)(g0 + q), x1 = (uint32_t)((g0 + q) >> 32), x2 = a.t, x3 = a.c3;
                philox_rounds(x0, x1, x2, x3, a.key);
                acc ^= x0 ^ x1 ^ x2 ^ x3;
            }
        } else if constexpr (FORM == 1) {
            const WordDraws d = word_draws_begin(a, a, g0);
#pragma unroll
            for (uint32_t q = 0; q < 8; ++q) {
                uint32_t u[4];
                word_draw_call(a, a, d, q, u);
                acc ^= u[0] ^ u[1] ^ u[2] ^ u[3];
            }
        } else {
            uint32_t p4[2], p8[2];
            word_draw_masks<8, FORM == 3 ? 1 : 0>(a, a, g0, p4, p8);
            acc ^= p4[0] ^ p4[1] ^ p8[0] ^ p8[1];
        }
    }
    out[tid] = acc;  // keeps the work alive
}

using MixKernel = void (*)(HalfSweepArgs, uint32_t, uint32_t *);

MixKernel mix_kernel(uint32_t form)
{
    if (form == 0) return k_mixbench<0>;
    if (form == 1) return k_mixbench<1>;
    if (form == 3) return k_mixbench<3>;
    return k_mixbench<2>;
}

}  // namespace
}  // namespace ising

using namespace ising;

extern "C" ISING_API ising_status ising_bench_mix(uint32_t form, uint32_t words_per_thread, double *ms,
                                                  double *draws_per_ns, void *cuda_stream)
{
    clear_error();
    if (form > 3) return fail(ISING_ERR_INVALID, "form must be 0 .. 3");
    if (words_per_thread == 0 || words_per_thread > (1u << 20))
        return fail(ISING_ERR_INVALID, "words_per_thread must be in [1, 2^20]");
    if (!ms || !draws_per_ns) return fail(ISING_ERR_INVALID, "null output");
    cudaStream_t s = (cudaStream_t)cuda_stream;
    const MixKernel k = mix_kernel(form);
    int dev = 0, sms = 0, per_sm = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    const int block = 512;
    if (e == cudaSuccess) e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k, block, 0);
    if (e != cudaSuccess) return fail(ISING_ERR_CUDA, "ising_bench_mix: %s", cudaGetErrorString(e));
    if (per_sm < 1) per_sm = 1;
    const int grid = sms * per_sm;  // one full wave of resident blocks
    const uint64_t threads = (uint64_t)grid * block;

    HalfSweepArgs a{};
    a.key = make_round_keys(0x243F6A8885A308D3ull);
    a.thr4 = threshold_for(4.0, 2.269185);
    a.thr8 = threshold_for(8.0, 2.269185);
    a.t = 12345u;
    a.c3 = 1u;
    a.words_per_row = 1u;
    prepare_half_sweep(a, grid, block);

    uint32_t *out = nullptr;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    e = cudaMallocAsync((void **)&out, threads * sizeof(uint32_t), s);
    if (e == cudaSuccess) e = cudaEventCreate(&e0);
    if (e == cudaSuccess) e = cudaEventCreate(&e1);
    // one untimed warm-up launch, then the timed one
    if (e == cudaSuccess) {
        k<<<grid, block, 0, s>>>(a, words_per_thread < 4 ? words_per_thread : 4, out);
        e = cudaGetLastError();
    }
    if (e == cudaSuccess) e = cudaEventRecord(e0, s);
    if (e == cudaSuccess) {
        k<<<grid, block, 0, s>>>(a, words_per_thread, out);
        e = cudaGetLastError();
    }
    if (e == cudaSuccess) e = cudaEventRecord(e1, s);
    if (e == cudaSuccess) e = cudaEventSynchronize(e1);
    float t = 0.f;
    if (e == cudaSuccess) e = cudaEventElapsedTime(&t, e0, e1);
    if (out) cudaFreeAsync(out, s);
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
    if (e != cudaSuccess) return fail(ISING_ERR_CUDA, "ising_bench_mix: %s", cudaGetErrorString(e));
    *ms = t;
    *draws_per_ns = (double)threads * words_per_thread * 32.0 / ((double)t * 1e6);
    return ISING_OK;
}

// The checkerboard step in a nonzero external field H (Sec. 3, Eq. 1 keeps the
// term -H sum_i S_i; the paper then sets H = 0).
//
// Flipping S with c anti-aligned neighbours (neighbour sum n = S (4 - 2c))
// changes the energy by dE = 2 S (n + H) = 2 (4 - 2c) + 2 S H, so the
// acceptance depends on the class (S, c): ten classes instead of the three of
// the zero-field update.  The host fixes, per class, either "always" (dE <= 0)
// or the threshold floor(2^32 exp(-dE/T)) (Sec. 3: the factors are computed on
// the CPU per temperature and passed to the kernel).
//
// Per word the kernel forms the four neighbour words and the bit-sliced count
// c = b0 + 2 b1 + 4 b2 of the energy variables of Sec. 4, Eq. 4 (a full adder
// tree instead of the "c >= 2 / c == 1 / c == 0" split), then
//   always = S & [c >= k+] | ~S & [c >= k-]        (bit-parallel)
//   P      = bits of the sites whose draw u < thr[S, c]   (per site, a table
//            lookup in shared memory indexed by the site's 4-bit class)
//   flip   = target mask & (always | P).
// The draws are the same Philox4x32-10 words as in the zero-field update (the
// counter contract does not depend on H), so H = 0 reproduces it bit for bit.
// Lattices are processed 32 bits at a time whatever their storage width (a
// 64-bit word is two consecutive 32-bit words).
#include "field.h"
#include "field_device.cuh"

#include <atomic>

namespace ising {

namespace {

// Work item = (block of R rows, word column); the thread walks down its column
// as in the zero-field kernel.  Whole periodic lattice.  Three blocks of 512 per
// SM (a 40-register cap) ran 3 % faster than four of 256 at 62 registers.
__global__ void __launch_bounds__(512, 3) k_half_sweep_field(const __grid_constant__ HalfSweepArgs a,
                                                          const __grid_constant__ FieldTable ft)
{
    dependent_launch_wait();
    __shared__ uint32_t tab[16];
    if (threadIdx.x < 16) tab[threadIdx.x] = ft.thr[threadIdx.x];
    __syncthreads();

    uint32_t *const S = static_cast<uint32_t *>(a.spins);
    const uint64_t rows = a.rows;
    const uint32_t W = a.words_per_row;
    const uint32_t R = a.rows_per_item;
    const uint32_t nrb = (uint32_t)(rows / R);
    const uint64_t groups_per_row = a.L >> 3;

    unsigned int cnt_up = 0, cnt_anti = 0;
    const uint32_t tid = blockIdx.x * blockDim.x + threadIdx.x;
    uint32_t rb = tid / W;
    uint32_t w = tid - rb * W;
    while (rb < nrb) {
        const int64_t dl = (w == 0) ? (int64_t)W - 1 : -1;
        const int64_t dr = (w + 1 == W) ? 1 - (int64_t)W : 1;
        const uint64_t y0 = (uint64_t)rb * R;
        uint32_t *p = S + y0 * W + w;
        uint32_t up = *((y0 == 0) ? S + (rows - 1) * W + w : p - W);
        uint32_t cur = *p;
        uint64_t g = y0 * groups_per_row + (uint64_t)w * 4;
        uint32_t off = (uint32_t)((y0 + a.p) & 1u);
        for (uint32_t r = 0; r < R; ++r) {
            uint32_t *const pn = (y0 + r + 1 == rows) ? S + w : p + W;
            const uint32_t dn = *pn;
            const uint32_t nw = update_word_field(a, a, tab, ft.k_up, ft.k_dn, cur, up, dn, p[dl], p[dr], off, g,
                                                  a.acc != nullptr, cnt_up, cnt_anti);
            *p = nw;
            up = nw;
            cur = dn;
            p = pn;
            g += groups_per_row;
            off ^= 1u;
        }
        rb += a.stride_rb;
        w += a.stride_w;
        if (w >= W) {
            w -= W;
            ++rb;
        }
    }
    dependent_launch_trigger();
    if (a.acc) block_accumulate(cnt_up, cnt_anti, a.acc);
}

constexpr int kFieldBlock = 512;
constexpr int kMaxDevices = 64;

}  // namespace

// dE = 2 S (n + H) with n = S (4 - 2c), in FP64, as the class table.
FieldTable make_field_table(double T, double H)
{
    FieldTable f{};
    f.k_up = 5;
    f.k_dn = 5;
    for (int i = 0; i < 2; ++i) {
        const int v = i ? 1 : -1;
        for (int c = 4; c >= 0; --c) {
            const int nsum = v * (4 - 2 * c);
            const double dE = 2.0 * (double)v * ((double)nsum + H);
            if (dE <= 0.0) {
                // dE falls as c grows, so the always-accepted classes are c >= k
                (i ? f.k_up : f.k_dn) = (uint32_t)c;
                f.thr[8 * i + c] = 0u;
            } else {
                f.thr[8 * i + c] = threshold_for(dE, T);
            }
        }
    }
    return f;
}

cudaError_t launch_half_sweep_field(HalfSweepArgs a, const FieldTable &ft, cudaStream_t s)
{
    a.rows = a.L;
    a.first_row = 0;
    a.update_rows = a.L;
    a.y_offset = 0;
    a.words_per_row = (uint32_t)(a.L / 32);
    a.rows_per_item = 8;  // L is a multiple of 64
    a.zero = 0u;
    // SMs and resident blocks per SM of the device, queried once per device
    static std::atomic<int> sms_of[kMaxDevices], per_sm_of[kMaxDevices];
    int dev = 0;
    cudaGetDevice(&dev);
    const bool cached = dev >= 0 && dev < kMaxDevices;
    int sms = cached ? sms_of[dev].load(std::memory_order_relaxed) : 0;
    int per_sm = cached ? per_sm_of[dev].load(std::memory_order_relaxed) : 0;
    if (sms <= 0 || per_sm <= 0) {
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_half_sweep_field, kFieldBlock, 0);
        if (sms <= 0) sms = 1;
        if (per_sm <= 0) per_sm = 1;
        if (cached) {
            sms_of[dev].store(sms, std::memory_order_relaxed);
            per_sm_of[dev].store(per_sm, std::memory_order_relaxed);
        }
    }
    const int cap = sms * per_sm;
    const uint64_t items = (a.L / 8) * (uint64_t)a.words_per_row;
    const uint64_t need = (items + kFieldBlock - 1) / kFieldBlock;
    const int grid = (int)(need < (uint64_t)cap ? need : (uint64_t)cap);
    prepare_half_sweep(a, grid, kFieldBlock);
    // programmatic stream serialization, as the zero-field step kernels, except for
    // grids between half and twice the SM count, where it measured slower
    // (L = 4096: 440 against 510 attempts/ns)
    const bool dependent = grid < sms / 2 || grid >= 2 * sms;
    cudaLaunchConfig_t cfg{};
    cfg.gridDim = dim3((unsigned)grid);
    cfg.blockDim = dim3((unsigned)kFieldBlock);
    cfg.stream = s;
    cudaLaunchAttribute attr{};
    attr.id = cudaLaunchAttributeProgrammaticStreamSerialization;
    attr.val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = &attr;
    cfg.numAttrs = dependent ? 1 : 0;
    return cudaLaunchKernelEx(&cfg, k_half_sweep_field, a, ft);
}

}  // namespace ising

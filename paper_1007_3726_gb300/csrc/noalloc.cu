// ising_sweep_noalloc: the sweep for callers that cannot allocate memory.
//
// Some callers own every byte of device memory themselves and must not see
// the library call cudaMalloc: a serving process that has reserved its whole
// HBM budget up front in its own pool, a host application that lends device
// buffers to plug-ins and forbids them the CUDA allocator, or a loop that
// cannot afford the device-wide synchronisation a cudaMalloc / cudaFree may
// bring.  For them this entry point runs ising_sweep's kernels on a lattice the
// caller owns (the one-CTA or cluster kernel where ising_sweep's default takes
// it, the half-sweep step kernels otherwise), and keeps the kernels' scratch
// (the per-sweep M/E counters) in a fixed array compiled into the library
// instead of allocating it.
#include "ising.h"
#include "handle.h"
#include "kernels.h"
#include "runtime.h"

#include <cstdint>
#include <cstdlib>
#include <cstring>
#include <mutex>

using namespace ising;

namespace {

// Two 64-bit counters per recorded sweep (number of +1 spins, number of
// anti-aligned bonds), plus one slot for the state after the call's last sweep
// that the one-CTA and cluster kernels always write and one for their error
// flag.  Every GPU that loads the library holds this 1 MiB (and 32 bytes)
// until the process exits.
constexpr uint64_t kMaxRecords = ISING_NOALLOC_MAX_RECORDS;
static __device__ __align__(256) unsigned long long g_noalloc_counters[2 * (kMaxRecords + 2)];

constexpr int kMaxDevices = 64;
std::mutex g_setup_mu;
unsigned long long *g_counters_addr[kMaxDevices] = {};

// Device address of the counters on the current device, looked up once per
// device.  In host code g_noalloc_counters names a host-side stand-in, not
// device memory, so it must never be handed to a kernel directly.
ising_status counters_for_current_device(unsigned long long **out)
{
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return fail(ISING_ERR_CUDA, "cudaGetDevice: %s", cudaGetErrorString(e));
    if (dev < 0 || dev >= kMaxDevices) return fail(ISING_ERR_INVALID, "device %d out of range", dev);
    std::lock_guard<std::mutex> lk(g_setup_mu);
    if (!g_counters_addr[dev]) {
        void *p = nullptr;
        e = cudaGetSymbolAddress(&p, g_noalloc_counters);
        if (e != cudaSuccess || !p)
            return fail(ISING_ERR_CUDA, "cudaGetSymbolAddress: %s", cudaGetErrorString(e));
        g_counters_addr[dev] = static_cast<unsigned long long *>(p);
    }
    *out = g_counters_addr[dev];
    return ISING_OK;
}

}  // namespace

extern "C" ISING_API ising_status ising_sweep_noalloc(void *d_spins, uint64_t L, uint32_t word_bits,
                                                      double T, uint64_t seed, uint32_t stream_id,
                                                      uint64_t t0, uint64_t nsweeps,
                                                      uint32_t record_every, int64_t *M_out,
                                                      int64_t *E_out, uint64_t cap,
                                                      void *cuda_stream)
{
    clear_error();
    if (!d_spins) return fail(ISING_ERR_INVALID, "d_spins is NULL");
    // the kernels read the lattice in 32- to 128-bit units whatever word_bits it
    // was stored with
    if (reinterpret_cast<uintptr_t>(d_spins) % 16 != 0)
        return fail(ISING_ERR_INVALID, "d_spins must be 16-byte aligned");
    if (L < 64 || L % 64 != 0 || L > (1ull << 20))
        return fail(ISING_ERR_INVALID, "L must be a multiple of 64 in [64, 2^20]");
    if (word_bits != 32 && word_bits != 64) return fail(ISING_ERR_INVALID, "word_bits must be 32 or 64");
    if (!valid_temperature(T)) return fail(ISING_ERR_INVALID, "T must be finite and > 0");
    if (stream_id >= (1u << 31)) return fail(ISING_ERR_INVALID, "stream_id must be < 2^31");
    if (t0 >= 0xFFFFFFFFull || nsweeps >= 0xFFFFFFFFull - t0)
        return fail(ISING_ERR_INVALID, "sweep counter would reach 2^32 - 1");
    {
        // device (or managed) memory of the current device only: a host pointer
        // or another GPU's memory is refused before any work
        int dev = 0;
        cudaError_t e = cudaGetDevice(&dev);
        if (e != cudaSuccess) return fail(ISING_ERR_CUDA, "cudaGetDevice: %s", cudaGetErrorString(e));
        cudaPointerAttributes pa{};
        e = cudaPointerGetAttributes(&pa, d_spins);
        if (e != cudaSuccess) {
            cudaGetLastError();  // not sticky: clear it
            return fail(ISING_ERR_INVALID, "d_spins is not device memory (%s)", cudaGetErrorString(e));
        }
        if ((pa.type != cudaMemoryTypeDevice && pa.type != cudaMemoryTypeManaged) || pa.device != dev)
            return fail(ISING_ERR_INVALID, "d_spins must be device memory of the current device %d", dev);
    }
    if ((M_out == nullptr) != (E_out == nullptr))
        return fail(ISING_ERR_INVALID, "M_out and E_out must both be set or both be NULL");
    const uint64_t nrec = record_every ? (t0 + nsweeps) / record_every - t0 / record_every : 0;
    if (nrec > kMaxRecords)
        return fail(ISING_ERR_INVALID,
                    "%llu samples in one call exceed the fixed scratch of %llu; split the call",
                    (unsigned long long)nrec, (unsigned long long)kMaxRecords);
    if (nrec > 0 && !M_out) return fail(ISING_ERR_INVALID, "samples requested but M_out is NULL");
    if (M_out && cap < nrec) return fail(ISING_ERR_INVALID, "cap is smaller than the samples");
    if (nsweeps == 0) return ISING_OK;

    unsigned long long *acc = nullptr;
    ising_status st = counters_for_current_device(&acc);
    if (st != ISING_OK) return st;

    cudaStream_t s = (cudaStream_t)cuda_stream;
    cudaError_t e = cudaSuccess;
    // the counters keep the previous call's values: clear the ones this call adds into
    if (nrec) e = cudaMemsetAsync(acc, 0, nrec * 2 * sizeof(unsigned long long), s);

    HalfSweepArgs a{};
    a.spins = d_spins;
    a.L = L;
    a.rows = L;
    a.key = make_round_keys(seed);
    a.thr4 = threshold_for(4.0, T);
    a.thr8 = threshold_for(8.0, T);
    int dev = 0;
    cudaGetDevice(&dev);
    const LaunchConfig dflt = default_launch(dev, L, word_bits);
    if (dflt.proc_bits == kTinyProcBits) {
        // a lattice that one CTA or one cluster holds: every sweep in one launch,
        // as ising_sweep runs it; its last slot (after the final sweep) is unused here
        TinyRunArgs ta{};
        ta.spins = d_spins;
        ta.L = L;
        ta.key = a.key;
        ta.thr4 = a.thr4;
        ta.thr8 = a.thr8;
        ta.c3base = stream_id << 1;
        ta.t0 = (uint32_t)t0;
        ta.nsweeps = (uint32_t)nsweeps;
        ta.record_every = record_every;
        ta.nrec = (uint32_t)nrec;
        ta.acc = acc;
        // the cluster kernel adds into every slot it writes, the last one included;
        // the slot after it is the error flag of the one-CTA kernels
        ta.err = reinterpret_cast<unsigned int *>(acc + 2 * (nrec + 1));
        e = cudaMemsetAsync(acc, 0, (nrec + 2) * 2 * sizeof(unsigned long long), s);
        // launches of at most 2^30 sweeps (a launch counts its steps in 32 bits),
        // as in ising_sweep: launch k records from slot rec_done on, and its
        // final-state slot, the next launch's first sample slot, is cleared
        uint64_t max_chunk = 1ull << 30;
        if (const char *mx = std::getenv("ISING_TINY_MAX_SWEEPS")) {  // testing only
            const uint64_t v = std::strtoull(mx, nullptr, 10);
            if (v > 0 && v < max_chunk) max_chunk = v;
        }
        uint64_t done = 0, rec_done = 0;
        while (e == cudaSuccess && done < nsweeps) {
            const uint64_t n = nsweeps - done < max_chunk ? nsweeps - done : max_chunk;
            const uint64_t tc = t0 + done;
            const uint64_t nrec_c = record_every ? (tc + n) / record_every - tc / record_every : 0;
            if (done > 0) e = cudaMemsetAsync(acc + 2 * rec_done, 0, 2 * sizeof(unsigned long long), s);
            ta.t0 = (uint32_t)tc;
            ta.nsweeps = (uint32_t)n;
            ta.nrec = (uint32_t)nrec_c;
            ta.acc = acc + 2 * rec_done;
            if (e == cudaSuccess) e = launch_tiny(ta, dflt.block, dflt.rows_per_item, dflt.grid, s);
            done += n;
            rec_done += nrec_c;
        }
    }
    const LaunchConfig cfg = plain_launch(dflt);
    uint64_t slot = 0;
    for (uint64_t i = 0; dflt.proc_bits != kTinyProcBits && i < nsweeps && e == cudaSuccess; ++i) {
        const uint64_t t = t0 + i;
        a.t = (uint32_t)t;
        for (uint32_t p = 0; p < 2 && e == cudaSuccess; ++p) {
            a.p = p;
            a.c3 = (stream_id << 1) | p;
            a.acc = (p == 1 && record_every && (t + 1) % record_every == 0) ? acc + 2 * (slot++)
                                                                          : nullptr;
            e = launch_half_sweep(a, cfg, s);
        }
    }
    unsigned long long err_flag = 0;
    if (e == cudaSuccess && nrec && dflt.proc_bits == kTinyProcBits)
        e = cudaMemcpyAsync(&err_flag, acc + 2 * (nrec + 1), sizeof err_flag, cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess && nrec) {
        // column 0 of the counters into M_out, column 1 into E_out
        e = cudaMemcpy2DAsync(M_out, sizeof(int64_t), acc, 2 * sizeof(unsigned long long),
                              sizeof(int64_t), nrec, cudaMemcpyDeviceToHost, s);
        if (e == cudaSuccess)
            e = cudaMemcpy2DAsync(E_out, sizeof(int64_t), acc + 1, 2 * sizeof(unsigned long long),
                                  sizeof(int64_t), nrec, cudaMemcpyDeviceToHost, s);
    }
    if (e == cudaSuccess && nrec) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) return fail(ISING_ERR_CUDA, "ising_sweep_noalloc: %s", cudaGetErrorString(e));
    if (err_flag) return fail(ISING_ERR_TIMEOUT, "a wait inside the one-CTA kernel ran out; the lattice is lost");
    const int64_t N = (int64_t)(L * L);
    for (uint64_t i = 0; i < nrec; ++i) {
        M_out[i] = 2 * M_out[i] - N;      // +1 spins -> magnetisation
        E_out[i] = 2 * E_out[i] - 2 * N;  // anti-aligned bonds -> energy
    }
    return ISING_OK;
}

// Launch configurations of the half-sweep and the autotuner that picks one.
//
// The per-site random-number contract makes every configuration give the same
// bits, so the choice is purely a speed question: processing width (32 or 64
// lattice bits per thread and row), register cap (occupancy against
// instruction-level parallelism), block size and rows per work item.  The
// autotuner times each candidate with CUDA events on a scratch copy of the
// lattice and keeps the fastest per (device, L, storage word width).
#include "handle.h"
#include "kernels.h"
#include "runtime.h"

#include <cstdio>
#include <cstdlib>
#include <map>
#include <mutex>
#include <tuple>

using namespace ising;

namespace {
std::mutex g_tuned_mu;
std::map<std::tuple<int, uint64_t, uint32_t>, LaunchConfig> g_tuned;

ising_launch to_abi(const LaunchConfig &c)
{
    return ising_launch{c.proc_bits, c.regcap, c.block, c.rows_per_item, c.grid, c.insert, c.persistent};
}
LaunchConfig from_abi(const ising_launch &l)
{
    return LaunchConfig{l.proc_bits, l.regcap, l.insert, l.block, l.rows_per_item, l.grid, l.persistent};
}
}  // namespace

namespace ising {

LaunchConfig default_launch(int device, uint64_t L, uint32_t word_bits)
{
    {
        std::lock_guard<std::mutex> lk(g_tuned_mu);
        auto it = g_tuned.find(std::make_tuple(device, L, word_bits));
        if (it != g_tuned.end()) return it->second;
    }
    // untuned: the shapes the autotuner picked on GB300 at these sizes
    // (fields: proc_bits, regcap, insert, block, rows_per_item, grid)
    // every sweep of a call in one launch: the warp-specialised cluster kernel
    // (L = 64: 4 CTAs, L = 128 and 256: 8 CTAs), a cluster of 8 CTAs (L = 512)
    if (L == 64) return LaunchConfig{kTinyProcBits, 0, 0, kTinyWsBlock, 1, 4};
    if (L == 128 || L == 256) return LaunchConfig{kTinyProcBits, 0, 0, kTinyWsBlock, 1, 8};
    if (L == 512) return LaunchConfig{kTinyProcBits, 0, 0, 512, 1, 8};
    if (L < 4096) return LaunchConfig{32, 1, 0, 256, 2, 0};
    if (L < 16384) return LaunchConfig{64, 0, 0, 512, 4, 0};
    return LaunchConfig{64, 1, 0, 512, 8, 0};
}

void remember_launch(int device, uint64_t L, uint32_t word_bits, const LaunchConfig &c)
{
    std::lock_guard<std::mutex> lk(g_tuned_mu);
    g_tuned[std::make_tuple(device, L, word_bits)] = c;
}

std::vector<LaunchConfig> launch_candidates(uint64_t L, uint64_t rows)
{
    std::vector<LaunchConfig> out;
    // the one-CTA kernel, for lattices one CTA holds, and the warp-specialised
    // forms at L = 64 and 128 (one CTA at L = 64, or a cluster)
    for (uint32_t ctas : {1u, 2u, 4u, 8u}) {
        LaunchConfig ws{kTinyProcBits, 0, 0, kTinyWsBlock, 1, ctas};
        if (launch_config_valid(ws, L, rows)) out.push_back(ws);
    }
    for (uint32_t ctas : {1u, 2u, 4u, 8u})
        for (uint32_t blk : {128u, 256u, 512u})
            for (uint32_t tpw : {1u, 2u, 4u}) {
                LaunchConfig c{kTinyProcBits, 0, 0, blk, tpw, ctas};
                if (launch_config_valid(c, L, rows)) out.push_back(c);
            }
    for (uint32_t pb : {32u, 64u})
        for (uint32_t rc : {0u, 1u, 2u})
            for (uint32_t ins : {0u, 1u, 2u})
                for (uint32_t blk : {128u, 256u, 512u})
                    for (uint32_t R : {4u, 8u, 16u}) {
                        LaunchConfig c{pb, rc, ins, blk, R, 0};
                        if (launch_config_valid(c, L, rows)) out.push_back(c);
                    }
    // every sweep of a call in one cooperative launch, for the step shapes that
    // suit the lattices whose steps are short
    for (uint32_t pb : {32u, 64u})
        for (uint32_t rc : {0u, 1u, 2u})
            for (uint32_t blk : {256u, 512u})
                for (uint32_t R : {2u, 4u, 8u}) {
                    LaunchConfig c{pb, rc, 0, blk, R, 0, 1};
                    if (launch_config_valid(c, L, rows)) out.push_back(c);
                }
    // larger grids than the resident one (the block scheduler evens out the tail):
    // for the shapes that use all registers of the 40-register cap
    for (uint32_t pb : {32u, 64u})
        for (uint32_t blk : {256u, 512u})
            for (uint32_t R : {2u, 4u, 8u}) {
                LaunchConfig c{pb, 1, 0, blk, R, 0};
                if (!launch_config_valid(c, L, rows)) continue;
                const uint64_t items = rows / R * (L / pb);
                const uint64_t full = (items + blk - 1) / blk;
                for (uint64_t g : {full, full / 4})
                    if (g > 0 && g <= 65535u * 16u) {
                        c.grid = (uint32_t)g;
                        out.push_back(c);
                    }
            }
    return out;
}

}  // namespace ising

extern "C" {

ISING_API ising_status ising_get_launch(const ising_lattice *h, ising_launch *out)
{
    clear_error();
    if (!h || !out) return fail(ISING_ERR_INVALID, "null argument");
    *out = to_abi(h->launch);
    return ISING_OK;
}

ISING_API ising_status ising_set_launch(ising_lattice *h, const ising_launch *cfg)
{
    clear_error();
    if (!h || !cfg) return fail(ISING_ERR_INVALID, "null argument");
    const LaunchConfig c = from_abi(*cfg);
    if (!launch_config_valid(c, h->L, h->L))
        return fail(ISING_ERR_INVALID, "launch configuration not valid for L = %llu",
                    (unsigned long long)h->L);
    h->launch = c;
    return ISING_OK;
}

ISING_API uint32_t ising_launch_candidates(uint64_t L, ising_launch *out, uint32_t cap)
{
    const std::vector<LaunchConfig> v = launch_candidates(L, L);
    for (uint32_t i = 0; out && i < cap && i < v.size(); ++i) out[i] = to_abi(v[i]);
    return (uint32_t)v.size();
}

ISING_API ising_status ising_autotune(ising_lattice *h, uint32_t reps, ising_launch *best,
                                      double *best_us_per_step)
{
    clear_error();
    ising_status st = check_live(h);
    if (st != ISING_OK) return st;
    if ((st = harvest(h)) != ISING_OK) return st;
    if (reps == 0) reps = 3;

    // scratch: the first rows of the lattice, at most 256 MiB, a multiple of 64 rows
    const uint64_t row_bytes = h->L / 8;
    uint64_t rows = (256ull << 20) / row_bytes;
    rows = rows - rows % 64;
    if (rows < 64) rows = 64;
    if (rows > h->L) rows = h->L;
    void *scratch = h->alloc.allocate(rows * row_bytes, h->stream);
    if (!scratch) return fail(ISING_ERR_OOM, "cannot allocate the autotuning scratch");
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    cudaError_t e = cudaMemcpyAsync(scratch, h->d_spins, rows * row_bytes, cudaMemcpyDeviceToDevice,
                                    h->stream);
    if (e == cudaSuccess) e = cudaEventCreate(&e0);
    if (e == cudaSuccess) e = cudaEventCreate(&e1);

    HalfSweepArgs a{};
    a.spins = scratch;
    a.L = h->L;
    a.rows = rows;
    a.key = h->key;
    a.thr4 = h->thr4;
    a.thr8 = h->thr8;
    a.t = 0xFFFFFFF0u;  // any value: the scratch is thrown away
    LaunchConfig best_c = h->launch;
    double best_step_ms = 1e30;  // per checkerboard step
    const std::vector<LaunchConfig> cands = launch_candidates(h->L, rows);
    const char *log_env = std::getenv("ISING_AUTOTUNE_LOG");
    const bool log = log_env && log_env[0] == '1';
    for (size_t i = 0; i < cands.size() && e == cudaSuccess; ++i) {
        const LaunchConfig &c = cands[i];
        uint32_t steps = 2 * reps;
        if (c.persistent) {
            // one launch runs many sweeps: time one of 8 reps sweeps after a 1-sweep launch
            HalfSweepArgs pa{};
            pa.spins = scratch;
            pa.L = h->L;
            pa.key = h->key;
            pa.thr4 = h->thr4;
            pa.thr8 = h->thr8;
            SweepsRun sr{};
            sr.t0 = 0xFFFFF000u;  // any value: the scratch is thrown away
            sr.nsweeps = 1;
            sr.c3base = h->stream_id << 1;
            sr.acc = h->d_acc;
            e = launch_sweeps(pa, c, sr, h->stream);
            if (e == cudaSuccess) e = cudaEventRecord(e0, h->stream);
            sr.nsweeps = 8 * reps;
            if (e == cudaSuccess) e = launch_sweeps(pa, c, sr, h->stream);
            steps = 16 * reps;
        } else if (c.proc_bits == kTinyProcBits) {
            // one launch runs many sweeps: time one of 8 reps sweeps after a 1-sweep warm-up
            TinyRunArgs ta{};
            ta.spins = scratch;
            ta.L = h->L;
            ta.key = h->key;
            ta.thr4 = h->thr4;
            ta.thr8 = h->thr8;
            ta.c3base = h->stream_id << 1;
            ta.t0 = 0xFFFFF000u;  // any value: the scratch is thrown away
            ta.record_every = 0;
            ta.nrec = 0;
            ta.acc = h->d_acc;
            ta.err = reinterpret_cast<unsigned int *>(h->d_acc + 2);  // after the one state slot
            ta.nsweeps = 1;
            e = cudaMemsetAsync(h->d_acc + 2, 0, 16, h->stream);
            if (e == cudaSuccess) e = launch_tiny(ta, c.block, c.rows_per_item, c.grid, h->stream);
            if (e == cudaSuccess) e = cudaEventRecord(e0, h->stream);
            ta.nsweeps = 8 * reps;
            if (e == cudaSuccess) e = launch_tiny(ta, c.block, c.rows_per_item, c.grid, h->stream);
            steps = 16 * reps;
        }
        for (uint32_t r = 0; r <= reps && e == cudaSuccess && c.proc_bits != kTinyProcBits && !c.persistent; ++r) {
            if (r == 1) e = cudaEventRecord(e0, h->stream);
            for (uint32_t p = 0; p < 2 && e == cudaSuccess; ++p) {
                a.p = p;
                a.c3 = (h->stream_id << 1) | p;
                a.acc = p == 1 ? h->d_acc : nullptr;  // step B reduces, as when recording
                e = launch_half_sweep(a, c, h->stream);
            }
        }
        if (e == cudaSuccess) e = cudaEventRecord(e1, h->stream);
        if (e == cudaSuccess) e = cudaEventSynchronize(e1);
        if (e == cudaSuccess && c.proc_bits == kTinyProcBits) {
            unsigned int flag = 0;
            e = cudaMemcpy(&flag, h->d_acc + 2, sizeof flag, cudaMemcpyDeviceToHost);
            if (e == cudaSuccess && flag) {
                if (e0) cudaEventDestroy(e0);
                if (e1) cudaEventDestroy(e1);
                h->alloc.release(scratch, h->stream);
                h->failed = true;
                return fail(ISING_ERR_TIMEOUT, "a wait inside the one-CTA kernel ran out during autotuning");
            }
        }
        float ms = 0;
        if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
        const double step_ms = (double)ms / steps;
        if (e == cudaSuccess && log)
            std::fprintf(stderr, "autotune L=%llu rows=%llu proc_bits=%u regcap=%u insert=%u block=%u R=%u grid=%u persistent=%u: %.2f us/step\n",
                         (unsigned long long)h->L, (unsigned long long)rows, c.proc_bits, c.regcap,
                         c.insert, c.block, c.rows_per_item, c.grid, c.persistent, 1e3 * step_ms);
        if (e == cudaSuccess && step_ms < best_step_ms) {
            best_step_ms = step_ms;
            best_c = c;
        }
    }
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
    h->alloc.release(scratch, h->stream);
    if (e != cudaSuccess) return cuda_fail(h, e, "autotune");
    h->launch = best_c;
    remember_launch(h->device, h->L, h->word_bits, best_c);
    if (best) *best = to_abi(best_c);
    if (best_us_per_step) *best_us_per_step = 1e3 * best_step_ms * ((double)h->L / rows);
    return ISING_OK;
}

}  // extern "C"

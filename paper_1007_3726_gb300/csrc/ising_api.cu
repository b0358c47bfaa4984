// Host side of the C ABI declared in include/ising.h: validation, FP64
// thresholds (Sec. 3), memory and stream management, sample bookkeeping and
// FP64 moments.  All lattice arithmetic runs in the kernels of kernels.cu.
#include "ising.h"
#include "kernels.h"
#include "handle.h"
#include "runtime.h"

#include <algorithm>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <mutex>
#include <new>
#include <string>
#include <vector>

using namespace ising;

// ------------------------------------------------------------ errors -------
namespace {
thread_local std::string g_last_error;
}

namespace ising {

ising_status fail(ising_status st, const char *fmt, ...)
{
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof buf, fmt, ap);
    va_end(ap);
    g_last_error = buf;
    return st;
}

void clear_error() { g_last_error.clear(); }

// ------------------------------------------------------------ allocator ----
namespace {
std::mutex g_alloc_mu;
ising_alloc_fn g_alloc = nullptr;
ising_free_fn g_free = nullptr;
void *g_alloc_ctx = nullptr;
}  // namespace

Allocator current_allocator()
{
    std::lock_guard<std::mutex> lk(g_alloc_mu);
    return Allocator{g_alloc, g_free, g_alloc_ctx};
}

void *Allocator::allocate(size_t bytes, cudaStream_t s) const
{
    if (bytes == 0) bytes = 16;
    if (alloc) return alloc(bytes, (void *)s, ctx);
    void *p = nullptr;
    if (cudaMalloc(&p, bytes) != cudaSuccess) {
        cudaGetLastError();  // clear the (non-sticky) allocation error
        return nullptr;
    }
    return p;
}

void Allocator::release(void *p, cudaStream_t s) const
{
    if (!p) return;
    if (free_fn)
        free_fn(p, (void *)s, ctx);
    else
        cudaFree(p);
}

// ------------------------------------------------------------ thresholds ---
// floor(2^32 exp(-dE / T)) in FP64 (Sec. 3: the acceptance factors of the two
// positive energy changes are fixed on the CPU for each temperature).
uint32_t threshold_for(double dE, double T)
{
    const double v = std::floor(std::ldexp(std::exp(-dE / T), 32));
    if (v >= 4294967295.0) return 0xFFFFFFFFu;
    if (v <= 0.0) return 0u;
    return (uint32_t)v;
}

bool valid_temperature(double T) { return std::isfinite(T) && T > 0.0; }

}  // namespace ising

namespace ising {

int64_t to_M(const ising_lattice *h, unsigned long long up)
{
    return 2 * (int64_t)up - (int64_t)(h->L * h->L);
}
int64_t to_E(const ising_lattice *h, unsigned long long anti)
{
    return 2 * (int64_t)anti - 2 * (int64_t)(h->L * h->L);
}

ising_status cuda_fail(ising_lattice *h, cudaError_t e, const char *what)
{
    if (h) h->failed = true;
    return fail(ISING_ERR_CUDA, "%s: %s", what, cudaGetErrorString(e));
}

#define CK(h, expr)                                             \
    do {                                                        \
        cudaError_t e_ = (expr);                                \
        if (e_ != cudaSuccess) return cuda_fail((h), e_, #expr); \
    } while (0)

ising_status check_live(ising_lattice *h)
{
    if (!h) return fail(ISING_ERR_INVALID, "null handle");
    if (h->failed) return fail(ISING_ERR_STATE, "handle failed earlier; destroy it");
    cudaError_t e = cudaSetDevice(h->device);
    if (e != cudaSuccess) return cuda_fail(h, e, "cudaSetDevice");
    return ISING_OK;
}

// Reads back the samples of the last queued call.
ising_status harvest(ising_lattice *h)
{
    if (!h->pending) return ISING_OK;
    CK(h, cudaEventSynchronize(h->ev));
    if (h->pending_err && h->h_acc[2 * (h->pending_rec + 1)] != 0) {
        // a bounded wait in the kernel ran out: the lattice is not to be trusted
        h->pending = false;
        h->pending_err = false;
        h->failed = true;
        return fail(ISING_ERR_TIMEOUT, "a wait inside the one-CTA kernel ran out; the lattice is lost");
    }
    h->pending_err = false;
    for (size_t i = 0; i < h->pending_rec; ++i) {
        h->sM.push_back(to_M(h, h->h_acc[2 * i]));
        h->sE.push_back(to_E(h, h->h_acc[2 * i + 1]));
    }
    // the last slot always holds the state after the call's final sweep
    const size_t last = h->pending_rec;
    h->M = to_M(h, h->h_acc[2 * last]);
    h->E = to_E(h, h->h_acc[2 * last + 1]);
    h->pending = false;
    return ISING_OK;
}

ising_status ensure_acc(ising_lattice *h, size_t slots)
{
    if (slots <= h->acc_slots) return ISING_OK;
    size_t n = h->acc_slots ? h->acc_slots : 64;
    while (n < slots) n *= 2;
    CK(h, cudaStreamSynchronize(h->stream));
    unsigned long long *d = (unsigned long long *)h->alloc.allocate(n * 16, h->stream);
    if (!d) return fail(ISING_ERR_OOM, "cannot allocate %zu bytes of accumulators", n * 16);
    unsigned long long *hp = nullptr;
    if (cudaHostAlloc((void **)&hp, n * 16, cudaHostAllocDefault) != cudaSuccess) {
        cudaGetLastError();
        h->alloc.release(d, h->stream);
        return fail(ISING_ERR_OOM, "cannot allocate %zu bytes of pinned host memory", n * 16);
    }
    h->alloc.release(h->d_acc, h->stream);
    if (h->h_acc) cudaFreeHost(h->h_acc);
    h->d_acc = d;
    h->h_acc = hp;
    h->acc_slots = n;
    return ISING_OK;
}

void destroy_all(ising_lattice *h)
{
    if (!h) return;
    cudaSetDevice(h->device);
    cudaStreamSynchronize(h->stream);
    h->alloc.release(h->d_base, h->stream);
    h->alloc.release(h->d_acc, h->stream);
    if (h->h_acc) cudaFreeHost(h->h_acc);
    if (h->ev) cudaEventDestroy(h->ev);
    delete h;
}

ising_status count_state(ising_lattice *h)
{
    CK(h, cudaMemsetAsync(h->d_acc, 0, 16, h->stream));
    CK(h, launch_recount(h->d_spins, h->L, h->word_bits, h->d_acc, h->stream));
    CK(h, cudaMemcpyAsync(h->h_acc, h->d_acc, 16, cudaMemcpyDeviceToHost, h->stream));
    CK(h, cudaStreamSynchronize(h->stream));
    h->M = to_M(h, h->h_acc[0]);
    h->E = to_E(h, h->h_acc[1]);
    return ISING_OK;
}

ising_status validate_params(const ising_params *p, uint32_t *word_bits)
{
    if (!p) return fail(ISING_ERR_INVALID, "params is NULL");
    if (p->L < 64 || p->L % 64 != 0 || p->L > (1ull << 20))
        return fail(ISING_ERR_INVALID, "L must be a multiple of 64 in [64, 2^20], got %llu",
                    (unsigned long long)p->L);
    if (!valid_temperature(p->T)) return fail(ISING_ERR_INVALID, "T must be finite and > 0");
    if (!std::isfinite(p->H)) return fail(ISING_ERR_INVALID, "H must be finite");
    if (p->stream_id >= (1u << 31)) return fail(ISING_ERR_INVALID, "stream_id must be < 2^31");
    if (p->init < ISING_COLD_UP || p->init > ISING_FROM_PACKED)
        return fail(ISING_ERR_INVALID, "unknown init mode %d", (int)p->init);
    if ((p->init == ISING_FROM_BUFFER || p->init == ISING_FROM_PACKED) && !p->init_data)
        return fail(ISING_ERR_INVALID, "init_data is NULL");
    if (p->first_sweep >= 0xFFFFFFFFull) return fail(ISING_ERR_INVALID, "first_sweep must be < 2^32 - 1");
    uint32_t wb = p->word_bits;
    if (wb == 0) wb = p->L >= 65536 ? 64 : 32;
    if (wb != 32 && wb != 64) return fail(ISING_ERR_INVALID, "word_bits must be 0, 32 or 64");
    *word_bits = wb;
    return ISING_OK;
}

}  // namespace ising

// ------------------------------------------------------------ ABI ----------
extern "C" {

const char *ising_last_error(void) { return g_last_error.c_str(); }

ising_status ising_thresholds(double T, uint32_t *thr4, uint32_t *thr8)
{
    if (!thr4 || !thr8) return fail(ISING_ERR_INVALID, "null output");
    if (!valid_temperature(T)) return fail(ISING_ERR_INVALID, "T must be finite and > 0");
    *thr4 = threshold_for(4.0, T);
    *thr8 = threshold_for(8.0, T);
    return ISING_OK;
}

ising_status ising_field_thresholds(double T, double H, uint32_t thr[10], uint8_t always[10])
{
    if (!thr || !always) return fail(ISING_ERR_INVALID, "null output");
    if (!valid_temperature(T)) return fail(ISING_ERR_INVALID, "T must be finite and > 0");
    if (!std::isfinite(H)) return fail(ISING_ERR_INVALID, "H must be finite");
    const FieldTable f = make_field_table(T, H);
    for (int i = 0; i < 2; ++i)
        for (int c = 0; c < 5; ++c) {
            thr[5 * i + c] = f.thr[8 * i + c];
            always[5 * i + c] = (uint32_t)c >= (i ? f.k_up : f.k_dn);
        }
    return ISING_OK;
}

ising_status ising_set_temperature(ising_lattice *h, double T)
{
    clear_error();
    if (!h) return fail(ISING_ERR_INVALID, "null handle");
    if (h->failed) return fail(ISING_ERR_STATE, "handle failed earlier; destroy it");
    if (!valid_temperature(T)) return fail(ISING_ERR_INVALID, "T must be finite and > 0");
    h->T = T;
    h->thr4 = threshold_for(4.0, T);
    h->thr8 = threshold_for(8.0, T);
    h->field = make_field_table(T, h->H);
    return ISING_OK;
}

ising_status ising_set_field(ising_lattice *h, double H)
{
    clear_error();
    if (!h) return fail(ISING_ERR_INVALID, "null handle");
    if (h->failed) return fail(ISING_ERR_STATE, "handle failed earlier; destroy it");
    if (!std::isfinite(H)) return fail(ISING_ERR_INVALID, "H must be finite");
    h->H = H;
    h->field = make_field_table(h->T, H);
    return ISING_OK;
}

ising_status ising_get_params(const ising_lattice *h, double *T, double *H)
{
    clear_error();
    if (!h) return fail(ISING_ERR_INVALID, "null handle");
    if (T) *T = h->T;
    if (H) *H = h->H;
    return ISING_OK;
}

ising_status ising_set_allocator(ising_alloc_fn alloc, ising_free_fn release, void *ctx)
{
    if ((alloc == nullptr) != (release == nullptr))
        return fail(ISING_ERR_INVALID, "alloc and release must both be set or both be NULL");
    std::lock_guard<std::mutex> lk(g_alloc_mu);
    g_alloc = alloc;
    g_free = release;
    g_alloc_ctx = ctx;
    return ISING_OK;
}

ising_status ising_create(const ising_params *params, void *cuda_stream, ising_lattice **out)
{
    clear_error();
    if (!out) return fail(ISING_ERR_INVALID, "out is NULL");
    *out = nullptr;
    uint32_t wb = 0;
    ising_status st = validate_params(params, &wb);
    if (st != ISING_OK) return st;

    ising_lattice *h = new (std::nothrow) ising_lattice();
    if (!h) return fail(ISING_ERR_OOM, "host allocation failed");
    h->L = params->L;
    h->T = params->T;
    h->seed = params->seed;
    h->stream_id = params->stream_id;
    h->word_bits = wb;
    h->W = (uint32_t)(params->L / wb);
    h->thr4 = threshold_for(4.0, params->T);
    h->thr8 = threshold_for(8.0, params->T);
    h->H = params->H;
    h->field = make_field_table(params->T, params->H);
    h->bytes = (size_t)(params->L * params->L / 8);
    h->stream = (cudaStream_t)cuda_stream;
    h->alloc = current_allocator();
    h->key = make_round_keys(params->seed);
    h->sweeps_done = params->first_sweep;
    cudaError_t e = cudaGetDevice(&h->device);
    if (e != cudaSuccess) {
        delete h;
        return fail(ISING_ERR_CUDA, "cudaGetDevice: %s", cudaGetErrorString(e));
    }
    auto bail = [&](ising_status s) {
        std::string msg = g_last_error;
        destroy_all(h);
        g_last_error = msg;
        return s;
    };
    if (cudaEventCreateWithFlags(&h->ev, cudaEventDisableTiming) != cudaSuccess) {
        cudaGetLastError();
        h->ev = nullptr;
        return bail(fail(ISING_ERR_CUDA, "cudaEventCreate failed"));
    }
    h->d_base = h->alloc.allocate(h->bytes + 2 * kGuardBytes, h->stream);
    if (!h->d_base)
        return bail(fail(ISING_ERR_OOM, "cannot allocate %zu bytes for the lattice", h->bytes));
    h->d_spins = static_cast<char *>(h->d_base) + kGuardBytes;
    e = cudaMemsetAsync(h->d_base, kGuardByte, kGuardBytes, h->stream);
    if (e == cudaSuccess)
        e = cudaMemsetAsync(static_cast<char *>(h->d_spins) + h->bytes, kGuardByte, kGuardBytes, h->stream);
    if (e != cudaSuccess) return bail(cuda_fail(h, e, "guard bytes"));
    if ((st = ensure_acc(h, 64)) != ISING_OK) return bail(st);

    h->launch = default_launch(h->device, h->L, wb);

    // initial state
    switch (params->init) {
    case ISING_COLD_UP:
        e = cudaMemsetAsync(h->d_spins, 0xFF, h->bytes, h->stream);
        break;
    case ISING_COLD_DOWN:
        e = cudaMemsetAsync(h->d_spins, 0x00, h->bytes, h->stream);
        break;
    case ISING_HOT:
        e = launch_init_hot(h->d_spins, h->L, wb, h->seed, h->stream_id, h->stream);
        break;
    case ISING_FROM_PACKED:
        e = cudaMemcpyAsync(h->d_spins, params->init_data, h->bytes, cudaMemcpyHostToDevice,
                            h->stream);
        break;
    case ISING_FROM_BUFFER: {
        const size_t n = (size_t)(h->L * h->L);
        int8_t *tmp = (int8_t *)h->alloc.allocate(n, h->stream);
        if (!tmp) return bail(fail(ISING_ERR_OOM, "cannot allocate %zu bytes of staging", n));
        e = cudaMemsetAsync(h->d_acc, 0, 16, h->stream);
        if (e == cudaSuccess)
            e = cudaMemcpyAsync(tmp, params->init_data, n, cudaMemcpyHostToDevice, h->stream);
        if (e == cudaSuccess)
            e = launch_pack(tmp, h->d_spins, h->L, wb, (unsigned int *)h->d_acc, h->stream);
        if (e == cudaSuccess)
            e = cudaMemcpyAsync(h->h_acc, h->d_acc, 16, cudaMemcpyDeviceToHost, h->stream);
        if (e == cudaSuccess) e = cudaStreamSynchronize(h->stream);
        h->alloc.release(tmp, h->stream);
        if (e == cudaSuccess && ((unsigned int *)h->h_acc)[0] != 0)
            return bail(fail(ISING_ERR_INVALID, "init_data holds %u values that are not +1/-1",
                             ((unsigned int *)h->h_acc)[0]));
        break;
    }
    default:
        break;
    }
    if (e != cudaSuccess) return bail(cuda_fail(h, e, "initial state"));
    if ((st = count_state(h)) != ISING_OK) return bail(st);
    *out = h;
    return ISING_OK;
}

ising_status ising_destroy(ising_lattice *h)
{
    clear_error();
    if (!h) return ISING_OK;
    destroy_all(h);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return fail(ISING_ERR_CUDA, "destroy: %s", cudaGetErrorString(e));
    return ISING_OK;
}

ising_status ising_sweep(ising_lattice *h, uint64_t nsweeps, uint32_t record_every, int64_t *M_out,
                         int64_t *E_out, uint64_t cap)
{
    clear_error();
    NvtxRange range("ising_sweep");
    ising_status st = check_live(h);
    if (st != ISING_OK) return st;
    if ((M_out == nullptr) != (E_out == nullptr))
        return fail(ISING_ERR_INVALID, "M_out and E_out must both be set or both be NULL");
    if (h->sweeps_done + nsweeps >= 0xFFFFFFFFull)
        return fail(ISING_ERR_INVALID, "sweep counter would reach 2^32 - 1");
    if (nsweeps == 0) return ISING_OK;

    const uint64_t t0 = h->sweeps_done;
    uint64_t nrec = 0;
    if (record_every)
        nrec = (t0 + nsweeps) / record_every - t0 / record_every;
    if (M_out && cap < nrec)
        return fail(ISING_ERR_INVALID, "cap %llu < %llu samples of this call",
                    (unsigned long long)cap, (unsigned long long)nrec);
    if ((st = harvest(h)) != ISING_OK) return st;
    if ((st = ensure_acc(h, nrec + 2)) != ISING_OK) return st;

    CK(h, cudaMemsetAsync(h->d_acc, 0, (nrec + 2) * 16, h->stream));
    if (h->launch.proc_bits == kTinyProcBits) {
        // the whole call in one launch of one CTA
        TinyRunArgs ta{};
        ta.spins = h->d_spins;
        ta.L = h->L;
        ta.key = h->key;
        ta.thr4 = h->thr4;
        ta.thr8 = h->thr8;
        ta.c3base = h->stream_id << 1;
        ta.t0 = (uint32_t)t0;
        ta.nsweeps = (uint32_t)nsweeps;
        ta.record_every = record_every;
        ta.nrec = (uint32_t)nrec;
        ta.acc = h->d_acc;
        if (h->H != 0.0) {
            ta.use_field = 1;
            for (int k = 0; k < 16; ++k) ta.field_thr[k] = h->field.thr[k];
            ta.k_up = h->field.k_up;
            ta.k_dn = h->field.k_dn;
        }
        ta.err = reinterpret_cast<unsigned int *>(h->d_acc + 2 * (nrec + 1));
        {
            // failure-detection testing only (see include/ising.h)
            const char *hold = std::getenv("ISING_TINY_HOLD_STEP");
            ta.hold_step = hold ? (uint32_t)std::strtoul(hold, nullptr, 10) : 0u;
        }
        // A launch counts its checkerboard steps (2 per sweep) in 32 bits: a
        // longer call runs as several launches of at most 2^30 sweeps.  Launch k
        // records its samples from slot rec_done on; its final-state slot is the
        // next launch's first sample slot, cleared in between (some of these
        // kernels add their counts into the slots).
        uint64_t max_chunk = 1ull << 30;
        if (const char *mx = std::getenv("ISING_TINY_MAX_SWEEPS")) {  // testing only
            const uint64_t v = std::strtoull(mx, nullptr, 10);
            if (v > 0 && v < max_chunk) max_chunk = v;
        }
        uint64_t done = 0, rec_done = 0;
        while (done < nsweeps) {
            const uint64_t n = std::min(nsweeps - done, max_chunk);
            const uint64_t tc = t0 + done;
            const uint64_t nrec_c = record_every ? (tc + n) / record_every - tc / record_every : 0;
            if (done > 0) CK(h, cudaMemsetAsync(h->d_acc + 2 * rec_done, 0, 16, h->stream));
            ta.t0 = (uint32_t)tc;
            ta.nsweeps = (uint32_t)n;
            ta.nrec = (uint32_t)nrec_c;
            ta.acc = h->d_acc + 2 * rec_done;
            CK(h, launch_tiny(ta, h->launch.block, h->launch.rows_per_item, h->launch.grid, h->stream));
            done += n;
            rec_done += nrec_c;
        }
        h->pending_err = true;
        return finish_sweep_call(h, t0, nsweeps, nrec, M_out, E_out);
    }
    if (h->launch.persistent && h->H == 0.0) {
        // the whole call in one cooperative launch
        HalfSweepArgs a{};
        a.spins = h->d_spins;
        a.L = h->L;
        a.key = h->key;
        a.thr4 = h->thr4;
        a.thr8 = h->thr8;
        SweepsRun sr{};
        sr.t0 = (uint32_t)t0;
        sr.nsweeps = (uint32_t)nsweeps;
        sr.record_every = record_every;
        sr.nrec = (uint32_t)nrec;
        sr.c3base = h->stream_id << 1;
        sr.acc = h->d_acc;
        CK(h, launch_sweeps(a, h->launch, sr, h->stream));
        return finish_sweep_call(h, t0, nsweeps, nrec, M_out, E_out);
    }
    HalfSweepArgs a{};
    a.spins = h->d_spins;
    a.L = h->L;
    a.rows = h->L;
    a.key = h->key;
    a.thr4 = h->thr4;
    a.thr8 = h->thr8;
    size_t slot = 0;
    for (uint64_t i = 0; i < nsweeps; ++i) {
        const uint64_t t = t0 + i;
        a.t = (uint32_t)t;
        for (uint32_t p = 0; p < 2; ++p) {
            a.p = p;
            a.c3 = (h->stream_id << 1) | p;
            a.acc = nullptr;
            if (p == 1) {
                const bool rec = record_every && ((t + 1) % record_every == 0);
                if (rec)
                    a.acc = h->d_acc + 2 * (slot++);
                else if (i + 1 == nsweeps)
                    a.acc = h->d_acc + 2 * nrec;  // state after the call
            }
            if (h->H != 0.0)
                CK(h, launch_half_sweep_field(a, h->field, h->stream));
            else
                CK(h, launch_half_sweep(a, plain_launch(h->launch), h->stream));
        }
    }
    if (slot == nrec && nrec > 0 && record_every && (t0 + nsweeps) % record_every == 0) {
        // the final sweep was recorded: copy its counters into the "state" slot too
        CK(h, cudaMemcpyAsync(h->d_acc + 2 * nrec, h->d_acc + 2 * (nrec - 1), 16,
                              cudaMemcpyDeviceToDevice, h->stream));
    }
    return finish_sweep_call(h, t0, nsweeps, nrec, M_out, E_out);
}

}  // extern "C"

namespace ising {

// Queues the read-back of a call's counters; with M_out, waits and copies the
// call's samples out.
ising_status finish_sweep_call(ising_lattice *h, uint64_t t0, uint64_t nsweeps, uint64_t nrec, int64_t *M_out,
                               int64_t *E_out)
{
    ising_status st;
    CK(h, cudaMemcpyAsync(h->h_acc, h->d_acc, (nrec + (h->pending_err ? 2 : 1)) * 16, cudaMemcpyDeviceToHost,
                          h->stream));
    CK(h, cudaEventRecord(h->ev, h->stream));
    h->sweeps_done = t0 + nsweeps;
    h->pending = true;
    h->pending_rec = nrec;
    if (M_out) {
        const size_t base = h->sM.size();
        if ((st = harvest(h)) != ISING_OK) return st;
        for (size_t i = 0; i < nrec; ++i) {
            M_out[i] = h->sM[base + i];
            E_out[i] = h->sE[base + i];
        }
    }
    return ISING_OK;
}

}  // namespace ising

extern "C" {

ising_status ising_measure_from(ising_lattice *h, uint64_t first_sample, ising_obs *out)
{
    clear_error();
    ising_status st = check_live(h);
    if (st != ISING_OK) return st;
    if (!out) return fail(ISING_ERR_INVALID, "out is NULL");
    if ((st = harvest(h)) != ISING_OK) return st;
    CK(h, cudaStreamSynchronize(h->stream));
    std::memset(out, 0, sizeof *out);
    out->sweeps_done = h->sweeps_done;
    out->n_samples = h->sM.size() > first_sample ? h->sM.size() - first_sample : 0;
    out->M = h->M;
    out->E = h->E;
    const size_t n = h->sM.size();
    if (out->n_samples == 0) return ISING_OK;
    // plain FP64 sums in sample order
    const double N = (double)h->L * (double)h->L;
    double sm = 0, sa = 0, s2 = 0, s4 = 0, se = 0, se2 = 0;
    for (size_t i = (size_t)first_sample; i < n; ++i) {
        const double m = (double)h->sM[i] / N;
        const double e = (double)h->sE[i] / N;
        sm += m;
        sa += std::fabs(m);
        s2 += m * m;
        s4 += m * m * m * m;
        se += e;
        se2 += e * e;
    }
    const double k = (double)(n - first_sample);
    out->mean_m = sm / k;
    out->mean_abs_m = sa / k;
    out->mean_m2 = s2 / k;
    out->mean_m4 = s4 / k;
    out->mean_e = se / k;
    out->mean_e2 = se2 / k;
    out->U4 = 1.0 - out->mean_m4 / (3.0 * out->mean_m2 * out->mean_m2);
    out->chi = N * (out->mean_m2 - out->mean_abs_m * out->mean_abs_m) / h->T;
    out->C = N * (out->mean_e2 - out->mean_e * out->mean_e) / (h->T * h->T);
    return ISING_OK;
}

ising_status ising_measure(ising_lattice *h, ising_obs *out) { return ising_measure_from(h, 0, out); }

ising_status ising_get_spins(ising_lattice *h, uint64_t row0, uint64_t nrows, int8_t *out)
{
    clear_error();
    ising_status st = check_live(h);
    if (st != ISING_OK) return st;
    if (!out && nrows) return fail(ISING_ERR_INVALID, "out is NULL");
    if (row0 >= h->L || nrows > h->L)
        return fail(ISING_ERR_INVALID, "rows out of range");
    if (nrows == 0) return ISING_OK;
    if ((st = harvest(h)) != ISING_OK) return st;
    const size_t n = (size_t)(nrows * h->L);
    int8_t *tmp = (int8_t *)h->alloc.allocate(n, h->stream);
    if (!tmp) return fail(ISING_ERR_OOM, "cannot allocate %zu bytes of staging", n);
    cudaError_t e = launch_unpack(h->d_spins, h->L, h->word_bits, row0, nrows, tmp, h->stream);
    if (e == cudaSuccess) e = cudaMemcpyAsync(out, tmp, n, cudaMemcpyDeviceToHost, h->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(h->stream);
    h->alloc.release(tmp, h->stream);
    if (e != cudaSuccess) return cuda_fail(h, e, "get_spins");
    return ISING_OK;
}

ising_status ising_get_packed(ising_lattice *h, void *out, size_t bytes)
{
    clear_error();
    ising_status st = check_live(h);
    if (st != ISING_OK) return st;
    if (!out || bytes != h->bytes)
        return fail(ISING_ERR_INVALID, "need a buffer of exactly %zu bytes", h->bytes);
    if ((st = harvest(h)) != ISING_OK) return st;
    CK(h, cudaMemcpyAsync(out, h->d_spins, h->bytes, cudaMemcpyDeviceToHost, h->stream));
    CK(h, cudaStreamSynchronize(h->stream));
    return ISING_OK;
}

ising_status ising_recount(ising_lattice *h, int64_t *M, int64_t *E)
{
    clear_error();
    ising_status st = check_live(h);
    if (st != ISING_OK) return st;
    if (!M || !E) return fail(ISING_ERR_INVALID, "null output");
    if ((st = harvest(h)) != ISING_OK) return st;
    CK(h, cudaMemsetAsync(h->d_acc, 0, 16, h->stream));
    CK(h, launch_recount(h->d_spins, h->L, h->word_bits, h->d_acc, h->stream));
    CK(h, cudaMemcpyAsync(h->h_acc, h->d_acc, 16, cudaMemcpyDeviceToHost, h->stream));
    CK(h, cudaStreamSynchronize(h->stream));
    *M = to_M(h, h->h_acc[0]);
    *E = to_E(h, h->h_acc[1]);
    return ISING_OK;
}

ising_status ising_get_samples(ising_lattice *h, uint64_t first, uint64_t count, int64_t *M, int64_t *E,
                               uint64_t *n_out)
{
    clear_error();
    ising_status st = check_live(h);
    if (st != ISING_OK) return st;
    if ((st = harvest(h)) != ISING_OK) return st;
    const uint64_t have = h->sM.size();
    const uint64_t n = first >= have ? 0 : std::min<uint64_t>(count, have - first);
    if (n_out) *n_out = n;
    if (n && (!M || !E)) return fail(ISING_ERR_INVALID, "null output");
    for (uint64_t i = 0; i < n; ++i) {
        M[i] = h->sM[first + i];
        E[i] = h->sE[first + i];
    }
    return ISING_OK;
}

ising_status ising_info(const ising_lattice *h, uint32_t *word_bits, uint64_t *L,
                        uint64_t *sweeps_done)
{
    clear_error();
    if (!h) return fail(ISING_ERR_INVALID, "null handle");
    if (word_bits) *word_bits = h->word_bits;
    if (L) *L = h->L;
    if (sweeps_done) *sweeps_done = h->sweeps_done;
    return ISING_OK;
}

ising_status ising_check_guards(ising_lattice *h, uint32_t *intact)
{
    clear_error();
    ising_status st = check_live(h);
    if (st != ISING_OK) return st;
    if (!intact) return fail(ISING_ERR_INVALID, "intact is NULL");
    unsigned char g[2 * kGuardBytes];
    CK(h, cudaMemcpyAsync(g, h->d_base, kGuardBytes, cudaMemcpyDeviceToHost, h->stream));
    CK(h, cudaMemcpyAsync(g + kGuardBytes, static_cast<char *>(h->d_spins) + h->bytes, kGuardBytes,
                          cudaMemcpyDeviceToHost, h->stream));
    CK(h, cudaStreamSynchronize(h->stream));
    uint32_t ok = 1;
    for (size_t i = 0; i < 2 * kGuardBytes; ++i) ok &= (g[i] == kGuardByte);
    *intact = ok;
    return ISING_OK;
}

ising_status ising_device_spins(const ising_lattice *h, void **dptr, size_t *bytes)
{
    clear_error();
    if (!h || !dptr || !bytes) return fail(ISING_ERR_INVALID, "null argument");
    *dptr = h->d_spins;
    *bytes = h->bytes;
    return ISING_OK;
}

}  // extern "C"

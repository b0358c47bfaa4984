// Request server: simulations arrive at any time, are admitted against a
// device-memory budget, stay resident on the GPU, and advance together in
// persistent multi-lattice launches (continuous batching: a request that
// arrives while others run joins at the next launch, a finished one leaves and
// frees its memory).  The per-site random-number contract makes every
// request's trajectory independent of what else shares the launch, so its
// samples are bit-identical to running it alone.
#include "batch_internal.h"
#include "handle.h"
#include "runtime.h"

#include <algorithm>
#include <chrono>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <mutex>
#include <string>
#include <thread>
#include <unordered_map>
#include <vector>

using namespace ising;

namespace {

struct Request {
    uint64_t id = 0;
    ising_request req{};
    ising_result res{};
    ising_lattice *h = nullptr;
    uint64_t remaining = 0;
    size_t bytes = 0;
    bool cancel = false;
    std::vector<int64_t> M, E;
};

size_t request_bytes(const ising_request &r)
{
    const uint64_t L = r.params.L;
    const uint64_t n = r.record_every ? r.nsweeps / r.record_every + 2 : 2;
    return (size_t)(L * L / 8) + (size_t)n * 16 + 4096;
}

}  // namespace

struct ising_server {
    ising_server_opts opts{};
    int device = 0;
    cudaStream_t stream = nullptr;
    std::chrono::steady_clock::time_point t0;
    std::thread worker;
    std::mutex mu;
    std::condition_variable cv_work, cv_done;
    bool stop = false;
    uint64_t next_id = 1;
    std::deque<Request *> incoming;                 // submitted, not yet seen by the worker
    std::deque<Request *> queue;                    // waiting for admission, in arrival order
    std::vector<Request *> resident;                // admitted, in admission order
    std::deque<Request *> finished;                 // results not yet polled
    std::unordered_map<uint64_t, Request *> kept;   // polled results whose samples are kept
    ising_server_counters stats{};
    ising_batch *batch = nullptr;
    std::vector<uint64_t> plan_ids;     // request ids of the current plan (handle addresses are reused)
    std::vector<uint64_t> plan_sweeps;
    std::string worker_error;

    double now() const
    {
        return std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
    }
};

namespace {

void finish(ising_server *s, Request *r, ising_status st)
{
    r->res.status = st;
    r->res.t_finish = s->now();
    if (r->h) {
        if (st == ISING_OK) {
            ising_measure(r->h, &r->res.obs);
            if (s->opts.keep_samples) {
                r->M = r->h->sM;
                r->E = r->h->sE;
            }
        }
        ising_destroy(r->h);
        r->h = nullptr;
        std::lock_guard<std::mutex> lk(s->mu);
        s->stats.mem_used -= r->bytes;
    }
    std::lock_guard<std::mutex> lk(s->mu);
    if (st == ISING_OK)
        ++s->stats.completed;
    else if (st == ISING_ERR_CANCELLED)
        ++s->stats.cancelled;
    else
        ++s->stats.failed;
    s->finished.push_back(r);
    s->cv_done.notify_all();
}

// Admits queued requests, in arrival order, while the budget allows.
void admit(ising_server *s)
{
    NvtxRange range("server_admit");
    while (true) {
        Request *r = nullptr;
        {
            std::lock_guard<std::mutex> lk(s->mu);
            if (s->queue.empty()) return;
            r = s->queue.front();
            if (!r->cancel && s->stats.mem_used + r->bytes > s->opts.hbm_budget_bytes &&
                r->bytes <= s->opts.hbm_budget_bytes)
                return;  // wait for memory to free up
            s->queue.pop_front();
        }
        if (r->cancel) {
            finish(s, r, ISING_ERR_CANCELLED);
            continue;
        }
        if (r->bytes > s->opts.hbm_budget_bytes) {
            finish(s, r, ISING_ERR_OOM);
            continue;
        }
        ising_lattice *h = nullptr;
        ising_status st = ising_create(&r->req.params, (void *)s->stream, &h);
        if (st != ISING_OK) {
            finish(s, r, st);
            continue;
        }
        r->h = h;
        r->res.t_admit = s->now();
        std::lock_guard<std::mutex> lk(s->mu);
        s->stats.mem_used += r->bytes;
        s->stats.peak_mem = std::max(s->stats.peak_mem, s->stats.mem_used);
        ++s->stats.admitted;
        s->resident.push_back(r);
    }
}

// One launch over the oldest resident requests that fit the batch.
void run_epoch(ising_server *s)
{
    NvtxRange range("server_epoch");
    std::vector<Request *> res;
    {
        std::lock_guard<std::mutex> lk(s->mu);
        res = s->resident;
    }
    // cancelled residents leave first
    std::vector<Request *> live;
    for (Request *r : res) {
        if (r->cancel) {
            {
                std::lock_guard<std::mutex> lk(s->mu);
                s->resident.erase(std::find(s->resident.begin(), s->resident.end(), r));
            }
            finish(s, r, ISING_ERR_CANCELLED);
        } else {
            live.push_back(r);
        }
    }
    if (live.empty()) return;
    const size_t cap = batch_capacity_bytes(s->batch);
    std::vector<Request *> act;
    size_t bytes = 0;
    for (Request *r : live) {
        const uint64_t L = r->req.params.L;
        const size_t need = (size_t)(L / 8) * (L + 8) + 1024;
        if (!act.empty() && (bytes + need > cap * 8 / 10 ||
                             (s->opts.max_active && act.size() >= s->opts.max_active)))
            break;
        act.push_back(r);
        bytes += need;
    }
    std::vector<ising_lattice *> hs;
    std::vector<uint64_t> sw, ids;
    std::vector<uint32_t> re;
    for (Request *r : act) {
        ids.push_back(r->id);
        hs.push_back(r->h);
        sw.push_back(std::min<uint64_t>(r->remaining, s->opts.epoch_sweeps));
        re.push_back(r->req.record_every);
    }
    ising_status st = ISING_OK;
    if (ids != s->plan_ids || sw != s->plan_sweeps) {
        // shrink the set until it plans (shared memory is the limit)
        while (true) {
            st = batch_replan(s->batch, hs, sw, re);
            if (st != ISING_ERR_INVALID || hs.size() == 1) break;
            const size_t keep = std::max<size_t>(1, hs.size() / 2);
            hs.resize(keep);
            sw.resize(keep);
            re.resize(keep);
            ids.resize(keep);
            act.resize(keep);
        }
        if (st != ISING_OK) {
            s->plan_ids.clear();
            s->plan_sweeps.clear();
            // the oldest request cannot be planned: it fails, the others go on
            Request *r = act.front();
            {
                std::lock_guard<std::mutex> lk(s->mu);
                s->resident.erase(std::find(s->resident.begin(), s->resident.end(), r));
            }
            finish(s, r, st);
            return;
        }
        s->plan_ids = ids;
        s->plan_sweeps = sw;
    }
    const double t_start = s->now();
    for (Request *r : act)
        if (r->res.epochs++ == 0) r->res.t_first_run = t_start;
    st = ising_batch_run(s->batch, 1);
    const double t_end = s->now();
    {
        std::lock_guard<std::mutex> lk(s->mu);
        ++s->stats.epochs;
        s->stats.busy_seconds += t_end - t_start;
        for (size_t i = 0; i < act.size(); ++i)
            if (st == ISING_OK) s->stats.attempts += act[i]->req.params.L * act[i]->req.params.L * sw[i];
    }
    if (st != ISING_OK) {
        // a failed launch loses the lattices it held; the batch is rebuilt
        for (Request *r : act) {
            {
                std::lock_guard<std::mutex> lk(s->mu);
                s->resident.erase(std::find(s->resident.begin(), s->resident.end(), r));
            }
            finish(s, r, st);
        }
        batch_free(s->batch);
        s->batch = nullptr;
        batch_new(s->device, &s->opts.batch, &s->batch);
        s->plan_ids.clear();
        s->plan_sweeps.clear();
        return;
    }
    for (size_t i = 0; i < act.size(); ++i) {
        Request *r = act[i];
        r->remaining -= sw[i];
        if (r->remaining == 0) {
            {
                std::lock_guard<std::mutex> lk(s->mu);
                s->resident.erase(std::find(s->resident.begin(), s->resident.end(), r));
            }
            finish(s, r, ISING_OK);
        }
    }
    // finished requests leave the plan; the rotation puts the next ones first
    {
        std::lock_guard<std::mutex> lk(s->mu);
        if (s->resident.size() > act.size()) {
            // round robin: the requests that just ran go behind the waiting ones
            std::vector<Request *> rot;
            for (Request *r : s->resident)
                if (std::find(act.begin(), act.end(), r) == act.end()) rot.push_back(r);
            for (Request *r : s->resident)
                if (std::find(act.begin(), act.end(), r) != act.end()) rot.push_back(r);
            s->resident = rot;
        }
    }
}

void worker_main(ising_server *s)
{
    cudaSetDevice(s->device);
    while (true) {
        {
            std::unique_lock<std::mutex> lk(s->mu);
            s->cv_work.wait(lk, [&] { return s->stop || !s->incoming.empty() || !s->resident.empty() ||
                                             !s->queue.empty(); });
            if (s->stop) break;
            while (!s->incoming.empty()) {
                s->queue.push_back(s->incoming.front());
                s->incoming.pop_front();
            }
        }
        admit(s);
        bool any;
        {
            std::lock_guard<std::mutex> lk(s->mu);
            any = !s->resident.empty();
        }
        if (any && s->batch) {
            run_epoch(s);
        } else if (!any) {
            // queue head waits for memory that only finishing requests free: nothing runs
            std::unique_lock<std::mutex> lk(s->mu);
            s->cv_work.wait_for(lk, std::chrono::milliseconds(5));
        }
    }
    // drop what is left
    std::vector<Request *> left;
    {
        std::lock_guard<std::mutex> lk(s->mu);
        left.assign(s->resident.begin(), s->resident.end());
        s->resident.clear();
        for (Request *r : s->queue) left.push_back(r);
        for (Request *r : s->incoming) left.push_back(r);
        s->queue.clear();
        s->incoming.clear();
    }
    for (Request *r : left) {
        if (r->h) ising_destroy(r->h);
        delete r;
    }
}

}  // namespace

extern "C" {

ISING_API ising_status ising_server_create(const ising_server_opts *opts, ising_server **out)
{
    clear_error();
    if (!out) return fail(ISING_ERR_INVALID, "out is NULL");
    *out = nullptr;
    ising_server *s = new (std::nothrow) ising_server();
    if (!s) return fail(ISING_ERR_OOM, "host allocation failed");
    if (opts) s->opts = *opts;
    if (s->opts.hbm_budget_bytes == 0) s->opts.hbm_budget_bytes = 64ull << 30;
    if (s->opts.epoch_sweeps == 0) s->opts.epoch_sweeps = 1000;
    if (s->opts.batch.block == 0) {
        s->opts.batch.block = 256;
        s->opts.batch.ctas_per_sm = s->opts.batch.ctas_per_sm ? s->opts.batch.ctas_per_sm : 4;
    }
    s->t0 = std::chrono::steady_clock::now();
    cudaError_t e = cudaGetDevice(&s->device);
    if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&s->stream, cudaStreamNonBlocking);
    if (e != cudaSuccess) {
        delete s;
        return fail(ISING_ERR_CUDA, "server set-up: %s", cudaGetErrorString(e));
    }
    ising_status st = batch_new(s->device, &s->opts.batch, &s->batch);
    if (st != ISING_OK) {
        cudaStreamDestroy(s->stream);
        delete s;
        return st;
    }
    s->worker = std::thread(worker_main, s);
    *out = s;
    return ISING_OK;
}

ISING_API ising_status ising_server_submit(ising_server *s, const ising_request *req, uint64_t *id)
{
    clear_error();
    if (!s || !req) return fail(ISING_ERR_INVALID, "null argument");
    uint32_t wb = 0;
    ising_status st = validate_params(&req->params, &wb);
    if (st != ISING_OK) return st;
    if (req->nsweeps == 0 || req->nsweeps >= 0xFFFFFFFFull)
        return fail(ISING_ERR_INVALID, "nsweeps must be in [1, 2^32 - 1)");
    Request *r = new (std::nothrow) Request();
    if (!r) return fail(ISING_ERR_OOM, "host allocation failed");
    r->req = *req;
    r->remaining = req->nsweeps;
    r->bytes = request_bytes(*req);
    std::lock_guard<std::mutex> lk(s->mu);
    r->id = s->next_id++;
    r->res.id = r->id;
    r->res.tag = req->tag;
    r->res.t_submit = s->now();
    ++s->stats.submitted;
    s->incoming.push_back(r);
    if (id) *id = r->id;
    s->cv_work.notify_all();
    return ISING_OK;
}

ISING_API ising_status ising_server_cancel(ising_server *s, uint64_t id)
{
    clear_error();
    if (!s) return fail(ISING_ERR_INVALID, "null server");
    std::lock_guard<std::mutex> lk(s->mu);
    for (auto *lst : {&s->incoming, &s->queue})
        for (Request *r : *lst)
            if (r->id == id) {
                r->cancel = true;
                s->cv_work.notify_all();
                return ISING_OK;
            }
    for (Request *r : s->resident)
        if (r->id == id) {
            r->cancel = true;  // leaves at the next launch boundary
            return ISING_OK;
        }
    return fail(ISING_ERR_INVALID, "no such pending request");
}

ISING_API ising_status ising_server_poll(ising_server *s, ising_result *out, uint32_t cap, uint32_t *n,
                                         double wait_s)
{
    clear_error();
    if (!s || !n || (cap && !out)) return fail(ISING_ERR_INVALID, "null argument");
    *n = 0;
    std::unique_lock<std::mutex> lk(s->mu);
    if (s->finished.empty() && wait_s > 0)
        s->cv_done.wait_for(lk, std::chrono::duration<double>(wait_s), [&] { return !s->finished.empty(); });
    while (*n < cap && !s->finished.empty()) {
        Request *r = s->finished.front();
        s->finished.pop_front();
        out[(*n)++] = r->res;
        if (s->opts.keep_samples && r->res.status == ISING_OK)
            s->kept[r->id] = r;
        else
            delete r;
    }
    return ISING_OK;
}

ISING_API ising_status ising_server_samples(ising_server *s, uint64_t id, int64_t *M, int64_t *E, uint64_t cap,
                                            uint64_t *n)
{
    clear_error();
    if (!s || !n) return fail(ISING_ERR_INVALID, "null argument");
    std::lock_guard<std::mutex> lk(s->mu);
    auto it = s->kept.find(id);
    if (it == s->kept.end()) return fail(ISING_ERR_INVALID, "no kept samples for request %llu",
                                         (unsigned long long)id);
    Request *r = it->second;
    *n = r->M.size();
    if (!M || !E) return ISING_OK;  // size query
    if (cap < r->M.size()) return fail(ISING_ERR_INVALID, "cap is smaller than the samples");
    std::memcpy(M, r->M.data(), r->M.size() * sizeof(int64_t));
    std::memcpy(E, r->E.data(), r->E.size() * sizeof(int64_t));
    s->kept.erase(it);
    delete r;
    return ISING_OK;
}

ISING_API ising_status ising_server_stats(ising_server *s, ising_server_counters *out)
{
    clear_error();
    if (!s || !out) return fail(ISING_ERR_INVALID, "null argument");
    std::lock_guard<std::mutex> lk(s->mu);
    *out = s->stats;
    out->queued = s->incoming.size() + s->queue.size();
    out->resident = s->resident.size();
    out->now = s->now();
    return ISING_OK;
}

ISING_API ising_status ising_server_destroy(ising_server *s)
{
    clear_error();
    if (!s) return ISING_OK;
    {
        std::lock_guard<std::mutex> lk(s->mu);
        s->stop = true;
        s->cv_work.notify_all();
    }
    if (s->worker.joinable()) s->worker.join();
    for (Request *r : s->finished) delete r;
    for (auto &kv : s->kept) delete kv.second;
    if (s->batch) batch_free(s->batch);
    if (s->stream) cudaStreamDestroy(s->stream);
    delete s;
    return ISING_OK;
}

}  // extern "C"

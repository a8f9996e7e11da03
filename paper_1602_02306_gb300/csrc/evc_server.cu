// evc_server.cu -- a request server for interval counts on several resident
// matrices (see evc_server_* in include/evc.h).
//
// Requests (matrix, xi, eta, probes, steps, tol, seed) arrive at any time.
// A scheduler thread keeps them in arrival order and, whenever an execution
// slot is idle, forms a batch: the oldest waiting request plus the later
// ones that can share its launch (same matrix, probe count and seed), as
// many as the HBM budget and the batch limit allow.  The batch runs as one
// batched count (two shifts per request, each with its request's tolerance
// and step limit) on the slot's own stream, so batches on different slots
// overlap on the device; under the identity preconditioner all shifts of the
// batch read one Lanczos run per probe (shared Krylov mode).
// A request that does not fit the remaining budget waits (first come, first
// served: nothing overtakes it); memory and slots are returned as batches
// finish, and waiting requests are admitted at once.  Every column of a
// batch is computed independently with batch-independent reductions, so a
// request's result does not depend on which other requests shared its
// launch.
#include "evc_internal.cuh"
#include "../../include/evc.h"

#include <algorithm>
#include <chrono>
#include <condition_variable>
#include <deque>
#include <map>
#include <memory>
#include <mutex>
#include <thread>
#include <vector>

namespace {

struct Req {
    int64_t ticket;
    int matrix;
    double xi, eta;
    int nprobe, maxsteps;
    double tol;
    uint64_t seed;
    double* quad_out;     // caller buffer [2*nprobe] or null
    evc_result res;
    bool done = false;
};

struct Batch {
    std::vector<Req*> reqs;
    size_t bytes = 0;
};

struct Slot {
    std::thread th;
    std::unique_ptr<Batch> work;    // assigned batch (null when idle)
    std::map<int, evc_ctx*> clones; // per matrix
};

}  // namespace

struct evc_server {
    size_t budget = 0, used = 0, peak = 0;
    int max_batch = 16;
    bool stop = false;
    int64_t next_ticket = 1;
    std::mutex mu;
    std::condition_variable cv_sched, cv_done, cv_slot;
    std::deque<Req*> pending;
    std::map<int64_t, std::unique_ptr<Req>> reqs;
    std::vector<evc_ctx*> matrices;
    std::vector<std::unique_ptr<Slot>> slots;
    std::thread sched;
    std::chrono::steady_clock::time_point t0 = std::chrono::steady_clock::now();
    int device = 0;
    int64_t batches = 0, completed = 0, merged = 0;

    double now() const
    {
        return std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
    }
};

namespace {

// Requests share a launch when they run the same probes on the same matrix;
// each shift keeps its own stop tolerance and step limit, so tolerances and
// limits may differ.  Under the identity preconditioner the merged shifts also
// share the Lanczos columns themselves (shared Krylov mode).
bool compatible(const Req* a, const Req* b)
{
    return a->matrix == b->matrix && a->nprobe == b->nprobe && a->seed == b->seed;
}

evc_ctx* clone_for(evc_server* s, Slot* sl, int matrix)
{
    auto it = sl->clones.find(matrix);
    if (it != sl->clones.end()) return it->second;
    evc_ctx* c = evc::clone_context(s->matrices[matrix]);
    sl->clones[matrix] = c;
    return c;
}

// Scheduler: forms batches in arrival order for idle slots (lock held).
void schedule(evc_server* s)
{
    for (auto& slp : s->slots) {
        Slot* sl = slp.get();
        if (sl->work || s->pending.empty()) continue;
        Req* head = s->pending.front();
        evc_ctx* c = clone_for(s, sl, head->matrix);
        if (!c) {
            head->res.status = EVC_ENOMEM;
            head->done = true;
            s->pending.pop_front();
            s->cv_done.notify_all();
            continue;
        }
        auto b = std::make_unique<Batch>();
        std::vector<size_t> take;
        size_t bytes = 0;
        for (size_t idx = 0; idx < s->pending.size() && (int)take.size() < s->max_batch; ++idx) {
            Req* r = s->pending[idx];
            if (!compatible(head, r)) continue;
            int kmx = r->maxsteps;
            for (size_t t : take) kmx = std::max(kmx, s->pending[t]->maxsteps);
            const size_t need = evc_workspace_bytes(c, 2 * ((int)take.size() + 1), r->nprobe, kmx);
            if (need == 0 || s->used + need > s->budget) break;
            take.push_back(idx);
            bytes = need;
        }
        if (take.empty()) {
            // the oldest request waits for memory; if nothing is running it can never fit
            bool any_busy = false;
            for (auto& o : s->slots) any_busy |= (bool)o->work;
            if (!any_busy) {
                head->res.status = EVC_ENOMEM;
                head->done = true;
                s->pending.pop_front();
                s->cv_done.notify_all();
                continue;
            }
            return;   // first come, first served: nothing overtakes the head
        }
        for (size_t t = take.size(); t-- > 0;) {
            b->reqs.insert(b->reqs.begin(), s->pending[take[t]]);
            s->pending.erase(s->pending.begin() + (std::ptrdiff_t)take[t]);
        }
        b->bytes = bytes;
        s->used += bytes;
        if (s->used > s->peak) s->peak = s->used;
        const double t = s->now();
        for (Req* r : b->reqs) {
            r->res.t_start = t;
            r->res.batch_size = (int)b->reqs.size();
        }
        ++s->batches;
        s->merged += (int64_t)b->reqs.size() - 1;
        sl->work = std::move(b);
        s->cv_slot.notify_all();
    }
}

void run_batch(evc_server* s, Slot* sl, Batch* b)
{
    evc::NvtxRange nv("evc: server batch");
    Req* head = b->reqs.front();
    evc_ctx* c;
    {
        std::lock_guard<std::mutex> g(s->mu);
        c = clone_for(s, sl, head->matrix);
    }
    const int R = (int)b->reqs.size();
    const int m = head->nprobe;
    std::vector<double> shifts(2 * R), tols(2 * R), L(2 * R), quad((size_t)2 * R * m);
    std::vector<int> steps(2 * R), kmax(2 * R);
    for (int q = 0; q < R; ++q) {
        shifts[2 * q] = b->reqs[q]->xi;
        shifts[2 * q + 1] = b->reqs[q]->eta;
        tols[2 * q] = tols[2 * q + 1] = b->reqs[q]->tol;
        kmax[2 * q] = kmax[2 * q + 1] = b->reqs[q]->maxsteps;
    }
    cudaSetDevice(s->device);
    int rc = EVC_OK;
    void* ws = nullptr;
    // the clone's own stream: the workspace comes from the device's
    // stream-ordered pool and goes back to it when the batch ends
    cudaStream_t st = evc::ctx_stream(c);
    if (cudaMallocAsync(&ws, b->bytes, st) != cudaSuccess) {
        cudaGetLastError();
        rc = EVC_ENOMEM;
    }
    if (rc == EVC_OK) rc = evc_set_workspace(c, ws, b->bytes);
    if (rc == EVC_OK)
        rc = evc::count_slices_each(c, shifts.data(), 2 * R, m, kmax.data(), tols.data(),
                                    head->seed, L.data(), quad.data(), steps.data());
    // A numeric failure is flagged once for the whole launch: run each request
    // of a merged batch alone (in the same workspace) so that only the request
    // whose own columns fail reports it, as it would have alone.
    std::vector<int> rcs(R, rc);
    if (rc == EVC_ENUMERIC && R > 1) {
        for (int q = 0; q < R; ++q)
            rcs[q] = evc::count_slices_each(c, shifts.data() + 2 * q, 2, m, kmax.data() + 2 * q,
                                            tols.data() + 2 * q, head->seed, L.data() + 2 * q,
                                            quad.data() + (size_t)2 * q * m, steps.data() + 2 * q);
    }
    evc_set_workspace(c, nullptr, 0);
    if (ws) {
        cudaFreeAsync(ws, st);
        cudaStreamSynchronize(st);
    }
    std::lock_guard<std::mutex> g(s->mu);
    const double t = s->now();
    for (int q = 0; q < R; ++q) {
        Req* r = b->reqs[q];
        r->res.status = rcs[q];
        if (rcs[q] == EVC_OK) {
            r->res.n_below[0] = L[2 * q];
            r->res.n_below[1] = L[2 * q + 1];
            r->res.estimate = L[2 * q + 1] - L[2 * q];
            r->res.steps[0] = steps[2 * q];
            r->res.steps[1] = steps[2 * q + 1];
            if (r->quad_out)
                for (int j = 0; j < 2 * m; ++j) r->quad_out[j] = quad[(size_t)2 * q * m + j];
        }
        r->res.t_done = t;
        r->done = true;
        ++s->completed;
    }
    s->used -= b->bytes;
    sl->work.reset();
    s->cv_done.notify_all();
    s->cv_sched.notify_all();
}

void slot_main(evc_server* s, Slot* sl)
{
    cudaSetDevice(s->device);
    std::unique_lock<std::mutex> lk(s->mu);
    for (;;) {
        s->cv_slot.wait(lk, [&] { return s->stop || (bool)sl->work; });
        if (!sl->work) return;   // stopping and idle
        Batch* b = sl->work.get();
        lk.unlock();
        run_batch(s, sl, b);
        lk.lock();
    }
}

void sched_main(evc_server* s)
{
    cudaSetDevice(s->device);
    std::unique_lock<std::mutex> lk(s->mu);
    for (;;) {
        schedule(s);
        if (s->stop) {
            bool busy = false;
            for (auto& sl : s->slots) busy |= (bool)sl->work;
            if (!busy && s->pending.empty()) break;
        }
        s->cv_sched.wait_for(lk, std::chrono::milliseconds(50));
    }
    s->cv_slot.notify_all();
}

}  // namespace

extern "C" {

int evc_server_create(size_t hbm_budget_bytes, int slots, int max_batch, evc_server** out)
{
    if (!out) return EVC_EINVAL;
    *out = nullptr;
    if (hbm_budget_bytes == 0 || slots < 1 || slots > 64 || max_batch < 1 || max_batch > 1024)
        return EVC_EINVAL;
    evc_server* s = new (std::nothrow) evc_server();
    if (!s) return EVC_ENOMEM;
    if (cudaGetDevice(&s->device) != cudaSuccess) {
        cudaGetLastError();
        delete s;
        return EVC_ECUDA;
    }
    // keep freed workspaces in the device's memory pool instead of returning
    // them to the driver between batches
    cudaMemPool_t pool;
    if (cudaDeviceGetDefaultMemPool(&pool, s->device) == cudaSuccess) {
        uint64_t thr = UINT64_MAX;
        cudaMemPoolSetAttribute(pool, cudaMemPoolAttrReleaseThreshold, &thr);
    }
    cudaGetLastError();
    s->budget = hbm_budget_bytes;
    s->max_batch = max_batch;
    for (int i = 0; i < slots; ++i) s->slots.push_back(std::make_unique<Slot>());
    for (auto& sl : s->slots) sl->th = std::thread(slot_main, s, sl.get());
    s->sched = std::thread(sched_main, s);
    *out = s;
    return EVC_OK;
}

int evc_server_add_matrix(evc_server* s, evc_ctx* ctx, int* matrix_id)
{
    if (!s || !ctx || !matrix_id) return EVC_EINVAL;
    std::lock_guard<std::mutex> g(s->mu);
    s->matrices.push_back(ctx);
    *matrix_id = (int)s->matrices.size() - 1;
    return EVC_OK;
}

int evc_server_submit(evc_server* s, int matrix_id, double xi, double eta, int nprobe,
                      int maxsteps, double tol, uint64_t seed, double* per_probe_quad,
                      int64_t* ticket)
{
    if (!s || !ticket) return EVC_EINVAL;
    if (!(xi < eta) || nprobe < 1 || maxsteps < 1 || maxsteps > EVC_MAX_STEPS) return EVC_EINVAL;
    std::lock_guard<std::mutex> g(s->mu);
    if (s->stop || matrix_id < 0 || matrix_id >= (int)s->matrices.size()) return EVC_EINVAL;
    auto r = std::make_unique<Req>();
    r->ticket = s->next_ticket++;
    r->matrix = matrix_id;
    r->xi = xi;
    r->eta = eta;
    r->nprobe = nprobe;
    r->maxsteps = maxsteps;
    r->tol = tol;
    r->seed = seed;
    r->quad_out = per_probe_quad;
    r->res = evc_result{};
    r->res.t_submit = s->now();
    *ticket = r->ticket;
    s->pending.push_back(r.get());
    s->reqs[r->ticket] = std::move(r);
    s->cv_sched.notify_all();
    return EVC_OK;
}

int evc_server_wait(evc_server* s, int64_t ticket, double timeout_s, evc_result* res)
{
    if (!s) return EVC_EINVAL;
    std::unique_lock<std::mutex> lk(s->mu);
    auto it = s->reqs.find(ticket);
    if (it == s->reqs.end()) return EVC_EINVAL;
    Req* r = it->second.get();
    auto pred = [&] { return r->done; };
    if (timeout_s < 0) s->cv_done.wait(lk, pred);
    else if (!s->cv_done.wait_for(lk, std::chrono::duration<double>(timeout_s), pred))
        return EVC_EAGAIN;
    if (res) *res = r->res;
    const int st = r->res.status;
    s->reqs.erase(it);
    return st;
}

int evc_server_poll(evc_server* s, int64_t ticket, evc_result* res)
{
    if (!s) return EVC_EINVAL;
    std::lock_guard<std::mutex> g(s->mu);
    auto it = s->reqs.find(ticket);
    if (it == s->reqs.end()) return EVC_EINVAL;
    if (!it->second->done) return EVC_EAGAIN;
    if (res) *res = it->second->res;
    const int st = it->second->res.status;
    s->reqs.erase(it);
    return st;
}

int evc_server_stats(evc_server* s, evc_server_counters* st)
{
    if (!s || !st) return EVC_EINVAL;
    std::lock_guard<std::mutex> g(s->mu);
    st->budget_bytes = s->budget;
    st->used_bytes = s->used;
    st->peak_bytes = s->peak;
    st->pending = (int64_t)s->pending.size();
    st->batches = s->batches;
    st->completed = s->completed;
    st->merged = s->merged;
    return EVC_OK;
}

void evc_server_destroy(evc_server* s)
{
    if (!s) return;
    {
        std::lock_guard<std::mutex> g(s->mu);
        s->stop = true;
    }
    s->cv_sched.notify_all();
    if (s->sched.joinable()) s->sched.join();
    s->cv_slot.notify_all();
    for (auto& sl : s->slots)
        if (sl->th.joinable()) sl->th.join();
    for (auto& sl : s->slots)
        for (auto& kv : sl->clones) evc_destroy(kv.second);
    delete s;
}

}  // extern "C"

// rb_server.cu - continuous-batching serving loop over a device-resident
// index (no paper counterpart; the serving pattern of this library).
//
// One host thread owns the loop.  Each iteration it (1) retires batches whose
// device work finished (a host callback enqueued after the batch stamps the
// completion time and wakes the loop), handing results to waiting tickets;
// (2) admits queued requests in arrival order while a stream slot is free and
// the memory budget covers the request's worst-case result bytes, forms a
// batch of them and enqueues it on that slot's stream.  Batches on different
// streams overlap on the device; requests that arrive meanwhile wait only for
// a free slot and budget, not for the running batches.  A result's memory is
// charged to the budget until the caller frees the result.
#include <chrono>
#include <condition_variable>
#include <deque>
#include <list>
#include <mutex>
#include <thread>
#include <unordered_map>

#include "rb_multi.h"

using namespace rbi;

namespace {

using clk = std::chrono::steady_clock;

struct Req {
    rb_request r;
    uint64_t bound = 0;
    clk::time_point t_submit;
    double latency = 0;
    int state = 0;   // 0 queued, 1 in flight, 2 done
    rb_t *out = nullptr;
    uint64_t card = 0;
    rb_status st = RB_OK;
};

struct Slot {
    cudaStream_t s = nullptr;
    PinnedBuf stage;
    bool busy = false;
};

struct Flight;

}  // namespace

struct rb_server {
    std::vector<const rb *> index;
    BmView *d_index = nullptr;
    uint32_t n = 0;
    uint64_t budget_cap = 0;
    RbBudget *budget = nullptr;
    uint32_t max_batch = 0;
    int device = 0;
    std::mutex mu;
    std::condition_variable cv_work, cv_done;
    std::deque<uint64_t> queue;
    std::deque<uint64_t> done;   // completed tickets in completion order (rb_server_poll)
    std::unordered_map<uint64_t, Req> reqs;
    std::vector<Slot> slots;
    std::list<Flight *> flights;
    std::thread th;
    bool stop = false;
    uint64_t next_ticket = 1, completed = 0, batches = 0, inflight = 0, peak_inflight = 0;
};

namespace {

struct Flight {
    rb_server *srv;
    int slot;
    MultiBatch *mb;
    RbArena *arena;
    std::vector<uint64_t> tickets;
    std::atomic<int> done{0};
    clk::time_point t_done;
};

void CUDART_CB on_batch_done(void *p) {
    Flight *f = (Flight *)p;
    f->t_done = clk::now();
    f->done.store(1);
    f->srv->cv_work.notify_all();
}

void budget_notify(void *ctx) { ((rb_server *)ctx)->cv_work.notify_all(); }

void retire(rb_server *S, Flight *f) {
    std::vector<rb_t *> outs(f->tickets.size(), nullptr);
    std::vector<uint64_t> cards(f->tickets.size(), 0);
    // the batch's device work is complete; its results may outlive the loop
    // and its streams, so their memory is released on the default stream
    if (f->arena) f->arena->stream = nullptr;
    rb_status st = multi_finish(f->mb, f->arena, outs.data(), cards.data());
    for (size_t i = 0; i < f->tickets.size(); i++) {
        auto it = S->reqs.find(f->tickets[i]);
        if (it == S->reqs.end()) {   // abandoned ticket
            rb_free(outs[i]);
            continue;
        }
        Req &r = it->second;
        r.st = st;
        r.out = outs[i];
        r.card = cards[i];
        r.latency = std::chrono::duration<double>(f->t_done - r.t_submit).count();
        r.state = 2;
        S->done.push_back(f->tickets[i]);
    }
    // tickets collected by rb_server_wait stay in `done` until a poll skips
    // them; drop them here when they pile up
    if (S->done.size() > 4096 && S->done.size() > 2 * S->reqs.size()) {
        std::deque<uint64_t> keep;
        for (uint64_t t : S->done)
            if (S->reqs.count(t)) keep.push_back(t);
        S->done.swap(keep);
    }
    S->completed += f->tickets.size();
    S->inflight -= f->tickets.size();
    multi_free(f->mb, S->slots[f->slot].s);
    arena_unref(f->arena);
    S->slots[f->slot].busy = false;
    delete f;
}

void loop(rb_server *S) {
    cudaSetDevice(S->device);
    std::unique_lock<std::mutex> lk(S->mu);
    for (;;) {
        bool retired = false;
        for (auto it = S->flights.begin(); it != S->flights.end();) {
            if ((*it)->done.load()) {
                retire(S, *it);
                it = S->flights.erase(it);
                retired = true;
            } else {
                ++it;
            }
        }
        if (retired) S->cv_done.notify_all();
        if (S->stop && S->flights.empty()) {
            // shutting down: requests never admitted fail with RB_EBUSY
            for (uint64_t t : S->queue) {
                auto it = S->reqs.find(t);
                if (it != S->reqs.end()) {
                    it->second.st = RB_EBUSY;
                    it->second.state = 2;
                    S->done.push_back(t);
                }
            }
            S->queue.clear();
            S->cv_done.notify_all();
            break;
        }
        if (S->stop) {
            S->cv_work.wait_for(lk, std::chrono::microseconds(200));
            continue;
        }
        // admission
        for (;;) {
            if (S->queue.empty()) break;
            int slot = -1;
            for (size_t i = 0; i < S->slots.size(); i++)
                if (!S->slots[i].busy) { slot = (int)i; break; }
            if (slot < 0) break;
            std::vector<MultiQuery> qs;
            std::vector<uint64_t> tk;
            uint64_t need = 0;
            const int64_t used = S->budget->used.load();
            while (!S->queue.empty() && qs.size() < S->max_batch) {
                Req &r = S->reqs[S->queue.front()];
                if ((uint64_t)used + need + r.bound > S->budget_cap) break;
                need += r.bound;
                MultiQuery mq;
                mq.op = r.r.op;
                mq.count_only = r.r.count_only;
                mq.members.assign(r.r.members, r.r.members + r.r.k);
                qs.push_back(mq);
                tk.push_back(S->queue.front());
                r.state = 1;
                S->queue.pop_front();
            }
            if (qs.empty()) break;   // wait for memory
            Slot &sl = S->slots[slot];
            sl.busy = true;
            S->budget->used.fetch_add((int64_t)need);
            Flight *f = new Flight;
            f->srv = S;
            f->slot = slot;
            f->mb = nullptr;
            f->arena = nullptr;
            f->tickets = tk;
            lk.unlock();
            uint64_t ab = 0;
            rb_status st = multi_prepare(S->index.data(), S->d_index, S->n, qs, sl.s, &f->mb, &ab, &sl.stage, true);
            if (st == RB_OK && ab) {
                f->arena = arena_new_native(ab, sl.s);
                if (!f->arena) st = RB_ENOMEM;
            }
            if (f->arena) {
                f->arena->budget = S->budget;
                f->arena->charge = need;
                S->budget->refs.fetch_add(1);
            } else {
                S->budget->used.fetch_sub((int64_t)need);   // nothing materialised
            }
            if (st == RB_OK) st = multi_enqueue(f->mb, f->arena, sl.s);
            if (st == RB_OK && cudaLaunchHostFunc(sl.s, on_batch_done, f) != cudaSuccess) st = RB_ECUDA;
            lk.lock();
            if (st != RB_OK) {
                // fail every request of the batch (no device work is pending on
                // its results: wait for the stream before releasing)
                cudaStreamSynchronize(sl.s);
                for (uint64_t t : tk) {
                    auto it = S->reqs.find(t);
                    if (it != S->reqs.end()) {
                        it->second.st = st;
                        it->second.state = 2;
                        S->done.push_back(t);
                    }
                }
                if (f->mb) multi_free(f->mb, sl.s);
                arena_unref(f->arena);
                sl.busy = false;
                delete f;
                S->cv_done.notify_all();
                continue;
            }
            S->flights.push_back(f);
            S->batches++;
            S->inflight += tk.size();
            if (S->inflight > S->peak_inflight) S->peak_inflight = S->inflight;
        }
        S->cv_work.wait_for(lk, std::chrono::microseconds(200));
    }
}

}  // namespace

extern "C" {

rb_status rb_server_create(const rb_t *const *index, uint32_t n, uint64_t mem_budget, uint32_t max_inflight_batches,
                           uint32_t max_batch, rb_server_t **out) {
    if (!out) return set_err(RB_EINVAL, "rb_server_create: out is NULL");
    *out = nullptr;
    if (n && !index) return set_err(RB_EINVAL, "rb_server_create: NULL index");
    if (max_inflight_batches < 1 || max_inflight_batches > 64) return set_err(RB_EINVAL, "max_inflight_batches in 1..64");
    if (max_batch < 1) return set_err(RB_EINVAL, "max_batch must be >= 1");
    rb_server *S = new rb_server;
    S->index.assign(index, index + n);
    S->n = n;
    S->budget_cap = mem_budget;
    S->max_batch = max_batch;
    cudaGetDevice(&S->device);
    S->budget = new RbBudget;
    S->budget->used.store(0);
    S->budget->refs.store(1);
    S->budget->notify = budget_notify;
    S->budget->ctx = S;
    std::vector<BmView> hv(n);
    for (uint32_t i = 0; i < n; i++) {
        if (!index[i]) { budget_unref(S->budget); delete S; return set_err(RB_EINVAL, "index[%u] is NULL", i); }
        hv[i] = view_of(index[i]);
    }
    // the index table comes from the installed allocator, on the calling
    // thread (the legacy default stream; the copy below completes before the
    // loop starts)
    S->d_index = (BmView *)dev_alloc(sizeof(BmView) * std::max<uint32_t>(n, 1), nullptr);
    if (!S->d_index) {
        budget_unref(S->budget);
        delete S;
        return RB_ENOMEM;
    }
    cudaError_t e = cudaSuccess;
    if (n) e = cudaMemcpy(S->d_index, hv.data(), sizeof(BmView) * n, cudaMemcpyHostToDevice);
    S->slots.resize(max_inflight_batches);
    for (auto &sl : S->slots)
        if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&sl.s, cudaStreamNonBlocking);
    if (e != cudaSuccess) {
        for (auto &sl : S->slots)
            if (sl.s) cudaStreamDestroy(sl.s);
        dev_free(S->d_index, sizeof(BmView) * std::max<uint32_t>(n, 1), nullptr);
        budget_unref(S->budget);
        delete S;
        return cuda_err(e, "rb_server_create");
    }
    S->th = std::thread(loop, S);
    *out = S;
    return RB_OK;
}

}  // extern "C"

namespace {

// checks one request and computes its worst-case result bytes
rb_status make_req(rb_server_t *S, const rb_request *r, Req &q) {
    if (r->op != RB_AND && r->op != RB_OR) return set_err(RB_EINVAL, "request op must be RB_AND or RB_OR");
    if (r->k < 1 || r->k > RB_SERVE_MAX_K) return set_err(RB_EINVAL, "request k must be 1..%d", RB_SERVE_MAX_K);
    MultiQuery mq;
    mq.op = r->op;
    mq.count_only = r->count_only;
    for (uint32_t i = 0; i < r->k; i++) {
        if (r->members[i] >= S->n) return set_err(RB_EINVAL, "request member %u out of range", r->members[i]);
        mq.members.push_back(r->members[i]);
    }
    q.r = *r;
    q.bound = multi_query_bound(S->index.data(), mq);
    if (q.bound > S->budget_cap) return set_err(RB_EBUSY, "request needs up to %llu bytes, above the whole budget",
                                                (unsigned long long)q.bound);
    return RB_OK;
}

}  // namespace

extern "C" {

rb_status rb_server_submit(rb_server_t *S, const rb_request *r, uint64_t *ticket) {
    if (!S || !r || !ticket) return set_err(RB_EINVAL, "rb_server_submit: NULL argument");
    return rb_server_submit_many(S, r, 1, ticket);
}

rb_status rb_server_submit_many(rb_server_t *S, const rb_request *r, uint32_t n, uint64_t *tickets) {
    if (!S || (n && (!r || !tickets))) return set_err(RB_EINVAL, "rb_server_submit_many: NULL argument");
    std::vector<Req> qs(n);
    for (uint32_t i = 0; i < n; i++) {
        rb_status st = make_req(S, r + i, qs[i]);
        if (st != RB_OK) return st;
    }
    const clk::time_point now = clk::now();
    {
        std::lock_guard<std::mutex> g(S->mu);
        for (uint32_t i = 0; i < n; i++) {
            qs[i].t_submit = now;
            tickets[i] = S->next_ticket++;
            S->reqs.emplace(tickets[i], qs[i]);
            S->queue.push_back(tickets[i]);
        }
    }
    S->cv_work.notify_all();
    return RB_OK;
}

rb_status rb_server_poll(rb_server_t *S, uint32_t cap, int timeout_ms, uint64_t *tickets, rb_status *status,
                         rb_t **outs, uint64_t *cards, double *latency_s, uint32_t *n_out) {
    if (!S || !n_out || (cap && !tickets)) return set_err(RB_EINVAL, "rb_server_poll: NULL argument");
    *n_out = 0;
    std::unique_lock<std::mutex> lk(S->mu);
    const auto deadline = clk::now() + std::chrono::milliseconds(timeout_ms < 0 ? 0 : timeout_ms);
    while (S->done.empty()) {
        if (S->cv_done.wait_until(lk, deadline) == std::cv_status::timeout && S->done.empty()) return RB_OK;
    }
    uint32_t k = 0;
    while (k < cap && !S->done.empty()) {
        const uint64_t t = S->done.front();
        S->done.pop_front();
        auto it = S->reqs.find(t);
        if (it == S->reqs.end()) continue;   // already collected by rb_server_wait
        Req &q = it->second;
        tickets[k] = t;
        if (status) status[k] = q.st;
        if (cards) cards[k] = q.st == RB_OK ? q.card : 0;
        if (latency_s) latency_s[k] = q.latency;
        if (outs) outs[k] = q.st == RB_OK ? q.out : nullptr;
        else rb_free(q.out);
        if (outs && q.st != RB_OK) rb_free(q.out);
        S->reqs.erase(it);
        k++;
    }
    *n_out = k;
    return RB_OK;
}

rb_status rb_server_wait(rb_server_t *S, uint64_t ticket, int timeout_ms, rb_t **out, uint64_t *card,
                         double *latency_s) {
    if (out) *out = nullptr;
    if (!S) return set_err(RB_EINVAL, "rb_server_wait: NULL server");
    std::unique_lock<std::mutex> lk(S->mu);
    const auto deadline = clk::now() + std::chrono::milliseconds(timeout_ms < 0 ? 0 : timeout_ms);
    // the ticket is looked up again after every wait: while the lock is
    // released a submission may rehash the map and a poll may collect the
    // ticket
    auto it = S->reqs.find(ticket);
    if (it == S->reqs.end()) return set_err(RB_EINVAL, "unknown ticket %llu", (unsigned long long)ticket);
    while (it->second.state != 2) {
        const bool timed_out = S->cv_done.wait_until(lk, deadline) == std::cv_status::timeout;
        it = S->reqs.find(ticket);
        if (it == S->reqs.end())
            return set_err(RB_EINVAL, "ticket %llu was collected by another call", (unsigned long long)ticket);
        if (timed_out && it->second.state != 2)
            return set_err(RB_ETIMEOUT, "ticket %llu not done within %d ms", (unsigned long long)ticket, timeout_ms);
    }
    Req r = it->second;
    S->reqs.erase(it);
    lk.unlock();
    if (r.st != RB_OK) {
        rb_free(r.out);
        return set_err(r.st, "request failed");
    }
    if (card) *card = r.card;
    if (latency_s) *latency_s = r.latency;
    if (out) *out = r.out;
    else rb_free(r.out);
    return RB_OK;
}

rb_status rb_server_stats(rb_server_t *S, uint64_t *completed, uint64_t *batches, uint64_t *peak) {
    if (!S) return set_err(RB_EINVAL, "rb_server_stats: NULL server");
    std::lock_guard<std::mutex> g(S->mu);
    if (completed) *completed = S->completed;
    if (batches) *batches = S->batches;
    if (peak) *peak = S->peak_inflight;
    return RB_OK;
}

void rb_server_destroy(rb_server_t *S) {
    if (!S) return;
    {
        std::lock_guard<std::mutex> g(S->mu);
        S->stop = true;
    }
    S->cv_work.notify_all();
    if (S->th.joinable()) S->th.join();
    for (auto &kv : S->reqs) rb_free(kv.second.out);
    for (auto &sl : S->slots) {
        if (sl.s) {
            cudaStreamSynchronize(sl.s);
            cudaStreamDestroy(sl.s);
        }
        if (sl.stage.p) cudaFreeHost(sl.stage.p);
    }
    dev_free(S->d_index, sizeof(BmView) * std::max<uint32_t>(S->n, 1), nullptr);
    {
        // results that outlive the loop stop waking it before it is deleted
        std::lock_guard<std::mutex> g(S->budget->mu);
        S->budget->notify = nullptr;
    }
    budget_unref(S->budget);
    delete S;
}

}  // extern "C"

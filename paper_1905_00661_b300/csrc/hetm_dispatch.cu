// Request queues, device affinity and work stealing (Sec. III-B, transaction
// scheduling and dispatching).
//
// Every registered transaction type owns up to three queues of single
// requests: CPU_Q and GPU_Q for requests submitted with an affinity for one
// device, SHARED_Q for those without one (a type with one implementation has
// only the queue of that device).  CPU worker threads pull one request at a
// time, from the CPU_Qs in round-robin order over the types and, when all of
// them are empty, from the SHARED_Qs.  The GPU controller packs a type's
// GPU_Q, topped up from its SHARED_Q, into one batch when they hold enough
// requests to feed the kernel (or the oldest has waited long enough) and
// hands it to the serving loop, which fuses batches into synchronization
// rounds.  A batch whose round was rolled back (GPU-loses conflict) is put
// back at the front of its queues and runs again.
//
// Queues hold spans of consecutive requests of one submission, so that a
// million-request submission is one queue entry until a device splits it.

#include <algorithm>
#include <chrono>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <memory>
#include <mutex>
#include <thread>
#include <unordered_map>
#include <vector>

#include "hetm.h"
#include "hetm_internal.cuh"

namespace {

using Clock = std::chrono::steady_clock;
constexpr int kCpuQ = 0, kGpuQ = 1, kSharedQ = 2;

struct Sub {  // one hetm_dispatch_submit call
    uint32_t type = 0, n = 0;
    const char *tx = nullptr;
    uint8_t *status = nullptr;
    char *out = nullptr;
    uint8_t *device = nullptr;
    uint32_t left = 0;  // requests not completed yet
    int rc = HETM_OK;
    bool done = false;
    Clock::time_point arrival{};
    double latency_ms = 0;
};

struct Span {  // requests first .. first + count - 1 of a submission
    Sub *s;
    uint32_t first, count;
};

struct Queue {
    std::deque<Span> spans;
    uint64_t n = 0;

    bool empty() const { return n == 0; }
    Clock::time_point oldest() const { return spans.front().s->arrival; }
    Span pop1() {
        Span &f = spans.front();
        const Span r{f.s, f.first, 1};
        ++f.first;
        if (--f.count == 0) spans.pop_front();
        --n;
        return r;
    }
    // Up to k requests from the front, appended to out as spans; returns how many.
    uint64_t take(uint64_t k, std::vector<Span> &out) {
        uint64_t got = 0;
        while (got < k && !spans.empty()) {
            Span &f = spans.front();
            const uint32_t c = (uint32_t)std::min<uint64_t>(f.count, k - got);
            out.push_back({f.s, f.first, c});
            f.first += c;
            f.count -= c;
            got += c;
            if (f.count == 0) spans.pop_front();
        }
        n -= got;
        return got;
    }
    void push_front(const Span &sp) {
        spans.push_front(sp);
        n += sp.count;
    }
    void push_back(const Span &sp) {
        spans.push_back(sp);
        n += sp.count;
    }
};

struct Type {
    hetm_tx_type t{};
    Queue q[3];
};

struct Act {  // one GPU activation (a batch of one type)
    Type *ty = nullptr;
    uint32_t n = 0;
    std::vector<Span> spans;
    std::vector<uint8_t> from;  // queue each span came from
    std::vector<char> tx, out;
    std::vector<uint8_t> status;
    uint64_t server_id = 0;
};

size_t wl_record_bytes(uint32_t wl) {
    switch (wl) {
        case HETM_WL_BANK: return sizeof(hetm_bank_tx);
        case HETM_WL_CACHE: return sizeof(hetm_cache_req);
        default: return 0;
    }
}

size_t wl_out_bytes(uint32_t wl) { return wl == HETM_WL_CACHE ? 8 : 0; }

}  // namespace

struct hetm_dispatch {
    hetm_server *server = nullptr;
    hetm_gpu_batch_fn gpu_fn = nullptr;
    void *gpu_user = nullptr;
    hetm_dispatch_config cfg{};
    std::mutex mu;
    std::condition_variable cv_cpu, cv_ctl, cv_cmp, cv_done;
    std::vector<std::unique_ptr<Type>> types;
    std::unordered_map<uint64_t, Sub *> subs;
    uint64_t next_ticket = 1;
    std::deque<Act *> inflight;  // submitted to the server, oldest first
    bool stop = false, ctl_done = false;
    std::vector<std::thread> workers;
    std::thread ctl, cmp;
    hetm_dispatch_stats st{};
};

namespace {

// Completes k requests of s (lock held).
void retire(hetm_dispatch *d, Sub *s, uint32_t k, int rc) {
    if (rc != HETM_OK && s->rc == HETM_OK) s->rc = rc;
    s->left -= k;
    if (s->left == 0) {
        s->done = true;
        s->latency_ms = std::chrono::duration<double, std::milli>(Clock::now() - s->arrival).count();
        d->cv_done.notify_all();
    }
}

bool gpu_work_left(const hetm_dispatch *d) {
    for (const auto &t : d->types)
        if (t->t.gpu_workload && (!t->q[kGpuQ].empty() || !t->q[kSharedQ].empty())) return true;
    return false;
}

void cpu_worker(hetm_dispatch *d, uint32_t w) {
    size_t cur = 0;  // this worker's round-robin position over the types
    std::unique_lock<std::mutex> lk(d->mu);
    for (;;) {
        Span sp{};
        int from = -1;
        Type *ty = nullptr;
        const size_t nt = d->types.size();
        for (int which : {kCpuQ, kSharedQ}) {
            for (size_t i = 0; i < nt && from < 0; ++i) {
                const size_t t = (cur + i) % nt;
                Queue &q = d->types[t]->q[which];
                if (q.empty()) continue;
                sp = q.pop1();
                from = which;
                ty = d->types[t].get();
                cur = t + 1;
            }
            if (from >= 0) break;
        }
        if (from < 0) {
            if (d->stop) return;
            d->cv_cpu.wait(lk);
            continue;
        }
        lk.unlock();
        const uint32_t i = sp.first;
        const char *rec = sp.s->tx + (size_t)i * ty->t.rec_bytes;
        char *out = sp.s->out && ty->t.out_bytes ? sp.s->out + (size_t)i * ty->t.out_bytes : nullptr;
        const int r = ty->t.cpu_fn(ty->t.cpu_user, w, rec, out);
        if (sp.s->status) sp.s->status[i] = r < 0 ? 0 : (uint8_t)r;
        if (sp.s->device) sp.s->device[i] = HETM_DEVICE_CPU;
        lk.lock();
        ++d->st.cpu_done;
        if (from == kSharedQ) ++d->st.cpu_stolen;
        retire(d, sp.s, 1, r < 0 ? r : HETM_OK);
    }
}

// Results of a finished activation back to its submissions, or -- when its
// round undid it -- its requests back to the front of their queues.
void complete(hetm_dispatch *d, Act *a, int rc, uint32_t outcome) {
    Type &ty = *a->ty;
    const bool undone = rc == HETM_OK && outcome == HETM_OUTCOME_GPU_ROLLED_BACK;
    uint64_t stolen = 0;
    if (!undone) {
        size_t pos = 0;
        const size_t ob = ty.t.out_bytes;
        for (size_t k = 0; k < a->spans.size(); ++k) {
            const Span &sp = a->spans[k];
            Sub *s = sp.s;
            if (s->status) std::memcpy(s->status + sp.first, a->status.data() + pos, sp.count);
            if (s->out && ob)
                std::memcpy(s->out + (size_t)sp.first * ob, a->out.data() + pos * ob, (size_t)sp.count * ob);
            if (s->device) std::memset(s->device + sp.first, HETM_DEVICE_GPU, sp.count);
            if (a->from[k] == kSharedQ) stolen += sp.count;
            pos += sp.count;
        }
    }
    std::lock_guard<std::mutex> g(d->mu);
    if (undone) {
        for (size_t k = a->spans.size(); k-- > 0;) ty.q[a->from[k]].push_front(a->spans[k]);
        d->st.requeued += a->n;
        d->cv_cpu.notify_all();
    } else {
        d->st.gpu_done += a->n;
        d->st.gpu_stolen += stolen;
        ++d->st.activations;
        for (const Span &sp : a->spans) retire(d, sp.s, sp.count, rc);
    }
    d->cv_ctl.notify_one();
    delete a;
}

// Pick the next activation (lock held): a type whose GPU_Q + SHARED_Q hold
// gpu_min_batch requests, or whose oldest waiting request is due.  Returns
// null and sets *wake to the next due time (or leaves it) when none is ready.
Act *pick_activation(hetm_dispatch *d, size_t *cur, Clock::time_point *wake) {
    const size_t nt = d->types.size();
    const auto now = Clock::now();
    const auto max_wait = std::chrono::microseconds(d->cfg.gpu_max_wait_us);
    for (size_t i = 0; i < nt; ++i) {
        const size_t t = (*cur + i) % nt;
        Type &ty = *d->types[t];
        if (!ty.t.gpu_workload) continue;
        Queue &g = ty.q[kGpuQ], &sh = ty.q[kSharedQ];
        if (g.empty() && sh.empty()) continue;
        auto oldest = Clock::time_point::max();
        if (!g.empty()) oldest = g.oldest();
        if (!sh.empty()) oldest = std::min(oldest, sh.oldest());
        const bool go = g.n + sh.n >= d->cfg.gpu_min_batch || now - oldest >= max_wait || d->stop;
        if (!go) {
            *wake = std::min(*wake, oldest + max_wait);
            continue;
        }
        Act *a = new Act();
        a->ty = &ty;
        const uint64_t cap = d->cfg.gpu_max_batch;
        uint64_t got = g.take(cap, a->spans);
        a->from.assign(a->spans.size(), kGpuQ);
        got += sh.take(cap - got, a->spans);
        a->from.resize(a->spans.size(), kSharedQ);
        a->n = (uint32_t)got;
        *cur = t + 1;
        return a;
    }
    return nullptr;
}

void controller(hetm_dispatch *d) {
    size_t cur = 0;
    std::unique_lock<std::mutex> lk(d->mu);
    for (;;) {
        if (d->stop && !gpu_work_left(d) && d->inflight.empty()) break;
        Act *a = nullptr;
        auto wake = Clock::time_point::max();
        if (d->inflight.size() < d->cfg.gpu_inflight) a = pick_activation(d, &cur, &wake);
        if (!a) {
            if (wake == Clock::time_point::max()) d->cv_ctl.wait(lk);
            else d->cv_ctl.wait_until(lk, wake);
            continue;
        }
        const hetm_tx_type tt = a->ty->t;
        lk.unlock();
        const hetm::Range range("hetm_dispatch activation");
        // pack the records of the batch
        const size_t rb = tt.rec_bytes, ob = tt.out_bytes;
        a->tx.resize((size_t)a->n * rb);
        a->status.assign(a->n, 0);
        a->out.resize((size_t)a->n * ob);
        size_t pos = 0;
        for (const Span &sp : a->spans) {
            std::memcpy(a->tx.data() + pos * rb, sp.s->tx + (size_t)sp.first * rb, (size_t)sp.count * rb);
            pos += sp.count;
        }
        if (!d->server) {
            uint32_t outcome = HETM_OUTCOME_CLEAN;
            const int rc = d->gpu_fn(d->gpu_user, tt.gpu_workload, tt.word_base, a->tx.data(), a->n,
                                     a->status.data(), ob ? a->out.data() : nullptr, &outcome);
            complete(d, a, rc, outcome);
            lk.lock();
            continue;
        }
        hetm_request r{};
        r.workload = tt.gpu_workload;
        r.n_tx = a->n;
        r.host_tx = a->tx.data();
        r.host_status = a->status.data();
        r.host_out = ob ? a->out.data() : nullptr;
        r.word_base = tt.word_base;
        const int rc = hetm_server_submit(d->server, &r, &a->server_id);
        if (rc != HETM_OK) {
            complete(d, a, rc, HETM_OUTCOME_CLEAN);
            lk.lock();
            continue;
        }
        lk.lock();
        d->inflight.push_back(a);
        d->cv_cmp.notify_one();
    }
    d->ctl_done = true;
    d->cv_cmp.notify_all();
}

// Waits for the server's batches in submission order.
void completer(hetm_dispatch *d) {
    std::unique_lock<std::mutex> lk(d->mu);
    for (;;) {
        d->cv_cmp.wait(lk, [&] { return !d->inflight.empty() || d->ctl_done; });
        if (d->inflight.empty()) return;
        Act *a = d->inflight.front();
        lk.unlock();
        uint32_t outcome = HETM_OUTCOME_CLEAN;
        const int rc = hetm_server_wait_outcome(d->server, a->server_id, nullptr, &outcome);
        lk.lock();
        d->inflight.pop_front();
        lk.unlock();
        complete(d, a, rc, outcome);
        lk.lock();
    }
}

}  // namespace

extern "C" {

int hetm_dispatch_config_default(hetm_dispatch_config *cfg) {
    if (!cfg) return HETM_EINVAL;
    std::memset(cfg, 0, sizeof(*cfg));
    cfg->cpu_workers = 2;
    cfg->gpu_min_batch = 1024;
    cfg->gpu_max_batch = 1u << 20;
    cfg->gpu_max_wait_us = 2000;
    cfg->gpu_inflight = 2;
    return HETM_OK;
}

int hetm_dispatch_create(hetm_dispatch **out, hetm_server *server, hetm_gpu_batch_fn gpu_fn,
                         void *gpu_user, const hetm_dispatch_config *cfg) {
    if (!out) return HETM_EINVAL;
    hetm_dispatch_config c;
    hetm_dispatch_config_default(&c);
    if (cfg) c = *cfg;
    if (c.gpu_min_batch == 0 || c.gpu_max_batch == 0 || c.gpu_inflight == 0) return HETM_EINVAL;
    if (server)
        c.gpu_max_batch = (uint32_t)std::min<uint64_t>(c.gpu_max_batch, hetm::server_max_round_tx(server));
    hetm_dispatch *d = new (std::nothrow) hetm_dispatch();
    if (!d) return HETM_ENOMEM;
    d->server = server;
    d->gpu_fn = server ? nullptr : gpu_fn;
    d->gpu_user = gpu_user;
    d->cfg = c;
    int dev = -1;
    if (server && cudaGetDevice(&dev) != cudaSuccess) dev = -1;
    try {
        for (uint32_t w = 0; w < c.cpu_workers; ++w) d->workers.emplace_back(cpu_worker, d, w);
        d->ctl = std::thread(controller, d);
        if (server)
            d->cmp = std::thread([d, dev] {
                if (dev >= 0) cudaSetDevice(dev);
                completer(d);
            });
    } catch (...) {  // a thread could not be started: stop the ones that were
        hetm_dispatch_destroy(d);
        return HETM_ENOMEM;
    }
    *out = d;
    return HETM_OK;
}

int hetm_dispatch_register(hetm_dispatch *d, const hetm_tx_type *t, uint32_t *type) {
    if (!d || !t || !type || t->rec_bytes == 0) return HETM_EINVAL;
    if (!t->cpu_fn && !t->gpu_workload) return HETM_EINVAL;
    if (t->cpu_fn && d->cfg.cpu_workers == 0) return HETM_EINVAL;
    if (t->gpu_workload) {
        if (!d->server && !d->gpu_fn) return HETM_EINVAL;
        if (wl_record_bytes(t->gpu_workload) == 0 || t->rec_bytes != wl_record_bytes(t->gpu_workload) ||
            t->out_bytes != wl_out_bytes(t->gpu_workload))
            return HETM_EINVAL;
    }
    std::unique_ptr<Type> ty(new (std::nothrow) Type());
    if (!ty) return HETM_ENOMEM;
    ty->t = *t;
    std::lock_guard<std::mutex> g(d->mu);
    if (d->stop) return HETM_EINVAL;
    *type = (uint32_t)d->types.size();
    d->types.push_back(std::move(ty));
    return HETM_OK;
}

int hetm_dispatch_submit(hetm_dispatch *d, uint32_t type, int affinity, const void *tx, uint32_t n,
                         uint8_t *status, void *out, uint8_t *device, uint64_t *ticket) {
    if (!d || !ticket || (n && !tx)) return HETM_EINVAL;
    if (affinity != HETM_AFFINITY_NONE && affinity != HETM_AFFINITY_CPU && affinity != HETM_AFFINITY_GPU)
        return HETM_EINVAL;
    std::lock_guard<std::mutex> g(d->mu);
    if (d->stop || type >= d->types.size()) return HETM_EINVAL;
    Type &ty = *d->types[type];
    const bool cpu = ty.t.cpu_fn != nullptr, gpu = ty.t.gpu_workload != 0;
    int which;
    if (cpu && gpu)
        which = affinity == HETM_AFFINITY_CPU ? kCpuQ : affinity == HETM_AFFINITY_GPU ? kGpuQ : kSharedQ;
    else if (cpu)
        which = affinity == HETM_AFFINITY_GPU ? -1 : kCpuQ;
    else
        which = affinity == HETM_AFFINITY_CPU ? -1 : kGpuQ;
    if (which < 0) return HETM_EINVAL;
    Sub *s = new (std::nothrow) Sub();
    if (!s) return HETM_ENOMEM;
    s->type = type;
    s->n = s->left = n;
    s->tx = static_cast<const char *>(tx);
    s->status = status;
    s->out = static_cast<char *>(out);
    s->device = device;
    s->arrival = Clock::now();
    const uint64_t id = d->next_ticket++;
    d->subs[id] = s;
    *ticket = id;
    if (n == 0) {
        s->done = true;
        return HETM_OK;
    }
    ty.q[which].push_back({s, 0, n});
    if (which != kGpuQ) d->cv_cpu.notify_all();
    if (which != kCpuQ) d->cv_ctl.notify_one();
    return HETM_OK;
}

int hetm_dispatch_wait(hetm_dispatch *d, uint64_t ticket, double *latency_ms) {
    if (!d) return HETM_EINVAL;
    std::unique_lock<std::mutex> lk(d->mu);
    auto it = d->subs.find(ticket);
    if (it == d->subs.end()) return HETM_EINVAL;
    Sub *s = it->second;
    if (!d->cv_done.wait_for(lk, std::chrono::seconds(120), [&] { return s->done; })) return HETM_ETIMEOUT;
    if (latency_ms) *latency_ms = s->latency_ms;
    const int rc = s->rc;
    d->subs.erase(it);
    delete s;
    return rc;
}

int hetm_dispatch_get_stats(hetm_dispatch *d, hetm_dispatch_stats *out) {
    if (!d || !out) return HETM_EINVAL;
    std::lock_guard<std::mutex> g(d->mu);
    *out = d->st;
    out->queued_cpu = out->queued_gpu = out->queued_shared = 0;
    for (const auto &t : d->types) {
        out->queued_cpu += t->q[kCpuQ].n;
        out->queued_gpu += t->q[kGpuQ].n;
        out->queued_shared += t->q[kSharedQ].n;
    }
    return HETM_OK;
}

void hetm_dispatch_destroy(hetm_dispatch *d) {
    if (!d) return;
    {
        std::lock_guard<std::mutex> g(d->mu);
        d->stop = true;
        d->cv_cpu.notify_all();
        d->cv_ctl.notify_all();
    }
    if (d->ctl.joinable()) d->ctl.join();
    if (d->cmp.joinable()) d->cmp.join();
    for (auto &w : d->workers)
        if (w.joinable()) w.join();
    for (auto &kv : d->subs) delete kv.second;
    delete d;
}

}  // extern "C"

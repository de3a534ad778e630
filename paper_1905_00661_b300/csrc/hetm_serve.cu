// Serving loop: continuous batching of transaction batches into SHeTM rounds.
//
// Client threads submit batches (host records) at any time.  One loop thread
// forms rounds: it admits waiting batches in arrival order while the
// device-memory budget and the round's transaction capacity allow, copies
// their records to the device on a copy stream while the previous round is
// still running on the GPU, and then runs one synchronization round for all
// admitted batches together (one persistent executor launch over uneven
// batches, validation, apply, merge: Sec. IV-C) -- or, in per-batch mode,
// one round per batch.  A batch commits when its round's merge is done and
// its results are back on the host; its latency is measured from submit to
// that point.  The STMR and all round state stay on the device throughout.

#include <cuda_runtime.h>

#include <algorithm>
#include <chrono>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <mutex>
#include <thread>
#include <unordered_map>
#include <vector>

#include "hetm.h"
#include "hetm_internal.cuh"

namespace {

using Clock = std::chrono::steady_clock;

size_t record_bytes(uint32_t wl) {
    switch (wl) {
        case HETM_WL_BANK: return sizeof(hetm_bank_tx);
        case HETM_WL_RMW: return sizeof(hetm_rmw_tx);
        case HETM_WL_CACHE: return sizeof(hetm_cache_req);
        case HETM_WL_W2: return sizeof(hetm_w2_tx);
        default: return 0;
    }
}

size_t out_bytes(uint32_t wl) {
    return wl == HETM_WL_RMW || wl == HETM_WL_W2 ? 4 : wl == HETM_WL_CACHE ? 8 : 0;
}

struct Req {
    uint64_t id;
    hetm_request r;
    Clock::time_point arrival;
    // device buffers (one allocation)
    void *dev = nullptr;
    size_t dev_bytes = 0;
    int done = 0;
    int rc = HETM_OK;
    double latency_ms = 0;
    uint32_t committed = 0;
    uint32_t outcome = 0;  // HETM_OUTCOME_* of its round
};

}  // namespace

struct hetm_server {
    hetm_ctx *ctx = nullptr;
    hetm_server_config cfg{};
    cudaStream_t copy = nullptr;
    cudaStream_t main = nullptr;
    cudaEvent_t rdone[2] = {nullptr, nullptr};  // end of a launched group's result copies
    std::mutex mu;
    std::condition_variable cv_in, cv_done;
    std::deque<Req *> waiting;
    std::unordered_map<uint64_t, Req *> all;
    uint64_t next_id = 1;
    bool stop = false;
    std::thread loop;
    size_t budget = 0, held = 0;  // budget 0: admission follows free device memory only
    size_t reserve = 0;           // device memory admission always leaves free
    // stats
    uint64_t rounds = 0, completed = 0, committed = 0, refused = 0;
    std::vector<double> lat;
    Clock::time_point first_arrival{}, last_done{};
    bool have_first = false;
};

namespace {

// Device footprint of a request: records + order + status + outputs, 256-aligned parts.
size_t footprint(const hetm_request &r) {
    auto al = [](size_t b) { return (b + 255) & ~size_t(255); };
    return al(r.n_tx * record_bytes(r.workload)) + al(r.n_tx * 8ull) + al(r.n_tx) +
           al(r.n_tx * out_bytes(r.workload)) + 256;
}

int stage(hetm_server *s, Req *q) {
    q->dev_bytes = footprint(q->r);
    if (cudaMallocAsync(&q->dev, q->dev_bytes, s->copy) != cudaSuccess) {
        cudaGetLastError();
        return HETM_ENOMEM;
    }
    const size_t rb = q->r.n_tx * record_bytes(q->r.workload);
    if (rb && cudaMemcpyAsync(q->dev, q->r.host_tx, rb, cudaMemcpyHostToDevice, s->copy) != cudaSuccess)
        return HETM_ECUDA;
    return HETM_OK;
}

void parts(Req *q, void **tx, uint64_t **order, uint8_t **status, void **out) {
    auto al = [](size_t b) { return (b + 255) & ~size_t(255); };
    char *p = static_cast<char *>(q->dev);
    *tx = p;
    p += al(q->r.n_tx * record_bytes(q->r.workload));
    *order = reinterpret_cast<uint64_t *>(p);
    p += al(q->r.n_tx * 8ull);
    *status = reinterpret_cast<uint8_t *>(p);
    p += al(q->r.n_tx);
    *out = out_bytes(q->r.workload) ? p : nullptr;
}

int submit_to_ctx(hetm_server *s, Req *q) {
    void *tx, *out;
    uint64_t *order;
    uint8_t *status;
    parts(q, &tx, &order, &status, &out);
    hetm_batch b{q->r.workload, q->r.n_tx, tx, order, status, out, q->r.txid_base, q->r.word_base};
    uint64_t bid = 0;
    return hetm_gpu_submit_batch(s->ctx, &b, &bid);
}

// Results back to the caller's host buffers, then release the device buffers.
int collect(hetm_server *s, Req *q) {
    void *tx, *out;
    uint64_t *order;
    uint8_t *status;
    parts(q, &tx, &order, &status, &out);
    const uint32_t n = q->r.n_tx;
    int rc = HETM_OK;
    if (q->r.host_order && cudaMemcpyAsync(q->r.host_order, order, n * 8ull, cudaMemcpyDeviceToHost, s->main) != cudaSuccess)
        rc = HETM_ECUDA;
    if (q->r.host_status && cudaMemcpyAsync(q->r.host_status, status, n, cudaMemcpyDeviceToHost, s->main) != cudaSuccess)
        rc = HETM_ECUDA;
    if (q->r.host_out && out &&
        cudaMemcpyAsync(q->r.host_out, out, n * out_bytes(q->r.workload), cudaMemcpyDeviceToHost, s->main) != cudaSuccess)
        rc = HETM_ECUDA;
    if (cudaFreeAsync(q->dev, s->main) != cudaSuccess) rc = HETM_ECUDA;
    return rc;
}

void finish(hetm_server *s, std::vector<Req *> &group, int rc) {
    const auto now = Clock::now();
    std::lock_guard<std::mutex> g(s->mu);
    for (Req *q : group) {
        q->rc = rc;
        q->done = 1;
        q->latency_ms = std::chrono::duration<double, std::milli>(now - q->arrival).count();
        s->held -= q->dev_bytes;
        s->lat.push_back(q->latency_ms);
        ++s->completed;
        s->committed += q->committed;
    }
    s->last_done = now;
    s->cv_done.notify_all();
    s->cv_in.notify_all();
}

// rounds of the context launched and not yet collected
int open_rounds(hetm_server *s) { return hetm::ctx_open_rounds(s->ctx); }
bool round_opened(hetm_server *s) { return open_rounds(s) > 0; }

// Launch one round for `group` (already staged): the executor waits for
// the staging copies; result copies are queued behind the round.
int launch_round(hetm_server *s, std::vector<Req *> &group, cudaEvent_t done) {
    const hetm::Range range("hetm_server round");
    cudaEvent_t ev;
    if (cudaEventCreateWithFlags(&ev, cudaEventDisableTiming) != cudaSuccess) return HETM_ECUDA;
    cudaEventRecord(ev, s->copy);
    cudaStreamWaitEvent(s->main, ev, 0);
    cudaEventDestroy(ev);
    int rc = HETM_OK;
    for (Req *q : group)
        if (rc == HETM_OK) rc = submit_to_ctx(s, q);
    if (rc == HETM_OK) rc = hetm_round(s->ctx, nullptr);
    for (Req *q : group) {
        const int c = collect(s, q);
        if (rc == HETM_OK) rc = c;
    }
    // results of this group are in host memory once the stream passes here
    if (cudaEventRecord(done, s->main) != cudaSuccess && rc == HETM_OK) rc = HETM_ECUDA;
    return rc;
}

// Wait for the round of `group` and complete its batches.
void complete_round(hetm_server *s, std::vector<Req *> &group, int rc, cudaEvent_t done) {
    hetm_round_stats st;
    std::memset(&st, 0, sizeof(st));
    const int w = hetm_round_wait(s->ctx, &st);
    if (rc == HETM_OK) rc = w;
    // this group's result copies only (the next round may already be queued)
    if (cudaEventSynchronize(done) != cudaSuccess && rc == HETM_OK) rc = HETM_ECUDA;
    // every transaction commits unless the round reports give-ups, which
    // are attributed to the batches in order
    uint64_t left = st.committed;
    for (Req *q : group) {
        q->committed = (uint32_t)std::min<uint64_t>(left, q->r.n_tx);
        left -= q->committed;
        q->outcome = st.outcome;
    }
    {
        std::lock_guard<std::mutex> g(s->mu);
        ++s->rounds;
    }
    finish(s, group, rc);
}

// Device memory free for batches now: what the device reports free (memory
// other allocations took since the server started counts against it), less
// the reserve.  Batches of earlier groups are already allocated when the
// loop admits the next group, so they are part of what is not free.
size_t free_for_batches(const hetm_server *s) {
    size_t free_b = 0, total_b = 0;
    if (cudaMemGetInfo(&free_b, &total_b) != cudaSuccess) return 0;
    return free_b > s->reserve ? free_b - s->reserve : 0;
}

// Admit waiting batches (arrival order) while their device footprint fits
// the memory free now (and the optional fixed budget) and the round's
// capacities.  A batch that does not fit while nothing is in flight cannot
// be admitted by waiting: it fails with HETM_ENOMEM (into `refused`).
// With `block`, wait until at least one batch is waiting (or stop).
bool admit(hetm_server *s, std::vector<Req *> &group, bool block, std::vector<Req *> &refused) {
    {
        std::unique_lock<std::mutex> lk(s->mu);
        if (block) s->cv_in.wait(lk, [&] { return s->stop || !s->waiting.empty(); });
        if (s->waiting.empty()) return !s->stop;
    }
    const size_t avail = free_for_batches(s);
    std::unique_lock<std::mutex> lk(s->mu);
    uint64_t tx = 0;
    size_t taken = 0;
    while (!s->waiting.empty()) {
        Req *q = s->waiting.front();
        const size_t f = footprint(q->r);
        if (!group.empty() && (s->cfg.per_batch || group.size() >= s->cfg.max_round_batches ||
                               tx + q->r.n_tx > s->cfg.max_round_tx))
            break;
        const bool fits = taken + f <= avail && (s->budget == 0 || s->held + f <= s->budget);
        if (!fits) {
            if (group.empty() && s->held == 0) {  // nothing in flight will free memory
                s->waiting.pop_front();
                ++s->refused;
                refused.push_back(q);
                continue;
            }
            break;  // wait for in-flight batches to free memory
        }
        s->waiting.pop_front();
        s->held += f;
        taken += f;
        tx += q->r.n_tx;
        group.push_back(q);
    }
    return true;
}

int stage_group(hetm_server *s, std::vector<Req *> &group) {
    int rc = HETM_OK;
    for (Req *q : group)
        if (rc == HETM_OK) rc = stage(s, q);
    return rc;
}

// Pipeline: while round k runs on the GPU, round k+1's batches are admitted,
// copied to the device and launched behind it (two rounds in flight on the
// context), so that the GPU goes from one round to the next without waiting
// for the host to complete the first.
void loop_main(hetm_server *s) {
    std::vector<Req *> cur;  // launched, not completed
    int cur_rc = HETM_OK;
    int ev = 0;  // s->rdone[ev]: the end of cur's result copies
    std::vector<Req *> refused;
    auto fail_refused = [&] {
        if (refused.empty()) return;
        for (Req *q : refused) q->dev_bytes = 0;  // never allocated
        finish(s, refused, HETM_ENOMEM);
        refused.clear();
    };
    for (;;) {
        if (cur.empty()) {  // nothing in flight: wait for work
            std::vector<Req *> g;
            const bool go = admit(s, g, true, refused);
            fail_refused();
            if (!go) return;
            if (g.empty()) {
                std::this_thread::sleep_for(std::chrono::microseconds(20));
                continue;
            }
            const int rc = stage_group(s, g);
            if (rc != HETM_OK) {
                finish(s, g, rc);
                continue;
            }
            cur_rc = launch_round(s, g, s->rdone[ev]);
            if (cur_rc != HETM_OK && !round_opened(s)) {
                finish(s, g, cur_rc);  // nothing was launched
                continue;
            }
            cur.swap(g);
        }
        std::vector<Req *> next;
        int next_rc = HETM_OK;
        admit(s, next, false, refused);
        fail_refused();
        bool next_open = false;
        if (!next.empty()) {
            next_rc = stage_group(s, next);
            if (next_rc == HETM_OK) {
                const int before = open_rounds(s);
                next_rc = launch_round(s, next, s->rdone[ev ^ 1]);
                next_open = open_rounds(s) > before;
            }
        }
        complete_round(s, cur, cur_rc, s->rdone[ev]);
        cur.clear();
        if (next_open) {
            cur.swap(next);
            cur_rc = next_rc;
            ev ^= 1;
        } else if (!next.empty()) {
            finish(s, next, next_rc);  // its round was never launched
        }
    }
}

}  // namespace

extern "C" {

int hetm_server_config_default(hetm_server_config *cfg) {
    if (!cfg) return HETM_EINVAL;
    std::memset(cfg, 0, sizeof(*cfg));
    cfg->per_batch = 0;
    cfg->device_budget = 0;
    cfg->max_round_batches = 1024;
    cfg->max_round_tx = 1ull << 22;
    return HETM_OK;
}

int hetm_server_create(hetm_server **out, hetm_ctx *ctx, const hetm_server_config *cfg) {
    if (!out || !ctx) return HETM_EINVAL;
    hetm_server *s = new (std::nothrow) hetm_server();
    if (!s) return HETM_ENOMEM;
    s->ctx = ctx;
    hetm_server_config d;
    hetm_server_config_default(&d);
    if (cfg) d = *cfg;
    if (d.max_round_batches == 0 || d.max_round_tx == 0) {
        delete s;
        return HETM_EINVAL;
    }
    s->cfg = d;
    size_t free_b = 0, total_b = 0;
    if (cudaMemGetInfo(&free_b, &total_b) != cudaSuccess) {
        delete s;
        return HETM_ECUDA;
    }
    s->budget = d.device_budget;
    s->reserve = d.free_reserve ? d.free_reserve : total_b / 16;
    s->main = static_cast<cudaStream_t>(hetm_ctx_stream(ctx));
    if (cudaStreamCreateWithFlags(&s->copy, cudaStreamNonBlocking) != cudaSuccess ||
        cudaEventCreateWithFlags(&s->rdone[0], cudaEventDisableTiming) != cudaSuccess ||
        cudaEventCreateWithFlags(&s->rdone[1], cudaEventDisableTiming) != cudaSuccess) {
        if (s->copy) cudaStreamDestroy(s->copy);
        for (auto e : s->rdone)
            if (e) cudaEventDestroy(e);
        delete s;
        return HETM_ECUDA;
    }
    int dev = 0;
    cudaGetDevice(&dev);
    try {
        s->loop = std::thread([s, dev] {
            cudaSetDevice(dev);
            loop_main(s);
        });
    } catch (...) {
        hetm_server_destroy(s);
        return HETM_ENOMEM;
    }
    *out = s;
    return HETM_OK;
}

int hetm_server_submit(hetm_server *s, const hetm_request *r, uint64_t *id) {
    if (!s || !r || !id || (r->n_tx && !r->host_tx) || record_bytes(r->workload) == 0)
        return HETM_EINVAL;
    Req *q = new (std::nothrow) Req();
    if (!q) return HETM_ENOMEM;
    q->r = *r;
    q->arrival = Clock::now();
    size_t free_b = 0, total_b = 0;
    if (cudaMemGetInfo(&free_b, &total_b) != cudaSuccess) {
        delete q;
        return HETM_ECUDA;
    }
    std::lock_guard<std::mutex> g(s->mu);
    const size_t f = footprint(*r);
    if ((s->budget && f > s->budget) || f + s->reserve > total_b || r->n_tx > s->cfg.max_round_tx) {
        ++s->refused;
        delete q;
        return HETM_EBUSY;
    }
    q->id = s->next_id++;
    if (!s->have_first) {
        s->first_arrival = q->arrival;
        s->have_first = true;
    }
    s->all[q->id] = q;
    s->waiting.push_back(q);
    *id = q->id;
    s->cv_in.notify_one();
    return HETM_OK;
}

int hetm_server_wait(hetm_server *s, uint64_t id, double *latency_ms) {
    return hetm_server_wait_outcome(s, id, latency_ms, nullptr);
}

int hetm_server_wait_outcome(hetm_server *s, uint64_t id, double *latency_ms, uint32_t *outcome) {
    if (!s) return HETM_EINVAL;
    std::unique_lock<std::mutex> lk(s->mu);
    auto it = s->all.find(id);
    if (it == s->all.end()) return HETM_EINVAL;
    Req *q = it->second;
    if (!s->cv_done.wait_for(lk, std::chrono::seconds(120), [&] { return q->done != 0; }))
        return HETM_ETIMEOUT;
    if (latency_ms) *latency_ms = q->latency_ms;
    if (outcome) *outcome = q->outcome;
    const int rc = q->rc;
    s->all.erase(it);
    delete q;
    return rc;
}

int hetm_server_get_stats(hetm_server *s, hetm_server_stats *out) {
    if (!s || !out) return HETM_EINVAL;
    std::lock_guard<std::mutex> g(s->mu);
    std::memset(out, 0, sizeof(*out));
    out->rounds = s->rounds;
    out->completed = s->completed;
    out->committed = s->committed;
    out->refused = s->refused;
    if (!s->lat.empty()) {
        std::vector<double> v = s->lat;
        std::sort(v.begin(), v.end());
        auto pct = [&](double p) {
            const size_t i = std::min(v.size() - 1, (size_t)(p * (v.size() - 1) + 0.5));
            return v[i];
        };
        out->p50_ms = pct(0.50);
        out->p99_ms = pct(0.99);
        out->max_ms = v.back();
    }
    if (s->have_first && s->completed)
        out->span_s = std::chrono::duration<double>(s->last_done - s->first_arrival).count();
    return HETM_OK;
}

void hetm_server_destroy(hetm_server *s) {
    if (!s) return;
    {
        std::lock_guard<std::mutex> g(s->mu);
        s->stop = true;
        s->cv_in.notify_all();
    }
    if (s->loop.joinable()) s->loop.join();
    for (auto &kv : s->all) delete kv.second;
    if (s->copy) cudaStreamDestroy(s->copy);
    for (auto e : s->rdone)
        if (e) cudaEventDestroy(e);
    delete s;
}

}  // extern "C"

namespace hetm {
uint64_t server_max_round_tx(const hetm_server *s) { return s->cfg.max_round_tx; }
}  // namespace hetm

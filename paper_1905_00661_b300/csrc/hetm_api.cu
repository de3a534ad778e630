// Host runtime and C ABI of the SHeTM round library.
//
// Owns the device state of one STMR (working copy W, shadow S, timestamp
// array TS, RS_bmp, WS_bmp, lock table, device log buffers), the pinned
// per-thread CPU logs and their H2D shipping on a side stream, the batch
// table of the current execution phase, and two captured CUDA graphs: the
// persistent executor launch and the validate -> apply -> merge -> clear
// chain (Sec. IV-C, IV-D).

#include <cuda_runtime.h>

#include <algorithm>
#include <atomic>
#include <chrono>
#include <cstdio>
#include <cstring>
#include <map>
#include <memory>
#include <mutex>
#include <new>
#include <vector>

#include "hetm_internal.cuh"
#include "hetm_testing.h"  // hetm_gpu_mark

using namespace hetm;

namespace {

constexpr unsigned long long kWatchBudgetNs = 20ull * 1000 * 1000 * 1000;  // as the executor's

struct Scratch {                    // device-resident counters
    unsigned long long gv;          // commit-version clock
    unsigned long long next;        // executor work counter
    unsigned long long counters[3]; // committed, gave up, aborts (cumulative)
    unsigned long long conflicts;   // hits of the last validation
    unsigned long long dirty;       // chunks merged by the last merge
    int err;
    int pad;
    unsigned int stop;              // early validation: conflict seen, stop executing
    unsigned int segs_done;         //   ordered-phase segments finished
    unsigned int segs_total;        //   their number + 1 (0 = not known yet)
    unsigned int exec_over;         //   nonzero once every executor kernel has finished
    unsigned long long v0;          // optimistic executor: commit clock before the launch
    unsigned long long rest_n;      //   indices the read-only phase left to the STM
    unsigned long long w2n;         // ordered executor: W2 updates listed for the STM tail
};

struct RoundOut {                   // pinned copy of the round's results
    unsigned long long counters[3];
    unsigned long long conflicts;
    unsigned long long dirty;
    int err;
    unsigned int stopped;           // early validation stopped the execution phase
};

struct ThreadLog {
    std::mutex mu;
    hetm_log_entry *buf[2] = {nullptr, nullptr};  // pinned, alternating rounds
    int cur = 0;
    uint64_t fill = 0;     // tuples written into buf[cur]
    uint64_t shipped = 0;  // tuples of buf[cur] already queued for H2D
};

int ilog2(uint64_t v) {
    int r = 0;
    while ((1ull << r) < v) ++r;
    return r;
}

bool pow2(uint64_t v) { return v && !(v & (v - 1)); }

}  // namespace

constexpr int kRoundRing = 64;        // rounds whose end hetm_batch_poll can still look up
constexpr size_t kBatchRecs = 65536;  // batches hetm_batch_poll keeps track of

struct hetm_ctx {
    int device = 0;
    int n_sm = 0;
    cudaStream_t stream = nullptr;
    bool own_stream = false;
    cudaStream_t ship = nullptr;
    hetm_config cfg{};
    uint64_t n_words = 0;
    uint32_t granule_bytes = 0, gshift = 0, cshift = 0;
    uint64_t rs_words = 0, ws_words = 0;

    int32_t *W = nullptr, *S = nullptr;
    uint32_t *TS = nullptr, *rs = nullptr, *ws = nullptr;
    uint32_t *filter = nullptr;    // shared-memory filter of RS_bmp (validation)
    unsigned long long *locks = nullptr;
    Scratch *scr = nullptr;
    DevRound *d_round = nullptr;   // [0] fused round, [1 + b] batch b alone
    DevBatch *d_batches = nullptr;
    uint64_t *d_prefix = nullptr;
    uint64_t *d_prefix0 = nullptr; // {0} for single-batch launches
    hetm_log_entry *dlog[2] = {nullptr, nullptr};

    // pinned staging of the batch table: two stagings per round (batches at
    // its start, the CPU log after the execution phase is launched), for two
    // rounds in flight; a slot is refilled once its copies are done
    static constexpr int kStages = 4;
    struct Stage {
        DevRound *rounds = nullptr;
        DevBatch *batches = nullptr;
        uint64_t *prefix = nullptr;
        cudaEvent_t used = nullptr;
    } stage[kStages];
    int stage_cur = 0;
    RoundOut *out = nullptr;       // pinned: [0] hetm_validate, [1 + slot] a round in flight

    std::vector<DevBatch> pending;
    std::vector<uint64_t> pending_ids;  // ids of `pending`, same order
    uint64_t next_batch_id = 1;

    // batch tracking for hetm_batch_poll: every round that runs batches gets a
    // sequence number; its end (after the merge) records an event and a pinned
    // copy of its conflict count in slot seq % kRoundRing
    struct BatchRec {
        uint32_t n_tx = 0;
        uint64_t round = 0;  // 0 while queued
        bool done = false;
        uint32_t outcome = 0;
        double latency_ms = 0;
        std::chrono::steady_clock::time_point t_submit;
    };
    std::map<uint64_t, BatchRec> brec;
    uint64_t round_seq = 0;             // rounds that ran batches so far
    uint64_t exec_round = 0;            // round whose execution ran, not merged yet (0: none)
    cudaEvent_t rend[kRoundRing] = {};  // end of round seq, slot seq % kRoundRing
    uint64_t rend_seq[kRoundRing] = {};
    int rend_force[kRoundRing] = {};    // conflict decided by the caller (-1: counted)
    unsigned long long *rconf = nullptr; // pinned: hits of round seq, same slot

    // CPU logs
    std::vector<std::unique_ptr<ThreadLog>> tlogs;
    std::atomic<uint64_t> dlog_fill{0};
    int dlog_cur = 0;
    cudaEvent_t dlog_free[2] = {nullptr, nullptr};  // last validation that read dlog[i]
    cudaEvent_t ship_done = nullptr;
    cudaEvent_t tlog_free[2] = {nullptr, nullptr};  // copies out of host buffers i
    const hetm_log_entry *attached = nullptr;
    uint64_t attached_n = 0;
    std::atomic<int> ship_err{0};

    // graphs
    // Up to kInFlight rounds launched by hetm_round(ctx, NULL) and not yet
    // collected by hetm_round_wait, oldest at slot r_head.  Each slot has its
    // own sync graph, timing events, pinned results and WS_bmp copy, so a
    // round can be launched before the previous one is collected.
    static constexpr int kInFlight = 2;
    cudaGraphExec_t g_exec = nullptr, g_sync[kInFlight] = {};
    uint32_t n_kern[2] = {0, 0};  // kernel nodes of g_exec / g_sync
    cudaEvent_t ev[kInFlight][7] = {};  // timing: 0/6 around the executor, 1..4 in the sync graph, 5 end
    uint64_t slot_n_log[kInFlight] = {};
    uint32_t slot_nb[kInFlight] = {};
    int r_head = 0, r_open = 0;
    // conflict policy: WS_bmp of the last round (pinned host copy, for
    // hetm_read_dirty), whether that round's GPU writes survived, and the
    // anti-starvation state
    uint32_t *ws_host = nullptr;   // kInFlight copies, one per round slot
    const uint32_t *ws_last = nullptr;  // the copy of the last collected round
    bool last_gpu_survived = false;
    uint32_t gpu_losses = 0;
    std::atomic<bool> cpu_read_only{false};
    // double-buffered merge to the host (hetm_read_dirty_async): its stream,
    // "round ended" / "copies done" events, and whether the next write of
    // STMR^S must still wait for the copies
    cudaStream_t d2h = nullptr;
    cudaEvent_t ev_d2h_from = nullptr, ev_d2h_done = nullptr;
    bool d2h_pending = false, d2h_recorded = false;
    // ordered executor: side stream of the read-only phase, and its fork/join
    cudaStream_t ro_side = nullptr;
    cudaEvent_t ro_fork = nullptr, ro_join = nullptr;
    // early validation: watcher stream, "stop flag reset" node of g_exec, watcher done
    bool early = false;
    cudaStream_t watch = nullptr;
    cudaEvent_t ev_watch_start = nullptr, ev_watch_done = nullptr;

    OrderArgs ord{};               // ordered-executor scratch (exec_mode ORDERED)
    uint32_t *rest = nullptr;      // optimistic executor: indices left by the read-only phase
    uint32_t *w2list = nullptr;    // ordered executor: the W2 updates of a launch
    int tail_blocks = 0;           //   grid of the STM that runs them after the ordered phase
    int ord_blocks = 0;
    int exec_blocks = 0, exec_threads = 256, stream_blocks = 0;
    unsigned long long prev_counters[3] = {0, 0, 0};

    std::vector<void *> dev_allocs;
};

#define CK(x)                                                                       \
    do {                                                                            \
        cudaError_t e_ = (x);                                                       \
        if (e_ != cudaSuccess) {                                                    \
            std::fprintf(stderr, "hetm: %s failed: %s (%s:%d)\n", #x,              \
                         cudaGetErrorString(e_), __FILE__, __LINE__);               \
            return HETM_ECUDA;                                                      \
        }                                                                           \
    } while (0)

namespace {

// Order the context stream after the host copies of hetm_read_dirty_async
// still reading STMR^S; every write of STMR^S (apply, merge, load) comes after.
cudaError_t after_host_copies(hetm_ctx *c) {
    if (!c->d2h_pending) return cudaSuccess;
    c->d2h_pending = false;
    return cudaStreamWaitEvent(c->stream, c->ev_d2h_done, 0);
}

void *dev_alloc(hetm_ctx *c, size_t bytes) {
    void *p = nullptr;
    if (bytes == 0) bytes = 16;
    if (c->cfg.dev_alloc) {
        p = c->cfg.dev_alloc(bytes, c->cfg.alloc_user);
    } else if (cudaMalloc(&p, bytes) != cudaSuccess) {
        cudaGetLastError();
        p = nullptr;
    }
    if (p) c->dev_allocs.push_back(p);
    return p;
}

template <class T>
bool dev_alloc_t(hetm_ctx *c, T **p, size_t count) {
    *p = static_cast<T *>(dev_alloc(c, count * sizeof(T)));
    return *p != nullptr;
}

template <class T>
bool host_alloc_t(T **p, size_t count) {
    if (cudaHostAlloc(reinterpret_cast<void **>(p), std::max<size_t>(count * sizeof(T), 16),
                      cudaHostAllocDefault) != cudaSuccess) {
        cudaGetLastError();
        *p = nullptr;
        return false;
    }
    return true;
}

// Queue k tuples of thread log L for H2D at the device log's next free slot.
int ship_locked(hetm_ctx *c, ThreadLog &L, uint64_t k) {
    if (k == 0) return HETM_OK;
    uint64_t off = c->dlog_fill.fetch_add(k);
    if (off + k > c->cfg.log_capacity) {
        c->dlog_fill.fetch_sub(k);
        return HETM_ECAPACITY;
    }
    cudaError_t e = cudaMemcpyAsync(c->dlog[c->dlog_cur] + off, L.buf[L.cur] + L.shipped,
                                    k * sizeof(hetm_log_entry), cudaMemcpyHostToDevice, c->ship);
    if (e != cudaSuccess) {
        c->ship_err.store(HETM_ECUDA);
        return HETM_ECUDA;
    }
    L.shipped += k;
    return HETM_OK;
}

// End the CPU side of a round: ship every partial chunk, switch every thread
// to its other host buffer and the device log to its other buffer.  On
// return *log / *n describe the round's device log; c->ship_done follows
// the last copy.
int flush_logs(hetm_ctx *c, const hetm_log_entry **log, uint64_t *n) {
    std::vector<std::unique_lock<std::mutex>> held;
    held.reserve(c->tlogs.size());
    for (auto &L : c->tlogs) held.emplace_back(L->mu);
    int rc = HETM_OK;
    for (auto &Lp : c->tlogs) {
        ThreadLog &L = *Lp;
        if (L.buf[L.cur]) {
            int r = ship_locked(c, L, L.fill - L.shipped);
            if (r != HETM_OK) rc = r;
        }
    }
    if (c->ship_err.load() != HETM_OK) rc = c->ship_err.exchange(HETM_OK);
    const int hb = c->tlogs.empty() ? 0 : c->tlogs[0]->cur;
    CK(cudaEventRecord(c->tlog_free[hb], c->ship));
    CK(cudaEventRecord(c->ship_done, c->ship));
    if (c->attached) {
        *log = c->attached;
        *n = c->attached_n;
    } else {
        *log = c->dlog[c->dlog_cur];
        *n = c->dlog_fill.load();
    }
    c->attached = nullptr;
    c->attached_n = 0;
    // next round: the other buffers; wait until the copies out of the other
    // host buffer (issued two rounds ago) are done before refilling it
    CK(cudaEventSynchronize(c->tlog_free[hb ^ 1]));
    for (auto &Lp : c->tlogs) {
        Lp->cur ^= 1;
        Lp->fill = 0;
        Lp->shipped = 0;
    }
    c->dlog_cur ^= 1;
    c->dlog_fill.store(0);
    // the other device buffer is refilled only after the validation that
    // last read it
    CK(cudaStreamWaitEvent(c->ship, c->dlog_free[c->dlog_cur], 0));
    return rc;
}

// Stage the pending batch table and the round sizes into device memory.
int stage_round(hetm_ctx *c, const hetm_log_entry *log, uint64_t n_log) {
    auto &st = c->stage[c->stage_cur];
    CK(cudaEventSynchronize(st.used));
    const uint32_t nb = (uint32_t)c->pending.size();
    uint64_t total = 0;
    for (uint32_t b = 0; b < nb; ++b) {
        st.batches[b] = c->pending[b];
        st.prefix[b] = total;
        st.rounds[1 + b] = DevRound{c->pending[b].n_tx, 0, nullptr, 1, 0};
        total += c->pending[b].n_tx;
    }
    st.prefix[nb] = total;
    st.rounds[0] = DevRound{total, n_log, log, nb, 0};
    CK(cudaMemcpyAsync(c->d_round, st.rounds, sizeof(DevRound) * (1 + nb), cudaMemcpyHostToDevice,
                       c->stream));
    if (nb) {
        CK(cudaMemcpyAsync(c->d_batches, st.batches, sizeof(DevBatch) * nb, cudaMemcpyHostToDevice,
                           c->stream));
        CK(cudaMemcpyAsync(c->d_prefix, st.prefix, sizeof(uint64_t) * (nb + 1),
                           cudaMemcpyHostToDevice, c->stream));
    }
    CK(cudaEventRecord(st.used, c->stream));
    c->stage_cur = (c->stage_cur + 1) % hetm_ctx::kStages;
    return HETM_OK;
}

ExecArgs exec_args(hetm_ctx *c, const DevRound *rp, const DevBatch *batches,
                   const uint64_t *prefix) {
    ExecArgs a{};
    a.W = c->W;
    a.n_words = c->n_words;
    a.locks = c->locks;
    a.lock_mask = (1u << c->cfg.lock_log2) - 1;
    a.lock_shift = c->cfg.lock_shift;
    a.gv = &c->scr->gv;
    a.rs = c->rs;
    a.filter = c->filter;
    a.gshift = c->gshift;
    a.ws = c->ws;
    a.cshift = c->cshift;
    a.rp = rp;
    a.batches = batches;
    a.prefix = prefix;
    a.next = &c->scr->next;
    a.max_attempts = c->cfg.max_attempts;
    a.budget_ns = c->cfg.exec_budget_us ? 1000ull * c->cfg.exec_budget_us : 20ull * 1000 * 1000 * 1000;
    a.counters = c->scr->counters;
    a.err = &c->scr->err;
    if (c->early) {
        a.stop = &c->scr->stop;
        a.segs_done = &c->scr->segs_done;
        a.segs_total = &c->scr->segs_total;
    }
    a.cache_log2_sets = c->cfg.cache_log2_sets;
    a.key_base = c->cfg.cache_key_base;
    a.val_base = c->cfg.cache_val_base;
    a.lru_base = c->cfg.cache_lru_base;
    a.ver_base = c->cfg.cache_ver_base;
    a.instrument = c->cfg.uninstrumented ? 0u : 1u;
    return a;
}

// Ordered mode: the W2 updates of the launch (listed by the ordering pre-pass)
// run under the STM after the ordered phase, serialized after every
// transaction of the launch (the pre-pass took the clock past the launch's
// versions); a launch without W2 updates draws nothing and ends at once.
cudaError_t launch_w2_tail(hetm_ctx *c, ExecArgs e) {
    e.skip_ro = 1;
    e.rest = c->w2list;
    e.rest_n = &c->scr->w2n;
    e.rest_cap = ~0ull;
    e.stop = nullptr;
    e.segs_done = e.segs_total = nullptr;
    cudaError_t err = cudaMemsetAsync(&c->scr->next, 0, sizeof(unsigned long long), c->stream);
    if (err == cudaSuccess) err = launch_exec(e, c->tail_blocks, 256, c->stream);
    return err;
}

// Executor launch(es) for the staged table: one persistent launch over all
// batches, or one launch per batch.
// `capturing`: recorded into g_exec, which then marks (ev_watch_start) the
// point where the early-validation stop flag has been cleared.
int enqueue_exec(hetm_ctx *c, bool per_batch, uint32_t nb, bool capturing = false) {
    if (c->cfg.exec_mode == HETM_EXEC_ORDERED) {
        OrderArgs o = c->ord;
        if (!per_batch) {
            o.e = exec_args(c, c->d_round, c->d_batches, c->d_prefix);
            if (c->early) {
                CK(cudaMemsetAsync(&c->scr->stop, 0, 4 * sizeof(unsigned int), c->stream));
                if (capturing)
                    CK(cudaEventRecordWithFlags(c->ev_watch_start, c->stream, cudaEventRecordExternal));
            }
            CK(cudaMemsetAsync(&c->scr->w2n, 0, sizeof(unsigned long long), c->stream));
            CK(launch_ordered(o, c->ord_blocks, c->stream_blocks, c->stream, c->ro_side, c->ro_fork,
                              c->ro_join));
            CK(launch_w2_tail(c, o.e));
            // stream order: set only after every kernel of the execution phase
            if (c->early) CK(cudaMemsetAsync(&c->scr->exec_over, 0xFF, sizeof(unsigned int), c->stream));
            return HETM_OK;
        }
        for (uint32_t b = 0; b < nb; ++b) {
            o.e = exec_args(c, c->d_round + 1 + b, c->d_batches + b, c->d_prefix0);
            o.e.stop = nullptr;  // no watcher runs beside per-batch launches
            o.e.segs_done = o.e.segs_total = nullptr;
            CK(cudaMemsetAsync(&c->scr->w2n, 0, sizeof(unsigned long long), c->stream));
            CK(launch_ordered(o, c->ord_blocks, c->stream_blocks, c->stream, c->ro_side, c->ro_fork,
                              c->ro_join));
            CK(launch_w2_tail(c, o.e));
        }
        return HETM_OK;
    }
    // Optimistic executor: the W1 read-only transactions of a launch run first,
    // lock-free on the launch-start state (serialized before every update of
    // the launch, commit key 2 * v0 + 1), so that the STM runs the updates only.
    auto run = [&](ExecArgs e) -> int {
        CK(cudaMemcpyAsync(&c->scr->v0, &c->scr->gv, sizeof(unsigned long long), cudaMemcpyDeviceToDevice,
                           c->stream));
        e.rest = c->rest;
        e.rest_n = &c->scr->rest_n;
        e.rest_cap = c->rest ? c->cfg.max_round_tx : 0;
        if (c->rest) CK(cudaMemsetAsync(&c->scr->rest_n, 0, sizeof(unsigned long long), c->stream));
        CK(launch_ro_phase(e, &c->scr->v0, c->stream_blocks, c->stream));
        e.skip_ro = 1;
        CK(cudaMemsetAsync(&c->scr->next, 0, sizeof(unsigned long long), c->stream));
        CK(launch_exec(e, c->exec_blocks, c->exec_threads, c->stream));
        return HETM_OK;
    };
    if (!per_batch) return run(exec_args(c, c->d_round, c->d_batches, c->d_prefix));
    for (uint32_t b = 0; b < nb; ++b) {
        const int rc = run(exec_args(c, c->d_round + 1 + b, c->d_batches + b, c->d_prefix0));
        if (rc != HETM_OK) return rc;
    }
    return HETM_OK;
}

// Validation + apply as the conflict policy wants them: GPU-loses fuses the
// TS max into validation and applies unconditionally; CPU-loses validates
// first and applies only when no tuple hit (both passes read the count).
int enqueue_validate_apply(hetm_ctx *c, uint32_t *flags, cudaEvent_t *e) {
    const bool cpu_loses = c->cfg.conflict_policy == HETM_POLICY_CPU_LOSES;
    CK(launch_validate(c->d_round, c->rs, c->gshift, c->n_words, flags, &c->scr->conflicts,
                       cpu_loses ? nullptr : c->TS, &c->scr->err, c->filter, c->n_sm, c->stream));
    if (e) CK(cudaEventRecordWithFlags(e[1], c->stream, cudaEventRecordExternal));
    if (cpu_loses)
        CK(launch_ts_max_if_clean(c->d_round, c->TS, c->n_words, &c->scr->conflicts, &c->scr->err,
                                  c->stream_blocks, c->stream));
    CK(launch_apply(c->d_round, c->TS, c->W, c->S, c->n_words, c->stream_blocks, c->stream,
                    cpu_loses ? &c->scr->conflicts : nullptr));
    return HETM_OK;
}

// validate (+ TS max) -> apply -> merge -> clear; events e[0..3] between
// phases when non-null.
int enqueue_sync(hetm_ctx *c, uint32_t *flags, int force, cudaEvent_t *e, RoundOut *out,
                 uint32_t *ws_dst) {
    CK(cudaMemsetAsync(&c->scr->conflicts, 0, 2 * sizeof(unsigned long long), c->stream));
    if (e) CK(cudaEventRecordWithFlags(e[0], c->stream, cudaEventRecordExternal));
    int rc = enqueue_validate_apply(c, flags, e);
    if (rc != HETM_OK) return rc;
    if (e) CK(cudaEventRecordWithFlags(e[2], c->stream, cudaEventRecordExternal));
    // CPU-loses: the GPU's writes stand whatever validation found (W -> S)
    if (c->cfg.conflict_policy == HETM_POLICY_CPU_LOSES) force = 0;
    CK(launch_merge(c->ws, c->cshift, c->W, c->S, c->n_words, &c->scr->conflicts, force,
                    &c->scr->dirty, c->stream_blocks, c->stream, &c->scr->err));
    CK(cudaMemcpyAsync(ws_dst, c->ws, c->ws_words * 4, cudaMemcpyDeviceToHost, c->stream));
    CK(cudaMemsetAsync(c->rs, 0, c->rs_words * 4, c->stream));
    CK(cudaMemsetAsync(c->filter, 0, kFilterBits / 8, c->stream));
    CK(cudaMemsetAsync(c->ws, 0, c->ws_words * 4, c->stream));
    if (e) CK(cudaEventRecordWithFlags(e[3], c->stream, cudaEventRecordExternal));
    CK(cudaMemcpyAsync(out, c->scr->counters, 5 * sizeof(unsigned long long),
                       cudaMemcpyDeviceToHost, c->stream));
    CK(cudaMemcpyAsync(&out->err, &c->scr->err, sizeof(int), cudaMemcpyDeviceToHost, c->stream));
    CK(cudaMemcpyAsync(&out->stopped, &c->scr->stop, sizeof(unsigned int), cudaMemcpyDeviceToHost,
                       c->stream));
    return HETM_OK;
}

// which: 0 = the execution phase, 1 = the sync phase of round slot `slot`
int capture(hetm_ctx *c, cudaGraphExec_t *out, int which, int slot = 0) {
    cudaGraph_t g = nullptr;
    CK(cudaStreamBeginCapture(c->stream, cudaStreamCaptureModeThreadLocal));
    int rc = which == 0 ? enqueue_exec(c, false, 0, true)
                        : enqueue_sync(c, nullptr, -1, c->ev[slot] + 1, c->out + 1 + slot,
                                       c->ws_host + (size_t)slot * c->ws_words);
    cudaError_t e = cudaStreamEndCapture(c->stream, &g);
    if (rc != HETM_OK) {
        if (g) cudaGraphDestroy(g);
        return rc;
    }
    if (e == cudaSuccess) {
        size_t nn = 0;
        e = cudaGraphGetNodes(g, nullptr, &nn);
        std::vector<cudaGraphNode_t> nodes(nn);
        if (e == cudaSuccess && nn) e = cudaGraphGetNodes(g, nodes.data(), &nn);
        uint32_t k = 0;
        for (size_t i = 0; e == cudaSuccess && i < nn; ++i) {
            cudaGraphNodeType t;
            e = cudaGraphNodeGetType(nodes[i], &t);
            k += t == cudaGraphNodeTypeKernel;
        }
        c->n_kern[which] = k;
    }
    if (e != cudaSuccess) {
        if (g) cudaGraphDestroy(g);
        CK(e);
    }
    e = cudaGraphInstantiate(out, g, 0);
    cudaGraphDestroy(g);
    CK(e);
    return HETM_OK;
}

}  // namespace

extern "C" {

const char *hetm_strerror(int code) {
    switch (code) {
        case HETM_OK: return "ok";
        case HETM_EINVAL: return "invalid argument or precondition violated";
        case HETM_ENOMEM: return "out of device or pinned host memory";
        case HETM_ECAPACITY: return "fixed-capacity buffer or table full";
        case HETM_ETIMEOUT: return "bounded device wait gave up";
        case HETM_ECUDA: return "CUDA runtime error";
        case HETM_EBUSY: return "not admitted now; retry later";
        case HETM_EDEVICE: return "kernel met an out-of-range address";
        default: return "unknown error";
    }
}

int hetm_config_default(hetm_config *cfg) {
    if (!cfg) return HETM_EINVAL;
    std::memset(cfg, 0, sizeof(*cfg));
    cfg->ws_chunk_bytes = 16384;
    cfg->lock_log2 = 22;
    cfg->lock_shift = 0;
    cfg->exec_blocks = 0;
    cfg->exec_threads = 256;
    cfg->max_attempts = 1u << 16;
    cfg->cpu_threads = 8;
    cfg->log_chunk_bytes = 49152;
    cfg->log_capacity = 1ull << 24;
    cfg->cpu_log_capacity = 1ull << 21;
    cfg->max_batches = 4096;
    cfg->exec_mode = HETM_EXEC_ORDERED;
    cfg->max_round_tx = 1ull << 22;
    return HETM_OK;
}

void hetm_destroy(hetm_ctx *c) {
    if (!c) return;
    cudaSetDevice(c->device);
    if (c->ship) cudaStreamSynchronize(c->ship);
    if (c->stream) cudaStreamSynchronize(c->stream);
    if (c->g_exec) cudaGraphExecDestroy(c->g_exec);
    for (auto &g : c->g_sync)
        if (g) cudaGraphExecDestroy(g);
    for (auto &slot : c->ev)
        for (auto &e : slot)
            if (e) cudaEventDestroy(e);
    for (auto &s : c->stage) {
        if (s.rounds) cudaFreeHost(s.rounds);
        if (s.batches) cudaFreeHost(s.batches);
        if (s.prefix) cudaFreeHost(s.prefix);
        if (s.used) cudaEventDestroy(s.used);
    }
    for (int i = 0; i < 2; ++i) {
        if (c->dlog_free[i]) cudaEventDestroy(c->dlog_free[i]);
        if (c->tlog_free[i]) cudaEventDestroy(c->tlog_free[i]);
    }
    if (c->ship_done) cudaEventDestroy(c->ship_done);
    if (c->watch) cudaStreamSynchronize(c->watch);
    if (c->ev_watch_start) cudaEventDestroy(c->ev_watch_start);
    if (c->ev_watch_done) cudaEventDestroy(c->ev_watch_done);
    if (c->watch) cudaStreamDestroy(c->watch);
    for (auto &L : c->tlogs)
        for (auto *b : L->buf)
            if (b) cudaFreeHost(b);
    if (c->out) cudaFreeHost(c->out);
    if (c->rconf) cudaFreeHost(c->rconf);
    if (c->ro_side) {
        cudaStreamSynchronize(c->ro_side);
        cudaStreamDestroy(c->ro_side);
    }
    if (c->d2h) {
        cudaStreamSynchronize(c->d2h);
        cudaStreamDestroy(c->d2h);
    }
    if (c->ev_d2h_from) cudaEventDestroy(c->ev_d2h_from);
    if (c->ev_d2h_done) cudaEventDestroy(c->ev_d2h_done);
    if (c->ro_fork) cudaEventDestroy(c->ro_fork);
    if (c->ro_join) cudaEventDestroy(c->ro_join);
    for (auto &e : c->rend)
        if (e) cudaEventDestroy(e);
    if (c->ws_host) cudaFreeHost(c->ws_host);
    for (void *p : c->dev_allocs) {
        if (c->cfg.dev_free) c->cfg.dev_free(p, c->cfg.alloc_user);
        else cudaFree(p);
    }
    if (c->ship) cudaStreamDestroy(c->ship);
    if (c->own_stream && c->stream) cudaStreamDestroy(c->stream);
    delete c;
}

int hetm_init(hetm_ctx **out, uint64_t stmr_words, uint32_t granule_bytes, const hetm_config *cfg,
              void *stream) {
    if (!out || stmr_words == 0 || stmr_words >= (1ull << 32)) return HETM_EINVAL;
    if (!pow2(granule_bytes) || granule_bytes < 4) return HETM_EINVAL;
    hetm_config d;
    hetm_config_default(&d);
    if (cfg) d = *cfg;
    if (!pow2(d.ws_chunk_bytes) || d.ws_chunk_bytes < 16) return HETM_EINVAL;
    if (d.lock_log2 < 1 || d.lock_log2 > 30 || d.lock_shift > 31) return HETM_EINVAL;
    if (d.exec_mode == HETM_EXEC_ORDERED) {
        if (d.exec_threads != 128 && d.exec_threads != 256 && d.exec_threads != 512)
            return HETM_EINVAL;
    } else if (d.exec_threads == 0 || d.exec_threads % 32 || d.exec_threads > 256) {
        return HETM_EINVAL;
    }
    if (d.log_chunk_bytes < 12 || d.log_chunk_bytes % 12 || d.max_attempts == 0) return HETM_EINVAL;
    if (d.max_batches == 0 || d.max_batches > 65535 || d.cpu_threads == 0 || d.log_capacity == 0)
        return HETM_EINVAL;
    if (d.cache_log2_sets > 28) return HETM_EINVAL;
    if (d.exec_mode > HETM_EXEC_OPTIMISTIC) return HETM_EINVAL;
    if (d.conflict_policy > HETM_POLICY_CPU_LOSES) return HETM_EINVAL;
    if (d.exec_mode == HETM_EXEC_ORDERED && (d.max_round_tx == 0 || d.max_round_tx > (1ull << 28)))
        return HETM_EINVAL;

    hetm_ctx *c = new (std::nothrow) hetm_ctx();
    if (!c) return HETM_ENOMEM;
    c->cfg = d;
    c->n_words = stmr_words;
    c->granule_bytes = granule_bytes;
    c->gshift = (uint32_t)ilog2(granule_bytes / 4);
    c->cshift = (uint32_t)ilog2(d.ws_chunk_bytes / 4);
    const uint64_t n_gran = ((stmr_words - 1) >> c->gshift) + 1;
    const uint64_t n_chunk = ((stmr_words - 1) >> c->cshift) + 1;
    c->rs_words = (n_gran + 31) / 32;
    c->ws_words = (n_chunk + 31) / 32;

    auto fail = [&](int rc) {
        hetm_destroy(c);
        return rc;
    };
    if (cudaGetDevice(&c->device) != cudaSuccess) return fail(HETM_ECUDA);
    if (cudaDeviceGetAttribute(&c->n_sm, cudaDevAttrMultiProcessorCount, c->device) != cudaSuccess)
        return fail(HETM_ECUDA);
    if (stream) {
        c->stream = static_cast<cudaStream_t>(stream);
    } else {
        if (cudaStreamCreateWithFlags(&c->stream, cudaStreamNonBlocking) != cudaSuccess)
            return fail(HETM_ECUDA);
        c->own_stream = true;
    }
    if (cudaStreamCreateWithFlags(&c->ship, cudaStreamNonBlocking) != cudaSuccess)
        return fail(HETM_ECUDA);
    c->early = d.early_validate != 0 && d.exec_mode == HETM_EXEC_ORDERED;
    if (c->early && (cudaStreamCreateWithFlags(&c->watch, cudaStreamNonBlocking) != cudaSuccess ||
                     cudaEventCreateWithFlags(&c->ev_watch_start, cudaEventDisableTiming) != cudaSuccess ||
                     cudaEventCreateWithFlags(&c->ev_watch_done, cudaEventDisableTiming) != cudaSuccess))
        return fail(HETM_ECUDA);

    const uint32_t nb = d.max_batches;
    if (!dev_alloc_t(c, &c->W, stmr_words) || !dev_alloc_t(c, &c->S, stmr_words) ||
        !dev_alloc_t(c, &c->TS, stmr_words) || !dev_alloc_t(c, &c->rs, c->rs_words) ||
        !dev_alloc_t(c, &c->ws, c->ws_words) || !dev_alloc_t(c, &c->locks, 1ull << d.lock_log2) ||
        !dev_alloc_t(c, &c->filter, kFilterBits / 32) ||
        !dev_alloc_t(c, &c->scr, 1) || !dev_alloc_t(c, &c->d_round, nb + 1) ||
        !dev_alloc_t(c, &c->d_batches, nb) || !dev_alloc_t(c, &c->d_prefix, nb + 1) ||
        !dev_alloc_t(c, &c->d_prefix0, 2) || !dev_alloc_t(c, &c->dlog[0], d.log_capacity) ||
        !dev_alloc_t(c, &c->dlog[1], d.log_capacity))
        return fail(HETM_ENOMEM);
    // optimistic executor: the list of indices its read-only phase leaves to
    // the STM (rounds above max_round_tx transactions go unlisted)
    if (d.exec_mode == HETM_EXEC_OPTIMISTIC && d.max_round_tx && d.max_round_tx <= (1ull << 32) &&
        !dev_alloc_t(c, &c->rest, d.max_round_tx))
        return fail(HETM_ENOMEM);
    if (d.exec_mode == HETM_EXEC_ORDERED) {
        OrderArgs &o = c->ord;
        o.cap_tx = (uint32_t)d.max_round_tx;
        o.cap_acc = 4 * o.cap_tx;
        o.seg_log2 = (uint32_t)ilog2(d.exec_threads);
        o.key_bits = (uint32_t)ilog2(stmr_words);
        if (o.key_bits == 0) o.key_bits = 1;
        const uint64_t hist_n = 256ull * ((o.cap_acc + 2047) / 2048);
        const uint64_t tot_n = std::max<uint64_t>(hist_n, o.cap_acc) / 1024 + 2;
        if (!dev_alloc_t(c, &o.scan_tot, tot_n) ||
            !dev_alloc_t(c, &o.keys0, o.cap_acc) || !dev_alloc_t(c, &o.vals0, o.cap_acc) ||
            !dev_alloc_t(c, &o.keys1, o.cap_acc) || !dev_alloc_t(c, &o.vals1, o.cap_acc) ||
            !dev_alloc_t(c, &o.hist, hist_n) || !dev_alloc_t(c, &o.runs, o.cap_acc) ||
            !dev_alloc_t(c, &o.rec, o.cap_tx) || !dev_alloc_t(c, &o.packed, o.cap_acc) ||
            !dev_alloc_t(c, &o.n_acc, 5) || !dev_alloc_t(c, &o.cache_heads, o.cap_tx) ||
            !dev_alloc_t(c, &o.v0, 1))
            return fail(HETM_ENOMEM);
        o.n_ord = o.n_acc + 1;
        o.n_tx32 = o.n_acc + 2;
        o.n_cache_runs = o.n_acc + 3;
        o.n_hist = o.n_acc + 4;
        if (!dev_alloc_t(c, &c->w2list, o.cap_tx)) return fail(HETM_ENOMEM);
        o.w2list = c->w2list;
        o.w2n = &c->scr->w2n;
    }
    for (auto &s : c->stage) {
        if (!host_alloc_t(&s.rounds, nb + 1) || !host_alloc_t(&s.batches, nb) ||
            !host_alloc_t(&s.prefix, nb + 1))
            return fail(HETM_ENOMEM);
        if (cudaEventCreateWithFlags(&s.used, cudaEventDisableTiming) != cudaSuccess)
            return fail(HETM_ECUDA);
    }
    if (!host_alloc_t(&c->out, 1 + hetm_ctx::kInFlight) ||
        !host_alloc_t(&c->ws_host, hetm_ctx::kInFlight * c->ws_words))
        return fail(HETM_ENOMEM);
    std::memset(c->ws_host, 0, hetm_ctx::kInFlight * c->ws_words * 4);
    std::memset(c->out, 0, (1 + hetm_ctx::kInFlight) * sizeof(RoundOut));
    c->ws_last = c->ws_host;
    for (int i = 0; i < 2; ++i) {
        if (cudaEventCreateWithFlags(&c->dlog_free[i], cudaEventDisableTiming) != cudaSuccess ||
            cudaEventCreateWithFlags(&c->tlog_free[i], cudaEventDisableTiming) != cudaSuccess)
            return fail(HETM_ECUDA);
    }
    if (cudaEventCreateWithFlags(&c->ship_done, cudaEventDisableTiming) != cudaSuccess)
        return fail(HETM_ECUDA);
    for (auto &slot : c->ev)
        for (auto &e : slot)
            if (cudaEventCreate(&e) != cudaSuccess) return fail(HETM_ECUDA);
    for (auto &e : c->rend)
        if (cudaEventCreateWithFlags(&e, cudaEventDisableTiming) != cudaSuccess) return fail(HETM_ECUDA);
    if (cudaStreamCreateWithFlags(&c->d2h, cudaStreamNonBlocking) != cudaSuccess ||
        cudaEventCreateWithFlags(&c->ev_d2h_from, cudaEventDisableTiming) != cudaSuccess ||
        cudaEventCreateWithFlags(&c->ev_d2h_done, cudaEventDisableTiming) != cudaSuccess)
        return fail(HETM_ECUDA);
    if (cudaStreamCreateWithFlags(&c->ro_side, cudaStreamNonBlocking) != cudaSuccess ||
        cudaEventCreateWithFlags(&c->ro_fork, cudaEventDisableTiming) != cudaSuccess ||
        cudaEventCreateWithFlags(&c->ro_join, cudaEventDisableTiming) != cudaSuccess)
        return fail(HETM_ECUDA);
    if (!host_alloc_t(&c->rconf, kRoundRing)) return fail(HETM_ENOMEM);
    std::memset(c->rconf, 0, kRoundRing * sizeof(unsigned long long));
    for (uint32_t t = 0; t < d.cpu_threads; ++t) c->tlogs.emplace_back(new ThreadLog());

    int occ = 0;
    c->exec_threads = (int)d.exec_threads;
    if (d.exec_mode == HETM_EXEC_ORDERED) {
        if (ordered_exec_occupancy(d.exec_threads, &occ) != 0 || occ < 1) occ = 1;
        c->ord_blocks = d.exec_blocks ? (int)d.exec_blocks : c->n_sm * occ;
        int tocc = 0;
        if (exec_occupancy(256, &tocc) != 0 || tocc < 1) tocc = 1;
        c->tail_blocks = c->n_sm * tocc;
    } else {
        if (exec_occupancy(c->exec_threads, &occ) != 0 || occ < 1) occ = 1;
        c->exec_blocks = d.exec_blocks ? (int)d.exec_blocks : c->n_sm * occ;
    }
    c->stream_blocks = c->n_sm * 8;
    if (validate_setup() != cudaSuccess) return fail(HETM_ECUDA);

    if (cudaMemsetAsync(c->locks, 0, (1ull << d.lock_log2) * 8, c->stream) != cudaSuccess ||
        cudaMemsetAsync(c->scr, 0, sizeof(Scratch), c->stream) != cudaSuccess ||
        cudaMemsetAsync(c->d_prefix0, 0, 16, c->stream) != cudaSuccess ||
        cudaMemsetAsync(c->rs, 0, c->rs_words * 4, c->stream) != cudaSuccess ||
        cudaMemsetAsync(c->filter, 0, kFilterBits / 8, c->stream) != cudaSuccess ||
        cudaMemsetAsync(c->ws, 0, c->ws_words * 4, c->stream) != cudaSuccess ||
        cudaMemsetAsync(c->TS, 0, stmr_words * 4, c->stream) != cudaSuccess ||
        cudaMemsetAsync(c->W, 0, stmr_words * 4, c->stream) != cudaSuccess ||
        cudaMemsetAsync(c->S, 0, stmr_words * 4, c->stream) != cudaSuccess)
        return fail(HETM_ECUDA);
    for (int i = 0; i < 2; ++i) {
        if (cudaEventRecord(c->dlog_free[i], c->stream) != cudaSuccess ||
            cudaEventRecord(c->tlog_free[i], c->ship) != cudaSuccess)
            return fail(HETM_ECUDA);
    }
    for (auto &st : c->stage)
        if (cudaEventRecord(st.used, c->stream) != cudaSuccess) return fail(HETM_ECUDA);
    if (cudaStreamSynchronize(c->stream) != cudaSuccess) return fail(HETM_ECUDA);
    *out = c;
    return HETM_OK;
}

int hetm_load(hetm_ctx *c, const int32_t *src, uint64_t n) {
    const Range range("hetm_load");
    if (!c || !src || n != c->n_words) return HETM_EINVAL;
    CK(cudaSetDevice(c->device));
    CK(cudaStreamSynchronize(c->ship));
    CK(after_host_copies(c));
    CK(cudaMemcpyAsync(c->W, src, n * 4, cudaMemcpyDefault, c->stream));
    CK(cudaMemcpyAsync(c->S, c->W, n * 4, cudaMemcpyDeviceToDevice, c->stream));
    CK(cudaMemsetAsync(c->TS, 0, n * 4, c->stream));
    CK(cudaMemsetAsync(c->rs, 0, c->rs_words * 4, c->stream));
    CK(cudaMemsetAsync(c->filter, 0, kFilterBits / 8, c->stream));
    CK(cudaMemsetAsync(c->ws, 0, c->ws_words * 4, c->stream));
    CK(cudaMemsetAsync(c->locks, 0, (1ull << c->cfg.lock_log2) * 8, c->stream));
    CK(cudaMemsetAsync(c->scr, 0, sizeof(Scratch), c->stream));
    CK(cudaStreamSynchronize(c->stream));
    for (auto &L : c->tlogs) {
        std::lock_guard<std::mutex> g(L->mu);
        L->fill = L->shipped = 0;
    }
    c->dlog_fill.store(0);
    c->pending.clear();
    // batches still queued, or run by an execution phase that never merged,
    // are discarded with the state: hetm_batch_poll forgets them
    for (uint64_t id : c->pending_ids) c->brec.erase(id);
    c->pending_ids.clear();
    if (c->exec_round) {
        for (auto it = c->brec.begin(); it != c->brec.end();)
            it = it->second.round == c->exec_round ? c->brec.erase(it) : std::next(it);
        c->exec_round = 0;
    }
    c->attached = nullptr;
    c->attached_n = 0;
    std::memset(c->prev_counters, 0, sizeof(c->prev_counters));
    // rounds still in flight have finished (stream synchronized) and are discarded
    c->r_open = 0;
    c->r_head = 0;
    return HETM_OK;
}

int hetm_read_stmr(hetm_ctx *c, int which, int32_t *dst, uint64_t off, uint64_t n) {
    if (!c || !dst || (which != 0 && which != 1) || off > c->n_words || n > c->n_words - off)
        return HETM_EINVAL;
    CK(cudaSetDevice(c->device));
    CK(cudaMemcpyAsync(dst, (which ? c->S : c->W) + off, n * 4, cudaMemcpyDeviceToHost, c->stream));
    CK(cudaStreamSynchronize(c->stream));
    return HETM_OK;
}

void *hetm_device_ptr(hetm_ctx *c, int which) {
    if (!c) return nullptr;
    switch (which) {
        case 0: return c->W;
        case 1: return c->S;
        case 2: return c->TS;
        case 3: return c->rs;
        case 4: return c->ws;
        default: return nullptr;
    }
}

int hetm_bitmap_words(hetm_ctx *c, uint64_t *rs_words, uint64_t *ws_words) {
    if (!c) return HETM_EINVAL;
    if (rs_words) *rs_words = c->rs_words;
    if (ws_words) *ws_words = c->ws_words;
    return HETM_OK;
}

void *hetm_ctx_stream(hetm_ctx *c) { return c ? static_cast<void *>(c->stream) : nullptr; }

int hetm_sync(hetm_ctx *c) {
    if (!c) return HETM_EINVAL;
    CK(cudaStreamSynchronize(c->ship));
    CK(cudaStreamSynchronize(c->stream));
    return HETM_OK;
}

int hetm_gpu_submit_batch(hetm_ctx *c, const hetm_batch *b, uint64_t *batch_id) {
    if (!c || !b) return HETM_EINVAL;
    if (b->workload < HETM_WL_BANK || b->workload > HETM_WL_W2) return HETM_EINVAL;
    if (b->n_tx && !b->tx) return HETM_EINVAL;
    if (b->workload == HETM_WL_CACHE) {
        const hetm_config &f = c->cfg;
        const uint64_t ns = 1ull << f.cache_log2_sets;
        // aligned regions (16-byte vector loads of a set's keys and stamps); the
        // optimistic executor also needs one lock stripe per set region
        if ((f.exec_mode == HETM_EXEC_OPTIMISTIC && f.lock_shift < 4) ||
            f.cache_key_base % 16 || f.cache_val_base % 16 ||
            f.cache_lru_base % 16 || f.cache_key_base + 16 * ns > c->n_words ||
            f.cache_val_base + 16 * ns > c->n_words || f.cache_lru_base + 8 * ns > c->n_words ||
            f.cache_ver_base + ns > c->n_words)
            return HETM_EINVAL;
    }
    if (c->pending.size() >= c->cfg.max_batches) return HETM_EBUSY;
    if (c->cfg.exec_mode == HETM_EXEC_ORDERED) {
        uint64_t queued = b->n_tx;
        for (const auto &p : c->pending) queued += p.n_tx;
        if (queued > c->cfg.max_round_tx) return HETM_EBUSY;
    }
    DevBatch d{b->workload, b->n_tx, b->tx, b->order, b->status, b->out, b->txid_base, b->word_base};
    c->pending.push_back(d);
    const uint64_t id = c->next_batch_id++;
    c->pending_ids.push_back(id);
    hetm_ctx::BatchRec rec;
    rec.n_tx = b->n_tx;
    rec.t_submit = std::chrono::steady_clock::now();
    c->brec.emplace(id, rec);
    while (c->brec.size() > kBatchRecs) c->brec.erase(c->brec.begin());
    if (batch_id) *batch_id = id;
    return HETM_OK;
}

// The queued batches join round `r` (their execution phase is being launched).
static void assign_round(hetm_ctx *c, uint64_t r) {
    for (uint64_t id : c->pending_ids) {
        auto it = c->brec.find(id);
        if (it != c->brec.end()) it->second.round = r;
    }
    c->pending_ids.clear();
}

// End of round `r` on the context stream (after its merge): its event and the
// conflict count of its validation (or the caller's decision, force >= 0).
static int end_round(hetm_ctx *c, uint64_t r, int force) {
    const int slot = (int)(r % kRoundRing);
    CK(cudaMemcpyAsync(&c->rconf[slot], &c->scr->conflicts, sizeof(unsigned long long),
                       cudaMemcpyDeviceToHost, c->stream));
    CK(cudaEventRecord(c->rend[slot], c->stream));
    c->rend_seq[slot] = r;
    c->rend_force[slot] = force;
    return HETM_OK;
}

int hetm_gpu_exec(hetm_ctx *c, int per_batch) {
    const Range range("hetm_gpu_exec");
    if (!c) return HETM_EINVAL;
    CK(cudaSetDevice(c->device));
    if (c->pending.empty()) return HETM_OK;
    int rc = stage_round(c, nullptr, 0);
    if (rc != HETM_OK) return rc;
    rc = enqueue_exec(c, per_batch != 0, (uint32_t)c->pending.size());
    c->pending.clear();
    if (!c->exec_round) c->exec_round = ++c->round_seq;
    assign_round(c, c->exec_round);
    return rc;
}

int hetm_exec_counters(hetm_ctx *c, uint64_t *committed, uint64_t *gave_up, uint64_t *aborts) {
    if (!c) return HETM_EINVAL;
    unsigned long long h[3];
    CK(cudaStreamSynchronize(c->stream));
    CK(cudaMemcpy(h, c->scr->counters, sizeof(h), cudaMemcpyDeviceToHost));
    if (committed) *committed = h[0];
    if (gave_up) *gave_up = h[1];
    if (aborts) *aborts = h[2];
    int err = 0;
    CK(cudaMemcpy(&err, &c->scr->err, sizeof(int), cudaMemcpyDeviceToHost));
    return err_code(err);
}

int hetm_gpu_mark(hetm_ctx *c, const uint32_t *addr, const int32_t *vals, uint64_t n) {
    if (!c || (n && !addr)) return HETM_EINVAL;
    CK(cudaSetDevice(c->device));
    CK(launch_mark(addr, vals, n, c->W, c->n_words, c->rs, c->filter, c->gshift, c->ws, c->cshift,
                   &c->scr->err, c->n_sm * 4, c->stream));
    return HETM_OK;
}

int hetm_cpu_log_write(hetm_ctx *c, uint32_t thread, const hetm_log_entry *e, uint32_t n) {
    if (!c || thread >= c->tlogs.size() || (n && !e)) return HETM_EINVAL;
    if (n && c->cpu_read_only.load()) return HETM_EBUSY;  // anti-starvation round
    ThreadLog &L = *c->tlogs[thread];
    std::lock_guard<std::mutex> g(L.mu);
    if (!L.buf[L.cur]) {
        if (cudaSetDevice(c->device) != cudaSuccess) return HETM_ECUDA;
        if (!host_alloc_t(&L.buf[0], c->cfg.cpu_log_capacity) ||
            !host_alloc_t(&L.buf[1], c->cfg.cpu_log_capacity))
            return HETM_ENOMEM;
    }
    if (L.fill + n > c->cfg.cpu_log_capacity) return HETM_ECAPACITY;
    std::memcpy(L.buf[L.cur] + L.fill, e, (size_t)n * sizeof(hetm_log_entry));
    L.fill += n;
    const uint64_t chunk = c->cfg.log_chunk_bytes / sizeof(hetm_log_entry);
    while (L.fill - L.shipped >= chunk) {
        int rc = ship_locked(c, L, chunk);
        if (rc != HETM_OK) return rc;
    }
    return HETM_OK;
}

int hetm_log_attach(hetm_ctx *c, const hetm_log_entry *dev_log, uint64_t n) {
    if (!c || (n && !dev_log) || (reinterpret_cast<uintptr_t>(dev_log) & 15)) return HETM_EINVAL;
    c->attached = dev_log;
    c->attached_n = n;
    return HETM_OK;
}

int hetm_validate(hetm_ctx *c, uint64_t *n_conflicts, uint32_t *dev_flag_bits) {
    const Range range("hetm_validate");
    if (!c) return HETM_EINVAL;
    CK(cudaSetDevice(c->device));
    const hetm_log_entry *log = nullptr;
    uint64_t n = 0;
    int rc = flush_logs(c, &log, &n);
    if (rc != HETM_OK) return rc;
    std::vector<DevBatch> keep;
    keep.swap(c->pending);  // the table is staged by the exec call, not here
    rc = stage_round(c, log, n);
    keep.swap(c->pending);
    if (rc != HETM_OK) return rc;
    CK(cudaStreamWaitEvent(c->stream, c->ship_done, 0));
    CK(after_host_copies(c));
    CK(cudaMemsetAsync(&c->scr->conflicts, 0, sizeof(unsigned long long), c->stream));
    rc = enqueue_validate_apply(c, dev_flag_bits, nullptr);
    if (rc != HETM_OK) return rc;
    CK(cudaEventRecord(c->dlog_free[c->dlog_cur ^ 1], c->stream));
    if (n_conflicts) {
        unsigned long long h = 0;
        int err = 0;
        CK(cudaMemcpyAsync(&c->out->conflicts, &c->scr->conflicts, 8, cudaMemcpyDeviceToHost,
                           c->stream));
        CK(cudaMemcpyAsync(&c->out->err, &c->scr->err, 4, cudaMemcpyDeviceToHost, c->stream));
        CK(cudaStreamSynchronize(c->stream));
        h = c->out->conflicts;
        err = c->out->err;
        *n_conflicts = h;
        if (err) return err_code(err);
    }
    return HETM_OK;
}

int hetm_validate_only(hetm_ctx *c, const hetm_log_entry *dev_log, uint64_t n,
                       uint32_t *dev_flag_bits, uint64_t *dev_count) {
    if (!c || (n && !dev_log) || (reinterpret_cast<uintptr_t>(dev_log) & 15)) return HETM_EINVAL;
    CK(cudaSetDevice(c->device));
    if (n == 0) return HETM_OK;
    CK(launch_validate_direct(dev_log, n, c->rs, c->gshift, c->n_words, dev_flag_bits,
                              reinterpret_cast<unsigned long long *>(dev_count), &c->scr->err,
                              c->filter, c->n_sm, c->stream));
    return HETM_OK;
}

int hetm_merge(hetm_ctx *c, int conflict) {
    const Range range("hetm_merge");
    if (!c || conflict < -1 || conflict > 1) return HETM_EINVAL;
    CK(cudaSetDevice(c->device));
    CK(after_host_copies(c));
    CK(cudaMemsetAsync(&c->scr->dirty, 0, sizeof(unsigned long long), c->stream));
    CK(launch_merge(c->ws, c->cshift, c->W, c->S, c->n_words, &c->scr->conflicts, conflict,
                    &c->scr->dirty, c->stream_blocks, c->stream, &c->scr->err));
    CK(cudaMemsetAsync(c->rs, 0, c->rs_words * 4, c->stream));
    CK(cudaMemsetAsync(c->filter, 0, kFilterBits / 8, c->stream));
    CK(cudaMemsetAsync(c->ws, 0, c->ws_words * 4, c->stream));
    if (c->exec_round) {
        const int rc = end_round(c, c->exec_round, conflict);
        c->exec_round = 0;
        if (rc != HETM_OK) return rc;
    }
    return HETM_OK;
}

int hetm_round(hetm_ctx *c, hetm_round_stats *stats) {
    const Range range("hetm_round");
    if (!c) return HETM_EINVAL;
    // the synchronous form collects its own round: no other may be in flight
    if (c->r_open == hetm_ctx::kInFlight || (stats && c->r_open)) return HETM_EBUSY;
    CK(cudaSetDevice(c->device));
    const int slot = (c->r_head + c->r_open) % hetm_ctx::kInFlight;
    if (!c->g_exec) {
        int rc = capture(c, &c->g_exec, 0);
        if (rc != HETM_OK) return rc;
    }
    if (!c->g_sync[slot]) {
        int rc = capture(c, &c->g_sync[slot], 1, slot);
        if (rc != HETM_OK) return rc;
    }
    cudaEvent_t *ev = c->ev[slot];
    const uint32_t nb = (uint32_t)c->pending.size();
    // the executor starts right away; log chunks keep shipping meanwhile
    int rc = stage_round(c, nullptr, 0);
    if (rc != HETM_OK) return rc;
    CK(cudaEventRecord(ev[0], c->stream));
    if (nb) CK(cudaGraphLaunch(c->g_exec, c->stream));
    CK(cudaEventRecord(ev[6], c->stream));
    c->pending.clear();
    if (nb || c->exec_round) {
        if (!c->exec_round) c->exec_round = ++c->round_seq;
        assign_round(c, c->exec_round);
    }
    // end of the execution phase: ship the rest of the logs, then validate
    const hetm_log_entry *log = nullptr;
    uint64_t n = 0;
    rc = flush_logs(c, &log, &n);
    if (rc != HETM_OK) return rc;
    rc = stage_round(c, log, n);
    if (rc != HETM_OK) return rc;
    if (c->early && nb && n) {
        // the watcher starts once the stop flag is clear and the log is on the
        // device, runs beside the executor, and the sync phase waits for it
        CK(cudaStreamWaitEvent(c->watch, c->ev_watch_start, 0));
        CK(cudaStreamWaitEvent(c->watch, c->ship_done, 0));
        CK(launch_watch(log, n, c->rs, c->gshift, c->n_words, &c->scr->stop, &c->scr->segs_done,
                        &c->scr->segs_total, &c->scr->exec_over, kWatchBudgetNs, c->n_sm, c->watch));
        CK(cudaEventRecord(c->ev_watch_done, c->watch));
        CK(cudaStreamWaitEvent(c->stream, c->ev_watch_done, 0));
    }
    CK(cudaStreamWaitEvent(c->stream, c->ship_done, 0));
    CK(after_host_copies(c));  // the execution phase above overlapped them
    CK(cudaGraphLaunch(c->g_sync[slot], c->stream));
    CK(cudaEventRecord(c->dlog_free[c->dlog_cur ^ 1], c->stream));
    if (c->exec_round) {
        rc = end_round(c, c->exec_round, c->cfg.conflict_policy == HETM_POLICY_CPU_LOSES ? 0 : -1);
        c->exec_round = 0;
        if (rc != HETM_OK) return rc;
    }
    CK(cudaEventRecord(ev[5], c->stream));
    c->slot_n_log[slot] = n;
    c->slot_nb[slot] = nb;
    ++c->r_open;
    if (!stats) return HETM_OK;
    return hetm_round_wait(c, stats);
}

int hetm_read_dirty(hetm_ctx *c, int32_t *host, uint64_t *n_chunks, uint64_t *n_bytes) {
    const Range range("hetm_read_dirty");
    if (!c || !host) return HETM_EINVAL;
    if (c->r_open) return HETM_EBUSY;  // a round in flight would change S under the copies
    CK(cudaSetDevice(c->device));
    CK(cudaStreamSynchronize(c->stream));
    uint64_t chunks = 0, bytes = 0;
    if (c->last_gpu_survived) {
        const uint64_t wpc = 1ull << c->cshift;
        const uint64_t n_chunk = (c->n_words + wpc - 1) / wpc;
        uint64_t ch = 0;
        while (ch < n_chunk) {
            if (!((c->ws_last[ch >> 5] >> (ch & 31)) & 1u)) {
                ++ch;
                continue;
            }
            uint64_t end = ch + 1;  // coalesce a run of dirty chunks into one copy
            while (end < n_chunk && ((c->ws_last[end >> 5] >> (end & 31)) & 1u)) ++end;
            const uint64_t w0 = ch * wpc, w1 = std::min<uint64_t>(end * wpc, c->n_words);
            CK(cudaMemcpyAsync(host + w0, c->S + w0, (w1 - w0) * 4, cudaMemcpyDeviceToHost, c->stream));
            chunks += end - ch;
            bytes += (w1 - w0) * 4;
            ch = end;
        }
        CK(cudaStreamSynchronize(c->stream));
    }
    if (n_chunks) *n_chunks = chunks;
    if (n_bytes) *n_bytes = bytes;
    return HETM_OK;
}

int hetm_read_dirty_async(hetm_ctx *c, int32_t *host, uint64_t *n_chunks, uint64_t *n_bytes) {
    const Range range("hetm_read_dirty_async");
    if (!c || !host) return HETM_EINVAL;
    if (c->r_open) return HETM_EBUSY;  // a round in flight would change S under the copies
    CK(cudaSetDevice(c->device));
    CK(cudaStreamSynchronize(c->stream));  // the dirty map and outcome of the last round
    uint64_t chunks = 0, bytes = 0;
    if (c->last_gpu_survived) {
        CK(cudaEventRecord(c->ev_d2h_from, c->stream));
        CK(cudaStreamWaitEvent(c->d2h, c->ev_d2h_from, 0));
        const uint64_t wpc = 1ull << c->cshift;
        const uint64_t n_chunk = (c->n_words + wpc - 1) / wpc;
        uint64_t ch = 0;
        while (ch < n_chunk) {
            if (!((c->ws_last[ch >> 5] >> (ch & 31)) & 1u)) {
                ++ch;
                continue;
            }
            uint64_t end = ch + 1;
            while (end < n_chunk && ((c->ws_last[end >> 5] >> (end & 31)) & 1u)) ++end;
            const uint64_t w0 = ch * wpc, w1 = std::min<uint64_t>(end * wpc, c->n_words);
            CK(cudaMemcpyAsync(host + w0, c->S + w0, (w1 - w0) * 4, cudaMemcpyDeviceToHost, c->d2h));
            chunks += end - ch;
            bytes += (w1 - w0) * 4;
            ch = end;
        }
        CK(cudaEventRecord(c->ev_d2h_done, c->d2h));
        c->d2h_pending = c->d2h_recorded = true;
    }
    if (n_chunks) *n_chunks = chunks;
    if (n_bytes) *n_bytes = bytes;
    return HETM_OK;
}

int hetm_read_dirty_wait(hetm_ctx *c) {
    if (!c) return HETM_EINVAL;
    CK(cudaSetDevice(c->device));
    if (c->d2h_recorded) CK(cudaEventSynchronize(c->ev_d2h_done));
    return HETM_OK;
}

int hetm_cpu_updates_allowed(hetm_ctx *c) { return c && !c->cpu_read_only.load() ? 1 : 0; }

int hetm_round_wait(hetm_ctx *c, hetm_round_stats *stats) {
    const Range range("hetm_round_wait");
    if (!c) return HETM_EINVAL;
    if (!c->r_open) {
        if (stats) std::memset(stats, 0, sizeof(*stats));
        return HETM_OK;
    }
    // the oldest round in flight
    const int slot = c->r_head;
    cudaEvent_t *ev = c->ev[slot];
    CK(cudaEventSynchronize(ev[5]));
    c->r_head = (c->r_head + 1) % hetm_ctx::kInFlight;
    --c->r_open;
    c->ws_last = c->ws_host + (size_t)slot * c->ws_words;
    const RoundOut *out = c->out + 1 + slot;
    const uint64_t n = c->slot_n_log[slot];
    const uint32_t nb = c->slot_nb[slot];
    hetm_round_stats local;
    if (!stats) stats = &local;
    std::memset(stats, 0, sizeof(*stats));
    stats->n_log = n;
    stats->n_conflicts = out->conflicts;
    stats->conflict = out->conflicts != 0;
    stats->err = err_code(out->err);
    stats->committed = out->counters[0] - c->prev_counters[0];
    stats->gave_up = out->counters[1] - c->prev_counters[1];
    stats->aborts = out->counters[2] - c->prev_counters[2];
    std::memcpy(c->prev_counters, out->counters, sizeof(c->prev_counters));
    stats->dirty_chunks = out->dirty;
    stats->n_batches = nb;
    stats->n_kernels = (nb ? c->n_kern[0] : 0) + c->n_kern[1] + (c->early && nb && n ? 1u : 0u);
    stats->stopped_early = c->early && nb && n ? out->stopped : 0u;
    const bool cpu_loses = c->cfg.conflict_policy == HETM_POLICY_CPU_LOSES;
    stats->outcome = !stats->conflict ? HETM_OUTCOME_CLEAN
                                      : (cpu_loses ? HETM_OUTCOME_CPU_DISCARDED : HETM_OUTCOME_GPU_ROLLED_BACK);
    // a timed-out execution phase was undone by the merge whatever validation found
    if (stats->err == HETM_ETIMEOUT) stats->outcome = HETM_OUTCOME_GPU_ROLLED_BACK;
    c->last_gpu_survived = stats->outcome != HETM_OUTCOME_GPU_ROLLED_BACK;
    // anti-starvation (Sec. IV-E): a read-only CPU phase ends with its round;
    // starve_limit consecutive GPU losses start one
    c->cpu_read_only.store(false);
    if (!cpu_loses && c->cfg.starve_limit && nb) {
        c->gpu_losses = stats->outcome == HETM_OUTCOME_GPU_ROLLED_BACK ? c->gpu_losses + 1 : 0;
        if (c->gpu_losses >= c->cfg.starve_limit) {
            c->gpu_losses = 0;
            c->cpu_read_only.store(true);
            stats->cpu_read_only_next = 1;
        }
    }
    float ms = 0;
    if (cudaEventElapsedTime(&ms, ev[0], ev[6]) == cudaSuccess) stats->ms_exec = ms;
    if (cudaEventElapsedTime(&ms, ev[1], ev[2]) == cudaSuccess) stats->ms_validate = ms;
    if (cudaEventElapsedTime(&ms, ev[2], ev[3]) == cudaSuccess) stats->ms_apply = ms;
    if (cudaEventElapsedTime(&ms, ev[3], ev[4]) == cudaSuccess) stats->ms_merge = ms;
    if (cudaEventElapsedTime(&ms, ev[0], ev[5]) == cudaSuccess) stats->ms_total = ms;
    return stats->err;
}

int hetm_batch_poll(hetm_ctx *c, uint64_t batch_id, hetm_batch_result *out) {
    if (!c || !out) return HETM_EINVAL;
    auto it = c->brec.find(batch_id);
    if (it == c->brec.end()) return HETM_EINVAL;
    hetm_ctx::BatchRec &b = it->second;
    std::memset(out, 0, sizeof(*out));
    out->n_tx = b.n_tx;
    out->round = b.round;
    if (!b.done && b.round) {
        const int slot = (int)(b.round % kRoundRing);
        if (c->rend_seq[slot] > b.round) {
            // a later round ended in this slot, so this one ended before it
            b.done = true;
            b.outcome = HETM_OUTCOME_UNKNOWN;
        } else if (c->rend_seq[slot] == b.round) {
            if (cudaSetDevice(c->device) != cudaSuccess) return HETM_ECUDA;
            const cudaError_t q = cudaEventQuery(c->rend[slot]);
            if (q == cudaSuccess) {
                const int f = c->rend_force[slot];
                const bool conflict = f >= 0 ? f != 0 : c->rconf[slot] != 0;
                const bool cpu_loses = c->cfg.conflict_policy == HETM_POLICY_CPU_LOSES;
                b.done = true;
                b.outcome = !conflict ? HETM_OUTCOME_CLEAN
                                      : (cpu_loses ? HETM_OUTCOME_CPU_DISCARDED : HETM_OUTCOME_GPU_ROLLED_BACK);
            } else if (q != cudaErrorNotReady) {
                return HETM_ECUDA;
            }
        }
        if (b.done)
            b.latency_ms = std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() -
                                                                     b.t_submit).count();
    }
    out->state = !b.round ? HETM_BATCH_QUEUED : (b.done ? HETM_BATCH_DONE : HETM_BATCH_RUNNING);
    out->outcome = b.done ? b.outcome : 0u;
    out->latency_ms = b.done ? b.latency_ms : 0.0;
    return HETM_OK;
}

}  // extern "C"

namespace hetm {
int ctx_open_rounds(const hetm_ctx *c) { return c->r_open; }
}  // namespace hetm

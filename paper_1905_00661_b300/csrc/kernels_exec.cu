// Speculative GPU transaction executor (execution phase, Sec. IV-C).
//
// One transaction per lane; a warp draws transactions in groups from a global
// counter over all admitted batches (uneven sizes, one persistent launch).
// Intra-GPU concurrency control is a word-based STM written for this
// library (the paper's guest GPU TM is PR-STM; any opaque TM may serve,
// Sec. IV-B):
//
//   * a table of 2^k striped 64-bit version locks, small enough to stay in
//     L2: unlocked = version << 1, locked = (owner << 1) | 1;
//   * transactions whose write-set is known up front (bank transfers, W1
//     updates, cache PUTs) lock it before reading (try-lock, abort on
//     failure, so no waiting and no deadlock), read under the locks, take a
//     commit version v from a global clock -- one atomicAdd per warp for
//     all its committing lanes -- write, and release the stripes at v;
//   * W1 read-only transactions run before this kernel, lock-free on the
//     launch-start state, in the ordered executor's read-only phase (commit
//     key 2 * v0 + 1: before every update of the launch; ExecArgs::skip_ro);
//     run here instead (skip_ro = 0), a read-only transaction reads (lock
//     versions, fence, values, fence, versions again) and commits when
//     nothing changed, with commit key 2 * (newest version seen) + 1, i.e.
//     right after the last writer it observed;
//   * a cache GET that hits writes its LRU stamp: it locks that stripe at
//     commit, takes v, then re-validates what it read (TL2 order);
//   * a W2 transaction (40 reads, Sec. V-A) reads against a snapshot rv of
//     the clock: it locks its 4 written words first (updates), checks that
//     every other word's stripe is unlocked with a version <= rv, fences,
//     reads the values, and after taking v checks the stripes again (TL2:
//     any writer that could have come between rv and v shows there).  An
//     update commits at 2v, a read-only transaction at 2 rv + 1.
//
// At commit a transaction ORs the granules of every word it read or wrote
// into RS_bmp and the chunks of every word it wrote into WS_bmp (Sec. IV-B,
// and writes into RS_bmp per Sec. IV-C).  Aborted attempts record nothing.
// Attempts are bounded (max_attempts) with randomized backoff; a
// transaction over the bound reports status 2 and has no effect.

#include "hetm_internal.cuh"

namespace hetm {
namespace {

constexpr uint64_t kNone = ~0ull;

struct Exec {
    const ExecArgs &a;
    __device__ __forceinline__ uint32_t stripe(uint64_t w) const {
        return ((uint32_t)(w >> a.lock_shift) * 2654435769u) & a.lock_mask;
    }
    __device__ __forceinline__ unsigned long long *lock(uint32_t s) const { return a.locks + s; }
    __device__ __forceinline__ void mark_read(uint64_t w0, uint32_t len) const {
        if (!a.instrument) return;
        for (uint64_t g = w0 >> a.gshift; g <= (w0 + len - 1) >> a.gshift; ++g)
            rs_mark(a.rs, a.filter, g);
    }
    __device__ __forceinline__ void mark_write(uint64_t w0, uint32_t len) const {
        if (!a.instrument) return;
        mark_read(w0, len);
        for (uint64_t c = w0 >> a.cshift; c <= (w0 + len - 1) >> a.cshift; ++c)
            atomicOr(a.ws + (c >> 5), 1u << (c & 31));
    }
};

__device__ __forceinline__ uint4 ld_vol16(const int32_t *p) {
    uint4 v;
    asm volatile("ld.volatile.global.v4.u32 {%0,%1,%2,%3}, [%4];"
                 : "=r"(v.x), "=r"(v.y), "=r"(v.z), "=r"(v.w)
                 : "l"(p)
                 : "memory");
    return v;
}

// Try to lock n stripes (duplicates allowed; only first occurrences are
// locked).  cur[] receives the versions the locks held.  Returns true with
// every stripe held, or false with none held.
template <int N>
__device__ __forceinline__ bool try_lock(const Exec &x, const uint32_t (&st)[N], int n,
                                         unsigned long long (&cur)[N], unsigned &own,
                                         unsigned long long mine) {
    own = 0;
#pragma unroll
    for (int k = 0; k < N; ++k) {
        if (k >= n) break;
        bool first = true;
#pragma unroll
        for (int j = 0; j < k; ++j) first &= st[j] != st[k];
        if (first) own |= 1u << k;
    }
#pragma unroll
    for (int k = 0; k < N; ++k)
        if (own & (1u << k)) cur[k] = ld_rlx64(x.lock(st[k]));
    bool ok = true;
#pragma unroll
    for (int k = 0; k < N; ++k)
        if (own & (1u << k)) ok &= !(cur[k] & 1ull);
    if (!ok) return false;
    unsigned got = 0;
#pragma unroll
    for (int k = 0; k < N; ++k)
        if (own & (1u << k))
            if (atomicCAS(x.lock(st[k]), cur[k], mine) == cur[k]) got |= 1u << k;
    if (got == own) {
        fence_gpu();  // acquire: reads below see the previous holders' writes
        return true;
    }
#pragma unroll
    for (int k = 0; k < N; ++k)
        if (got & (1u << k)) st_rlx64(x.lock(st[k]), cur[k]);
    return false;
}

template <int N>
__device__ __forceinline__ void release(const Exec &x, const uint32_t (&st)[N], unsigned own,
                                        unsigned long long word) {
    fence_gpu();  // release: the writes above are visible before the unlock
#pragma unroll
    for (int k = 0; k < N; ++k)
        if (own & (1u << k)) st_rlx64(x.lock(st[k]), word);
}

// W2: a word's stripe is usable when this lane holds it or when it is
// unlocked at a version no newer than the snapshot rv.
__device__ __forceinline__ bool w2_stripe_ok(const Exec &x, uint64_t w, unsigned long long rv,
                                             unsigned long long mine) {
    const unsigned long long l = ld_rlx64(x.lock(x.stripe(w)));
    return l == mine || (!(l & 1ull) && (l >> 1) <= rv);
}

// Stripes of words j0..39 of a W2 transaction (all usable: true).
__device__ __forceinline__ bool w2_check(const Exec &x, const hetm_w2_tx *t, int j0,
                                         unsigned long long rv, unsigned long long mine) {
    bool ok = true;
#pragma unroll 4
    for (int j = j0; j < 40; ++j) ok &= w2_stripe_ok(x, __ldg(&t->addr[j]), rv, mine);
    return ok;
}

// 32-bit wrapping sum of words j0..39 (after w2_check and a fence).
__device__ __forceinline__ int32_t w2_sum(const Exec &x, const hetm_w2_tx *t, int j0) {
    int32_t s = 0;
#pragma unroll 4
    for (int j = j0; j < 40; ++j) s += ld_rlx32(x.a.W + __ldg(&t->addr[j]));
    return s;
}

__device__ __forceinline__ int binsearch(const uint64_t *prefix, uint32_t n, uint64_t gi) {
    uint32_t lo = 0, hi = n;  // prefix[lo] <= gi < prefix[hi]
    while (hi - lo > 1) {
        uint32_t mid = (lo + hi) >> 1;
        if (__ldg(prefix + mid) <= gi) lo = mid; else hi = mid;
    }
    return (int)lo;
}

__global__ void __launch_bounds__(256) k_exec(ExecArgs a) {
    const Exec x{a};
    const uint32_t n_batches = a.rp->n_batches;
    const uint64_t total = a.rp->total_tx;
    // after the read-only phase: draw only the indices it left (when listed)
    const bool listed = a.skip_ro && a.rest && total <= a.rest_cap;
    const uint64_t n_draw = listed ? *a.rest_n : total;
    const unsigned lane = threadIdx.x & 31u;
    const unsigned long long mine =
        ((unsigned long long)(blockIdx.x * blockDim.x + threadIdx.x + 1) << 1) | 1ull;

    uint64_t gi = kNone;
    bool done = false;
    uint32_t attempts = 0, sit = 0;
    // the lane's transaction
    uint32_t wl = 0, li = 0, txid = 0, na = 0;
    uint32_t addr[4] = {0, 0, 0, 0};
    bool upd = false;
    int32_t amt = 0;
    uint64_t ckey = 0, cval = 0;
    uint32_t cop = 0;
    const hetm_w2_tx *w2 = nullptr;  // W2: the record (its 40 words are re-read from it)
    uint64_t *o_order = nullptr;
    uint8_t *o_status = nullptr;
    void *o_out = nullptr;
    unsigned long long n_commit = 0, n_gaveup = 0, n_abort = 0;
    // lane 0's clock decides for the whole warp, so the warp leaves together
    const unsigned long long t0 = __shfl_sync(kFull, globaltimer_ns(), 0);
    uint32_t iter = 0;
    bool expired = false;  // past the budget: draw what is left only to report it

    for (;;) {
        // wall-clock bound: past it, every unfinished transaction gives up
        if (!expired && (++iter & 63u) == 0 &&
            __shfl_sync(kFull, globaltimer_ns(), 0) - t0 > a.budget_ns) {
            expired = true;
            if (gi != kNone) {
                if (o_status) o_status[li] = kGaveUp;
                ++n_gaveup;
                gi = kNone;
            }
            if (lane == 0) set_err(a.err, kErrTimeout);
        }
        // ---------------------------------------------------- draw new work
        const bool need = gi == kNone && !done;
        const unsigned nm = __ballot_sync(kFull, need);
        if (nm) {
            const int leader = __ffs(nm) - 1;
            unsigned long long base = 0;
            if ((int)lane == leader) base = atomicAdd(a.next, (unsigned long long)__popc(nm));
            base = __shfl_sync(kFull, base, leader);
            if (need) {
                const uint64_t my = base + __popc(nm & lanemask_lt());
                if (my < n_draw) {
                    gi = listed ? a.rest[my] : my;
                    attempts = 0;
                    sit = 0;
                    const int b = binsearch(a.prefix, n_batches, gi);
                    const DevBatch &d = a.batches[b];
                    wl = d.workload;
                    li = (uint32_t)(gi - a.prefix[b]);
                    o_order = d.order;
                    o_status = d.status;
                    o_out = d.out;
                    bool bad = false;
                    if (wl == HETM_WL_BANK) {
                        const hetm_bank_tx t = static_cast<const hetm_bank_tx *>(d.tx)[li];
                        addr[0] = d.word_base + t.src;
                        addr[1] = d.word_base + t.dst;
                        amt = t.amount;
                        na = 2;
                        upd = true;
                        bad = addr[0] >= a.n_words || addr[1] >= a.n_words;
                    } else if (wl == HETM_WL_RMW) {
                        const hetm_rmw_tx *t = static_cast<const hetm_rmw_tx *>(d.tx) + li;
#pragma unroll
                        for (int k = 0; k < 4; ++k) {
                            addr[k] = t->addr[k];
                            bad |= addr[k] >= a.n_words;
                        }
                        upd = t->flags & 1u;
                        txid = d.txid_base + li;
                        na = 4;
                    } else if (wl == HETM_WL_CACHE) {
                        const hetm_cache_req *r = static_cast<const hetm_cache_req *>(d.tx) + li;
                        ckey = r->key;
                        cval = r->value;
                        cop = r->op;
                        na = 0;
                    } else if (wl == HETM_WL_W2) {
                        w2 = static_cast<const hetm_w2_tx *>(d.tx) + li;
                        for (int k = 0; k < 40; ++k) {
                            const uint32_t ad = w2->addr[k];
                            if (k < 4) addr[k] = ad;
                            bad |= ad >= a.n_words;
                        }
                        upd = w2->flags & 1u;
                        txid = d.txid_base + li;
                        na = 4;
                    } else {
                        bad = true;
                    }
                    if (bad) {
                        set_err(a.err, kErrAddr);
                        if (o_status) o_status[li] = kGaveUp;
                        ++n_gaveup;
                        gi = kNone;  // drawn again next iteration
                    } else if (a.skip_ro && (wl == HETM_WL_RMW || wl == HETM_WL_W2) && !upd) {
                        gi = kNone;  // ran in the read-only phase
                    } else if (expired) {
                        if (o_status) o_status[li] = kGaveUp;
                        ++n_gaveup;
                        gi = kNone;
                    }
                } else {
                    done = true;
                }
            }
        }
        if (__all_sync(kFull, gi == kNone && done)) break;
        const bool busy = gi != kNone;
        const bool active = busy && sit == 0;
        if (busy && sit > 0) --sit;
        if (!__any_sync(kFull, active)) {
            __nanosleep(64);
            continue;
        }

        // ------------------------------------------ phase 1: lock and read
        bool want_v = false, ro_ok = false, fail = false;
        uint32_t st[4] = {0, 0, 0, 0};
        unsigned long long cur[4] = {0, 0, 0, 0};
        unsigned own = 0;
        int32_t val[4] = {0, 0, 0, 0};
        unsigned long long ro_key = 0;
        // cache state
        uint32_t set = 0, way = 0;
        int hit = -1;
        uint64_t found = 0;
        unsigned long long ck = 0, cv = 0, cl = 0;
        uint32_t kst = 0, vst = 0, lst = 0;
        bool evict = false;
        int32_t ver_old = 0;

        unsigned long long rv = 0;  // W2: clock snapshot
        if (active && wl == HETM_WL_W2) {
            rv = ld_rlx64(a.gv);
            fence_gpu();
#pragma unroll
            for (int k = 0; k < 4; ++k) st[k] = x.stripe(addr[k]);
            bool ok = true, locked = false;
            if (upd) ok = locked = try_lock<4>(x, st, 4, cur, own, mine);
            // updates hold their 4 words; the rest (all 40 for a read-only
            // transaction) must be unlocked at a version <= rv
            if (ok) ok = w2_check(x, w2, upd ? 4 : 0, rv, mine);
            if (ok) {
                fence_gpu();
                if (upd) {
#pragma unroll
                    for (int k = 0; k < 4; ++k) val[k] = ld_rlx32(a.W + addr[k]);
                    val[0] += w2_sum(x, w2, 4);  // val[0..3] summed at commit
                    want_v = true;
                } else {
                    val[0] = w2_sum(x, w2, 0);
                    fence_gpu();
                    ro_ok = w2_check(x, w2, 0, rv, mine);
                    fail = !ro_ok;
                    ro_key = 2 * rv + 1;
                }
            } else {
                // nothing written: give the stripes back at their versions
#pragma unroll
                for (int k = 0; k < 4; ++k)
                    if (locked && (own & (1u << k))) st_rlx64(x.lock(st[k]), cur[k]);
                fail = true;
            }
        } else if (active && wl != HETM_WL_CACHE) {
#pragma unroll
            for (int k = 0; k < 4; ++k) st[k] = x.stripe(addr[k]);
            if (upd) {
                if (try_lock<4>(x, st, (int)na, cur, own, mine)) {
#pragma unroll
                    for (int k = 0; k < 4; ++k)
                        if (k < (int)na) val[k] = ld_rlx32(a.W + addr[k]);
                    want_v = true;
                } else {
                    fail = true;
                }
            } else {
#pragma unroll
                for (int k = 0; k < 4; ++k) cur[k] = ld_rlx64(x.lock(st[k]));
                fence_gpu();
#pragma unroll
                for (int k = 0; k < 4; ++k) val[k] = ld_rlx32(a.W + addr[k]);
                fence_gpu();
                bool ok = true;
                unsigned long long mx = 0;
#pragma unroll
                for (int k = 0; k < 4; ++k) {
                    const unsigned long long again = ld_rlx64(x.lock(st[k]));
                    ok &= !(cur[k] & 1ull) && again == cur[k];
                    mx = cur[k] > mx ? cur[k] : mx;
                }
                ro_ok = ok;
                fail = !ok;
                ro_key = mx | 1ull;
            }
        } else if (active) {  // object cache
            set = (uint32_t)(splitmix_fin(ckey) & ((1ull << a.cache_log2_sets) - 1));
            const uint64_t kw = a.key_base + 16ull * set;
            kst = x.stripe(kw);
            if (cop == 0) {
                // GET: optimistic read of the set's keys
                ck = ld_rlx64(x.lock(kst));
                fence_gpu();
                uint64_t keys[8];
#pragma unroll
                for (int q = 0; q < 4; ++q) {
                    const uint4 v = ld_vol16(a.W + kw + 4 * q);
                    keys[2 * q] = ((uint64_t)v.y << 32) | v.x;
                    keys[2 * q + 1] = ((uint64_t)v.w << 32) | v.z;
                }
#pragma unroll
                for (int w = 7; w >= 0; --w)
                    if (keys[w] == ckey) hit = w;
                if (ck & 1ull) {
                    fail = true;
                } else if (hit < 0) {
                    fence_gpu();
                    ro_ok = ld_rlx64(x.lock(kst)) == ck;
                    fail = !ro_ok;
                    ro_key = ck | 1ull;
                } else {
                    const uint64_t vw = a.val_base + 2ull * (8ull * set + hit);
                    const uint64_t lw = a.lru_base + 8ull * set + hit;
                    vst = x.stripe(vw);
                    lst = x.stripe(lw);
                    cv = ld_rlx64(x.lock(vst));
                    cl = ld_rlx64(x.lock(lst));
                    fence_gpu();
                    found = ld_rlx_u64(a.W + vw);
                    if ((cv & 1ull) || (cl & 1ull) ||
                        atomicCAS(x.lock(lst), cl, mine) != cl) {
                        fail = true;
                    } else {
                        fence_gpu();
                        want_v = true;
                    }
                }
            } else {
                // PUT: lock keys, values, LRU stamps and version of the set up front
                const uint32_t pst[4] = {kst, x.stripe(a.val_base + 16ull * set),
                                         x.stripe(a.lru_base + 8ull * set),
                                         x.stripe(a.ver_base + set)};
#pragma unroll
                for (int k = 0; k < 4; ++k) st[k] = pst[k];
                if (try_lock<4>(x, st, 4, cur, own, mine)) {
                    uint64_t keys[8];
#pragma unroll
                    for (int q = 0; q < 4; ++q) {
                        const uint4 v = ld_vol16(a.W + kw + 4 * q);
                        keys[2 * q] = ((uint64_t)v.y << 32) | v.x;
                        keys[2 * q + 1] = ((uint64_t)v.w << 32) | v.z;
                    }
                    int empty = -1;
#pragma unroll
                    for (int w = 7; w >= 0; --w) {
                        if (keys[w] == ckey) hit = w;
                        if (keys[w] == 0) empty = w;
                    }
                    ver_old = ld_rlx32(a.W + a.ver_base + set);
                    if (hit >= 0) {
                        way = (uint32_t)hit;
                    } else if (empty >= 0) {
                        way = (uint32_t)empty;
                    } else {
                        evict = true;
                        uint32_t best = 0;
                        const uint4 l0 = ld_vol16(a.W + a.lru_base + 8ull * set);
                        const uint4 l1 = ld_vol16(a.W + a.lru_base + 8ull * set + 4);
                        const uint32_t l[8] = {l0.x, l0.y, l0.z, l0.w, l1.x, l1.y, l1.z, l1.w};
                        way = 0;
                        best = l[0];
#pragma unroll
                        for (int w = 1; w < 8; ++w)
                            if (l[w] < best) {
                                best = l[w];
                                way = (uint32_t)w;
                            }
                    }
                    want_v = true;
                } else {
                    fail = true;
                }
            }
        }

        // ------------------------------- commit versions, one atomic per warp
        const unsigned vm = __ballot_sync(kFull, want_v);
        unsigned long long v = 0;
        if (vm) {
            const int leader = __ffs(vm) - 1;
            unsigned long long base = 0;
            if ((int)lane == leader) base = atomicAdd(a.gv, (unsigned long long)__popc(vm));
            base = __shfl_sync(kFull, base, leader);
            v = base + 1 + __popc(vm & lanemask_lt());
        }

        // ------------------------------- phase 2: validate, write, release
        bool committed = false;
        if (want_v && wl == HETM_WL_W2) {
            // TL2 commit: a writer of a read word that came after rv shows
            // in its stripe now (locked, or a version > rv)
            fence_gpu();
            if (w2_check(x, w2, 4, rv, mine)) {
                const int32_t s = val[0] + val[1] + val[2] + val[3];
#pragma unroll
                for (int k = 0; k < 4; ++k) st_rlx32(a.W + addr[k], s + k + (int32_t)txid);
                release<4>(x, st, own, v << 1);
                if (o_order) o_order[li] = v << 1;
                if (o_out) static_cast<int32_t *>(o_out)[li] = s;
                for (int j = 4; j < 40; ++j) x.mark_read(__ldg(&w2->addr[j]), 1);
#pragma unroll
                for (int k = 0; k < 4; ++k) x.mark_write(addr[k], 1);
                committed = true;
            } else {
#pragma unroll
                for (int k = 0; k < 4; ++k)
                    if (own & (1u << k)) st_rlx64(x.lock(st[k]), cur[k]);
                fail = true;
            }
        } else if (ro_ok && wl == HETM_WL_W2) {
            if (o_order) o_order[li] = ro_key;
            if (o_out) static_cast<int32_t *>(o_out)[li] = val[0];
            for (int j = 0; j < 40; ++j) x.mark_read(__ldg(&w2->addr[j]), 1);
            committed = true;
        } else if (want_v && wl != HETM_WL_CACHE) {
            int32_t nv[4];
            int32_t s = 0;
            if (wl == HETM_WL_RMW) {
#pragma unroll
                for (int k = 0; k < 4; ++k) s += val[k];
#pragma unroll
                for (int k = 0; k < 4; ++k) nv[k] = s + k + (int32_t)txid;
            } else {  // bank: src -= amt, then dst += amt (dst may equal src)
                nv[0] = val[0] - amt;
                nv[1] = (addr[1] == addr[0] ? nv[0] : val[1]) + amt;
            }
#pragma unroll
            for (int k = 0; k < 4; ++k)
                if (k < (int)na) st_rlx32(a.W + addr[k], nv[k]);
            release<4>(x, st, own, v << 1);
            if (o_order) o_order[li] = v << 1;
            if (o_out && wl == HETM_WL_RMW) static_cast<int32_t *>(o_out)[li] = s;
#pragma unroll
            for (int k = 0; k < 4; ++k)
                if (k < (int)na) x.mark_write(addr[k], 1);
            committed = true;
        } else if (ro_ok && wl != HETM_WL_CACHE && wl != HETM_WL_W2) {
            int32_t s = 0;
#pragma unroll
            for (int k = 0; k < 4; ++k) s += val[k];
            if (o_order) o_order[li] = ro_key;
            if (o_out) static_cast<int32_t *>(o_out)[li] = s;
#pragma unroll
            for (int k = 0; k < 4; ++k) x.mark_read(addr[k], 1);
            committed = true;
        } else if (wl == HETM_WL_CACHE && (want_v || ro_ok)) {
            const uint64_t kw = a.key_base + 16ull * set;
            if (cop == 0 && ro_ok) {  // GET miss
                if (o_order) o_order[li] = ro_key;
                if (o_out) static_cast<uint64_t *>(o_out)[li] = ~0ull;
                x.mark_read(kw, 16);
                committed = true;
            } else if (cop == 0) {  // GET hit: validate the reads after taking v
                const bool ok_k = kst == lst ? cl == ck : ld_rlx64(x.lock(kst)) == ck;
                const bool ok_v = vst == lst ? cl == cv : ld_rlx64(x.lock(vst)) == cv;
                if (ok_k && ok_v && ck == (ck & ~1ull)) {
                    const uint64_t lw = a.lru_base + 8ull * set + hit;
                    st_rlx32(a.W + lw, (int32_t)(uint32_t)v);
                    fence_gpu();
                    st_rlx64(x.lock(lst), v << 1);
                    if (o_order) o_order[li] = v << 1;
                    if (o_out) static_cast<uint64_t *>(o_out)[li] = found;
                    x.mark_read(kw, 16);
                    x.mark_read(a.val_base + 2ull * (8ull * set + hit), 2);
                    x.mark_write(lw, 1);
                    committed = true;
                } else {
                    st_rlx64(x.lock(lst), cl);  // nothing written: restore
                    fail = true;
                }
            } else {  // PUT under the set's locks
                const uint64_t slot = 8ull * set + way;
                if (hit < 0) st_rlx_u64w(a.W + a.key_base + 2 * slot, ckey);
                st_rlx_u64w(a.W + a.val_base + 2 * slot, cval);
                st_rlx32(a.W + a.lru_base + slot, (int32_t)(uint32_t)v);
                st_rlx32(a.W + a.ver_base + set, ver_old + 1);
                release<4>(x, st, own, v << 1);
                if (o_order) o_order[li] = v << 1;
                if (o_out) static_cast<uint64_t *>(o_out)[li] = way;
                x.mark_read(kw, 16);
                x.mark_write(a.ver_base + set, 1);
                if (evict) x.mark_read(a.lru_base + 8ull * set, 8);
                if (hit < 0) x.mark_write(a.key_base + 2 * slot, 2);
                x.mark_write(a.val_base + 2 * slot, 2);
                x.mark_write(a.lru_base + slot, 1);
                committed = true;
            }
        }

        if (committed) {
            if (o_status) o_status[li] = kCommitted;
            ++n_commit;
            gi = kNone;
        } else if (fail) {
            ++n_abort;
            if (++attempts >= a.max_attempts) {
                if (o_status) o_status[li] = kGaveUp;
                ++n_gaveup;
                gi = kNone;
            } else {
                const uint32_t h = (uint32_t)gi * 0x9E3779B1u + attempts * 0x85EBCA6Bu + lane;
                const uint32_t span = attempts < 6 ? (1u << attempts) : 64u;
                sit = (h >> 16) & (span - 1);
            }
        }
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        n_commit += __shfl_xor_sync(kFull, n_commit, o);
        n_gaveup += __shfl_xor_sync(kFull, n_gaveup, o);
        n_abort += __shfl_xor_sync(kFull, n_abort, o);
    }
    if (lane == 0) {
        if (n_commit) atomicAdd(a.counters + 0, n_commit);
        if (n_gaveup) atomicAdd(a.counters + 1, n_gaveup);
        if (n_abort) atomicAdd(a.counters + 2, n_abort);
    }
}

}  // namespace

cudaError_t launch_exec(const ExecArgs &a, int blocks, int threads, cudaStream_t s) {
    k_exec<<<blocks, threads, 0, s>>>(a);
    return cudaGetLastError();
}

int exec_occupancy(int threads, int *blocks_per_sm) {
    return (int)cudaOccupancyMaxActiveBlocksPerMultiprocessor(blocks_per_sm, k_exec, threads, 0);
}

}  // namespace hetm

// Ordered execution of a batch (execution phase, Sec. IV-C), the default
// GPU guest TM of this library.
//
// The paper lets any TM that keeps committed transactions serializable and
// every running transaction consistent drive the GPU side (Sec. IV-B); here
// the serial order is fixed up front instead of discovered by aborts:
//
//   1. read-only W1 transactions of the launch come first in the order: they
//      all observe the launch-start state, take no locks and never wait;
//   2. every other transaction (W1 updates, bank transfers, cache requests)
//      follows in launch index order.  Each names its resources up front
//      (its words; a cache request its set).  A stable radix sort of the
//      (resource, index) pairs gives, for every access, its position among
//      the accesses to that resource; a transaction runs when every resource
//      has reached its position, so each one executes atomically at its
//      place in the order and nothing ever aborts or rolls back.
//   3. for word resources the last writer hands the next one the word's
//      value inside a packed (count, value) word, so one 8-byte store
//      publishes both the turn and the data; cache sets use reader/writer
//      turns (GETs of one set run concurrently, PUTs alone).
//
// Commit keys: 2*V0 + 1 for the read-only phase (V0 = commit clock before the
// launch), 2*(V0 + 1 + u) for transaction u of the ordered phase; the clock
// then advances by the launch size.  RS_bmp / WS_bmp are recorded at commit
// exactly as in the optimistic executor.
//
// Every wait is a poll inside the warp's iteration, bounded by a wall-clock
// budget; transactions are handed out in index order to resident warps, so
// the lowest unfinished transaction can always run.

#include <algorithm>
#include <type_traits>

#include "hetm_internal.cuh"

namespace hetm {
namespace {

// ----------------------------------------------------------------------------
// block-wide inclusive scan of one 64-bit value per thread (256 threads)
// ----------------------------------------------------------------------------
struct SumOp {
    __device__ __forceinline__ uint64_t operator()(uint64_t a, uint64_t b) const { return a + b; }
};
struct PairMaxOp {  // independent max of the high and low 32-bit halves
    __device__ __forceinline__ uint64_t operator()(uint64_t a, uint64_t b) const {
        const uint32_t hi = max((uint32_t)(a >> 32), (uint32_t)(b >> 32));
        const uint32_t lo = max((uint32_t)a, (uint32_t)b);
        return ((uint64_t)hi << 32) | lo;
    }
};

constexpr int kScanThreads = 256;
constexpr int kScanItems = 4;                        // per thread
constexpr int kScanTile = kScanThreads * kScanItems; // 1024 items per block

template <class Op>
__device__ __forceinline__ uint64_t block_scan_incl(uint64_t v, Op op, uint64_t *s_warp) {
    const unsigned lane = threadIdx.x & 31u, warp = threadIdx.x >> 5;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const uint64_t t = __shfl_up_sync(kFull, v, o);
        if ((int)lane >= o) v = op(t, v);
    }
    if (lane == 31) s_warp[warp] = v;
    __syncthreads();
    if (warp == 0) {
        uint64_t w = lane < kScanThreads / 32 ? s_warp[lane] : 0;
#pragma unroll
        for (int o = 1; o < kScanThreads / 32; o <<= 1) {
            const uint64_t t = __shfl_up_sync(kFull, w, o);
            if ((int)lane >= o) w = op(t, w);
        }
        if (lane < kScanThreads / 32) s_warp[lane] = w;
    }
    __syncthreads();
    if (warp > 0) v = op(s_warp[warp - 1], v);
    __syncthreads();
    return v;
}

// Tile-local inclusive scan of in[0..n) (n read from *n_dev); tile totals
// to tot[block].  For kExclusive the written value is the exclusive prefix.
template <class Op, bool kExclusive>
__global__ void __launch_bounds__(kScanThreads) k_scan_tiles(const uint64_t *in, uint64_t *out,
                                                             const uint32_t *n_dev, uint32_t n_fix,
                                                             uint64_t *tot, uint64_t identity) {
    __shared__ uint64_t s_warp[kScanThreads / 32];
    const uint32_t n = n_dev ? *n_dev : n_fix;
    const uint32_t nt = (n + kScanTile - 1) / kScanTile;
    Op op;
    // a grid of the machine's size walks the tiles the count fills
    for (uint32_t tile = blockIdx.x; tile < nt; tile += gridDim.x) {
        const uint64_t base = (uint64_t)tile * kScanTile;
        uint64_t x[kScanItems];
        uint64_t run = identity;
#pragma unroll
        for (int k = 0; k < kScanItems; ++k) {
            const uint64_t i = base + threadIdx.x * kScanItems + k;
            x[k] = i < n ? in[i] : identity;
            run = op(run, x[k]);
        }
        const uint64_t incl = block_scan_incl(run, op, s_warp);
        uint64_t pre = __shfl_up_sync(kFull, incl, 1);
        // exclusive prefix of this thread's items inside the tile
        {
            const unsigned lane = threadIdx.x & 31u, warp = threadIdx.x >> 5;
            if (lane == 0) pre = warp == 0 ? identity : s_warp[warp - 1];
            // s_warp was overwritten by the scan with inclusive warp totals
        }
        uint64_t acc = pre;
#pragma unroll
        for (int k = 0; k < kScanItems; ++k) {
            const uint64_t i = base + threadIdx.x * kScanItems + k;
            const uint64_t nxt = op(acc, x[k]);
            if (i < n) out[i] = kExclusive ? acc : nxt;
            acc = nxt;
        }
        if (threadIdx.x == kScanThreads - 1) tot[tile] = incl;
        __syncthreads();  // s_warp is refilled by the next tile's scan
    }
}

// Exclusive scan of the tile totals in place (one block, any count).
template <class Op>
__global__ void __launch_bounds__(kScanThreads) k_scan_totals(uint64_t *tot, const uint32_t *n_dev,
                                                              uint32_t n_fix, uint64_t identity) {
    __shared__ uint64_t s_warp[kScanThreads / 32];
    __shared__ uint64_t s_carry;
    const uint32_t n = n_dev ? *n_dev : n_fix;
    const uint32_t nt = (n + kScanTile - 1) / kScanTile;
    Op op;
    if (threadIdx.x == 0) s_carry = identity;
    __syncthreads();
    for (uint32_t b0 = 0; b0 < nt; b0 += kScanThreads) {
        const uint32_t b = b0 + threadIdx.x;
        const uint64_t v = b < nt ? tot[b] : identity;
        const uint64_t incl = block_scan_incl(v, op, s_warp);
        const uint64_t carry = s_carry;
        uint64_t ex = __shfl_up_sync(kFull, incl, 1);
        const unsigned lane = threadIdx.x & 31u, warp = threadIdx.x >> 5;
        if (lane == 0) ex = warp == 0 ? identity : s_warp[warp - 1];
        __syncthreads();
        if (b < nt) tot[b] = op(carry, ex);
        if (threadIdx.x == kScanThreads - 1) s_carry = op(carry, incl);
        __syncthreads();
    }
}

// out[i] = op(tot[tile], out[i]) for every item.
template <class Op>
__global__ void __launch_bounds__(kScanThreads) k_scan_fix(uint64_t *out, const uint32_t *n_dev,
                                                           uint32_t n_fix, const uint64_t *tot) {
    const uint32_t n = n_dev ? *n_dev : n_fix;
    const uint32_t nt = (n + kScanTile - 1) / kScanTile;
    Op op;
    for (uint32_t tile = blockIdx.x; tile < nt; tile += gridDim.x) {
        const uint64_t base = (uint64_t)tile * kScanTile;
        const uint64_t c = tot[tile];
#pragma unroll
        for (int k = 0; k < kScanItems; ++k) {
            const uint64_t i = base + k * kScanThreads + threadIdx.x;
            if (i < n) out[i] = op(c, out[i]);
        }
    }
}

}  // namespace

// Device-wide scan of n (device or fixed) 64-bit values; `grid` blocks walk
// the tiles of kScanTile (any grid works); tot holds one value per tile of
// the capacity.
template <class Op, bool kExclusive>
static cudaError_t device_scan(const uint64_t *in, uint64_t *out, const uint32_t *n_dev,
                               uint32_t n_fix, uint32_t grid, uint64_t *tot, uint64_t identity,
                               cudaStream_t s) {
    k_scan_tiles<Op, kExclusive><<<grid, kScanThreads, 0, s>>>(in, out, n_dev, n_fix, tot, identity);
    k_scan_totals<Op><<<1, kScanThreads, 0, s>>>(tot, n_dev, n_fix, identity);
    k_scan_fix<Op><<<grid, kScanThreads, 0, s>>>(out, n_dev, n_fix, tot);
    return cudaGetLastError();
}

namespace {

// ----------------------------------------------------------------------------
// stable LSD radix sort of (key, value) u32 pairs, 8-bit digits
// ----------------------------------------------------------------------------
constexpr int kSortThreads = 256;
constexpr int kSortItems = 8;
constexpr int kSortTile = kSortThreads * kSortItems;  // 2048

// hist[d * n_tiles + tile] = count of digit d in the tile, n_tiles = the
// tiles the n (device) keys fill, so that the scan after it covers those
// and not the capacity; *hist_n = 256 * n_tiles, the scan's count.
__global__ void __launch_bounds__(kSortThreads) k_radix_hist(const uint32_t *keys, const uint32_t *n_dev,
                                                             uint32_t shift, uint64_t *hist,
                                                             uint32_t *hist_n) {
    __shared__ uint32_t s_cnt[256];
    const uint32_t n = *n_dev;
    const uint32_t n_tiles = (n + kSortTile - 1) / kSortTile;
    if (blockIdx.x == 0 && threadIdx.x == 0) *hist_n = 256u * n_tiles;
    for (uint32_t tile = blockIdx.x; tile < n_tiles; tile += gridDim.x) {
        const uint64_t base = (uint64_t)tile * kSortTile;
        s_cnt[threadIdx.x] = 0;
        __syncthreads();
#pragma unroll
        for (int k = 0; k < kSortItems; ++k) {
            const uint64_t i = base + k * kSortThreads + threadIdx.x;
            if (i < n) atomicAdd(&s_cnt[(keys[i] >> shift) & 255u], 1u);
        }
        __syncthreads();
        hist[(uint64_t)threadIdx.x * n_tiles + tile] = s_cnt[threadIdx.x];
        __syncthreads();  // s_cnt is cleared for the next tile
    }
}

// Stable scatter: items keep their input order within a digit.
__global__ void __launch_bounds__(kSortThreads) k_radix_scatter(const uint32_t *kin, const uint32_t *vin,
                                                                uint32_t *kout, uint32_t *vout,
                                                                const uint32_t *n_dev, uint32_t shift,
                                                                const uint64_t *hist_ex) {
    __shared__ uint32_t s_base[256];                      // running output position per digit
    __shared__ uint32_t s_wcnt[kSortThreads / 32][256];   // per-warp digit counts of a round
    const uint32_t n = *n_dev;
    const uint32_t n_tiles = (n + kSortTile - 1) / kSortTile;
    const unsigned lane = threadIdx.x & 31u, warp = threadIdx.x >> 5;
    for (uint32_t tile = blockIdx.x; tile < n_tiles; tile += gridDim.x) {
        const uint64_t base = (uint64_t)tile * kSortTile;
        s_base[threadIdx.x] = (uint32_t)hist_ex[(uint64_t)threadIdx.x * n_tiles + tile];
        for (int r = 0; r < kSortItems; ++r) {
            for (int w = 0; w < kSortThreads / 32; ++w) s_wcnt[w][threadIdx.x] = 0;
            __syncthreads();
            const uint64_t i = base + (uint64_t)r * kSortThreads + threadIdx.x;
            const bool ok = i < n;
            const uint32_t key = ok ? kin[i] : 0u;
            const uint32_t val = ok ? vin[i] : 0u;
            const uint32_t d = ok ? (key >> shift) & 255u : 256u + lane;  // padding: unique
            const unsigned peers = __match_any_sync(kFull, d);
            const uint32_t rank = __popc(peers & lanemask_lt());
            if (ok && rank == 0) s_wcnt[warp][d] = __popc(peers);
            __syncthreads();
            // digit-wise exclusive prefix over the warps of this round
            uint32_t run = 0;
            {
                const uint32_t dd = threadIdx.x;
                for (int w = 0; w < kSortThreads / 32; ++w) {
                    const uint32_t c = s_wcnt[w][dd];
                    s_wcnt[w][dd] = run;
                    run += c;
                }
            }
            __syncthreads();
            if (ok) {
                const uint32_t pos = s_base[d] + s_wcnt[warp][d] + rank;
                if (pos < n) {  // always true for a consistent histogram
                    kout[pos] = key;
                    vout[pos] = val;
                }
            }
            __syncthreads();
            s_base[threadIdx.x] += run;
            __syncthreads();
        }
    }
}

}  // namespace

// Sort n (device) pairs by key, `bits` significant key bits, in place in
// (k0, v0) using (k1, v1) as the other buffer.  hist holds 256 *
// n_tiles_cap values; tot one value per scan tile of it; hist_n one device
// word (the histogram's length for the n at hand).
static cudaError_t radix_sort(uint32_t *k0, uint32_t *v0, uint32_t *k1, uint32_t *v1,
                              const uint32_t *n_dev, uint32_t cap, uint32_t bits, uint64_t *hist,
                              uint64_t *tot, uint32_t *hist_n, uint32_t max_blocks, cudaStream_t s) {
    const uint32_t n_tiles_cap = (cap + kSortTile - 1) / kSortTile;
    // grids of the machine's size that walk the tiles the keys fill
    const uint32_t grid = std::max(1u, std::min(n_tiles_cap, max_blocks));
    const uint32_t scan_grid =
        std::max(1u, std::min((256u * n_tiles_cap + kScanTile - 1) / kScanTile, max_blocks));
    uint32_t passes = (bits + 7) / 8;
    if (passes & 1u) ++passes;  // even pass count: the result lands back in (k0, v0)
    for (uint32_t p = 0; p < passes; ++p) {
        const uint32_t shift = 8 * p;
        uint32_t *ki = (p & 1) ? k1 : k0, *vi = (p & 1) ? v1 : v0;
        uint32_t *ko = (p & 1) ? k0 : k1, *vo = (p & 1) ? v0 : v1;
        if (shift >= 32) {  // padding pass: plain copy keeps the order
            cudaError_t e = cudaMemcpyAsync(ko, ki, (size_t)cap * 4, cudaMemcpyDeviceToDevice, s);
            if (e != cudaSuccess) return e;
            e = cudaMemcpyAsync(vo, vi, (size_t)cap * 4, cudaMemcpyDeviceToDevice, s);
            if (e != cudaSuccess) return e;
            continue;
        }
        k_radix_hist<<<grid, kSortThreads, 0, s>>>(ki, n_dev, shift, hist, hist_n);
        cudaError_t e = device_scan<SumOp, true>(hist, hist, hist_n, 0, scan_grid, tot, 0, s);
        if (e != cudaSuccess) return e;
        k_radix_scatter<<<grid, kSortThreads, 0, s>>>(ki, vi, ko, vo, n_dev, shift, hist);
    }
    return cudaGetLastError();
}

namespace {

// Resources (conflict units) of transaction u for the ordered phase: its
// distinct words for bank / W1 updates (all written), its set's version word
// for a cache request (PUT writes, GET reads).  W1 read-only transactions
// have none: they run in the read-only phase.
struct TxView {
    uint32_t wl, li, b, n;
    uint32_t addr[4];
    uint32_t wmask;    // bit k: resource k is written
    uint32_t map;      // W1: 2-bit slot of the j-th declared word
    uint32_t aux;      // W1: txid; bank: amount
    const DevBatch *d;
    bool tail;         // W2 update: runs under the STM after the ordered phase
};

__device__ __forceinline__ int find_batch(const uint64_t *prefix, uint32_t nb, uint64_t gi) {
    uint32_t lo = 0, hi = nb;
    while (hi - lo > 1) {
        const uint32_t mid = (lo + hi) >> 1;
        if (__ldg(prefix + mid) <= gi) lo = mid; else hi = mid;
    }
    return (int)lo;
}

__device__ __forceinline__ bool view_tx(const ExecArgs &a, uint64_t u, TxView &t) {
    t.b = (uint32_t)find_batch(a.prefix, a.rp->n_batches, u);
    t.d = a.batches + t.b;
    t.wl = t.d->workload;
    t.li = (uint32_t)(u - a.prefix[t.b]);
    t.n = 0;
    t.wmask = 0;
    t.map = 0;
    t.aux = 0;
    t.tail = false;
    if (t.wl == HETM_WL_W2) {
        // no resources here: read-only W2 transactions run in the read-only
        // phase, updates under the STM after the ordered phase (40 words do
        // not fit the ordered record)
        const hetm_w2_tx *x = static_cast<const hetm_w2_tx *>(t.d->tx) + t.li;
        bool ok = true;
        for (int j = 0; j < 40; ++j) ok &= __ldg(&x->addr[j]) < a.n_words;
        t.tail = (x->flags & 1u) != 0;
        return ok;
    }
    if (t.wl == HETM_WL_BANK) {
        const hetm_bank_tx x = static_cast<const hetm_bank_tx *>(t.d->tx)[t.li];
        t.addr[0] = t.d->word_base + x.src;
        t.addr[1] = t.d->word_base + x.dst;
        t.n = t.addr[1] == t.addr[0] ? 1 : 2;
        t.wmask = 3;
        t.aux = (uint32_t)x.amount;
        return t.addr[0] < a.n_words && t.addr[1] < a.n_words;
    }
    if (t.wl == HETM_WL_RMW) {
        const hetm_rmw_tx *x = static_cast<const hetm_rmw_tx *>(t.d->tx) + t.li;
        uint32_t orig[4];
        bool ok = true;
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            orig[j] = x->addr[j];
            ok &= orig[j] < a.n_words;
        }
        if (x->flags & 1u) {
            uint32_t m = 0;
#pragma unroll
            for (int j = 0; j < 4; ++j) {
                uint32_t slot = m;
#pragma unroll
                for (int k = 0; k < 4; ++k)
                    if (k < (int)m && t.addr[k] == orig[j]) slot = k;
                if (slot == m) t.addr[m++] = orig[j];
                t.map |= slot << (2 * j);
            }
            t.n = m;
            t.wmask = (1u << m) - 1;
            t.aux = t.d->txid_base + t.li;
        }
        return ok;
    }
    if (t.wl == HETM_WL_CACHE) {
        const hetm_cache_req *r = static_cast<const hetm_cache_req *>(t.d->tx) + t.li;
        const uint32_t set = (uint32_t)(splitmix_fin(r->key) & ((1ull << a.cache_log2_sets) - 1));
        t.addr[0] = (uint32_t)(a.ver_base + set);
        t.n = 1;
        t.wmask = r->op == 1 ? 1u : 0u;
        return true;
    }
    return false;
}

// Ranks of the ordered phase.  The serial order is the launch order, so a
// transaction's rank and the offset of its accesses are the exclusive
// prefix, over the launch, of (1 << 32 | its resource count) for the
// transactions the ordered phase runs.  k_ord_count sums that value over
// each tile of kScanTile launch indices into scan_tot[tile]; the tile sums
// are scanned in place (k_scan_totals); k_ord_emit works each value out
// again and scans inside its tile.  Tiles are walked in rounds of 256
// consecutive indices, one per thread, so that a warp's record loads are
// contiguous.
__device__ __forceinline__ uint64_t ord_value(bool ok, const TxView &t) {
    return ok && t.n ? (1ull << 32) | t.n : 0ull;
}

__global__ void __launch_bounds__(kScanThreads) k_ord_count(OrderArgs o) {
    __shared__ uint64_t s_warp[kScanThreads / 32];
    const ExecArgs &a = o.e;
    const uint64_t total = a.rp->total_tx;
    if (blockIdx.x == 0 && threadIdx.x == 0) {
        *o.n_tx32 = (uint32_t)total;
        *o.n_cache_runs = 0;
        const unsigned long long v0 = *a.gv;
        *o.v0 = v0;
        *a.gv = v0 + total + 1;  // this launch owns versions v0+1 .. v0+total+1
    }
    unsigned long long bad = 0;
    const unsigned lane = threadIdx.x & 31u;
    const uint64_t nt = (total + kScanTile - 1) / kScanTile;
    for (uint64_t tile = blockIdx.x; tile < nt; tile += gridDim.x) {
        uint64_t sum = 0;
        for (int r = 0; r < kScanItems; ++r) {
            const uint64_t u = tile * kScanTile + (uint64_t)r * kScanThreads + threadIdx.x;
            TxView t;
            bool ok = false, tail = false;
            if (u < total) {
                ok = view_tx(a, u, t);
                sum += ord_value(ok, t);
                if (!ok) {  // out-of-range words or unknown workload: not executed
                    if (t.d->status) t.d->status[t.li] = kGaveUp;
                    ++bad;
                }
                tail = ok && t.tail;
            }
            // the W2 updates are listed warp by warp
            const unsigned m = __ballot_sync(kFull, tail);
            if (m && o.w2list) {
                unsigned long long base = 0;
                if (lane == (unsigned)(__ffs(m) - 1)) base = atomicAdd(o.w2n, (unsigned long long)__popc(m));
                base = __shfl_sync(kFull, base, __ffs(m) - 1);
                if (tail) o.w2list[base + __popc(m & lanemask_lt())] = (uint32_t)u;
            }
        }
        const uint64_t incl = block_scan_incl(sum, SumOp(), s_warp);
        if (threadIdx.x == kScanThreads - 1) o.scan_tot[tile] = incl;
    }
    if (bad) {
        set_err(a.err, kErrAddr);
        atomicAdd(a.counters + 1, bad);
    }
}

// access list entry: key = resource word, value = rank << 4 | slot << 2 | cache << 1 | writer
__global__ void __launch_bounds__(kScanThreads) k_ord_emit(OrderArgs o) {
    __shared__ uint64_t s_warp[kScanThreads / 32];
    const ExecArgs &a = o.e;
    const uint64_t total = a.rp->total_tx;
    const uint64_t nt = (total + kScanTile - 1) / kScanTile;
    for (uint64_t tile = blockIdx.x; tile < nt; tile += gridDim.x) {
        uint64_t carry = o.scan_tot[tile];  // exclusive prefix of the tile
        for (int r = 0; r < kScanItems; ++r) {
            const uint64_t u = tile * kScanTile + (uint64_t)r * kScanThreads + threadIdx.x;
            TxView t;
            bool ok = false;
            if (u < total) ok = view_tx(a, u, t);
            const uint64_t v = u < total ? ord_value(ok, t) : 0ull;
            const uint64_t incl = block_scan_incl(v, SumOp(), s_warp);
            const uint64_t c = carry + incl - v;  // exclusive prefix: (rank << 32) | offset
            carry += s_warp[kScanThreads / 32 - 1];  // the round's total
            __syncthreads();  // s_warp is rewritten by the next round's scan
            if (u >= total) continue;
            const uint32_t n = ok ? t.n : 0;
            if (n) {
                const uint32_t rank = (uint32_t)(c >> 32);
                OrdRec &rr = o.rec[rank];
                rr.u = (uint32_t)u;
                rr.meta = n | (t.wl << 3) | (t.map << 8) | (t.b << 16);
                rr.aux = t.aux;
                rr.li = t.li;
                const uint32_t cache = t.wl == HETM_WL_CACHE ? 2u : 0u;
                for (uint32_t k = 0; k < n; ++k) {
                    rr.addr[k] = t.addr[k];
                    o.keys0[(uint32_t)c + k] = t.addr[k];
                    o.vals0[(uint32_t)c + k] = (rank << 4) | (k << 2) | cache | ((t.wmask >> k) & 1u);
                }
            }
            if (u == total - 1) {
                *o.n_acc = (uint32_t)c + n;
                *o.n_ord = (uint32_t)(c >> 32) + (n ? 1u : 0u);
            }
        }
    }
    if (total == 0 && blockIdx.x == 0 && threadIdx.x == 0) {
        *o.n_acc = 0;
        *o.n_ord = 0;
    }
}

// per sorted access: (run head index << 32) | (index + 1 if a writer)
__global__ void __launch_bounds__(256) k_ord_runs(OrderArgs o) {
    const uint32_t n = *o.n_acc;
    const uint64_t stride = gridDim.x * (uint64_t)blockDim.x;
    // bound rounded up to whole warps: the cache run heads are appended warp by warp
    const uint64_t span = (n + 31ull) & ~31ull;
    for (uint64_t i = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; i < span; i += stride) {
        bool cache_head = false;
        if (i < n) {
            const bool head = i == 0 || o.keys0[i] != o.keys0[i - 1];
            const uint32_t v = o.vals0[i];
            o.runs[i] = ((head ? i : 0ull) << 32) | ((v & 1u) ? i + 1 : 0ull);
            o.packed[i] = 0ull;
            cache_head = head && (v & 2u);
        }
        const unsigned m = __ballot_sync(kFull, cache_head);
        if (m) {
            uint32_t base = 0;
            if ((threadIdx.x & 31u) == 0) base = atomicAdd(o.n_cache_runs, (uint32_t)__popc(m));
            base = __shfl_sync(kFull, base, 0);
            if (cache_head) o.cache_heads[base + __popc(m & lanemask_lt())] = (uint32_t)i;
        }
    }
}

// Per access: resource id (its run head), its turn, and whether it takes its
// input from a transaction of the same segment (then it does not wait on
// the global turn) and must publish to a later segment.
__global__ void __launch_bounds__(256) k_ord_acc(OrderArgs o) {
    const uint32_t n = *o.n_acc;
    const uint64_t stride = gridDim.x * (uint64_t)blockDim.x;
    for (uint64_t i = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; i < n; i += stride) {
        const uint32_t start = (uint32_t)(o.runs[i] >> 32);
        const uint32_t v = o.vals0[i];
        const uint32_t rank = v >> 4, k = (v >> 2) & 3u;
        const bool cache = v & 2u, writer = v & 1u;
        uint32_t turn, src = 0;
        if (cache) {  // reader/writer turns on the set's counter
            uint32_t need;
            if (writer) {
                need = (uint32_t)i - start;
            } else {
                const uint32_t lw = i ? (uint32_t)o.runs[i - 1] : 0u;  // last writer before i, + 1
                need = lw > start ? lw - start : 0u;
            }
            turn = need | (writer ? kFWriter : 0u);
        } else {
            turn = ((uint32_t)i - start) | kFWriter;
            if (i > start) {
                const uint32_t pv = o.vals0[i - 1];
                if ((pv >> 4) >> o.seg_log2 == rank >> o.seg_log2) {
                    turn |= kFLocal;
                    src = (((pv >> 4) & ((1u << o.seg_log2) - 1u)) << 2) | ((pv >> 2) & 3u);
                }
            }
            const bool last = i + 1 == n || o.keys0[i + 1] != o.keys0[i];
            if (last) turn |= kFLast;
            else if ((o.vals0[i + 1] >> 4) >> o.seg_log2 != rank >> o.seg_log2) turn |= kFPublish;
        }
        OrdRec &r = o.rec[rank];
        r.res[k] = start;
        r.turn[k] = turn;
        r.src[k] = src;
    }
}

// Read-only phase: W1 read-only transactions on the launch-start state.
__global__ void __launch_bounds__(256) k_ord_ro(OrderArgs o) {
    const ExecArgs &a = o.e;
    const uint64_t total = a.rp->total_tx;
    const unsigned long long key = 2ull * (*o.v0) + 1;
    const uint64_t stride = gridDim.x * (uint64_t)blockDim.x;
    const bool listing = a.rest && total <= a.rest_cap;
    unsigned long long n_commit = 0;
    // runs launch index u if it is a W1 read-only transaction; true if it ran
    auto run_ro = [&](uint64_t u) -> bool {
        const int b = find_batch(a.prefix, a.rp->n_batches, u);
        const DevBatch &d = a.batches[b];
        const uint32_t li = (uint32_t)(u - a.prefix[b]);
        if (d.workload == HETM_WL_W2) {  // W2 read-only: 40 words
            const hetm_w2_tx *x = static_cast<const hetm_w2_tx *>(d.tx) + li;
            if (x->flags & 1u) return false;
            bool ok = true;
            int32_t s = 0;
#pragma unroll 8
            for (int k = 0; k < 40; ++k) {
                const uint32_t ad = __ldg(&x->addr[k]);
                ok &= ad < a.n_words;
                if (ad < a.n_words) s += a.W[ad];
            }
            if (!ok) return false;  // reported by the STM
            if (a.instrument) {
#pragma unroll 8
                for (int k = 0; k < 40; ++k) rs_mark(a.rs, a.filter, __ldg(&x->addr[k]) >> a.gshift);
            }
            if (d.order) d.order[li] = key;
            if (d.out) static_cast<int32_t *>(d.out)[li] = s;
            if (d.status) d.status[li] = kCommitted;
            return true;
        }
        if (d.workload != HETM_WL_RMW) return false;
        const hetm_rmw_tx *x = static_cast<const hetm_rmw_tx *>(d.tx) + li;
        if (x->flags & 1u) return false;
        uint32_t ad[4];
        bool ok = true;
#pragma unroll
        for (int k = 0; k < 4; ++k) {
            ad[k] = x->addr[k];
            ok &= ad[k] < a.n_words;
        }
        if (!ok) return false;  // reported by k_ord_count or the STM
        int32_t s = 0;
#pragma unroll
        for (int k = 0; k < 4; ++k) s += a.W[ad[k]];
        if (a.instrument) {
#pragma unroll
            for (int k = 0; k < 4; ++k) rs_mark(a.rs, a.filter, ad[k] >> a.gshift);
        }
        if (d.order) d.order[li] = key;
        if (d.out) static_cast<int32_t *>(d.out)[li] = s;
        if (d.status) d.status[li] = kCommitted;
        return true;
    };
    // The indices left to the STM are gathered in shared memory (one shared
    // atomic per warp and iteration) and appended to the list with one global
    // atomic per block at the end: one counter for the whole launch would
    // serialize the appends.  What does not fit the block's buffer goes to
    // the list directly, one atomic per warp.
    constexpr uint32_t kCap = 4096;
    __shared__ uint32_t s_list[kCap];
    __shared__ uint32_t s_n;
    __shared__ unsigned long long s_base;
    const unsigned lane = threadIdx.x & 31u;
    if (threadIdx.x == 0) s_n = 0;
    __syncthreads();
    // loop bound rounded up to whole warps so that the warp collectives are convergent
    const uint64_t span = (total + 31) & ~31ull;
    for (uint64_t u = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; u < span; u += stride) {
        const bool ran = u < total && run_ro(u);
        n_commit += ran ? 1u : 0u;
        if (listing) {
            const bool left = u < total && !ran;
            const unsigned m = __ballot_sync(kFull, left);
            if (m) {
                uint32_t base = 0;
                if (lane == 0) base = atomicAdd(&s_n, (uint32_t)__popc(m));
                base = __shfl_sync(kFull, base, 0);
                const uint32_t pos = base + __popc(m & lanemask_lt());
                const bool spill = left && pos >= kCap;
                if (left && !spill) s_list[pos] = (uint32_t)u;
                const unsigned ms = __ballot_sync(kFull, spill);
                if (ms) {
                    unsigned long long g = 0;
                    if (lane == (unsigned)(__ffs(ms) - 1)) g = atomicAdd(a.rest_n, (unsigned long long)__popc(ms));
                    g = __shfl_sync(kFull, g, __ffs(ms) - 1);
                    if (spill) a.rest[g + __popc(ms & lanemask_lt())] = (uint32_t)u;
                }
            }
        }
    }
    __syncthreads();
    if (listing) {
        const uint32_t n = min(s_n, kCap);
        if (threadIdx.x == 0) s_base = n ? atomicAdd(a.rest_n, (unsigned long long)n) : 0ull;
        __syncthreads();
        for (uint32_t i = threadIdx.x; i < n; i += blockDim.x) a.rest[s_base + i] = s_list[i];
    }
#pragma unroll
    for (int w = 16; w > 0; w >>= 1) n_commit += __shfl_xor_sync(kFull, n_commit, w);
    if ((threadIdx.x & 31u) == 0 && n_commit) atomicAdd(a.counters + 0, n_commit);
}

__device__ __forceinline__ void mark_range(const ExecArgs &a, uint64_t w0, uint32_t len, bool write) {
    if (!a.instrument) return;
    for (uint64_t g = w0 >> a.gshift; g <= (w0 + len - 1) >> a.gshift; ++g)
        rs_mark(a.rs, a.filter, g);
    if (write)
        for (uint64_t c = w0 >> a.cshift; c <= (w0 + len - 1) >> a.cshift; ++c)
            atomicOr(a.ws + (c >> 5), 1u << (c & 31));
}


// Object cache (Sec. V-D).  A request touches only its own set, so the
// requests of different sets never depend on each other and only each set's
// own requests need the launch order.  The sorted access list holds them as
// one run per set; one warp takes a run, keeps the set (8 keys, 8 values, 8
// GPU stamps, version) in registers -- the same copy in every lane -- and
// applies the run's requests in rank order, 32 staged at a time (each lane
// loads one, then every lane applies them all in turn).  The changed words go
// back once per run, and the read/write-set marks of all its requests are
// applied once, spread over the lanes.  No hand-on between warps is needed.
// (Word transactions of the same launch must not touch the cache regions.)
struct CacheMarks {
    uint32_t keys_read, lru_all_read, ver_write;
    uint32_t val_read, val_write, key_write, lru_write;  // bit w: way w
};

// One request applied to the set copy; returns the request's output.
__device__ __forceinline__ uint64_t cache_apply(uint64_t (&keys)[8], uint64_t (&vals)[8], uint32_t (&lru)[8],
                                                uint32_t &ver, uint32_t &dirty_kv, uint32_t &dirty_lru,
                                                uint64_t key, uint64_t value, uint32_t op, uint32_t stamp,
                                                CacheMarks &mk) {
    int hit = -1, empty = -1;
#pragma unroll
    for (int w = 7; w >= 0; --w) {
        if (keys[w] == key) hit = w;
        if (keys[w] == 0) empty = w;
    }
    mk.keys_read = 1;
    if (op == 0) {  // GET: a hit reads the value and stamps the way
        if (hit < 0) return ~0ull;
        uint64_t out = 0;
#pragma unroll
        for (int w = 0; w < 8; ++w)
            if (w == hit) {
                out = vals[w];
                lru[w] = max(lru[w], stamp);
            }
        dirty_lru |= 1u << hit;
        mk.val_read |= 1u << hit;
        mk.lru_write |= 1u << hit;
        return out;
    }
    // PUT: update in place, else the first empty way, else the least recently
    // stamped way (lowest way on ties)
    int way;
    if (hit >= 0) {
        way = hit;
    } else if (empty >= 0) {
        way = empty;
    } else {
        way = 0;
        uint32_t best = lru[0];
#pragma unroll
        for (int w = 1; w < 8; ++w)
            if (lru[w] < best) {
                best = lru[w];
                way = w;
            }
        mk.lru_all_read = 1;
    }
#pragma unroll
    for (int w = 0; w < 8; ++w)
        if (w == way) {
            keys[w] = key;
            vals[w] = value;
            lru[w] = stamp;
        }
    if (hit < 0) mk.key_write |= 1u << way;
    dirty_kv |= 1u << way;
    dirty_lru |= 1u << way;
    ++ver;
    mk.val_write |= 1u << way;
    mk.lru_write |= 1u << way;
    mk.ver_write = 1;
    return (uint64_t)way;
}

__device__ __forceinline__ uint64_t shfl64(uint64_t v, int l) {
    return ((uint64_t)__shfl_sync(kFull, (uint32_t)(v >> 32), l) << 32) | __shfl_sync(kFull, (uint32_t)v, l);
}

// Ordered phase, CTA-segment executor.  A CTA takes segments of SEG
// consecutive ranks in rank order; executor thread t owns rank g*SEG + t,
// and one extra warp (the poll warp) watches the words that earlier segments
// hand on.  Each executor warp runs its 32 transactions in waves: in one
// wave every lane whose inputs are all available executes (lanes ready at
// the same time never depend on each other), then the warp syncs.  Inputs
// come from a predecessor in the same segment (its value in shared memory,
// tagged with the segment) or from an earlier segment (the resource's packed
// (turns done, value) word in global memory).  The executor warps issue no
// global load inside the wave loop: a load in flight would stall the whole
// warp, and with it the lanes at the front of a chain, for an L2 round trip
// at every wave.  Instead each lane checks its external inputs once when the
// segment starts, and the poll warp polls the ones still pending and hands
// each one over through shared memory as soon as it is satisfied.  A warp
// none of whose lanes ran in a pass sleeps briefly, leaving the issue slots
// to the warps at the front of the chains.  (Measured on the 4M-transaction
// Zipf(0.99) batch: 20 ns after each idle pass is 1-2% faster than 50 or
// 100 ns and a few percent faster than spinning; sleeps scaled by an estimate
// of the turns still ahead are no better.  The poll warp itself does not
// sleep: a sleep scaled by the turns still ahead of its nearest wait cost
// 0.5%, and 10 ns a link on a chain inside one warp.)
#ifndef HETM_IDLE_SLEEP_NS
#define HETM_IDLE_SLEEP_NS 20  // ns of sleep after a pass in which no lane of the warp ran
#endif
#ifndef HETM_IDLE_PASSES
#define HETM_IDLE_PASSES 4  // idle passes between two looks at the abort flag and the clock
#endif

template <uint32_t SEG>
struct SegSmem {
    // (segment + 1) << 32 | value: one aligned 8-byte store hands a word on
    // to a later transaction of the segment, flag and data together
    // slot-major, so that the lanes of a warp read 8-byte words 8 bytes apart
    unsigned long long pack[4][SEG];  // output of thread t for slot k: pack[k][t]
    unsigned long long ext[4][SEG];   // external input of slot k, from the poll warp
    uint32_t list_slot[SEG * 4];      // pending external slots: t << 2 | k
    uint32_t list_res[SEG * 4];       //   their resource
    uint32_t list_turn[SEG * 4];      //   their turn word
    uint32_t seg, n_list;
    int abort;
};

template <uint32_t SEG>
__global__ void __launch_bounds__(SEG + 32) k_seg_exec(OrderArgs o) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    SegSmem<SEG> &sm = *reinterpret_cast<SegSmem<SEG> *>(smem_raw);
    const ExecArgs &a = o.e;
    const uint32_t n_ord = *o.n_ord;
    const uint32_t n_seg = (n_ord + SEG - 1) / SEG;
    const unsigned long long v0 = *o.v0;
    const unsigned t = threadIdx.x;
    const unsigned lane = t & 31u;
    const bool poller = t >= SEG;
    const unsigned long long t0 = __shfl_sync(kFull, globaltimer_ns(), 0);
    unsigned long long n_commit = 0, n_gaveup = 0;
    if (!poller) {
#pragma unroll
        for (int k = 0; k < 4; ++k) sm.pack[k][t] = 0ull;
#pragma unroll
        for (int k = 0; k < 4; ++k) sm.ext[k][t] = 0ull;
    }
    if (t == 0) sm.abort = 0;
    if (t == 0 && blockIdx.x == 0 && a.segs_total) st_rlx32((int32_t *)a.segs_total, (int32_t)(n_seg + 1));
    __syncthreads();
    for (;;) {
        if (t == 0) {
            // sm.abort: 1 = the time budget ran out, 2 = early validation
            // found a conflict; either way this CTA runs no more transactions
            // and only reports the ones of the segments it still takes
            if (!sm.abort && a.stop && ld_rlx32((const int32_t *)a.stop)) sm.abort = 2;
            sm.seg = (uint32_t)atomicAdd(a.next, 1ull);
            sm.n_list = 0;
        }
        __syncthreads();
        const uint32_t g = sm.seg;
        if (g >= n_seg) break;
        const unsigned long long tag = (unsigned long long)(g + 1) << 32;
        if (sm.abort) {
            // stopped by early validation (the round is lost to the CPU: not
            // run) or past the time budget (gave up; cache requests are left
            // to k_cache_runs, and the merge undoes the whole phase)
            const uint32_t r = g * SEG + t;
            if (!poller && r < n_ord) {
                const OrdRec &q = o.rec[r];
                const DevBatch &d = a.batches[q.meta >> 16];
                if (sm.abort == 2) {
                    if (d.status) d.status[q.li] = kNotRun;
                } else if (((q.meta >> 3) & 3u) != HETM_WL_CACHE) {
                    if (d.status) d.status[q.li] = kGaveUp;
                    ++n_gaveup;
                }
            }
            __syncthreads();
            if (t == 0 && a.segs_done) atomicAdd(a.segs_done, 1u);
            continue;
        }

        if (poller) {
            // ---------------- poll warp: external inputs still pending
            __syncthreads();  // the executors have listed them
            uint32_t n = sm.n_list;
            uint32_t passes = 0;
            while (n) {
                if (*(volatile int *)&sm.abort) break;
                if (a.stop && ld_rlx32((const int32_t *)a.stop)) {
                    if (lane == 0) atomicCAS(&sm.abort, 0, 2);
                    break;
                }
                if ((++passes & 15u) == 0 &&
                    __shfl_sync(kFull, globaltimer_ns(), 0) - t0 > a.budget_ns)
                    break;  // the executors see the budget run out themselves
                uint32_t kept = 0;
                for (uint32_t base = 0; base < n; base += 128) {
                    uint32_t sl[4], rs[4], tf[4];
                    unsigned long long pv[4];
#pragma unroll
                    for (int j = 0; j < 4; ++j) {
                        const uint32_t i = base + 32 * j + lane;
                        sl[j] = 0xFFFFFFFFu;
                        if (i < n) {
                            sl[j] = sm.list_slot[i];
                            rs[j] = sm.list_res[i];
                            tf[j] = sm.list_turn[i];
                            pv[j] = ld_rlx64(o.packed + rs[j]);
                        }
                    }
                    bool ok[4];
#pragma unroll
                    for (int j = 0; j < 4; ++j) {
                        ok[j] = false;
                        if (sl[j] == 0xFFFFFFFFu) continue;
                        const uint32_t c = (uint32_t)(pv[j] >> 32), need = tf[j] & kTurnMask;
                        ok[j] = (tf[j] & kFWriter) ? c == need : c >= need;
                    }
                    // No fence before handing the inputs on: every pending input
                    // is a word whose value travels in the same 8-byte word as
                    // its turn count (cache requests do not run here), so the
                    // relaxed load above already holds everything the consumer
                    // reads.
#pragma unroll
                    for (int j = 0; j < 4; ++j)
                        if (ok[j])
                            *(volatile unsigned long long *)&sm.ext[sl[j] & 3u][sl[j] >> 2] =
                                tag | (uint32_t)pv[j];
                    __syncwarp();
                    // compact the pending entries in place (writes land below
                    // every index this warp still has to read)
#pragma unroll
                    for (int j = 0; j < 4; ++j) {
                        const bool keep = sl[j] != 0xFFFFFFFFu && !ok[j];
                        const unsigned m = __ballot_sync(kFull, keep);
                        if (keep) {
                            const uint32_t p = kept + __popc(m & lanemask_lt());
                            sm.list_slot[p] = sl[j];
                            sm.list_res[p] = rs[j];
                            sm.list_turn[p] = tf[j];
                        }
                        kept += __popc(m);
                    }
                    __syncwarp();
                }
                n = kept;
            }
            __syncthreads();  // end of segment
            continue;
        }

        // ---------------- executor lanes
        const uint32_t r = g * SEG + t;
        OrdRec rc;
        uint32_t n = 0, wl = 0;
        if (r < n_ord) {
            rc = o.rec[r];
            n = rc.meta & 7u;
            wl = (rc.meta >> 3) & 3u;
        }
        const bool cache = wl == HETM_WL_CACHE;
        // output pointers now, so that no global load sits on the handoff path
        uint64_t *o_order = nullptr;
        uint8_t *o_status = nullptr;
        void *o_out = nullptr;
        if (n) {
            const DevBatch &d = a.batches[rc.meta >> 16];
            o_order = d.order;
            o_status = d.status;
            o_out = d.out;
        }
        // W1 update naming 4 distinct words (the common case): slot j = word j
        const bool rmw4 = wl == HETM_WL_RMW && n == 4 && ((rc.meta >> 8) & 0xFFu) == 0xE4u;
        int32_t cur[4] = {0, 0, 0, 0};
        int32_t nv[4] = {0, 0, 0, 0};
        int32_t sum = 0;
        uint32_t ext = 0, loc = 0;  // slots still waiting on an earlier segment / this segment
#pragma unroll
        for (int k = 0; k < 4; ++k) {
            if (k >= (int)n || cache) continue;
            const uint32_t tf = rc.turn[k];
            if (!cache && (tf & kFLocal)) loc |= 1u << k;
            else if (cache || (tf & kTurnMask)) ext |= 1u << k;
            else cur[k] = ld_rlx32(a.W + rc.addr[k]);  // first access: launch-start value
        }
        unsigned long long pv[4] = {0, 0, 0, 0};
#pragma unroll
        for (int k = 0; k < 4; ++k)
            if (ext & (1u << k)) pv[k] = ld_rlx64(o.packed + rc.res[k]);
        // one look at the external inputs; what is not there yet goes to the poll warp
#pragma unroll
        for (int k = 0; k < 4; ++k) {
            if (!(ext & (1u << k))) continue;
            const uint32_t c = (uint32_t)(pv[k] >> 32), need = rc.turn[k] & kTurnMask;
            if ((rc.turn[k] & kFWriter) ? c == need : c >= need) {
                ext &= ~(1u << k);
                cur[k] = (int32_t)(uint32_t)pv[k];
            }
        }
        {
            const uint32_t cnt = __popc(ext);
            uint32_t incl = cnt;
#pragma unroll
            for (int w = 1; w < 32; w <<= 1) {
                const uint32_t y = __shfl_up_sync(kFull, incl, w);
                if (lane >= (unsigned)w) incl += y;
            }
            const uint32_t total = __shfl_sync(kFull, incl, 31);
            uint32_t base = 0;
            if (lane == 31 && total) base = atomicAdd(&sm.n_list, total);
            base = __shfl_sync(kFull, base, 31);
            uint32_t p = base + incl - cnt;
#pragma unroll
            for (int k = 0; k < 4; ++k) {
                if (!(ext & (1u << k))) continue;
                sm.list_slot[p] = (t << 2) | (uint32_t)k;
                sm.list_res[p] = rc.res[k];
                sm.list_turn[p] = rc.turn[k];
                ++p;
            }
        }
        __syncthreads();  // the pending list is complete: the poll warp starts

        bool finished = n == 0 || cache;  // cache requests run in k_cache_runs
        bool executed = false;
        bool timed_out = false;
        // Each slot still pending watches one shared word: its predecessor's
        // output slot in this segment, or its external input from the poll
        // warp; a slot no longer pending watches this lane's own output cell
        // (never tagged before the lane runs; written only for slots whose
        // next access is in this segment).  One pass is four
        // independent shared loads and selects, with no per-slot branching,
        // so that a hand-on inside the segment costs one short pass.
        uint32_t watch[4];
        uint32_t pend = ext | loc;
#pragma unroll
        for (int k = 0; k < 4; ++k) {
            const unsigned long long *w = &sm.pack[k][t];
            if (loc & (1u << k)) w = &sm.pack[rc.src[k] & 3u][rc.src[k] >> 2];
            else if (ext & (1u << k)) w = &sm.ext[k][t];
            watch[k] = (uint32_t)__cvta_generic_to_shared(w);
        }
        // what the pass needs, worked out once: every instruction in the pass
        // is on the path of each hand-on inside a warp
        const uint32_t gt = g + 1;
        uint32_t pubmask = 0;
        uint32_t pturn[4];
#pragma unroll
        for (int k = 0; k < 4; ++k) {
            pturn[k] = (rc.turn[k] & kTurnMask) + 1u;
            if (k < (int)n && (rc.turn[k] & kFPublish)) pubmask |= 1u << k;
        }
        const int32_t aux0 = (int32_t)rc.aux;
        // slots whose next access is in this segment: only those hand on through
        // shared memory, and only those are stored (a shared store in the pass
        // lengthens every hand-on)
        uint32_t locmask = 0;
#pragma unroll
        for (int k = 0; k < 4; ++k)
            if (k < (int)n && !(rc.turn[k] & (kFLast | kFPublish))) locmask |= 1u << k;
        auto run_tx = [&]() {
            if (rmw4) {
                sum = (cur[0] + cur[1]) + (cur[2] + cur[3]);
#pragma unroll
                for (int k = 0; k < 4; ++k) nv[k] = sum + (aux0 + k);
            } else if (wl == HETM_WL_RMW) {
#pragma unroll
                for (int j = 0; j < 4; ++j) {
                    const uint32_t sl = (rc.meta >> (8 + 2 * j)) & 3u;
#pragma unroll
                    for (int k = 0; k < 4; ++k)
                        if ((uint32_t)k == sl) sum += cur[k];
                }
                // a word named twice keeps the value of its last position
#pragma unroll
                for (int j = 0; j < 4; ++j) {
                    const uint32_t sl = (rc.meta >> (8 + 2 * j)) & 3u;
#pragma unroll
                    for (int k = 0; k < 4; ++k)
                        if ((uint32_t)k == sl) nv[k] = sum + j + (int32_t)rc.aux;
                }
            } else if (n == 1) {  // bank transfer onto the same account
                nv[0] = cur[0];
            } else {
                nv[0] = cur[0] - (int32_t)rc.aux;
                nv[1] = cur[1] + (int32_t)rc.aux;
            }
#pragma unroll
            for (int k = 0; k < 4; ++k)
                if (locmask & (1u << k)) *(volatile unsigned long long *)&sm.pack[k][t] = tag | (uint32_t)nv[k];
#pragma unroll
            for (int k = 0; k < 4; ++k)
                if (pubmask & (1u << k))
                    st_rlx64(o.packed + rc.res[k], ((unsigned long long)pturn[k] << 32) | (uint32_t)nv[k]);
            finished = true;
            executed = true;
        };
        const bool all_rmw4 = __all_sync(kFull, rmw4 || finished);
        // The pass loop, compiled twice: for a warp whose lanes are all 4-word
        // W1 updates (or none) a loop of its own with the straight body, for
        // every other warp the general one.
        auto passes = [&](auto w1_only) {
            constexpr bool kW1 = decltype(w1_only)::value;
            uint32_t idle = 0, checks = 0;
            for (;;) {
                unsigned long long v[4];
#pragma unroll
                for (int k = 0; k < 4; ++k)
                    asm volatile("ld.volatile.shared.u64 %0, [%1];" : "=l"(v[k]) : "r"(watch[k]) : "memory");
                // a watched cell tagged with this segment holds the slot's input; a
                // slot that is not pending watches this lane's own output cell,
                // tagged (if at all) only once the lane has run, so its value is
                // never taken
                uint32_t gotm = 0;
#pragma unroll
                for (int k = 0; k < 4; ++k) {
                    const bool got = (uint32_t)(v[k] >> 32) == gt;
                    cur[k] = got ? (int32_t)(uint32_t)v[k] : cur[k];
                    gotm |= got ? (1u << k) : 0u;
                }
                const bool ready = !finished && (pend & ~gotm) == 0;
                if constexpr (kW1) {
                    const int32_t s4 = (cur[0] + cur[1]) + (cur[2] + cur[3]);
                    if (ready) {
                        sum = s4;
#pragma unroll
                        for (int k = 0; k < 4; ++k) {
                            nv[k] = s4 + (aux0 + k);
                            if (locmask & (1u << k))
                                *(volatile unsigned long long *)&sm.pack[k][t] = tag | (uint32_t)nv[k];
                        }
#pragma unroll
                        for (int k = 0; k < 4; ++k)
                            if (pubmask & (1u << k))
                                st_rlx64(o.packed + rc.res[k],
                                         ((unsigned long long)pturn[k] << 32) | (uint32_t)nv[k]);
                        finished = true;
                        executed = true;
                    }
                } else {
                    if (ready) run_tx();
                }
                __syncwarp();
                // a pass in which a lane ran is followed by another: the warp
                // leaves from an idle pass, so a busy pass takes one vote
                if (__any_sync(kFull, ready)) {
                    idle = 0;
                    continue;
                }
                if (__all_sync(kFull, finished)) break;
                // an idle pass leaves the issue slots to the warps that can run
                if (HETM_IDLE_SLEEP_NS) __nanosleep(HETM_IDLE_SLEEP_NS);
                if (++idle < HETM_IDLE_PASSES) continue;
                idle = 0;
                if (__any_sync(kFull, *(volatile int *)&sm.abort != 0) ||
                    ((++checks & 3u) == 0 &&
                     __shfl_sync(kFull, globaltimer_ns(), 0) - t0 > a.budget_ns)) {
                    timed_out = true;
                    break;
                }
            }
        };
        if (all_rmw4) passes(std::true_type{});
        else passes(std::false_type{});
        if (executed) {
            const unsigned long long key = 2ull * (v0 + 1 + rc.u);
            if (!cache) {
#pragma unroll
                for (int k = 0; k < 4; ++k) {
                    if (k >= (int)n) continue;
                    if (rc.turn[k] & kFLast) st_rlx32(a.W + rc.addr[k], nv[k]);
                    // the bitmaps are unions over the round: the word's first
                    // writer marks it for all of its writers
                    if ((rc.turn[k] & kTurnMask) == 0) mark_range(a, rc.addr[k], 1, true);
                }
                if (wl == HETM_WL_RMW && o_out) static_cast<int32_t *>(o_out)[rc.li] = sum;
            }
            if (o_order) o_order[rc.li] = key;
            if (o_status) o_status[rc.li] = kCommitted;
            ++n_commit;
        }
        if (timed_out && !finished) {
            if (*(volatile int *)&sm.abort == 2) {
                // stopped by early validation: the round is lost to the CPU,
                // this transaction never runs (its successors stop too)
                if (o_status) o_status[rc.li] = kNotRun;
            } else {
                if (o_status) o_status[rc.li] = kGaveUp;
                ++n_gaveup;
                set_err(a.err, kErrTimeout);
                // the other warps of the CTA see it at their next idle pass and
                // give up too; a successor waiting on this transaction never
                // sees its input arrive, so it cannot run on a missing value
                sm.abort = 1;
            }
        }
        __syncthreads();  // end of segment
        if (t == 0 && a.segs_done) atomicAdd(a.segs_done, 1u);
    }
    if (poller) return;
#pragma unroll
    for (int w = 16; w > 0; w >>= 1) {
        n_commit += __shfl_xor_sync(kFull, n_commit, w);
        n_gaveup += __shfl_xor_sync(kFull, n_gaveup, w);
    }
    if (lane == 0) {
        if (n_commit) atomicAdd(a.counters + 0, n_commit);
        if (n_gaveup) atomicAdd(a.counters + 1, n_gaveup);
    }
}

// Staging of every cache access's request in access-list order, so that the
// run kernel reads it with coalesced loads instead of a chain of dependent
// random ones (access -> record -> request).  It reuses scratch that is free
// once the turns are computed: packed (key), runs (value), keys1 (batch << 1
// | op), vals1 (index in the batch) and vals0 (the transaction's launch
// index, which gives its commit version).
__global__ void __launch_bounds__(256) k_cache_gather(OrderArgs o) {
    const ExecArgs &a = o.e;
    if (*o.n_cache_runs == 0) return;
    const uint32_t n = *o.n_acc;
    const uint64_t stride = gridDim.x * (uint64_t)blockDim.x;
    for (uint64_t j = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; j < n; j += stride) {
        const uint32_t v = o.vals0[j];
        if (!(v & 2u)) continue;
        const OrdRec &q = o.rec[v >> 4];
        const uint32_t li = q.li, b = q.meta >> 16;
        const hetm_cache_req r = static_cast<const hetm_cache_req *>(a.batches[b].tx)[li];
        o.packed[j] = r.key;
        o.runs[j] = r.value;
        o.keys1[j] = (b << 1) | (r.op & 1u);
        o.vals1[j] = li;
        o.vals0[j] = q.u;
    }
}

// One warp per cache run (see cache_apply); the next 32 staged requests are
// loaded while the current ones are applied.  Early validation's stop flag
// leaves runs not yet started as not run.
// One staged cache request of a run (a lane's slot of a 32-request chunk).
struct CacheStage {
    uint64_t key, value;
    uint32_t meta, li, u, res;
};
__device__ __forceinline__ void cp_async8(void *dst, const void *src) {
    asm volatile("cp.async.ca.shared.global [%0], [%1], 8;" ::"r"((uint32_t)__cvta_generic_to_shared(dst)),
                 "l"(src)
                 : "memory");
}
__device__ __forceinline__ void cp_async4(void *dst, const void *src) {
    asm volatile("cp.async.ca.shared.global [%0], [%1], 4;" ::"r"((uint32_t)__cvta_generic_to_shared(dst)),
                 "l"(src)
                 : "memory");
}
__global__ void __launch_bounds__(256) k_cache_runs(OrderArgs o) {
    const ExecArgs &a = o.e;
    const uint32_t n_runs = *o.n_cache_runs;
    if (n_runs == 0) return;
    const uint32_t n_acc = *o.n_acc;
    const unsigned long long v0 = *o.v0;
    const unsigned lane = threadIdx.x & 31u;
    const uint32_t warp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const uint32_t n_warps = (gridDim.x * blockDim.x) >> 5;
    __shared__ CacheStage stage_ring[8][2][32];  // per warp: the chunk in use and the next one
    unsigned long long n_commit = 0;
    for (uint32_t ri = warp; ri < n_runs; ri += n_warps) {
        const uint32_t head = o.cache_heads[ri];
        const uint32_t res = o.keys0[head];  // the set's version word
        const uint32_t set = res - (uint32_t)a.ver_base;
        const bool stopped = a.stop && __shfl_sync(kFull, ld_rlx32((const int32_t *)a.stop), 0);
        const uint64_t kw = a.key_base + 16ull * set, vb = a.val_base + 16ull * set;
        const uint64_t lb = a.lru_base + 8ull * set;
        uint64_t keys[8], vals[8];
        uint32_t lru[8];
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            const uint4 k = *reinterpret_cast<const uint4 *>(a.W + kw + 4 * q);
            const uint4 v = *reinterpret_cast<const uint4 *>(a.W + vb + 4 * q);
            keys[2 * q] = ((uint64_t)k.y << 32) | k.x;
            keys[2 * q + 1] = ((uint64_t)k.w << 32) | k.z;
            vals[2 * q] = ((uint64_t)v.y << 32) | v.x;
            vals[2 * q + 1] = ((uint64_t)v.w << 32) | v.z;
        }
#pragma unroll
        for (int q = 0; q < 2; ++q) {
            const uint4 l = *reinterpret_cast<const uint4 *>(a.W + lb + 4 * q);
            lru[4 * q] = l.x;
            lru[4 * q + 1] = l.y;
            lru[4 * q + 2] = l.z;
            lru[4 * q + 3] = l.w;
        }
        uint32_t ver = (uint32_t)a.W[res], ver0 = ver, dirty_kv = 0, dirty_lru = 0;
        CacheMarks mk{};
        // Chunk c of the run (its 32 requests, one per lane) is copied into
        // this warp's shared-memory slot c & 1 by cp.async while chunk c - 1
        // is applied: the six copies of a lane issue at once and hold no
        // registers, where register staging had to wait for the access-list
        // key (is the request in the run?) before loading the rest.  Each
        // lane copies and reads only its own slot entry.
        CacheStage(&ring)[2][32] = stage_ring[threadIdx.x >> 5];
        auto issue = [&](uint32_t c) {
            const uint32_t j = head + 32u * c + lane;
            CacheStage &e = ring[c & 1u][lane];
            if (j < n_acc) {
                cp_async8(&e.key, o.packed + j);
                cp_async8(&e.value, o.runs + j);
                cp_async4(&e.meta, o.keys1 + j);
                cp_async4(&e.li, o.vals1 + j);
                cp_async4(&e.u, o.vals0 + j);
                cp_async4(&e.res, o.keys0 + j);
            }
            asm volatile("cp.async.commit_group;" ::: "memory");
        };
        // GPU stamps only grow, and stamps grow with the rank, so a way's
        // stamp is the largest stamp of any access to it.  A GET therefore
        // only raises this lane's own running maximum for the way it hit;
        // the lanes' maxima are folded into the set copy (warp reductions)
        // only where a stamp is read: before a PUT that must evict, and at
        // the end of the run.
        uint32_t pl[8] = {0, 0, 0, 0, 0, 0, 0, 0};  // this lane's newest GET stamp per way
        uint32_t pend_ways = 0, mark_ways = 0;        // ways with unfolded stamps / hit by this lane
        bool any_get = false;
        auto fold = [&]() {
            const uint32_t wa = __reduce_or_sync(kFull, pend_ways);
#pragma unroll
            for (int w = 0; w < 8; ++w)
                if ((wa >> w) & 1u) lru[w] = max(lru[w], __reduce_max_sync(kFull, pl[w]));
            pend_ways = 0;
        };
        bool in = false;
        uint64_t key = 0, value = 0;
        uint32_t meta = 0, li = 0, u = 0;
        issue(0);
        for (uint32_t c = 0;; ++c) {
            asm volatile("cp.async.wait_group 0;" ::: "memory");
            {
                const uint32_t j = head + 32u * c + lane;
                const CacheStage &e = ring[c & 1u][lane];
                in = j < n_acc && e.res == res;  // the run is contiguous: a prefix of lanes
                key = e.key;
                value = e.value;
                meta = e.meta;
                li = e.li;
                u = e.u;
            }
            const unsigned m = __ballot_sync(kFull, in);
            const int cnt = __popc(m);
            if (cnt == 32) issue(c + 1);  // the run goes on: copy its next chunk
            const uint32_t op = meta & 1u;
            const DevBatch *d = in ? a.batches + (meta >> 1) : nullptr;
            uint64_t my_out = 0;
            const unsigned puts = __ballot_sync(kFull, in && op == 1u);
            const uint32_t my_stamp = (uint32_t)(v0 + 1 + u);
            if (!stopped) {
                // The chunk is cut at every PUT of a key that is not in the set
                // at that point (an insert, possibly evicting): such a PUT runs
                // alone, in order.  In the stretch before it no key moves, since
                // its PUTs all update keys already in the set in place: each GET
                // reads the value of the last PUT to its way before it in the
                // stretch, else the copy at the stretch's start, and each way
                // written ends the stretch with its last PUT's value.
                int pos = 0;
                while (pos < cnt) {
                    int h0 = -1;  // this lane's key in the current copy
#pragma unroll
                    for (int w = 7; w >= 0; --w)
                        if (keys[w] == key) h0 = w;
                    const unsigned from = ~((1u << pos) - 1u);
                    const unsigned ins = __ballot_sync(kFull, in && op == 1u && h0 < 0) & from;
                    const int np = ins ? __ffs(ins) - 1 : cnt;  // next inserting PUT (or the end)
                    const unsigned range = from & (np < 32 ? (1u << np) - 1u : kFull);
                    if (np > pos) {
                        const bool inr = in && ((range >> lane) & 1u);
                        const unsigned rputs = puts & range;
                        const unsigned same = __match_any_sync(kFull, inr ? h0 : -2);
                        const unsigned before = same & rputs & lanemask_lt();
                        const uint64_t pv = shfl64(value, before ? 31 - __clz(before) : (int)lane);
                        if (inr) {
                            if (op == 1u) {
                                my_out = (uint64_t)h0;
                            } else {
                                uint64_t cv = ~0ull;
#pragma unroll
                                for (int w = 0; w < 8; ++w)
                                    if (w == h0) cv = vals[w];
                                my_out = before ? pv : cv;
                                any_get = true;
                                if (h0 >= 0) mark_ways |= 1u << h0;
                            }
                            if (h0 >= 0) {
#pragma unroll
                                for (int w = 0; w < 8; ++w)
                                    if (w == h0) pl[w] = max(pl[w], my_stamp);
                                pend_ways |= 1u << h0;
                            }
                        }
                        if (rputs) {
                            const bool last_put =
                                ((rputs >> lane) & 1u) && !(same & rputs & ~lanemask_lt() & ~(1u << lane));
                            const uint32_t wput = __reduce_or_sync(kFull, last_put ? 1u << h0 : 0u);
#pragma unroll
                            for (int w = 0; w < 8; ++w) {
                                if (!((wput >> w) & 1u)) continue;
                                const unsigned lb = __ballot_sync(kFull, last_put && h0 == w);
                                vals[w] = shfl64(value, __ffs(lb) - 1);
                            }
                            dirty_kv |= wput;
                            dirty_lru |= wput;
                            mk.val_write |= wput;
                            mk.lru_write |= wput;
                            mk.ver_write = 1;
                            ver += (uint32_t)__popc(rputs);
                        }
                        mk.keys_read = 1;
                    }
                    if (np < cnt) {
                        const uint64_t k_ = shfl64(key, np), v_ = shfl64(value, np);
                        const uint32_t stamp = (uint32_t)__shfl_sync(kFull, my_stamp, np);
                        // a PUT that finds no empty way evicts by stamp: bring the
                        // stamps up to date first (warp-uniform: every lane holds
                        // the same copy)
                        bool has_empty = false;
#pragma unroll
                        for (int w = 0; w < 8; ++w) has_empty |= keys[w] == 0;
                        if (!has_empty) fold();
                        const uint64_t out = cache_apply(keys, vals, lru, ver, dirty_kv, dirty_lru, k_, v_, 1u,
                                                         stamp, mk);
                        if ((int)lane == np) my_out = out;
                    }
                    pos = np + 1;
                }
            }
            if (in) {
                if (stopped) {
                    if (d->status) d->status[li] = kNotRun;
                } else {
                    if (d->out) static_cast<uint64_t *>(d->out)[li] = my_out;
                    if (d->order) d->order[li] = 2ull * (v0 + 1 + u);
                    if (d->status) d->status[li] = kCommitted;
                }
            }
            if (!stopped) n_commit += in ? 1u : 0u;
            if (cnt < 32) break;
        }
        asm volatile("cp.async.wait_all;" ::: "memory");
        if (stopped) continue;
        fold();
        {
            const uint32_t wm = __reduce_or_sync(kFull, mark_ways);
            dirty_lru |= wm;
            mk.val_read |= wm;
            mk.lru_write |= wm;
            if (__any_sync(kFull, any_get)) mk.keys_read = 1;
        }
        // write back what changed: lane w owns way w
        if (lane < 8) {
#pragma unroll
            for (int w = 0; w < 8; ++w)
                if ((int)lane == w) {
                    if (dirty_kv & (1u << w)) {
                        st_rlx_u64w(a.W + kw + 2 * w, keys[w]);
                        st_rlx_u64w(a.W + vb + 2 * w, vals[w]);
                    }
                    if (dirty_lru & (1u << w)) st_rlx32(a.W + lb + w, (int32_t)lru[w]);
                }
        }
        if (lane == 8 && ver != ver0) st_rlx32(a.W + res, (int32_t)ver);
        // read/write-set marks of the whole run, one range per lane
        if (lane == 9 && mk.keys_read) mark_range(a, kw, 16, false);
        if (lane == 10 && mk.lru_all_read) mark_range(a, lb, 8, false);
        if (lane == 11 && mk.ver_write) mark_range(a, res, 1, true);
        if (lane >= 12 && lane < 20) {
            const uint32_t w = lane - 12;
            if (mk.key_write & (1u << w)) mark_range(a, kw + 2 * w, 2, true);
            if (mk.val_write & (1u << w)) mark_range(a, vb + 2 * w, 2, true);
            else if (mk.val_read & (1u << w)) mark_range(a, vb + 2 * w, 2, false);
            if (mk.lru_write & (1u << w)) mark_range(a, lb + w, 1, true);
        }
    }
#pragma unroll
    for (int w = 16; w > 0; w >>= 1) n_commit += __shfl_xor_sync(kFull, n_commit, w);
    if (lane == 0 && n_commit) atomicAdd(a.counters + 0, n_commit);
}

}  // namespace

cudaError_t launch_ro_phase(const ExecArgs &e, unsigned long long *v0, int blocks, cudaStream_t s) {
    OrderArgs o{};
    o.e = e;
    o.v0 = v0;
    k_ord_ro<<<blocks, 256, 0, s>>>(o);
    return cudaGetLastError();
}

cudaError_t launch_ordered(const OrderArgs &o, int exec_blocks, int stream_blocks,
                           cudaStream_t s, cudaStream_t side, cudaEvent_t fork, cudaEvent_t join) {
    k_ord_count<<<stream_blocks, kScanThreads, 0, s>>>(o);
    // The read-only phase needs only the clock snapshot k_ord_count takes and
    // the launch-start STMR^W, which nothing changes before k_seg_exec: with a
    // side stream it runs beside the ordering pre-pass.
    const bool beside = side && fork && join;
    if (beside) {
        cudaError_t e0 = cudaEventRecord(fork, s);
        if (e0 == cudaSuccess) e0 = cudaStreamWaitEvent(side, fork, 0);
        if (e0 != cudaSuccess) return e0;
        k_ord_ro<<<stream_blocks, 256, 0, side>>>(o);
        e0 = cudaEventRecord(join, side);
        if (e0 != cudaSuccess) return e0;
    }
    // Every return from here on first joins the side stream back into s, so
    // that a failure during a stream capture ends the capture with its own
    // error instead of an unjoined fork.
    auto joined = [&](cudaError_t err) -> cudaError_t {
        if (beside) {
            const cudaError_t ej = cudaStreamWaitEvent(s, join, 0);
            if (err == cudaSuccess) err = ej;
        }
        return err;
    };
    const uint32_t max_blocks = (uint32_t)std::max(stream_blocks, 1);
    k_scan_totals<SumOp><<<1, kScanThreads, 0, s>>>(o.scan_tot, o.n_tx32, 0, 0ull);
    k_ord_emit<<<stream_blocks, kScanThreads, 0, s>>>(o);
    cudaError_t e = cudaGetLastError();
    e = radix_sort(o.keys0, o.vals0, o.keys1, o.vals1, o.n_acc, o.cap_acc, o.key_bits, o.hist,
                   o.scan_tot, o.n_hist, max_blocks, s);
    if (e != cudaSuccess) return joined(e);
    k_ord_runs<<<stream_blocks, 256, 0, s>>>(o);
    const uint32_t acc_grid = std::min((o.cap_acc + kScanTile - 1) / kScanTile, max_blocks);
    e = device_scan<PairMaxOp, false>(o.runs, o.runs, o.n_acc, 0, acc_grid, o.scan_tot, 0, s);
    if (e != cudaSuccess) return joined(e);
    k_ord_acc<<<stream_blocks, 256, 0, s>>>(o);
    if (beside) e = joined(cudaSuccess);
    else k_ord_ro<<<stream_blocks, 256, 0, s>>>(o);
    if (e != cudaSuccess) return e;
    e = cudaMemsetAsync(o.e.next, 0, sizeof(unsigned long long), s);
    if (e != cudaSuccess) return e;
    switch (o.seg_log2) {
    case 7: k_seg_exec<128><<<exec_blocks, 128 + 32, sizeof(SegSmem<128>), s>>>(o); break;
    case 8: k_seg_exec<256><<<exec_blocks, 256 + 32, sizeof(SegSmem<256>), s>>>(o); break;
    case 9: k_seg_exec<512><<<exec_blocks, 512 + 32, sizeof(SegSmem<512>), s>>>(o); break;
    default: return cudaErrorInvalidValue;
    }
    k_cache_gather<<<stream_blocks, 256, 0, s>>>(o);
    k_cache_runs<<<stream_blocks, 256, 0, s>>>(o);
    return cudaGetLastError();
}

namespace {
template <uint32_t SEG>
int seg_occupancy(int *blocks_per_sm) {
    cudaError_t e = cudaFuncSetAttribute(k_seg_exec<SEG>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)sizeof(SegSmem<SEG>));
    if (e != cudaSuccess) return (int)e;
    return (int)cudaOccupancyMaxActiveBlocksPerMultiprocessor(blocks_per_sm, k_seg_exec<SEG>, SEG + 32,
                                                              sizeof(SegSmem<SEG>));
}
}  // namespace

// Also raises the kernels' dynamic shared-memory limit; called once per
// context before the first launch.
int ordered_exec_occupancy(uint32_t seg, int *blocks_per_sm) {
    switch (seg) {
    case 128: return seg_occupancy<128>(blocks_per_sm);
    case 256: return seg_occupancy<256>(blocks_per_sm);
    case 512: return seg_occupancy<512>(blocks_per_sm);
    default: return (int)cudaErrorInvalidValue;
    }
}

}  // namespace hetm

// Validation, apply and merge kernels of a SHeTM round (Sec. IV-C, IV-D).
//
// All three stream an HBM-resident array once: the CPU write-set log (12-byte
// tuples) for validate/apply, STMR^W and STMR^S on the dirty chunks for the
// merge.  Loads do not allocate in L1, and every warp keeps its next loads in
// flight while it works on the current ones: apply and merge read 16-byte
// vectors, validation reads only the tuple fields it tests.

#include "hetm_internal.cuh"

namespace hetm {
namespace {

// A warp tile is 128 log tuples = 1536 B, loaded by three coalesced 512-byte
// vector instructions (lane l takes vectors l, 32 + l, 64 + l), so each
// sector of the log crosses L2 once.  The warp then swaps the tile through
// shared memory so that lane l owns tuples 4l..4l+3, three 16-byte vectors,
// in which tuple j of the lane sits at:
//   addr  q0.x q0.w q1.z q2.y
//   value q0.y q1.x q1.w q2.z
//   ts    q0.z q1.y q2.x q2.w
struct Tile {
    uint4 q0, q1, q2;
};

constexpr int kTileVec = 96;  // 16-byte vectors per tile

__device__ __forceinline__ Tile load_tile(const hetm_log_entry *log, uint64_t tile, unsigned lane) {
    const uint4 *p = reinterpret_cast<const uint4 *>(reinterpret_cast<const char *>(log) + tile * 1536ull);
    Tile t;
    t.q0 = ld_stream16(p + lane);
    t.q1 = ld_stream16(p + 32 + lane);
    t.q2 = ld_stream16(p + 64 + lane);
    return t;
}

// From the coalesced load order to per-lane tuple ownership (stage: this
// warp's kTileVec vectors of shared memory).
__device__ __forceinline__ Tile own_tile(const Tile &in, uint4 *stage, unsigned lane) {
    stage[lane] = in.q0;
    stage[32 + lane] = in.q1;
    stage[64 + lane] = in.q2;
    __syncwarp();
    Tile t;
    t.q0 = stage[3 * lane];
    t.q1 = stage[3 * lane + 1];
    t.q2 = stage[3 * lane + 2];
    __syncwarp();
    return t;
}

__device__ __forceinline__ void tile_fields(const Tile &t, uint32_t a[4], int32_t v[4], uint32_t s[4]) {
    a[0] = t.q0.x; a[1] = t.q0.w; a[2] = t.q1.z; a[3] = t.q2.y;
    v[0] = (int32_t)t.q0.y; v[1] = (int32_t)t.q1.x; v[2] = (int32_t)t.q1.w; v[3] = (int32_t)t.q2.z;
    s[0] = t.q0.z; s[1] = t.q1.y; s[2] = t.q2.x; s[3] = t.q2.w;
}

// Shared-memory filter of RS_bmp.  Every random probe of the L2-resident
// bitmap costs one 32-byte L2 sector and, while it is in flight, one L1
// line of the SM, and at 16.8M probes per validation those probes bound the
// kernel.  Each CTA therefore first looks a tuple's granule up in a 1M-bit
// hashed summary of the set granules (a Bloom filter with one hash,
// maintained next to RS_bmp) kept in its shared memory: a clear filter bit
// proves the granule is not in RS_bmp, and only tuples whose filter bit is
// set probe L2.  A CTA uses the filter only while at most 3/4 of its bits
// are set (else it would pass almost everything).  The filter is not made
// larger: the shared memory it takes comes out of the L1 lines that hold
// the probes and log loads in flight, and a 1.5M- or 1.75M-bit filter made
// the kernel slower on the validation-at-scale log.
__device__ __forceinline__ const uint32_t *load_filter(const uint32_t *filter, uint32_t *smem) {
    __shared__ uint32_t s_fill;
    if (threadIdx.x == 0) s_fill = 0;
    __syncthreads();
    if (!filter) return nullptr;
    const uint4 *src = reinterpret_cast<const uint4 *>(filter);
    uint4 *dst = reinterpret_cast<uint4 *>(smem);
    uint32_t fill = 0;
    for (uint32_t i = threadIdx.x; i < kFilterBits / 128; i += blockDim.x) {
        const uint4 v = __ldcg(src + i);
        dst[i] = v;
        fill += __popc(v.x) + __popc(v.y) + __popc(v.z) + __popc(v.w);
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) fill += __shfl_xor_sync(kFull, fill, o);
    if ((threadIdx.x & 31) == 0) atomicAdd(&s_fill, fill);
    __syncthreads();
    return s_fill <= kFilterBits / 4 * 3 ? smem : nullptr;
}

// Raise TS[a] to timestamp s.  A skewed log sends many tuples to a few hot
// words, and atomics on one word serialize in its L2 slice; a tuple whose
// timestamp is not above the value seen through L1 cannot change TS and
// skips the atomic.  TS only grows during the pass, so a stale cached value
// is at most the current one: a skip is always safe, at worst an atomic is
// not saved.
//
// The value a tuple sees (through L1, else returned by its atomic) is one
// TS held, and when it equals s the timestamp is repeated: by another tuple
// of the round or by one applied in an earlier round.  Of the tuples of one
// word carrying its newest timestamp all but the first to reach L2 see s,
// so a repeat of the timestamp the apply writes is always caught; a repeat
// below it may go unseen and changes nothing.
__device__ __forceinline__ uint32_t ts_seen(const uint32_t *ts, uint32_t a) {
    uint32_t seen;
    asm volatile("ld.global.ca.u32 %0, [%1];" : "=r"(seen) : "l"(ts + a));
    return seen;
}
// true when s repeats a timestamp TS holds for the word
__device__ __forceinline__ bool ts_raise(uint32_t *ts, uint32_t a, uint32_t s) {
    uint32_t seen = ts_seen(ts, a);
    if (seen < s) seen = atomicMax(ts + a, s);
    return seen == s;
}

// 4-byte load of a log field that is read once (no L1 allocation)
__device__ __forceinline__ uint32_t ld_field(const uint32_t *p) {
    uint32_t v;
    asm volatile("ld.global.nc.L1::no_allocate.u32 %0, [%1];" : "=r"(v) : "l"(p));
    return v;
}

// Validation (Sec. IV-C): flag = RS_bmp[granule(addr)] for every tuple, the
// flags bit-packed in log order, the hits counted.  kMax additionally raises
// TS[addr] to the tuple's timestamp (first pass of the apply).
//
// The log is read in groups of 32 consecutive tuples, lane l holding tuple
// 32g + l: one 4-byte load per lane fetches the group's addresses (384
// contiguous bytes, so each sector of the log crosses L2 once), and a warp
// ballot over the group's probes is directly its flag word.  Only the fields
// the pass uses are loaded (the timestamp only for kMax), and there is no
// staging buffer, which leaves the shared memory to the filter.  Each warp
// owns a contiguous range of groups and keeps kValGroups of them in flight:
// the next kValGroups groups' loads are issued before the current ones are
// probed.
constexpr int kValGroups = 4;

template <bool kMax>
__device__ __forceinline__ void validate_body(const hetm_log_entry *__restrict__ log, uint64_t n,
                                              const uint32_t *__restrict__ rs, uint32_t gshift,
                                              uint64_t n_words, uint32_t *__restrict__ flags,
                                              unsigned long long *count, uint32_t *ts, int *err,
                                              const uint32_t *filter, uint32_t *s_filter) {
    constexpr int U = kValGroups;
    const uint32_t *lw = reinterpret_cast<const uint32_t *>(log);  // 3 words per tuple
    const unsigned lane = threadIdx.x & 31u;
    const uint64_t warp = (blockIdx.x * (uint64_t)blockDim.x + threadIdx.x) >> 5;
    const uint64_t n_warps = (gridDim.x * (uint64_t)blockDim.x) >> 5;
    const uint64_t n_groups = (n + 31) / 32;
    const uint64_t g0 = warp * n_groups / n_warps, g1 = (warp + 1) * n_groups / n_warps;
    uint32_t hits = 0;
    bool bad = false, bad_ts = false;

    uint32_t a[U], s[U];
    bool v[U];
#pragma unroll
    for (int u = 0; u < U; ++u) {
        const uint64_t t = (g0 + u) * 32 + lane;
        v[u] = g0 + u < g1 && t < n;
        a[u] = v[u] ? ld_field(lw + 3 * t) : 0u;
        s[u] = kMax && v[u] ? ld_field(lw + 3 * t + 2) : 0u;
    }
    // the filter is copied while the first groups' loads are in flight
    const uint32_t *flt = load_filter(filter, s_filter);
    for (uint64_t g = g0; g < g1; g += U) {
        uint32_t na[U], ns[U];
        bool nv[U];
#pragma unroll
        for (int u = 0; u < U; ++u) {
            const uint64_t t = (g + U + u) * 32 + lane;
            nv[u] = g + U + u < g1 && t < n;
            na[u] = nv[u] ? ld_field(lw + 3 * t) : 0u;
            ns[u] = kMax && nv[u] ? ld_field(lw + 3 * t + 2) : 0u;
        }
        uint32_t gr[U], w[U];
        bool in[U];
#pragma unroll
        for (int u = 0; u < U; ++u) {
            in[u] = v[u] && a[u] < n_words;
            bad |= v[u] && !in[u];
            if (kMax) bad_ts |= in[u] && !ts_valid(s[u]);
            gr[u] = a[u] >> gshift;
            bool p = in[u];
            if (flt && p) {
                const uint32_t sl = filter_slot(gr[u]);
                p = (flt[sl >> 5] >> (sl & 31)) & 1u;
            }
            w[u] = p ? __ldg(rs + (gr[u] >> 5)) : 0u;
        }
        uint32_t seen[U];
        if (kMax) {
#pragma unroll
            for (int u = 0; u < U; ++u) seen[u] = in[u] && ts_valid(s[u]) ? ts_seen(ts, a[u]) : ~0u;
#pragma unroll
            for (int u = 0; u < U; ++u)
                if (seen[u] < s[u]) seen[u] = atomicMax(ts + a[u], s[u]);
        }
        uint32_t mine = 0;
#pragma unroll
        for (int u = 0; u < U; ++u) {
            const uint32_t b = __ballot_sync(kFull, (w[u] >> (gr[u] & 31)) & 1u);
            if (lane == (unsigned)u) mine = b;
        }
        hits += __popc(mine);
        if (flags && lane < (unsigned)U && g + lane < g1) flags[g + lane] = mine;
        if (kMax) {  // the atomics' old values, read last (see ts_raise)
#pragma unroll
            for (int u = 0; u < U; ++u)
                bad_ts |= in[u] && ts_valid(s[u]) && seen[u] == s[u];
        }
#pragma unroll
        for (int u = 0; u < U; ++u) {
            a[u] = na[u];
            s[u] = ns[u];
            v[u] = nv[u];
        }
    }
    if (bad) set_err(err, kErrAddr);
    if (bad_ts) set_err(err, kErrLogTs);
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) hits += __shfl_xor_sync(kFull, hits, o);
    if (lane == 0 && hits && count) atomicAdd(count, (unsigned long long)hits);
}

template <bool kMax>
__global__ void __launch_bounds__(kValThreads, 1) k_validate_round(const DevRound *rp, const uint32_t *rs,
                                                                   uint32_t gshift, uint64_t n_words,
                                                                   uint32_t *flags,
                                                                   unsigned long long *count,
                                                                   uint32_t *ts, int *err,
                                                                   const uint32_t *filter) {
    extern __shared__ uint4 s_dyn[];  // the filter
    validate_body<kMax>(rp->log, rp->n_log, rs, gshift, n_words, flags, count, ts, err, filter,
                        reinterpret_cast<uint32_t *>(s_dyn));
}

__global__ void __launch_bounds__(kValThreads, 1) k_validate_direct(const hetm_log_entry *log, uint64_t n,
                                                                    const uint32_t *rs, uint32_t gshift,
                                                                    uint64_t n_words, uint32_t *flags,
                                                                    unsigned long long *count, int *err,
                                                                    const uint32_t *filter) {
    extern __shared__ uint4 s_dyn[];  // the filter
    validate_body<false>(log, n, rs, gshift, n_words, flags, count, nullptr, err, filter,
                         reinterpret_cast<uint32_t *>(s_dyn));
}

// Early validation (Sec. IV-D): while the ordered executor runs, the round's
// CPU log (already on the device) is validated again and again against
// RS_bmp, whose bits the executor sets as transactions commit.  A hit means
// the round will conflict whatever else commits, and under GPU-loses its
// whole batch is rolled back: the watcher raises *stop and the executor
// takes no new segment and runs no further transaction.  The final
// validation still checks the whole log against the whole RS_bmp; the
// watcher only saves the time of work that would be discarded.  It reads
// RS_bmp through L2 (the executor's atomicOr lands there); a bit it misses
// is caught by the final validation.  Every CTA leaves when the executor has
// finished all its segments (*segs_done + 1 >= *segs_total), when the
// execution phase is over (*exec_over, set by the context stream after its
// last kernel), on a hit, or after budget_ns.
__global__ void __launch_bounds__(128) k_watch(const hetm_log_entry *__restrict__ log, uint64_t n,
                                               const uint32_t *rs, uint32_t gshift, uint64_t n_words,
                                               unsigned int *stop, const unsigned int *segs_done,
                                               const unsigned int *segs_total,
                                               const unsigned int *exec_over,
                                               unsigned long long budget_ns) {
    __shared__ int s_quit;
    const unsigned long long t0 = globaltimer_ns();
    const uint64_t stride = gridDim.x * (uint64_t)blockDim.x;
    for (uint32_t scan = 0;; ++scan) {
        bool hit = false;
        for (uint64_t i = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; i < n && !hit; i += stride) {
            const uint32_t a = __ldg(&log[i].addr);
            if (a < n_words) {
                const uint32_t g = a >> gshift;
                hit = (__ldcg(rs + (g >> 5)) >> (g & 31)) & 1u;
            }
        }
        if (hit) atomicExch(stop, 1u);
        __syncthreads();
        if (threadIdx.x == 0) {
            const unsigned int tot = *(volatile const unsigned int *)segs_total;
            const unsigned int done = *(volatile const unsigned int *)segs_done;
            s_quit = *(volatile unsigned int *)stop != 0 || (tot != 0 && done + 1 >= tot) ||
                     *(volatile const unsigned int *)exec_over != 0 || globaltimer_ns() - t0 > budget_ns;
        }
        __syncthreads();
        if (s_quit) return;
    }
}

// CPU-loses policy (Sec. IV-E): the CPU log is applied only when the whole
// validation came back clean, so the TS max runs as its own pass after
// validation and, like the apply, does nothing once a conflict was counted.
__global__ void __launch_bounds__(256) k_ts_max_if_clean(const DevRound *rp, uint32_t *ts,
                                                         uint64_t n_words,
                                                         const unsigned long long *conflicts,
                                                         int *err) {
    if (*(volatile const unsigned long long *)conflicts) return;
    const hetm_log_entry *log = rp->log;
    const uint64_t n = rp->n_log;
    const uint64_t stride = gridDim.x * (uint64_t)blockDim.x;
    bool bad_ts = false;
    for (uint64_t i = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; i < n; i += stride) {
        const uint32_t a = __ldg(&log[i].addr), s = __ldg(&log[i].ts);
        if (a >= n_words) continue;
        bad_ts |= !ts_valid(s) || ts_raise(ts, a, s);
    }
    if (bad_ts) set_err(err, kErrLogTs);
}

// Apply, second pass (Sec. IV-C): after TS holds the newest timestamp of
// every logged word, exactly the tuple carrying it writes its value into
// STMR^W and into the shadow STMR^S (Sec. IV-D: the shadow plus the CPU log
// is the CPU's state).  Out-of-range tuples were reported by validation,
// timestamps out of range or repeated by the timestamp pass.
// skip_if (may be null): the round's conflict count; a nonzero count skips
// the apply (CPU-loses policy).
__global__ void __launch_bounds__(256) k_apply(const DevRound *rp, const uint32_t *__restrict__ ts,
                                               int32_t *__restrict__ W, int32_t *__restrict__ S,
                                               uint64_t n_words, const unsigned long long *skip_if) {
    if (skip_if && *(volatile const unsigned long long *)skip_if) return;
    __shared__ uint4 s_stage[256 / 32 * kTileVec];
    const hetm_log_entry *log = rp->log;
    const uint64_t n = rp->n_log;
    const unsigned lane = threadIdx.x & 31u;
    uint4 *stage = s_stage + (threadIdx.x >> 5) * kTileVec;
    const uint64_t warp = (blockIdx.x * (uint64_t)blockDim.x + threadIdx.x) >> 5;
    const uint64_t n_warps = (gridDim.x * (uint64_t)blockDim.x) >> 5;
    const uint64_t n_tiles = n / 128;
    uint64_t c = warp;
    Tile next;
    if (c < n_tiles) next = load_tile(log, c, lane);
    for (; c < n_tiles; c += n_warps) {
        const Tile cur = own_tile(next, stage, lane);
        if (c + n_warps < n_tiles) next = load_tile(log, c + n_warps, lane);
        uint32_t a[4], s[4];
        int32_t v[4];
        tile_fields(cur, a, v, s);
        bool ok[4];
        uint32_t t[4];
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            ok[j] = a[j] < n_words && ts_valid(s[j]);
            t[j] = ok[j] ? __ldcg(ts + a[j]) : 0u;
        }
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            if (ok[j] && t[j] == s[j]) {
                W[a[j]] = v[j];
                S[a[j]] = v[j];
            }
        }
    }
    if (warp == n_warps - 1) {
        for (uint64_t i = n_tiles * 128 + lane; i < n; i += 32) {
            const uint32_t a = log[i].addr, s = log[i].ts;
            if (a < n_words && ts_valid(s) && __ldcg(ts + a) == s) {
                W[a] = log[i].value;
                S[a] = log[i].value;
            }
        }
    }
}

// Merge (Sec. IV-C Merge Phase, Sec. IV-D): every WS_bmp chunk is copied
// W -> S when validation succeeded (the GPU's speculative commits become
// final) or S -> W when it failed (the GPU batch is undone; S already holds
// start + CPU writes).  Warps walk the chunks: a clean chunk costs one
// (cached) bitmap load, so the cost follows the dirty bytes; a dirty chunk
// is copied with 16-byte vectors, 4 in flight per lane.  Chunks smaller
// than a warp's 32 vectors are packed several to a warp.
__device__ __forceinline__ bool chunk_dirty(const uint32_t *ws, uint64_t c) {
    return (__ldg(ws + (c >> 5)) >> (c & 31)) & 1u;
}

__global__ void __launch_bounds__(256) k_merge(const uint32_t *__restrict__ ws, uint32_t cshift,
                                               int32_t *W, int32_t *S, uint64_t n_words,
                                               const unsigned long long *conflicts, int force,
                                               unsigned long long *dirty_count, const int *err) {
    // an execution phase that ran out of its time budget is undone like a
    // batch that lost a conflict (its transactions ran only in part)
    const bool conflict =
        (err && (*err & kErrTimeout)) || (force >= 0 ? force != 0 : (*conflicts != 0ull));
    const uint4 *src = reinterpret_cast<const uint4 *>(conflict ? S : W);
    uint4 *dst = reinterpret_cast<uint4 *>(conflict ? W : S);
    const unsigned lane = threadIdx.x & 31u;
    const uint64_t tid = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x;
    const uint64_t n_threads = gridDim.x * (uint64_t)blockDim.x;
    const uint64_t warp = tid >> 5, n_warps = n_threads >> 5;
    const uint64_t n_vec = n_words / 4;
    const uint64_t wpc = 1ull << cshift;              // words per chunk (>= 4)
    const uint64_t vpc = wpc / 4;                     // vectors per chunk
    const uint64_t n_chunks = (n_words + wpc - 1) / wpc;
    if (vpc >= 32) {
        for (uint64_t c = warp; c < n_chunks; c += n_warps) {
            if (!chunk_dirty(ws, c)) continue;
            const uint64_t v0 = c * vpc;
            const uint64_t v1 = v0 + vpc < n_vec ? v0 + vpc : n_vec;
            for (uint64_t v = v0 + lane; v < v1; v += 128) {
                uint4 r[4];
#pragma unroll
                for (int k = 0; k < 4; ++k)
                    if (v + 32u * k < v1) r[k] = __ldcs(src + v + 32u * k);
#pragma unroll
                for (int k = 0; k < 4; ++k)
                    if (v + 32u * k < v1) __stcs(dst + v + 32u * k, r[k]);
            }
        }
    } else {
        const uint64_t per = 32 / vpc;  // chunks per warp step
        for (uint64_t c0 = warp * per; c0 < n_chunks; c0 += n_warps * per) {
            const uint64_t c = c0 + lane / vpc;
            const uint64_t v = c * vpc + lane % vpc;
            if (c < n_chunks && v < n_vec && chunk_dirty(ws, c)) __stcs(dst + v, __ldcs(src + v));
        }
    }
    // the last n_words % 4 words
    if (tid == 0) {
        for (uint64_t w = n_vec * 4; w < n_words; ++w) {
            if (chunk_dirty(ws, w >> cshift)) {
                int32_t *d = conflict ? W : S;
                const int32_t *s = conflict ? S : W;
                d[w] = s[w];
            }
        }
    }
    if (dirty_count) {
        const uint64_t n_ws = (n_chunks + 31) / 32;
        unsigned long long cnt = 0;
        for (uint64_t i = tid; i < n_ws; i += n_threads) cnt += __popc(ws[i]);
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) cnt += __shfl_xor_sync(kFull, cnt, o);
        if (lane == 0 && cnt) atomicAdd(dirty_count, cnt);
    }
}

// Planted GPU accesses: non-transactional writes (or reads, vals == NULL)
// recorded in RS_bmp, and writes also in WS_bmp, as a committing GPU
// transaction would (Sec. IV-B, IV-C).
__global__ void k_mark(const uint32_t *__restrict__ addr, const int32_t *__restrict__ vals,
                       uint64_t n, int32_t *W, uint64_t n_words, uint32_t *rs, uint32_t *filter,
                       uint32_t gshift, uint32_t *ws, uint32_t cshift, int *err) {
    const uint64_t stride = gridDim.x * (uint64_t)blockDim.x;
    for (uint64_t i = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; i < n; i += stride) {
        uint32_t a = addr[i];
        if (a >= n_words) {
            set_err(err, kErrAddr);
            continue;
        }
        rs_mark(rs, filter, a >> gshift);
        if (vals) {
            W[a] = vals[i];
            uint32_t ch = a >> cshift;
            atomicOr(ws + (ch >> 5), 1u << (ch & 31));
        }
    }
}

}  // namespace

constexpr size_t kValSmem = kFilterBits / 8;

cudaError_t validate_setup() {
    const int smem = (int)kValSmem;
    cudaError_t e = cudaFuncSetAttribute(k_validate_round<true>,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
    if (e == cudaSuccess)
        e = cudaFuncSetAttribute(k_validate_round<false>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
    if (e == cudaSuccess)
        e = cudaFuncSetAttribute(k_validate_direct, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
    return e;
}

cudaError_t launch_validate(const DevRound *rp, const uint32_t *rs, uint32_t gshift,
                            uint64_t n_words, uint32_t *flags, unsigned long long *count,
                            uint32_t *ts, int *err, const uint32_t *filter, int blocks,
                            cudaStream_t s) {
    const size_t smem = kValSmem;
    if (ts)
        k_validate_round<true><<<blocks, kValThreads, smem, s>>>(rp, rs, gshift, n_words, flags, count,
                                                                 ts, err, filter);
    else
        k_validate_round<false><<<blocks, kValThreads, smem, s>>>(rp, rs, gshift, n_words, flags, count,
                                                                  ts, err, filter);
    return cudaGetLastError();
}

cudaError_t launch_watch(const hetm_log_entry *log, uint64_t n, const uint32_t *rs, uint32_t gshift,
                         uint64_t n_words, unsigned int *stop, const unsigned int *segs_done,
                         const unsigned int *segs_total, const unsigned int *exec_over,
                         unsigned long long budget_ns, int blocks, cudaStream_t s) {
    k_watch<<<blocks, 128, 0, s>>>(log, n, rs, gshift, n_words, stop, segs_done, segs_total, exec_over,
                                   budget_ns);
    return cudaGetLastError();
}

cudaError_t launch_validate_direct(const hetm_log_entry *log, uint64_t n, const uint32_t *rs,
                                   uint32_t gshift, uint64_t n_words, uint32_t *flags,
                                   unsigned long long *count, int *err, const uint32_t *filter,
                                   int blocks, cudaStream_t s) {
    const size_t smem = kValSmem;
    k_validate_direct<<<blocks, kValThreads, smem, s>>>(log, n, rs, gshift, n_words, flags, count, err,
                                                        filter);
    return cudaGetLastError();
}

cudaError_t launch_apply(const DevRound *rp, const uint32_t *ts, int32_t *W, int32_t *S,
                         uint64_t n_words, int blocks, cudaStream_t s,
                         const unsigned long long *skip_if) {
    k_apply<<<blocks, 256, 0, s>>>(rp, ts, W, S, n_words, skip_if);
    return cudaGetLastError();
}

cudaError_t launch_ts_max_if_clean(const DevRound *rp, uint32_t *ts, uint64_t n_words,
                                   const unsigned long long *conflicts, int *err, int blocks,
                                   cudaStream_t s) {
    k_ts_max_if_clean<<<blocks, 256, 0, s>>>(rp, ts, n_words, conflicts, err);
    return cudaGetLastError();
}

cudaError_t launch_merge(const uint32_t *ws, uint32_t cshift, int32_t *W, int32_t *S,
                         uint64_t n_words, const unsigned long long *conflicts, int force,
                         unsigned long long *dirty_count, int blocks, cudaStream_t s,
                        const int *err) {
    k_merge<<<blocks, 256, 0, s>>>(ws, cshift, W, S, n_words, conflicts, force, dirty_count, err);
    return cudaGetLastError();
}

cudaError_t launch_mark(const uint32_t *addr, const int32_t *vals, uint64_t n, int32_t *W,
                        uint64_t n_words, uint32_t *rs, uint32_t *filter, uint32_t gshift,
                        uint32_t *ws, uint32_t cshift, int *err, int blocks, cudaStream_t s) {
    if (n == 0) return cudaSuccess;
    k_mark<<<blocks, 256, 0, s>>>(addr, vals, n, W, n_words, rs, filter, gshift, ws, cshift, err);
    return cudaGetLastError();
}

}  // namespace hetm

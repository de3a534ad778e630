// Internal declarations of the SHeTM round library (CUDA, sm_103a).
#pragma once

#include <cuda_runtime.h>
#include <nvtx3/nvToolsExt.h>
#include <stdint.h>

#include "hetm.h"

namespace hetm {

// Host-side NVTX range over one library call (what the host enqueued, and
// when): visible to a profiler that is attached, free otherwise.
struct Range {
    explicit Range(const char *name) { nvtxRangePushA(name); }
    ~Range() { nvtxRangePop(); }
    Range(const Range &) = delete;
    Range &operator=(const Range &) = delete;
};

constexpr uint8_t kCommitted = 1;
constexpr uint8_t kGaveUp = 2;
constexpr uint8_t kNotRun = 3;  // the execution phase stopped early (early validation)
constexpr unsigned kFull = 0xffffffffu;

// Device-side batch descriptor (one per admitted batch).
struct DevBatch {
    uint32_t workload;
    uint32_t n_tx;
    const void *tx;
    uint64_t *order;
    uint8_t *status;
    void *out;
    uint32_t txid_base;
    uint32_t word_base;
};

// Per-round sizes, read by the kernels from device memory so that one
// captured graph serves every round.
struct DevRound {
    uint64_t total_tx;            // transactions over all batches
    uint64_t n_log;               // CPU tuples to validate
    const hetm_log_entry *log;    // device log of this round
    uint32_t n_batches;
    uint32_t pad;
};

// Device error word: a set of bits, each site ORs its own in, so that no
// error hides another (a timeout must still undo the batch after an address
// error of the same or an earlier round).
constexpr int kErrAddr = 1;
constexpr int kErrTimeout = 2;
constexpr int kErrLogTs = 4;  // a CPU tuple's timestamp out of range, or repeated

// HETM_ETIMEOUT when the execution phase ran out of its budget (whatever else
// went wrong), HETM_EDEVICE for an out-of-range address, HETM_EINVAL for a
// CPU log that broke the timestamp rule, else HETM_OK.
inline int err_code(int bits) {
    if (bits & kErrTimeout) return HETM_ETIMEOUT;
    if (bits & kErrAddr) return HETM_EDEVICE;
    return bits ? HETM_EINVAL : HETM_OK;
}

// CPU timestamps are 1 .. 2^32 - 2 (0 is TS's "none yet").
__host__ __device__ __forceinline__ bool ts_valid(uint32_t ts) { return ts - 1u < 0xFFFFFFFEu; }

// Arguments of the executor kernel.
struct ExecArgs {
    int32_t *W;
    uint64_t n_words;
    unsigned long long *locks;
    uint32_t lock_mask;
    uint32_t lock_shift;
    unsigned long long *gv;        // global commit-version clock
    uint32_t *rs;                  // RS_bmp
    uint32_t *filter;              // its shared-memory filter (may be null)
    uint32_t gshift;               // granule(a) = a >> gshift
    uint32_t *ws;                  // WS_bmp
    uint32_t cshift;               // chunk(a) = a >> cshift
    const DevRound *rp;
    const DevBatch *batches;
    const uint64_t *prefix;        // n_batches + 1 prefix sums of n_tx
    unsigned long long *next;      // work counter (reset per launch)
    uint32_t max_attempts;
    unsigned long long budget_ns;  // wall-clock bound of one launch
    unsigned long long *counters;  // [0] committed [1] gave up [2] aborts
    int *err;
    // early validation (null when off): the watcher's stop flag, segments
    // the ordered phase finished, and its segment count + 1 (0 = not known yet)
    const unsigned int *stop;
    unsigned int *segs_done, *segs_total;
    uint32_t cache_log2_sets;
    uint64_t key_base, val_base, lru_base, ver_base;
    // optimistic executor: W1 read-only transactions already ran (lock-free,
    // on the launch-start state, before every update of the launch)
    uint32_t skip_ro;
    // optimistic executor (null otherwise): the read-only phase lists the
    // launch indices it did not run (rest[0 .. *rest_n)), so that the STM
    // draws only those; a launch of more than rest_cap transactions is not
    // listed and the STM draws every index
    uint32_t *rest;
    unsigned long long *rest_n;
    uint64_t rest_cap;
    // 0: commits record nothing in RS_bmp / WS_bmp (the uninstrumented
    // executor that instrumentation costs are measured against, Sec. V-A)
    uint32_t instrument;
};

// One transaction of the ordered phase (indexed by its rank in that phase).
// Slot k of a word transaction is one distinct word; turn[k] carries the
// access's position among the accesses to its resource plus flags.
constexpr uint32_t kSegMin = 128, kSegMax = 512;  // CTA segment sizes (threads)
constexpr uint32_t kTurnMask = 0x0FFFFFFFu;
constexpr uint32_t kFWriter = 1u << 31;     // the access writes the resource
constexpr uint32_t kFLast = 1u << 30;       // last access of the word in the launch
constexpr uint32_t kFLocal = 1u << 29;      // predecessor is in the same segment
constexpr uint32_t kFPublish = 1u << 28;    // successor is in a later segment
struct __align__(16) OrdRec {
    uint32_t u;        // launch index
    uint32_t meta;     // n (bits 0-2) | workload (3-4) | map (8-15) | batch (16-31)
    uint32_t aux;      // W1: txid; bank: amount
    uint32_t li;       // index inside its batch
    uint32_t addr[4];  // distinct words (bank: src, dst); cache: set version word
    uint32_t res[4];   // resource id (index of its run in the sorted access list)
    uint32_t turn[4];  // position | flags
    uint32_t src[4];   // local predecessor: (thread << 2) | slot
};
static_assert(sizeof(OrdRec) == 80, "80-byte record");

// Scratch of the ordered executor (capacities fixed at context creation).
struct OrderArgs {
    ExecArgs e;
    uint64_t *scan_tot;         // per-tile totals of the scans (and of the ranking)
    uint32_t *keys0, *vals0;    // [cap_acc] access list, sorted in place
    uint32_t *keys1, *vals1;    // [cap_acc] radix-sort ping-pong buffers
    uint64_t *hist;             // [256 * ceil(cap_acc / 2048)] digit counts
    uint64_t *runs;             // [cap_acc] (run head << 32 | last writer + 1), max-scanned
    OrdRec *rec;                // [cap_tx] ordered-phase transactions by rank
    unsigned long long *packed; // [cap_acc] per resource: (turns done << 32) | value
    uint32_t *n_acc, *n_ord, *n_tx32;
    uint32_t *n_hist;           // the radix sort's histogram length for the launch
    uint32_t *cache_heads;      // [cap_tx] first access of every cache set's run
    uint32_t *n_cache_runs;     //   their number
    unsigned long long *v0;     // commit clock before the launch
    uint32_t cap_tx, cap_acc, key_bits;
    uint32_t seg_log2;          // transactions per CTA segment = 2^seg_log2 (7, 8 or 9)
    // W2 updates of the launch (null: none can occur), run under the STM
    // after the ordered phase: w2list[0 .. *w2n)
    uint32_t *w2list;
    unsigned long long *w2n;
};

// ------------------------------------------------------------------ PTX helpers
__device__ __forceinline__ unsigned long long ld_rlx64(const unsigned long long *p) {
    unsigned long long v;
    asm volatile("ld.relaxed.gpu.global.u64 %0, [%1];" : "=l"(v) : "l"(p) : "memory");
    return v;
}
__device__ __forceinline__ int32_t ld_rlx32(const int32_t *p) {
    int32_t v;
    asm volatile("ld.relaxed.gpu.global.s32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}
__device__ __forceinline__ uint64_t ld_rlx_u64(const int32_t *p) {
    unsigned long long v;
    asm volatile("ld.relaxed.gpu.global.u64 %0, [%1];" : "=l"(v) : "l"(p) : "memory");
    return v;
}
__device__ __forceinline__ void st_rlx32(int32_t *p, int32_t v) {
    asm volatile("st.relaxed.gpu.global.s32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}
__device__ __forceinline__ void st_rlx_u64w(int32_t *p, uint64_t v) {
    asm volatile("st.relaxed.gpu.global.u64 [%0], %1;" ::"l"(p), "l"(v) : "memory");
}
__device__ __forceinline__ void st_rlx64(unsigned long long *p, unsigned long long v) {
    asm volatile("st.relaxed.gpu.global.u64 [%0], %1;" ::"l"(p), "l"(v) : "memory");
}
__device__ __forceinline__ void fence_gpu() { asm volatile("fence.acq_rel.gpu;" ::: "memory"); }
__device__ __forceinline__ unsigned lanemask_lt() {
    unsigned m;
    asm("mov.u32 %0, %%lanemask_lt;" : "=r"(m));
    return m;
}

// streaming 16-byte load that does not allocate in L1
__device__ __forceinline__ uint4 ld_stream16(const void *p) {
    uint4 v;
    asm volatile("ld.global.nc.L1::no_allocate.v4.u32 {%0,%1,%2,%3}, [%4];"
                 : "=r"(v.x), "=r"(v.y), "=r"(v.z), "=r"(v.w)
                 : "l"(p));
    return v;
}

__device__ __forceinline__ unsigned long long globaltimer_ns() {
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

__device__ __forceinline__ void set_err(int *err, int bit) {
    if (err && !(*(volatile int *)err & bit)) atomicOr(err, bit);
}

// SplitMix64 finalizer (Steele, Lea & Flood 2014): the cache's set hash.
__device__ __forceinline__ uint64_t splitmix_fin(uint64_t z) {
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
}

// ----------------------------------------------------------- host launchers
cudaError_t launch_exec(const ExecArgs &a, int blocks, int threads, cudaStream_t s);
int exec_occupancy(int threads, int *blocks_per_sm);
// side / fork / join (all or none): the read-only phase runs on `side`, beside
// the ordering pre-pass on `s`
cudaError_t launch_ordered(const OrderArgs &o, int exec_blocks, int stream_blocks, cudaStream_t s,
                           cudaStream_t side = nullptr, cudaEvent_t fork = nullptr,
                           cudaEvent_t join = nullptr);
// W1 read-only transactions of a launch, lock-free on the launch-start state
// (commit key 2 * *v0 + 1: before every update of the launch)
cudaError_t launch_ro_phase(const ExecArgs &e, unsigned long long *v0, int blocks, cudaStream_t s);
int ordered_exec_occupancy(uint32_t seg, int *blocks_per_sm);

// validation kernels: one CTA of kValThreads per SM, RS_bmp filter in shared memory
constexpr uint32_t kFilterBits = 1u << 20;  // 128 KiB
constexpr int kValThreads = 1024;

// Filter of RS_bmp (a one-hash Bloom filter of the set granules), kept next
// to RS_bmp: every site that sets a granule bit also sets the granule's
// filter bit, and both are cleared together after the merge.
__device__ __forceinline__ uint32_t filter_slot(uint32_t g) {
    uint32_t h = g * 0x9E3779B1u;
    h ^= h >> 15;
    h *= 0x85EBCA77u;
    h ^= h >> 13;
    return __umulhi(h, kFilterBits);
}

// Set granule g in RS_bmp (and its filter bit), skipping bits already set.
__device__ __forceinline__ void rs_mark(uint32_t *rs, uint32_t *filter, uint64_t g) {
    const uint32_t m = 1u << (g & 31);
    if (rs[g >> 5] & m) return;
    atomicOr(rs + (g >> 5), m);
    if (filter) {
        const uint32_t sl = filter_slot((uint32_t)g);
        atomicOr(filter + (sl >> 5), 1u << (sl & 31));
    }
}
cudaError_t validate_setup();
cudaError_t launch_watch(const hetm_log_entry *log, uint64_t n, const uint32_t *rs, uint32_t gshift,
                         uint64_t n_words, unsigned int *stop, const unsigned int *segs_done,
                         const unsigned int *segs_total, const unsigned int *exec_over,
                         unsigned long long budget_ns, int blocks, cudaStream_t s);
cudaError_t launch_validate(const DevRound *rp, const uint32_t *rs, uint32_t gshift,
                            uint64_t n_words, uint32_t *flags, unsigned long long *count,
                            uint32_t *ts, int *err, const uint32_t *filter, int blocks,
                            cudaStream_t s);
cudaError_t launch_validate_direct(const hetm_log_entry *log, uint64_t n, const uint32_t *rs,
                                   uint32_t gshift, uint64_t n_words, uint32_t *flags,
                                   unsigned long long *count, int *err, const uint32_t *filter,
                                   int blocks, cudaStream_t s);
cudaError_t launch_apply(const DevRound *rp, const uint32_t *ts, int32_t *W, int32_t *S,
                         uint64_t n_words, int blocks, cudaStream_t s,
                         const unsigned long long *skip_if = nullptr);
cudaError_t launch_ts_max_if_clean(const DevRound *rp, uint32_t *ts, uint64_t n_words,
                                   const unsigned long long *conflicts, int *err, int blocks,
                                   cudaStream_t s);
// err (may be null): a kErrTimeout there undoes the batch (S -> W) whatever
// conflicts / force say
cudaError_t launch_merge(const uint32_t *ws, uint32_t cshift, int32_t *W, int32_t *S,
                         uint64_t n_words, const unsigned long long *conflicts, int force,
                         unsigned long long *dirty_count, int blocks, cudaStream_t s,
                         const int *err);
// the serving loop's transactions-per-round capacity
uint64_t server_max_round_tx(const hetm_server *s);
// rounds launched by hetm_round(ctx, NULL) and not yet collected
int ctx_open_rounds(const hetm_ctx *c);
cudaError_t launch_mark(const uint32_t *addr, const int32_t *vals, uint64_t n, int32_t *W,
                        uint64_t n_words, uint32_t *rs, uint32_t *filter, uint32_t gshift,
                        uint32_t *ws, uint32_t cshift, int *err, int blocks, cudaStream_t s);

}  // namespace hetm

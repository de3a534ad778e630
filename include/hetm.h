/*
 * hetm.h -- C ABI of the GPU side of a Speculative HeTM (SHeTM)
 * synchronization round, after Castro, Romano, Ilic and Khan, "HeTM:
 * Transactional Memory for Heterogeneous Systems" (arXiv 1905.00661).
 *
 * A round (Sec. IV-C) has three phases:
 *   execution  -- GPU transaction batches run speculatively on the working
 *                 copy STMR^W; every commit ORs the granules it read or wrote
 *                 into RS_bmp and the transfer chunks it wrote into WS_bmp
 *                 (Sec. IV-B "GPU instrumentation"; writes also go to RS_bmp,
 *                 Sec. IV-C, so one test covers write-write conflicts);
 *   validation -- the CPU write-set log of <addr, value, ts> tuples, shipped
 *                 to the device in chunks (Sec. IV-D), is tested against
 *                 RS_bmp; a hit marks the round as conflicting, and every
 *                 tuple is applied anyway to STMR^W and the shadow STMR^S when
 *                 its timestamp is the newest for its word (array TS);
 *   merge      -- the chunks marked in WS_bmp are copied W -> S when
 *                 validation succeeded and S -> W when it failed, undoing the
 *                 GPU batch (GPU-loses policy, Sec. IV-C; shadow-copy
 *                 rollback, Sec. IV-D).  Afterwards W == S.
 *
 * Conventions for every call:
 *   - return 0 (HETM_OK) or a negative HETM_E* code; hetm_strerror() names it;
 *   - "device pointer" = memory of the context's CUDA device (cudaMalloc,
 *     a torch CUDA tensor's data_ptr(), ...); "host pointer" = any host
 *     memory unless stated as pinned;
 *   - the library never takes ownership of caller memory; caller device
 *     buffers passed to an asynchronous call must stay valid until that
 *     work has completed on the context stream (hetm_sync);
 *   - one controller thread drives a context; only hetm_cpu_log_write may be
 *     called concurrently, from distinct `thread` ids.
 */
#ifndef HETM_H
#define HETM_H

#include <stddef.h>
#include <stdint.h>

#if defined(__GNUC__)
#define HETM_API __attribute__((visibility("default")))
#else
#define HETM_API
#endif

#ifdef __cplusplus
extern "C" {
#endif

/* ---------------------------------------------------------------- errors */
#define HETM_OK 0
#define HETM_EINVAL (-1)    /* bad argument or precondition violated; from a
                               round: a CPU tuple's ts out of range or
                               repeated (hetm_log_entry), reported until
                               hetm_load */
#define HETM_ENOMEM (-2)    /* device or pinned host allocation failed        */
#define HETM_ECAPACITY (-3) /* a fixed-capacity buffer or table is full       */
#define HETM_ETIMEOUT (-4)  /* a bounded device wait gave up                  */
#define HETM_ECUDA (-5)     /* a CUDA runtime call failed                     */
#define HETM_EBUSY (-6)     /* not admitted now (memory or slots); retry later */
#define HETM_EDEVICE (-7)   /* a kernel met an out-of-range address; the
                               offending item was skipped, state is undefined;
                               the context keeps reporting it until hetm_load */

HETM_API const char *hetm_strerror(int code);

/* --------------------------------------------------------------- records */
/* CPU write-set log tuple (Sec. IV-B, CPU instrumentation).  12 bytes,
 * packed.  `ts` totally orders the writes to one word: 1 <= ts < 2^32 - 1
 * and unique per word over the lifetime of the context (until hetm_load).
 * A tuple is applied when its ts is the newest of its word.  The device
 * checks the rule where it raises TS (under CPU_LOSES only in rounds that
 * validate clean), and the round then reports HETM_EINVAL: for a ts out of
 * range (the tuple is validated, not applied), and for a ts repeated on the
 * newest ts of a word, within the round or from an earlier one (the word
 * holds one of the values concerned; for a tie within the round W and S
 * need not hold the same one).  A repeat below a word's newest ts changes
 * nothing and may go unreported. */
typedef struct hetm_log_entry {
    uint32_t addr;  /* word index into the STMR, < stmr_words */
    int32_t value;  /* value the CPU transaction wrote          */
    uint32_t ts;    /* commit timestamp of the CPU transaction  */
} hetm_log_entry;

/* Transactional workloads run by the GPU executor. */
#define HETM_WL_BANK 1  /* hetm_bank_tx                      */
#define HETM_WL_RMW 2   /* hetm_rmw_tx (W1 of Sec. V-A)       */
#define HETM_WL_CACHE 3 /* hetm_cache_req (Sec. V-D)          */
#define HETM_WL_W2 4    /* hetm_w2_tx (W2 of Sec. V-A)        */

/* bank transfer: bal[src] -= amount; bal[dst] += amount (int32, wrapping).
 * Accounts are words base+src, base+dst with base = hetm_batch.word_base. */
typedef struct hetm_bank_tx {
    uint32_t src, dst;
    int32_t amount;
} hetm_bank_tx;

/* Four word reads; with flags bit 0 set the transaction also writes
 * s + j + txid to its j-th word, s = the 32-bit sum it read, txid =
 * hetm_batch.txid_base + index.  out (int32) receives s. */
typedef struct hetm_rmw_tx {
    uint32_t addr[4];
    uint32_t flags;
} hetm_rmw_tx;

/* W2 of Sec. V-A: like W1, but every transaction reads 40 words.  A
 * read-only transaction outputs the 32-bit sum s of its 40 words; with flags
 * bit 0 set it also writes s + j + txid to its j-th word for j = 0..3 (the
 * update transactions of both workloads update 4 positions).  The 40 words
 * of one transaction must be distinct.  176 bytes (16-byte multiple).
 * Read-only W2 transactions run in either executor's read-only phase
 * (lock-free, on the launch-start state).  Updates run under the STM with
 * their 36 read-only words validated against a clock snapshot: in
 * HETM_EXEC_OPTIMISTIC with the launch's other updates, in
 * HETM_EXEC_ORDERED after the ordered phase, serialized after every other
 * transaction of the launch. */
typedef struct hetm_w2_tx {
    uint32_t addr[40];
    uint32_t flags;
    uint32_t pad[3];
} hetm_w2_tx;

/* Object-cache request, op 0 = GET, 1 = PUT.  Set = SplitMix64 finalizer of
 * key mod 2^cache_log2_sets.  GET hit: out = value and the GPU LRU stamp of
 * the slot is set to the commit version; miss: out = UINT64_MAX.  PUT: hit
 * way, else the first empty way (key 0), else the way with the smallest GPU
 * LRU stamp (lowest way on ties) takes key and value, its stamp becomes the
 * commit version and the set version word is incremented; out = way.
 * Requests conflict only with requests on the same set; word transactions
 * (bank, W1) of the same execution phase must not address the cache regions
 * (the ordered executor orders words and sets separately). */
typedef struct hetm_cache_req {
    uint64_t key;
    uint64_t value;
    uint32_t op;
    uint32_t pad;
} hetm_cache_req;

/* ---------------------------------------------------------- configuration */
/* GPU guest TM of the execution phase (any TM that keeps committed
 * transactions serializable may serve, Sec. IV-B):
 *   ORDERED    -- the serial order is fixed before execution: W1 read-only
 *                 transactions first (lock-free, on the phase-start state),
 *                 then every other transaction in index order, each running
 *                 when its declared words / cache set reach its turn.  No
 *                 aborts.  Needs max_round_tx capacity (~200 B per tx).
 *   OPTIMISTIC -- word-based STM with striped version locks (try-lock for
 *                 known write sets, validated reads, bounded retries). */
#define HETM_EXEC_ORDERED 0
#define HETM_EXEC_OPTIMISTIC 1

typedef struct hetm_config {
    uint32_t ws_chunk_bytes;   /* WS_bmp / merge chunk, power of two >= 16
                                  (Sec. IV-D uses 16 KB); default 16384    */
    uint32_t lock_log2;        /* 2^lock_log2 striped version locks; 22   */
    uint32_t lock_shift;       /* words per lock stripe = 2^lock_shift; 0  */
    uint32_t exec_blocks;      /* executor grid; 0 = one wave (SMs x occ.) */
    uint32_t exec_threads;     /* executor CTA size; 256.  Ordered mode: 128,
                                  256 or 512 transactions per CTA segment;
                                  optimistic: multiple of 32, <= 256          */
    uint32_t max_attempts;     /* per-transaction attempt bound; 1<<20     */
    uint32_t cpu_threads;      /* number of per-thread CPU logs; 8         */
    uint32_t log_chunk_bytes;  /* H2D shipping chunk, multiple of 12; 49152 */
    uint64_t log_capacity;     /* device log entries per round; 1<<24      */
    uint64_t cpu_log_capacity; /* pinned entries per CPU thread per round; 1<<22 */
    uint32_t max_batches;      /* pending batches per round; 4096          */
    uint32_t cache_log2_sets;  /* object-cache layout (HETM_WL_CACHE)      */
    uint64_t cache_key_base, cache_val_base, cache_lru_base, cache_ver_base;
    uint32_t exec_mode;        /* HETM_EXEC_ORDERED (default) or HETM_EXEC_OPTIMISTIC */
    uint32_t early_validate;   /* 1: early validation (Sec. IV-D) in hetm_round --
                                  while the ordered executor runs, a watcher
                                  kernel re-scans the round's CPU log against
                                  RS_bmp as commits set its bits; a hit stops
                                  the execution phase (the round is lost to the
                                  CPU anyway under GPU-loses).  Ordered mode,
                                  fused rounds only; 0                        */
    uint64_t max_round_tx;     /* ordered mode: transactions per execution phase; 1<<22.
                                  Optimistic mode: launches up to this size
                                  hand the STM a list of the transactions
                                  their read-only phase left (4 B per tx) */
    /* Optional device allocator (e.g. a framework's caching allocator);
     * NULL = cudaMalloc/cudaFree.  Called only from hetm_init/hetm_destroy. */
    void *(*dev_alloc)(size_t bytes, void *user);
    void (*dev_free)(void *ptr, void *user);
    void *alloc_user;
    /* Inter-device conflict resolution (Sec. IV-E).  HETM_POLICY_GPU_LOSES
     * (the paper's prototype): the CPU log is always applied and a conflict
     * rolls the GPU batch back.  HETM_POLICY_CPU_LOSES: the CPU log is applied
     * only after the whole validation came back clean; on a conflict the GPU
     * state stands, the CPU log is discarded, and the host re-aligns its
     * replica from its shadow and the GPU-dirty chunks (hetm_read_dirty). */
    uint32_t conflict_policy;
    /* GPU_LOSES only: after this many consecutive rounds that rolled the GPU
     * back, the next execution phase admits only read-only CPU transactions
     * (Sec. IV-E's anti-starvation rule; hetm_cpu_updates_allowed reports it
     * and hetm_cpu_log_write refuses writes), so that round validates clean.
     * 0 = off (default). */
    uint32_t starve_limit;
    /* Wall-clock bound of the waits of one execution phase, in microseconds
     * (0 = 20 s).  Past it every transaction not yet run gives up (status 2),
     * the round reports HETM_ETIMEOUT and HETM_OUTCOME_GPU_ROLLED_BACK, and
     * its merge undoes the whole batch (S -> W), as after a lost conflict.
     * The error stays reported until hetm_load. */
    uint32_t exec_budget_us;
    /* 1: the executors record nothing in RS_bmp / WS_bmp.  Only for measuring
     * what the GPU instrumentation costs (Sec. V-A compares against the
     * uninstrumented GPU TM): validation then cannot see the batch's reads
     * and the merge moves no chunk, so a round's result is not SHeTM's.
     * 0 (default): instrumented. */
    uint32_t uninstrumented;
} hetm_config;

#define HETM_POLICY_GPU_LOSES 0
#define HETM_POLICY_CPU_LOSES 1

/* Fill *cfg with the defaults listed above. */
HETM_API int hetm_config_default(hetm_config *cfg);

/* ------------------------------------------------------------- lifecycle */
typedef struct hetm_ctx hetm_ctx;

/* Create a context on the current CUDA device for an STMR of `stmr_words`
 * int32 words (1 <= stmr_words < 2^32) with conflict granule
 * `granule_bytes` (power of two, >= 4; Sec. V-A studies 4 B and 1 KB).
 * Allocates STMR^W, STMR^S, TS, RS_bmp, WS_bmp, the lock table, two device
 * log buffers and the pinned per-thread CPU logs.  `stream` is a
 * cudaStream_t for all device work (NULL = a new non-blocking stream owned
 * by the context).  cfg NULL = defaults.  On success *out owns everything. */
HETM_API int hetm_init(hetm_ctx **out, uint64_t stmr_words, uint32_t granule_bytes,
              const hetm_config *cfg, void *stream);

/* Release every resource of the context (synchronizes its streams). */
HETM_API void hetm_destroy(hetm_ctx *ctx);

/* STMR^W = STMR^S = src[0..n), TS = 0, bitmaps and logs cleared.  src is a
 * host or device pointer (n == stmr_words).  Synchronous. */
HETM_API int hetm_load(hetm_ctx *ctx, const int32_t *src, uint64_t n);

/* Copy n words from offset `off` of STMR^W (which = 0) or STMR^S
 * (which = 1) to host memory.  Synchronizes the context stream. */
HETM_API int hetm_read_stmr(hetm_ctx *ctx, int which, int32_t *host_dst, uint64_t off, uint64_t n);

/* Device address of STMR^W (0), STMR^S (1), TS (2), RS_bmp (3), WS_bmp (4);
 * NULL for other values.  Borrowed: valid until hetm_destroy. */
HETM_API void *hetm_device_ptr(hetm_ctx *ctx, int which);

/* Size in 32-bit words of RS_bmp and WS_bmp (bit g of word g/32, LSB first). */
HETM_API int hetm_bitmap_words(hetm_ctx *ctx, uint64_t *rs_words, uint64_t *ws_words);

/* Wait for all work queued on the context stream. */
HETM_API int hetm_sync(hetm_ctx *ctx);

/* The cudaStream_t all device work of the context runs on. */
HETM_API void *hetm_ctx_stream(hetm_ctx *ctx);

/* -------------------------------------------------- execution phase (A1) */
/* One transaction batch.  All pointers are device pointers; outputs may be
 * NULL.  order[i] is the commit key of transaction i: sorting the committed
 * transactions by (order, index) gives a serial order that reproduces
 * STMR^W and every output (property P1, Sec. III).  An update commit has
 * key 2v (v = its commit version, unique); a read-only commit has key
 * 2v'+1 where v' is the newest version it observed.  status[i] = 1
 * committed, 2 gave up after max_attempts (no effect, no bitmap bits), 3
 * not run: early validation found a conflict and stopped the execution
 * phase (the round rolls the whole batch back). */
typedef struct hetm_batch {
    uint32_t workload;   /* HETM_WL_* */
    uint32_t n_tx;
    const void *tx;      /* n_tx records of the workload's type            */
    uint64_t *order;     /* out: commit key per transaction                */
    uint8_t *status;     /* out: 1 committed, 2 gave up, 3 not run         */
    void *out;           /* out: int32 (RMW, W2) or uint64 (cache) per tx  */
    uint32_t txid_base;  /* RMW, W2: txid = txid_base + index               */
    uint32_t word_base;  /* BANK: account a is word word_base + a           */
} hetm_batch;

/* Admit a batch into the current round's execution phase.  The batch is
 * queued; hetm_gpu_exec (or hetm_round) runs every queued batch in one
 * persistent launch.  Returns HETM_EBUSY when the batch table is full or
 * the device lacks `reserve_bytes` of free memory for its buffers.  With
 * cfg->max_batches reached, call hetm_gpu_exec first.  *batch_id gets a
 * context-unique id. */
HETM_API int hetm_gpu_submit_batch(hetm_ctx *ctx, const hetm_batch *batch, uint64_t *batch_id);

/* Run every queued batch now: one launch of the persistent executor that
 * drains all of them (uneven sizes), asynchronous on the context stream.
 * per_batch != 0 instead launches the executor once per batch. */
HETM_API int hetm_gpu_exec(hetm_ctx *ctx, int per_batch);

/* Execution statistics since the last hetm_load: committed transactions,
 * transactions that gave up, and aborted attempts.  Synchronizes. */
HETM_API int hetm_exec_counters(hetm_ctx *ctx, uint64_t *committed, uint64_t *gave_up, uint64_t *aborts);


/* ---------------------------------------------------- log shipping (A2) */
/* Append n tuples (host memory) to CPU thread `thread`'s pinned log.  Each
 * full log_chunk_bytes chunk is copied to the device log with
 * cudaMemcpyAsync on a side stream right away, overlapping the GPU's work
 * (Sec. IV-D).  Thread-safe for distinct `thread` values.  HETM_ECAPACITY
 * if the thread's pinned log or the device log would overflow. */
HETM_API int hetm_cpu_log_write(hetm_ctx *ctx, uint32_t thread, const hetm_log_entry *e, uint32_t n);

/* Use caller device memory as this round's CPU log instead of the shipped
 * one (no copy).  `dev_log` must be 16-byte aligned and stay valid until the
 * round's validation has completed. */
HETM_API int hetm_log_attach(hetm_ctx *ctx, const hetm_log_entry *dev_log, uint64_t n);

/* ------------------------------------------------- validation (A3..A5) */
/* Ship the rest of the CPU logs, then validate them against RS_bmp and
 * apply every tuple whose timestamp is the newest for its word and newer
 * than TS to STMR^W and STMR^S (Sec. IV-C).  dev_flag_bits (device, may be
 * NULL) receives bit i = "tuple i of the device log hit a read granule",
 * ceil(n/32) words.  If n_conflicts is non-NULL the call synchronizes and
 * stores the number of hits; otherwise the count stays on the device for
 * hetm_merge(ctx, -1). */
HETM_API int hetm_validate(hetm_ctx *ctx, uint64_t *n_conflicts, uint32_t *dev_flag_bits);

/* Validation only (no apply) of a device log: the early-validation test of
 * Sec. IV-D.  Asynchronous; *dev_count (device uint64) is incremented by
 * the number of hits, flags as in hetm_validate (may be NULL). */
HETM_API int hetm_validate_only(hetm_ctx *ctx, const hetm_log_entry *dev_log, uint64_t n,
                       uint32_t *dev_flag_bits, uint64_t *dev_count);

/* Allocation-free validation (no counterpart in the paper: the paper's
 * validation always runs inside its own runtime, which owns its memory).
 * For callers that must not allocate device memory at the moment they
 * validate: work recorded into a CUDA graph under capture, serving loops
 * that cannot afford cudaMalloc's device-wide synchronization, and plug-ins
 * whose host framework hands them only input and output buffers.  It needs
 * no context: the same per-tuple test as hetm_validate_only is run against
 * the caller's RS_bmp (dev_rs_bmp, bit g of word g/32, for a STMR of
 * stmr_words words and conflict granule granule_bytes).
 *   dev_log          device, 16-byte aligned, n tuples (n <= HETM_NOALLOC_MAX_TUPLES,
 *                    else HETM_ECAPACITY)
 *   dev_flag_bits    device, ceil(n/32) words, or NULL
 *   dev_n_conflicts  device uint64: receives (not adds) the number of hits
 *   dev_err          device int32 or NULL: HETM_OK, or HETM_EDEVICE when a
 *                    tuple's address was >= stmr_words (that tuple is skipped)
 *   stream           cudaStream_t (NULL = legacy default stream)
 * Asynchronous; calls no cudaMalloc, cudaFree or allocating library routine.
 * Its scratch is one static device array of about 48 KiB per GPU that loads
 * the library, kept until the process exits and shared by every call on
 * that GPU: calls that overlap on the GPU (different streams without
 * ordering) race on it and give undefined results.  Each call rewrites every
 * scratch slot it reads, so nothing needs clearing between calls.  The first
 * call on a device looks up the array's device address with that device
 * current; make that first call before any stream capture begins. */
#define HETM_NOALLOC_MAX_TUPLES (1ull << 25)
HETM_API int hetm_validate_noalloc(const hetm_log_entry *dev_log, uint64_t n,
                                   const uint32_t *dev_rs_bmp, uint32_t granule_bytes,
                                   uint64_t stmr_words, uint32_t *dev_flag_bits,
                                   uint64_t *dev_n_conflicts, int32_t *dev_err, void *stream);

/* -------------------------------------------------------- merge (A6) */
/* Copy the WS_bmp chunks W -> S (conflict == 0) or S -> W (conflict == 1);
 * conflict == -1 takes the decision from the last hetm_validate on the
 * device, without a host round trip.  Then clears RS_bmp and WS_bmp. */
HETM_API int hetm_merge(hetm_ctx *ctx, int conflict);

/* ------------------------------------------------------ round (A1..A7) */
typedef struct hetm_round_stats {
    uint64_t n_log;          /* CPU tuples validated                     */
    uint64_t n_conflicts;    /* tuples that hit RS_bmp                    */
    int32_t conflict;        /* 1: GPU batch undone                       */
    int32_t err;             /* HETM_OK; HETM_ETIMEOUT when the execution
                                phase ran out of its budget (the batch was
                                undone), whatever else went wrong; else
                                HETM_EDEVICE after an out-of-range address;
                                else HETM_EINVAL after a CPU timestamp out of
                                range or repeated (hetm_log_entry) */
    uint64_t committed;      /* GPU transactions committed this round     */
    uint64_t gave_up;        /* GPU transactions that gave up             */
    uint64_t aborts;         /* aborted GPU attempts this round           */
    uint64_t dirty_chunks;   /* WS_bmp chunks merged                      */
    uint32_t n_batches;      /* batches executed this round               */
    float ms_exec, ms_validate, ms_apply, ms_merge, ms_total;
    uint32_t n_kernels;      /* kernel launches this round (graph kernel nodes) */
    uint32_t stopped_early;  /* 1: early validation stopped the execution phase */
    uint32_t outcome;        /* HETM_OUTCOME_*: who won the round            */
    uint32_t cpu_read_only_next; /* 1: anti-starvation -- the next execution
                                    phase admits only read-only CPU transactions */
} hetm_round_stats;

#define HETM_OUTCOME_CLEAN 0          /* no conflict: both devices' commits stand   */
#define HETM_OUTCOME_GPU_ROLLED_BACK 1 /* conflict, GPU loses: its batch is undone  */
#define HETM_OUTCOME_CPU_DISCARDED 2  /* conflict, CPU loses: its log is discarded */

/* One whole round: run the queued batches (persistent executor), ship the
 * CPU logs, validate, apply, merge, clear.  The device part is CUDA graphs
 * captured on first use and replayed.  stats NULL = asynchronous (no host
 * synchronization): up to two rounds may be in flight, the second queued on
 * the device behind the first (its batches and CPU log are the ones
 * submitted before this call), so that the GPU does not wait for the host
 * to collect a round before the next starts; HETM_EBUSY with two in flight.
 * Otherwise (stats non-NULL) it needs none in flight (HETM_EBUSY), waits
 * and fills *stats.  With two rounds in flight, the anti-starvation rule set
 * by the first applies to the execution phase launched after it is
 * collected. */
HETM_API int hetm_round(hetm_ctx *ctx, hetm_round_stats *stats);

/* Wait for the oldest round launched by hetm_round(ctx, NULL) and not yet
 * collected, and fill *stats (may be NULL; zeroed when none is in flight).
 * Returns the round's status like hetm_round. */
HETM_API int hetm_round_wait(hetm_ctx *ctx, hetm_round_stats *stats);

/* Where a submitted batch is, without blocking (the GPU-controller's view of
 * its queue, Sec. III-A: a transactional kernel's requests finish when the
 * synchronization round that ran them has merged).  A batch is QUEUED until
 * hetm_gpu_exec or hetm_round launches it, RUNNING until the round that ran
 * it has finished its merge on the device (hetm_round, or hetm_merge after
 * hetm_gpu_exec and hetm_validate), then DONE: its order, status and out
 * buffers hold their final values, `outcome` is that round's HETM_OUTCOME_*
 * (HETM_OUTCOME_UNKNOWN when it ended more than 64 rounds before the first
 * poll that saw it done) and `latency_ms` is host time from its submission
 * to that first poll.  Ids are those hetm_gpu_submit_batch returned; the
 * context remembers the last 65,536 batches, and forgets those that
 * hetm_load discarded.  HETM_EINVAL for an unknown id or NULL pointer,
 * HETM_ECUDA if the device query failed.  Call from the controller thread,
 * and not while a hetm_server drives the context (its loop thread is then the
 * controller). */
#define HETM_BATCH_QUEUED 1
#define HETM_BATCH_RUNNING 2
#define HETM_BATCH_DONE 3
#define HETM_OUTCOME_UNKNOWN 0xFFFFFFFFu
typedef struct {
    uint32_t state;      /* HETM_BATCH_QUEUED / _RUNNING / _DONE             */
    uint32_t outcome;    /* DONE: the round's HETM_OUTCOME_* (else 0)        */
    uint64_t round;      /* sequence number of the round that runs it, 0 while queued */
    uint32_t n_tx;       /* transactions of the batch                        */
    uint32_t reserved;
    double latency_ms;   /* DONE: submission -> first poll that saw it done  */
} hetm_batch_result;

HETM_API int hetm_batch_poll(hetm_ctx *ctx, uint64_t batch_id, hetm_batch_result *out);

/* Host side of the merge (Sec. IV-C merge phase, Sec. IV-E): copy into the
 * host replica `host_stmr` (stmr_words int32, host memory) every WS_bmp
 * chunk of the last completed round whose GPU writes survived it (a clean
 * round, or a conflict the CPU lost), from STMR^S, contiguous dirty chunks
 * in one copy.  After a round the GPU lost nothing is copied (the host
 * replica already holds the round's outcome).  Under CPU_LOSES the caller
 * first restores the words its discarded log wrote from its own shadow.
 * *n_chunks / *n_bytes (may be NULL) get what was copied.  Synchronous.
 * HETM_EBUSY while a round is in flight (it would change STMR^S under the
 * copies): collect it with hetm_round_wait first. */
HETM_API int hetm_read_dirty(hetm_ctx *ctx, int32_t *host_stmr, uint64_t *n_chunks, uint64_t *n_bytes);

/* Double-buffered form of hetm_read_dirty (Sec. IV-D: the shadow STMR^S lets
 * the copy to the host overlap the next execution phase, which reads and
 * writes STMR^W only).  Queues the same copies on a side stream and returns;
 * the next call that writes STMR^S (the synchronization phase of
 * hetm_round, hetm_validate, hetm_merge, hetm_load) waits for them on the
 * device, so they see the last round's STMR^S.  host_stmr must be pinned
 * (cudaHostAlloc / cudaHostRegister) for the copies to be asynchronous, and
 * must not be read before hetm_read_dirty_wait returns.  Same precondition
 * as hetm_read_dirty: the last round's stats were collected. */
HETM_API int hetm_read_dirty_async(hetm_ctx *ctx, int32_t *host_stmr, uint64_t *n_chunks,
                                   uint64_t *n_bytes);
/* Block until the copies of the last hetm_read_dirty_async are in host memory. */
HETM_API int hetm_read_dirty_wait(hetm_ctx *ctx);

/* 1 when CPU update transactions may run in the current execution phase; 0
 * while the anti-starvation rule holds the CPU to read-only transactions
 * (starve_limit). */
HETM_API int hetm_cpu_updates_allowed(hetm_ctx *ctx);

/* ---------------------------------------------------------- serving (A7) */
/* A serving loop over one context: client threads submit transaction
 * batches (host records) at any time; one loop thread admits waiting
 * batches in arrival order while the device-memory budget and the round's
 * capacity allow, stages their records on the device while the previous
 * round still runs, and executes all admitted batches in one round (one
 * persistent executor launch over uneven batches, then validation, apply,
 * merge; Sec. IV-C) -- or one round per batch with per_batch = 1.  A batch
 * completes when its round is merged and its results are in the caller's
 * host buffers; its commit latency runs from submit to that point.  While a
 * server exists, only it drives the context (hetm_cpu_log_write stays open
 * to CPU threads). */
typedef struct hetm_request {
    uint32_t workload, n_tx;
    const void *host_tx;     /* n_tx records (host; read during admission)   */
    uint64_t *host_order;    /* out (host, may be NULL): commit keys          */
    uint8_t *host_status;    /* out (host, may be NULL): 1 committed          */
    void *host_out;          /* out (host, may be NULL): RMW int32 / cache u64 */
    uint32_t txid_base, word_base;
} hetm_request;

/* Admission: a waiting batch is admitted (in arrival order) when its device
 * footprint (records + order + status + outputs) fits the device memory free
 * at that moment, as cudaMemGetInfo reports it, less free_reserve -- memory
 * that other allocations take after the server started is seen -- and, when
 * device_budget is set, when the bytes of admitted batches stay within it.
 * A batch that does not fit while no batch is in flight completes with
 * HETM_ENOMEM (counted in `refused`); otherwise it waits for in-flight
 * batches to finish. */
typedef struct hetm_server_config {
    int32_t per_batch;           /* 1: one round per batch (the plain form)        */
    uint32_t max_round_batches;  /* batches per round; 1024                        */
    uint64_t max_round_tx;       /* transactions per round; 1<<22                  */
    uint64_t device_budget;      /* fixed cap on in-flight batch bytes; 0 = none    */
    uint64_t free_reserve;       /* device bytes admission leaves free; 0 = 1/16 of
                                    the device's memory                          */
} hetm_server_config;

typedef struct hetm_server_stats {
    uint64_t rounds, completed, committed, refused;
    double p50_ms, p99_ms, max_ms;  /* commit latency of completed batches   */
    double span_s;                  /* first submit to last completion        */
} hetm_server_stats;

typedef struct hetm_server hetm_server;
HETM_API int hetm_server_config_default(hetm_server_config *cfg);
/* Start the loop thread.  The context must outlive the server. */
HETM_API int hetm_server_create(hetm_server **out, hetm_ctx *ctx, const hetm_server_config *cfg);
/* Queue a batch (thread-safe).  HETM_EBUSY if it can never fit (larger than
 * device_budget, or than the device's memory less free_reserve) or exceeds
 * the round capacity.  The host buffers must stay valid until wait. */
HETM_API int hetm_server_submit(hetm_server *s, const hetm_request *r, uint64_t *id);
/* Block until batch `id` completed (bounded: HETM_ETIMEOUT after 120 s). */
HETM_API int hetm_server_wait(hetm_server *s, uint64_t id, double *latency_ms);
/* hetm_server_wait that also gives the HETM_OUTCOME_* of the round that ran
 * the batch (*outcome may be NULL).  After HETM_OUTCOME_GPU_ROLLED_BACK the
 * batch's effects on the STMR were undone by the merge: its status and out
 * buffers hold what the undone execution produced. */
HETM_API int hetm_server_wait_outcome(hetm_server *s, uint64_t id, double *latency_ms,
                                      uint32_t *outcome);
HETM_API int hetm_server_get_stats(hetm_server *s, hetm_server_stats *out);
/* Drain the queue, stop the loop thread, free the server. */
HETM_API void hetm_server_destroy(hetm_server *s);

/* ------------------------------------------------------------- dispatch */
/* Request queues and device affinity (Sec. III-B, transaction scheduling and
 * dispatching).  Requests are single transactions of a registered type.  A
 * type has a transactional function (runs one request on the CPU), a
 * transactional kernel (one of the executor's workloads, runs requests in
 * batches on the GPU), or both.  A type with one implementation has one
 * queue; a type with both has three: CPU_Q, GPU_Q and SHARED_Q, chosen by
 * the affinity given at submission (none -> SHARED_Q), so that requests known
 * to conflict can be kept on one device.
 *   - CPU workers (cpu_workers threads) take one request at a time from the
 *     CPU_Qs of all types in round-robin order; when every CPU_Q is empty they
 *     steal one from a SHARED_Q (round-robin too).
 *   - A GPU controller thread activates a type's kernel when its GPU_Q plus
 *     SHARED_Q hold gpu_min_batch requests (the GPU steals from SHARED_Q only
 *     what its own GPU_Q leaves of the batch), or when the oldest of them has
 *     waited gpu_max_wait_us; a batch takes at most gpu_max_batch requests,
 *     and at most gpu_inflight batches are outstanding.  Batches go to a
 *     hetm_server (which fuses them into synchronization rounds) or, with no
 *     server, to a caller-supplied batch function.
 *   - A batch whose round ended HETM_OUTCOME_GPU_ROLLED_BACK had its effects
 *     undone: its requests go back to the front of the queues they came from
 *     and run again, so every request completes exactly once.
 * The transactional function runs the request through the application's
 * CPU TM and hands its writes to hetm_cpu_log_write (thread id = the worker
 * index it is given).  Under HETM_POLICY_CPU_LOSES the application undoes
 * and re-runs discarded CPU transactions itself (Sec. IV-E); the dispatcher
 * completes a CPU request when its function returns. */
#define HETM_AFFINITY_NONE 0
#define HETM_AFFINITY_CPU 1
#define HETM_AFFINITY_GPU 2
#define HETM_DEVICE_CPU 1 /* hetm_dispatch_submit's device[] values */
#define HETM_DEVICE_GPU 2

/* Runs request `tx` on the CPU (worker index `worker`), writing out_bytes to
 * `out` when out is not NULL.  Returns the request's status byte (0..255, 1 =
 * committed) or a negative HETM_E* code, which fails its submission.  Called
 * from the dispatcher's worker threads, several at a time. */
typedef int (*hetm_cpu_tx_fn)(void *user, uint32_t worker, const void *tx, void *out);
/* Runs n requests (packed records) on the GPU with no hetm_server attached:
 * fills status[n] (and out, n x out_bytes, when not NULL) and *outcome with
 * the HETM_OUTCOME_* of the round that ran them.  Returns HETM_OK or an error
 * code, which fails every submission in the batch.  Called from the
 * controller thread only. */
typedef int (*hetm_gpu_batch_fn)(void *user, uint32_t workload, uint32_t word_base, const void *tx,
                                 uint32_t n, uint8_t *status, void *out, uint32_t *outcome);

typedef struct hetm_tx_type {
    uint32_t gpu_workload;   /* HETM_WL_BANK / HETM_WL_CACHE, or 0: no kernel.
                                HETM_WL_RMW is refused: its txid is a position
                                in the batch, which dispatch does not fix */
    uint32_t rec_bytes;      /* bytes of one request; the workload's record
                                size when gpu_workload != 0                */
    uint32_t out_bytes;      /* bytes of one result; the workload's (bank 0,
                                cache 8) when gpu_workload != 0            */
    uint32_t word_base;      /* the kernel's hetm_request.word_base       */
    hetm_cpu_tx_fn cpu_fn;   /* transactional function, or NULL           */
    void *cpu_user;
} hetm_tx_type;

typedef struct hetm_dispatch_config {
    uint32_t cpu_workers;      /* CPU worker threads; 2                          */
    uint32_t gpu_min_batch;    /* requests that make an activation worth it; 1024 */
    uint32_t gpu_max_batch;    /* requests per activation; 1 << 20, clamped to the
                                  server's max_round_tx                           */
    uint32_t gpu_max_wait_us;  /* fewer requests activate after this wait; 2000   */
    uint32_t gpu_inflight;     /* outstanding activations; 2                      */
} hetm_dispatch_config;

typedef struct hetm_dispatch_stats {
    uint64_t cpu_done, gpu_done;        /* requests completed on each device      */
    uint64_t cpu_stolen, gpu_stolen;    /* of those, taken from a SHARED_Q        */
    uint64_t activations;               /* GPU batches completed                  */
    uint64_t requeued;                  /* requests re-run after a rolled-back round */
    uint64_t queued_cpu, queued_gpu, queued_shared;  /* waiting now            */
} hetm_dispatch_stats;

typedef struct hetm_dispatch hetm_dispatch;
HETM_API int hetm_dispatch_config_default(hetm_dispatch_config *cfg);
/* Start the worker and controller threads.  GPU batches go to `server` when
 * it is not NULL (it must outlive the dispatcher), else to `gpu_fn`; with
 * neither, only CPU-only types can be registered.  HETM_EINVAL for a bad
 * config (gpu_min_batch, gpu_max_batch or gpu_inflight 0). */
HETM_API int hetm_dispatch_create(hetm_dispatch **out, hetm_server *server, hetm_gpu_batch_fn gpu_fn,
                                  void *gpu_user, const hetm_dispatch_config *cfg);
/* Register a transaction type; *type gets its id (0, 1, ...).  HETM_EINVAL
 * when it has no implementation, a record size that does not match its
 * workload, a CPU function but no CPU workers, or a kernel but neither a
 * server nor a batch function. */
HETM_API int hetm_dispatch_register(hetm_dispatch *d, const hetm_tx_type *t, uint32_t *type);
/* Queue n requests of `type` (records packed in tx, host memory) with an
 * affinity (HETM_AFFINITY_*).  Results: status[n] (may be NULL), out (n x
 * out_bytes, may be NULL), device[n] (HETM_DEVICE_*, may be NULL).  All
 * buffers stay the caller's and must stay valid until hetm_dispatch_wait.
 * Thread-safe.  HETM_EINVAL for an unknown type, an affinity naming a device
 * the type has no implementation for, or after destroy began. */
HETM_API int hetm_dispatch_submit(hetm_dispatch *d, uint32_t type, int affinity, const void *tx,
                                  uint32_t n, uint8_t *status, void *out, uint8_t *device,
                                  uint64_t *ticket);
/* Block until every request of `ticket` completed (bounded: HETM_ETIMEOUT
 * after 120 s); returns the first error among them, and frees the ticket.
 * *latency_ms (may be NULL): submission to the last completion. */
HETM_API int hetm_dispatch_wait(hetm_dispatch *d, uint64_t ticket, double *latency_ms);
HETM_API int hetm_dispatch_get_stats(hetm_dispatch *d, hetm_dispatch_stats *out);
/* Run every queued request, stop the threads, free the dispatcher. */
HETM_API void hetm_dispatch_destroy(hetm_dispatch *d);

/* ------------------------------------------------------------ autotuner */
/* The paper runs one executor shape and studies the conflict granule (Sec.
 * V-A: 4 B against 1 KB granules, instrumentation cost against false
 * conflicts) and the merge chunk (Sec. IV-D: 16 KB) by hand.  The autotuner
 * measures these choices on the caller's own sample instead: it creates a
 * scratch context per candidate on the current device (3 x stmr_words x 4
 * bytes plus the executor's per-round state, freed after the candidate),
 * loads `init`, and times 1 + reps whole rounds (hetm_round) of the sample
 * batches (+ the CPU log), the first round untimed.  A round with the CPU
 * log starts from `init` loaded again (a log's timestamps are applied once
 * per context).
 *
 * Search, a coordinate search in three stages:
 *   0  executor shape -- every (mode, exec_threads, blocks per SM, lock_log2)
 *      of the space at granules[0], no CPU log; score = transactions
 *      committed per second of execution phase;
 *   1  granule -- each granule with the CPU log and the best shape; score =
 *      commits of rounds that validated clean per second of round (a
 *      conflicting round rolls the GPU batch back), or minus the round time
 *      when every candidate conflicts;
 *   2  merge chunk -- each ws_chunk_bytes, scored as stage 1.
 * In stage 0 a candidate whose warm-up round is slower than cut x the best
 * candidate so far keeps that measurement alone. */
typedef struct hetm_tune_space {
    uint32_t modes;             /* bit 0: HETM_EXEC_ORDERED, bit 1: OPTIMISTIC; 3 */
    uint32_t threads[4];        /* exec_threads candidates, 0-terminated (ordered:
                                   128/256/512; optimistic: multiple of 32 <= 256;
                                   others are skipped per mode); 128, 256, 512  */
    uint32_t blocks_per_sm[4];  /* grid = SMs x this; 0 = occupancy limit.  The
                                   first entry is always tried, the rest up to
                                   the first 0; 0, 1                           */
    uint32_t lock_log2[4];      /* optimistic lock-table sizes, 0-terminated; 22 */
    uint32_t granules[8];       /* conflict granules (bytes), 0-terminated;
                                   4, 64, 1024                                  */
    uint32_t ws_chunk_bytes[6]; /* merge chunks, 0-terminated; 1K, 4K, 16K      */
    uint32_t reps;              /* timed rounds per candidate (median); 3       */
    float cut;                  /* stage-0 early cut factor; 4                  */
} hetm_tune_space;

/* One measured candidate. */
typedef struct hetm_tune_trial {
    uint32_t stage;             /* 0 shape, 1 granule, 2 merge chunk            */
    uint32_t exec_mode, exec_threads, exec_blocks, lock_log2;
    uint32_t granule_bytes, ws_chunk_bytes;
    int32_t rc;                 /* HETM_OK, or why the candidate failed          */
    uint32_t rounds;            /* rounds measured                               */
    uint32_t conflicts;         /* of those, rounds that conflicted              */
    uint64_t committed;         /* GPU commits per round (median round)          */
    float ms_exec, ms_round;    /* medians over the measured rounds              */
    float score;                /* the stage's score (higher is better)          */
    uint32_t reserved;
} hetm_tune_trial;

HETM_API int hetm_tune_space_default(hetm_tune_space *space);

/* Tune for a sample.  init: stmr_words int32 (host or device).  batches:
 * n_batches descriptors as for hetm_gpu_submit_batch (device records; the
 * output buffers are overwritten by every candidate).  log: n_log device
 * log entries attached to every round of stages 1-2 (NULL/0: none; 16-byte
 * aligned).  base: every field the search does not set (capacities, cache
 * layout, allocator); NULL = defaults.  space NULL = defaults.  On
 * HETM_OK, *best_cfg = base with exec_mode, exec_threads, exec_blocks,
 * lock_log2 and ws_chunk_bytes tuned and *best_granule is the granule to
 * pass to hetm_init.  trials (may be NULL when max_trials is 0) receives up
 * to max_trials candidates in the order run; *n_trials (may be NULL) the
 * number run.  Synchronous; do not run it while another context of the
 * same device is mid-round if timings are to mean anything.
 * HETM_EINVAL for bad arguments or when no stage-0 candidate ran. */
HETM_API int hetm_autotune(uint64_t stmr_words, const int32_t *init, const hetm_batch *batches,
                           uint32_t n_batches, const hetm_log_entry *log, uint64_t n_log,
                           const hetm_config *base, const hetm_tune_space *space,
                           hetm_config *best_cfg, uint32_t *best_granule, hetm_tune_trial *trials,
                           uint32_t max_trials, uint32_t *n_trials);

#ifdef __cplusplus
}
#endif
#endif /* HETM_H */

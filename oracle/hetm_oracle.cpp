// Oracle for one SHeTM synchronization round -- TEST INFRASTRUCTURE ONLY.
//
// Plain, slow, single-threaded C++ that computes the *definitions* the GPU
// path must reach, written from the paper (Castro, Romano, Ilic, Khan,
// "HeTM: Transactional Memory for Heterogeneous Systems", arXiv 1905.00661):
//
//   * serial replay of the GPU's committed transactions in their reported
//     commit order (property P1, Sec. III), which also yields the exact
//     read/write granule sets the GPU instrumentation must record
//     (Sec. IV-B "GPU instrumentation", Sec. IV-C, with WS contained in RS);
//   * inter-device conflicts by brute-force set intersection of the CPU
//     write-set with the GPU read-set (Sec. IV-C, Validation Phase);
//   * the CPU write image: per word, the tuple with the newest timestamp,
//     applied only if newer than the word's stored timestamp (Sec. IV-C,
//     timestamp array TS);
//   * the final state of both GPU copies (Sec. IV-C Merge Phase, Sec. IV-D
//     rollback through the shadow copy): the replayed GPU state when
//     validation succeeds, the round-start state when it fails, in both cases
//     overlaid with the CPU image.
//
// Only tests/, the package's smoke check and the bench's CPU-baseline leg
// load this library.  It shares no source with the CUDA library.

#include <algorithm>
#include <cstdint>
#include <cstring>
#include <map>
#include <numeric>
#include <set>
#include <unordered_set>
#include <vector>

namespace {

struct LogEntry {      // <address, value, timestamp>, Sec. IV-B CPU instrumentation
    uint32_t addr;
    int32_t value;
    uint32_t ts;
};
static_assert(sizeof(LogEntry) == 12, "log tuple is 12 bytes");

struct BankTx {
    uint32_t src;
    uint32_t dst;
    int32_t amount;
};
static_assert(sizeof(BankTx) == 12, "bank tx is 12 bytes");

struct RmwTx {
    uint32_t addr[4];
    uint32_t flags;    // bit 0: update transaction
};
static_assert(sizeof(RmwTx) == 20, "rmw tx is 20 bytes");

struct W2Tx {
    uint32_t addr[40];
    uint32_t flags;    // bit 0: update transaction
    uint32_t pad[3];
};
static_assert(sizeof(W2Tx) == 176, "W2 tx is 176 bytes");

struct CacheReq {
    uint64_t key;
    uint64_t value;
    uint32_t op;       // 0 GET, 1 PUT
    uint32_t pad;
};
static_assert(sizeof(CacheReq) == 24, "cache request is 24 bytes");

const uint8_t kCommitted = 1;

// 32-bit two's-complement addition, written out so that overflow wraps.
int32_t add32(int32_t a, int32_t b) {
    return (int32_t)((uint32_t)a + (uint32_t)b);
}

uint64_t granule_of(uint64_t word, uint32_t granule_bytes) {
    return word * 4 / granule_bytes;
}

// The serial order: committed transactions sorted by their reported commit
// key, ties (read-only transactions that observed the same state) by index.
std::vector<uint64_t> serial_order(uint64_t n, const uint64_t* order, const uint8_t* status) {
    std::vector<uint64_t> idx;
    for (uint64_t i = 0; i < n; ++i)
        if (status[i] == kCommitted) idx.push_back(i);
    std::stable_sort(idx.begin(), idx.end(),
                     [&](uint64_t a, uint64_t b) { return order[a] < order[b]; });
    return idx;
}

struct Footprint {
    std::set<uint64_t> granules;   // everything read or written (WS is inside RS)
    std::set<uint64_t> chunks;     // write-set at transfer-chunk granularity
    uint32_t granule_bytes, chunk_bytes;
    void read(uint64_t w) { granules.insert(granule_of(w, granule_bytes)); }
    void write(uint64_t w) {
        granules.insert(granule_of(w, granule_bytes));
        chunks.insert(w * 4 / chunk_bytes);
    }
};

int64_t emit(const std::set<uint64_t>& s, uint32_t* out, uint64_t cap) {
    if (s.size() > cap) return -1;
    uint64_t k = 0;
    for (uint64_t v : s) out[k++] = (uint32_t)v;
    return (int64_t)k;
}

uint64_t splitmix64_finalizer(uint64_t z) {
    // SplitMix64 output function (Steele, Lea & Flood 2014)
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ULL;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBULL;
    return z ^ (z >> 31);
}

uint64_t load_u64(const int32_t* m, uint64_t word) {
    uint64_t v;
    std::memcpy(&v, m + word, 8);
    return v;
}

void store_u64(int32_t* m, uint64_t word, uint64_t v) {
    std::memcpy(m + word, &v, 8);
}

}  // namespace

extern "C" {

// ---------------------------------------------------------------------------
// Serial replay of a bank batch (property P1, Sec. III).  A transfer reads
// and writes both accounts: bal[src] -= amount, then bal[dst] += amount, in
// 32-bit wrapping arithmetic.  `stmr` is replayed in place; the granule and
// chunk sets of the committed transactions are written to r_out / d_out
// (sorted ascending) and their sizes to *n_r / *n_d.  Returns 0, or -1 if an
// output array is too small or an address is out of range.
// ---------------------------------------------------------------------------
int hetm_oracle_replay_bank(int32_t* stmr, uint64_t n_words, const void* txs, uint64_t n_tx,
                            const uint64_t* order, const uint8_t* status,
                            uint32_t granule_bytes, uint32_t chunk_bytes,
                            uint32_t* r_out, uint64_t r_cap, uint64_t* n_r,
                            uint32_t* d_out, uint64_t d_cap, uint64_t* n_d) {
    const BankTx* tx = static_cast<const BankTx*>(txs);
    Footprint fp{{}, {}, granule_bytes, chunk_bytes};
    for (uint64_t i : serial_order(n_tx, order, status)) {
        const BankTx& t = tx[i];
        if (t.src >= n_words || t.dst >= n_words) return -1;
        stmr[t.src] = add32(stmr[t.src], -t.amount);
        stmr[t.dst] = add32(stmr[t.dst], t.amount);
        fp.write(t.src);
        fp.write(t.dst);
    }
    int64_t a = emit(fp.granules, r_out, r_cap), b = emit(fp.chunks, d_out, d_cap);
    if (a < 0 || b < 0) return -1;
    *n_r = (uint64_t)a;
    *n_d = (uint64_t)b;
    return 0;
}

// ---------------------------------------------------------------------------
// Serial replay of W1-style transactions (Sec. V-A): each reads 4 words and
// outputs their 32-bit wrapping sum s; an update transaction then writes
// s + j + txid to its j-th word (txid = txid_base + index in the batch).
// The per-transaction output (the sum each committed transaction observed)
// goes to out_sum[i]; aborted transactions keep out_sum unchanged.
// ---------------------------------------------------------------------------
int hetm_oracle_replay_rmw(int32_t* stmr, uint64_t n_words, const void* txs, uint64_t n_tx,
                           const uint64_t* order, const uint8_t* status, uint32_t txid_base,
                           int32_t* out_sum, uint32_t granule_bytes, uint32_t chunk_bytes,
                           uint32_t* r_out, uint64_t r_cap, uint64_t* n_r,
                           uint32_t* d_out, uint64_t d_cap, uint64_t* n_d) {
    const RmwTx* tx = static_cast<const RmwTx*>(txs);
    Footprint fp{{}, {}, granule_bytes, chunk_bytes};
    for (uint64_t i : serial_order(n_tx, order, status)) {
        const RmwTx& t = tx[i];
        int32_t s = 0;
        for (int j = 0; j < 4; ++j) {
            if (t.addr[j] >= n_words) return -1;
            s = add32(s, stmr[t.addr[j]]);
            fp.read(t.addr[j]);
        }
        out_sum[i] = s;
        if (t.flags & 1u) {
            uint32_t txid = txid_base + (uint32_t)i;
            for (int j = 0; j < 4; ++j) {
                stmr[t.addr[j]] = add32(add32(s, j), (int32_t)txid);
                fp.write(t.addr[j]);
            }
        }
    }
    int64_t a = emit(fp.granules, r_out, r_cap), b = emit(fp.chunks, d_out, d_cap);
    if (a < 0 || b < 0) return -1;
    *n_r = (uint64_t)a;
    *n_d = (uint64_t)b;
    return 0;
}

// ---------------------------------------------------------------------------
// Serial replay of W2 transactions (Sec. V-A: W1 with 40 reads instead of 4
// in both transaction types).  Each reads its 40 words and outputs their
// 32-bit wrapping sum s; an update transaction then writes s + j + txid to
// its first 4 words, j = 0..3 (both workloads' updates update 4 positions).
// Outputs and footprints as for hetm_oracle_replay_rmw.
// ---------------------------------------------------------------------------
int hetm_oracle_replay_w2(int32_t* stmr, uint64_t n_words, const void* txs, uint64_t n_tx,
                          const uint64_t* order, const uint8_t* status, uint32_t txid_base,
                          int32_t* out_sum, uint32_t granule_bytes, uint32_t chunk_bytes,
                          uint32_t* r_out, uint64_t r_cap, uint64_t* n_r,
                          uint32_t* d_out, uint64_t d_cap, uint64_t* n_d) {
    const W2Tx* tx = static_cast<const W2Tx*>(txs);
    Footprint fp{{}, {}, granule_bytes, chunk_bytes};
    for (uint64_t i : serial_order(n_tx, order, status)) {
        const W2Tx& t = tx[i];
        int32_t s = 0;
        for (int j = 0; j < 40; ++j) {
            if (t.addr[j] >= n_words) return -1;
            s = add32(s, stmr[t.addr[j]]);
            fp.read(t.addr[j]);
        }
        out_sum[i] = s;
        if (t.flags & 1u) {
            uint32_t txid = txid_base + (uint32_t)i;
            for (int j = 0; j < 4; ++j) {
                stmr[t.addr[j]] = add32(add32(s, j), (int32_t)txid);
                fp.write(t.addr[j]);
            }
        }
    }
    int64_t a = emit(fp.granules, r_out, r_cap), b = emit(fp.chunks, d_out, d_cap);
    if (a < 0 || b < 0) return -1;
    *n_r = (uint64_t)a;
    *n_d = (uint64_t)b;
    return 0;
}

// ---------------------------------------------------------------------------
// Serial replay of object-cache requests (Sec. V-D).  Layout per set s,
// way w (word offsets): key u64 at key_base + 2(8s+w), value u64 at
// val_base + 2(8s+w), GPU LRU stamp at lru_base + 8s + w, per-set version
// at ver_base + s.  set = splitmix64_finalizer(key) mod n_sets.
//   GET hit at w : out = value; GPU LRU[w] = stamp.       reads keys, value[w]
//   GET miss     : out = ~0; no writes.                    reads keys
//   PUT          : hit way, else first empty way (key 0), else the way with
//                  the smallest GPU LRU stamp (lowest way on ties);
//                  key[w] = key (if it changes), value[w] = value,
//                  GPU LRU[w] = stamp, version += 1; out = w.
//                  reads keys, version (and all 8 LRU stamps when evicting)
// stamp = the low 32 bits of (commit key >> 1), i.e. the writer's commit
// version.  Every write is also recorded as a read (WS inside RS, Sec. IV-C).
// ---------------------------------------------------------------------------
int hetm_oracle_replay_cache(int32_t* stmr, uint64_t n_words, uint32_t log2_sets,
                             uint64_t key_base, uint64_t val_base, uint64_t lru_base,
                             uint64_t ver_base, const void* reqs, uint64_t n_req,
                             const uint64_t* order, const uint8_t* status, uint64_t* out,
                             uint32_t granule_bytes, uint32_t chunk_bytes,
                             uint32_t* r_out, uint64_t r_cap, uint64_t* n_r,
                             uint32_t* d_out, uint64_t d_cap, uint64_t* n_d) {
    const CacheReq* rq = static_cast<const CacheReq*>(reqs);
    const uint64_t n_sets = 1ull << log2_sets;
    const int ways = 8;
    if (ver_base + n_sets > n_words) return -1;
    Footprint fp{{}, {}, granule_bytes, chunk_bytes};
    for (uint64_t i : serial_order(n_req, order, status)) {
        const CacheReq& r = rq[i];
        uint64_t s = splitmix64_finalizer(r.key) & (n_sets - 1);
        uint32_t stamp = (uint32_t)(order[i] >> 1);
        int hit = -1, empty = -1;
        for (int w = 0; w < ways; ++w) {
            uint64_t kw = key_base + 2 * (s * ways + w);
            fp.read(kw);
            fp.read(kw + 1);
            uint64_t k = load_u64(stmr, kw);
            if (k == r.key && hit < 0) hit = w;
            if (k == 0 && empty < 0) empty = w;
        }
        if (r.op == 0) {  // GET
            if (hit < 0) {
                out[i] = ~0ull;
                continue;
            }
            uint64_t vw = val_base + 2 * (s * ways + hit);
            fp.read(vw);
            fp.read(vw + 1);
            out[i] = load_u64(stmr, vw);
            uint64_t lw = lru_base + s * ways + hit;
            stmr[lw] = (int32_t)stamp;
            fp.write(lw);
            continue;
        }
        // PUT
        uint64_t verw = ver_base + s;
        fp.read(verw);
        int w = hit;
        if (w < 0) w = empty;
        if (w < 0) {
            uint32_t best = 0;
            for (int v = 0; v < ways; ++v) {
                uint64_t lw = lru_base + s * ways + v;
                fp.read(lw);
                uint32_t l = (uint32_t)stmr[lw];
                if (w < 0 || l < best) {
                    best = l;
                    w = v;
                }
            }
        }
        uint64_t kw = key_base + 2 * (s * ways + w);
        uint64_t vw = val_base + 2 * (s * ways + w);
        uint64_t lw = lru_base + s * ways + w;
        if (hit < 0) {
            store_u64(stmr, kw, r.key);
            fp.write(kw);
            fp.write(kw + 1);
        }
        store_u64(stmr, vw, r.value);
        fp.write(vw);
        fp.write(vw + 1);
        stmr[lw] = (int32_t)stamp;
        fp.write(lw);
        stmr[verw] = add32(stmr[verw], 1);
        fp.write(verw);
        out[i] = (uint64_t)w;
    }
    int64_t a = emit(fp.granules, r_out, r_cap), b = emit(fp.chunks, d_out, d_cap);
    if (a < 0 || b < 0) return -1;
    *n_r = (uint64_t)a;
    *n_d = (uint64_t)b;
    return 0;
}

// ---------------------------------------------------------------------------
// Inter-device conflicts (Sec. IV-C, Validation Phase): the CPU write-set is
// tested against the GPU read-set, WS^CPU intersect RS^GPU, by brute force.
// flags[i] = 1 iff granule(log[i].addr) is in the set of GPU-read granules.
// Returns the number of flagged entries.
// ---------------------------------------------------------------------------
int64_t hetm_oracle_conflicts(const void* log, uint64_t n, const uint32_t* read_granules,
                              uint64_t n_read, uint32_t granule_bytes, uint8_t* flags) {
    const LogEntry* e = static_cast<const LogEntry*>(log);
    std::unordered_set<uint64_t> rs(read_granules, read_granules + n_read);
    int64_t hits = 0;
    for (uint64_t i = 0; i < n; ++i) {
        flags[i] = rs.count(granule_of(e[i].addr, granule_bytes)) ? 1 : 0;
        hits += flags[i];
    }
    return hits;
}

// ---------------------------------------------------------------------------
// The CPU write image (Sec. IV-C, timestamp array): for every word named in
// the log, the tuple with the largest timestamp wins; it is written into
// `state` only when that timestamp is newer than ts_state[word], which is
// then raised to it.  `state` may be NULL to update ts_state alone.
// Returns the number of timestamp ties between tuples of one word (the
// timestamp must totally order the writes to a position, so a tie is an
// invalid input), or -1 if an address is out of range.
// ---------------------------------------------------------------------------
int64_t hetm_oracle_cpu_image(int32_t* state, uint32_t* ts_state, uint64_t n_words,
                              const void* log, uint64_t n) {
    const LogEntry* e = static_cast<const LogEntry*>(log);
    std::map<uint32_t, std::pair<uint32_t, int32_t>> newest;
    int64_t ties = 0;
    for (uint64_t i = 0; i < n; ++i) {
        if (e[i].addr >= n_words) return -1;
        auto it = newest.find(e[i].addr);
        if (it == newest.end()) {
            newest[e[i].addr] = {e[i].ts, e[i].value};
        } else if (e[i].ts > it->second.first) {
            it->second = {e[i].ts, e[i].value};
        } else if (e[i].ts == it->second.first) {
            ++ties;
        }
    }
    for (const auto& kv : newest) {
        uint32_t a = kv.first;
        if (kv.second.first > ts_state[a]) {
            if (state) state[a] = kv.second.second;
            ts_state[a] = kv.second.first;
        }
    }
    return ties;
}

// ---------------------------------------------------------------------------
// Final state of STMR^W and STMR^S after the merge phase (Sec. IV-C Merge
// Phase; Sec. IV-D rollback).  Under the GPU-loses policy the round keeps
// the GPU's transactions only when validation found no conflict:
//   final = (conflict ? start : replayed) overlaid with the CPU image.
// `final_out` receives the result; ts_state is advanced as by the apply.
// ---------------------------------------------------------------------------
int64_t hetm_oracle_final_state(const int32_t* start, const int32_t* replayed, uint64_t n_words,
                                int conflict, const void* log, uint64_t n, uint32_t* ts_state,
                                int32_t* final_out) {
    const int32_t* base = conflict ? start : replayed;
    std::memcpy(final_out, base, n_words * sizeof(int32_t));
    return hetm_oracle_cpu_image(final_out, ts_state, n_words, log, n);
}

// ---------------------------------------------------------------------------
// Planted GPU writes (no transaction logic): words written by the GPU batch
// of a validation-at-scale round.  Applies them in order to `stmr`.
// ---------------------------------------------------------------------------
int hetm_oracle_plant(int32_t* stmr, uint64_t n_words, const uint32_t* addr, const int32_t* value,
                      uint64_t n) {
    for (uint64_t i = 0; i < n; ++i) {
        if (addr[i] >= n_words) return -1;
        stmr[addr[i]] = value[i];
    }
    return 0;
}

// Sum of all words in 64-bit arithmetic (bank conservation checks).
int64_t hetm_oracle_sum64(const int32_t* stmr, uint64_t n_words) {
    int64_t s = 0;
    for (uint64_t i = 0; i < n_words; ++i) s += stmr[i];
    return s;
}

}  // extern "C"

"""Seeded synthetic inputs for SHeTM synchronization rounds.

This module produces *inputs only*: initial STMR images, GPU transaction
batches, CPU write-set logs and planted GPU read/write sets.  It holds none of
the round's arithmetic (no validation, no timestamp resolution, no merge, no
replay) and is the one module that both the CUDA path's tests/bench and the
CPU oracle consume.

Random numbers come from a counter-based SplitMix64 (Steele, Lea & Flood,
"Fast splittable pseudorandom number generators", OOPSLA 2014): draw ``i`` of
stream ``s`` under seed ``k`` is ``mix64(key(k, s) + (i + 1) * GAMMA)``, so any
element can be regenerated independently and the inputs are identical on any
machine and numpy version.  Zipf ranks use rejection-inversion (Hoermann &
Derflinger, "Rejection-inversion to generate variates from monotone discrete
distributions", ACM TOMACS 1996), which needs no table over the 2^28 support.

Workload shapes follow the paper's evaluation (Sec. V): uniform or skewed
word-granular accesses for the synthetic benchmarks (Sec. V-A/V-B, W1), and an
8-way set-associative object cache with per-device LRU stamps and a per-set
version word for the MemcachedGPU-shaped workload (Sec. V-D).
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np

# --------------------------------------------------------------------------
# record layouts shared by the C ABI, the oracle and the tests
# --------------------------------------------------------------------------
#: CPU write-set log tuple <address, value, timestamp> (Sec. IV-B, CPU instrumentation)
LOG_DTYPE = np.dtype([("addr", "<u4"), ("value", "<i4"), ("ts", "<u4")])
#: bank transfer: bal[src] -= amount; bal[dst] += amount
BANK_DTYPE = np.dtype([("src", "<u4"), ("dst", "<u4"), ("amount", "<i4")])
#: W1-style transaction: 4 word addresses, flags bit0 = update (Sec. V-A)
RMW_DTYPE = np.dtype([("addr", "<u4", (4,)), ("flags", "<u4")])
#: object-cache request (Sec. V-D): op 0 = GET, 1 = PUT
W2_DTYPE = np.dtype([("addr", "<u4", (40,)), ("flags", "<u4"), ("pad", "<u4", (3,))])
CACHE_DTYPE = np.dtype([("key", "<u8"), ("value", "<u8"), ("op", "<u4"), ("pad", "<u4")])

assert LOG_DTYPE.itemsize == 12 and BANK_DTYPE.itemsize == 12
assert RMW_DTYPE.itemsize == 20 and CACHE_DTYPE.itemsize == 24

WORKLOAD_BANK = 1
WORKLOAD_RMW = 2
WORKLOAD_CACHE = 3
WORKLOAD_W2 = 4

# --------------------------------------------------------------------------
# counter-based SplitMix64
# --------------------------------------------------------------------------
GAMMA = np.uint64(0x9E3779B97F4A7C15)
_M1 = np.uint64(0xBF58476D1CE4E5B9)
_M2 = np.uint64(0x94D049BB133111EB)
_S30, _S27, _S31 = np.uint64(30), np.uint64(27), np.uint64(31)


def mix64(z: np.ndarray) -> np.ndarray:
    """SplitMix64 output function (variant 13 of Stafford's mixers)."""
    z = np.asarray(z, dtype=np.uint64).copy()
    z ^= z >> _S30
    z *= _M1
    z ^= z >> _S27
    z *= _M2
    z ^= z >> _S31
    return z


def _key(seed: int, stream: int) -> np.uint64:
    k = np.array([(seed * 0x100000001B3 + stream * 0x9E3779B97F4A7C15) & (2**64 - 1)],
                 dtype=np.uint64)
    return mix64(k)[0]


def draws(seed: int, stream: int, idx) -> np.ndarray:
    """uint64 draws for counter indices ``idx`` of ``stream``."""
    idx = np.asarray(idx, dtype=np.uint64)
    return mix64(_key(seed, stream) + (idx + np.uint64(1)) * GAMMA)


def draws_range(seed: int, stream: int, count: int, start: int = 0) -> np.ndarray:
    return draws(seed, stream, np.arange(start, start + count, dtype=np.uint64))


def uniform_below(bits: np.ndarray, n) -> np.ndarray:
    """Lemire multiply-shift: top 32 bits scaled into [0, n) for n <= 2^32."""
    n = np.asarray(n, dtype=np.uint64)
    return ((bits >> np.uint64(32)) * n) >> np.uint64(32)


def uniform01(bits: np.ndarray) -> np.ndarray:
    return (bits >> np.uint64(11)).astype(np.float64) * (1.0 / 9007199254740992.0)


# --------------------------------------------------------------------------
# Zipf(q) over ranks 1..n by rejection-inversion
# --------------------------------------------------------------------------
class Zipf:
    """Rejection-inversion sampler for P(k) proportional to k^-q, k in 1..n.

    With h(x) = x^-q and H an antiderivative of h, a continuous variate is
    drawn by inverting H on [H(1.5) - h(1), H(n + 0.5)], rounded to the
    nearest integer k, and accepted when it falls inside the region under
    the step function at k (Hoermann & Derflinger 1996, Sec. 3).
    """

    def __init__(self, n: int, q: float):
        if n < 1 or q <= 0:
            raise ValueError("Zipf needs n >= 1 and q > 0")
        self.n, self.q = int(n), float(q)
        self.a = 1.0 - self.q
        self.h_x1 = self.H(1.5) - 1.0
        self.h_n = self.H(self.n + 0.5)
        self.s = 2.0 - self.Hinv(self.H(2.5) - self.h(2.0))

    def h(self, x):
        return np.exp(-self.q * np.log(x))

    def H(self, x):
        lx = np.log(x)
        if abs(self.a) < 1e-12:
            return lx
        return np.expm1(self.a * lx) / self.a

    def Hinv(self, y):
        if abs(self.a) < 1e-12:
            return np.exp(y)
        t = np.maximum(y * self.a, -1.0 + 1e-300)
        return np.exp(np.log1p(t) / self.a)

    def pmf(self, k: np.ndarray) -> np.ndarray:
        """Exact probabilities, for tests (sums k^-q over the full support)."""
        ks = np.arange(1, self.n + 1, dtype=np.float64)
        z = np.sum(ks ** -self.q)
        return np.asarray(k, dtype=np.float64) ** -self.q / z

    def sample(self, seed: int, stream: int, count: int, start: int = 0) -> np.ndarray:
        out = np.zeros(count, dtype=np.int64)
        pending = np.arange(count, dtype=np.int64)
        for attempt in range(64):
            if pending.size == 0:
                break
            ctr = (pending + start).astype(np.uint64) * np.uint64(64) + np.uint64(attempt)
            u = self.h_n + uniform01(draws(seed, stream, ctr)) * (self.h_x1 - self.h_n)
            x = self.Hinv(u)
            k = np.clip(np.floor(x + 0.5), 1, self.n)
            acc = (k - x <= self.s) | (u >= self.H(k + 0.5) - self.h(k))
            out[pending[acc]] = k[acc].astype(np.int64)
            pending = pending[~acc]
        if pending.size:
            raise RuntimeError("Zipf sampler did not converge")
        return out


#: odd multiplier of the rank -> address bijection modulo a power of two
RANK_MULT = 2654435761


def rank_to_index(rank: np.ndarray, log2_n: int) -> np.ndarray:
    """Scatter Zipf rank r (1-based) over [0, 2^log2_n) by an odd-multiplier bijection."""
    m = np.uint64((1 << log2_n) - 1)
    r = np.asarray(rank, dtype=np.uint64) - np.uint64(1)
    return ((r * np.uint64(RANK_MULT)) & m).astype(np.uint32)


def permutation(seed: int, stream: int, n: int) -> np.ndarray:
    """Random permutation of 0..n-1 by sorting counter draws."""
    return np.argsort(draws_range(seed, stream, n), kind="stable").astype(np.int64)


# --------------------------------------------------------------------------
# streams (distinct ids per use)
# --------------------------------------------------------------------------
class S:
    INIT, SRC, DST, AMT = 1, 2, 3, 4
    CPU_SRC, CPU_DST, CPU_AMT = 5, 6, 7
    GRAN, HIT_G, HIT_W, ZIPF, VAL, TS, POS = 10, 11, 12, 13, 14, 15, 16
    PLANT, PLANT_VAL = 17, 18
    RMW_ADDR, RMW_UPD = 20, 21
    W2_ADDR, W2_UPD = 24, 25
    LOG_ADDR, LOG_VAL = 22, 23
    KEY, OP, PUTVAL, PREFILL = 30, 31, 32, 33
    ARRIVE, SIZE, KIND = 40, 41, 42


# --------------------------------------------------------------------------
# config 0: bank (one round, G = 4 B)
# --------------------------------------------------------------------------
@dataclass
class BankRound:
    n_accounts: int
    init: np.ndarray             # int32[N]
    gpu_tx: np.ndarray           # BANK_DTYPE[n_gpu]
    cpu_logs: list               # per CPU thread: LOG_DTYPE arrays
    cpu_final: np.ndarray        # host replica after the CPU transactions
    granule_bytes: int = 4

    @property
    def cpu_log(self) -> np.ndarray:
        return np.concatenate(self.cpu_logs) if self.cpu_logs else np.zeros(0, LOG_DTYPE)


def bank_transfers(seed: int, streams, count: int, lo: int, hi: int) -> np.ndarray:
    """`count` transfers over accounts [lo, hi): src uniform, dst != src, amount in 1..10."""
    s_src, s_dst, s_amt = streams
    span = hi - lo
    tx = np.zeros(count, dtype=BANK_DTYPE)
    src = uniform_below(draws_range(seed, s_src, count), span)
    off = uniform_below(draws_range(seed, s_dst, count), max(span - 1, 1))
    dst = (src + np.uint64(1) + off) % np.uint64(span)
    tx["src"] = (src + np.uint64(lo)).astype(np.uint32)
    tx["dst"] = (dst + np.uint64(lo)).astype(np.uint32)
    tx["amount"] = (uniform_below(draws_range(seed, s_amt, count), 10) + np.uint64(1)).astype(np.int32)
    return tx


def run_cpu_bank(init: np.ndarray, per_thread: list, ts_base: int = 0):
    """Execute CPU transfers in a fixed round-robin interleaving on a host replica.

    This stands in for the CPU guest TM: a serial execution is a legal STM
    history, and each commit hands <addr, value, ts> of both written words to
    the per-thread log, with ts a global commit clock (Sec. IV-B).
    """
    bal = init.astype(np.int64).copy()
    n_thr = len(per_thread)
    logs = [[] for _ in range(n_thr)]
    ts = ts_base
    longest = max((len(t) for t in per_thread), default=0)
    for i in range(longest):
        for t in range(n_thr):
            if i >= len(per_thread[t]):
                continue
            src, dst, amt = (int(per_thread[t][i]["src"]), int(per_thread[t][i]["dst"]),
                             int(per_thread[t][i]["amount"]))
            ts += 1
            bal[src] = _wrap32(bal[src] - amt)
            bal[dst] = _wrap32(bal[dst] + amt)
            logs[t].append((src, bal[src], ts))
            logs[t].append((dst, bal[dst], ts))
    out = []
    for t in range(n_thr):
        a = np.zeros(len(logs[t]), dtype=LOG_DTYPE)
        if logs[t]:
            arr = np.array(logs[t], dtype=np.int64)
            a["addr"], a["value"], a["ts"] = arr[:, 0], arr[:, 1], arr[:, 2]
        out.append(a)
    return out, bal.astype(np.int32)


def _wrap32(x: int) -> int:
    return ((int(x) + 2**31) % 2**32) - 2**31


def bank_round(seed: int = 0, n_accounts: int = 1 << 20, n_gpu: int = 65536,
               cpu_threads: int = 4, cpu_tx_per_thread: int = 10000,
               partitioned: bool = False, init_balance: int = 1000) -> BankRound:
    """Bank round: GPU batch and CPU per-thread logs over one STMR of accounts.

    ``partitioned`` confines the CPU to [0, N/2) and the GPU to [N/2, N), the
    disjoint-halves setup of Sec. V-B, which can never conflict.
    """
    init = np.full(n_accounts, init_balance, dtype=np.int32)
    half = n_accounts // 2
    g_lo, g_hi = (half, n_accounts) if partitioned else (0, n_accounts)
    c_lo, c_hi = (0, half) if partitioned else (0, n_accounts)
    gpu = bank_transfers(seed, (S.SRC, S.DST, S.AMT), n_gpu, g_lo, g_hi)
    per_thread = []
    for t in range(cpu_threads):
        all_cpu = bank_transfers(seed + 1000 * (t + 1), (S.CPU_SRC, S.CPU_DST, S.CPU_AMT),
                                 cpu_tx_per_thread, c_lo, c_hi)
        per_thread.append(all_cpu)
    logs, final = run_cpu_bank(init, per_thread)
    return BankRound(n_accounts, init, gpu, logs, final)


# --------------------------------------------------------------------------
# config 1: validation + merge at scale (planted GPU read/write sets)
# --------------------------------------------------------------------------
@dataclass
class ValidationRound:
    log2_words: int
    granule_bytes: int
    init: np.ndarray | None      # int32[N] (None: caller derives with init_words)
    read_granules: np.ndarray    # sorted uint32 granule ids read by the GPU batch
    plant_addr: np.ndarray       # uint32 words written by the GPU batch
    plant_value: np.ndarray      # int32 values written
    log: np.ndarray              # LOG_DTYPE[n]
    n_hits_planted: int
    meta: dict = field(default_factory=dict)


def init_words(seed: int, start: int, count: int) -> np.ndarray:
    """Initial STMR words: uniform int32, regenerable for any window."""
    return (draws_range(seed, S.INIT, count, start) >> np.uint64(32)).astype(np.uint32).view(np.int32)


def init_stmr(seed: int, n: int, chunk: int = 1 << 24) -> np.ndarray:
    """``init_words`` for the whole STMR, generated in bounded-memory chunks."""
    out = np.empty(n, dtype=np.int32)
    for s in range(0, n, chunk):
        out[s:s + chunk] = init_words(seed, s, min(chunk, n - s))
    return out


def validation_round(seed: int = 1, log2_words: int = 28, granule_bytes: int = 64,
                     read_frac: float = 0.05, n_log: int = 1 << 24, hit_frac: float = 0.02,
                     zipf_q: float = 0.9, write_frac_of_read: float = 0.20,
                     cpu_threads: int = 4, with_init: bool = True) -> ValidationRound:
    """Validation-at-scale round: planted read-set bitmap and a skewed CPU log.

    * ``read_frac`` of the granules are GPU-read (uniform, without replacement);
    * ``hit_frac`` of the log entries land on read granules (uniform granule,
      then uniform word); the rest are Zipf(q) ranks mapped to words,
      redrawn while they land on a read granule;
    * timestamps are a random permutation of 1..n_log, cut into
      ``cpu_threads`` contiguous per-thread segments, each sorted;
    * the GPU wrote every word of ``write_frac_of_read`` of the read granules.
    """
    n_words = 1 << log2_words
    wpg = granule_bytes // 4
    n_gran = n_words // wpg
    n_read = int(round(read_frac * n_gran))
    gperm = permutation(seed, S.GRAN, n_gran)
    read_g = np.sort(gperm[:n_read]).astype(np.uint32)
    is_read = np.zeros(n_gran, dtype=bool)
    is_read[read_g] = True

    n_hit = int(round(hit_frac * n_log))
    n_miss = n_log - n_hit
    # hits: uniform read granule, then uniform word inside it
    hg = read_g[uniform_below(draws_range(seed, S.HIT_G, n_hit), n_read).astype(np.int64)]
    hw = uniform_below(draws_range(seed, S.HIT_W, n_hit), wpg).astype(np.uint32)
    hit_addr = hg.astype(np.uint32) * np.uint32(wpg) + hw
    # misses: Zipf ranks over the words, redrawn while they hit a read granule
    z = Zipf(n_words, zipf_q)
    miss_addr = np.zeros(n_miss, dtype=np.uint32)
    pending = np.arange(n_miss, dtype=np.int64)
    redraw = 0
    while pending.size:
        r = z.sample(seed, S.ZIPF, pending.size, start=redraw * n_miss + 0)
        # distinct counters for every redraw pass: shift by pass * n_miss
        a = rank_to_index(r, log2_words)
        ok = ~is_read[a // wpg]
        miss_addr[pending[ok]] = a[ok]
        pending = pending[~ok]
        redraw += 1
        if redraw > 64:
            raise RuntimeError("miss address redraw did not converge")
    addr = np.concatenate([hit_addr, miss_addr])
    pos = permutation(seed, S.POS, n_log)
    log = np.zeros(n_log, dtype=LOG_DTYPE)
    log["addr"] = addr[pos]
    log["value"] = (draws_range(seed, S.VAL, n_log) >> np.uint64(32)).astype(np.uint32).view(np.int32)
    ts = (permutation(seed, S.TS, n_log) + 1).astype(np.uint32)
    seg = -(-n_log // cpu_threads)
    for t in range(cpu_threads):
        lo, hi = t * seg, min(n_log, (t + 1) * seg)
        ts[lo:hi] = np.sort(ts[lo:hi])
    log["ts"] = ts
    # GPU writes: every word of a subset of the read granules
    n_plant_g = int(round(write_frac_of_read * n_read))
    pg = np.sort(read_g[permutation(seed, S.PLANT, n_read)[:n_plant_g]])
    plant_addr = (pg.astype(np.uint64)[:, None] * np.uint64(wpg)
                  + np.arange(wpg, dtype=np.uint64)[None, :]).reshape(-1).astype(np.uint32)
    plant_value = (draws_range(seed, S.PLANT_VAL, plant_addr.size) >> np.uint64(32)).astype(
        np.uint32).view(np.int32)
    init = init_stmr(seed, n_words) if with_init else None
    return ValidationRound(log2_words, granule_bytes, init, read_g, plant_addr, plant_value,
                           log, n_hit, meta={"n_read_granules": n_read,
                                             "n_plant_granules": n_plant_g})


# --------------------------------------------------------------------------
# config 2: W1-style read/modify/write transactions under Zipf(0.99)
# --------------------------------------------------------------------------
def rmw_batch(seed: int, batch: int, n_tx: int, log2_words: int, q: float = 0.99,
              update_frac: float = 0.10, uniform: bool = False,
              lo: int = 0, hi: int | None = None) -> np.ndarray:
    """Transactions of 4 distinct word addresses; ``update_frac`` of them are updates.

    Addresses are Zipf(q) ranks scattered by the rank bijection, or uniform
    over [lo, hi) when ``uniform`` (the paper's W1 accesses the STMR uniformly).
    Duplicate addresses inside a transaction are redrawn.
    """
    n_words = 1 << log2_words
    hi = n_words if hi is None else hi
    tx = np.zeros(n_tx, dtype=RMW_DTYPE)
    base = batch * n_tx * 4
    z = None if uniform else Zipf(n_words, q)

    def gen(idx_counter):
        if uniform:
            return (uniform_below(draws(seed, S.RMW_ADDR, idx_counter), hi - lo)
                    + np.uint64(lo)).astype(np.uint32)
        r = np.empty(idx_counter.size, dtype=np.int64)
        # Zipf.sample indexes its own counters; draw through a per-element call
        r[:] = z.sample(seed, S.RMW_ADDR, idx_counter.size, start=int(idx_counter[0]))
        return rank_to_index(r, log2_words)

    addr = np.zeros((n_tx, 4), dtype=np.uint32)
    flat = gen(np.arange(base, base + n_tx * 4, dtype=np.uint64)).reshape(n_tx, 4)
    addr[:] = flat
    # redraw duplicates inside a transaction (fresh counters past the batch block)
    extra = 0
    while True:
        dup = np.zeros(n_tx, dtype=bool)
        for i in range(4):
            for j in range(i):
                dup |= addr[:, i] == addr[:, j]
        rows = np.nonzero(dup)[0]
        if rows.size == 0:
            break
        extra += 1
        ctr0 = (1 << 40) + (batch << 24) * 64 + extra * (n_tx * 4)
        fresh = gen(np.arange(ctr0, ctr0 + rows.size * 4, dtype=np.uint64)).reshape(-1, 4)
        addr[rows] = fresh
        if extra > 256:
            raise RuntimeError("duplicate redraw did not converge")
    tx["addr"] = addr
    upd = uniform01(draws_range(seed, S.RMW_UPD, n_tx, batch * n_tx)) < update_frac
    tx["flags"] = upd.astype(np.uint32)
    return tx


def w2_batch(seed: int, batch: int, n_tx: int, log2_words: int, update_frac: float = 0.10,
             lo: int = 0, hi: int | None = None) -> np.ndarray:
    """W2 of Sec. V-A: transactions of 40 distinct words drawn uniformly over
    [lo, hi); ``update_frac`` of them are updates (they write their first 4
    words).  A transaction with a repeated word is redrawn whole."""
    hi = (1 << log2_words) if hi is None else hi
    tx = np.zeros(n_tx, dtype=W2_DTYPE)
    base = batch * n_tx * 40

    def gen(c0, rows):
        ctr = np.arange(c0, c0 + rows * 40, dtype=np.uint64)
        return (uniform_below(draws(seed, S.W2_ADDR, ctr), hi - lo)
                + np.uint64(lo)).astype(np.uint32).reshape(rows, 40)

    addr = gen(base, n_tx)
    extra = 0
    while True:
        srt = np.sort(addr, axis=1)
        rows = np.nonzero((srt[:, 1:] == srt[:, :-1]).any(axis=1))[0]
        if rows.size == 0:
            break
        extra += 1
        addr[rows] = gen((1 << 41) + (batch << 24) * 64 + extra * (n_tx * 40), rows.size)
        if extra > 256:
            raise RuntimeError("duplicate redraw did not converge")
    tx["addr"] = addr
    upd = uniform01(draws_range(seed, S.W2_UPD, n_tx, batch * n_tx)) < update_frac
    tx["flags"] = upd.astype(np.uint32)
    return tx


def cpu_write_log(seed: int, rnd: int, n: int, log2_words: int, q: float = 0.99,
                  ts_base: int = 0, cpu_threads: int = 4, uniform: bool = False,
                  lo: int = 0, hi: int | None = None, offset: int = 0) -> list:
    """Per-thread CPU logs of plain writes for one round; ts = ts_base + 1 .. ts_base + n.

    Zipf addresses fall in [offset, offset + 2^log2_words): with ``offset`` the
    log covers another partition of the STMR than the GPU's (Sec. V-B splits
    the STMR in two halves, one per device)."""
    n_words = 1 << log2_words
    hi = n_words if hi is None else hi
    if uniform:
        addr = (uniform_below(draws_range(seed, S.LOG_ADDR, n, rnd * n), hi - lo)
                + np.uint64(lo)).astype(np.uint32)
    else:
        addr = (rank_to_index(Zipf(n_words, q).sample(seed, S.LOG_ADDR, n, start=rnd * n),
                              log2_words).astype(np.uint64) + np.uint64(offset)).astype(np.uint32)
    val = (draws_range(seed, S.LOG_VAL, n, rnd * n) >> np.uint64(32)).astype(np.uint32).view(np.int32)
    log = np.zeros(n, dtype=LOG_DTYPE)
    log["addr"], log["value"] = addr, val
    log["ts"] = np.arange(ts_base + 1, ts_base + n + 1, dtype=np.uint64).astype(np.uint32)
    # thread t owns commits t, t + T, t + 2T, ... (a round-robin commit clock)
    return [log[t::cpu_threads].copy() for t in range(cpu_threads)]


# --------------------------------------------------------------------------
# config 3: object cache (8-way set associative)
# --------------------------------------------------------------------------
@dataclass
class CacheLayout:
    """Word layout of the cache inside the STMR (structure-of-arrays per region).

    Per set s and way w:
      keys   : u64 at words key_base + 2*(8 s + w)      (one 64 B block per set)
      values : u64 at words val_base + 2*(8 s + w)
      gpu_lru: u32 at gpu_lru_base + 8 s + w            (GPU-local LRU stamps)
      cpu_lru: u32 at cpu_lru_base + 8 s + w            (CPU-local LRU stamps)
      version: u32 at ver_base + s                      (bumped by every PUT)
    """
    log2_sets: int
    ways: int = 8

    @property
    def n_sets(self):
        return 1 << self.log2_sets

    @property
    def key_base(self):
        return 0

    @property
    def val_base(self):
        return 2 * self.ways * self.n_sets

    @property
    def gpu_lru_base(self):
        return 4 * self.ways * self.n_sets

    @property
    def cpu_lru_base(self):
        return 5 * self.ways * self.n_sets

    @property
    def ver_base(self):
        return 6 * self.ways * self.n_sets

    @property
    def n_words(self):
        return 6 * self.ways * self.n_sets + self.n_sets


def set_of_key(keys: np.ndarray, log2_sets: int) -> np.ndarray:
    """Set index: SplitMix64 finalizer of the key, low bits."""
    return (mix64(np.asarray(keys, dtype=np.uint64)) & np.uint64((1 << log2_sets) - 1)).astype(np.uint32)


def cache_prefill(layout: CacheLayout, n_keys: int) -> np.ndarray:
    """Initial STMR image with keys 1..n_keys inserted in ascending order.

    A key goes to the first empty way of its set; a full set keeps its
    first 8 keys (later keys are simply not cached).  Values are key * 3,
    LRU stamps 0, versions 0.
    """
    img = np.zeros(layout.n_words, dtype=np.int32)
    keys = np.arange(1, n_keys + 1, dtype=np.uint64)
    sets = set_of_key(keys, layout.log2_sets).astype(np.int64)
    order = np.argsort(sets, kind="stable")
    ss = sets[order]
    first = np.searchsorted(ss, ss, side="left")
    way = np.arange(ss.size) - first
    keep = way < layout.ways
    slot = ss[keep] * layout.ways + way[keep]
    k = keys[order][keep]
    v = k * np.uint64(3)
    kw = img[layout.key_base: layout.val_base].view(np.uint64)
    vw = img[layout.val_base: layout.gpu_lru_base].view(np.uint64)
    kw[slot] = k
    vw[slot] = v
    return img


def cache_batch(seed: int, batch: int, n_req: int, n_keys: int, q: float = 0.99,
                get_frac: float = 0.90) -> np.ndarray:
    """GET/PUT requests with Zipf(q) key popularity over 1..n_keys (power of two)."""
    log2_keys = int(math.log2(n_keys))
    assert 1 << log2_keys == n_keys
    r = Zipf(n_keys, q).sample(seed, S.KEY, n_req, start=batch * n_req)
    keys = rank_to_index(r, log2_keys).astype(np.uint64) + np.uint64(1)
    req = np.zeros(n_req, dtype=CACHE_DTYPE)
    req["key"] = keys
    req["op"] = (uniform01(draws_range(seed, S.OP, n_req, batch * n_req)) >= get_frac).astype(np.uint32)
    req["value"] = draws_range(seed, S.PUTVAL, n_req, batch * n_req)
    return req


def log_uniform_sizes(seed: int, stream: int, count: int, lo: int, hi: int, start: int = 0):
    """Batch sizes log-uniform over [lo, hi]."""
    u = uniform01(draws_range(seed, stream, count, start))
    return np.floor(np.exp(np.log(lo) + u * (np.log(hi + 1) - np.log(lo)))).astype(np.int64).clip(lo, hi)


def poisson_arrivals(seed: int, count: int, rate_per_s: float) -> np.ndarray:
    """Arrival times (seconds) of a Poisson process: exponential inter-arrivals."""
    u = uniform01(draws_range(seed, S.ARRIVE, count))
    gaps = -np.log1p(-u) / rate_per_s
    return np.cumsum(gaps)

"""Pins for the CPU oracle (no GPU): hand-enumerated rounds, closed forms,
invariants and brute force.  Each test names the passage it pins."""
import itertools
import json
import os

import numpy as np
import pytest

import oracle
import workloads as wl

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _golden(name):
    with open(os.path.join(GOLDEN, name)) as f:
        return json.load(f)


def _log(rows):
    a = np.zeros(len(rows), wl.LOG_DTYPE)
    for i, (addr, val, ts) in enumerate(rows):
        a[i] = (addr, val, ts)
    return a


def _bank(rows):
    a = np.zeros(len(rows), wl.BANK_DTYPE)
    for i, r in enumerate(rows):
        a[i] = tuple(r)
    return a


def _rmw(rows):
    a = np.zeros(len(rows), wl.RMW_DTYPE)
    for i, r in enumerate(rows):
        a[i]["addr"] = r[:4]
        a[i]["flags"] = r[4]
    return a


@pytest.mark.parametrize("name", ["bank_no_conflict.json", "bank_conflict.json",
                                  "granule_false_sharing.json", "rmw_order.json",
                                  "rmw_order_swapped.json"])
def test_golden_round(name):
    """Hand-enumerated rounds (Sec. III P1; Sec. IV-C validation, TS, merge; Sec. IV-D)."""
    g = _golden(name)
    start = np.array(g["start"], np.int32)
    log = _log(g["log"])
    ex = g["expect"]
    if g["kind"] == "bank":
        res = oracle.round_bank(start, _bank(g["gpu_tx"]), g["order"], g["status"], log,
                                g["granule_bytes"], g["chunk_bytes"])
    else:
        res = oracle.round_rmw(start, _rmw(g["gpu_tx"]), g["order"], g["status"], log,
                               g["granule_bytes"], g["chunk_bytes"])
        st = np.array(g["status"])
        assert res.out[st == 1].tolist() == [o for o, s in zip(ex["out"], g["status"]) if s == 1]
    assert res.replayed.tolist() == ex["replayed"]
    assert res.R.tolist() == ex["R"]
    assert res.D.tolist() == ex["D"]
    assert res.flags.tolist() == ex["flags"]
    assert res.conflict == ex["conflict"]
    assert res.final.tolist() == ex["final"]
    assert res.ties == 0


def test_golden_ts_freshness():
    """Sec. IV-C: apply a tuple only if newer than the stored timestamp."""
    g = _golden("ts_freshness.json")
    state = np.array(g["start"], np.int32)
    ts = np.array(g["ts_state"], np.uint32)
    ties = oracle.cpu_image(state, ts, _log(g["log"]))
    assert state.tolist() == g["expect"]["final"]
    assert ts.tolist() == g["expect"]["ts_state"]
    assert ties == g["expect"]["ties"]


def _cache_image(g, layout):
    img = np.zeros(layout.n_words, np.int32)
    img[layout.key_base:layout.val_base].view(np.uint64)[:8] = g["keys"]
    img[layout.val_base:layout.gpu_lru_base].view(np.uint64)[:8] = g["values"]
    img[layout.gpu_lru_base:layout.gpu_lru_base + 8] = g["gpu_lru"]
    img[layout.ver_base] = g["version"]
    return img


@pytest.mark.parametrize("name", ["cache_one_set.json", "cache_evict.json"])
def test_golden_cache(name):
    """Sec. V-D object cache: GET/PUT, per-device LRU, per-set version."""
    g = _golden(name)
    layout = wl.CacheLayout(log2_sets=g["log2_sets"])
    assert layout.n_words == 49
    img = _cache_image(g, layout)
    reqs = np.zeros(len(g["reqs"]), wl.CACHE_DTYPE)
    for i, (k, v, op) in enumerate(g["reqs"]):
        reqs[i]["key"], reqs[i]["value"], reqs[i]["op"] = k, v, op
    out, R, D = oracle.replay_cache(img, layout, reqs, g["order"], g["status"],
                                    g["granule_bytes"], g["chunk_bytes"])
    ex = g["expect"]
    assert out.tolist() == ex["out"]
    assert img[0:16].view(np.uint64).tolist() == ex["keys"]
    assert img[16:32].view(np.uint64).tolist() == ex["values"]
    assert img[32:40].tolist() == ex["gpu_lru"]
    assert int(img[48]) == ex["version"]
    assert img[40:48].tolist() == [0] * 8          # the CPU LRU region is never touched
    assert R.tolist() == ex["R"] and D.tolist() == ex["D"]


def test_golden_cache_sets():
    """Sec. V-D object cache over four sets: the set index is the SplitMix64
    finalizer of the key (worked by hand in the golden), so a dropped hash,
    a wrong shift or constant puts a key in the wrong set and fails here."""
    g = _golden("cache_sets.json")
    layout = wl.CacheLayout(log2_sets=g["log2_sets"])
    assert layout.n_words == 196
    img = np.zeros(layout.n_words, np.int32)
    kw = img[layout.key_base:layout.val_base].view(np.uint64).reshape(4, 8)
    vw = img[layout.val_base:layout.gpu_lru_base].view(np.uint64).reshape(4, 8)
    for s_, (ks, vs) in enumerate(zip(g["start"]["keys"], g["start"]["values"])):
        kw[s_, :len(ks)] = ks
        vw[s_, :len(vs)] = vs
    reqs = np.zeros(len(g["reqs"]), wl.CACHE_DTYPE)
    for i, (k, v, op) in enumerate(g["reqs"]):
        reqs[i]["key"], reqs[i]["value"], reqs[i]["op"] = k, v, op
    out, R, D = oracle.replay_cache(img, layout, reqs, g["order"], g["status"],
                                    g["granule_bytes"], g["chunk_bytes"])
    ex = g["expect"]
    assert out.tolist() == ex["out"]
    assert kw.tolist() == ex["keys"]
    assert vw.tolist() == ex["values"]
    lru = img[layout.gpu_lru_base:layout.cpu_lru_base].reshape(4, 8)
    assert lru.tolist() == ex["gpu_lru"]
    assert img[layout.ver_base:layout.ver_base + 4].tolist() == ex["version"]
    assert img[layout.cpu_lru_base:layout.ver_base].tolist() == [0] * 32
    assert R.tolist() == ex["R"] and D.tolist() == ex["D"]


def _w2_golden_txs(g):
    txs = np.zeros(len(g["txs"]), wl.W2_DTYPE)
    spans = [list(range(0, 40)), list(range(2, 42)), [47, 46, 45, 44] + list(range(0, 36))]
    for i, t in enumerate(g["txs"]):
        txs[i]["addr"] = spans[i]
        txs[i]["flags"] = t["flags"]
    return txs


def test_golden_w2():
    """Sec. V-A W2 (40 reads): hand-derived sums and final words for two serial
    orders of the same three transactions."""
    g = _golden("w2_order.json")
    txs = _w2_golden_txs(g)
    for case in g["cases"]:
        st = np.arange(g["n_words"], dtype=np.int32)
        out, R, D = oracle.replay_w2(st, txs, case["order"], np.ones(3, np.uint8),
                                     g["granule_bytes"], g["chunk_bytes"])
        assert out.tolist() == case["out"]
        assert st[0:4].tolist() == g["expect_common"]["final_0_3"]
        assert st[44:48].tolist() == case["final_44_47"]
        assert st[4:44].tolist() == list(range(4, 44))
        assert R.tolist() == g["expect_common"]["R"] and D.tolist() == g["expect_common"]["D"]


def test_w2_with_zero_padding_reads_is_w1():
    """A W2 transaction whose 36 extra words hold 0 and are never written
    computes what the W1 transaction on its first 4 words computes."""
    n = 1 << 12
    w1 = wl.rmw_batch(seed=5, batch=0, n_tx=300, log2_words=11, update_frac=0.5)
    w2 = np.zeros(len(w1), wl.W2_DTYPE)
    w2["addr"][:, :4] = w1["addr"]
    w2["addr"][:, 4:] = (n // 2 + np.arange(36, dtype=np.uint32))[None, :] + \
        (np.arange(len(w1), dtype=np.uint32) % 7)[:, None] * 36
    w2["flags"] = w1["flags"]
    start = wl.init_words(5, 0, n)
    start[n // 2:] = 0
    order = np.arange(len(w1), dtype=np.uint64)[::-1] * 2 + 2   # reverse launch order
    status = np.ones(len(w1), np.uint8)
    s1, s2 = start.copy(), start.copy()
    o1, R1, D1 = oracle.replay_rmw(s1, w1, order, status, 4, 64, txid_base=11)
    o2, R2, D2 = oracle.replay_w2(s2, w2, order, status, 4, 64, txid_base=11)
    np.testing.assert_array_equal(o1, o2)
    np.testing.assert_array_equal(s1, s2)
    np.testing.assert_array_equal(D1, D2)
    np.testing.assert_array_equal(R2[R2 < n // 2], R1)
    assert (R2 >= n // 2).sum() == 36 + 6 * 36   # the padding words, one granule each


def test_cache_replay_finds_every_prefilled_key():
    """The prefill places keys by workloads.mix64 (pinned to published
    SplitMix64 outputs); a GET of every placed key through the oracle's own
    set index must hit and return the prefill's value (key * 3) on 256 sets."""
    layout = wl.CacheLayout(log2_sets=8)
    n_keys = 1024
    img = wl.cache_prefill(layout, n_keys)
    keys = np.arange(1, n_keys + 1, dtype=np.uint64)
    placed = np.isin(keys, img[layout.key_base:layout.val_base].view(np.uint64))
    assert placed.sum() > 0.95 * n_keys          # ~4 keys a set: few sets overflow
    reqs = np.zeros(int(placed.sum()), wl.CACHE_DTYPE)
    reqs["key"] = keys[placed]
    order = np.arange(1, reqs.size + 1, dtype=np.uint64) * 2
    out, _, _ = oracle.replay_cache(img.copy(), layout, reqs, order, np.ones(reqs.size, np.uint8),
                                    64, 64)
    np.testing.assert_array_equal(out, keys[placed] * np.uint64(3))
    # the keys the prefill could not place (full sets) miss
    missed = np.zeros(int((~placed).sum()), wl.CACHE_DTYPE)
    missed["key"] = keys[~placed]
    if missed.size:
        out, _, _ = oracle.replay_cache(img.copy(), layout, missed,
                                        np.arange(1, missed.size + 1, dtype=np.uint64) * 2 + 1,
                                        np.ones(missed.size, np.uint8), 64, 64)
        assert (out == np.uint64(2**64 - 1)).all()


# ---------------------------------------------------------------------------
# closed-form special cases (Sec. IV-C)
# ---------------------------------------------------------------------------
def _small_bank(seed=3, n=64, n_gpu=20, partitioned=False):
    return wl.bank_round(seed=seed, n_accounts=n, n_gpu=n_gpu, cpu_threads=2,
                         cpu_tx_per_thread=6, partitioned=partitioned)


def _all_committed(n):
    return np.arange(n, dtype=np.uint64) * 2 + 2, np.ones(n, np.uint8)


def test_empty_cpu_log_keeps_gpu_replay():
    """No CPU writes: validation cannot fail, final = GPU replay (Sec. IV-C)."""
    b = _small_bank()
    order, st = _all_committed(len(b.gpu_tx))
    res = oracle.round_bank(b.init, b.gpu_tx, order, st, np.zeros(0, wl.LOG_DTYPE), 4, 16)
    assert not res.conflict and res.n_conflicts == 0
    np.testing.assert_array_equal(res.final, res.replayed)


def test_empty_gpu_batch_gives_cpu_state():
    """No GPU transactions: final = start + CPU image = the CPU's own replica."""
    b = _small_bank()
    order, st = _all_committed(0)
    res = oracle.round_bank(b.init, b.gpu_tx[:0], order, st, b.cpu_log, 4, 16)
    assert not res.conflict
    np.testing.assert_array_equal(res.final, b.cpu_final)


def test_whole_stmr_granule_always_conflicts():
    """Granule = whole STMR, GPU read >= 1 word, log non-empty -> conflict."""
    b = _small_bank()
    order, st = _all_committed(len(b.gpu_tx))
    G = 4 * b.n_accounts
    res = oracle.round_bank(b.init, b.gpu_tx, order, st, b.cpu_log, G, G)
    assert res.conflict and res.flags.all()
    np.testing.assert_array_equal(res.final, b.cpu_final)


def test_partitioned_halves_never_conflict():
    """Sec. V-B setup: CPU and GPU on disjoint halves -> never a conflict; both kept."""
    b = _small_bank(partitioned=True)
    order, st = _all_committed(len(b.gpu_tx))
    res = oracle.round_bank(b.init, b.gpu_tx, order, st, b.cpu_log, 4, 16)
    assert not res.conflict
    half = b.n_accounts // 2
    np.testing.assert_array_equal(res.final[:half], b.cpu_final[:half])
    np.testing.assert_array_equal(res.final[half:], res.replayed[half:])
    np.testing.assert_array_equal(res.replayed[:half], b.init[:half])


def test_every_entry_on_read_granule_sets_every_flag():
    b = _small_bank()
    log = b.cpu_log
    flags, n = oracle.conflicts(log, np.unique(log["addr"] // 1), 4)
    assert n == len(log) and flags.all()


def test_conflict_flags_match_set_membership():
    """Brute-force check of the flags by numpy set membership (different algorithm)."""
    rng = np.random.default_rng(5)
    log = np.zeros(500, wl.LOG_DTYPE)
    log["addr"] = rng.integers(0, 4096, 500)
    for G in (4, 64, 1024):
        R = np.unique(rng.integers(0, 4096 * 4 // G, 40)).astype(np.uint32)
        flags, n = oracle.conflicts(log, R, G)
        expect = np.isin(log["addr"].astype(np.int64) * 4 // G, R)
        assert flags.astype(bool).tolist() == expect.tolist() and n == expect.sum()


def test_cpu_image_equals_sequential_apply_in_ts_order():
    """Newest-ts image == applying tuples one by one in timestamp order (Sec. IV-C)."""
    rng = np.random.default_rng(7)
    n_words = 32
    log = np.zeros(300, wl.LOG_DTYPE)
    log["addr"] = rng.integers(0, n_words, 300)
    log["value"] = rng.integers(-1000, 1000, 300)
    log["ts"] = rng.permutation(300) + 1
    ts0 = rng.integers(0, 150, n_words).astype(np.uint32)
    state = rng.integers(-5, 5, n_words).astype(np.int32)
    expect_state, expect_ts = state.copy(), ts0.copy()
    for e in sorted(log.tolist(), key=lambda r: r[2]):
        a, v, t = e
        if t > expect_ts[a]:
            expect_state[a], expect_ts[a] = v, t
    ts = ts0.copy()
    assert oracle.cpu_image(state, ts, log) == 0
    np.testing.assert_array_equal(state, expect_state)
    np.testing.assert_array_equal(ts, expect_ts)


def test_cpu_image_counts_ties():
    log = _log([(1, 5, 3), (1, 6, 3), (2, 1, 1)])
    assert oracle.cpu_image(None, np.zeros(4, np.uint32), log) == 1


# ---------------------------------------------------------------------------
# invariants
# ---------------------------------------------------------------------------
@pytest.mark.parametrize("partitioned", [False, True])
def test_bank_conservation_both_outcomes(partitioned):
    """Transfers conserve the int64 total under either outcome (bank invariant)."""
    b = wl.bank_round(seed=11, n_accounts=1 << 12, n_gpu=3000, cpu_threads=4,
                      cpu_tx_per_thread=300, partitioned=partitioned)
    order, st = _all_committed(len(b.gpu_tx))
    res = oracle.round_bank(b.init, b.gpu_tx, order, st, b.cpu_log, 4, 64)
    assert res.conflict == (not partitioned)
    assert oracle.sum64(res.final) == oracle.sum64(b.init) == 1000 * (1 << 12)
    if not partitioned:
        np.testing.assert_array_equal(res.final, b.cpu_final)


def test_sum64_does_not_overflow():
    x = np.full(1 << 12, 2**31 - 1, np.int32)
    assert oracle.sum64(x) == (2**31 - 1) * (1 << 12)


def test_rs_contains_ws_and_wrapping_arithmetic():
    """Writes are recorded in RS (Sec. IV-C) and int32 arithmetic wraps."""
    start = np.array([2**31 - 1, -2**31, 0, 0], np.int32)
    tx = _bank([(0, 1, 1)])
    res = oracle.round_bank(start, tx, [2], [1], np.zeros(0, wl.LOG_DTYPE), 4, 4)
    assert res.replayed.tolist() == [2**31 - 2, -2**31 + 1, 0, 0]
    tx = _bank([(1, 0, 5)])
    r2 = oracle.round_bank(start, tx, [2], [1], np.zeros(0, wl.LOG_DTYPE), 4, 4)
    assert r2.replayed.tolist() == [-2**31 + 4, 2**31 - 5, 0, 0]
    assert set(r2.D.tolist()) <= set(r2.R.tolist())


# ---------------------------------------------------------------------------
# brute force over serial orders (P1)
# ---------------------------------------------------------------------------
def test_replay_follows_reported_order_bruteforce():
    """For 3 conflicting transactions, each of the 6 orders gives its own state,
    and the replay of order p equals a direct hand-loop execution in order p."""
    start = np.array([3, 1, 4, 1, 5, 9, 2, 6], np.int32)
    txs = _rmw([[0, 1, 2, 3, 1], [2, 3, 4, 5, 1], [5, 6, 7, 0, 0]])
    seen = {}
    for perm in itertools.permutations(range(3)):
        order = np.zeros(3, np.uint64)
        for rank, i in enumerate(perm):
            order[i] = 2 * rank + 2
        st = start.copy()
        out, _, _ = oracle.replay_rmw(st, txs, order, np.ones(3, np.uint8), 4, 4)
        ref = start.astype(np.int64).tolist()
        ref_out = [0] * 3
        for i in perm:
            a = txs[i]["addr"].tolist()
            s = sum(ref[x] for x in a)
            s = ((s + 2**31) % 2**32) - 2**31
            ref_out[i] = s
            if txs[i]["flags"] & 1:
                for j, x in enumerate(a):
                    ref[x] = ((s + j + i + 2**31) % 2**32) - 2**31
        assert st.tolist() == ref and out.tolist() == ref_out
        seen[perm] = (tuple(st.tolist()), tuple(out.tolist()))
    assert len(set(seen.values())) == 6


def test_aborted_transactions_leave_no_trace():
    """Sec. IV-B: bitmaps are updated only at commit; aborted tx are not replayed."""
    start = np.arange(8, dtype=np.int32)
    txs = _rmw([[0, 1, 2, 3, 1], [4, 5, 6, 7, 1]])
    st = start.copy()
    out, R, D = oracle.replay_rmw(st, txs, [2, 0], [1, 2], 4, 4)
    assert R.tolist() == [0, 1, 2, 3] and D.tolist() == [0, 1, 2, 3]
    assert st[4:].tolist() == [4, 5, 6, 7]


# ---------------------------------------------------------------------------
# sizing sanity of the configurations
# ---------------------------------------------------------------------------
def test_bank_config_expects_conflict():
    """2^20 accounts, 65,536 GPU transfers vs 80,000 CPU writes: overlap ~ 1e4 words."""
    b = wl.bank_round(seed=0)
    gpu_words = np.union1d(b.gpu_tx["src"], b.gpu_tx["dst"])
    hits = np.isin(b.cpu_log["addr"], gpu_words).sum()
    assert len(b.cpu_log) == 80000 and 5000 < hits < 20000


def test_validation_config_hits_exact_at_small_scale():
    """The planted hit count is exact (2% of the log) at a reduced size."""
    v = wl.validation_round(seed=1, log2_words=18, n_log=1 << 15)
    flags, n = oracle.conflicts(v.log, v.read_granules, v.granule_bytes)
    assert n == v.n_hits_planted == round(0.02 * (1 << 15))


def _log_rows(rows):
    a = np.zeros(len(rows), wl.LOG_DTYPE)
    for i, r in enumerate(rows):
        a[i] = tuple(r)
    return a


def test_cpu_loses_policy_hand_enumerated():
    """Sec. IV-E: under CPU-loses the CPU write-sets are applied only after a
    clean validation.  Eight words 10..17; the GPU's replay wrote 99 into word 2
    and read word 3 (G = 4 B: granules 2 and 3)."""
    start = np.arange(10, 18, dtype=np.int32)
    replayed = start.copy()
    replayed[2] = 99
    R = np.array([2, 3], np.uint32)
    hit = _log_rows([(3, 50, 1), (6, 60, 2)])     # word 3 was read by the GPU
    clean = _log_rows([(6, 60, 2)])
    # conflict, GPU loses: start + CPU writes
    g = oracle.round_from_replay(start, replayed, R, hit, 4, np.zeros(8, np.uint32))
    assert g.conflict
    np.testing.assert_array_equal(g.final, [10, 11, 12, 50, 14, 15, 60, 17])
    # conflict, CPU loses: the GPU's state, no CPU write, TS untouched
    ts = np.zeros(8, np.uint32)
    c = oracle.round_from_replay(start, replayed, R, hit, 4, ts, cpu_loses=True)
    assert c.conflict
    np.testing.assert_array_equal(c.final, [10, 11, 99, 13, 14, 15, 16, 17])
    assert not ts.any()
    # no conflict: both policies give replay + CPU writes
    for cpu_loses in (False, True):
        r = oracle.round_from_replay(start, replayed, R, clean, 4, np.zeros(8, np.uint32),
                                     cpu_loses=cpu_loses)
        assert not r.conflict
        np.testing.assert_array_equal(r.final, [10, 11, 99, 13, 14, 15, 60, 17])


def test_cpu_baseline_mt_matches_oracle():
    """The timed multithreaded CPU baseline computes what the oracle defines:
    the same flags and hit count, and the same newest-timestamp apply."""
    v = wl.validation_round(seed=3, log2_words=18, n_log=1 << 15)
    n = 1 << 18
    wpg = v.granule_bytes // 4
    R = v.read_granules
    rs = np.zeros((n // wpg + 31) // 32, np.uint32)
    np.bitwise_or.at(rs, R // 32, (np.uint32(1) << (R % 32).astype(np.uint32)))
    ref_flags, ref_n = oracle.conflicts(v.log, R, v.granule_bytes)
    for threads in (1, 3, 8):
        W = v.init.copy()
        S = v.init.copy()
        TS = np.zeros(n, np.uint32)
        flags = np.zeros(len(v.log), np.uint8)
        hits = oracle.cpu_validate_apply_mt(v.log, rs, v.granule_bytes, W, S, TS, threads, flags)
        assert hits == ref_n == v.n_hits_planted
        np.testing.assert_array_equal(flags, ref_flags)
        want = v.init.copy()
        ts = np.zeros(n, np.uint32)
        assert oracle.cpu_image(want, ts, v.log) == 0
        np.testing.assert_array_equal(W, want)
        np.testing.assert_array_equal(S, want)
        np.testing.assert_array_equal(TS, ts)

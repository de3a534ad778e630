"""CUDA path vs the oracle, element by element, on seeded inputs (needs a GPU).

Every round is run through the C ABI (Python binding = marshalling only) and
compared bit-exact with the oracle: STMR^W after execution against the serial
replay in the GPU's reported commit order (P1), RS_bmp / WS_bmp against the
replay's granule and chunk sets, conflict flags against brute-force set
intersection, and the final STMR^W == STMR^S against the final-state rule.
Integer work throughout: the tolerance is zero.
"""
import json
import os
import threading

import numpy as np
import pytest

import oracle
import workloads as wl
import paper_1905_00661_b300.testing as hetm_testing
from roundkit import bits_of, check_keys, flags_of, gpu_bitmaps, submit, to_dev

pytestmark = pytest.mark.gpu
GOLDEN = os.path.join(os.path.dirname(__file__), "golden")
#: both GPU guest TMs: 0 = ordered (default), 1 = optimistic STM
MODES = [0, 1]


def cfg(mode, **kw):
    kw["exec_mode"] = mode
    return kw


@pytest.fixture(scope="module")
def torch():
    import torch as t
    if not t.cuda.is_available():
        pytest.skip("no CUDA device")
    return t


def _log(rows):
    a = np.zeros(len(rows), wl.LOG_DTYPE)
    for i, r in enumerate(rows):
        a[i] = tuple(r)
    return a


def _exec_and_check_replay(ctx, h, torch, start, batches, G, C, kind="rmw", layout=None):
    """Run the queued batches (one launch), then check STMR^W against the serial
    replay in the GPU's reported order and the bitmaps against the replay's sets.

    ``batches`` = [(records, BatchOut, txid_base)]; for RMW the bases must be
    cumulative so that the concatenation replays as one history."""
    ctx.gpu_exec()
    ctx.sync()
    torch.cuda.synchronize()
    W = ctx.read_stmr(h.STMR_W)
    S = ctx.read_stmr(h.STMR_S)
    np.testing.assert_array_equal(S, start)  # execution never touches the shadow
    rs_bits, ws_bits = gpu_bitmaps(ctx, h)
    keys = np.concatenate([b[1].host()[0] for b in batches])
    stat = np.concatenate([b[1].host()[1] for b in batches])
    got_out = np.concatenate([b[1].host()[2] for b in batches])
    check_keys(keys, stat)
    recs = np.concatenate([b[0] for b in batches])
    replayed = start.copy()
    if kind == "rmw":
        base0 = batches[0][2]
        sizes = np.cumsum([0] + [len(b[0]) for b in batches[:-1]])
        assert all(b[2] == base0 + int(o) for b, o in zip(batches, sizes))
        out, R, D = oracle.replay_rmw(replayed, recs, keys, stat, G, C, txid_base=base0)
        np.testing.assert_array_equal(got_out[stat == 1], out[stat == 1])
    elif kind == "bank":
        R, D = oracle.replay_bank(replayed, recs, keys, stat, G, C)
    else:
        out, R, D = oracle.replay_cache(replayed, layout, recs, keys, stat, G, C)
        np.testing.assert_array_equal(got_out.view(np.uint64)[stat == 1], out[stat == 1])
    np.testing.assert_array_equal(W, replayed)
    np.testing.assert_array_equal(rs_bits, R)
    np.testing.assert_array_equal(ws_bits, D)
    return replayed, R, D, keys, stat


def _finish_round(ctx, h, torch, start, replayed, R, log, G, ts_state=None, ship_threads=1):
    """Ship `log` (split over threads), validate with flags, merge; compare."""
    n = len(log)
    if ship_threads > 1:
        parts = np.array_split(log, ship_threads)
        th = [threading.Thread(target=ctx.cpu_log_write, args=(t, p)) for t, p in enumerate(parts)]
        [t.start() for t in th]
        [t.join() for t in th]
        shipped = np.concatenate(parts)
    else:
        if n:
            ctx.cpu_log_write(0, log)
        shipped = log
    flags = torch.zeros(max((n + 31) // 32, 1), dtype=torch.int32, device="cuda")
    n_conf = ctx.validate(flags=flags)
    ref = oracle.round_from_replay(start, replayed, R, shipped if ship_threads == 1 else log, G,
                                   np.zeros(start.size, np.uint32) if ts_state is None else ts_state)
    assert n_conf == ref.n_conflicts
    if ship_threads == 1:
        got = flags_of(flags.cpu().numpy().view(np.uint32), n)
        np.testing.assert_array_equal(got, ref.flags)
    ctx.merge(-1)
    ctx.sync()
    torch.cuda.synchronize()
    W = ctx.read_stmr(h.STMR_W)
    S = ctx.read_stmr(h.STMR_S)
    np.testing.assert_array_equal(W, ref.final)
    np.testing.assert_array_equal(S, ref.final)
    rs_bits, ws_bits = gpu_bitmaps(ctx, h)
    assert rs_bits.size == 0 and ws_bits.size == 0
    return ref


# ---------------------------------------------------------------------------
@pytest.mark.parametrize("mode", MODES)
@pytest.mark.parametrize("name", ["bank_no_conflict.json", "bank_conflict.json",
                                  "granule_false_sharing.json"])
def test_golden_bank_on_gpu(hetm, torch, name, mode):
    """Hand-enumerated bank rounds (Sec. IV-C) through the CUDA path."""
    g = json.load(open(os.path.join(GOLDEN, name)))
    h = hetm
    start = np.array(g["start"], np.int32)
    tx = np.zeros(len(g["gpu_tx"]), wl.BANK_DTYPE)
    for i, r in enumerate(g["gpu_tx"]):
        tx[i] = tuple(r)
    keep = np.array(g["status"]) == 1
    tx = tx[keep]
    with h.Context(len(start), g["granule_bytes"], cfg(mode, ws_chunk_bytes=16, lock_log2=4)) as ctx:
        ctx.load(start)
        b = submit(ctx, torch, wl.WORKLOAD_BANK, tx)
        replayed, R, D, _, _ = _exec_and_check_replay(ctx, h, torch, start, [(tx, b, 0)],
                                                      g["granule_bytes"], 16, kind="bank")
        assert replayed.tolist() == g["expect"]["replayed"]
        ref = _finish_round(ctx, h, torch, start, replayed, R, _log(g["log"]), g["granule_bytes"])
        assert ref.final.tolist() == g["expect"]["final"]
        assert ref.flags.tolist() == g["expect"]["flags"]


@pytest.mark.parametrize("mode", MODES)
@pytest.mark.parametrize("partitioned", [False, True])
def test_bank_config_round(hetm, torch, partitioned, mode):
    """Bank: 2^20 accounts, 65,536 GPU transfers, 4 x 10,000 CPU transfers, G = 4 B, seed 0."""
    h = hetm
    b = wl.bank_round(seed=0, partitioned=partitioned)
    with h.Context(b.n_accounts, 4, cfg(mode)) as ctx:
        ctx.load(b.init)
        bo = submit(ctx, torch, wl.WORKLOAD_BANK, b.gpu_tx)
        replayed, R, D, keys, stat = _exec_and_check_replay(ctx, h, torch, b.init,
                                                            [(b.gpu_tx, bo, 0)], 4, 16384,
                                                            kind="bank")
        assert (stat == 1).all()
        assert oracle.sum64(replayed) == oracle.sum64(b.init)
        ref = _finish_round(ctx, h, torch, b.init, replayed, R, b.cpu_log, 4)
        assert ref.conflict == (not partitioned)
        assert oracle.sum64(ref.final) == oracle.sum64(b.init)


@pytest.mark.parametrize("mode", MODES)
@pytest.mark.parametrize("uniform", [False, True])
def test_rmw_round(hetm, torch, uniform, mode):
    """W1-style transactions, Zipf(0.99) or uniform, 10% updates: replay parity + round."""
    h = hetm
    log2w, G = 16, 64
    start = wl.init_words(5, 0, 1 << log2w)
    tx = wl.rmw_batch(seed=5, batch=0, n_tx=30000, log2_words=log2w, uniform=uniform)
    log = wl.cpu_write_log(5, 0, 3000, log2w, cpu_threads=1, uniform=uniform)[0]
    with h.Context(1 << log2w, G, cfg(mode, ws_chunk_bytes=1024)) as ctx:
        ctx.load(start)
        bo = submit(ctx, torch, wl.WORKLOAD_RMW, tx, txid_base=7)
        replayed, R, D, keys, stat = _exec_and_check_replay(ctx, h, torch, start,
                                                            [(tx, bo, 7)], G, 1024)
        assert (stat == 1).all()
        _finish_round(ctx, h, torch, start, replayed, R, log, G)


@pytest.mark.parametrize("mode", MODES)
def test_rmw_uneven_batches_one_launch_and_per_batch(hetm, torch, mode):
    """Many uneven batches drained by one persistent launch, and one launch per batch."""
    h = hetm
    log2w, G = 15, 4
    start = wl.init_words(9, 0, 1 << log2w)
    sizes = [1, 31, 32, 33, 1000, 4097, 77, 12000]
    txs = [wl.rmw_batch(seed=9, batch=i, n_tx=n, log2_words=log2w) for i, n in enumerate(sizes)]
    for per_batch in (False, True):
        with h.Context(1 << log2w, G, cfg(mode, ws_chunk_bytes=64)) as ctx:
            ctx.load(start)
            bases = np.cumsum([0] + sizes[:-1])
            batches = [(t, submit(ctx, torch, wl.WORKLOAD_RMW, t, txid_base=int(bb)), int(bb))
                       for t, bb in zip(txs, bases)]
            if per_batch:
                ctx.gpu_exec(per_batch=True)
            _exec_and_check_replay(ctx, h, torch, start, batches, G, 64)


def test_optimistic_launches_above_the_listing_capacity(hetm, torch):
    """Optimistic executor with max_round_tx = 1000: a launch of at most 1000
    transactions hands the STM the list of updates its read-only phase left, a
    larger one is not listed and the STM draws every index.  Fused (one
    unlisted launch) and per batch (listed and unlisted launches): replay parity."""
    h = hetm
    log2w, G = 15, 4
    start = wl.init_words(19, 0, 1 << log2w)
    sizes = [1000, 33, 4097, 999, 1001]
    txs = [wl.rmw_batch(seed=19, batch=i, n_tx=n, log2_words=log2w, update_frac=0.3)
           for i, n in enumerate(sizes)]
    for per_batch in (False, True):
        with h.Context(1 << log2w, G, cfg(1, ws_chunk_bytes=64, max_round_tx=1000)) as ctx:
            ctx.load(start)
            bases = np.cumsum([0] + sizes[:-1])
            batches = [(t, submit(ctx, torch, wl.WORKLOAD_RMW, t, txid_base=int(bb)), int(bb))
                       for t, bb in zip(txs, bases)]
            if per_batch:
                ctx.gpu_exec(per_batch=True)
            _exec_and_check_replay(ctx, h, torch, start, batches, G, 64)


@pytest.mark.parametrize("n_log", [0, 1, 31, 128, (1 << 16) + 77])
def test_validation_planted(hetm, torch, n_log):
    """Validation-at-scale recipe at 2^20 words, ragged log sizes: flags, count, final."""
    h = hetm
    v = wl.validation_round(seed=1, log2_words=20, n_log=max(n_log, 1))
    log = v.log[:n_log]
    with h.Context(1 << 20, v.granule_bytes) as ctx:
        ctx.load(v.init)
        first = (v.read_granules.astype(np.uint64) * (v.granule_bytes // 4)).astype(np.uint32)
        hetm_testing.gpu_mark(ctx, torch.from_numpy(first).cuda())
        hetm_testing.gpu_mark(ctx, torch.from_numpy(v.plant_addr).cuda(), torch.from_numpy(v.plant_value).cuda())
        ref0 = oracle.round_planted(v.init, v.read_granules, v.plant_addr, v.plant_value,
                                    log, v.granule_bytes)
        rs_bits, ws_bits = gpu_bitmaps(ctx, h)
        np.testing.assert_array_equal(rs_bits, ref0.R)
        _finish_round(ctx, h, torch, v.init, ref0.replayed, ref0.R, log, v.granule_bytes)


def test_log_shipped_by_concurrent_threads(hetm, torch):
    """Four CPU threads append concurrently; chunks ship while they write (Sec. IV-D)."""
    h = hetm
    v = wl.validation_round(seed=2, log2_words=20, n_log=200000)
    with h.Context(1 << 20, v.granule_bytes, {"cpu_threads": 4, "log_chunk_bytes": 4800}) as ctx:
        ctx.load(v.init)
        first = (v.read_granules.astype(np.uint64) * (v.granule_bytes // 4)).astype(np.uint32)
        hetm_testing.gpu_mark(ctx, torch.from_numpy(first).cuda())
        ref0 = oracle.round_planted(v.init, v.read_granules, v.plant_addr[:0], v.plant_value[:0],
                                    v.log, v.granule_bytes)
        _finish_round(ctx, h, torch, v.init, ref0.replayed, ref0.R, v.log, v.granule_bytes,
                      ship_threads=4)


@pytest.mark.parametrize("mode", MODES)
def test_rounds_chain_with_graph(hetm, torch, mode):
    """Five whole rounds through hetm_round (captured graphs), TS carried across rounds."""
    h = hetm
    log2w, G = 16, 64
    n = 1 << log2w
    state = wl.init_words(3, 0, n)
    ts_state = np.zeros(n, np.uint32)
    with h.Context(n, G, cfg(mode, cpu_threads=2, ws_chunk_bytes=256)) as ctx:
        ctx.load(state)
        for r in range(5):
            uniform = r % 2 == 1
            tx = wl.rmw_batch(seed=3, batch=r, n_tx=20000, log2_words=log2w, uniform=uniform)
            logs = wl.cpu_write_log(3, r, 4000, log2w, ts_base=r * 4000, cpu_threads=2,
                                    uniform=uniform)
            bo = submit(ctx, torch, wl.WORKLOAD_RMW, tx, txid_base=r * 20000)
            for t, lg in enumerate(logs):
                ctx.cpu_log_write(t, lg)
            st = ctx.round(stats=True)
            assert st["rc"] == h.HETM_OK and st["n_log"] == 4000 and st["n_batches"] == 1
            # executor (ordered: sort + turn kernels + CTA segments; optimistic: one
            # launch) plus validation, apply and merge
            assert st["n_kernels"] >= (9 if mode == 0 else 4)
            keys, stat, out = bo.host()
            assert (stat == 1).all() and st["committed"] == 20000
            replayed = state.copy()
            rout, R, D = oracle.replay_rmw(replayed, tx, keys, stat, G, 256, txid_base=r * 20000)
            np.testing.assert_array_equal(out, rout)
            # ts_state is advanced in place by the oracle's apply
            ref = oracle.round_from_replay(state, replayed, R, np.concatenate(logs), G, ts_state)
            assert st["n_conflicts"] == ref.n_conflicts and bool(st["conflict"]) == ref.conflict
            W, S = ctx.read_stmr(h.STMR_W), ctx.read_stmr(h.STMR_S)
            np.testing.assert_array_equal(W, ref.final)
            np.testing.assert_array_equal(S, ref.final)
            state = ref.final


@pytest.mark.parametrize("mode", MODES)
def test_cache_round(hetm, torch, mode):
    """Object cache (Sec. V-D): GET/PUT replay parity, outputs, bitmaps, CPU PUT conflicts."""
    h = hetm
    lay = wl.CacheLayout(log2_sets=12)
    n_keys = 1 << 16
    start = wl.cache_prefill(lay, 1 << 15)
    cfg = {"lock_shift": 4, "cache_log2_sets": lay.log2_sets, "cache_key_base": lay.key_base,
           "cache_val_base": lay.val_base, "cache_lru_base": lay.gpu_lru_base,
           "cache_ver_base": lay.ver_base, "ws_chunk_bytes": 64, "exec_mode": mode}
    reqs = wl.cache_batch(seed=4, batch=0, n_req=40000, n_keys=n_keys)
    with h.Context(lay.n_words, 64, cfg) as ctx:
        ctx.load(start)
        bo = submit(ctx, torch, wl.WORKLOAD_CACHE, reqs)
        replayed, R, D, keys, stat = _exec_and_check_replay(ctx, h, torch, start, [(reqs, bo, 0)],
                                                            64, 64, kind="cache", layout=lay)
        assert (stat == 1).all()
        # CPU: PUT-shaped writes into the value region and the CPU LRU region
        log = np.zeros(500, wl.LOG_DTYPE)
        log["addr"] = np.concatenate([lay.cpu_lru_base + np.arange(250) * 8,
                                      lay.val_base + np.arange(250) * 16])
        log["value"] = np.arange(500)
        log["ts"] = np.arange(1, 501)
        _finish_round(ctx, h, torch, start, replayed, R, log, 64)


def test_validate_only_leaves_state(hetm, torch):
    """Early validation (Sec. IV-D): flags and count without applying anything."""
    h = hetm
    v = wl.validation_round(seed=6, log2_words=18, n_log=50001)
    with h.Context(1 << 18, v.granule_bytes) as ctx:
        ctx.load(v.init)
        first = (v.read_granules.astype(np.uint64) * (v.granule_bytes // 4)).astype(np.uint32)
        hetm_testing.gpu_mark(ctx, torch.from_numpy(first).cuda())
        dlog = to_dev(torch, v.log)
        flags = torch.zeros((len(v.log) + 31) // 32, dtype=torch.int32, device="cuda")
        cnt = torch.zeros(1, dtype=torch.int64, device="cuda")
        ctx.validate_only(dlog, len(v.log), flags, cnt)
        torch.cuda.synchronize()
        ref_flags, ref_n = oracle.conflicts(v.log, v.read_granules, v.granule_bytes)
        assert int(cnt.item()) == ref_n == v.n_hits_planted
        np.testing.assert_array_equal(flags_of(flags.cpu().numpy().view(np.uint32), len(v.log)),
                                      ref_flags)
        np.testing.assert_array_equal(ctx.read_stmr(h.STMR_W), v.init)


@pytest.mark.parametrize("mode", MODES)
def test_whole_stmr_granule_conflicts(hetm, torch, mode):
    """Granule = whole STMR: any GPU access + any CPU write conflicts."""
    h = hetm
    n = 4096
    start = np.arange(n, dtype=np.int32)
    tx = wl.rmw_batch(seed=8, batch=0, n_tx=100, log2_words=12, uniform=True)
    log = _log([(5, 1, 1)])
    with h.Context(n, 4 * n, cfg(mode, ws_chunk_bytes=4 * n)) as ctx:
        ctx.load(start)
        bo = submit(ctx, torch, wl.WORKLOAD_RMW, tx)
        replayed, R, D, _, _ = _exec_and_check_replay(ctx, h, torch, start, [(tx, bo, 0)], 4 * n,
                                                      4 * n)
        ref = _finish_round(ctx, h, torch, start, replayed, R, log, 4 * n)
        assert ref.conflict and ref.final[5] == 1


@pytest.mark.parametrize("mode", MODES)
def test_cache_one_hot_set_chunks(hetm, torch, mode):
    """One set, requests in launch order over whole 32-request chunks: chunks whose
    PUTs all update keys already in the set (GETs then read the newest value
    written to their way earlier in the chunk), and chunks with a PUT of an absent
    key into the full set (an eviction by stamp), followed by GETs of the new and
    the evicted key.  Outputs and the final STMR against the oracle's replay."""
    h = hetm
    lay = wl.CacheLayout(log2_sets=4)
    start = wl.cache_prefill(lay, 512)
    keys_of_set = start[lay.key_base: lay.val_base].view(np.uint64).reshape(lay.n_sets, 8)
    s = 5
    present = [int(k) for k in keys_of_set[s]]
    assert all(present) and len(set(present)) == 8
    allk = np.arange(1, 4096, dtype=np.uint64)
    absent = [int(k) for k in allk[wl.set_of_key(allk, lay.log2_sets) == s] if int(k) not in present][:3]
    k1, k2 = present[2], present[6]
    seq = []
    # chunk 1 and 2: PUTs that hit, GETs between them on the same and other ways
    for i in range(64):
        r = i % 8
        if r in (1, 5):
            seq.append((k1, 1000 + i, 1))
        elif r == 3:
            seq.append((k2, 2000 + i, 1))
        elif r == 7:
            seq.append((absent[0] if i % 16 == 7 else k2, 0, 0))
        else:
            seq.append((k1 if r % 2 == 0 else present[i % 8], 0, 0))
    # chunk 3: an eviction in the middle, then GETs of the new and an evicted key
    for i in range(32):
        if i == 10:
            seq.append((absent[1], 777, 1))
        elif i == 20:
            seq.append((absent[2], 888, 1))
        elif i % 3 == 0:
            seq.append((k1, 3000 + i, 1))
        else:
            seq.append(((absent[1], present[0], absent[2], k2)[i % 4], 0, 0))
    reqs = np.zeros(len(seq), dtype=wl.CACHE_DTYPE)
    reqs["key"] = [k for k, _, _ in seq]
    reqs["value"] = [v for _, v, _ in seq]
    reqs["op"] = [op for _, _, op in seq]
    cfg = {"lock_shift": 4, "cache_log2_sets": lay.log2_sets, "cache_key_base": lay.key_base,
           "cache_val_base": lay.val_base, "cache_lru_base": lay.gpu_lru_base,
           "cache_ver_base": lay.ver_base, "ws_chunk_bytes": 64, "exec_mode": mode}
    with h.Context(lay.n_words, 64, cfg) as ctx:
        ctx.load(start)
        bo = submit(ctx, torch, wl.WORKLOAD_CACHE, reqs)
        _, _, _, _, stat = _exec_and_check_replay(ctx, h, torch, start, [(reqs, bo, 0)], 64, 64,
                                                  kind="cache", layout=lay)
        assert (stat == 1).all()

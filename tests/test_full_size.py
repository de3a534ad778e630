"""CUDA path vs the oracle at full size (needs a GPU): the validation-at-scale
round, the RMW round configuration's 4M-transaction batch, the object-cache
configuration's 24 fused batches, and a serving mix of the serving
configuration's shapes.

The benchmark's validation workload, unchanged: 2^28 STMR words (1 GiB) and its
shadow, 64-byte granules (a 2 MiB RS_bmp), 5% of the granules read by the GPU
batch and every word of 20% of those written, and a 16,777,216-tuple CPU log
whose 2% planted hits land on read granules while the rest follow Zipf(0.9) off
them (Sec. IV-C validation, Sec. IV-D merge).  The kernels run in the launch
configuration the benchmark times (validation: one 1024-thread CTA per SM).
Every conflict flag, the conflict count, and every word of STMR^W and STMR^S
after the round are compared with the oracle; integer work, tolerance zero.
"""
import numpy as np
import pytest

import oracle
import workloads as wl
import paper_1905_00661_b300.testing as hetm_testing
from roundkit import flags_of, to_dev

pytestmark = pytest.mark.gpu
LOG2W = 28


@pytest.fixture(scope="module")
def torch():
    import torch as t
    if not t.cuda.is_available():
        pytest.skip("no CUDA device")
    return t


@pytest.fixture(scope="module")
def vr():
    return wl.validation_round(seed=1, log2_words=LOG2W, granule_bytes=64, with_init=False)


def _first_words(v):
    return (v.read_granules.astype(np.uint64) * (v.granule_bytes // 4)).astype(np.uint32)


def test_validate_only_full_size_every_flag(hetm, torch, vr):
    """Two validate-only calls in a row over the 16.8M-tuple log: every flag and the count."""
    h = hetm
    n = len(vr.log)
    ref_flags, ref_n = oracle.conflicts(vr.log, vr.read_granules, vr.granule_bytes)
    assert ref_n == vr.n_hits_planted
    with h.Context(1 << LOG2W, vr.granule_bytes, {"log_capacity": 1 << 12}) as ctx:
        hetm_testing.gpu_mark(ctx, torch.from_numpy(_first_words(vr)).cuda())
        dlog = to_dev(torch, vr.log)
        flags = torch.zeros((n + 31) // 32, dtype=torch.int32, device="cuda")
        cnt = torch.zeros(1, dtype=torch.int64, device="cuda")
        for _ in range(2):
            flags.fill_(-1)
            cnt.zero_()
            ctx.validate_only(dlog, n, flags, cnt)
            torch.cuda.synchronize()
            assert int(cnt.item()) == ref_n
            got = flags_of(flags.cpu().numpy().view(np.uint32), n)
            np.testing.assert_array_equal(got, ref_flags)
            # bits past the last tuple of the last flag word stay clear
            tail = flags.cpu().numpy().view(np.uint32)[-1] >> np.uint32(n % 32) if n % 32 else 0
            assert int(tail) == 0


@pytest.mark.parametrize("variant", ["conflict", "clean"])
def test_round_full_size_final_state(hetm, torch, vr, variant):
    """Validation + TS max, apply and merge of the whole round: the conflicting log
    (dirty chunks restored from S) and the log without its hits (dirty chunks W -> S)."""
    h = hetm
    wpg = vr.granule_bytes // 4
    log = vr.log
    if variant == "clean":
        is_read = np.zeros((1 << LOG2W) // wpg, dtype=bool)
        is_read[vr.read_granules] = True
        log = np.ascontiguousarray(log[~is_read[log["addr"] // wpg]])
    start = np.zeros(1 << LOG2W, np.int32)
    ref = oracle.round_planted(start, vr.read_granules, vr.plant_addr, vr.plant_value, log,
                               vr.granule_bytes)
    assert ref.ties == 0
    assert bool(ref.conflict) == (variant == "conflict")
    with h.Context(1 << LOG2W, vr.granule_bytes, {"log_capacity": 1 << 12, "cpu_threads": 1}) as ctx:
        ctx.load(torch.zeros(1 << LOG2W, dtype=torch.int32, device="cuda"))
        hetm_testing.gpu_mark(ctx, torch.from_numpy(_first_words(vr)).cuda())
        hetm_testing.gpu_mark(ctx, torch.from_numpy(vr.plant_addr).cuda(), torch.from_numpy(vr.plant_value).cuda())
        dlog = to_dev(torch, log)
        ctx.log_attach(dlog, len(log))
        st = ctx.round(stats=True)
        assert st["rc"] == h.HETM_OK
        assert st["n_conflicts"] == ref.n_conflicts
        assert bool(st["conflict"]) == bool(ref.conflict)
        np.testing.assert_array_equal(ctx.read_stmr(h.STMR_W), ref.final)
        np.testing.assert_array_equal(ctx.read_stmr(h.STMR_S), ref.final)


@pytest.mark.parametrize("mode,uniform", [(0, False), (1, False), (1, True)])
def test_executor_full_size_replay(hetm, torch, mode, uniform):
    """The RMW round configuration's batch at full size: 4M W1 transactions (10%
    updates, 4 distinct Zipf(0.99) words each over the lower 2^27 words of a
    2^28-word STMR) with 1 KiB granules and 16 KiB chunks: the ordered executor
    in 512-transaction segments (the shape the benchmark times) and the
    optimistic STM (256-thread CTAs; the hot words make it retry a lot), and
    the W1-uniform batch under the STM (its read-only phase lists the updates
    it leaves; Sec. V-A's W1, uniform words over the whole STMR).  The
    oracle replays the reported order: every committed transaction's sum,
    every word of STMR^W, and RS_bmp / WS_bmp exactly."""
    from roundkit import gpu_bitmaps, submit
    h = hetm
    g, c = 1024, 16384
    start = wl.init_stmr(2, 1 << LOG2W)
    tx = (wl.rmw_batch(seed=2, batch=7, n_tx=1 << 22, log2_words=LOG2W, uniform=True) if uniform
          else wl.rmw_batch(seed=2, batch=0, n_tx=1 << 22, log2_words=LOG2W - 1))
    cfg = {"exec_mode": mode, "exec_threads": 512 if mode == 0 else 256, "ws_chunk_bytes": c,
           "cpu_threads": 1}
    with h.Context(1 << LOG2W, g, cfg) as ctx:
        ctx.load(start)
        bo = submit(ctx, torch, wl.WORKLOAD_RMW, tx)
        ctx.gpu_exec()
        ctx.sync()
        torch.cuda.synchronize()
        w = ctx.read_stmr(h.STMR_W)
        rs_bits, ws_bits = gpu_bitmaps(ctx, h)
        keys, stat, out = bo.host()
    if mode == 0:
        assert (stat == 1).all()  # the ordered executor never aborts
    else:  # the STM's bounded retries may give some up: they must leave no trace
        assert np.isin(stat, [1, 2]).all() and (stat == 1).mean() > 0.9
    replayed = start.copy()
    ref_out, R, D = oracle.replay_rmw(replayed, tx, keys, stat, g, c)
    ok = stat == 1
    np.testing.assert_array_equal(out[ok], ref_out[ok])
    np.testing.assert_array_equal(w, replayed)
    np.testing.assert_array_equal(rs_bits, R)
    np.testing.assert_array_equal(ws_bits, D)


def test_object_cache_full_size_replay(hetm, torch):
    """The object-cache configuration at full size: 2^22 sets x 8 ways prefilled
    with 2^25 keys, 24 uneven batches (1K-512K requests, log-uniform, 90% GET,
    Zipf(0.99) over 2^26 keys) fused into one launch of the ordered executor.
    The oracle replays the reported order: every result, the cache regions of
    STMR^W, and RS_bmp / WS_bmp exactly."""
    from roundkit import gpu_bitmaps, submit
    h = hetm
    lay = wl.CacheLayout(22)
    start = wl.cache_prefill(lay, 1 << 25)
    sizes = wl.log_uniform_sizes(6, wl.S.SIZE, 24, 1 << 10, 1 << 19)
    reqs = [wl.cache_batch(6, i, int(n), 1 << 26) for i, n in enumerate(sizes)]
    cfg = {"cache_log2_sets": 22, "cache_key_base": lay.key_base, "cache_val_base": lay.val_base,
           "cache_lru_base": lay.gpu_lru_base, "cache_ver_base": lay.ver_base, "lock_shift": 4,
           "cpu_threads": 1, "ws_chunk_bytes": 16384}
    g, c = 64, 16384
    with h.Context(lay.n_words, g, cfg) as ctx:
        ctx.load(start)
        bos = [submit(ctx, torch, wl.WORKLOAD_CACHE, r) for r in reqs]
        ctx.gpu_exec()
        ctx.sync()
        torch.cuda.synchronize()
        w = ctx.read_stmr(h.STMR_W)
        rs_bits, ws_bits = gpu_bitmaps(ctx, h)
        res = [b.host() for b in bos]
    keys = np.concatenate([r[0] for r in res])
    stat = np.concatenate([r[1] for r in res])
    out = np.concatenate([r[2] for r in res]).view(np.uint64)
    assert (stat == 1).all()
    replayed = start.copy()
    ref_out, R, D = oracle.replay_cache(replayed, lay, np.concatenate(reqs), keys, stat, g, c)
    np.testing.assert_array_equal(out, ref_out)
    np.testing.assert_array_equal(w, replayed)
    np.testing.assert_array_equal(rs_bits, R)
    np.testing.assert_array_equal(ws_bits, D)


def test_serving_mix_full_size(hetm, torch):
    """The serving configuration's shapes at full size: one STMR holding the
    object cache (2^22 sets) and 2^26 bank accounts, 12 batches of 1K-1M
    transactions (log-uniform, bank or cache at random) submitted at once to
    the serving loop, which fuses them into rounds.  Every bank transfer
    commits and the accounts end at start + their net amounts (transfers
    commute); the cache requests, replayed by the oracle in the reported
    order, give every result and the final cache regions exactly."""
    h = hetm
    seed, n_batches, bank_log2 = 4, 12, 26
    lay = wl.CacheLayout(22)
    bank_base = (lay.n_words + 15) // 16 * 16
    start = np.zeros(bank_base + (1 << bank_log2), np.int32)
    start[:lay.n_words] = wl.cache_prefill(lay, 1 << 25)
    start[bank_base:] = 1000
    sizes = wl.log_uniform_sizes(seed, wl.S.SIZE, n_batches, 1 << 10, 1 << 20)
    kinds = wl.uniform01(wl.draws_range(seed, wl.S.KIND, n_batches)) < 0.5
    batches = [(1, wl.bank_transfers(seed * 1000 + i, (wl.S.SRC, wl.S.DST, wl.S.AMT), int(sizes[i]),
                                     0, 1 << bank_log2)) if kinds[i]
               else (3, wl.cache_batch(seed, i, int(sizes[i]), 1 << 26)) for i in range(n_batches)]
    assert {k for k, _ in batches} == {1, 3}
    cfg = {"cache_log2_sets": 22, "cache_key_base": lay.key_base, "cache_val_base": lay.val_base,
           "cache_lru_base": lay.gpu_lru_base, "cache_ver_base": lay.ver_base, "lock_shift": 4,
           "cpu_threads": 1}
    with h.Context(len(start), 64, cfg) as ctx:
        ctx.load(start)
        with h.Server(ctx) as srv:
            outs, ids = [], []
            for wk, tx in batches:
                o, s = np.zeros(len(tx), np.uint64), np.zeros(len(tx), np.uint8)
                out = np.zeros(len(tx), np.uint64) if wk == 3 else None
                ids.append(srv.submit(wk, tx, o, s, out, word_base=bank_base if wk == 1 else 0))
                outs.append((o, s, out))
            for i in ids:
                srv.wait(i)
        final = ctx.read_stmr(h.STMR_W)
        np.testing.assert_array_equal(final, ctx.read_stmr(h.STMR_S))
    bank = [(tx, o) for (wk, tx), o in zip(batches, outs) if wk == 1]
    expect = start[bank_base:].astype(np.int64)
    for tx, (o, s, _) in bank:
        assert (s == 1).all()
        np.add.at(expect, tx["src"], -tx["amount"].astype(np.int64))
        np.add.at(expect, tx["dst"], tx["amount"].astype(np.int64))
    np.testing.assert_array_equal(final[bank_base:], expect.astype(np.int32))
    cache = [(tx, o) for (wk, tx), o in zip(batches, outs) if wk == 3]
    reqs = np.concatenate([tx for tx, _ in cache])
    keys = np.concatenate([o[0] for _, o in cache])
    stat = np.concatenate([o[1] for _, o in cache])
    got = np.concatenate([o[2] for _, o in cache])
    assert (stat == 1).all()
    rep = start[:lay.n_words].copy()
    ref_out, _, _ = oracle.replay_cache(rep, lay, reqs, keys, stat, 64, 16384)
    np.testing.assert_array_equal(got, ref_out)
    np.testing.assert_array_equal(final[:lay.n_words], rep)

"""Serving loop (continuous batching into rounds) vs each batch run alone.

Bank batches on disjoint account ranges and an object-cache batch share one
STMR.  Submitted together to the server (fused rounds or one round per
batch), every batch must produce exactly what it produces alone on the same
start state -- per-transaction results and its region's final state -- and
that must equal the oracle's serial replay.  Integers: tolerance zero.
"""
import numpy as np
import pytest

import oracle
import workloads as wl

pytestmark = pytest.mark.gpu

LOG2_SETS = 10
RANGE = 4096
SIZES = [1000, 3000, 257, 5000]


def _setup():
    lay = wl.CacheLayout(LOG2_SETS)
    bank_base = (lay.n_words + 15) // 16 * 16
    n_words = bank_base + len(SIZES) * RANGE
    start = np.zeros(n_words, np.int32)
    start[:lay.n_words] = wl.cache_prefill(lay, 1 << (LOG2_SETS + 3))
    start[bank_base:] = 1000
    cfg = {"cache_log2_sets": LOG2_SETS, "cache_key_base": lay.key_base,
           "cache_val_base": lay.val_base, "cache_lru_base": lay.gpu_lru_base,
           "cache_ver_base": lay.ver_base, "ws_chunk_bytes": 256, "lock_shift": 4}
    banks = [wl.bank_transfers(40 + i, (wl.S.SRC, wl.S.DST, wl.S.AMT), n, 0, RANGE)
             for i, n in enumerate(SIZES)]
    cache = wl.cache_batch(seed=41, batch=0, n_req=2000, n_keys=1 << (LOG2_SETS + 4))
    return lay, bank_base, start, cfg, banks, cache


def _alone(h, start, cfg, workload, tx, word_base=0):
    import torch
    from roundkit import submit
    with h.Context(len(start), 64, cfg) as ctx:
        ctx.load(start)
        bo = submit(ctx, torch, workload, tx, word_base=word_base)
        st = ctx.round(stats=True)
        assert st["rc"] == h.HETM_OK
        keys, stat, out = bo.host()
        return ctx.read_stmr(h.STMR_W), keys, stat, out


@pytest.mark.parametrize("per_batch", [False, True])
@pytest.mark.parametrize("mode", [0, 1])
def test_mix_equals_alone_and_oracle(hetm, per_batch, mode):
    h = hetm
    lay, bank_base, start, cfg, banks, cache = _setup()
    cfg = dict(cfg, exec_mode=mode)
    with h.Context(len(start), 64, cfg) as ctx:
        ctx.load(start)
        with h.Server(ctx, per_batch=per_batch) as srv:
            ids = []
            outs = []
            for i, tx in enumerate(banks):
                o, s = np.zeros(len(tx), np.uint64), np.zeros(len(tx), np.uint8)
                ids.append(srv.submit(h.HETM_WL_BANK, tx, o, s, word_base=bank_base + i * RANGE))
                outs.append((o, s, None))
            o, s, out = (np.zeros(len(cache), np.uint64), np.zeros(len(cache), np.uint8),
                         np.zeros(len(cache), np.uint64))
            ids.append(srv.submit(h.HETM_WL_CACHE, cache, o, s, out))
            outs.append((o, s, out))
            lat = [srv.wait(i) for i in ids]
            st = srv.stats()
        final = ctx.read_stmr(h.STMR_W)
        np.testing.assert_array_equal(final, ctx.read_stmr(h.STMR_S))
    assert st["completed"] == len(ids) and st["committed"] == sum(SIZES) + len(cache)
    assert all(x > 0 for x in lat)
    if per_batch:
        assert st["rounds"] == len(ids)
    for i, tx in enumerate(banks):
        o, s, _ = outs[i]
        assert (s == 1).all()
        lo, hi = bank_base + i * RANGE, bank_base + (i + 1) * RANGE
        w_alone, k_alone, s_alone, _ = _alone(h, start, cfg, h.HETM_WL_BANK, tx, lo)
        np.testing.assert_array_equal(final[lo:hi], w_alone[lo:hi])  # transfers commute
        # oracle: the range replayed alone in the reported order
        rep = start.copy()
        txo = tx.copy()
        txo["src"] += lo
        txo["dst"] += lo
        oracle.replay_bank(rep, txo, o, s, 64, 256)
        np.testing.assert_array_equal(final[lo:hi], rep[lo:hi])
        assert oracle.sum64(final[lo:hi]) == 1000 * RANGE
    o, s, out = outs[-1]
    assert (s == 1).all()
    if mode == 0:
        # the ordered executor fixes the serial order by launch index, so the
        # cache batch sees exactly the same history alone and in the mix; the
        # optimistic one may pick another (equally serializable) order of
        # requests on one set, so only its oracle replay is checked
        w_alone, _, _, out_alone = _alone(h, start, cfg, h.HETM_WL_CACHE, cache)
        np.testing.assert_array_equal(out, out_alone.view(np.uint64))
        ckeys = slice(lay.key_base, lay.gpu_lru_base)  # keys and values
        np.testing.assert_array_equal(final[ckeys], w_alone[ckeys])
    rep = start.copy()
    rout, _, _ = oracle.replay_cache(rep, lay, cache, o, s, 64, 256)
    np.testing.assert_array_equal(out, rout)
    np.testing.assert_array_equal(final[:lay.n_words], rep[:lay.n_words])


def test_admission_by_device_budget(hetm):
    """A budget that holds one batch at a time still serves every batch, in order."""
    h = hetm
    lay, bank_base, start, cfg, banks, cache = _setup()
    with h.Context(len(start), 64, cfg) as ctx:
        ctx.load(start)
        with h.Server(ctx, device_budget=120_000) as srv:
            big = wl.bank_transfers(7, (wl.S.SRC, wl.S.DST, wl.S.AMT), 20000, 0, RANGE)
            with pytest.raises(h.HetmError) as e:
                srv.submit(h.HETM_WL_BANK, big, word_base=bank_base)
            assert e.value.code == h.HETM_EBUSY
            ids = [srv.submit(h.HETM_WL_BANK, tx, word_base=bank_base + i * RANGE)
                   for i, tx in enumerate(banks)]
            for i in ids:
                srv.wait(i)
            st = srv.stats()
        assert st["completed"] == len(banks) and st["refused"] == 1
        assert st["rounds"] >= 2
        final = ctx.read_stmr(h.STMR_W)
        for i in range(len(banks)):
            lo = bank_base + i * RANGE
            assert oracle.sum64(final[lo:lo + RANGE]) == 1000 * RANGE


def test_admission_follows_free_device_memory(hetm):
    """Admission reads the device's free memory at every admission, so memory
    taken by another allocation after the server started is seen: with
    admission leaving all but ~600 MB free, a 48 MB batch is served; once a
    1 GB tensor is allocated beside the server the same batch no longer fits
    (nothing is in flight to free memory: it completes with HETM_ENOMEM);
    after the tensor is released it is served again."""
    import torch
    h = hetm
    lay, bank_base, start, cfg, banks, cache = _setup()
    tx = wl.bank_transfers(8, (wl.S.SRC, wl.S.DST, wl.S.AMT), 1 << 21, 0, RANGE)  # ~48 MB on device
    with h.Context(len(start), 64, cfg) as ctx:
        ctx.load(start)
        torch.cuda.synchronize()
        torch.cuda.empty_cache()
        free, _ = torch.cuda.mem_get_info()
        reserve = free - (600 << 20)
        with h.Server(ctx, free_reserve=reserve) as srv:
            srv.wait(srv.submit(h.HETM_WL_BANK, tx, word_base=bank_base))
            hog = torch.empty(1 << 30, dtype=torch.uint8, device="cuda")
            torch.cuda.synchronize()
            bid = srv.submit(h.HETM_WL_BANK, tx, word_base=bank_base)
            with pytest.raises(h.HetmError) as e:
                srv.wait(bid)
            assert e.value.code == h.HETM_ENOMEM
            del hog
            torch.cuda.synchronize()
            torch.cuda.empty_cache()
            srv.wait(srv.submit(h.HETM_WL_BANK, tx, word_base=bank_base))
            st = srv.stats()
        assert st["refused"] == 1
        final = ctx.read_stmr(h.STMR_W)
        assert oracle.sum64(final[bank_base:bank_base + RANGE]) == 1000 * RANGE

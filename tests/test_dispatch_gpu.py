"""Dispatcher over the serving loop on the GPU (Sec. III-B dispatching, Sec. IV-C
rounds, needs a GPU).

1. Exactly once under rollback: CPU-only requests write CPU log tuples to
   words that share 64-byte granules with the accounts of GPU-only bank
   transfers, so the first round that runs transfers conflicts and the GPU
   batch is undone (GPU loses).  The dispatcher re-queues it; in the end every
   transfer has run once: each account holds its start balance plus the
   transfers' net amount (transfers commute), the poked words hold the CPU
   values, and W == S.
2. Results: object-cache requests through the dispatcher (one activation)
   give the per-request results and final cache state of the same requests
   run as one batch on their own, and of the oracle's serial replay.
Integers throughout: tolerance zero.
"""
import itertools
import threading

import numpy as np
import pytest

import oracle
import workloads as wl

pytestmark = pytest.mark.gpu

BANK = np.dtype([("src", "<u4"), ("dst", "<u4"), ("amount", "<i4")])
POKE = np.dtype([("addr", "<u4"), ("value", "<i4")])


def test_rolled_back_transfers_run_exactly_once(hetm):
    h = hetm
    n_words, n_acc = 1 << 16, 512          # accounts at even words 0 .. 1022
    rng = np.random.default_rng(11)
    tx = np.zeros(8192, BANK)
    a = rng.integers(0, n_acc, tx.size)
    b = (a + 1 + rng.integers(0, n_acc - 1, tx.size)) % n_acc
    tx["src"], tx["dst"] = 2 * a, 2 * b
    tx["amount"] = rng.integers(1, 10, tx.size)
    pokes = np.zeros(64, POKE)
    pokes["addr"] = 2 * rng.choice(n_acc, pokes.size, replace=False) + 1
    pokes["value"] = rng.integers(-10**6, 10**6, pokes.size)
    ts = itertools.count(1)
    ts_lock = threading.Lock()

    start = np.full(n_words, 1000, np.int32)
    with h.Context(n_words, 64, {"cpu_threads": 2, "ws_chunk_bytes": 256}) as ctx:
        ctx.load(start)

        def poke(worker, rec):
            r = np.frombuffer(rec, POKE)[0]
            with ts_lock:
                t = next(ts)
            e = np.zeros(1, h.LOG_DTYPE)
            e["addr"], e["value"], e["ts"] = r["addr"], r["value"], t
            ctx.cpu_log_write(worker, e)
            return 1, None

        with h.Server(ctx) as srv:
            with h.Dispatcher(srv, cpu_workers=2, gpu_min_batch=1024, gpu_max_wait_us=2000) as d:
                tp = d.register(8, cpu_fn=poke)
                tb = d.register(12, gpu_workload=h.HETM_WL_BANK)
                p = d.submit(tp, pokes)
                d.wait(p[0])             # the CPU log now holds every poke
                subs = [d.submit(tb, tx[i:i + 2048]) for i in range(0, tx.size, 2048)]
                for s in subs:
                    d.wait(s[0])
                st = d.stats()
            sst = srv.stats()
        w = ctx.read_stmr(h.STMR_W)
        np.testing.assert_array_equal(w, ctx.read_stmr(h.STMR_S))
    assert (p[3] == h.HETM_DEVICE_CPU).all() and (p[1] == 1).all()
    for s in subs:
        assert (s[3] == h.HETM_DEVICE_GPU).all() and (s[1] == 1).all()
    assert st["requeued"] >= 1, st          # the first transfer round was undone
    assert st["gpu_done"] == tx.size and st["cpu_done"] == pokes.size
    assert sst["rounds"] >= 2
    expect = start.astype(np.int64)
    np.add.at(expect, tx["src"], -tx["amount"].astype(np.int64))
    np.add.at(expect, tx["dst"], tx["amount"].astype(np.int64))
    expect[pokes["addr"]] = pokes["value"]
    np.testing.assert_array_equal(w, expect.astype(np.int32))


def test_cache_requests_match_a_batch_alone_and_the_oracle(hetm):
    import torch
    from roundkit import submit
    h = hetm
    log2_sets = 10
    lay = wl.CacheLayout(log2_sets)
    start = np.zeros(lay.n_words, np.int32)
    start[:] = wl.cache_prefill(lay, 1 << (log2_sets + 3))
    cfg = {"cache_log2_sets": log2_sets, "cache_key_base": lay.key_base,
           "cache_val_base": lay.val_base, "cache_lru_base": lay.gpu_lru_base,
           "cache_ver_base": lay.ver_base, "ws_chunk_bytes": 256}
    reqs = wl.cache_batch(seed=43, batch=0, n_req=3000, n_keys=1 << (log2_sets + 4))
    with h.Context(lay.n_words, 64, cfg) as ctx:
        ctx.load(start)
        with h.Server(ctx) as srv:
            with h.Dispatcher(srv, cpu_workers=0, gpu_min_batch=len(reqs)) as d:
                t = d.register(24, gpu_workload=h.HETM_WL_CACHE, out_bytes=8)
                tk, status, out, dev = d.submit(t, reqs)
                d.wait(tk)
                st = d.stats()
        final = ctx.read_stmr(h.STMR_W)
    assert st["activations"] == 1 and (dev == h.HETM_DEVICE_GPU).all() and (status == 1).all()
    out = out.view(np.uint64)
    with h.Context(lay.n_words, 64, cfg) as ctx:
        ctx.load(start)
        bo = submit(ctx, torch, h.HETM_WL_CACHE, reqs)
        assert ctx.round(stats=True)["rc"] == h.HETM_OK
        keys, stat, out_alone = bo.host()
        w_alone = ctx.read_stmr(h.STMR_W)
    np.testing.assert_array_equal(out, out_alone.view(np.uint64))
    ckeys = slice(lay.key_base, lay.gpu_lru_base)  # keys and values
    np.testing.assert_array_equal(final[ckeys], w_alone[ckeys])
    rep = start.copy()
    rout, _, _ = oracle.replay_cache(rep, lay, reqs, keys, stat, 64, 256)
    np.testing.assert_array_equal(out, rout)
    np.testing.assert_array_equal(final[:lay.n_words], rep[:lay.n_words])

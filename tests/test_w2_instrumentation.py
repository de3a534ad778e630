"""W2 (40 reads, Sec. V-A) and the uninstrumented executor, against the oracle
(needs a GPU).

* W2 batches under both executors (read-only transactions in the read-only
  phase, updates under the STM with reads validated against a clock
  snapshot -- with the launch's other updates in optimistic mode, after the
  ordered phase in ordered mode): STMR^W after execution equals the serial
  replay in the GPU's reported commit order, every committed sum equals the
  replay's, and RS_bmp / WS_bmp equal the replay's granule and chunk sets.
  A small STMR makes the 40-word read sets collide often, so validation
  failures and retries are exercised; then a whole round (CPU log,
  validation, merge) against the oracle's final state.
* In ordered mode, W2 mixed with W1 updates in one launch: the W2 updates
  commit after every W1 transaction of the launch, and the replay of both in
  the reported order reproduces STMR^W.
* uninstrumented = 1 (what Sec. V-A measures instrumentation costs against):
  the same transactions give the same STMR^W and outputs, and RS_bmp and
  WS_bmp stay empty.
Integer work: the tolerance is zero.
"""
import numpy as np
import pytest

import oracle
import workloads as wl
from roundkit import check_keys, gpu_bitmaps, submit

pytestmark = pytest.mark.gpu
G, C = 64, 1024


@pytest.fixture(scope="module")
def torch():
    import torch as t
    if not t.cuda.is_available():
        pytest.skip("no CUDA device")
    return t


def _exec(ctx, h, torch, batches):
    ctx.gpu_exec()
    ctx.sync()
    torch.cuda.synchronize()
    keys = np.concatenate([b.host()[0] for b in batches])
    stat = np.concatenate([b.host()[1] for b in batches])
    out = np.concatenate([b.host()[2] for b in batches])
    return keys, stat, out


@pytest.mark.parametrize("mode", [1, 0])
@pytest.mark.parametrize("log2w,n_tx,upd", [(16, 30000, 0.1), (16, 30000, 0.9), (12, 6000, 0.5)])
def test_w2_matches_the_oracle(hetm, torch, log2w, n_tx, upd, mode):
    h = hetm
    n = 1 << log2w
    start = wl.init_words(41, 0, n)
    # two uneven batches in one launch (txid bases continue across them)
    tx = wl.w2_batch(seed=41, batch=0, n_tx=n_tx, log2_words=log2w, update_frac=upd)
    cut = n_tx // 3
    with h.Context(n, G, {"exec_mode": mode, "ws_chunk_bytes": C, "cpu_threads": 1}) as ctx:
        ctx.load(start)
        b0 = submit(ctx, torch, wl.WORKLOAD_W2, tx[:cut], txid_base=100)
        b1 = submit(ctx, torch, wl.WORKLOAD_W2, tx[cut:], txid_base=100 + cut)
        keys, stat, out = _exec(ctx, h, torch, [b0, b1])
        assert (stat == 1).all()
        check_keys(keys, stat)
        W = ctx.read_stmr(h.STMR_W)
        rs_bits, ws_bits = gpu_bitmaps(ctx, h)
        replayed = start.copy()
        ref_out, R, D = oracle.replay_w2(replayed, tx, keys, stat, G, C, txid_base=100)
        np.testing.assert_array_equal(out, ref_out)
        np.testing.assert_array_equal(W, replayed)
        np.testing.assert_array_equal(rs_bits, R)
        np.testing.assert_array_equal(ws_bits, D)
        # the rest of the round: a CPU log on words the batch read, validation, merge
        log = np.concatenate(wl.cpu_write_log(42, 0, 500, log2w, cpu_threads=1, uniform=True))
        ctx.cpu_log_write(0, log)
        n_conf = ctx.validate()
        ref = oracle.round_from_replay(start, replayed, R, log, G, np.zeros(n, np.uint32))
        assert n_conf == ref.n_conflicts
        ctx.merge(-1)
        ctx.sync()
        np.testing.assert_array_equal(ctx.read_stmr(h.STMR_W), ref.final)
        np.testing.assert_array_equal(ctx.read_stmr(h.STMR_S), ref.final)
        if log2w == 12:
            assert ctx.exec_counters()["aborts"] > 0  # the contended case retried


def test_ordered_mode_runs_w2_after_its_ordered_phase(hetm, torch):
    h = hetm
    n = 1 << 13
    start = wl.init_words(45, 0, n)
    w1 = wl.rmw_batch(seed=45, batch=0, n_tx=5000, log2_words=13, update_frac=0.5)
    w2 = wl.w2_batch(seed=46, batch=0, n_tx=2000, log2_words=13, update_frac=0.5)
    with h.Context(n, G, {"exec_mode": 0, "ws_chunk_bytes": C, "cpu_threads": 1}) as ctx:
        ctx.load(start)
        b1 = submit(ctx, torch, wl.WORKLOAD_RMW, w1, txid_base=0)
        b2 = submit(ctx, torch, wl.WORKLOAD_W2, w2, txid_base=7)
        k1, s1, o1 = _exec(ctx, h, torch, [b1])
        k2, s2, o2 = b2.host()
        assert (s1 == 1).all() and (s2 == 1).all()
        upd1 = w1["flags"] == 1
        upd2 = w2["flags"] == 1
        # W2 updates after every W1 transaction; W2 read-only ones before every update
        assert k2[upd2].min() > k1.max()
        assert k2[~upd2].max() < k1[upd1].min()
        # one history: replay both kinds merged by their commit keys
        rep = start.copy()
        order = np.argsort(np.concatenate([k1, k2]), kind="stable")
        ref1, ref2 = np.zeros(len(w1), np.int32), np.zeros(len(w2), np.int32)
        for i in order:
            if i < len(w1):
                one = w1[i:i + 1]
                out, _, _ = oracle.replay_rmw(rep, one, [2], [1], G, C, txid_base=int(i))
                ref1[i] = out[0]
            else:
                j = i - len(w1)
                one = w2[j:j + 1]
                out, _, _ = oracle.replay_w2(rep, one, [2], [1], G, C, txid_base=7 + int(j))
                ref2[j] = out[0]
        np.testing.assert_array_equal(o1, ref1)
        np.testing.assert_array_equal(o2, ref2)
        np.testing.assert_array_equal(ctx.read_stmr(h.STMR_W), rep)


@pytest.mark.parametrize("mode,kind", [(1, "w1"), (1, "w2"), (0, "w1"), (0, "w2")])
def test_uninstrumented_executor_records_nothing(hetm, torch, mode, kind):
    h = hetm
    n = 1 << 14
    start = wl.init_words(44, 0, n)
    if kind == "w1":
        tx = wl.rmw_batch(seed=44, batch=0, n_tx=8000, log2_words=14, update_frac=0.5)
        wk, replay = wl.WORKLOAD_RMW, oracle.replay_rmw
    else:
        tx = wl.w2_batch(seed=44, batch=0, n_tx=4000, log2_words=14, update_frac=0.5)
        wk, replay = wl.WORKLOAD_W2, oracle.replay_w2
    results = []
    for unins in (0, 1):
        with h.Context(n, G, {"exec_mode": mode, "ws_chunk_bytes": C, "cpu_threads": 1,
                              "uninstrumented": unins}) as ctx:
            ctx.load(start)
            b = submit(ctx, torch, wk, tx)
            keys, stat, out = _exec(ctx, h, torch, [b])
            assert (stat == 1).all()
            W = ctx.read_stmr(h.STMR_W)
            rs_bits, ws_bits = gpu_bitmaps(ctx, h)
            replayed = start.copy()
            ref_out, R, D = replay(replayed, tx, keys, stat, G, C)
            np.testing.assert_array_equal(out, ref_out)
            np.testing.assert_array_equal(W, replayed)
            if unins:
                assert rs_bits.size == 0 and ws_bits.size == 0
            else:
                np.testing.assert_array_equal(rs_bits, R)
                np.testing.assert_array_equal(ws_bits, D)
            results.append(R.size)
    assert results[0] > 0

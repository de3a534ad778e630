"""W2 (40 reads, Sec. V-A) and the uninstrumented executor, against the oracle
(needs a GPU).

* W2 batches under the optimistic executor (read-only transactions in the
  read-only phase, updates under the STM with reads validated against a
  clock snapshot): STMR^W after execution equals the serial replay in the
  GPU's reported commit order, every committed sum equals the replay's, and
  RS_bmp / WS_bmp equal the replay's granule and chunk sets.  A small STMR
  makes the 40-word read sets collide often, so validation failures and
  retries are exercised; then a whole round (CPU log, validation, merge)
  against the oracle's final state.
* A context in ordered mode refuses W2 batches.
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


@pytest.mark.parametrize("log2w,n_tx,upd", [(16, 30000, 0.1), (16, 30000, 0.9), (12, 6000, 0.5)])
def test_w2_matches_the_oracle(hetm, torch, log2w, n_tx, upd):
    h = hetm
    n = 1 << log2w
    start = wl.init_words(41, 0, n)
    # two uneven batches in one launch (txid bases continue across them)
    tx = wl.w2_batch(seed=41, batch=0, n_tx=n_tx, log2_words=log2w, update_frac=upd)
    cut = n_tx // 3
    with h.Context(n, G, {"exec_mode": 1, "ws_chunk_bytes": C, "cpu_threads": 1}) as ctx:
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


def test_ordered_mode_refuses_w2(hetm, torch):
    h = hetm
    tx = wl.w2_batch(seed=43, batch=0, n_tx=64, log2_words=12)
    with h.Context(1 << 12, G, {"exec_mode": 0, "cpu_threads": 1}) as ctx:
        with pytest.raises(h.HetmError) as e:
            submit(ctx, torch, wl.WORKLOAD_W2, tx)
        assert e.value.code == h.HETM_EINVAL


@pytest.mark.parametrize("mode,kind", [(1, "w1"), (1, "w2"), (0, "w1")])
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

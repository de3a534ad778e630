"""Early validation (Sec. IV-D): a watcher validates the round's CPU log while
the ordered executor runs and stops the execution phase at the first hit.

Under GPU-loses a round with any hit rolls the GPU batch back, so stopping
early must not change the round's outcome: STMR^W == STMR^S == the oracle's
final state (start overlaid with the newest CPU writes), bit-exact.  Without a
hit the watcher must change nothing at all: every output equals the run with
early validation off.
"""
import numpy as np
import pytest

import oracle
import workloads as wl
from roundkit import BatchOut, to_dev

pytestmark = pytest.mark.gpu


def _round(h, torch, start, tx, log, G, early, chunk=1024):
    n = len(start)
    cfg = {"early_validate": int(early), "cpu_threads": 1, "ws_chunk_bytes": chunk,
           "max_round_tx": max(len(tx), 1)}
    with h.Context(n, G, cfg) as ctx:
        ctx.load(start)
        dtx = to_dev(torch, tx)
        bo = BatchOut(torch, len(tx), torch.int32)
        ctx.submit_batch(h.HETM_WL_RMW, dtx, bo.order, bo.status, bo.out, n_tx=len(tx))
        dlog = to_dev(torch, log)
        ctx.log_attach(dlog, len(log))
        st = ctx.round(stats=True)
        keys, stat, out = bo.host()
        return st, keys, stat, out, ctx.read_stmr(h.STMR_W), ctx.read_stmr(h.STMR_S)


def test_no_conflict_is_unchanged(hetm):
    """CPU log on the other half of the STMR: the watcher finds nothing and the
    round is identical to one without it."""
    import torch
    h = hetm
    log2w = 18
    start = wl.init_words(21, 0, 1 << log2w)
    tx = wl.rmw_batch(seed=21, batch=0, n_tx=50000, log2_words=log2w - 1)
    log = np.concatenate(wl.cpu_write_log(21, 0, 20000, log2w - 1, cpu_threads=1,
                                          offset=1 << (log2w - 1)))
    a = _round(h, torch, start, tx, log, 64, early=True)
    b = _round(h, torch, start, tx, log, 64, early=False)
    assert a[0]["rc"] == h.HETM_OK and not a[0]["conflict"] and a[0]["stopped_early"] == 0
    assert a[0]["committed"] == len(tx)
    for x, y in zip(a[1:], b[1:]):
        np.testing.assert_array_equal(x, y)
    # and the oracle agrees
    replayed = start.copy()
    rout, R, D = oracle.replay_rmw(replayed, tx, a[1], a[2], 64, 1024)
    ref = oracle.round_from_replay(start, replayed, R, log, 64, np.zeros(len(start), np.uint32))
    np.testing.assert_array_equal(a[3], rout)
    np.testing.assert_array_equal(a[4], ref.final)
    np.testing.assert_array_equal(a[5], ref.final)


def test_conflict_stops_execution_and_round_matches_oracle(hetm):
    """A 4M-transaction Zipf batch (tens of ms of execution) and a CPU log that
    writes the batch's hottest word: the watcher stops the execution phase long
    before its end, and the round's final state is the oracle's (start + CPU
    writes, the batch rolled back)."""
    import torch
    h = hetm
    log2w = 22
    n = 1 << log2w
    start = wl.init_words(22, 0, n)
    tx = wl.rmw_batch(seed=22, batch=0, n_tx=1 << 22, log2_words=log2w)
    hot = np.bincount(tx["addr"].reshape(-1).astype(np.int64), minlength=n).argmax()
    log = np.zeros(1000, wl.LOG_DTYPE)
    log["addr"] = (np.arange(1000, dtype=np.uint32) * 7919 + 5) % n
    log["addr"][500] = hot
    log["value"] = np.arange(1000, dtype=np.int32)
    log["ts"] = np.arange(1, 1001, dtype=np.uint32)
    st, keys, stat, out, W, S = _round(h, torch, start, tx, log, 64, early=True, chunk=16384)
    assert st["rc"] == h.HETM_OK and st["conflict"] and st["n_conflicts"] >= 1
    assert st["stopped_early"] == 1
    assert set(np.unique(stat)) <= {1, 3}
    assert st["committed"] == int((stat == 1).sum()) < len(tx)
    # GPU-loses: final = start overlaid with the newest CPU value of each word,
    # whatever the stopped batch had executed
    final, ties = oracle.final_state(start, start, True, log, np.zeros(n, np.uint32))
    assert ties == 0
    np.testing.assert_array_equal(W, final)
    np.testing.assert_array_equal(S, final)

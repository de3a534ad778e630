"""Degenerate rounds on the GPU against the closed forms the paper fixes
(Sec. IV-C; needs a GPU): a round with no GPU batch leaves start + the CPU
log (newest timestamp per word) and reports no conflict; a round with an
empty CPU log leaves the GPU's serial replay; a batch of zero transactions
among others changes nothing; an empty round (no batch, no log) leaves the
state as it was.  Both executors; integers, tolerance zero.
"""
import numpy as np
import pytest

import oracle
import workloads as wl
from roundkit import submit

pytestmark = pytest.mark.gpu

LOG2W = 15
N = 1 << LOG2W
G, C = 64, 1024


@pytest.fixture(scope="module")
def torch():
    import torch as t
    if not t.cuda.is_available():
        pytest.skip("no CUDA device")
    return t


def _cpu_image(state, log):
    out = state.copy()
    order = np.argsort(log["ts"], kind="stable")
    out[log["addr"][order]] = log["value"][order]
    return out


@pytest.mark.parametrize("mode", [0, 1])
def test_degenerate_rounds(hetm, torch, mode):
    h = hetm
    start = wl.init_words(41, 0, N)
    log = np.concatenate(wl.cpu_write_log(41, 0, 2500, LOG2W, cpu_threads=1))
    tx = wl.rmw_batch(seed=41, batch=0, n_tx=6000, log2_words=LOG2W)
    with h.Context(N, G, {"exec_mode": mode, "cpu_threads": 1, "ws_chunk_bytes": C}) as ctx:
        # no batch, no log
        ctx.load(start)
        st = ctx.round(stats=True)
        assert st["rc"] == h.HETM_OK and st["n_batches"] == 0 and st["n_log"] == 0
        assert not st["conflict"] and st["committed"] == 0
        np.testing.assert_array_equal(ctx.read_stmr(h.STMR_W), start)
        # no batch, a CPU log: start + the log, no conflict
        ctx.cpu_log_write(0, log)
        st = ctx.round(stats=True)
        assert st["rc"] == h.HETM_OK and not st["conflict"] and st["n_log"] == len(log)
        expect = _cpu_image(start, log)
        np.testing.assert_array_equal(ctx.read_stmr(h.STMR_W), expect)
        np.testing.assert_array_equal(ctx.read_stmr(h.STMR_S), expect)
        # a batch of zero transactions beside a real one, and no log: the replay
        ctx.load(start)
        empty = submit(ctx, torch, wl.WORKLOAD_RMW, tx[:0])
        bo = submit(ctx, torch, wl.WORKLOAD_RMW, tx)
        st = ctx.round(stats=True)
        assert st["rc"] == h.HETM_OK and st["n_batches"] == 2 and st["n_log"] == 0
        assert not st["conflict"] and st["committed"] == len(tx)
        keys, stat, out = bo.host()
        replayed = start.copy()
        ref_out, _, _ = oracle.replay_rmw(replayed, tx, keys, stat, G, C)
        np.testing.assert_array_equal(out, ref_out)
        np.testing.assert_array_equal(ctx.read_stmr(h.STMR_W), replayed)
        np.testing.assert_array_equal(ctx.read_stmr(h.STMR_S), replayed)
        del empty

"""Two rounds in flight (needs a GPU): the second round is launched before the
first is collected, queued on the device behind it (Sec. IV-C rounds back to
back).  The result must be that of the two rounds run one after the other:
each batch replayed in its reported order from the state the previous round
left, each round's CPU log overlaid by timestamp (GPU and CPU on disjoint
halves, Sec. V-B, so both rounds validate clean), W == S, and each round's
own statistics.  A third launch, a synchronous round and a host merge are
refused while two are in flight.  Integers: tolerance zero.
"""
import numpy as np
import pytest

import oracle
import workloads as wl
from roundkit import submit

pytestmark = pytest.mark.gpu

LOG2W = 16
N = 1 << LOG2W
G, C = 64, 1024


@pytest.fixture(scope="module")
def torch():
    import torch as t
    if not t.cuda.is_available():
        pytest.skip("no CUDA device")
    return t


def _overlay(state, log):
    order = np.argsort(log["ts"], kind="stable")
    state[log["addr"][order]] = log["value"][order]


@pytest.mark.parametrize("mode,early", [(0, 0), (1, 0), (0, 1)])
def test_two_rounds_in_flight_equal_two_rounds_in_sequence(hetm, torch, mode, early):
    h = hetm
    start = wl.init_words(31, 0, N)
    txa = wl.rmw_batch(seed=31, batch=0, n_tx=20000, log2_words=LOG2W - 1)
    txb = wl.rmw_batch(seed=31, batch=1, n_tx=15000, log2_words=LOG2W - 1, update_frac=0.3)
    loga = np.concatenate(wl.cpu_write_log(31, 0, 3000, LOG2W - 1, cpu_threads=1, offset=N // 2))
    logb = np.concatenate(wl.cpu_write_log(31, 1, 2000, LOG2W - 1, cpu_threads=1, offset=N // 2))
    logb["ts"] += loga["ts"].max()
    cfg = {"exec_mode": mode, "cpu_threads": 1, "ws_chunk_bytes": C, "early_validate": early}
    with h.Context(N, G, cfg) as ctx:
        ctx.load(start)
        boa = submit(ctx, torch, wl.WORKLOAD_RMW, txa)
        ctx.cpu_log_write(0, loga)
        ctx.round(stats=False)
        bob = submit(ctx, torch, wl.WORKLOAD_RMW, txb, txid_base=len(txa))
        ctx.cpu_log_write(0, logb)
        ctx.round(stats=False)
        for refused in (lambda: ctx.round(stats=False), lambda: ctx.round(stats=True),
                        lambda: ctx.read_dirty(np.zeros(N, np.int32))):
            with pytest.raises(h.HetmError) as e:
                refused()
            assert e.value.code == h.HETM_EBUSY
        sta = ctx.round_wait()
        stb = ctx.round_wait()
        none = ctx.round_wait()
        w = ctx.read_stmr(h.STMR_W)
        np.testing.assert_array_equal(w, ctx.read_stmr(h.STMR_S))
    assert sta["rc"] == stb["rc"] == h.HETM_OK and not sta["conflict"] and not stb["conflict"]
    assert (sta["committed"], sta["n_log"], sta["n_batches"]) == (len(txa), len(loga), 1)
    assert (stb["committed"], stb["n_log"], stb["n_batches"]) == (len(txb), len(logb), 1)
    assert none["n_log"] == 0 and none["committed"] == 0
    ka, sa, outa = boa.host()
    kb, sb, outb = bob.host()
    assert (sa == 1).all() and (sb == 1).all()
    assert kb[kb % 2 == 0].min() > ka.max()  # round b's updates commit after all of round a
    expect = start.copy()
    ref_a, _, _ = oracle.replay_rmw(expect, txa, ka, sa, G, C)
    np.testing.assert_array_equal(outa, ref_a)
    _overlay(expect, loga)
    ref_b, _, _ = oracle.replay_rmw(expect, txb, kb, sb, G, C, txid_base=len(txa))
    np.testing.assert_array_equal(outb, ref_b)
    _overlay(expect, logb)
    np.testing.assert_array_equal(w, expect)

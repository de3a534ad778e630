"""Failure paths, made on the host or by a wait that runs out -- no GPU fault
(needs a GPU).

* A device wait that runs out: an execution phase with a 200 us budget on a
  batch whose longest conflict chain needs milliseconds.  Every transaction
  is reported committed or gave up, the round reports HETM_ETIMEOUT and
  HETM_OUTCOME_GPU_ROLLED_BACK, and its merge undoes the whole batch: W == S
  == the start state with the CPU log applied (Sec. IV-C conflict case).  The
  error stays until hetm_load; after it the same context runs a short batch
  to the oracle's result.
* A timeout after an address error: one transaction of the batch names a word
  out of range (the device error word records it before the executor runs),
  or an earlier round on the same context left that error standing.  The
  timeout must still be reported and the batch undone, since a partly
  executed batch must never be merged as committed (Sec. IV-C merge phase,
  Sec. IV-D rollback).
* Allocation failure in hetm_init (the device allocator hook refuses the k-th
  request): HETM_ENOMEM, and every buffer it got is given back.
"""
import ctypes

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


def _cpu_image(start, log):
    img = start.copy()
    order = np.argsort(log["ts"], kind="stable")
    img[log["addr"][order]] = log["value"][order]
    return img


@pytest.mark.parametrize("mode", [0, 1])
def test_execution_budget_runs_out_and_the_batch_is_undone(hetm, torch, mode):
    h = hetm
    start = wl.init_words(23, 0, N)
    # Zipf(0.99) updates on the GPU's half: a chain of thousands of conflicting
    # transactions on the hottest word
    tx = wl.rmw_batch(seed=23, batch=0, n_tx=200000, log2_words=LOG2W - 1, update_frac=1.0)
    log = np.concatenate(wl.cpu_write_log(23, 0, 2000, LOG2W - 1, cpu_threads=1, offset=N // 2))
    cfg = {"exec_mode": mode, "exec_budget_us": 200, "cpu_threads": 1, "ws_chunk_bytes": C,
           "max_round_tx": 1 << 18}
    with h.Context(N, G, cfg) as ctx:
        ctx.load(start)
        bo = submit(ctx, torch, wl.WORKLOAD_RMW, tx)
        ctx.cpu_log_write(0, log)
        st = ctx.round(stats=True)
        assert st["rc"] == h.HETM_ETIMEOUT
        assert st["outcome"] == h.HETM_OUTCOME_GPU_ROLLED_BACK
        _, stat, _ = bo.host()
        assert np.isin(stat, [1, 2]).all()
        assert (stat == 2).sum() == st["gave_up"] > 0
        expect = _cpu_image(start, log)
        np.testing.assert_array_equal(ctx.read_stmr(h.STMR_W), expect)
        np.testing.assert_array_equal(ctx.read_stmr(h.STMR_S), expect)
        assert ctx.exec_counters()["rc"] == h.HETM_ETIMEOUT  # until hetm_load

        ctx.load(start)
        assert ctx.exec_counters()["rc"] == h.HETM_OK
        small = wl.rmw_batch(seed=24, batch=0, n_tx=512, log2_words=LOG2W, uniform=True)
        bo = submit(ctx, torch, wl.WORKLOAD_RMW, small)
        st = ctx.round(stats=True)
        assert st["rc"] == h.HETM_OK and st["outcome"] == h.HETM_OUTCOME_CLEAN
        keys, stat, out = bo.host()
        assert (stat == 1).all()
        replayed = start.copy()
        ref_out, _, _ = oracle.replay_rmw(replayed, small, keys, stat, G, C)
        np.testing.assert_array_equal(out, ref_out)
        np.testing.assert_array_equal(ctx.read_stmr(h.STMR_W), replayed)


def _chain_round(h, ctx, torch, start, bad_tx, seed=23):
    """One round whose execution phase runs out of its 200 us budget; bad_tx
    puts one out-of-range word into the batch."""
    tx = wl.rmw_batch(seed=seed, batch=0, n_tx=200000, log2_words=LOG2W - 1, update_frac=1.0)
    if bad_tx:
        tx["addr"][777, 2] = N + 5
    log = np.concatenate(wl.cpu_write_log(seed, 0, 2000, LOG2W - 1, cpu_threads=1, offset=N // 2))
    bo = submit(ctx, torch, wl.WORKLOAD_RMW, tx)
    ctx.cpu_log_write(0, log)
    st = ctx.round(stats=True)
    return st, bo, log


@pytest.mark.parametrize("mode", [0, 1])
@pytest.mark.parametrize("where", ["same_batch", "earlier_round"])
def test_timeout_after_an_address_error_still_undoes_the_batch(hetm, torch, mode, where):
    h = hetm
    start = wl.init_words(29, 0, N)
    cfg = {"exec_mode": mode, "exec_budget_us": 200, "cpu_threads": 1, "ws_chunk_bytes": C,
           "max_round_tx": 1 << 18}
    with h.Context(N, G, cfg) as ctx:
        ctx.load(start)
        ts_state = np.zeros(N, np.uint32)
        if where == "earlier_round":
            # a short clean round whose only fault is one out-of-range word
            small = wl.rmw_batch(seed=30, batch=0, n_tx=256, log2_words=LOG2W, uniform=True)
            small["addr"][5, 0] = N + 1
            bo = submit(ctx, torch, wl.WORKLOAD_RMW, small)
            st = ctx.round(stats=True)
            assert st["rc"] == h.HETM_EDEVICE
            assert st["outcome"] == h.HETM_OUTCOME_CLEAN
            keys, stat, _ = bo.host()
            assert stat[5] == 2 and (np.delete(stat, 5) == 1).all()
            replayed = start.copy()
            oracle.replay_rmw(replayed, small, keys, stat, G, C)
            np.testing.assert_array_equal(ctx.read_stmr(h.STMR_W), replayed)
            start = replayed
        st, bo, log = _chain_round(h, ctx, torch, start, bad_tx=where == "same_batch")
        assert st["rc"] == h.HETM_ETIMEOUT
        assert st["outcome"] == h.HETM_OUTCOME_GPU_ROLLED_BACK
        _, stat, _ = bo.host()
        assert np.isin(stat, [1, 2]).all() and st["gave_up"] > 0
        # the rolled-back round's final state is the oracle's conflict case
        expect, ties = oracle.final_state(start, start, True, log, ts_state.copy())
        assert ties == 0
        np.testing.assert_array_equal(ctx.read_stmr(h.STMR_W), expect)
        np.testing.assert_array_equal(ctx.read_stmr(h.STMR_S), expect)
        assert ctx.exec_counters()["rc"] == h.HETM_ETIMEOUT


@pytest.mark.parametrize("fail_at", [0, 3, 9])
def test_init_gives_back_every_buffer_when_an_allocation_fails(hetm, torch, fail_at):
    h = hetm
    dev = torch.cuda.current_device()
    live, calls = {}, [0]

    def alloc(nbytes, user):
        calls[0] += 1
        if calls[0] - 1 == fail_at:
            return None
        p = torch.cuda.caching_allocator_alloc(int(nbytes), dev)
        live[p] = nbytes
        return p

    def free(p, user):
        del live[p]
        torch.cuda.caching_allocator_delete(p)

    cb = (h._ALLOC(alloc), h._FREE(free))
    cfg = h.hetm_config_default()
    cfg.dev_alloc, cfg.dev_free = cb
    cfg.max_round_tx = 1 << 16
    out = ctypes.c_void_p()
    rc = h.lib().hetm_init(ctypes.byref(out), N, G, ctypes.byref(cfg), None)
    assert rc == h.HETM_ENOMEM
    assert calls[0] == fail_at + 1
    assert live == {}

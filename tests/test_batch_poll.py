"""hetm_batch_poll (needs a GPU): a batch is queued until an execution phase
launches it, running until the round that ran it has merged, then done with
that round's outcome (Sec. IV-C: a GPU batch's commits are final only once its
synchronization round validated and merged).  The per-transaction results of a
done batch equal the serial replay, as in the parity tests."""
import numpy as np
import pytest

import workloads as wl
from roundkit import submit

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def torch():
    import torch as t
    if not t.cuda.is_available():
        pytest.skip("no CUDA device")
    return t


def _bank(seed, n, lo, hi):
    return wl.bank_transfers(seed, (wl.S.SRC, wl.S.DST, wl.S.AMT), n, lo, hi)


def test_batch_states_through_a_round(hetm, torch):
    h = hetm
    n_words = 1 << 16
    with h.Context(n_words, 64, {"cpu_threads": 1}) as ctx:
        ctx.load(np.full(n_words, 1000, np.int32))
        b1 = submit(ctx, torch, wl.WORKLOAD_BANK, _bank(1, 3000, 0, n_words))
        b2 = submit(ctx, torch, wl.WORKLOAD_BANK, _bank(2, 500, 0, n_words))
        ids = [1, 2]  # the context's first ids
        for i in ids:
            r = ctx.batch_poll(i)
            assert r["state"] == h.HETM_BATCH_QUEUED and r["round"] == 0
        assert ctx.batch_poll(1)["n_tx"] == 3000 and ctx.batch_poll(2)["n_tx"] == 500
        ctx.round(stats=False)
        r = ctx.batch_poll(1)
        assert r["state"] in (h.HETM_BATCH_RUNNING, h.HETM_BATCH_DONE) and r["round"] == 1
        ctx.round_wait()
        for i, bo in zip(ids, (b1, b2)):
            r = ctx.batch_poll(i)
            assert r["state"] == h.HETM_BATCH_DONE
            assert r["outcome"] == h.HETM_OUTCOME_CLEAN and r["round"] == 1
            assert r["latency_ms"] > 0
            torch.cuda.synchronize()
            assert (bo.status.cpu().numpy() == 1).all()
        # a done batch stays done, with the latency first seen
        first = ctx.batch_poll(2)["latency_ms"]
        assert ctx.batch_poll(2)["latency_ms"] == first
        with pytest.raises(h.HetmError) as e:
            ctx.batch_poll(99)
        assert e.value.code == h.HETM_EINVAL


def test_batch_states_through_exec_validate_merge(hetm, torch):
    """The round written out by hand: running after hetm_gpu_exec however long the
    executor has been done, done once hetm_merge has run; a conflicting CPU log
    gives the GPU-rolled-back outcome."""
    h = hetm
    n_words = 1 << 16
    with h.Context(n_words, 64, {"cpu_threads": 1}) as ctx:
        ctx.load(np.full(n_words, 1000, np.int32))
        tx = _bank(3, 2000, 0, n_words)
        submit(ctx, torch, wl.WORKLOAD_BANK, tx)
        bid = 1
        ctx.gpu_exec()
        ctx.sync()
        torch.cuda.synchronize()
        assert ctx.batch_poll(bid)["state"] == h.HETM_BATCH_RUNNING
        log = np.zeros(1, dtype=wl.LOG_DTYPE)
        log["addr"] = tx["src"][0]  # a word the batch read and wrote
        log["value"] = 7
        log["ts"] = 1
        ctx.cpu_log_write(0, log)
        assert ctx.validate() == 1
        assert ctx.batch_poll(bid)["state"] == h.HETM_BATCH_RUNNING
        ctx.merge(-1)
        ctx.sync()
        r = ctx.batch_poll(bid)
        assert r["state"] == h.HETM_BATCH_DONE
        assert r["outcome"] == h.HETM_OUTCOME_GPU_ROLLED_BACK and r["round"] == 1
        # the next round gets the next number
        submit(ctx, torch, wl.WORKLOAD_BANK, _bank(4, 100, 0, n_words))
        ctx.round(stats=True)
        assert ctx.batch_poll(2)["round"] == 2 and ctx.batch_poll(2)["state"] == h.HETM_BATCH_DONE


def test_load_forgets_queued_batches(hetm, torch):
    h = hetm
    n_words = 1 << 12
    with h.Context(n_words, 64, {"cpu_threads": 1}) as ctx:
        ctx.load(np.full(n_words, 1000, np.int32))
        submit(ctx, torch, wl.WORKLOAD_BANK, _bank(5, 10, 0, n_words))
        assert ctx.batch_poll(1)["state"] == h.HETM_BATCH_QUEUED
        ctx.load(np.full(n_words, 1000, np.int32))
        with pytest.raises(h.HetmError):
            ctx.batch_poll(1)

"""Double-buffered host side of the merge (Sec. IV-D: STMR^S lets the copy of
the GPU-dirty chunks to the host overlap the next execution phase; needs a GPU).

Round k's surviving dirty chunks are queued for the host replica
(``read_dirty_async``) and round k+1 is launched at once on the same chunks.
The copies must hold round k's STMR^S, not round k+1's: the host replica
after ``read_dirty_wait`` equals STMR^S as it was after round k, word for
word (no CPU log: the non-dirty chunks still hold the start values).  A round
the GPU lost copies nothing, and a pageable replica gives the same words.
"""
import numpy as np
import pytest

import workloads as wl
from roundkit import BatchOut, to_dev

pytestmark = pytest.mark.gpu

LOG2W = 18
N = 1 << LOG2W
CHUNK = 256


def _bank(seed, n=20000):
    return wl.bank_transfers(seed, (wl.S.SRC, wl.S.DST, wl.S.AMT), n, 0, N // 4)


def _submit(h, torch, ctx, tx, keep):
    dtx = to_dev(torch, tx)
    bo = BatchOut(torch, len(tx), torch.int32)
    ctx.submit_batch(h.HETM_WL_BANK, dtx, bo.order, bo.status, bo.out, n_tx=len(tx))
    keep.append((dtx, bo))


@pytest.mark.parametrize("pinned", [True, False])
def test_async_copies_hold_the_previous_round(hetm, pinned):
    import torch
    h = hetm
    start = np.full(N, 1000, np.int32)
    keep = []
    with h.Context(N, 64, {"ws_chunk_bytes": CHUNK, "cpu_threads": 1}) as ctx:
        ctx.load(start)
        if pinned:
            host = torch.from_numpy(start.copy()).pin_memory()
            view = host.numpy()
        else:
            host = start.copy()
            view = host
        prev = start
        for k in range(3):
            _submit(h, torch, ctx, _bank(60 + k), keep)
            st = ctx.round(stats=True)
            assert st["rc"] == h.HETM_OK and st["outcome"] == h.HETM_OUTCOME_CLEAN
            s_k = ctx.read_stmr(h.STMR_S)
            chunks, nbytes = ctx.read_dirty_async(host)
            assert chunks == st["dirty_chunks"] and nbytes == chunks * CHUNK
            # the next round writes the same chunks while the copies may still run
            _submit(h, torch, ctx, _bank(70 + k), keep)
            st2 = ctx.round(stats=True)
            assert st2["rc"] == h.HETM_OK
            ctx.read_dirty_wait()
            np.testing.assert_array_equal(view, s_k)
            assert not np.array_equal(s_k, prev)
            # bring the replica up to date with the round just run
            ctx.read_dirty_async(host)
            ctx.read_dirty_wait()
            prev = ctx.read_stmr(h.STMR_S)
            np.testing.assert_array_equal(view, prev)


def test_lost_round_copies_nothing(hetm):
    import torch
    h = hetm
    start = np.full(N, 1000, np.int32)
    keep = []
    with h.Context(N, 64, {"ws_chunk_bytes": CHUNK, "cpu_threads": 1}) as ctx:
        ctx.load(start)
        tx = _bank(80)
        _submit(h, torch, ctx, tx, keep)
        log = np.zeros(1, h.LOG_DTYPE)
        log["addr"], log["value"], log["ts"] = tx["src"][0], -5, 1   # a word the batch reads
        ctx.cpu_log_write(0, log)
        st = ctx.round(stats=True)
        assert st["outcome"] == h.HETM_OUTCOME_GPU_ROLLED_BACK
        host = torch.from_numpy(start.copy()).pin_memory()
        assert ctx.read_dirty_async(host) == (0, 0)
        ctx.read_dirty_wait()
        np.testing.assert_array_equal(host.numpy(), start)

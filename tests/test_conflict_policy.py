"""Conflict-resolution policies (Sec. IV-E) and the host side of the merge.

* CPU-loses: the CPU log is applied only after a clean validation; on a
  conflict the GPU state stands.  STMR^W == STMR^S == the oracle's
  ``final_state_cpu_loses``, bit-exact.
* Host re-alignment: a host replica that ran the CPU's transactions
  speculatively (start + its log) is brought to the round's outcome by undoing
  its log from its shadow when the CPU lost, then copying the surviving
  GPU-dirty chunks (``hetm_read_dirty``); it must equal STMR^W, for both
  policies and both outcomes.
* Anti-starvation: after ``starve_limit`` consecutive GPU losses the next
  execution phase admits no CPU writes, so that round validates clean.
"""
import numpy as np
import pytest

import oracle
import workloads as wl
from roundkit import BatchOut, to_dev

pytestmark = pytest.mark.gpu

LOG2W = 16
N = 1 << LOG2W
G = 64
CHUNK = 1024


def _inputs(seed, conflicting):
    start = wl.init_words(seed, 0, N)
    tx = wl.rmw_batch(seed=seed, batch=0, n_tx=8000, log2_words=LOG2W - 1)
    if conflicting:  # Zipf words of the GPU's half: hits its read set
        log = np.concatenate(wl.cpu_write_log(seed, 0, 3000, LOG2W - 1, cpu_threads=1))
    else:            # the other half of the STMR (Sec. V-B's partition)
        log = np.concatenate(wl.cpu_write_log(seed, 0, 3000, LOG2W - 1, cpu_threads=1,
                                              offset=N // 2))
    return start, tx, log


def _host_speculative(start, log):
    """The CPU's replica after its speculative commits: newest ts per word."""
    h = start.copy()
    order = np.argsort(log["ts"], kind="stable")
    h[log["addr"][order]] = log["value"][order]
    return h


@pytest.mark.parametrize("policy", [0, 1])
@pytest.mark.parametrize("conflicting", [False, True])
def test_policy_round_and_host_realignment(hetm, policy, conflicting):
    import torch
    h = hetm
    start, tx, log = _inputs(31 + policy, conflicting)
    cfg = {"conflict_policy": policy, "ws_chunk_bytes": CHUNK, "cpu_threads": 1}
    with h.Context(N, G, cfg) as ctx:
        ctx.load(start)
        dtx = to_dev(torch, tx)
        bo = BatchOut(torch, len(tx), torch.int32)
        ctx.submit_batch(h.HETM_WL_RMW, dtx, bo.order, bo.status, bo.out, n_tx=len(tx))
        ctx.cpu_log_write(0, log)
        st = ctx.round(stats=True)
        assert st["rc"] == h.HETM_OK and bool(st["conflict"]) == conflicting
        want = (h.HETM_OUTCOME_CLEAN if not conflicting else
                h.HETM_OUTCOME_CPU_DISCARDED if policy == 1 else h.HETM_OUTCOME_GPU_ROLLED_BACK)
        assert st["outcome"] == want
        keys, stat, out = bo.host()
        W, S = ctx.read_stmr(h.STMR_W), ctx.read_stmr(h.STMR_S)
        # oracle
        replayed = start.copy()
        rout, R, D = oracle.replay_rmw(replayed, tx, keys, stat, G, CHUNK)
        np.testing.assert_array_equal(out, rout)
        ref = oracle.round_from_replay(start, replayed, R, log, G, np.zeros(N, np.uint32),
                                       cpu_loses=policy == 1)
        assert ref.conflict == conflicting and ref.n_conflicts == st["n_conflicts"]
        np.testing.assert_array_equal(W, ref.final)
        np.testing.assert_array_equal(S, ref.final)
        # host side: speculative replica -> undo if the CPU lost -> GPU chunks
        host = _host_speculative(start, log)
        if st["outcome"] == h.HETM_OUTCOME_CPU_DISCARDED:
            host[log["addr"]] = start[log["addr"]]  # from the CPU's shadow
        n_chunks, n_bytes = ctx.read_dirty(host)
        if st["outcome"] == h.HETM_OUTCOME_GPU_ROLLED_BACK:
            assert n_chunks == 0
        else:
            assert n_chunks == len(np.unique(D)) and n_bytes <= n_chunks * CHUNK
        np.testing.assert_array_equal(host, W)


def test_anti_starvation_read_only_cpu_round(hetm):
    """GPU-loses with starve_limit = 2: two lost rounds in a row make the next
    execution phase read-only on the CPU (writes refused), which then validates
    clean and lets the GPU's batch stand; afterwards CPU writes are allowed again."""
    import torch
    h = hetm
    start, tx, log = _inputs(41, True)
    with h.Context(N, G, {"starve_limit": 2, "ws_chunk_bytes": CHUNK, "cpu_threads": 1}) as ctx:
        ctx.load(start)
        dtx = to_dev(torch, tx)
        bo = BatchOut(torch, len(tx), torch.int32)
        outcomes = []
        for r in range(4):
            ctx.submit_batch(h.HETM_WL_RMW, dtx, bo.order, bo.status, bo.out, n_tx=len(tx),
                             txid_base=r * len(tx))
            lg = log.copy()
            lg["ts"] = lg["ts"] + r * len(log)
            if ctx.cpu_updates_allowed():
                ctx.cpu_log_write(0, lg)
            else:
                with pytest.raises(h.HetmError) as e:
                    ctx.cpu_log_write(0, lg)
                assert e.value.code == h.HETM_EBUSY
            st = ctx.round(stats=True)
            assert st["rc"] == h.HETM_OK
            outcomes.append((st["outcome"], st["cpu_read_only_next"]))
        assert outcomes == [(h.HETM_OUTCOME_GPU_ROLLED_BACK, 0), (h.HETM_OUTCOME_GPU_ROLLED_BACK, 1),
                            (h.HETM_OUTCOME_CLEAN, 0), (h.HETM_OUTCOME_GPU_ROLLED_BACK, 0)]
        assert ctx.cpu_updates_allowed()

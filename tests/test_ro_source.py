"""Where the ordered executor's read-only phase reads the launch-start state
(Sec. IV-C execution phase; needs a GPU).

A launch serializes its W1 read-only transactions before every update, on
the state the launch starts from, which is STMR^W.  After a load or a merge
STMR^S equals it, but not in these cases, where the read-only phase must see
what STMR^W holds:

* a second execution launch of the same round (step API: two gpu_exec calls
  before the merge): its read-only transactions see the first launch's
  writes;
* planted GPU writes (the testing library's gpu_mark with values) before a
  round: its read-only transactions see the planted words;
* the uninstrumented executor (no WS_bmp, so the merge cannot bring S level).

Each is checked bit-exact against the oracle's serial replay, with the
read-only batch's outputs (the sum of its 4 words) compared one by one.
"""
import numpy as np
import pytest

import oracle
import workloads as wl
import paper_1905_00661_b300.testing as hetm_testing
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


def _reads(seed, n):
    """Read-only W1 transactions over the whole STMR (uniform words)."""
    return wl.rmw_batch(seed=seed, batch=1, n_tx=n, log2_words=LOG2W, uniform=True, update_frac=0.0)


def _expected_sums(state, tx):
    return state[tx["addr"].astype(np.int64)].sum(axis=1, dtype=np.int64).astype(np.int32)


def test_second_launch_of_a_round_reads_the_first_launchs_writes(hetm, torch):
    h = hetm
    start = wl.init_words(71, 0, N)
    upd = wl.rmw_batch(seed=71, batch=0, n_tx=30000, log2_words=LOG2W, update_frac=1.0)
    ro = _reads(72, 20000)
    with h.Context(N, G, {"cpu_threads": 1, "ws_chunk_bytes": C}) as ctx:
        ctx.load(start)
        bu = submit(ctx, torch, wl.WORKLOAD_RMW, upd)
        ctx.gpu_exec()
        br = submit(ctx, torch, wl.WORKLOAD_RMW, ro, txid_base=len(upd))
        ctx.gpu_exec()
        ctx.sync()
        torch.cuda.synchronize()
        keys, stat, _ = bu.host()
        assert (stat == 1).all()
        after = start.copy()
        oracle.replay_rmw(after, upd, keys, stat, G, C)
        np.testing.assert_array_equal(ctx.read_stmr(h.STMR_W), after)
        _, rstat, rout = br.host()
        assert (rstat == 1).all()
        np.testing.assert_array_equal(rout, _expected_sums(after, ro))
        # the round closes as usual; the next round starts from the merged state
        assert ctx.validate() == 0
        ctx.merge(-1)
        ro2 = _reads(73, 20000)
        b2 = submit(ctx, torch, wl.WORKLOAD_RMW, ro2)
        st = ctx.round(stats=True)
        assert st["rc"] == h.HETM_OK
        _, s2, o2 = b2.host()
        assert (s2 == 1).all()
        np.testing.assert_array_equal(o2, _expected_sums(after, ro2))
        np.testing.assert_array_equal(ctx.read_stmr(h.STMR_S), after)


def test_read_only_phase_sees_planted_writes(hetm, torch):
    h = hetm
    start = wl.init_words(74, 0, N)
    rng = np.random.default_rng(74)
    addr = np.unique(rng.integers(0, N, 5000, dtype=np.uint32))
    vals = rng.integers(-1000, 1000, addr.size, dtype=np.int32)
    ro = _reads(75, 20000)
    with h.Context(N, G, {"cpu_threads": 1, "ws_chunk_bytes": C}) as ctx:
        ctx.load(start)
        hetm_testing.gpu_mark(ctx, torch.from_numpy(addr).cuda(), torch.from_numpy(vals).cuda())
        b = submit(ctx, torch, wl.WORKLOAD_RMW, ro)
        st = ctx.round(stats=True)
        assert st["rc"] == h.HETM_OK
        planted = start.copy()
        oracle.plant(planted, addr, vals)
        _, s, o = b.host()
        assert (s == 1).all()
        np.testing.assert_array_equal(o, _expected_sums(planted, ro))
        np.testing.assert_array_equal(ctx.read_stmr(h.STMR_W), planted)
        np.testing.assert_array_equal(ctx.read_stmr(h.STMR_S), planted)


def test_uninstrumented_rounds_read_stmr_w(hetm, torch):
    h = hetm
    start = wl.init_words(76, 0, N)
    upd = wl.rmw_batch(seed=76, batch=0, n_tx=30000, log2_words=LOG2W, update_frac=1.0)
    ro = _reads(77, 20000)
    with h.Context(N, G, {"cpu_threads": 1, "ws_chunk_bytes": C, "uninstrumented": 1}) as ctx:
        ctx.load(start)
        bu = submit(ctx, torch, wl.WORKLOAD_RMW, upd)
        assert ctx.round(stats=True)["rc"] == h.HETM_OK
        keys, stat, _ = bu.host()
        after = start.copy()
        oracle.replay_rmw(after, upd, keys, stat, G, C)
        np.testing.assert_array_equal(ctx.read_stmr(h.STMR_W), after)
        b = submit(ctx, torch, wl.WORKLOAD_RMW, ro, txid_base=len(upd))
        assert ctx.round(stats=True)["rc"] == h.HETM_OK
        _, s, o = b.host()
        assert (s == 1).all()
        np.testing.assert_array_equal(o, _expected_sums(after, ro))

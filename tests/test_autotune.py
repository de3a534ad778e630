"""Autotuner (executor shape, conflict granule, merge chunk) on a sample round.

The tuner runs whole rounds per candidate; these tests check that it picks
the best-scoring candidate of each stage, that a granule coarse enough to
create false conflicts loses (Sec. V-A's granule trade-off), and that a round
run with the tuned configuration still matches the oracle bit-exact.
"""
import numpy as np
import pytest

import oracle
import workloads as wl

pytestmark = pytest.mark.gpu

LOG2W = 16
N = 1 << LOG2W


def _sample():
    """GPU transactions touch only the first 64 B of every 1 KB block; the CPU
    log writes only the upper half of blocks.  4 B and 64 B granules see no
    conflict, 1 KB granules a false one."""
    tx = wl.rmw_batch(seed=11, batch=0, n_tx=6000, log2_words=LOG2W - 4, uniform=True)
    a = tx["addr"].astype(np.uint64)
    tx["addr"] = ((a >> np.uint64(4)) * np.uint64(256) + (a & np.uint64(15))).astype(np.uint32)
    logs = wl.cpu_write_log(11, 0, 3000, LOG2W - 4, uniform=True, cpu_threads=1)
    lg = logs[0]
    b = lg["addr"].astype(np.uint64)
    lg["addr"] = ((b >> np.uint64(4)) * np.uint64(256) + np.uint64(128) + (b & np.uint64(15))).astype(np.uint32)
    return wl.init_words(5, 0, N), tx, lg


def test_autotune_picks_best_and_avoids_false_conflicts(hetm):
    import torch
    from roundkit import BatchOut, to_dev
    h = hetm
    init, tx, lg = _sample()
    dtx = to_dev(torch, tx)
    bo = BatchOut(torch, len(tx), torch.int32)
    dlog = to_dev(torch, lg)
    space = {"threads": [128, 256], "blocks_per_sm": [0, 1], "granules": [1024, 64, 4],
             "ws_chunk_bytes": [256, 4096], "reps": 2}
    res = h.autotune(N, init, [(h.HETM_WL_RMW, dtx, bo.order, bo.status, bo.out)], log=dlog,
                     n_log=len(lg), base={"max_round_tx": 1 << 14}, space=space)
    tr = res["trials"]
    assert all(t["rc"] == h.HETM_OK for t in tr)
    st0 = [t for t in tr if t["stage"] == 0]
    st1 = [t for t in tr if t["stage"] == 1]
    st2 = [t for t in tr if t["stage"] == 2]
    # ordered: 2 sizes x 2 grids; optimistic: 2 sizes x 2 grids x 1 lock table
    assert len(st0) == 8 and len(st1) == 3 and len(st2) == 2
    assert all(t["committed"] == len(tx) for t in st0 if t["rounds"])
    b0 = max(st0, key=lambda t: t["score"])
    cfg = res["config"]
    assert (cfg["exec_mode"], cfg["exec_threads"], cfg["exec_blocks"]) == (
        b0["exec_mode"], b0["exec_threads"], b0["exec_blocks"])
    by_g = {t["granule_bytes"]: t for t in st1}
    assert by_g[1024]["conflicts"] == by_g[1024]["rounds"] > 0
    assert by_g[64]["conflicts"] == 0 and by_g[4]["conflicts"] == 0
    assert res["granule_bytes"] == max(st1, key=lambda t: t["score"])["granule_bytes"]
    assert res["granule_bytes"] in (4, 64)
    assert cfg["ws_chunk_bytes"] == max(st2, key=lambda t: t["score"])["ws_chunk_bytes"]

    # a round with the tuned configuration matches the oracle
    G = res["granule_bytes"]
    with h.Context(N, G, dict(cfg, max_round_tx=1 << 14, cpu_threads=1)) as ctx:
        ctx.load(init)
        ctx.submit_batch(h.HETM_WL_RMW, dtx, bo.order, bo.status, bo.out, n_tx=len(tx))
        ctx.cpu_log_write(0, lg)
        st = ctx.round(stats=True)
        assert st["rc"] == h.HETM_OK and not st["conflict"]
        keys, stat, out = bo.host()
        replayed = init.copy()
        rout, R, D = oracle.replay_rmw(replayed, tx, keys, stat, G, cfg["ws_chunk_bytes"])
        np.testing.assert_array_equal(out, rout)
        ref = oracle.round_from_replay(init, replayed, R, lg, G, np.zeros(N, np.uint32))
        assert ref.n_conflicts == 0
        np.testing.assert_array_equal(ctx.read_stmr(h.STMR_W), ref.final)
        np.testing.assert_array_equal(ctx.read_stmr(h.STMR_S), ref.final)


def test_handoff_latency_probe(hetm):
    """Hand-on of a word: through shared memory (two warps of a CTA) well under
    a microsecond, and no slower than across two SMs through L2."""
    import paper_1905_00661_b300.testing as t
    g, sh = t.handoff_latency(5000)
    assert 5.0 < sh < 2000.0
    assert 20.0 < g < 20000.0
    assert sh < g


def test_random_access_probe(hetm):
    """Random 4-byte reads and writes over 1 GiB: between 1e9 and 1e12 per second."""
    import paper_1905_00661_b300.testing as t
    r, w = t.random_access_rate(28, 1 << 26)
    assert 1e9 < r < 1e12 and 1e9 < w < 1e12


def test_l2_probe(hetm):
    """Random 4-byte probes of a 2 MiB (L2-resident) array in the validation
    kernel's launch shape: faster than random DRAM sectors, below 1e13/s."""
    import paper_1905_00661_b300.testing as t
    p = t.l2_probe_rate(19, 1 << 24)
    r, _ = t.random_access_rate(28, 1 << 26)
    assert r < p < 1e13

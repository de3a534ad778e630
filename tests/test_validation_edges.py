"""Validation kernels at their edges (needs a GPU): a read set dense enough that
the shared-memory filter of RS_bmp is bypassed, log sizes around the kernel's
work split, and tuples whose address is outside the STMR (Sec. IV-C validation).
Flags and counts are compared bit-exact with the oracle's brute-force set
intersection; integer work, tolerance zero.
"""
import numpy as np
import pytest

import oracle
import workloads as wl
import paper_1905_00661_b300.testing as hetm_testing
from roundkit import flags_of, to_dev

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def torch():
    import torch as t
    if not t.cuda.is_available():
        pytest.skip("no CUDA device")
    return t


def _validate_only(h, torch, ctx, log):
    n = len(log)
    dlog = to_dev(torch, log)
    flags = torch.full((max((n + 31) // 32, 1),), -1, dtype=torch.int32, device="cuda")
    cnt = torch.zeros(1, dtype=torch.int64, device="cuda")
    ctx.validate_only(dlog, n, flags, cnt)
    torch.cuda.synchronize()
    return flags_of(flags.cpu().numpy().view(np.uint32), n), int(cnt.item())


def _mark_read(ctx, torch, v):
    first = (v.read_granules.astype(np.uint64) * (v.granule_bytes // 4)).astype(np.uint32)
    hetm_testing.gpu_mark(ctx, torch.from_numpy(first).cuda())


def test_dense_read_set_bypasses_filter(hetm, torch):
    """Half of 2^22 one-word granules read: the 1M-bit filter would be ~86% set,
    above the 3/4 at which each CTA stops using it and probes RS_bmp directly."""
    h = hetm
    v = wl.validation_round(seed=7, log2_words=22, granule_bytes=4, read_frac=0.5, n_log=200003,
                            with_init=False)
    assert len(v.read_granules) == 1 << 21
    with h.Context(1 << 22, 4) as ctx:
        _mark_read(ctx, torch, v)
        got, n = _validate_only(h, torch, ctx, v.log)
    ref_flags, ref_n = oracle.conflicts(v.log, v.read_granules, v.granule_bytes)
    assert n == ref_n == v.n_hits_planted
    np.testing.assert_array_equal(got, ref_flags)


@pytest.mark.parametrize("n_log", [1, 33, 127, 129, 148 * 32 * 128 + 7])
def test_validate_only_ragged_sizes(hetm, torch, n_log):
    """Sizes around the work split: groups of 32 tuples, 4 groups in flight per
    warp, one 1024-thread CTA per SM (148 x 32 warps)."""
    h = hetm
    v = wl.validation_round(seed=9, log2_words=20, n_log=n_log, with_init=False)
    with h.Context(1 << 20, v.granule_bytes) as ctx:
        _mark_read(ctx, torch, v)
        got, n = _validate_only(h, torch, ctx, v.log)
    ref_flags, ref_n = oracle.conflicts(v.log, v.read_granules, v.granule_bytes)
    assert n == ref_n
    np.testing.assert_array_equal(got, ref_flags)


def test_out_of_range_tuples_are_skipped_and_reported(hetm, torch):
    """A tuple whose address is >= stmr_words is skipped (flag 0) and reported as
    HETM_EDEVICE; every other tuple's flag is still exact, and the error stays
    reported until hetm_load resets the context."""
    h = hetm
    log2w = 18
    v = wl.validation_round(seed=8, log2_words=log2w, n_log=4099, with_init=False)
    log = v.log.copy()
    bad = np.array([0, 37, 2048, 4098])
    log["addr"][bad] = (1 << log2w) + np.arange(bad.size, dtype=np.uint32) * 977
    good = np.ones(len(log), bool)
    good[bad] = False
    with h.Context(1 << log2w, v.granule_bytes) as ctx:
        _mark_read(ctx, torch, v)
        got, n = _validate_only(h, torch, ctx, log)
        ref_flags, ref_n = oracle.conflicts(log[good], v.read_granules, v.granule_bytes)
        assert n == ref_n
        np.testing.assert_array_equal(got[good], ref_flags)
        assert not got[bad].any()
        assert ctx.exec_counters()["rc"] == h.HETM_EDEVICE
        # the round path reports it too, through hetm_validate
        ctx.cpu_log_write(0, log)
        with pytest.raises(h.HetmError) as e:
            ctx.validate()
        assert e.value.code == h.HETM_EDEVICE
        # hetm_load clears the error
        ctx.load(np.zeros(1 << log2w, np.int32))
        assert ctx.exec_counters()["rc"] == h.HETM_OK

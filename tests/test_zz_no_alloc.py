"""hetm_validate_noalloc against hetm_validate_only and the oracle.

The allocation-free entry point serves callers that cannot allocate device
memory when they validate -- work being captured into a CUDA graph, serving
loops that must not pay cudaMalloc's device-wide synchronization, plug-ins
whose host framework owns all device memory.  It keeps its scratch in one
static device array shared by every call, so the check runs two calls in a
row (a large log, then a shorter one that must not see the first call's
leftovers) and compares flags, hit count and status with the context-based
entry point on the same inputs, and the flags and count with the oracle's
brute-force set intersection.  Further cases: out-of-range tuples (reported
as HETM_EDEVICE and left out of the count), no flag output, an empty log,
and logs shorter than one 128-tuple tile.  Integer results: they must match
exactly.
"""
import ctypes

import numpy as np
import pytest

import oracle
import workloads as wl
import paper_1905_00661_b300.testing as hetm_testing
from roundkit import flags_of, to_dev


def test_noalloc_rejects_oversized_input_without_device_work():
    import paper_1905_00661_b300 as h
    rc = h.lib().hetm_validate_noalloc(None, h.HETM_NOALLOC_MAX_TUPLES + 1, None, 64, 1 << 20,
                                       None, None, None, None)
    assert rc == h.HETM_ECAPACITY
    assert h.lib().hetm_validate_noalloc(None, 0, None, 48, 1 << 20, None, None, None,
                                         None) == h.HETM_EINVAL


@pytest.mark.gpu
def test_noalloc_matches_validate_only_on_two_calls(hetm):
    import torch
    h = hetm
    v = wl.validation_round(seed=12, log2_words=20, n_log=300001)  # 37 blocks, ragged end
    n_words = 1 << 20
    with h.Context(n_words, v.granule_bytes) as ctx:
        first = (v.read_granules.astype(np.uint64) * (v.granule_bytes // 4)).astype(np.uint32)
        hetm_testing.gpu_mark(ctx, torch.from_numpy(first).cuda())
        rs = ctx.device_tensor(h.RS_BMP)
        dlog = to_dev(torch, v.log)
        stream = ctx.stream
        for n in (len(v.log), 20011):  # second call: shorter log, scratch reused
            words = (n + 31) // 32
            ref_flags = torch.zeros(words, dtype=torch.int32, device="cuda")
            ref_cnt = torch.zeros(1, dtype=torch.int64, device="cuda")
            ctx.validate_only(dlog, n, ref_flags, ref_cnt)
            flags = torch.full((words,), -1, dtype=torch.int32, device="cuda")
            cnt = torch.full((1,), 12345, dtype=torch.int64, device="cuda")
            err = torch.full((1,), 99, dtype=torch.int32, device="cuda")
            torch.cuda.synchronize()
            rc = h.hetm_validate_noalloc(dlog, n, rs, v.granule_bytes, n_words, flags, cnt, err,
                                         stream.cuda_stream)
            assert rc == h.HETM_OK
            stream.synchronize()
            assert int(err.item()) == h.HETM_OK
            assert int(cnt.item()) == int(ref_cnt.item())
            got = flags_of(flags.cpu().numpy().view(np.uint32), n)
            exp = flags_of(ref_flags.cpu().numpy().view(np.uint32), n)
            np.testing.assert_array_equal(got, exp)
            o_flags, o_n = oracle.conflicts(v.log[:n], v.read_granules, v.granule_bytes)
            np.testing.assert_array_equal(got, o_flags)
            assert int(cnt.item()) == o_n
            if n == len(v.log):  # the planted recipe fixes the hit count of the full log
                assert o_n == v.n_hits_planted


@pytest.mark.gpu
def test_noalloc_edge_cases(hetm):
    import torch
    h = hetm
    n_words, G = 1 << 16, 64
    v = wl.validation_round(seed=13, log2_words=16, granule_bytes=G, n_log=4099, with_init=False)
    log = v.log.copy()
    bad = np.array([3, 64, 200, 4098])
    log["addr"][bad] = n_words + np.arange(bad.size, dtype=np.uint32)
    with h.Context(n_words, G) as ctx:
        first = (v.read_granules.astype(np.uint64) * (G // 4)).astype(np.uint32)
        hetm_testing.gpu_mark(ctx, torch.from_numpy(first).cuda())
        rs = ctx.device_tensor(h.RS_BMP)
        stream = ctx.stream
        for n in (0, 1, 31, 127, 128, 129, len(log)):
            part = log[:n]
            dlog = to_dev(torch, part)
            words = max((n + 31) // 32, 1)
            flags = torch.full((words,), -1, dtype=torch.int32, device="cuda")
            cnt = torch.full((1,), 777, dtype=torch.int64, device="cuda")
            err = torch.full((1,), 99, dtype=torch.int32, device="cuda")
            for with_flags in (True, False):
                torch.cuda.synchronize()
                rc = h.hetm_validate_noalloc(dlog, n, rs, G, n_words, flags if with_flags else None,
                                             cnt, err, stream.cuda_stream)
                assert rc == h.HETM_OK
                stream.synchronize()
                o_flags, o_n = oracle.conflicts(part, v.read_granules, G)
                assert int(cnt.item()) == o_n
                n_bad = int((part["addr"] >= n_words).sum())
                assert int(err.item()) == (h.HETM_EDEVICE if n_bad else h.HETM_OK)
                if with_flags and n:
                    got = flags_of(flags.cpu().numpy().view(np.uint32), n)
                    np.testing.assert_array_equal(got, o_flags)
            if n and n_bad:
                # the context-based entry point reports the same tuples
                ref_flags = torch.zeros(words, dtype=torch.int32, device="cuda")
                ref_cnt = torch.zeros(1, dtype=torch.int64, device="cuda")
                ctx.validate_only(dlog, n, ref_flags, ref_cnt)
                assert ctx.exec_counters()["rc"] == h.HETM_EDEVICE
                assert int(ref_cnt.item()) == o_n
                np.testing.assert_array_equal(
                    flags_of(ref_flags.cpu().numpy().view(np.uint32), n), o_flags)

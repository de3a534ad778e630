"""CUDA path vs the oracle at the validation-at-scale configuration's full size (needs a GPU).

The benchmark's validation workload, unchanged: 2^28 STMR words (1 GiB) and its
shadow, 64-byte granules (a 2 MiB RS_bmp), 5% of the granules read by the GPU
batch and every word of 20% of those written, and a 16,777,216-tuple CPU log
whose 2% planted hits land on read granules while the rest follow Zipf(0.9) off
them (Sec. IV-C validation, Sec. IV-D merge).  The kernels run in the launch
configuration the benchmark times (validation: one 1024-thread CTA per SM).
Every conflict flag, the conflict count, and every word of STMR^W and STMR^S
after the round are compared with the oracle; integer work, tolerance zero.
"""
import numpy as np
import pytest

import oracle
import workloads as wl
from roundkit import flags_of, to_dev

pytestmark = pytest.mark.gpu
LOG2W = 28


@pytest.fixture(scope="module")
def torch():
    import torch as t
    if not t.cuda.is_available():
        pytest.skip("no CUDA device")
    return t


@pytest.fixture(scope="module")
def vr():
    return wl.validation_round(seed=1, log2_words=LOG2W, granule_bytes=64, with_init=False)


def _first_words(v):
    return (v.read_granules.astype(np.uint64) * (v.granule_bytes // 4)).astype(np.uint32)


def test_validate_only_full_size_every_flag(hetm, torch, vr):
    """Two validate-only calls in a row over the 16.8M-tuple log: every flag and the count."""
    h = hetm
    n = len(vr.log)
    ref_flags, ref_n = oracle.conflicts(vr.log, vr.read_granules, vr.granule_bytes)
    assert ref_n == vr.n_hits_planted
    with h.Context(1 << LOG2W, vr.granule_bytes, {"log_capacity": 1 << 12}) as ctx:
        ctx.gpu_mark(torch.from_numpy(_first_words(vr)).cuda())
        dlog = to_dev(torch, vr.log)
        flags = torch.zeros((n + 31) // 32, dtype=torch.int32, device="cuda")
        cnt = torch.zeros(1, dtype=torch.int64, device="cuda")
        for _ in range(2):
            flags.fill_(-1)
            cnt.zero_()
            ctx.validate_only(dlog, n, flags, cnt)
            torch.cuda.synchronize()
            assert int(cnt.item()) == ref_n
            got = flags_of(flags.cpu().numpy().view(np.uint32), n)
            np.testing.assert_array_equal(got, ref_flags)
            # bits past the last tuple of the last flag word stay clear
            tail = flags.cpu().numpy().view(np.uint32)[-1] >> np.uint32(n % 32) if n % 32 else 0
            assert int(tail) == 0


@pytest.mark.parametrize("variant", ["conflict", "clean"])
def test_round_full_size_final_state(hetm, torch, vr, variant):
    """Validation + TS max, apply and merge of the whole round: the conflicting log
    (dirty chunks restored from S) and the log without its hits (dirty chunks W -> S)."""
    h = hetm
    wpg = vr.granule_bytes // 4
    log = vr.log
    if variant == "clean":
        is_read = np.zeros((1 << LOG2W) // wpg, dtype=bool)
        is_read[vr.read_granules] = True
        log = np.ascontiguousarray(log[~is_read[log["addr"] // wpg]])
    start = np.zeros(1 << LOG2W, np.int32)
    ref = oracle.round_planted(start, vr.read_granules, vr.plant_addr, vr.plant_value, log,
                               vr.granule_bytes)
    assert ref.ties == 0
    assert bool(ref.conflict) == (variant == "conflict")
    with h.Context(1 << LOG2W, vr.granule_bytes, {"log_capacity": 1 << 12, "cpu_threads": 1}) as ctx:
        ctx.load(torch.zeros(1 << LOG2W, dtype=torch.int32, device="cuda"))
        ctx.gpu_mark(torch.from_numpy(_first_words(vr)).cuda())
        ctx.gpu_mark(torch.from_numpy(vr.plant_addr).cuda(), torch.from_numpy(vr.plant_value).cuda())
        dlog = to_dev(torch, log)
        ctx.log_attach(dlog, len(log))
        st = ctx.round(stats=True)
        assert st["rc"] == h.HETM_OK
        assert st["n_conflicts"] == ref.n_conflicts
        assert bool(st["conflict"]) == bool(ref.conflict)
        np.testing.assert_array_equal(ctx.read_stmr(h.STMR_W), ref.final)
        np.testing.assert_array_equal(ctx.read_stmr(h.STMR_S), ref.final)

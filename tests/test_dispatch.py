"""Request queues, device affinity and work stealing (Sec. III-B, transaction
scheduling and dispatching) -- host logic, no GPU: the GPU side is a batch
function standing in for the serving loop.

Checked: affinity picks the queue (CPU_Q / GPU_Q / SHARED_Q, one queue for a
type with one implementation), CPU workers take CPU_Qs in round-robin order
and steal from SHARED_Q only when every CPU_Q is empty, the GPU activates on
gpu_min_batch or after gpu_max_wait_us and tops its batch up from SHARED_Q, a
batch whose round was rolled back runs again (every request completes exactly
once), errors reach the submission, and destroy drains the queues.
"""
import threading
import time

import numpy as np
import pytest

import paper_1905_00661_b300 as h

BANK = np.dtype([("src", "<u4"), ("dst", "<u4"), ("amount", "<i4")])
CACHE = np.dtype([("key", "<u8"), ("value", "<u8"), ("op", "<u4"), ("pad", "<u4")])
POKE = np.dtype([("addr", "<u4"), ("value", "<i4")])


def _bank(n, seed=0):
    r = np.random.default_rng(seed)
    t = np.zeros(n, BANK)
    t["src"] = np.arange(n)
    t["dst"] = r.integers(0, 1 << 20, n)
    t["amount"] = r.integers(1, 10, n)
    return t


class FakeGpu:
    """Batch function: records the batches it ran; cache outputs = 3 * key."""

    def __init__(self, outcomes=()):
        self.batches = []
        self.outcomes = list(outcomes)
        self.lock = threading.Lock()

    def __call__(self, workload, word_base, tx, n, status, out):
        rb = 24 if workload == h.HETM_WL_CACHE else 12
        assert tx.size == n * rb
        with self.lock:
            self.batches.append(tx.copy())
            oc = self.outcomes.pop(0) if self.outcomes else h.HETM_OUTCOME_CLEAN
        status[:] = 1
        if out is not None:
            keys = tx.view(CACHE)["key"]
            out.view(np.uint64)[:] = keys * 3
        return oc


def test_affinity_picks_the_queue():
    gpu = FakeGpu()
    ran_cpu = []
    lk = threading.Lock()

    def cpu(worker, rec):
        with lk:
            ran_cpu.append(np.frombuffer(rec, BANK)[0]["src"])
        return 1, None

    with h.Dispatcher(gpu_batch=gpu, cpu_workers=2, gpu_min_batch=256, gpu_max_wait_us=1000) as d:
        t = d.register(12, gpu_workload=h.HETM_WL_BANK, cpu_fn=cpu)
        recs = _bank(3000)
        a = d.submit(t, recs[:200], h.HETM_AFFINITY_CPU)
        b = d.submit(t, recs[200:1200], h.HETM_AFFINITY_GPU)
        c = d.submit(t, recs[1200:], h.HETM_AFFINITY_NONE)
        for tk, *_ in (a, b, c):
            d.wait(tk)
        st = d.stats()
    assert (a[3] == h.HETM_DEVICE_CPU).all() and (a[1] == 1).all()
    assert (b[3] == h.HETM_DEVICE_GPU).all() and (b[1] == 1).all()
    assert np.isin(c[3], [h.HETM_DEVICE_CPU, h.HETM_DEVICE_GPU]).all() and (c[1] == 1).all()
    # every request ran once, on the device its device[] entry names
    gpu_srcs = np.concatenate([x.view(BANK)["src"] for x in gpu.batches])
    cpu_srcs = np.array(ran_cpu)
    assert np.array_equal(np.sort(np.concatenate([gpu_srcs, cpu_srcs])), np.arange(3000))
    dev = np.concatenate([a[3], b[3], c[3]])
    assert np.array_equal(np.sort(cpu_srcs), np.flatnonzero(dev == h.HETM_DEVICE_CPU))
    assert st["cpu_done"] == len(cpu_srcs) and st["gpu_done"] == len(gpu_srcs)
    assert st["cpu_stolen"] + st["gpu_stolen"] == 1800
    assert st["cpu_done"] - st["cpu_stolen"] == 200
    assert st["queued_cpu"] == st["queued_gpu"] == st["queued_shared"] == 0


def test_single_implementation_types_have_one_queue():
    gpu = FakeGpu()
    with h.Dispatcher(gpu_batch=gpu, cpu_workers=1, gpu_min_batch=1, gpu_max_wait_us=100) as d:
        cpu_only = d.register(8, cpu_fn=lambda w, rec: (1, None))
        gpu_only = d.register(12, gpu_workload=h.HETM_WL_BANK)
        with pytest.raises(h.HetmError) as e:
            d.submit(cpu_only, np.zeros(4, POKE), h.HETM_AFFINITY_GPU)
        assert e.value.code == h.HETM_EINVAL
        with pytest.raises(h.HetmError):
            d.submit(gpu_only, _bank(4), h.HETM_AFFINITY_CPU)
        x = d.submit(cpu_only, np.zeros(5, POKE))
        y = d.submit(gpu_only, _bank(7))
        d.wait(x[0])
        d.wait(y[0])
    assert (x[3] == h.HETM_DEVICE_CPU).all() and (y[3] == h.HETM_DEVICE_GPU).all()


def test_register_rejects_bad_types():
    with h.Dispatcher(gpu_batch=FakeGpu(), cpu_workers=1) as d:
        for kw in (dict(rec_bytes=12),                                   # no implementation
                   dict(rec_bytes=20, gpu_workload=h.HETM_WL_RMW),      # txid is a batch position
                   dict(rec_bytes=16, gpu_workload=h.HETM_WL_BANK),     # record size
                   dict(rec_bytes=24, gpu_workload=h.HETM_WL_CACHE)):   # cache out is 8 bytes
            with pytest.raises(h.HetmError) as e:
                d.register(**kw)
            assert e.value.code == h.HETM_EINVAL
    with h.Dispatcher(cpu_workers=0) as d:
        with pytest.raises(h.HetmError):
            d.register(8, cpu_fn=lambda w, r: (1, None))                # no workers
        with pytest.raises(h.HetmError):
            d.register(12, gpu_workload=h.HETM_WL_BANK)                 # no GPU side


def test_gpu_activation_threshold_wait_and_batch_cap():
    gpu = FakeGpu()
    with h.Dispatcher(gpu_batch=gpu, cpu_workers=0, gpu_min_batch=50, gpu_max_batch=64,
                      gpu_max_wait_us=300000) as d:
        t = d.register(12, gpu_workload=h.HETM_WL_BANK)
        tk = d.submit(t, _bank(250))[0]
        lat_full = d.wait(tk)
        sizes = [len(b) // 12 for b in gpu.batches]
        assert sizes == [64, 64, 64, 58]
        assert lat_full < 250.0
        tk = d.submit(t, _bank(30, seed=1))[0]   # below the threshold: waits gpu_max_wait_us
        lat_small = d.wait(tk)
        assert lat_small >= 270.0
        assert len(gpu.batches[-1]) // 12 == 30


def test_gpu_tops_up_from_shared():
    gpu = FakeGpu()
    gate, started = threading.Event(), threading.Event()

    def slow_cpu(worker, rec):
        started.set()
        gate.wait(5)
        return 1, None

    with h.Dispatcher(gpu_batch=gpu, cpu_workers=1, gpu_min_batch=100, gpu_max_batch=1000,
                      gpu_max_wait_us=10 ** 7) as d:
        t = d.register(12, gpu_workload=h.HETM_WL_BANK, cpu_fn=slow_cpu)
        # the worker is held by its first SHARED request; the GPU takes its
        # own 60 plus 40+ stolen ones once the two queues hold 100
        s = d.submit(t, _bank(60), h.HETM_AFFINITY_NONE)
        assert started.wait(5)
        g = d.submit(t, _bank(60, seed=2), h.HETM_AFFINITY_GPU)
        t0 = time.time()
        while not gpu.batches and time.time() - t0 < 5:
            time.sleep(0.001)
        gate.set()
        d.wait(s[0])
        d.wait(g[0])
        st = d.stats()
    first = gpu.batches[0].view(BANK)
    assert len(first) == 60 + 59                       # all of GPU_Q, then SHARED_Q
    assert np.array_equal(first["src"][:60], np.arange(60))  # GPU_Q first, in order
    assert (g[3] == h.HETM_DEVICE_GPU).all()
    assert st["gpu_stolen"] == 59 and st["cpu_stolen"] == 1


def test_rolled_back_batch_runs_again():
    gpu = FakeGpu(outcomes=[h.HETM_OUTCOME_GPU_ROLLED_BACK, h.HETM_OUTCOME_CLEAN])
    r = np.zeros(500, CACHE)
    r["key"] = np.arange(1, 501)
    with h.Dispatcher(gpu_batch=gpu, cpu_workers=0, gpu_min_batch=500, gpu_max_wait_us=10 ** 6) as d:
        t = d.register(24, gpu_workload=h.HETM_WL_CACHE, out_bytes=8)
        tk, status, out, dev = d.submit(t, r, h.HETM_AFFINITY_GPU)
        d.wait(tk)
        st = d.stats()
    assert len(gpu.batches) == 2
    assert np.array_equal(gpu.batches[0], gpu.batches[1])   # same requests, same order
    assert np.array_equal(out.view(np.uint64), r["key"] * 3)
    assert (status == 1).all() and (dev == h.HETM_DEVICE_GPU).all()
    assert st["requeued"] == 500 and st["activations"] == 1 and st["gpu_done"] == 500


def test_cpu_workers_round_robin_then_steal():
    order = []
    gate, started = threading.Event(), threading.Event()

    def fn(tag):
        def f(worker, rec):
            if tag == "A" and not order:
                order.append("A")
                started.set()
                gate.wait(5)
                return 1, None
            order.append(tag)
            return 1, None
        return f

    with h.Dispatcher(gpu_batch=FakeGpu(), cpu_workers=1, gpu_min_batch=10 ** 6,
                      gpu_max_wait_us=10 ** 7) as d:
        ta = d.register(8, cpu_fn=fn("A"))
        tb = d.register(8, cpu_fn=fn("B"))
        tc = d.register(12, gpu_workload=h.HETM_WL_BANK, cpu_fn=fn("C"))
        first = d.submit(ta, np.zeros(1, POKE))
        assert started.wait(5)                # the worker now holds the first A
        subs = [d.submit(tc, _bank(2)), d.submit(ta, np.zeros(3, POKE)),
                d.submit(tb, np.zeros(3, POKE))]
        gate.set()
        for tk, *_ in [first] + subs:
            d.wait(tk)
    assert order == ["A", "B", "A", "B", "A", "B", "A", "C", "C"]


def test_errors_reach_the_submission():
    def bad_cpu(worker, rec):
        return h.HETM_ECAPACITY, None

    def bad_gpu(*a):
        raise RuntimeError("kernel failed")

    with h.Dispatcher(gpu_batch=bad_gpu, cpu_workers=1, gpu_min_batch=1) as d:
        tc = d.register(8, cpu_fn=bad_cpu)
        tg = d.register(12, gpu_workload=h.HETM_WL_BANK)
        x = d.submit(tc, np.zeros(2, POKE))
        y = d.submit(tg, _bank(3))
        with pytest.raises(h.HetmError) as e:
            d.wait(x[0])
        assert e.value.code == h.HETM_ECAPACITY
        with pytest.raises(h.HetmError) as e:
            d.wait(y[0])
        assert e.value.code == h.HETM_EINVAL
        with pytest.raises(h.HetmError):
            d.wait(12345)                     # unknown ticket


def test_destroy_runs_every_queued_request():
    gpu = FakeGpu()
    n_cpu = []

    def cpu(worker, rec):
        n_cpu.append(1)
        return 1, None

    d = h.Dispatcher(gpu_batch=gpu, cpu_workers=2, gpu_min_batch=10 ** 6, gpu_max_wait_us=10 ** 7)
    t = d.register(12, gpu_workload=h.HETM_WL_BANK, cpu_fn=cpu)
    keep = [d.submit(t, _bank(700), a) for a in (h.HETM_AFFINITY_CPU, h.HETM_AFFINITY_GPU,
                                                 h.HETM_AFFINITY_NONE)]
    d.close()
    assert len(n_cpu) + sum(len(b) // 12 for b in gpu.batches) == 2100
    assert (keep[0][3] == h.HETM_DEVICE_CPU).all() and (keep[1][3] == h.HETM_DEVICE_GPU).all()
    assert all((k[1] == 1).all() for k in keep)

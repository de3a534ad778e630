"""Python binding of libhetm.so -- the GPU side of a SHeTM synchronization round.

Argument marshalling only: every step of the round runs in the CUDA library
(``csrc/``), whose C ABI is ``include/hetm.h``.  PyTorch supplies device
memory (the context allocates through torch's caching allocator) and streams
(each context owns a torch CUDA stream, ordered against the caller's current
stream on every call).  There is no CPU fallback: importing this package
without the built library, or using it without a CUDA device, raises.

The module-level ``hetm_*`` functions carry the C names; ``Context`` is the
same API on an object.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libhetm.so")

HETM_OK, HETM_EINVAL, HETM_ENOMEM, HETM_ECAPACITY = 0, -1, -2, -3
HETM_ETIMEOUT, HETM_ECUDA, HETM_EBUSY, HETM_EDEVICE = -4, -5, -6, -7
HETM_WL_BANK, HETM_WL_RMW, HETM_WL_CACHE, HETM_WL_W2 = 1, 2, 3, 4
HETM_POLICY_GPU_LOSES, HETM_POLICY_CPU_LOSES = 0, 1
HETM_OUTCOME_CLEAN, HETM_OUTCOME_GPU_ROLLED_BACK, HETM_OUTCOME_CPU_DISCARDED = 0, 1, 2
HETM_EXEC_ORDERED, HETM_EXEC_OPTIMISTIC = 0, 1
HETM_BATCH_QUEUED, HETM_BATCH_RUNNING, HETM_BATCH_DONE = 1, 2, 3
HETM_OUTCOME_UNKNOWN = 0xFFFFFFFF
HETM_AFFINITY_NONE, HETM_AFFINITY_CPU, HETM_AFFINITY_GPU = 0, 1, 2
HETM_DEVICE_CPU, HETM_DEVICE_GPU = 1, 2
STMR_W, STMR_S, TS, RS_BMP, WS_BMP = 0, 1, 2, 3, 4

LOG_DTYPE = np.dtype([("addr", "<u4"), ("value", "<i4"), ("ts", "<u4")])

_vp, _u32, _u64, _i32, _int = (ctypes.c_void_p, ctypes.c_uint32, ctypes.c_uint64,
                               ctypes.c_int32, ctypes.c_int)
_ALLOC = ctypes.CFUNCTYPE(ctypes.c_void_p, ctypes.c_size_t, ctypes.c_void_p)
_FREE = ctypes.CFUNCTYPE(None, ctypes.c_void_p, ctypes.c_void_p)


class hetm_config(ctypes.Structure):
    _fields_ = [("ws_chunk_bytes", _u32), ("lock_log2", _u32), ("lock_shift", _u32),
                ("exec_blocks", _u32), ("exec_threads", _u32), ("max_attempts", _u32),
                ("cpu_threads", _u32), ("log_chunk_bytes", _u32), ("log_capacity", _u64),
                ("cpu_log_capacity", _u64), ("max_batches", _u32), ("cache_log2_sets", _u32),
                ("cache_key_base", _u64), ("cache_val_base", _u64), ("cache_lru_base", _u64),
                ("cache_ver_base", _u64), ("exec_mode", _u32), ("early_validate", _u32),
                ("max_round_tx", _u64), ("dev_alloc", _ALLOC), ("dev_free", _FREE),
                ("alloc_user", _vp), ("conflict_policy", _u32), ("starve_limit", _u32),
                ("exec_budget_us", _u32), ("uninstrumented", _u32)]


class hetm_batch(ctypes.Structure):
    _fields_ = [("workload", _u32), ("n_tx", _u32), ("tx", _vp), ("order", _vp), ("status", _vp),
                ("out", _vp), ("txid_base", _u32), ("word_base", _u32)]


class hetm_batch_result(ctypes.Structure):
    _fields_ = [("state", _u32), ("outcome", _u32), ("round", _u64), ("n_tx", _u32),
                ("reserved", _u32), ("latency_ms", ctypes.c_double)]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_ if k != "reserved"}


class hetm_round_stats(ctypes.Structure):
    _fields_ = [("n_log", _u64), ("n_conflicts", _u64), ("conflict", _i32), ("err", _i32),
                ("committed", _u64), ("gave_up", _u64), ("aborts", _u64), ("dirty_chunks", _u64),
                ("n_batches", _u32), ("ms_exec", ctypes.c_float), ("ms_validate", ctypes.c_float),
                ("ms_apply", ctypes.c_float), ("ms_merge", ctypes.c_float),
                ("ms_total", ctypes.c_float), ("n_kernels", _u32), ("stopped_early", _u32),
                ("outcome", _u32), ("cpu_read_only_next", _u32)]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


#: every symbol include/hetm.h declares
SYMBOLS = ("hetm_strerror", "hetm_config_default", "hetm_init", "hetm_destroy", "hetm_load",
           "hetm_read_stmr", "hetm_device_ptr", "hetm_bitmap_words", "hetm_sync",
           "hetm_gpu_submit_batch", "hetm_gpu_exec", "hetm_exec_counters",
           "hetm_cpu_log_write", "hetm_log_attach", "hetm_validate", "hetm_validate_only",
           "hetm_merge", "hetm_round", "hetm_validate_noalloc", "hetm_ctx_stream",
           "hetm_round_wait", "hetm_server_config_default", "hetm_server_create",
           "hetm_server_submit", "hetm_server_wait", "hetm_server_get_stats",
           "hetm_server_destroy", "hetm_tune_space_default", "hetm_autotune",
           "hetm_read_dirty",
           "hetm_cpu_updates_allowed", "hetm_batch_poll", "hetm_server_wait_outcome",
           "hetm_dispatch_config_default", "hetm_dispatch_create", "hetm_dispatch_register",
           "hetm_dispatch_submit", "hetm_dispatch_wait", "hetm_dispatch_get_stats",
           "hetm_dispatch_destroy", "hetm_read_dirty_async", "hetm_read_dirty_wait")


class hetm_tune_space(ctypes.Structure):
    _fields_ = [("modes", _u32), ("threads", _u32 * 4), ("blocks_per_sm", _u32 * 4),
                ("lock_log2", _u32 * 4), ("granules", _u32 * 8), ("ws_chunk_bytes", _u32 * 6),
                ("reps", _u32), ("cut", ctypes.c_float)]


class hetm_tune_trial(ctypes.Structure):
    _fields_ = [("stage", _u32), ("exec_mode", _u32), ("exec_threads", _u32),
                ("exec_blocks", _u32), ("lock_log2", _u32), ("granule_bytes", _u32),
                ("ws_chunk_bytes", _u32), ("rc", _i32), ("rounds", _u32), ("conflicts", _u32),
                ("committed", _u64), ("ms_exec", ctypes.c_float), ("ms_round", ctypes.c_float),
                ("score", ctypes.c_float), ("reserved", _u32)]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_ if k != "reserved"}


class hetm_request(ctypes.Structure):
    _fields_ = [("workload", _u32), ("n_tx", _u32), ("host_tx", _vp), ("host_order", _vp),
                ("host_status", _vp), ("host_out", _vp), ("txid_base", _u32), ("word_base", _u32)]


class hetm_server_config(ctypes.Structure):
    _fields_ = [("per_batch", _i32), ("max_round_batches", _u32), ("max_round_tx", _u64),
                ("device_budget", _u64), ("free_reserve", _u64)]


class hetm_server_stats(ctypes.Structure):
    _fields_ = [("rounds", _u64), ("completed", _u64), ("committed", _u64), ("refused", _u64),
                ("p50_ms", ctypes.c_double), ("p99_ms", ctypes.c_double), ("max_ms", ctypes.c_double),
                ("span_s", ctypes.c_double)]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


#: hetm_cpu_tx_fn(user, worker, tx, out) -> status byte or negative HETM_E* code
CPU_TX_FN = ctypes.CFUNCTYPE(_int, _vp, _u32, _vp, _vp)
#: hetm_gpu_batch_fn(user, workload, word_base, tx, n, status, out, outcome) -> rc
GPU_BATCH_FN = ctypes.CFUNCTYPE(_int, _vp, _u32, _u32, _vp, _u32, _vp, _vp, ctypes.POINTER(_u32))


class hetm_tx_type(ctypes.Structure):
    _fields_ = [("gpu_workload", _u32), ("rec_bytes", _u32), ("out_bytes", _u32),
                ("word_base", _u32), ("cpu_fn", CPU_TX_FN), ("cpu_user", _vp)]


class hetm_dispatch_config(ctypes.Structure):
    _fields_ = [("cpu_workers", _u32), ("gpu_min_batch", _u32), ("gpu_max_batch", _u32),
                ("gpu_max_wait_us", _u32), ("gpu_inflight", _u32)]


class hetm_dispatch_stats(ctypes.Structure):
    _fields_ = [("cpu_done", _u64), ("gpu_done", _u64), ("cpu_stolen", _u64), ("gpu_stolen", _u64),
                ("activations", _u64), ("requeued", _u64), ("queued_cpu", _u64),
                ("queued_gpu", _u64), ("queued_shared", _u64)]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


class HetmError(RuntimeError):
    def __init__(self, code, what=""):
        self.code = code
        super().__init__(f"{what}: {code} ({strerror(code)})")


def _declare(L):
    P = ctypes.POINTER
    sig = {
        "hetm_strerror": (ctypes.c_char_p, [_int]),
        "hetm_config_default": (_int, [P(hetm_config)]),
        "hetm_init": (_int, [P(_vp), _u64, _u32, P(hetm_config), _vp]),
        "hetm_destroy": (None, [_vp]),
        "hetm_load": (_int, [_vp, _vp, _u64]),
        "hetm_read_stmr": (_int, [_vp, _int, _vp, _u64, _u64]),
        "hetm_device_ptr": (_vp, [_vp, _int]),
        "hetm_bitmap_words": (_int, [_vp, P(_u64), P(_u64)]),
        "hetm_sync": (_int, [_vp]),
        "hetm_gpu_submit_batch": (_int, [_vp, P(hetm_batch), P(_u64)]),
        "hetm_gpu_exec": (_int, [_vp, _int]),
        "hetm_exec_counters": (_int, [_vp, P(_u64), P(_u64), P(_u64)]),
        "hetm_cpu_log_write": (_int, [_vp, _u32, _vp, _u32]),
        "hetm_log_attach": (_int, [_vp, _vp, _u64]),
        "hetm_validate": (_int, [_vp, P(_u64), _vp]),
        "hetm_validate_only": (_int, [_vp, _vp, _u64, _vp, _vp]),
        "hetm_merge": (_int, [_vp, _int]),
        "hetm_round": (_int, [_vp, P(hetm_round_stats)]),
        "hetm_validate_noalloc": (_int, [_vp, _u64, _vp, _u32, _u64, _vp, _vp, _vp, _vp]),
        "hetm_ctx_stream": (_vp, [_vp]),
        "hetm_round_wait": (_int, [_vp, P(hetm_round_stats)]),
        "hetm_batch_poll": (_int, [_vp, _u64, P(hetm_batch_result)]),
        "hetm_server_config_default": (_int, [P(hetm_server_config)]),
        "hetm_server_create": (_int, [P(_vp), _vp, P(hetm_server_config)]),
        "hetm_server_submit": (_int, [_vp, P(hetm_request), P(_u64)]),
        "hetm_server_wait": (_int, [_vp, _u64, P(ctypes.c_double)]),
        "hetm_server_wait_outcome": (_int, [_vp, _u64, P(ctypes.c_double), P(_u32)]),
        "hetm_dispatch_config_default": (_int, [P(hetm_dispatch_config)]),
        "hetm_dispatch_create": (_int, [P(_vp), _vp, GPU_BATCH_FN, _vp, P(hetm_dispatch_config)]),
        "hetm_dispatch_register": (_int, [_vp, P(hetm_tx_type), P(_u32)]),
        "hetm_dispatch_submit": (_int, [_vp, _u32, _int, _vp, _u32, _vp, _vp, _vp, P(_u64)]),
        "hetm_dispatch_wait": (_int, [_vp, _u64, P(ctypes.c_double)]),
        "hetm_dispatch_get_stats": (_int, [_vp, P(hetm_dispatch_stats)]),
        "hetm_dispatch_destroy": (None, [_vp]),
        "hetm_server_get_stats": (_int, [_vp, P(hetm_server_stats)]),
        "hetm_server_destroy": (None, [_vp]),
        "hetm_tune_space_default": (_int, [P(hetm_tune_space)]),
        "hetm_read_dirty": (_int, [_vp, _vp, P(_u64), P(_u64)]),
        "hetm_read_dirty_async": (_int, [_vp, _vp, P(_u64), P(_u64)]),
        "hetm_read_dirty_wait": (_int, [_vp]),
        "hetm_cpu_updates_allowed": (_int, [_vp]),
        "hetm_autotune": (_int, [_u64, _vp, P(hetm_batch), _u32, _vp, _u64, P(hetm_config),
                                 P(hetm_tune_space), P(hetm_config), P(_u32), P(hetm_tune_trial),
                                 _u32, P(_u32)]),
    }
    for name, (res, args) in sig.items():
        f = getattr(L, name)
        f.restype, f.argtypes = res, args
    return L


def load_library(path: str = LIB_PATH):
    """ctypes handle of the library; raises if it has not been built."""
    if not os.path.exists(path):
        raise ImportError(f"{path} is missing: build it with `python paper_1905_00661_b300/build.py`")
    return _declare(ctypes.CDLL(path))


_lib = load_library()


def lib():
    return _lib


def strerror(code: int) -> str:
    return _lib.hetm_strerror(code).decode()


def _ck(rc, what):
    if rc != HETM_OK:
        raise HetmError(rc, what)
    return rc


def _round_reported(rc, stats):
    """A round call's code that its stats explain (the round ran): OK, or the
    device error the round reports in ``err``."""
    return rc == HETM_OK or (rc in (HETM_EDEVICE, HETM_ETIMEOUT, HETM_EINVAL) and rc == stats["err"])


# ---------------------------------------------------------------------------
# C-named wrappers
# ---------------------------------------------------------------------------
def hetm_config_default() -> hetm_config:
    cfg = hetm_config()
    _ck(_lib.hetm_config_default(ctypes.byref(cfg)), "hetm_config_default")
    return cfg


def hetm_init(stmr_words, granule_bytes, cfg=None, stream=None):
    h = _vp()
    _ck(_lib.hetm_init(ctypes.byref(h), stmr_words, granule_bytes,
                       ctypes.byref(cfg) if cfg is not None else None, stream), "hetm_init")
    return h


def _ptr(x):
    """Device or host address of a torch tensor, numpy array, int or None."""
    if x is None:
        return None
    if isinstance(x, int):
        return x
    if isinstance(x, np.ndarray):
        assert x.flags["C_CONTIGUOUS"]
        return x.ctypes.data
    assert x.is_contiguous(), "tensors passed to the library must be contiguous"
    return x.data_ptr()


class _CudaArray:
    def __init__(self, ptr, n, typestr):
        self.__cuda_array_interface__ = {"shape": (n,), "typestr": typestr, "data": (ptr, False),
                                         "version": 3, "strides": None}


HETM_NOALLOC_MAX_TUPLES = 1 << 25


def hetm_validate_noalloc(dev_log, n, dev_rs_bmp, granule_bytes, stmr_words, dev_flag_bits,
                          dev_n_conflicts, dev_err=None, stream=None):
    """Allocation-free validation (see include/hetm.h): device pointers or tensors in,
    hit count (and optional error code) written to device memory; returns the C status."""
    return _lib.hetm_validate_noalloc(_ptr(dev_log), n, _ptr(dev_rs_bmp), granule_bytes,
                                      stmr_words, _ptr(dev_flag_bits), _ptr(dev_n_conflicts),
                                      _ptr(dev_err), stream)


def hetm_tune_space_default() -> hetm_tune_space:
    sp = hetm_tune_space()
    _ck(_lib.hetm_tune_space_default(ctypes.byref(sp)), "hetm_tune_space_default")
    return sp




_TUNED = ("exec_mode", "exec_threads", "exec_blocks", "lock_log2", "ws_chunk_bytes")


def autotune(stmr_words, init, batches, log=None, n_log=None, base=None, space=None,
             max_trials=128):
    """Pick the executor shape, conflict granule and merge chunk for a sample
    (hetm_autotune).  ``batches``: list of (workload, tx, order, status, out)
    or dicts with those keys plus optional n_tx / txid_base / word_base, device
    tensors.  ``log``: device tensor of log entries or None.  ``base`` and
    ``space``: dicts of hetm_config / hetm_tune_space fields.  Returns
    {"config": tuned fields, "granule_bytes": G, "trials": [...]}."""
    import torch
    if isinstance(init, np.ndarray):
        init = np.ascontiguousarray(init, dtype=np.int32)
    torch.cuda.current_stream().synchronize()
    descs = (hetm_batch * len(batches))()
    for i, b in enumerate(batches):
        if not isinstance(b, dict):
            b = dict(zip(("workload", "tx", "order", "status", "out"), b))
        tx = b["tx"]
        n_tx = b.get("n_tx")
        if n_tx is None:
            n_tx = len(tx) if isinstance(tx, np.ndarray) else tx.numel() * tx.element_size() // {
                HETM_WL_BANK: 12, HETM_WL_RMW: 20, HETM_WL_CACHE: 24}[b["workload"]]
        descs[i] = hetm_batch(b["workload"], int(n_tx), _ptr(tx), _ptr(b.get("order")),
                              _ptr(b.get("status")), _ptr(b.get("out")), b.get("txid_base", 0),
                              b.get("word_base", 0))
    cfg = hetm_config_default()
    for k, v in (base or {}).items():
        setattr(cfg, k, v)
    sp = hetm_tune_space_default()
    for k, v in (space or {}).items():
        if isinstance(getattr(sp, k), ctypes.Array):
            arr = getattr(sp, k)
            for j in range(len(arr)):
                arr[j] = v[j] if j < len(v) else 0
        else:
            setattr(sp, k, v)
    if log is not None and n_log is None:
        n_log = log.numel() * log.element_size() // 12
    best, g = hetm_config(), _u32()
    trials = (hetm_tune_trial * max_trials)()
    nt = _u32()
    _ck(_lib.hetm_autotune(int(stmr_words), _ptr(init), descs, len(batches), _ptr(log),
                           int(n_log or 0), ctypes.byref(cfg), ctypes.byref(sp), ctypes.byref(best),
                           ctypes.byref(g), trials, max_trials, ctypes.byref(nt)), "hetm_autotune")
    return {"config": {k: getattr(best, k) for k in _TUNED}, "granule_bytes": g.value,
            "trials": [trials[i].as_dict() for i in range(min(nt.value, max_trials))]}


# ---------------------------------------------------------------------------
# object API
# ---------------------------------------------------------------------------
class Context:
    """One STMR replica on the GPU plus the state of its synchronization rounds."""

    def __init__(self, stmr_words: int, granule_bytes: int, config: dict | None = None,
                 torch_allocator: bool = True):
        import torch
        if not torch.cuda.is_available():
            raise RuntimeError("the SHeTM round library needs a CUDA device")
        self.torch = torch
        self.n_words = int(stmr_words)
        self.granule_bytes = int(granule_bytes)
        self.stream = torch.cuda.Stream()
        cfg = hetm_config_default()
        for k, v in (config or {}).items():
            setattr(cfg, k, v)
        self._cb = None
        if torch_allocator:
            dev = torch.cuda.current_device()
            stream = self.stream

            def _alloc(nbytes, user):
                try:
                    return torch.cuda.caching_allocator_alloc(int(nbytes), dev, stream)
                except Exception:
                    return None

            def _free(p, user):
                torch.cuda.caching_allocator_delete(p)

            self._cb = (_ALLOC(_alloc), _FREE(_free))
            cfg.dev_alloc, cfg.dev_free = self._cb
        self.config = cfg
        self.h = hetm_init(self.n_words, self.granule_bytes, cfg, self.stream.cuda_stream)
        rw, ww = _u64(), _u64()
        _ck(_lib.hetm_bitmap_words(self.h, ctypes.byref(rw), ctypes.byref(ww)), "hetm_bitmap_words")
        self.rs_words, self.ws_words = rw.value, ww.value

    # stream ordering against the caller's torch stream
    def _enter(self):
        self.stream.wait_stream(self.torch.cuda.current_stream())

    def _leave(self):
        self.torch.cuda.current_stream().wait_stream(self.stream)

    def close(self):
        if getattr(self, "h", None):
            _lib.hetm_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    # ------------------------------------------------------------- state
    def load(self, src):
        """STMR^W = STMR^S = src (numpy int32 or CUDA int32 tensor); TS and bitmaps cleared."""
        if isinstance(src, np.ndarray):
            src = np.ascontiguousarray(src, dtype=np.int32)
        else:
            self._enter()
        _ck(_lib.hetm_load(self.h, _ptr(src), len(src)), "hetm_load")

    def read_stmr(self, which=STMR_W, off=0, n=None) -> np.ndarray:
        n = self.n_words - off if n is None else n
        out = np.empty(n, np.int32)
        _ck(_lib.hetm_read_stmr(self.h, which, out.ctypes.data, off, n), "hetm_read_stmr")
        return out

    def device_tensor(self, which):
        """Zero-copy torch view of STMR^W, STMR^S, TS, RS_bmp or WS_bmp."""
        p = _lib.hetm_device_ptr(self.h, which)
        n = {STMR_W: self.n_words, STMR_S: self.n_words, TS: self.n_words,
             RS_BMP: self.rs_words, WS_BMP: self.ws_words}[which]
        ts = "<i4" if which in (STMR_W, STMR_S) else "<u4"
        t = self.torch.as_tensor(_CudaArray(p, n, ts), device="cuda")
        return t

    def sync(self):
        _ck(_lib.hetm_sync(self.h), "hetm_sync")

    # ------------------------------------------------------------- execution
    def submit_batch(self, workload, tx, order=None, status=None, out=None, txid_base=0,
                     word_base=0, n_tx=None) -> int:
        b = hetm_batch(workload, int(len(tx) if n_tx is None else n_tx), _ptr(tx), _ptr(order),
                       _ptr(status), _ptr(out), txid_base, word_base)
        bid = _u64()
        _ck(_lib.hetm_gpu_submit_batch(self.h, ctypes.byref(b), ctypes.byref(bid)),
            "hetm_gpu_submit_batch")
        return bid.value

    def gpu_exec(self, per_batch=False):
        self._enter()
        _ck(_lib.hetm_gpu_exec(self.h, int(per_batch)), "hetm_gpu_exec")
        self._leave()

    def exec_counters(self):
        c, g, a = _u64(), _u64(), _u64()
        rc = _lib.hetm_exec_counters(self.h, ctypes.byref(c), ctypes.byref(g), ctypes.byref(a))
        return {"committed": c.value, "gave_up": g.value, "aborts": a.value, "rc": rc}

    # ------------------------------------------------------------- CPU logs
    def cpu_log_write(self, thread, entries: np.ndarray):
        e = np.ascontiguousarray(entries)
        assert e.dtype.itemsize == 12
        _ck(_lib.hetm_cpu_log_write(self.h, thread, e.ctypes.data, len(e)), "hetm_cpu_log_write")

    def log_attach(self, dev_log, n=None):
        n = dev_log.numel() * dev_log.element_size() // 12 if n is None else n
        _ck(_lib.hetm_log_attach(self.h, _ptr(dev_log), n), "hetm_log_attach")

    # ------------------------------------------------------------- validation / merge
    def validate(self, flags=None, sync=True):
        self._enter()
        n = _u64()
        _ck(_lib.hetm_validate(self.h, ctypes.byref(n) if sync else None, _ptr(flags)),
            "hetm_validate")
        self._leave()
        return n.value if sync else None

    def validate_only(self, dev_log, n, flags=None, count=None):
        self._enter()
        _ck(_lib.hetm_validate_only(self.h, _ptr(dev_log), n, _ptr(flags), _ptr(count)),
            "hetm_validate_only")
        self._leave()

    def read_dirty(self, host_stmr: np.ndarray):
        """Copy the last round's surviving GPU-dirty chunks into the host replica
        (int32 numpy array of stmr_words); returns (chunks, bytes) copied."""
        assert host_stmr.dtype == np.int32 and host_stmr.size == self.n_words
        assert host_stmr.flags["C_CONTIGUOUS"]
        c, b = _u64(), _u64()
        _ck(_lib.hetm_read_dirty(self.h, host_stmr.ctypes.data, ctypes.byref(c), ctypes.byref(b)),
            "hetm_read_dirty")
        return c.value, b.value

    def read_dirty_async(self, host_stmr):
        """Double-buffered read_dirty: queue the copies into ``host_stmr`` (a pinned
        int32 torch CPU tensor of stmr_words, or a numpy array -- then the copies
        are synchronous) and return (chunks, bytes) at once; the next write of
        STMR^S waits for them on the device.  Read the replica after
        :meth:`read_dirty_wait`."""
        if isinstance(host_stmr, np.ndarray):
            assert host_stmr.dtype == np.int32 and host_stmr.flags["C_CONTIGUOUS"]
            size, addr = host_stmr.size, host_stmr.ctypes.data
        else:
            assert host_stmr.dtype == self.torch.int32 and not host_stmr.is_cuda
            assert host_stmr.is_contiguous()
            size, addr = host_stmr.numel(), host_stmr.data_ptr()
        assert size == self.n_words
        c, b = _u64(), _u64()
        _ck(_lib.hetm_read_dirty_async(self.h, addr, ctypes.byref(c), ctypes.byref(b)),
            "hetm_read_dirty_async")
        return c.value, b.value

    def read_dirty_wait(self):
        _ck(_lib.hetm_read_dirty_wait(self.h), "hetm_read_dirty_wait")

    def cpu_updates_allowed(self) -> bool:
        return bool(_lib.hetm_cpu_updates_allowed(self.h))

    def merge(self, conflict=-1):
        self._enter()
        _ck(_lib.hetm_merge(self.h, int(conflict)), "hetm_merge")
        self._leave()

    def round(self, stats=True):
        self._enter()
        if stats:
            st = hetm_round_stats()
            rc = _lib.hetm_round(self.h, ctypes.byref(st))
            self._leave()
            d = st.as_dict()
            d["rc"] = rc
            if not _round_reported(rc, d):
                raise HetmError(rc, "hetm_round")
            return d
        rc = _lib.hetm_round(self.h, None)
        self._leave()
        _ck(rc, "hetm_round")
        return None

    def round_wait(self):
        """Wait for the oldest round started by ``round(stats=False)`` and not yet
        collected (two may be in flight); its stats."""
        st = hetm_round_stats()
        rc = _lib.hetm_round_wait(self.h, ctypes.byref(st))
        d = st.as_dict()
        d["rc"] = rc
        if not _round_reported(rc, d):
            raise HetmError(rc, "hetm_round_wait")
        return d

    def batch_poll(self, batch_id):
        """State of a submitted batch without blocking (HETM_BATCH_*), the outcome
        of the round that ran it, its round number and its latency once done."""
        r = hetm_batch_result()
        _ck(_lib.hetm_batch_poll(self.h, int(batch_id), ctypes.byref(r)), "hetm_batch_poll")
        return r.as_dict()


class Server:
    """Serving loop over a Context (continuous batching into rounds, see include/hetm.h).

    ``submit`` takes numpy record arrays and fills numpy result arrays that the
    caller keeps alive until ``wait``; ``per_batch`` selects one round per batch."""

    def __init__(self, ctx: Context, per_batch=False, max_round_batches=1024,
                 max_round_tx=1 << 22, device_budget=0, free_reserve=0):
        cfg = hetm_server_config()
        _ck(_lib.hetm_server_config_default(ctypes.byref(cfg)), "hetm_server_config_default")
        cfg.per_batch = int(per_batch)
        cfg.max_round_batches = max_round_batches
        cfg.max_round_tx = max_round_tx
        cfg.device_budget = device_budget
        cfg.free_reserve = free_reserve
        self.ctx = ctx
        self.h = _vp()
        ctx.torch.cuda.synchronize()
        _ck(_lib.hetm_server_create(ctypes.byref(self.h), ctx.h, ctypes.byref(cfg)),
            "hetm_server_create")
        self._keep = {}

    def submit(self, workload, tx, order=None, status=None, out=None, txid_base=0, word_base=0):
        tx = np.ascontiguousarray(tx)
        r = hetm_request(workload, len(tx), tx.ctypes.data, _ptr(order), _ptr(status), _ptr(out),
                         txid_base, word_base)
        bid = _u64()
        _ck(_lib.hetm_server_submit(self.h, ctypes.byref(r), ctypes.byref(bid)), "hetm_server_submit")
        self._keep[bid.value] = (tx, order, status, out)
        return bid.value

    def wait(self, bid):
        lat = ctypes.c_double()
        rc = _lib.hetm_server_wait(self.h, bid, ctypes.byref(lat))
        self._keep.pop(bid, None)
        _ck(rc, "hetm_server_wait")
        return lat.value

    def stats(self):
        st = hetm_server_stats()
        _ck(_lib.hetm_server_get_stats(self.h, ctypes.byref(st)), "hetm_server_get_stats")
        return st.as_dict()

    def close(self):
        if getattr(self, "h", None):
            _lib.hetm_server_destroy(self.h)
            self.h = None

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()


class Dispatcher:
    """Request queues with device affinity and work stealing (see include/hetm.h).

    GPU batches go to ``server`` (a :class:`Server`) or, without one, to
    ``gpu_batch(workload, word_base, tx_bytes, n, status, out) -> outcome``, a
    Python function that fills the numpy arrays ``status`` (uint8[n]) and ``out``
    (uint8[n * out_bytes] or None) and returns the HETM_OUTCOME_* of the round.
    CPU functions registered with :meth:`register` are called as
    ``cpu_fn(worker, record_bytes) -> (status, out_bytes or None)`` from the
    dispatcher's worker threads.  This class needs no CUDA device unless a
    server is attached."""

    def __init__(self, server=None, gpu_batch=None, cpu_workers=2, gpu_min_batch=1024,
                 gpu_max_batch=1 << 20, gpu_max_wait_us=2000, gpu_inflight=2):
        cfg = hetm_dispatch_config()
        _ck(_lib.hetm_dispatch_config_default(ctypes.byref(cfg)), "hetm_dispatch_config_default")
        cfg.cpu_workers, cfg.gpu_min_batch, cfg.gpu_max_batch = cpu_workers, gpu_min_batch, gpu_max_batch
        cfg.gpu_max_wait_us, cfg.gpu_inflight = gpu_max_wait_us, gpu_inflight
        self._types = []   # (record bytes, out bytes, callback object)
        self._keep = {}
        self._gpu_cb = GPU_BATCH_FN(self._gpu_trampoline) if gpu_batch else GPU_BATCH_FN()
        self._gpu_batch = gpu_batch
        self.h = _vp()
        _ck(_lib.hetm_dispatch_create(ctypes.byref(self.h), server.h if server else None,
                                      self._gpu_cb, None, ctypes.byref(cfg)), "hetm_dispatch_create")

    def _gpu_trampoline(self, user, workload, word_base, tx, n, status, out, outcome):
        try:
            rb = {HETM_WL_BANK: 12, HETM_WL_CACHE: 24}[workload]
            ob = 8 if workload == HETM_WL_CACHE else 0
            txb = np.frombuffer(ctypes.string_at(tx, n * rb), np.uint8)
            st = np.zeros(n, np.uint8)
            o = np.zeros(n * ob, np.uint8) if ob and out else None
            outcome[0] = int(self._gpu_batch(workload, word_base, txb, n, st, o))
            ctypes.memmove(status, st.ctypes.data, n)
            if o is not None:
                ctypes.memmove(out, o.ctypes.data, o.nbytes)
            return HETM_OK
        except Exception:  # reported to the submissions of the batch
            return HETM_EINVAL

    def register(self, rec_bytes, gpu_workload=0, out_bytes=0, word_base=0, cpu_fn=None):
        """Register a transaction type; returns its id."""
        cb = CPU_TX_FN()
        if cpu_fn is not None:
            def tramp(user, worker, tx, out, _f=cpu_fn, _rb=rec_bytes, _ob=out_bytes):
                try:
                    st, o = _f(worker, ctypes.string_at(tx, _rb))
                    if out and _ob and o is not None:
                        ctypes.memmove(out, bytes(o)[:_ob], _ob)
                    return int(st)
                except Exception:
                    return HETM_EINVAL
            cb = CPU_TX_FN(tramp)
        t = hetm_tx_type(gpu_workload, rec_bytes, out_bytes, word_base, cb, None)
        tid = _u32()
        _ck(_lib.hetm_dispatch_register(self.h, ctypes.byref(t), ctypes.byref(tid)),
            "hetm_dispatch_register")
        self._types.append((rec_bytes, out_bytes, cb))
        return tid.value

    def submit(self, type_id, records, affinity=HETM_AFFINITY_NONE):
        """Queue the requests in ``records`` (a numpy record array); returns
        (ticket, status uint8[n], out uint8[n * out_bytes] or None, device uint8[n]),
        the result arrays being filled by the time :meth:`wait` returns."""
        rec = np.ascontiguousarray(records)
        rb, ob, _ = self._types[type_id]
        assert rec.dtype.itemsize == rb
        n = len(rec)
        status = np.zeros(n, np.uint8)
        device = np.zeros(n, np.uint8)
        out = np.zeros(n * ob, np.uint8) if ob else None
        tk = _u64()
        _ck(_lib.hetm_dispatch_submit(self.h, type_id, affinity, rec.ctypes.data, n,
                                      status.ctypes.data, _ptr(out), device.ctypes.data,
                                      ctypes.byref(tk)), "hetm_dispatch_submit")
        self._keep[tk.value] = rec
        return tk.value, status, out, device

    def wait(self, ticket):
        lat = ctypes.c_double()
        rc = _lib.hetm_dispatch_wait(self.h, ticket, ctypes.byref(lat))
        self._keep.pop(ticket, None)
        _ck(rc, "hetm_dispatch_wait")
        return lat.value

    def stats(self):
        st = hetm_dispatch_stats()
        _ck(_lib.hetm_dispatch_get_stats(self.h, ctypes.byref(st)), "hetm_dispatch_get_stats")
        return st.as_dict()

    def close(self):
        if getattr(self, "h", None):
            _lib.hetm_dispatch_destroy(self.h)
            self.h = None

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

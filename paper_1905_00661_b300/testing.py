"""Python binding of the measurement probes and test scaffolding
(``include/hetm_testing.h``): not part of a synchronization round.

* ``gpu_mark`` plants a GPU batch's footprint (``hetm_gpu_mark``, in
  libhetm.so): the tests and the benchmark drive validation and merge with an
  exactly known read and write set through it.
* ``handoff_latency``, ``random_access_rate`` and ``l2_probe_rate`` measure
  the hardware floors the round's kernels are compared with (libhetm_testing.so).

Argument marshalling only, like the package itself.
"""
from __future__ import annotations

import ctypes
import os

from . import _ck, _lib, _ptr, _u32, _u64, _vp, _int

LIB_PATH = os.path.join(os.path.dirname(os.path.abspath(__file__)), "libhetm_testing.so")

#: every symbol include/hetm_testing.h declares, and the library that exports it
SYMBOLS = {"hetm_gpu_mark": "libhetm.so", "hetm_handoff_latency": "libhetm_testing.so",
           "hetm_random_access_rate": "libhetm_testing.so",
           "hetm_l2_probe_rate": "libhetm_testing.so",
           "hetm_log_stream_time": "libhetm_testing.so"}

_D = ctypes.POINTER(ctypes.c_double)
_lib.hetm_gpu_mark.restype, _lib.hetm_gpu_mark.argtypes = _int, [_vp, _vp, _vp, _u64]
_tl = None


def lib():
    """ctypes handle of libhetm_testing.so; raises if it has not been built."""
    global _tl
    if _tl is None:
        if not os.path.exists(LIB_PATH):
            raise ImportError(f"{LIB_PATH} is missing: build it with "
                              "`python paper_1905_00661_b300/build.py`")
        L = ctypes.CDLL(LIB_PATH)
        L.hetm_handoff_latency.restype, L.hetm_handoff_latency.argtypes = _int, [_u32, _D, _D]
        L.hetm_random_access_rate.restype, L.hetm_random_access_rate.argtypes = _int, [_u32, _u64, _D, _D]
        L.hetm_l2_probe_rate.restype, L.hetm_l2_probe_rate.argtypes = _int, [_u32, _u64, _u32, _D]
        L.hetm_log_stream_time.restype, L.hetm_log_stream_time.argtypes = _int, [_vp, _u64, _u32, _D]
        _tl = L
    return _tl


def gpu_mark(ctx, addr, vals=None):
    """Plant the words a GPU batch read (vals None) or wrote (device tensors)."""
    ctx._enter()
    _ck(_lib.hetm_gpu_mark(ctx.h, _ptr(addr), _ptr(vals), len(addr)), "hetm_gpu_mark")
    ctx._leave()


def handoff_latency(rounds=20000):
    """(cross-SM ns, cross-warp ns) for one hand-on of a word (hetm_handoff_latency)."""
    g, sh = ctypes.c_double(), ctypes.c_double()
    _ck(lib().hetm_handoff_latency(int(rounds), ctypes.byref(g), ctypes.byref(sh)),
        "hetm_handoff_latency")
    return g.value, sh.value


def random_access_rate(log2_words=28, n_access=1 << 28):
    """(random 4-byte reads/s, writes/s) over a 2^log2_words-word array (hetm_random_access_rate)."""
    r, w = ctypes.c_double(), ctypes.c_double()
    _ck(lib().hetm_random_access_rate(int(log2_words), int(n_access), ctypes.byref(r),
                                      ctypes.byref(w)), "hetm_random_access_rate")
    return r.value, w.value


def l2_probe_rate(log2_words=19, n_probe=1 << 24, smem_bytes=128 * 1024):
    """Random 4-byte probes per second of an L2-resident 2^log2_words-word array,
    in the validation kernel's launch shape (hetm_l2_probe_rate)."""
    r = ctypes.c_double()
    _ck(lib().hetm_l2_probe_rate(int(log2_words), int(n_probe), int(smem_bytes), ctypes.byref(r)),
        "hetm_l2_probe_rate")
    return r.value


def log_stream_time(dev_log, n, smem_bytes=128 * 1024):
    """Seconds for the validation kernel's log stream alone over n tuples of a
    device log (hetm_log_stream_time)."""
    r = ctypes.c_double()
    _ck(lib().hetm_log_stream_time(_ptr(dev_log), int(n), int(smem_bytes), ctypes.byref(r)),
        "hetm_log_stream_time")
    return r.value

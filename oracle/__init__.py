"""CPU oracle for SHeTM synchronization rounds -- test infrastructure only.

Plain single-threaded C++ (``hetm_oracle.cpp``) behind ctypes.  It computes
what a round must produce, from the definitions in the paper
(arXiv 1905.00661):

* ``replay_*``   -- serial replay in the reported commit order (P1, Sec. III)
                    of bank, W1, W2 (Sec. V-A) and object-cache batches,
                    plus the exact read/write granule sets (Sec. IV-B/IV-C);
* ``conflicts``  -- CPU write-set vs GPU read-set by brute-force set
                    intersection (Sec. IV-C, Validation Phase);
* ``cpu_image``  -- newest-timestamp tuple per word, applied only when newer
                    than the stored timestamp (Sec. IV-C, array TS);
* ``final_state``-- (conflict ? start : replayed) overlaid with the CPU image
                    (Sec. IV-C Merge Phase, Sec. IV-D rollback);
* ``final_state_cpu_loses`` -- the CPU-loses policy (Sec. IV-E): the CPU
                    image only after a clean validation, else the replay;
* ``round_*``    -- the above composed for one round.

``cpu_validate_apply_mt`` is not part of the oracle: it is the timed CPU
baseline of the synchronization phase (``cpu_baseline.cpp``, std::thread),
checked against the oracle in ``tests/test_oracle.py`` and timed by
``bench.py``.

Pins: every function is checked by ``tests/test_oracle.py`` against
hand-enumerated rounds (``tests/golden/``), closed forms, invariants and
brute force over serial orders.  No function here is "parity unpinned".

Only ``tests/``, ``__graft_entry__.smoke()`` and ``bench.py``'s CPU-baseline
leg may import this package.  It shares no code with the CUDA library.
"""
from __future__ import annotations

import ctypes
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "hetm_oracle.cpp")
_LIB = os.path.join(_HERE, "liboracle.so")

_c_u64p = ctypes.POINTER(ctypes.c_uint64)


_MT_SRC = os.path.join(_HERE, "cpu_baseline.cpp")
_MT_LIB = os.path.join(_HERE, "libcpubase.so")


def build(force: bool = False) -> str:
    """Compile the oracle into ``oracle/liboracle.so`` and the timed CPU
    baseline into ``oracle/libcpubase.so`` (g++, no GPU needed)."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        subprocess.check_call(["g++", "-O2", "-std=c++17", "-shared", "-fPIC", _SRC, "-o", _LIB])
    if force or not os.path.exists(_MT_LIB) or os.path.getmtime(_MT_LIB) < os.path.getmtime(_MT_SRC):
        subprocess.check_call(["g++", "-O3", "-std=c++17", "-pthread", "-shared", "-fPIC", _MT_SRC,
                               "-o", _MT_LIB])
    return _LIB


_lib = None


def lib():
    global _lib
    if _lib is None:
        build()
        L = ctypes.CDLL(_LIB)
        vp, u64, u32, i64, ci = ctypes.c_void_p, ctypes.c_uint64, ctypes.c_uint32, ctypes.c_int64, ctypes.c_int
        L.hetm_oracle_replay_bank.argtypes = [vp, u64, vp, u64, vp, vp, u32, u32, vp, u64, vp, vp, u64, vp]
        L.hetm_oracle_replay_bank.restype = ci
        L.hetm_oracle_replay_rmw.argtypes = [vp, u64, vp, u64, vp, vp, u32, vp, u32, u32, vp, u64, vp,
                                             vp, u64, vp]
        L.hetm_oracle_replay_rmw.restype = ci
        L.hetm_oracle_replay_w2.argtypes = [vp, u64, vp, u64, vp, vp, u32, vp, u32, u32, vp, u64, vp,
                                            vp, u64, vp]
        L.hetm_oracle_replay_w2.restype = ci
        L.hetm_oracle_replay_cache.argtypes = [vp, u64, u32, u64, u64, u64, u64, vp, u64, vp, vp, vp,
                                               u32, u32, vp, u64, vp, vp, u64, vp]
        L.hetm_oracle_replay_cache.restype = ci
        L.hetm_oracle_conflicts.argtypes = [vp, u64, vp, u64, u32, vp]
        L.hetm_oracle_conflicts.restype = i64
        L.hetm_oracle_cpu_image.argtypes = [vp, vp, u64, vp, u64]
        L.hetm_oracle_cpu_image.restype = i64
        L.hetm_oracle_final_state.argtypes = [vp, vp, u64, ci, vp, u64, vp, vp]
        L.hetm_oracle_final_state.restype = i64
        L.hetm_oracle_plant.argtypes = [vp, u64, vp, vp, u64]
        L.hetm_oracle_plant.restype = ci
        L.hetm_oracle_sum64.argtypes = [vp, u64]
        L.hetm_oracle_sum64.restype = i64
        _lib = L
    return _lib


def _p(a: np.ndarray):
    assert a.flags["C_CONTIGUOUS"], "oracle arrays must be contiguous"
    return a.ctypes.data


def _u8(a):
    return np.ascontiguousarray(a, dtype=np.uint8)


def _u64(a):
    return np.ascontiguousarray(a, dtype=np.uint64)


def _sets_out(cap_r, cap_d):
    return (np.zeros(max(cap_r, 1), np.uint32), np.zeros(max(cap_d, 1), np.uint32),
            np.zeros(1, np.uint64), np.zeros(1, np.uint64))


def replay_bank(stmr, txs, order, status, granule_bytes, chunk_bytes):
    """Replay committed transfers on ``stmr`` (in place); returns (R, D) granule/chunk ids."""
    order, status = _u64(order), _u8(status)
    r, d, nr, nd = _sets_out(2 * len(txs), 2 * len(txs))
    rc = lib().hetm_oracle_replay_bank(_p(stmr), stmr.size, _p(txs), len(txs), _p(order), _p(status),
                                       granule_bytes, chunk_bytes, _p(r), r.size, _p(nr),
                                       _p(d), d.size, _p(nd))
    if rc != 0:
        raise ValueError("oracle bank replay failed")
    return r[: int(nr[0])].copy(), d[: int(nd[0])].copy()


def replay_rmw(stmr, txs, order, status, granule_bytes, chunk_bytes, txid_base=0):
    """Replay W1-style transactions; returns (out_sum int32[n], R, D)."""
    order, status = _u64(order), _u8(status)
    out = np.zeros(len(txs), np.int32)
    r, d, nr, nd = _sets_out(4 * len(txs), 4 * len(txs))
    rc = lib().hetm_oracle_replay_rmw(_p(stmr), stmr.size, _p(txs), len(txs), _p(order), _p(status),
                                      txid_base, _p(out), granule_bytes, chunk_bytes, _p(r), r.size,
                                      _p(nr), _p(d), d.size, _p(nd))
    if rc != 0:
        raise ValueError("oracle rmw replay failed")
    return out, r[: int(nr[0])].copy(), d[: int(nd[0])].copy()


def replay_w2(stmr, txs, order, status, granule_bytes, chunk_bytes, txid_base=0):
    """Replay W2 transactions (40 reads, updates write their first 4 words);
    returns (out_sum int32[n], R, D)."""
    order, status = _u64(order), _u8(status)
    out = np.zeros(len(txs), np.int32)
    r, d, nr, nd = _sets_out(40 * len(txs), 4 * len(txs))
    rc = lib().hetm_oracle_replay_w2(_p(stmr), stmr.size, _p(txs), len(txs), _p(order), _p(status),
                                     txid_base, _p(out), granule_bytes, chunk_bytes, _p(r), r.size,
                                     _p(nr), _p(d), d.size, _p(nd))
    if rc != 0:
        raise ValueError("oracle W2 replay failed")
    return out, r[: int(nr[0])].copy(), d[: int(nd[0])].copy()


def replay_cache(stmr, layout, reqs, order, status, granule_bytes, chunk_bytes):
    """Replay cache requests; returns (out uint64[n], R, D).  ``layout`` is a workloads.CacheLayout."""
    order, status = _u64(order), _u8(status)
    out = np.zeros(len(reqs), np.uint64)
    cap = 40 * len(reqs) + 8
    r, d, nr, nd = _sets_out(cap, cap)
    rc = lib().hetm_oracle_replay_cache(_p(stmr), stmr.size, layout.log2_sets, layout.key_base,
                                        layout.val_base, layout.gpu_lru_base, layout.ver_base,
                                        _p(reqs), len(reqs), _p(order), _p(status), _p(out),
                                        granule_bytes, chunk_bytes, _p(r), r.size, _p(nr),
                                        _p(d), d.size, _p(nd))
    if rc != 0:
        raise ValueError("oracle cache replay failed")
    return out, r[: int(nr[0])].copy(), d[: int(nd[0])].copy()


def conflicts(log, read_granules, granule_bytes):
    """Per-entry conflict flags (uint8) and their count."""
    rg = np.ascontiguousarray(read_granules, dtype=np.uint32)
    flags = np.zeros(max(len(log), 1), np.uint8)
    n = lib().hetm_oracle_conflicts(_p(log), len(log), _p(rg), rg.size, granule_bytes, _p(flags))
    return flags[: len(log)], int(n)


def cpu_image(state, ts_state, log):
    """Overlay the newest-timestamp CPU writes on ``state`` (may be None); returns #ties."""
    st = 0 if state is None else _p(state)
    n = ts_state.size
    ties = lib().hetm_oracle_cpu_image(st, _p(ts_state), n, _p(log), len(log))
    if ties < 0:
        raise ValueError("log address out of range")
    return int(ties)


def final_state(start, replayed, conflict, log, ts_state):
    out = np.empty_like(start)
    ties = lib().hetm_oracle_final_state(_p(start), _p(replayed), start.size, int(bool(conflict)),
                                         _p(log), len(log), _p(ts_state), _p(out))
    if ties < 0:
        raise ValueError("log address out of range")
    return out, int(ties)


def plant(stmr, addr, value):
    addr = np.ascontiguousarray(addr, np.uint32)
    value = np.ascontiguousarray(value, np.int32)
    if lib().hetm_oracle_plant(_p(stmr), stmr.size, _p(addr), _p(value), addr.size) != 0:
        raise ValueError("planted address out of range")


def sum64(stmr):
    return int(lib().hetm_oracle_sum64(_p(stmr), stmr.size))


# ---------------------------------------------------------------------------
# composed rounds
# ---------------------------------------------------------------------------
class RoundResult:
    def __init__(self, **kw):
        self.__dict__.update(kw)


def final_state_cpu_loses(replayed, conflict, log, ts_state):
    """Final STMR under the CPU-loses policy (Sec. IV-E): the CPU write-sets
    are applied only when the whole validation found no conflict.  On a
    conflict the apply is skipped, so the GPU's replayed state stands and
    ``ts_state`` is left as it was; without one the round ends as under
    GPU-loses (the replay overlaid with the newest-timestamp CPU image)."""
    if conflict:
        return replayed.copy(), 0
    return final_state(replayed, replayed, False, log, ts_state)


def round_from_replay(start, replayed, R, log, granule_bytes, ts_state, cpu_loses=False):
    """Validation + final state, given the GPU's replayed state and read granules R."""
    flags, n_conf = conflicts(log, R, granule_bytes)
    if cpu_loses:
        final, ties = final_state_cpu_loses(replayed, n_conf > 0, log, ts_state)
    else:
        final, ties = final_state(start, replayed, n_conf > 0, log, ts_state)
    return RoundResult(flags=flags, n_conflicts=n_conf, conflict=n_conf > 0, final=final, ties=ties)


def round_bank(start, txs, order, status, log, granule_bytes, chunk_bytes, ts_state=None):
    ts_state = np.zeros(start.size, np.uint32) if ts_state is None else ts_state
    replayed = start.copy()
    R, D = replay_bank(replayed, txs, order, status, granule_bytes, chunk_bytes)
    res = round_from_replay(start, replayed, R, log, granule_bytes, ts_state)
    res.replayed, res.R, res.D, res.ts_state = replayed, R, D, ts_state
    return res


def round_rmw(start, txs, order, status, log, granule_bytes, chunk_bytes, ts_state=None,
              txid_base=0):
    ts_state = np.zeros(start.size, np.uint32) if ts_state is None else ts_state
    replayed = start.copy()
    out, R, D = replay_rmw(replayed, txs, order, status, granule_bytes, chunk_bytes, txid_base)
    res = round_from_replay(start, replayed, R, log, granule_bytes, ts_state)
    res.replayed, res.R, res.D, res.out, res.ts_state = replayed, R, D, out, ts_state
    return res


def round_planted(start, read_granules, plant_addr, plant_value, log, granule_bytes,
                  ts_state=None):
    """Validation-at-scale round: the GPU batch is given as read granules + written words."""
    ts_state = np.zeros(start.size, np.uint32) if ts_state is None else ts_state
    replayed = start.copy()
    plant(replayed, plant_addr, plant_value)
    wpg = granule_bytes // 4
    R = np.union1d(np.asarray(read_granules, np.uint32),
                   (np.asarray(plant_addr, np.uint64) // wpg).astype(np.uint32))
    res = round_from_replay(start, replayed, R, log, granule_bytes, ts_state)
    res.replayed, res.R, res.ts_state = replayed, R, ts_state
    return res


_mt = None


def cpu_validate_apply_mt(log, rs_words, granule_bytes, W, S, TS, threads, flags=None):
    """Timed CPU baseline: validation + apply of ``log`` against the RS_bmp
    words ``rs_words`` on host W, S, TS (updated in place) with ``threads``
    std::threads; returns the hit count."""
    global _mt
    if _mt is None:
        build()
        _mt = ctypes.CDLL(_MT_LIB)
        vp = ctypes.c_void_p
        _mt.hetm_cpu_validate_apply_mt.argtypes = [vp, ctypes.c_uint64, vp, ctypes.c_uint32,
                                                   ctypes.c_uint64, vp, vp, vp, vp, ctypes.c_int]
        _mt.hetm_cpu_validate_apply_mt.restype = ctypes.c_int64
    rs = np.ascontiguousarray(rs_words, np.uint32)
    gshift = int(np.log2(granule_bytes // 4))
    n = _mt.hetm_cpu_validate_apply_mt(_p(log), len(log), _p(rs), gshift, W.size, _p(W), _p(S), _p(TS),
                                       None if flags is None else _p(flags), int(threads))
    if n < 0:
        raise ValueError("log address out of range")
    return int(n)

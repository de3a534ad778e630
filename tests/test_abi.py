"""The C-ABI libraries load and export every symbol include/hetm.h and
include/hetm_testing.h declare (no GPU)."""
import ctypes
import os
import re

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared(header="hetm.h"):
    src = open(os.path.join(ROOT, "include", header)).read()
    return set(re.findall(r"HETM_API[^;(]*?\b(hetm_\w+)\s*\(", src))


def test_header_declares_binding_symbols():
    import paper_1905_00661_b300 as h
    import paper_1905_00661_b300.testing as t
    assert _declared() == set(h.SYMBOLS)
    assert _declared("hetm_testing.h") == set(t.SYMBOLS)
    assert not _declared() & _declared("hetm_testing.h")


def test_library_exports_every_declared_symbol():
    import paper_1905_00661_b300 as h
    import paper_1905_00661_b300.testing as t
    L = ctypes.CDLL(h.LIB_PATH)
    for name in _declared():
        assert hasattr(L, name), name
    libs = {"libhetm.so": L, "libhetm_testing.so": ctypes.CDLL(t.LIB_PATH)}
    for name, where in t.SYMBOLS.items():
        assert hasattr(libs[where], name), name
    # the probes are not part of the round library
    for name in ("hetm_handoff_latency", "hetm_random_access_rate", "hetm_l2_probe_rate",
                 "hetm_log_stream_time"):
        assert not hasattr(L, name), name


def test_strerror_and_defaults_without_gpu():
    import paper_1905_00661_b300 as h
    assert h.strerror(h.HETM_OK) == "ok"
    assert "capacity" in h.strerror(h.HETM_ECAPACITY)
    cfg = h.hetm_config_default()
    assert cfg.ws_chunk_bytes == 16384 and cfg.log_chunk_bytes == 49152
    assert cfg.lock_log2 == 22 and cfg.max_batches == 4096
    assert cfg.exec_mode == h.HETM_EXEC_ORDERED and cfg.max_round_tx == 1 << 22


def test_round_codes_the_binding_returns_as_stats():
    """A round call returns its stats when the code is the device error the
    round itself reports (a timeout, an address error, a CPU timestamp out of
    range or repeated); any other code -- an argument error before the round
    ran, a CUDA failure -- raises."""
    import paper_1905_00661_b300 as h
    ok = h._round_reported
    assert ok(h.HETM_OK, {"err": h.HETM_OK})
    for code in (h.HETM_ETIMEOUT, h.HETM_EDEVICE, h.HETM_EINVAL):
        assert ok(code, {"err": code})
        assert not ok(code, {"err": h.HETM_OK})
    assert not ok(h.HETM_ECUDA, {"err": h.HETM_OK})
    assert not ok(h.HETM_EBUSY, {"err": h.HETM_OK})
    assert not ok(h.HETM_EINVAL, {"err": h.HETM_EDEVICE})


def test_record_layouts_match_workloads():
    import paper_1905_00661_b300 as h
    import workloads as wl
    assert h.LOG_DTYPE == wl.LOG_DTYPE
    assert ctypes.sizeof(h.hetm_batch) == 48
    assert ctypes.sizeof(h.hetm_config) == 144
    assert ctypes.sizeof(h.hetm_round_stats) == 96


def test_init_rejects_bad_arguments_before_touching_the_device():
    import paper_1905_00661_b300 as h
    L = h.lib()
    p = ctypes.c_void_p()
    assert L.hetm_init(ctypes.byref(p), 0, 64, None, None) == h.HETM_EINVAL
    assert L.hetm_init(ctypes.byref(p), 1024, 48, None, None) == h.HETM_EINVAL
    assert L.hetm_init(ctypes.byref(p), 1 << 32, 64, None, None) == h.HETM_EINVAL
    cfg = h.hetm_config_default()
    cfg.ws_chunk_bytes = 100
    assert L.hetm_init(ctypes.byref(p), 1024, 64, ctypes.byref(cfg), None) == h.HETM_EINVAL


def test_autotune_space_and_argument_checks_without_gpu():
    import paper_1905_00661_b300 as h
    assert ctypes.sizeof(h.hetm_tune_space) == 116
    assert ctypes.sizeof(h.hetm_tune_trial) == 64
    sp = h.hetm_tune_space_default()
    assert sp.modes == 3 and list(sp.threads) == [128, 256, 512, 0]
    assert list(sp.granules)[:4] == [4, 64, 1024, 0] and sp.reps == 3
    best, g = h.hetm_config(), ctypes.c_uint32()
    # no sample: rejected before any device call
    rc = h.lib().hetm_autotune(1 << 10, None, None, 0, None, 0, None, None, ctypes.byref(best),
                               ctypes.byref(g), None, 0, None)
    assert rc == h.HETM_EINVAL


def test_handoff_probe_rejects_bad_arguments_without_gpu():
    import paper_1905_00661_b300 as h
    import paper_1905_00661_b300.testing as t
    g = ctypes.c_double()
    assert t.lib().hetm_handoff_latency(0, ctypes.byref(g), None) == h.HETM_EINVAL
    assert t.lib().hetm_handoff_latency(100, None, None) == h.HETM_EINVAL


def test_random_access_probe_rejects_bad_arguments_without_gpu():
    import paper_1905_00661_b300 as h
    import paper_1905_00661_b300.testing as t
    r = ctypes.c_double()
    assert t.lib().hetm_l2_probe_rate(9, 100, 0, ctypes.byref(r)) == h.HETM_EINVAL
    assert t.lib().hetm_l2_probe_rate(19, 100, 300 * 1024, ctypes.byref(r)) == h.HETM_EINVAL
    assert t.lib().hetm_log_stream_time(None, 100, 0, ctypes.byref(r)) == h.HETM_EINVAL
    assert t.lib().hetm_random_access_rate(10, 100, ctypes.byref(r), None) == h.HETM_EINVAL
    assert t.lib().hetm_random_access_rate(24, 0, ctypes.byref(r), None) == h.HETM_EINVAL
    assert t.lib().hetm_random_access_rate(24, 100, None, None) == h.HETM_EINVAL


def test_early_validation_fields_keep_layouts():
    import paper_1905_00661_b300 as h
    cfg = h.hetm_config_default()
    assert cfg.early_validate == 0
    assert cfg.conflict_policy == h.HETM_POLICY_GPU_LOSES and cfg.starve_limit == 0
    assert h.hetm_round_stats.stopped_early.offset == 84


def test_struct_layouts_match_the_c_compiler(tmp_path):
    """Every ctypes struct of the binding has the size and field offsets that
    gcc gives the same struct from include/hetm.h."""
    import shutil
    import subprocess
    import paper_1905_00661_b300 as h
    if not shutil.which("gcc"):
        import pytest
        pytest.skip("no gcc")
    structs = [h.hetm_config, h.hetm_round_stats, h.hetm_batch, h.hetm_tune_space,
               h.hetm_tune_trial, h.hetm_request, h.hetm_server_config, h.hetm_server_stats]
    lines = ['#include <stdio.h>', '#include <stddef.h>', '#include "hetm.h"', "int main(void) {"]
    for st in structs:
        n = st.__name__
        lines.append(f'printf("{n} %zu\\n", sizeof({n}));')
        for f, _ in st._fields_:
            lines.append(f'printf("{n}.{f} %zu\\n", offsetof({n}, {f}));')
    lines.append("return 0; }")
    src = tmp_path / "layout.c"
    src.write_text("\n".join(lines))
    exe = tmp_path / "layout"
    subprocess.check_call(["gcc", "-std=c11", "-I", os.path.join(ROOT, "include"), str(src),
                           "-o", str(exe)])
    got = dict(line.split() for line in subprocess.check_output([str(exe)]).decode().splitlines())
    for st in structs:
        n = st.__name__
        assert int(got[n]) == ctypes.sizeof(st), n
        for f, _ in st._fields_:
            assert int(got[f"{n}.{f}"]) == getattr(st, f).offset, f"{n}.{f}"


def test_batch_poll_rejects_bad_arguments_without_gpu():
    import paper_1905_00661_b300 as h
    L = h.lib()
    r = h.hetm_batch_result()
    assert L.hetm_batch_poll(None, 1, ctypes.byref(r)) == h.HETM_EINVAL
    assert L.hetm_batch_poll(None, 1, None) == h.HETM_EINVAL
    assert ctypes.sizeof(h.hetm_batch_result) == 32

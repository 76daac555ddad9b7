"""The C-ABI library builds for sm_103a, loads, and exports every entry point
declared in include/sbr.h (no GPU needed; no compute calls)."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    src = open(os.path.join(ROOT, "include", "sbr.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(sbr_[A-Za-z_0-9]+)\s*\(", src)))


@pytest.fixture(scope="module")
def lib():
    from paper_2208_10006_gb300 import build as b
    b.build()
    from paper_2208_10006_gb300 import _lib
    return _lib.load()


def test_every_declared_symbol_is_exported(lib):
    names = _declared()
    assert len(names) >= 15
    for n in names:
        assert hasattr(lib, n), n
    from paper_2208_10006_gb300 import _lib
    assert sorted(_lib.EXPORTS) == names


def test_version_and_error_string_without_gpu(lib):
    assert b"sm_103a" in lib.sbr_version()
    assert lib.sbr_last_error() == b""


def test_host_validation_rejects_bad_arguments_before_any_launch(lib):
    from paper_2208_10006_gb300 import _lib
    # N out of range: rejected on the host, no CUDA call made
    assert lib.sbr_launch_dirs(0, None, None, None) == 1
    assert b"N in" in lib.sbr_last_error()
    out = ctypes.c_void_p()
    assert lib.sbr_build_bvh(None, None, -1, 1, ctypes.byref(out), None) == 1
    assert lib.sbr_build_bvh_ex(None, None, 0, 1, ctypes.c_uint32(2), ctypes.byref(out), None) == 1
    assert b"flags" in lib.sbr_last_error()
    assert lib.sbr_trace(None, None, ctypes.byref(out), None) == 1
    assert lib.sbr_capacity(None, 1, 1, 1, None, 1, None, None) == 1


def test_library_is_built_for_sm103a_only():
    from paper_2208_10006_gb300 import build as b
    assert b.ARCH == "-gencode=arch=compute_103a,code=sm_103a"
    assert all("-gencode" not in f or f == b.ARCH for f in b.flags())


def test_ctypes_struct_layouts_match_the_header(tmp_path):
    # sizes and field offsets of the binding's structs against a C compile of sbr.h
    import shutil
    import subprocess
    if shutil.which("gcc") is None:
        pytest.skip("no C compiler")
    from paper_2208_10006_gb300 import _lib
    checks = {"sbr_trace_params": (_lib.TraceParams, ["tx", "rx_xyz", "alpha", "flags", "ray_begin", "ray_end"]),
              "sbr_trace_counters": (_lib.TraceCounters, ["near_edge_hits", "queue", "alpha", "bounce_ms"]),
              "sbr_path_info": (_lib.PathInfo, ["n_paths", "status"]),
              "sbr_batch_job": (_lib.BatchJob, ["tx", "alpha", "F", "freqs_hz", "H"]),
              "sbr_batch_config": (_lib.BatchConfig, ["path_cap", "use_graph", "breadth_first"]),
              "sbr_batch_info": (_lib.BatchInfo, ["max_keys", "rays", "config"]),
              "sbr_mlp_config": (_lib.MlpConfig, ["seed", "x_lo", "lr", "err_channel", "err_of"])}
    lines = ["#include <stdio.h>", "#include <stddef.h>", '#include "sbr.h"', "int main(void) {"]
    for cname, (_, fields) in checks.items():
        lines.append('printf("%%zu\\n", sizeof(%s));' % cname)
        for f in fields:
            lines.append('printf("%%zu\\n", offsetof(%s, %s));' % (cname, f))
    lines.append("return 0; }")
    src = tmp_path / "layout.c"
    src.write_text("\n".join(lines))
    exe = tmp_path / "layout"
    cuda_inc = "/usr/local/cuda/include"
    subprocess.run(["gcc", "-I", os.path.join(ROOT, "include"), "-I", cuda_inc, str(src), "-o", str(exe)],
                   check=True)
    got = [int(x) for x in subprocess.run([str(exe)], check=True, capture_output=True, text=True).stdout.split()]
    want = []
    for cname, (cls, fields) in checks.items():
        want.append(ctypes.sizeof(cls))
        want += [getattr(cls, f).offset for f in fields]
    assert got == want


@pytest.mark.parametrize("n", [65, 96, 128])
def test_capacity_rejects_arrays_above_64_on_the_host(lib, n):
    # the header's contract: min(Nr, Nt) <= 64 (the Cholesky of one frequency
    # lives in shared memory); larger arrays are refused before any CUDA call,
    # by both capacity entry points, with the limit named in the message
    snr = (ctypes.c_double * 1)(0.0)
    fake = ctypes.c_void_p(256)   # never dereferenced: the check comes first
    for entry in (lib.sbr_capacity, lib.sbr_capacity_noalloc):
        assert entry(fake, 1, n, n + 3, snr, 1, fake, None) == 1
        assert b"64" in lib.sbr_last_error()
    # n = 64 passes the array check and fails only on the SNR count (33 > 32)
    snr33 = (ctypes.c_double * 33)()
    assert lib.sbr_capacity(fake, 1, 64, 64, snr33, 33, fake, None) == 1
    assert b"n_snr" in lib.sbr_last_error()

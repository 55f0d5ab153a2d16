"""CPU checks of the boundary: the library loads and exports every entry point
include/clight.h declares, and the Python record layouts match the header."""
import ctypes
import os
import re

import numpy as np

import paper_2309_15861_gb300 as G
from paper_2309_15861_gb300 import build, inputs as I

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    txt = open(os.path.join(ROOT, "include", "clight.h")).read()
    txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
    return sorted(set(re.findall(r"\b(clight_[a-z0-9_]+)\s*\(", txt)))


def test_library_exports_every_declared_symbol():
    build.build()
    lib = ctypes.CDLL(G.LIB_PATH)
    names = _declared()
    assert "clight_trace" in names and "clight_create" in names
    missing = [n for n in names if not hasattr(lib, n)]
    assert not missing, missing


def test_record_layouts_match_the_header():
    assert I.SEG_DTYPE.itemsize == 64
    assert G.HIT_DTYPE.itemsize == 48
    assert ctypes.sizeof(G.Stats) == 104
    assert ctypes.sizeof(G.Params) == 192
    assert ctypes.sizeof(G.Atmosphere) == 8 + 3 * 64 + 7 * 8 + 8 + 16
    offs = {n: I.SEG_DTYPE.fields[n][1] for n in I.SEG_DTYPE.names}
    assert offs == {"x": 0, "y": 8, "z": 16, "t0": 24, "dx": 32, "dy": 36, "dz": 40, "L": 44,
                    "eps": 48, "dE": 52, "charge": 56, "shower": 60}
    hoffs = {n: G.HIT_DTYPE.fields[n][1] for n in G.HIT_DTYPE.names}
    assert hoffs == {"seg": 0, "k": 8, "tel": 12, "x_rel": 16, "y_rel": 20, "cx": 24, "cy": 28,
                     "lambda": 32, "weight": 36, "t": 40}


def test_status_strings_and_no_device_on_cpu():
    lib = G.lib()
    assert lib.clight_status_string(G.ERR_HIT_CAPACITY) == b"hit capacity exceeded"
    import torch
    if not torch.cuda.is_available():
        h = ctypes.c_void_p()
        assert lib.clight_create(ctypes.byref(h), 0) == G.ERR_NO_DEVICE
        rates = G.PipeRates()
        assert lib.clight_measure_pipes(0, ctypes.byref(rates)) == G.ERR_NO_DEVICE


def test_entry_points_refuse_what_they_cannot_use_before_any_device_call():
    """Argument checks on the host: a NULL context or output is refused with
    CLIGHT_ERR_ARG before any CUDA call (so this runs without a GPU)."""
    lib = G.lib()
    n64 = ctypes.c_int64()
    st = G.Stats()
    assert lib.clight_measure_pipes(0, None) == G.ERR_ARG
    assert lib.clight_trace(None, None, 0, 1, None, 0, None, None, ctypes.byref(st), ctypes.byref(n64), None) == G.ERR_ARG
    assert lib.clight_trace_fp64(None, None, 0, 1, None, 0, None, None, ctypes.byref(st), ctypes.byref(n64),
                                 None) == G.ERR_ARG
    assert lib.clight_trace_host(None, None, 0, 1, None, 0, None, None, ctypes.byref(st), ctypes.byref(n64),
                                 None) == G.ERR_ARG
    assert lib.clight_trace_noalloc(None, None, 0, 1, None, 0, None, ctypes.byref(st), ctypes.byref(n64),
                                    None) == G.ERR_ARG
    grad = (ctypes.c_double * 10)()
    assert lib.clight_trace_adjoint(None, None, 0, 1, None, 0, None, None, None, None, 0.5, 20.0, None, grad,
                                    None) == G.ERR_ARG
    t = G.Tune()
    assert lib.clight_autotune(None, None, 1, 1, 1, None, 0, 5.0, 1, ctypes.byref(t), None) == G.ERR_ARG
    ms = (ctypes.c_float * 3)()
    assert lib.clight_last_timing(None, ms) == G.ERR_ARG
    assert lib.clight_last_adjoint(None, None, None, ms) == G.ERR_ARG
    assert lib.clight_set_atmosphere(None, None) == G.ERR_ARG
    assert lib.clight_set_telescopes(None, None, 0) == G.ERR_ARG
    assert lib.clight_set_params(None, None) == G.ERR_ARG


def _c_layouts(tmp_path):
    """sizeof and field offsets of the header's records, printed by a C
    program that includes include/clight.h (gcc)."""
    import shutil
    import subprocess
    cc = shutil.which("gcc") or shutil.which("cc")
    if cc is None:
        import pytest
        pytest.skip("no C compiler")
    recs = {
        "clight_segment": ["x", "y", "z", "t0", "dx", "dy", "dz", "L", "eps", "dE", "charge", "shower"],
        "clight_hit": ["seg", "k", "tel", "x_rel", "y_rel", "cx", "cy", "lambda", "weight", "t"],
        "clight_stats": [n for n, _ in G.Stats._fields_],
        "clight_params": [n for n, _ in G.Params._fields_],
        "clight_atmosphere": [n for n, _ in G.Atmosphere._fields_],
        "clight_tune": [n for n, _ in G.Tune._fields_],
        "clight_pipe_rates": [n for n, _ in G.PipeRates._fields_],
    }
    lines = ['#include <stdio.h>', '#include <stddef.h>', '#include "clight.h"', "int main(void) {"]
    for r, fields in recs.items():
        lines.append(f'printf("{r} size %zu\\n", sizeof({r}));')
        for f in fields:
            lines.append(f'printf("{r} {f} %zu\\n", offsetof({r}, {f}));')
    lines.append("return 0; }")
    src = tmp_path / "layouts.c"
    src.write_text("\n".join(lines))
    exe = tmp_path / "layouts"
    subprocess.run([cc, "-std=c99", "-I", os.path.join(ROOT, "include"), str(src), "-o", str(exe)], check=True)
    out = subprocess.run([str(exe)], check=True, capture_output=True, text=True).stdout
    got = {}
    for line in out.splitlines():
        r, f, v = line.split()
        got[(r, f)] = int(v)
    return got


def test_binding_layouts_equal_the_c_header(tmp_path):
    """Every record the binding passes through the ABI has the C header's
    size and field offsets (compiled from include/clight.h)."""
    import ctypes as C
    got = _c_layouts(tmp_path)
    for name, cls in (("clight_stats", G.Stats), ("clight_params", G.Params), ("clight_atmosphere", G.Atmosphere),
                      ("clight_tune", G.Tune), ("clight_pipe_rates", G.PipeRates)):
        assert got[(name, "size")] == C.sizeof(cls), name
        for f, _ in cls._fields_:
            assert got[(name, f)] == getattr(cls, f).offset, (name, f)
    assert got[("clight_segment", "size")] == I.SEG_DTYPE.itemsize
    for f in I.SEG_DTYPE.names:
        assert got[("clight_segment", f)] == I.SEG_DTYPE.fields[f][1], f
    assert got[("clight_hit", "size")] == G.HIT_DTYPE.itemsize
    for f in G.HIT_DTYPE.names:
        assert got[("clight_hit", f)] == G.HIT_DTYPE.fields[f][1], f

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
    assert ctypes.sizeof(G.Stats) == 96
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

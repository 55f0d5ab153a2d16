"""GB300 library for Cherenkov / fluorescence light generation and
atmospheric propagation to telescopes (Baack & Alameddine, ICRC 2023).

Thin ctypes binding over the C ABI in ``include/clight.h``: argument
marshalling only.  Every step of the computation runs in the CUDA kernels of
``libclight.so``; there is no CPU fallback, and loading fails loudly when the
library has not been built.  PyTorch supplies device memory and streams.
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

from . import inputs

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libclight.so")

HIT_DTYPE = np.dtype([
    ("seg", "<i8"), ("k", "<u4"), ("tel", "<u4"),
    ("x_rel", "<f4"), ("y_rel", "<f4"), ("cx", "<f4"), ("cy", "<f4"),
    ("lambda", "<f4"), ("weight", "<f4"), ("t", "<f8"),
])
assert HIT_DTYPE.itemsize == 48

STATUS = {0: "ok", 1: "invalid argument", 2: "CUDA runtime error", 3: "hit capacity exceeded",
          4: "invalid segment", 5: "limit exceeded", 6: "no usable CUDA device"}
OK, ERR_ARG, ERR_CUDA, ERR_HIT_CAPACITY, ERR_BAD_SEGMENT, ERR_LIMIT, ERR_NO_DEVICE = range(7)
PROP_EXACT, PROP_STRAIGHT = 0, 1
PREC_FLOAT_PAIR, PREC_FP64_GUARD = 0, 1


class ClightError(RuntimeError):
    def __init__(self, code, where=""):
        super().__init__(f"{where}: {STATUS.get(code, code)} ({code})")
        self.code = code


class Atmosphere(C.Structure):
    _fields_ = [("n_layers", C.c_int32), ("spherical", C.c_int32),
                ("h_lo", C.c_double * 8), ("b", C.c_double * 8), ("c", C.c_double * 8),
                ("h_top", C.c_double), ("K", C.c_double), ("rho_ref", C.c_double),
                ("L0", C.c_double), ("lambda_ref", C.c_double), ("R_E", C.c_double),
                ("h_obs", C.c_double), ("refraction", C.c_int32), ("absorption", C.c_int32),
                ("disp_B", C.c_double), ("disp_lref", C.c_double)]


class Params(C.Structure):
    _fields_ = [("lambda1", C.c_double), ("lambda2", C.c_double), ("bunch", C.c_double),
                ("seed", C.c_uint32), ("stream", C.c_uint32), ("fluor_yield", C.c_double),
                ("fl_lambda1", C.c_double), ("fl_lambda2", C.c_double), ("seg_base", C.c_int64),
                ("precision", C.c_int32), ("block", C.c_int32), ("ctas_per_sm", C.c_int32),
                ("use_graph", C.c_int32), ("cell_width", C.c_float), ("key_bunch_bits", C.c_int32),
                ("cut_mode", C.c_int32), ("cut_pad", C.c_int32), ("cut_deg", C.c_double),
                ("cut_centre", C.c_double * 3), ("fl_beaming", C.c_int32), ("propagator", C.c_int32),
                ("beam_centre", C.c_double * 3), ("beam_radius", C.c_double), ("fl_roulette", C.c_int32),
                ("roulette_pad", C.c_int32), ("defer_cap", C.c_int64), ("trace_all", C.c_int32),
                ("work_chunk", C.c_int32)]


class Stats(C.Structure):
    _fields_ = [(n, C.c_int64) for n in
                ("rays", "escaped", "under", "turned", "reached", "hits", "guarded", "status", "cells", "cut",
                 "skipped", "deferred", "step_skipped")]

    def as_dict(self):
        return {n: getattr(self, n) for n, _ in self._fields_}


class PipeRates(C.Structure):
    _fields_ = [(n, C.c_double) for n in ("ffma_per_s", "mufu_ex2_per_s", "dfma_per_s", "imad_per_s", "lop3_per_s",
                                          "ffma_mhz", "mufu_mhz", "dfma_mhz", "imad_mhz", "lop3_mhz")] + \
               [("n_sm", C.c_int32), ("pad", C.c_int32)]

    def as_dict(self):
        return {n: getattr(self, n) for n, _ in self._fields_ if n != "pad"}


class Tune(C.Structure):
    _fields_ = [("block", C.c_int32), ("ctas_per_sm", C.c_int32), ("cell_width", C.c_float),
                ("work_chunk", C.c_int32), ("bunch", C.c_double), ("best_ms", C.c_double),
                ("default_ms", C.c_double), ("n_tried", C.c_int32), ("pad", C.c_int32), ("n_sample", C.c_int64)]

    def as_dict(self):
        return {n: getattr(self, n) for n, _ in self._fields_ if not n.startswith("pad")}


_lib = None


def lib():
    """The loaded CUDA library; raises if it has not been built."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise RuntimeError(f"{LIB_PATH} is missing: run paper_2309_15861_gb300.build.build() "
                               "(there is no CPU fallback)")
        L = C.CDLL(LIB_PATH)
        P = C.c_void_p
        L.clight_create.argtypes = [C.POINTER(P), C.c_int]
        L.clight_destroy.argtypes = [P]
        L.clight_destroy.restype = None
        L.clight_set_atmosphere.argtypes = [P, C.POINTER(Atmosphere)]
        L.clight_set_telescopes.argtypes = [P, P, C.c_int32]
        L.clight_set_params.argtypes = [P, C.POINTER(Params)]
        for fn in (L.clight_trace, L.clight_trace_fp64, L.clight_trace_host):
            fn.argtypes = [P, P, C.c_int64, C.c_int32, P, C.c_int64, P, P, C.POINTER(Stats),
                           C.POINTER(C.c_int64), P]
        L.clight_status_string.argtypes = [C.c_int]
        L.clight_status_string.restype = C.c_char_p
        L.clight_version.restype = C.c_int
        L.clight_last_timing.argtypes = [P, P]
        L.clight_trace_adjoint.argtypes = [P, P, C.c_int64, C.c_int32, P, C.c_int64, P, P, P, P,
                                           C.c_float, C.c_float, P, P, P]
        L.clight_autotune.argtypes = [P, P, C.c_int64, C.c_int64, C.c_int32, P, C.c_int64, C.c_double, C.c_int32,
                                      C.POINTER(Tune), P]
        L.clight_trace_noalloc.argtypes = [P, P, C.c_int64, C.c_int32, P, C.c_int64, P,
                                           C.POINTER(Stats), C.POINTER(C.c_int64), P]
        L.clight_measure_pipes.argtypes = [C.c_int, C.POINTER(PipeRates)]
        L.clight_last_adjoint.argtypes = [P, C.POINTER(C.c_int64), C.POINTER(C.c_int64), P]
        _lib = L
    return _lib


def atmosphere_struct(a: inputs.Atmosphere) -> Atmosphere:
    s = Atmosphere()
    s.n_layers = a.n_layers
    s.spherical = int(a.spherical)
    for i in range(a.n_layers):
        s.h_lo[i], s.b[i], s.c[i] = a.h_lo[i], a.b[i], a.c[i]
    s.h_top, s.K, s.rho_ref = a.h_top, a.K, a.rho_ref
    s.L0, s.lambda_ref, s.R_E, s.h_obs = a.L0, a.lambda_ref, a.R_E, a.h_obs
    s.refraction, s.absorption = int(a.refraction), int(a.absorption)
    s.disp_B, s.disp_lref = float(getattr(a, "disp_B", 0.0)), float(getattr(a, "disp_lref", 400.0))
    return s


def params_struct(p: inputs.Params, **kw) -> Params:
    s = Params()
    s.lambda1, s.lambda2, s.bunch = p.lambda1, p.lambda2, p.bunch
    s.seed, s.stream = p.seed & 0xFFFFFFFF, p.stream & 0xFFFFFFFF
    s.fluor_yield, s.fl_lambda1, s.fl_lambda2 = p.fluor_yield, p.fl_lambda1, p.fl_lambda2
    s.cut_mode = int(getattr(p, "cut_mode", 0))
    s.cut_deg = float(getattr(p, "cut_deg", 6.0))
    if s.cut_mode == 1:
        if p.cut_centre is None:
            raise ValueError("the centre cut needs Params.cut_centre")
        for i in range(3):
            s.cut_centre[i] = float(p.cut_centre[i])
    if getattr(p, "fl_beaming", 0):
        s.fl_beaming = 1
        for i in range(3):
            s.beam_centre[i] = float(p.beam_centre[i])
        s.beam_radius = float(p.beam_radius)
    s.fl_roulette = int(getattr(p, "fl_roulette", 0))
    for k, v in kw.items():
        setattr(s, k, v)
    return s


def _check(code, where):
    if code != OK:
        raise ClightError(code, where)


def _stream_handle(stream):
    if stream is None:
        import torch
        return C.c_void_p(torch.cuda.current_stream().cuda_stream)
    if isinstance(stream, int):
        return C.c_void_p(stream)
    return C.c_void_p(stream.cuda_stream)


class Context:
    """One library context on one device (owns tables, scratch and graphs)."""

    def __init__(self, device: int = 0):
        self._h = C.c_void_p()
        _check(lib().clight_create(C.byref(self._h), int(device)), "clight_create")
        self.n_tel = 0
        self.params = None

    def close(self):
        if self._h:
            lib().clight_destroy(self._h)
            self._h = C.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def set_atmosphere(self, atm: inputs.Atmosphere):
        s = atmosphere_struct(atm)
        _check(lib().clight_set_atmosphere(self._h, C.byref(s)), "clight_set_atmosphere")

    def set_telescopes(self, tels: np.ndarray):
        t = np.ascontiguousarray(tels, dtype=inputs.TEL_DTYPE)
        _check(lib().clight_set_telescopes(self._h, C.c_void_p(t.ctypes.data), len(t)),
               "clight_set_telescopes")
        self.n_tel = len(t)

    def set_params(self, par: inputs.Params, **kw):
        s = params_struct(par, **kw)
        _check(lib().clight_set_params(self._h, C.byref(s)), "clight_set_params")
        self.params = s

    def setup(self, workload: inputs.Workload, **kw):
        self.set_atmosphere(workload.atmosphere)
        self.set_telescopes(workload.telescopes)
        self.set_params(workload.params, **kw)

    # -- device-buffer entry points ---------------------------------------
    def trace(self, d_segs, n_segs, n_showers, d_hits, capacity, d_counts=None, d_sums=None,
              stream=None, fp64=False, raise_on_error=True):
        """Run the path on device buffers (torch tensors or raw pointers).

        Returns (status, n_hits, stats dict)."""
        fn = lib().clight_trace_fp64 if fp64 else lib().clight_trace
        _need(d_segs, int(n_segs) * 64, "d_segs")
        _need(d_hits, int(capacity) * 48, "d_hits")
        _need(d_counts, int(n_showers) * self.n_tel * 8, "d_counts")
        _need(d_sums, int(n_showers) * self.n_tel * 8, "d_sums")
        st = Stats()
        nh = C.c_int64()
        code = fn(self._h, _ptr(d_segs), int(n_segs), int(n_showers), _ptr(d_hits), int(capacity),
                  _ptr(d_counts), _ptr(d_sums), C.byref(st), C.byref(nh), _stream_handle(stream))
        if raise_on_error and code not in (OK,):
            raise ClightError(code, "clight_trace_fp64" if fp64 else "clight_trace")
        return code, nh.value, st.as_dict()

    def trace_adjoint(self, d_segs, n_segs, n_showers, d_hits, n_hits, gx=None, gy=None, gt=None, gY=None,
                      soft_s=0.5, soft_w=20.0, d_yield=None, stream=None, n_params=None):
        """Gradient of sum(gx x + gy y + gt t) + sum(gY Y) with respect to
        (c_1..c_L, K, L0); optionally the soft-edged yields Y into d_yield."""
        n = n_params if n_params is not None else 10
        out = np.zeros(max(n, 10))
        code = lib().clight_trace_adjoint(self._h, _ptr(d_segs), int(n_segs), int(n_showers), _ptr(d_hits),
                                          int(n_hits), _ptr(gx), _ptr(gy), _ptr(gt), _ptr(gY), float(soft_s),
                                          float(soft_w), _ptr(d_yield), C.c_void_p(out.ctypes.data),
                                          _stream_handle(stream))
        _check(code, "clight_trace_adjoint")
        return out

    def last_adjoint(self):
        """The last trace_adjoint: candidate rays, hits, and device ms of its
        candidate pass, candidate sort and tangent kernels."""
        nc, nh = C.c_int64(), C.c_int64()
        ms = (C.c_float * 3)()
        _check(lib().clight_last_adjoint(self._h, C.byref(nc), C.byref(nh), ms), "clight_last_adjoint")
        return {"candidates": nc.value, "hits": nh.value, "candidate_ms": float(ms[0]), "sort_ms": float(ms[1]),
                "tangent_ms": float(ms[2])}

    def autotune(self, d_segs, n_segs, n_sample, n_showers, d_hits, capacity, bunch_max, reps=5, stream=None):
        """Time bunch sizes, launch shapes, work chunks and cell widths on a sample of n_sample
        steps spread over all n_segs; the context keeps the choice (never slower than the
        defaults by the tuner's own timing).  -> dict of the choice and timings."""
        _need(d_segs, int(n_segs) * 64, "d_segs")
        _need(d_hits, int(capacity) * 48, "d_hits")
        t = Tune()
        code = lib().clight_autotune(self._h, _ptr(d_segs), int(n_segs), int(n_sample), int(n_showers),
                                     _ptr(d_hits), int(capacity), float(bunch_max), int(reps), C.byref(t),
                                     _stream_handle(stream))
        _check(code, "clight_autotune")
        if self.params is not None:
            self.params.block, self.params.ctas_per_sm = t.block, t.ctas_per_sm
            self.params.cell_width, self.params.bunch = t.cell_width, t.bunch
            self.params.work_chunk = t.work_chunk
        return t.as_dict()

    def trace_noalloc(self, d_segs, n_segs, n_showers, d_hits, capacity, d_counts=None, stream=None,
                      raise_on_error=True):
        """The path without any allocation: unsorted hits straight into d_hits,
        per-(shower, telescope) hit counts into d_counts.  For callers that
        cannot allocate device memory while they run.  -> (status, n_hits, stats)"""
        _need(d_segs, int(n_segs) * 64, "d_segs")
        _need(d_hits, int(capacity) * 48, "d_hits")
        _need(d_counts, int(n_showers) * self.n_tel * 8, "d_counts")
        st = Stats()
        nh = C.c_int64()
        code = lib().clight_trace_noalloc(self._h, _ptr(d_segs), int(n_segs), int(n_showers), _ptr(d_hits),
                                          int(capacity), _ptr(d_counts), C.byref(st), C.byref(nh),
                                          _stream_handle(stream))
        if raise_on_error and code != OK:
            raise ClightError(code, "clight_trace_noalloc")
        return code, nh.value, st.as_dict()

    def last_timing(self):
        """(trace-kernel ms, sort+reduce ms) of the last trace call (CUDA events)."""
        ms = (C.c_float * 2)()
        _check(lib().clight_last_timing(self._h, ms), "clight_last_timing")
        return float(ms[0]), float(ms[1])

    def trace_host(self, segs: np.ndarray, n_showers, capacity, stream=None, hits_out=None,
                   counts_out=None, sums_out=None, raise_on_error=True):
        """Run the path on host buffers (copies inside the call)."""
        segs = np.ascontiguousarray(segs)
        hits = hits_out if hits_out is not None else np.zeros(max(capacity, 1), dtype=HIT_DTYPE)
        ng = n_showers * self.n_tel
        counts = counts_out if counts_out is not None else np.zeros(ng, dtype=np.int64)
        sums = sums_out if sums_out is not None else np.zeros(ng, dtype=np.float64)
        st = Stats()
        nh = C.c_int64()
        code = lib().clight_trace_host(self._h, C.c_void_p(segs.ctypes.data), len(segs), int(n_showers),
                                       C.c_void_p(hits.ctypes.data), int(capacity),
                                       C.c_void_p(counts.ctypes.data), C.c_void_p(sums.ctypes.data),
                                       C.byref(st), C.byref(nh), _stream_handle(stream))
        if raise_on_error and code != OK:
            raise ClightError(code, "clight_trace_host")
        n = min(nh.value, capacity)
        return code, hits[:n], counts.reshape(n_showers, self.n_tel), sums.reshape(n_showers, self.n_tel), st.as_dict()


def pipe_rates(device: int = 0) -> dict:
    """Measured FP32-FMA, MUFU, FP64-FMA, integer-multiply and logic
    throughput of the GPU (operations/s) and the SM clock during each probe."""
    r = PipeRates()
    _check(lib().clight_measure_pipes(int(device), C.byref(r)), "clight_measure_pipes")
    return r.as_dict()


def _need(x, nbytes, what):
    """Refuse a torch buffer smaller than the call would read or write
    (raw integer pointers cannot be checked and are the caller's risk)."""
    if x is None or isinstance(x, int) or nbytes <= 0:
        return
    if hasattr(x, "numel") and hasattr(x, "element_size"):
        have = x.numel() * x.element_size()
        if have < nbytes:
            raise ValueError(f"{what}: {have} bytes, the call needs {nbytes}")


def _ptr(x):
    if x is None:
        return C.c_void_p(0)
    if isinstance(x, int):
        return C.c_void_p(x)
    if hasattr(x, "data_ptr"):
        return C.c_void_p(x.data_ptr())
    raise TypeError(f"cannot take a device pointer of {type(x)}")


def hits_from_bytes(buf) -> np.ndarray:
    """Decode a byte buffer (numpy or torch uint8, on host) into HIT_DTYPE records."""
    arr = buf.numpy() if hasattr(buf, "numpy") else np.asarray(buf)
    return arr.view(HIT_DTYPE)


def run_workload(ctx: Context, workload: inputs.Workload, capacity=None, fp64=False, stream=None,
                 device="cuda"):
    """Upload a workload, trace it on the device, return host results.

    -> (hits[HIT_DTYPE], counts, sums, stats)."""
    import torch
    segs = torch.from_numpy(workload.segments.view(np.uint8).reshape(-1)).to(device)
    n = len(workload.segments)
    cap = capacity if capacity is not None else max(1024, n * 4)
    hits = torch.empty(cap * 48, dtype=torch.uint8, device=device)
    ng = workload.n_showers * ctx.n_tel
    counts = torch.zeros(ng, dtype=torch.int64, device=device)
    sums = torch.zeros(ng, dtype=torch.float64, device=device)
    code, nh, st = ctx.trace(segs, n, workload.n_showers, hits, cap, counts, sums, stream=stream,
                             fp64=fp64, raise_on_error=False)
    if code == ERR_HIT_CAPACITY:
        return run_workload(ctx, workload, capacity=nh + 16, fp64=fp64, stream=stream, device=device)
    if code != OK:
        raise ClightError(code, "run_workload")
    h = hits[: nh * 48].cpu().numpy().view(HIT_DTYPE).copy()
    return (h, counts.cpu().numpy().reshape(workload.n_showers, ctx.n_tel),
            sums.cpu().numpy().reshape(workload.n_showers, ctx.n_tel), st)

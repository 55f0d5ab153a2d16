"""Plain FP64 CPU oracle (ctypes wrapper around oracle.c).

TEST INFRASTRUCTURE.  Only the tests, ``__graft_entry__.smoke()`` and the CPU
baseline leg of ``bench.py`` may import this package.  The CUDA library never
calls it and shares no code with it.
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_LIB = os.path.join(_HERE, "liboracle.so")

OR_TRACED, OR_ESCAPED, OR_UNDER, OR_TURNED = 0, 1, 2, 3

HIT_DTYPE = np.dtype([
    ("seg", "<i8"), ("k", "<u4"), ("tel", "<u4"),
    ("x_rel", "<f8"), ("y_rel", "<f8"), ("cx", "<f8"), ("cy", "<f8"),
    ("lambda", "<f8"), ("weight", "<f8"), ("t", "<f8"), ("dperp", "<f8"),
])
assert HIT_DTYPE.itemsize == 80


def build(force: bool = False) -> str:
    """Compile liboracle.so with gcc (plain C, OpenMP)."""
    src = os.path.join(_HERE, "oracle.c")
    if not force and os.path.exists(_LIB) and os.path.getmtime(_LIB) >= max(
            os.path.getmtime(src), os.path.getmtime(os.path.join(_HERE, "oracle.h"))):
        return _LIB
    tmp = _LIB + f".tmp{os.getpid()}"
    # no contraction into FMA: the same binary64 expressions give the same
    # bits on every host (the angular cut's decisions depend on it)
    cmd = ["gcc", "-O2", "-std=gnu11", "-ffp-contract=off", "-fopenmp", "-fPIC", "-shared", src, "-o", tmp, "-lm"]
    subprocess.run(cmd, check=True)
    os.replace(tmp, _LIB)
    return _LIB


class _Atm(C.Structure):
    _fields_ = [("n_layers", C.c_int),
                ("h_lo", C.c_double * 8), ("b", C.c_double * 8), ("c", C.c_double * 8),
                ("h_top", C.c_double), ("K", C.c_double), ("rho_ref", C.c_double),
                ("L0", C.c_double), ("lambda_ref", C.c_double),
                ("R_E", C.c_double), ("h_obs", C.c_double),
                ("spherical", C.c_int), ("refraction", C.c_int), ("absorption", C.c_int),
                ("disp_B", C.c_double), ("disp_lref", C.c_double)]


class _Par(C.Structure):
    _fields_ = [("lambda1", C.c_double), ("lambda2", C.c_double), ("bunch", C.c_double),
                ("seed", C.c_uint32), ("stream", C.c_uint32), ("fluor_yield", C.c_double),
                ("fl_lambda1", C.c_double), ("fl_lambda2", C.c_double),
                ("seg_base", C.c_int64), ("cut_mode", C.c_int32), ("cut_deg", C.c_double),
                ("cut_centre", C.c_double * 3), ("cut_tels", C.c_void_p), ("cut_n_tel", C.c_int32),
                ("fl_beaming", C.c_int32), ("beam_centre", C.c_double * 3), ("beam_radius", C.c_double),
                ("fl_roulette", C.c_int32)]


_lib = None


def lib():
    global _lib
    if _lib is None:
        build()
        L = C.CDLL(_LIB)
        P = C.c_void_p
        L.or_philox4x32_10.argtypes = [P, P, P]
        L.or_u01.argtypes = [C.c_uint32]
        L.or_u01.restype = C.c_double
        L.or_yield.argtypes = [P, P, P, P]
        L.or_yield_at.argtypes = [P, C.c_int64, P, P, P]
        L.or_rotation.argtypes = [P, P]
        L.or_photon.argtypes = [P, C.c_int64, C.c_uint32, P, P, P]
        L.or_propagate.argtypes = [P, P, P, C.c_double, C.c_double, P]
        L.or_delta.argtypes = [P, C.c_double]
        L.or_delta.restype = C.c_double
        L.or_density.argtypes = [P, C.c_double]
        L.or_density.restype = C.c_double
        L.or_disp_g.argtypes = [P, C.c_double]
        L.or_disp_g.restype = C.c_double
        L.or_trace.argtypes = [P, C.c_int64, P, P, C.c_int, P, C.c_int, P, C.c_int64,
                               P, P, P, C.c_int]
        L.or_trace.restype = C.c_int64
        L.or_soft_yield.argtypes = [P, C.c_int64, P, P, P, P, C.c_int, P, C.c_int,
                                    C.c_double, C.c_double, P, C.c_int]
        L.or_eval_rays.argtypes = [P, P, P, P, P, P, C.c_int64, P, P, P, P, C.c_int]
        L.or_grad_rays.argtypes = [P, P, P, P, P, P, C.c_int64, P, P, P, P, P, P, P, P, C.c_int]
        L.or_grad_soft.argtypes = [P, C.c_int64, P, P, P, P, C.c_int, P, C.c_int, C.c_double, C.c_double, P, P,
                                   C.c_int]
        _lib = L
    return _lib


def _ptr(a: np.ndarray):
    return C.c_void_p(0) if a is None else C.c_void_p(a.ctypes.data)


def atm_struct(atm) -> _Atm:
    s = _Atm()
    s.n_layers = atm.n_layers
    for i in range(atm.n_layers):
        s.h_lo[i] = atm.h_lo[i]
        s.b[i] = atm.b[i]
        s.c[i] = atm.c[i]
    s.h_top = atm.h_top
    s.K = atm.K
    s.rho_ref = atm.rho_ref
    s.L0 = atm.L0
    s.lambda_ref = atm.lambda_ref
    s.R_E = atm.R_E
    s.h_obs = atm.h_obs
    s.spherical = int(atm.spherical)
    s.refraction = int(atm.refraction)
    s.absorption = int(atm.absorption)
    s.disp_B = float(getattr(atm, "disp_B", 0.0))
    s.disp_lref = float(getattr(atm, "disp_lref", 400.0))
    return s


def par_struct(p, seg_base: int = 0, tels=None) -> _Par:
    """The C parameter block.  For the per-telescope angular cut `tels` must
    be given and must stay alive while the block is used."""
    s = _Par()
    s.seg_base = int(seg_base)
    s.lambda1, s.lambda2, s.bunch = p.lambda1, p.lambda2, p.bunch
    s.seed, s.stream = p.seed & 0xFFFFFFFF, p.stream & 0xFFFFFFFF
    s.fluor_yield, s.fl_lambda1, s.fl_lambda2 = p.fluor_yield, p.fl_lambda1, p.fl_lambda2
    mode = int(getattr(p, "cut_mode", 0))
    s.cut_mode = mode
    s.cut_deg = float(getattr(p, "cut_deg", 6.0))
    if mode == 1:
        if p.cut_centre is None:
            raise ValueError("the centre cut needs Params.cut_centre")
        for i in range(3):
            s.cut_centre[i] = float(p.cut_centre[i])
    if mode == 2:
        if tels is None:
            raise ValueError("the per-telescope cut needs the telescopes")
        s.cut_tels = tels.ctypes.data
        s.cut_n_tel = len(tels)
    if getattr(p, "fl_beaming", 0):
        s.fl_beaming = 1
        for i in range(3):
            s.beam_centre[i] = float(p.beam_centre[i])
        s.beam_radius = float(p.beam_radius)
    s.fl_roulette = int(getattr(p, "fl_roulette", 0))
    return s


# --------------------------------------------------------------------------
def philox(ctr, key):
    c = np.asarray(ctr, dtype=np.uint32)
    k = np.asarray(key, dtype=np.uint32)
    o = np.zeros(4, dtype=np.uint32)
    lib().or_philox4x32_10(_ptr(c), _ptr(k), _ptr(o))
    return o


def u01(x: int) -> float:
    return lib().or_u01(int(x) & 0xFFFFFFFF)


def yield_of(seg, atm, par, tels=None, seg_index=0):
    """-> dict(n_c, w_c, n_f, w_f, cos_tc, sin_tc, Nc, Nf, delta, h_mid) of the
    step whose global index is seg_index."""
    s = np.ascontiguousarray(np.asarray(seg).reshape(1))
    o = np.zeros(10)
    tels = None if tels is None else np.ascontiguousarray(tels)
    a, p = atm_struct(atm), par_struct(par, 0, tels)
    lib().or_yield_at(_ptr(s), int(seg_index), C.byref(a), C.byref(p), _ptr(o))
    keys = ["n_c", "w_c", "n_f", "w_f", "cos_tc", "sin_tc", "Nc", "Nf", "delta", "h_mid"]
    return dict(zip(keys, o.tolist()))


def rotation(d):
    dd = np.asarray(d, dtype=np.float64)
    M = np.zeros(9)
    lib().or_rotation(_ptr(dd), _ptr(M))
    return M.reshape(3, 3)


def photon(seg, seg_index, k, atm, par, tels=None):
    """-> (r_e[3], d[3], t_e, lambda, weight, process)."""
    s = np.ascontiguousarray(np.asarray(seg).reshape(1))
    o = np.zeros(10)
    tels = None if tels is None else np.ascontiguousarray(tels)
    a, p = atm_struct(atm), par_struct(par, 0, tels)
    lib().or_photon(_ptr(s), int(seg_index), int(k), C.byref(a), C.byref(p), _ptr(o))
    return o[0:3].copy(), o[3:6].copy(), o[6], o[7], o[8], int(o[9])


def propagate(atm, r_e, d, t_e=0.0, lam=400.0):
    """-> dict(status, P, dL, t, tau, n_obs)."""
    r = np.asarray(r_e, dtype=np.float64)
    dd = np.asarray(d, dtype=np.float64)
    o = np.zeros(10)
    a = atm_struct(atm)
    lib().or_propagate(C.byref(a), _ptr(r), _ptr(dd), float(t_e), float(lam), _ptr(o))
    return dict(status=int(o[0]), P=o[1:4].copy(), dL=o[4:7].copy(), t=o[7], tau=o[8], n_obs=o[9])


def disp_g(atm, lam):
    return lib().or_disp_g(C.byref(atm_struct(atm)), float(lam))


def delta(atm, h):
    return lib().or_delta(C.byref(atm_struct(atm)), float(h))


def density(atm, h):
    return lib().or_density(C.byref(atm_struct(atm)), float(h))


def trace(segs, atm, tels, par, n_showers=1, capacity=None, threads=0, seg_base=0):
    """Full oracle trace -> (hits[HIT_DTYPE], counts, sums, stats dict).

    seg_base is the global index of segs[0] (it keys the random numbers)."""
    segs = np.ascontiguousarray(segs)
    tels = np.ascontiguousarray(tels)
    a, p = atm_struct(atm), par_struct(par, seg_base, tels)
    n_tel = len(tels)
    counts = np.zeros(n_showers * n_tel, dtype=np.int64)
    sums = np.zeros(n_showers * n_tel, dtype=np.float64)
    stats = np.zeros(5, dtype=np.int64)
    cap = capacity if capacity is not None else 0
    hits = np.zeros(max(cap, 1), dtype=HIT_DTYPE)
    total = lib().or_trace(_ptr(segs), len(segs), C.byref(a), _ptr(tels), n_tel, C.byref(p),
                           n_showers, _ptr(hits), cap, _ptr(counts), _ptr(sums), _ptr(stats),
                           int(threads))
    if capacity is None or total > cap:
        hits = np.zeros(max(total, 1), dtype=HIT_DTYPE)
        total = lib().or_trace(_ptr(segs), len(segs), C.byref(a), _ptr(tels), n_tel,
                               C.byref(p), n_showers, _ptr(hits), total, _ptr(counts),
                               _ptr(sums), _ptr(stats), int(threads))
    st = dict(zip(["rays", "escaped", "under", "turned", "reached"], stats.tolist()))
    return hits[:total], counts.reshape(n_showers, n_tel), sums.reshape(n_showers, n_tel), st


def bunch_counts(segs, atm, par, tels=None, seg_base=0):
    """Nominal Cherenkov and fluorescence bunch counts of every segment
    (`tels` is needed for the per-telescope angular cut, seg_base for the
    fluorescence count rule 1)."""
    nc = np.zeros(len(segs), dtype=np.uint32)
    nf = np.zeros(len(segs), dtype=np.uint32)
    for i in range(len(segs)):
        y = yield_of(segs[i], atm, par, tels, seg_index=seg_base + i)
        nc[i] = int(y["n_c"])
        nf[i] = int(y["n_f"])
    return nc, nf


def soft_yield(segs, nbc, nbf, atm, tels, par, n_showers=1, s=0.5, W=10.0, threads=0, seg_base=0):
    segs = np.ascontiguousarray(segs)
    tels = np.ascontiguousarray(tels)
    nbc = np.ascontiguousarray(nbc, dtype=np.uint32)
    nbf = np.ascontiguousarray(nbf, dtype=np.uint32)
    out = np.zeros(n_showers * len(tels))
    a, p = atm_struct(atm), par_struct(par, seg_base, tels)
    lib().or_soft_yield(_ptr(segs), len(segs), _ptr(nbc), _ptr(nbf), C.byref(a), _ptr(tels),
                        len(tels), C.byref(p), n_showers, float(s), float(W), _ptr(out),
                        int(threads))
    return out.reshape(n_showers, len(tels))


def eval_rays(segs, seg_idx, k, tel, nbc, nbf, atm, tels, par, threads=0, seg_base=0):
    """-> (n, 5) array: x_rel, y_rel, t, weight*exp(-tau), dperp.

    seg_idx indexes segs; seg_base is the global index of segs[0] (it keys
    the random numbers)."""
    segs = np.ascontiguousarray(segs)
    tels = np.ascontiguousarray(tels)
    seg_idx = np.ascontiguousarray(seg_idx, dtype=np.int64)
    k = np.ascontiguousarray(k, dtype=np.uint32)
    tel = np.ascontiguousarray(tel, dtype=np.uint32)
    nbc = np.ascontiguousarray(nbc, dtype=np.uint32)
    nbf = np.ascontiguousarray(nbf, dtype=np.uint32)
    out = np.zeros((len(seg_idx), 5))
    a, p = atm_struct(atm), par_struct(par, seg_base, tels)
    lib().or_eval_rays(_ptr(segs), _ptr(seg_idx), _ptr(k), _ptr(tel), _ptr(nbc), _ptr(nbf),
                       len(seg_idx), C.byref(a), _ptr(tels), C.byref(p), _ptr(out), int(threads))
    return out


def grad_rays(segs, seg_idx, k, tel, nbc, nbf, atm, tels, par, gx=None, gy=None, gt=None, gw=None,
              threads=0, seg_base=0):
    """FP64 gradient (dual numbers) of sum gx x_rel + gy y_rel + gt t + gw weight*exp(-tau)
    over the given hits with respect to (c_1..c_L, K, L0)."""
    segs = np.ascontiguousarray(segs)
    tels = np.ascontiguousarray(tels)
    seg_idx = np.ascontiguousarray(seg_idx, dtype=np.int64)
    k = np.ascontiguousarray(k, dtype=np.uint32)
    tel = np.ascontiguousarray(tel, dtype=np.uint32)
    nbc = np.ascontiguousarray(nbc, dtype=np.uint32)
    nbf = np.ascontiguousarray(nbf, dtype=np.uint32)
    f = lambda v: None if v is None else np.ascontiguousarray(v, dtype=np.float64)
    gx, gy, gt, gw = f(gx), f(gy), f(gt), f(gw)
    out = np.zeros(atm.n_layers + 2)
    a, p = atm_struct(atm), par_struct(par, seg_base, tels)
    lib().or_grad_rays(_ptr(segs), _ptr(seg_idx), _ptr(k), _ptr(tel), _ptr(nbc), _ptr(nbf), len(seg_idx),
                       C.byref(a), _ptr(tels), C.byref(p), _ptr(gx), _ptr(gy), _ptr(gt), _ptr(gw), _ptr(out),
                       int(threads))
    return out


def grad_soft(segs, nbc, nbf, atm, tels, par, gY, n_showers=1, s=0.5, W=10.0, threads=0, seg_base=0):
    """FP64 gradient (dual numbers) of sum gY Y of the soft yield."""
    segs = np.ascontiguousarray(segs)
    tels = np.ascontiguousarray(tels)
    nbc = np.ascontiguousarray(nbc, dtype=np.uint32)
    nbf = np.ascontiguousarray(nbf, dtype=np.uint32)
    gY = np.ascontiguousarray(gY, dtype=np.float64).reshape(-1)
    out = np.zeros(atm.n_layers + 2)
    a, p = atm_struct(atm), par_struct(par, seg_base, tels)
    lib().or_grad_soft(_ptr(segs), len(segs), _ptr(nbc), _ptr(nbf), C.byref(a), _ptr(tels), len(tels),
                       C.byref(p), int(n_showers), float(s), float(W), _ptr(gY), _ptr(out), int(threads))
    return out

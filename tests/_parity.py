"""Element-by-element comparison of CUDA hits with oracle hits.

Tolerances (from the path's stated accuracy):
  x_rel, y_rel   1 cm
  t              0.01 ns
  weight         2e-5 relative (near the Cherenkov threshold, where binary32
                 would lose kappa/2 of its digits in beta n - 1, kappa =
                 (delta + eps)/(beta n - 1), the kernels compute the
                 refractivity in FP32 pairs from kappa = 16 on)
  lambda         2e-6 relative
  cx, cy         2e-6 absolute
A hit whose impact parameter lies within 1 cm of the aperture edge may be
present on one side only; such hits are listed and excluded from the count
comparison.
"""
import json
import os

import numpy as np

TOL_XY = 0.01
TOL_T = 0.01
TOL_W = 2e-5
TOL_LAM = 2e-6
TOL_DIR = 2e-6
EDGE = 0.01


def _key(h):
    return h["seg"].astype(np.int64) * (1 << 24) * 4096 + h["k"].astype(np.int64) * 4096 + h["tel"].astype(np.int64)


def weight_tolerance(segs, ref, atm, par, seg_base=0):
    """Per-hit weight tolerance of the oracle hits: the fixed bound TOL_W for
    every hit (the arguments are kept for the callers)."""
    return np.full(len(ref), TOL_W)


def compare(gpu, ref, tels, edge=EDGE, tol_xy=TOL_XY, tol_t=TOL_T, ref_dperp_of=None, w_tol=None):
    """Return a report dict; raise AssertionError on any violation.

    gpu: HIT_DTYPE (binary32 fields) records; ref: oracle records (FP64).
    ref_dperp_of(missing_gpu_hits) -> impact parameters from the oracle for
    hits only the GPU found (to check they are edge cases)."""
    kg, kr = _key(gpu), _key(ref)
    assert len(np.unique(kg)) == len(kg), "duplicate GPU hits"
    common, ig, ir = np.intersect1d(kg, kr, return_indices=True)
    only_ref = np.setdiff1d(np.arange(len(ref)), ir)
    only_gpu = np.setdiff1d(np.arange(len(gpu)), ig)
    R = tels["R"].astype(np.float64)
    # hits only the oracle has must sit at the aperture edge
    if len(only_ref):
        d = ref["dperp"][only_ref] - R[ref["tel"][only_ref]]
        bad = np.abs(d) >= edge
        assert not bad.any(), f"{bad.sum()} oracle hits missing on GPU away from the edge: {ref[only_ref][bad][:5]}"
    if len(only_gpu):
        assert ref_dperp_of is not None, f"{len(only_gpu)} GPU-only hits and no way to check them"
        dp = ref_dperp_of(gpu[only_gpu])
        d = dp - R[gpu["tel"][only_gpu]]
        bad = np.abs(d) >= edge
        assert not bad.any(), f"{bad.sum()} GPU-only hits away from the edge: {gpu[only_gpu][bad][:5]} d={d[bad][:5]}"
    g = gpu[ig]
    r = ref[ir]
    ex = np.abs(g["x_rel"] - r["x_rel"])
    ey = np.abs(g["y_rel"] - r["y_rel"])
    et = np.abs(g["t"] - r["t"])
    ew = np.abs(g["weight"] / r["weight"] - 1.0)
    el = np.abs(g["lambda"] / r["lambda"] - 1.0)
    ec = np.maximum(np.abs(g["cx"] - r["cx"]), np.abs(g["cy"] - r["cy"]))
    rep = dict(n_gpu=len(gpu), n_ref=len(ref), n_common=len(common), only_ref=len(only_ref),
               only_gpu=len(only_gpu))
    for name, e in (("x", ex), ("y", ey), ("t", et), ("w", ew), ("lam", el), ("dir", ec)):
        rep[f"max_{name}"] = float(e.max()) if len(e) else 0.0
        rep[f"rms_{name}"] = float(np.sqrt(np.mean(e ** 2))) if len(e) else 0.0
    path = os.environ.get("CLIGHT_PARITY_REPORT")
    if path:
        with open(path, "a") as f:
            f.write(json.dumps({"test": os.environ.get("PYTEST_CURRENT_TEST", "?").split(" ")[0], **rep}) + "\n")
    assert rep["max_x"] < tol_xy and rep["max_y"] < tol_xy, rep
    assert rep["max_t"] < tol_t, rep
    wt = np.full(len(r), TOL_W) if w_tol is None else np.asarray(w_tol)[ir]
    bad = ew >= wt
    assert not bad.any(), (rep, g[bad][:3], r[bad][:3], ew[bad][:3], wt[bad][:3])
    assert rep["max_lam"] < TOL_LAM, rep
    assert rep["max_dir"] < TOL_DIR, rep
    return rep


def compare_counts(gpu_counts, ref_counts, gpu_hits, ref_hits, n_tel, shower_of_seg):
    """Per-(shower, telescope) counts equal after removing one-sided edge hits."""
    kg, kr = _key(gpu_hits), _key(ref_hits)
    only_g = gpu_hits[~np.isin(kg, kr)]
    only_r = ref_hits[~np.isin(kr, kg)]
    adj = np.array(ref_counts, dtype=np.int64).copy()
    for h in only_r:
        adj[shower_of_seg(h["seg"]), h["tel"]] -= 1
    for h in only_g:
        adj[shower_of_seg(h["seg"]), h["tel"]] += 1
    np.testing.assert_array_equal(np.asarray(gpu_counts), adj)

"""Seeded synthetic workloads: track segments, atmospheres, telescope arrays.

This module only *makes inputs*.  It holds none of the light-generation or
propagation arithmetic; both the CUDA library and the CPU oracle consume what
it returns, byte for byte.

The paper's own showers come from CORSIKA 7/8 runs (Sec. 3), which are not
available; these generators stand in for them with the shapes the paper's
workloads have: electron track steps of a few metres (Sec. 1.2), emitted along
a Gaisser-Hillas longitudinal profile of a gamma shower, with angular and
lateral spread, in a layered exponential atmosphere.

Record layouts (little endian, shared by every consumer as a *format*):

segment (64 B)::

    double x, y, z      start of the step, local frame, metres (z up,
                        origin at sea level below the array centre)
    double t0           time at the start of the step, ns
    float  dx, dy, dz   direction of flight (unit vector)
    float  L            step length, m
    float  eps          1 - beta of the charged particle
    float  dE           energy deposited over the step, MeV (fluorescence)
    int32  charge       charge number z
    uint32 shower       shower index

telescope (16 B)::  float x, y, z, R   sphere centre and radius, m
"""
from __future__ import annotations

import dataclasses
import math

import numpy as np

SEG_DTYPE = np.dtype([
    ("x", "<f8"), ("y", "<f8"), ("z", "<f8"), ("t0", "<f8"),
    ("dx", "<f4"), ("dy", "<f4"), ("dz", "<f4"), ("L", "<f4"),
    ("eps", "<f4"), ("dE", "<f4"), ("charge", "<i4"), ("shower", "<u4"),
])
assert SEG_DTYPE.itemsize == 64

TEL_DTYPE = np.dtype([("x", "<f4"), ("y", "<f4"), ("z", "<f4"), ("R", "<f4")])
assert TEL_DTYPE.itemsize == 16

C_M_PER_NS = 0.299792458          # speed of light, m/ns
M_E_MEV = 0.51099895069           # electron mass, MeV
RHO_SEA = 1.225e-3                # sea-level density used to normalise, g/cm^3
DELTA_SEA = 2.9e-4                # n - 1 at sea level


@dataclasses.dataclass
class Atmosphere:
    """Layered exponential atmosphere rho_i(h) = b_i / c_i * exp(-h / c_i).

    b_i in g/cm^2, c_i and h in metres, so rho = b_i / (100 c_i) e^{-h/c_i}
    in g/cm^3.  n - 1 = K rho.  Layer i covers [h_lo[i], h_lo[i+1]); the last
    layer ends at h_top, above which rho = 0.  a_i (the thickness offsets,
    T(h) = a_i + b_i e^{-h/c_i}) are only used to synthesise shower depths.
    """
    h_lo: list
    b: list
    c: list
    a: list
    h_top: float
    K: float
    rho_ref: float = RHO_SEA
    L0: float = 20000.0          # extinction length at lambda_ref, m
    lambda_ref: float = 400.0    # nm
    spherical: bool = True
    R_E: float = 6371000.0
    h_obs: float = 2000.0
    refraction: bool = True
    absorption: bool = True
    disp_B: float = 0.0          # dispersion: n - 1 = delta(h) (1 + B/l^2)/(1 + B/l_d^2); 0 = none
    disp_lref: float = 400.0     # nm, the wavelength at which delta(h) holds

    @property
    def n_layers(self) -> int:
        return len(self.h_lo)

    # ---- helpers for input synthesis only -------------------------------
    def _layer(self, h):
        h = np.asarray(h, dtype=np.float64)
        idx = np.searchsorted(np.asarray(self.h_lo), h, side="right") - 1
        return np.clip(idx, 0, self.n_layers - 1)

    def density(self, h):
        """rho(h) in g/cm^3 (used to give synthetic steps their dE)."""
        h = np.asarray(h, dtype=np.float64)
        i = self._layer(h)
        b = np.asarray(self.b)[i]
        c = np.asarray(self.c)[i]
        rho = b / (100.0 * c) * np.exp(-h / c)
        return np.where(h >= self.h_top, 0.0, rho)

    def thickness(self, h):
        """Vertical thickness T(h) above altitude h, g/cm^2."""
        h = np.asarray(h, dtype=np.float64)
        i = self._layer(h)
        a = np.asarray(self.a)[i]
        b = np.asarray(self.b)[i]
        c = np.asarray(self.c)[i]
        return np.where(h >= self.h_top, 0.0, a + b * np.exp(-h / c))

    def altitude_of_thickness(self, T):
        """Inverse of thickness() (per layer, closed form)."""
        T = np.asarray(T, dtype=np.float64)
        edges = np.append(np.asarray(self.h_lo[1:], dtype=np.float64), self.h_top)
        Tb = self.thickness(edges - 1e-9)     # thickness at each layer's top
        i = np.searchsorted(-Tb, -T, side="left")
        i = np.clip(i, 0, self.n_layers - 1)
        a = np.asarray(self.a)[i]
        b = np.asarray(self.b)[i]
        c = np.asarray(self.c)[i]
        arg = np.clip((T - a) / b, 1e-300, None)
        return -c * np.log(arg)


def atmosphere_layered(spherical=True, h_obs=2000.0, refraction=True,
                       absorption=True) -> Atmosphere:
    """Synthetic, stated 5-layer parameter set.

    Lower edges 0, 4, 10, 40, 100 km and top of atmosphere 120 km; scale
    heights 9.9, 8.8, 6.4, 7.7, 7.0 km; b_i fixed by rho(0) = 1.225e-3 g/cm^3
    and continuity of rho at every edge; a_i by continuity of T and
    T(h_top) = 0; K by n(0) - 1 = 2.9e-4.
    """
    h_lo = [0.0, 4000.0, 10000.0, 40000.0, 100000.0]
    c = [9900.0, 8800.0, 6400.0, 7700.0, 7000.0]
    h_top = 120000.0
    b = [RHO_SEA * 100.0 * c[0]]
    for i in range(1, 5):
        rho_edge = b[i - 1] / (100.0 * c[i - 1]) * math.exp(-h_lo[i] / c[i - 1])
        b.append(rho_edge * 100.0 * c[i] * math.exp(h_lo[i] / c[i]))
    a = [0.0] * 5
    a[4] = -b[4] * math.exp(-h_top / c[4])
    for i in range(3, -1, -1):
        T_edge = a[i + 1] + b[i + 1] * math.exp(-h_lo[i + 1] / c[i + 1])
        a[i] = T_edge - b[i] * math.exp(-h_lo[i + 1] / c[i])
    return Atmosphere(h_lo=h_lo, b=b, c=c, a=a, h_top=h_top,
                      K=DELTA_SEA / RHO_SEA, spherical=spherical, h_obs=h_obs,
                      refraction=refraction, absorption=absorption)


def atmosphere_single_exponential(H=8400.0, h_obs=2000.0, spherical=False,
                                  refraction=True, absorption=False) -> Atmosphere:
    """n - 1 = 2.9e-4 exp(-h / H) as one layer with an unreachable top."""
    b = RHO_SEA * 100.0 * H
    return Atmosphere(h_lo=[0.0], b=[b], c=[H], a=[0.0], h_top=1.0e6,
                      K=DELTA_SEA / RHO_SEA, spherical=spherical, h_obs=h_obs,
                      refraction=refraction, absorption=absorption)


@dataclasses.dataclass
class Params:
    lambda1: float = 300.0        # nm, Cherenkov band
    lambda2: float = 600.0
    bunch: float = 1.0            # maximum photons per bunch
    seed: int = 1
    stream: int = 0
    fluor_yield: float = 0.0      # photons per MeV deposited
    fl_lambda1: float = 340.0     # nm, fluorescence band
    fl_lambda2: float = 450.0
    cut_mode: int = 0             # Cherenkov angular cut: 0 off, 1 array centre, 2 each telescope
    cut_deg: float = 6.0          # cut angle, degrees
    cut_centre: tuple = None      # array centre for cut_mode 1 (see array_centre)
    fl_beaming: int = 0           # fluorescence beamed toward the array (see beam_cone)
    beam_centre: tuple = None
    beam_radius: float = None
    fl_roulette: int = 0          # fluorescence steps with N < B: one bunch of weight B with probability N/B


def array_centre(tels: np.ndarray) -> tuple:
    """Mean of the telescope centres (the 'experiment centre' of the angular cut)."""
    return (float(np.mean(tels["x"].astype(np.float64))), float(np.mean(tels["y"].astype(np.float64))),
            float(np.mean(tels["z"].astype(np.float64))))


def beam_cone(tels: np.ndarray) -> tuple:
    """(centre, radius) of the sphere about the mean telescope centre that
    holds every telescope sphere (the target of fluorescence beaming)."""
    c = np.array(array_centre(tels))
    xyz = np.stack([tels["x"], tels["y"], tels["z"]], axis=1).astype(np.float64)
    r = float(np.max(np.linalg.norm(xyz - c[None, :], axis=1) + tels["R"].astype(np.float64)))
    return tuple(float(v) for v in c), r


def telescope_grid(nx, ny, spacing, R=6.0, z=2000.0):
    xs = (np.arange(nx) - (nx - 1) / 2.0) * spacing
    ys = (np.arange(ny) - (ny - 1) / 2.0) * spacing
    X, Y = np.meshgrid(xs, ys, indexing="ij")
    t = np.zeros(nx * ny, dtype=TEL_DTYPE)
    t["x"] = X.ravel()
    t["y"] = Y.ravel()
    t["z"] = z
    t["R"] = R
    return t


def telescopes_c0(z=2000.0):
    t = np.zeros(4, dtype=TEL_DTYPE)
    t["x"] = [100.0, 100.0, -100.0, -100.0]
    t["y"] = [100.0, -100.0, 100.0, -100.0]
    t["z"] = z
    t["R"] = 6.0
    return t


# --------------------------------------------------------------------------
# segment generators
# --------------------------------------------------------------------------
def segments_vertical(n, seed=1, h_range=(5000.0, 20000.0), xy_half=250.0,
                      beta_range=(0.995, 0.99999), L=1.0, charge=-1):
    """Straight vertical 1 m electron steps (the plain FP64 flat-Earth case)."""
    rng = np.random.default_rng(np.random.SeedSequence([seed, 0xC0]))
    s = np.zeros(n, dtype=SEG_DTYPE)
    z = rng.uniform(h_range[0], h_range[1], n)
    s["x"] = rng.uniform(-xy_half, xy_half, n)
    s["y"] = rng.uniform(-xy_half, xy_half, n)
    s["z"] = z
    s["t0"] = (h_range[1] - z) / C_M_PER_NS
    s["dx"] = 0.0
    s["dy"] = 0.0
    s["dz"] = -1.0
    s["L"] = L
    beta = rng.uniform(beta_range[0], beta_range[1], n)
    s["eps"] = (1.0 - beta).astype(np.float32)
    s["dE"] = 0.0
    s["charge"] = charge
    s["shower"] = 0
    return s


def _unit_frame(u):
    """Two unit vectors perpendicular to unit vector u (rows)."""
    u = np.asarray(u, dtype=np.float64)
    ref = np.array([1.0, 0.0, 0.0]) if abs(u[0]) < 0.9 else np.array([0.0, 1.0, 0.0])
    e1 = np.cross(u, ref)
    e1 /= np.linalg.norm(e1)
    e2 = np.cross(u, e1)
    return e1, e2


def segments_shower(n, atm: Atmosphere, seed=1, zenith_deg=0.0, azimuth_deg=0.0,
                    shower=0, core=(0.0, 0.0), Xmax=350.0, lam=70.0,
                    tilt_sigma_deg=5.0, lateral_scale=80.0,
                    E_range_MeV=(10.0, 1000.0), L_range=(0.5, 5.0),
                    dEdX=2.0, t_ref_alt=100000.0, chunk=1 << 22, workers=0):
    """Charged track steps of one gamma shower.

    Depth along the axis X ~ Gamma(k = Xmax/lam + 1, lam) (the Gaisser-Hillas
    profile with X0 = 0), truncated at the observation level; lateral offset
    ~ Exp(lateral_scale); direction tilted from the axis by Gaussian angles of
    tilt_sigma_deg in two perpendicular planes; electron energy log-uniform
    in E_range_MeV; step length uniform in L_range; dE = dEdX * rho * L.
    The geometry of the axis is taken in the local (flat) frame.  Blocks of
    `chunk` steps draw from independent child seeds, so `workers` processes
    give the same array as one.
    """
    spec = _ShowerSpec(atm, seed, zenith_deg, azimuth_deg, shower, core, Xmax, lam, tilt_sigma_deg,
                       lateral_scale, E_range_MeV, L_range, dEdX, t_ref_alt)
    tasks = [(spec, lo, min(chunk, n - lo), i) for i, lo in enumerate(range(0, n, chunk))]
    return _run_tasks(tasks, n, workers)


@dataclasses.dataclass
class _ShowerSpec:
    atm: Atmosphere
    seed: int
    zenith_deg: float
    azimuth_deg: float
    shower: int
    core: tuple
    Xmax: float
    lam: float
    tilt_sigma_deg: float
    lateral_scale: float
    E_range_MeV: tuple
    L_range: tuple
    dEdX: float
    t_ref_alt: float


def _shower_chunk(sp: _ShowerSpec, m: int, index: int) -> np.ndarray:
    """Block `index` (m steps) of a shower; its generator is child `index` of the shower's seed."""
    atm = sp.atm
    out = np.zeros(m, dtype=SEG_DTYPE)
    zen = math.radians(sp.zenith_deg)
    az = math.radians(sp.azimuth_deg)
    u_ax = np.array([math.sin(zen) * math.cos(az), math.sin(zen) * math.sin(az),
                     -math.cos(zen)])
    e1, e2 = _unit_frame(u_ax)
    cosz = math.cos(zen)
    X_obs = float(atm.thickness(np.array([atm.h_obs]))[0]) / cosz
    k = sp.Xmax / sp.lam + 1.0
    core3 = np.array([sp.core[0], sp.core[1], atm.h_obs])
    top_pt = core3 - u_ax * (sp.t_ref_alt - atm.h_obs) / cosz
    rng = np.random.default_rng(np.random.SeedSequence([sp.seed, 0x5E6, sp.shower], spawn_key=(index,)))
    X = rng.gamma(k, sp.lam, m)
    bad = X >= X_obs
    while bad.any():
        X[bad] = rng.gamma(k, sp.lam, int(bad.sum()))
        bad = X >= X_obs
    h = atm.altitude_of_thickness(X * cosz)
    axis_pt = core3[None, :] - u_ax[None, :] * ((h - atm.h_obs) / cosz)[:, None]
    r = rng.exponential(sp.lateral_scale, m)
    phi = rng.uniform(0.0, 2.0 * math.pi, m)
    pos = axis_pt + (r * np.cos(phi))[:, None] * e1[None, :] \
        + (r * np.sin(phi))[:, None] * e2[None, :]
    g1 = np.tan(rng.normal(0.0, math.radians(sp.tilt_sigma_deg), m))
    g2 = np.tan(rng.normal(0.0, math.radians(sp.tilt_sigma_deg), m))
    d = u_ax[None, :] + g1[:, None] * e1[None, :] + g2[:, None] * e2[None, :]
    d /= np.linalg.norm(d, axis=1)[:, None]
    L = rng.uniform(sp.L_range[0], sp.L_range[1], m)
    E = np.exp(rng.uniform(math.log(sp.E_range_MeV[0]), math.log(sp.E_range_MeV[1]), m))
    gam = E / M_E_MEV
    beta = np.sqrt(1.0 - 1.0 / gam ** 2)
    eps = 1.0 / (gam ** 2 * (1.0 + beta))
    charge = np.where(rng.random(m) < 0.5, -1, 1)
    out["x"] = pos[:, 0]
    out["y"] = pos[:, 1]
    out["z"] = pos[:, 2]
    out["t0"] = ((pos - top_pt[None, :]) @ u_ax) / C_M_PER_NS
    out["dx"] = d[:, 0]
    out["dy"] = d[:, 1]
    out["dz"] = d[:, 2]
    out["L"] = L
    out["eps"] = eps
    out["dE"] = sp.dEdX * atm.density(h) * L * 100.0
    out["charge"] = charge
    out["shower"] = sp.shower
    return out


def _chunk_into(args):
    shm_name, n_total, (spec, lo, m, index) = args
    from multiprocessing import shared_memory
    shm = shared_memory.SharedMemory(name=shm_name)
    try:
        dst = np.ndarray((n_total,), dtype=SEG_DTYPE, buffer=shm.buf)
        dst[lo:lo + m] = _shower_chunk(spec, m, index)
        del dst
    finally:
        shm.close()
    return m


class _SharedArray(np.ndarray):
    """An ndarray that keeps its shared-memory block mapped."""
    _shm = None

    def __array_finalize__(self, obj):
        if obj is not None:
            self._shm = getattr(obj, "_shm", None)


def _run_tasks(tasks, n_total, workers):
    """Fill an n_total array from (spec, lo, m, index) blocks, in this process or in `workers` spawned ones."""
    if workers is None or workers <= 1 or len(tasks) <= 1:
        out = np.zeros(n_total, dtype=SEG_DTYPE)
        for spec, lo, m, index in tasks:
            out[lo:lo + m] = _shower_chunk(spec, m, index)
        return out
    import concurrent.futures as cf
    import multiprocessing as mp
    from multiprocessing import shared_memory
    shm = shared_memory.SharedMemory(create=True, size=max(1, n_total * SEG_DTYPE.itemsize))
    try:
        ctx = mp.get_context("spawn")
        with cf.ProcessPoolExecutor(max_workers=workers, mp_context=ctx) as ex:
            done = sum(ex.map(_chunk_into, [(shm.name, n_total, t) for t in tasks]))
        assert done == n_total
    except BaseException:
        shm.close()
        shm.unlink()
        raise
    shm.unlink()          # the mapping stays valid while this process holds it
    arr = np.ndarray((n_total,), dtype=SEG_DTYPE, buffer=shm.buf).view(_SharedArray)
    arr._shm = shm
    return arr


def default_workers() -> int:
    """Processes for input generation: the host's cores, at most 32."""
    import os
    return max(1, min(32, os.cpu_count() or 1))


# --------------------------------------------------------------------------
# the named workloads
# --------------------------------------------------------------------------
@dataclasses.dataclass
class Workload:
    name: str
    segments: np.ndarray
    atmosphere: Atmosphere
    telescopes: np.ndarray
    params: Params
    n_showers: int = 1
    description: str = ""


def workload_flat_vertical(n=10_000, seed=1):
    """1e4 vertical 1 m steps, single exponential, flat Earth, 4 telescopes."""
    atm = atmosphere_single_exponential()
    return Workload("flat_vertical_1e4", segments_vertical(n, seed=seed), atm,
                    telescopes_c0(atm.h_obs), Params(bunch=1.0, seed=seed),
                    description="vertical 1 m electron steps, h U[5,20] km, "
                                "beta U[0.995,0.99999], flat Earth, no absorption, B=1")


def workload_shower_1tev(n=20_000_000, seed=1, zenith_deg=0.0, telescopes=None,
                         bunch=5.0, name=None, workers=0):
    """One 1 TeV gamma shower, 5 layers, spherical Earth, absorption, B=5."""
    atm = atmosphere_layered()
    tel = telescopes if telescopes is not None else telescope_grid(10, 10, 100.0, z=atm.h_obs)
    segs = segments_shower(n, atm, seed=seed, zenith_deg=zenith_deg, workers=workers)
    nm = name or f"shower_1tev_z{int(zenith_deg)}_{n:.0e}".replace("+0", "")
    return Workload(nm, segs, atm, tel, Params(bunch=bunch, seed=seed),
                    description=f"1 TeV gamma shower, zenith {zenith_deg} deg, {n} steps, "
                                f"{len(tel)} telescopes, B={bunch}")


def workload_inclined(n=100_000_000, seed=1, workers=0):
    """Zenith 60 deg, 21 x 21 telescopes on a 400 m square at 20 m spacing."""
    atm = atmosphere_layered()
    return workload_shower_1tev(n, seed=seed, zenith_deg=60.0,
                                telescopes=telescope_grid(21, 21, 20.0, z=atm.h_obs),
                                name=f"shower_1tev_z60_{n:.0e}".replace("+0", ""), workers=workers)


def batch_showers(n_showers=256, seed=1, segs_per_10gev=20_000,
                  E_range_GeV=(10.0, 10_000.0), zen_max_deg=45.0, scale=1.0,
                  fluor_yield=5.0, bunch=5.0, workers=0):
    """Many showers with uneven sizes plus fluorescence (yield per MeV)."""
    atm = atmosphere_layered()
    rng = np.random.default_rng(np.random.SeedSequence([seed, 0xBA7]))
    E = np.exp(rng.uniform(math.log(E_range_GeV[0]), math.log(E_range_GeV[1]), n_showers))
    zen = rng.uniform(0.0, zen_max_deg, n_showers)
    az = rng.uniform(0.0, 360.0, n_showers)
    counts = np.maximum(1, np.round(segs_per_10gev * E / 10.0 * scale)).astype(np.int64)
    chunk = 1 << 22
    tasks, lo = [], 0
    for i in range(n_showers):
        spec = _ShowerSpec(atm, seed, float(zen[i]), float(az[i]), i, (0.0, 0.0), 350.0, 70.0, 5.0, 80.0,
                           (10.0, 1000.0), (0.5, 5.0), 2.0, 100000.0)
        n_i = int(counts[i])
        for j, a in enumerate(range(0, n_i, chunk)):
            tasks.append((spec, lo + a, min(chunk, n_i - a), j))
        lo += n_i
    segs = _run_tasks(tasks, lo, workers)
    tel = telescope_grid(10, 10, 100.0, z=atm.h_obs)
    return Workload(f"batch_{n_showers}_showers", segs, atm, tel,
                    Params(bunch=bunch, seed=seed, fluor_yield=fluor_yield),
                    n_showers=n_showers,
                    description=f"{n_showers} showers, E log-U{E_range_GeV} GeV, "
                                f"zenith U[0,{zen_max_deg}], fluorescence {fluor_yield}/MeV")


def shower_offsets(segs: np.ndarray, n_showers: int) -> np.ndarray:
    """First segment index of every shower (segments grouped by shower)."""
    return np.searchsorted(segs["shower"], np.arange(n_showers + 1)).astype(np.int64)

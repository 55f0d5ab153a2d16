"""The bound behind the kernel's quadrature skip, checked against the exact
FP64 oracle on the CPU.

The kernel skips the refraction quadrature for a ray whose vacuum crossing
of the plane z = h_obs lies farther from every telescope centre than the
hit test's search radius plus a bound on how far refraction can move that
crossing.  With mu the smaller of the vacuum line's zenith cosine at its
landing point on the observation sphere and its global |d_z|, s the sine
that goes with it and delta_max the largest refractivity above h_obs:

  |X_refracted - X_vacuum| <= s delta_max (h_e - h_obs + zeta) / mu^3
  angle(arrival direction, d) <= s delta_max / mu

(zeta = rho^2 / r_obs bounds the depth of the sphere below the plane).
The kernel adds a factor 1.25 and 5 cm on top; here the bare bound must
hold on every ray the oracle lands, also for an atmosphere whose
refractivity jumps upward at a layer edge.
"""
import dataclasses
import math

import numpy as np
import pytest

import oracle as O
from paper_2309_15861_gb300 import inputs as I


def _delta_max(atm):
    hs = np.concatenate([np.linspace(atm.h_obs, atm.h_top, 20001), np.asarray(atm.h_lo, float) + 1e-6])
    hs = hs[(hs >= atm.h_obs) & (hs < atm.h_top)]
    return max(O.delta(atm, float(h)) for h in hs)


def _vacuum(atm, r, d):
    """Crossing of the plane z = h_obs and the zenith cosine at the sphere landing."""
    t = (r[2] - atm.h_obs) / -d[2]
    X = r + t * d
    if not atm.spherical:
        return X, -d[2]
    c = np.array([0.0, 0.0, -atm.R_E])
    r_obs = atm.R_E + atm.h_obs
    R0 = r - c
    b = -(d @ R0)
    disc = b * b - (R0 @ R0 - r_obs * r_obs)
    if disc <= 0:
        return X, None
    s = b - math.sqrt(disc)
    L = R0 + s * d
    return X, -(d @ L) / r_obs


def _atmospheres():
    a1 = I.atmosphere_layered(spherical=True)
    a2 = I.atmosphere_layered(spherical=False)
    a3 = I.atmosphere_layered(spherical=True)
    b = list(a3.b)
    b[2] *= 1.15                        # refractivity jumps up at 10 km
    a3 = dataclasses.replace(a3, b=b)
    return [a1, a2, a3]


@pytest.mark.parametrize("ai", [0, 1, 2])
def test_refraction_moves_the_plane_crossing_less_than_the_bound(ai):
    atm = _atmospheres()[ai]
    dmax = _delta_max(atm)
    rng = np.random.default_rng(100 + ai)
    worst_x = worst_a = 0.0
    n_landed = 0
    for _ in range(3000):
        h = rng.uniform(atm.h_obs + 50.0, 30000.0)
        r = np.array([rng.uniform(-20000, 20000), rng.uniform(-20000, 20000), h])
        th = math.radians(rng.uniform(0.0, 85.0))
        ph = rng.uniform(0, 2 * math.pi)
        d = np.array([math.sin(th) * math.cos(ph), math.sin(th) * math.sin(ph), -math.cos(th)])
        res = O.propagate(atm, r, d)
        if res["status"] != 0:
            continue
        Xv, cos_obs = _vacuum(atm, r, d)
        if cos_obs is None:
            continue
        mu = min(cos_obs, -d[2])
        s = math.sqrt(max(0.0, 1.0 - mu * mu))
        P, dL = res["P"], res["dL"]
        t = (atm.h_obs - P[2]) / dL[2]
        X = P + t * dL
        zeta = (Xv[0] ** 2 + Xv[1] ** 2) / (atm.R_E + atm.h_obs) if atm.spherical else 0.0
        he = h if not atm.spherical else (np.linalg.norm(r - [0, 0, -atm.R_E]) - atm.R_E)
        bound = s * dmax * (he - atm.h_obs + zeta) / mu ** 3
        moved = math.hypot(X[0] - Xv[0], X[1] - Xv[1])
        assert moved <= bound + 1e-6, (r, d, moved, bound)
        ang = math.acos(min(1.0, float(dL @ d) / np.linalg.norm(dL)))
        assert ang <= s * dmax / mu + 1e-9, (r, d, ang, s * dmax / mu)
        worst_x = max(worst_x, moved / (bound + 1e-12))
        worst_a = max(worst_a, ang / (s * dmax / mu + 1e-15))
        n_landed += 1
    assert n_landed > 1500
    # the bound is not vacuous: it is within a small factor of the worst case
    print("worst fraction of the bound: crossing %.3f, angle %.3f" % (worst_x, worst_a))
    assert worst_x > 0.2 and worst_a > 0.2, (worst_x, worst_a)


def test_dispersion_cone_angles_stay_within_the_band_spread():
    """With dispersion the first pass builds each Cherenkov photon's cone at
    the middle of its step's band and widens its margins by the band's
    spread of cone angles, asin(sin theta(u_hi)) - asin(sin theta(u_lo)).
    That holds because every photon leaves at an angle between the band
    edges' (n grows with u = 1/lambda): checked on the oracle's photons."""
    atm = I.atmosphere_layered()
    atm.disp_B = 20000.0
    atm.disp_lref = 400.0
    par = I.Params(bunch=1.0, seed=5)
    rng = np.random.default_rng(7)
    checked = 0
    for i in range(40):
        s = np.zeros(1, dtype=I.SEG_DTYPE)[0]
        s["z"] = rng.uniform(3000.0, 15000.0)
        s["dz"] = -1.0
        s["L"] = 2.0
        s["charge"] = -1
        d0 = O.yield_of(s, atm, I.Params())["delta"]
        s["eps"] = d0 * rng.uniform(0.2, 1.05)      # some steps with the threshold inside the band
        y = O.yield_of(s, atm, par, seg_index=i)
        if y["n_c"] < 1:
            continue
        delta, beta = y["delta"], 1.0 - float(s["eps"])

        def theta(lam):
            return math.acos(min(1.0, 1.0 / (beta * (1.0 + delta * O.disp_g(atm, lam)))))
        lo, hi = theta(par.lambda2), theta(par.lambda1)       # longest wavelength: smallest angle
        for k in range(int(y["n_c"])):
            r, d, te, lam, w, proc = O.photon(s, i, k, atm, par)
            th = math.acos(min(1.0, -d[2]))
            assert lo - 1e-12 <= th <= hi + 1e-12, (i, k, lam, th, lo, hi)
            checked += 1
    assert checked > 200

"""Pins of the FP64 oracle against facts fixed outside it.

Each test checks the oracle against something other than its own formulas:
an independent library (cuRAND's host Philox, scipy constants and
quadrature), a closed form, a brute-force ray tracer of the eikonal
equation, an invariant, or a geometric brute force.  Each is chosen so that a
plausible slip (a dropped factor, a wrong sign, a transposed operand) fails.
"""
import ctypes
import dataclasses
import math
import os

import numpy as np
import pytest
import scipy.constants as SC
from scipy import integrate, stats

import oracle as O
from paper_2309_15861_gb300 import inputs as I
from tests import _eikonal

C_M_NS = SC.c * 1e-9


# ---------------------------------------------------------------- Philox
def _curand_host():
    for path in ("/usr/local/cuda/lib64/libcurand.so", "libcurand.so", "libcurand.so.10"):
        try:
            return ctypes.CDLL(path)
        except OSError:
            continue
    return None


@pytest.mark.parametrize("seed", [1, 0xDEADBEEF, 0x123456789ABCDEF])
def test_philox_matches_curand_host_generator(seed):
    """cuRAND's host PHILOX4_32_10 generator emits block j of its stream from
    counter (0, 0, j, 0) and key (seed lo, seed hi); the oracle's Philox must
    reproduce that stream bit for bit."""
    cr = _curand_host()
    if cr is None:
        pytest.skip("libcurand not available")
    gen = ctypes.c_void_p()
    assert cr.curandCreateGeneratorHost(ctypes.byref(gen), 161) == 0  # PHILOX4_32_10
    try:
        assert cr.curandSetPseudoRandomGeneratorSeed(gen, ctypes.c_ulonglong(seed)) == 0
        n = 4 * 512
        buf = np.zeros(n, dtype=np.uint32)
        assert cr.curandGenerate(gen, ctypes.c_void_p(buf.ctypes.data), ctypes.c_size_t(n)) == 0
    finally:
        cr.curandDestroyGenerator(gen)
    key = [seed & 0xFFFFFFFF, (seed >> 32) & 0xFFFFFFFF]
    ours = np.concatenate([O.philox([0, 0, j, 0], key) for j in range(n // 4)])
    np.testing.assert_array_equal(ours, buf)


def test_philox_uses_every_counter_word_and_key_word():
    base = O.philox([1, 2, 3, 4], [5, 6])
    for i in range(4):
        c = [1, 2, 3, 4]
        c[i] ^= 1
        assert not np.array_equal(O.philox(c, [5, 6]), base)
    for i in range(2):
        k = [5, 6]
        k[i] ^= 1
        assert not np.array_equal(O.philox([1, 2, 3, 4], k), base)


def test_u01_mapping_is_exact_in_binary32():
    for x in [0, 1, 255, 256, 0x7FFFFFFF, 0xFFFFFFFF, 0x12345678]:
        u = O.u01(x)
        assert 0.0 < u < 1.0
        assert float(np.float32(u)) == u
        assert u == ((x >> 9) + 0.5) / 2 ** 23


# ---------------------------------------------------------------- yield
def _one_seg(eps=1e-5, z=10000.0, L=1.0, charge=-1, d=(0.0, 0.0, -1.0), dE=0.0):
    s = np.zeros(1, dtype=I.SEG_DTYPE)
    s["z"] = z
    s["dx"], s["dy"], s["dz"] = d
    s["L"] = L
    s["eps"] = eps
    s["charge"] = charge
    s["dE"] = dE
    return s[0]


def test_frank_tamm_yield_against_codata_prefactor_and_quadrature():
    """N = mu_r pi z^2 e^2 / (h eps0 c0) int dlambda/lambda^2 (1 - 1/(beta n)^2) L
    with CODATA constants from scipy and the wavelength integral done by
    quadrature; catches a wrong prefactor, band factor, charge or length."""
    atm = I.atmosphere_single_exponential()
    par = I.Params(lambda1=300.0, lambda2=600.0, bunch=1.0)
    pref = math.pi * SC.e ** 2 / (SC.h * SC.epsilon_0 * SC.c)
    lam_int, _ = integrate.quad(lambda lam: 1.0 / lam ** 2, 300e-9, 600e-9)
    for charge, L, eps, z in [(-1, 1.0, 1e-5, 10000.0), (2, 3.5, 2e-6, 4000.0),
                              (1, 0.25, 1e-4, 3000.0)]:
        seg = _one_seg(eps=eps, z=z, L=L, charge=charge)
        y = O.yield_of(seg, atm, par)
        h_mid = z - 0.5 * L
        n = 1.0 + 2.9e-4 * math.exp(-h_mid / 8400.0)
        beta = 1.0 - float(np.float32(eps))
        want = pref * charge ** 2 * lam_int * (1.0 - 1.0 / (beta * n) ** 2) * L
        assert y["Nc"] == pytest.approx(want, rel=2e-9)
        assert y["cos_tc"] == pytest.approx(1.0 / (beta * n), rel=1e-14)
        assert y["n_c"] == math.ceil(want)
        assert y["w_c"] * y["n_c"] == pytest.approx(y["Nc"], rel=1e-14)
    # 300-600 nm: 2 pi alpha (1/l1 - 1/l2) = 76417.7 photons/m at sin^2 = 1
    assert 2 * math.pi * SC.alpha * (1 / 300e-9 - 1 / 600e-9) == pytest.approx(76417.7, abs=0.1)


def test_cherenkov_threshold_and_beta_one_limit():
    atm = I.atmosphere_single_exponential()
    par = I.Params(bunch=1.0)
    z = 10000.0
    n = 1.0 + 2.9e-4 * math.exp(-(z - 0.5) / 8400.0)
    eps_thr = 1.0 - 1.0 / n
    below = O.yield_of(_one_seg(eps=float(np.float32(eps_thr * 1.001)), z=z), atm, par)
    above = O.yield_of(_one_seg(eps=float(np.float32(eps_thr * 0.999)), z=z), atm, par)
    assert below["Nc"] == 0.0 and below["n_c"] == 0
    assert above["Nc"] > 0 and above["n_c"] >= 1
    lim = O.yield_of(_one_seg(eps=0.0, z=z), atm, par)
    assert lim["sin_tc"] ** 2 == pytest.approx(1.0 - 1.0 / n ** 2, rel=1e-12)
    assert O.yield_of(_one_seg(charge=0), atm, par)["n_c"] == 0


def test_bunching_and_fluorescence_yield():
    atm = I.atmosphere_layered()
    par = I.Params(bunch=5.0, fluor_yield=5.0)
    seg = _one_seg(eps=1e-5, z=8000.0, L=4.0, dE=1.7)
    y = O.yield_of(seg, atm, par)
    assert y["n_c"] == math.ceil(y["Nc"] / 5.0) and y["w_c"] <= 5.0 + 1e-12
    assert y["Nf"] == pytest.approx(5.0 * float(np.float32(1.7)), rel=1e-15)
    assert y["n_f"] == math.ceil(y["Nf"] / 5.0)
    assert y["w_f"] * y["n_f"] == pytest.approx(y["Nf"], rel=1e-14)


def test_wavelengths_follow_one_over_lambda_squared():
    atm = I.atmosphere_single_exponential()
    par = I.Params(lambda1=300.0, lambda2=600.0, bunch=1.0)
    seg = _one_seg(eps=0.0, z=6000.0, L=20.0)
    nb = int(O.yield_of(seg, atm, par)["n_c"])
    lam = np.array([O.photon(seg, 7, k, atm, par)[3] for k in range(min(nb, 4000))])
    cdf = lambda l: (1 / 300.0 - 1 / l) / (1 / 300.0 - 1 / 600.0)
    assert stats.kstest(lam, cdf).pvalue > 1e-3
    assert lam.min() >= 300.0 and lam.max() <= 600.0


# ---------------------------------------------------------------- cone
def test_rotation_matrix_properties():
    rng = np.random.default_rng(3)
    dirs = list(rng.normal(size=(50, 3))) + [np.array([0, 0, -1.0]), np.array([0, 0, 1.0]),
                                             np.array([1.0, 0, 0]), np.array([0, 1e-9, 1.0])]
    for d in dirs:
        d = d / np.linalg.norm(d)
        M = O.rotation(d)
        np.testing.assert_allclose(M @ M.T, np.eye(3), atol=1e-13)
        assert np.linalg.det(M) == pytest.approx(1.0, abs=1e-13)
        np.testing.assert_allclose(M @ np.array([0, 0, -1.0]), d, atol=1e-9)
        np.testing.assert_allclose(M, M.T, atol=1e-15)          # half turn: symmetric


def test_cone_angle_and_azimuth_are_preserved():
    """Every photon sits at theta_c from the track; the azimuth difference of
    two photons of one step equals 2 pi (u2 - u2') from their Philox words."""
    atm = I.atmosphere_layered()
    par = I.Params(bunch=1.0)
    rng = np.random.default_rng(5)
    for t in range(10):
        d = rng.normal(size=3)
        d[2] = -abs(d[2]) - 0.3
        d /= np.linalg.norm(d)
        seg = _one_seg(eps=2e-6, z=7000.0, L=2.0, d=tuple(d.astype(np.float32)))
        dd = np.array([seg["dx"], seg["dy"], seg["dz"]], dtype=np.float64)
        dd /= np.linalg.norm(dd)
        y = O.yield_of(seg, atm, par)
        e1 = np.cross(dd, [0.3, 0.5, 0.8]); e1 /= np.linalg.norm(e1)
        e2 = np.cross(e1, dd)     # (e1, e2, -d) right-handed, as (x, y, z) about -z
        az, u2 = [], []
        for k in range(8):
            r_e, dg, t_e, lam, w, proc = O.photon(seg, 100 + t, k, atm, par)
            assert proc == 0
            assert np.linalg.norm(dg) == pytest.approx(1.0, abs=1e-14)
            assert math.acos(np.clip(dg @ dd, -1, 1)) == pytest.approx(math.acos(y["cos_tc"]), abs=1e-10)
            az.append(math.atan2(dg @ e2, dg @ e1))
            x = O.philox([100 + t, 0, k, 0], [1, 0])
            u2.append(O.u01(x[2]))
            ell = np.linalg.norm(r_e - np.array([0, 0, 7000.0]))
            assert t_e == pytest.approx(ell / ((1 - float(np.float32(2e-6))) * C_M_NS), rel=1e-12)
        for k in range(1, 8):
            da = (az[k] - az[0]) - 2 * math.pi * (u2[k] - u2[0])
            da = (da + math.pi) % (2 * math.pi) - math.pi
            assert abs(da) < 1e-9


def test_fluorescence_is_isotropic():
    atm = I.atmosphere_layered()
    par = I.Params(bunch=1.0, fluor_yield=50.0)
    seg = _one_seg(eps=0.5, z=9000.0, L=2.0, dE=80.0)      # below Cherenkov threshold
    y = O.yield_of(seg, atm, par)
    assert y["n_c"] == 0 and y["n_f"] == 4000
    dz = np.array([O.photon(seg, 3, k, atm, par)[1][2] for k in range(4000)])
    assert stats.kstest(dz, "uniform", args=(-1, 2)).pvalue > 1e-3
    lam = np.array([O.photon(seg, 3, k, atm, par)[3] for k in range(0, 4000, 4)])
    assert stats.kstest(lam, "uniform", args=(340, 110)).pvalue > 1e-3


# ---------------------------------------------------------------- propagation
def _dirs(rng, n, max_zen_deg):
    zen = np.radians(rng.uniform(0, max_zen_deg, n))
    az = rng.uniform(0, 2 * np.pi, n)
    return np.stack([np.sin(zen) * np.cos(az), np.sin(zen) * np.sin(az), -np.cos(zen)], 1)


def test_straight_flat_single_exponential_closed_form():
    """Refraction off, flat Earth, n - 1 = a e^{-h/H}: landing point, time and
    optical depth have closed forms."""
    atm = I.atmosphere_single_exponential(refraction=False, absorption=True)
    a, H = 2.9e-4, 8400.0
    rng = np.random.default_rng(11)
    for d in _dirs(rng, 20, 70):
        r_e = np.array([rng.uniform(-500, 500), rng.uniform(-500, 500), rng.uniform(3000, 30000)])
        lam = rng.uniform(300, 600)
        res = O.propagate(atm, r_e, d, t_e=5.0, lam=lam)
        dz = abs(d[2])
        dh = r_e[2] - atm.h_obs
        P = r_e + d * dh / dz
        np.testing.assert_allclose(res["P"], P, rtol=0, atol=1e-9)
        np.testing.assert_allclose(res["dL"], d, atol=1e-14)
        ex = math.exp(-atm.h_obs / H) - math.exp(-r_e[2] / H)
        t = 5.0 + (dh + a * H * ex) / (C_M_NS * dz)
        assert res["t"] == pytest.approx(t, rel=0, abs=1e-9)
        tau = (I.RHO_SEA / atm.rho_ref) * H * ex / (atm.L0 * (lam / 400.0) ** 4 * dz)
        assert res["tau"] == pytest.approx(tau, rel=1e-11)


def test_straight_spherical_line_sphere_intersection():
    atm = I.atmosphere_layered(refraction=False)
    rng = np.random.default_rng(12)
    r_obs = atm.R_E + atm.h_obs
    for d in _dirs(rng, 12, 75):
        r_e = np.array([rng.uniform(-3e4, 3e4), rng.uniform(-3e4, 3e4), rng.uniform(5000, 35000)])
        res = O.propagate(atm, r_e, d, t_e=0.0, lam=450.0)
        Rv = r_e + np.array([0, 0, atm.R_E])
        b = -(Rv @ d)
        s = b - math.sqrt(b * b - (Rv @ Rv - r_obs ** 2))
        P = r_e + s * d
        np.testing.assert_allclose(res["P"], P, atol=2e-6)
        np.testing.assert_allclose(res["dL"], d, atol=1e-12)

        def n_along(u):
            p = r_e + u * d
            h = np.linalg.norm(p + [0, 0, atm.R_E]) - atm.R_E
            return 1.0 + atm.K * float(atm.density(h))
        pts = sorted([u for u in np.linspace(0, s, 2) ])
        Lopt, _ = integrate.quad(n_along, 0.0, s, epsabs=1e-9, epsrel=1e-13, limit=400)
        assert res["t"] == pytest.approx(Lopt / C_M_NS, abs=2e-6)


@pytest.mark.parametrize("spherical", [False, True])
def test_refracted_rays_match_brute_force_eikonal(spherical):
    atm = I.atmosphere_layered(spherical=spherical)
    rng = np.random.default_rng(21 + spherical)
    N = 12
    d = _dirs(rng, N, 65)
    r_e = np.stack([rng.uniform(-2e4, 2e4, N), rng.uniform(-2e4, 2e4, N),
                    rng.uniform(4000, 16000, N)], 1)
    P, D, Lopt, Ltau = _eikonal.trace(atm, r_e, d, ds=2.0)
    for i in range(N):
        res = O.propagate(atm, r_e[i], d[i], t_e=0.0, lam=400.0)
        assert res["status"] == O.OR_TRACED
        np.testing.assert_allclose(res["P"], P[i], atol=2e-4)
        np.testing.assert_allclose(res["dL"], D[i], atol=1e-9)
        # RK4 loses accuracy where grad n jumps at layer edges (~1e-5 m of
        # optical path, not monotone in the step): 5e-4 ns = 0.15 mm
        assert res["t"] == pytest.approx(Lopt[i] / C_M_NS, abs=5e-4)
        assert res["tau"] == pytest.approx(Ltau[i] / atm.L0, rel=1e-6)


def test_refraction_invariants_vertical_and_flat_limit():
    atm = I.atmosphere_layered(spherical=False)
    # vertical rays are not bent
    res = O.propagate(atm, [12.5, -7.0, 15000.0], [0, 0, -1.0])
    np.testing.assert_allclose(res["P"][:2], [12.5, -7.0], atol=1e-12)
    # Snell: n sin(theta) is the same at emission and arrival
    d = np.array([0.5, 0.2, -0.8]); d /= np.linalg.norm(d)
    res = O.propagate(atm, [0, 0, 12000.0], d)
    n_e = 1 + O.delta(atm, 12000.0)
    assert res["n_obs"] * math.hypot(*res["dL"][:2]) == pytest.approx(n_e * math.hypot(*d[:2]), rel=1e-13)
    # a spherical Earth of huge radius approaches the flat result
    big = I.atmosphere_layered(spherical=True)
    big.R_E = 1e13
    flat = O.propagate(atm, [100.0, 50.0, 12000.0], d, lam=380.0)
    sph = O.propagate(big, [100.0, 50.0, 12000.0], d, lam=380.0)
    np.testing.assert_allclose(sph["P"], flat["P"], atol=1e-4)
    # residual curvature: drop D^2 / 2R ~ 3e-6 m over D ~ 7.5 km -> 1e-5 ns
    assert sph["t"] == pytest.approx(flat["t"], abs=5e-5)
    assert sph["tau"] == pytest.approx(flat["tau"], rel=1e-7)


def test_fermat_refracted_path_is_shortest_in_optical_length():
    atm = I.atmosphere_layered(spherical=True)
    rng = np.random.default_rng(31)
    for d in _dirs(rng, 6, 70):
        r_e = np.array([0.0, 0.0, rng.uniform(6000, 20000)])
        res = O.propagate(atm, r_e, d)
        P = res["P"]
        chord = P - r_e
        Ls = np.linalg.norm(chord)

        def n_along(u):
            p = r_e + u * chord / Ls
            h = np.linalg.norm(p + [0, 0, atm.R_E]) - atm.R_E
            return 1.0 + atm.K * float(atm.density(h))
        Lchord, _ = integrate.quad(n_along, 0, Ls, epsabs=1e-10, epsrel=1e-14, limit=400,
                                   points=None)
        Lref = res["t"] * C_M_NS
        assert Lref <= Lchord + 1e-7
        assert Lchord - Lref < 1e-3 * Ls * 1e-3


def test_escaped_and_turned_rays():
    atm = I.atmosphere_layered(spherical=True)
    assert O.propagate(atm, [0, 0, 9000.0], [0.3, 0, 0.95])["status"] == O.OR_ESCAPED
    # almost horizontal at 30 km: misses the observation sphere
    d = np.array([1.0, 0.0, -0.001]); d /= np.linalg.norm(d)
    assert O.propagate(atm, [0, 0, 30000.0], d)["status"] == O.OR_TURNED
    assert O.propagate(atm, [0, 0, 1500.0], [0, 0, -1.0])["status"] == O.OR_UNDER


# ---------------------------------------------------------------- hit test
def test_hit_decision_matches_brute_force_distance():
    """Impact parameter from the oracle vs. the minimum distance found by
    sampling points along the line."""
    atm = I.atmosphere_single_exponential()
    rng = np.random.default_rng(41)
    tels = np.zeros(3, dtype=I.TEL_DTYPE)
    tels["x"] = [0.0, 14.0, -9.0]
    tels["y"] = [0.0, 3.0, 11.0]
    tels["z"] = atm.h_obs
    tels["R"] = [6.0, 4.0, 5.0]
    segs = np.zeros(200, dtype=I.SEG_DTYPE)
    segs["x"] = rng.uniform(-120, 120, 200)
    segs["y"] = rng.uniform(-120, 120, 200)
    segs["z"] = rng.uniform(4000, 7000, 200)
    segs["dz"] = -1.0
    segs["L"] = 1.0
    segs["eps"] = 1e-5
    segs["charge"] = -1
    hits, counts, sums, st = O.trace(segs, atm, tels, I.Params(bunch=1.0))
    assert len(hits) > 0
    for h in hits[:50]:
        r_e, dg, t_e, lam, w, _ = O.photon(segs[h["seg"]], h["seg"], h["k"], atm, I.Params(bunch=1.0))
        res = O.propagate(atm, r_e, dg, t_e, lam)
        T = tels[h["tel"]]
        C3 = np.array([T["x"], T["y"], T["z"]], dtype=np.float64)
        s = np.linspace(-40, 40, 400001)
        pts = res["P"][None, :] + s[:, None] * res["dL"][None, :]
        dmin = np.min(np.linalg.norm(pts - C3[None, :], axis=1))
        assert dmin == pytest.approx(h["dperp"], abs=1e-6)
        assert h["dperp"] < T["R"]
    # the sorted list, the counts and the sums agree
    assert np.all(np.diff(hits["tel"].astype(np.int64) * 10 ** 12 + hits["seg"] * 10 ** 4 + hits["k"]) > 0)
    assert counts.sum() == len(hits)
    for j in range(3):
        assert sums[0, j] == pytest.approx(hits["weight"][hits["tel"] == j].sum(), rel=1e-14)


# ---------------------------------------------------------------- inputs
def test_shower_generator_distributions():
    atm = I.atmosphere_layered()
    s = I.segments_shower(200_000, atm, seed=3, zenith_deg=0.0)
    assert s.dtype.itemsize == 64
    r = np.hypot(s["x"], s["y"])
    assert stats.kstest(r, "expon", args=(0, 80)).pvalue > 1e-4
    nrm = np.sqrt(s["dx"].astype(np.float64) ** 2 + s["dy"] ** 2 + s["dz"] ** 2)
    assert np.abs(nrm - 1).max() < 3e-7
    assert (s["z"] > atm.h_obs).all()
    X = atm.thickness(s["z"])
    X_obs = float(atm.thickness(np.array([atm.h_obs]))[0])
    g = stats.gamma(6, scale=70.0)                        # Gaisser-Hillas, Xmax 350, lambda 70
    assert stats.kstest(X, lambda x: g.cdf(x) / g.cdf(X_obs)).pvalue > 1e-4
    L = s["L"]
    assert L.min() >= 0.5 and L.max() <= 5.0


# ---------------------------------------------------------------- adjoint reference
def _fluorescence_steps(n, seed):
    """Uncharged steps (no Cherenkov light) that emit fluorescence only."""
    rng = np.random.default_rng(seed)
    s = np.zeros(n, dtype=I.SEG_DTYPE)
    s["x"] = rng.uniform(-50, 50, n)
    s["y"] = rng.uniform(-50, 50, n)
    s["z"] = rng.uniform(5000, 15000, n)
    s["dz"] = -1.0
    s["L"] = 1.0
    s["eps"] = 1e-3
    s["dE"] = rng.uniform(0.5, 2.0, n)
    s["charge"] = 0
    return s


def test_oracle_gradient_matches_closed_form_for_straight_rays():
    """Refraction off, flat Earth, one exponential layer, fluorescence only:
    the emission does not depend on the atmosphere, the ray is straight, and
    t - t_e = (s + K b/(100 |dz|) (e^{-h_obs/c} - e^{-h_e/c})) / c_light,
    tau = b (e^{-h_obs/c} - e^{-h_e/c}) / (100 rho_ref |dz| L0 (lambda/lambda_ref)^4).
    Central differences of the oracle (h = 1e-4 relative) against the
    derivatives of these in K, c and L0."""
    atm = I.atmosphere_single_exponential(refraction=False, absorption=True, spherical=False)
    par = I.Params(bunch=1.0, seed=3, fluor_yield=5.0)
    segs = _fluorescence_steps(40, seed=2)
    tel = np.zeros(1, dtype=I.TEL_DTYPE)
    tel["z"] = atm.h_obs
    tel["R"] = 1e6
    nbc, nbf = O.bunch_counts(segs, atm, par)
    assert nbc.sum() == 0 and nbf.sum() > 100
    rows = []
    for i in range(len(segs)):
        for k in range(int(nbf[i])):
            r, d, te, lam, w, proc = O.photon(segs[i], i, k, atm, par)
            if d[2] < -0.2:
                rows.append((i, k, r[2], abs(d[2]), lam, w, te))
    rows = np.array(rows)
    si, kk = rows[:, 0].astype(np.int64), rows[:, 1].astype(np.uint32)
    he, adz, lam, w = rows[:, 2], rows[:, 3], rows[:, 4], rows[:, 5]
    tt = np.zeros(len(rows), dtype=np.uint32)
    b, c, K, L0, ho = atm.b[0], atm.c[0], atm.K, atm.L0, atm.h_obs

    def ev(a):
        return O.eval_rays(segs, si, kk, tt, nbc, nbf, a, tel, par)

    base = ev(atm)
    # the closed form of the values themselves
    E = np.exp(-ho / c) - np.exp(-he / c)
    t_cf = rows[:, 6] + ((he - ho) / adz + K * b / (100 * adz) * E) / C_M_NS
    tau = b * E / (100 * atm.rho_ref * adz * L0 * (lam / atm.lambda_ref) ** 4)
    np.testing.assert_allclose(base[:, 2], t_cf, rtol=1e-12, atol=1e-9)
    np.testing.assert_allclose(base[:, 3], w * np.exp(-tau), rtol=1e-10)
    dE_dc = (ho * np.exp(-ho / c) - he * np.exp(-he / c)) / c ** 2
    expect = {
        "K": (b / (100 * adz) * E / C_M_NS, np.zeros(len(rows))),
        "c": (K * b / (100 * adz) * dE_dc / C_M_NS, -w * np.exp(-tau) * tau / E * dE_dc),
        "L0": (np.zeros(len(rows)), w * np.exp(-tau) * tau / L0),
    }
    for name, (dt, dw) in expect.items():
        val = {"K": K, "c": c, "L0": L0}[name]
        h = 1e-4 * val
        out = []
        for sgn in (1, -1):
            a = I.Atmosphere(**{**atm.__dict__})
            if name == "c":
                a.c = [c + sgn * h]
            else:
                setattr(a, name, val + sgn * h)
            out.append(ev(a))
        fd = (out[0] - out[1]) / (2 * h)
        np.testing.assert_allclose(fd[:, 2], dt, rtol=1e-6, atol=1e-12 * np.abs(dt).max())
        np.testing.assert_allclose(fd[:, 3], dw, rtol=1e-6, atol=1e-9 * np.abs(dw).max() + 1e-300)
        np.testing.assert_allclose(fd[:, 0], 0.0, atol=1e-9)      # straight rays do not move


def test_eval_rays_reproduces_the_traced_hits():
    w = I.workload_shower_1tev(n=3000, seed=7)
    h, cnt, sums, st = O.trace(w.segments, w.atmosphere, w.telescopes, w.params)
    assert len(h) > 50
    nbc, nbf = O.bunch_counts(w.segments, w.atmosphere, w.params)
    ev = O.eval_rays(w.segments, h["seg"], h["k"], h["tel"], nbc, nbf, w.atmosphere, w.telescopes, w.params)
    np.testing.assert_allclose(ev[:, 0], h["x_rel"], atol=1e-9)
    np.testing.assert_allclose(ev[:, 1], h["y_rel"], atol=1e-9)
    np.testing.assert_allclose(ev[:, 2], h["t"], rtol=0, atol=1e-9)
    np.testing.assert_allclose(ev[:, 3], h["weight"], rtol=1e-12)
    np.testing.assert_allclose(ev[:, 4], h["dperp"], atol=1e-9)


def test_soft_yield_limits():
    """s -> 0 gives the hard-aperture photon sums; the cut at R + W does not matter."""
    w = I.workload_shower_1tev(n=3000, seed=9)
    h, cnt, sums, st = O.trace(w.segments, w.atmosphere, w.telescopes, w.params)
    nbc, nbf = O.bunch_counts(w.segments, w.atmosphere, w.params)
    hard = O.soft_yield(w.segments, nbc, nbf, w.atmosphere, w.telescopes, w.params, s=1e-9, W=0.01)
    edge = np.abs(h["dperp"] - w.telescopes["R"][h["tel"]]) < 1e-6
    assert not edge.any()
    np.testing.assert_allclose(hard, sums, rtol=1e-9, atol=1e-9)
    y20 = O.soft_yield(w.segments, nbc, nbf, w.atmosphere, w.telescopes, w.params, s=0.5, W=20.0)
    y40 = O.soft_yield(w.segments, nbc, nbf, w.atmosphere, w.telescopes, w.params, s=0.5, W=40.0)
    np.testing.assert_allclose(y20, y40, rtol=1e-12, atol=1e-15 * y40.max())
    assert y20.sum() > 0


# ---------------------------------------------------------------- angular cut
def _aimed_steps(targets_and_angles, z=10000.0):
    """One vertical-ish step per (target point, extra angle): the step at
    (0, 0, z) points at the target, then tilts by the extra angle about y."""
    s = np.zeros(len(targets_and_angles), dtype=I.SEG_DTYPE)
    for i, (tgt, extra) in enumerate(targets_and_angles):
        v = np.asarray(tgt, dtype=np.float64) - np.array([0.0, 0.0, z])
        v /= np.linalg.norm(v)
        a = math.radians(extra)
        R = np.array([[math.cos(a), 0, math.sin(a)], [0, 1, 0], [-math.sin(a), 0, math.cos(a)]])
        d = R @ v
        s[i]["x"], s[i]["y"], s[i]["z"] = 0.0, 0.0, z
        s[i]["dx"], s[i]["dy"], s[i]["dz"] = d
    s["L"] = 1e-3          # the midpoint is the start to 1e-4 rad
    s["eps"] = 1e-6
    s["charge"] = -1
    return s


def test_angular_cut_decisions_against_brute_force_angles():
    """Sec. 1.2.1: Cherenkov light of a step survives when its direction is
    within the cut angle of the direction to the array centre (mode 1) or to
    some telescope (mode 2).  Angles by arccos, away from the boundary."""
    atm = I.atmosphere_layered()
    tels = I.telescope_grid(3, 3, 300.0, z=atm.h_obs)
    centre = I.array_centre(tels)
    far = (tels["x"][0], tels["y"][0], tels["z"][0])            # a corner telescope
    cases = [(centre, 0.0), (centre, 5.0), (centre, 7.0), (centre, -5.5), (centre, 20.0),
             (far, 1.0), (far, 5.0), (far, 8.0)]
    segs = _aimed_steps(cases)
    for mode in (1, 2):
        par = I.Params(bunch=1.0, cut_mode=mode, cut_deg=6.0, cut_centre=centre)
        for s, (tgt, extra) in zip(segs, cases):
            d = np.array([s["dx"], s["dy"], s["dz"]], dtype=np.float64)
            d /= np.linalg.norm(d)
            m = np.array([s["x"], s["y"], s["z"]]) + 0.5 * float(s["L"]) * d
            targets = [np.array(centre)] if mode == 1 else [np.array([t["x"], t["y"], t["z"]], float) for t in tels]
            ang = min(math.degrees(math.acos(np.clip(d @ (c - m) / np.linalg.norm(c - m), -1, 1))) for c in targets)
            assert abs(ang - 6.0) > 0.05
            y = O.yield_of(s, atm, par, tels)
            y0 = O.yield_of(s, atm, I.Params(bunch=1.0))
            assert y0["n_c"] > 0
            assert (y["n_c"] > 0) == (ang < 6.0), (mode, tgt, extra, ang)
            if y["n_c"] > 0:
                assert y["n_c"] == y0["n_c"] and y["w_c"] == y0["w_c"]


def test_angular_cut_keeps_a_subset_of_the_hits():
    """With the cut the oracle's hits are exactly the uncut hits of the kept
    steps (same keys, same values); fluorescence is untouched."""
    w = I.workload_shower_1tev(n=4000, seed=21)
    h0, c0, s0, st0 = O.trace(w.segments, w.atmosphere, w.telescopes, w.params)
    par = I.Params(**{**w.params.__dict__, "cut_mode": 1, "cut_deg": 6.0,
                      "cut_centre": I.array_centre(w.telescopes)})
    h1, c1, s1, st1 = O.trace(w.segments, w.atmosphere, w.telescopes, par)
    assert st1["rays"] < st0["rays"] and len(h1) > 0
    nc1, _ = O.bunch_counts(w.segments, w.atmosphere, par)
    kept = nc1[h0["seg"]] > 0
    np.testing.assert_array_equal(h1, h0[kept])


# ---------------------------------------------------------------- fluorescence beaming
def _fluor_workload(n, seed, beaming, dE=(20.0, 40.0), xy=3000.0, z=(3000.0, 9000.0)):
    atm = I.atmosphere_layered()
    tels = I.telescope_grid(4, 4, 100.0, z=atm.h_obs)
    rng = np.random.default_rng(seed)
    s = np.zeros(n, dtype=I.SEG_DTYPE)
    s["x"] = rng.uniform(-xy, xy, n)
    s["y"] = rng.uniform(-xy, xy, n)
    s["z"] = rng.uniform(z[0], z[1], n)
    d = rng.normal(size=(n, 3))
    d /= np.linalg.norm(d, axis=1)[:, None]
    s["dx"], s["dy"], s["dz"] = d[:, 0], d[:, 1], d[:, 2]
    s["L"] = rng.uniform(0.5, 5.0, n)
    s["eps"] = 1e-3
    s["dE"] = rng.uniform(dE[0], dE[1], n)
    s["charge"] = 0
    c, r = I.beam_cone(tels)
    par = I.Params(bunch=1.0, seed=seed, fluor_yield=5.0, fl_beaming=beaming, beam_centre=c, beam_radius=r)
    return I.Workload("fluor", s, atm, tels, par)


def test_beamed_fluorescence_fills_its_cone_uniformly():
    """Sec. 1.1.1: beamed directions lie in the cone about the step-to-array
    axis, uniform in solid angle (cos of the angle to the axis uniform on
    [cos alpha, 1]); the photon number scales by sin^2(alpha/2)."""
    w = _fluor_workload(200, 3, 1, dE=(2000.0, 4000.0))
    c, R = np.array(w.params.beam_centre), w.params.beam_radius
    cosines = []
    for i, s in enumerate(w.segments[:60]):
        d = np.array([s["dx"], s["dy"], s["dz"]], dtype=np.float64)
        d /= np.linalg.norm(d)
        m = np.array([s["x"], s["y"], s["z"]]) + 0.5 * float(s["L"]) * d
        D = np.linalg.norm(c - m)
        alpha = math.asin(R / D) + 5e-3 + float(s["L"]) / D
        u = (c - m) / D
        y = O.yield_of(s, w.atmosphere, w.params)
        y0 = O.yield_of(s, w.atmosphere, dataclasses.replace(w.params, fl_beaming=0))
        np.testing.assert_allclose(y["Nf"], y0["Nf"] * math.sin(alpha / 2) ** 2, rtol=1e-12)
        for k in range(int(y["n_f"])):
            r, dg, te, lam, wt, proc = O.photon(s, i, k, w.atmosphere, w.params)
            assert proc == 1
            cosines.append((dg @ u - math.cos(alpha)) / (1 - math.cos(alpha)))
    cosines = np.array(cosines)
    assert cosines.min() >= -1e-12 and cosines.max() <= 1 + 1e-12 and len(cosines) > 200
    assert stats.kstest(cosines, "uniform").pvalue > 1e-3


def test_beaming_loses_no_hits_and_keeps_the_mean():
    """Every hit of isotropic emission left its step inside that step's
    cone, so beaming removes no reachable direction; the beamed photon sums
    agree with the isotropic ones within their statistical error."""
    kw = dict(dE=(300.0, 500.0), xy=1000.0, z=(3000.0, 4500.0))
    wi = _fluor_workload(1200, 5, 0, **kw)
    wb = _fluor_workload(1200, 5, 1, **kw)
    hi, ci, si, sti = O.trace(wi.segments, wi.atmosphere, wi.telescopes, wi.params)
    hb, cb, sb, stb = O.trace(wb.segments, wb.atmosphere, wb.telescopes, wb.params)
    assert len(hi) > 30 and stb["rays"] < 0.2 * sti["rays"]
    c, R = np.array(wb.params.beam_centre), wb.params.beam_radius
    for h in hi:
        s = wi.segments[h["seg"]]
        d = np.array([s["dx"], s["dy"], s["dz"]], dtype=np.float64)
        d /= np.linalg.norm(d)
        m = np.array([s["x"], s["y"], s["z"]]) + 0.5 * float(s["L"]) * d
        D = np.linalg.norm(c - m)
        assert D >= 2 * R
        alpha = math.asin(R / D) + 5e-3 + float(s["L"]) / D
        r, dg, te, lam, wt, proc = O.photon(s, int(h["seg"]), int(h["k"]), wi.atmosphere, wi.params)
        assert math.acos(np.clip(dg @ (c - m) / D, -1, 1)) < alpha
    # means: isotropic photons hit with bunch weight 1 (Poisson); beamed ones carry the cone share
    tot_i, tot_b = si.sum(), sb.sum()
    assert abs(tot_b - tot_i) < 5 * math.sqrt(tot_i) + 5 * math.sqrt(max(1.0, (sb ** 2).sum() / max(1, len(hb)))), (tot_i, tot_b)


def test_fluorescence_roulette_is_unbiased_and_keeps_large_counts():
    """Count rule 1 (the reading that lets beaming cut rays): a step with
    N_f < B emits one bunch of weight B with probability N_f/B, the number
    drawn from the (cuRAND-pinned) Philox at counter (step, 0xFFFFFFFF, 1);
    its expectation is N_f.  Steps with N_f >= B keep ceil bunching."""
    w = _fluor_workload(1, 7, 0, dE=(1.0, 1.0))
    s = w.segments[0]
    par = dataclasses.replace(w.params, bunch=10.0, fl_roulette=1)
    Nf = O.yield_of(s, w.atmosphere, par)["Nf"]
    assert Nf == pytest.approx(5.0)
    x = Nf / par.bunch
    n = 4000
    picks = np.zeros(n)
    for i in range(n):
        y = O.yield_of(s, w.atmosphere, par, seg_index=i)
        assert y["n_c"] == 0 and y["n_f"] in (0, 1)
        assert y["w_f"] == (par.bunch if y["n_f"] else 0.0)
        u = O.u01(O.philox([i, 0, 0xFFFFFFFF, 1], [par.seed, par.stream])[0])
        assert y["n_f"] == (1 if u < x else 0)
        picks[i] = y["n_f"]
    # mean photon number N_f within 5 sigma of the binomial
    assert abs(picks.mean() * par.bunch - Nf) < 5 * par.bunch * math.sqrt(x * (1 - x) / n)
    # a high word of the step index reaches the counter
    big = (1 << 32) + 17
    u = O.u01(O.philox([17, 1, 0xFFFFFFFF, 1], [par.seed, par.stream])[0])
    assert O.yield_of(s, w.atmosphere, par, seg_index=big)["n_f"] == (1 if u < x else 0)
    # N_f >= B: unchanged
    s2 = s.copy()
    s2["dE"] = 7.3
    y1 = O.yield_of(s2, w.atmosphere, par, seg_index=3)
    y0 = O.yield_of(s2, w.atmosphere, dataclasses.replace(par, fl_roulette=0), seg_index=3)
    assert (y1["n_f"], y1["w_f"]) == (y0["n_f"], y0["w_f"]) == (4.0, pytest.approx(36.5 / 4))


def test_fluorescence_roulette_keeps_the_mean_photon_sums():
    """Beamed steps with few photons under count rule 1: far fewer rays,
    the same expected photon sums at the telescopes."""
    kw = dict(dE=(50.0, 150.0), xy=1000.0, z=(3000.0, 4500.0))
    wb = _fluor_workload(100000, 11, 1, **kw)
    wb.params = dataclasses.replace(wb.params, bunch=10.0)
    wr = _fluor_workload(100000, 11, 1, **kw)
    wr.params = dataclasses.replace(wr.params, bunch=10.0, fl_roulette=1)
    hb, cb, sb, stb = O.trace(wb.segments, wb.atmosphere, wb.telescopes, wb.params)
    hr, cr, sr, str_ = O.trace(wr.segments, wr.atmosphere, wr.telescopes, wr.params)
    assert str_["rays"] < 0.5 * stb["rays"]
    # emitted with weight B (the hit weight is that times the transmission)
    for h in hr[:20]:
        assert O.photon(wr.segments[h["seg"]], int(h["seg"]), int(h["k"]), wr.atmosphere, wr.params)[4] == 10.0
    assert np.all(hr["weight"] <= 10.0)
    tb, tr = sb.sum(), sr.sum()
    # roulette hits: counts of weight 10 (Poisson-like); the ceil side is nearly exact
    assert len(hr) > 30
    assert abs(tr - tb) < 5 * 10.0 * math.sqrt(tb / 10.0 + 1), (tb, tr)


# ---------------------------------------------------------------- dispersion
def _disp_atm(B):
    a = I.atmosphere_layered()
    a.disp_B = B
    a.disp_lref = 400.0
    return a


def _one_step(eps, z=8000.0):
    s = np.zeros(1, dtype=I.SEG_DTYPE)
    s["z"] = z
    s["dz"] = -1.0
    s["L"] = 2.0
    s["eps"] = eps
    s["charge"] = -1
    return s[0]


def test_dispersion_yield_against_the_wavelength_integral():
    """Sec. 1.2's Frank-Tamm double integral with n depending on lambda:
    the oracle's integral in u = 1/lambda against scipy's quadrature in
    lambda, below and across the Cherenkov threshold; B -> 0 gives the
    closed form of the dispersion-free yield."""
    par = I.Params(bunch=1.0)
    alpha = SC.fine_structure
    for B in (5000.0, 20000.0):
        atm = _disp_atm(B)
        for eps in (1e-6, 5e-5, 1.5e-4):
            s = _one_step(eps)
            y = O.yield_of(s, atm, par)
            delta = y["delta"]
            beta = 1.0 - eps

            def integrand(lam):
                n = 1.0 + delta * O.disp_g(atm, lam)
                return max(0.0, 1.0 - 1.0 / (beta * n) ** 2) / lam ** 2
            ref = integrate.quad(integrand, par.lambda1, par.lambda2, limit=400, epsabs=0, epsrel=1e-12)[0]
            Nref = 2 * math.pi * alpha * 1e9 * ref * float(s["L"])
            assert (y["Nc"] > 0) == (Nref > 0)
            if Nref > 0:
                np.testing.assert_allclose(y["Nc"], Nref, rtol=2e-6)
    atm0 = _disp_atm(1e-9)
    s = _one_step(1e-5)
    y = O.yield_of(s, atm0, par)
    y_nd = O.yield_of(s, I.atmosphere_layered(), par)
    np.testing.assert_allclose(y["Nc"], y_nd["Nc"], rtol=1e-9)


def test_dispersion_wavelengths_and_cherenkov_angles():
    """Photon wavelengths follow (1/lambda^2)(1 - 1/(beta n(lambda))^2) on the
    band above threshold (KS against scipy's CDF), and each photon leaves at
    cos(theta) = 1/(beta n(lambda)) to its track."""
    atm = _disp_atm(20000.0)
    s = _one_step(0.0, z=4000.0)
    d0 = O.yield_of(s, atm, I.Params())["delta"]
    eps = 1.02 * d0            # the threshold falls inside 300-600 nm
    s["eps"] = eps
    s["L"] = 5.0
    par = I.Params(bunch=1.0, seed=11)
    y = O.yield_of(s, atm, par)
    delta, beta = y["delta"], 1.0 - eps
    assert y["n_c"] >= 1
    lams = []
    segs = np.repeat(s[None], 300)
    for i in range(300):
        for k in range(int(y["n_c"])):
            r, d, te, lam, w, proc = O.photon(segs[i], i, k, atm, par)
            n = 1.0 + delta * O.disp_g(atm, lam)
            assert abs(-d[2] - 1.0 / (beta * n)) < 1e-10
            lams.append(lam)
    lams = np.array(lams)
    assert len(lams) >= 300

    def dens(lam):
        n = 1.0 + delta * O.disp_g(atm, lam)
        return max(0.0, 1.0 - 1.0 / (beta * n) ** 2) / lam ** 2
    top = integrate.quad(dens, par.lambda1, par.lambda2, epsrel=1e-10, limit=200)[0]
    cdf = lambda x: np.array([integrate.quad(dens, par.lambda1, v, epsrel=1e-9, limit=200)[0] / top for v in np.atleast_1d(x)])
    assert lams.max() < par.lambda2 and dens(lams.max()) > 0
    assert stats.kstest(lams, cdf).pvalue > 1e-3


# ---------------------------------------------------------------- FP64 reference gradient
def _atm_at(base, th):
    a = I.Atmosphere(**{**base.__dict__})
    L = a.n_layers
    a.c = list(th[:L])
    a.K = th[L]
    a.L0 = th[L + 1]
    return a


@pytest.mark.parametrize("case", ["vertical", "inclined"])
def test_dual_number_gradient_matches_central_differences(case):
    """The oracle's FP64 gradient by dual numbers (a separate derivation of
    the same physics) against its own central differences (h = 1e-4
    relative): hit positions, times and weights, and the soft yield."""
    w = (I.workload_shower_1tev(n=2500, seed=41) if case == "vertical"
         else I.workload_inclined(n=1500, seed=43))
    h, c, s, st = O.trace(w.segments, w.atmosphere, w.telescopes, w.params)
    assert len(h) > 20
    nbc, nbf = O.bunch_counts(w.segments, w.atmosphere, w.params)
    rng = np.random.default_rng(1)
    gx, gy, gt, gw = rng.normal(size=(4, len(h)))
    gY = rng.normal(size=len(w.telescopes))
    g = O.grad_rays(w.segments, h["seg"], h["k"], h["tel"], nbc, nbf, w.atmosphere, w.telescopes, w.params,
                    gx, gy, gt, gw)
    gs = O.grad_soft(w.segments, nbc, nbf, w.atmosphere, w.telescopes, w.params, gY, s=0.5, W=20.0)
    theta = np.array(list(w.atmosphere.c) + [w.atmosphere.K, w.atmosphere.L0])

    def loss(th):
        ev = O.eval_rays(w.segments, h["seg"], h["k"], h["tel"], nbc, nbf, _atm_at(w.atmosphere, th),
                         w.telescopes, w.params)
        return gx @ ev[:, 0] + gy @ ev[:, 1] + gt @ ev[:, 2] + gw @ ev[:, 3]

    def lsoft(th):
        return float(gY @ O.soft_yield(w.segments, nbc, nbf, _atm_at(w.atmosphere, th), w.telescopes, w.params,
                                       s=0.5, W=20.0).ravel())
    for p in range(len(theta)):
        hp = 1e-4 * theta[p]
        tp, tm = theta.copy(), theta.copy()
        tp[p] += hp
        tm[p] -= hp
        fd = (loss(tp) - loss(tm)) / (2 * hp)
        fds = (lsoft(tp) - lsoft(tm)) / (2 * hp)
        scale = max(abs(fd), 1e-9 * np.abs(g).max())
        assert abs(g[p] - fd) <= 2e-5 * scale, (p, g[p], fd)
        scale_s = max(abs(fds), 1e-9 * np.abs(gs).max())
        assert abs(gs[p] - fds) <= 1e-4 * scale_s, (p, gs[p], fds)


# ---------------------------------------------------------------- the paper's rule of thumb for the cut
def _cut_rule_workload(n, seed, d_lo, d_hi, R=300.0):
    """Electron steps at distance D in [d_lo, d_hi] radii from one large
    telescope sphere (radius R, at the observation level), flying toward it
    within 0-10 degrees of the direction to its centre."""
    atm = I.atmosphere_layered()
    tels = I.telescope_grid(1, 1, 1.0, R=R, z=atm.h_obs)
    C = np.array([float(tels["x"][0]), float(tels["y"][0]), float(tels["z"][0])])
    rng = np.random.default_rng(seed)
    s = np.zeros(n, dtype=I.SEG_DTYPE)
    for i in range(n):
        D = rng.uniform(d_lo, d_hi) * R
        a = math.radians(rng.uniform(0.0, 30.0))
        ph = rng.uniform(0.0, 2.0 * math.pi)
        P = C + D * np.array([math.sin(a) * math.cos(ph), math.sin(a) * math.sin(ph), math.cos(a)])
        u = (C - P) / D
        # tilt u by 0-10 degrees about a random axis perpendicular to it
        t = rng.normal(size=3)
        t -= (t @ u) * u
        t /= np.linalg.norm(t)
        b = math.radians(rng.uniform(0.0, 10.0))
        d = math.cos(b) * u + math.sin(b) * t
        s[i]["x"], s[i]["y"], s[i]["z"] = P
        s[i]["dx"], s[i]["dy"], s[i]["dz"] = d
    s["L"] = 1.0
    s["eps"] = 1e-5
    s["charge"] = -1
    par = I.Params(bunch=5.0, seed=seed)
    return s, atm, tels, par


def test_cut_loses_no_photons_beyond_fifteen_radii_as_the_paper_states():
    """The paper's rule of thumb for its angular cut (golden fixture
    tests/golden/angular_cut_rule.json): with a 6 degree cut a telescope more
    than ~15 radii away loses no photons.  Oracle: per-telescope cut on steps
    15-25 radii from a 300 m sphere -- same hits as without the cut, though the
    cut removes a good share of the steps; at 2-3 radii it loses photons."""
    import json
    rule = json.load(open(os.path.join(os.path.dirname(__file__), "golden", "angular_cut_rule.json")))
    s, atm, tels, par = _cut_rule_workload(1500, 3, rule["min_distance_in_radii"], 25.0)
    cut = dataclasses.replace(par, cut_mode=2, cut_deg=rule["cut_deg"])
    h0, c0, s0, st0 = O.trace(s, atm, tels, par)
    h1, c1, s1, st1 = O.trace(s, atm, tels, cut)
    nc0, _ = O.bunch_counts(s, atm, par, tels)
    nc1, _ = O.bunch_counts(s, atm, cut, tels)
    cut_steps = int(np.sum((nc0 > 0) & (nc1 == 0)))
    assert cut_steps > 0.2 * len(s) and len(h0) > 1000
    loss = 1.0 - s1.sum() / s0.sum()
    assert loss == rule["expected_photon_loss"], loss
    np.testing.assert_array_equal(h1, h0)
    # the rule is not vacuous: close to the telescope the same cut loses photons
    s, atm, tels, par = _cut_rule_workload(1500, 4, 2.0, 3.0)
    cut = dataclasses.replace(par, cut_mode=2, cut_deg=rule["cut_deg"])
    _, _, s0, _ = O.trace(s, atm, tels, par)
    _, _, s1, _ = O.trace(s, atm, tels, cut)
    assert s1.sum() < 0.99 * s0.sum()


def test_yield_near_threshold_matches_high_precision():
    """Sec. 1.2: N = 2 pi alpha z^2 (1/l1 - 1/l2)(1 - 1/(beta n)^2) L above the
    threshold beta n > 1, n = 1 + delta(h_mid).  Near the threshold the
    oracle's yield equals a 50-digit evaluation of that formula (written as
    printed, 1 - 1/(beta n)^2) to binary64's conditioning, 4e-16 over the
    relative distance r of beta n - 1 from the threshold (r down to 1e-9 of
    the refractivity), and both sides agree which steps emit."""
    mp = pytest.importorskip("mpmath")
    mp.mp.dps = 50
    atm = I.atmosphere_layered()
    par = I.Params(bunch=5.0)
    rng = np.random.default_rng(11)
    for r in (1e-2, 1e-4, 1e-6, 1e-8, 1e-9, -1e-8):
        s = np.zeros(1, dtype=I.SEG_DTYPE)
        s["x"], s["y"], s["z"] = rng.uniform(-100, 100), rng.uniform(-100, 100), rng.uniform(3e3, 1.5e4)
        s["dx"], s["dy"], s["dz"] = 0.01, -0.02, -1.0
        s["L"] = 2.5
        s["charge"] = -1
        d = [mp.mpf(float(s["dx"][0])), mp.mpf(float(s["dy"][0])), mp.mpf(float(s["dz"][0]))]
        nrm = mp.sqrt(sum(v * v for v in d))
        d = [v / nrm for v in d]
        L = mp.mpf(float(s["L"][0]))
        m = [mp.mpf(float(s[k][0])) + L / 2 * d[i] for i, k in enumerate(("x", "y", "z"))]
        RE = mp.mpf(atm.R_E)
        h = mp.sqrt(m[0] ** 2 + m[1] ** 2 + (m[2] + RE) ** 2) - RE
        i = int(np.searchsorted(np.asarray(atm.h_lo), float(h), side="right") - 1)
        delta = mp.mpf(atm.K) * mp.mpf(atm.b[i]) / (100 * mp.mpf(atm.c[i])) * mp.exp(-h / mp.mpf(atm.c[i]))
        s["eps"] = np.float32(float(delta * (1 - r) / (1 + delta)))
        beta_n = (1 - mp.mpf(float(s["eps"][0]))) * (1 + delta)
        y = O.yield_of(s[0], atm, par)
        if beta_n <= 1:
            assert y["Nc"] == 0.0 and y["n_c"] == 0.0
            continue
        N = 2 * mp.pi * mp.mpf(7.2973525643e-3) * (mp.mpf(1) / 300 - mp.mpf(1) / 600) * mp.mpf(10) ** 9 * \
            (1 - 1 / beta_n ** 2) * L
        # binary64 conditioning: delta's ~1e-16 relative error, times
        # delta / (beta n - 1) ~ 1 / r
        assert abs(y["Nc"] / float(N) - 1.0) < 4e-16 / abs(r) + 1e-12, (r, y["Nc"], float(N))

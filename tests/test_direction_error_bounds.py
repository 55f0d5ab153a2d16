"""Direction errors the classification carries as margins.

1. The MUFU azimuth (kAzErr = 1e-6 in the classification kernel).  The kernel forms the angle as
the binary32 product 6.28318531f * (u - 0.5f), u = m 2^-23 + 2^-24 the
Philox uniform, and takes the MUFU sine and cosine of it (each within
2^-21.41 of the value at its argument, documented for [-pi, pi]).  The
argument's rounding is checked here for every possible u; with the MUFU
error the unit vector (cos c, sin c) stays within 1e-6 of the exact one.

2. The Cherenkov cone from a binary32 beta n - 1 = g' (Sec. 1.2: cos theta_c
= 1/(beta n)), the exact g within eg of it: the kernel takes
eg (2.2 / sin theta_c' + 1.1) as the rays' direction error.  theta_c grows
like sqrt(2 g), so the largest change is toward g' - eg, about
2 eg / theta_c'; the set-up recomputes in binary64 every count its bound
leaves uncertain, which includes every step with g' <= 2 eg."""
import numpy as np


def test_binary32_azimuth_argument_for_every_uniform():
    m = np.arange(1 << 23, dtype=np.float64)
    u64 = m * 2.0 ** -23 + 2.0 ** -24
    u = u64.astype(np.float32)
    assert np.array_equal(u.astype(np.float64), u64)                  # the uniforms are exact in binary32
    du = u - np.float32(0.5)
    assert np.array_equal(du.astype(np.float64), u64 - 0.5)           # and so is u - 1/2
    arg = np.float32(6.28318531) * du                                  # the kernel's binary32 product
    exact = 2.0 * np.pi * (u64 - 0.5)
    err = np.abs(arg.astype(np.float64) - exact)
    assert np.abs(arg).max() <= np.pi                                  # inside the documented range
    assert err.max() <= 3.8e-7                                         # the argument's share of the bound
    # (cos, sin) of an angle off by e moves by at most e; the MUFU pair adds
    # at most sqrt(2) 2^-21.41 -- together below kAzErr
    assert err.max() + np.sqrt(2.0) * 2.0 ** -21.41 < 1.0e-6


def _theta(g):
    # cos theta_c = 1 / (1 + g) for beta n = 1 + g
    return np.arccos(1.0 / (1.0 + g))


def test_cone_angle_error_from_a_binary32_beta_n_minus_one():
    for eg in (1e-12, 1e-10, 1.2e-9, 1e-8, 1e-6):
        gp = eg * np.concatenate([np.linspace(1.0001, 3.0, 2001), np.logspace(0.5, 6, 2001)])
        thp = _theta(gp)
        bound = eg * (2.2 / np.sin(thp) + 1.1)
        for g in (gp - eg, gp + eg):
            err = np.abs(_theta(g) - thp)
            assert np.all(err <= bound), (eg, float((err / bound).max()))
        # the change toward g' - eg is what needs the factor 2: 1.1 would not do
        near = gp < 3.0 * eg
        old = eg * 1.1 * (1.0 / np.sin(thp[near]) + 1.0)
        assert np.any(np.abs(_theta(gp[near] - eg) - thp[near]) > old)


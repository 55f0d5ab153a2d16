"""The direction error the classification carries for its MUFU azimuth
(kAzErr = 1e-6 in the classification kernel).  The kernel forms the angle as
the binary32 product 6.28318531f * (u - 0.5f), u = m 2^-23 + 2^-24 the
Philox uniform, and takes the MUFU sine and cosine of it (each within
2^-21.41 of the value at its argument, documented for [-pi, pi]).  The
argument's rounding is checked here for every possible u; with the MUFU
error the unit vector (cos c, sin c) stays within 1e-6 of the exact one."""
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

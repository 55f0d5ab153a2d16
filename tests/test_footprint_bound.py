"""The footprint box of the whole-step skip (the classification kernel's
cone_lands_clear), in binary64 on the CPU.

A Cherenkov photon of a step with unit direction d leaves along
u(c) = cos(theta_c) d + sin(theta_c) (cos c e1 + sin c e2), where e1, e2 are
the first two columns of M_Rod for d (Sec. 1.2.1), and from height dz above
the plane z = h_obs it crosses the plane at dz u_xy / (-u_z) from its
emission point.  With v = (cos c, sin c), u_x / (-u_z) = (a0 + a . v) / (b0 + b . v),
and its range over c is spanned by the two roots of
(b0^2 - |b|^2) l^2 - 2 (a0 b0 - a . b) l + a0^2 - |a|^2 = 0.  These tests check that
statement against dense sampling of c, and that the box the kernel spans
from the two ends of a step holds every crossing of every emission point
in between."""
import numpy as np


def _frame(d):
    # M_Rod = 2 A A^T - 1 with A the unit bisector of d and -z (maps -z to d)
    A = np.array([d[0], d[1], d[2] - 1.0])
    A /= np.linalg.norm(A)
    e1 = 2.0 * A[0] * A - np.array([1.0, 0.0, 0.0])
    e2 = 2.0 * A[1] * A - np.array([0.0, 1.0, 0.0])
    return e1, e2


def _roots(a0, a1, a2, b0, b1, b2):
    A2 = b0 * b0 - (b1 * b1 + b2 * b2)
    B1 = a0 * b0 - (a1 * b1 + a2 * b2)
    C0 = a0 * a0 - (a1 * a1 + a2 * a2)
    sq = np.sqrt(max(B1 * B1 - A2 * C0, 0.0))
    return (B1 - sq) / A2, (B1 + sq) / A2


def _cases(rng, n):
    for _ in range(n):
        zen = np.radians(rng.uniform(0.0, 75.0))
        az = rng.uniform(0.0, 2 * np.pi)
        d = np.array([np.sin(zen) * np.cos(az), np.sin(zen) * np.sin(az), -np.cos(zen)])
        th = np.radians(rng.uniform(0.01, 2.0))
        yield d, th


def test_cone_vectors_are_unit_at_the_cherenkov_angle():
    rng = np.random.default_rng(3)
    c = np.linspace(0.0, 2 * np.pi, 257)
    for d, th in _cases(rng, 50):
        e1, e2 = _frame(d)
        assert abs(e1 @ d) < 1e-12 and abs(e2 @ d) < 1e-12 and abs(e1 @ e2) < 1e-12
        u = np.cos(th) * d[:, None] + np.sin(th) * (np.cos(c) * e1[:, None] + np.sin(c) * e2[:, None])
        np.testing.assert_allclose(np.linalg.norm(u, axis=0), 1.0, atol=1e-12)
        np.testing.assert_allclose(np.arccos(np.clip(d @ u, -1, 1)), th, atol=1e-7)


def test_ratio_range_is_spanned_by_the_roots():
    rng = np.random.default_rng(5)
    c = np.linspace(0.0, 2 * np.pi, 200_001)
    v = np.stack([np.cos(c), np.sin(c)])
    for d, th in _cases(rng, 60):
        e1, e2 = _frame(d)
        ct, st = np.cos(th), np.sin(th)
        b0, b1, b2 = -ct * d[2], -st * e1[2], -st * e2[2]
        assert b0 * b0 - (b1 * b1 + b2 * b2) > 0.0          # every photon heads down
        for k in (0, 1):                                      # x and y
            a0, a1, a2 = ct * d[k], st * e1[k], st * e2[k]
            r = (a0 + a1 * v[0] + a2 * v[1]) / (b0 + b1 * v[0] + b2 * v[1])
            lo, hi = _roots(a0, a1, a2, b0, b1, b2)
            span = hi - lo
            assert r.min() >= lo - 1e-12 * (1 + abs(lo)) and r.max() <= hi + 1e-12 * (1 + abs(hi))
            # the extremes are reached (dense sampling: within the sampling step's effect)
            assert r.min() - lo <= 1e-8 * max(span, 1e-3) + 1e-12
            assert hi - r.max() <= 1e-8 * max(span, 1e-3) + 1e-12


def test_box_of_the_step_ends_holds_every_crossing():
    rng = np.random.default_rng(7)
    c = np.linspace(0.0, 2 * np.pi, 721)
    v = np.stack([np.cos(c), np.sin(c)])
    for d, th in _cases(rng, 40):
        e1, e2 = _frame(d)
        ct, st = np.cos(th), np.sin(th)
        x0 = rng.uniform(-2000, 2000, size=2)
        z0 = rng.uniform(3000.0, 15000.0)                    # start height above the plane
        L = rng.uniform(0.5, 50.0)
        b0, b1, b2 = -ct * d[2], -st * e1[2], -st * e2[2]
        (xl, xh), (yl, yh) = (_roots(ct * d[k], st * e1[k], st * e2[k], b0, b1, b2) for k in (0, 1))
        dz0, dz1 = z0, z0 + L * d[2]
        x1 = x0 + L * d[:2]
        box = (min(x0[0] + dz0 * xl, x1[0] + dz1 * xl), max(x0[0] + dz0 * xh, x1[0] + dz1 * xh),
               min(x0[1] + dz0 * yl, x1[1] + dz1 * yl), max(x0[1] + dz0 * yh, x1[1] + dz1 * yh))
        u = ct * d[:, None] + st * (v[0] * e1[:, None] + v[1] * e2[:, None])
        for f in np.linspace(0.0, 1.0, 11):                  # emission points along the step
            p = np.array([x0[0], x0[1], z0]) + f * L * d
            X = p[0] + p[2] * u[0] / (-u[2])
            Y = p[1] + p[2] * u[1] / (-u[2])
            tol = 1e-9 * (1 + np.abs(X).max() + np.abs(Y).max())
            assert X.min() >= box[0] - tol and X.max() <= box[1] + tol
            assert Y.min() >= box[2] - tol and Y.max() <= box[3] + tol


def test_binary32_roots_with_their_margin_contain_the_exact_roots():
    """The kernel forms the roots in binary32 with approximate square roots and
    reciprocals (within a few ulp) and widens them by
    m = (sqrt(4e-7 (B1^2 + |A2 C0|)) + 4e-7 (|B1| + sqrt(disc))) / A2 + 1e-6.
    Emulated here in binary32 with every approximate result perturbed by up
    to 4 ulp: the widened interval holds the binary64 roots."""
    f = np.float32
    rng = np.random.default_rng(11)
    for d, th in _cases(rng, 4000):
        e1, e2 = _frame(d)
        ct, st = np.cos(th), np.sin(th)
        d32, e132, e232 = d.astype(f), e1.astype(f), e2.astype(f)
        ct32, st32 = f(ct), f(st)
        b0, b1, b2 = -ct32 * d32[2], -st32 * e132[2], -st32 * e232[2]
        A2 = b0 * b0 - (b1 * b1 + b2 * b2)
        iA = f(1.0) / A2 * f(1.0 + rng.uniform(-4, 4) * 2.0 ** -23)
        for k in (0, 1):
            a0, a1, a2 = ct32 * d32[k], st32 * e132[k], st32 * e232[k]
            B1 = a0 * b0 - (a1 * b1 + a2 * b2)
            C0 = a0 * a0 - (a1 * a1 + a2 * a2)
            disc = max(B1 * B1 - A2 * C0, f(0.0))
            sq = np.sqrt(disc) * f(1.0 + rng.uniform(-4, 4) * 2.0 ** -23)
            m = (np.sqrt(f(4.0e-7) * (B1 * B1 + abs(A2 * C0))) + f(4.0e-7) * (abs(B1) + sq)) * iA + f(1.0e-6)
            lo, hi = (B1 - sq) * iA - m, (B1 + sq) * iA + m
            lo64, hi64 = _roots(ct * d[k], st * e1[k], st * e2[k], -ct * d[2], -st * e1[2], -st * e2[2])
            assert lo <= lo64 and hi >= hi64, (lo, lo64, hi, hi64)

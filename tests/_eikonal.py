"""Brute-force ray tracing of the eikonal equation, used only to pin the
oracle's invariant quadrature.

The ray equation d(n t)/ds = grad n is integrated in Cartesian coordinates by
classical fourth-order Runge-Kutta with a small fixed step, carrying the
optical path int n ds and the density-weighted path int rho/rho_ref ds.  It
knows nothing of the Snell/Bouguer invariant the oracle uses.
"""
import numpy as np


def _rho_and_grad(atm, h):
    """rho(h) and d rho / dh for the layered model (vectorised)."""
    h_lo = np.asarray(atm.h_lo, dtype=np.float64)
    i = np.clip(np.searchsorted(h_lo, h, side="right") - 1, 0, len(h_lo) - 1)
    b = np.asarray(atm.b)[i]
    c = np.asarray(atm.c)[i]
    rho = b / (100.0 * c) * np.exp(-h / c)
    rho = np.where(h >= atm.h_top, 0.0, rho)
    return rho, -rho / c


def _alt_and_up(atm, r):
    if atm.spherical:
        R = r.copy()
        R[:, 2] += atm.R_E
        rn = np.linalg.norm(R, axis=1)
        return rn - atm.R_E, R / rn[:, None]
    up = np.zeros_like(r)
    up[:, 2] = 1.0
    return r[:, 2].copy(), up


def _deriv(atm, y):
    r, v = y[:, 0:3], y[:, 3:6]
    h, up = _alt_and_up(atm, r)
    rho, drho = _rho_and_grad(atm, h)
    n = 1.0 + atm.K * rho
    gradn = (atm.K * drho)[:, None] * up
    out = np.empty_like(y)
    out[:, 0:3] = v / n[:, None]
    out[:, 3:6] = gradn
    out[:, 6] = n                       # d(optical path)/ds
    out[:, 7] = rho / atm.rho_ref       # d(density path)/ds
    return out


def trace(atm, r_e, d, ds=1.0, refraction=True):
    """Trace rays from r_e (N,3) along unit d (N,3) to the observation level.

    Returns landing points (N,3), directions (N,3), optical path (N,),
    density-weighted path (N,).  Refraction off: straight lines, n only in
    the optical path.
    """
    r_e = np.atleast_2d(np.asarray(r_e, dtype=np.float64))
    d = np.atleast_2d(np.asarray(d, dtype=np.float64))
    d = d / np.linalg.norm(d, axis=1)[:, None]
    N = len(r_e)
    h0, _ = _alt_and_up(atm, r_e)
    rho0, _ = _rho_and_grad(atm, h0)
    n0 = 1.0 + atm.K * rho0
    y = np.zeros((N, 8))
    y[:, 0:3] = r_e
    y[:, 3:6] = d * (n0[:, None] if refraction else 1.0)
    active = np.ones(N, dtype=bool)
    P = np.zeros((N, 3))
    D = np.zeros((N, 3))
    Lopt = np.zeros(N)
    Ltau = np.zeros(N)

    def f(yy):
        if refraction:
            return _deriv(atm, yy)
        out = _deriv(atm, yy)
        h, _ = _alt_and_up(atm, yy[:, 0:3])
        out[:, 0:3] = yy[:, 3:6]
        out[:, 3:6] = 0.0
        return out

    for _ in range(10_000_000):
        if not active.any():
            break
        ya = y[active]
        k1 = f(ya)
        k2 = f(ya + 0.5 * ds * k1)
        k3 = f(ya + 0.5 * ds * k2)
        k4 = f(ya + ds * k3)
        yn = ya + ds / 6.0 * (k1 + 2 * k2 + 2 * k3 + k4)
        hn, _ = _alt_and_up(atm, yn[:, 0:3])
        crossed = hn <= atm.h_obs
        idx = np.nonzero(active)[0]
        if crossed.any():
            # finish the crossing rays with a shortened step found by bisection
            for j in np.nonzero(crossed)[0]:
                lo, hi = 0.0, ds
                y0 = ya[j:j + 1]
                for _ in range(60):
                    mid = 0.5 * (lo + hi)
                    a1 = f(y0)
                    a2 = f(y0 + 0.5 * mid * a1)
                    a3 = f(y0 + 0.5 * mid * a2)
                    a4 = f(y0 + mid * a3)
                    ym = y0 + mid / 6.0 * (a1 + 2 * a2 + 2 * a3 + a4)
                    hm, _ = _alt_and_up(atm, ym[:, 0:3])
                    if hm[0] > atm.h_obs:
                        lo = mid
                    else:
                        hi = mid
                k = idx[j]
                P[k] = ym[0, 0:3]
                vv = ym[0, 3:6]
                D[k] = vv / np.linalg.norm(vv)
                Lopt[k] = ym[0, 6]
                Ltau[k] = ym[0, 7]
            active[idx[crossed]] = False
        y[idx[~crossed]] = yn[~crossed]
    return P, D, Lopt, Ltau

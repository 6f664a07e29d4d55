"""Macroscopic moments, Hermite equilibria and BGK collision (Sec. 2).

Units (reading of Eqs. (feq-2)-(feq-4)): the printed equilibria carry "1 + u.c" with no 1/c_s^2
factor, so they are read in normalized units where c_s = 1, the reference temperature is 1,
and the abscissae are xi_i = r e_i (r from stencil.py). All prefactors 1/(n! c_s^(2n-2)) then
reduce to 1/n!.

Equilibrium, D = 2, with s = xi.u, u2 = u.u, c2 = xi.xi, theta = T - 1:
  order 2 (Eq. feq-2): w rho [1 + s + (s^2 - u2 + theta (c2 - 2)) / 2]
  order 3 (Eq. feq-3): + w rho s (s^2 - 3 u2 + 3 theta (c2 - 4)) / 6
  order 4 (Eq. feq-4): + w rho [s^4 - 6 s^2 u2 + 3 u2^2
                                + 6 theta (s^2 (c2 - 6) + u2 (4 - c2))
                                + 3 theta^2 (c2^2 - 8 c2 + 8)] / 24
Reading: Eq. (feq-4) prints (c2 - 4) in the mixed theta-term; the fourth Hermite polynomial
contracted with delta u u in D = 2 gives (c2 - D - 4) = (c2 - 6), and only that value lets the
equilibrium return the density it was built from (Sec. 2 requires Eq. (macro) to hold). The
printed constant is kept available as `mixed4_shift` so a test can show it breaks Eq. (macro).

Moments, Eq. (macro), with d = D = 2 and e = (d/2) T:
  rho = sum f,  rho u = sum f xi,  and the energy moment read as the kinetic definition
  sum f |xi - u|^2 = D rho T (for d = 2 this equals the printed d rho e with e = (d/2) T).
"""
from __future__ import annotations

import numpy as np

D = 2


def moments(f: np.ndarray, xi: np.ndarray):
    """Eq. (macro): f (q, ...) -> rho, u (2, ...), T."""
    rho = f.sum(axis=0)
    j = np.tensordot(xi.T, f, axes=(1, 0))            # (2, ...)
    u = j / rho
    dev2 = ((xi[:, 0].reshape((-1,) + (1,) * (f.ndim - 1)) - u[0]) ** 2
            + (xi[:, 1].reshape((-1,) + (1,) * (f.ndim - 1)) - u[1]) ** 2)
    T = (f * dev2).sum(axis=0) / (D * rho)
    return rho, u, T


def feq(rho, u, T, xi: np.ndarray, w: np.ndarray, order: int, mixed4_shift: float = 6.0):
    """Eqs. (feq-2), (feq-3), (feq-4): equilibrium populations, shape (q, ...)."""
    sh = (-1,) + (1,) * np.ndim(rho)
    xx = xi[:, 0].reshape(sh)
    xy = xi[:, 1].reshape(sh)
    ww = w.reshape(sh)
    s = xx * u[0] + xy * u[1]                 # u . c_i
    u2 = u[0] * u[0] + u[1] * u[1]            # u^2
    c2 = xx * xx + xy * xy                    # c_i^2
    th = T - 1.0
    poly = 1.0 + s + 0.5 * (s * s - u2 + th * (c2 - 2.0))                       # Eq. (feq-2)
    if order >= 3:
        poly = poly + s / 6.0 * (s * s - 3.0 * u2 + 3.0 * th * (c2 - 4.0))      # Eq. (feq-3)
    if order >= 4:
        poly = poly + (s ** 4 - 6.0 * s * s * u2 + 3.0 * u2 * u2                 # Eq. (feq-4)
                       + 6.0 * th * (s * s * (c2 - mixed4_shift) + u2 * (4.0 - c2))
                       + 3.0 * th * th * (c2 * c2 - 8.0 * c2 + 8.0)) / 24.0
    return ww * rho * poly


def bgk(f, f_eq, tau):
    """Omega^BGK of Eq. (lbe): post-collision f + Omega = f - (f - f_eq) / tau."""
    return f - (f - f_eq) / tau

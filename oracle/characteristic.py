"""Characteristic boundary conditions of Sec. 4 ("Characteristic BC").

Macroscopic state U = (rho, u_x, u_y, T), ideal gas P = rho T c_s^2 with c_s = 1 (normalized
units), internal energy e = (D/2) T, D = 2, so gamma = (D + 2)/D = 2 and the sound speed is
c = sqrt(gamma T).

Inviscid primitive equations dU/dt = -A dU/dx - B dU/dy (Eq. NSF-CHAR with the transverse
part written out). A = S^-1 Lambda S, Lambda = diag(u_n - c, u_n, u_n, u_n + c), where u_n is
the velocity along the boundary normal axis. Wave amplitudes L = Lambda S dU/dn (normal axis),
transverse amplitudes T_cal = S B dU/dt_axis (tangential axis), so that
Eq. (thermal_CBC_macro_evo):  dU/dt = -S^-1 (L_bar + T_cal)   (viscous part V = 0: the paper
                                                             gives no formula for it)
Eq. (thermal_LODI_macro_evo): dU/dt = -S^-1 L_bar.

Readings where the paper defers to its ref. [klass-camwa-2024] (not available):
* Boundary nodes are the M = 3 layers outside F. Each edge node carries its own target U_tgt,
  advanced over one time step by classical RK4 with the fluid moments frozen at time n
  (solver.py; explicit Euler is unstable here).
* Normal derivative at a boundary node x_b: one-sided second order along the outward normal n,
  (3 U(x_b) - 4 U(x_b - n) + U(x_b - 2n)) / 2, using U_tgt for boundary nodes and the moments
  for fluid nodes. Tangential derivative: central along the boundary layer, one-sided second
  order at the two ends of the layer (central with wrap-around along a periodic axis).
* Lattice spacing: a population with xi_i = r e_i crosses e_i nodes per step, so one node is r
  normalized length units and d/dx = (1/r) d/d(node index).
* Incoming waves are those with Lambda_k * (outward sign) < 0.
* PNR (Eq. PNR): incoming L_bar = 0, used with the LODI evolution.
* CBC relax (Eq. CBC-Relax), used with the CBC evolution. As printed,
  L_bar_inc = (1 - Ma) T_cal_inc; together with dU/dt = -S^-1 (L_bar + T_cal) that would add the
  transverse term twice. Reading (transverse damping of the cited Yoo & Im scheme):
  L_bar_inc = -(1 - beta) T_cal_inc with beta = Ma; beta = 1 leaves the incoming transverse
  term untouched, beta = 0 freezes the incoming characteristic. The printed sign is
  available with relax_sign = +1.
* Corner nodes (outside F along both axes) use the zero-gradient copy.

PML-aware characteristic BC (Appendix, Eq. NSF-CHAR-PML). The PML adds the velocity moments of
Omega^PML to the conservation laws: terms I (gradient part), II (f_hat part), III (Q part).
Readings: the source of a band node is the moment of the selected parts of Omega^PML, exactly
as the discrete collision applies them (Eq. pml-general, per time step), at the nearest fluid
node x_f (the outermost PML layer, where sigma = sigma_max), with the sign of the collision
term (a damping; the printed "+" of Eq. NSF-CHAR-PML is available as an option); the conserved-variable
source (mass, momentum, energy = sum f |xi|^2 / 2) is mapped to the primitive variables by the
exact chain rule at the time-n state of x_f (the printed scaling vector S is its diagonal
part), and added to dU/dt of every layer of the band, frozen over the Runge-Kutta stages like
the fluid moments.
"""
from __future__ import annotations

import numpy as np

D = 2
GAMMA = (D + 2.0) / D


def jacobian(U: np.ndarray, axis: int) -> np.ndarray:
    """Primitive Euler flux Jacobian along `axis` (0 = x, 1 = y); U (..., 4) -> (..., 4, 4).

    rho_t + u_a rho_a + rho (u_a)_a = 0;  (u_a)_t + u_a (u_a)_a + P_a / rho = 0;
    (u_t)_t + u_a (u_t)_a = 0;  T_t + u_a T_a + (2/D) T (u_a)_a = 0;  P_a = T rho_a + rho T_a.
    """
    rho, T = U[..., 0], U[..., 3]
    un = U[..., 1 + axis]
    n = 1 + axis          # index of the normal velocity in U
    A = np.zeros(U.shape[:-1] + (4, 4))
    A[..., 0, 0] = un
    A[..., 0, n] = rho
    A[..., n, 0] = T / rho
    A[..., n, n] = un
    A[..., n, 3] = 1.0
    t = 2 - axis          # index of the tangential velocity in U
    A[..., t, t] = un
    A[..., 3, n] = (2.0 / D) * T
    A[..., 3, 3] = un
    return A


def eigen(U: np.ndarray, axis: int):
    """Left eigenvectors S (rows) and eigenvalues Lambda of jacobian(U, axis)."""
    rho, T = U[..., 0], U[..., 3]
    un = U[..., 1 + axis]
    c = np.sqrt(GAMMA * T)
    n, t = 1 + axis, 2 - axis
    S = np.zeros(U.shape[:-1] + (4, 4))
    # acoustic wave u_n - c:  dP - rho c du_n
    S[..., 0, 0] = T
    S[..., 0, n] = -rho * c
    S[..., 0, 3] = rho
    # entropy wave u_n:  (2/D) T drho - rho dT
    S[..., 1, 0] = (2.0 / D) * T
    S[..., 1, 3] = -rho
    # shear wave u_n:  du_t
    S[..., 2, t] = 1.0
    # acoustic wave u_n + c:  dP + rho c du_n
    S[..., 3, 0] = T
    S[..., 3, n] = rho * c
    S[..., 3, 3] = rho
    lam = np.stack([un - c, un, un, un + c], axis=-1)
    return S, lam


def rate(U, dUn, dUt, axis, out_sign, variant, beta, r, relax_sign=-1.0):
    """dU/dt at boundary nodes.

    U (n, 4) state at the node; dUn, dUt (n, 4) derivatives per node index along the normal
    axis `axis` and the tangential axis; out_sign = +1/-1 the outward direction along `axis`;
    variant 0 = PNR with LODI evolution, 1 = CBC relax with the CBC evolution.
    """
    S, lam = eigen(U, axis)
    Sinv = np.linalg.inv(S)
    L = lam * np.einsum("nij,nj->ni", S, dUn / r)                    # Lambda S dU/dx
    incoming = lam * out_sign < 0.0
    if variant == 0:
        Lbar = np.where(incoming, 0.0, L)                               # Eq. (PNR)
        return -np.einsum("nij,nj->ni", Sinv, Lbar)                     # Eq. (LODI evo)
    B = jacobian(U, 1 - axis)
    Tcal = np.einsum("nij,njk,nk->ni", S, B, dUt / r)                   # S B dU/dy
    Lbar = np.where(incoming, relax_sign * (1.0 - beta) * Tcal, L)      # Eq. (CBC-Relax)
    return -np.einsum("nij,nj->ni", Sinv, Lbar + Tcal)                  # Eq. (CBC evo)


def one_sided(u0, u1, u2):
    """Second-order one-sided derivative toward u0 from u1 = U(x - n), u2 = U(x - 2n)."""
    return 0.5 * (3.0 * u0 - 4.0 * u1 + u2)


def tangential(Uline: np.ndarray, periodic: bool = False) -> np.ndarray:
    """d/d(index) along a line of nodes (m, 4): central inside, one-sided at the two ends, or
    central everywhere with wrap-around when the line is periodic."""
    if periodic:
        return 0.5 * (np.roll(Uline, -1, axis=0) - np.roll(Uline, 1, axis=0))
    d = np.zeros_like(Uline)
    d[1:-1] = 0.5 * (Uline[2:] - Uline[:-2])
    d[0] = -one_sided(Uline[0], Uline[1], Uline[2])
    d[-1] = one_sided(Uline[-1], Uline[-2], Uline[-3])
    return d


def conserved_to_primitive_rate(s_mass, s_mom, s_energy, U):
    """d(rho, u_x, u_y, T)/dt from d(rho, rho u, E)/dt at state U (..., 4), E = rho (u^2 + D T)/2.
    d rho = s_m;  rho du = s_mom - u s_m;  (D/2) rho dT = s_E - u . s_mom + (u^2/2 - (D/2) T) s_m."""
    rho, ux, uy, T = U[..., 0], U[..., 1], U[..., 2], U[..., 3]
    u2 = ux * ux + uy * uy
    dux = (s_mom[0] - ux * s_mass) / rho
    duy = (s_mom[1] - uy * s_mass) / rho
    dT = (s_energy - ux * s_mom[0] - uy * s_mom[1] + (0.5 * u2 - 0.5 * D * T) * s_mass) \
        / (0.5 * D * rho)
    return np.stack([s_mass, dux, duy, dT], axis=-1)

"""Perfectly matched layer of Sec. 3.

Geometry (Fig. 2): the bulk B of nx x ny nodes is padded by W PML layers on every side; the
fluid region F = B + P has Lx x Ly = (nx + 2W) x (ny + 2W) nodes. The PML layer index of a node
is i = 1 .. W counted outward from the bulk (Eq. PML_ramp). Reading for the corner regions,
where a node is outside the bulk along both axes: i = max(i_x, i_y) (Chebyshev distance from
the bulk). Exponent: Eq. (PML_ramp) uses p = 2; the profile exponent is a parameter p.

Auxiliary variable Q, Eq. (PMLQ) dQ/dt = f_hat with the trapezoidal rule. The printed discrete
rule lacks the previous value of Q; reading: Q^n = Q^(n-1) + (f_hat^(n-1) + f_hat^n) / 2 with
Q^0 = 0, where f_hat = f_eq - f_eq_bar (Eq. decomp-NJ) and f_eq_bar is the equilibrium of the
constant mean state. Q is kept on P and on the ring of bulk nodes next to P, because the
central difference of the innermost PML layer reaches into that ring ("central differences
for all other cases"); Omega^PML itself acts on P only.

Gradient: Eq. (FD-dx-center) everywhere except along an axis whose outward neighbour lies
outside F (outermost layer), where Eq. (FD-dx-bw) is used along the outward normal n:
dQ/dn = (3 Q(x) - 4 Q(x - n) + Q(x - 2n)) / 2, dQ/dx_a = n_a dQ/dn.

Collision term, Eq. (PMLCOLL) with sigma_x = sigma_y = sigma:
Omega^PML_i = -sigma (c_i . grad Q_i + 2 f_hat_i + sigma Q_i), with c_i the integer lattice
velocity e_i (the discrete equation is written with dx = dt = 1), sigma per time step.
"""
from __future__ import annotations

import numpy as np


def _axis_layers(L, W):
    """PML layer index along one axis: W - (distance to the nearer end), 0 outside the PML."""
    if W == 0:
        return np.zeros(L, dtype=np.int64)
    z = np.arange(L)
    return np.maximum(0, np.maximum(W - z, z - (L - 1 - W)))


def layer_index(Lx: int, Ly: int, W: int, Wy: int = None) -> np.ndarray:
    """(Ly, Lx) int array: PML layer index i in 1..W on P, 0 in the bulk (equal widths)."""
    Wy = W if Wy is None else Wy
    return np.maximum(_axis_layers(Lx, W)[None, :], _axis_layers(Ly, Wy)[:, None])


def sigma_field(Lx, Ly, W, sigma_max, power, Wy=None):
    """Eq. (PML_ramp): sigma = sigma_max (i / W)^p on P, 0 in the bulk. With different widths
    on the x edges (W) and y edges (Wy) the layer fraction is max(i_x / W, i_y / Wy)."""
    Wy = W if Wy is None else Wy
    fx = _axis_layers(Lx, W) / W if W > 0 else np.zeros(Lx)
    fy = _axis_layers(Ly, Wy) / Wy if Wy > 0 else np.zeros(Ly)
    frac = np.maximum(fx[None, :], fy[:, None])
    return np.where(frac > 0, sigma_max * frac ** power, 0.0)


def in_pml(Lx, Ly, W, Wy=None) -> np.ndarray:
    """Nodes of P (PML layer index >= 1 along some axis)."""
    Wy = W if Wy is None else Wy
    return (_axis_layers(Lx, W)[None, :] > 0) | (_axis_layers(Ly, Wy)[:, None] > 0)


def q_support(Lx, Ly, W, Wy=None) -> np.ndarray:
    """Nodes where Q is kept: P plus the bulk nodes one step inside it along each PML axis (the
    ring the central difference of the innermost layer reaches)."""
    Wy = W if Wy is None else Wy
    x = np.arange(Lx)
    y = np.arange(Ly)
    dx = np.minimum(x, Lx - 1 - x)
    dy = np.minimum(y, Ly - 1 - y)
    sx = (dx <= W) if W > 0 else np.zeros(Lx, dtype=bool)
    sy = (dy <= Wy) if Wy > 0 else np.zeros(Ly, dtype=bool)
    return sx[None, :] | sy[:, None]


def trapezoid_update(Q_prev, fhat_prev, fhat_now):
    """Q^n = Q^(n-1) + (f_hat^(n-1) + f_hat^n) / 2."""
    return Q_prev + 0.5 * (fhat_prev + fhat_now)


def gradient(Q: np.ndarray, periodic_y: bool = False):
    """Per-axis finite differences of Q (q, Ly, Lx) over F.

    Central differences Eq. (FD-dx-center) in the interior; at the outermost layer of F the
    one-sided Eq. (FD-dx-bw) along the outward normal. Along a periodic y axis the central
    difference wraps. Values are only used on P.
    """
    gx = np.zeros_like(Q)
    gy = np.zeros_like(Q)
    gx[:, :, 1:-1] = 0.5 * (Q[:, :, 2:] - Q[:, :, :-2])
    # right edge: outward normal +x; left edge: outward normal -x
    gx[:, :, -1] = +0.5 * (3.0 * Q[:, :, -1] - 4.0 * Q[:, :, -2] + Q[:, :, -3])
    gx[:, :, 0] = -0.5 * (3.0 * Q[:, :, 0] - 4.0 * Q[:, :, 1] + Q[:, :, 2])
    if periodic_y:
        gy[:] = 0.5 * (np.roll(Q, -1, axis=1) - np.roll(Q, 1, axis=1))
    else:
        gy[:, 1:-1, :] = 0.5 * (Q[:, 2:, :] - Q[:, :-2, :])
        gy[:, -1, :] = +0.5 * (3.0 * Q[:, -1, :] - 4.0 * Q[:, -2, :] + Q[:, -3, :])
        gy[:, 0, :] = -0.5 * (3.0 * Q[:, 0, :] - 4.0 * Q[:, 1, :] + Q[:, 2, :])
    return gx, gy


def omega_pml(e: np.ndarray, gx, gy, fhat, Q, sigma):
    """Eq. (PMLCOLL): -sigma (c_i . grad Q_i + 2 f_hat_i + sigma Q_i), shape (q, Ly, Lx)."""
    ex = e[:, 0].astype(np.float64).reshape(-1, 1, 1)
    ey = e[:, 1].astype(np.float64).reshape(-1, 1, 1)
    return -sigma * (ex * gx + ey * gy + 2.0 * fhat + sigma * Q)

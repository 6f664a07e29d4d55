"""Perfectly matched layer of Sec. 3.

Geometry (Fig. 2): the bulk B of nx x ny nodes is padded by PML layers; the fluid region
F = B + P has Lx x Ly nodes. Widths are per edge, (W_w, W_e, W_s, W_n), so that the damping
zones away from the outlet can be thinner (the closing remark of Sec. 5); equal widths W on
every side are the paper's setting, Lx x Ly = (nx + 2W) x (ny + 2W). The PML layer index of a
node along an axis is i = 1 .. W_side counted outward from the bulk (Eq. PML_ramp), and its
layer fraction along that axis is i / W_side.

Absorption coefficients. Eq. (pml-general) has sigma_x and sigma_y; the paper then sets
sigma_x = sigma_y = sigma (Eq. PMLCOLL). Default ("isotropic") reading: sigma_x = sigma_y =
sigma_max f^p with f = max(f_x, f_y) the larger layer fraction (with equal widths this is the
Chebyshev distance from the bulk, i = max(i_x, i_y), in the corners). Option "split": the
general form with sigma_x = sigma_max f_x^p and sigma_y = sigma_max f_y^p (each nonzero only
in the slab of its own axis; both in the corners). Exponent: Eq. (PML_ramp) uses p = 2; the
profile exponent is a parameter p.

Auxiliary variable Q, Eq. (PMLQ) dQ/dt = f_hat with the trapezoidal rule. The printed discrete
rule lacks the previous value of Q; reading: Q^n = Q^(n-1) + (f_hat^(n-1) + f_hat^n) / 2 with
Q^0 = 0, where f_hat = f_eq - f_eq_bar (Eq. decomp-NJ) and f_eq_bar is the equilibrium of the
constant mean state. Q is kept on P and on the ring of bulk nodes next to P, because the
central difference of the innermost PML layer reaches into that ring ("central differences
for all other cases"); Omega^PML itself acts on P only.

Gradient: Eq. (FD-dx-center) everywhere except along an axis whose outward neighbour lies
outside F (outermost layer), where Eq. (FD-dx-bw) is used along the outward normal n:
dQ/dn = (3 Q(x) - 4 Q(x - n) + Q(x - 2n)) / 2, dQ/dx_a = n_a dQ/dn.

Link-integrated gradient (an option, not the printed scheme). The printed per-axis central
differences make the scheme linearly unstable for every sigma > 0 (von Neumann analysis in the
tests): the lattice streams each population exactly along its link while grad Q is taken by
differences that do not follow the link, so at wavenumbers where the two disagree (e.g.
k = 2 pi / 3 for the speed-3 populations of D2Q37, which alias to zero phase) the identity
that makes the continuous PML stable is lost. The option pml_grad = "link" replaces
c_i . grad Q_i by its exact integral along the path the population travels in one step,
Q_i(x + e_i) - Q_i(x); for a field linear in x this equals the printed form. Q is then needed up to
M nodes away from P (inside the bulk and in the boundary band Gamma), and is integrated there by
the same trapezoidal rule from the moments of those nodes.

Collision term, Eq. (pml-general):
Omega^PML_i = -(sigma_y c_ix dQ_i/dx + sigma_x c_iy dQ_i/dy + (sigma_x + sigma_y) f_hat_i
               + sigma_x sigma_y Q_i),
which for sigma_x = sigma_y = sigma is Eq. (PMLCOLL), -sigma (c_i . grad Q_i + 2 f_hat_i +
sigma Q_i); c_i is the integer lattice velocity e_i (the discrete equation is written with
dx = dt = 1), sigma per time step.
"""
from __future__ import annotations

import numpy as np


def widths4(W, Wy=None):
    """(W_w, W_e, W_s, W_n) from an int W (all edges, or the W/E edges when Wy is given) or
    a 4-tuple."""
    if np.ndim(W) == 1:
        if Wy is not None:
            raise ValueError("give either per-edge widths or W and Wy")
        w = tuple(int(v) for v in W)
        if len(w) != 4:
            raise ValueError("per-edge widths are (W_w, W_e, W_s, W_n)")
        return w
    Wy = W if Wy is None else Wy
    return (int(W), int(W), int(Wy), int(Wy))


def _axis_layers(L, lo, hi):
    """(layer index, layer fraction) along one axis with lo layers at its start and hi at its
    end: i = lo - z on the low side, z - (L - 1 - hi) on the high side, 0 in between."""
    z = np.arange(L)
    i_lo = np.maximum(0, lo - z) if lo > 0 else np.zeros(L, dtype=np.int64)
    i_hi = np.maximum(0, z - (L - 1 - hi)) if hi > 0 else np.zeros(L, dtype=np.int64)
    frac = np.zeros(L)
    if lo > 0:
        frac = np.where(i_lo > 0, i_lo / lo, frac)
    if hi > 0:
        frac = np.where(i_hi > 0, i_hi / hi, frac)
    return i_lo + i_hi, frac


def layer_index(Lx: int, Ly: int, W, Wy=None) -> np.ndarray:
    """(Ly, Lx) int array: max(i_x, i_y) on P, 0 in the bulk."""
    ww, we, ws, wn = widths4(W, Wy)
    ix, _ = _axis_layers(Lx, ww, we)
    iy, _ = _axis_layers(Ly, ws, wn)
    return np.maximum(ix[None, :], iy[:, None])


def sigma_fields(Lx, Ly, W, sigma_max, power, Wy=None, split=False):
    """(sigma_x, sigma_y), each (Ly, Lx): Eq. (PML_ramp) with the reading of the module
    docstring ("isotropic": both equal sigma_max max(f_x, f_y)^p; "split": per axis)."""
    ww, we, ws, wn = widths4(W, Wy)
    _, fx = _axis_layers(Lx, ww, we)
    _, fy = _axis_layers(Ly, ws, wn)
    FX = np.broadcast_to(fx[None, :], (Ly, Lx))
    FY = np.broadcast_to(fy[:, None], (Ly, Lx))
    if split:
        return (np.where(FX > 0, sigma_max * FX ** power, 0.0),
                np.where(FY > 0, sigma_max * FY ** power, 0.0))
    f = np.maximum(FX, FY)
    s = np.where(f > 0, sigma_max * f ** power, 0.0)
    return s, s.copy()


def sigma_field(Lx, Ly, W, sigma_max, power, Wy=None):
    """Eq. (PML_ramp) with sigma_x = sigma_y: sigma_max max(f_x, f_y)^p on P, 0 in the bulk."""
    return sigma_fields(Lx, Ly, W, sigma_max, power, Wy)[0]


def in_pml(Lx, Ly, W, Wy=None) -> np.ndarray:
    """Nodes of P (PML layer index >= 1 along some axis)."""
    return layer_index(Lx, Ly, W, Wy) > 0


def q_support(Lx, Ly, W, Wy=None) -> np.ndarray:
    """Nodes where Q is kept: P plus the bulk nodes one step inside it along each PML edge (the
    ring the central difference of the innermost layer reaches)."""
    ww, we, ws, wn = widths4(W, Wy)
    x = np.arange(Lx)
    y = np.arange(Ly)
    sx = np.zeros(Lx, dtype=bool)
    sy = np.zeros(Ly, dtype=bool)
    if ww > 0:
        sx |= x <= ww
    if we > 0:
        sx |= Lx - 1 - x <= we
    if ws > 0:
        sy |= y <= ws
    if wn > 0:
        sy |= Ly - 1 - y <= wn
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


def omega_pml_terms(e: np.ndarray, gx, gy, fhat, Q, sigma_x, sigma_y=None):
    """The three parts of Eq. (pml-general), each (q, Ly, Lx): the gradient part
    -(sigma_y c_x dQ/dx + sigma_x c_y dQ/dy), the f_hat part -(sigma_x + sigma_y) f_hat and the
    Q part -sigma_x sigma_y Q (their moments are the terms I, II, III of Eq. NSF-CHAR-PML)."""
    sigma_y = sigma_x if sigma_y is None else sigma_y
    ex = e[:, 0].astype(np.float64).reshape(-1, 1, 1)
    ey = e[:, 1].astype(np.float64).reshape(-1, 1, 1)
    return (-(sigma_y * ex * gx + sigma_x * ey * gy), -(sigma_x + sigma_y) * fhat,
            -(sigma_x * sigma_y) * Q)


def omega_pml(e: np.ndarray, gx, gy, fhat, Q, sigma_x, sigma_y=None):
    """Eq. (pml-general), shape (q, Ly, Lx):
    -(sigma_y c_x dQ/dx + sigma_x c_y dQ/dy + (sigma_x + sigma_y) f_hat + sigma_x sigma_y Q);
    sigma_y defaults to sigma_x (Eq. PMLCOLL)."""
    sigma_y = sigma_x if sigma_y is None else sigma_y
    ex = e[:, 0].astype(np.float64).reshape(-1, 1, 1)
    ey = e[:, 1].astype(np.float64).reshape(-1, 1, 1)
    return -(sigma_y * ex * gx + sigma_x * ey * gy + (sigma_x + sigma_y) * fhat
             + sigma_x * sigma_y * Q)


def link_difference(QG: np.ndarray, e: np.ndarray, M: int, Ly: int, Lx: int) -> np.ndarray:
    """Q_i(x + e_i) - Q_i(x) for every node x of F, shape (q, Ly, Lx); QG is Q on the whole
    grid G = F + M boundary layers, shape (q, Ly + 2M, Lx + 2M) (node (x, y) of F at
    [M + y, M + x])."""
    out = np.empty((QG.shape[0], Ly, Lx))
    for i, (ex, ey) in enumerate(e):
        ahead = QG[i, M + ey:M + ey + Ly, M + ex:M + ex + Lx]
        here = QG[i, M:M + Ly, M:M + Lx]
        out[i] = ahead - here
    return out


def omega_pml_link_terms(link, fhat, Q, sigma):
    """The three parts of Eq. (PMLCOLL) with c_i . grad Q_i replaced by the link difference
    `link` (q, Ly, Lx): -sigma link, -2 sigma f_hat, -sigma^2 Q."""
    return (-sigma * link, -2.0 * sigma * fhat, -(sigma * sigma) * Q)

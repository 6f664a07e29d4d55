"""Error metrics of Sec. 5 ("Reference Simulation").

e_Z       = ( sum_(x,y) ( |Z - Z_ref| / |Z_ref| )^2 )^(1/2)     (printed without 1/N)
e~_Z(x,y) = |Z - Z_ref| / |Z_ref|
e_bar_Z   = mean of e_Z over the sampled iterations;  C_Z = e_bar_Z / e_bar_Z^ZG.
Normwise relative L2 ||Z - Z_o||_2 / ||Z_o||_2 is the parity measure between two solvers.
"""
from __future__ import annotations

import numpy as np


def e_Z(Z, Zref):
    return float(np.sqrt(np.sum((np.abs(Z - Zref) / np.abs(Zref)) ** 2)))


def pointwise(Z, Zref):
    return np.abs(Z - Zref) / np.abs(Zref)


def rel_l2(Z, Zref):
    den = np.sqrt(np.sum(Zref * Zref))
    return float(np.sqrt(np.sum((Z - Zref) ** 2)) / den) if den > 0 else float(
        np.sqrt(np.sum((Z - Zref) ** 2)))


def C_Z(ebar, ebar_zg):
    return ebar / ebar_zg

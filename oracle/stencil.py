"""Velocity stencils (Sec. 2, "Velocity stencils"; Fig. 1).

The paper names D2Q9, D2Q17 and D2Q37 as the minimal integer stencils (maximum displacement
M = 3) that carry Gauss-Hermite quadratures of degree 5, 7 and 9 with non-negative weights,
but it prints neither the velocities nor the weights. Reading taken here:

* velocity shells (all sign / axis permutations of each base vector):
    D2Q9  : (0,0) (1,0) (1,1)
    D2Q17 : (0,0) (1,0) (1,1) (2,2) (3,0)
    D2Q37 : (0,0) (1,0) (1,1) (2,0) (2,1) (2,2) (3,0) (3,1)
* normalized abscissae xi_i = r e_i with an unknown scale r, one weight per shell. Weights and
  r follow from requiring that the rule integrates exactly every even monomial
  xi_x^a xi_y^b (a + b < degree) against the unit Gaussian weight, whose moments are
  (a-1)!! (b-1)!!. With x <-> y symmetry there are exactly (#shells + 1) such conditions;
  for a fixed r they are linear in the weights, so r is a root of the determinant of the
  augmented system. Of the roots, the one with all weights positive is taken.

This is the oracle's own derivation (determinant root + linear solve). It is test
infrastructure only.
"""
from __future__ import annotations

from dataclasses import dataclass
from functools import lru_cache

import numpy as np
from scipy.optimize import brentq, root

SHELLS = {
    9: [(0, 0), (1, 0), (1, 1)],
    17: [(0, 0), (1, 0), (1, 1), (2, 2), (3, 0)],
    37: [(0, 0), (1, 0), (1, 1), (2, 0), (2, 1), (2, 2), (3, 0), (3, 1)],
}
DEGREE = {9: 5, 17: 7, 37: 9}        # quadrature degree (Sec. 2)
EQ_ORDER = {9: 2, 17: 3, 37: 4}      # Hermite order of the equilibrium: Eqs. (feq-2/3/4)


def shell_members(a: int, b: int) -> list[tuple[int, int]]:
    """All distinct vectors obtained from (a, b) by sign changes and swapping the axes."""
    out = set()
    for p, q in ((a, b), (b, a)):
        for sp in (1, -1):
            for sq in (1, -1):
                out.add((sp * p, sq * q))
    return sorted(out)


def odd_double_factorial(n: int) -> int:
    """(n-1)!! for even n >= 0: the n-th moment of the unit Gaussian."""
    v = 1
    for k in range(n - 1, 0, -2):
        v *= k
    return v


def _conditions(degree: int):
    """Even exponent pairs (a, b), a >= b, a + b < degree."""
    return [(a, b) for s in range(0, degree, 2) for a in range(s, -1, -1)
            for b in [s - a] if a % 2 == 0 and b % 2 == 0 and a >= b]


def _system(shells, conds, r):
    A = np.zeros((len(conds), len(shells)))
    rhs = np.zeros(len(conds))
    for k, (a, b) in enumerate(conds):
        rhs[k] = odd_double_factorial(a) * odd_double_factorial(b)
        for s, base in enumerate(shells):
            A[k, s] = r ** (a + b) * sum(ex ** a * ey ** b for ex, ey in shell_members(*base))
    return A, rhs


@dataclass(frozen=True)
class Lattice:
    q: int
    r: float                 # scale: xi_i = r * e_i (normalized units, c_s = 1)
    e: np.ndarray            # (q, 2) integer lattice velocities
    w: np.ndarray            # (q,) weights
    shell_of: np.ndarray     # (q,) shell index of each velocity
    order: int               # Hermite order of the equilibrium
    M: int                   # maximum displacement (halo depth)

    @property
    def xi(self) -> np.ndarray:
        return self.r * self.e.astype(np.float64)

    @property
    def cs_lattice(self) -> float:
        """Speed of sound c_s in lattice units (nodes per step) = 1 / r."""
        return 1.0 / self.r


@lru_cache(maxsize=None)
def lattice(q: int = 37) -> Lattice:
    shells = SHELLS[q]
    conds = _conditions(DEGREE[q])
    assert len(conds) == len(shells) + 1

    def det(r):
        A, rhs = _system(shells, conds, r)
        return np.linalg.det(np.column_stack([A, rhs]))

    def full_system(x):
        # the conditions as a square nonlinear system in (weights, r)
        A, rhs = _system(shells, conds, x[-1])
        return A @ x[:-1] - rhs

    grid = np.linspace(0.5, 4.0, 3501)
    vals = np.array([det(r) for r in grid])
    best = None
    for k in range(len(grid) - 1):
        if vals[k] == 0.0 or vals[k] * vals[k + 1] < 0:
            r0 = brentq(det, grid[k], grid[k + 1], xtol=1e-15, maxiter=500)
            A, rhs = _system(shells, conds, r0)
            W0, *_ = np.linalg.lstsq(A, rhs, rcond=None)
            # polish the determinant root with Newton steps on the full system
            sol = root(full_system, np.append(W0, r0), method="hybr", tol=1e-15)
            W, r = sol.x[:-1], float(sol.x[-1])
            A, rhs = _system(shells, conds, r)
            if np.all(W > 0) and np.allclose(A @ W, rhs, rtol=1e-13, atol=1e-14):
                assert best is None, "more than one admissible quadrature"
                best = (r, W)
    assert best is not None, f"no admissible quadrature for D2Q{q}"
    r, W = best
    e, w, shell_of = [], [], []
    for s, base in enumerate(shells):
        for v in shell_members(*base):
            e.append(v)
            w.append(W[s])
            shell_of.append(s)
    e = np.array(e, dtype=np.int64)
    assert len(e) == q
    return Lattice(q=q, r=float(r), e=e, w=np.array(w), shell_of=np.array(shell_of),
                   order=EQ_ORDER[q], M=int(np.abs(e).max()))

"""Seeded synthetic inputs shared by the oracle tests, the CUDA path tests and the benchmark.

This module holds no arithmetic of the lattice Boltzmann method. It only produces initial
macroscopic fields (rho, u_x, u_y, T) on the fluid region F = bulk + PML, and the seeded
parameter draws of the batched / serving workloads. Every field is a float64 numpy array of
shape (Ly, Lx) = (ny + 2W, nx + 2W), row-major (y outer, x inner), in the normalized units
of the method: sound speed c_s = 1, reference temperature T0 = 1, velocities in units of c_s.

Coordinates: bulk node (i, j) with 0 <= i < nx sits at F column W + i. Centres are given in
bulk coordinates; the default centre is ((nx-1)/2, (ny-1)/2).

Case definitions (the paper defines only the density step and its own vortex; the pulse and
the isentropic vortex below are the synthetic stand-ins used for the GB300 workloads):

* pressure pulse: p = 1 + A g, g = exp(-ln2 r^2 / b^2) (b = half-width), isentropic with
  gamma = (D+2)/D = 2: rho = p^(1/gamma), T = p / rho, u = u0.
* isentropic Gaussian vortex: u_theta = Mv (r/R) exp((1 - r^2/R^2)/2),
  T = T0 - (Mv^2/4) exp(1 - r^2/R^2), rho = rho0 (T/T0)^(1/(gamma-1)), plus uniform mean flow.
* density step (Sec. 5.1): tanh profile of the paper with rho0 = 1, rho1 = 1.05, s = 0.5.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np

GAMMA = 2.0  # (D + 2) / D for D = 2, monatomic ideal gas


def _edges(W, Wy=None):
    """(W_w, W_e, W_s, W_n) from W (every edge, or W/E with Wy on S/N) or a 4-tuple."""
    if np.ndim(W) == 1:
        return tuple(int(v) for v in W)
    Wy = W if Wy is None else Wy
    return (int(W), int(W), int(Wy), int(Wy))


def f_shape(nx: int, ny: int, W, Wy=None) -> tuple[int, int]:
    """(Ly, Lx) of the fluid region F (W PML layers per edge, Wy on the y edges if given, or
    per-edge widths (W_w, W_e, W_s, W_n))."""
    ww, we, ws, wn = _edges(W, Wy)
    return (ny + ws + wn, nx + ww + we)


def _bulk_coords(nx, ny, W, Wy=None):
    ww, we, ws, wn = _edges(W, Wy)
    Ly, Lx = f_shape(nx, ny, W, Wy)
    y, x = np.meshgrid(np.arange(Ly, dtype=np.float64) - ws,
                       np.arange(Lx, dtype=np.float64) - ww, indexing="ij")
    return x, y


def uniform(nx, ny, W, rho=1.0, ux=0.0, uy=0.0, T=1.0):
    shp = f_shape(nx, ny, W)
    return (np.full(shp, rho), np.full(shp, ux), np.full(shp, uy), np.full(shp, T))


def pressure_pulse(nx, ny, W, amp=1e-3, halfwidth=4.0, u0=(0.0, 0.0), center=None, Wy=None):
    """Isentropic Gaussian pressure pulse on a uniform state (rho = T = 1)."""
    x, y = _bulk_coords(nx, ny, W, Wy)
    cx, cy = center if center is not None else ((nx - 1) / 2.0, (ny - 1) / 2.0)
    r2 = (x - cx) ** 2 + (y - cy) ** 2
    p = 1.0 + amp * np.exp(-math.log(2.0) * r2 / (halfwidth * halfwidth))
    rho = p ** (1.0 / GAMMA)
    T = p / rho
    return rho, np.full_like(rho, u0[0]), np.full_like(rho, u0[1]), T


def multi_pulse(nx, ny, W, amps, centers, halfwidth=4.0, u0=(0.0, 0.0)):
    """Superposed isentropic pulses: p = 1 + sum_k A_k g_k."""
    x, y = _bulk_coords(nx, ny, W)
    p = np.ones_like(x)
    for a, (cx, cy) in zip(amps, centers):
        r2 = (x - cx) ** 2 + (y - cy) ** 2
        p += a * np.exp(-math.log(2.0) * r2 / (halfwidth * halfwidth))
    rho = p ** (1.0 / GAMMA)
    T = p / rho
    return rho, np.full_like(rho, u0[0]), np.full_like(rho, u0[1]), T


def isentropic_vortex(nx, ny, W, R=20.0, Mv=0.05, mean_u=(0.3, 0.0), T0=1.0, rho0=1.0,
                      center=None):
    """Isentropic Gaussian vortex convected by a uniform mean flow."""
    x, y = _bulk_coords(nx, ny, W)
    cx, cy = center if center is not None else ((nx - 1) / 2.0, (ny - 1) / 2.0)
    dx, dy = x - cx, y - cy
    r2 = dx * dx + dy * dy
    e = np.exp(1.0 - r2 / (R * R))
    amp = Mv / R * np.sqrt(e)          # u_theta / r
    ux = mean_u[0] - amp * dy
    uy = mean_u[1] + amp * dx
    T = T0 - 0.25 * Mv * Mv * e
    rho = rho0 * (T / T0) ** (1.0 / (GAMMA - 1.0))
    return rho, ux, uy, T


def density_step(Lx, Ly, Ma=0.05, rho0=1.0, rho1=1.05, s=0.5, W=0, Wy=None):
    """Sec. 5.1 density step on an Lx x Ly bulk (periodic in y in the paper), padded by W
    nodes on the x edges and Wy (default W) on the y edges (or per-edge widths); the profile
    formula continues into the padding. Background rho0 with a plateau rho1 on
    [Lx/4, 3Lx/4]. Reading: the printed right branch, rho1 - (rho1 - rho0)/2 (tanh(.) - 1),
    jumps to 2 rho1 - rho0 at Lx/2 and ends at rho1; with (tanh(.) + 1) it is continuous and
    returns to rho0, the state of the PML's mean equilibrium."""
    x, y = _bulk_coords(Lx, Ly, W, Wy)
    xs = x + 1.0  # the paper counts nodes from 1
    half = (rho1 - rho0) / 2.0
    left = rho1 + half * (np.tanh(s * (xs - 0.25 * Lx)) - 1.0)
    right = rho1 - half * (np.tanh(s * (xs - 0.75 * Lx)) + 1.0)
    rho = np.where(xs <= Lx / 2.0, left, right)
    return rho, np.full_like(rho, Ma), np.zeros_like(rho), np.ones_like(rho)


def paper_vortex(nx, ny, W, Ma=0.1, b=0.2, rstar=0.5, K=180.0, rho0=1.0, T0=1.0, pad=0):
    """Sec. 5.2 thermal vortex on an nx x ny bulk: normalized coordinates
    x* = 2(x - 1)/(nx - 1) - 1 (x counted from 1 over the bulk), centre (K/(nx - 1), 0); inside
    radius r*: u = u0 + (5/2) u0 2^(-(x^2 + y^2)/b^2) (y, -x), T = T0 + y (5/2) u0 2^(...),
    rho = rho0; u0 = Ma (c_s = 1). The paper does not give b, r*, K: b = 0.2, r* = 0.5, K = 180
    are chosen here. `pad` extends the grid by pad nodes per side with the same formula
    (periodic reference runs), on top of the W PML layers."""
    Ly, Lx = ny + 2 * (W + pad), nx + 2 * (W + pad)
    y, x = np.meshgrid(np.arange(Ly, dtype=np.float64) - (W + pad) + 1.0,
                       np.arange(Lx, dtype=np.float64) - (W + pad) + 1.0, indexing="ij")
    xs = 2.0 * (x - 1.0) / (nx - 1.0) - 1.0 - K / (nx - 1.0)
    ys = 2.0 * (y - 1.0) / (ny - 1.0) - 1.0
    inside = xs * xs + ys * ys < rstar * rstar
    g = 2.5 * Ma * np.power(2.0, -(xs * xs + ys * ys) / (b * b))
    ux = Ma + np.where(inside, g * ys, 0.0)
    uy = np.where(inside, -g * xs, 0.0)
    T = T0 + np.where(inside, ys * g, 0.0)
    return np.full_like(ux, rho0), ux, uy, T


def random_smooth_state(nx, ny, W, seed, du=0.05, drho=0.02, dT=0.02, mean_u=(0.0, 0.0),
                        modes=4, Wy=None):
    """Seeded smooth random perturbation (sum of low Fourier modes) around a mean state."""
    rng = np.random.default_rng(seed)
    x, y = _bulk_coords(nx, ny, W, Wy)
    Ly, Lx = x.shape
    out = []
    for amp, base in ((drho, 1.0), (du, mean_u[0]), (du, mean_u[1]), (dT, 1.0)):
        fld = np.full_like(x, base)
        for _ in range(modes):
            kx, ky = rng.integers(1, 4, size=2)
            ph = rng.uniform(0, 2 * np.pi, size=2)
            a = rng.uniform(-1, 1) * amp / modes
            fld += a * np.sin(2 * np.pi * kx * x / Lx + ph[0]) * np.cos(2 * np.pi * ky * y / Ly + ph[1])
        out.append(fld)
    return tuple(out)


# --------------------------------------------------------------------------------------------
# Workload configurations (sizes and parameter draws of the GB300 workloads)
# --------------------------------------------------------------------------------------------

@dataclass
class Case:
    """One solve: geometry, physics parameters and initial fields recipe."""
    name: str
    nx: int
    ny: int
    W: int
    tau: float
    sigma_max: float
    sigma_power: int
    bc: str                      # "periodic" | "zg" | "nrbc"
    steps: int
    ic: str                      # "pulse" | "vortex" | "multi_pulse" | "uniform" | "step"
    ic_args: dict = field(default_factory=dict)
    nrbc_edges: tuple = (0, 1, 0, 0)   # W, E, S, N: 0 = PNR-LODI, 1 = CBC relax
    beta: float = 0.3
    mean: tuple = (1.0, 0.0, 0.0, 1.0)  # rho0, u0x, u0y, T0 (mean equilibrium of the PML)
    pml_grad: str = "central"    # "central" (printed differences) | "link" (link difference)

    def fields(self):
        if self.ic == "pulse":
            return pressure_pulse(self.nx, self.ny, self.W, **self.ic_args)
        if self.ic == "vortex":
            return isentropic_vortex(self.nx, self.ny, self.W, **self.ic_args)
        if self.ic == "multi_pulse":
            return multi_pulse(self.nx, self.ny, self.W, **self.ic_args)
        if self.ic == "uniform":
            return uniform(self.nx, self.ny, self.W, **self.ic_args)
        if self.ic == "step":
            return density_step(self.nx, self.ny, W=self.W, **self.ic_args)
        raise ValueError(self.ic)


def pulse_64():
    """64x64 bulk + 8-node PML, zero-gradient edge, tau 0.8, cubic sigma 0.1, 200 steps."""
    return Case("pulse64_w8_zg", 64, 64, 8, 0.8, 0.1, 3, "zg", 200, "pulse",
                dict(amp=1e-3, halfwidth=4.0))


def vortex_2048(n=2048, W=32):
    """2048^2 bulk + PML 32 (cubic), NRBC (east CBC relax, others PNR-LODI), isentropic vortex
    R = 20, Mv = 0.05 in a Mach 0.3 mean flow, tau 0.55."""
    return Case(f"vortex{n}_w{W}_nrbc", n, n, W, 0.55, 0.1, 3, "nrbc", 20000, "vortex",
                dict(R=20.0, Mv=0.05, mean_u=(0.3, 0.0)), nrbc_edges=(0, 1, 0, 0), beta=0.3,
                mean=(1.0, 0.3, 0.0, 1.0))


def stress_8192(n=8192, W=64, seed=0):
    """8192^2 bulk + PML 64, NRBC, four superposed pulses in a Mach 0.2 mean flow, tau 0.52."""
    rng = np.random.default_rng(seed)
    amps = rng.uniform(1e-3, 1e-2, size=4).tolist()
    centers = [tuple(c) for c in rng.uniform(0, n - 1, size=(4, 2)).tolist()]
    return Case(f"stress{n}_w{W}_nrbc", n, n, W, 0.52, 0.1, 3, "nrbc", 10000, "multi_pulse",
                dict(amps=amps, centers=centers, halfwidth=4.0 * n / 1024, u0=(0.2, 0.0)),
                nrbc_edges=(0, 1, 0, 0), beta=0.2, mean=(1.0, 0.2, 0.0, 1.0))


def batched_sweep(count=256, seed=0, steps=5000, pml_grad="central", nrbc_edges=(0, 1, 0, 0)):
    """Seeded uneven instances: N ~ U{128..1024}, W ~ U{4..64}, log sigma ~ U[ln .01, ln .5],
    bc 50/50 zg/nrbc, case 50/50 pulse (A = 1e-3) / vortex (mean Mach ~ U[0.1, 0.5]).
    pml_grad and nrbc_edges (W, E, S, N variants of the characteristic BC) apply to every
    instance; the draws do not depend on them."""
    rng = np.random.default_rng(seed)
    cases = []
    for k in range(count):
        n = int(rng.integers(128, 1025))
        W = int(rng.integers(4, 65))
        sig = float(np.exp(rng.uniform(np.log(0.01), np.log(0.5))))
        bc = "zg" if rng.random() < 0.5 else "nrbc"
        if rng.random() < 0.5:
            cases.append(Case(f"b{k}", n, n, W, 0.8, sig, 3, bc, steps, "pulse",
                              dict(amp=1e-3, halfwidth=4.0), nrbc_edges=tuple(nrbc_edges),
                              pml_grad=pml_grad))
        else:
            ma = float(rng.uniform(0.1, 0.5))
            cases.append(Case(f"b{k}", n, n, W, 0.8, sig, 3, bc, steps, "vortex",
                              dict(R=20.0, Mv=0.05, mean_u=(ma, 0.0)), beta=ma,
                              mean=(1.0, ma, 0.0, 1.0), nrbc_edges=tuple(nrbc_edges),
                              pml_grad=pml_grad))
    return cases


def request_stream(count=500, rate=50.0, seed=0, nmin=64, nmax=2048, smin=1000, smax=20000,
                   pml_grad="central", nrbc_edges=(0, 1, 0, 0)):
    """Poisson request stream: (arrival_time_s, Case). Bulk N log-uniform, W ~ U{8..64}.
    pml_grad and nrbc_edges apply to every request; the draws do not depend on them."""
    rng = np.random.default_rng(seed)
    t = 0.0
    out = []
    for k in range(count):
        t += float(rng.exponential(1.0 / rate))
        n = int(round(math.exp(rng.uniform(math.log(nmin), math.log(nmax)))))
        W = int(rng.integers(8, 65))
        steps = int(rng.integers(smin, smax + 1))
        if rng.random() < 0.5:
            c = Case(f"r{k}", n, n, W, 0.8, 0.1, 3, "zg", steps, "pulse",
                     dict(amp=1e-3, halfwidth=4.0), pml_grad=pml_grad)
        else:
            c = Case(f"r{k}", n, n, W, 0.8, 0.05, 3, "nrbc", steps, "vortex",
                     dict(R=min(20.0, n / 8), Mv=0.05, mean_u=(0.1, 0.0)), beta=0.1,
                     mean=(1.0, 0.1, 0.0, 1.0), nrbc_edges=tuple(nrbc_edges),
                     pml_grad=pml_grad)
        out.append((t, c))
    return out

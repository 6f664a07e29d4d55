"""One time step of the PML + outer-BC lattice Boltzmann scheme, written out literally.

Grid. Bulk nx x ny; fluid region F = bulk + PML layers (W per side, or per-edge widths;
Lx x Ly); boundary band
Gamma = M layers outside F (M = maximum displacement of the stencil, 3 for D2Q37), so every
pull source x - e_i of a node of F lies on the allocated grid G = F + Gamma. Reading of the
boundary nodes x_(b,j), j = 1..M, of Sec. 4: they are the nodes of Gamma; after streaming
their populations are defined by the BC and they then take part in the collision (BGK only,
no PML term) like any other node. "(L + 2W)^2" in Sec. 5.2 counts F only.

State after n steps: f^n on G, post-stream with Gamma already set by the BC. One step
(Sec. 2 outline: collision, streaming, boundary condition, then moments):
  1. moments U^n on G                                      Eq. (macro)
  2. f_eq^n on G                                           Eqs. (feq-2..4)
  3. on P + ring: f_hat^n = f_eq^n - f_eq_bar, Q^n by the trapezoidal rule
     (option pml_grad = "link": on all of G, boundary band included)
  4. on P: grad Q^n and Omega^PML                          Eqs. (PMLCOLL), (FD-dx-*)
     (option "link": c_i . grad Q_i as Q_i(x + e_i) - Q_i(x), pml.py)
  5. collide: f* = f - (f - f_eq)/tau on G, + Omega^PML on P      Eq. (lbe)
  6. stream (pull): f^(n+1)(x) = f*(x - e_i) for x in F
  7. boundary: Gamma of f^(n+1) from
       periodic: periodic images (reference simulations of Sec. 5),
       zg:       f(x_b) = f(x_f), x_f the nearest node of F   Eq. (zg-bc),
       nrbc:     U_tgt^(n+1) from U_tgt^n by integrating dU/dt (characteristic.py) over one
                 step (RK4, fluid moments frozen at time n) on the edge bands, then
                 f(x_b) = f_eq(U_tgt^(n+1)) + [f(x_f) - f_eq(U(f(x_f)))] (non-equilibrium
                 extrapolation); corner blocks of Gamma use the zg copy.
Initialization (Sec. 2): f^0 = f_eq(initial fields) on F; Gamma by the BC rule with
U_tgt^0 = initial fields at x_f; Q^0 = 0.
"""
from __future__ import annotations

import numpy as np

from . import characteristic as ch
from . import pml
from .equilibrium import bgk, feq, moments
from .stencil import lattice

EDGES = ("W", "E", "S", "N")


def rk4_step(y0, rate, dt):
    """One step of the classical fourth-order Runge-Kutta method for the autonomous system
    dy/dt = rate(y): stages k1 = rate(y0), k2 = rate(y0 + dt k1 / 2), k3 = rate(y0 + dt k2 / 2),
    k4 = rate(y0 + dt k3); y1 = y0 + dt (k1 + 2 k2 + 2 k3 + k4) / 6."""
    k1 = rate(y0)
    k2 = rate(y0 + 0.5 * dt * k1)
    k3 = rate(y0 + 0.5 * dt * k2)
    k4 = rate(y0 + dt * k3)
    return y0 + dt * (k1 + 2.0 * k2 + 2.0 * k3 + k4) / 6.0


class OracleLBM:
    def __init__(self, nx, ny, W, tau, sigma_max=0.0, sigma_power=2, bc="zg", q=37,
                 nrbc_edges=(0, 0, 0, 0), beta=0.0, mean=(1.0, 0.0, 0.0, 1.0),
                 relax_sign=-1.0, pml_on=True, Wy=None, periodic_y=False, sigma_split=False,
                 pml_source=0, pml_grad="central"):
        """W: PML layers on every edge, or on the W and E edges when Wy (S and N edges) is
        given, or a per-edge tuple (W_w, W_e, W_s, W_n). periodic_y: the y axis wraps (no PML
        on it; Wy defaults to 0 then); the x edges keep the chosen BC. sigma_split: the
        general sigma_x != sigma_y form of Eq. (pml-general) instead of sigma_x = sigma_y.
        pml_source: bitmask of the PML source terms I (1), II (2), III (4) of Eq. NSF-CHAR-PML
        added to the characteristic targets (Appendix; 0 = the characteristic BC of Sec. 4);
        + 8: the sign printed there instead of the collision term's."""
        self.lat = lattice(q)
        self.pml_on = pml_on
        if pml_grad not in ("central", "link"):
            raise ValueError("pml_grad is 'central' or 'link'")
        if pml_grad == "link" and sigma_split:
            raise ValueError("the link-integrated gradient is defined for sigma_x = sigma_y")
        self.pml_grad = pml_grad
        self.periodic_y = bool(periodic_y)
        if self.periodic_y and Wy is None and np.ndim(W) == 0:
            Wy = 0
        self.widths = pml.widths4(W, Wy)
        ww, we, ws, wn = self.widths
        if any(w < 0 or w == 1 for w in self.widths):
            raise ValueError("a PML needs W >= 2 (one-sided difference reaches 2 nodes in)")
        if bc == "periodic" and any(self.widths):
            raise ValueError("periodic mode has no PML")
        if self.periodic_y and (ws or wn or bc == "periodic"):
            raise ValueError("a periodic y axis has no PML and needs a zg/nrbc x edge")
        self.nx, self.ny = nx, ny
        self.Lx, self.Ly = nx + ww + we, ny + ws + wn
        self.M = self.lat.M
        self.tau = tau
        self.bc = bc
        self.nrbc_edges = tuple(nrbc_edges)
        self.pml_source = int(pml_source)
        self._src = None
        self.beta = beta
        self.relax_sign = relax_sign
        M, Lx, Ly = self.M, self.Lx, self.Ly
        self.Gx, self.Gy = Lx + 2 * M, Ly + 2 * M
        self.sigma_x, self.sigma_y = pml.sigma_fields(Lx, Ly, self.widths, sigma_max,
                                                      sigma_power, split=sigma_split)
        self.in_P = pml.in_pml(Lx, Ly, self.widths)
        self.qsup = pml.q_support(Lx, Ly, self.widths)
        self.edges = ("W", "E") if self.periodic_y else EDGES
        rho0, u0x, u0y, T0 = mean
        self.fbar = feq(np.float64(rho0), np.array([u0x, u0y]), np.float64(T0),
                        self.lat.xi, self.lat.w, self.lat.order)          # f_eq_bar (Eq. decomp-NJ)
        self.step_count = 0
        gx = np.arange(self.Gx) - M
        gy = np.arange(self.Gy) - M
        self._clx = np.clip(gx, 0, Lx - 1) + M
        self._cly = np.clip(gy, 0, Ly - 1) + M
        self._wrx = np.mod(gx, Lx) + M
        self._wry = np.mod(gy, Ly) + M

    # ---------------------------------------------------------------- helpers
    @property
    def Fs(self):
        M = self.M
        return (slice(None), slice(M, M + self.Ly), slice(M, M + self.Lx))

    def _feq(self, rho, u, T):
        return feq(rho, u, T, self.lat.xi, self.lat.w, self.lat.order)

    def _edge_nodes(self, edge, j):
        """G indices (gy, gx) of the layer-j nodes of an edge band, and their x_f."""
        M, Lx, Ly = self.M, self.Lx, self.Ly
        if edge == "W":
            gy = np.arange(Ly) + M
            return gy, np.full(Ly, M - j), gy, np.full(Ly, M)
        if edge == "E":
            gy = np.arange(Ly) + M
            return gy, np.full(Ly, M + Lx - 1 + j), gy, np.full(Ly, M + Lx - 1)
        if edge == "S":
            gx = np.arange(Lx) + M
            return np.full(Lx, M - j), gx, np.full(Lx, M), gx
        gx = np.arange(Lx) + M
        return np.full(Lx, M + Ly - 1 + j), gx, np.full(Lx, M + Ly - 1), gx

    def _fill_gamma(self, f):
        """Gamma of the post-stream populations f (in place), Sec. 4 / Sec. 5."""
        if self.bc == "periodic":
            f[:] = f[:, self._wry[:, None], self._wrx[None, :]]
            return
        # zero-gradient copy, Eq. (zg-bc); in nrbc mode this also fills the corner blocks
        f[:] = f[:, self._cly[:, None], self._clx[None, :]]
        if self.bc == "nrbc":
            for k, edge in enumerate(EDGES):
                if edge not in self.edges:
                    continue
                for j in range(1, self.M + 1):
                    by, bx, fy, fx = self._edge_nodes(edge, j)
                    ff = f[:, fy, fx]
                    rho, u, T = moments(ff, self.lat.xi)
                    Ut = self.Utgt[edge][j - 1]
                    f[:, by, bx] = (self._feq(Ut[:, 0], Ut[:, 1:3].T, Ut[:, 3])
                                    + ff - self._feq(rho, u, T))
        if self.periodic_y:
            # rows outside F along the periodic axis are images of rows inside, boundary
            # columns included (those hold the x-edge boundary values just set)
            f[:] = f[:, self._wry, :]

    def _edge_sources(self, om, Uf):
        """Primitive-variable PML sources (Appendix) at the outermost fluid node of every band
        position: edge -> (m, 4), from the selected parts om (q, Ly, Lx) of Omega^PML."""
        xi = self.lat.xi
        mass = om.sum(axis=0)
        mom = np.tensordot(xi.T, om, axes=(1, 0))                          # (2, Ly, Lx)
        energy = 0.5 * np.tensordot((xi ** 2).sum(1), om, axes=(0, 0))
        prim = ch.conserved_to_primitive_rate(mass, mom, energy, Uf)     # (Ly, Lx, 4)
        return {"W": prim[:, 0], "E": prim[:, -1], "S": prim[0, :], "N": prim[-1, :]}

    def _set_sources(self, parts, rho, u, T):
        """Appendix sources from the three parts (gradient, f_hat, Q) of Omega^PML on F."""
        sel = sum(pt for k, pt in enumerate(parts) if self.pml_source >> k & 1)
        M = self.M
        Uf = np.stack([rho, u[0], u[1], T], axis=-1)[M:M + self.Ly, M:M + self.Lx]
        if self.pml_source & 8:                          # printed "+" of Eq. NSF-CHAR-PML
            sel = -sel
        self._src = self._edge_sources(np.where(self.in_P, sel, 0.0), Uf)

    def _target_rates(self, V, U):
        """dU/dt of every edge-band node for the boundary state V (dict edge -> M layers of
        (m, 4) arrays) and the time-n fluid moments U (Ly, Lx, 4) on F."""
        M = self.M
        rates = {}
        for k, edge in enumerate(EDGES):
            if edge not in self.edges:
                continue
            axis = 0 if edge in ("W", "E") else 1
            out = -1.0 if edge in ("W", "S") else 1.0
            layers = []
            for j in range(1, M + 1):
                by, bx, fy, fx = self._edge_nodes(edge, j)

                def U_at(jj):
                    # layer jj >= 1: boundary state; jj = 0: the outermost fluid node x_f;
                    # jj = -1: the fluid node one further inside
                    if jj >= 1:
                        return V[edge][jj - 1]
                    d = -jj
                    if axis == 0:
                        return U[fy - M, fx - M - int(out) * d]
                    return U[fy - M - int(out) * d, fx - M]

                U0 = V[edge][j - 1]
                dUn = out * ch.one_sided(U0, U_at(j - 1), U_at(j - 2))
                dUt = ch.tangential(U0, periodic=self.periodic_y and axis == 0)
                rt = ch.rate(U0, dUn, dUt, axis, out, self.nrbc_edges[k], self.beta,
                             self.lat.r, self.relax_sign)
                if self._src is not None:
                    rt = rt + self._src[edge]                                # Appendix source
                layers.append(rt)
            rates[edge] = layers
        return rates

    def _advance_targets(self, U):
        """U_tgt^n -> U_tgt^(n+1): classical fourth-order Runge-Kutta over one time step with
        the fluid moments frozen at time n. (Explicit Euler with the one-sided difference is
        unstable here: its self-coefficient 1 - 3 nu / 2 leaves the unit disc once the
        acoustic CFL nu = (|u_n| + c) / r exceeds 4/3, i.e. already near Mach 0.2.)"""
        edges = self.edges
        names = [(e, j) for e in edges for j in range(len(self.Utgt[e]))]

        sizes = [len(self.Utgt[e][j]) for e, j in names]
        offs = np.concatenate([[0], np.cumsum(sizes)])

        def pack(V):
            return np.concatenate([V[e][j] for e, j in names])

        def unpack(X):
            V = {e: [] for e in edges}
            for k, (e, j) in enumerate(names):
                V[e].append(X[offs[k]:offs[k + 1]])
            return V

        X = rk4_step(pack(self.Utgt), lambda X: pack(self._target_rates(unpack(X), U)), 1.0)
        self.Utgt = unpack(X)

    # ---------------------------------------------------------------- public
    def init(self, rho, ux, uy, T):
        """f^0 = f_eq(fields) on F; Gamma by the BC; Q^0 = 0."""
        M = self.M
        f = np.zeros((self.lat.q, self.Gy, self.Gx))
        f[self.Fs] = self._feq(rho, np.stack([ux, uy]), T)
        if self.bc == "nrbc":
            Uf = np.stack([rho, ux, uy, T], axis=-1)
            self.Utgt = {}
            for edge in self.edges:
                layers = []
                for j in range(1, M + 1):
                    by, bx, fy, fx = self._edge_nodes(edge, j)
                    layers.append(Uf[fy - M, fx - M].copy())
                self.Utgt[edge] = layers
        self._fill_gamma(f)
        self.f = f
        self.Q = None
        self.fhat_prev = None
        self._src = None
        self.step_count = 0

    def step(self, n=1):
        lat = self.lat
        for _ in range(n):
            f = self.f
            rho, u, T = moments(f, lat.xi)                                   # 1
            fe = self._feq(rho, u, T)                                        # 2
            fstar = bgk(f, fe, self.tau)                                     # 5 (BGK part)
            if any(self.widths) and self.pml_on and self.pml_grad == "link":
                Fs = self.Fs
                fhatG = fe - self.fbar[:, None, None]                        # 3, on all of G
                if self.Q is None:
                    QG = np.zeros_like(fhatG)                                # Q^0 = 0
                else:
                    QG = pml.trapezoid_update(self.Q, self.fhat_prev, fhatG)
                self.Q, self.fhat_prev = QG, fhatG
                link = pml.link_difference(QG, lat.e, self.M, self.Ly, self.Lx)      # 4
                parts = pml.omega_pml_link_terms(link, fhatG[Fs], QG[Fs], self.sigma_x)
                om = parts[0] + parts[1] + parts[2]
                fstar[Fs] = fstar[Fs] + np.where(self.in_P, om, 0.0)         # 5 (PML part)
                if self.bc == "nrbc" and self.pml_source & 7:
                    self._set_sources(parts, rho, u, T)
            elif any(self.widths) and self.pml_on:
                Fs = self.Fs
                fhat = np.where(self.qsup, fe[Fs] - self.fbar[:, None, None], 0.0)   # 3
                if self.Q is None:
                    Q = np.zeros_like(fhat)                                  # Q^0 = 0
                else:
                    Q = np.where(self.qsup, pml.trapezoid_update(self.Q, self.fhat_prev, fhat),
                                 0.0)
                self.Q, self.fhat_prev = Q, fhat
                gx, gy = pml.gradient(Q, self.periodic_y)                    # 4
                om = pml.omega_pml(lat.e, gx, gy, fhat, Q, self.sigma_x, self.sigma_y)
                fstar[Fs] = fstar[Fs] + np.where(self.in_P, om, 0.0)         # 5 (PML part)
                if self.bc == "nrbc" and self.pml_source & 7:
                    parts = pml.omega_pml_terms(lat.e, gx, gy, fhat, Q, self.sigma_x,
                                                self.sigma_y)
                    self._set_sources(parts, rho, u, T)
            if self.periodic_y:
                # the rows beyond a periodic y axis carry the post-collision populations of
                # the rows they image (PML term included), as on an unbounded periodic lattice
                fstar[:] = fstar[:, self._wry, :]
            fnew = np.empty_like(f)                                          # 6
            M = self.M
            for i, (ex, ey) in enumerate(lat.e):
                fnew[i, M:M + self.Ly, M:M + self.Lx] = fstar[
                    i, M - ey:M - ey + self.Ly, M - ex:M - ex + self.Lx]
            if self.bc == "nrbc":                                            # 7
                U = np.stack([rho, u[0], u[1], T], axis=-1)[M:M + self.Ly, M:M + self.Lx]
                self._advance_targets(U)
            self._fill_gamma(fnew)
            self.f = fnew
            self.step_count += 1

    def fields(self, region="F"):
        """rho, u_x, u_y, T of f^n on F (region "F") or on the bulk (region "bulk")."""
        rho, u, T = moments(self.f[self.Fs], self.lat.xi)
        out = (rho, u[0], u[1], T)
        if region == "bulk":
            ww, ws = self.widths[0], self.widths[2]
            out = tuple(a[ws:ws + self.ny, ww:ww + self.nx] for a in out)
        return out

    def totals(self):
        """Mass, x/y momentum and energy (1/2 sum f |xi|^2) summed over F."""
        fF = self.f[self.Fs]
        xi = self.lat.xi
        mass = fF.sum()
        mx = np.tensordot(xi[:, 0], fF, axes=(0, 0)).sum()
        my = np.tensordot(xi[:, 1], fF, axes=(0, 0)).sum()
        en = 0.5 * np.tensordot((xi ** 2).sum(1), fF, axes=(0, 0)).sum()
        return np.array([mass, mx, my, en])

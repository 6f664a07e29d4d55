"""Pins of the parts of the oracle that the field-level tests leave loose: the gradient and
sigma^2 Q parts of Omega^PML (Eqs. pml-general / PMLCOLL), the trapezoidal accumulator over two
steps (Eq. PMLQ), the link-integrated gradient option, the Runge-Kutta integrator of the
characteristic targets and the CBC-relax branch (Eq. CBC-Relax).

Each closed form below is derived by hand from the equations, not by re-running the oracle's
own formula; the planted-mistake tests show that a flipped sign or a wrong coefficient in the
term a pin guards makes that pin fail.
"""
import numpy as np
import pytest

import workloads as wl
from oracle import OracleLBM, pml
from oracle import solver as osolver


# ------------------------------------------------------------------ planted accumulator Q
def _uniform(o, rho=1.0):
    shp = (o.Ly, o.Lx)
    return np.full(shp, rho), np.zeros(shp), np.zeros(shp), np.ones(shp)


def _planted_q_error(mode, kind, a=2e-4, sigma=0.3):
    """Rest state f = w (the PML mean state), so f_hat = 0 and Q stays as planted. Q_i is the
    same scalar field q(x) for every direction: q = a x (kind "lin") or a x^2 (kind "quad"),
    x the F column. PML on the x edges only, periodic y, sigma = sigma_max on P (power 0).
    One step: f*_i(z) = w_i + Omega_i(z) on P with (sigma_x = sigma_y = sigma)
      printed central / one-sided differences (exact for these fields):
          Omega_i = -sigma (e_ix q'(z) + sigma q(z))
      link difference: Omega_i = -sigma (q(z + e_i) - q(z) + sigma q(z)).
    After the pull, f_i(x) = f*_i(x - e_i). Returns the largest deviation from the closed form
    over the nodes whose source lies in F."""
    nx, ny, W = 6, 4, 6
    o = OracleLBM(nx, ny, W, 0.8, sigma, 0, "zg", q=37, periodic_y=True, pml_grad=mode)
    o.init(*_uniform(o))
    lat, M, Lx, Ly = o.lat, o.M, o.Lx, o.Ly

    def q_of(x):
        x = np.asarray(x, dtype=np.float64)
        return a * x if kind == "lin" else a * x * x

    def dq_of(x):
        x = np.asarray(x, dtype=np.float64)
        return a * np.ones_like(x) if kind == "lin" else 2.0 * a * x

    if mode == "link":
        xs = np.arange(Lx + 2 * M) - M                       # F column of every G column
        o.Q = np.broadcast_to(q_of(xs)[None, None, :], (37, Ly + 2 * M, Lx + 2 * M)).copy()
    else:
        xs = np.arange(Lx)
        Q = np.broadcast_to(q_of(xs)[None, None, :], (37, Ly, Lx)).copy()
        o.Q = np.where(o.qsup, Q, 0.0)
    o.fhat_prev = np.zeros_like(o.Q)
    o.step(1)
    worst = 0.0
    w = lat.w
    inP = o.in_P[0]
    for i, (ex, ey) in enumerate(lat.e):
        for x in range(Lx):
            z = x - ex
            if z < 0 or z >= Lx:
                continue
            if inP[z]:
                if mode == "link":
                    grad = q_of(z + ex) - q_of(z)
                else:
                    grad = ex * dq_of(z)
                om = -sigma * (grad + sigma * q_of(z))
            else:
                om = 0.0
            got = o.f[i, M:M + Ly, M + x]
            worst = max(worst, float(np.max(np.abs(got - (w[i] + om)))))
    return worst


@pytest.mark.parametrize("mode", ["central", "link"])
def test_planted_linear_q_gives_the_gradient_and_sigma2_parts(mode):
    assert _planted_q_error(mode, "lin") < 1e-16


@pytest.mark.parametrize("mode", ["central", "link"])
def test_planted_quadratic_q(mode):
    """Quadratic q: the central / one-sided differences are exact derivatives; the link
    difference is the exact path integral a (2 z e_x + e_x^2) — the two options differ."""
    assert _planted_q_error(mode, "quad") < 1e-15


def test_link_and_central_differ_on_a_quadratic():
    """The extra a e_x^2 of the path integral is present in link mode only."""
    assert _planted_q_error("central", "quad") < 1e-15
    # evaluate the central closed form against the link run: must miss by ~sigma a e_x^2
    o_err = _planted_q_error_cross()
    assert o_err > 1e-6


def _planted_q_error_cross(a=2e-4, sigma=0.3):
    """Link run checked against the central closed form (must not match)."""
    nx, ny, W = 6, 4, 6
    o = OracleLBM(nx, ny, W, 0.8, sigma, 0, "zg", q=37, periodic_y=True, pml_grad="link")
    o.init(*_uniform(o))
    M, Lx, Ly = o.M, o.Lx, o.Ly
    xs = np.arange(Lx + 2 * M) - M
    o.Q = np.broadcast_to((a * xs * xs)[None, None, :], (37, Ly + 2 * M, Lx + 2 * M)).copy()
    o.fhat_prev = np.zeros_like(o.Q)
    o.step(1)
    worst = 0.0
    for i, (ex, ey) in enumerate(o.lat.e):
        for x in range(Lx):
            z = x - ex
            if 0 <= z < Lx and o.in_P[0][z]:
                om = -sigma * (ex * 2 * a * z + sigma * a * z * z)
                worst = max(worst, float(np.max(np.abs(o.f[i, M:M + Ly, M + x] - (o.lat.w[i] + om)))))
    return worst


def test_planted_mistake_in_the_gradient_sign_breaks_the_pin(monkeypatch):
    real = pml.omega_pml

    def flipped(e, gx, gy, fhat, Q, sx, sy=None):
        return real(e, -gx, -gy, fhat, Q, sx, sy)
    monkeypatch.setattr(pml, "omega_pml", flipped)
    assert _planted_q_error("central", "lin") > 1e-6


def test_planted_mistake_in_the_sigma2_term_breaks_the_pin(monkeypatch):
    real = pml.omega_pml_link_terms

    def flipped(link, fhat, Q, sigma):
        g, f, q = real(link, fhat, Q, sigma)
        return g, f, -q
    monkeypatch.setattr(pml, "omega_pml_link_terms", flipped)
    assert _planted_q_error("link", "lin") > 1e-6


def test_link_difference_is_the_path_integral_of_a_quadratic():
    """Q(x + e) - Q(x) for Q = al x^2 + be x y + ga y^2 + de x + ep y, on every node of F, from
    a field given on G (boundary band included)."""
    from oracle.stencil import lattice
    lat = lattice(37)
    M, Ly, Lx = 3, 5, 7
    al, be, ga, de, ep = 0.3, -0.7, 0.2, 1.1, -2.0
    gy, gx = np.meshgrid(np.arange(Ly + 2 * M) - M, np.arange(Lx + 2 * M) - M, indexing="ij")
    q = al * gx * gx + be * gx * gy + ga * gy * gy + de * gx + ep * gy
    QG = np.broadcast_to(q, (37,) + q.shape).copy()
    got = pml.link_difference(QG, lat.e, M, Ly, Lx)
    y, x = np.meshgrid(np.arange(Ly), np.arange(Lx), indexing="ij")
    for i, (ex, ey) in enumerate(lat.e):
        want = (al * (2 * x * ex + ex * ex) + be * (x * ey + y * ex + ex * ey)
                + ga * (2 * y * ey + ey * ey) + de * ex + ep * ey)
        assert np.allclose(got[i], want, rtol=0, atol=1e-12)


# ------------------------------------------------------------------ two steps of a uniform excess
def _two_step_error(mode, sigma=0.3, d=1e-3):
    """Uniform density excess d at rest, sigma = sigma_max on P (power 0), PML on the x edges,
    periodic y. Step 0: f_hat^0 = d w, Q^0 = 0, Omega^0 = -2 sigma d w, so deep in a slab
    f^1 = w (1 + d (1 - 2 sigma)). Step 1: f_hat^1 = d (1 - 2 sigma) w, Q^1 = (f_hat^0 + f_hat^1)/2
    = d (1 - sigma) w, grad Q^1 = 0, Omega^1 = -sigma (2 f_hat^1 + sigma Q^1), hence
    rho^2 = 1 + d (1 - 4 sigma + 3 sigma^2 + sigma^3) at nodes nine or more links from the bulk
    and from the boundary band."""
    nx, ny, W = 6, 4, 24
    o = OracleLBM(nx, ny, W, 0.8, sigma, 0, "zg", q=37, periodic_y=True, pml_grad=mode)
    o.init(*_uniform(o, 1.0 + d))
    o.step(2)
    rho = o.fields("F")[0]
    want = 1.0 + d * (1.0 - 4.0 * sigma + 3.0 * sigma ** 2 + sigma ** 3)
    deep = rho[:, 9:W - 9]
    return float(np.max(np.abs(deep - want)))


@pytest.mark.parametrize("mode", ["central", "link"])
def test_two_step_closed_form_of_a_uniform_excess(mode):
    assert _two_step_error(mode) < 1e-15


def test_planted_mistake_in_the_trapezoid_breaks_the_two_step_pin(monkeypatch):
    monkeypatch.setattr(pml, "trapezoid_update", lambda Q, a, b: Q + b)   # implicit Euler
    assert _two_step_error("central") > 1e-6


def test_planted_mistake_in_the_sigma2_sign_breaks_the_two_step_pin(monkeypatch):
    real = pml.omega_pml

    def flipped(e, gx, gy, fhat, Q, sx, sy=None):
        return real(e, gx, gy, fhat, -Q, sx, sy)
    monkeypatch.setattr(pml, "omega_pml", flipped)
    assert _two_step_error("central") > 1e-6


# ------------------------------------------------------------------ Runge-Kutta integrator
@pytest.mark.parametrize("z", [0.3, -1.7, 0.5 + 2.0j])
def test_rk4_step_is_the_fourth_order_taylor_polynomial_on_a_linear_system(z):
    """For dy/dt = lam y the classical RK4 step is exactly y (1 + z + z^2/2 + z^3/6 + z^4/24),
    z = lam dt; a wrong stage weight or stage point changes the polynomial."""
    y0 = np.array([1.0 + 0.0j, -0.25 + 0.5j])
    dt = 0.7
    lam = z / dt
    got = osolver.rk4_step(y0, lambda y: lam * y, dt)
    want = y0 * (1 + z + z ** 2 / 2 + z ** 3 / 6 + z ** 4 / 24)
    assert np.allclose(got, want, rtol=1e-15, atol=1e-15)


def test_rk4_converges_at_fourth_order():
    """Nonlinear autonomous system dy/dt = -y^2 (y(t) = 1 / (1 + t)): halving dt divides the
    error at t = 1 by 2^4."""
    def run(n):
        y = np.array([1.0])
        for _ in range(n):
            y = osolver.rk4_step(y, lambda v: -v * v, 1.0 / n)
        return abs(y[0] - 0.5)
    e1, e2 = run(8), run(16)
    assert 14.0 < e1 / e2 < 18.0


def test_planted_mistake_in_an_rk4_weight_breaks_the_pin(monkeypatch):
    def wrong(y0, rate, dt):
        k1 = rate(y0)
        k2 = rate(y0 + 0.5 * dt * k1)
        k3 = rate(y0 + 0.5 * dt * k2)
        k4 = rate(y0 + dt * k3)
        return y0 + dt * (k1 + 2.0 * k2 + k3 + 2.0 * k4) / 6.0
    y0 = np.array([1.0])
    z = 0.3
    assert abs(wrong(y0, lambda y: z * y, 1.0)[0] - (1 + z + z * z / 2 + z ** 3 / 6 + z ** 4 / 24)) > 1e-4


# ------------------------------------------------------------------ CBC relax
def _y_invariant_run(edges, beta):
    fields = wl.density_step(30, 6, Ma=0.1, W=0, Wy=0)
    o = OracleLBM(30, 6, 0, 0.8, 0.0, 2, "nrbc", q=17, nrbc_edges=edges, beta=beta,
                  mean=(1.0, 0.1, 0.0, 1.0), periodic_y=True)
    o.init(*fields)
    o.step(40)
    return o


def test_cbc_relax_equals_pnr_on_a_y_invariant_state():
    """On a y-invariant state the transverse amplitudes T_cal vanish, so Eq. (CBC-Relax) with
    the CBC evolution reduces to Eq. (PNR) with the LODI evolution, bit for bit."""
    a = _y_invariant_run((1, 1, 0, 0), 0.3)
    b = _y_invariant_run((0, 0, 0, 0), 0.3)
    assert np.array_equal(a.f, b.f)
    for e in ("W", "E"):
        for va, vb in zip(a.Utgt[e], b.Utgt[e]):
            assert np.array_equal(va, vb)


def test_cbc_relax_rate_uses_the_transverse_term():
    """At a single east-edge band node with tangential gradients only (of rho, u_y and T):
    PNR-LODI sees no normal variation (zero rate); CBC relax with beta = 1 keeps the whole
    transverse term, dU/dt = -B dU/dy (B the primitive Jacobian along y); beta = 0 makes the
    incoming (u - c) characteristic rate zero and leaves the other three as with beta = 1."""
    from oracle import characteristic as ch
    U = np.array([[1.0, 0.2, 0.0, 1.0]])           # rho, u_x, u_y, T at an east-edge node
    dUn = np.zeros((1, 4))
    dUt = np.array([[0.01, 0.0, 0.03, 0.02]])       # d/dy of rho, u_y, T (per node index)
    r = 1.3
    pnr = ch.rate(U, dUn, dUt, 0, +1.0, 0, 0.0, r)
    assert np.all(pnr == 0.0)
    full = ch.rate(U, dUn, dUt, 0, +1.0, 1, 1.0, r)
    B = ch.jacobian(U, 1)
    want = -np.einsum("nij,nj->ni", B, dUt / r)
    assert np.allclose(full, want, rtol=1e-14, atol=1e-16)
    # beta = 0: the incoming (u - c) amplitude plus its transverse part is zero, so the
    # incoming characteristic variable S_0 . dU/dt is zero and the others keep -T_cal
    frozen = ch.rate(U, dUn, dUt, 0, +1.0, 1, 0.0, r)
    S, lam = ch.eigen(U, 0)
    w = np.einsum("nij,nj->ni", S, frozen)
    wf = np.einsum("nij,nj->ni", S, full)
    assert abs(w[0, 0]) < 1e-16 and abs(wf[0, 0]) > 1e-4
    assert np.allclose(w[0, 1:], wf[0, 1:], rtol=1e-14, atol=1e-18)


@pytest.mark.parametrize("Ma", [0.1, 0.3])
def test_oblique_wave_reflects_less_with_cbc_relax_than_with_pnr(Ma):
    """Sec. 5.2 ordering on a wave that leaves through the east edge at an angle (pulse near the
    south-east corner, mean flow Mach Ma along x, D2Q17, no PML): the east edge with
    Eq. (CBC-Relax) at beta = Ma (reading: incoming L_bar = -(1 - beta) T_cal) lets less of the
    wave back into the domain than Eq. (PNR); the printed sign (relax_sign = +1), which adds
    the transverse term twice, reflects more than both. Error: L2 of rho - rho_ref over the
    domain after 40 steps, rho_ref from a periodic run padded beyond every signal."""
    N, steps, pad, tau = 48, 40, 80, 0.8
    centre = (N - 12, N // 2 - 14)

    def run(bc, edges=(0, 0, 0, 0), beta=0.0, rs=-1.0, p=0):
        n = N + 2 * p
        f = wl.pressure_pulse(n, n, 0, amp=1e-3, halfwidth=3, u0=(Ma, 0.0),
                              center=(centre[0] + p, centre[1] + p))
        o = OracleLBM(n, n, 0, tau, 0.0, 2, bc, q=17, nrbc_edges=edges, beta=beta,
                      mean=(1.0, Ma, 0.0, 1.0), relax_sign=rs)
        o.init(*f)
        o.step(steps)
        return o.fields()[0][p:p + N, p:p + N]

    ref = run("periodic", p=pad)
    err = {k: float(np.sqrt(np.sum((run("nrbc", *a) - ref) ** 2))) for k, a in
           {"pnr": ((0, 0, 0, 0),), "relax": ((0, 1, 0, 0), Ma),
            "printed": ((0, 1, 0, 0), Ma, +1.0)}.items()}
    assert err["relax"] < 0.95 * err["pnr"]
    assert err["printed"] > 1.2 * err["pnr"]

"""Pins of the oracle's time step, PML and boundary conditions (Secs. 2-5)."""
import math

import numpy as np
import pytest

import workloads as wl
from oracle import OracleLBM, characteristic as ch, metrics, pml
from oracle.stencil import lattice


def test_free_streaming_is_an_exact_permutation():
    """tau = inf (no collision) on a periodic grid: n steps move each population by n e_i."""
    nx, ny, n = 13, 11, 5
    o = OracleLBM(nx, ny, 0, float("inf"), bc="periodic")
    o.init(*wl.uniform(nx, ny, 0))
    M = o.M
    ids = (1000.0 + np.arange(37 * ny * nx, dtype=np.float64)).reshape(37, ny, nx)
    o.f[o.Fs] = ids
    o._fill_gamma(o.f)
    o.step(n)
    got = o.f[o.Fs]
    y, x = np.meshgrid(np.arange(ny), np.arange(nx), indexing="ij")
    for i, (ex, ey) in enumerate(o.lat.e):
        src = ids[i, (y - n * ey) % ny, (x - n * ex) % nx]
        assert np.array_equal(got[i], src)


def test_periodic_run_conserves_totals():
    o = OracleLBM(24, 20, 0, 0.6, bc="periodic")
    o.init(*wl.random_smooth_state(24, 20, 0, seed=5, du=0.1, mean_u=(0.1, -0.05)))
    a = o.totals()
    o.step(200)
    b = o.totals()
    assert np.all(np.abs(b - a) <= 1e-13 * np.abs(a).max())


def test_sigma_profile():
    Lx, Ly, W = 20, 16, 4
    i = pml.layer_index(Lx, Ly, W)
    assert i[8, 0] == W and i[8, W - 1] == 1 and i[8, W] == 0       # left strip
    assert i[0, 0] == W and i[1, 2] == max(W - 1, W - 2)            # corner: Chebyshev
    s = pml.sigma_field(Lx, Ly, W, 0.2, 3)
    assert s[8, 0] == pytest.approx(0.2) and s[8, W - 1] == pytest.approx(0.2 / W ** 3)
    assert s[8, W] == 0.0


def test_gradient_exact_on_quadratics():
    """Both Eq. (FD-dx-center) and Eq. (FD-dx-bw) are exact for quadratic fields; a sign or
    index slip in either is caught at the interior or at the outermost layer."""
    Ly, Lx = 9, 12
    y, x = np.meshgrid(np.arange(Ly, dtype=float), np.arange(Lx, dtype=float), indexing="ij")
    Q = np.stack([0.3 * x * x - 0.7 * x * y + 0.2 * y * y + x - 2 * y + 0.5,
                  -x * x + 3 * x * y + 0.1 * y])
    gx, gy = pml.gradient(Q)
    assert np.allclose(gx[0], 0.6 * x - 0.7 * y + 1, atol=1e-12)
    assert np.allclose(gy[0], -0.7 * x + 0.4 * y - 2, atol=1e-12)
    assert np.allclose(gx[1], -2 * x + 3 * y, atol=1e-12)
    assert np.allclose(gy[1], 3 * x + 0.1, atol=1e-12)


def test_trapezoid_exact_for_linear_in_time():
    """Q(t) = int_0^t f_hat: exact for f_hat linear in t (trapezoidal rule)."""
    a, b = 0.3, -0.05
    Q = np.zeros(1)
    prev = np.array([a])
    for n in range(1, 20):
        now = np.array([a + b * n])
        Q = pml.trapezoid_update(Q, prev, now)
        prev = now
        assert Q[0] == pytest.approx(a * n + 0.5 * b * n * n, abs=1e-13)


def test_pml_with_zero_sigma_is_plain_lbm_bit_for_bit():
    """Sec. 3: the PML acts only through the modified collision; sigma_max = 0 reproduces the
    plain scheme on the same grid bit for bit."""
    a = OracleLBM(24, 24, 6, 0.7, 0.0, 3, "zg")
    b = OracleLBM(24, 24, 6, 0.7, 0.0, 3, "zg", pml_on=False)   # same grid, no PML branch
    fields = wl.pressure_pulse(24, 24, 6, amp=1e-3, halfwidth=3)
    a.init(*fields)
    b.init(*fields)
    a.step(30)
    b.step(30)
    assert np.array_equal(a.f, b.f)


def test_mean_state_is_a_fixed_point_with_pml_and_nrbc():
    mean = (1.0, 0.2, -0.1, 1.05)
    o = OracleLBM(20, 20, 4, 0.6, 0.3, 3, "nrbc", nrbc_edges=(1, 0, 1, 0), beta=0.4, mean=mean)
    o.init(*wl.uniform(20, 20, 4, *mean))
    o.step(20)
    for fld, m in zip(o.fields(), mean):
        assert np.max(np.abs(fld - m)) < 1e-13


def test_characteristic_decomposition():
    """S A S^-1 = Lambda with A from the primitive Euler equations (Eq. NSF-CHAR), and keeping
    every wave reproduces dU/dt = -A dU/dx."""
    rng = np.random.default_rng(7)
    U = np.stack([rng.uniform(0.8, 1.2, 30), rng.uniform(-0.4, 0.4, 30),
                  rng.uniform(-0.4, 0.4, 30), rng.uniform(0.8, 1.2, 30)], -1)
    for axis in (0, 1):
        A = ch.jacobian(U, axis)
        S, lam = ch.eigen(U, axis)
        SASi = S @ A @ np.linalg.inv(S)
        assert np.allclose(SASi, np.einsum("ni,ij->nij", lam, np.eye(4)), atol=1e-13)
        # eigenvalues from numpy's general eigen-solver
        ev = np.sort(np.linalg.eigvals(A).real, axis=-1)
        assert np.allclose(ev, np.sort(lam, axis=-1), atol=1e-12)
        dU = rng.standard_normal((30, 4))
        full = -np.einsum("nij,nj->ni", np.linalg.inv(S),
                          lam * np.einsum("nij,nj->ni", S, dU))
        assert np.allclose(full, -np.einsum("nij,nj->ni", A, dU), atol=1e-12)


def test_sound_speed_is_adiabatic():
    """c^2 = gamma T with gamma = (D + 2) / D = 2 for the monatomic gas of Sec. 2."""
    U = np.array([[1.0, 0.0, 0.0, 1.3]])
    _, lam = ch.eigen(U, 0)
    assert lam[0, 3] == pytest.approx(math.sqrt(2 * 1.3), abs=1e-15)


@pytest.mark.slow
def test_pml_and_nrbc_reduce_reflections():
    """Directional claims of Sec. 5 on the averaged global error e_bar_Z (Sec. 5 metrics) of a
    pulse leaving a 40^2 bulk, against a periodic reference on a 240^2 grid: ZG + PML beats
    ZG alone, the characteristic BC beats ZG, and adding the PML to it helps further."""
    nx, tau, pad = 40, 0.8, 100
    pulse = lambda n, W: wl.pressure_pulse(n, n, W, amp=1e-3, halfwidth=3.0)
    big = nx + 2 * pad
    ref = OracleLBM(big, big, 0, tau, bc="periodic")
    ref.init(*pulse(big, 0))
    refs = []
    for _ in range(7):
        ref.step(10)
        refs.append(ref.fields()[0][pad:pad + nx, pad:pad + nx])

    def ebar(W, sig, bc):
        o = OracleLBM(nx, nx, W, tau, sig, 3, bc)
        o.init(*pulse(nx, W))
        errs = []
        for k in range(7):
            o.step(10)
            errs.append(metrics.e_Z(o.fields("bulk")[0], refs[k]))
        return float(np.mean(errs))

    zg, zg_pml = ebar(0, 0.0, "zg"), ebar(12, 0.3, "zg")
    nrbc, nrbc_pml = ebar(0, 0.0, "nrbc"), ebar(12, 0.1, "nrbc")
    assert zg_pml < zg / 2
    assert nrbc < zg
    assert nrbc_pml < nrbc / 1.5


def test_centred_pulse_symmetry():
    nx, W = 30, 6
    o = OracleLBM(nx, nx, W, 0.7, 0.1, 3, "zg")
    o.init(*wl.pressure_pulse(nx, nx, W, amp=1e-3, halfwidth=3.0))
    o.step(40)
    rho = o.fields()[0] - 1.0
    # the signal is ~1e-5; a mirrored index or sign slip breaks symmetry at that scale, while
    # summation order leaves a few ulps of rho ~ 1
    assert np.abs(rho).max() > 1e-6
    assert np.max(np.abs(rho - rho[:, ::-1])) < 1e-13
    assert np.max(np.abs(rho - rho[::-1, :])) < 1e-13
    assert np.max(np.abs(rho - rho.T)) < 1e-13


def test_light_cone_bit_exact():
    """Bulk nodes farther than 4n from P and Gamma after n steps equal a periodic run of the
    same size bit for bit (the BC and PML have not reached them)."""
    nx, W, n = 40, 4, 3
    L = nx + 2 * W
    fields = wl.random_smooth_state(nx, nx, W, seed=9)
    a = OracleLBM(nx, nx, W, 0.7, 0.2, 2, "nrbc", nrbc_edges=(1, 1, 0, 0), beta=0.3)
    b = OracleLBM(L, L, 0, 0.7, bc="periodic")
    a.init(*fields)
    b.init(*fields)
    a.step(n)
    b.step(n)
    d = W + 4 * n + 1
    sl = (slice(None), slice(a.M + d, a.M + L - d), slice(a.M + d, a.M + L - d))
    assert np.array_equal(a.f[sl], b.f[sl])
    assert not np.array_equal(a.f, b.f)


@pytest.mark.slow
def test_acoustic_pulse_against_linear_closed_form():
    """Small isentropic pulse, u0 = 0: p'(r, t) = (A / 2a) int e^{-k^2/4a} e^{-nu k^2 t}
    cos(c k t) J0(k r) k dk with a = ln2 / b^2, c = sqrt(gamma) c_s = sqrt(2)/r nodes/step and
    sound damping nu = (tau - 1/2) c_s^2 (D = 2, Pr = 1). Pins feq, moments, collision and
    streaming together: an isothermal or mis-scaled equilibrium changes the sound speed."""
    from scipy.integrate import quad
    from scipy.special import j0
    lat = lattice(37)
    nx, tau, amp, b, t = 96, 0.8, 1e-4, 6.0, 24
    o = OracleLBM(nx, nx, 0, tau, bc="periodic")
    o.init(*wl.pressure_pulse(nx, nx, 0, amp=amp, halfwidth=b))
    o.step(t)
    rho, ux, uy, T = o.fields()
    p = rho * T - 1.0
    cy = (nx - 1) / 2.0
    a = math.log(2.0) / b ** 2
    c = math.sqrt(2.0) / lat.r
    nu = (tau - 0.5) / lat.r ** 2
    xs = np.arange(nx // 2, nx - 4)
    row = int(cy)                      # nodes of this row sit half a node off the centre line
    rr = np.sqrt((xs - cy) ** 2 + (row - cy) ** 2)
    want = np.array([amp / (2 * a) * quad(
        lambda k: math.exp(-k * k / (4 * a) - nu * k * k * t) * math.cos(c * k * t) * j0(k * r) * k,
        0, 12 * math.sqrt(a), limit=400)[0] for r in rr])
    got = p[row, xs]
    assert np.max(np.abs(got - want)) < 0.005 * amp   # measured 0.11 %; isothermal c: 18 %


@pytest.mark.parametrize("bc,W", [("zg", 0), ("zg", 6), ("nrbc", 6)])
def test_periodic_y_keeps_a_y_invariant_state_y_invariant(bc, W):
    """Sec. 5.1 setting: a density step that does not depend on y, on a y-periodic grid with
    PML / outflow BC on the x edges, stays y-invariant, and the row does not depend on ny (a
    wrong wrap or a y-boundary treatment applied on the periodic axis breaks both)."""
    rows = []
    for ny in (8, 11):
        o = OracleLBM(40, ny, W, 0.7, 0.05, 2, bc, periodic_y=True)
        o.init(*wl.density_step(40, ny, Ma=0.05, W=W, Wy=0))
        o.step(25)
        rho = o.fields("F")[0]
        assert rho.shape == (ny, 40 + 2 * W)
        assert np.array_equal(rho, np.broadcast_to(rho[0], rho.shape))
        rows.append(rho[0])
    assert np.array_equal(rows[0], rows[1])
    assert np.abs(rows[0][W:W + 40] - rows[0][W:W + 40].mean()).max() > 1e-3


def test_periodic_y_light_cone_matches_fully_periodic_run():
    """Away from the x edges a y-periodic run equals a fully periodic one bit for bit."""
    nx, ny, n = 40, 14, 3
    fields = wl.random_smooth_state(nx, ny, 0, seed=5)
    a = OracleLBM(nx, ny, 0, 0.7, bc="zg", periodic_y=True)
    b = OracleLBM(nx, ny, 0, 0.7, bc="periodic")
    a.init(*fields)
    b.init(*fields)
    a.step(n)
    b.step(n)
    d = 4 * n + 1
    fa, fb = a.fields(), b.fields()
    for za, zb in zip(fa, fb):
        assert np.array_equal(za[:, d:nx - d], zb[:, d:nx - d])
    assert not np.array_equal(fa[0], fb[0])


def test_per_axis_pml_widths_transpose():
    """W on the x edges and Wy on the y edges: the run of the transposed problem, with the
    widths swapped, is the transposed run (catches a width used on the wrong axis)."""
    nx, ny, W, Wy = 30, 22, 6, 3
    a = OracleLBM(nx, ny, W, 0.7, 0.1, 2, "zg", Wy=Wy)
    b = OracleLBM(ny, nx, Wy, 0.7, 0.1, 2, "zg", Wy=W)
    c = (11.0, 7.0)
    a.init(*wl.pressure_pulse(nx, ny, W, amp=1e-3, halfwidth=3.0, center=c, Wy=Wy))
    b.init(*wl.pressure_pulse(ny, nx, Wy, amp=1e-3, halfwidth=3.0, center=c[::-1], Wy=W))
    a.step(40)
    b.step(40)
    ra, rb = a.fields("F")[0] - 1.0, b.fields("F")[0] - 1.0
    assert ra.shape == (ny + 2 * Wy, nx + 2 * W)
    assert np.abs(ra[:, :W]).max() > 1e-8          # the pulse has reached both PML slabs
    assert np.abs(ra[:Wy, :]).max() > 1e-8
    assert np.max(np.abs(ra - rb.T)) < 1e-13
    sa = pml.sigma_field(nx + 2 * W, ny + 2 * Wy, W, 0.1, 2, Wy)
    assert sa[Wy + 5, 0] == pytest.approx(0.1) and sa[0, W + 5] == pytest.approx(0.1)
    assert sa[Wy + 5, 1] == pytest.approx(0.1 * (5 / 6) ** 2)
    assert sa[1, W + 5] == pytest.approx(0.1 * (2 / 3) ** 2)


@pytest.mark.parametrize("split", [False, True])
def test_pml_first_step_closed_form(split):
    """Uniform density excess delta at rest, sigma = sigma_max on all of P (p = 0), Q^0 = 0:
    the first step adds -(sigma_x + sigma_y) f_hat (Eq. pml-general), and a node whose pull
    sources all lie in one zone reads rho = 1 + delta (1 - sigma_x - sigma_y), T = 1, u = 0.
    Equal sigmas (Eq. PMLCOLL): 1 - 2 sigma on all of P. Split: 1 - sigma in a slab, 1 - 2 sigma
    in a corner. Bulk: 1 + delta."""
    nx, W, s, d = 16, 10, 0.05, 1e-3
    o = OracleLBM(nx, nx, W, 0.7, s, 0, "zg", sigma_split=split)
    L = nx + 2 * W
    o.init(*wl.uniform(nx, nx, W, rho=1.0 + d))
    o.step(1)
    rho, ux, uy, T = o.fields("F")
    slab = rho[L // 2, 5]
    corner = rho[5, 5]
    bulk = rho[L // 2, L // 2]
    assert bulk == pytest.approx(1.0 + d, abs=1e-14)
    assert slab == pytest.approx(1.0 + d * (1.0 - (1.0 if split else 2.0) * s), abs=1e-14)
    assert corner == pytest.approx(1.0 + d * (1.0 - 2.0 * s), abs=1e-14)
    for z in (slab, corner):
        assert abs(z - (1.0 + d)) > 0.5 * s * d          # the term acted
    for (y, x) in ((L // 2, 5), (5, 5), (L // 2, L // 2)):
        assert abs(T[y, x] - 1.0) < 1e-13 and abs(ux[y, x]) < 1e-13 and abs(uy[y, x]) < 1e-13


def test_split_x_slab_ignores_the_x_gradient(monkeypatch):
    """In the split form the x derivative of Q is weighted by sigma_y, which is zero in a PML
    slab on the x edges: on a y-periodic grid with PML only on the x edges and a y-invariant
    state, scaling the x derivative changes nothing (and changes the sigma_x = sigma_y run)."""
    nx, ny, W = 40, 8, 8

    def run(split):
        o = OracleLBM(nx, ny, W, 0.7, 0.1, 2, "zg", periodic_y=True, sigma_split=split)
        o.init(*wl.density_step(nx, ny, Ma=0.05, W=W, Wy=0))
        o.step(12)
        return o.fields("F")[0]

    base = {sp: run(sp) for sp in (False, True)}
    orig = pml.gradient

    def scaled(Q, periodic_y=False):
        gx, gy = orig(Q, periodic_y)
        return 3.0 * gx, gy

    monkeypatch.setattr(pml, "gradient", scaled)
    assert np.array_equal(run(True), base[True])
    assert np.abs(run(False) - base[False]).max() > 1e-9


@pytest.mark.parametrize("split,src", [(False, 0), (True, 0), (False, 7), (True, 1)])
def test_per_edge_widths_mirror(split, src):
    """Widths (W_w, W_e) = (3, 7) and the x-mirrored problem with (7, 3): mirrored results
    (catches a width, a layer fraction or an Appendix PML source taken from the wrong edge)."""
    nx, ny = 26, 20
    a = OracleLBM(nx, ny, (3, 7, 4, 2), 0.7, 0.1, 2, "nrbc", sigma_split=split, pml_source=src)
    b = OracleLBM(nx, ny, (7, 3, 4, 2), 0.7, 0.1, 2, "nrbc", sigma_split=split, pml_source=src)
    c = (9.0, 8.0)
    a.init(*wl.pressure_pulse(nx, ny, (3, 7, 4, 2), amp=1e-3, halfwidth=3.0, center=c))
    b.init(*wl.pressure_pulse(nx, ny, (7, 3, 4, 2), amp=1e-3, halfwidth=3.0,
                              center=(nx - 1 - c[0], c[1])))
    a.step(40)
    b.step(40)
    ra, rb = a.fields("F")[0] - 1.0, b.fields("F")[0] - 1.0
    assert ra.shape == (ny + 6, nx + 10)
    assert np.abs(ra[:, :3]).max() > 1e-8 and np.abs(ra[:, -7:]).max() > 1e-8
    assert np.max(np.abs(ra - rb[:, ::-1])) < 1e-13


def test_density_step_profile():
    """Sec. 5.1 initial density: rho0 at both ends, plateau rho1 around the centre, continuous
    at Lx/2, half-way values at Lx/4 and 3Lx/4 (node counting from 1)."""
    rho, ux, uy, T = wl.density_step(200, 20, Ma=0.05)
    r = rho[0]
    assert r[0] == pytest.approx(1.0, abs=1e-12) and r[-1] == pytest.approx(1.0, abs=1e-12)
    assert r[99] == pytest.approx(1.05, abs=1e-9) and r[100] == pytest.approx(1.05, abs=1e-9)
    assert r[49] == pytest.approx(1.025) and r[149] == pytest.approx(1.025)
    assert np.abs(np.diff(r)).max() < 0.05 * 0.5 / 2 + 1e-12     # no jump anywhere
    assert np.all(ux == 0.05) and np.all(uy == 0.0) and np.all(T == 1.0)


def test_conserved_to_primitive_rate_is_the_derivative_of_the_variable_map():
    """Appendix source mapping: d(rho, u, T) from d(rho, rho u, E) equals the derivative of
    u = m / rho, T = (2 E / rho - u^2) / D along the same conserved perturbation."""
    rng = np.random.default_rng(3)
    U = np.column_stack([1 + 0.1 * rng.random(5), 0.2 * rng.standard_normal(5),
                         0.2 * rng.standard_normal(5), 1 + 0.1 * rng.random(5)])

    def cons(U):
        rho, ux, uy, T = U.T
        return np.column_stack([rho, rho * ux, rho * uy, 0.5 * rho * (ux * ux + uy * uy + 2 * T)])

    def prim(C):
        rho, mx, my, E = C.T
        ux, uy = mx / rho, my / rho
        return np.column_stack([rho, ux, uy, (2 * E / rho - ux * ux - uy * uy) / 2])

    dC = rng.standard_normal((5, 4))
    h = 1e-6
    fd = (prim(cons(U) + h * dC) - prim(cons(U) - h * dC)) / (2 * h)
    got = ch.conserved_to_primitive_rate(dC[:, 0], dC[:, 1:3].T, dC[:, 3], U)
    assert np.max(np.abs(got - fd)) < 1e-8


def test_pml_source_first_step_closed_form():
    """Appendix term II at the first step from a uniform density excess delta at rest (Q^0 = 0,
    so terms I and III vanish): the outermost PML layer (sigma = sigma_max) gets
    d rho / dt = -2 sigma_max delta (the mass moment of -2 sigma f_hat), du = dT = 0; term I
    alone gives zero."""
    nx, W, s, d = 16, 6, 0.05, 1e-3
    for src, want in ((2, -2.0 * s * d), (1, 0.0), (7, -2.0 * s * d), (10, 2.0 * s * d)):
        o = OracleLBM(nx, nx, W, 0.7, s, 2, "nrbc", pml_source=src)
        o.init(*wl.uniform(nx, nx, W, rho=1.0 + d))
        o.step(1)
        for edge in ("W", "E", "S", "N"):
            v = o._src[edge]
            assert np.allclose(v[:, 0], want, rtol=1e-12, atol=1e-18), (src, edge)
            assert np.abs(v[:, 1:]).max() < 1e-16
    o = OracleLBM(nx, nx, W, 0.7, s, 2, "nrbc")
    o.init(*wl.uniform(nx, nx, W, rho=1.0 + d))
    o.step(1)
    assert o._src is None

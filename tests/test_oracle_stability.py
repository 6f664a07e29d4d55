"""Linear stability of the PML collision (Sec. 3), rest state, homogeneous sigma.

Von Neumann analysis of one step per Fourier mode k: f_hat = J f with J the Jacobian of
f -> f_eq(U(f)) taken from the oracle's own equilibrium; collide
f* = f - (f - f_hat)/tau - sigma (G Q + 2 f_hat + sigma Q); stream f_i <- e^{-i k.e_i} f*_i.
G is the symbol of c_i . grad:
  central (Eqs. FD-dx-center, as printed): i (e_ix sin k_x + e_iy sin k_y)
  link (integral of c_i . grad Q along one lattice link, the pml_grad = "link" option):
       e^{i k.e_i} - 1.
Readings of the time levels tried with the printed central differences (state per mode:
f^n, Q^(n-1), f_hat^(n-1)):
  trapezoid   Q^n = Q^(n-1) + (f_hat^(n-1) + f_hat^n)/2, Omega^n uses Q^n (the oracle)
  lagged_grad grad Q^(n-1) in Omega^n (cheaper reading of "(x, t)")
  lagged_q    Q^(n-1) everywhere in Omega^n
  euler       Q^n = Q^(n-1) + f_hat^(n-1) (explicit rule instead of the trapezoid)
  predictor   Q^(n+1) = Q^n + (f_hat^n + f_hat(f*^n))/2 from the post-collision state at the same
              node, Omega^n uses Q^n (the printed "f_eq at t + dt" read as a predictor)
Finding pinned here: every one of these readings of the printed central differences has
modes with |lambda| > 1 for sigma > 0, and for D2Q37 the y-invariant modes (the Sec. 5.1
density-step setting) grow at about 0.4 sigma per step (k_x near 2 pi / 3, where the speed-3
populations stream with phase 1 but the central difference does not vanish); the link form
keeps max |lambda| = 1.
"""
import numpy as np
import pytest

from oracle.equilibrium import feq, moments
from oracle.stencil import lattice

_J = {}


def _jacobian(q):
    if q not in _J:
        L = lattice(q)
        f0 = feq(np.float64(1.0), np.zeros(2), np.float64(1.0), L.xi, L.w, L.order)

        def g(f):
            r, u, T = moments(f, L.xi)
            return feq(r, u, T, L.xi, L.w, L.order)
        J = np.zeros((q, q))
        h = 1e-7
        for j in range(q):
            d = np.zeros(q)
            d[j] = h
            J[:, j] = (g(f0 + d) - g(f0 - d)) / (2 * h)
        _J[q] = (L, J)
    return _J[q]


def amplification(q, sigma, tau, kx, ky, grad="central", reading="trapezoid"):
    L, J = _jacobian(q)
    e = L.e.astype(float)
    n = q
    I, Z = np.eye(n), np.zeros((n, n))
    phase = e[:, 0] * kx + e[:, 1] * ky
    if grad == "central":
        G = np.diag(1j * (e[:, 0] * np.sin(kx) + e[:, 1] * np.sin(ky)))
    else:
        G = np.diag(np.exp(1j * phase) - 1.0)
    S = np.diag(np.exp(-1j * phase))
    fn = np.hstack([I, Z, Z])
    fh = np.hstack([J, Z, Z])
    Qprev = np.hstack([Z, I, Z])
    Qtrap = np.hstack([0.5 * J, I, 0.5 * I])
    if reading == "predictor":
        # state (f^n, Q^n, unused): Omega^n uses Q^n, then Q^(n+1) from f^n and f*^n
        Qn = Qprev
        fs = fn - (fn - fh) / tau - sigma * (G @ Qn + 2 * fh + sigma * Qn)
        Qnext = Qn + 0.5 * (fh + J @ fs)
        A = np.vstack([S @ fs, Qnext, np.hstack([Z, Z, I])])
        return float(np.abs(np.linalg.eigvals(A)).max())
    if reading == "euler":
        Qn = np.hstack([Z, I, I])
        gq, qq = G @ Qn, Qn
    elif reading == "lagged_grad":
        Qn = Qtrap
        gq, qq = G @ Qprev, Qn
    elif reading == "lagged_q":
        Qn = Qtrap
        gq, qq = G @ Qprev, Qprev
    else:
        Qn = Qtrap
        gq, qq = G @ Qn, Qn
    fs = fn - (fn - fh) / tau - sigma * (gq + 2 * fh + sigma * qq)
    A = np.vstack([S @ fs, Qn, fh])
    return float(np.abs(np.linalg.eigvals(A)).max())


def worst(q, sigma, tau, grad="central", reading="trapezoid", nk=13, ky_zero=False):
    ks = np.linspace(0, np.pi, nk)
    kys = [0.0] if ky_zero else ks
    return max(amplification(q, sigma, tau, kx, ky, grad, reading) for kx in ks for ky in kys)


def test_plain_lbm_is_neutrally_stable():
    assert worst(37, 0.0, 0.8) == pytest.approx(1.0, abs=1e-9)


@pytest.mark.parametrize("tau", [0.55, 0.8])
def test_printed_central_gradient_is_unstable(tau):
    assert worst(37, 0.05, tau) > 1.005


@pytest.mark.parametrize("reading", ["trapezoid", "lagged_grad", "lagged_q", "euler", "predictor"])
def test_every_time_level_reading_of_the_printed_scheme_is_unstable_for_d2q37(reading):
    """y-invariant modes (k_y = 0) of D2Q37, tau 0.8: growth per step above 1 + 0.1 sigma for
    sigma 0.01 and 0.1, whatever the time level of Q and grad Q."""
    for sigma in (0.01, 0.1):
        assert worst(37, sigma, 0.8, "central", reading, nk=49, ky_zero=True) > 1 + 0.1 * sigma


def test_d2q37_grows_much_faster_than_d2q17_on_y_invariant_modes():
    """Why the Sec. 5.1 D2Q17 runs survive 2000 steps and the D2Q37 runs do not: at sigma 0.01
    the y-invariant growth rate of D2Q37 is more than ten times that of D2Q17."""
    g37 = worst(37, 0.01, 0.8, nk=49, ky_zero=True) - 1.0
    g17 = worst(17, 0.01, 0.8, nk=49, ky_zero=True) - 1.0
    assert g37 > 10.0 * g17 > 0.0


@pytest.mark.parametrize("q", [9, 17, 37])
@pytest.mark.parametrize("tau", [0.55, 0.8])
def test_link_gradient_is_stable(q, tau):
    for sigma in (0.01, 0.1, 0.35):
        assert worst(q, sigma, tau, "link", nk=9) <= 1.0 + 1e-9


def test_density_step_d2q37_diverges_with_the_printed_gradient_and_not_with_the_link_form():
    """The Sec. 5.1 setting in small (60 x 4 bulk, periodic y, PML W 20 on the x edges, Table 1
    D2Q37 ZG sigma_max 0.175, quadratic ramp, tau 0.8, Mach 0.05): the printed central
    differences blow up within 400 steps; the link-integrated gradient stays bounded by the
    initial step height over 600 steps."""
    import workloads as wl
    from oracle import OracleLBM
    out = {}
    for mode in ("central", "link"):
        f = wl.density_step(60, 4, Ma=0.05, W=20, Wy=0)
        o = OracleLBM(60, 4, 20, 0.8, 0.175, 2, "zg", q=37, mean=(1.0, 0.05, 0.0, 1.0),
                      periodic_y=True, pml_grad=mode)
        o.init(*f)
        peak = 0.0
        with np.errstate(all="ignore"):
            for _ in range(12 if mode == "link" else 8):
                o.step(50)
                r = o.fields()[0]
                peak = float(np.max(np.abs(r - 1.0))) if np.all(np.isfinite(r)) else np.inf
                if peak > 1.0:
                    break
        out[mode] = peak
    assert out["central"] > 1.0
    assert out["link"] < 0.05

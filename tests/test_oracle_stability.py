"""Linear stability of the PML collision as printed (Sec. 3), D2Q37, rest state.

Von Neumann analysis of one step with a homogeneous sigma: state (f^n, Q^(n-1), f_hat^(n-1))
per Fourier mode k; f_hat = J f with J the Jacobian of f -> f_eq(U(f)) taken from the
oracle's own equilibrium; Q^n = Q^(n-1) + (f_hat^(n-1) + f_hat^n)/2; collide
f* = f - (f - f_hat)/tau - sigma (e_i . G Q^n + 2 f_hat + sigma Q^n); stream f_i <- e^{-i k.e_i} f*_i.
G is the symbol of the gradient:
  central (Eqs. FD-dx-center, as printed): i sin(k_x), i sin(k_y) per axis
  characteristic (integral of c_i . grad Q along one lattice link): e^{i k.e_i} - 1.
Finding pinned here: with the printed central differences the scheme has modes with
|lambda| > 1 for every sigma > 0, so long runs with a PML grow unboundedly (the growth is
convective and slow for a thin ramped layer, fast for small tau); the characteristic form
keeps max |lambda| = 1. This motivates reporting LBM_EUNSTABLE rather than masking it.
"""
import numpy as np
import pytest

from oracle.equilibrium import feq, moments
from oracle.stencil import lattice


def _jacobian():
    L = lattice(37)
    f0 = feq(np.float64(1.0), np.zeros(2), np.float64(1.0), L.xi, L.w, 4)

    def g(f):
        r, u, T = moments(f, L.xi)
        return feq(r, u, T, L.xi, L.w, 4)
    J = np.zeros((37, 37))
    h = 1e-7
    for j in range(37):
        d = np.zeros(37)
        d[j] = h
        J[:, j] = (g(f0 + d) - g(f0 - d)) / (2 * h)
    return L, J


def max_amplification(sigma, tau, grad, nk=13):
    L, J = _jacobian()
    e = L.e.astype(float)
    I, Z = np.eye(37), np.zeros((37, 37))
    worst = 0.0
    for kx in np.linspace(0, np.pi, nk):
        for ky in np.linspace(0, np.pi, nk):
            phase = e[:, 0] * kx + e[:, 1] * ky
            if grad == "central":
                G = np.diag(e[:, 0] * 1j * np.sin(kx) + e[:, 1] * 1j * np.sin(ky))
            else:
                G = np.diag(np.exp(1j * phase) - 1.0)
            Qn = np.hstack([0.5 * J, I, 0.5 * I])
            fh = np.hstack([J, Z, Z])
            fn = np.hstack([I, Z, Z])
            fs = fn - (fn - fh) / tau - sigma * (G @ Qn + 2 * fh + sigma * Qn)
            A = np.vstack([np.diag(np.exp(-1j * phase)) @ fs, Qn, fh])
            worst = max(worst, float(np.abs(np.linalg.eigvals(A)).max()))
    return worst


def test_plain_lbm_is_neutrally_stable():
    assert max_amplification(0.0, 0.8, "central") == pytest.approx(1.0, abs=1e-9)


@pytest.mark.parametrize("tau", [0.55, 0.8])
def test_printed_central_gradient_is_unstable(tau):
    assert max_amplification(0.05, tau, "central") > 1.005


@pytest.mark.parametrize("tau", [0.55, 0.8])
def test_characteristic_gradient_is_stable(tau):
    assert max_amplification(0.1, tau, "characteristic") <= 1.0 + 1e-9

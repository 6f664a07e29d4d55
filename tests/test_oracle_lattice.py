"""Pins of the oracle's stencils, equilibria and BGK collision (Sec. 2).

Each check is against something other than the oracle's own formulas: textbook closed forms,
an independent Gauss-Hermite product rule from numpy, closed-form Gaussian moments, and the
conservation laws the method must satisfy.
"""
import numpy as np
import pytest
from numpy.polynomial.hermite_e import hermegauss

from oracle import equilibrium as eq
from oracle import stencil
from oracle.stencil import lattice


def gaussian_expectation(a, b, n=16):
    """E[x^a y^b] under the unit 2-D Gaussian via numpy's Gauss-HermiteE product rule."""
    x, w = hermegauss(n)
    w = w / w.sum()
    return float(np.sum(w * x ** a) * np.sum(w * x ** b))


@pytest.mark.parametrize("q", [9, 17, 37])
def test_velocity_sets(q):
    L = lattice(q)
    assert L.e.shape == (q, 2)
    assert len({tuple(v) for v in L.e.tolist()}) == q          # distinct
    assert int(np.abs(L.e).max()) == (1 if q == 9 else 3)     # max displacement M (Sec. 2)
    assert np.all(L.w > 0)                                      # non-negative weights
    # closed under the square's symmetry group
    s = {tuple(v) for v in L.e.tolist()}
    for ex, ey in s:
        assert (-ex, ey) in s and (ey, ex) in s


def test_d2q9_textbook_values():
    L = lattice(9)
    assert L.r == pytest.approx(np.sqrt(3.0), abs=1e-15)
    by_norm = {0: 4 / 9, 1: 1 / 9, 2: 1 / 36}
    for v, w in zip(L.e, L.w):
        assert w == pytest.approx(by_norm[int(v @ v)], abs=1e-15)


@pytest.mark.parametrize("q,deg", [(9, 5), (17, 7), (37, 9)])
def test_quadrature_degree_against_gauss_hermite(q, deg):
    """Every monomial of degree <= deg (odd, mixed, all) is integrated exactly; the rule is not
    exact one degree higher, so the degrees 5 / 7 / 9 of Sec. 2 are met and not exceeded."""
    L = lattice(q)
    xi = L.xi
    for a in range(deg + 1):
        for b in range(deg + 1 - a):
            got = float(np.sum(L.w * xi[:, 0] ** a * xi[:, 1] ** b))
            assert got == pytest.approx(gaussian_expectation(a, b), abs=2e-13), (a, b)
    misses = [abs(float(np.sum(L.w * xi[:, 0] ** a * xi[:, 1] ** (deg + 1 - a)))
                  - gaussian_expectation(a, deg + 1 - a))
              for a in range(0, deg + 2, 2)]
    assert max(misses) > 1e-3


def test_dropped_velocity_breaks_the_rule(monkeypatch):
    """Planted mistake: a shell generator that loses one mirror image must fail the rule."""
    orig = stencil.shell_members

    def lossy(a, b):
        m = orig(a, b)
        return m[:-1] if (a, b) == (2, 1) else m

    monkeypatch.setattr(stencil, "shell_members", lossy)
    stencil.lattice.cache_clear()
    try:
        with pytest.raises(AssertionError):
            stencil.lattice(37)
    finally:
        monkeypatch.undo()
        stencil.lattice.cache_clear()


def random_states(n, seed):
    rng = np.random.default_rng(seed)
    rho = rng.uniform(0.5, 2.0, n)
    ang = rng.uniform(0, 2 * np.pi, n)
    mag = rng.uniform(0, 0.5, n)
    u = np.stack([mag * np.cos(ang), mag * np.sin(ang)])
    T = rng.uniform(0.7, 1.5, n)
    return rho, u, T


@pytest.mark.parametrize("q", [9, 17, 37])
def test_equilibrium_returns_its_moments(q):
    """Sec. 2: the stencil/equilibrium pair must reproduce Eq. (macro)."""
    L = lattice(q)
    rho, u, T = random_states(500, 1)
    f = eq.feq(rho, u, T, L.xi, L.w, L.order)
    r2, u2, T2 = eq.moments(f, L.xi)
    assert np.max(np.abs(r2 / rho - 1)) < 1e-13
    assert np.max(np.abs(u2 - u)) < 1e-13
    assert np.max(np.abs(T2 / T - 1)) < 1e-13


def test_printed_mixed_term_breaks_mass():
    """Eq. (feq-4) as printed, (c^2 - 4), does not return rho; (c^2 - 6) does."""
    L = lattice(37)
    rho, u, T = np.array([1.1]), np.array([[0.2], [-0.1]]), np.array([1.3])
    printed = eq.feq(rho, u, T, L.xi, L.w, 4, mixed4_shift=4.0).sum(0)
    fixed = eq.feq(rho, u, T, L.xi, L.w, 4).sum(0)
    assert abs(fixed[0] - 1.1) < 1e-14
    # closed form of the printed error: rho (1 + (T - 1) u^2 / 2)
    assert printed[0] == pytest.approx(1.1 * (1 + 0.3 * 0.05 / 2), abs=1e-13)


def gaussian_moment_tensor(rho, u, T, idx):
    """rho E[prod xi_k] for xi ~ N(u, T I) (Isserlis / Wick), closed form."""
    idx = list(idx)
    if not idx:
        return rho

    def rec(rem):
        if not rem:
            return 1.0
        a = rem[0]
        rest = rem[1:]
        tot = u[a] * rec(rest)
        for k in range(len(rest)):
            if rest[k] == a:
                tot = tot + T * rec(rest[:k] + rest[k + 1:])
        return tot
    return rho * rec(idx)


@pytest.mark.parametrize("q,top", [(9, 2), (17, 3), (37, 4)])
def test_equilibrium_moments_match_maxwellian(q, top):
    """The Hermite equilibrium of order N carries the Maxwellian's moments up to order N."""
    L = lattice(q)
    rho, u, T = random_states(50, 2)
    f = eq.feq(rho, u, T, L.xi, L.w, L.order)
    import itertools
    for n in range(top + 1):
        for idx in itertools.product((0, 1), repeat=n):
            m = np.ones_like(L.xi[:, 0])
            for a in idx:
                m = m * L.xi[:, a]
            got = (f * m[:, None]).sum(0)
            want = gaussian_moment_tensor(rho, u, T, idx)
            assert np.max(np.abs(got - want)) < 1e-12, (q, idx)


def test_rest_equilibrium_is_the_weights():
    L = lattice(37)
    f = eq.feq(np.float64(1.0), np.array([0.0, 0.0]), np.float64(1.0), L.xi, L.w, 4)
    assert np.array_equal(f, L.w)


@pytest.mark.parametrize("tau", [0.52, 0.8, 2.0])
def test_bgk_conserves_mass_momentum_energy(tau):
    L = lattice(37)
    rng = np.random.default_rng(3)
    rho, u, T = random_states(200, 4)
    f = eq.feq(rho, u, T, L.xi, L.w, 4) * (1 + 0.05 * rng.standard_normal((37, 200)))
    r, uu, TT = eq.moments(f, L.xi)
    fs = eq.bgk(f, eq.feq(r, uu, TT, L.xi, L.w, 4), tau)
    xi = L.xi
    for m in (np.ones(37), xi[:, 0], xi[:, 1], (xi ** 2).sum(1)):
        a = (f * m[:, None]).sum(0)
        b = (fs * m[:, None]).sum(0)
        assert np.max(np.abs(a - b) / (np.abs(a) + 1)) < 1e-14

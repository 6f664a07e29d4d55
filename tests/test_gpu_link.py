"""Parity of the link-integrated PML gradient option (pml_grad = "link": c_i . grad Q_i as
Q_i(x + e_i) - Q_i(x), with Q also on the M-node bulk ring and on the boundary nodes outside F)
with the oracle's link mode, and its long-run stability where the printed central differences
blow up (the Sec. 5.1 D2Q37 setting).

Same tolerances as the other parity tests: FP64 path 1e-12, FP32-deviation path 1e-5.
"""
import numpy as np
import pytest

import workloads as wl
from parity_helpers import case_kwargs, check as _check, make_solver

pytestmark = pytest.mark.gpu


def check(kw, fields, steps, precision):
    _check(kw, fields, steps, precision, tag="link ")


@pytest.mark.parametrize("precision", ["fp64", "fp32dev"])
def test_link_pulse_64_pml8_zg(precision):
    c = wl.pulse_64()
    kw = case_kwargs(nx=c.nx, ny=c.ny, W=c.W, tau=c.tau, sigma_max=c.sigma_max,
                     sigma_power=c.sigma_power, bc=c.bc, pml_grad="link")
    check(kw, c.fields(), c.steps, precision)


@pytest.mark.parametrize("precision", ["fp64", "fp32dev"])
def test_link_vortex_nrbc_pml(precision):
    kw = case_kwargs(nx=48, ny=44, W=6, tau=0.6, sigma_max=0.05, sigma_power=3, bc="nrbc",
                     nrbc_edges=(0, 1, 0, 0), beta=0.3, mean=(1.0, 0.3, 0.0, 1.0),
                     pml_grad="link")
    fields = wl.isentropic_vortex(48, 44, 6, R=8.0, Mv=0.05, mean_u=(0.3, 0.0))
    check(kw, fields, 60, precision)


@pytest.mark.parametrize("precision", ["fp64", "fp32dev"])
@pytest.mark.parametrize("nx,ny,W", [(45, 37, 5), (33, 70, 2), (200, 9, 64)])
def test_link_ragged_pml_sizes(nx, ny, W, precision):
    kw = case_kwargs(nx=nx, ny=ny, W=W, tau=0.75, sigma_max=0.2, sigma_power=2, bc="zg",
                     pml_grad="link")
    fields = wl.random_smooth_state(nx, ny, W, seed=nx + ny, du=0.05)
    check(kw, fields, 30, precision)


@pytest.mark.parametrize("precision", ["fp64", "fp32dev"])
@pytest.mark.parametrize("widths,bc", [((2, 9, 0, 5), "zg"), ((0, 7, 4, 0), "nrbc"),
                                       ((6, 0, 0, 3), "zg")])
def test_link_per_edge_widths(widths, bc, precision):
    """Per-edge widths with edges without PML: P nodes next to such an edge reach boundary
    nodes outside F through the link difference."""
    nx, ny = 30, 26
    kw = case_kwargs(nx=nx, ny=ny, W=widths[0], widths=widths, tau=0.7, sigma_max=0.1,
                     sigma_power=2, bc=bc, mean=(1.0, 0.05, 0.0, 1.0), pml_grad="link")
    Ly, Lx = wl.f_shape(nx, ny, widths)
    rng_fields = wl.random_smooth_state(nx, ny, widths, seed=7, du=0.03, mean_u=(0.05, 0.0))
    assert rng_fields[0].shape == (Ly, Lx)
    check(kw, rng_fields, 40, precision)


@pytest.mark.parametrize("precision", ["fp64", "fp32dev"])
@pytest.mark.parametrize("src", [0, 7])
def test_link_density_step_periodic_y(src, precision):
    """Sec. 5.1 setting: periodic y, PML on the x edges, PNR-LODI, with and without the Appendix
    PML sources (term I is the link difference's moment in this mode)."""
    kw = case_kwargs(nx=60, ny=8, W=10, tau=0.8, sigma_max=0.1, sigma_power=2, bc="nrbc",
                     mean=(1.0, 0.05, 0.0, 1.0), periodic_y=True, pml_source=src,
                     pml_grad="link")
    fields = wl.density_step(60, 8, Ma=0.05, W=10, Wy=0)
    check(kw, fields, 60, precision)


@pytest.mark.parametrize("q", [17, 9])
@pytest.mark.parametrize("precision", ["fp64", "fp32dev"])
def test_link_other_stencils(q, precision):
    kw = case_kwargs(nx=36, ny=30, W=6, tau=0.7, sigma_max=0.1, sigma_power=2, bc="nrbc",
                     nrbc_edges=(0, 1, 0, 0), beta=0.1, mean=(1.0, 0.1, 0.0, 1.0), q=q,
                     pml_grad="link")
    fields = wl.pressure_pulse(36, 30, 6, amp=2e-3, halfwidth=3.0, u0=(0.1, 0.0))
    check(kw, fields, 50, precision)


@pytest.mark.parametrize("precision", ["fp64", "fp32dev"])
def test_link_checkpoint_restore_continues_bit_for_bit(precision):
    kw = case_kwargs(nx=40, ny=32, W=6, tau=0.7, sigma_max=0.1, sigma_power=3, bc="nrbc",
                     nrbc_edges=(0, 1, 0, 0), beta=0.2, mean=(1.0, 0.1, 0.0, 1.0),
                     pml_grad="link")
    fields = wl.pressure_pulse(40, 32, 6, amp=2e-3, halfwidth=3.0, u0=(0.1, 0.0))
    with make_solver(kw, precision) as a, make_solver(kw, precision) as b:
        a.init(*fields)
        a.step(17)
        ck = a.checkpoint()
        a.step(23)
        want = a.moments()
        b.init(*wl.uniform(40, 32, 6))
        b.restore(ck)
        b.step(23)
        got = b.moments()
        assert a.guards_intact() and b.guards_intact()
    for g, w in zip(got, want):
        assert np.array_equal(g, w)


@pytest.mark.parametrize("precision", ["fp64", "fp32dev"])
def test_d2q37_density_step_stays_finite_for_2000_steps_with_the_link_gradient(precision):
    """Table 1 D2Q37 ZG W 20 sigma_max 0.175, quadratic ramp, tau 0.8, 200 x 20 bulk, periodic
    y: the printed gradient is flagged unphysical within a few hundred steps, the link
    gradient runs 2000 steps with the bulk density within the initial step's range."""
    from paper_2504_20169_gb300 import LBMError
    fields = wl.density_step(200, 20, Ma=0.05, W=20, Wy=0)
    out = {}
    for mode in ("central", "link"):
        kw = case_kwargs(nx=200, ny=20, W=20, tau=0.8, sigma_max=0.175, sigma_power=2,
                         bc="zg", mean=(1.0, 0.05, 0.0, 1.0), periodic_y=True, pml_grad=mode)
        with make_solver(kw, precision) as s:
            s.init(*fields)
            try:
                s.step(2000)
                s.sync()
                rho = s.moments("bulk")[0]
                out[mode] = float(np.max(np.abs(rho - 1.0)))
            except LBMError:
                out[mode] = np.inf
    assert out["central"] == np.inf
    assert out["link"] < 0.05

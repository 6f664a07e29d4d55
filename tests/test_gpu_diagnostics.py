"""Bit-exact checks of the index maps the kernels use (pull sources of Eq. lbe, PML site
classification and absorption coefficients of Eqs. PML_ramp / pml-general) against the
oracle, and the measured FMA peaks used as the FP64 path's ALU roofline."""
import numpy as np
import pytest

import workloads as wl
from oracle import OracleLBM, pml
from parity_helpers import case_kwargs, make_solver

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("q", [37, 17, 9])
@pytest.mark.parametrize("nx,ny,W", [(20, 13, 0), (17, 30, 5), (9, 9, 2)])
def test_pull_index_matches_the_oracle_streaming(q, nx, ny, W):
    kw = case_kwargs(nx=nx, ny=ny, W=W, q=q, sigma_max=0.1 if W else 0.0)
    with make_solver(kw) as s:
        got = s.pull_index()
        M, Lx, Ly = s.M, s.Lx, s.Ly
    from paper_2504_20169_gb300 import lattice_info
    e_lib, _, _ = lattice_info(q)          # the library's direction order
    o = OracleLBM(nx, ny, W, 0.8, 0.1 if W else 0.0, 3, "zg", q=q)
    assert sorted(map(tuple, e_lib.tolist())) == sorted(map(tuple, o.lat.e.tolist()))
    Gx = Lx + 2 * M
    y, x = np.meshgrid(np.arange(Ly), np.arange(Lx), indexing="ij")
    for i, (ex, ey) in enumerate(e_lib.tolist()):
        # the oracle's streaming pulls velocity e from fstar[:, M - ey + y, M - ex + x]
        want = (M - ey + y) * Gx + (M - ex + x)
        assert np.array_equal(got[i], want), i


@pytest.mark.parametrize("widths,py,split,grad", [
    ((6, 6, 6, 6), False, False, "central"), ((2, 9, 0, 5), False, False, "central"),
    ((4, 7, 3, 6), False, True, "central"), ((8, 5, 0, 0), True, False, "central"),
    ((6, 6, 6, 6), False, False, "link"), ((0, 7, 4, 0), False, False, "link")])
def test_site_class_matches_the_oracle(widths, py, split, grad):
    nx, ny, smax, p = 21, 18, 0.3, 3
    kw = case_kwargs(nx=nx, ny=ny, W=widths[0], widths=widths, sigma_max=smax, sigma_power=p,
                     periodic_y=py, split=split, pml_grad=grad)
    with make_solver(kw) as s:
        layer, hq, sx, sy = s.site_class()
        M = s.M
    Lx, Ly = nx + widths[0] + widths[1], ny + widths[2] + widths[3]
    assert np.array_equal(layer, pml.layer_index(Lx, Ly, widths))
    want_sx, want_sy = pml.sigma_fields(Lx, Ly, widths, smax, p, split=split)
    assert np.allclose(sx, want_sx, rtol=1e-15, atol=0) and np.allclose(sy, want_sy, rtol=1e-15, atol=0)
    inP = pml.in_pml(Lx, Ly, widths)
    if grad == "central":
        assert np.array_equal(hq, pml.q_support(Lx, Ly, widths))
    else:
        # link mode: every node within M links (Chebyshev) of P carries Q
        near = np.zeros_like(inP)
        for dy in range(-M, M + 1):
            for dx in range(-M, M + 1):
                sh = np.zeros_like(inP)
                ys = slice(max(0, dy), Ly + min(0, dy)), slice(max(0, -dy), Ly + min(0, -dy))
                xs = slice(max(0, dx), Lx + min(0, dx)), slice(max(0, -dx), Lx + min(0, -dx))
                sh[ys[0], xs[0]] = inP[ys[1], xs[1]]
                near |= sh
        assert np.array_equal(hq, near)


def test_fma_peaks_are_measured():
    from paper_2504_20169_gb300 import peak_fma
    f64, ms64 = peak_fma("fp64")
    f32, ms32 = peak_fma("fp32dev")
    print(f"FMA peak: FP64 {f64:.3f} TFLOP/s ({ms64:.1f} ms), FP32 {f32:.2f} TFLOP/s ({ms32:.1f} ms)")
    assert 0.1 < f64 < 100.0 and 10.0 < f32 < 200.0
    assert f32 > 5 * f64

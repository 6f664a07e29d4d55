"""Host-only checks of liblbm: loading, exported symbols, the library's own quadrature, and
argument validation (none of these launches a kernel)."""
import ctypes as C
import os
import re
import subprocess

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "lbm.h")


@pytest.fixture(scope="module")
def L():
    from paper_2504_20169_gb300 import build
    build.build()
    from paper_2504_20169_gb300 import _lib
    return _lib


def declared_functions():
    text = open(HEADER).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(lbm_[a-z_0-9]+)\s*\(", text)))


def test_header_declares_the_core_calls():
    names = declared_functions()
    for core in ("lbm_create", "lbm_init", "lbm_step", "lbm_moments", "lbm_destroy"):
        assert core in names


def test_every_declared_symbol_is_exported(L):
    names = declared_functions()
    out = subprocess.run(["nm", "-D", "--defined-only", L.LIB_PATH], capture_output=True,
                         text=True, check=True).stdout
    exported = set(re.findall(r"\sT\s(lbm_[a-z_0-9]+)$", out, flags=re.M))
    missing = [n for n in names if n not in exported]
    assert not missing, missing
    # and the ctypes binding declares exactly the header's functions
    assert sorted(L.PROTOTYPES) == names
    lib = L.lib()
    for n in names:
        assert getattr(lib, n) is not None


def read_golden(q):
    path = os.path.join(ROOT, "tests", "golden", f"lattice_d2q{q}.txt")
    r, rows = None, []
    for line in open(path):
        if line.startswith("#"):
            continue
        parts = line.split()
        if parts[0] == "r":
            r = float(parts[1])
        else:
            rows.append((int(parts[0]), int(parts[1]), float(parts[2])))
    return r, rows


@pytest.mark.parametrize("q", [9, 17, 37])
def test_library_quadrature_matches_oracle(L, q):
    from paper_2504_20169_gb300 import lattice_info
    e, w, r = lattice_info(q)
    r_gold, rows = read_golden(q)
    assert r == pytest.approx(r_gold, abs=1e-14)
    gold = {(ex, ey): ww for ex, ey, ww in rows}
    assert len({tuple(v) for v in e.tolist()}) == q
    for (ex, ey), ww in zip(e.tolist(), w.tolist()):
        assert ww == pytest.approx(gold[(ex, ey)], rel=1e-13, abs=1e-16)


def _create(L, **kw):
    args = dict(nx=32, ny=32, q=37, tau=0.8, W=4, sigma=(0.1, 3), bc=L.LBM_BC_ZG,
                prec=L.LBM_FP64)
    args.update(kw)
    grid = L.lbm_grid(args["nx"], args["ny"])
    sig = L.lbm_sigma_profile(*args["sigma"])
    bp = L.lbm_bc_params()
    bp.rho0, bp.T0 = 1.0, 1.0
    for k, v in kw.get("edges", {}).items():
        bp.edge[k] = v
    out = C.c_void_p(123)
    st = L.lib().lbm_create(C.byref(grid), args["q"], args["tau"], args["W"], C.byref(sig),
                            args["bc"], C.byref(bp), args["prec"], None, C.byref(out))
    return st, out


@pytest.mark.parametrize("kw", [dict(nx=4), dict(tau=0.5), dict(tau=0.3), dict(W=1), dict(W=-2),
                                dict(q=19), dict(bc=7), dict(prec=5), dict(sigma=(-0.1, 2)),
                                dict(bc=0, W=4), dict(edges={1: 3})])
def test_invalid_arguments_are_rejected_before_any_allocation(L, kw):
    st, out = _create(L, **kw)
    assert st == L.LBM_EINVAL
    assert out.value is None
    assert L.lib().lbm_last_error(None)


def test_null_safety(L):
    lib = L.lib()
    assert lib.lbm_destroy(None) == L.LBM_OK
    assert lib.lbm_step(None, 1) == L.LBM_EINVAL
    assert lib.lbm_geometry(None, None) == L.LBM_EINVAL


def test_estimate_bytes_bc_follows_the_grid_shape(L):
    """lbm_estimate_bytes_bc (host only) budgets per-edge widths, the periodic y axis and the
    link gradient's wider accumulator; with equal widths it equals lbm_estimate_bytes."""
    from paper_2504_20169_gb300 import estimate_bytes
    grid = L.lbm_grid(256, 256)
    n = C.c_size_t()
    assert L.lib().lbm_estimate_bytes(C.byref(grid), 37, 32, L.LBM_BC_NRBC, L.LBM_FP32_DEV,
                                      C.byref(n)) == L.LBM_OK
    base = estimate_bytes(256, 256, 32, bc="nrbc")
    assert base == n.value
    thin = estimate_bytes(256, 256, 32, bc="nrbc", pml_widths=(8, 32, 8, 8))
    py = estimate_bytes(256, 256, 32, bc="nrbc", periodic_y=True)
    link = estimate_bytes(256, 256, 32, bc="nrbc", pml_grad="link")
    assert thin < base and py < base and link > base
    # FP64 holds twice the populations
    assert estimate_bytes(256, 256, 32, bc="nrbc", precision="fp64") > 1.9 * base


@pytest.mark.parametrize("kw", [dict(pml_grad="link", sigma_split=True),
                                dict(pml_widths=(1, 4, 4, 4)), dict(bc="periodic")])
def test_estimate_bytes_bc_rejects_what_create_rejects(L, kw):
    from paper_2504_20169_gb300 import LBMError, estimate_bytes
    with pytest.raises(LBMError):
        estimate_bytes(64, 64, 8, **kw)


def test_link_gradient_needs_equal_sigmas(L):
    grid = L.lbm_grid(32, 32)
    sig = L.lbm_sigma_profile(0.1, 3, 1)
    bp = L.lbm_bc_params()
    bp.rho0, bp.T0, bp.pml_grad = 1.0, 1.0, 1
    out = C.c_void_p(123)
    st = L.lib().lbm_create(C.byref(grid), 37, 0.8, 4, C.byref(sig), L.LBM_BC_ZG, C.byref(bp),
                            L.LBM_FP64, None, C.byref(out))
    assert st == L.LBM_EINVAL and out.value is None
    bp.pml_grad = 2
    sig.split = 0
    st = L.lib().lbm_create(C.byref(grid), 37, 0.8, 4, C.byref(sig), L.LBM_BC_ZG, C.byref(bp),
                            L.LBM_FP64, None, C.byref(out))
    assert st == L.LBM_EINVAL

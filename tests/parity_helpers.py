"""Shared helpers of the GPU parity tests: run the same seeded case through the oracle and
through liblbm, and compare fields."""
import numpy as np

from oracle import OracleLBM


def case_kwargs(**kw):
    base = dict(nx=32, ny=32, W=4, tau=0.8, sigma_max=0.1, sigma_power=3, bc="zg", q=37,
                nrbc_edges=(0, 0, 0, 0), beta=0.0, mean=(1.0, 0.0, 0.0, 1.0), relax_sign=-1.0,
                widths=None, periodic_y=False, split=False, pml_source=0, pml_grad="central")
    base.update(kw)
    return base


def run_oracle(kw, fields, steps):
    W = kw["W"] if kw["widths"] is None else tuple(kw["widths"])
    o = OracleLBM(kw["nx"], kw["ny"], W, kw["tau"], kw["sigma_max"], kw["sigma_power"],
                  kw["bc"], q=kw["q"], nrbc_edges=kw["nrbc_edges"], beta=kw["beta"],
                  mean=kw["mean"], relax_sign=kw["relax_sign"],
                  periodic_y=kw["periodic_y"], sigma_split=kw["split"],
                  pml_source=kw["pml_source"], pml_grad=kw["pml_grad"])
    o.init(*fields)
    o.step(steps)
    return o.fields(), o


def make_solver(kw, precision="fp64"):
    from paper_2504_20169_gb300 import Solver
    return Solver(kw["nx"], kw["ny"], kw["W"], kw["tau"], kw["sigma_max"], kw["sigma_power"],
                  kw["bc"], kw["q"], kw["nrbc_edges"], kw["beta"], kw["mean"],
                  kw["relax_sign"], precision, pml_widths=kw["widths"],
                  periodic_y=kw["periodic_y"], sigma_split=kw["split"],
                  pml_source=kw["pml_source"], pml_grad=kw["pml_grad"])


def run_gpu(kw, fields, steps, precision="fp64"):
    with make_solver(kw, precision) as s:
        s.init(*fields)
        s.step(steps)
        return s.moments()


def rel_l2(a, b):
    den = np.sqrt(np.sum(b * b))
    return float(np.sqrt(np.sum((a - b) ** 2)) / den)


def vel_l2(a, b):
    """L2 error of a velocity component: plain relative L2 when ||b|| >= c_s sqrt(N) / 10
    (an RMS velocity of at least a tenth of the sound speed, c_s = 1), else relative to that
    floor.

    A plain relative L2 is ill-conditioned when the velocity field is nearly zero: the FP64
    oracle rerun from inputs perturbed by one ulp differs from itself by 1e-9 .. 5e-8 in that
    measure after 200 steps of the 64^2 pulse case, while rho and T agree to 1e-15."""
    den = max(np.sqrt(np.sum(b * b)), 0.1 * np.sqrt(b.size))
    return float(np.sqrt(np.sum((a - b) ** 2)) / den)


# Relative L2 of the perturbations rho - 1 and T - 1. The perturbations of the test cases are
# 1e-3 .. 5e-2 of the fields, and they pass through zero where the waves have left, so these
# measures are 10^2 .. 10^5 times more sensitive than the relative L2 of the fields: the FP32
# deviation storage resolves g = f - w to about 1e-7 of w, i.e. 1e-4 of a 1e-3 perturbation per
# step, which over 200 steps gives up to ~1e-2.
PERT_TOL = {"fp64": 1e-8, "fp32dev": 5e-2}
TOL = {"fp64": 1e-12, "fp32dev": 1e-5}


def field_errors(gpu, ora):
    """Errors of (rho, u_x, u_y, T): relative L2 for rho and T, vel_l2 for the velocity; and
    the relative L2 of the perturbations rho - 1, T - 1."""
    full = [rel_l2(gpu[0], ora[0]), vel_l2(gpu[1], ora[1]), vel_l2(gpu[2], ora[2]),
            rel_l2(gpu[3], ora[3])]
    pert = [rel_l2(gpu[0] - 1, ora[0] - 1), rel_l2(gpu[3] - 1, ora[3] - 1)]
    return full, pert


def check(kw, fields, steps, precision="fp64", pert_tol=None, tag=""):
    """Run oracle and GPU on the same inputs; bound the field errors by TOL and the
    perturbation errors by PERT_TOL (or pert_tol)."""
    ora, _ = run_oracle(kw, fields, steps)
    gpu = run_gpu(kw, fields, steps, precision)
    full, pert = field_errors(gpu, ora)
    print(f"{tag}{precision} full={['%.2e' % e for e in full]} pert={['%.2e' % e for e in pert]}")
    assert max(full) < TOL[precision], full
    assert max(pert) < (PERT_TOL[precision] if pert_tol is None else pert_tol), pert
    return full, pert

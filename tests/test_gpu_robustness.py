"""Out-of-bounds writes and allocation failure, checked without a memory checker and without
faulting the GPU: every device buffer of a context carries guard bands that must survive every
operation on every geometry the library supports; an allocation budget set through the
environment makes lbm_create fail cleanly with LBM_ENOMEM and leave nothing allocated."""
import os

import numpy as np
import pytest

import workloads as wl
from parity_helpers import case_kwargs, make_solver

pytestmark = pytest.mark.gpu

GEOMETRIES = [
    (case_kwargs(nx=45, ny=37, W=5, tau=0.75, sigma_max=0.2, bc="zg"), None),
    (case_kwargs(nx=200, ny=9, W=64, tau=0.75, sigma_max=0.2, bc="zg"), None),
    (case_kwargs(nx=16, ny=12, W=2, tau=0.7, sigma_max=0.05, bc="nrbc", nrbc_edges=(1, 1, 1, 1),
                 beta=0.3, mean=(1.0, 0.1, 0.05, 1.0)), None),
    (case_kwargs(nx=8, ny=8, W=2, tau=0.8, sigma_max=0.05, bc="zg"), None),
    (case_kwargs(nx=8, ny=8, W=0, tau=0.8, sigma_max=0.0, bc="periodic"), None),
    (case_kwargs(nx=60, ny=12, W=8, tau=0.8, sigma_max=0.05, bc="nrbc", nrbc_edges=(1, 1, 0, 0),
                 beta=0.2, mean=(1.0, 0.05, 0.0, 1.0), periodic_y=True, pml_source=7), None),
    (case_kwargs(nx=33, ny=41, W=0, tau=0.75, sigma_max=0.15, bc="nrbc", widths=(35, 2, 0, 6),
                 split=True, pml_source=1), None),
    (case_kwargs(nx=36, ny=30, W=4, tau=0.7, sigma_max=0.1, bc="nrbc", q=17,
                 nrbc_edges=(0, 1, 0, 1), beta=0.2), None),
    (case_kwargs(nx=36, ny=30, W=4, tau=0.7, sigma_max=0.1, bc="nrbc", q=9,
                 nrbc_edges=(0, 1, 0, 1), beta=0.2), None),
]


def _fields(kw):
    W = kw["widths"] if kw["widths"] is not None else kw["W"]
    Wy = 0 if kw["periodic_y"] else None
    return wl.random_smooth_state(kw["nx"], kw["ny"], W, seed=1, du=0.02, Wy=Wy)


@pytest.mark.parametrize("precision", ["fp64", "fp32dev"])
@pytest.mark.parametrize("k", range(len(GEOMETRIES)))
def test_guard_bands_survive_every_operation(k, precision):
    import torch
    kw = GEOMETRIES[k][0]
    fields = _fields(kw)
    with make_solver(kw, precision) as s:
        assert s.guards_intact()
        s.init(*fields)
        s.step(7)
        s.moments()
        s.moments(region="bulk")
        s.reduce()
        ref = [torch.as_tensor(np.ascontiguousarray(a), device="cuda")
               for a in s.moments(region="bulk")]
        s.error_sums(ref)
        blob = s.checkpoint()
        s.step(3)
        s.restore(blob)
        s.import_populations(s.export_populations())
        s.step(2)
        s.profile_enable(2)
        s.step(2)
        s.profile_read()
        assert s.guards_intact()


def test_allocation_budget_fails_cleanly():
    import torch
    from paper_2504_20169_gb300._lib import LBMError, LBM_ENOMEM
    kw = case_kwargs(nx=256, ny=256, W=16, tau=0.8, sigma_max=0.1, bc="nrbc")
    torch.cuda.synchronize()
    free0 = torch.cuda.mem_get_info()[0]
    os.environ["LBM_DEBUG_ALLOC_BUDGET"] = str(4 << 20)     # far less than the populations
    try:
        for _ in range(3):
            with pytest.raises(LBMError) as ei:
                make_solver(kw, "fp64")
            assert ei.value.status == LBM_ENOMEM
            assert "allocation failed" in str(ei.value)
    finally:
        del os.environ["LBM_DEBUG_ALLOC_BUDGET"]
    torch.cuda.synchronize()
    assert abs(torch.cuda.mem_get_info()[0] - free0) < (8 << 20)
    with make_solver(kw, "fp64") as s:                         # without the budget: fine
        s.init(*wl.uniform(256, 256, 16))
        s.step(2)
        assert s.guards_intact()

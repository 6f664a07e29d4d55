"""lbm_totals_noalloc: the allocation-free totals reduction, for callers that cannot call
cudaMalloc (graph capture in progress, memory owned by a host application's pool, fixed
budgets). Its partial sums live in a fixed device array of the library instead of memory
allocated per call; this checks it against the context-based lbm_reduce, twice in a row."""
import ctypes as C

import numpy as np
import pytest

import workloads as wl
from parity_helpers import case_kwargs, make_solver

pytestmark = pytest.mark.gpu


def _call(L, fields, out, n=None):
    ptrs = [C.c_void_p(f.data_ptr()) for f in fields]
    n = fields[0].numel() if n is None else n
    return L.lib().lbm_totals_noalloc(*ptrs, C.c_int64(n), C.c_void_p(out.data_ptr()), None)


def test_noalloc_totals_match_lbm_reduce_on_two_calls():
    import torch
    from paper_2504_20169_gb300 import _lib as L
    kw = case_kwargs(nx=120, ny=90, W=8, tau=0.7, sigma_max=0.1, bc="nrbc",
                     nrbc_edges=(0, 1, 0, 0), beta=0.3, mean=(1.0, 0.2, 0.0, 1.0))
    fields = wl.isentropic_vortex(120, 90, 8, R=10.0, mean_u=(0.2, 0.0))
    with make_solver(kw) as s:
        s.init(*fields)
        for call in range(2):
            s.step(7)
            ref = s.reduce()                                   # existing entry point
            dev_fields = [t.reshape(-1) for t in s.moments(region="F", device=True)]
            out = torch.full((7,), float("nan"), dtype=torch.float64, device="cuda")
            free_before = torch.cuda.mem_get_info()[0]
            st = _call(L, dev_fields, out)
            torch.cuda.synchronize()
            assert st == L.LBM_OK, L.lib().lbm_last_error(None)
            if call == 1:
                # the first call on the device may load the module; later calls allocate nothing
                assert torch.cuda.mem_get_info()[0] == free_before
            got = out.cpu().numpy()
            assert np.allclose(got[:4], ref[:4], rtol=1e-13, atol=1e-12), (got, ref)
            assert got[4] == ref[4] and got[5] == ref[5] and got[6] == ref[6]


def test_noalloc_rejects_sizes_beyond_its_maximum():
    import torch
    from paper_2504_20169_gb300 import _lib as L
    x = torch.ones(16, dtype=torch.float64, device="cuda")
    out = torch.zeros(7, dtype=torch.float64, device="cuda")
    st = _call(L, [x, x, x, x], out, n=L.LBM_TOTALS_NOALLOC_MAX_N + 1)
    assert st == L.LBM_EINVAL
    assert b"LBM_TOTALS_NOALLOC_MAX_N" in L.lib().lbm_last_error(None)
    assert _call(L, [x, x, x, x], out, n=0) == L.LBM_EINVAL

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


def test_noalloc_large_field_with_bad_entries_matches_numpy():
    """n = 2^21 + 5 values (more than 1024 blocks x 256 threads, so the grid-stride loop goes
    round more than once and the second pass folds all 1024 partial rows), with non-positive
    and non-finite entries: sums against numpy in FP64 (rtol 1e-12; NaN where numpy gives NaN),
    minima (fmin ignores NaN, like numpy.nanmin) and the bad-entry count exactly; two calls."""
    import torch
    from paper_2504_20169_gb300 import _lib as L
    n = (1 << 21) + 5
    rng = np.random.default_rng(3)
    rho = rng.uniform(0.5, 1.5, n)
    ux = rng.uniform(-0.3, 0.3, n)
    uy = rng.uniform(-0.3, 0.3, n)
    T = rng.uniform(0.8, 1.2, n)
    bad = rng.choice(n, size=9, replace=False)
    rho[bad[:3]] = [-0.5, 0.0, -2.0]
    T[bad[3:6]] = [0.0, -1.0, 2e30]
    for field in (True, False):
        if field:
            T2 = T.copy()
            T2[bad[6]] = np.nan
        else:
            T2 = T
        want_sum = [rho.sum(), (rho * ux).sum(), (rho * uy).sum(),
                    (0.5 * rho * (ux * ux + uy * uy + 2.0 * T2)).sum()]
        want_min = [np.nanmin(rho), np.nanmin(T2)]
        ok = (rho > 0) & (T2 > 0) & (rho < 1e30) & (T2 < 1e30)
        want_bad = float(np.count_nonzero(~ok))
        dev = [torch.from_numpy(a).cuda() for a in (rho, ux, uy, T2)]
        for call in range(2):
            out = torch.full((7,), 123.0, dtype=torch.float64, device="cuda")
            assert _call(L, dev, out) == L.LBM_OK, L.lib().lbm_last_error(None)
            got = out.cpu().numpy()
            assert np.allclose(got[:4], want_sum, rtol=1e-12, atol=0, equal_nan=True), (got, want_sum)
            assert got[4] == want_min[0] and got[5] == want_min[1]
            assert got[6] == want_bad


def test_noalloc_rejects_sizes_beyond_its_maximum():
    import torch
    from paper_2504_20169_gb300 import _lib as L
    x = torch.ones(16, dtype=torch.float64, device="cuda")
    out = torch.zeros(7, dtype=torch.float64, device="cuda")
    st = _call(L, [x, x, x, x], out, n=L.LBM_TOTALS_NOALLOC_MAX_N + 1)
    assert st == L.LBM_EINVAL
    assert b"LBM_TOTALS_NOALLOC_MAX_N" in L.lib().lbm_last_error(None)
    assert _call(L, [x, x, x, x], out, n=0) == L.LBM_EINVAL

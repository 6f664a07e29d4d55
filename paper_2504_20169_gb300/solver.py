"""Python wrapper of one liblbm context (argument marshalling only).

Host arrays are numpy float64 (C-contiguous); device arrays are torch float64 CUDA tensors,
whose data pointers are passed straight to the library. The CUDA stream of a context is a
torch.cuda.Stream (default: torch's current stream at creation).
"""
from __future__ import annotations

import ctypes as C

import numpy as np

from . import _lib as L

_BC = {"periodic": L.LBM_BC_PERIODIC, "zg": L.LBM_BC_ZG, "nrbc": L.LBM_BC_NRBC}
_PREC = {"fp64": L.LBM_FP64, "fp32dev": L.LBM_FP32_DEV}


def _check(status, ctx=None):
    if status != L.LBM_OK:
        msg = L.lib().lbm_last_error(ctx)
        raise L.LBMError(status, msg.decode() if msg else "")


def lattice_info(q=37):
    """(e (q, 2) int array, w (q,), r) as derived by the library (host only, no GPU)."""
    qq = C.c_int()
    e = (C.c_int * (2 * q))()
    w = (C.c_double * q)()
    r = C.c_double()
    _check(L.lib().lbm_lattice_info(q, C.byref(qq), e, w, C.byref(r)))
    return np.array(e[:], dtype=np.int64).reshape(q, 2), np.array(w[:]), r.value


def _host(a):
    a = np.ascontiguousarray(a, dtype=np.float64)
    return a, a.ctypes.data_as(C.c_void_p)


class Solver:
    def __init__(self, nx, ny, W, tau, sigma_max=0.0, sigma_power=2, bc="zg", q=37,
                 nrbc_edges=(0, 0, 0, 0), beta=0.0, mean=(1.0, 0.0, 0.0, 1.0), relax_sign=-1.0,
                 precision="fp64", stream=None, pml_widths=None, periodic_y=False,
                 sigma_split=False, pml_source=0, pml_grad="central"):
        """W: PML layers on every edge, unless pml_widths = (W_w, W_e, W_s, W_n) is given;
        periodic_y: the y axis wraps (no S/N boundary, no PML there); sigma_split: the
        sigma_x != sigma_y form of Eq. (pml-general); pml_source: bitmask of the Appendix PML
        source terms I (1), II (2), III (4) added to the characteristic targets; pml_grad:
        "central" (the printed differences) or "link" (Q_i(x + e_i) - Q_i(x))."""
        import torch
        self.torch = torch
        self.stream = stream if stream is not None else torch.cuda.current_stream()
        self.nx, self.ny, self.W, self.q = nx, ny, W, q
        self.precision = precision
        grid = L.lbm_grid(nx, ny)
        sig = L.lbm_sigma_profile(sigma_max, sigma_power, 1 if sigma_split else 0)
        bp = L.lbm_bc_params()
        for k in range(4):
            bp.edge[k] = int(nrbc_edges[k])
        bp.beta = beta
        bp.relax_sign = relax_sign
        bp.rho0, bp.u0x, bp.u0y, bp.T0 = mean
        if pml_widths is not None:
            bp.use_pml_widths = 1
            for k in range(4):
                bp.pml_widths[k] = int(pml_widths[k])
        bp.periodic_y = 1 if periodic_y else 0
        bp.pml_source = int(pml_source)
        bp.pml_grad = {"central": 0, "link": 1}[pml_grad]
        out = C.c_void_p()
        with torch.cuda.device(self.stream.device):
            _check(L.lib().lbm_create(C.byref(grid), q, float(tau), W, C.byref(sig), _BC[bc],
                                      C.byref(bp), _PREC[precision],
                                      C.c_void_p(self.stream.cuda_stream), C.byref(out)))
        self.ctx = out
        g = (C.c_int64 * 12)()
        _check(L.lib().lbm_geometry(self.ctx, g), self.ctx)
        self.M = int(g[3])
        self.Lx, self.Ly = int(g[4]), int(g[5])
        self.widths = tuple(int(v) for v in g[8:12])

    # ---------------------------------------------------------------- lifecycle
    def close(self):
        if getattr(self, "ctx", None):
            L.lib().lbm_destroy(self.ctx)
            self.ctx = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()

    # ---------------------------------------------------------------- calls
    def init(self, rho, ux, uy, T):
        torch = self.torch
        if isinstance(rho, torch.Tensor):
            fl = [t.contiguous() for t in (rho, ux, uy, T)]
            for t in fl:
                assert t.is_cuda and t.dtype == torch.float64 and t.numel() == self.Lx * self.Ly
            ptrs = [C.c_void_p(t.data_ptr()) for t in fl]
            _check(L.lib().lbm_init(self.ctx, *ptrs, 1), self.ctx)
            self._keep = fl
        else:
            arrs = [_host(a) for a in (rho, ux, uy, T)]
            for a, _ in arrs:
                assert a.size == self.Lx * self.Ly
            _check(L.lib().lbm_init(self.ctx, *[p for _, p in arrs], 0), self.ctx)

    def step(self, n=1):
        _check(L.lib().lbm_step(self.ctx, int(n)), self.ctx)

    def sync(self):
        _check(L.lib().lbm_sync(self.ctx), self.ctx)

    def moments(self, region="F", device=False):
        reg = 1 if region == "F" else 0
        shape = (self.Ly, self.Lx) if reg else (self.ny, self.nx)
        if device:
            torch = self.torch
            outs = [torch.empty(shape, dtype=torch.float64, device=self.stream.device)
                    for _ in range(4)]
            _check(L.lib().lbm_moments(self.ctx, *[C.c_void_p(t.data_ptr()) for t in outs], reg,
                                       1), self.ctx)
            return tuple(outs)
        outs = [np.empty(shape) for _ in range(4)]
        _check(L.lib().lbm_moments(self.ctx, *[o.ctypes.data_as(C.c_void_p) for o in outs], reg,
                                   0), self.ctx)
        return tuple(outs)

    def reduce(self):
        out = (C.c_double * 7)()
        _check(L.lib().lbm_reduce(self.ctx, out), self.ctx)
        return np.array(out[:])

    def error_sums(self, ref):
        """ref: four torch float64 CUDA tensors over the bulk; returns 12 sums."""
        out = (C.c_double * 12)()
        refs = [r.contiguous() for r in ref]
        _check(L.lib().lbm_error_sums(self.ctx, *[C.c_void_p(r.data_ptr()) for r in refs], out),
               self.ctx)
        return np.array(out[:])

    def export_populations(self):
        Gx, Gy = self.Lx + 2 * self.M, self.Ly + 2 * self.M
        out = np.empty((self.q, Gy, Gx))
        _check(L.lib().lbm_export_populations(self.ctx, out.ctypes.data_as(L._dp)), self.ctx)
        return out

    def import_populations(self, arr):
        a = np.ascontiguousarray(arr, dtype=np.float64)
        Gx, Gy = self.Lx + 2 * self.M, self.Ly + 2 * self.M
        assert a.shape == (self.q, Gy, Gx)
        _check(L.lib().lbm_import_populations(self.ctx, a.ctypes.data_as(L._dp)), self.ctx)

    def checkpoint(self) -> bytes:
        n = C.c_size_t()
        _check(L.lib().lbm_checkpoint_size(self.ctx, C.byref(n)), self.ctx)
        buf = C.create_string_buffer(n.value)
        _check(L.lib().lbm_checkpoint(self.ctx, buf, n.value), self.ctx)
        return buf.raw

    def restore(self, data: bytes):
        buf = C.create_string_buffer(data, len(data))
        _check(L.lib().lbm_restore(self.ctx, buf, len(data)), self.ctx)

    def pull_index(self):
        """(q, Ly, Lx) int64: G index gy * (Lx + 2M) + gx of every pull source x - e_i."""
        out = np.empty((self.q, self.Ly, self.Lx), dtype=np.int64)
        _check(L.lib().lbm_export_pull_index(self.ctx, out.ctypes.data_as(C.c_void_p)), self.ctx)
        return out

    def site_class(self):
        """(layer index, has_q, sigma_x, sigma_y) per node of F, each (Ly, Lx)."""
        shp = (self.Ly, self.Lx)
        layer = np.empty(shp, dtype=np.int32)
        hq = np.empty(shp, dtype=np.uint8)
        sx, sy = np.empty(shp), np.empty(shp)
        _check(L.lib().lbm_export_site_class(self.ctx, *[a.ctypes.data_as(C.c_void_p)
                                                         for a in (layer, hq, sx, sy)]),
               self.ctx)
        return layer, hq.astype(bool), sx, sy

    KERNEL_CLASSES = ("targets", "interior", "frame1", "frame2", "band")

    def profile_enable(self, max_steps):
        _check(L.lib().lbm_profile_enable(self.ctx, int(max_steps)), self.ctx)

    def profile_read(self):
        """{kernel class: summed GPU ms}, recorded steps; restarts recording."""
        ms = (C.c_double * 5)()
        n = C.c_int()
        _check(L.lib().lbm_profile_read(self.ctx, ms, C.byref(n)), self.ctx)
        return dict(zip(self.KERNEL_CLASSES, ms[:])), n.value

    def guards_intact(self):
        """True if no kernel wrote outside the context's device buffers (guard bands)."""
        v = C.c_int()
        _check(L.lib().lbm_debug_check_guards(self.ctx, C.byref(v)), self.ctx)
        return bool(v.value)

    @property
    def steps(self):
        g = (C.c_int64 * 12)()
        _check(L.lib().lbm_geometry(self.ctx, g), self.ctx)
        return int(g[7])


def estimate_bytes(nx, ny, W, q=37, bc="zg", precision="fp32dev", pml_widths=None,
                   periodic_y=False, pml_grad="central", sigma_split=False):
    """Device bytes lbm_create would allocate (lbm_estimate_bytes_bc; host only)."""
    grid = L.lbm_grid(nx, ny)
    sig = L.lbm_sigma_profile(0.1, 2, 1 if sigma_split else 0)
    bp = L.lbm_bc_params()
    bp.rho0, bp.T0 = 1.0, 1.0
    if pml_widths is not None:
        bp.use_pml_widths = 1
        for k in range(4):
            bp.pml_widths[k] = int(pml_widths[k])
    bp.periodic_y = 1 if periodic_y else 0
    bp.pml_grad = {"central": 0, "link": 1}[pml_grad]
    n = C.c_size_t()
    _check(L.lib().lbm_estimate_bytes_bc(C.byref(grid), q, int(W), C.byref(sig), _BC[bc],
                                         C.byref(bp), _PREC[precision], C.byref(n)))
    return n.value


def peak_fma(precision="fp64", stream=None):
    """Measured FMA throughput of the current device in TFLOP/s (lbm_peak_fma)."""
    t, ms = C.c_double(), C.c_double()
    _check(L.lib().lbm_peak_fma(_PREC[precision], C.byref(t), C.byref(ms),
                                C.c_void_p(stream.cuda_stream if stream is not None else 0)))
    return t.value, ms.value

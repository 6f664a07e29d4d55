// Launchers of one (stencil, precision) combination. Instantiated once per combination in the
// ops_*.cu translation units so they compile in parallel.
#pragma once
#include <cfloat>
#include <cmath>

#include "lbm_device.cuh"
#include "lbm_internal.h"
#include "pml_fused.cuh"

namespace lbm {

// f^0 = f_eq(rho, u, T) on F (Sec. 2 initialization) and, on P and its ring, the accumulator
// S^(-1) = -f_hat^0 / 2 so that Q^0 = S^(-1) + f_hat^0 / 2 = 0.
template <class S, class Real, bool DEV>
__global__ void k_init_eq(Geom g, Consts<Real> c, const double* __restrict__ rho,
                          const double* __restrict__ ux, const double* __restrict__ uy,
                          const double* __restrict__ T, Real* __restrict__ A, Real* __restrict__ Sold) {
  const int x = blockIdx.x * blockDim.x + threadIdx.x;
  const int y = blockIdx.y;
  if (x >= g.Lx) return;
  const int k = y * g.Lx + x;
  const double r0 = rho[k], vx = ux[k], vy = uy[k], T0 = T[k];
  Macro<Real> m;
  m.rho = Real(r0);
  m.drho = Real(r0 - 1.0);
  m.inv_rho = Real(1.0 / r0);
  m.urx = c.r * Real(vx);
  m.ury = c.r * Real(vy);
  m.u2 = Real(vx * vx + vy * vy);
  m.theta = Real(T0 - 1.0);
  const EqCoef<Real> kc = eq_coef<S::ORDER, Real>(m);
  const long long idx = gindex(g, x, y);
  const bool has_q = pml_node<Real>(g, x, y).has_q;
  const int fi = has_q ? frame_index(g, x, y) : 0;
#pragma unroll
  for (int i = 0; i < S::Q; ++i) {
    const Real eq = eq_dir<S, Real, DEV>(i, m, kc, c);
    A[(long long)i * g.plane + idx] = eq;
    if (has_q) Sold[(long long)i * g.Sp + fi] = Real(-0.5) * (eq - c.eqbar[i]);
  }
}

// Link mode: the accumulator of the boundary nodes outside F, S^(-1) = -f_hat^0 / 2 with f_hat^0
// from the fields at the nearest fluid node (the state the boundary rule gives those nodes at
// initialization: zero-gradient copy, or characteristic targets equal to the fields there).
template <class S, class Real, bool DEV>
__global__ void k_init_gamma_s(Geom g, Consts<Real> c, const double* __restrict__ rho,
                               const double* __restrict__ ux, const double* __restrict__ uy,
                               const double* __restrict__ T, Real* __restrict__ Sold) {
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= g.ngamma) return;
  int x, y;
  gamma_xy(g, t, x, y);
  if (g.py && (y < 0 || y >= g.Ly)) return;   // images of rows inside F (wrapped lookups)
  const int k = min(max(y, 0), g.Ly - 1) * g.Lx + min(max(x, 0), g.Lx - 1);
  const double r0 = rho[k], vx = ux[k], vy = uy[k], T0 = T[k];
  Macro<Real> m;
  m.rho = Real(r0);
  m.drho = Real(r0 - 1.0);
  m.inv_rho = Real(1.0 / r0);
  m.urx = c.r * Real(vx);
  m.ury = c.r * Real(vy);
  m.u2 = Real(vx * vx + vy * vy);
  m.theta = Real(T0 - 1.0);
  const EqCoef<Real> kc = eq_coef<S::ORDER, Real>(m);
#pragma unroll
  for (int i = 0; i < S::Q; ++i)
    Sold[(long long)i * g.Sp + g.frame_n + t] =
        Real(-0.5) * (eq_dir<S, Real, DEV>(i, m, kc, c) - c.eqbar[i]);
}

// Block-wide reduction of NV doubles (sums, except slots flagged in min_mask which take the
// minimum); thread 0 writes the block's partials.
template <int NV>
__device__ inline void block_reduce_store(double (&v)[NV], unsigned min_mask, double* out) {
  __shared__ double sh[32][NV];
  const int lane = threadIdx.x & 31;
  const int tid = threadIdx.y * blockDim.x + threadIdx.x;
  const int warp = tid >> 5;
  const int nwarps = (blockDim.x * blockDim.y + 31) >> 5;
#pragma unroll
  for (int k = 0; k < NV; ++k) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      const double t = __shfl_down_sync(0xffffffffu, v[k], o);
      v[k] = ((min_mask >> k) & 1u) ? fmin(v[k], t) : v[k] + t;
    }
  }
  if (lane == 0) {
#pragma unroll
    for (int k = 0; k < NV; ++k) sh[warp][k] = v[k];
  }
  __syncthreads();
  if (warp == 0) {
#pragma unroll
    for (int k = 0; k < NV; ++k) {
      double a = lane < nwarps ? sh[lane][k] : (((min_mask >> k) & 1u) ? DBL_MAX : 0.0);
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) {
        const double t = __shfl_down_sync(0xffffffffu, a, o);
        a = ((min_mask >> k) & 1u) ? fmin(a, t) : a + t;
      }
      if (lane == 0) out[k] = a;
    }
  }
}

// Moments of the current time level over the bulk (region 0) or F (region 1): pulled from the
// previous post-collision buffer (STREAM) or read in place from the initial equilibrium.
// mode bit 1: write the fields; bit 2: conserved totals; bit 4: error sums vs reference fields.
template <class S, class Real, bool DEV, bool STREAM>
__global__ void __launch_bounds__(256) k_fields(Geom g, Consts<Real> c, const Real* __restrict__ A,
                                                int region, double* o0, double* o1, double* o2,
                                                double* o3, const double* r0, const double* r1,
                                                const double* r2, const double* r3,
                                                double* partials, int mode) {
  const int nxr = region ? g.Lx : g.nx, nyr = region ? g.Ly : g.ny;
  const int offx = region ? 0 : g.Ww, offy = region ? 0 : g.Ws;
  const int xr = blockIdx.x * blockDim.x + threadIdx.x;
  const int yr = blockIdx.y * blockDim.y + threadIdx.y;
  const bool live = xr < nxr && yr < nyr;
  double v[12];
#pragma unroll
  for (int k = 0; k < 12; ++k) v[k] = 0.0;
  unsigned min_mask = 0;
  if (mode & 2) {
    min_mask = (1u << 4) | (1u << 5);
    v[4] = DBL_MAX;
    v[5] = DBL_MAX;
  }
  if (live) {
    Real p[S::Q];
    load_pop<S, Real, STREAM>(p, A, g, gindex(g, xr + offx, yr + offy));
    const Macro<Real> m = moments<S, Real, DEV>(p, c);
    const double rho = double(m.rho), ux = double(m.urx / c.r), uy = double(m.ury / c.r);
    const double T = 1.0 + double(m.theta);
    const long long k = (long long)yr * nxr + xr;
    if (mode & 1) {
      if (o0) o0[k] = rho;
      if (o1) o1[k] = ux;
      if (o2) o2[k] = uy;
      if (o3) o3[k] = T;
    }
    if (mode & 2) {
      v[0] = rho;
      v[1] = rho * ux;
      v[2] = rho * uy;
      v[3] = 0.5 * rho * (ux * ux + uy * uy + 2.0 * T);
      v[4] = rho;
      v[5] = T;
      v[6] = (rho > 0.0 && T > 0.0 && rho < 1e30 && T < 1e30) ? 0.0 : 1.0;
    } else if (mode & 4) {
      const double z[4] = {rho, ux, uy, T};
      const double zr[4] = {r0[k], r1[k], r2[k], r3[k]};
#pragma unroll
      for (int q = 0; q < 4; ++q) {
        const double dz = z[q] - zr[q];
        v[3 * q] = dz * dz;
        v[3 * q + 1] = zr[q] * zr[q];
        const double rel = dz / zr[q];
        v[3 * q + 2] = rel * rel;
      }
    }
  }
  if (mode & 6) block_reduce_store<12>(v, min_mask, partials + 12ll * (blockIdx.y * gridDim.x + blockIdx.x));
}

// Stored populations <-> absolute FP64 populations on the whole grid G ([i][gy][gx]).
template <class S, class Real, bool DEV>
__global__ void k_export(Geom g, Consts<Real> c, const Real* __restrict__ A, double* __restrict__ out) {
  const int Gx = g.Lx + 2 * g.M, Gy = g.Ly + 2 * g.M;
  const long long n = (long long)S::Q * Gx * Gy;
  for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < n;
       t += (long long)gridDim.x * blockDim.x) {
    const int i = int(t / ((long long)Gx * Gy));
    const int rem = int(t - (long long)i * Gx * Gy);
    const int gy = rem / Gx, gx = rem - gy * Gx;
    const Real v = A[(long long)i * g.plane + gindex(g, gx - g.M, gy - g.M)];
    out[t] = DEV ? double(v) + double(c.w[i]) : double(v);
  }
}

template <class S, class Real, bool DEV>
__global__ void k_import(Geom g, Consts<Real> c, const double* __restrict__ in, Real* __restrict__ A) {
  const int Gx = g.Lx + 2 * g.M, Gy = g.Ly + 2 * g.M;
  const long long n = (long long)S::Q * Gx * Gy;
  for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < n;
       t += (long long)gridDim.x * blockDim.x) {
    const int i = int(t / ((long long)Gx * Gy));
    const int rem = int(t - (long long)i * Gx * Gy);
    const int gy = rem / Gx, gx = rem - gy * Gx;
    A[(long long)i * g.plane + gindex(g, gx - g.M, gy - g.M)] =
        DEV ? Real(in[t] - double(c.w[i])) : Real(in[t]);
  }
}

template <class S, class Real, bool DEV>
struct Ops {
  static const Consts<Real>& consts(const Dev& d) {
    if constexpr (sizeof(Real) == 8) return d.cd; else return d.cf;
  }

  template <bool STREAM>
  static cudaError_t step_impl(const Dev& d) {
    const Geom& g = d.g;
    const Consts<Real>& c = consts(d);
    const Real* A = static_cast<const Real*>(d.A);
    Real* B = static_cast<Real*>(d.B);
    // characteristic targets then boundary band on bs, PML frame on fs, interior on d.st; all
    // read A and write disjoint parts of B
    const bool link = g.link && has_pml(g);
    const cudaStream_t bs = d.aux ? d.aux : d.st;
    // link mode: the gradient pass reads the boundary nodes' new accumulator, so the frame
    // runs on the boundary stream in the order frame phase 1, band, frame phase 2
    const cudaStream_t fs = link ? bs : (d.aux2 ? d.aux2 : bs);
    auto mark = [&](int k, cudaStream_t s) {
      if (d.ev) cudaEventRecord(d.ev[k], s);
    };
    if (d.aux) {
      cudaEventRecord(d.fork, d.st);
      cudaStreamWaitEvent(d.aux, d.fork, 0);
      if (d.aux2) cudaStreamWaitEvent(d.aux2, d.fork, 0);
    }
    // Appendix PML source terms: only with a characteristic BC and a PML
    const int src_mask = (d.bc.bc == 2 && has_pml(g)) ? (d.bc.pml_source & 7) : 0;
    mark(0, bs);
    if (STREAM && d.bc.bc == 2) launch_nrbc_stages(d, sizeof(Real) == 4, bs);
    mark(1, bs);
    mark(4, fs);
    bool fused = false;
    if constexpr (DEV) {
      if (has_pml(g) && !link) {
        // FP32: single-pass frame (tile + halo in shared memory)
        const FrameTiles ft = make_frame_tiles(g, 256);
        const size_t smem = pml_fused_smem<S>(ft);
        k_pml_fused<S, STREAM><<<frame_tile_count(ft), 256, smem, fs>>>(
            g, c, ft, A, B, static_cast<const float*>(d.Sold), static_cast<float*>(d.Snew),
            d.Uedge_out, d.bc.bc == 2 ? 1 : 0, d.flag, d.Sedge_out, src_mask);
        fused = true;
      }
    }
    if (!fused)
      k_frame1<S, Real, DEV, STREAM><<<(g.frame_n + 127) / 128, 128, 0, fs>>>(
          g, c, A, B, static_cast<const Real*>(d.Sold), static_cast<Real*>(d.Snew), d.Uedge_out,
          d.bc.bc == 2 ? 1 : 0, d.flag, d.Sedge_out, src_mask);
    mark(5, fs);
    auto band = [&]() {
      mark(8, bs);
      k_gamma<S, Real, DEV, STREAM><<<(g.ngamma + 127) / 128, 128, 0, bs>>>(
          g, c, d.bc, A, B, d.Vtgt, link ? static_cast<const Real*>(d.Sold) : nullptr,
          link ? static_cast<Real*>(d.Snew) : nullptr);
      mark(9, bs);
    };
    if (link) band();
    mark(6, fs);
    if (has_pml(g) && !fused)
      k_frame2<S, Real><<<(g.frame_n + 127) / 128, 128, 0, fs>>>(
          g, c, B, static_cast<const Real*>(d.Sold), static_cast<const Real*>(d.Snew),
          d.Sedge_out, src_mask);
    mark(7, fs);
    if (!link) band();
    const int nbx = (g.Lx - g.Fe - (g.Fw / 32) * 32 + 31) / 32;
    const int ny_in = g.Ly - g.Fs - g.Fn;
    constexpr int BY = 4;
    mark(2, d.st);
    if (nbx > 0 && ny_in > 0) {
      dim3 grid(nbx, (ny_in + BY - 1) / BY);
      k_bulk<S, Real, DEV, STREAM><<<grid, dim3(32, BY), 0, d.st>>>(g, c, A, B, d.flag);
    }
    mark(3, d.st);
    if (d.aux) {
      cudaEventRecord(d.join, d.aux);
      cudaStreamWaitEvent(d.st, d.join, 0);
      if (d.aux2) {
        cudaEventRecord(d.join2, d.aux2);
        cudaStreamWaitEvent(d.st, d.join2, 0);
      }
    }
    if (g.py) {
      const long long n = (long long)(g.Lx + 2 * g.M) * g.M;
      k_wrap_y<Real><<<dim3(unsigned((n + 255) / 256), S::Q), 256, 0, d.st>>>(g, B);
    }
    return cudaGetLastError();
  }

  static cudaError_t step(const Dev& d, bool stream) {
    return stream ? step_impl<true>(d) : step_impl<false>(d);
  }

  static cudaError_t init_eq(const Dev& d, const double* rho, const double* ux, const double* uy,
                             const double* T) {
    const Geom& g = d.g;
    dim3 grid((g.Lx + 127) / 128, g.Ly);
    k_init_eq<S, Real, DEV><<<grid, 128, 0, d.st>>>(g, consts(d), rho, ux, uy, T,
                                                   static_cast<Real*>(const_cast<void*>(d.A)),
                                                   static_cast<Real*>(const_cast<void*>(d.Sold)));
    if (g.link && has_pml(g))
      k_init_gamma_s<S, Real, DEV><<<(g.ngamma + 127) / 128, 128, 0, d.st>>>(
          g, consts(d), rho, ux, uy, T, static_cast<Real*>(const_cast<void*>(d.Sold)));
    return cudaGetLastError();
  }

  static cudaError_t fields(const Dev& d, const void* src, bool stream, int region, double* const o[4],
                            const double* const r[4], int mode, double* partials, int* nblocks) {
    const Geom& g = d.g;
    const int nxr = region ? g.Lx : g.nx, nyr = region ? g.Ly : g.ny;
    dim3 blk(32, 8), grid((nxr + 31) / 32, (nyr + 7) / 8);
    *nblocks = grid.x * grid.y;
    if (stream)
      k_fields<S, Real, DEV, true><<<grid, blk, 0, d.st>>>(g, consts(d), static_cast<const Real*>(src),
                                                           region, o[0], o[1], o[2], o[3], r[0], r[1],
                                                           r[2], r[3], partials, mode);
    else
      k_fields<S, Real, DEV, false><<<grid, blk, 0, d.st>>>(g, consts(d), static_cast<const Real*>(src),
                                                            region, o[0], o[1], o[2], o[3], r[0], r[1],
                                                            r[2], r[3], partials, mode);
    return cudaGetLastError();
  }

  static cudaError_t export_pop(const Dev& d, const void* src, double* out) {
    k_export<S, Real, DEV><<<1024, 256, 0, d.st>>>(d.g, consts(d), static_cast<const Real*>(src), out);
    return cudaGetLastError();
  }
  static cudaError_t import_pop(const Dev& d, const double* in, void* dst) {
    k_import<S, Real, DEV><<<1024, 256, 0, d.st>>>(d.g, consts(d), in, static_cast<Real*>(dst));
    return cudaGetLastError();
  }

  // per-device kernel attributes, set once for every context on the context's device
  static cudaError_t prepare() {
    if constexpr (DEV) {
      cudaError_t e = cudaFuncSetAttribute(k_pml_fused<S, true>,
                                           cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024);
      if (e == cudaSuccess)
        e = cudaFuncSetAttribute(k_pml_fused<S, false>,
                                 cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024);
      return e;
    }
    return cudaSuccess;
  }

  static OpsTable table() {
    OpsTable t;
    t.prepare = &prepare;
    t.step = &step;
    t.init_eq = &init_eq;
    t.fields = &fields;
    t.export_pop = &export_pop;
    t.import_pop = &import_pop;
    t.elem_size = sizeof(Real);
    return t;
  }
};

}  // namespace lbm

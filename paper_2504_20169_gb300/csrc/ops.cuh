// Launchers of one (stencil, precision) combination. Instantiated once per combination in the
// ops_*.cu translation units so they compile in parallel.
#pragma once
#include <algorithm>
#include <cfloat>
#include <cmath>
#include <cstring>
#include <mutex>
#include <vector>

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

// ------------------------------------------------------------------------------------------
// Batched execution: one launch per kernel class over a table spanning every instance of the
// batch. Each block reads its (member, tile) entry and runs the same per-node / per-tile body
// as the single-instance kernels, so every member computes bit for bit what it computes alone.
// ------------------------------------------------------------------------------------------
template <class Real>
struct MemberDev {
  Geom g;
  Consts<Real> c;
  BcParams bc;
  FrameTiles ft;
  const Real* A;
  Real* B;
  Real* Sold;
  Real* Snew;
  double* Vtgt;
  double* Uedge_out;
  double* Sedge_out;
  int* flag;
  int src_mask;
};

template <class S, class Real, bool DEV>
__global__ void __launch_bounds__(256) kb_bulk(const MemberDev<Real>* __restrict__ mem,
                                               const int* __restrict__ tab) {
  const int* e = tab + 3 * blockIdx.x;
  const MemberDev<Real>& md = mem[e[0]];
  const Geom g = md.g;
  const int x0 = (g.Fw / 32) * 32;
  bulk_node<S, Real, DEV, true>(g, md.c, md.A, md.B, md.flag,
                                x0 + e[1] * blockDim.x + threadIdx.x,
                                g.Fs + e[2] * blockDim.y + threadIdx.y);
}

template <class S>
__global__ void __launch_bounds__(256) kb_pml_fused(const MemberDev<float>* __restrict__ mem,
                                                    const int* __restrict__ tab) {
  extern __shared__ float smem[];
  const int* e = tab + 2 * blockIdx.x;
  const MemberDev<float>& md = mem[e[0]];
  pml_fused_tile<S, true>(md.g, md.c, md.ft, md.A, md.B, md.Sold, md.Snew, md.Uedge_out,
                          md.bc.bc == 2 ? 1 : 0, md.flag, md.Sedge_out, md.src_mask, e[1], smem);
}

template <class S, class Real, bool DEV>
__global__ void __launch_bounds__(128) kb_frame1(const MemberDev<Real>* __restrict__ mem,
                                                 const int* __restrict__ tab) {
  const int* e = tab + 2 * blockIdx.x;
  const MemberDev<Real>& md = mem[e[0]];
  const Geom g = md.g;
  if constexpr (sizeof(Real) == 4) {
    // FP32: the node's accumulator is staged in shared memory by cp.async during the pull
    __shared__ float stage[128 * S::Q];
    frame1_node<S, Real, DEV, true, true>(g, md.c, md.A, md.B, md.Sold, md.Snew, md.Uedge_out,
                                          md.bc.bc == 2 ? 1 : 0, md.flag, md.Sedge_out,
                                          md.src_mask, e[1] * blockDim.x + threadIdx.x,
                                          reinterpret_cast<Real*>(stage) + threadIdx.x * S::Q);
  } else {
    frame1_node<S, Real, DEV, true>(g, md.c, md.A, md.B, md.Sold, md.Snew, md.Uedge_out,
                                    md.bc.bc == 2 ? 1 : 0, md.flag, md.Sedge_out, md.src_mask,
                                    e[1] * blockDim.x + threadIdx.x);
  }
}

template <class S, class Real>
__global__ void __launch_bounds__(128) kb_frame2(const MemberDev<Real>* __restrict__ mem,
                                                 const int* __restrict__ tab) {
  const int* e = tab + 2 * blockIdx.x;
  const MemberDev<Real>& md = mem[e[0]];
  const Geom g = md.g;
  if constexpr (sizeof(Real) == 4) {
    // FP32: the gathers and the loads of B are staged in shared memory by cp.async
    __shared__ float stq[128 * S::Q], stb[128 * S::Q];
    frame2_node<S, Real, true>(g, md.c, md.B, md.Sold, md.Snew, md.Sedge_out, md.src_mask,
                               e[1] * blockDim.x + threadIdx.x,
                               reinterpret_cast<Real*>(stq) + threadIdx.x * S::Q,
                               reinterpret_cast<Real*>(stb) + threadIdx.x * S::Q);
  } else {
    frame2_node<S, Real>(g, md.c, md.B, md.Sold, md.Snew, md.Sedge_out, md.src_mask,
                         e[1] * blockDim.x + threadIdx.x);
  }
}

template <class S, class Real, bool DEV>
__global__ void __launch_bounds__(128) kb_gamma(const MemberDev<Real>* __restrict__ mem,
                                                const int* __restrict__ tab) {
  const int* e = tab + 2 * blockIdx.x;
  const MemberDev<Real>& md = mem[e[0]];
  const Geom g = md.g;
  const bool link = g.link && has_pml(g);
  gamma_node<S, Real, DEV, true>(g, md.c, md.bc, md.A, md.B, md.Vtgt,
                                 link ? md.Sold : nullptr, link ? md.Snew : nullptr,
                                 e[1] * blockDim.x + threadIdx.x);
}

template <class Real>
__global__ void __launch_bounds__(256) kb_wrap_y(const MemberDev<Real>* __restrict__ mem,
                                                 const int* __restrict__ tab) {
  const int* e = tab + 2 * blockIdx.x;
  const MemberDev<Real>& md = mem[e[0]];
  const Geom g = md.g;
  wrap_y_elem<Real>(g, md.B, (long long)e[1] * blockDim.x + threadIdx.x, blockIdx.y);
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
    // Streaming steps of a context run the boundary-side classes through the table-driven
    // kernels of its one-member plan (the kernels a batch runs), so that a context computes
    // bit for bit the same alone and in any batch; the interior kernel is the same either way.
    const BatchPlan* pl = STREAM ? d.plan : nullptr;
    const MemberDev<Real>* pm = pl ? static_cast<const MemberDev<Real>*>(pl->desc[d.which]) : nullptr;
    if (pl) {
      launch_nrbc_batch(pl->tgt[d.which], pl->tgt_tab, pl->n_tgt, sizeof(Real) == 4,
                        pl->tgt_threads, pl->tgt_smem, bs);
    } else if (STREAM && d.bc.bc == 2) {
      launch_nrbc_stages(d, sizeof(Real) == 4, bs);
    }
    mark(1, bs);
    mark(4, fs);
    if (pl) {
      if constexpr (DEV) {
        if (pl->n_frame)
          kb_pml_fused<S><<<pl->n_frame, 256, pl->frame_smem, fs>>>(
              reinterpret_cast<const MemberDev<float>*>(pm), pl->frame_tab);
      }
      if (pl->n_f1) kb_frame1<S, Real, DEV><<<pl->n_f1, 128, 0, fs>>>(pm, pl->f1_tab);
      mark(5, fs);
      auto band_b = [&]() {
        mark(8, bs);
        if (pl->n_band) kb_gamma<S, Real, DEV><<<pl->n_band, 128, 0, bs>>>(pm, pl->band_tab);
        mark(9, bs);
      };
      if (link) band_b();
      mark(6, fs);
      if (pl->n_f2) kb_frame2<S, Real><<<pl->n_f2, 128, 0, fs>>>(pm, pl->f2_tab);
      mark(7, fs);
      if (!link) band_b();
    }
    bool fused = false;
    if constexpr (DEV) {
      if (!pl && has_pml(g) && !link) {
        // FP32: single-pass frame (tile + halo in shared memory)
        const FrameTiles ft = make_frame_tiles(g, 256);
        const size_t smem = pml_fused_smem<S>(ft);
        k_pml_fused<S, STREAM><<<frame_tile_count(ft), 256, smem, fs>>>(
            g, c, ft, A, B, static_cast<const float*>(d.Sold), static_cast<float*>(d.Snew),
            d.Uedge_out, d.bc.bc == 2 ? 1 : 0, d.flag, d.Sedge_out, src_mask);
        fused = true;
      }
    }
    if (!fused && !pl)
      k_frame1<S, Real, DEV, STREAM><<<(g.frame_n + 127) / 128, 128, 0, fs>>>(
          g, c, A, B, static_cast<Real*>(d.Sold), static_cast<Real*>(d.Snew), d.Uedge_out,
          d.bc.bc == 2 ? 1 : 0, d.flag, d.Sedge_out, src_mask);
    if (!pl) mark(5, fs);
    auto band = [&]() {
      mark(8, bs);
      k_gamma<S, Real, DEV, STREAM><<<(g.ngamma + 127) / 128, 128, 0, bs>>>(
          g, c, d.bc, A, B, d.Vtgt, link ? static_cast<Real*>(d.Sold) : nullptr,
          link ? static_cast<Real*>(d.Snew) : nullptr);
      mark(9, bs);
    };
    if (!pl) {
      if (link) band();
      mark(6, fs);
      if (has_pml(g) && !fused)
        k_frame2<S, Real><<<(g.frame_n + 127) / 128, 128, 0, fs>>>(
            g, c, B, static_cast<const Real*>(d.Sold), static_cast<const Real*>(d.Snew),
            d.Sedge_out, src_mask);
      mark(7, fs);
      if (!link) band();
    }
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
    if (pl) {
      if (pl->n_wrap) kb_wrap_y<Real><<<dim3(pl->n_wrap, S::Q), 256, 0, d.st>>>(pm, pl->wrap_tab);
    } else if (g.py) {
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
                                                   static_cast<Real*>(d.Sold));
    if (g.link && has_pml(g))
      k_init_gamma_s<S, Real, DEV><<<(g.ngamma + 127) / 128, 128, 0, d.st>>>(
          g, consts(d), rho, ux, uy, T, static_cast<Real*>(d.Sold));
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
  static cudaError_t prepare(const double* w) {
    // weights in constant memory, once per device (the values never change)
    {
      static std::mutex mu;
      static bool done[64] = {};
      int dev = 0;
      cudaError_t e = cudaGetDevice(&dev);
      if (e != cudaSuccess) return e;
      std::lock_guard<std::mutex> lock(mu);
      if (dev < 0 || dev >= 64 || !done[dev]) {
        Real wr[S::Q];
        for (int i = 0; i < S::Q; ++i) wr[i] = Real(w[i]);
        const void* sym;
        if constexpr (sizeof(Real) == 8)
          sym = S::Q == 37 ? (const void*)&kw37d : S::Q == 17 ? (const void*)&kw17d : (const void*)&kw9d;
        else
          sym = S::Q == 37 ? (const void*)&kw37f : S::Q == 17 ? (const void*)&kw17f : (const void*)&kw9f;
        e = cudaMemcpyToSymbol(sym, wr, sizeof(wr));
        if (e != cudaSuccess) return e;
        if (dev >= 0 && dev < 64) done[dev] = true;
      }
    }
    if constexpr (DEV) {
      cudaError_t e = cudaFuncSetAttribute(k_pml_fused<S, true>,
                                           cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024);
      if (e == cudaSuccess)
        e = cudaFuncSetAttribute(k_pml_fused<S, false>,
                                 cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024);
      if (e == cudaSuccess)
        e = cudaFuncSetAttribute(kb_pml_fused<S>,
                                 cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024);
      return e;
    }
    return cudaSuccess;
  }

  // ---------------------------------------------------------------- batched execution
  static MemberDev<Real> member_of(const Dev& d) {
    MemberDev<Real> m;
    std::memset(&m, 0, sizeof m);
    m.g = d.g;
    m.c = consts(d);
    m.bc = d.bc;
    m.ft = make_frame_tiles(d.g, 256);
    m.A = static_cast<const Real*>(d.A);
    m.B = static_cast<Real*>(d.B);
    m.Sold = static_cast<Real*>(d.Sold);
    m.Snew = static_cast<Real*>(d.Snew);
    m.Vtgt = d.Vtgt;
    m.Uedge_out = d.Uedge_out;
    m.Sedge_out = d.Sedge_out;
    m.flag = d.flag;
    m.src_mask = (d.bc.bc == 2 && has_pml(d.g)) ? (d.bc.pml_source & 7) : 0;
    return m;
  }

  static bool fused_of(const Geom& g) { return DEV && has_pml(g) && !g.link; }

  static cudaError_t batch_plan(const Dev* const* dev0, const Dev* const* dev1, int n, int tx,
                                int by, BatchPlan* plan) {
    BatchPlan p;
    p.n = n;
    p.tx = tx;
    p.by = by;
    p.q = S::Q;
    p.link = n > 0 && dev0[0]->g.link;
    std::vector<int> bulk, frame, f1, f2, band, tgt, wrap;
    for (int m = 0; m < n; ++m) {
      const Geom& g = dev0[m]->g;
      const int x0 = (g.Fw / 32) * 32;
      const int nbx = (g.Lx - g.Fe - x0 + tx - 1) / tx, nby = (g.Ly - g.Fs - g.Fn + by - 1) / by;
      if (g.Lx - g.Fe - x0 > 0 && g.Ly - g.Fs - g.Fn > 0)
        for (int j = 0; j < nby; ++j)
          for (int i = 0; i < nbx; ++i) bulk.insert(bulk.end(), {m, i, j});
      if (fused_of(g)) {
        const FrameTiles ft = make_frame_tiles(g, 256);
        const int nt = frame_tile_count(ft);
        for (int k = 0; k < nt; ++k) frame.insert(frame.end(), {m, k});
        p.frame_smem = std::max(p.frame_smem, pml_fused_smem<S>(ft));
      } else {
        for (int b = 0; b < (g.frame_n + 127) / 128; ++b) f1.insert(f1.end(), {m, b});
        if (has_pml(g))
          for (int b = 0; b < (g.frame_n + 127) / 128; ++b) f2.insert(f2.end(), {m, b});
      }
      for (int b = 0; b < (g.ngamma + 127) / 128; ++b) band.insert(band.end(), {m, b});
      if (dev0[m]->bc.bc == 2) {
        int chunks, threads;
        size_t smem;
        nrbc_shape(g, &chunks, &threads, &smem);
        for (int k = 0; k < chunks; ++k) tgt.insert(tgt.end(), {m, k});
        p.tgt_threads = std::max(p.tgt_threads, threads);
        p.tgt_smem = std::max(p.tgt_smem, smem);
      }
      if (g.py) {
        const long long nw = (long long)(g.Lx + 2 * g.M) * g.M;
        for (int b = 0; b < (int)((nw + 255) / 256); ++b) wrap.insert(wrap.end(), {m, b});
      }
    }
    p.n_bulk = (int)bulk.size() / 3;
    p.n_frame = (int)frame.size() / 2;
    p.n_f1 = (int)f1.size() / 2;
    p.n_f2 = (int)f2.size() / 2;
    p.n_band = (int)band.size() / 2;
    p.n_tgt = (int)tgt.size() / 2;
    p.n_wrap = (int)wrap.size() / 2;
    // one device allocation: descriptors (2 parity states), target descriptors, tables
    std::vector<MemberDev<Real>> d0(n), d1(n);
    std::vector<TgtDesc> t0(n), t1(n);
    for (int m = 0; m < n; ++m) {
      d0[m] = member_of(*dev0[m]);
      d1[m] = member_of(*dev1[m]);
      t0[m] = TgtDesc{dev0[m]->g, dev0[m]->bc, dev0[m]->Uedge_in, dev0[m]->Sedge_in, dev0[m]->Vtgt};
      t1[m] = TgtDesc{dev1[m]->g, dev1[m]->bc, dev1[m]->Uedge_in, dev1[m]->Sedge_in, dev1[m]->Vtgt};
    }
    auto al = [](size_t b) { return (b + 255) / 256 * 256; };
    const size_t bd = al(sizeof(MemberDev<Real>) * n), bt = al(sizeof(TgtDesc) * n);
    const std::vector<int>* tabs[7] = {&bulk, &frame, &f1, &f2, &band, &tgt, &wrap};
    size_t total = 2 * bd + 2 * bt;
    for (auto* t : tabs) total += al(sizeof(int) * t->size() + 4);
    char* mem = nullptr;
    cudaError_t e = cudaMalloc(&mem, total);
    if (e != cudaSuccess) return e;
    p.mem = mem;
    size_t off = 0;
    auto put = [&](const void* src, size_t bytes, size_t slot) {
      void* dst = mem + off;
      if (bytes && e == cudaSuccess) e = cudaMemcpy(dst, src, bytes, cudaMemcpyHostToDevice);
      off += slot;
      return dst;
    };
    p.desc[0] = put(d0.data(), sizeof(MemberDev<Real>) * n, bd);
    p.desc[1] = put(d1.data(), sizeof(MemberDev<Real>) * n, bd);
    p.tgt[0] = static_cast<TgtDesc*>(put(t0.data(), sizeof(TgtDesc) * n, bt));
    p.tgt[1] = static_cast<TgtDesc*>(put(t1.data(), sizeof(TgtDesc) * n, bt));
    int** dst[7] = {&p.bulk_tab, &p.frame_tab, &p.f1_tab, &p.f2_tab, &p.band_tab, &p.tgt_tab,
                    &p.wrap_tab};
    for (int k = 0; k < 7; ++k)
      *dst[k] = static_cast<int*>(put(tabs[k]->data(), sizeof(int) * tabs[k]->size(),
                                      al(sizeof(int) * tabs[k]->size() + 4)));
    if (e != cudaSuccess) {
      cudaFree(mem);
      return e;
    }
    *plan = p;
    return cudaSuccess;
  }

  static cudaError_t batch_step(const BatchPlan& p, int which, cudaStream_t st, cudaStream_t aux,
                                cudaStream_t aux2, cudaEvent_t fork, cudaEvent_t join,
                                cudaEvent_t join2) {
    const MemberDev<Real>* mem = static_cast<const MemberDev<Real>*>(p.desc[which]);
    const cudaStream_t bs = aux ? aux : st;
    const cudaStream_t fs = p.link ? bs : (aux2 ? aux2 : bs);
    if (aux) {
      cudaEventRecord(fork, st);
      cudaStreamWaitEvent(aux, fork, 0);
      if (aux2) cudaStreamWaitEvent(aux2, fork, 0);
    }
    // characteristic targets, then (printed gradient) the boundary band, on bs
    cudaError_t e = launch_nrbc_batch(p.tgt[which], p.tgt_tab, p.n_tgt, sizeof(Real) == 4,
                                      p.tgt_threads, p.tgt_smem, bs);
    if (e != cudaSuccess) return e;
    auto band = [&]() {
      if (p.n_band) kb_gamma<S, Real, DEV><<<p.n_band, 128, 0, bs>>>(mem, p.band_tab);
    };
    if (!p.link) band();
    // the frame on fs
    if constexpr (DEV) {
      if (p.n_frame)
        kb_pml_fused<S><<<p.n_frame, 256, p.frame_smem, fs>>>(mem, p.frame_tab);
    }
    if (p.n_f1) kb_frame1<S, Real, DEV><<<p.n_f1, 128, 0, fs>>>(mem, p.f1_tab);
    if (p.link) band();
    if (p.n_f2) kb_frame2<S, Real><<<p.n_f2, 128, 0, fs>>>(mem, p.f2_tab);
    // the interiors of every member on st
    if (p.n_bulk)
      kb_bulk<S, Real, DEV><<<p.n_bulk, dim3(p.tx, p.by), 0, st>>>(mem, p.bulk_tab);
    if (aux) {
      cudaEventRecord(join, aux);
      cudaStreamWaitEvent(st, join, 0);
      if (aux2) {
        cudaEventRecord(join2, aux2);
        cudaStreamWaitEvent(st, join2, 0);
      }
    }
    if (p.n_wrap) kb_wrap_y<Real><<<dim3(p.n_wrap, S::Q), 256, 0, st>>>(mem, p.wrap_tab);
    return cudaGetLastError();
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
    t.batch_plan = &batch_plan;
    t.batch_step = &batch_step;
    return t;
  }
};

}  // namespace lbm

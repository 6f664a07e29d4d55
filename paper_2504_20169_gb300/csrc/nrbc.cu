// Characteristic boundary targets (Sec. 4) and the final pass of the FP64 reductions.
#include <cfloat>

#include "lbm_internal.h"

namespace lbm {

// Rate dU/dt of one edge-band node (Sec. 4). U0: the node; U1, U2: the states one and two nodes
// inward along the normal (band layers or fluid moments); Va, Vb, Vc: three consecutive nodes of
// the same layer around it along the tangent with weights (ca, cb, cc) of the tangential
// derivative. PNR-LODI: Eq. (PNR) with Eq. (thermal_LODI_macro_evo); CBC relax: Eq. (CBC-Relax)
// with Eq. (thermal_CBC_macro_evo); viscous part zero. Differences in FP64, algebra in R.
template <class R>
__device__ inline void char_rate(const BcParams& bc, int variant, double out, const Prim& U0d,
                                 const Prim& U1, const Prim& U2, const Prim& Va, const Prim& Vb,
                                 const Prim& Vc, double ca, double cb, double cc, bool xaxis,
                                 double kk[4]) {
  const double hs = 0.5 * out;
  PrimT<R> dn;
  dn.rho = R(hs * (3.0 * U0d.rho - 4.0 * U1.rho + U2.rho));
  dn.un = R(hs * (3.0 * U0d.un - 4.0 * U1.un + U2.un));
  dn.ut = R(hs * (3.0 * U0d.ut - 4.0 * U1.ut + U2.ut));
  dn.T = R(hs * (3.0 * U0d.T - 4.0 * U1.T + U2.T));
  const PrimT<R> U0 = to<R>(U0d);
  const R inv_r = R(bc.inv_r);
  const R c = sqrt(R(2) * U0.T);  // gamma T with gamma = (D + 2) / D = 2
  const R lam[4] = {U0.un - c, U0.un, U0.un, U0.un + c};
  R wn[4];
  char_forward(U0, c, dn, wn);
  const R sgn = R(out);
  R tot[4];
  if (variant == 0) {
    for (int k = 0; k < 4; ++k) tot[k] = (lam[k] * sgn < R(0)) ? R(0) : lam[k] * wn[k] * inv_r;
  } else {
    PrimT<R> dt;
    dt.rho = R(ca * Va.rho + cb * Vb.rho + cc * Vc.rho);
    dt.un = R(ca * Va.un + cb * Vb.un + cc * Vc.un);
    dt.ut = R(ca * Va.ut + cb * Vb.ut + cc * Vc.ut);
    dt.T = R(ca * Va.T + cb * Vb.T + cc * Vc.T);
    // B dU along the tangential axis (u_t advects; P_t = T rho_t + rho T_t; (2/D) T = T)
    PrimT<R> bd;
    bd.rho = U0.ut * dt.rho + U0.rho * dt.ut;
    bd.un = U0.ut * dt.un;
    bd.ut = (U0.T / U0.rho) * dt.rho + U0.ut * dt.ut + dt.T;
    bd.T = U0.T * dt.ut + U0.ut * dt.T;
    R Tc[4];
    char_forward(U0, c, bd, Tc);
    const R relax = R(bc.relax_sign * (1.0 - bc.beta));
    for (int k = 0; k < 4; ++k) {
      const R Lbar = (lam[k] * sgn < R(0)) ? relax * Tc[k] : lam[k] * wn[k];
      tot[k] = (Lbar + Tc[k]) * inv_r;
    }
  }
  const PrimT<R> r = char_inverse(U0, c, tot);
  kk[0] = -double(r.rho);
  kk[1] = xaxis ? -double(r.un) : -double(r.ut);
  kk[2] = xaxis ? -double(r.ut) : -double(r.un);
  kk[3] = -double(r.T);
}

// All four stages of classical RK4 for the targets of one chunk of one edge band, in shared
// memory (fluid moments Ue frozen at time n). Block = one edge, tangential chunk [t0, t0 + T)
// plus a 4-node halo on each side where the chunk does not end the band; thread = (layer,
// position). Each stage shrinks the valid range by one node at a chunk cut, so the chunk's own
// nodes see exactly the values a full-band evaluation would. On a periodic y axis the W and E
// bands wrap around (central tangential differences everywhere, halo taken modulo Ly).
constexpr int kChunk = 32, kHalo = 4, kText = kChunk + 2 * kHalo;

// (nrbc_chunk is the per-block work, shared with the batched launch over many instances;
// chunk = index over the four bands' chunks, sm = 16 M kText doubles of shared memory.)
template <class R>
__device__ __forceinline__ void nrbc_chunk(const Geom& g, const BcParams& bc,
                                           const double* __restrict__ Ue,
                                           const double* __restrict__ Se,
                                           double* __restrict__ Vg, int chunk, double* sm) {
  const int M = g.M, Lx = g.Lx, Ly = g.Ly;
  const int cw = (Ly + kChunk - 1) / kChunk, cs = (Lx + kChunk - 1) / kChunk;
  int e, k = chunk;
  if (k < cw) e = 0;
  else if (k < 2 * cw) { e = 1; k -= cw; }
  else if (k < 2 * cw + cs) { e = 2; k -= 2 * cw; }
  else { e = 3; k -= 2 * cw + cs; }
  if (g.py && e >= 2) return;   // no S / N boundary on a periodic y axis
  const int len = e < 2 ? Ly : Lx;
  const int off = e == 0 ? 0 : e == 1 ? M * Ly : e == 2 ? 2 * M * Ly : 2 * M * Ly + M * Lx;
  const int ueoff = e == 0 ? 0 : e == 1 ? 2 * Ly : e == 2 ? 4 * Ly : 4 * Ly + 2 * Lx;
  const bool xaxis = e < 2;
  const double out = (e == 0 || e == 2) ? -1.0 : 1.0;
  const int t0 = k * kChunk;
  // along a periodic y axis the W / E bands are closed loops: the halo wraps around
  const bool wrap = g.py && e < 2;
  const int lo = wrap ? t0 - kHalo : max(0, t0 - kHalo);
  const int hi = wrap ? t0 + kChunk + kHalo : min(len, t0 + kChunk + kHalo);
  auto wr = [&](int tt) { return wrap ? ((tt % len) + len) % len : tt; };
  // shared state: [4 buffers][4 comps][M][kText] : V0, stage a, stage b, accumulator
  const int plane = M * kText;
  auto at = [&](int buf, int q, int j, int t) -> double& {
    return sm[(buf * 4 + q) * plane + (j - 1) * kText + (t - lo)];
  };
  const int tid = threadIdx.x;
  const int j = tid / kText + 1, t = lo + tid % kText;
  const bool live = j <= M && t < hi;
  if (live)
    for (int q = 0; q < 4; ++q) at(0, q, j, t) = Vg[q * g.nb + off + (j - 1) * len + wr(t)];
  __syncthreads();
  auto prim = [&](int buf, int jj, int tt) {
    Prim u;
    u.rho = at(buf, 0, jj, tt);
    const double ux = at(buf, 1, jj, tt), uy = at(buf, 2, jj, tt);
    u.un = xaxis ? ux : uy;
    u.ut = xaxis ? uy : ux;
    u.T = at(buf, 3, jj, tt);
    return u;
  };
  auto fluid = [&](int layer, int tt) {
    return load_prim(Ue, g.ne, ueoff + layer * len + wr(tt), xaxis);
  };
  const int variant = bc.edge[e];
  // Appendix PML source of this band position, mapped to (rho, u_x, u_y, T) rates at the
  // time-n state of the outermost fluid node: d rho = s_m, rho du = s_mom - u s_m,
  // (D/2) rho dT = s_E - u . s_mom + (u^2/2 - (D/2) T) s_m (D = 2); constant over the stages
  double src[4] = {0, 0, 0, 0};
  if ((bc.pml_source & 7) && live) {
    const int ns = 2 * (Lx + Ly);
    const int sb = (e == 0 ? 0 : e == 1 ? Ly : e == 2 ? 2 * Ly : 2 * Ly + Lx) + wr(t);
    const int ub = ueoff + wr(t);
    const double rho = Ue[ub], ux = Ue[g.ne + ub], uy = Ue[2 * g.ne + ub], T = Ue[3 * g.ne + ub];
    const double sm = Se[sb], sx = Se[ns + sb], sy = Se[2 * ns + sb], sE = Se[3 * ns + sb];
    src[0] = sm;
    src[1] = (sx - ux * sm) / rho;
    src[2] = (sy - uy * sm) / rho;
    src[3] = (sE - ux * sx - uy * sy + (0.5 * (ux * ux + uy * uy) - T) * sm) / rho;
    if (bc.pml_source & 8)   // the sign printed in Eq. (NSF-CHAR-PML)
      for (int q = 0; q < 4; ++q) src[q] = -src[q];
  }
  double kk[4] = {0, 0, 0, 0};
  for (int s = 1; s <= 4; ++s) {
    const int in_buf = s == 1 ? 0 : (s == 3 ? 2 : 1);  // V0, a, b, a
    const int slo = (!wrap && lo == 0) ? 0 : lo + s, shi = (!wrap && hi == len) ? len : hi - s;
    if (live && t >= slo && t < shi) {
      const Prim U0 = prim(in_buf, j, t);
      const Prim U1 = j >= 2 ? prim(in_buf, j - 1, t) : fluid(0, t);
      const Prim U2 = j >= 3 ? prim(in_buf, j - 2, t) : (j == 2 ? fluid(0, t) : fluid(1, t));
      int ta;
      double ca, cb, cc;
      if (!wrap && t == 0) { ta = 0; ca = -1.5; cb = 2.0; cc = -0.5; }
      else if (!wrap && t == len - 1) { ta = t - 2; ca = 0.5; cb = -2.0; cc = 1.5; }
      else { ta = t - 1; ca = -0.5; cb = 0.0; cc = 0.5; }
      Prim Va = U0, Vb = U0, Vc = U0;
      if (variant != 0) {
        Va = prim(in_buf, j, ta);
        Vb = prim(in_buf, j, ta + 1);
        Vc = prim(in_buf, j, ta + 2);
      }
      char_rate<R>(bc, variant, out, U0, U1, U2, Va, Vb, Vc, ca, cb, cc, xaxis, kk);
      for (int q = 0; q < 4; ++q) kk[q] += src[q];
    }
    __syncthreads();   // everyone has read the stage input before it is overwritten
    if (live && t >= slo && t < shi) {
      if (s < 4) {
        const int out_buf = s == 2 ? 2 : 1;            // a, b, a
        const double a = s == 3 ? 1.0 : 0.5, wgt = s == 1 ? 1.0 : 2.0;
        for (int q = 0; q < 4; ++q) {
          at(out_buf, q, j, t) = at(0, q, j, t) + a * kk[q];
          at(3, q, j, t) = (s == 1 ? 0.0 : at(3, q, j, t)) + wgt * kk[q];
        }
      } else if (t >= t0 && t < t0 + kChunk && t < len) {
        const double sixth = 1.0 / 6.0;
        for (int q = 0; q < 4; ++q)
          Vg[q * g.nb + off + (j - 1) * len + t] = at(0, q, j, t) + (at(3, q, j, t) + kk[q]) * sixth;
      }
    }
    __syncthreads();
  }
}

template <class R>
__global__ void k_nrbc_rk4(Geom g, BcParams bc, const double* __restrict__ Ue,
                           const double* __restrict__ Se, double* __restrict__ Vg) {
  extern __shared__ double sm[];
  nrbc_chunk<R>(g, bc, Ue, Se, Vg, blockIdx.x, sm);
}

template <class R>
__global__ void kb_nrbc_rk4(const TgtDesc* __restrict__ d, const int* __restrict__ tab) {
  extern __shared__ double sm[];
  const int m = tab[2 * blockIdx.x], chunk = tab[2 * blockIdx.x + 1];
  const TgtDesc& t = d[m];
  nrbc_chunk<R>(t.g, t.bc, t.Ue, t.Se, t.V, chunk, sm);
}

void nrbc_shape(const Geom& g, int* chunks, int* threads, size_t* smem) {
  *chunks = 2 * ((g.Ly + kChunk - 1) / kChunk) + 2 * ((g.Lx + kChunk - 1) / kChunk);
  *threads = (g.M * kText + 31) / 32 * 32;
  *smem = sizeof(double) * 16 * g.M * kText;
}

cudaError_t launch_nrbc_batch(const TgtDesc* d, const int* tab, int n, bool fp32, int threads,
                              size_t smem, cudaStream_t s) {
  if (n <= 0) return cudaSuccess;
  if (fp32) kb_nrbc_rk4<float><<<n, threads, smem, s>>>(d, tab);
  else kb_nrbc_rk4<double><<<n, threads, smem, s>>>(d, tab);
  return cudaGetLastError();
}

// The four RK4 stages of one step in one launch; fp32 selects FP32 characteristic algebra
// (targets and differences stay FP64).
cudaError_t launch_nrbc_stages(const Dev& d, bool fp32, cudaStream_t s) {
  const Geom& g = d.g;
  int blocks, threads;
  size_t smem;
  nrbc_shape(g, &blocks, &threads, &smem);
  if (fp32)
    k_nrbc_rk4<float><<<blocks, threads, smem, s>>>(g, d.bc, d.Uedge_in, d.Sedge_in, d.Vtgt);
  else
    k_nrbc_rk4<double><<<blocks, threads, smem, s>>>(g, d.bc, d.Uedge_in, d.Sedge_in, d.Vtgt);
  return cudaGetLastError();
}

// Final pass of the FP64 reductions: one block of 1024 threads; each thread folds whole
// 12-value records (contiguous, so a warp reads 32 consecutive records), then warp shuffles and
// one shared-memory round combine the 32 warps. Sums, except the slots flagged in min_mask
// (minimum).
__global__ void __launch_bounds__(1024) k_reduce_final(const double* __restrict__ partials, int n,
                                                      unsigned min_mask,
                                                      double* __restrict__ out) {
  __shared__ double sh[32][12];
  double a[12];
#pragma unroll
  for (int k = 0; k < 12; ++k) a[k] = ((min_mask >> k) & 1u) ? DBL_MAX : 0.0;
  for (int i = threadIdx.x; i < n; i += blockDim.x) {
    const double* r = partials + 12ll * i;
#pragma unroll
    for (int k = 0; k < 12; ++k) a[k] = ((min_mask >> k) & 1u) ? fmin(a[k], r[k]) : a[k] + r[k];
  }
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nwarps = blockDim.x >> 5;
#pragma unroll
  for (int k = 0; k < 12; ++k)
    for (int o = 16; o > 0; o >>= 1) {
      const double t = __shfl_down_sync(0xffffffffu, a[k], o);
      a[k] = ((min_mask >> k) & 1u) ? fmin(a[k], t) : a[k] + t;
    }
  if (lane == 0)
    for (int k = 0; k < 12; ++k) sh[warp][k] = a[k];
  __syncthreads();
  if (warp == 0) {
    for (int k = 0; k < 12; ++k) {
      const bool mn = (min_mask >> k) & 1u;
      double b = lane < nwarps ? sh[lane][k] : (mn ? DBL_MAX : 0.0);
      for (int o = 16; o > 0; o >>= 1) {
        const double t = __shfl_down_sync(0xffffffffu, b, o);
        b = mn ? fmin(b, t) : b + t;
      }
      if (lane == 0) out[k] = b;
    }
  }
}

cudaError_t reduce_partials(const double* partials, int n, unsigned min_mask, double* out,
                            cudaStream_t st) {
  k_reduce_final<<<1, 1024, 0, st>>>(partials, n, min_mask, out);
  return cudaGetLastError();
}

}  // namespace lbm

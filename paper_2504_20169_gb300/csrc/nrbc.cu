// Characteristic boundary targets (Sec. 4) and the final pass of the FP64 reductions.
#include <cfloat>

#include "lbm_internal.h"

namespace lbm {

// stage 1..4 of classical RK4 over one time step; fluid moments Ue frozen at time n. Targets,
// stage values and all differences are FP64; the characteristic algebra runs in R.
// One stage of classical RK4 for dU/dt of every edge-band node (fluid moments Ue frozen at
// time n). Band node b -> edge (W, E, S, N), layer j = 1..M outward, tangential index t.
// Rates: Eq. (thermal_LODI_macro_evo) with Eq. (PNR) for PNR-LODI edges, Eq.
// (thermal_CBC_macro_evo) with Eq. (CBC-Relax) for CBC-relax edges; viscous part zero.
// Derivatives per node index: normal one-sided 2nd order toward the outside, tangential
// central (one-sided at the band ends); one node is r normalized lengths.
template <class R>
__global__ void k_nrbc_stage(Geom g, BcParams bc, const double* __restrict__ Ue,
                             double* __restrict__ V0, const double* __restrict__ Vin,
                             double* __restrict__ Vout, double* __restrict__ acc, int stage) {
  const int b = blockIdx.x * blockDim.x + threadIdx.x;
  if (b >= g.nb) return;
  const int M = g.M, Lx = g.Lx, Ly = g.Ly;
  int e, off, len, ueoff;
  if (b < M * Ly) { e = 0; off = 0; len = Ly; ueoff = 0; }
  else if (b < 2 * M * Ly) { e = 1; off = M * Ly; len = Ly; ueoff = 2 * Ly; }
  else if (b < 2 * M * Ly + M * Lx) { e = 2; off = 2 * M * Ly; len = Lx; ueoff = 4 * Ly; }
  else { e = 3; off = 2 * M * Ly + M * Lx; len = Lx; ueoff = 4 * Ly + 2 * Lx; }
  const int loc = b - off;
  const int j = loc / len + 1, t = loc - (j - 1) * len;
  const bool xaxis = e < 2;
  const double out = (e == 0 || e == 2) ? -1.0 : 1.0;
  const int nb = g.nb, ne = g.ne;
  auto node = [&](int jj, int tt) { return off + (jj - 1) * len + tt; };

  const Prim U0d = load_prim(Vin, nb, b, xaxis);
  const Prim U1 = j >= 2 ? load_prim(Vin, nb, node(j - 1, t), xaxis)
                         : load_prim(Ue, ne, ueoff + t, xaxis);
  const Prim U2 = j >= 3 ? load_prim(Vin, nb, node(j - 2, t), xaxis)
                         : (j == 2 ? load_prim(Ue, ne, ueoff + t, xaxis)
                                   : load_prim(Ue, ne, ueoff + len + t, xaxis));
  // d/dx_axis per node = out * (3 U(x_b) - 4 U(x_b - n) + U(x_b - 2n)) / 2; differences in FP64
  const double hs = 0.5 * out;
  PrimT<R> dn;
  dn.rho = R(hs * (3.0 * U0d.rho - 4.0 * U1.rho + U2.rho));
  dn.un = R(hs * (3.0 * U0d.un - 4.0 * U1.un + U2.un));
  dn.ut = R(hs * (3.0 * U0d.ut - 4.0 * U1.ut + U2.ut));
  dn.T = R(hs * (3.0 * U0d.T - 4.0 * U1.T + U2.T));

  const PrimT<R> U0 = to<R>(U0d);
  const R inv_r = R(1.0 / bc.r);
  const R c = sqrt(R(2) * U0.T);  // gamma T with gamma = (D + 2) / D = 2
  const R lam[4] = {U0.un - c, U0.un, U0.un, U0.un + c};
  R wn[4];
  char_forward(U0, c, dn, wn);
  const R sgn = R(out);
  R tot[4];
  if (bc.edge[e] == 0) {
    // PNR-LODI: incoming amplitudes vanish, transverse terms dropped
    for (int k = 0; k < 4; ++k) tot[k] = (lam[k] * sgn < R(0)) ? R(0) : lam[k] * wn[k] * inv_r;
  } else {
    // CBC relax: transverse amplitudes T = S B dU/dt_axis
    const int ta = t == 0 ? 0 : (t == len - 1 ? t - 2 : t - 1);
    const Prim Va = load_prim(Vin, nb, node(j, ta), xaxis);
    const Prim Vb = load_prim(Vin, nb, node(j, ta + 1), xaxis);
    const Prim Vc = load_prim(Vin, nb, node(j, ta + 2), xaxis);
    double ca, cb, cc;
    if (t == 0) { ca = -1.5; cb = 2.0; cc = -0.5; }
    else if (t == len - 1) { ca = 0.5; cb = -2.0; cc = 1.5; }
    else { ca = -0.5; cb = 0.0; cc = 0.5; }
    PrimT<R> dt;
    dt.rho = R(ca * Va.rho + cb * Vb.rho + cc * Vc.rho);
    dt.un = R(ca * Va.un + cb * Vb.un + cc * Vc.un);
    dt.ut = R(ca * Va.ut + cb * Vb.ut + cc * Vc.ut);
    dt.T = R(ca * Va.T + cb * Vb.T + cc * Vc.T);
    // B dU along the tangential axis (tangential velocity u_t advects; P_t = T rho_t + rho T_t)
    PrimT<R> bd;
    bd.rho = U0.ut * dt.rho + U0.rho * dt.ut;
    bd.un = U0.ut * dt.un;
    bd.ut = (U0.T / U0.rho) * dt.rho + U0.ut * dt.ut + dt.T;
    bd.T = U0.T * dt.ut + U0.ut * dt.T;  // (2/D) T with D = 2
    R Tc[4];
    char_forward(U0, c, bd, Tc);
    const R relax = R((bc.relax_sign == 0.0 ? -1.0 : bc.relax_sign) * (1.0 - bc.beta));
    for (int k = 0; k < 4; ++k) {
      const R Lbar = (lam[k] * sgn < R(0)) ? relax * Tc[k] : lam[k] * wn[k];
      tot[k] = (Lbar + Tc[k]) * inv_r;
    }
  }
  const PrimT<R> r = char_inverse(U0, c, tot);
  // rate k = -S^-1 (...) in (rho, u_x, u_y, T)
  const double k0 = -double(r.rho), k3 = -double(r.T);
  const double kx = xaxis ? -double(r.un) : -double(r.ut), ky = xaxis ? -double(r.ut) : -double(r.un);
  const double kk[4] = {k0, kx, ky, k3};
  if (stage < 4) {
    const double a = stage == 3 ? 1.0 : 0.5;
    const double wgt = stage == 1 ? 1.0 : 2.0;
    for (int q = 0; q < 4; ++q) {
      Vout[q * nb + b] = V0[q * nb + b] + a * kk[q];
      acc[q * nb + b] = (stage == 1 ? 0.0 : acc[q * nb + b]) + wgt * kk[q];
    }
  } else {
    for (int q = 0; q < 4; ++q) V0[q * nb + b] = V0[q * nb + b] + (acc[q * nb + b] + kk[q]) / 6.0;
  }
}

// The four RK4 stages of one step (buffers: stage input Vtgt -> Va -> Vb -> Va; Vtgt updated in
// place by the last stage).
cudaError_t launch_nrbc_stages(const Dev& d, bool fp32, cudaStream_t s) {
  const Geom& g = d.g;
  const int nbk = (g.nb + 127) / 128;
  const double* Vin[4] = {d.Vtgt, d.Va, d.Vb, d.Va};
  double* Vout[4] = {d.Va, d.Vb, d.Va, nullptr};
  for (int k = 1; k <= 4; ++k) {
    if (fp32)
      k_nrbc_stage<float><<<nbk, 128, 0, s>>>(g, d.bc, d.Uedge, d.Vtgt, Vin[k - 1], Vout[k - 1],
                                               d.Vacc, k);
    else
      k_nrbc_stage<double><<<nbk, 128, 0, s>>>(g, d.bc, d.Uedge, d.Vtgt, Vin[k - 1], Vout[k - 1],
                                                d.Vacc, k);
  }
  return cudaGetLastError();
}

__global__ void k_reduce_final(const double* __restrict__ partials, int n, unsigned min_mask,
                               double* __restrict__ out) {
  __shared__ double sh[256];
  for (int k = 0; k < 12; ++k) {
    const bool is_min = (min_mask >> k) & 1u;
    double a = is_min ? DBL_MAX : 0.0;
    for (int i = threadIdx.x; i < n; i += blockDim.x) {
      const double v = partials[12ll * i + k];
      a = is_min ? fmin(a, v) : a + v;
    }
    sh[threadIdx.x] = a;
    __syncthreads();
    for (int s = blockDim.x / 2; s > 0; s >>= 1) {
      if (threadIdx.x < s) {
        const double o = sh[threadIdx.x + s];
        sh[threadIdx.x] = is_min ? fmin(sh[threadIdx.x], o) : sh[threadIdx.x] + o;
      }
      __syncthreads();
    }
    if (threadIdx.x == 0) out[k] = sh[0];
    __syncthreads();
  }
}

cudaError_t reduce_partials(const double* partials, int n, unsigned min_mask, double* out,
                            cudaStream_t st) {
  k_reduce_final<<<1, 256, 0, st>>>(partials, n, min_mask, out);
  return cudaGetLastError();
}

}  // namespace lbm

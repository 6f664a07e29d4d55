// Device side of the PML + outer-boundary thermal lattice Boltzmann step (arXiv 2504.20169).
//
// Storage. Populations are SoA planes p[i][row][col] over the grid G = F + M boundary layers.
// Node (x, y) of F (0 <= x < Lx) sits at row y + M, column cF0 + x, where cF0 is a multiple of
// 32, so every warp-aligned run of 32 nodes of F starts on a 128 B (FP32) / 256 B (FP64)
// boundary. In LBM_FP32_DEV storage each value is g_i = f_i - w_i (deviation from the rest
// state), otherwise the absolute f_i in FP64.
//
// A stored buffer always holds post-collision populations f* of one time level; a step pulls
// f^(n+1)(x) = f*^n(x - e_i) (Eq. lbe), collides, and writes f*^(n+1).
//
// Work split of one step (all kernels read buffer A and write disjoint parts of buffer B):
//   k_nrbc_rk4        characteristic targets U_tgt^(n+1) on the edge bands, four RK4 stages (Sec. 4)
//   k_bulk            nodes of F inside the frame depths (Fw, Fe, Fs, Fn): BGK only
//   k_frame1          the frame (the outer Fw / Fe / Fs / Fn layers of F): BGK, PML
//                     accumulator, local PML terms,
//                     saving the outer two layers' moments for the characteristic BC
//   k_frame2          PML nodes: the gradient part of Omega^PML (needs the frame's new Q)
//   k_gamma           the M boundary layers outside F (zero gradient, characteristic BC with
//                     non-equilibrium extrapolation, or periodic images)
//   k_wrap_y          periodic y axis only, after all of the above: the M rows beyond each y
//                     end copy the finished rows they image
#pragma once
#include <cstdint>
#include <cuda_runtime.h>

#include "stencils.cuh"

namespace lbm {

constexpr int kMaxQ = 37;

struct Geom {
  int nx, ny, M, Lx, Ly;
  int Ww, We, Ws, Wn; // PML layers on the W, E, S and N edges (0: none there)
  int py;            // 1: the y axis is periodic (then Ws = Wn = 0)
  int pitch;         // storage row length (elements), multiple of 32
  int cF0;           // storage column of x = 0 of F, multiple of 32
  long long plane;   // elements per direction plane (pitch * (Ly + 2M))
  int Fw, Fe, Fs, Fn; // frame depth per edge: max(W_edge + qr, M, 2) with a PML there, else
                     // max(M, 2) (the two outer layers feed the characteristic targets);
                     // Fs = Fn = 0 on a periodic y axis
  int frame_n;       // number of frame nodes
  int link;          // 1: c_i . grad Q_i as the link difference Q_i(x + e_i) - Q_i(x) (an
                     // option; 0: the printed per-axis differences, Eqs. FD-dx-center / -bw)
  int qr;            // depth of the ring of bulk nodes next to P that carries Q: 1 (printed
                     // central difference), M (link difference)
  long long Sp;      // PML accumulator stride per direction: the frame nodes, then (link
                     // mode) the ngamma boundary nodes outside F
  int nb;            // characteristic-BC band nodes: 2 M (Lx + Ly)
  int ne;            // saved fluid-moment slots: 4 (Lx + Ly) (two layers per edge)
  int ngamma;        // boundary nodes outside F: 2M(Lx + 2M) + 2M Ly
};

__host__ __device__ inline bool has_pml(const Geom& g) { return (g.Ww | g.We | g.Ws | g.Wn) > 0; }

// Lattice and physics constants in the arithmetic type of a kernel. eqbar holds the
// equilibrium of the PML mean state (Eq. decomp-NJ) in the storage representation.
template <class Real>
struct Consts {
  Real w[kMaxQ];
  Real eqbar[kMaxQ];
  Real r, r2, omega, sigma_max;
  int power;
  int split;         // 1: sigma_x != sigma_y (Eq. pml-general), 0: sigma_x = sigma_y (Eq. PMLCOLL)
};

struct BcParams {
  int bc;            // 0 periodic, 1 zero gradient, 2 characteristic
  int edge[4];       // W E S N: 0 PNR-LODI, 1 CBC relax
  double beta, relax_sign, r, omega, inv_r;
  int pml_source;    // bitmask of the Appendix PML source terms I (1), II (2), III (4);
                     // 8: with the printed sign instead of the collision's
};

__host__ __device__ inline long long gindex(const Geom& g, int x, int y) {
  return (long long)(y + g.M) * g.pitch + g.cF0 + x;
}

__device__ inline int dist_out(const Geom& g, int x, int y) {
  return min(min(x, g.Lx - 1 - x), min(y, g.Ly - 1 - y));
}

// PML classification of node (x, y) of F. Layer index along x: i = W_w - x near the W edge,
// x - (Lx - 1 - W_e) near the E edge, 0 between (likewise along y with W_s, W_n); layer
// fraction f_x = i / (width of that edge). P = {f_x > 0 or f_y > 0}; the accumulator Q is kept
// on P and on the ring of qr nodes inside each PML edge (in link mode also on every boundary
// node outside F, see q_slot).
template <class Real>
struct PmlNode {
  bool has_q, in_p;
  int ix, iy;        // layer index along x and along y (0 outside that axis' slabs)
  Real fx, fy;
};

template <class Real>
__device__ inline PmlNode<Real> pml_node(const Geom& g, int x, int y) {
  const int ex = g.Lx - 1 - x, ey = g.Ly - 1 - y;
  const int iw = g.Ww > 0 ? max(0, g.Ww - x) : 0, ie = g.We > 0 ? max(0, g.We - ex) : 0;
  const int is = g.Ws > 0 ? max(0, g.Ws - y) : 0, in = g.Wn > 0 ? max(0, g.Wn - ey) : 0;
  PmlNode<Real> n;
  n.in_p = (iw | ie | is | in) > 0;
  n.ix = iw + ie;
  n.iy = is + in;
  const int r = g.qr - 1;
  n.has_q = (g.Ww > 0 && x <= g.Ww + r) || (g.We > 0 && ex <= g.We + r) ||
            (g.Ws > 0 && y <= g.Ws + r) || (g.Wn > 0 && ey <= g.Wn + r);
  n.fx = iw > 0 ? Real(iw) / Real(g.Ww) : (ie > 0 ? Real(ie) / Real(g.We) : Real(0));
  n.fy = is > 0 ? Real(is) / Real(g.Ws) : (in > 0 ? Real(in) / Real(g.Wn) : Real(0));
  return n;
}

// Frame: bottom rows (Fs), top rows (Fn), then left (Fw) and right (Fe) columns of the
// middle rows.
__device__ inline void frame_xy(const Geom& g, int fi, int& x, int& y) {
  const int Lx = g.Lx;
  const int bot = g.Fs * Lx, top = g.Fn * Lx;
  if (fi < bot) { y = fi / Lx; x = fi - y * Lx; return; }
  fi -= bot;
  if (fi < top) { int t = fi / Lx; y = g.Ly - g.Fn + t; x = fi - t * Lx; return; }
  fi -= top;
  const int mid = g.Ly - g.Fs - g.Fn;
  const int left = mid * g.Fw;
  if (fi < left) { int t = fi / g.Fw; y = g.Fs + t; x = fi - t * g.Fw; return; }
  fi -= left;
  int t = fi / g.Fe;
  y = g.Fs + t;
  x = g.Lx - g.Fe + (fi - t * g.Fe);
}

__device__ inline int frame_index(const Geom& g, int x, int y) {
  const int Lx = g.Lx;
  if (y < g.Fs) return y * Lx + x;
  if (y >= g.Ly - g.Fn) return g.Fs * Lx + (y - (g.Ly - g.Fn)) * Lx + x;
  const int base = (g.Fs + g.Fn) * Lx;
  if (x < g.Fw) return base + (y - g.Fs) * g.Fw + x;
  return base + (g.Ly - g.Fs - g.Fn) * g.Fw + (y - g.Fs) * g.Fe + (x - (g.Lx - g.Fe));
}

// sigma of Eq. (PML_ramp) for layer fraction frac = i / W.
template <class Real>
__device__ inline Real sigma_of(const Consts<Real>& c, Real frac) {
  Real p = Real(1);
  for (int k = 0; k < c.power; ++k) p *= frac;
  return c.sigma_max * p;
}

// (sigma_x, sigma_y) of a node of P: both sigma(max(f_x, f_y)) (Eq. PMLCOLL, corners by the
// larger fraction), or per axis in the split form of Eq. (pml-general).
template <class Real>
__device__ inline void pml_sigmas(const Consts<Real>& c, const PmlNode<Real>& n, Real& sx,
                                  Real& sy) {
  if (c.split) {
    sx = n.fx > Real(0) ? sigma_of(c, n.fx) : Real(0);
    sy = n.fy > Real(0) ? sigma_of(c, n.fy) : Real(0);
  } else {
    sx = sigma_of(c, n.fx > n.fy ? n.fx : n.fy);
    sy = sx;
  }
}

// ------------------------------------------------------------------------------------------
// Per-node arithmetic
// ------------------------------------------------------------------------------------------

// Macroscopic state of a node: rho, the velocity scaled by r (so xi_i . u = ex urx + ey ury),
// u^2 and theta = T - 1. drho = rho - 1 is kept for the deviation storage.
template <class Real>
struct Macro {
  Real rho, drho, urx, ury, u2, theta, inv_rho;
};

// Eq. (macro) on stored values p (absolute f, or g = f - w when DEV).
template <class S, class Real, bool DEV>
__host__ __device__ inline Macro<Real> moments(const Real (&p)[S::Q], const Consts<Real>& c) {
  // column sums cx[k] = sum of p_i with e_ix = k and row sums cy[k] (k = -3..3): every moment
  // below follows from them (rho, sum p e_x, sum p e_x^2 and the y counterparts)
  Real cx[7] = {0, 0, 0, 0, 0, 0, 0}, cy[7] = {0, 0, 0, 0, 0, 0, 0};
#pragma unroll
  for (int i = 0; i < S::Q; ++i) {
    cx[S::ex(i) + 3] += p[i];
    cy[S::ey(i) + 3] += p[i];
  }
  const Real s0 = ((cx[0] + cx[6]) + (cx[1] + cx[5])) + ((cx[2] + cx[4]) + cx[3]);
  const Real sx = (cx[4] - cx[2]) + Real(2) * (cx[5] - cx[1]) + Real(3) * (cx[6] - cx[0]);
  const Real sy = (cy[4] - cy[2]) + Real(2) * (cy[5] - cy[1]) + Real(3) * (cy[6] - cy[0]);
  const Real sxx = (cx[4] + cx[2]) + Real(4) * (cx[5] + cx[1]) + Real(9) * (cx[6] + cx[0]);
  const Real syy = (cy[4] + cy[2]) + Real(4) * (cy[5] + cy[1]) + Real(9) * (cy[6] + cy[0]);
  const Real s2 = sxx + syy;
  Macro<Real> m;
  if (DEV) {
    m.drho = s0;
    m.rho = Real(1) + s0;
  } else {
    m.rho = s0;
    m.drho = s0 - Real(1);
  }
  m.inv_rho = Real(1) / m.rho;
  // rho u = sum f xi = r sum f e (the rest weights carry no momentum)
  const Real ux = c.r * sx * m.inv_rho, uy = c.r * sy * m.inv_rho;
  m.urx = c.r * ux;
  m.ury = c.r * uy;
  m.u2 = ux * ux + uy * uy;
  // D rho T = sum f |xi|^2 - rho u^2 with D = 2; sum w |xi|^2 = D for the deviation form
  if (DEV)
    m.theta = Real(0.5) * (c.r2 * s2 * m.inv_rho - m.u2 - Real(2) * m.drho * m.inv_rho);
  else
    m.theta = Real(0.5) * (c.r2 * s2 * m.inv_rho - m.u2) - Real(1);
  return m;
}

// Quadrature weights in constant memory, one table per stencil and precision (filled once per
// device when the first context is created there): with a direction index known at compile
// time, a kernel reads its weight as an instruction operand instead of a load. Host code (the
// mean equilibrium) reads the context's constants.
static __constant__ double kw37d[37], kw17d[17], kw9d[9];
static __constant__ float kw37f[37], kw17f[17], kw9f[9];

template <class S, class Real>
__host__ __device__ inline Real weight(const Consts<Real>& c, int i) {
#ifdef __CUDA_ARCH__
  if constexpr (sizeof(Real) == 8) {
    if constexpr (S::Q == 37) return kw37d[i];
    else if constexpr (S::Q == 17) return kw17d[i];
    else return kw9d[i];
  } else {
    if constexpr (S::Q == 37) return kw37f[i];
    else if constexpr (S::Q == 17) return kw17f[i];
    else return kw9f[i];
  }
#else
  return c.w[i];
#endif
}

// Site coefficients of the equilibrium polynomial in a = xi . u (Eqs. feq-2/3/4):
//   P(a) = C0 + C1 a + C2 a^2 + C3 a^3 + C4 a^4,   C0 = k00 + c2 (k01 + c2 k02),
//   C1 = k10 + c2 k11, C2 = k20 + c2 k21, C3 = 1/6 (order >= 3), C4 = 1/24 (order 4),
// with c2 = |xi|^2 of the shell. k00m = k00 - 1 (for the deviation form, no cancellation).
template <class Real>
struct EqCoef {
  Real k00m, k01, k02, k10, k11, k20, k21;
};

template <int ORDER, class Real>
__host__ __device__ inline EqCoef<Real> eq_coef(const Macro<Real>& m) {
  const Real u2 = m.u2, th = m.theta;
  EqCoef<Real> k;
  if (ORDER >= 4) {
    k.k00m = -Real(0.5) * u2 - th + Real(0.125) * u2 * u2 + th * u2 + th * th;
    k.k01 = Real(0.5) * th - Real(0.25) * th * u2 - th * th;
    k.k02 = Real(0.125) * th * th;
    k.k20 = Real(0.5) - Real(0.25) * u2 - Real(1.5) * th;
    k.k21 = Real(0.25) * th;
  } else {
    k.k00m = -Real(0.5) * u2 - th;
    k.k01 = Real(0.5) * th;
    k.k02 = Real(0);
    k.k20 = Real(0.5);
    k.k21 = Real(0);
  }
  if (ORDER >= 3) {
    k.k10 = Real(1) - Real(0.5) * u2 - Real(2) * th;
    k.k11 = Real(0.5) * th;
  } else {
    k.k10 = Real(1);
    k.k11 = Real(0);
  }
  return k;
}

// Equilibrium of direction i in the storage representation: f_eq (absolute) or
// f_eq - w = w (rho (P - 1) + drho) (deviation).
template <class S, class Real, bool DEV>
__host__ __device__ inline Real eq_dir(int i, const Macro<Real>& m, const EqCoef<Real>& k,
                              const Consts<Real>& c) {
  const Real c2 = c.r2 * Real(e2_of<S>(i));
  const Real a = Real(S::ex(i)) * m.urx + Real(S::ey(i)) * m.ury;
  const Real C0m = k.k00m + c2 * (k.k01 + c2 * k.k02);
  const Real C1 = k.k10 + c2 * k.k11;
  const Real C2 = k.k20 + c2 * k.k21;
  Real poly = C2;
  if (S::ORDER >= 3) {
    Real C34 = Real(1.0 / 6.0);
    if (S::ORDER >= 4) C34 = C34 + a * Real(1.0 / 24.0);
    poly = poly + a * C34;
  }
  const Real Pm1 = C0m + a * (C1 + a * poly);  // P - 1
  if (DEV) return weight<S, Real>(c, i) * (m.rho * Pm1 + m.drho);
  return weight<S, Real>(c, i) * m.rho * (Real(1) + Pm1);
}

// Same, for all directions at once using the +/- pairing: E(a) = C0 + a^2 (C2 + a^2 C4),
// O(a) = a (C1 + a^2 C3), P(+-a) = E +- O. Writes the post-collision value
// f + omega (eq - f) = (1 - omega) f + omega eq, with omega folded into the weights.
template <class S, class Real, bool DEV>
__device__ inline void collide_bgk(Real (&p)[S::Q], const Macro<Real>& m,
                                   const Consts<Real>& c) {
  const EqCoef<Real> k = eq_coef<S::ORDER, Real>(m);
  const Real om = c.omega;
#pragma unroll
  for (int s = 0; s < S::NSHELL; ++s) {
    const int i0 = S::shell_first(s);
    const int n = S::shell_size(s);
    const Real c2 = c.r2 * Real(e2_of<S>(i0));
    const Real C0m = k.k00m + c2 * (k.k01 + c2 * k.k02);
    const Real C1 = k.k10 + c2 * k.k11;
    const Real C2 = k.k20 + c2 * k.k21;
    const Real wr = om * weight<S, Real>(c, i0) * m.rho;     // omega w rho (a shell shares w)
    const Real wd = om * weight<S, Real>(c, i0) * m.drho;
    const Real keep = Real(1) - om;
    if (n == 1) {
      const Real eq = DEV ? (wr * C0m + wd) : (wr + wr * C0m);
      p[i0] = keep * p[i0] + eq;
      continue;
    }
#pragma unroll
    for (int h = 0; h < n / 2; ++h) {
      const int ip = i0 + h, im = i0 + h + n / 2;
      const Real a = Real(S::ex(ip)) * m.urx + Real(S::ey(ip)) * m.ury;
      const Real a2 = a * a;
      Real Ev = C2;
      if (S::ORDER >= 4) Ev = Ev + a2 * Real(1.0 / 24.0);
      Ev = C0m + a2 * Ev;                      // E - 1
      Real Ov = C1;
      if (S::ORDER >= 3) Ov = Ov + a2 * Real(1.0 / 6.0);
      Ov = a * Ov;
      Real eqp, eqm;
      if (DEV) {
        const Real base = wr * Ev + wd;
        const Real odd = wr * Ov;
        eqp = base + odd;
        eqm = base - odd;
      } else {
        const Real base = wr + wr * Ev;
        const Real odd = wr * Ov;
        eqp = base + odd;
        eqm = base - odd;
      }
      p[ip] = keep * p[ip] + eqp;
      p[im] = keep * p[im] + eqm;
    }
  }
}

template <class Real>
__device__ inline bool unphysical(const Macro<Real>& m) {
  const Real T = Real(1) + m.theta;
  return !(m.rho > Real(0)) || !(T > Real(0)) || !(m.rho < Real(1e30)) || !(T < Real(1e30));
}

// Storage index of the pull source x - e_i of the node at storage index idx (Eq. lbe).
__host__ __device__ inline long long pull_src(const Geom& g, long long idx, int ex, int ey) {
  return idx - (long long)ey * g.pitch - ex;
}

template <class S, class Real, bool STREAM>
__device__ inline void load_pop(Real (&p)[S::Q], const Real* __restrict__ A, const Geom& g,
                                long long idx) {
#pragma unroll
  for (int i = 0; i < S::Q; ++i) {
    const long long src = STREAM ? pull_src(g, idx, S::ex(i), S::ey(i)) : idx;
    p[i] = __ldg(A + (long long)i * g.plane + src);
  }
}

// ------------------------------------------------------------------------------------------
// Kernels
// ------------------------------------------------------------------------------------------

// Interior of F (inside the frame depths Fw, Fe, Fs, Fn): pull, moments, BGK, store.
// Block: 32 x BY threads; the x tiles start on a 32-node boundary of F.
// (bulk_node is the per-node work, shared with the batched launch over many instances.)
template <class S, class Real, bool DEV, bool STREAM>
__device__ __forceinline__ void bulk_node(const Geom& g, const Consts<Real>& c,
                                          const Real* __restrict__ A, Real* __restrict__ B,
                                          int* flag, int x, int y) {
  if (x < g.Fw || x >= g.Lx - g.Fe || y >= g.Ly - g.Fn) return;
  const long long idx = gindex(g, x, y);
  Real p[S::Q];
  load_pop<S, Real, STREAM>(p, A, g, idx);
  const Macro<Real> m = moments<S, Real, DEV>(p, c);
  if (unphysical(m)) *flag = 1;
  collide_bgk<S, Real, DEV>(p, m, c);
#pragma unroll
  for (int i = 0; i < S::Q; ++i) B[(long long)i * g.plane + idx] = p[i];
}

template <class S, class Real, bool DEV, bool STREAM>
__global__ void __launch_bounds__(256) k_bulk(Geom g, Consts<Real> c, const Real* __restrict__ A,
                                              Real* __restrict__ B, int* flag) {
  const int x0 = (g.Fw / 32) * 32;
  bulk_node<S, Real, DEV, STREAM>(g, c, A, B, flag, x0 + blockIdx.x * 32 + threadIdx.x,
                                  g.Fs + blockIdx.y * blockDim.y + threadIdx.y);
}

// Writes the time-level moments of a node in the outer two layers of F into every edge slot
// that refers to it (the characteristic BC reads them at the next step).
template <class Real>
__device__ inline void save_edge_moments(const Geom& g, double* Ue, int x, int y,
                                         const Macro<Real>& m, Real r) {
  const double rho = double(m.rho), ux = double(m.urx / r), uy = double(m.ury / r);
  const double T = 1.0 + double(m.theta);
  const int ne = g.ne;
  auto put = [&](int slot) {
    Ue[slot] = rho;
    Ue[ne + slot] = ux;
    Ue[2 * ne + slot] = uy;
    Ue[3 * ne + slot] = T;
  };
  const int Lx = g.Lx, Ly = g.Ly;
  // slot layout: W [2][Ly], E [2][Ly], S [2][Lx], N [2][Lx]
  if (x < 2) put(x * Ly + y);
  if (x >= Lx - 2) put(2 * Ly + (Lx - 1 - x) * Ly + y);
  if (y < 2) put(4 * Ly + y * Lx + x);
  if (y >= Ly - 2) put(4 * Ly + 2 * Lx + (Ly - 1 - y) * Lx + x);
}

// Slot of the outermost fluid node (x, y) in the PML-source arrays of edge e (W E S N):
// W [Ly], E [Ly], S [Lx], N [Lx]; -1 when the node is not on that edge.
__device__ inline int src_slot(const Geom& g, int e, int x, int y) {
  if (e == 0) return x == 0 ? y : -1;
  if (e == 1) return x == g.Lx - 1 ? g.Ly + y : -1;
  if (g.py) return -1;
  if (e == 2) return y == 0 ? 2 * g.Ly + x : -1;
  return y == g.Ly - 1 ? 2 * g.Ly + g.Lx + x : -1;
}

// Mass, momentum and energy moments (sum of |xi|^2 / 2) of a per-direction PML part, written
// (add = false) or added (add = true) into every edge slot of an outermost fluid node.
template <class Real>
__device__ inline void put_pml_source(const Geom& g, double* Se, int x, int y, const Real mom[4],
                                      bool add) {
  const int ns = 2 * (g.Lx + g.Ly);
  for (int e = 0; e < 4; ++e) {
    const int k = src_slot(g, e, x, y);
    if (k < 0) continue;
    for (int q = 0; q < 4; ++q) Se[q * ns + k] = (add ? Se[q * ns + k] : 0.0) + double(mom[q]);
  }
}

__device__ inline bool outermost(const Geom& g, int x, int y) {
  return x == 0 || x == g.Lx - 1 || (!g.py && (y == 0 || y == g.Ly - 1));
}

// 4-byte asynchronous global -> shared copy (cp.async) and the wait for all of this thread's
// copies.
__device__ __forceinline__ void cp_async4(float* dst, const float* src) {
  const unsigned d = static_cast<unsigned>(__cvta_generic_to_shared(dst));
  asm volatile("cp.async.ca.shared.global [%0], [%1], 4;\n" ::"r"(d), "l"(src) : "memory");
}
__device__ __forceinline__ void cp_async_wait_all() {
  asm volatile("cp.async.wait_all;\n" ::: "memory");
}

// Frame, phase 1: BGK plus, on P and its inner ring, the trapezoidal accumulator
// S = Q + f_hat / 2 (Eq. PMLQ: Q^n = S^(n-1) + f_hat^n / 2, S^n = S^(n-1) + f_hat^n), and on P
// the local part -((sigma_x + sigma_y) f_hat + sigma_x sigma_y Q) of Eq. (pml-general)
// (-sigma (2 f_hat + sigma Q) of Eq. PMLCOLL when sigma_x = sigma_y). With the link gradient
// the node also stores Q^n in place of S^(n-1) (no kernel of the step reads S^(n-1) after its
// own node's phase 1; the next step writes S^(n+1) there) and adds its own share
// +sigma Q_i(x) of the link difference, so phase 2 gathers one value per direction.
// STAGE (FP32 table-driven launch): S^(n-1) of the node is copied into `stage` (Q values of
// shared memory owned by this thread) by cp.async while the populations are pulled, instead
// of being held in registers.
template <class S, class Real, bool DEV, bool STREAM, bool STAGE = false>
__device__ __forceinline__ void frame1_node(const Geom& g, const Consts<Real>& c,
                                            const Real* __restrict__ A, Real* __restrict__ B,
                                            Real* __restrict__ Sold,
                                            Real* __restrict__ Snew, double* Uedge,
                                            int save_edges, int* flag, double* Sedge,
                                            int src_mask, int fi, Real* stage = nullptr) {
  if (fi >= g.frame_n) return;
  int x, y;
  frame_xy(g, fi, x, y);
  const int d = dist_out(g, x, y);
  const long long idx = gindex(g, x, y);
  if constexpr (STAGE) {
    if (pml_node<Real>(g, x, y).has_q) {
#pragma unroll
      for (int i = 0; i < S::Q; ++i) cp_async4(stage + i, Sold + (long long)i * g.Sp + fi);
    }
  }
  Real p[S::Q];
  load_pop<S, Real, STREAM>(p, A, g, idx);
  const Macro<Real> m = moments<S, Real, DEV>(p, c);
  if (unphysical(m)) *flag = 1;
  if (save_edges && d < 2) save_edge_moments(g, Uedge, x, y, m, c.r);
  const PmlNode<Real> pn = pml_node<Real>(g, x, y);
  const bool has_q = pn.has_q;
  const bool in_p = pn.in_p;
  Real sx = Real(0), sy = Real(0);
  if (in_p) pml_sigmas(c, pn, sx, sy);
  const Real ssum = sx + sy, sprod = sx * sy;
  const EqCoef<Real> k = eq_coef<S::ORDER, Real>(m);
  // Appendix PML source at the outermost layer: moments of the f_hat (II) and Q (III) parts
  // here; the gradient part (I) is added by k_frame2
  const bool src = src_mask && outermost(g, x, y);
  double smom[4] = {0.0, 0.0, 0.0, 0.0};   // FP64 sums (cancellation)
  if (has_q) {
    // FP32: all accumulator loads in flight before any store (the FP64 build has no registers
    // to spare for them next to its populations)
    constexpr bool kHoist = sizeof(Real) == 4 && !STAGE;
    Real so[S::Q];
    if (kHoist) {
#pragma unroll
      for (int i = 0; i < S::Q; ++i) so[i] = Sold[(long long)i * g.Sp + fi];
    }
    if constexpr (STAGE) cp_async_wait_all();
#pragma unroll
    for (int i = 0; i < S::Q; ++i) {
      const Real eq = eq_dir<S, Real, DEV>(i, m, k, c);
      const Real fhat = eq - c.eqbar[i];
      const Real s0 = STAGE ? stage[i] : (kHoist ? so[i] : Sold[(long long)i * g.Sp + fi]);
      const Real q = s0 + Real(0.5) * fhat;
      Snew[(long long)i * g.Sp + fi] = s0 + fhat;
      if (g.link) Sold[(long long)i * g.Sp + fi] = q;   // Q^n over S^(n-1), gathered by phase 2
      Real out = p[i] + c.omega * (eq - p[i]);
      if (in_p) {
        out = out - (ssum * fhat + sprod * q);
        // link mode: the node's own share +sigma Q_i(x) of -sigma (Q_i(x + e_i) - Q_i(x))
        if (g.link && (S::ex(i) != 0 || S::ey(i) != 0)) out = out + sx * q;
      }
      B[(long long)i * g.plane + idx] = out;
      if (src && in_p) {
        const double part = -(((src_mask & 2) ? double(ssum) * double(fhat) : 0.0) +
                              ((src_mask & 4) ? double(sprod) * double(q) : 0.0));
        smom[0] += part;
        smom[1] += double(S::ex(i)) * part;
        smom[2] += double(S::ey(i)) * part;
        smom[3] += double(S::ex(i) * S::ex(i) + S::ey(i) * S::ey(i)) * part;
      }
    }
  } else {
    collide_bgk<S, Real, DEV>(p, m, c);
#pragma unroll
    for (int i = 0; i < S::Q; ++i) B[(long long)i * g.plane + idx] = p[i];
  }
  if (src) {
    // lattice moments -> physical: xi = r e, |xi|^2 / 2 = r^2 |e|^2 / 2
    smom[1] *= double(c.r);
    smom[2] *= double(c.r);
    smom[3] *= 0.5 * double(c.r2);
    put_pml_source(g, Sedge, x, y, smom, false);
  }
}

template <class S, class Real, bool DEV, bool STREAM>
__global__ void __launch_bounds__(128) k_frame1(Geom g, Consts<Real> c, const Real* __restrict__ A,
                                                Real* __restrict__ B, Real* __restrict__ Sold,
                                                Real* __restrict__ Snew, double* Uedge, int save_edges,
                                                int* flag, double* Sedge, int src_mask) {
  frame1_node<S, Real, DEV, STREAM>(g, c, A, B, Sold, Snew, Uedge, save_edges, flag, Sedge,
                                    src_mask, blockIdx.x * blockDim.x + threadIdx.x);
}

// Frame, phase 2 (PML nodes): subtract sigma_y c_ix dQ_i/dx + sigma_x c_iy dQ_i/dy (sigma
// e_i . grad Q_i when sigma_x = sigma_y) with Q = (S^(n-1) + S^n) / 2,
// Eq. (FD-dx-center) per axis, Eq. (FD-dx-bw) along the outward normal at the outermost layer;
// with the link gradient, the neighbour's share of the link difference (Q^n read in place).
template <class S, class Real, bool STAGE = false>
__device__ __forceinline__ void frame2_node(const Geom& g, const Consts<Real>& c,
                                            Real* __restrict__ B, const Real* __restrict__ Sold,
                                            const Real* __restrict__ Snew, double* Sedge,
                                            int src_mask, int fi, Real* stq = nullptr,
                                            Real* stb = nullptr) {
  if (fi >= g.frame_n) return;
  int x, y;
  frame_xy(g, fi, x, y);
  const PmlNode<Real> pn = pml_node<Real>(g, x, y);
  if (!pn.in_p) return;
  Real sx, sy;
  pml_sigmas(c, pn, sx, sy);
  if (g.link) {
    // link mode: the remaining -sigma Q_i(x + e_i) of -sigma (Q_i(x + e_i) - Q_i(x)), the
    // integral of sigma c_i . grad Q_i along the link the population travels (sigma_x =
    // sigma_y); phase 1 added +sigma Q_i(x), and Q^n sits in the S^(n-1) slots of the frame and
    // of the boundary nodes outside F, where phase 1 and the band kernel stored it
    const long long idx = gindex(g, x, y);
    const bool src = (src_mask & 1) && outermost(g, x, y);   // Appendix term I
    // a node whose whole stencil lies in its own band finds a neighbour's slot at a linear
    // offset (row length rl) from its own; other nodes use q_slot
    constexpr int R = S::M;
    int rl = 0;
    if (y < g.Fs) {
      if (x >= R && x < g.Lx - R && y >= R && y + R < g.Fs) rl = g.Lx;
    } else if (y >= g.Ly - g.Fn) {
      if (x >= R && x < g.Lx - R && y - R >= g.Ly - g.Fn && y + R < g.Ly) rl = g.Lx;
    } else if (x < g.Fw) {
      if (x >= R && x + R < g.Fw && y - R >= g.Fs && y + R < g.Ly - g.Fn) rl = g.Fw;
    } else {
      if (x - R >= g.Lx - g.Fe && x + R < g.Lx && y - R >= g.Fs && y + R < g.Ly - g.Fn) rl = g.Fe;
    }
    double smom[4] = {0.0, 0.0, 0.0, 0.0};   // FP64 sums (cancellation)
    // every gather (and in FP32 every load of B) in flight before the first update of B:
    // in registers, or (STAGE) copied into this thread's shared-memory rows by cp.async
    constexpr bool kHoistB = sizeof(Real) == 4 && !STAGE;
    Real qg[S::Q], bg[S::Q];
#pragma unroll
    for (int i = 0; i < S::Q; ++i) {
      if (S::ex(i) == 0 && S::ey(i) == 0) continue;
      const int nb = rl ? fi + S::ey(i) * rl + S::ex(i) : q_slot(g, x + S::ex(i), y + S::ey(i));
      if constexpr (STAGE) {
        cp_async4(stq + i, Sold + (long long)i * g.Sp + nb);
        cp_async4(stb + i, B + (long long)i * g.plane + idx);
      } else {
        qg[i] = __ldg(Sold + (long long)i * g.Sp + nb);
        if (kHoistB) bg[i] = B[(long long)i * g.plane + idx];
      }
    }
    if constexpr (STAGE) cp_async_wait_all();
#pragma unroll
    for (int i = 0; i < S::Q; ++i) {
      if (S::ex(i) == 0 && S::ey(i) == 0) continue;
      const Real* sq = Sold + (long long)i * g.Sp;
      const Real qn = STAGE ? stq[i] : qg[i];
      Real* b = B + (long long)i * g.plane + idx;
      *b = (STAGE ? stb[i] : (kHoistB ? bg[i] : *b)) - sx * qn;
      if (src) {
        const double part = -double(sx) * (double(qn) - double(__ldg(sq + fi)));
        smom[0] += part;
        smom[1] += double(S::ex(i)) * part;
        smom[2] += double(S::ey(i)) * part;
        smom[3] += double(S::ex(i) * S::ex(i) + S::ey(i) * S::ey(i)) * part;
      }
    }
    if (src) {
      smom[1] *= double(c.r);
      smom[2] *= double(c.r);
      smom[3] *= 0.5 * double(c.r2);
      put_pml_source(g, Sedge, x, y, smom, true);
    }
    return;
  }
  // x axis: neighbours / one-sided stencil
  int ax0, ax1, ax2;  // frame indices; derivative = cx0*Q(ax0) + cx1*Q(ax1) + cx2*Q(ax2)
  Real cx0, cx1, cx2;
  if (x == 0) {  // outward normal -x: dQ/dx = -(3Q(x) - 4Q(x+1) + Q(x+2))/2
    ax0 = fi; ax1 = frame_index(g, 1, y); ax2 = frame_index(g, 2, y);
    cx0 = Real(-1.5); cx1 = Real(2); cx2 = Real(-0.5);
  } else if (x == g.Lx - 1) {
    ax0 = fi; ax1 = frame_index(g, x - 1, y); ax2 = frame_index(g, x - 2, y);
    cx0 = Real(1.5); cx1 = Real(-2); cx2 = Real(0.5);
  } else {
    ax0 = frame_index(g, x + 1, y); ax1 = frame_index(g, x - 1, y); ax2 = fi;
    cx0 = Real(0.5); cx1 = Real(-0.5); cx2 = Real(0);
  }
  int ay0, ay1, ay2;
  Real cy0, cy1, cy2;
  if (g.py) {  // periodic y: central difference with wrap
    ay0 = frame_index(g, x, y + 1 < g.Ly ? y + 1 : 0);
    ay1 = frame_index(g, x, y > 0 ? y - 1 : g.Ly - 1);
    ay2 = fi;
    cy0 = Real(0.5); cy1 = Real(-0.5); cy2 = Real(0);
  } else if (y == 0) {
    ay0 = fi; ay1 = frame_index(g, x, 1); ay2 = frame_index(g, x, 2);
    cy0 = Real(-1.5); cy1 = Real(2); cy2 = Real(-0.5);
  } else if (y == g.Ly - 1) {
    ay0 = fi; ay1 = frame_index(g, x, y - 1); ay2 = frame_index(g, x, y - 2);
    cy0 = Real(1.5); cy1 = Real(-2); cy2 = Real(0.5);
  } else {
    ay0 = frame_index(g, x, y + 1); ay1 = frame_index(g, x, y - 1); ay2 = fi;
    cy0 = Real(0.5); cy1 = Real(-0.5); cy2 = Real(0);
  }
  const long long idx = gindex(g, x, y);
  const bool src = (src_mask & 1) && outermost(g, x, y);   // Appendix term I
  double smom[4] = {0.0, 0.0, 0.0, 0.0};   // FP64 sums (cancellation)
#pragma unroll
  for (int i = 0; i < S::Q; ++i) {
    const Real* so = Sold + (long long)i * g.Sp;
    const Real* sn = Snew + (long long)i * g.Sp;
    Real gq = 0;   // sigma_y c_x dQ/dx + sigma_x c_y dQ/dy, with 2Q
    if (S::ex(i) != 0) {
      const Real dx = cx0 * (__ldg(so + ax0) + __ldg(sn + ax0)) +
                      cx1 * (__ldg(so + ax1) + __ldg(sn + ax1)) +
                      cx2 * (__ldg(so + ax2) + __ldg(sn + ax2));
      gq += sy * Real(S::ex(i)) * dx;
    }
    if (S::ey(i) != 0) {
      const Real dy = cy0 * (__ldg(so + ay0) + __ldg(sn + ay0)) +
                      cy1 * (__ldg(so + ay1) + __ldg(sn + ay1)) +
                      cy2 * (__ldg(so + ay2) + __ldg(sn + ay2));
      gq += sx * Real(S::ey(i)) * dy;
    }
    Real* b = B + (long long)i * g.plane + idx;
    *b = *b - Real(0.5) * gq;   // Q = (S^(n-1) + S^n) / 2
    if (src) {
      const double part = -0.5 * double(gq);
      smom[0] += part;
      smom[1] += double(S::ex(i)) * part;
      smom[2] += double(S::ey(i)) * part;
      smom[3] += double(S::ex(i) * S::ex(i) + S::ey(i) * S::ey(i)) * part;
    }
  }
  if (src) {
    smom[1] *= double(c.r);
    smom[2] *= double(c.r);
    smom[3] *= 0.5 * double(c.r2);
    put_pml_source(g, Sedge, x, y, smom, true);
  }
}

template <class S, class Real>
__global__ void __launch_bounds__(128) k_frame2(Geom g, Consts<Real> c, Real* __restrict__ B,
                                                const Real* __restrict__ Sold,
                                                const Real* __restrict__ Snew, double* Sedge,
                                                int src_mask) {
  frame2_node<S, Real>(g, c, B, Sold, Snew, Sedge, src_mask, blockIdx.x * blockDim.x + threadIdx.x);
}

__device__ inline void gamma_xy(const Geom& g, int t, int& x, int& y) {
  const int M = g.M, Gx = g.Lx + 2 * M;
  if (t < M * Gx) { y = t / Gx; x = t - y * Gx - M; y -= M; return; }
  t -= M * Gx;
  if (t < M * Gx) { int r = t / Gx; y = g.Ly + r; x = t - r * Gx - M; return; }
  t -= M * Gx;
  const int r = t / (2 * M), k = t - r * 2 * M;
  y = r;
  x = k < M ? k - M : g.Lx + (k - M);
}

// Inverse of gamma_xy: index of a boundary node (x, y) outside F.
__device__ inline int gamma_index(const Geom& g, int x, int y) {
  const int M = g.M, Gx = g.Lx + 2 * M;
  if (y < 0) return (y + M) * Gx + (x + M);
  if (y >= g.Ly) return M * Gx + (y - g.Ly) * Gx + (x + M);
  return 2 * M * Gx + y * 2 * M + (x < 0 ? x + M : M + (x - g.Lx));
}

// Slot of node (x, y) of G in the accumulator arrays in link mode: its frame index inside F,
// frame_n + its boundary index outside F; along a periodic y axis y is wrapped first.
__device__ inline int q_slot(const Geom& g, int x, int y) {
  if (g.py) y = y < 0 ? y + g.Ly : (y >= g.Ly ? y - g.Ly : y);
  if (x >= 0 && x < g.Lx && y >= 0 && y < g.Ly) return frame_index(g, x, y);
  return g.frame_n + gamma_index(g, x, y);
}

// Boundary layers outside F (Sec. 4): the post-stream populations there are set by the BC and
// then BGK-collided (no PML term). Zero gradient (Eq. zg-bc): copy of the nearest fluid node x_f,
// so the result equals the BGK post-collision of x_f. Characteristic BC on the edge bands:
// f = f_eq(U_tgt) + f_neq(x_f), whose moments are U_tgt, so the collided value is
// f_eq(U_tgt) + (1 - omega) f_neq(x_f); the corner blocks use the zero-gradient copy.
// Periodic: the post-collision value of the periodic image.
// Link mode with a PML (Sold != nullptr): the node also advances its accumulator
// S^n = S^(n-1) + f_hat^n (slot frame_n + t) from the moments of its pre-collision state, and
// stores Q^n = S^(n-1) + f_hat^n / 2 in place of S^(n-1) for the frame's phase 2.
template <class S, class Real, bool DEV, bool STREAM>
__device__ __forceinline__ void gamma_node(const Geom& g, const Consts<Real>& c,
                                           const BcParams& bc, const Real* __restrict__ A,
                                           Real* __restrict__ B,
                                           const double* __restrict__ Vtgt,
                                           Real* __restrict__ Sold,
                                           Real* __restrict__ Snew, int t) {
  if (t >= g.ngamma) return;
  int x, y;
  gamma_xy(g, t, x, y);
  // rows beyond a periodic y axis are copied from the finished rows they image (k_wrap_y)
  if (g.py && (y < 0 || y >= g.Ly)) return;
  const long long dst = gindex(g, x, y);
  int sx, sy;
  if (bc.bc == 0) {
    sx = (x + g.Lx) % g.Lx;
    sy = (y + g.Ly) % g.Ly;
  } else {
    sx = min(max(x, 0), g.Lx - 1);
    sy = min(max(y, 0), g.Ly - 1);
  }
  Real p[S::Q];
  load_pop<S, Real, STREAM>(p, A, g, gindex(g, sx, sy));
  const Macro<Real> m = moments<S, Real, DEV>(p, c);
  const bool xo = x < 0 || x >= g.Lx, yo = y < 0 || y >= g.Ly;
  if (bc.bc == 2 && xo != yo) {
    // edge band node: index into the target arrays
    int b;
    const int M = g.M, Lx = g.Lx, Ly = g.Ly;
    if (x < 0) b = (-x - 1) * Ly + y;
    else if (x >= Lx) b = M * Ly + (x - Lx) * Ly + y;
    else if (y < 0) b = 2 * M * Ly + (-y - 1) * Lx + x;
    else b = 2 * M * Ly + M * Lx + (y - Ly) * Lx + x;
    Macro<Real> mt;
    const double trho = Vtgt[b], tux = Vtgt[g.nb + b], tuy = Vtgt[2 * g.nb + b],
                 tT = Vtgt[3 * g.nb + b];
    mt.rho = Real(trho);
    mt.drho = Real(trho - 1.0);
    mt.inv_rho = Real(1.0 / trho);
    mt.urx = Real(bc.r * tux);
    mt.ury = Real(bc.r * tuy);
    mt.u2 = Real(tux * tux + tuy * tuy);
    mt.theta = Real(tT - 1.0);
    const EqCoef<Real> kf = eq_coef<S::ORDER, Real>(m);
    const EqCoef<Real> kt = eq_coef<S::ORDER, Real>(mt);
    const Real keep = Real(1) - c.omega;
    // FP32: accumulator loads in flight before any store (FP64 has no registers to spare)
    constexpr bool kHoist = sizeof(Real) == 4;
    Real so[S::Q];
    if (kHoist && Sold) {
#pragma unroll
      for (int i = 0; i < S::Q; ++i) so[i] = Sold[(long long)i * g.Sp + g.frame_n + t];
    }
#pragma unroll
    for (int i = 0; i < S::Q; ++i) {
      const Real neq = p[i] - eq_dir<S, Real, DEV>(i, m, kf, c);
      const Real eqt = eq_dir<S, Real, DEV>(i, mt, kt, c);
      B[(long long)i * g.plane + dst] = eqt + keep * neq;
      if (Sold) {
        const long long k = (long long)i * g.Sp + g.frame_n + t;
        const Real s0 = kHoist ? so[i] : Sold[k], fh = eqt - c.eqbar[i];
        Snew[k] = s0 + fh;
        Sold[k] = s0 + Real(0.5) * fh;   // Q^n in place, gathered by the frame's phase 2
      }
    }
    return;
  }
  if (Sold) {
    const EqCoef<Real> kf = eq_coef<S::ORDER, Real>(m);
    constexpr bool kHoist = sizeof(Real) == 4;   // as above
    Real so[S::Q];
    if (kHoist) {
#pragma unroll
      for (int i = 0; i < S::Q; ++i) so[i] = Sold[(long long)i * g.Sp + g.frame_n + t];
    }
#pragma unroll
    for (int i = 0; i < S::Q; ++i) {
      const long long k = (long long)i * g.Sp + g.frame_n + t;
      const Real s0 = kHoist ? so[i] : Sold[k];
      const Real fh = eq_dir<S, Real, DEV>(i, m, kf, c) - c.eqbar[i];
      Snew[k] = s0 + fh;
      Sold[k] = s0 + Real(0.5) * fh;   // Q^n in place, gathered by the frame's phase 2
    }
  }
  collide_bgk<S, Real, DEV>(p, m, c);
#pragma unroll
  for (int i = 0; i < S::Q; ++i) B[(long long)i * g.plane + dst] = p[i];
}

template <class S, class Real, bool DEV, bool STREAM>
__global__ void __launch_bounds__(128) k_gamma(Geom g, Consts<Real> c, BcParams bc,
                                               const Real* __restrict__ A, Real* __restrict__ B,
                                               const double* __restrict__ Vtgt,
                                               Real* __restrict__ Sold,
                                               Real* __restrict__ Snew) {
  gamma_node<S, Real, DEV, STREAM>(g, c, bc, A, B, Vtgt, Sold, Snew,
                                   blockIdx.x * blockDim.x + threadIdx.x);
}

// Periodic y axis: the M rows below y = 0 and above y = Ly - 1 (boundary columns included)
// take the post-collision populations of the rows they image, PML term included, once every
// other kernel of the step has written B. Thread = (direction, row pair j, column).
template <class Real>
__device__ __forceinline__ void wrap_y_elem(const Geom& g, Real* __restrict__ B, long long t,
                                            int dir) {
  const int Gx = g.Lx + 2 * g.M;
  const long long n = (long long)Gx * g.M;
  if (t >= n) return;
  const int j = int(t / Gx) + 1, x = int(t % Gx) - g.M;
  Real* plane = B + (long long)dir * g.plane;
  plane[gindex(g, x, -j)] = plane[gindex(g, x, g.Ly - j)];
  plane[gindex(g, x, g.Ly - 1 + j)] = plane[gindex(g, x, j - 1)];
}

template <class Real>
__global__ void __launch_bounds__(256) k_wrap_y(Geom g, Real* __restrict__ B) {
  wrap_y_elem<Real>(g, B, (long long)blockIdx.x * blockDim.x + threadIdx.x, blockIdx.y);
}

// ------------------------------------------------------------------------------------------
// Characteristic targets (Sec. 4): one Runge-Kutta stage for every edge-band node.
// ------------------------------------------------------------------------------------------
template <class R>
struct PrimT { R rho, un, ut, T; };
using Prim = PrimT<double>;

// Inverse of the characteristic map: given w = S dU (acoustic-, entropy, shear, acoustic+),
// return dU = S^-1 w in (rho, u_n, u_t, T). With P = rho T (c_s = 1), c^2 = 2 T (gamma = 2):
// dP = (w1 + w4)/2, du_n = (w4 - w1)/(2 rho c), du_t = w3, drho = (dP + w2)/c^2,
// dT = (dP - T drho)/rho.
template <class R>
__device__ inline PrimT<R> char_inverse(const PrimT<R>& U, R c, const R w[4]) {
  PrimT<R> d;
  const R dP = R(0.5) * (w[0] + w[3]);
  d.un = (w[3] - w[0]) / (R(2) * U.rho * c);
  d.ut = w[2];
  d.rho = (dP + w[1]) / (c * c);
  d.T = (dP - U.T * d.rho) / U.rho;
  return d;
}

// w = S dU for the normal axis: w1 = T drho - rho c du_n + rho dT, w2 = T drho - rho dT,
// w3 = du_t, w4 = T drho + rho c du_n + rho dT (left eigenvectors of the Euler Jacobian).
template <class R>
__device__ inline void char_forward(const PrimT<R>& U, R c, const PrimT<R>& dU, R w[4]) {
  const R dP = U.T * dU.rho + U.rho * dU.T;
  w[0] = dP - U.rho * c * dU.un;
  w[1] = U.T * dU.rho - U.rho * dU.T;
  w[2] = dU.ut;
  w[3] = dP + U.rho * c * dU.un;
}

__device__ inline Prim load_prim(const double* V, int stride, int slot, bool xaxis) {
  Prim u;
  u.rho = V[slot];
  const double ux = V[stride + slot], uy = V[2 * stride + slot];
  u.un = xaxis ? ux : uy;
  u.ut = xaxis ? uy : ux;
  u.T = V[3 * stride + slot];
  return u;
}

template <class R>
__device__ inline PrimT<R> to(const Prim& p) {
  return PrimT<R>{R(p.rho), R(p.un), R(p.ut), R(p.T)};
}



}  // namespace lbm

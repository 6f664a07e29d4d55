// Single-pass PML frame kernel (FP32 deviation storage): one block per tile of the frame
// (P + inner ring: the outer Fw / Fe / Fs / Fn layers of F) with a 2-node halo.
//
//  A  every owned node and every halo node phase C reads that carries Q (distance <= W along
//     a PML axis) pulls its populations and takes its moments; the latter store
//     Q_i = S_i^(n-1) + f_hat_i^n / 2 for all i in shared memory (trapezoidal accumulator,
//     Eq. PMLQ; f_hat = f_eq - f_eq_bar, Eq. decomp-NJ);
//  C  every owned node pulls again (cache hits), collides with BGK (moments kept from A),
//     adds on P the PML term of Eq. (pml-general) (Eq. PMLCOLL when sigma_x = sigma_y) with
//     grad Q from shared memory
//     (Eq. FD-dx-center; Eq. FD-dx-bw along the outward normal on the outermost layer; the
//     2-node halo covers both), writes the post-collision populations and
//     S^n = S^(n-1) + f_hat^n.
//
// Tiles: the bottom and top bands (Fs / Fn rows, full width) use 32-wide tiles whose height
// splits the band depth evenly; the left and right bands (Fw / Fe columns of the middle rows)
// use tiles whose width splits the band depth evenly.
#pragma once
#include "lbm_device.cuh"

namespace lbm {

struct BandTiles {
  int tw, th;        // tile size
  int cols, rows;    // tiles across / along the band
  int n;             // cols * rows
};

struct FrameTiles {
  BandTiles b[4];    // bottom, top, left, right
  int ext_max;       // largest (tw + 4) (th + 4)
};

inline BandTiles row_band(int depth, int Lx) {
  BandTiles t{};
  t.tw = 32;
  t.rows = (depth + 7) / 8;
  t.th = t.rows > 0 ? (depth + t.rows - 1) / t.rows : 1;
  t.cols = (Lx + 31) / 32;
  t.n = t.rows * t.cols;
  return t;
}

inline BandTiles column_band(int depth, int height, int threads) {
  BandTiles t{};
  t.cols = (depth + 31) / 32;
  t.tw = (depth + t.cols - 1) / t.cols;
  t.th = threads / t.tw;
  if (t.th > 32) t.th = 32;
  t.rows = (height + t.th - 1) / t.th;
  t.n = t.rows * t.cols;
  return t;
}

inline FrameTiles make_frame_tiles(const Geom& g, int threads) {
  FrameTiles t{};
  const int mid = g.Ly - g.Fs - g.Fn;
  t.b[0] = row_band(g.Fs, g.Lx);
  t.b[1] = row_band(g.Fn, g.Lx);
  t.b[2] = column_band(g.Fw, mid, threads);
  t.b[3] = column_band(g.Fe, mid, threads);
  t.ext_max = 0;
  for (int k = 0; k < 4; ++k) {
    const int e = (t.b[k].tw + 4) * (t.b[k].th + 4);
    if (t.b[k].n > 0 && e > t.ext_max) t.ext_max = e;
  }
  return t;
}

inline int frame_tile_count(const FrameTiles& t) { return t.b[0].n + t.b[1].n + t.b[2].n + t.b[3].n; }

// shared memory of k_pml_fused: Q on the extended tile and the moments of the owned nodes
template <class S>
inline size_t pml_fused_smem(const FrameTiles& ft) {
  return sizeof(float) * ((size_t)S::Q * ft.ext_max + 7 * 256);
}

// One frame tile (tile = index over the four bands' tiles) on one block; smem holds
// pml_fused_smem bytes. Shared with the batched launch over many instances.
template <class S, bool STREAM>
__device__ __forceinline__ void pml_fused_tile(const Geom& g, const Consts<float>& c,
                                               const FrameTiles& ft,
                                               const float* __restrict__ A,
                                               float* __restrict__ B,
                                               const float* __restrict__ Sold,
                                               float* __restrict__ Snew, double* Uedge,
                                               int save_edges, int* flag, double* Sedge,
                                               int src_mask, int tile, float* smem) {
  // ---- tile of this block
  int x0, y0, tw, th, band;  // band 0 bottom, 1 top, 2 left, 3 right
  {
    int k = tile;
    band = 0;
    while (band < 3 && k >= ft.b[band].n) k -= ft.b[band++].n;
    const BandTiles& bt = ft.b[band];
    const int r = k / bt.cols, cc = k - r * bt.cols;
    tw = bt.tw;
    th = bt.th;
    if (band == 0) { x0 = cc * tw; y0 = r * th; }
    else if (band == 1) { x0 = cc * tw; y0 = g.Ly - g.Fn + r * th; }
    else if (band == 2) { x0 = cc * tw; y0 = g.Fs + r * th; }
    else { x0 = g.Lx - g.Fe + cc * tw; y0 = g.Fs + r * th; }
  }
  const int ew = tw + 4, eh = th + 4, next = ew * eh;
  const int nown = tw * th;
  float* Qs = smem;                       // [Q][next]   Q = S^(n-1) + f_hat / 2
  float* Mc = Qs + S::Q * ft.ext_max;     // [7][256]    moments of the owned nodes
  const int tid = threadIdx.x;

  // ---- A: Q on tile + halo; equilibria and moments of the owned nodes kept for phase C
  for (int e = tid; e < next; e += blockDim.x) {
    const int ex = e % ew, ey = e / ew;
    const int tx = ex - 2, ty = ey - 2;
    // halo nodes phase C never reads: the corners (the differences are per axis), and the
    // second halo column / row unless the tile's edge column / row is an outermost layer of F
    // whose one-sided stencil (Eq. FD-dx-bw) reaches two nodes inward
    const bool xin = tx >= 0 && tx < tw, yin = ty >= 0 && ty < th;
    if (!xin && !yin) continue;
    if (tx == -2 && x0 != g.Lx - 1) continue;
    if (tx == tw + 1 && x0 + tw - 1 != 0) continue;
    if (ty == -2 && (g.py || y0 != g.Ly - 1)) continue;
    if (ty == th + 1 && (g.py || y0 + th - 1 != 0)) continue;
    const int x = x0 - 2 + ex;
    int y = y0 - 2 + ey;
    if (g.py) y = (y + g.Ly) % g.Ly;   // halo rows wrap along a periodic y axis
    if (x < 0 || y < 0 || x >= g.Lx || y >= g.Ly) continue;
    const int own = (xin && yin) ? ty * tw + tx : -1;
    // frame nodes farther out than the PML along neither axis (a frame depth set by M
    // where an axis has no PML) still need their moments for phase C
    const bool hq = pml_node<float>(g, x, y).has_q;
    if (!hq && own < 0) continue;
    float p[S::Q];
    load_pop<S, float, STREAM>(p, A, g, gindex(g, x, y));
    const Macro<float> m = moments<S, float, true>(p, c);
    if (own >= 0) {
      Mc[0 * 256 + own] = m.rho;
      Mc[1 * 256 + own] = m.drho;
      Mc[2 * 256 + own] = m.inv_rho;
      Mc[3 * 256 + own] = m.urx;
      Mc[4 * 256 + own] = m.ury;
      Mc[5 * 256 + own] = m.u2;
      Mc[6 * 256 + own] = m.theta;
    }
    if (!hq) continue;
    const EqCoef<float> kc = eq_coef<S::ORDER, float>(m);
    const int fi = frame_index(g, x, y);
#pragma unroll
    for (int i = 0; i < S::Q; ++i) {
      const float eq = eq_dir<S, float, true>(i, m, kc, c);
      Qs[i * next + e] = __ldg(Sold + (long long)i * g.Sp + fi) + 0.5f * (eq - c.eqbar[i]);
    }
  }
  __syncthreads();

  // ---- C: owned nodes
  if (tid >= nown) return;
  const int tx = tid % tw, ty = tid / tw;
  const int x = x0 + tx, y = y0 + ty;
  if (x >= g.Lx || y >= g.Ly) return;
  bool owned;
  if (band == 0) owned = y < g.Fs;
  else if (band == 1) owned = y >= g.Ly - g.Fn;
  else if (band == 2) owned = x < g.Fw && y < g.Ly - g.Fn;
  else owned = y < g.Ly - g.Fn;
  if (!owned) return;
  const int d = dist_out(g, x, y);
  const long long idx = gindex(g, x, y);
  float p[S::Q];
  load_pop<S, float, STREAM>(p, A, g, idx);
  Macro<float> m;
  m.rho = Mc[0 * 256 + tid];
  m.drho = Mc[1 * 256 + tid];
  m.inv_rho = Mc[2 * 256 + tid];
  m.urx = Mc[3 * 256 + tid];
  m.ury = Mc[4 * 256 + tid];
  m.u2 = Mc[5 * 256 + tid];
  m.theta = Mc[6 * 256 + tid];
  if (unphysical(m)) *flag = 1;
  if (save_edges && d < 2) save_edge_moments(g, Uedge, x, y, m, c.r);
  const EqCoef<float> kc = eq_coef<S::ORDER, float>(m);
  const int fi = frame_index(g, x, y);
  const int e0 = (ty + 2) * ew + (tx + 2);
  const PmlNode<float> pn = pml_node<float>(g, x, y);
  const bool in_p = pn.in_p;
  float sx = 0.f, sy = 0.f;
  if (in_p) pml_sigmas(c, pn, sx, sy);
  const float ssum = sx + sy, sprod = sx * sy;
  // gradient stencils on the shared-memory tile (offsets in extended-tile units)
  float cx0 = 0.5f, cx1 = -0.5f, cx2 = 0.f, cy0 = 0.5f, cy1 = -0.5f, cy2 = 0.f;
  int ox0 = 1, ox1 = -1, ox2 = 0, oy0 = ew, oy1 = -ew, oy2 = 0;
  if (x == 0) { cx0 = -1.5f; cx1 = 2.f; cx2 = -0.5f; ox0 = 0; ox1 = 1; ox2 = 2; }
  else if (x == g.Lx - 1) { cx0 = 1.5f; cx1 = -2.f; cx2 = 0.5f; ox0 = 0; ox1 = -1; ox2 = -2; }
  if (!g.py && y == 0) { cy0 = -1.5f; cy1 = 2.f; cy2 = -0.5f; oy0 = 0; oy1 = ew; oy2 = 2 * ew; }
  else if (!g.py && y == g.Ly - 1) {
    cy0 = 1.5f; cy1 = -2.f; cy2 = 0.5f; oy0 = 0; oy1 = -ew; oy2 = -2 * ew;
  }
  // Appendix PML source at the outermost layer: moments of the selected parts of Omega^PML
  const bool src = src_mask && outermost(g, x, y);
  float smom[4] = {0.f, 0.f, 0.f, 0.f};
#pragma unroll
  for (int i = 0; i < S::Q; ++i) {
    const float eq = eq_dir<S, float, true>(i, m, kc, c);
    const float fhat = eq - c.eqbar[i];
    const float* q = Qs + i * next + e0;
    const float qn = q[0];
    Snew[(long long)i * g.Sp + fi] = __ldg(Sold + (long long)i * g.Sp + fi) + fhat;  // S^n
    float out = p[i] + c.omega * (eq - p[i]);
    if (in_p) {
      float gq = 0.f;   // sigma_y c_x dQ/dx + sigma_x c_y dQ/dy
      if (S::ex(i) != 0) gq += sy * float(S::ex(i)) * (cx0 * q[ox0] + cx1 * q[ox1] + cx2 * q[ox2]);
      if (S::ey(i) != 0) gq += sx * float(S::ey(i)) * (cy0 * q[oy0] + cy1 * q[oy1] + cy2 * q[oy2]);
      out = out - (gq + ssum * fhat + sprod * qn);
      if (src) {
        const float part = -(((src_mask & 1) ? gq : 0.f) + ((src_mask & 2) ? ssum * fhat : 0.f) +
                             ((src_mask & 4) ? sprod * qn : 0.f));
        smom[0] += part;
        smom[1] += float(S::ex(i)) * part;
        smom[2] += float(S::ey(i)) * part;
        smom[3] += float(S::ex(i) * S::ex(i) + S::ey(i) * S::ey(i)) * part;
      }
    }
    B[(long long)i * g.plane + idx] = out;
  }
  if (src) {
    smom[1] *= c.r;
    smom[2] *= c.r;
    smom[3] *= 0.5f * c.r2;
    put_pml_source(g, Sedge, x, y, smom, false);
  }
}

template <class S, bool STREAM>
__global__ void __launch_bounds__(256) k_pml_fused(Geom g, Consts<float> c, FrameTiles ft,
                                                   const float* __restrict__ A,
                                                   float* __restrict__ B,
                                                   const float* __restrict__ Sold,
                                                   float* __restrict__ Snew, double* Uedge,
                                                   int save_edges, int* flag, double* Sedge,
                                                   int src_mask) {
  extern __shared__ float smem[];
  pml_fused_tile<S, STREAM>(g, c, ft, A, B, Sold, Snew, Uedge, save_edges, flag, Sedge, src_mask,
                            blockIdx.x, smem);
}

}  // namespace lbm

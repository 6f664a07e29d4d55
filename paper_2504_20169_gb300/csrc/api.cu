// C ABI of liblbm (include/lbm.h): context management, validation, the quadrature of Sec. 2,
// and the host-side sequencing of the kernels.
#include <cmath>
#include <mutex>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <string>
#include <vector>

#include "../../include/lbm.h"
#include "lbm_internal.h"

using namespace lbm;

namespace {

thread_local std::string g_create_error;

// --------------------------------------------------------------------------------------------
// Gauss-Hermite rule of a stencil (Sec. 2): one weight per velocity shell and the scale r of
// xi_i = r e_i such that sum_i w_i xi_x^p xi_y^q equals the unit-Gaussian moment
// (p-1)!!(q-1)!! for every even pair p >= q with p + q below the quadrature degree. Solved by
// Newton's method on the square system in (weights, r), started from a least-squares fit.
// --------------------------------------------------------------------------------------------
long double odd_df(int n) {
  long double v = 1;
  for (int k = n - 1; k > 0; k -= 2) v *= k;
  return v;
}

bool solve_linear(std::vector<long double>& A, std::vector<long double>& b, int n) {
  for (int c = 0; c < n; ++c) {
    int piv = c;
    for (int r = c + 1; r < n; ++r)
      if (std::fabs((double)A[r * n + c]) > std::fabs((double)A[piv * n + c])) piv = r;
    if (A[piv * n + c] == 0) return false;
    if (piv != c) {
      for (int k = 0; k < n; ++k) std::swap(A[c * n + k], A[piv * n + k]);
      std::swap(b[c], b[piv]);
    }
    for (int r = c + 1; r < n; ++r) {
      const long double f = A[r * n + c] / A[c * n + c];
      for (int k = c; k < n; ++k) A[r * n + k] -= f * A[c * n + k];
      b[r] -= f * b[c];
    }
  }
  for (int c = n - 1; c >= 0; --c) {
    long double s = b[c];
    for (int k = c + 1; k < n; ++k) s -= A[c * n + k] * b[k];
    b[c] = s / A[c * n + c];
  }
  return true;
}

template <class S>
bool derive_quadrature(int degree, double r0, double* w_dir, double* r_out, std::string& err) {
  const int ns = S::NSHELL;
  std::vector<int> cp, cq;
  for (int s = 0; s < degree; s += 2)
    for (int p = s; p >= 0; --p) {
      const int q = s - p;
      if (p % 2 == 0 && q % 2 == 0 && p >= q) { cp.push_back(p); cq.push_back(q); }
    }
  const int ne = (int)cp.size();
  if (ne != ns + 1) { err = "quadrature: condition count mismatch"; return false; }
  // lattice moments of every shell: m[k][s] = sum over members of ex^p ey^q
  std::vector<long double> m(ne * ns, 0);
  for (int k = 0; k < ne; ++k)
    for (int s = 0; s < ns; ++s)
      for (int i = S::shell_first(s); i < S::shell_first(s) + S::shell_size(s); ++i)
        m[k * ns + s] += std::pow((long double)S::ex(i), cp[k]) * std::pow((long double)S::ey(i), cq[k]);
  std::vector<long double> rhs(ne);
  for (int k = 0; k < ne; ++k) rhs[k] = odd_df(cp[k]) * odd_df(cq[k]);
  auto mat = [&](long double r, std::vector<long double>& A) {
    A.assign(ne * ns, 0);
    for (int k = 0; k < ne; ++k)
      for (int s = 0; s < ns; ++s) A[k * ns + s] = std::pow(r, cp[k] + cq[k]) * m[k * ns + s];
  };
  // least-squares start at r0
  std::vector<long double> A, N(ns * ns, 0), y(ns, 0);
  long double r = r0;
  mat(r, A);
  for (int a = 0; a < ns; ++a) {
    for (int b = 0; b < ns; ++b)
      for (int k = 0; k < ne; ++k) N[a * ns + b] += A[k * ns + a] * A[k * ns + b];
    for (int k = 0; k < ne; ++k) y[a] += A[k * ns + a] * rhs[k];
  }
  if (!solve_linear(N, y, ns)) { err = "quadrature: singular start"; return false; }
  std::vector<long double> W = y;
  const int n = ns + 1;
  for (int it = 0; it < 100; ++it) {
    std::vector<long double> J(n * n, 0), F(n, 0);
    mat(r, A);
    for (int k = 0; k < ne; ++k) {
      long double s = 0, sd = 0;
      for (int j = 0; j < ns; ++j) {
        s += A[k * ns + j] * W[j];
        J[k * n + j] = A[k * ns + j];
        sd += (long double)(cp[k] + cq[k]) * std::pow(r, cp[k] + cq[k] - 1) * m[k * ns + j] * W[j];
      }
      J[k * n + ns] = (cp[k] + cq[k]) > 0 ? sd : 0;
      F[k] = -(s - rhs[k]);
    }
    if (!solve_linear(J, F, n)) { err = "quadrature: singular Newton step"; return false; }
    long double step = 0;
    for (int j = 0; j < ns; ++j) { W[j] += F[j]; step = std::max(step, std::fabs(F[j])); }
    r += F[ns];
    step = std::max(step, std::fabs(F[ns]));
    if (step < 1e-17L) break;
  }
  mat(r, A);
  double worst = 0;
  for (int k = 0; k < ne; ++k) {
    long double s = 0;
    for (int j = 0; j < ns; ++j) s += A[k * ns + j] * W[j];
    worst = std::max(worst, (double)std::fabs(s - rhs[k]));
  }
  for (int j = 0; j < ns; ++j)
    if (!(W[j] > 0)) { err = "quadrature: negative weight"; return false; }
  if (!(worst < 1e-11)) { err = "quadrature: Newton did not converge"; return false; }
  for (int s = 0; s < ns; ++s)
    for (int i = S::shell_first(s); i < S::shell_first(s) + S::shell_size(s); ++i)
      w_dir[i] = (double)W[s];
  *r_out = (double)r;
  return true;
}

bool lattice_of(int q, double* w, double* r, std::string& err) {
  switch (q) {
    case 37: return derive_quadrature<D2Q37>(9, 1.2, w, r, err);
    case 17: return derive_quadrature<D2Q17>(7, 1.64, w, r, err);
    case 9: return derive_quadrature<D2Q9>(5, 1.73, w, r, err);
  }
  err = "unknown stencil";
  return false;
}

template <class S>
void velocities(int* e) {
  for (int i = 0; i < S::Q; ++i) { e[2 * i] = S::ex(i); e[2 * i + 1] = S::ey(i); }
}

template <class S>
void mean_equilibrium(const double* w, double r, const lbm_bc_params& bp, double* out) {
  Consts<double> c{};
  for (int i = 0; i < S::Q; ++i) c.w[i] = w[i];
  c.r = r;
  c.r2 = r * r;
  Macro<double> m;
  m.rho = bp.rho0;
  m.drho = bp.rho0 - 1.0;
  m.inv_rho = 1.0 / bp.rho0;
  m.urx = r * bp.u0x;
  m.ury = r * bp.u0y;
  m.u2 = bp.u0x * bp.u0x + bp.u0y * bp.u0y;
  m.theta = bp.T0 - 1.0;
  const EqCoef<double> k = eq_coef<S::ORDER, double>(m);
  for (int i = 0; i < S::Q; ++i) out[i] = eq_dir<S, double, false>(i, m, k, c);
}

int halo_of(int q) { return q == 9 ? 1 : 3; }

}  // namespace

void lbm::set_global_error(const std::string& msg) { g_create_error = msg; }

// --------------------------------------------------------------------------------------------
struct lbm_ctx {
  int q = 0;
  lbm_precision prec = LBM_FP64;
  lbm_bc_kind bc = LBM_BC_ZG;
  int device = 0;
  Geom g{};
  OpsTable ops{};
  Dev dev{};
  double w[kMaxQ]{}, r = 0, tau = 0, omega = 0;
  cudaStream_t st = nullptr;
  void* f[2] = {nullptr, nullptr};
  void* S[2] = {nullptr, nullptr};
  double* V = nullptr;        // 4 arrays of [4][nb]: targets, stage a, stage b, accumulator
  double* Uedge = nullptr;    // two buffers of [4][ne] (ping-pong with the populations)
  double* Sedge = nullptr;    // two buffers of [4][2 (Lx + Ly)]: Appendix PML source
  double* staging = nullptr;  // [4][Lx*Ly]
  double* partials = nullptr;
  int max_blocks = 0;
  double* dout = nullptr;
  double* hout = nullptr;     // pinned
  int* hflag = nullptr;       // mapped pinned
  int* dflag = nullptr;
  size_t fbytes = 0, sbytes = 0;
  int cur = 0, scur = 0;
  bool initialized = false, prev_valid = false, prev_prestream = false;
  long long steps = 0;
  cudaStream_t aux = nullptr, aux2 = nullptr, cap = nullptr;  // boundary streams, capture
  cudaEvent_t fork = nullptr, join = nullptr, join2 = nullptr, ready = nullptr;
  cudaGraphExec_t graph[2] = {nullptr, nullptr};  // one step, keyed by the buffer parity
  cudaGraph_t gtemplate[2] = {nullptr, nullptr};  // the captured graphs (child graphs of batches)
  bool use_graphs = true;
  std::vector<cudaEvent_t> prof;   // kKernelClasses * 2 events per recorded step
  int prof_cap = 0, prof_used = 0;
  // device buffers: base pointer (guard band of kGuard bytes on both sides) and payload size
  BatchPlan plan{};           // one-member plan: the table-driven boundary-side launches
  std::vector<std::pair<char*, size_t>> allocs;
  size_t alloc_total = 0, alloc_budget = 0;  // budget 0: unlimited (test hook, see lbm.h)
  std::string err;
};

// Every device buffer of a context sits between two guard bands of kGuard bytes filled with
// kGuardByte; lbm_debug_check_guards reports whether any kernel wrote into them.
static const size_t kGuard = 256;
static const int kGuardByte = 0xA5;

static cudaError_t dalloc(lbm_ctx* ctx, void** p, size_t bytes) {
  *p = nullptr;
  if (ctx->alloc_budget && ctx->alloc_total + bytes > ctx->alloc_budget)
    return cudaErrorMemoryAllocation;
  char* base = nullptr;
  cudaError_t e = cudaMalloc((void**)&base, bytes + 2 * kGuard);
  if (e != cudaSuccess) return e;
  ctx->allocs.push_back({base, bytes});
  ctx->alloc_total += bytes;
  // on the context's stream: creating a context does not wait for other streams' work
  if ((e = cudaMemsetAsync(base, kGuardByte, kGuard, ctx->st)) != cudaSuccess) return e;
  if ((e = cudaMemsetAsync(base + kGuard + bytes, kGuardByte, kGuard, ctx->st)) != cudaSuccess)
    return e;
  *p = base + kGuard;
  return cudaSuccess;
}

#define LBM_CK(call)                                                          \
  do {                                                                        \
    cudaError_t e_ = (call);                                                  \
    if (e_ != cudaSuccess) {                                                  \
      ctx->err = std::string(#call) + ": " + cudaGetErrorString(e_);          \
      return LBM_ECUDA;                                                       \
    }                                                                         \
  } while (0)

static void free_all(lbm_ctx* ctx) {
  if (!ctx) return;
  cudaSetDevice(ctx->device);
  if (ctx->st) cudaStreamSynchronize(ctx->st); else cudaDeviceSynchronize();
  for (cudaEvent_t e : ctx->prof) cudaEventDestroy(e);
  ctx->prof.clear();
  for (int k = 0; k < 2; ++k) {
    if (ctx->graph[k]) cudaGraphExecDestroy(ctx->graph[k]);
    if (ctx->gtemplate[k]) cudaGraphDestroy(ctx->gtemplate[k]);
  }
  if (ctx->aux) cudaStreamDestroy(ctx->aux);
  if (ctx->aux2) cudaStreamDestroy(ctx->aux2);
  if (ctx->cap) cudaStreamDestroy(ctx->cap);
  if (ctx->fork) cudaEventDestroy(ctx->fork);
  if (ctx->join) cudaEventDestroy(ctx->join);
  if (ctx->join2) cudaEventDestroy(ctx->join2);
  if (ctx->ready) cudaEventDestroy(ctx->ready);
  batch_plan_free(&ctx->plan);
  for (auto& a : ctx->allocs) cudaFree(a.first);
  ctx->allocs.clear();
  if (ctx->hout) cudaFreeHost(ctx->hout);
  if (ctx->hflag) cudaFreeHost(ctx->hflag);
}

static size_t edge_slots(const Geom& g) { return 4 * (size_t)g.ne; }
static size_t source_slots(const Geom& g) { return 4 * 2 * ((size_t)g.Lx + g.Ly); }

static void set_roles(lbm_ctx* ctx, int a, int s) {
  Dev& d = ctx->dev;
  d.which = a;
  d.A = ctx->f[a];
  d.B = ctx->f[1 - a];
  d.Sold = ctx->S[s];
  d.Snew = ctx->S[1 - s];
  d.Uedge_in = ctx->Uedge + a * edge_slots(ctx->g);
  d.Uedge_out = ctx->Uedge + (1 - a) * edge_slots(ctx->g);
  d.Sedge_in = ctx->Sedge + a * source_slots(ctx->g);
  d.Sedge_out = ctx->Sedge + (1 - a) * source_slots(ctx->g);
}

static lbm_status check_ready(lbm_ctx* ctx) {
  if (!ctx) return LBM_EINVAL;
  if (!ctx->initialized) { ctx->err = "context not initialized"; return LBM_ESTATE; }
  if (cudaSetDevice(ctx->device) != cudaSuccess) { ctx->err = "cudaSetDevice failed"; return LBM_ECUDA; }
  return LBM_OK;
}

extern "C" {

lbm_status lbm_lattice_info(lbm_stencil stencil, int* q, int* e, double* w, double* r) {
  double ww[kMaxQ], rr;
  std::string err;
  if (!lattice_of((int)stencil, ww, &rr, err)) { g_create_error = err; return LBM_EINVAL; }
  const int qq = (int)stencil;
  if (q) *q = qq;
  if (w) std::memcpy(w, ww, sizeof(double) * qq);
  if (r) *r = rr;
  if (e) {
    if (qq == 37) velocities<D2Q37>(e);
    else if (qq == 17) velocities<D2Q17>(e);
    else velocities<D2Q9>(e);
  }
  return LBM_OK;
}

// Storage geometry of a grid (section "Storage" of lbm_device.cuh) and the bytes it needs.
static Geom make_geom(int nx, int ny, const int W[4], int M, int py, int link) {
  Geom g{};
  g.nx = nx;
  g.ny = ny;
  g.Ww = W[0];
  g.We = W[1];
  g.Ws = W[2];
  g.Wn = W[3];
  g.py = py;
  g.M = M;
  g.Lx = nx + g.Ww + g.We;
  g.Ly = ny + g.Ws + g.Wn;
  g.cF0 = 32;
  g.pitch = ((g.cF0 + g.Lx + g.M) + 31) / 32 * 32;
  g.plane = ((long long)g.pitch * (g.Ly + 2 * g.M) + 63) / 64 * 64;
  // the frame holds the PML and its inner ring (1 node for the printed central difference, M
  // for the link difference), and at least the two outer layers whose moments the
  // characteristic targets read (so also for D2Q9, M = 1)
  g.link = link;
  g.qr = link ? M : 1;
  auto depth = [&](int w) { return std::max(w > 0 ? w + g.qr : 0, std::max(g.M, 2)); };
  g.Fw = depth(g.Ww);
  g.Fe = depth(g.We);
  g.Fs = py ? 0 : depth(g.Ws);
  g.Fn = py ? 0 : depth(g.Wn);
  g.frame_n = (g.Fs + g.Fn) * g.Lx + (g.Ly - g.Fs - g.Fn) * (g.Fw + g.Fe);
  g.nb = 2 * g.M * (g.Lx + g.Ly);
  g.ne = 4 * (g.Lx + g.Ly);
  g.ngamma = 2 * g.M * (g.Lx + 2 * g.M) + 2 * g.M * g.Ly;
  // accumulator slots: the frame, then (link mode) the boundary nodes outside F
  g.Sp = has_pml(g) ? ((long long)g.frame_n + (link ? g.ngamma : 0) + 31) / 32 * 32 : 0;
  return g;
}

static size_t bytes_of(const Geom& g, int q, int es) {
  const size_t max_blocks = (size_t)((g.Lx + 31) / 32) * ((g.Ly + 7) / 8);
  return 2 * (size_t)q * g.plane * es + 2 * (size_t)q * g.Sp * es +
         sizeof(double) * (16 * (size_t)g.nb + 2 * edge_slots(g) + 2 * source_slots(g) +
                           4 * (size_t)g.Lx * g.Ly +
                           12 * max_blocks + 16) +
         10 * 2 * kGuard;   // guard bands of the (at most ten) device buffers
}

extern "C" lbm_status lbm_estimate_bytes(const lbm_grid* grid, lbm_stencil stencil, int pml_width,
                                         lbm_bc_kind bc, lbm_precision precision, size_t* bytes) {
  if (!grid || !bytes) return LBM_EINVAL;
  const int q = (int)stencil;
  if ((q != 37 && q != 17 && q != 9) || grid->nx < 8 || grid->ny < 8 || pml_width < 0 ||
      pml_width == 1 || (bc == LBM_BC_PERIODIC && pml_width != 0) ||
      (precision != LBM_FP64 && precision != LBM_FP32_DEV))
    return LBM_EINVAL;
  const int W4[4] = {pml_width, pml_width, pml_width, pml_width};
  const Geom g = make_geom(grid->nx, grid->ny, W4, halo_of(q), 0, 0);
  *bytes = bytes_of(g, q, precision == LBM_FP64 ? 8 : 4);
  return LBM_OK;
}

// Argument checks of lbm_create (shared with lbm_estimate_bytes_bc): the resolved sigma
// profile, boundary parameters and per-edge PML widths, or LBM_EINVAL with the reason.
static lbm_status check_args(const lbm_grid* grid, lbm_stencil stencil, double tau, int pml_width,
                             const lbm_sigma_profile* sigma, lbm_bc_kind bc,
                             const lbm_bc_params* bcp, lbm_precision precision,
                             lbm_sigma_profile& sg, lbm_bc_params& bp, int W4[4]) {
  auto fail = [](const char* m) { g_create_error = m; return LBM_EINVAL; };
  if (!grid) return fail("grid is NULL");
  const int q = (int)stencil;
  if (q != 37 && q != 17 && q != 9) return fail("stencil must be 9, 17 or 37");
  if (grid->nx < 8 || grid->ny < 8) return fail("bulk must be at least 8 x 8");
  if (!(tau > 0.5)) return fail("tau must exceed 1/2");
  if (pml_width < 0 || pml_width == 1 || pml_width > 4096)
    return fail("pml_width must be 0 or 2..4096");
  if (bc != LBM_BC_PERIODIC && bc != LBM_BC_ZG && bc != LBM_BC_NRBC) return fail("bad bc kind");
  if (precision != LBM_FP64 && precision != LBM_FP32_DEV) return fail("bad precision");
  sg = sigma ? *sigma : lbm_sigma_profile{0.0, 2, 0};
  if (!(sg.sigma_max >= 0.0) || !std::isfinite(sg.sigma_max) || sg.power < 0 || sg.power > 16 ||
      (sg.split != 0 && sg.split != 1))
    return fail("bad sigma profile");
  if (bcp) bp = *bcp;
  else { std::memset(&bp, 0, sizeof bp); bp.rho0 = 1.0; bp.T0 = 1.0; }
  if (bp.periodic_y != 0 && bp.periodic_y != 1) return fail("periodic_y must be 0 or 1");
  if (bp.use_pml_widths != 0 && bp.use_pml_widths != 1) return fail("use_pml_widths must be 0 or 1");
  for (int k = 0; k < 4; ++k) W4[k] = bp.use_pml_widths ? bp.pml_widths[k] : pml_width;
  if (bp.periodic_y && !bp.use_pml_widths) W4[2] = W4[3] = 0;
  for (int k = 0; k < 4; ++k)
    if (W4[k] < 0 || W4[k] == 1 || W4[k] > 4096) return fail("PML widths must be 0 or 2..4096");
  if (bc == LBM_BC_PERIODIC && (W4[0] | W4[1] | W4[2] | W4[3]))
    return fail("periodic mode has no PML");
  if (bp.periodic_y && (W4[2] || W4[3])) return fail("a periodic y axis has no PML");
  if (bp.periodic_y && bc == LBM_BC_PERIODIC) return fail("periodic_y needs a ZG or NRBC x edge");
  if (bp.pml_source < 0 || bp.pml_source > 15) return fail("pml_source is a bitmask of 1, 2, 4, 8");
  if (bp.pml_grad != 0 && bp.pml_grad != 1) return fail("pml_grad must be 0 or 1");
  if (bp.pml_grad == 1 && sg.split) return fail("the link gradient needs sigma_x = sigma_y");
  if (!(bp.rho0 > 0) || !(bp.T0 > 0) || !std::isfinite(bp.u0x) || !std::isfinite(bp.u0y) ||
      !std::isfinite(bp.beta))
    return fail("bad mean state or beta");
  for (int k = 0; k < 4; ++k)
    if (bp.edge[k] != 0 && bp.edge[k] != 1) return fail("bad characteristic BC variant");
  if (bp.relax_sign != 0.0 && bp.relax_sign != 1.0 && bp.relax_sign != -1.0)
    return fail("relax_sign must be -1, +1 or 0");
  if ((long long)grid->nx * grid->ny > (1ll << 31) / 2) return fail("grid too large");
  return LBM_OK;
}

lbm_status lbm_estimate_bytes_bc(const lbm_grid* grid, lbm_stencil stencil, int pml_width,
                                 const lbm_sigma_profile* sigma, lbm_bc_kind bc,
                                 const lbm_bc_params* bc_params, lbm_precision precision,
                                 size_t* bytes) {
  if (!bytes) return LBM_EINVAL;
  lbm_sigma_profile sg;
  lbm_bc_params bp;
  int W4[4];
  const lbm_status st = check_args(grid, stencil, 0.75, pml_width, sigma, bc, bc_params,
                                   precision, sg, bp, W4);
  if (st != LBM_OK) return st;
  const int q = (int)stencil;
  const Geom g = make_geom(grid->nx, grid->ny, W4, halo_of(q), bp.periodic_y, bp.pml_grad);
  *bytes = bytes_of(g, q, precision == LBM_FP64 ? 8 : 4);
  return LBM_OK;
}

lbm_status lbm_create(const lbm_grid* grid, lbm_stencil stencil, double tau, int pml_width,
                      const lbm_sigma_profile* sigma, lbm_bc_kind bc, const lbm_bc_params* bcp,
                      lbm_precision precision, void* cuda_stream, lbm_ctx** out) {
  if (!out) return LBM_EINVAL;
  *out = nullptr;
  auto fail = [](const char* m) { g_create_error = m; return LBM_EINVAL; };
  lbm_sigma_profile sg;
  lbm_bc_params bp;
  int W4[4];
  {
    const lbm_status st = check_args(grid, stencil, tau, pml_width, sigma, bc, bcp, precision,
                                     sg, bp, W4);
    if (st != LBM_OK) return st;
  }
  const int q = (int)stencil;

  lbm_ctx* ctx = new lbm_ctx();
  if (const char* b = std::getenv("LBM_DEBUG_ALLOC_BUDGET")) ctx->alloc_budget = std::strtoull(b, nullptr, 10);
  ctx->q = q;
  ctx->prec = precision;
  ctx->bc = bc;
  ctx->tau = tau;
  ctx->omega = std::isinf(tau) ? 0.0 : 1.0 / tau;
  ctx->st = (cudaStream_t)cuda_stream;
  std::string lerr;
  if (!lattice_of(q, ctx->w, &ctx->r, lerr)) { delete ctx; return fail("quadrature failed"); }
  cudaGetDevice(&ctx->device);

  ctx->g = make_geom(grid->nx, grid->ny, W4, halo_of(q), bp.periodic_y, bp.pml_grad);
  Geom& g = ctx->g;

  switch (q * 2 + (precision == LBM_FP32_DEV)) {
    case 74: ctx->ops = ops_q37_f64(); break;
    case 75: ctx->ops = ops_q37_f32(); break;
    case 34: ctx->ops = ops_q17_f64(); break;
    case 35: ctx->ops = ops_q17_f32(); break;
    case 18: ctx->ops = ops_q9_f64(); break;
    default: ctx->ops = ops_q9_f32(); break;
  }
  const int es = ctx->ops.elem_size;
  ctx->fbytes = (size_t)q * g.plane * es;
  ctx->sbytes = (size_t)q * g.Sp * es;
  const size_t fieldbytes = (size_t)4 * g.Lx * g.Ly * sizeof(double);
  ctx->max_blocks = ((g.Lx + 31) / 32) * ((g.Ly + 7) / 8);

  auto oom = [&](const char* what) {
    g_create_error = std::string("allocation failed: ") + what;
    free_all(ctx);
    delete ctx;
    return LBM_ENOMEM;
  };
  for (int k = 0; k < 2; ++k) {
    if (dalloc(ctx, &ctx->f[k], ctx->fbytes) != cudaSuccess) return oom("populations");
    if (cudaMemsetAsync(ctx->f[k], 0, ctx->fbytes, ctx->st) != cudaSuccess) return oom("populations");
    if (has_pml(g)) {
      if (dalloc(ctx, &ctx->S[k], ctx->sbytes) != cudaSuccess) return oom("PML accumulator");
      if (cudaMemsetAsync(ctx->S[k], 0, ctx->sbytes, ctx->st) != cudaSuccess)
        return oom("PML accumulator");
    }
  }
  if (dalloc(ctx, (void**)&ctx->V, sizeof(double) * 16 * (size_t)g.nb) != cudaSuccess)
    return oom("targets");
  if (dalloc(ctx, (void**)&ctx->Uedge, sizeof(double) * 2 * edge_slots(g)) != cudaSuccess)
    return oom("edges");
  if (cudaMemsetAsync(ctx->V, 0, sizeof(double) * 16 * (size_t)g.nb, ctx->st) != cudaSuccess ||
      cudaMemsetAsync(ctx->Uedge, 0, sizeof(double) * 2 * edge_slots(g), ctx->st) != cudaSuccess)
    return oom("targets");
  if (dalloc(ctx, (void**)&ctx->Sedge, sizeof(double) * 2 * source_slots(g)) != cudaSuccess ||
      cudaMemsetAsync(ctx->Sedge, 0, sizeof(double) * 2 * source_slots(g), ctx->st) != cudaSuccess)
    return oom("PML source");
  if (dalloc(ctx, (void**)&ctx->staging, fieldbytes) != cudaSuccess) return oom("staging");
  if (dalloc(ctx, (void**)&ctx->partials, sizeof(double) * 12 * (size_t)ctx->max_blocks) !=
      cudaSuccess)
    return oom("partials");
  if (dalloc(ctx, (void**)&ctx->dout, sizeof(double) * 16) != cudaSuccess) return oom("outputs");
  if (cudaHostAlloc(&ctx->hout, sizeof(double) * 16, cudaHostAllocDefault) != cudaSuccess)
    return oom("pinned outputs");
  if (cudaHostAlloc(&ctx->hflag, sizeof(int), cudaHostAllocMapped) != cudaSuccess)
    return oom("status flag");
  *ctx->hflag = 0;
  if (cudaHostGetDevicePointer((void**)&ctx->dflag, ctx->hflag, 0) != cudaSuccess)
    return oom("status flag mapping");

  // the boundary chain is latency-bound: give its stream the highest priority so its blocks
  // are scheduled ahead of the interior kernel's as SM slots free up
  int prio_low = 0, prio_high = 0;
  cudaDeviceGetStreamPriorityRange(&prio_low, &prio_high);
  if (cudaStreamCreateWithPriority(&ctx->aux, cudaStreamNonBlocking, prio_high) != cudaSuccess ||
      cudaStreamCreateWithPriority(&ctx->aux2, cudaStreamNonBlocking, prio_high) != cudaSuccess ||
      cudaStreamCreateWithFlags(&ctx->cap, cudaStreamNonBlocking) != cudaSuccess ||
      cudaEventCreateWithFlags(&ctx->fork, cudaEventDisableTiming) != cudaSuccess ||
      cudaEventCreateWithFlags(&ctx->join, cudaEventDisableTiming) != cudaSuccess ||
      cudaEventCreateWithFlags(&ctx->join2, cudaEventDisableTiming) != cudaSuccess ||
      cudaEventCreateWithFlags(&ctx->ready, cudaEventDisableTiming) != cudaSuccess)
    return oom("streams and events");
  Dev& d = ctx->dev;
  d.g = g;
  d.st = ctx->st;
  d.aux = ctx->aux;
  d.aux2 = ctx->aux2;
  d.fork = ctx->fork;
  d.join = ctx->join;
  d.join2 = ctx->join2;
  d.flag = ctx->dflag;
  d.Vtgt = ctx->V;
  d.Va = ctx->V + 4 * (size_t)g.nb;
  d.Vb = ctx->V + 8 * (size_t)g.nb;
  d.Vacc = ctx->V + 12 * (size_t)g.nb;
  d.bc.bc = (int)bc;
  for (int k = 0; k < 4; ++k) d.bc.edge[k] = bp.edge[k];
  d.bc.beta = bp.beta;
  d.bc.relax_sign = bp.relax_sign == 0.0 ? -1.0 : bp.relax_sign;
  d.bc.pml_source = bp.pml_source;
  d.bc.r = ctx->r;
  d.bc.inv_r = 1.0 / ctx->r;
  d.bc.omega = ctx->omega;
  double fbar[kMaxQ];
  if (q == 37) mean_equilibrium<D2Q37>(ctx->w, ctx->r, bp, fbar);
  else if (q == 17) mean_equilibrium<D2Q17>(ctx->w, ctx->r, bp, fbar);
  else mean_equilibrium<D2Q9>(ctx->w, ctx->r, bp, fbar);
  std::memset(&d.cd, 0, sizeof d.cd);
  std::memset(&d.cf, 0, sizeof d.cf);
  for (int i = 0; i < q; ++i) {
    d.cd.w[i] = ctx->w[i];
    d.cd.eqbar[i] = fbar[i];
    d.cf.w[i] = (float)ctx->w[i];
    d.cf.eqbar[i] = (float)(fbar[i] - ctx->w[i]);
  }
  d.cd.r = ctx->r; d.cd.r2 = ctx->r * ctx->r; d.cd.omega = ctx->omega;
  d.cd.sigma_max = sg.sigma_max; d.cd.power = sg.power; d.cd.split = sg.split;
  d.cf.r = (float)ctx->r; d.cf.r2 = (float)(ctx->r * ctx->r); d.cf.omega = (float)ctx->omega;
  d.cf.sigma_max = (float)sg.sigma_max; d.cf.power = sg.power; d.cf.split = sg.split;
  if (ctx->ops.prepare(ctx->w) != cudaSuccess) return oom("kernel attributes");
  {
    // the context's one-member plan, for buffer parity 0 and 1
    set_roles(ctx, 0, 0);
    Dev d0 = ctx->dev;
    set_roles(ctx, 1, 1);
    Dev d1 = ctx->dev;
    const Dev* p0 = &d0;
    const Dev* p1 = &d1;
    if (ctx->ops.batch_plan(&p0, &p1, 1, 32, 4, &ctx->plan) != cudaSuccess) return oom("plan");
    ctx->dev.plan = &ctx->plan;
  }
  if (cudaStreamSynchronize(ctx->st) != cudaSuccess) return oom("stream sync");
  *out = ctx;
  return LBM_OK;
}

lbm_status lbm_destroy(lbm_ctx* ctx) {
  if (!ctx) return LBM_OK;
  free_all(ctx);
  delete ctx;
  return LBM_OK;
}

const char* lbm_last_error(const lbm_ctx* ctx) {
  return ctx ? ctx->err.c_str() : g_create_error.c_str();
}

lbm_status lbm_debug_check_guards(lbm_ctx* ctx, int* intact) {
  if (!ctx || !intact) return LBM_EINVAL;
  LBM_CK(cudaSetDevice(ctx->device));
  LBM_CK(cudaStreamSynchronize(ctx->st));
  *intact = 1;
  std::vector<unsigned char> h(kGuard);
  for (const auto& a : ctx->allocs)
    for (int side = 0; side < 2; ++side) {
      LBM_CK(cudaMemcpy(h.data(), a.first + (side ? kGuard + a.second : 0), kGuard,
                        cudaMemcpyDeviceToHost));
      for (unsigned char v : h)
        if (v != (unsigned char)kGuardByte) *intact = 0;
    }
  return LBM_OK;
}

lbm_status lbm_geometry(const lbm_ctx* ctx, int64_t* out) {
  if (!ctx || !out) return LBM_EINVAL;
  const Geom& g = ctx->g;
  out[0] = g.nx; out[1] = g.ny; out[2] = g.Ww; out[3] = g.M;
  out[4] = g.Lx; out[5] = g.Ly; out[6] = ctx->q; out[7] = ctx->steps;
  out[8] = g.Ww; out[9] = g.We; out[10] = g.Ws; out[11] = g.Wn;
  return LBM_OK;
}

}  // extern "C"

// characteristic targets at initialization: the fields at the nearest fluid node x_f
namespace lbm {
__global__ void k_init_targets(Geom g, const double* rho, const double* ux, const double* uy,
                               const double* T, double* V) {
  const int b = blockIdx.x * blockDim.x + threadIdx.x;
  if (b >= g.nb) return;
  const int M = g.M, Lx = g.Lx, Ly = g.Ly;
  int x, y;
  if (b < M * Ly) { y = b % Ly; x = 0; }
  else if (b < 2 * M * Ly) { y = (b - M * Ly) % Ly; x = Lx - 1; }
  else if (b < 2 * M * Ly + M * Lx) { x = (b - 2 * M * Ly) % Lx; y = 0; }
  else { x = (b - 2 * M * Ly - M * Lx) % Lx; y = Ly - 1; }
  const int k = y * Lx + x;
  V[b] = rho[k];
  V[g.nb + b] = ux[k];
  V[2 * g.nb + b] = uy[k];
  V[3 * g.nb + b] = T[k];
}
}  // namespace lbm

extern "C" {

lbm_status lbm_init(lbm_ctx* ctx, const double* rho, const double* ux, const double* uy,
                    const double* T, int fields_on_device) {
  if (!ctx) return LBM_EINVAL;
  if (!rho || !ux || !uy || !T) { ctx->err = "NULL field"; return LBM_EINVAL; }
  LBM_CK(cudaSetDevice(ctx->device));
  const Geom& g = ctx->g;
  const size_t n = (size_t)g.Lx * g.Ly;
  const double* src[4] = {rho, ux, uy, T};
  if (!fields_on_device) {
    for (int k = 0; k < 4; ++k)
      LBM_CK(cudaMemcpyAsync(ctx->staging + k * n, src[k], n * sizeof(double),
                             cudaMemcpyHostToDevice, ctx->st));
    for (int k = 0; k < 4; ++k) src[k] = ctx->staging + k * n;
  }
  *ctx->hflag = 0;
  Dev& d = ctx->dev;
  set_roles(ctx, 0, 0);
  LBM_CK(ctx->ops.init_eq(d, src[0], src[1], src[2], src[3]));
  if (ctx->bc == LBM_BC_NRBC) {
    k_init_targets<<<(g.nb + 127) / 128, 128, 0, ctx->st>>>(g, src[0], src[1], src[2], src[3],
                                                            d.Vtgt);
    LBM_CK(cudaGetLastError());
  }
  // initial collision (no streaming): buffer 0 holds f^0, buffer 1 receives f*^0
  LBM_CK(ctx->ops.step(d, false));
  LBM_CK(cudaStreamSynchronize(ctx->st));
  ctx->cur = 1;
  ctx->scur = 1;
  ctx->steps = 0;
  ctx->initialized = true;
  ctx->prev_valid = true;
  ctx->prev_prestream = true;
  return LBM_OK;
}

// Captures one step for the current buffer parity into an executable graph (on the internal
// capture stream; the boundary chain forks onto aux inside the capture).
static lbm_status build_graph(lbm_ctx* ctx, int parity) {
  set_roles(ctx, parity, parity);
  Dev d = ctx->dev;
  d.st = ctx->cap;
  d.ev = nullptr;
  LBM_CK(cudaStreamBeginCapture(ctx->cap, cudaStreamCaptureModeThreadLocal));
  cudaError_t e = ctx->ops.step(d, true);
  cudaGraph_t graph = nullptr;
  cudaError_t e2 = cudaStreamEndCapture(ctx->cap, &graph);
  LBM_CK(e);
  LBM_CK(e2);
  e = cudaGraphInstantiate(&ctx->graph[parity], graph, 0);
  if (e != cudaSuccess) cudaGraphDestroy(graph);
  LBM_CK(e);
  ctx->gtemplate[parity] = graph;
  return LBM_OK;
}

lbm_status lbm_step(lbm_ctx* ctx, int n) {
  lbm_status s = check_ready(ctx);
  if (s != LBM_OK) return s;
  if (n < 0) { ctx->err = "negative step count"; return LBM_EINVAL; }
  if (*(volatile int*)ctx->hflag) { ctx->err = "unphysical state flagged"; return LBM_EUNSTABLE; }
  for (int k = 0; k < n; ++k) {
    const bool profiled = ctx->prof_used < ctx->prof_cap;
    if (ctx->use_graphs && !profiled) {
      if (!ctx->graph[ctx->cur]) {
        lbm_status gs = build_graph(ctx, ctx->cur);
        if (gs != LBM_OK) return gs;
      }
      LBM_CK(cudaGraphLaunch(ctx->graph[ctx->cur], ctx->st));
    } else {
      set_roles(ctx, ctx->cur, ctx->scur);
      Dev d = ctx->dev;
      if (profiled) {
        // attribution: each kernel class runs alone (boundary chain after the interior kernel on
        // one stream), so its events measure that class and nothing concurrent
        d.ev = &ctx->prof[(size_t)2 * kKernelClasses * ctx->prof_used++];
        d.aux = nullptr;
        d.aux2 = nullptr;
      }
      LBM_CK(ctx->ops.step(d, true));
    }
    ctx->cur ^= 1;
    ctx->scur ^= 1;
    ctx->steps++;
  }
  if (n > 0) { ctx->prev_valid = true; ctx->prev_prestream = false; }
  return LBM_OK;
}

lbm_status lbm_sync(lbm_ctx* ctx) {
  if (!ctx) return LBM_EINVAL;
  LBM_CK(cudaSetDevice(ctx->device));
  LBM_CK(cudaStreamSynchronize(ctx->st));
  if (*(volatile int*)ctx->hflag) { ctx->err = "unphysical state flagged"; return LBM_EUNSTABLE; }
  return LBM_OK;
}

lbm_status lbm_moments(lbm_ctx* ctx, double* rho, double* ux, double* uy, double* T, int region,
                       int out_on_device) {
  lbm_status s = check_ready(ctx);
  if (s != LBM_OK) return s;
  if (!ctx->prev_valid) { ctx->err = "populations were imported; step first"; return LBM_ESTATE; }
  const Geom& g = ctx->g;
  const size_t n = region ? (size_t)g.Lx * g.Ly : (size_t)g.nx * g.ny;
  double* user[4] = {rho, ux, uy, T};
  double* o[4];
  for (int k = 0; k < 4; ++k) o[k] = out_on_device ? user[k] : (user[k] ? ctx->staging + k * n : nullptr);
  const double* r[4] = {nullptr, nullptr, nullptr, nullptr};
  int nblk = 0;
  LBM_CK(ctx->ops.fields(ctx->dev, ctx->f[1 - ctx->cur], !ctx->prev_prestream, region ? 1 : 0, o,
                         r, 1, nullptr, &nblk));
  if (!out_on_device)
    for (int k = 0; k < 4; ++k)
      if (user[k])
        LBM_CK(cudaMemcpyAsync(user[k], o[k], n * sizeof(double), cudaMemcpyDeviceToHost, ctx->st));
  LBM_CK(cudaStreamSynchronize(ctx->st));
  if (*(volatile int*)ctx->hflag) { ctx->err = "unphysical state flagged"; return LBM_EUNSTABLE; }
  return LBM_OK;
}

static lbm_status reduce_common(lbm_ctx* ctx, int mode, const double* const r[4], unsigned min_mask,
                                double* out, int nout) {
  double* o[4] = {nullptr, nullptr, nullptr, nullptr};
  int nblk = 0;
  LBM_CK(ctx->ops.fields(ctx->dev, ctx->f[1 - ctx->cur], !ctx->prev_prestream, mode == 2 ? 1 : 0,
                         o, r, mode, ctx->partials, &nblk));
  LBM_CK(reduce_partials(ctx->partials, nblk, min_mask, ctx->dout, ctx->st));
  LBM_CK(cudaMemcpyAsync(ctx->hout, ctx->dout, sizeof(double) * 12, cudaMemcpyDeviceToHost, ctx->st));
  LBM_CK(cudaStreamSynchronize(ctx->st));
  std::memcpy(out, ctx->hout, sizeof(double) * nout);
  return LBM_OK;
}

lbm_status lbm_reduce(lbm_ctx* ctx, double* out) {
  lbm_status s = check_ready(ctx);
  if (s != LBM_OK) return s;
  if (!out) return LBM_EINVAL;
  if (!ctx->prev_valid) { ctx->err = "populations were imported; step first"; return LBM_ESTATE; }
  const double* r[4] = {nullptr, nullptr, nullptr, nullptr};
  return reduce_common(ctx, 2, r, (1u << 4) | (1u << 5), out, 7);
}

lbm_status lbm_error_sums(lbm_ctx* ctx, const double* ref_rho, const double* ref_ux,
                          const double* ref_uy, const double* ref_T, double* out) {
  lbm_status s = check_ready(ctx);
  if (s != LBM_OK) return s;
  if (!out || !ref_rho || !ref_ux || !ref_uy || !ref_T) return LBM_EINVAL;
  if (!ctx->prev_valid) { ctx->err = "populations were imported; step first"; return LBM_ESTATE; }
  const double* r[4] = {ref_rho, ref_ux, ref_uy, ref_T};
  return reduce_common(ctx, 4, r, 0u, out, 12);
}

lbm_status lbm_export_populations(lbm_ctx* ctx, double* host) {
  lbm_status s = check_ready(ctx);
  if (s != LBM_OK) return s;
  if (!host) return LBM_EINVAL;
  const Geom& g = ctx->g;
  const size_t n = (size_t)ctx->q * (g.Lx + 2 * g.M) * (g.Ly + 2 * g.M);
  double* tmp = nullptr;
  LBM_CK(cudaMalloc(&tmp, n * sizeof(double)));
  cudaError_t e = ctx->ops.export_pop(ctx->dev, ctx->f[ctx->cur], tmp);
  if (e == cudaSuccess) e = cudaMemcpyAsync(host, tmp, n * sizeof(double), cudaMemcpyDeviceToHost, ctx->st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(ctx->st);
  cudaFree(tmp);
  LBM_CK(e);
  return LBM_OK;
}

lbm_status lbm_import_populations(lbm_ctx* ctx, const double* host) {
  lbm_status s = check_ready(ctx);
  if (s != LBM_OK) return s;
  if (!host) return LBM_EINVAL;
  const Geom& g = ctx->g;
  const size_t n = (size_t)ctx->q * (g.Lx + 2 * g.M) * (g.Ly + 2 * g.M);
  double* tmp = nullptr;
  LBM_CK(cudaMalloc(&tmp, n * sizeof(double)));
  cudaError_t e = cudaMemcpyAsync(tmp, host, n * sizeof(double), cudaMemcpyHostToDevice, ctx->st);
  if (e == cudaSuccess) e = ctx->ops.import_pop(ctx->dev, tmp, ctx->f[ctx->cur]);
  if (e == cudaSuccess) e = cudaStreamSynchronize(ctx->st);
  cudaFree(tmp);
  LBM_CK(e);
  ctx->prev_valid = false;
  return LBM_OK;
}

}  // extern "C"

// Diagnostic exports: the index maps and the site classification as the kernels compute them.
namespace lbm {
template <class S>
__global__ void k_pull_index(Geom g, long long* __restrict__ out) {
  const long long nf = (long long)g.Lx * g.Ly, n = (long long)S::Q * nf;
  const int Gx = g.Lx + 2 * g.M;
  for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < n;
       t += (long long)gridDim.x * blockDim.x) {
    const int i = int(t / nf);
    const long long k = t - (long long)i * nf;
    const int y = int(k / g.Lx), x = int(k - (long long)y * g.Lx);
    const long long src = pull_src(g, gindex(g, x, y), S::ex(i), S::ey(i));
    const long long row = src / g.pitch, col = src - row * g.pitch;
    out[t] = row * Gx + (col - g.cF0 + g.M);   // G coordinates (gy, gx), row-major
  }
}

__global__ void k_site_class(Geom g, Consts<double> c, int* __restrict__ layer,
                             unsigned char* __restrict__ hasq, double* __restrict__ sxo,
                             double* __restrict__ syo) {
  const int x = blockIdx.x * blockDim.x + threadIdx.x, y = blockIdx.y;
  if (x >= g.Lx) return;
  const PmlNode<double> n = pml_node<double>(g, x, y);
  const long long k = (long long)y * g.Lx + x;
  layer[k] = max(n.ix, n.iy);
  hasq[k] = has_pml(g) && n.has_q ? 1 : 0;
  double sx = 0.0, sy = 0.0;
  if (n.in_p) pml_sigmas(c, n, sx, sy);
  sxo[k] = sx;
  syo[k] = sy;
}
}  // namespace lbm

extern "C" {

lbm_status lbm_export_pull_index(lbm_ctx* ctx, int64_t* host) {
  if (!ctx) return LBM_EINVAL;
  if (!host) { ctx->err = "NULL output"; return LBM_EINVAL; }
  LBM_CK(cudaSetDevice(ctx->device));
  const Geom& g = ctx->g;
  const size_t n = (size_t)ctx->q * g.Lx * g.Ly;
  long long* tmp = nullptr;
  LBM_CK(cudaMalloc(&tmp, n * sizeof(long long)));
  if (ctx->q == 37) k_pull_index<D2Q37><<<512, 256, 0, ctx->st>>>(g, tmp);
  else if (ctx->q == 17) k_pull_index<D2Q17><<<512, 256, 0, ctx->st>>>(g, tmp);
  else k_pull_index<D2Q9><<<512, 256, 0, ctx->st>>>(g, tmp);
  cudaError_t e = cudaGetLastError();
  if (e == cudaSuccess) e = cudaMemcpyAsync(host, tmp, n * sizeof(long long), cudaMemcpyDeviceToHost, ctx->st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(ctx->st);
  cudaFree(tmp);
  LBM_CK(e);
  return LBM_OK;
}

lbm_status lbm_export_site_class(lbm_ctx* ctx, int32_t* layer, uint8_t* has_q, double* sigma_x,
                                 double* sigma_y) {
  if (!ctx) return LBM_EINVAL;
  LBM_CK(cudaSetDevice(ctx->device));
  const Geom& g = ctx->g;
  const size_t n = (size_t)g.Lx * g.Ly;
  char* tmp = nullptr;
  const size_t bytes = n * (sizeof(int) + 1 + 2 * sizeof(double)) + 64;
  LBM_CK(cudaMalloc(&tmp, bytes));
  double* sx = reinterpret_cast<double*>(tmp);
  double* sy = sx + n;
  int* ly = reinterpret_cast<int*>(sy + n);
  unsigned char* hq = reinterpret_cast<unsigned char*>(ly + n);
  k_site_class<<<dim3((g.Lx + 127) / 128, g.Ly), 128, 0, ctx->st>>>(g, ctx->dev.cd, ly, hq, sx, sy);
  cudaError_t e = cudaGetLastError();
  auto get = [&](void* dst, const void* src, size_t b) {
    if (dst && e == cudaSuccess) e = cudaMemcpyAsync(dst, src, b, cudaMemcpyDeviceToHost, ctx->st);
  };
  get(layer, ly, n * sizeof(int));
  get(has_q, hq, n);
  get(sigma_x, sx, n * sizeof(double));
  get(sigma_y, sy, n * sizeof(double));
  if (e == cudaSuccess) e = cudaStreamSynchronize(ctx->st);
  cudaFree(tmp);
  LBM_CK(e);
  return LBM_OK;
}

lbm_status lbm_profile_enable(lbm_ctx* ctx, int max_steps) {
  if (!ctx || max_steps < 0) return LBM_EINVAL;
  LBM_CK(cudaSetDevice(ctx->device));
  LBM_CK(cudaStreamSynchronize(ctx->st));
  for (cudaEvent_t e : ctx->prof) cudaEventDestroy(e);
  ctx->prof.clear();
  ctx->prof_cap = ctx->prof_used = 0;
  ctx->prof.resize((size_t)2 * kKernelClasses * max_steps);
  for (auto& e : ctx->prof) LBM_CK(cudaEventCreate(&e));
  ctx->prof_cap = max_steps;
  return LBM_OK;
}

lbm_status lbm_profile_read(lbm_ctx* ctx, double* ms, int* steps) {
  if (!ctx || !ms) return LBM_EINVAL;
  LBM_CK(cudaSetDevice(ctx->device));
  LBM_CK(cudaStreamSynchronize(ctx->st));
  for (int k = 0; k < kKernelClasses; ++k) ms[k] = 0.0;
  for (int s = 0; s < ctx->prof_used; ++s)
    for (int k = 0; k < kKernelClasses; ++k) {
      float t = 0.f;
      LBM_CK(cudaEventElapsedTime(&t, ctx->prof[(size_t)2 * kKernelClasses * s + 2 * k],
                                  ctx->prof[(size_t)2 * kKernelClasses * s + 2 * k + 1]));
      ms[k] += t;
    }
  if (steps) *steps = ctx->prof_used;
  ctx->prof_used = 0;
  return LBM_OK;
}

// checkpoint layout: header of 8 int64, then current and previous population buffers, the PML
// accumulator of the current level, the targets, the saved edge moments and PML sources
struct CkptHeader { int64_t magic, q, nx, ny, widths, prec, steps, flags; };

// the four PML widths (each <= 4096) packed 16 bits apiece, and the sigma form
static int64_t pack_widths(const lbm_ctx* ctx) {
  const Geom& g = ctx->g;
  return (int64_t)g.Ww | ((int64_t)g.We << 16) | ((int64_t)g.Ws << 32) | ((int64_t)g.Wn << 48);
}
static const int64_t kMagic = 0x4c424d434b505431ll;

lbm_status lbm_checkpoint_size(const lbm_ctx* ctx, size_t* bytes) {
  if (!ctx || !bytes) return LBM_EINVAL;
  *bytes = sizeof(CkptHeader) + 2 * ctx->fbytes + ctx->sbytes +
           sizeof(double) * (4 * (size_t)ctx->g.nb + edge_slots(ctx->g) + source_slots(ctx->g));
  return LBM_OK;
}

lbm_status lbm_checkpoint(lbm_ctx* ctx, void* host, size_t bytes) {
  lbm_status s = check_ready(ctx);
  if (s != LBM_OK) return s;
  size_t need;
  lbm_checkpoint_size(ctx, &need);
  if (!host || bytes < need) { ctx->err = "checkpoint buffer too small"; return LBM_EINVAL; }
  char* p = static_cast<char*>(host);
  CkptHeader h{kMagic, ctx->q, ctx->g.nx, ctx->g.ny, pack_widths(ctx), (int64_t)ctx->prec,
               ctx->steps,
               (int64_t)(ctx->prev_valid ? 1 : 0) | (int64_t)(ctx->prev_prestream ? 2 : 0) |
                   ((int64_t)ctx->g.py << 2) | ((int64_t)ctx->g.link << 3)};
  std::memcpy(p, &h, sizeof h);
  p += sizeof h;
  const cudaMemcpyKind k = cudaMemcpyDeviceToHost;
  LBM_CK(cudaMemcpyAsync(p, ctx->f[ctx->cur], ctx->fbytes, k, ctx->st)); p += ctx->fbytes;
  LBM_CK(cudaMemcpyAsync(p, ctx->f[1 - ctx->cur], ctx->fbytes, k, ctx->st)); p += ctx->fbytes;
  if (ctx->sbytes) { LBM_CK(cudaMemcpyAsync(p, ctx->S[ctx->scur], ctx->sbytes, k, ctx->st)); p += ctx->sbytes; }
  LBM_CK(cudaMemcpyAsync(p, ctx->V, sizeof(double) * 4 * ctx->g.nb, k, ctx->st)); p += sizeof(double) * 4 * ctx->g.nb;
  // the edge moments the next step's targets read
  LBM_CK(cudaMemcpyAsync(p, ctx->Uedge + ctx->cur * edge_slots(ctx->g),
                         sizeof(double) * edge_slots(ctx->g), k, ctx->st));
  p += sizeof(double) * edge_slots(ctx->g);
  LBM_CK(cudaMemcpyAsync(p, ctx->Sedge + ctx->cur * source_slots(ctx->g),
                         sizeof(double) * source_slots(ctx->g), k, ctx->st));
  LBM_CK(cudaStreamSynchronize(ctx->st));
  return LBM_OK;
}

lbm_status lbm_restore(lbm_ctx* ctx, const void* host, size_t bytes) {
  if (!ctx || !host) return LBM_EINVAL;
  LBM_CK(cudaSetDevice(ctx->device));
  size_t need;
  lbm_checkpoint_size(ctx, &need);
  if (bytes < need) { ctx->err = "checkpoint buffer too small"; return LBM_EINVAL; }
  const char* p = static_cast<const char*>(host);
  CkptHeader h;
  std::memcpy(&h, p, sizeof h);
  if (h.magic != kMagic || h.q != ctx->q || h.nx != ctx->g.nx || h.ny != ctx->g.ny ||
      h.widths != pack_widths(ctx) || h.prec != (int64_t)ctx->prec ||
      ((h.flags >> 2) & 1) != ctx->g.py || ((h.flags >> 3) & 1) != ctx->g.link) {
    ctx->err = "checkpoint does not match this context";
    return LBM_EINVAL;
  }
  p += sizeof h;
  const cudaMemcpyKind k = cudaMemcpyHostToDevice;
  ctx->cur = 0;
  ctx->scur = 0;
  LBM_CK(cudaMemcpyAsync(ctx->f[0], p, ctx->fbytes, k, ctx->st)); p += ctx->fbytes;
  LBM_CK(cudaMemcpyAsync(ctx->f[1], p, ctx->fbytes, k, ctx->st)); p += ctx->fbytes;
  if (ctx->sbytes) { LBM_CK(cudaMemcpyAsync(ctx->S[0], p, ctx->sbytes, k, ctx->st)); p += ctx->sbytes; }
  LBM_CK(cudaMemcpyAsync(ctx->V, p, sizeof(double) * 4 * ctx->g.nb, k, ctx->st)); p += sizeof(double) * 4 * ctx->g.nb;
  LBM_CK(cudaMemcpyAsync(ctx->Uedge, p, sizeof(double) * edge_slots(ctx->g), k, ctx->st));
  p += sizeof(double) * edge_slots(ctx->g);
  LBM_CK(cudaMemcpyAsync(ctx->Sedge, p, sizeof(double) * source_slots(ctx->g), k, ctx->st));
  LBM_CK(cudaStreamSynchronize(ctx->st));
  ctx->steps = h.steps;
  ctx->prev_valid = (h.flags & 1) != 0;
  ctx->prev_prestream = (h.flags & 2) != 0;
  ctx->initialized = true;
  *ctx->hflag = 0;
  return LBM_OK;
}

}  // extern "C"

// --------------------------------------------------------------------------------------------
// Batched execution (see lbm.h): the members are grouped by (stencil, precision, PML gradient
// mode); each group is one plan whose kernels each cover every member of the group in one
// launch (a table of (member, tile) entries), and one step of all groups is one captured graph
// per buffer-parity state.
#include <map>
#include <tuple>

namespace {
struct BatchGroup {
  OpsTable ops;
  std::vector<int> idx;     // member indices
  BatchPlan plan;
};
// autotuned bulk tile shape per (stencil, precision, PML gradient mode, device name)
std::mutex g_tune_mutex;
std::map<std::tuple<int, int, int, std::string>, std::pair<int, int>> g_tune_cache;

std::string device_name(int dev) {
  cudaDeviceProp pr;
  if (cudaGetDeviceProperties(&pr, dev) != cudaSuccess) return "?";
  return pr.name;
}
}  // namespace

struct lbm_batch {
  cudaStream_t st = nullptr;              // the caller's stream
  cudaStream_t cap = nullptr, aux = nullptr, aux2 = nullptr;
  cudaEvent_t fork = nullptr, join = nullptr, join2 = nullptr;
  int device = -1;
  std::vector<lbm_ctx*> members;
  std::vector<int> base;                  // members' buffer parity when the plans were built
  std::vector<BatchGroup> groups;
  cudaGraphExec_t graph[2] = {nullptr, nullptr};
  int tx = 0, by = 0;                     // bulk tile shape; 0: from the tuning cache / default
  bool built = false;
  std::string err;
};

static void batch_clear(lbm_batch* b) {
  for (int k = 0; k < 2; ++k)
    if (b->graph[k]) { cudaGraphExecDestroy(b->graph[k]); b->graph[k] = nullptr; }
  for (auto& g : b->groups) batch_plan_free(&g.plan);
  b->groups.clear();
  b->built = false;
}

void lbm::batch_plan_free(BatchPlan* p) {
  if (p->mem) cudaFree(p->mem);
  *p = BatchPlan();
}

static std::tuple<int, int, int, std::string> tune_key(const lbm_ctx* c) {
  return {c->q, (int)c->prec, c->g.link, device_name(c->device)};
}

// Plans and the two step graphs for the current member set and tile shape.
static lbm_status batch_build(lbm_batch* b) {
  batch_clear(b);
  if (b->members.empty()) return LBM_OK;
  lbm_ctx* ctx = b->members[0];   // for LBM_CK messages
  LBM_CK(cudaSetDevice(b->device));
  int tx = b->tx, by = b->by;
  if (!tx) {
    std::lock_guard<std::mutex> lock(g_tune_mutex);
    auto it = g_tune_cache.find(tune_key(ctx));
    tx = it != g_tune_cache.end() ? it->second.first : 32;
    by = it != g_tune_cache.end() ? it->second.second : 4;
  }
  std::map<std::tuple<int, int, int>, int> gi;
  for (int m = 0; m < (int)b->members.size(); ++m) {
    lbm_ctx* c = b->members[m];
    auto key = std::make_tuple(c->q, (int)c->prec, c->g.link);
    auto it = gi.find(key);
    if (it == gi.end()) {
      gi[key] = (int)b->groups.size();
      b->groups.push_back(BatchGroup{c->ops, {m}, BatchPlan()});
    } else {
      b->groups[it->second].idx.push_back(m);
    }
  }
  b->base.resize(b->members.size());
  for (auto& G : b->groups) {
    std::vector<Dev> d0, d1;
    for (int m : G.idx) {
      lbm_ctx* c = b->members[m];
      b->base[m] = c->cur;
      set_roles(c, c->cur, c->scur);
      d0.push_back(c->dev);
      set_roles(c, c->cur ^ 1, c->scur ^ 1);
      d1.push_back(c->dev);
    }
    std::vector<const Dev*> p0, p1;
    for (size_t k = 0; k < d0.size(); ++k) { p0.push_back(&d0[k]); p1.push_back(&d1[k]); }
    const cudaError_t e = G.ops.batch_plan(p0.data(), p1.data(), (int)p0.size(), tx, by, &G.plan);
    if (e != cudaSuccess) {
      b->err = std::string("batch plan: ") + cudaGetErrorString(e);
      batch_clear(b);
      return e == cudaErrorMemoryAllocation ? LBM_ENOMEM : LBM_ECUDA;
    }
  }
  for (int w = 0; w < 2; ++w) {
    cudaError_t e = cudaStreamBeginCapture(b->cap, cudaStreamCaptureModeThreadLocal);
    if (e == cudaSuccess) {
      for (auto& G : b->groups)
        if (e == cudaSuccess)
          e = G.ops.batch_step(G.plan, w, b->cap, b->aux, b->aux2, b->fork, b->join, b->join2);
      cudaGraph_t graph = nullptr;
      const cudaError_t e2 = cudaStreamEndCapture(b->cap, &graph);
      if (e == cudaSuccess) e = e2;
      if (e == cudaSuccess) e = cudaGraphInstantiate(&b->graph[w], graph, 0);
      if (graph) cudaGraphDestroy(graph);
    }
    if (e != cudaSuccess) {
      b->err = std::string("batch graph: ") + cudaGetErrorString(e);
      batch_clear(b);
      return LBM_ECUDA;
    }
  }
  b->built = true;
  return LBM_OK;
}

extern "C" {

lbm_status lbm_batch_create(void* cuda_stream, lbm_batch** out) {
  if (!out) return LBM_EINVAL;
  *out = nullptr;
  lbm_batch* b = new lbm_batch();
  b->st = (cudaStream_t)cuda_stream;
  cudaGetDevice(&b->device);
  int lo = 0, hi = 0;
  cudaDeviceGetStreamPriorityRange(&lo, &hi);
  if (cudaStreamCreateWithFlags(&b->cap, cudaStreamNonBlocking) != cudaSuccess ||
      cudaStreamCreateWithPriority(&b->aux, cudaStreamNonBlocking, hi) != cudaSuccess ||
      cudaStreamCreateWithPriority(&b->aux2, cudaStreamNonBlocking, hi) != cudaSuccess ||
      cudaEventCreateWithFlags(&b->fork, cudaEventDisableTiming) != cudaSuccess ||
      cudaEventCreateWithFlags(&b->join, cudaEventDisableTiming) != cudaSuccess ||
      cudaEventCreateWithFlags(&b->join2, cudaEventDisableTiming) != cudaSuccess) {
    lbm_batch_destroy(b);
    g_create_error = "lbm_batch_create: stream or event creation failed";
    return LBM_ECUDA;
  }
  *out = b;
  return LBM_OK;
}

lbm_status lbm_batch_set(lbm_batch* b, lbm_ctx* const* ctxs, int count) {
  if (!b || count < 0 || (count > 0 && !ctxs)) return LBM_EINVAL;
  for (int k = 0; k < count; ++k) {
    if (!ctxs[k] || !ctxs[k]->initialized) { b->err = "batch member not initialized"; return LBM_ESTATE; }
    if (ctxs[k]->device != b->device) { b->err = "batch member on another device"; return LBM_EINVAL; }
    for (int j = 0; j < k; ++j)
      if (ctxs[j] == ctxs[k]) { b->err = "context listed twice"; return LBM_EINVAL; }
  }
  if (cudaStreamSynchronize(b->st) != cudaSuccess) { b->err = "stream sync failed"; return LBM_ECUDA; }
  batch_clear(b);
  b->members.assign(ctxs, ctxs + count);
  return LBM_OK;
}

lbm_status lbm_batch_tile(lbm_batch* b, int tx, int by) {
  if (!b) return LBM_EINVAL;
  if (!((tx == 0 && by == 0) || ((tx == 32 || tx == 64 || tx == 128 || tx == 256) && by >= 1 &&
                                  tx * by <= 256))) {
    b->err = "tile: tx in {32, 64, 128, 256}, by >= 1, tx * by <= 256 (or 0, 0)";
    return LBM_EINVAL;
  }
  if (cudaStreamSynchronize(b->st) != cudaSuccess) { b->err = "stream sync failed"; return LBM_ECUDA; }
  b->tx = tx;
  b->by = by;
  batch_clear(b);
  return LBM_OK;
}

lbm_status lbm_batch_step(lbm_batch* b, int n) {
  if (!b || n < 0) return LBM_EINVAL;
  if (b->members.empty() || n == 0) return LBM_OK;
  for (lbm_ctx* c : b->members)
    if (*(volatile int*)c->hflag) { b->err = "a member flagged an unphysical state"; return LBM_EUNSTABLE; }
  lbm_ctx* ctx = b->members[0];  // for LBM_CK messages
  LBM_CK(cudaSetDevice(b->device));
  for (int k = 0; k < n; ++k) {
    // parity state of the members against the plans (a member stepped on its own since
    // then makes the states disagree: rebuild)
    int state = -1;
    if (b->built) {
      for (size_t m = 0; m < b->members.size(); ++m) {
        const int s = b->members[m]->cur != b->base[m] ? 1 : 0;
        if (state < 0) state = s;
        else if (s != state) { state = -2; break; }
      }
    }
    if (!b->built || state < 0) {
      lbm_status bs = batch_build(b);
      if (bs != LBM_OK) return bs;
      state = 0;
    }
    LBM_CK(cudaGraphLaunch(b->graph[state], b->st));
    for (lbm_ctx* c : b->members) {
      c->cur ^= 1;
      c->scur ^= 1;
      c->steps++;
      c->prev_valid = true;
      c->prev_prestream = false;
    }
  }
  return LBM_OK;
}

lbm_status lbm_batch_autotune(lbm_batch* b, int steps, int* tx_out, int* by_out) {
  if (!b || steps < 1) return LBM_EINVAL;
  if (b->members.empty()) { b->err = "empty batch"; return LBM_ESTATE; }
  lbm_ctx* ctx = b->members[0];
  LBM_CK(cudaSetDevice(b->device));
  static const int cand[][2] = {{32, 2}, {32, 4}, {32, 8}, {64, 2}, {64, 4}, {128, 1},
                                {128, 2}, {256, 1}};
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  LBM_CK(cudaEventCreate(&e0));
  cudaError_t ce = cudaEventCreate(&e1);
  if (ce != cudaSuccess) { cudaEventDestroy(e0); LBM_CK(ce); }
  float best = 1e30f;
  int bt = 32, bb = 4;
  lbm_status st = LBM_OK;
  for (const auto& c : cand) {
    b->tx = c[0];
    b->by = c[1];
    batch_clear(b);
    st = lbm_batch_step(b, 1);   // builds the plan and graphs (one untimed step)
    if (st != LBM_OK) break;
    cudaEventRecord(e0, b->st);
    st = lbm_batch_step(b, steps);
    if (st != LBM_OK) break;
    cudaEventRecord(e1, b->st);
    if (cudaEventSynchronize(e1) != cudaSuccess) { st = LBM_ECUDA; break; }
    float ms = 0.f;
    cudaEventElapsedTime(&ms, e0, e1);
    if (ms < best) { best = ms; bt = c[0]; bb = c[1]; }
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  b->tx = bt;
  b->by = bb;
  batch_clear(b);
  if (st != LBM_OK) return st;
  {
    std::lock_guard<std::mutex> lock(g_tune_mutex);
    g_tune_cache[tune_key(ctx)] = {bt, bb};
  }
  if (tx_out) *tx_out = bt;
  if (by_out) *by_out = bb;
  return LBM_OK;
}

lbm_status lbm_batch_destroy(lbm_batch* b) {
  if (!b) return LBM_OK;
  if (b->device >= 0) cudaSetDevice(b->device);
  cudaStreamSynchronize(b->st);
  batch_clear(b);
  if (b->cap) cudaStreamDestroy(b->cap);
  if (b->aux) cudaStreamDestroy(b->aux);
  if (b->aux2) cudaStreamDestroy(b->aux2);
  if (b->fork) cudaEventDestroy(b->fork);
  if (b->join) cudaEventDestroy(b->join);
  if (b->join2) cudaEventDestroy(b->join2);
  delete b;
  return LBM_OK;
}

}  // extern "C"

/*
 * lbm.h - C ABI of the GB300 PML + outer-boundary thermal lattice Boltzmann step.
 *
 * Method: Klass, Gabbana, Bartel, "Perfectly Matched Layers and Characteristic Boundaries in
 * Lattice Boltzmann: Accuracy vs. Cost" (arXiv 2504.20169).
 *   - lattice BGK step, Eq. (lbe); moments, Eq. (macro); Hermite equilibria Eqs. (feq-2..4),
 *     with the fourth-order mixed temperature term read as (c^2 - 6) (the printed (c^2 - 4)
 *     does not return the density it was built from);
 *   - PML: Eqs. (decomp-NJ), (PMLCOLL), (PML_ramp), (PMLQ) with the trapezoidal rule, gradients
 *     Eqs. (FD-dx-center) / (FD-dx-bw); optionally the general sigma_x != sigma_y form of
 *     Eq. (pml-general) and per-edge widths (closing remark of Sec. 5);
 *   - outer boundary: zero gradient, Eq. (zg-bc), or the characteristic BC of Sec. 4
 *     (Eqs. NSF-CHAR, PNR, thermal_LODI_macro_evo, thermal_CBC_macro_evo, CBC-Relax) with
 *     non-equilibrium extrapolation, optionally with the PML source terms of the Appendix
 *     (Eq. NSF-CHAR-PML); a periodic y axis for the Sec. 5.1 setting.
 *
 * Geometry. Bulk nx x ny nodes; W PML layers on every side give the fluid region F of
 * Lx x Ly = (nx + 2W) x (ny + 2W) nodes (Fig. 2) (with per-edge widths, see lbm_bc_params:
 * Lx = nx + W_w + W_e, Ly = ny + W_s + W_n); M boundary layers outside F (M = 3 for D2Q37
 * and D2Q17, 1 for D2Q9) hold the boundary nodes x_(b,j) of Sec. 4. Field arrays passed through
 * this ABI are float64, row-major with y outer: element (y, x) at index y * Lx + x over F, or
 * y * nx + x over the bulk.
 *
 * Units. Normalized Hermite units of the equilibria: c_s = 1, reference temperature 1, velocity
 * in units of c_s. The lattice moves e_i (integer) nodes per step with xi_i = r e_i, so one node
 * is r normalized lengths; lbm_lattice_info returns r.
 *
 * Conventions. Every call returns an lbm_status and never aborts. The library owns all device
 * memory of a context; the caller owns every pointer it passes. Work is queued on the context's
 * CUDA stream; calls that return host data synchronize that stream. A context is not
 * thread-safe; separate contexts are independent. After LBM_EUNSTABLE the context is poisoned:
 * lbm_moments, lbm_export_populations, lbm_last_error and lbm_destroy still work.
 */
#ifndef LBM_H
#define LBM_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct lbm_ctx lbm_ctx;

typedef enum {
  LBM_OK = 0,
  LBM_EINVAL = 1,     /* invalid argument or combination; nothing allocated */
  LBM_ENOMEM = 2,     /* device or pinned allocation failed */
  LBM_ECUDA = 3,      /* a CUDA call failed; lbm_last_error has the message */
  LBM_EUNSTABLE = 4,  /* a non-finite or non-positive density / temperature was produced */
  LBM_ETIMEOUT = 5,   /* reserved: no kernel of this library waits on another, so no call
                          returns it */
  LBM_ESTATE = 6      /* call not valid in the context's state (e.g. step before init) */
} lbm_status;

/* Velocity stencils of Sec. 2 (Fig. 1): q velocities; equilibrium order 2 / 3 / 4. */
typedef enum { LBM_D2Q9 = 9, LBM_D2Q17 = 17, LBM_D2Q37 = 37 } lbm_stencil;

/* Outer boundary of the PML-extended grid. PERIODIC is the fully periodic reference mode of
 * Sec. 5 ("Reference Simulation") and requires pml_width == 0. */
typedef enum { LBM_BC_PERIODIC = 0, LBM_BC_ZG = 1, LBM_BC_NRBC = 2 } lbm_bc_kind;

/* Characteristic BC variant per edge (Sec. 4, Sec. 5.2):
 * PNR_LODI   incoming amplitudes zero, Eq. (PNR), LODI evolution Eq. (thermal_LODI_macro_evo);
 * CBC_RELAX  incoming amplitudes relaxed against the transverse terms, Eq. (CBC-Relax), with
 *            the CBC evolution Eq. (thermal_CBC_macro_evo). Reading of the printed sign: the
 *            incoming amplitude is relax_sign * (1 - beta) * T_inc, relax_sign = -1 by default
 *            (beta = 1 leaves the transverse term, beta = 0 freezes the incoming wave). */
typedef enum { LBM_NRBC_PNR_LODI = 0, LBM_NRBC_CBC_RELAX = 1 } lbm_nrbc_variant;

typedef enum { LBM_FP64 = 0, LBM_FP32_DEV = 1 } lbm_precision;

typedef struct { int nx, ny; } lbm_grid;

/* Eq. (PML_ramp): sigma = sigma_max (i / W)^power on PML layer i = 1..W of an edge of width W
 * (power 2 in the paper); a node's layer fraction along an axis is i / W of the nearer edge.
 * split = 0: sigma_x = sigma_y = sigma(max(f_x, f_y)), Eq. (PMLCOLL) (the paper's choice;
 * corners by the larger fraction). split = 1: the general form of Eq. (pml-general) with
 * sigma_x = sigma(f_x), sigma_y = sigma(f_y), each zero outside the slab of its own axis. */
typedef struct { double sigma_max; int power; int split; } lbm_sigma_profile;

typedef struct {
  int edge[4];                  /* lbm_nrbc_variant for the W, E, S, N edges               */
  double beta;                  /* relaxation Mach number "Ma" of Eq. (CBC-Relax)            */
  double relax_sign;            /* -1 (default reading) or +1 (as printed); 0 means -1      */
  double rho0, u0x, u0y, T0;    /* mean state: f_eq_bar of the PML (Eq. decomp-NJ)          */
  int use_pml_widths;           /* 0: pml_width on every edge; 1: pml_widths below          */
  int pml_widths[4];            /* PML layers on the W, E, S, N edges (0 or 2..4096); thin  */
                                /* layers away from the outlet (closing remark of Sec. 5)   */
  int pml_source;               /* bitmask, LBM_BC_NRBC with a PML only: add the PML source */
                                /* terms I (1), II (2), III (4) of Eq. (NSF-CHAR-PML)       */
                                /* (Appendix) to the characteristic targets: the moments of  */
                                /* those parts of Omega^PML at the outermost fluid node      */
                                /* (0: the characteristic BC of Sec. 4); adding 8 takes the  */
                                /* "+" printed in Eq. (NSF-CHAR-PML) instead of the sign of  */
                                /* the collision term                                        */
  int periodic_y;               /* 1: the y axis is periodic (Sec. 5.1 setting): no S / N    */
                                /* boundary and no PML there (with use_pml_widths = 0 the    */
                                /* S / N widths are taken as 0; otherwise they must be 0)    */
  int pml_grad;                 /* 0: c_i . grad Q_i of Eq. (PMLCOLL) by the printed per-axis */
                                /* differences, Eqs. (FD-dx-center) / (FD-dx-bw) (default).  */
                                /* 1: by the link difference Q_i(x + e_i) - Q_i(x), the     */
                                /* integral of c_i . grad Q_i along the path the population  */
                                /* travels in one step. Not the paper's printed scheme: an   */
                                /* option, because the printed differences let grid-scale    */
                                /* modes grow for every sigma > 0 (fast for D2Q37), while    */
                                /* the link form stays stable. Q is then also integrated on  */
                                /* the M-node bulk ring next to the PML and on every boundary */
                                /* node outside F. Needs split = 0 (sigma_x = sigma_y).      */
} lbm_bc_params;

/* Create a context. tau > 1/2 (tau = +INFINITY gives collisionless free streaming);
 * pml_width 0 or 2..4096 (the one-sided gradient reaches two nodes inward); bc_params may be
 * NULL for the rest state (1, 0, 0, 1), PNR_LODI on every edge and pml_width on every edge.
 * cuda_stream is a cudaStream_t (NULL = the legacy default stream). Allocates the populations
 * (2 x q x |grid| values of the precision), the PML accumulator on the PML and its inner
 * ring, the boundary targets and the edge moments / sources (lbm_estimate_bytes gives the
 * total). On failure *out is NULL and nothing stays allocated. */
lbm_status lbm_create(const lbm_grid* grid, lbm_stencil stencil, double tau, int pml_width,
                      const lbm_sigma_profile* sigma, lbm_bc_kind bc, const lbm_bc_params* bc_params,
                      lbm_precision precision, void* cuda_stream, lbm_ctx** out);

/* Initialize from macroscopic fields over F (Lx * Ly float64 each, layout above):
 * f^0 = f_eq(fields) (Sec. 2), Q^0 = 0, boundary targets = fields at the nearest fluid node.
 * fields_on_device != 0: the four pointers are device pointers; else host pointers (copied
 * through the library's staging buffer, synchronizing the stream). */
lbm_status lbm_init(lbm_ctx* ctx, const double* rho, const double* ux, const double* uy,
                    const double* T, int fields_on_device);

/* Advance n >= 0 time steps (collide with PML, stream, boundary). Asynchronous on the
 * context stream. Returns LBM_EUNSTABLE if an earlier step has already flagged an unphysical
 * state (the flag lives in mapped host memory and is read without synchronizing). */
lbm_status lbm_step(lbm_ctx* ctx, int n);

/* Wait for queued work; returns LBM_EUNSTABLE if any step flagged an unphysical state. */
lbm_status lbm_sync(lbm_ctx* ctx);

/* Macroscopic fields rho, u_x, u_y, T of the current time level over F (region 1) or the bulk
 * (region 0), float64, layout above. out_on_device != 0: device pointers. Any output pointer may
 * be NULL. Synchronizes the stream. */
lbm_status lbm_moments(lbm_ctx* ctx, double* rho, double* ux, double* uy, double* T, int region,
                       int out_on_device);

/* Conserved totals over F at the current time level, FP64 reduction on the device:
 * out[0] = sum rho, out[1] = sum rho u_x, out[2] = sum rho u_y, out[3] = sum (1/2) sum_i f_i |xi_i|^2,
 * out[4] = min rho, out[5] = min T, out[6] = number of non-finite or non-positive rho or T.
 * out is a host array of 7 doubles. Synchronizes. */
lbm_status lbm_reduce(lbm_ctx* ctx, double* out);

/* Error sums against reference fields over the bulk (Sec. 5 metrics), FP64 on the device.
 * ref: four device arrays (rho, u_x, u_y, T) of nx * ny float64. out (host, 12 doubles): for
 * each field Z in that order, out[3k] = sum (Z - Zref)^2, out[3k+1] = sum Zref^2,
 * out[3k+2] = sum ((Z - Zref) / Zref)^2 (the square of e_Z). Synchronizes. */
lbm_status lbm_error_sums(lbm_ctx* ctx, const double* ref_rho, const double* ref_ux,
                          const double* ref_uy, const double* ref_T, double* out);

/* Velocity set and quadrature derived by the library (Sec. 2). Host-only, needs no GPU.
 * e: 2*q ints (ex, ey per velocity), w: q doubles, r: scale. Any output may be NULL. */
lbm_status lbm_lattice_info(lbm_stencil stencil, int* q, int* e, double* w, double* r);

/* Grid description of a context: out[0..11] = nx, ny, W (of the W edge), M, Lx, Ly, q, step
 * count, then the PML widths of the W, E, S, N edges. Lx = nx + W_w + W_e, Ly = ny + W_s + W_n;
 * the bulk starts at (W_w, W_s) of F. */
lbm_status lbm_geometry(const lbm_ctx* ctx, int64_t* out);

/* Debugging aid (no counterpart in the paper; stands in for a memory checker). Every device
 * buffer a context allocates sits between two 256-byte guard bands filled with 0xA5 at
 * creation. Synchronizes the context stream and sets *intact = 1 if every guard band still
 * holds its pattern, 0 if a kernel wrote outside a buffer. Test hook: if the environment
 * variable LBM_DEBUG_ALLOC_BUDGET holds a byte count when lbm_create runs, allocations beyond
 * that many payload bytes fail as if the device were out of memory (LBM_ENOMEM, nothing left
 * allocated). */
lbm_status lbm_debug_check_guards(lbm_ctx* ctx, int* intact);

/* Debug / checkpoint: the stored post-collision populations of the last completed step (or
 * of the initial collision) on the whole grid G = (Lx + 2M) x (Ly + 2M), as float64 absolute
 * populations, layout [i][gy][gx]; host buffer of q * Gx * Gy doubles. Synchronizes. */
lbm_status lbm_export_populations(lbm_ctx* ctx, double* host);
/* Replace the stored post-collision populations (same layout); the PML accumulator and the
 * boundary targets are left as they are. Intended for bit-exact streaming tests. */
lbm_status lbm_import_populations(lbm_ctx* ctx, const double* host);

/* Full checkpoint of a context (populations, PML accumulator, boundary targets and moments,
 * step count) into a host buffer. lbm_checkpoint_size gives the byte count. A context restored
 * with lbm_restore into an identically created context continues bit-identically. */
lbm_status lbm_checkpoint_size(const lbm_ctx* ctx, size_t* bytes);
lbm_status lbm_checkpoint(lbm_ctx* ctx, void* host, size_t bytes);
lbm_status lbm_restore(lbm_ctx* ctx, const void* host, size_t bytes);

/* Per-kernel timing (tracing). lbm_profile_enable(ctx, max_steps) makes the next max_steps
 * steps record CUDA events on the context stream around each kernel class: 0 characteristic
 * targets, 1 interior (BGK only), 2 PML frame phase 1, 3 PML frame phase 2, 4 boundary band;
 * max_steps = 0 disables. Recorded steps are launched directly with every class running alone
 * (no concurrency between the interior kernel and the boundary chain), so each class's time
 * is its own; unrecorded steps keep the concurrent graph replay. lbm_profile_read synchronizes, writes the summed GPU milliseconds of
 * each class into ms[5] and the number of recorded steps into *steps, and restarts recording. */
lbm_status lbm_profile_enable(lbm_ctx* ctx, int max_steps);
lbm_status lbm_profile_read(lbm_ctx* ctx, double* ms, int* steps);

/* Device bytes lbm_create would allocate for these arguments (no allocation, no GPU needed);
 * used for admission by HBM budget. Returns LBM_EINVAL for arguments lbm_create rejects. */
lbm_status lbm_estimate_bytes(const lbm_grid* grid, lbm_stencil stencil, int pml_width,
                              lbm_bc_kind bc, lbm_precision precision, size_t* bytes);

/* Same as lbm_estimate_bytes for the full set of lbm_create arguments that shape the grid:
 * per-edge PML widths and the periodic y axis (bc_params->use_pml_widths, pml_widths,
 * periodic_y) and the link gradient's wider accumulator (bc_params->pml_grad); sigma and
 * bc_params may be NULL as in lbm_create. Runs lbm_create's argument checks (LBM_EINVAL with
 * lbm_last_error(NULL) set for arguments lbm_create rejects); no allocation, no GPU needed. */
lbm_status lbm_estimate_bytes_bc(const lbm_grid* grid, lbm_stencil stencil, int pml_width,
                                 const lbm_sigma_profile* sigma, lbm_bc_kind bc,
                                 const lbm_bc_params* bc_params, lbm_precision precision,
                                 size_t* bytes);

/* Diagnostic exports for bit-exact tests of the index maps (no counterpart in the paper; the
 * maps are those of Eq. (lbe) and of Eqs. (PML_ramp), (pml-general)). Neither needs lbm_init.
 * lbm_export_pull_index: for every direction i and node (x, y) of F, the grid-G index
 * gy * (Lx + 2M) + gx of the node the pull of direction i reads, x - e_i, as the kernels compute
 * it (G coordinates: gx = x + M, gy = y + M); host buffer of q * Lx * Ly int64, layout
 * [i][y][x]. lbm_export_site_class: per node of F (host buffers of Lx * Ly, layout [y][x], any
 * may be NULL): layer = the PML layer index max(i_x, i_y) (0 in the bulk), has_q = 1 where the
 * PML accumulator Q is kept (P and its inner ring), sigma_x / sigma_y = the absorption
 * coefficients the collision applies (0 off P). Both allocate a temporary device buffer and
 * synchronize the context stream. */
lbm_status lbm_export_pull_index(lbm_ctx* ctx, int64_t* host);
lbm_status lbm_export_site_class(lbm_ctx* ctx, int32_t* layer, uint8_t* has_q, double* sigma_x,
                                 double* sigma_y);

/* Measured vector FMA throughput of the current CUDA device (no counterpart in the paper: the
 * ALU roofline of the FP64 path, whose interior kernel is bound by the FP64 pipe). precision
 * LBM_FP64 times double FMAs, LBM_FP32_DEV float FMAs: every SM filled with threads running
 * eight independent FMA chains, one warm-up launch, then one timed launch (CUDA events on
 * cuda_stream, a cudaStream_t or NULL). *tflops = 2 x FMAs / time, *ms = the timed launch
 * (ms may be NULL). Synchronizes; errors by lbm_last_error(NULL). */
lbm_status lbm_peak_fma(lbm_precision precision, double* tflops, double* ms, void* cuda_stream);

/* Batched execution of independent instances (serving). A batch holds a resident set of
 * initialized contexts on one device and advances all of them together. Members are grouped
 * by (stencil, precision, PML gradient mode); within a group every kernel class (characteristic
 * targets, interior, PML frame, boundary band, periodic row copies) is one launch whose blocks
 * walk a table of (member, tile) entries spanning all members of the group, so instances of
 * different sizes, PML widths and boundary conditions share each launch and fill the GPU
 * together; one step of the whole batch is one CUDA-graph launch on the batch's stream. Each
 * block runs the same per-node code as lbm_step, so every member computes bit for bit what it
 * computes alone, whatever the tile shape. lbm_batch_set replaces the resident set (continuous
 * batching: call it between steps as instances are admitted or retired; the plans and graphs are
 * rebuilt on the next step, as they are when a member was stepped on its own in between).
 * lbm_batch_step returns LBM_EUNSTABLE without stepping anyone if a member has flagged an
 * unphysical state (find it with lbm_sync, drop it with lbm_batch_set). The batch does not own
 * its members; destroy a context only after removing it from every batch.
 * lbm_batch_tile sets the interior kernel's block shape tx x by (tx in {32, 64, 128, 256},
 * by >= 1, tx * by <= 256; 0, 0 = the tuned shape for this stencil, precision and device if
 * one was found in this process, else 32 x 4). lbm_batch_autotune times `steps` batch steps
 * with each of the candidate shapes 32x2, 32x4, 32x8, 64x2, 64x4, 128x1, 128x2, 256x1 (one
 * untimed step each to build them), keeps the fastest for this batch, records it for
 * (stencil, precision, PML gradient mode, device name) for later batches of the process, and
 * returns it in *tx, *by (either may be NULL). Tuning steps are real steps: every member
 * advances by 8 (steps + 1); the shape never changes the results. */
typedef struct lbm_batch lbm_batch;
lbm_status lbm_batch_create(void* cuda_stream, lbm_batch** out);
lbm_status lbm_batch_set(lbm_batch* batch, lbm_ctx* const* ctxs, int count);
lbm_status lbm_batch_step(lbm_batch* batch, int n);
lbm_status lbm_batch_tile(lbm_batch* batch, int tx, int by);
lbm_status lbm_batch_autotune(lbm_batch* batch, int steps, int* tx, int* by);
lbm_status lbm_batch_destroy(lbm_batch* batch);

/* Conserved totals of macroscopic fields that the caller already holds on the device, computed
 * without allocating anything. The paper has no counterpart: this exists for callers that cannot
 * call cudaMalloc - code running while a CUDA graph is captured, plugins inside an application
 * that owns all device memory through its own pool, processes with a fixed memory budget.
 * rho, ux, uy, T: device arrays of n float64 values each (e.g. the fields of lbm_moments);
 * out: device array of 7 float64 written with the same quantities as lbm_reduce (sum rho,
 * sum rho u_x, sum rho u_y, sum (1/2) rho (|u|^2 + 2 T), min rho, min T, count of non-finite or
 * non-positive rho / T). n must be 1 .. LBM_TOTALS_NOALLOC_MAX_N, else LBM_EINVAL.
 * The per-block partial sums live in one fixed 64 KiB device array of the library (1024 blocks
 * x 8 doubles), which every GPU that loads the library keeps until the process exits; every
 * call on a device shares it and rewrites all the slots it uses, so nothing needs clearing, but
 * calls that overlap on the GPU (other streams, other threads) race on it. The first call on a
 * device looks up the array's device address (cudaGetSymbolAddress) with that device current:
 * make that first call before any stream capture. The looked-up address is kept for the life of
 * the process, so do not call this after cudaDeviceReset of that device (the module, and with it
 * the array, may then sit elsewhere). No cudaMalloc, cudaFree or allocating library
 * routine is called. Asynchronous on cuda_stream (a cudaStream_t, NULL = legacy default stream).
 * Errors are reported by lbm_last_error(NULL). */
#define LBM_TOTALS_NOALLOC_MAX_N ((int64_t)1 << 28)
lbm_status lbm_totals_noalloc(const double* rho, const double* ux, const double* uy,
                              const double* T, int64_t n, double* out, void* cuda_stream);

/* Last error message of the context (or of the last failed lbm_create when ctx is NULL). */
const char* lbm_last_error(const lbm_ctx* ctx);

/* Release everything; NULL is allowed. */
lbm_status lbm_destroy(lbm_ctx* ctx);

#ifdef __cplusplus
}
#endif
#endif /* LBM_H */

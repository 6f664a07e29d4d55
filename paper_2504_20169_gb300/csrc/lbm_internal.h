// Host-side plumbing shared by the translation units of liblbm (not part of the C ABI).
#pragma once
#include <string>

#include <cuda_runtime.h>

#include "lbm_device.cuh"

namespace lbm {

// Everything a launch needs: geometry, constants, the current buffer roles, the stream.
struct Dev {
  Geom g;
  BcParams bc;
  Consts<double> cd;
  Consts<float> cf;
  const void* A;     // post-collision populations of the current level (read)
  void* B;           // next level (written)
  void* Sold;        // PML accumulator S^(n-1) (link mode: Q^n in place during the step)
  void* Snew;        // S^n
  double* Vtgt;      // characteristic targets U_tgt [4][nb]
  double* Va;        // Runge-Kutta stage buffers [4][nb]
  double* Vb;
  double* Vacc;
  // fluid moments of the outer two layers of F [4][ne], two buffers: the characteristic
  // targets read the level-n moments (Uedge_in, written by the previous step's frame) while
  // this step's frame writes the next level's (Uedge_out), so the two can run concurrently
  const double* Uedge_in;
  double* Uedge_out;
  // Appendix PML source (mass, momentum, energy rates) at the outermost fluid node of every
  // edge position [4][2 (Lx + Ly)], double-buffered like Uedge
  const double* Sedge_in;
  double* Sedge_out;
  int* flag;         // device-visible address of the mapped "unphysical state" flag
  cudaStream_t st;
  // Boundary-side work runs forked from and joined back into st, concurrently with the
  // interior kernel on st: the characteristic targets and then the boundary band on aux, the
  // PML frame on aux2 (both may be null: everything then runs in order on st).
  cudaStream_t aux, aux2;
  cudaEvent_t fork, join, join2;
  // optional timing: when ev is set, event 2k / 2k+1 are recorded around kernel class k
  // (0 characteristic targets, 1 interior, 2 frame phase 1, 3 frame phase 2, 4 boundary band)
  cudaEvent_t* ev;
  // the context's one-member batch plan (its descriptors for buffer parity 0 and 1) and the
  // parity of this launch; streaming steps run the boundary-side classes through it
  const struct BatchPlan* plan;
  int which;
};

constexpr int kKernelClasses = 5;

// Characteristic-target work of one batch member (the batched RK4 launch).
struct TgtDesc {
  Geom g;
  BcParams bc;
  const double* Ue;
  const double* Se;
  double* V;
};

// Work list of a batch of instances with the same stencil, precision and PML gradient mode:
// one launch per kernel class over a table of (member, tile / block) entries that spans all
// instances (see lbm_batch_step). The member descriptors exist for the two buffer-parity
// states the batch alternates between; everything lives in one device allocation.
struct BatchPlan {
  int n = 0;                  // members
  void* desc[2] = {nullptr, nullptr};   // member descriptors, parity state 0 / 1
  TgtDesc* tgt[2] = {nullptr, nullptr};
  int* bulk_tab = nullptr;    // (member, bx, by)
  int* frame_tab = nullptr;   // fused FP32 frame tiles: (member, tile)
  int* f1_tab = nullptr;      // frame phase 1 blocks of 128 nodes: (member, block)
  int* f2_tab = nullptr;      // frame phase 2 blocks (members with a PML): (member, block)
  int* band_tab = nullptr;    // boundary-band blocks of 128 nodes: (member, block)
  int* tgt_tab = nullptr;     // characteristic-target chunks: (member, chunk)
  int* wrap_tab = nullptr;    // periodic-y row copies, blocks of 256: (member, block)
  int n_bulk = 0, n_frame = 0, n_f1 = 0, n_f2 = 0, n_band = 0, n_tgt = 0, n_wrap = 0;
  size_t frame_smem = 0, tgt_smem = 0;
  int tgt_threads = 0, q = 0;
  int tx = 32, by = 4;        // bulk tile shape (blockDim)
  bool link = false;
  void* mem = nullptr;
};

struct OpsTable {
  cudaError_t (*prepare)(const double* w);   // kernel attributes and the quadrature weights
                                             // (constant memory) on the current device
  cudaError_t (*step)(const Dev&, bool stream);
  cudaError_t (*init_eq)(const Dev&, const double*, const double*, const double*, const double*);
  cudaError_t (*fields)(const Dev&, const void* src, bool stream, int region, double* const o[4],
                        const double* const r[4], int mode, double* partials, int* nblocks);
  cudaError_t (*export_pop)(const Dev&, const void* src, double* out);
  cudaError_t (*import_pop)(const Dev&, const double* in, void* dst);
  int elem_size;
  // batched execution (lbm_batch): build the plan of n members from their launch state in
  // the two parity states (dev0[m], dev1[m]), launch one step of parity state `which`
  // (boundary-side work forked onto aux / aux2 and joined back into st), free the plan
  cudaError_t (*batch_plan)(const Dev* const* dev0, const Dev* const* dev1, int n, int tx,
                            int by, BatchPlan* plan);
  cudaError_t (*batch_step)(const BatchPlan& plan, int which, cudaStream_t st, cudaStream_t aux,
                            cudaStream_t aux2, cudaEvent_t fork, cudaEvent_t join,
                            cudaEvent_t join2);
};

void batch_plan_free(BatchPlan* plan);

// Launch shape of the characteristic-target kernel of one grid: chunks (blocks), threads per
// block, dynamic shared memory.
void nrbc_shape(const Geom& g, int* chunks, int* threads, size_t* smem);

// Batched characteristic targets: one block per table entry (member, chunk).
cudaError_t launch_nrbc_batch(const TgtDesc* d, const int* tab, int n, bool fp32, int threads,
                              size_t smem, cudaStream_t s);

OpsTable ops_q37_f64();
OpsTable ops_q37_f32();
OpsTable ops_q17_f64();
OpsTable ops_q17_f32();
OpsTable ops_q9_f64();
OpsTable ops_q9_f32();

// Characteristic-target RK4 stages of one step on stream s; fp32 selects FP32 characteristic
// algebra (targets and differences stay FP64).
cudaError_t launch_nrbc_stages(const Dev& d, bool fp32, cudaStream_t s);

// Message returned by lbm_last_error(NULL) (calls without a context).
void set_global_error(const std::string& msg);

// Final pass of the deterministic two-pass FP64 reduction: n partial rows of 12 values ->
// out[12] (slots in min_mask take the minimum).
cudaError_t reduce_partials(const double* partials, int n, unsigned min_mask, double* out,
                            cudaStream_t st);

}  // namespace lbm

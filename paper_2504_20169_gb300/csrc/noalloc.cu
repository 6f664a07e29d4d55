// Allocation-free variant of the conserved-totals reduction (lbm_totals_noalloc in lbm.h).
//
// Some callers cannot call cudaMalloc at all: code running while a CUDA graph is being
// captured, plugins hosted by an application that owns every allocation through its own pool,
// and processes whose device memory budget is fixed before they start. This entry point lets
// them reduce fields they already hold without the library allocating anything: the per-block
// partial sums live in the fixed array below, which every GPU that loads this library keeps
// until the process exits.
#include <cfloat>
#include <cstdint>
#include <mutex>
#include <string>

#include "../../include/lbm.h"
#include "lbm_internal.h"

namespace {

constexpr int kBlocks = 1024;          // maximum blocks of the first pass
constexpr int kThreads = 256;
constexpr int kSlots = 8;              // partial values per block
constexpr int kMaxDevices = 64;

// The scratch of every call on a device: kBlocks x kSlots doubles (64 KiB). In host code this
// name is only a stand-in for the device symbol; kernels receive its device address, looked up
// once per device with cudaGetSymbolAddress.
static __device__ __align__(256) double g_totals_scratch[kBlocks * kSlots];

std::mutex g_mutex;
double* g_scratch_ptr[kMaxDevices] = {};

__device__ inline void reduce_slot(double& a, double b, int k) {
  a = (k == 4 || k == 5) ? fmin(a, b) : a + b;
}

__global__ void k_totals_pass1(const double* __restrict__ rho, const double* __restrict__ ux,
                               const double* __restrict__ uy, const double* __restrict__ T,
                               long long n, double* __restrict__ scratch) {
  double v[kSlots] = {0, 0, 0, 0, DBL_MAX, DBL_MAX, 0, 0};
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n;
       i += (long long)gridDim.x * blockDim.x) {
    const double r = rho[i], a = ux[i], b = uy[i], t = T[i];
    v[0] += r;
    v[1] += r * a;
    v[2] += r * b;
    v[3] += 0.5 * r * (a * a + b * b + 2.0 * t);
    v[4] = fmin(v[4], r);
    v[5] = fmin(v[5], t);
    v[6] += (r > 0.0 && t > 0.0 && r < 1e30 && t < 1e30) ? 0.0 : 1.0;
  }
  __shared__ double sh[kThreads / 32][kSlots];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
  for (int k = 0; k < kSlots; ++k) {
    for (int o = 16; o > 0; o >>= 1) reduce_slot(v[k], __shfl_down_sync(0xffffffffu, v[k], o), k);
    if (lane == 0) sh[warp][k] = v[k];
  }
  __syncthreads();
  if (threadIdx.x < kSlots) {
    const int k = threadIdx.x;
    double a = sh[0][k];
    for (int w = 1; w < kThreads / 32; ++w) reduce_slot(a, sh[w][k], k);
    scratch[blockIdx.x * kSlots + k] = a;   // every used slot is rewritten on each call
  }
}

__global__ void k_totals_pass2(const double* __restrict__ scratch, int nblocks,
                               double* __restrict__ out) {
  if (threadIdx.x >= kSlots) return;
  const int k = threadIdx.x;
  double a = scratch[k];
  for (int b = 1; b < nblocks; ++b) reduce_slot(a, scratch[b * kSlots + k], k);
  if (k < 7) out[k] = a;
}

// Device address of the scratch on the current device; looked up on the first call there.
lbm_status scratch_of_current_device(double** ptr) {
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) {
    lbm::set_global_error("lbm_totals_noalloc: no usable current device");
    return LBM_ECUDA;
  }
  std::lock_guard<std::mutex> lock(g_mutex);
  if (!g_scratch_ptr[dev]) {
    void* p = nullptr;
    const cudaError_t e = cudaGetSymbolAddress(&p, g_totals_scratch);
    if (e != cudaSuccess || !p) {
      lbm::set_global_error(std::string("lbm_totals_noalloc: cudaGetSymbolAddress failed: ") +
                            cudaGetErrorString(e));
      return LBM_ECUDA;
    }
    g_scratch_ptr[dev] = static_cast<double*>(p);
  }
  *ptr = g_scratch_ptr[dev];
  return LBM_OK;
}

}  // namespace

extern "C" lbm_status lbm_totals_noalloc(const double* rho, const double* ux, const double* uy,
                                         const double* T, int64_t n, double* out,
                                         void* cuda_stream) {
  if (!rho || !ux || !uy || !T || !out || n <= 0) {
    lbm::set_global_error("lbm_totals_noalloc: NULL pointer or empty field");
    return LBM_EINVAL;
  }
  if (n > LBM_TOTALS_NOALLOC_MAX_N) {
    lbm::set_global_error("lbm_totals_noalloc: n exceeds LBM_TOTALS_NOALLOC_MAX_N (2^28 nodes)");
    return LBM_EINVAL;
  }
  double* scratch = nullptr;
  const lbm_status s = scratch_of_current_device(&scratch);
  if (s != LBM_OK) return s;
  const cudaStream_t st = static_cast<cudaStream_t>(cuda_stream);
  const long long want = (n + kThreads - 1) / kThreads;
  const int blocks = (int)(want < kBlocks ? want : kBlocks);
  k_totals_pass1<<<blocks, kThreads, 0, st>>>(rho, ux, uy, T, (long long)n, scratch);
  k_totals_pass2<<<1, 32, 0, st>>>(scratch, blocks, out);
  const cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) {
    lbm::set_global_error(std::string("lbm_totals_noalloc: launch failed: ") +
                          cudaGetErrorString(e));
    return LBM_ECUDA;
  }
  return LBM_OK;
}


// Vector FMA throughput of the current device (lbm_peak_fma in lbm.h): the ALU roofline of
// the FP64 path, whose interior kernel is bound by the FP64 pipe rather than by HBM.
//
// Every thread runs eight independent fused multiply-add chains a = a * b + c (enough
// independent work per warp to keep the pipe busy); the grid fills every SM to its thread
// limit. FLOPs = threads x iterations x 8 chains x 2. The chains' sum is compared against a
// value it never takes, so the compiler cannot drop them.
#include <string>

#include "../../include/lbm.h"
#include "lbm_internal.h"

namespace {

static __device__ double g_fma_sink[2];

template <class T>
__global__ void __launch_bounds__(256) k_fma_chains(int iters, T seed) {
  const T b = T(0.9999999), c = T(1e-7);
  T a[8];
#pragma unroll
  for (int k = 0; k < 8; ++k) a[k] = seed + T(threadIdx.x + k) * T(1e-6);
  for (int n = 0; n < iters; ++n) {
#pragma unroll
    for (int k = 0; k < 8; ++k) a[k] = fma(a[k], b, c);
  }
  T s = T(0);
#pragma unroll
  for (int k = 0; k < 8; ++k) s += a[k];
  if (s == T(-12345.0)) g_fma_sink[sizeof(T) == 8 ? 0 : 1] = double(s);
}

template <class T>
cudaError_t run(int iters, cudaStream_t st, int blocks, float* ms) {
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  cudaError_t e = cudaEventCreate(&e0);
  if (e == cudaSuccess) e = cudaEventCreate(&e1);
  if (e == cudaSuccess) {
    k_fma_chains<T><<<blocks, 256, 0, st>>>(iters / 16 + 1, T(1));   // warm-up
    cudaEventRecord(e0, st);
    k_fma_chains<T><<<blocks, 256, 0, st>>>(iters, T(1));
    cudaEventRecord(e1, st);
    e = cudaGetLastError();
  }
  if (e == cudaSuccess) e = cudaEventSynchronize(e1);
  if (e == cudaSuccess) e = cudaEventElapsedTime(ms, e0, e1);
  if (e0) cudaEventDestroy(e0);
  if (e1) cudaEventDestroy(e1);
  return e;
}

}  // namespace

extern "C" lbm_status lbm_peak_fma(lbm_precision precision, double* tflops, double* ms,
                                   void* cuda_stream) {
  if (!tflops || (precision != LBM_FP64 && precision != LBM_FP32_DEV)) {
    lbm::set_global_error("lbm_peak_fma: bad precision or NULL output");
    return LBM_EINVAL;
  }
  int dev = 0, sms = 0, tpm = 0;
  if (cudaGetDevice(&dev) != cudaSuccess ||
      cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess ||
      cudaDeviceGetAttribute(&tpm, cudaDevAttrMaxThreadsPerMultiProcessor, dev) != cudaSuccess) {
    lbm::set_global_error("lbm_peak_fma: no CUDA device");
    return LBM_ECUDA;
  }
  const int blocks = sms * (tpm / 256);
  // about 50-100 ms per timed launch at the nominal rates (FP64 ~1 TFLOP/s, FP32 ~80)
  const int iters = precision == LBM_FP64 ? 12000 : 600000;
  float t = 0.f;
  const cudaError_t e = precision == LBM_FP64
                            ? run<double>(iters, (cudaStream_t)cuda_stream, blocks, &t)
                            : run<float>(iters, (cudaStream_t)cuda_stream, blocks, &t);
  if (e != cudaSuccess) {
    lbm::set_global_error(std::string("lbm_peak_fma: ") + cudaGetErrorString(e));
    return LBM_ECUDA;
  }
  const double flops = double(blocks) * 256.0 * double(iters) * 8.0 * 2.0;
  *tflops = flops / (double(t) * 1e-3) / 1e12;
  if (ms) *ms = t;
  return LBM_OK;
}

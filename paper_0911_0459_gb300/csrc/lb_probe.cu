// Device rate diagnostics: the FP64 fused multiply-add throughput of this GPU.
//
// The liquid-gas model runs in FP64 (its densities near 4 leave FP32 too few
// bits for the coexistence pins), and GB300's FP64 rate is a small fraction of
// its FP32 rate, so that path is bound by FP64 arithmetic before HBM.  This
// measures the ceiling its roofline is quoted against.
#include <cuda_runtime.h>

#include "lb.h"

namespace {

constexpr int kChains = 8;        // independent FMA chains per thread
constexpr int kThreads = 256;
constexpr int kBlocksPerSM = 8;

__global__ void __launch_bounds__(kThreads) fp64_fma_kernel(double* out, int iters, double a, double b) {
  double x[kChains];
#pragma unroll
  for (int k = 0; k < kChains; ++k) x[k] = 1e-3 * (threadIdx.x + 1) + k;
  for (int i = 0; i < iters; ++i) {
#pragma unroll
    for (int k = 0; k < kChains; ++k) x[k] = fma(x[k], a, b);
  }
  double s = 0.0;
#pragma unroll
  for (int k = 0; k < kChains; ++k) s += x[k];
  if (s == -1.0) out[blockIdx.x] = s;  // never true: keeps the chains live
}

}  // namespace

extern "C" lb_status lb_fp64_fma_rate(void* stream, double* tflops) {
  if (!tflops) return LB_ERR_ARG;
  *tflops = 0.0;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  int dev = 0, sms = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) !=
                                                cudaSuccess)
    return LB_ERR_CUDA;
  const int grid = sms * kBlocksPerSM;
  const int iters = 2048;
  double* out = nullptr;
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  cudaError_t e = cudaMalloc(&out, sizeof(double) * grid);
  if (e == cudaSuccess) e = cudaEventCreate(&e0);
  if (e == cudaSuccess) e = cudaEventCreate(&e1);
  float best = 0.f;
  // a warm-up launch, then the best of three timed launches
  for (int r = 0; r < 4 && e == cudaSuccess; ++r) {
    e = cudaEventRecord(e0, s);
    if (e == cudaSuccess) {
      fp64_fma_kernel<<<grid, kThreads, 0, s>>>(out, iters, 0.9999999, 1e-9);
      e = cudaGetLastError();
    }
    if (e == cudaSuccess) e = cudaEventRecord(e1, s);
    if (e == cudaSuccess) e = cudaEventSynchronize(e1);
    float ms = 0.f;
    if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
    if (e == cudaSuccess && r > 0 && (best == 0.f || ms < best)) best = ms;
  }
  if (e0) cudaEventDestroy(e0);
  if (e1) cudaEventDestroy(e1);
  if (out) cudaFree(out);
  if (e != cudaSuccess || best <= 0.f) return LB_ERR_CUDA;
  const double flops = 2.0 * kChains * (double)iters * grid * kThreads;
  *tflops = flops / (best * 1e-3) / 1e12;
  return LB_OK;
}

// measure.cu -- instrumentation that measures the device rather than the
// method (no counterpart in the paper): the double-precision FMA throughput
// that bounds the FP64 form of the transport sweeps, against which the bench
// states that form's arithmetic rate. Changes no device setting.
#include <cuda_runtime.h>

#include <string>

#include "../../include/reg.h"
#include "internal.h"

using namespace reg;

namespace {

constexpr int kChains = 8;  // independent FMA chains per thread

// Every thread runs kChains independent chains a <- a*b + c for `iters`
// steps (2 flops each). The chains converge to c/(1-b) = 1, so no value
// overflows or becomes subnormal; the sum is compared with a value it never
// takes so that no chain can be removed.
__global__ void __launch_bounds__(256) k_fp64_fma(double* sink, int iters, double b, double c) {
  double a[kChains];
#pragma unroll
  for (int k = 0; k < kChains; ++k) a[k] = 1e-3 * (threadIdx.x + k);
  for (int i = 0; i < iters; ++i) {
#pragma unroll
    for (int k = 0; k < kChains; ++k) a[k] = fma(a[k], b, c);
  }
  double s = 0.0;
#pragma unroll
  for (int k = 0; k < kChains; ++k) s += a[k];
  if (s == -1.0) sink[blockIdx.x] = s;
}

}  // namespace

extern "C" {

reg_status reg_fp64_peak(double* gflops) {
  if (!gflops) {
    set_thread_error("reg_fp64_peak: gflops is null");
    return REG_EINVAL;
  }
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  double* sink = nullptr;
  try {
    int dev = 0, sms = 0, per_sm = 0;
    REG_CUDA(cudaGetDevice(&dev));
    REG_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
    REG_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_fp64_fma, 256, 0));
    const int blocks = sms * (per_sm < 1 ? 1 : per_sm);
    REG_CUDA(cudaMalloc(&sink, sizeof(double) * blocks));
    REG_CUDA(cudaEventCreate(&e0));
    REG_CUDA(cudaEventCreate(&e1));
    const int iters = 1 << 14;
    k_fp64_fma<<<blocks, 256>>>(sink, 64, 0.9999, 1e-4);  // warm-up
    REG_LAUNCH();
    float best = 1e30f;
    for (int r = 0; r < 3; ++r) {
      REG_CUDA(cudaEventRecord(e0));
      k_fp64_fma<<<blocks, 256>>>(sink, iters, 0.9999, 1e-4);
      REG_LAUNCH();
      REG_CUDA(cudaEventRecord(e1));
      REG_CUDA(cudaEventSynchronize(e1));
      float ms = 0.f;
      REG_CUDA(cudaEventElapsedTime(&ms, e0, e1));
      if (ms < best) best = ms;
    }
    const double flops = 2.0 * kChains * (double)iters * blocks * 256.0;
    *gflops = flops / (best * 1e-3) / 1e9;
  } catch (const CudaError& e) {
    if (sink) cudaFree(sink);
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
    set_thread_error("reg_fp64_peak: " + e.what);
    return REG_ECUDA;
  }
  cudaFree(sink);
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  return REG_OK;
}

}  // extern "C"

// fused_f32.cu -- single precision instantiation of the fused transport stages.
#include "../../include/reg.h"
#include "fused_launch.cuh"

namespace reg {
template <>
void adv_stage<float>(Spectral<float>& sp, const float* u, const fused::AdvEpi<float>& e, float2* U, float2* Zx,
                      float2* Zy, bool u_ready, bool emit) {
  fused::adv_stage_impl<float>(sp, u, e, U, Zx, Zy, u_ready, emit);
}
template <>
void adv2_stage<float>(Spectral<float>& sp, const float* uA, const fused::AdvEpi<float>& eA, const float* uB,
                      const fused::AdvEpi<float>& eB, float2* const* Z) {
  fused::adv2_stage_impl<float>(sp, uA, eA, uB, eB, Z);
}
template <>
void div_stage<float>(Spectral<float>& sp, const float* lam, const float* a, const fused::DivEpi<float>& e,
                      float2* Q0, float2* Q1, float2* Q2) {
  fused::div_stage_impl<float>(sp, lam, a, e, Q0, Q1, Q2);
}

// timeouts of the TMA column pass of this precision since the last call (reset on read)
int take_tma_timeouts_f32(cudaStream_t s) {
  int h = 0;
  REG_CUDA(cudaMemcpyFromSymbolAsync(&h, fused::g_tma_timeouts, sizeof(int), 0, cudaMemcpyDeviceToHost, s));
  REG_CUDA(cudaStreamSynchronize(s));
  if (h) {
    const int z = 0;
    REG_CUDA(cudaMemcpyToSymbolAsync(fused::g_tma_timeouts, &z, sizeof(int), 0, cudaMemcpyHostToDevice, s));
    REG_CUDA(cudaStreamSynchronize(s));
  }
  return h;
}
}  // namespace reg

extern "C" reg_status reg_selftest_copy_timeout(int* counted) {
  if (!counted) return REG_EINVAL;
  try {
    reg::fused::k_wait_timeout_probe<<<1, 32>>>(1 << 12);
    REG_CUDA(cudaGetLastError());
    REG_CUDA(cudaDeviceSynchronize());
    *counted = reg::take_tma_timeouts_f32(nullptr);
  } catch (const reg::CudaError& e) {
    reg::set_thread_error(e.what);
    return REG_ECUDA;
  }
  return REG_OK;
}

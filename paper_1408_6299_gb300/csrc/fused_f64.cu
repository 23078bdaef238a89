// fused_f64.cu -- double precision instantiation of the fused transport stages.
#include "fused_launch.cuh"

namespace reg {
template <>
void adv_stage<double>(Spectral<double>& sp, const double* u, const fused::AdvEpi<double>& e, double2* U,
                       double2* Zx, double2* Zy, bool u_ready, bool emit) {
  fused::adv_stage_impl<double>(sp, u, e, U, Zx, Zy, u_ready, emit);
}
template <>
void adv2_stage<double>(Spectral<double>& sp, const double* uA, const fused::AdvEpi<double>& eA, const double* uB,
                      const fused::AdvEpi<double>& eB, double2* const* Z) {
  fused::adv2_stage_impl<double>(sp, uA, eA, uB, eB, Z);
}
template <>
void div_stage<double>(Spectral<double>& sp, const double* lam, const double* a, const fused::DivEpi<double>& e,
                       double2* Q0, double2* Q1, double2* Q2) {
  fused::div_stage_impl<double>(sp, lam, a, e, Q0, Q1, Q2);
}

// timeouts of the TMA column pass of this precision since the last call (reset on read)
int take_tma_timeouts_f64(cudaStream_t s) {
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

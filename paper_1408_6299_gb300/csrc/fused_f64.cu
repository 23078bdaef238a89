// fused_f64.cu -- double precision instantiation of the fused transport stages.
#include "fused_launch.cuh"

namespace reg {
template <>
void adv_stage<double>(Spectral<double>& sp, const double* u, const fused::AdvEpi<double>& e, double2* U,
                       double2* Zx, double2* Zy) {
  fused::adv_stage_impl<double>(sp, u, e, U, Zx, Zy);
}
template <>
void div_stage<double>(Spectral<double>& sp, const double* lam, const double* a, const fused::DivEpi<double>& e,
                       double2* Q0, double2* Q1, double2* Q2) {
  fused::div_stage_impl<double>(sp, lam, a, e, Q0, Q1, Q2);
}
}  // namespace reg

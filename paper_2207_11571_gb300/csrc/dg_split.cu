// Split-form phase B (kinetic-energy-preserving volume term) in both precisions: a
// translation unit of its own, so that these instantiations build in parallel with the
// default kernels.
#include "dg_launch.cuh"

namespace dgnn {
cudaError_t flux_split_f32(const dg_ctx* c, double* q, double* dqdt, const Forcing& f, int mode, double A, double B,
                           double dt, double invB1, cudaStream_t st) {
  return flux_split_t<float>(c, q, dqdt, f, mode, A, B, dt, invB1, st);
}
cudaError_t flux_split_f64(const dg_ctx* c, double* q, double* dqdt, const Forcing& f, int mode, double A, double B,
                           double dt, double invB1, cudaStream_t st) {
  return flux_split_t<double>(c, q, dqdt, f, mode, A, B, dt, invB1, st);
}
}  // namespace dgnn

// FP32 instantiation of the operator kernels (FP32 fluxes and contractions, FP64 state).
#include "dg_launch.cuh"

namespace dgnn {
cudaError_t gradient_f32(const dg_ctx* c, const double* q, int src, cudaStream_t st) {
  return gradient_t<float>(c, q, src, st);
}
cudaError_t flux_f32(const dg_ctx* c, double* q, double* dqdt, const Forcing& f, int mode, double A, double B,
                     double dt, double invB1, cudaStream_t st) {
  return flux_t<float>(c, q, dqdt, f, mode, A, B, dt, invB1, st);
}
// Constant-memory tables of this unit's kernels (see upload_const_D).
cudaError_t prepare_f32_constants() { return upload_const_D(); }
}  // namespace dgnn

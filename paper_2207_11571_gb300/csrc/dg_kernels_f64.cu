// FP64 instantiation of the operator kernels (the parity path).
#include "dg_launch.cuh"

namespace dgnn {
cudaError_t gradient_f64(const dg_ctx* c, const double* q, int src, cudaStream_t st) {
  return gradient_t<double>(c, q, src, st);
}
cudaError_t flux_f64(const dg_ctx* c, double* q, double* dqdt, const Forcing& f, int mode, double A, double B,
                     double dt, double invB1, cudaStream_t st) {
  return flux_t<double>(c, q, dqdt, f, mode, A, B, dt, invB1, st);
}
}  // namespace dgnn

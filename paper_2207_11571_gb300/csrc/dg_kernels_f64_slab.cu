// FP64 operator kernels of slab contexts (see dg_kernels_f32_slab.cu).
#include "dg_launch.cuh"

namespace dgnn {
cudaError_t gradient_f64_slab(const dg_ctx* c, const double* q, int src, cudaStream_t st) {
  return gradient_t<double, true>(c, q, src, st);
}
cudaError_t flux_f64_slab(const dg_ctx* c, double* q, double* dqdt, const Forcing& f, int mode, double A, double B,
                          double dt, double invB1, cudaStream_t st) {
  return flux_t<double, true>(c, q, dqdt, f, mode, A, B, dt, invB1, st);
}
cudaError_t flux_split_f64_slab(const dg_ctx* c, double* q, double* dqdt, const Forcing& f, int mode, double A,
                                double B, double dt, double invB1, cudaStream_t st) {
  return flux_split_t<double, true>(c, q, dqdt, f, mode, A, B, dt, invB1, st);
}
}  // namespace dgnn

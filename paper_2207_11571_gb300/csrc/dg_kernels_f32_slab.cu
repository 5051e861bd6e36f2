// FP32 operator kernels of slab contexts (dg_create_part: an owned range of element
// layers and ghost layers); their own translation unit, so that the whole-mesh kernels
// compile without the slab arithmetic and the two build in parallel.
#include "dg_launch.cuh"

namespace dgnn {
cudaError_t gradient_f32_slab(const dg_ctx* c, const double* q, int src, cudaStream_t st) {
  return gradient_t<float, true>(c, q, src, st);
}
cudaError_t flux_f32_slab(const dg_ctx* c, double* q, double* dqdt, const Forcing& f, int mode, double A, double B,
                          double dt, double invB1, cudaStream_t st) {
  return flux_t<float, true>(c, q, dqdt, f, mode, A, B, dt, invB1, st);
}
cudaError_t flux_split_f32_slab(const dg_ctx* c, double* q, double* dqdt, const Forcing& f, int mode, double A,
                                double B, double dt, double invB1, cudaStream_t st) {
  return flux_split_t<float, true>(c, q, dqdt, f, mode, A, B, dt, invB1, st);
}
// Constant-memory tables of this unit's kernels (see upload_const_D).
cudaError_t prepare_f32_slab_constants() { return upload_const_D(); }
}  // namespace dgnn

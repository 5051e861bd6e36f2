// FP32 instantiation of the batched RK-stage kernels (several meshes of one
// order per launch).
#include "dg_aux.h"
#include "dg_launch.cuh"

namespace dgnn {
cudaError_t batch_stage_f32(int P, dg_ctx* const* ctx, double* const* q, const double* dt, int n, int k, double A,
                            double B, double invB1, cudaStream_t st) {
  return batch_stage_t<float>(P, ctx, q, dt, n, k, A, B, invB1, st);
}
cudaError_t batch_prepare_f32(int P, int E) { return batch_prepare_t<float>(P, E); }
// Constant-memory tables of this unit's kernels (see upload_const_D).
cudaError_t prepare_batch_f32_constants() { return upload_const_D(); }
}  // namespace dgnn

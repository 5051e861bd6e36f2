// Host launchers of the operator kernels for one operator precision T; included by
// dg_kernels_f32.cu and dg_kernels_f64.cu so that the two precisions compile in
// parallel translation units.
#pragma once

#include "dg_kernels.cuh"

namespace dgnn {

inline int block_threads(int P, int E) {
  const int np = (P + 1) * (P + 1) * (P + 1);
  return ((E * np + 31) / 32) * 32;
}

template <typename K>
cudaError_t set_smem(K kern, size_t smem) {
  if (smem > 48 * 1024) return cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  return cudaSuccess;
}

template <int P, typename T, int SRC>
cudaError_t gradient_p(const dg_ctx* c, const double* q, cudaStream_t st) {
  constexpr int n = P + 1, np = n * n * n;
  const int E = c->geom.E;
  const size_t smem = sizeof(T) * (n * n + 4 * E * np);
  auto kern = k_gradient<P, T, SRC>;
  cudaError_t e = set_smem(kern, smem);
  if (e != cudaSuccess) return e;
  const int grid = (c->nel + E - 1) / E;
  kern<<<grid, block_threads(P, E), smem, st>>>(q, c->qn32, c->dlt, static_cast<T*>(c->qf),
                                                SRC == 0 ? c->qn32 : nullptr, static_cast<T*>(c->vis), c->geom,
                                                c->phys);
  return cudaGetLastError();
}

template <int P, typename T, int MODE, typename GT>
cudaError_t flux_p(const dg_ctx* c, double* q, double* dqdt, const Forcing& f, const RkArgs& rk, cudaStream_t st) {
  constexpr int n = P + 1, np = n * n * n;
  const int E = c->geom.E;
  const size_t smem = sizeof(T) * (n * n + 5 * E * np);
  auto kern = k_flux<P, T, MODE, GT>;
  cudaError_t e = set_smem(kern, smem);
  if (e != cudaSuccess) return e;
  const int grid = (c->nel + E - 1) / E;
  kern<<<grid, block_threads(P, E), smem, st>>>(q, static_cast<const T*>(c->qf), static_cast<const T*>(c->vis), dqdt,
                                                static_cast<GT*>(c->g), c->dlt, f, c->geom, c->phys, rk);
  return cudaGetLastError();
}

// FP64 operator: modes 0 (dq/dt) and 1 (FP64 RK stage).  FP32 operator: modes 0, 2, 3, 4.
template <int P, typename T>
cudaError_t flux_dispatch_mode(const dg_ctx* c, double* q, double* dqdt, const Forcing& f, int mode,
                               const RkArgs& rk, cudaStream_t st) {
  using GT = T;  // RK register in the operator precision
  switch (mode) {
    case 0: return flux_p<P, T, 0, GT>(c, q, dqdt, f, rk, st);
    case 1: return flux_p<P, T, 1, GT>(c, q, dqdt, f, rk, st);
    case 2: return flux_p<P, T, 2, GT>(c, q, dqdt, f, rk, st);
    case 3: return flux_p<P, T, 3, GT>(c, q, dqdt, f, rk, st);
    case 4: return flux_p<P, T, 4, GT>(c, q, dqdt, f, rk, st);
  }
  return cudaErrorInvalidValue;
}

template <int P, typename T>
cudaError_t gradient_dispatch_src(const dg_ctx* c, const double* q, int src, cudaStream_t st) {
  if (src == 0) return gradient_p<P, T, 0>(c, q, st);
  return gradient_p<P, T, 1>(c, q, st);
}

#define DG_FOR_EACH_P(CALL)        \
  switch (c->P) {                  \
    case 1: return CALL(1);        \
    case 2: return CALL(2);        \
    case 3: return CALL(3);        \
    case 4: return CALL(4);        \
    case 5: return CALL(5);        \
    case 6: return CALL(6);        \
    case 7: return CALL(7);        \
    case 8: return CALL(8);        \
  }                                \
  return cudaErrorInvalidValue;

template <typename T>
cudaError_t gradient_t(const dg_ctx* c, const double* q, int src, cudaStream_t st) {
#define DG_G(PP) gradient_dispatch_src<PP, T>(c, q, src, st)
  DG_FOR_EACH_P(DG_G)
#undef DG_G
}

template <typename T>
cudaError_t flux_t(const dg_ctx* c, double* q, double* dqdt, const Forcing& f, int mode, const RkArgs& rk,
                   cudaStream_t st) {
#define DG_F(PP) flux_dispatch_mode<PP, T>(c, q, dqdt, f, mode, rk, st)
  DG_FOR_EACH_P(DG_F)
#undef DG_F
}

}  // namespace dgnn

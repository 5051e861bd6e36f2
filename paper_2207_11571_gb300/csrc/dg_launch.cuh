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

template <int P, typename T>
cudaError_t gradient_p(const dg_ctx* c, const double* q, cudaStream_t st) {
  constexpr int n = P + 1, np = n * n * n;
  const int E = c->geom.E;
  const size_t smem = sizeof(T) * (n * n + 4 * E * np);
  auto kern = k_gradient<P, T>;
  if (smem > 48 * 1024) {
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
  }
  const int grid = (c->nel + E - 1) / E;
  kern<<<grid, block_threads(P, E), smem, st>>>(q, static_cast<T*>(c->qf), static_cast<T*>(c->vis), c->geom, c->phys);
  return cudaGetLastError();
}

template <int P, typename T, int MODE, typename GT>
cudaError_t flux_p(const dg_ctx* c, double* q, double* dqdt, const Forcing& f, double A, double B,
                   double dt, cudaStream_t st) {
  constexpr int n = P + 1, np = n * n * n;
  const int E = c->geom.E;
  const size_t smem = sizeof(T) * (n * n + 5 * E * np);
  auto kern = k_flux<P, T, MODE, GT>;
  if (smem > 48 * 1024) {
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
  }
  const int grid = (c->nel + E - 1) / E;
  kern<<<grid, block_threads(P, E), smem, st>>>(q, static_cast<const T*>(c->qf), static_cast<const T*>(c->vis),
                                                dqdt, static_cast<GT*>(c->g), f, c->geom, c->phys, A, B, dt);
  return cudaGetLastError();
}

template <int P, typename T>
cudaError_t flux_dispatch_mode(const dg_ctx* c, double* q, double* dqdt, const Forcing& f, int mode,
                               double A, double B, double dt, cudaStream_t st) {
  if (mode == 0) return flux_p<P, T, 0, double>(c, q, dqdt, f, A, B, dt, st);
  if (c->opts.rk_register_fp32) return flux_p<P, T, 1, float>(c, q, dqdt, f, A, B, dt, st);
  return flux_p<P, T, 1, double>(c, q, dqdt, f, A, B, dt, st);
}

template <typename T>
cudaError_t gradient_t(const dg_ctx* c, const double* q, cudaStream_t st) {
  switch (c->P) {
    case 1: return gradient_p<1, T>(c, q, st);
    case 2: return gradient_p<2, T>(c, q, st);
    case 3: return gradient_p<3, T>(c, q, st);
    case 4: return gradient_p<4, T>(c, q, st);
    case 5: return gradient_p<5, T>(c, q, st);
    case 6: return gradient_p<6, T>(c, q, st);
    case 7: return gradient_p<7, T>(c, q, st);
    case 8: return gradient_p<8, T>(c, q, st);
  }
  return cudaErrorInvalidValue;
}

template <typename T>
cudaError_t flux_t(const dg_ctx* c, double* q, double* dqdt, const Forcing& f, int mode, double A,
                   double B, double dt, cudaStream_t st) {
  switch (c->P) {
    case 1: return flux_dispatch_mode<1, T>(c, q, dqdt, f, mode, A, B, dt, st);
    case 2: return flux_dispatch_mode<2, T>(c, q, dqdt, f, mode, A, B, dt, st);
    case 3: return flux_dispatch_mode<3, T>(c, q, dqdt, f, mode, A, B, dt, st);
    case 4: return flux_dispatch_mode<4, T>(c, q, dqdt, f, mode, A, B, dt, st);
    case 5: return flux_dispatch_mode<5, T>(c, q, dqdt, f, mode, A, B, dt, st);
    case 6: return flux_dispatch_mode<6, T>(c, q, dqdt, f, mode, A, B, dt, st);
    case 7: return flux_dispatch_mode<7, T>(c, q, dqdt, f, mode, A, B, dt, st);
    case 8: return flux_dispatch_mode<8, T>(c, q, dqdt, f, mode, A, B, dt, st);
  }
  return cudaErrorInvalidValue;
}

}  // namespace dgnn

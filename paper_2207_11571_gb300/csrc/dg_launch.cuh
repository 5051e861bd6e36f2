// Host launchers of the operator kernels for one operator precision T; included by
// dg_kernels_f32.cu and dg_kernels_f64.cu so that the two precisions compile in
// parallel translation units.
#pragma once

#include <algorithm>
#include <type_traits>

#include "dg_kernels.cuh"

namespace dgnn {

// Elements a launch processes: the whole mesh, or a slab's own layers.
inline int owned_elems(const dg_ctx* c) { return c->e_end - c->e_begin; }

inline int block_threads(int P, int E) {
  const int np = (P + 1) * (P + 1) * (P + 1);
  return ((E * np + 31) / 32) * 32;
}

// Threads of a flux block: flux_npt(P) nodes per thread.
inline int flux_threads(int P, int E) {
  const int np = (P + 1) * (P + 1) * (P + 1);
  const int npt = flux_npt(P);
  return (((E * np + npt - 1) / npt + 31) / 32) * 32;
}

template <typename T>
OpConst<T> make_const(const dg_ctx* c) {
  OpConst<T> k;
  k.K = c->K;
  k.E = c->geom.E;
  k.nel = c->e_end;
  k.Kz = c->Kz;
  k.e_begin = c->e_begin;
  k.N = c->N;
  const Phys& ph = c->phys;
  k.gm1 = T(ph.gamma - 1.0);
  k.rho_ref = T(ph.rho_ref);
  k.theta_ref = T(ph.theta_ref);
  k.Hc = T(ph.Hc);
  k.s2h = T(c->geom.two_over_h);
  k.winv = T(c->geom.winv);
  k.mu = T(ph.mu);
  k.lam = T(ph.lam);
  k.csd2 = T(ph.csd2);
  k.lam_t = T(ph.lam_t);
  k.les = ph.les;
  k.drho_ref = ph.rho_ref;
  k.dE_ref = ph.E_ref;
  k.feat = c->feat_out;
  for (int i = 0; i < kMaxN1 * kMaxN1; ++i) k.D[i] = T(c->geom.D[i]);
  return k;
}

// Fills this translation unit's constant-memory derivative matrices (c_D32) on the
// current device, once per device.  Synchronous: called from dg_create, outside any
// stream capture.
static cudaError_t upload_const_D() {
  static bool done[64] = {};
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  if (dev >= 0 && dev < 64 && done[dev]) return cudaSuccess;
  float h[kMaxP + 1][kMaxN1 * kMaxN1] = {};
  for (int P = 1; P <= kMaxP; ++P) {
    Basis1D b;
    if (build_basis(P, &b) != 0) return cudaErrorInvalidValue;
    for (int i = 0; i < (P + 1) * (P + 1); ++i) h[P][i] = (float)b.D[i];
  }
  e = cudaMemcpyToSymbol(c_D32, h, sizeof(h));
  if (e == cudaSuccess && dev >= 0 && dev < 64) done[dev] = true;
  return e;
}

// Launch with programmatic stream serialization (the kernels wait for their predecessor
// themselves, see pdl_wait in dg_kernels.cuh).
template <typename... KArgs, typename... Args>
cudaError_t launch_pdl(void (*kern)(KArgs...), dim3 grid, dim3 block, size_t smem, cudaStream_t st, Args&&... args) {
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = grid;
  cfg.blockDim = block;
  cfg.dynamicSmemBytes = smem;
  cfg.stream = st;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  attr[0].val.programmaticStreamSerializationAllowed = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  return cudaLaunchKernelEx(&cfg, kern, std::forward<Args>(args)...);
}

template <typename K>
cudaError_t set_smem(K kern, size_t smem) {
  if (smem > 48 * 1024) return cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  return cudaSuccess;
}

// Shared memory of the kernels (layouts in dg_kernels.cuh).
template <int P, typename T>
size_t gradient_smem(int E) {
  constexpr int n = P + 1, n2 = n * n, np = n2 * n;
  // FP32 at P >= 7 with one element per block adds the line-wise derivative buffer [12][np]
  const int lines = (std::is_same<T, float>::value && P >= 7 && E == 1) ? 12 * np : 0;
  return sizeof(T) * (n2 + 4 * E * np + 4 * E * 6 * n2 + lines);
}

// Cube blocks: eight elements, halo of the 24 external faces only, lifted terms of all 48.
template <int P, typename T>
size_t gradient_smem_cube() {
  constexpr int n = P + 1, n2 = n * n, np = n2 * n;
  return sizeof(T) * (n2 + 4 * kCubeElems * np + 4 * 3 * kCubeElems * n2);
}

template <int P, typename T>
size_t flux_smem_cube() {
  constexpr int n = P + 1, n2 = n * n, np = n2 * n;
  const int tile = flux_early(P, sizeof(T)) ? 14 + kTileComponents : kTileComponents;
  return sizeof(T) * (n2 + tile * kCubeElems * np + kFaceComponents * 3 * kCubeElems * n2 + 5 * kCubeElems * 6 * n2);
}

template <int P, typename T>
size_t flux_smem(int E) {
  constexpr int n = P + 1, n2 = n * n, np = n2 * n;
  // early volume fluxes: own tile [14] and flux tile [15] apart
  const int tile = flux_early(P, sizeof(T)) ? 14 + kTileComponents : kTileComponents;
  return sizeof(T) * (n2 + tile * E * np + (kFaceComponents + 5) * E * 6 * n2);
}

// Phase A.  SLAB: a slab context (owned range, local z extent; no network features);
// whole meshes pick the variant that also writes the network's features when the context
// asks for them (c->feat_out), so that the plain kernel compiles as it did without them.
template <int P, typename T, int SRC, bool SLAB, bool FEAT>
cudaError_t gradient_launch(const dg_ctx* c, const double* q, cudaStream_t st) {
  if constexpr (cube_ok(P) && !SLAB) {
    if (c->geom.cube) {
      const size_t smem = gradient_smem_cube<P, T>();
      auto kern = k_gradient<P, T, SRC, true, false, FEAT>;
      cudaError_t e = set_smem(kern, smem);
      if (e != cudaSuccess) return e;
      const int h = c->K / 2;
      return launch_pdl(kern, dim3(h * h * h), dim3(block_threads(P, kCubeElems)), smem, st,
          q, c->qn32, c->dlt, static_cast<T*>(c->qf), SRC == 0 ? c->qn32 : nullptr, static_cast<T*>(c->vis),
          make_const<T>(c));
    }
  }
  const int E = c->geom.E;
  const size_t smem = gradient_smem<P, T>(E);
  auto kern = k_gradient<P, T, SRC, false, SLAB, FEAT>;
  cudaError_t e = set_smem(kern, smem);
  if (e != cudaSuccess) return e;
  const int grid = (owned_elems(c) + E - 1) / E;
  return launch_pdl(kern, dim3(grid), dim3(block_threads(P, E)), smem, st, q, c->qn32, c->dlt, static_cast<T*>(c->qf),
                                                SRC == 0 ? c->qn32 : nullptr, static_cast<T*>(c->vis),
                                                make_const<T>(c));
}

template <int P, typename T, int SRC, bool SLAB>
cudaError_t gradient_p(const dg_ctx* c, const double* q, cudaStream_t st) {
  if constexpr (!SLAB) {
    if (c->feat_out.out != nullptr) return gradient_launch<P, T, SRC, false, true>(c, q, st);
  }
  return gradient_launch<P, T, SRC, SLAB, false>(c, q, st);
}

// Grid of a persistent streamed launch: resident blocks on every SM, at most one per item.
template <typename K>
cudaError_t stream_grid(K kern, int threads, size_t smem, int items, int* grid) {
  static int sms = 0;
  if (!sms) {
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (e != cudaSuccess) return e;
  }
  int per_sm = 0;
  cudaError_t e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, threads, smem);
  if (e != cudaSuccess) return e;
  if (per_sm < 1) return cudaErrorInvalidConfiguration;
  *grid = std::min(items, per_sm * sms);
  return cudaSuccess;
}

// Own tiles of the streamed kernel by TMA bulk copies: every component row of qf and vis
// must start on a 16-byte boundary up to the element's shift (e np) mod 4.
inline int stream_bulk_ok(const dg_ctx* c) {
  return (reinterpret_cast<uintptr_t>(c->qf) % 16 == 0) && (reinterpret_cast<uintptr_t>(c->vis) % 16 == 0) &&
         (c->N % 4 == 0);
}

// Streamed phase B (FP32 operator, P >= 6, one element per block step).
template <int P, int MODE, bool SLAB>
cudaError_t flux_stream_launch(const dg_ctx* c, double* q, double* dqdt, const Forcing& f,
                               const RkArgs<float>& rk, cudaStream_t st) {
  const size_t smem = sizeof(float) * stream_smem_floats<P>();
  auto kern = k_flux_stream<P, MODE, SLAB>;
  cudaError_t e = set_smem(kern, smem);
  if (e != cudaSuccess) return e;
  int grid = 0;
  if ((e = stream_grid(kern, stream_threads(P), smem, owned_elems(c), &grid)) != cudaSuccess) return e;
  StreamMesh m;
  m.q = q;
  m.qf = static_cast<const float*>(c->qf);
  m.vis = static_cast<const float*>(c->vis);
  m.dqdt = dqdt;
  m.greg = static_cast<float*>(c->g);
  m.dlt = c->dlt;
  m.fc = f;
  m.C = make_const<float>(c);
  m.rk = rk;
  m.bulk = stream_bulk_ok(c);
  m.err = c->err_dev;
  return launch_pdl(kern, dim3(grid), dim3(stream_threads(P)), smem, st, m);
}

template <int P, typename T, int MODE, bool SLAB>
cudaError_t flux_p(const dg_ctx* c, double* q, double* dqdt, const Forcing& f, const RkArgs<T>& rk,
                   cudaStream_t st) {
  if constexpr (std::is_same<T, float>::value && P >= 6 && MODE != 1) {
    if (c->geom.E == 1) return flux_stream_launch<P, MODE, SLAB>(c, q, dqdt, f, rk, st);
  }
  if constexpr (cube_ok(P) && !SLAB) {
    if (c->geom.cube) {
      const size_t smem = flux_smem_cube<P, T>();
      auto kern = k_flux<P, T, MODE, true>;
      cudaError_t e = set_smem(kern, smem);
      if (e != cudaSuccess) return e;
      const int h = c->K / 2;
      return launch_pdl(kern, dim3(h * h * h), dim3(flux_threads(P, kCubeElems)), smem, st, 
          q, static_cast<const T*>(c->qf), static_cast<const T*>(c->vis), dqdt, static_cast<T*>(c->g), c->dlt, f,
          make_const<T>(c), rk);
    }
  }
  const int E = c->geom.E;
  const size_t smem = flux_smem<P, T>(E);
  auto kern = k_flux<P, T, MODE, false, false, SLAB>;
  cudaError_t e = set_smem(kern, smem);
  if (e != cudaSuccess) return e;
  const int grid = (owned_elems(c) + E - 1) / E;
  return launch_pdl(kern, dim3(grid), dim3(flux_threads(P, E)), smem, st, q, static_cast<const T*>(c->qf), static_cast<const T*>(c->vis), dqdt,
                                                static_cast<T*>(c->g), c->dlt, f, make_const<T>(c), rk);
}

// FP64 operator: modes 0 (dq/dt) and 1 (FP64 RK stage).  FP32 operator: modes 0, 2, 3, 4.
template <int P, typename T, bool SLAB>
cudaError_t flux_dispatch_mode(const dg_ctx* c, double* q, double* dqdt, const Forcing& f, int mode,
                               const RkArgs<T>& rk, cudaStream_t st) {
  switch (mode) {
    case 0: return flux_p<P, T, 0, SLAB>(c, q, dqdt, f, rk, st);
    case 1: return flux_p<P, T, 1, SLAB>(c, q, dqdt, f, rk, st);
    case 2: return flux_p<P, T, 2, SLAB>(c, q, dqdt, f, rk, st);
    case 3: return flux_p<P, T, 3, SLAB>(c, q, dqdt, f, rk, st);
    case 4: return flux_p<P, T, 4, SLAB>(c, q, dqdt, f, rk, st);
  }
  return cudaErrorInvalidValue;
}

template <int P, typename T, bool SLAB>
cudaError_t gradient_dispatch_src(const dg_ctx* c, const double* q, int src, cudaStream_t st) {
  if (src == 0) return gradient_p<P, T, 0, SLAB>(c, q, st);
  return gradient_p<P, T, 1, SLAB>(c, q, st);
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

template <typename T, bool SLAB = false>
cudaError_t gradient_t(const dg_ctx* c, const double* q, int src, cudaStream_t st) {
#define DG_G(PP) gradient_dispatch_src<PP, T, SLAB>(c, q, src, st)
  DG_FOR_EACH_P(DG_G)
#undef DG_G
}

template <typename T, bool SLAB = false>
cudaError_t flux_t(const dg_ctx* c, double* q, double* dqdt, const Forcing& f, int mode, double A, double B,
                   double dt, double invB1, cudaStream_t st) {
  const RkArgs<T> rk{T(A), T(B), T(dt), T(invB1)};
#define DG_F(PP) flux_dispatch_mode<PP, T, SLAB>(c, q, dqdt, f, mode, rk, st)
  DG_FOR_EACH_P(DG_F)
#undef DG_F
}

// ---------------------------------------------------------------------------------------
// Split-form phase B (rows of E elements, every order, both precisions): k_flux with the
// two-point-flux volume term and a tile of primitives [6][E np] on top of flux_smem.
template <int P, typename T, int MODE, bool SLAB>
cudaError_t flux_split_p(const dg_ctx* c, double* q, double* dqdt, const Forcing& f, const RkArgs<T>& rk,
                         cudaStream_t st) {
  constexpr int np = (P + 1) * (P + 1) * (P + 1);
  const int E = c->geom.E;
  const size_t smem = flux_smem<P, T>(E) + sizeof(T) * 6 * E * np;
  auto kern = k_flux<P, T, MODE, false, true, SLAB>;
  cudaError_t e = set_smem(kern, smem);
  if (e != cudaSuccess) return e;
  const int grid = (owned_elems(c) + E - 1) / E;
  return launch_pdl(kern, dim3(grid), dim3(flux_threads(P, E)), smem, st, q, static_cast<const T*>(c->qf), static_cast<const T*>(c->vis), dqdt,
                                                static_cast<T*>(c->g), c->dlt, f, make_const<T>(c), rk);
}

template <int P, typename T, bool SLAB>
cudaError_t flux_split_dispatch_mode(const dg_ctx* c, double* q, double* dqdt, const Forcing& f, int mode,
                                     const RkArgs<T>& rk, cudaStream_t st) {
  if constexpr (std::is_same<T, float>::value) {
    switch (mode) {
      case 0: return flux_split_p<P, T, 0, SLAB>(c, q, dqdt, f, rk, st);
      case 2: return flux_split_p<P, T, 2, SLAB>(c, q, dqdt, f, rk, st);
      case 3: return flux_split_p<P, T, 3, SLAB>(c, q, dqdt, f, rk, st);
      case 4: return flux_split_p<P, T, 4, SLAB>(c, q, dqdt, f, rk, st);
    }
  } else {
    switch (mode) {
      case 0: return flux_split_p<P, T, 0, SLAB>(c, q, dqdt, f, rk, st);
      case 1: return flux_split_p<P, T, 1, SLAB>(c, q, dqdt, f, rk, st);
    }
  }
  return cudaErrorInvalidValue;
}

template <typename T, bool SLAB = false>
cudaError_t flux_split_t(const dg_ctx* c, double* q, double* dqdt, const Forcing& f, int mode, double A, double B,
                         double dt, double invB1, cudaStream_t st) {
  const RkArgs<T> rk{T(A), T(B), T(dt), T(invB1)};
#define DG_S(PP) flux_split_dispatch_mode<PP, T, SLAB>(c, q, dqdt, f, mode, rk, st)
  DG_FOR_EACH_P(DG_S)
#undef DG_S
}

// ---------------------------------------------------------------------------------------
// Batched RK stage: one phase-A and one phase-B launch for all instances of order P.
// Instances must share the operator precision T and the elements-per-block E.

template <typename T>
void fill_batch(BatchTable<T>* tb, dg_ctx* const* ctx, double* const* q, const double* dt, int n, double A,
                double B, double invB1) {
  tb->n = n;
  int blocks = 0;
  for (int i = 0; i < n; ++i) {
    const dg_ctx* c = ctx[i];
    tb->block_start[i] = blocks;
    blocks += (owned_elems(c) + c->geom.E - 1) / c->geom.E;
    tb->q[i] = q[i];
    tb->qn32[i] = c->qn32;
    tb->dlt[i] = c->dlt;
    tb->qf[i] = static_cast<T*>(c->qf);
    tb->vis[i] = static_cast<T*>(c->vis);
    tb->g[i] = static_cast<T*>(c->g);
    tb->rk[i] = RkArgs<T>{T(A), T(B), T(dt[i]), T(invB1)};
    tb->C[i] = make_const<T>(c);
    tb->bulk[i] = stream_bulk_ok(c);
    tb->err[i] = c->err_dev;
  }
  tb->block_start[n] = blocks;
}

// Stage k of the RK3 step: the same source and mode sequence as the single-mesh path
// (FP32 operator: sources 0, 1, 1 and modes 2, 3, 4; FP64 operator: source 0, mode 1).
template <int P, typename T>
cudaError_t batch_stage_p(const BatchTable<T>& tb, int E, int k, cudaStream_t st) {
  constexpr bool f32 = std::is_same<T, float>::value;
  const int grid = tb.block_start[tb.n];
  const int threads = block_threads(P, E);
  const size_t gs = gradient_smem<P, T>(E), fs = flux_smem<P, T>(E);
  cudaError_t e;
  if constexpr (std::is_same<T, float>::value && P >= 6) {
    if (E == 1) {
      auto kg = k == 0 ? k_gradient_batch<P, T, 0> : k_gradient_batch<P, T, 1>;
      auto kf = k == 0 ? k_flux_stream_batch<P, 2> : k == 1 ? k_flux_stream_batch<P, 3> : k_flux_stream_batch<P, 4>;
      const size_t ss = sizeof(float) * stream_smem_floats<P>();
      int sgrid = 0;
      if ((e = stream_grid(kf, stream_threads(P), ss, grid, &sgrid)) != cudaSuccess) return e;
      if ((e = launch_pdl(kg, dim3(grid), dim3(threads), gs, st, tb)) != cudaSuccess) return e;
      return launch_pdl(kf, dim3(sgrid), dim3(stream_threads(P)), ss, st, tb);
    }
  }
  void (*kg)(const BatchTable<T>);
  void (*kf)(const BatchTable<T>);
  if constexpr (f32) {
    kg = k == 0 ? k_gradient_batch<P, T, 0> : k_gradient_batch<P, T, 1>;
    kf = k == 0 ? k_flux_batch<P, T, 2> : k == 1 ? k_flux_batch<P, T, 3> : k_flux_batch<P, T, 4>;
  } else {
    kg = k_gradient_batch<P, T, 0>;
    kf = k_flux_batch<P, T, 1>;
  }
  if ((e = launch_pdl(kg, dim3(grid), dim3(threads), gs, st, tb)) != cudaSuccess) return e;
  return launch_pdl(kf, dim3(grid), dim3(flux_threads(P, E)), fs, st, tb);
}

// Dynamic shared-memory attributes of the batched kernels of order P at E elements per
// block; set before any launch (and outside stream capture).
template <int P, typename T>
cudaError_t batch_prepare_p(int E) {
  const size_t gs = gradient_smem<P, T>(E), fs = flux_smem<P, T>(E);
  cudaError_t e;
  if constexpr (std::is_same<T, float>::value && P >= 6) {
    if (E == 1) {
      const size_t ss = sizeof(float) * stream_smem_floats<P>();
      if ((e = set_smem(k_flux_stream_batch<P, 2>, ss)) != cudaSuccess) return e;
      if ((e = set_smem(k_flux_stream_batch<P, 3>, ss)) != cudaSuccess) return e;
      if ((e = set_smem(k_flux_stream_batch<P, 4>, ss)) != cudaSuccess) return e;
    }
  }
  if constexpr (std::is_same<T, float>::value) {
    if ((e = set_smem(k_gradient_batch<P, T, 0>, gs)) != cudaSuccess) return e;
    if ((e = set_smem(k_gradient_batch<P, T, 1>, gs)) != cudaSuccess) return e;
    if ((e = set_smem(k_flux_batch<P, T, 2>, fs)) != cudaSuccess) return e;
    if ((e = set_smem(k_flux_batch<P, T, 3>, fs)) != cudaSuccess) return e;
    return set_smem(k_flux_batch<P, T, 4>, fs);
  } else {
    if ((e = set_smem(k_gradient_batch<P, T, 0>, gs)) != cudaSuccess) return e;
    return set_smem(k_flux_batch<P, T, 1>, fs);
  }
}

template <typename T>
cudaError_t batch_prepare_t(int P, int E) {
  switch (P) {
    case 1: return batch_prepare_p<1, T>(E);
    case 2: return batch_prepare_p<2, T>(E);
    case 3: return batch_prepare_p<3, T>(E);
    case 4: return batch_prepare_p<4, T>(E);
    case 5: return batch_prepare_p<5, T>(E);
    case 6: return batch_prepare_p<6, T>(E);
    case 7: return batch_prepare_p<7, T>(E);
    case 8: return batch_prepare_p<8, T>(E);
  }
  return cudaErrorInvalidValue;
}

template <typename T>
cudaError_t batch_stage_t(int P, dg_ctx* const* ctx, double* const* q, const double* dt, int n, int k, double A,
                          double B, double invB1, cudaStream_t st) {
  if (n < 1 || n > kMaxBatch) return cudaErrorInvalidValue;
  BatchTable<T> tb;
  fill_batch<T>(&tb, ctx, q, dt, n, A, B, invB1);
  const int E = ctx[0]->geom.E;
  switch (P) {
    case 1: return batch_stage_p<1, T>(tb, E, k, st);
    case 2: return batch_stage_p<2, T>(tb, E, k, st);
    case 3: return batch_stage_p<3, T>(tb, E, k, st);
    case 4: return batch_stage_p<4, T>(tb, E, k, st);
    case 5: return batch_stage_p<5, T>(tb, E, k, st);
    case 6: return batch_stage_p<6, T>(tb, E, k, st);
    case 7: return batch_stage_p<7, T>(tb, E, k, st);
    case 8: return batch_stage_p<8, T>(tb, E, k, st);
  }
  return cudaErrorInvalidValue;
}

}  // namespace dgnn

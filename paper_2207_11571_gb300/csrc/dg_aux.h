// Declarations of the auxiliary kernels (initial state, filter, diagnostics, pairs).
#pragma once

#include "dg_common.h"

namespace dgnn {

// Node coordinates and quadrature weights of a context, by value for kernels.
// t_begin, t_end: the owned nodes (a whole mesh: 0, N; a slab: its own layers);
// z_off: global element layer of local layer 0 (a slab's lower ghost layer).
struct NodeGeom {
  int K, n;
  long long N;
  long long t_begin, t_end;
  int z_off;
  double h;
  double xi[kMaxN1];
  double w[kMaxN1];
};

inline NodeGeom node_geom(const dg_ctx* c) {
  NodeGeom g;
  g.K = c->K;
  g.n = c->n;
  g.N = c->N;
  g.t_begin = (long long)c->e_begin * c->np;
  g.t_end = (long long)c->e_end * c->np;
  g.z_off = c->part ? (c->z_begin - 1 + c->K) % c->K : 0;
  g.h = 2.0 * M_PI / c->K;
  for (int i = 0; i < kMaxN1; ++i) {
    g.xi[i] = i < c->n ? c->basis.xi[i] : 0.0;
    g.w[i] = i < c->n ? c->basis.w[i] : 0.0;
  }
  return g;
}

// Diagnostic vector: [0] mass, [1..3] momentum, [4] energy, [5] 2 pi^3 ke, [6] 2 pi^3 dke/dt,
// [7] non-finite count (summed); [8..10] e_inf, [11] max wave speed (maxima).
constexpr int kDiagSum = 8;
constexpr int kDiagLen = 12;
constexpr int kDiagNonfinite = 7;
constexpr int kDiagThreads = 256;
constexpr int kDiagBlocks = 1024;

cudaError_t launch_init_tgv(const dg_ctx* c, double* q, const double* pert, cudaStream_t st);
cudaError_t launch_project(const dg_ctx* hi, const dg_ctx* lo, const double* qh, double* ql, const double* Gdev,
                           cudaStream_t st);
// The same tensor-product transform from the lower to the higher order (I: n_hi x n_lo).
cudaError_t launch_prolong(const dg_ctx* lo, const dg_ctx* hi, const double* ql, double* qh, const double* Idev,
                           cudaStream_t st);
// host[0..n) = src[0..n), then *flag as an int in the next slot; host is pinned host memory
// (the SMs write it through the coherent mapping).  n < 1024.
cudaError_t launch_store_host(const double* src, int n, const int* flag, double* host, cudaStream_t st);
cudaError_t launch_diagnostics(const dg_ctx* c, const double* q, const double* R, const double* qref,
                               double* partial, int nblocks, double* out, cudaStream_t st);
cudaError_t launch_make_pairs(const dg_ctx* lo, const double* qb_n, const double* qnn_np1, const double* qb_np1,
                              double dt, int first_var, int n_vars, float* X, float* Y, cudaStream_t st);
// Face traces of a slab (element-layer partition).  pack: the owned boundary layers'
// faces normal to z, from the first owned layer's lower faces into send_lo and the last
// owned layer's upper faces into send_hi; unpack: recv_lo into the lower ghost layer's
// upper faces, recv_hi into the upper ghost layer's lower faces.  Buffer layout
// [component][element of the layer][face node].
//   what 0: the FP64 state q (5 doubles per face node);
//   what 1: the FP32 stage state qn32 + dlt (5 floats; unpacked into qn32, the ghost dlt
//           stays zero);
//   what 2: the operator-precision stage state qf and the z-normal viscous quantities
//           (tau_xz, tau_yz, tau_zz, k theta_z): 9 values.
cudaError_t launch_trace_pack(const dg_ctx* c, const double* q, int what, void* send_lo, void* send_hi,
                              cudaStream_t st);
cudaError_t launch_trace_unpack(const dg_ctx* c, double* q, int what, const void* recv_lo, const void* recv_hi,
                                cudaStream_t st);
// Bytes of one side's traces for `what`.
size_t trace_bytes_for(const dg_ctx* c, int what);

// q += dt s on the forced variables (Algorithm 1's correction after the step).
cudaError_t launch_add_forcing(const dg_ctx* c, double* q, const Forcing& f, double dt, cudaStream_t st);

// Operator kernels per precision (dg_kernels_f32.cu / dg_kernels_f64.cu).
cudaError_t gradient_f32(const dg_ctx* c, const double* q, int src, cudaStream_t st);
cudaError_t gradient_f64(const dg_ctx* c, const double* q, int src, cudaStream_t st);
cudaError_t flux_f32(const dg_ctx* c, double* q, double* dqdt, const Forcing& f, int mode, double A, double B,
                     double dt, double invB1, cudaStream_t st);
cudaError_t flux_split_f32(const dg_ctx* c, double* q, double* dqdt, const Forcing& f, int mode, double A, double B,
                           double dt, double invB1, cudaStream_t st);
cudaError_t flux_split_f64(const dg_ctx* c, double* q, double* dqdt, const Forcing& f, int mode, double A, double B,
                           double dt, double invB1, cudaStream_t st);
cudaError_t flux_f64(const dg_ctx* c, double* q, double* dqdt, const Forcing& f, int mode, double A, double B,
                     double dt, double invB1, cudaStream_t st);

// The same for slab contexts (dg_kernels_f32_slab.cu, dg_kernels_f64_slab.cu).
cudaError_t gradient_f32_slab(const dg_ctx* c, const double* q, int src, cudaStream_t st);
cudaError_t gradient_f64_slab(const dg_ctx* c, const double* q, int src, cudaStream_t st);
cudaError_t flux_f32_slab(const dg_ctx* c, double* q, double* dqdt, const Forcing& f, int mode, double A, double B,
                          double dt, double invB1, cudaStream_t st);
cudaError_t flux_f64_slab(const dg_ctx* c, double* q, double* dqdt, const Forcing& f, int mode, double A, double B,
                          double dt, double invB1, cudaStream_t st);
cudaError_t flux_split_f32_slab(const dg_ctx* c, double* q, double* dqdt, const Forcing& f, int mode, double A,
                                double B, double dt, double invB1, cudaStream_t st);
cudaError_t flux_split_f64_slab(const dg_ctx* c, double* q, double* dqdt, const Forcing& f, int mode, double A,
                                double B, double dt, double invB1, cudaStream_t st);
cudaError_t prepare_f32_slab_constants();

// Derivative matrices in the constant memory of the FP32 kernels (dg_kernels_f32.cu,
// dg_batch_f32.cu); once per device, before the first FP32 launch.
cudaError_t prepare_f32_constants();
cudaError_t prepare_batch_f32_constants();

// Batched RK stage k for n instances of order P sharing precision and elements per block
// (dg_batch_f32.cu / dg_batch_f64.cu): q[i] is instance i's FP64 state, dt[i] its step.
cudaError_t batch_stage_f32(int P, dg_ctx* const* ctx, double* const* q, const double* dt, int n, int k, double A,
                            double B, double invB1, cudaStream_t st);
// Sets the kernels' shared-memory attributes for order P at E elements per block; call
// before batch_stage_* (never inside a stream capture).
cudaError_t batch_prepare_f32(int P, int E);
cudaError_t batch_prepare_f64(int P, int E);
cudaError_t batch_stage_f64(int P, dg_ctx* const* ctx, double* const* q, const double* dt, int n, int k, double A,
                            double B, double invB1, cudaStream_t st);

// Persistent batched RK stage (dg_batch_persist.cu, FP32 operator, orders 1..6): one
// cooperative launch per stage for every member; bar: the grid barrier's two counters
// (zero before the first stage of a step).  prepare sets the kernels' shared-memory
// attribute for the orders present and returns the shared memory and co-resident grid.
bool batch_persistent_ok(int P);
cudaError_t batch_persistent_prepare(const int* orders, int n, size_t* smem, int* grid);
cudaError_t batch_persistent_stage(dg_ctx* const* ctx, double* const* q, const double* dt, int n, int k, double A,
                                   double B, double invB1, unsigned* bar, size_t smem, int grid, cudaStream_t st);

}  // namespace dgnn

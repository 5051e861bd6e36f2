// Internal declarations shared by the translation units of libdgnn.so.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <string>

#include "../../include/dgnn.h"

namespace dgnn {

constexpr int kMaxP = 8;
constexpr int kMaxN1 = kMaxP + 1;

// Thread-local error message; returns the status for convenient `return fail(...)`.
int fail(int status, const std::string& msg);
int cuda_fail(cudaError_t err, const char* what);

#define DG_CUDA(call)                                              \
  do {                                                             \
    cudaError_t e_ = (call);                                       \
    if (e_ != cudaSuccess) return ::dgnn::cuda_fail(e_, #call);    \
  } while (0)

// 1D Gauss-Lobatto basis of order P, built on the host in FP64.
struct Basis1D {
  int P = 0;
  double xi[kMaxN1];
  double w[kMaxN1];
  double D[kMaxN1 * kMaxN1];  // D[i * n + m] = l_m'(xi_i)
};
int build_basis(int P, Basis1D* out);
// Filter G of Eq. 2 in 1D: (P_lo+1) x (P_hi+1), row-major.
int build_filter(int P_hi, int P_lo, double* G);
// Interpolation from the order-P_lo nodes to the order-P_hi nodes in 1D, (P_hi+1) x
// (P_lo+1) row-major: I[a][j] = l_j(xi_hi_a), l_j the Lagrange basis on the P_lo nodes.
int build_prolongation(int P_lo, int P_hi, double* I);

// Mesh and basis constants passed by value to every kernel.
struct Geom {
  int K;            // elements per direction
  int nel;          // K^3
  long long N;      // nodes = nel * n^3
  int E;            // elements per block
  int cube;         // 1: blocks are 2 x 2 x 2 cubes of elements (E = 8; P <= 3, even K)
  int split;        // 1: kinetic-energy-preserving split-form volume term (rows of elements)
  double two_over_h;
  double winv;      // 1 / w_0 = 1 / w_P
  double D[kMaxN1 * kMaxN1];
};

// Physical constants of the operator.  The operator works on the state relative to a
// constant reference (rho_ref, E_ref): r = rho - rho_ref, e = rho e - E_ref, with
// p' = p - p_ref and theta' = theta - p_ref / rho_ref.  Constant parts of the fluxes
// have zero divergence and cancel in the interface terms, so the operator is unchanged;
// in FP32 this keeps the Mach-0.1 background pressure (p0 ~ 71) out of the momentum
// flux derivatives.  The FP64 operator uses zero references (the plain formulas).
struct Phys {
  double gamma;
  double mu;         // 1 / Re
  double lam;        // mu gamma / ((gamma-1) Pr): heat coefficient on grad(p/rho)
  int les;           // Smagorinsky on/off
  double csd2;       // (Cs * delta)^2
  double lam_t;      // gamma / ((gamma-1) Prt): turbulent heat coefficient per unit mu_t
  double rho_ref, E_ref, p_ref;  // reference state (zero in the FP64 operator)
  double Hc;         // E_ref + p_ref: constant part of the total enthalpy flux density
  double theta_ref;  // p_ref / rho_ref
};

// Network features that a phase-A launch writes besides its outputs (Sec. 2.2: the
// element's scaled state): out[e * ld + slot * n^3 + node] = bf16((s_v - mean_f) / sd_f)
// for v = first_var + slot, from the stage state s the launch forms; mean_f is taken
// relative to the operator's reference state (shift32, FP32 operator) or as is (mean64,
// FP64 operator).  out == nullptr: none.
struct FeatureOut {
  void* out = nullptr;   // bf16
  int ld = 0;
  int first_var = 0;
  int n_vars = 0;
  const float* shift32 = nullptr;
  const double* mean64 = nullptr;
  const float* sd = nullptr;
};

// Optional forcing source added to the operator: s[e * stride + slot * n^3 + node]
// for variables first_var .. first_var + n_vars - 1.
struct Forcing {
  const float* s = nullptr;
  int first_var = 0;
  int n_vars = 0;
  int stride = 0;
};

}  // namespace dgnn

// The solver context behind the opaque dg_ctx handle.
struct dg_ctx {
  int K = 0, P = 0, n = 0, np = 0;
  int closure = 0;
  double Re = 0, Mach = 0, Pr = 0;
  dg_opts opts{};
  dgnn::Basis1D basis;
  dgnn::Geom geom{};
  dgnn::Phys phys{};
  long long N = 0;   // nodes of the local arrays (a slab: its own layers and two ghost layers)
  int nel = 0;       // elements of the local arrays
  // Owned elements [e_begin, e_end) of the local K x K x Kz element array.  A whole mesh:
  // 0, K^3, Kz = K.  A slab of the periodic mesh (dg_create_part): global element layers
  // [z_begin, z_begin + z_count) at local layers 1 .. z_count, with one ghost layer on
  // each side (local layers 0 and z_count + 1) that holds the neighbouring layers' face
  // data, filled by the trace exchange before each phase.
  int part = 0;
  int z_begin = 0, z_count = 0, Kz = 0;
  int e_begin = 0, e_end = 0;
  void* trace[4] = {};           // device face-trace buffers: send_lo, send_hi, recv_lo, recv_hi
  size_t trace_bytes = 0;        // bytes of each buffer
  dg_exchange_fn xfn = nullptr;  // exchange of a slab's traces with its neighbours (dg_part_set_exchange)
  void* xuser = nullptr;
  // workspace (device)
  void* qf = nullptr;     // operator-precision stage state (reference-shifted), [5][N]
  float* qn32 = nullptr;  // FP32 operator: reference-shifted FP32 image of q at the step start, [5][N]
  float* dlt = nullptr;   // FP32 operator: RK increment accumulated within the step, [5][N]
  void* vis = nullptr;    // viscous stresses and heat flux, [9][N] operator precision
  void* g = nullptr;      // RK register [5][N] (double or float)
  double* rhs_tmp = nullptr;  // [5][N] FP64 operator value for diagnostics
  double* red = nullptr;  // reduction partials
  int red_blocks = 0;
  double* red_host = nullptr;  // pinned host copy of the final reduction
  double* q_dev = nullptr;     // device state for dg_advance_host
  int* err_dev = nullptr;      // device error flag: a bounded wait in a kernel expired
  // dg_advance_host_async calls in flight (at most two, on one stream), oldest at slot
  // host_head: each has an event after its last copy and, if it asked for diagnostics,
  // its results in its slot of the pinned ring [2][kHostSlot]
  int host_pending = 0, host_head = 0;
  bool host_want[2] = {};
  cudaEvent_t host_evt[2] = {};
  cudaStream_t host_stream = nullptr;
  double* host_ring = nullptr;
  double* host_ring_dev = nullptr;   // the ring's device address (cudaHostGetDevicePointer)
  int forcing_mode = DG_FORCING_STAGE;  // where dg_rk3_step applies a network forcing
  float* s_buf = nullptr;      // forcing buffer [nel][5 n^3]
  dgnn::FeatureOut feat_out;   // features the next phase-A launch also writes (set per launch)
  double* filter_dev[dgnn::kMaxP + 1] = {};  // filter G to each lower order (dg_project)
  double* prolong_dev[dgnn::kMaxP + 1] = {};  // interpolation to each higher order (dg_prolong)
  bool borrowed = false;       // member of a dg_batch: released by dg_batch_destroy only
};

namespace dgnn {

// Launchers of the operator kernels.  All return cudaError_t.
// Phase A.  src 0: stage state from q (FP64); src 1: from qn32 + dlt (FP32 operator,
// RK stages 2 and 3).
cudaError_t launch_gradient(const dg_ctx* c, const double* q, int src, cudaStream_t st);
// Phase B.  mode 0: dqdt = R (+ s).  mode 1: FP64 RK stage, g = A g + dt R, q += B g.
// modes 2, 3, 4: FP32 operator RK stages 1, 2, 3 on the FP32 increment; stage 3 adds
// the increment to the FP64 state.
cudaError_t launch_flux(const dg_ctx* c, double* q, double* dqdt, const Forcing& f, int mode,
                        double rkA, double rkB, double dt, cudaStream_t st);

// Fills the sizes, basis, geometry and physics constants of a context from validated
// arguments (host only; no device memory is touched).  Shared by dg_create and the
// no-allocation operator so that both run the kernels with the same constants.
int setup_ctx(dg_ctx* c, int K, int P, double Re, double Mach, double Pr, int closure, const dg_opts& o);
// dg_create for a local array of K x K x Kz elements (Kz = K: the whole periodic mesh).
int dg_create_local(int K, int P, double Re, double Mach, double Pr, int closure, const dg_opts* opts, int Kz,
                    dg_ctx** out);

}  // namespace dgnn

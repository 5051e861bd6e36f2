// C ABI of libdgnn.so (declared in include/dgnn.h): context management and the
// solver entry points.  Argument checking, workspace ownership and stage sequencing
// live here; all arithmetic runs in the kernels.
#include <cmath>
#include <cstdio>
#include <cstring>
#include <string>
#include <vector>

#include "dg_aux.h"
#include "dg_kernels.cuh"
#include "nn_bridge.h"
#include "tc_common.cuh"

namespace dgnn {

namespace {
thread_local std::string g_last_error;

// Williamson (1980) 2N-storage RK3 coefficients (the paper's third-order three-stage
// Runge-Kutta scheme, Sec. 3.1, is unnamed; this is the reading).
constexpr double kRkA[3] = {0.0, -5.0 / 9.0, -153.0 / 128.0};
constexpr double kRkB[3] = {1.0 / 3.0, 15.0 / 16.0, 8.0 / 15.0};

int default_elems_per_block(int P) {
  static const int E[9] = {0, 32, 16, 4, 2, 2, 1, 1, 1};
  return E[P];
}

int max_elems_per_block(int P) {
  const int np = (P + 1) * (P + 1) * (P + 1);
  int E = 1;
  while (((E + 1) * np + 31) / 32 * 32 <= max_threads_for(P)) ++E;
  return E;
}
}  // namespace

int fail(int status, const std::string& msg) {
  g_last_error = msg;
  return status;
}

int cuda_fail(cudaError_t err, const char* what) {
  return fail(DG_ERR_CUDA, std::string(what) + ": " + cudaGetErrorString(err));
}

cudaError_t launch_gradient(const dg_ctx* c, const double* q, int src, cudaStream_t st) {
  const bool f32 = c->opts.precision == DG_PREC_FP32;
  if (c->part) return f32 ? gradient_f32_slab(c, q, src, st) : gradient_f64_slab(c, q, src, st);
  return f32 ? gradient_f32(c, q, src, st) : gradient_f64(c, q, src, st);
}

cudaError_t launch_flux(const dg_ctx* c, double* q, double* dqdt, const Forcing& f, int mode, double A, double B,
                        double dt, cudaStream_t st) {
  const double invB1 = 1.0 / kRkB[0];
  if (c->part) {
    const bool f32 = c->opts.precision == DG_PREC_FP32;
    if (c->geom.split)
      return f32 ? flux_split_f32_slab(c, q, dqdt, f, mode, A, B, dt, invB1, st)
                 : flux_split_f64_slab(c, q, dqdt, f, mode, A, B, dt, invB1, st);
    return f32 ? flux_f32_slab(c, q, dqdt, f, mode, A, B, dt, invB1, st)
               : flux_f64_slab(c, q, dqdt, f, mode, A, B, dt, invB1, st);
  }
  if (c->geom.split)
    return c->opts.precision == DG_PREC_FP32 ? flux_split_f32(c, q, dqdt, f, mode, A, B, dt, invB1, st)
                                             : flux_split_f64(c, q, dqdt, f, mode, A, B, dt, invB1, st);
  return c->opts.precision == DG_PREC_FP32 ? flux_f32(c, q, dqdt, f, mode, A, B, dt, invB1, st)
                                           : flux_f64(c, q, dqdt, f, mode, A, B, dt, invB1, st);
}

// Launch plan of RK stage k (0, 1, 2): source of the phase-A stage state and phase-B mode.
static void stage_plan(const dg_ctx* c, int k, int* src, int* mode) {
  if (c->opts.precision == DG_PREC_FP32) {
    *src = (k == 0) ? 0 : 1;
    *mode = 2 + k;
  } else {
    *src = 0;
    *mode = 1;
  }
}

// Algorithmic bytes per node of the phase-A and phase-B launches of stage k: every value
// the kernel must read or write once (neighbour interface reads are L2 hits, not counted).
static void stage_bytes(const dg_ctx* c, int k, double* grad, double* flux) {
  if (c->opts.precision == DG_PREC_FP32) {
    const double A[3] = {40 + 20 + 20 + 36, 20 + 20 + 20 + 36, 20 + 20 + 20 + 36};
    const double B[3] = {20 + 36 + 20, 20 + 36 + 20 + 20 + 20, 20 + 36 + 20 + 20 + 40 + 40};
    *grad = A[k];
    *flux = B[k];
  } else {
    *grad = 40 + 40 + 72;
    *flux = 40 + 72 + (k ? 40 : 0) + 40 + 40 + 40;
  }
}

// Evaluates the network forcing on the current state q (all elements) into c->s_buf;
// features_ready: the phase-A launch before it wrote the network's input features.
static int forcing_for(dg_ctx* c, const double* q, const nn_model* net, Forcing* f, cudaStream_t st,
                       bool features_ready = false) {
  *f = Forcing{};
  if (!net) return DG_OK;
  int first = 0, nv = 0;
  int rc = nn_forcing_on_state(net, c, q, c->s_buf, &first, &nv, st, features_ready);
  if (rc) return rc;
  f->s = c->s_buf;
  f->first_var = first;
  f->n_vars = nv;
  f->stride = nv * c->np;
  return DG_OK;
}

// Trace exchange of slabs before a phase (what: see launch_trace_pack): every part packs
// its owned boundary faces; a group of slabs of one mesh on this device moves them by
// device copies between neighbours (a single slab that spans the mesh: onto itself); a
// single slab with an exchange function hands its buffers to that function; every part
// then unpacks into its ghost layers.  Whole-mesh contexts exchange nothing.
static int exchange_traces(dg_ctx* const* cs, int n, double* const* qs, int what, cudaStream_t st) {
  if (!cs[0]->part) return DG_OK;
  for (int i = 0; i < n; ++i) DG_CUDA(launch_trace_pack(cs[i], qs[i], what, cs[i]->trace[0], cs[i]->trace[1], st));
  const size_t bytes = trace_bytes_for(cs[0], what);
  if (n == 1 && cs[0]->xfn) {
    const int rc = cs[0]->xfn(cs[0]->xuser, what, cs[0]->trace[0], cs[0]->trace[1], cs[0]->trace[2],
                              cs[0]->trace[3], bytes, (void*)st);
    if (rc != 0) return fail(DG_ERR_EXCHANGE, "the slab's exchange function returned " + std::to_string(rc));
  } else {
    for (int i = 0; i < n; ++i) {
      const dg_ctx* lower = cs[(i + n - 1) % n];
      const dg_ctx* upper = cs[(i + 1) % n];
      DG_CUDA(cudaMemcpyAsync(cs[i]->trace[2], lower->trace[1], bytes, cudaMemcpyDeviceToDevice, st));
      DG_CUDA(cudaMemcpyAsync(cs[i]->trace[3], upper->trace[0], bytes, cudaMemcpyDeviceToDevice, st));
    }
  }
  for (int i = 0; i < n; ++i)
    DG_CUDA(launch_trace_unpack(cs[i], qs[i], what, cs[i]->trace[2], cs[i]->trace[3], st));
  return DG_OK;
}

// Phase-A trace of stage state source src (0: the FP64 state; 1: the FP32 increment scheme).
static int phase_a_what(const dg_ctx* c, int src) { return (c->opts.precision == DG_PREC_FP32 && src == 1) ? 1 : 0; }
constexpr int kWhatPhaseB = 2;

// dq/dt of n contexts: one whole mesh, or the slabs of one mesh exchanging traces.
static int rhs_into_n(dg_ctx* const* cs, int n, double* const* qs, double* const* outs, const nn_model* net,
                      cudaStream_t st) {
  int rc = exchange_traces(cs, n, qs, phase_a_what(cs[0], 0), st);
  if (rc) return rc;
  const bool feats = n == 1 && net && nn_phase_a_features(net, cs[0], &cs[0]->feat_out);
  for (int i = 0; i < n; ++i) {
    const cudaError_t e = launch_gradient(cs[i], qs[i], 0, st);
    cs[i]->feat_out = FeatureOut{};
    DG_CUDA(e);
  }
  Forcing f;
  if (n == 1) {
    rc = forcing_for(cs[0], qs[0], net, &f, st, feats);
    if (rc) return rc;
  }
  rc = exchange_traces(cs, n, qs, kWhatPhaseB, st);
  if (rc) return rc;
  for (int i = 0; i < n; ++i) DG_CUDA(launch_flux(cs[i], qs[i], outs[i], f, 0, 0.0, 0.0, 0.0, st));
  return DG_OK;
}

static int rhs_into(dg_ctx* c, const double* q, double* out, const nn_model* net, cudaStream_t st) {
  double* qq = const_cast<double*>(q);
  return rhs_into_n(&c, 1, &qq, &out, net, st);
}

// With a network forcing: DG_FORCING_STAGE adds s(q_k) to the operator in every stage
// (Eq. 4 integrated by RK3); DG_FORCING_POST evaluates s once on q^n (the stage-1 state),
// takes the uncorrected step and adds dt s(q^n) (Algorithm 1, third loop).  n > 1: the
// slabs of one mesh advanced in lockstep (no forcing).  exchange = false (the autotuner's
// timing on a scratch state) skips the slabs' trace exchange.
static int rk3_steps_n(dg_ctx* const* cs, int n, double* const* qs, double dt, int nsteps, const nn_model* net,
                       cudaStream_t st, bool exchange = true) {
  dg_ctx* c = cs[0];
  const bool post = net && c->forcing_mode == DG_FORCING_POST;
  for (int s = 0; s < nsteps; ++s) {
    Forcing fpost;
    for (int k = 0; k < 3; ++k) {
      int src, mode;
      stage_plan(c, k, &src, &mode);
      int rc = exchange ? exchange_traces(cs, n, qs, phase_a_what(c, src), st) : DG_OK;
      if (rc) return rc;
      // the forcing's input features come out of the phase-A launch when the network allows
      const bool want = net && (!post || k == 0);
      const bool feats = want && n == 1 && nn_phase_a_features(net, c, &c->feat_out);
      for (int i = 0; i < n; ++i) {
        const cudaError_t e = launch_gradient(cs[i], qs[i], src, st);
        cs[i]->feat_out = FeatureOut{};
        DG_CUDA(e);
      }
      Forcing f;
      if (want) {
        rc = forcing_for(c, qs[0], net, &f, st, feats);
        if (rc) return rc;
      }
      if (post) {
        if (k == 0) fpost = f;
        f = Forcing{};
      }
      rc = exchange ? exchange_traces(cs, n, qs, kWhatPhaseB, st) : DG_OK;
      if (rc) return rc;
      for (int i = 0; i < n; ++i) DG_CUDA(launch_flux(cs[i], qs[i], nullptr, f, mode, kRkA[k], kRkB[k], dt, st));
    }
    if (post) DG_CUDA(launch_add_forcing(c, qs[0], fpost, dt, st));
  }
  return DG_OK;
}

static int rk3_steps(dg_ctx* c, double* q, double dt, int nsteps, const nn_model* net, cudaStream_t st,
                     bool exchange = true) {
  return rk3_steps_n(&c, 1, &q, dt, nsteps, net, st, exchange);
}

// Diagnostics in two parts: the reductions and the copy of their result into a pinned
// host buffer (the context's, or a slot of its host-advance ring) are enqueued on st;
// diag_collect waits for st and fills out from the context's buffer.
constexpr int kHostSlot = kDiagLen + 1;   // the diagnostics and the error flag
// slot: the device address of a mapped host-advance slot, or NULL for the context's buffer.
static int diag_enqueue(dg_ctx* c, const double* q, const double* qref, const nn_model* net, bool with_rhs,
                        cudaStream_t st, double* slot = nullptr) {
  double* host = slot ? slot : c->red_host;
  const double* R = nullptr;
  if (with_rhs) {
    int rc = rhs_into(c, q, c->rhs_tmp, net, st);
    if (rc) return rc;
    R = c->rhs_tmp;
  }
  double* dev_out = c->red + (size_t)c->red_blocks * kDiagLen;
  DG_CUDA(launch_diagnostics(c, q, R, qref, c->red, c->red_blocks, dev_out, st));
  // the kernels' error flag rides along in the slot after the diagnostics.  A host-advance
  // slot is written by a kernel (its few bytes do not wait behind other streams' state
  // copies on the copy engine); the synchronous paths copy.
  if (slot) {
    DG_CUDA(launch_store_host(dev_out, kDiagLen, c->err_dev, host, st));
    return DG_OK;
  }
  DG_CUDA(cudaMemcpyAsync(host, dev_out, kDiagLen * sizeof(double), cudaMemcpyDeviceToHost, st));
  DG_CUDA(cudaMemcpyAsync(host + kDiagLen, c->err_dev, sizeof(int), cudaMemcpyDeviceToHost, st));
  return DG_OK;
}

// Fills out from the copied diagnostics r (and their error flag).
static int diag_parse(dg_ctx* c, const double* r, bool with_rhs, bool with_ref, dg_diag* out) {
  int err = 0;
  std::memcpy(&err, r + kDiagLen, sizeof(int));
  if (err) {
    DG_CUDA(cudaMemset(c->err_dev, 0, sizeof(int)));
    return fail(DG_ERR_TIMEOUT, "a bounded wait in the streamed flux kernel expired (its results are invalid)");
  }
  const double vol = 8.0 * M_PI * M_PI * M_PI;
  std::memset(out, 0, sizeof(*out));
  out->mass = r[0];
  for (int i = 0; i < 3; ++i) out->momentum[i] = r[1 + i];
  out->energy = r[4];
  out->ke = r[5] / vol;
  out->dke_dt = with_rhs ? r[6] / vol : 0.0;
  out->nonfinite = (int64_t)r[kDiagNonfinite];
  for (int i = 0; i < 3; ++i) out->e_inf[i] = with_ref ? r[8 + i] : 0.0;
  out->max_wave = r[11];
  return out->nonfinite ? fail(DG_ERR_NONFINITE, "state holds non-finite values") : DG_OK;
}

static int diag_collect(dg_ctx* c, bool with_rhs, bool with_ref, dg_diag* out, cudaStream_t st) {
  DG_CUDA(cudaStreamSynchronize(st));
  return diag_parse(c, c->red_host, with_rhs, with_ref, out);
}

static int diagnostics_into(dg_ctx* c, const double* q, const double* qref, const nn_model* net, bool with_rhs,
                            dg_diag* out, cudaStream_t st) {
  int rc = diag_enqueue(c, q, qref, net, with_rhs, st);
  if (rc) return rc;
  return diag_collect(c, with_rhs, qref != nullptr, out, st);
}

int setup_ctx(dg_ctx* c, int K, int P, double Re, double Mach, double Pr, int closure, const dg_opts& o) {
  c->K = K;
  c->P = P;
  c->n = P + 1;
  c->np = c->n * c->n * c->n;
  c->nel = K * K * K;
  c->N = (long long)c->nel * c->np;
  c->Kz = K;
  c->e_begin = 0;
  c->e_end = c->nel;
  c->closure = closure;
  c->Re = Re;
  c->Mach = Mach;
  c->Pr = Pr;
  c->opts = o;
  int rc = build_basis(P, &c->basis);
  if (rc) return rc;
  const double h = 2.0 * M_PI / K;
  c->geom.K = K;
  c->geom.nel = c->nel;
  c->geom.N = c->N;
  c->geom.E = o.elems_per_block > 0 ? o.elems_per_block : default_elems_per_block(P);
  c->geom.cube = o.block_shape;
  if (c->geom.cube) c->geom.E = kCubeElems;
  c->geom.split = o.volume_flux;
  c->geom.two_over_h = 2.0 / h;
  c->geom.winv = 1.0 / c->basis.w[0];
  std::memset(c->geom.D, 0, sizeof(c->geom.D));
  std::memcpy(c->geom.D, c->basis.D, sizeof(double) * c->n * c->n);
  const double g = o.gamma;
  c->phys.gamma = g;
  c->phys.mu = 1.0 / Re;
  c->phys.lam = c->phys.mu * g / ((g - 1.0) * Pr);
  c->phys.les = closure;
  const double delta = o.les_delta > 0 ? o.les_delta : h / (P + 1);
  c->phys.csd2 = (o.Cs * delta) * (o.Cs * delta);
  c->phys.lam_t = g / ((g - 1.0) * o.Prt);
  if (o.precision == DG_PREC_FP32) {
    // reference state: rho0 = 1 and the background pressure p0 = 1/(gamma M^2)
    c->phys.rho_ref = 1.0;
    c->phys.p_ref = 1.0 / (g * Mach * Mach);
    c->phys.E_ref = c->phys.p_ref / (g - 1.0);
  } else {
    c->phys.rho_ref = c->phys.p_ref = c->phys.E_ref = 0.0;
  }
  c->phys.Hc = c->phys.E_ref + c->phys.p_ref;
  c->phys.theta_ref = c->phys.rho_ref > 0 ? c->phys.p_ref / c->phys.rho_ref : 0.0;
  return DG_OK;
}

// A slab evaluates the operator only with its neighbours' traces: it needs an exchange
// function unless it spans the whole mesh (its own lower and upper faces are then its
// neighbours').  The network forcing is not offered on slabs.
static int part_usable(const dg_ctx* c, const nn_model* net, const char* who) {
  if (!c->part) return DG_OK;
  if (net) return fail(DG_ERR_UNSUPPORTED, std::string(who) + ": no network forcing on a slab (dg_create_part)");
  if (!c->xfn && c->z_count < c->K)
    return fail(DG_ERR_INVALID_ARG, std::string(who) + ": a slab needs an exchange function (dg_part_set_exchange) "
                                                       "or a group call (dg_group_*)");
  return DG_OK;
}

// The parts of a group call must be the slabs of one mesh in order: same mesh, order,
// flow and precision, consecutive layers covering 0 .. K-1, states given for each.
static int check_group(dg_ctx* const* parts, int n, double* const* q, const char* who) {
  if (!parts || !q || n < 1) return fail(DG_ERR_INVALID_ARG, std::string(who) + ": NULL argument or n < 1");
  int z = 0;
  for (int i = 0; i < n; ++i) {
    const dg_ctx* c = parts[i];
    if (!c || !q[i]) return fail(DG_ERR_INVALID_ARG, std::string(who) + ": NULL part or state");
    if (!c->part) return fail(DG_ERR_INVALID_ARG, std::string(who) + ": part " + std::to_string(i) + " is not a slab");
    const dg_ctx* a = parts[0];
    if (c->K != a->K || c->P != a->P || c->Re != a->Re || c->Mach != a->Mach || c->Pr != a->Pr ||
        c->closure != a->closure || c->opts.precision != a->opts.precision || c->geom.split != a->geom.split)
      return fail(DG_ERR_INVALID_ARG, std::string(who) + ": parts of different meshes, orders, flows or precisions");
    if (c->z_begin != z)
      return fail(DG_ERR_INVALID_ARG, std::string(who) + ": part " + std::to_string(i) + " does not start at layer " +
                                          std::to_string(z));
    z += c->z_count;
  }
  if (z != parts[0]->K) return fail(DG_ERR_INVALID_ARG, std::string(who) + ": the parts do not cover the K layers");
  return DG_OK;
}

}  // namespace dgnn

using namespace dgnn;

extern "C" {

int dg_create_part(int K, int P, double Re, double Mach, double Pr, int closure, const dg_opts* opts, int z_begin,
                   int z_count, dg_ctx** out) {
  if (!out) return fail(DG_ERR_INVALID_ARG, "dg_create_part: out is NULL");
  *out = nullptr;
  if (K < 1 || K > 256) return fail(DG_ERR_INVALID_ARG, "dg_create_part: K must be in [1, 256]");
  if (z_begin < 0 || z_count < 1 || z_begin + z_count > K)
    return fail(DG_ERR_INVALID_ARG, "dg_create_part: layers [z_begin, z_begin + z_count) must lie in [0, K)");
  dg_opts o;
  dg_opts_default(&o);
  if (opts) o = *opts;
  if (o.block_shape != 0) return fail(DG_ERR_INVALID_ARG, "dg_create_part: slabs run rows of elements (block_shape 0)");
  // a whole-mesh context for the slab's local array of z_count + 2 layers: same checks,
  // basis and constants; its element and node counts are then the local ones
  dg_ctx* c = nullptr;
  int rc = dg_create_local(K, P, Re, Mach, Pr, closure, &o, z_count + 2, &c);
  if (rc) return rc;
  if (o.precision == DG_PREC_FP32) {
    const cudaError_t ec = prepare_f32_slab_constants();
    if (ec != cudaSuccess) {
      dg_destroy(c);
      return cuda_fail(ec, "dg_create_part: constant tables");
    }
  }
  c->part = 1;
  c->z_begin = z_begin;
  c->z_count = z_count;
  c->e_begin = K * K;
  c->e_end = K * K * (z_count + 1);
  size_t tb = 0;
  for (int w = 0; w < 3; ++w) tb = std::max(tb, trace_bytes_for(c, w));
  c->trace_bytes = tb;
  cudaError_t e = cudaSuccess;
  for (int i = 0; i < 4 && e == cudaSuccess; ++i) e = cudaMalloc(&c->trace[i], tb);
  // the ghost layers' FP32 increment stays zero: their stage state arrives whole in qn32
  if (e == cudaSuccess && c->dlt) e = cudaMemset(c->dlt, 0, 5 * c->N * sizeof(float));
  if (e != cudaSuccess) {
    dg_destroy(c);
    return cuda_fail(e, "dg_create_part: trace buffers");
  }
  *out = c;
  return DG_OK;
}

int dg_part_layout(const dg_ctx* c, int* z_begin, int* z_count, int64_t* first_owned_node, int64_t* owned_nodes) {
  if (!c) return fail(DG_ERR_INVALID_ARG, "dg_part_layout: NULL context");
  if (z_begin) *z_begin = c->part ? c->z_begin : 0;
  if (z_count) *z_count = c->part ? c->z_count : c->K;
  if (first_owned_node) *first_owned_node = (int64_t)c->e_begin * c->np;
  if (owned_nodes) *owned_nodes = (int64_t)(c->e_end - c->e_begin) * c->np;
  return DG_OK;
}

int dg_part_set_exchange(dg_ctx* c, dg_exchange_fn fn, void* user) {
  if (!c) return fail(DG_ERR_INVALID_ARG, "dg_part_set_exchange: NULL context");
  if (!c->part) return fail(DG_ERR_INVALID_ARG, "dg_part_set_exchange: not a slab (dg_create_part)");
  c->xfn = fn;
  c->xuser = user;
  return DG_OK;
}

int dg_part_trace_bytes(const dg_ctx* c, int what, size_t* bytes) {
  if (!c || !bytes) return fail(DG_ERR_INVALID_ARG, "dg_part_trace_bytes: NULL argument");
  if (!c->part) return fail(DG_ERR_INVALID_ARG, "dg_part_trace_bytes: not a slab (dg_create_part)");
  if (what < 0 || what > 2) return fail(DG_ERR_INVALID_ARG, "dg_part_trace_bytes: what must be 0, 1 or 2");
  *bytes = trace_bytes_for(c, what);
  return DG_OK;
}

int dg_group_rk3_step(dg_ctx* const* parts, int n, double* const* q, double dt, int nsteps, void* stream) {
  int rc = check_group(parts, n, q, "dg_group_rk3_step");
  if (rc) return rc;
  if (nsteps < 0 || !std::isfinite(dt)) return fail(DG_ERR_INVALID_ARG, "dg_group_rk3_step: bad nsteps or dt");
  return rk3_steps_n(parts, n, q, dt, nsteps, nullptr, (cudaStream_t)stream);
}

int dg_group_rhs(dg_ctx* const* parts, int n, double* const* q, double* const* dqdt, void* stream) {
  int rc = check_group(parts, n, q, "dg_group_rhs");
  if (rc) return rc;
  if (!dqdt) return fail(DG_ERR_INVALID_ARG, "dg_group_rhs: NULL dqdt");
  for (int i = 0; i < n; ++i)
    if (!dqdt[i] || dqdt[i] == q[i]) return fail(DG_ERR_INVALID_ARG, "dg_group_rhs: NULL or aliasing dqdt");
  return rhs_into_n(parts, n, q, dqdt, nullptr, (cudaStream_t)stream);
}

int dg_diag_combine(const dg_diag* parts, int n, dg_diag* out) {
  if (!parts || !out || n < 1) return fail(DG_ERR_INVALID_ARG, "dg_diag_combine: NULL argument or n < 1");
  dg_diag r = parts[0];
  for (int i = 1; i < n; ++i) {   // in part order: the same sums on every rank
    const dg_diag& p = parts[i];
    r.mass += p.mass;
    for (int k = 0; k < 3; ++k) r.momentum[k] += p.momentum[k];
    r.energy += p.energy;
    r.ke += p.ke;
    r.dke_dt += p.dke_dt;
    for (int k = 0; k < 3; ++k) r.e_inf[k] = std::max(r.e_inf[k], p.e_inf[k]);
    r.max_wave = std::max(r.max_wave, p.max_wave);
    r.nonfinite += p.nonfinite;
  }
  *out = r;
  return r.nonfinite ? fail(DG_ERR_NONFINITE, "state holds non-finite values") : DG_OK;
}

int dg_group_diagnostics(dg_ctx* const* parts, int n, double* const* q, dg_diag* out, void* stream) {
  int rc = check_group(parts, n, q, "dg_group_diagnostics");
  if (rc) return rc;
  if (!out) return fail(DG_ERR_INVALID_ARG, "dg_group_diagnostics: NULL out");
  cudaStream_t st = (cudaStream_t)stream;
  std::vector<double*> R(n);
  for (int i = 0; i < n; ++i) R[i] = parts[i]->rhs_tmp;
  rc = rhs_into_n(parts, n, q, R.data(), nullptr, st);
  if (rc) return rc;
  std::vector<dg_diag> d(n);
  for (int i = 0; i < n; ++i) {
    dg_ctx* c = parts[i];
    double* dev_out = c->red + (size_t)c->red_blocks * kDiagLen;
    DG_CUDA(launch_diagnostics(c, q[i], c->rhs_tmp, nullptr, c->red, c->red_blocks, dev_out, st));
    DG_CUDA(cudaMemcpyAsync(c->red_host, dev_out, kDiagLen * sizeof(double), cudaMemcpyDeviceToHost, st));
    DG_CUDA(cudaMemcpyAsync(c->red_host + kDiagLen, c->err_dev, sizeof(int), cudaMemcpyDeviceToHost, st));
  }
  for (int i = 0; i < n; ++i) {
    rc = diag_collect(parts[i], true, false, &d[i], st);
    if (rc && rc != DG_ERR_NONFINITE) return rc;
  }
  return dg_diag_combine(d.data(), n, out);
}

int dg_opts_default(dg_opts* o) {
  if (!o) return fail(DG_ERR_INVALID_ARG, "dg_opts_default: NULL");
  std::memset(o, 0, sizeof(*o));
  o->precision = DG_PREC_FP64;
  o->gamma = 1.4;
  o->Cs = 0.1;
  o->Prt = 0.9;
  o->les_delta = 0.0;
  o->elems_per_block = 0;
  return DG_OK;
}

int dg_create(int K, int P, double Re, double Mach, double Pr, int closure, const dg_opts* opts, dg_ctx** out) {
  return dg_create_local(K, P, Re, Mach, Pr, closure, opts, K, out);
}

}  // extern "C"

namespace dgnn {
// dg_create for a local array of K x K x Kz elements (Kz = K: the whole periodic mesh).
int dg_create_local(int K, int P, double Re, double Mach, double Pr, int closure, const dg_opts* opts, int Kz,
                    dg_ctx** out) {
  if (!out) return fail(DG_ERR_INVALID_ARG, "dg_create: out is NULL");
  *out = nullptr;
  if (K < 1 || K > 256) return fail(DG_ERR_INVALID_ARG, "dg_create: K must be in [1, 256]");
  if (P < 1 || P > kMaxP) return fail(DG_ERR_INVALID_ARG, "dg_create: P must be in [1, 8]");
  if (!(Re > 0) || !(Mach > 0) || !(Pr > 0)) return fail(DG_ERR_INVALID_ARG, "dg_create: Re, Mach, Pr must be > 0");
  if (closure != 0 && closure != 1) return fail(DG_ERR_INVALID_ARG, "dg_create: closure must be 0 or 1");
  dg_opts o;
  dg_opts_default(&o);
  if (opts) o = *opts;
  if (o.precision != DG_PREC_FP64 && o.precision != DG_PREC_FP32)
    return fail(DG_ERR_INVALID_ARG, "dg_create: unknown precision");
  if (!(o.gamma > 1.0) || !std::isfinite(o.gamma)) return fail(DG_ERR_INVALID_ARG, "dg_create: gamma must be finite and > 1");
  if (!(o.Cs >= 0.0) || !std::isfinite(o.Cs)) return fail(DG_ERR_INVALID_ARG, "dg_create: Cs must be finite and >= 0");
  if (!(o.Prt > 0.0) || !std::isfinite(o.Prt)) return fail(DG_ERR_INVALID_ARG, "dg_create: Prt must be finite and > 0");
  if (!std::isfinite(o.les_delta)) return fail(DG_ERR_INVALID_ARG, "dg_create: les_delta must be finite");
  if (o.elems_per_block > max_elems_per_block(P))
    return fail(DG_ERR_INVALID_ARG, "dg_create: elems_per_block exceeds the block size limit for this P");
  if (o.block_shape != 0 && o.block_shape != 1) return fail(DG_ERR_INVALID_ARG, "dg_create: block_shape must be 0 or 1");
  if (o.block_shape == 1 && (!cube_ok(P) || K % 2 != 0))
    return fail(DG_ERR_INVALID_ARG, "dg_create: cube blocks need P <= 3 and an even K");
  if (o.volume_flux != 0 && o.volume_flux != 1) return fail(DG_ERR_INVALID_ARG, "dg_create: volume_flux must be 0 or 1");
  if (o.volume_flux == 1 && o.block_shape != 0)
    return fail(DG_ERR_INVALID_ARG, "dg_create: the split-form volume term runs on rows of elements (block_shape 0)");

  dg_ctx* c = new dg_ctx();
  int rc = setup_ctx(c, K, P, Re, Mach, Pr, closure, o);
  if (rc) {
    delete c;
    return rc;
  }
  if (Kz != K) {   // a slab's local array: element and node counts of its Kz layers
    c->Kz = Kz;
    c->nel = K * K * Kz;
    c->N = (long long)c->nel * c->np;
    c->e_end = c->nel;
    c->geom.nel = c->nel;
    c->geom.N = c->N;
  }

  const bool f32 = o.precision == DG_PREC_FP32;
  if (f32) {
    cudaError_t ec = prepare_f32_constants();
    if (ec == cudaSuccess) ec = prepare_batch_f32_constants();
    if (ec != cudaSuccess) {
      delete c;
      return cuda_fail(ec, "dg_create: constant tables");
    }
  }
  const size_t tsz = f32 ? sizeof(float) : sizeof(double);
  c->red_blocks = kDiagBlocks;
  cudaError_t e = cudaSuccess;
  if (e == cudaSuccess) e = cudaMalloc(&c->qf, 5 * c->N * tsz);
  if (e == cudaSuccess) e = cudaMalloc(&c->vis, 9 * c->N * tsz);
  if (e == cudaSuccess) e = cudaMalloc(&c->g, 5 * c->N * tsz);
  if (f32 && e == cudaSuccess) e = cudaMalloc(&c->qn32, 5 * c->N * sizeof(float));
  if (f32 && e == cudaSuccess) e = cudaMalloc(&c->dlt, 5 * c->N * sizeof(float));
  if (e == cudaSuccess) e = cudaMalloc(&c->rhs_tmp, 5 * c->N * sizeof(double));
  if (e == cudaSuccess) e = cudaMalloc(&c->red, (size_t)(c->red_blocks + 1) * kDiagLen * sizeof(double));
  if (e == cudaSuccess) e = cudaMallocHost(&c->red_host, (kDiagLen + 1) * sizeof(double));
  if (e == cudaSuccess) e = cudaMalloc(&c->err_dev, sizeof(int));
  if (e == cudaSuccess) e = cudaMemset(c->err_dev, 0, sizeof(int));
  if (e == cudaSuccess) e = cudaMalloc(&c->s_buf, 5 * c->N * sizeof(float));
  if (e != cudaSuccess) {
    dg_destroy(c);
    return cuda_fail(e, "dg_create: workspace allocation");
  }
  *out = c;
  return DG_OK;
}
}  // namespace dgnn

extern "C" {

int dg_destroy(dg_ctx* c) {
  if (!c) return fail(DG_ERR_INVALID_ARG, "dg_destroy: NULL");
  if (c->borrowed) return fail(DG_ERR_INVALID_ARG, "dg_destroy: the context belongs to a batch (dg_batch_destroy)");
  cudaFree(c->qf);
  cudaFree(c->vis);
  cudaFree(c->g);
  cudaFree(c->qn32);
  cudaFree(c->dlt);
  cudaFree(c->rhs_tmp);
  cudaFree(c->red);
  cudaFree(c->s_buf);
  cudaFree(c->q_dev);
  if (c->red_host) cudaFreeHost(c->red_host);
  if (c->host_ring) cudaFreeHost(c->host_ring);
  for (int i = 0; i < 2; ++i)
    if (c->host_evt[i]) cudaEventDestroy(c->host_evt[i]);
  if (c->err_dev) cudaFree(c->err_dev);
  for (int i = 0; i <= kMaxP; ++i) cudaFree(c->filter_dev[i]);
  for (int i = 0; i <= kMaxP; ++i) cudaFree(c->prolong_dev[i]);
  for (int i = 0; i < 4; ++i) cudaFree(c->trace[i]);
  delete c;
  return DG_OK;
}

int dg_sizes(const dg_ctx* c, int64_t* nodes, int64_t* elems) {
  if (!c) return fail(DG_ERR_INVALID_ARG, "dg_sizes: NULL context");
  if (nodes) *nodes = c->N;
  if (elems) *elems = c->nel;
  return DG_OK;
}

int dg_basis_1d(int P, double* xi, double* w, double* D) {
  Basis1D b;
  int rc = build_basis(P, &b);
  if (rc) return rc;
  const int n = P + 1;
  for (int i = 0; i < n; ++i) {
    if (xi) xi[i] = b.xi[i];
    if (w) w[i] = b.w[i];
  }
  if (D) std::memcpy(D, b.D, sizeof(double) * n * n);
  return DG_OK;
}

int dg_init_tgv(dg_ctx* c, double* q, const double* pert, void* stream) {
  if (!c || !q) return fail(DG_ERR_INVALID_ARG, "dg_init_tgv: NULL argument");
  DG_CUDA(launch_init_tgv(c, q, pert, (cudaStream_t)stream));
  return DG_OK;
}

int dg_rhs(dg_ctx* c, const double* q, double* dqdt, const nn_model* forcing, void* stream) {
  if (!c || !q || !dqdt) return fail(DG_ERR_INVALID_ARG, "dg_rhs: NULL argument");
  if (q == dqdt) return fail(DG_ERR_INVALID_ARG, "dg_rhs: q and dqdt must not alias");
  int rc = part_usable(c, forcing, "dg_rhs");
  if (rc) return rc;
  return rhs_into(c, q, dqdt, forcing, (cudaStream_t)stream);
}

int dg_rk3_step(dg_ctx* c, double* q, double dt, int nsteps, const nn_model* forcing, void* stream) {
  if (!c || !q) return fail(DG_ERR_INVALID_ARG, "dg_rk3_step: NULL argument");
  if (nsteps < 0 || !std::isfinite(dt)) return fail(DG_ERR_INVALID_ARG, "dg_rk3_step: bad nsteps or dt");
  int rc = part_usable(c, forcing, "dg_rk3_step");
  if (rc) return rc;
  return rk3_steps(c, q, dt, nsteps, forcing, (cudaStream_t)stream);
}

int dg_advance_host_async(dg_ctx* c, double* q_host, double dt, int nsteps, const nn_model* forcing, int want_diag,
                          void* stream) {
  if (!c || !q_host) return fail(DG_ERR_INVALID_ARG, "dg_advance_host_async: NULL argument");
  if (nsteps < 0 || !std::isfinite(dt)) return fail(DG_ERR_INVALID_ARG, "dg_advance_host_async: bad nsteps or dt");
  int prc = part_usable(c, forcing, "dg_advance_host_async");
  if (prc) return prc;
  cudaStream_t st = (cudaStream_t)stream;
  if (c->host_pending == 2)
    return fail(DG_ERR_INVALID_ARG, "dg_advance_host_async: two calls pending: collect one with dg_advance_host_wait");
  if (c->host_pending == 1 && st != c->host_stream)
    return fail(DG_ERR_INVALID_ARG, "dg_advance_host_async: a pending call is on another stream");
  const size_t bytes = 5 * c->N * sizeof(double);
  if (!c->q_dev) DG_CUDA(cudaMalloc(&c->q_dev, bytes));
  if (!c->host_ring) {
    DG_CUDA(cudaHostAlloc(&c->host_ring, 2 * kHostSlot * sizeof(double), cudaHostAllocMapped));
    DG_CUDA(cudaHostGetDevicePointer(&c->host_ring_dev, c->host_ring, 0));
    for (int i = 0; i < 2; ++i) DG_CUDA(cudaEventCreateWithFlags(&c->host_evt[i], cudaEventDisableTiming));
  }
  const int slot = (c->host_head + c->host_pending) % 2;
  // a second pending call reuses the device state after the first's copy back (same stream)
  DG_CUDA(cudaMemcpyAsync(c->q_dev, q_host, bytes, cudaMemcpyHostToDevice, st));
  int rc = rk3_steps(c, c->q_dev, dt, nsteps, forcing, st);
  if (rc) return rc;
  DG_CUDA(cudaMemcpyAsync(q_host, c->q_dev, bytes, cudaMemcpyDeviceToHost, st));
  if (want_diag) {
    rc = diag_enqueue(c, c->q_dev, nullptr, forcing, false, st, c->host_ring_dev + slot * kHostSlot);
    if (rc) return rc;
  }
  DG_CUDA(cudaEventRecord(c->host_evt[slot], st));
  c->host_want[slot] = want_diag != 0;
  c->host_stream = st;
  ++c->host_pending;
  return DG_OK;
}

int dg_advance_host_wait(dg_ctx* c, dg_diag* diag, void* stream) {
  if (!c) return fail(DG_ERR_INVALID_ARG, "dg_advance_host_wait: NULL argument");
  if (c->host_pending == 0) {
    DG_CUDA(cudaStreamSynchronize((cudaStream_t)stream));
    if (diag) return fail(DG_ERR_INVALID_ARG, "dg_advance_host_wait: no call is pending");
    return DG_OK;
  }
  // the oldest pending call: its copy back and its diagnostics have landed after its event
  const int slot = c->host_head;
  c->host_head = (slot + 1) % 2;
  --c->host_pending;
  DG_CUDA(cudaEventSynchronize(c->host_evt[slot]));
  if (!diag) return DG_OK;
  if (!c->host_want[slot]) return fail(DG_ERR_INVALID_ARG, "dg_advance_host_wait: no diagnostics were requested");
  return diag_parse(c, c->host_ring + slot * kHostSlot, false, false, diag);
}

int dg_advance_host(dg_ctx* c, double* q_host, double dt, int nsteps, const nn_model* forcing, dg_diag* diag,
                    void* stream) {
  if (!c || !q_host) return fail(DG_ERR_INVALID_ARG, "dg_advance_host: NULL argument");
  if (nsteps < 0 || !std::isfinite(dt)) return fail(DG_ERR_INVALID_ARG, "dg_advance_host: bad nsteps or dt");
  // its wait must collect this call, not an older pending one
  if (c->host_pending) return fail(DG_ERR_INVALID_ARG, "dg_advance_host: dg_advance_host_async calls are pending");
  int rc = dg_advance_host_async(c, q_host, dt, nsteps, forcing, diag != nullptr, stream);
  if (rc) return rc;
  return dg_advance_host_wait(c, diag, stream);
}

int dg_project(const dg_ctx* hi, const dg_ctx* lo, const double* q_hi, double* q_lo, void* stream) {
  if (!hi || !lo || !q_hi || !q_lo) return fail(DG_ERR_INVALID_ARG, "dg_project: NULL argument");
  if (hi->K != lo->K) return fail(DG_ERR_INVALID_ARG, "dg_project: contexts must share K");
  if (lo->P > hi->P) return fail(DG_ERR_INVALID_ARG, "dg_project: needs P_lo <= P_hi");
  dg_ctx* h = const_cast<dg_ctx*>(hi);
  if (!h->filter_dev[lo->P]) {
    double G[kMaxN1 * kMaxN1];
    int rc = build_filter(hi->P, lo->P, G);
    if (rc) return rc;
    DG_CUDA(cudaMalloc(&h->filter_dev[lo->P], sizeof(G)));
    DG_CUDA(cudaMemcpy(h->filter_dev[lo->P], G, sizeof(double) * lo->n * hi->n, cudaMemcpyHostToDevice));
  }
  DG_CUDA(launch_project(hi, lo, q_hi, q_lo, h->filter_dev[lo->P], (cudaStream_t)stream));
  return DG_OK;
}

int dg_prolong(const dg_ctx* lo, const dg_ctx* hi, const double* q_lo, double* q_hi, void* stream) {
  if (!hi || !lo || !q_hi || !q_lo) return fail(DG_ERR_INVALID_ARG, "dg_prolong: NULL argument");
  if (hi->K != lo->K) return fail(DG_ERR_INVALID_ARG, "dg_prolong: contexts must share K");
  if (lo->P > hi->P) return fail(DG_ERR_INVALID_ARG, "dg_prolong: needs P_lo <= P_hi");
  dg_ctx* l = const_cast<dg_ctx*>(lo);
  if (!l->prolong_dev[hi->P]) {
    double I[kMaxN1 * kMaxN1];
    int rc = build_prolongation(lo->P, hi->P, I);
    if (rc) return rc;
    DG_CUDA(cudaMalloc(&l->prolong_dev[hi->P], sizeof(I)));
    DG_CUDA(cudaMemcpy(l->prolong_dev[hi->P], I, sizeof(double) * lo->n * hi->n, cudaMemcpyHostToDevice));
  }
  DG_CUDA(launch_prolong(lo, hi, q_lo, q_hi, l->prolong_dev[hi->P], (cudaStream_t)stream));
  return DG_OK;
}

int dg_diagnostics(dg_ctx* c, const double* q, const double* q_ref, const nn_model* forcing, dg_diag* out,
                   void* stream) {
  if (!c || !q || !out) return fail(DG_ERR_INVALID_ARG, "dg_diagnostics: NULL argument");
  int rc = part_usable(c, forcing, "dg_diagnostics");
  if (rc) return rc;
  return diagnostics_into(c, q, q_ref, forcing, true, out, (cudaStream_t)stream);
}

int dg_stable_dt(dg_ctx* c, const double* q, double cfl, double* dt_out, void* stream) {
  if (!c || !q || !dt_out) return fail(DG_ERR_INVALID_ARG, "dg_stable_dt: NULL argument");
  if (!(cfl > 0)) return fail(DG_ERR_INVALID_ARG, "dg_stable_dt: cfl must be > 0");
  dg_diag d;
  int rc = diagnostics_into(c, q, nullptr, nullptr, false, &d, (cudaStream_t)stream);
  if (rc) return rc;
  const double h = 2.0 * M_PI / c->K;
  *dt_out = cfl * h / ((c->P + 1.0) * (c->P + 1.0) * d.max_wave);
  return DG_OK;
}

int dg_make_pairs(const dg_ctx* lo, const double* q_bar_n, const double* q_nn_np1, const double* q_bar_np1,
                  double dt, int first_var, int n_vars, float* X, float* Y, void* stream) {
  if (!lo || !q_bar_n || !q_nn_np1 || !q_bar_np1 || !X || !Y)
    return fail(DG_ERR_INVALID_ARG, "dg_make_pairs: NULL argument");
  if (!(dt != 0.0) || !std::isfinite(dt)) return fail(DG_ERR_INVALID_ARG, "dg_make_pairs: dt must be finite, nonzero");
  if (first_var < 0 || n_vars < 1 || first_var + n_vars > 5)
    return fail(DG_ERR_INVALID_ARG, "dg_make_pairs: variable range outside 0..4");
  DG_CUDA(launch_make_pairs(lo, q_bar_n, q_nn_np1, q_bar_np1, dt, first_var, n_vars, X, Y, (cudaStream_t)stream));
  return DG_OK;
}

int dg_profile_rk3(dg_ctx* c, double* q, double dt, int nsteps, double* ms_gradient, double* ms_flux,
                   int* launches_gradient, int* launches_flux, double* flux_bytes, double* grad_bytes,
                   void* stream) {
  if (!c || !q) return fail(DG_ERR_INVALID_ARG, "dg_profile_rk3: NULL argument");
  if (nsteps < 1 || !std::isfinite(dt)) return fail(DG_ERR_INVALID_ARG, "dg_profile_rk3: bad nsteps or dt");
  cudaStream_t st = (cudaStream_t)stream;
  const int nl = 3 * nsteps;
  std::vector<cudaEvent_t> ev(4 * nl);
  int created = 0;
  cudaError_t e = cudaSuccess;
  for (; created < 4 * nl && e == cudaSuccess; ++created) e = cudaEventCreate(&ev[created]);
  double tg = 0.0, tf = 0.0, bg = 0.0, bf = 0.0;
  if (e == cudaSuccess) {
    for (int s = 0; s < nsteps && e == cudaSuccess; ++s)
      for (int k = 0; k < 3 && e == cudaSuccess; ++k) {
        const int i = 4 * (3 * s + k);
        int src, mode;
        stage_plan(c, k, &src, &mode);
        double gb, fb;
        stage_bytes(c, k, &gb, &fb);
        bg += gb;
        bf += fb;
        cudaEventRecord(ev[i], st);
        e = launch_gradient(c, q, src, st);
        cudaEventRecord(ev[i + 1], st);
        cudaEventRecord(ev[i + 2], st);
        if (e == cudaSuccess) e = launch_flux(c, q, nullptr, Forcing{}, mode, kRkA[k], kRkB[k], dt, st);
        cudaEventRecord(ev[i + 3], st);
      }
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    for (int l = 0; l < nl && e == cudaSuccess; ++l) {
      float a = 0.f, b = 0.f;
      cudaEventElapsedTime(&a, ev[4 * l], ev[4 * l + 1]);
      cudaEventElapsedTime(&b, ev[4 * l + 2], ev[4 * l + 3]);
      tg += a;
      tf += b;
    }
  }
  for (int i = 0; i < created; ++i) cudaEventDestroy(ev[i]);
  if (e != cudaSuccess) return cuda_fail(e, "dg_profile_rk3");
  if (ms_gradient) *ms_gradient = tg;
  if (ms_flux) *ms_flux = tf;
  if (launches_gradient) *launches_gradient = nl;
  if (launches_flux) *launches_flux = nl;
  if (flux_bytes) *flux_bytes = bf / nl * (double)c->N;
  if (grad_bytes) *grad_bytes = bg / nl * (double)c->N;
  return DG_OK;
}

const char* dg_last_error(void) { return g_last_error.c_str(); }

}  // extern "C"

// ---------------------------------------------------------------- autotuner

extern "C" int dg_autotune(dg_ctx* c, const double* q, double dt, int* best_E, double* best_ms, void* stream) {
  using namespace dgnn;
  if (!c || !q) return fail(DG_ERR_INVALID_ARG, "dg_autotune: NULL argument");
  if (!std::isfinite(dt)) return fail(DG_ERR_INVALID_ARG, "dg_autotune: bad dt");
  cudaStream_t st = (cudaStream_t)stream;
  const size_t bytes = 5 * c->N * sizeof(double);
  double* work = nullptr;
  DG_CUDA(cudaMalloc(&work, bytes));
  cudaEvent_t a = nullptr, b = nullptr;
  cudaError_t e = cudaEventCreate(&a);
  if (e == cudaSuccess) e = cudaEventCreate(&b);
  const int E0 = c->geom.E, cube0 = c->geom.cube;
  int bestE = E0, bestCube = cube0;
  double best = 1e300;
  // candidates: rows of E = 1, 2, 4, ... elements, then (where allowed) cubes
  std::vector<std::pair<int, int>> cand;  // (E, cube)
  for (int E = 1; E <= max_elems_per_block(c->P); E *= 2) cand.push_back({E, 0});
  if (cube_ok(c->P) && c->K % 2 == 0 && !c->borrowed && !c->geom.split && !c->part) cand.push_back({kCubeElems, 1});
  for (const auto& ce : cand) {
    if (e != cudaSuccess) break;
    c->geom.E = ce.first;
    c->geom.cube = ce.second;
    e = cudaMemcpyAsync(work, q, bytes, cudaMemcpyDeviceToDevice, st);
    if (e != cudaSuccess) break;
    if (rk3_steps(c, work, dt, 1, nullptr, st, false) != DG_OK) {  // shared memory too large for this E: skip
      cudaGetLastError();
      continue;
    }
    cudaEventRecord(a, st);
    const int reps = 3;
    if (rk3_steps(c, work, dt, reps, nullptr, st, false) != DG_OK) {
      cudaGetLastError();
      continue;
    }
    cudaEventRecord(b, st);
    e = cudaEventSynchronize(b);
    float ms = 0.f;
    if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, a, b);
    if (e == cudaSuccess && ms / reps < best) {
      best = ms / reps;
      bestE = c->geom.E;
      bestCube = c->geom.cube;
    }
  }
  c->geom.E = (best < 1e300) ? bestE : E0;
  c->geom.cube = (best < 1e300) ? bestCube : cube0;
  if (a) cudaEventDestroy(a);
  if (b) cudaEventDestroy(b);
  cudaFree(work);
  if (e != cudaSuccess) return cuda_fail(e, "dg_autotune");
  if (best_E) *best_E = c->geom.E;
  if (best_ms) *best_ms = best;
  return DG_OK;
}

extern "C" int dg_set_forcing_mode(dg_ctx* c, int mode) {
  using namespace dgnn;
  if (!c) return fail(DG_ERR_INVALID_ARG, "dg_set_forcing_mode: NULL context");
  if (mode != DG_FORCING_STAGE && mode != DG_FORCING_POST)
    return fail(DG_ERR_INVALID_ARG, "dg_set_forcing_mode: unknown mode");
  c->forcing_mode = mode;
  return DG_OK;
}

namespace dgnn {
// Two bounded waits on mbarriers that never complete (no arrivals): out[0] from the
// operator's bulk-copy wait, out[1] from the tensor-core wait; 1 = reported completion.
__global__ void k_wait_selfcheck(int* out) {
  __shared__ unsigned long long bars[2];
  if (threadIdx.x == 0) {
    bulk_bar_init(&bars[0]);
    bulk_bar_init(&bars[1]);
    bulk_bar_fence_init();
  }
  __syncthreads();
  if (threadIdx.x == 0) out[0] = bulk_wait(&bars[0], 0u) ? 1 : 0;
  if (threadIdx.x == 32) out[1] = tc::mbar_wait(reinterpret_cast<uint64_t*>(&bars[1]), 0u) ? 1 : 0;
}
}  // namespace dgnn

extern "C" int dg_check_bounded_waits(double* seconds, void* stream) {
  using namespace dgnn;
  cudaStream_t st = (cudaStream_t)stream;
  int* d = nullptr;
  DG_CUDA(cudaMalloc(&d, 2 * sizeof(int)));
  int h[2] = {-1, -1};
  cudaEvent_t a = nullptr, b = nullptr;
  cudaError_t e = cudaEventCreate(&a);
  if (e == cudaSuccess) e = cudaEventCreate(&b);
  if (e == cudaSuccess) e = cudaMemsetAsync(d, 0xFF, 2 * sizeof(int), st);
  if (e == cudaSuccess) e = cudaEventRecord(a, st);
  if (e == cudaSuccess) {
    k_wait_selfcheck<<<1, 64, 0, st>>>(d);
    e = cudaGetLastError();
  }
  if (e == cudaSuccess) e = cudaEventRecord(b, st);
  if (e == cudaSuccess) e = cudaMemcpyAsync(h, d, sizeof(h), cudaMemcpyDeviceToHost, st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  float ms = 0.f;
  if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, a, b);
  if (a) cudaEventDestroy(a);
  if (b) cudaEventDestroy(b);
  cudaFree(d);
  if (e != cudaSuccess) return cuda_fail(e, "dg_check_bounded_waits");
  if (h[0] != 0 || h[1] != 0)
    return fail(DG_ERR_CUDA, "dg_check_bounded_waits: a wait reported completion without arrivals");
  if (seconds) *seconds = ms / 1e3;
  return DG_OK;
}

extern "C" int dg_blocking(const dg_ctx* c, int* elems_per_block, int* block_shape) {
  using namespace dgnn;
  if (!c) return fail(DG_ERR_INVALID_ARG, "dg_blocking: NULL context");
  if (elems_per_block) *elems_per_block = c->geom.E;
  if (block_shape) *block_shape = c->geom.cube;
  return DG_OK;
}

// Batches of independent solvers advanced together (C ABI in include/dgnn.h).
//
// Each member is an ordinary context (its own mesh, flow, closure and workspace).  A
// batched RK3 step groups the members by order P: every group runs one phase-A and one
// phase-B launch per stage covering all of its members' element blocks (k_gradient_batch,
// k_flux_batch), so twelve small meshes cost six launches per step per order instead of
// six per mesh.  Groups of different orders do not depend on each other and run as
// parallel branches.  The whole step is recorded once into a CUDA graph on private
// streams and replayed on the caller's stream; it is recorded again when the member
// states, step sizes or elements-per-block change.
#include <cmath>
#include <map>
#include <vector>

#include "dg_aux.h"

namespace dgnn {
namespace {

// Williamson 2N RK3 (the same coefficients as the single-mesh path).
constexpr double kA[3] = {0.0, -5.0 / 9.0, -153.0 / 128.0};
constexpr double kB[3] = {1.0 / 3.0, 15.0 / 16.0, 8.0 / 15.0};

struct Group {
  int P = 0;
  std::vector<int> members;
};

struct GraphKey {
  std::vector<double*> q;
  std::vector<double> dt;
  std::vector<int> E;
  int persistent = 0;
  bool operator==(const GraphKey& o) const {
    return q == o.q && dt == o.dt && E == o.E && persistent == o.persistent;
  }
};

}  // namespace
}  // namespace dgnn

struct dg_batch {
  std::vector<dg_ctx*> inst;
  std::vector<dgnn::Group> groups;
  int precision = DG_PREC_FP64;
  std::vector<cudaStream_t> cap;     // one capture stream per group
  std::vector<cudaEvent_t> join;     // one per group
  cudaEvent_t fork = nullptr;
  cudaGraphExec_t exec = nullptr;
  dgnn::GraphKey key;
  unsigned* bar = nullptr;           // grid barrier of the persistent stage kernel (2 counters)
};

namespace dgnn {
namespace {

cudaError_t stage_group(const dg_batch* b, const Group& g, double* const* q, const double* dt, int k,
                        cudaStream_t st) {
  dg_ctx* ctx[DG_BATCH_MAX];
  double* qs[DG_BATCH_MAX];
  double dts[DG_BATCH_MAX];
  const int n = (int)g.members.size();
  for (int j = 0; j < n; ++j) {
    ctx[j] = b->inst[g.members[j]];
    qs[j] = q[g.members[j]];
    dts[j] = dt[g.members[j]];
  }
  const double invB1 = 1.0 / kB[0];
  return b->precision == DG_PREC_FP32 ? batch_stage_f32(g.P, ctx, qs, dts, n, k, kA[k], kB[k], invB1, st)
                                      : batch_stage_f64(g.P, ctx, qs, dts, n, k, kA[k], kB[k], invB1, st);
}

cudaError_t prepare_groups(const dg_batch* b) {
  for (const Group& g : b->groups) {
    const int E = b->inst[g.members[0]]->geom.E;
    cudaError_t e = b->precision == DG_PREC_FP32 ? batch_prepare_f32(g.P, E) : batch_prepare_f64(g.P, E);
    if (e != cudaSuccess) return e;
  }
  return cudaSuccess;
}

// One RK3 step of every group, the groups one after another on one stream.
cudaError_t step_direct(const dg_batch* b, double* const* q, const double* dt, cudaStream_t st) {
  cudaError_t e0 = prepare_groups(b);
  if (e0 != cudaSuccess) return e0;
  for (int k = 0; k < 3; ++k)
    for (const Group& g : b->groups) {
      cudaError_t e = stage_group(b, g, q, dt, k, st);
      if (e != cudaSuccess) return e;
    }
  return cudaSuccess;
}

// One RK3 step of every member as three persistent launches (one per stage, every order
// together), after a reset of the grid barrier's counters.
cudaError_t step_persistent(const dg_batch* b, double* const* q, const double* dt, size_t smem, int grid,
                            cudaStream_t st) {
  cudaError_t e = cudaMemsetAsync(b->bar, 0, 2 * sizeof(unsigned), st);
  const int n = (int)b->inst.size();
  const double invB1 = 1.0 / kB[0];
  for (int k = 0; k < 3 && e == cudaSuccess; ++k)
    e = batch_persistent_stage(b->inst.data(), q, dt, n, k, kA[k], kB[k], invB1, b->bar, smem, grid, st);
  return e;
}

int prepare_persistent(const dg_batch* b, size_t* smem, int* grid) {
  if (b->precision != DG_PREC_FP32)
    return fail(DG_ERR_UNSUPPORTED, "dg_batch_rk3_step: the persistent stage kernel runs the FP32 operator");
  std::vector<int> orders;
  for (const dg_ctx* c : b->inst) {
    if (!batch_persistent_ok(c->P))
      return fail(DG_ERR_UNSUPPORTED, "dg_batch_rk3_step: the persistent stage kernel takes orders 1 to 6");
    orders.push_back(c->P);
  }
  DG_CUDA(batch_persistent_prepare(orders.data(), (int)orders.size(), smem, grid));
  return DG_OK;
}

// Records one step with the groups as parallel branches: fork from cap[0], each group on
// its own stream, join back into cap[0].  persistent: three cooperative launches on cap[0].
int record_step(dg_batch* b, double* const* q, const double* dt, bool persistent) {
  size_t psmem = 0;
  int pgrid = 0;
  if (persistent) {
    int rc = prepare_persistent(b, &psmem, &pgrid);
    if (rc) return rc;
  }
  // kernel attributes (dynamic shared memory) are set outside the recording
  cudaError_t ea = prepare_groups(b);
  if (ea != cudaSuccess) return cuda_fail(ea, "dg_batch_rk3_step: kernel attributes");
  if (b->exec) {
    cudaGraphExecDestroy(b->exec);
    b->exec = nullptr;
  }
  cudaStream_t s0 = b->cap[0];
  DG_CUDA(cudaStreamBeginCapture(s0, cudaStreamCaptureModeThreadLocal));
  cudaError_t e = cudaEventRecord(b->fork, s0);
  if (persistent && e == cudaSuccess) e = step_persistent(b, q, dt, psmem, pgrid, s0);
  for (size_t gi = 0; gi < b->groups.size() && e == cudaSuccess && !persistent; ++gi) {
    cudaStream_t s = b->cap[gi];
    if (gi > 0) e = cudaStreamWaitEvent(s, b->fork, 0);
    for (int k = 0; k < 3 && e == cudaSuccess; ++k) e = stage_group(b, b->groups[gi], q, dt, k, s);
    if (gi > 0 && e == cudaSuccess) e = cudaEventRecord(b->join[gi], s);
    if (gi > 0 && e == cudaSuccess) e = cudaStreamWaitEvent(s0, b->join[gi], 0);
  }
  cudaGraph_t graph = nullptr;
  cudaError_t e2 = cudaStreamEndCapture(s0, &graph);
  if (e == cudaSuccess) e = e2;
  if (e == cudaSuccess) e = cudaGraphInstantiate(&b->exec, graph, 0);
  if (graph) cudaGraphDestroy(graph);
  if (e != cudaSuccess) {
    b->exec = nullptr;
    cudaGetLastError();
    return cuda_fail(e, "dg_batch_rk3_step: recording the step graph");
  }
  return DG_OK;
}

GraphKey key_of(const dg_batch* b, double* const* q, const double* dt, bool persistent) {
  GraphKey k;
  k.persistent = persistent;
  const size_t n = b->inst.size();
  k.q.assign(q, q + n);
  k.dt.assign(dt, dt + n);
  for (const dg_ctx* c : b->inst) k.E.push_back(c->geom.E);
  return k;
}

}  // namespace
}  // namespace dgnn

using namespace dgnn;

extern "C" {

int dg_batch_destroy(dg_batch* b) {
  if (!b) return fail(DG_ERR_INVALID_ARG, "dg_batch_destroy: NULL");
  if (b->exec) cudaGraphExecDestroy(b->exec);
  for (cudaStream_t s : b->cap)
    if (s) cudaStreamDestroy(s);
  for (cudaEvent_t e : b->join)
    if (e) cudaEventDestroy(e);
  if (b->fork) cudaEventDestroy(b->fork);
  if (b->bar) cudaFree(b->bar);
  for (dg_ctx* c : b->inst) {
    c->borrowed = false;
    dg_destroy(c);
  }
  delete b;
  return DG_OK;
}

int dg_create_batch(const dg_instance_desc* desc, int n, const dg_opts* opts, dg_batch** out) {
  if (!out) return fail(DG_ERR_INVALID_ARG, "dg_create_batch: out is NULL");
  *out = nullptr;
  if (!desc) return fail(DG_ERR_INVALID_ARG, "dg_create_batch: desc is NULL");
  if (n < 1 || n > DG_BATCH_MAX) return fail(DG_ERR_INVALID_ARG, "dg_create_batch: n must be in [1, 16]");
  for (int i = 0; i < n; ++i)
    if (desc[i].P < 1 || desc[i].P > kMaxP) return fail(DG_ERR_INVALID_ARG, "dg_create_batch: P must be in [1, 8]");
  dg_opts o;
  dg_opts_default(&o);
  if (opts) o = *opts;
  if (o.block_shape != 0) return fail(DG_ERR_INVALID_ARG, "dg_create_batch: batch members use rows of elements (block_shape 0)");
  if (o.volume_flux != 0) return fail(DG_ERR_INVALID_ARG, "dg_create_batch: batch members use the standard volume term");
  dg_batch* b = new dg_batch();
  b->precision = o.precision;
  for (int i = 0; i < n; ++i) {
    dg_ctx* c = nullptr;
    const dg_instance_desc& d = desc[i];
    int rc = dg_create(d.K, d.P, d.Re, d.Mach, d.Pr, d.closure, &o, &c);
    if (rc) {
      std::string msg = std::string("dg_create_batch: member ") + std::to_string(i) + ": " + dg_last_error();
      dg_batch_destroy(b);
      return fail(rc, msg);
    }
    c->borrowed = true;
    b->inst.push_back(c);
  }
  std::map<int, int> slot;
  for (int i = 0; i < n; ++i) {
    const int P = desc[i].P;
    if (!slot.count(P)) {
      slot[P] = (int)b->groups.size();
      b->groups.push_back(Group{P, {}});
    }
    b->groups[slot[P]].members.push_back(i);
  }
  // one elements-per-block per order (the first member's choice)
  for (const Group& g : b->groups)
    for (int m : g.members) b->inst[m]->geom.E = b->inst[g.members[0]]->geom.E;
  cudaError_t e = cudaEventCreateWithFlags(&b->fork, cudaEventDisableTiming);
  b->cap.assign(b->groups.size(), nullptr);
  b->join.assign(b->groups.size(), nullptr);
  for (size_t gi = 0; gi < b->groups.size() && e == cudaSuccess; ++gi) {
    e = cudaStreamCreateWithFlags(&b->cap[gi], cudaStreamNonBlocking);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&b->join[gi], cudaEventDisableTiming);
  }
  if (e == cudaSuccess) e = cudaMalloc(&b->bar, 2 * sizeof(unsigned));
  if (e == cudaSuccess) e = cudaMemset(b->bar, 0, 2 * sizeof(unsigned));
  if (e != cudaSuccess) {
    dg_batch_destroy(b);
    return cuda_fail(e, "dg_create_batch: streams, events and barrier");
  }
  *out = b;
  return DG_OK;
}

int dg_batch_size(const dg_batch* b, int* n) {
  if (!b || !n) return fail(DG_ERR_INVALID_ARG, "dg_batch_size: NULL argument");
  *n = (int)b->inst.size();
  return DG_OK;
}

int dg_batch_member(dg_batch* b, int i, dg_ctx** out) {
  if (!b || !out) return fail(DG_ERR_INVALID_ARG, "dg_batch_member: NULL argument");
  if (i < 0 || i >= (int)b->inst.size()) return fail(DG_ERR_INVALID_ARG, "dg_batch_member: index out of range");
  *out = b->inst[i];
  return DG_OK;
}

int dg_batch_rk3_step(dg_batch* b, double* const* q, const double* dt, int nsteps, int flags, void* stream) {
  if (!b || !q || !dt) return fail(DG_ERR_INVALID_ARG, "dg_batch_rk3_step: NULL argument");
  if (nsteps < 0) return fail(DG_ERR_INVALID_ARG, "dg_batch_rk3_step: nsteps < 0");
  if (flags & ~(DG_BATCH_NO_GRAPH | DG_BATCH_PERSISTENT))
    return fail(DG_ERR_INVALID_ARG, "dg_batch_rk3_step: unknown flags");
  const bool persistent = (flags & DG_BATCH_PERSISTENT) != 0;
  for (size_t i = 0; i < b->inst.size(); ++i) {
    if (!q[i]) return fail(DG_ERR_INVALID_ARG, "dg_batch_rk3_step: NULL member state");
    if (!std::isfinite(dt[i])) return fail(DG_ERR_INVALID_ARG, "dg_batch_rk3_step: non-finite dt");
    for (size_t j = 0; j < i; ++j)
      if (q[j] == q[i]) return fail(DG_ERR_INVALID_ARG, "dg_batch_rk3_step: two members share one state");
  }
  cudaStream_t st = (cudaStream_t)stream;
  if (flags & DG_BATCH_NO_GRAPH) {
    if (persistent) {
      size_t smem = 0;
      int grid = 0;
      int rc = prepare_persistent(b, &smem, &grid);
      if (rc) return rc;
      for (int s = 0; s < nsteps; ++s) DG_CUDA(step_persistent(b, q, dt, smem, grid, st));
      return DG_OK;
    }
    for (int s = 0; s < nsteps; ++s) DG_CUDA(step_direct(b, q, dt, st));
    return DG_OK;
  }
  if (nsteps == 0) return DG_OK;
  GraphKey k = key_of(b, q, dt, persistent);
  if (!b->exec || !(k == b->key)) {
    int rc = record_step(b, q, dt, persistent);
    if (rc) return rc;
    b->key = k;
  }
  for (int s = 0; s < nsteps; ++s) DG_CUDA(cudaGraphLaunch(b->exec, st));
  return DG_OK;
}

int dg_batch_autotune(dg_batch* b, double* const* q, const double* dt, void* stream) {
  if (!b || !q || !dt) return fail(DG_ERR_INVALID_ARG, "dg_batch_autotune: NULL argument");
  for (const Group& g : b->groups) {
    int big = g.members[0];
    for (int m : g.members)
      if (b->inst[m]->N > b->inst[big]->N) big = m;
    int E = 0;
    int rc = dg_autotune(b->inst[big], q[big], dt[big], &E, nullptr, stream);
    if (rc) return rc;
    for (int m : g.members) b->inst[m]->geom.E = E;
  }
  return DG_OK;
}

}  // extern "C"

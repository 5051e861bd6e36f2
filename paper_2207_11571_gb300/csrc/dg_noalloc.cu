// dg_rhs_noalloc: the DGSEM operator for callers that must not allocate device memory.
//
// Who needs it: code that calls the operator from a place where cudaMalloc is not
// allowed or not wanted -- an in-situ analysis hook inside another solver's time loop
// whose device memory was budgeted and locked at start-up, or a host thread that must
// not take the allocator's locks or synchronise the device (cudaMalloc and cudaFree may
// do both).  dg_create allocates its workspace (stage state and viscous stresses, ~112
// bytes per node in FP64); this entry point instead uses one fixed scratch array that
// lives in the library's own device image.
//
// The scratch array holds the two intermediate fields of one operator evaluation: the
// stage state (5 values per node) and the viscous stresses and heat flux (9 values per
// node), at most kNoallocMaxNodes nodes.  Every GPU that loads the library keeps it
// (3.7 MB) until the process exits.  All calls on a device share it and it keeps the
// last call's contents; nothing in it needs to start at zero, because the first kernel
// of every call writes every entry it later reads.  Calls whose work overlaps on the GPU
// (different streams, or different host threads) race on the array: serialise them.
//
// In host code the array's name is only a host-side stand-in; its device address comes
// from cudaGetSymbolAddress, taken once per device (with that device current) on the
// first call made while it is current.  The same first call uploads the FP32 kernels'
// constant tables for that device (synchronous copies), whatever precision it asks for,
// so later calls of either precision enqueue kernels only.  Make that first call before
// any stream capture.  The cached address belongs to the device's context: after
// cudaDeviceReset the library must not be called again in the process.
#include <mutex>

#include "dg_aux.h"
#include "dg_kernels.cuh"

namespace dgnn {
namespace {

constexpr long long kNoallocMaxNodes = 32768;  // e.g. 8^3 elements at P = 3, 4^3 at P = 7
constexpr long long kNoallocDoubles = 14 * kNoallocMaxNodes;
constexpr int kNoallocMaxDevices = 64;

static __device__ __align__(256) double g_noalloc_scratch[kNoallocDoubles];

std::mutex g_noalloc_mu;
double* g_noalloc_addr[kNoallocMaxDevices] = {};

// Device address of the scratch array on the current device (looked up once per device,
// together with the upload of the FP32 constant tables).
int noalloc_scratch(double** out) {
  int dev = 0;
  DG_CUDA(cudaGetDevice(&dev));
  if (dev < 0 || dev >= kNoallocMaxDevices) return fail(DG_ERR_UNSUPPORTED, "dg_rhs_noalloc: device index too large");
  std::lock_guard<std::mutex> lock(g_noalloc_mu);
  if (!g_noalloc_addr[dev]) {
    void* p = nullptr;
    cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
    if (e != cudaSuccess) return cuda_fail(e, "dg_rhs_noalloc: cudaGetSymbolAddress of the scratch array");
    // FP32 derivative tables in constant memory: uploaded here, at set-up, for both
    // precisions, so that no later call issues a synchronous copy
    e = prepare_f32_constants();
    if (e != cudaSuccess) return cuda_fail(e, "dg_rhs_noalloc: constant tables");
    g_noalloc_addr[dev] = static_cast<double*>(p);
  }
  *out = g_noalloc_addr[dev];
  return DG_OK;
}

}  // namespace
}  // namespace dgnn

using namespace dgnn;

extern "C" int dg_rhs_noalloc(int K, int P, double Re, double Mach, double Pr, int closure, int precision,
                              const double* q, double* dqdt, void* stream) {
  if (!q || !dqdt) return fail(DG_ERR_INVALID_ARG, "dg_rhs_noalloc: NULL argument");
  if (q == dqdt) return fail(DG_ERR_INVALID_ARG, "dg_rhs_noalloc: q and dqdt must not alias");
  if (K < 1 || K > 256) return fail(DG_ERR_INVALID_ARG, "dg_rhs_noalloc: K must be in [1, 256]");
  if (P < 1 || P > kMaxP) return fail(DG_ERR_INVALID_ARG, "dg_rhs_noalloc: P must be in [1, 8]");
  if (!(Re > 0) || !(Mach > 0) || !(Pr > 0)) return fail(DG_ERR_INVALID_ARG, "dg_rhs_noalloc: Re, Mach, Pr must be > 0");
  if (closure != 0 && closure != 1) return fail(DG_ERR_INVALID_ARG, "dg_rhs_noalloc: closure must be 0 or 1");
  if (precision != DG_PREC_FP64 && precision != DG_PREC_FP32)
    return fail(DG_ERR_INVALID_ARG, "dg_rhs_noalloc: unknown precision");
  const long long nodes = (long long)K * K * K * (P + 1) * (P + 1) * (P + 1);
  if (nodes > kNoallocMaxNodes)
    return fail(DG_ERR_INVALID_ARG, "dg_rhs_noalloc: " + std::to_string(nodes) +
                                        " nodes exceed the no-allocation limit of 32768 nodes (K^3 (P+1)^3); "
                                        "use dg_create / dg_rhs");

  double* scratch = nullptr;
  int rc = noalloc_scratch(&scratch);
  if (rc) return rc;

  // A solver description on the host stack, with its workspace in the scratch array.
  dg_opts o;
  dg_opts_default(&o);
  o.precision = precision;
  dg_ctx c;
  rc = setup_ctx(&c, K, P, Re, Mach, Pr, closure, o);
  if (rc) return rc;
  // stage state then viscous quantities, in the operator precision
  if (precision == DG_PREC_FP32) {
    float* s = reinterpret_cast<float*>(scratch);
    c.qf = s;
    c.vis = s + 5 * nodes;
  } else {
    c.qf = scratch;
    c.vis = scratch + 5 * nodes;
  }
  cudaStream_t st = (cudaStream_t)stream;
  DG_CUDA(launch_gradient(&c, q, 0, st));
  DG_CUDA(launch_flux(&c, const_cast<double*>(q), dqdt, Forcing{}, 0, 0.0, 0.0, 0.0, st));
  // the context lives on the stack and owns nothing: keep its destructor-free fields empty
  c.qf = c.vis = nullptr;
  return DG_OK;
}

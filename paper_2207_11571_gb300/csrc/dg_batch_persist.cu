// Persistent batched RK stage (FP32 operator): one cooperative launch per RK stage for
// every member of a batch, whatever its order (P = 1 .. 6).
//
// Each block of kPersistThreads threads walks the phase-A work items of all members
// (blocks of E_P consecutive elements of a member, E_P = the elements of order P that
// fill the block), meets every other block at a grid barrier, then walks the phase-B items
// of all members.  The per-item arithmetic is the single-mesh kernels' (gradient_block,
// flux_block), so a member computes what it computes alone; only the blocking differs.
// The grid holds as many blocks as are resident at once (a cooperative launch), and the
// barrier's wait is bounded (about a second): on expiry the block sets the batch's error
// flag and returns.  The launches of a step form one CUDA graph, after a reset of the
// barrier's counter.
#include "dg_aux.h"
#include "dg_launch.cuh"

namespace dgnn {

constexpr int kPersistThreads = 384;
__host__ __device__ constexpr int persist_elems(int P) { return kPersistThreads / ((P + 1) * (P + 1) * (P + 1)); }

struct PersistTable {
  BatchTable<float> tb;   // block_start: first work item of each member (the same items in both phases)
  int P[kMaxBatch];
  unsigned* bar;          // [0] arrivals at the barrier, [1] its generation
};

// Bounded grid barrier: every block's thread 0 counts its arrival; the last to arrive
// resets the count and advances the generation, the others wait for the new generation.
// Writes before the barrier are visible after it (fences around the count).  Returns
// false in every thread of a block whose wait expired.
__device__ __forceinline__ bool grid_barrier_bounded(unsigned* bar) {
  __syncthreads();
  int expired = 0;
  if (threadIdx.x == 0) {
    volatile unsigned* gen = bar + 1;
    const unsigned g = *gen;
    __threadfence();
    if (atomicAdd(bar, 1u) == gridDim.x - 1) {
      atomicExch(bar, 0u);
      __threadfence();
      atomicAdd(bar + 1, 1u);
    } else {
      const long long t0 = clock64();
      while (*gen == g) {
        if (clock64() - t0 > 2000000000LL) {
          expired = 1;
          break;
        }
      }
    }
    __threadfence();
  }
  return __syncthreads_or(expired) == 0;
}

template <int SRC, int MODE>
__global__ void __launch_bounds__(kPersistThreads, 2) k_batch_persistent(const __grid_constant__ PersistTable pt) {
  const BatchTable<float>& tb = pt.tb;
  const int items = tb.block_start[tb.n];
  for (int item = blockIdx.x; item < items; item += gridDim.x) {
    const int i = batch_instance(tb.block_start, tb.n, item);
    const int blk = item - tb.block_start[i];
    float* qn32_out = SRC == 0 ? tb.qn32[i] : nullptr;
    switch (pt.P[i]) {
#define DG_PA(PP)                                                                                                  \
  case PP:                                                                                                         \
    gradient_block<PP, float, SRC>(blk, tb.q[i], tb.qn32[i], tb.dlt[i], tb.qf[i], qn32_out, tb.vis[i], tb.C[i]); \
    break;
      DG_PA(1) DG_PA(2) DG_PA(3) DG_PA(4) DG_PA(5) DG_PA(6)
#undef DG_PA
    }
    __syncthreads();   // the next item reuses the shared memory
  }
  if (!grid_barrier_bounded(pt.bar)) {
    if (threadIdx.x == 0 && tb.err[0]) atomicExch(tb.err[0], 1);
    return;
  }
  for (int item = blockIdx.x; item < items; item += gridDim.x) {
    const int i = batch_instance(tb.block_start, tb.n, item);
    const int blk = item - tb.block_start[i];
    switch (pt.P[i]) {
#define DG_PB(PP)                                                                                                 \
  case PP:                                                                                                        \
    flux_block<PP, float, MODE>(blk, tb.q[i], tb.qf[i], tb.vis[i], nullptr, tb.g[i], tb.dlt[i], Forcing{}, tb.C[i], \
                                tb.rk[i]);                                                                        \
    break;
      DG_PB(1) DG_PB(2) DG_PB(3) DG_PB(4) DG_PB(5) DG_PB(6)
#undef DG_PB
    }
    __syncthreads();
  }
}

namespace {

// Shared memory of one work item of order P in the persistent kernel (the larger phase).
size_t persist_smem_p(int P) {
  switch (P) {
#define DG_SM(PP) \
  case PP: return std::max(gradient_smem<PP, float>(persist_elems(PP)), flux_smem<PP, float>(persist_elems(PP)));
    DG_SM(1) DG_SM(2) DG_SM(3) DG_SM(4) DG_SM(5) DG_SM(6)
#undef DG_SM
  }
  return 0;
}

using PersistKernel = void (*)(const PersistTable);

PersistKernel persist_kernel(int k) {
  return k == 0 ? k_batch_persistent<0, 2> : k == 1 ? k_batch_persistent<1, 3> : k_batch_persistent<1, 4>;
}

}  // namespace

bool batch_persistent_ok(int P) { return P >= 1 && P <= 6; }

cudaError_t batch_persistent_prepare(const int* orders, int n, size_t* smem_out, int* grid_out) {
  size_t smem = 0;
  for (int i = 0; i < n; ++i) smem = std::max(smem, persist_smem_p(orders[i]));
  int grid = 0;
  for (int k = 0; k < 3; ++k) {
    PersistKernel kern = persist_kernel(k);
    cudaError_t e = set_smem(kern, smem);
    if (e != cudaSuccess) return e;
    int per_sm = 0;
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, kPersistThreads, smem);
    if (e != cudaSuccess) return e;
    int dev = 0, sms = 0;
    if ((e = cudaGetDevice(&dev)) != cudaSuccess) return e;
    if ((e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev)) != cudaSuccess) return e;
    const int g = per_sm * sms;
    grid = (k == 0) ? g : std::min(grid, g);
  }
  if (grid < 1) return cudaErrorInvalidConfiguration;
  *smem_out = smem;
  *grid_out = grid;
  return cudaSuccess;
}

cudaError_t batch_persistent_stage(dg_ctx* const* ctx, double* const* q, const double* dt, int n, int k, double A,
                                   double B, double invB1, unsigned* bar, size_t smem, int grid, cudaStream_t st) {
  if (n < 1 || n > kMaxBatch) return cudaErrorInvalidValue;
  PersistTable pt;
  fill_batch<float>(&pt.tb, ctx, q, dt, n, A, B, invB1);
  // work items of E_P elements per member, whatever blocking the member uses alone
  int items = 0;
  for (int i = 0; i < n; ++i) {
    const int P = ctx[i]->P;
    if (!batch_persistent_ok(P)) return cudaErrorInvalidValue;
    pt.P[i] = P;
    pt.tb.C[i].E = persist_elems(P);
    pt.tb.block_start[i] = items;
    items += (owned_elems(ctx[i]) + persist_elems(P) - 1) / persist_elems(P);
  }
  pt.tb.block_start[n] = items;
  pt.bar = bar;
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(std::min(grid, items));
  cfg.blockDim = dim3(kPersistThreads);
  cfg.dynamicSmemBytes = smem;
  cfg.stream = st;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeCooperative;
  attr[0].val.cooperative = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  return cudaLaunchKernelEx(&cfg, persist_kernel(k), pt);
}

}  // namespace dgnn

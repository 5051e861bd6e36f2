// The corrective forcing s(q) of an RK stage (Sec. 2.2, Fig. 2; Eq. 4): every layer of
// the network on the tcgen05 tensor cores in one launch, from the bf16 element features to
// the unscaled forcing in the layout the flux kernel adds to the operator.
//
// A cluster of C CTAs (C = 1, 2 or 4) carries one tile of 128 elements (MMA M = 128)
// through the network.  Each CTA loads the tile's features by TMA.  CTA j of the cluster
// owns output columns [j N/C, (j+1) N/C) of every layer: it streams only that slice of
// each weight matrix, writes its bf16 slice of each hidden layer's output into its own
// activation panels, and copies that slice (64-column panels, one bulk copy per panel and
// peer on the asynchronous copy engine) into the same panels of every other CTA of the
// cluster (distributed shared memory), so that each CTA holds the whole input of the next
// layer.  With C = 4 a 4096-element mesh occupies 128 SMs, and every weight byte read from
// L2 feeds 128 rows.
//
// Warps: 0 TMA producer (the feature tile, then weight tiles through a 5-stage ring),
// 1 TMEM allocation and the MMA issuer, 2..9 epilogue: two warps per TMEM lane quarter
// (one TMEM lane = one element per thread), taking alternate 16-column groups, one 64-column
// panel of the CTA's slice after the other; 10 the exchange (lane k talks to CTA k): the
// arrivals at the peers, the slice copies and the receipts, off the epilogue's path.  The layers' biases and the output scaling of
// this CTA's slices sit in shared memory.  Ordering uses mbarriers only:
//   panel_ready[i] (one arrival per epilogue thread): panel i of this CTA's slice of the
//       next input is written (a CTA's own panels are free once its own MMAs of the layer
//       have completed, since only they read them);
//   act_from[k] (k != own rank): one local arrival carrying the bytes of CTA k's slice,
//       which CTA k's bulk copies complete;
//   peers_done (C arrivals): every CTA's MMAs of the current layer have completed, so no
//       tensor core still reads the panels that the slice copies overwrite, and every
//       earlier slice copy has landed (those MMAs waited for it);
//   copies_landed (C - 1 arrivals, one from each receiver's exchange warp): this CTA's
//       slice has landed everywhere, so the copy engine no longer reads the panels that
//       the next slice overwrites.
// A hidden layer's K loop starts on the CTA's own panels as each is written and then takes
// the peers' slices in rank order after its own (j + 1, j + 2, ...), each on its own
// barrier, so the tensor core works while the other slices are still in flight; the
// weight tiles stream in the same order.  Where a slice is at most 256 columns, layers
// alternate between two TMEM accumulators, so the next layer's MMAs may start while the
// epilogue still reads the last panels of this one.
// Every wait is bounded (about a second): on expiry a thread sets the error flag and the
// CTA skips the rest of its work; all threads meet at a final cluster barrier, so that no
// CTA leaves while a peer may still write into its shared memory.
#include <cudaTypedefs.h>

#include <cstring>

#include "dg_common.h"
#include "nn_forcing.h"
#include "nn_gemm.h"
#include "nn_mlp.h"
#include "tc_common.cuh"

namespace dgnn {

using namespace tc;

namespace {

constexpr int kRows = 128;
constexpr int kChunk = 128;                       // output columns per MMA at most
constexpr int kPanel = 64;                        // input columns per panel / weight tile
constexpr int kPanelBytes = kRows * kPanel * 2;   // 16 KB
constexpr int kTileBytes = kChunk * kPanel * 2;   // 16 KB (largest weight tile)
constexpr int kMaxPanels = kMlpMaxWidth / kPanel; // 8
constexpr int kRing = 5;
constexpr int kMaxCluster = 4;
constexpr int kEpiWarps = 8;                      // two per TMEM lane quarter
constexpr int kXchgWarp = 2 + kEpiWarps;          // the warp that sends the slices
constexpr int kThreads = 64 + 32 * kEpiWarps + 32;
constexpr int kTmemCols = 512;
constexpr int kActBytes = kMaxPanels * kPanelBytes;
constexpr int kRingOffset = kActBytes;
constexpr int kConstFloats = kMlpMaxLayers * kMlpMaxWidth / 2 + 2 * kMlpMaxWidth;   // bias slices, scale, shift
constexpr int kConstOffset = kRingOffset + kRing * kTileBytes;
constexpr int kBarOffset = kConstOffset + kConstFloats * 4;
constexpr int kSmemBytes = kBarOffset + 256 + 1024;
static_assert(kSmemBytes <= 227 * 1024, "forcing kernel exceeds shared memory");

struct ForcingArgs {
  CUtensorMap act0;               // features [rows][pad(d0)] bf16, box 64 x 128
  CUtensorMap w[kMlpMaxLayers];   // Wb[l] [d(l+1)][pad(d(l))] bf16, box 64 x min(128, slice)
  const float* bias[kMlpMaxLayers];
  int dims[kMlpMaxLayers + 1];
  int L;
  int rows;                       // elements
  int csize;                      // CTAs per cluster = column slices
  // output s[e][f] = (y + b) scale + shift
  const float* scale;
  const float* shift;
  float* out;
  int ldo;
};

__device__ __forceinline__ int panels_of(int d) { return (d + kPanel - 1) / kPanel; }
__device__ __forceinline__ uint32_t panel_offset(int r, int j) { return r * 128 + ((j ^ (r & 7)) << 4); }

__device__ __forceinline__ uint32_t cluster_rank() {
  uint32_t r;
  asm volatile("mov.u32 %0, %%cluster_ctarank;" : "=r"(r));
  return r;
}
// Address of the same shared-memory location in CTA `cta` of the cluster.
__device__ __forceinline__ uint32_t mapa(uint32_t saddr, uint32_t cta) {
  uint32_t r;
  asm volatile("mapa.shared::cluster.u32 %0, %1, %2;" : "=r"(r) : "r"(saddr), "r"(cta));
  return r;
}
// Arrival on the mbarrier at the same offset in CTA `cta`, releasing this thread's prior
// writes at cluster scope.
__device__ __forceinline__ void arrive_remote(uint64_t* bar, uint32_t cta) {
  asm volatile("mbarrier.arrive.release.cluster.shared::cluster.b64 _, [%0];" ::"r"(mapa(smem_u32(bar), cta))
               : "memory");
}
__device__ __forceinline__ bool try_wait_cluster(uint64_t* bar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n .reg .pred p;\n"
      " mbarrier.try_wait.parity.acquire.cluster.shared::cta.b64 p, [%1], %2;\n"
      " selp.u32 %0, 1, 0, p;\n}\n"
      : "=r"(ok)
      : "r"(smem_u32(bar)), "r"(parity)
      : "memory");
  return ok != 0;
}
// Bounded wait (acquire at cluster scope); false when the limit expires.
__device__ __forceinline__ bool wait_cluster(uint64_t* bar, uint32_t parity) {
  if (try_wait_cluster(bar, parity)) return true;
  const long long t0 = clock64();
  while (!try_wait_cluster(bar, parity))
    if (clock64() - t0 > kWaitCycles) return false;
  return true;
}
__device__ __forceinline__ void cluster_sync_all() {
  asm volatile("barrier.cluster.arrive.release.aligned;\n barrier.cluster.wait.acquire.aligned;" ::: "memory");
}

// 16 consecutive bf16 values of row r at global column gc (a multiple of 16) into this
// CTA's own activation panels.
__device__ __forceinline__ void put16_local(uint8_t* act, int r, int gc, const float v[16]) {
  const uint4 lo = make_uint4(pack_bf16(v[0], v[1]), pack_bf16(v[2], v[3]), pack_bf16(v[4], v[5]),
                              pack_bf16(v[6], v[7]));
  const uint4 hi = make_uint4(pack_bf16(v[8], v[9]), pack_bf16(v[10], v[11]), pack_bf16(v[12], v[13]),
                              pack_bf16(v[14], v[15]));
  uint8_t* pan = act + (gc / kPanel) * kPanelBytes;
  const int j = (gc % kPanel) / 8;
  *reinterpret_cast<uint4*>(pan + panel_offset(r, j)) = lo;
  *reinterpret_cast<uint4*>(pan + panel_offset(r, j + 1)) = hi;
}

// Bulk copy (the asynchronous copy engine) of `bytes` of this CTA's shared memory at
// `src` to the same offset in CTA `cta`, completing its bytes on that CTA's mbarrier `bar`.
__device__ __forceinline__ void bulk_to_peer(const void* src, uint32_t bytes, uint64_t* bar, uint32_t cta) {
  const uint32_t s = smem_u32(src);
  asm volatile(
      "cp.async.bulk.shared::cluster.shared::cta.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
          mapa(s, cta)),
      "r"(s), "r"(bytes), "r"(mapa(smem_u32(bar), cta))
      : "memory");
}

// Two 16-column TMEM loads of this thread's lane, one wait.
__device__ __forceinline__ void tmem_ld16x2(uint32_t ta, uint32_t tb, float va[16], float vb[16]) {
  uint32_t r[32];
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%32];\n"
      "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%16,%17,%18,%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31}, [%33];\n"
      "tcgen05.wait::ld.sync.aligned;\n"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
        "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15]),
        "=r"(r[16]), "=r"(r[17]), "=r"(r[18]), "=r"(r[19]), "=r"(r[20]), "=r"(r[21]), "=r"(r[22]), "=r"(r[23]),
        "=r"(r[24]), "=r"(r[25]), "=r"(r[26]), "=r"(r[27]), "=r"(r[28]), "=r"(r[29]), "=r"(r[30]), "=r"(r[31])
      : "r"(ta), "r"(tb)
      : "memory");
#pragma unroll
  for (int i = 0; i < 16; ++i) {
    va[i] = __uint_as_float(r[i]);
    vb[i] = __uint_as_float(r[16 + i]);
  }
}

// First TMEM column of layer l's accumulator (slice width ns): where a slice fits in 256
// columns, layers alternate between columns 0 and 256; wider slices always start at 0.
__device__ __forceinline__ uint32_t acc_column(int ns, int l) { return (ns <= 256 && (l & 1)) ? 256u : 0u; }

// Named barrier of the epilogue warps only.
__device__ __forceinline__ void epilogue_sync() {
  asm volatile("bar.sync 1, %0;" ::"n"(32 * kEpiWarps) : "memory");
}

__global__ void __launch_bounds__(kThreads, 1) k_forcing_cluster(const __grid_constant__ ForcingArgs a,
                                                                  int* __restrict__ err_flag) {
  extern __shared__ uint8_t smem_raw[];
  uint8_t* base = reinterpret_cast<uint8_t*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
  uint8_t* act = base;
  uint8_t* ring = base + kRingOffset;
  uint64_t* full = reinterpret_cast<uint64_t*>(base + kBarOffset);
  uint64_t* empty = full + kRing;
  uint64_t* a0_full = empty + kRing;
  uint64_t* mma_done = a0_full + 1;
  uint64_t* panel_ready = mma_done + 1;      // [kMaxPanels], panels of this CTA's slice
  uint64_t* act_from = panel_ready + kMaxPanels;   // [kMaxCluster], indexed by the sending CTA
  uint64_t* peers_done = act_from + kMaxCluster;
  uint64_t* copies_landed = peers_done + 1;
  uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(copies_landed + 1);
  int* abort_flag = reinterpret_cast<int*>(tmem_slot + 1);

  const int warp = threadIdx.x / 32, lane = threadIdx.x % 32;
  const int C = a.csize;
  const int j = (int)cluster_rank();
  const int m0 = (blockIdx.x / C) * kRows;

  if (threadIdx.x == 0) {
    for (int s = 0; s < kRing; ++s) {
      mbar_init(&full[s], 1);
      mbar_init(&empty[s], 1);
    }
    mbar_init(a0_full, 1);
    mbar_init(mma_done, 1);
    for (int i = 0; i < kMaxPanels; ++i) mbar_init(&panel_ready[i], 32 * kEpiWarps);
    for (int k = 0; k < kMaxCluster; ++k) mbar_init(&act_from[k], 1);   // local arrival + CTA k's bytes
    mbar_init(peers_done, C);      // one arrival per CTA
    mbar_init(copies_landed, C > 1 ? C - 1 : 1);
    *abort_flag = 0;
    mbar_fence_init();
  }
  if (warp == 1) tmem_alloc(tmem_slot, kTmemCols);
  tc_fence_before();
  __syncthreads();
  cluster_sync_all();   // every CTA's barriers exist before any remote arrival
  tc_fence_after();
  const uint32_t tmem = *tmem_slot;
  // programmatic dependent launch: the set-up above overlaps the previous kernel; every
  // global read (stage state, weights: a training step may just have written them) waits
  asm volatile("griddepcontrol.wait;" ::: "memory");

  if (warp == 0) {
    if (lane == 0) {
      // the tile's features, then the weight tiles of this CTA's column slice, layer by
      // layer, chunk by chunk
      const int P0 = panels_of(a.dims[0]);
      mbar_expect_tx(a0_full, P0 * kPanelBytes);
      for (int p = 0; p < P0; ++p) tma_load_2d(act + p * kPanelBytes, &a.act0, a0_full, p * kPanel, m0);
      int issued = 0;
      bool ok = true;
      for (int l = 0; l < a.L && ok; ++l) {
        const int ns = a.dims[l + 1] / C, KP = panels_of(a.dims[l]);
        const int own0 = l == 0 ? 0 : j * (KP / C);   // the K loop's first panel
        for (int c0 = 0; c0 < ns && ok; c0 += kChunk) {
          const int nc = min(kChunk, ns - c0);
          for (int i = 0; i < KP; ++i) {
            const int p = (own0 + i) % KP;
            const int s = issued % kRing;
            const uint32_t ph = (issued / kRing) & 1;
            if (*(volatile int*)abort_flag || !mbar_wait(&empty[s], ph ^ 1)) {
              *(volatile int*)abort_flag = 1;
              atomicExch(err_flag, 21);
              ok = false;
              break;
            }
            mbar_expect_tx(&full[s], (uint32_t)(min(kChunk, ns) * kPanel * 2));
            tma_load_2d(ring + s * kTileBytes, &a.w[l], &full[s], p * kPanel, j * ns + c0);
            ++issued;
            (void)nc;
          }
        }
      }
      for (int i = (issued > kRing ? issued - kRing : 0); i < issued; ++i)
        if (!mbar_wait(&full[i % kRing], (i / kRing) & 1)) atomicExch(err_flag, 22);
      if (!mbar_wait(a0_full, 0)) atomicExch(err_flag, 27);
    }
  } else if (warp == 1) {
    if (lane == 0) {
      int used = 0;
      bool ok = true;
      for (int l = 0; l < a.L && ok; ++l) {
        const int ns = a.dims[l + 1] / C, KP = panels_of(a.dims[l]);
        const int pps = l == 0 ? KP : KP / C;   // panels per slice of the input
        const int own0 = l == 0 ? 0 : j * pps;
        const uint32_t acc = acc_column(ns, l);
        // layer 0: the features by TMA.  Layer l > 0: this CTA's own panels as the epilogue
        // writes them, then each peer's slice when its copies have landed; where this
        // layer's accumulator overlaps the previous one, first the epilogue's last panel
        // (it has read the whole accumulator then).
        uint32_t have = l == 0 ? 0xFFu : 0u;    // bit p: input panel p is in shared memory
        bool in_ok = true;
        if (l == 0) {
          in_ok = mbar_wait(a0_full, 0);
        } else {
          const int pns = a.dims[l] / C;
          const uint32_t pacc = acc_column(pns, l - 1);
          if (pacc < acc + ns && acc < pacc + pns) in_ok = mbar_wait(&panel_ready[pps - 1], (l - 1) & 1);
        }
        if (*(volatile int*)abort_flag || !in_ok) {
          *(volatile int*)abort_flag = 1;
          atomicExch(err_flag, 23);
          break;
        }
        fence_async_smem();
        tc_fence_after();
        for (int c0 = 0; c0 < ns && ok; c0 += kChunk) {
          const uint32_t idesc = idesc_bf16(kRows, min(kChunk, ns - c0));
          for (int i = 0; i < KP; ++i) {
            const int p = (own0 + i) % KP;
            if (!((have >> p) & 1u)) {
              const int src = p / pps;
              const bool got = src == j ? mbar_wait(&panel_ready[p - own0], (l - 1) & 1)
                                        : wait_cluster(&act_from[src], (l - 1) & 1);
              if (*(volatile int*)abort_flag || !got) {
                *(volatile int*)abort_flag = 1;
                atomicExch(err_flag, 28);
                ok = false;
                break;
              }
              fence_async_smem();
              tc_fence_after();
              have |= src == j ? (1u << p) : (((1u << pps) - 1u) << (src * pps));
            }
            const int s = used % kRing;
            const uint32_t ph = (used / kRing) & 1;
            if (*(volatile int*)abort_flag || !mbar_wait(&full[s], ph)) {
              *(volatile int*)abort_flag = 1;
              atomicExch(err_flag, 24);
              ok = false;
              break;
            }
            tc_fence_after();
            const uint32_t aa = smem_u32(act + p * kPanelBytes), bb = smem_u32(ring + s * kTileBytes);
#pragma unroll
            for (int kk = 0; kk < kPanel / 16; ++kk)
              umma_bf16(tmem + acc + c0, sw128_desc(aa + kk * 32), sw128_desc(bb + kk * 32), idesc, (i | kk) != 0);
            umma_commit(&empty[s]);
            ++used;
          }
        }
        if (ok) umma_commit(mma_done);
      }
    }
    __syncwarp();
  } else if (warp == kXchgWarp) {
    if (C > 1) {
      // per hidden layer: once this CTA's MMAs are done, expect the peers' slices and
      // announce it to every CTA; once every CTA's are done, copy each panel of this CTA's
      // slice to every peer as the epilogue finishes it; then tell each peer when its
      // slice has landed here.  Lane k talks to CTA k (lane i >= 1 copies to CTA j - i),
      // so the remote operations of one step fly together.
      bool ok = true;
      for (int l = 0; l + 1 < a.L && ok; ++l) {
        const int ns = a.dims[l + 1] / C, pps = ns / kPanel;
        const uint32_t slice = (uint32_t)pps * kPanelBytes;
        ok = mbar_wait(mma_done, l & 1) && !*(volatile int*)abort_flag;
        if (ok) {
          if (lane < C && lane != j) mbar_expect_tx(&act_from[lane], slice);
          __syncwarp();
          if (lane < C) arrive_remote(peers_done, (uint32_t)lane);
          ok = wait_cluster(peers_done, l & 1) && !*(volatile int*)abort_flag;
        }
        ok = __all_sync(0xffffffffu, ok);
        for (int pi = 0; pi < pps && ok; ++pi) {
          ok = __all_sync(0xffffffffu, mbar_wait(&panel_ready[pi], l & 1) && !*(volatile int*)abort_flag);
          if (ok && lane >= 1 && lane < C)
            bulk_to_peer(act + (j * pps + pi) * kPanelBytes, kPanelBytes, &act_from[j], (uint32_t)((j - lane + C) % C));
        }
        if (ok && lane >= 1 && lane < C) {
          const uint32_t k = (uint32_t)((j + lane) % C);
          ok = wait_cluster(&act_from[k], l & 1);
          if (ok) arrive_remote(copies_landed, k);
        }
        ok = __all_sync(0xffffffffu, ok);
        if (!ok && lane == 0) {
          *(volatile int*)abort_flag = 1;
          atomicExch(err_flag, 26);
        }
      }
    }
  } else {
    // epilogue: warp w owns TMEM lanes (rows) 32 (w % 4) .. +31 and the 16-column groups
    // g of each slice with g % 2 == half
    const int ew = warp - 2;
    const int quarter = warp % 4, half = ew / 4;
    const int r = quarter * 32 + lane;
    const int m = m0 + r;
    const bool row_ok = m < a.rows;
    const uint32_t lane_base = tmem + ((uint32_t)(quarter * 32) << 16);
    // this CTA's column slices of every bias, and of the output scaling, into shared memory
    float* cbias = reinterpret_cast<float*>(base + kConstOffset);
    {
      int off = 0;
      for (int l = 0; l < a.L; ++l) {
        const int ns = a.dims[l + 1] / C;
        for (int i = ew * 32 + lane; i < ns; i += 32 * kEpiWarps) cbias[off + i] = a.bias[l][j * ns + i];
        off += ns;
      }
      const int nsL = a.dims[a.L] / C;
      for (int i = ew * 32 + lane; i < nsL; i += 32 * kEpiWarps) {
        cbias[off + i] = a.scale ? a.scale[j * nsL + i] : 1.f;
        cbias[off + nsL + i] = a.shift ? a.shift[j * nsL + i] : 0.f;
      }
      epilogue_sync();
    }
    bool ok = true;
    int boff = 0;
    for (int l = 0; l < a.L && ok; ++l) {
      const int N = a.dims[l + 1], ns = N / C, cbase = j * ns;
      const bool last = (l == a.L - 1);
      const float* cb = cbias + boff;
      const float* cs = cb + ns;       // last layer: scale, then shift
      const float* ch = cs + ns;
      boff += ns;
      ok = mbar_wait(mma_done, l & 1) && !*(volatile int*)abort_flag;
      tc_fence_after();
      if (!__all_sync(0xffffffffu, ok)) {
        *(volatile int*)abort_flag = 1;
        atomicExch(err_flag, 25);
        ok = false;
        break;
      }
      const int groups = ns / 16;
      const uint32_t lane_acc = lane_base + acc_column(ns, l);
      if (!last) {
        // this CTA's slice of the next layer's input into its own panels, one panel after
        // the other: its own MMAs of this layer are done, and (from the second hidden layer
        // on) the copy engine has sent the slice these panels hold
        if (C > 1 && l > 0) {
          ok = mbar_wait(copies_landed, (l - 1) & 1) && !*(volatile int*)abort_flag;
          if (!__all_sync(0xffffffffu, ok)) {
            *(volatile int*)abort_flag = 1;
            atomicExch(err_flag, 29);
            ok = false;
            break;
          }
        }
#pragma unroll 1
        for (int g = half; g < groups; g += 4) {
          // groups g and g + 2 of this warp: two TMEM loads, one wait
          const bool two = g + 2 < groups;
          float va[16], vb[16];
          tmem_ld16x2(lane_acc + 16 * g, lane_acc + 16 * (two ? g + 2 : g), va, vb);
#pragma unroll
          for (int i = 0; i < 16; ++i) va[i] = fmaxf(va[i] + cb[16 * g + i], 0.f);
          put16_local(act, r, cbase + 16 * g, va);
          if (two) {
#pragma unroll
            for (int i = 0; i < 16; ++i) vb[i] = fmaxf(vb[i] + cb[16 * (g + 2) + i], 0.f);
            put16_local(act, r, cbase + 16 * (g + 2), vb);
          }
          // the panel is read by the copy engine and the tensor core
          fence_async_smem();
          tc_fence_before();
          mbar_arrive(&panel_ready[g / 4]);
        }
      } else {
#pragma unroll 1
        for (int g = half; g < groups; g += 2) {
          float v[16];
          tmem_ld16(lane_acc + 16 * g, v);
#pragma unroll
          for (int i = 0; i < 16; ++i) v[i] = (v[i] + cb[16 * g + i]) * cs[16 * g + i] + ch[16 * g + i];
          if (row_ok) {
            float4* o = reinterpret_cast<float4*>(a.out + (size_t)m * a.ldo + cbase + 16 * g);
#pragma unroll
            for (int i = 0; i < 4; ++i) o[i] = make_float4(v[4 * i], v[4 * i + 1], v[4 * i + 2], v[4 * i + 3]);
          }
        }
      }
    }
  }
  tc_fence_before();
  __syncthreads();
  if (warp == 1) tmem_dealloc(tmem, kTmemCols);
  cluster_sync_all();   // no CTA leaves while a peer may still write into its shared memory
}

}  // namespace

int forcing_cluster_size(const int* dims, int L, int rows, int sms) {
  if (L < 1 || L > kMlpMaxLayers || rows < 1) return 0;
  const int tiles = (rows + kRows - 1) / kRows;
  for (int C : {4, 2, 1}) {
    if (C > 1 && tiles * C > sms) continue;   // one wave of clusters
    bool fits = true;
    for (int l = 0; l <= L; ++l)
      if (dims[l] < 16 * C || dims[l] > kMlpMaxWidth || dims[l] % (16 * C)) fits = false;
    for (int l = 1; l < L; ++l)   // hidden layers: each CTA's slice is whole 64-column panels
      if (dims[l] % (kPanel * C)) fits = false;
    int consts = 2 * dims[L] / C;   // the slices of every bias and of the output scaling
    for (int l = 1; l <= L; ++l) consts += dims[l] / C;
    if (consts > kConstFloats) fits = false;
    if (fits) return C;
  }
  return 0;
}

int forcing_fused(const ForcingLaunch& f, cudaStream_t st) {
  const int C = f.csize;
  if (C != 1 && C != 2 && C != 4) return fail(DG_ERR_INVALID_ARG, "fused forcing: cluster size must be 1, 2 or 4");
  ForcingArgs a;
  std::memset(&a, 0, sizeof(a));
  int rc = make_map(&a.act0, f.act0, f.rows, f.dims[0], f.ld0, kRows);
  if (rc) return rc;
  for (int l = 0; l < f.L; ++l) {
    const int ns = f.dims[l + 1] / C;
    rc = make_map(&a.w[l], f.Wb[l], f.dims[l + 1], f.dims[l], f.ldw[l], ns < kChunk ? ns : kChunk);
    if (rc) return rc;
    a.bias[l] = f.bias[l];
  }
  for (int l = 0; l <= f.L; ++l) a.dims[l] = f.dims[l];
  a.L = f.L;
  a.rows = f.rows;
  a.csize = C;
  a.scale = f.scale;
  a.shift = f.shift;
  a.out = f.out;
  a.ldo = f.ldo;
  static bool configured = false;
  if (!configured) {
    DG_CUDA(cudaFuncSetAttribute(k_forcing_cluster, cudaFuncAttributeMaxDynamicSharedMemorySize, kSmemBytes));
    configured = true;
  }
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(((f.rows + kRows - 1) / kRows) * C);
  cfg.blockDim = dim3(kThreads);
  cfg.dynamicSmemBytes = kSmemBytes;
  cfg.stream = st;
  cudaLaunchAttribute attr[2];
  attr[0].id = cudaLaunchAttributeClusterDimension;
  attr[0].val.clusterDim.x = C;
  attr[0].val.clusterDim.y = 1;
  attr[0].val.clusterDim.z = 1;
  attr[1].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  attr[1].val.programmaticStreamSerializationAllowed = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 2;
  DG_CUDA(cudaLaunchKernelEx(&cfg, k_forcing_cluster, a, f.err));
  return DG_OK;
}

}  // namespace dgnn

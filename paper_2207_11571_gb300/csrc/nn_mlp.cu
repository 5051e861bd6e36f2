// Fused forward pass of the forcing network (Sec. 2.2, Fig. 2) on the tcgen05 tensor
// cores: one CTA carries 128 rows (elements) through every layer without leaving the SM.
//
// The layer input lives in shared memory as 64-column panels in the 128-byte-swizzled
// K-major layout the tensor core reads; the accumulator of the layer output lives in
// TMEM (up to 512 FP32 columns).  Six warps:
//   warp 0 (one elected thread): TMA producer.  It loads the 128-row input of layer 0
//          into the activation panels, then streams every weight tile of every layer
//          (128 output rows x 64 input columns, bf16) through a 6-stage ring;
//   warp 1: allocates the 512 TMEM columns; one thread issues tcgen05.mma (M = 128,
//          N = 128 per output chunk, K = 16) over the panels of the current layer and
//          commits each ring stage back to the producer and each finished layer to the
//          epilogue;
//   warps 2..5: epilogue.  Each reads its 32 TMEM lanes (rows), adds the bias, and for a
//          hidden layer applies ReLU and writes the bf16 result over the activation
//          panels (they are free: every MMA of the layer has completed), then signals
//          the next layer; for the output layer it applies the output scaling and
//          writes FP32 to global memory.
// Weights of layer l+1 stream in while the epilogue of layer l runs.  Every wait is
// bounded (about one second); on expiry the thread sets the error flag, the producer
// drains its copies with bounded waits, TMEM is released and the kernel returns.
#include <cudaTypedefs.h>

#include <cstring>

#include "dg_common.h"
#include "nn_gemm.h"
#include "nn_mlp.h"
#include "tc_common.cuh"

namespace dgnn {

using namespace tc;

namespace {

constexpr int kRows = 128;           // rows per CTA (MMA M)
constexpr int kChunk = 128;          // output columns per MMA (N) and per weight tile
constexpr int kPanel = 64;           // input columns per panel / weight tile (K slice)
constexpr int kPanelBytes = kRows * kPanel * 2;     // 16 KB
constexpr int kTileBytes = kChunk * kPanel * 2;     // 16 KB
constexpr int kMaxPanels = kMlpMaxWidth / kPanel;   // 8
constexpr int kRing = 6;
constexpr int kThreads = 192;
constexpr int kTmemCols = 512;

struct MlpSmem {
  static constexpr int kActBytes = kMaxPanels * kPanelBytes;   // 128 KB
  static constexpr int kRingOffset = kActBytes;
  static constexpr int kBarOffset = kRingOffset + kRing * kTileBytes;
  static constexpr int kBytes = kBarOffset + 256 + 1024;       // barriers, TMEM slot, alignment
};
static_assert(MlpSmem::kBytes <= 227 * 1024, "fused network kernel exceeds shared memory");

struct MlpArgs {
  CUtensorMap act0;                 // layer-0 input [rows][pad(d0)] bf16, box 64 x 128
  CUtensorMap w[kMlpMaxLayers];     // Wb[l] [d(l+1)][pad(d(l))] bf16, box 64 x 128
  const float* bias[kMlpMaxLayers];
  int dims[kMlpMaxLayers + 1];
  int L;
  int rows;
  const float* scale;               // output scaling (per output column) or NULL
  const float* shift;
  float* out;                       // [rows][ldo] FP32
  int ldo;
};

__device__ __forceinline__ int panels_of(int d) { return (d + kPanel - 1) / kPanel; }
__device__ __forceinline__ int chunks_of(int d) { return (d + kChunk - 1) / kChunk; }

// Byte offset of 16-byte chunk j (0..7) of row r in a 128-row panel with the 128-byte
// swizzle: rows are 128 bytes apart, chunk index XOR (row mod 8).
__device__ __forceinline__ uint32_t panel_offset(int r, int j) { return r * 128 + ((j ^ (r & 7)) << 4); }

__global__ void __launch_bounds__(kThreads, 1) k_mlp_fused(const __grid_constant__ MlpArgs a, int* __restrict__ err_flag) {
  extern __shared__ uint8_t smem_raw[];
  uint8_t* base = reinterpret_cast<uint8_t*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
  uint8_t* act = base;
  uint8_t* ring = base + MlpSmem::kRingOffset;
  uint64_t* full = reinterpret_cast<uint64_t*>(base + MlpSmem::kBarOffset);
  uint64_t* empty = full + kRing;
  uint64_t* a0_full = empty + kRing;
  uint64_t* mma_done = a0_full + 1;
  uint64_t* act_ready = mma_done + 1;
  uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(act_ready + 1);
  int* abort_flag = reinterpret_cast<int*>(tmem_slot + 1);

  const int warp = threadIdx.x / 32, lane = threadIdx.x % 32;
  const int m0 = blockIdx.x * kRows;

  if (threadIdx.x == 0) {
    for (int s = 0; s < kRing; ++s) {
      mbar_init(&full[s], 1);
      mbar_init(&empty[s], 1);
    }
    mbar_init(a0_full, 1);
    mbar_init(mma_done, 1);
    mbar_init(act_ready, 4);  // one arrival per epilogue warp
    *abort_flag = 0;
    mbar_fence_init();
  }
  if (warp == 1) tmem_alloc(tmem_slot, kTmemCols);
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = *tmem_slot;

  if (warp == 0) {
    if (lane == 0) {
      const int P0 = panels_of(a.dims[0]);
      mbar_expect_tx(a0_full, P0 * kPanelBytes);
      for (int p = 0; p < P0; ++p) tma_load_2d(act + p * kPanelBytes, &a.act0, a0_full, p * kPanel, m0);
      int issued = 0;
      bool ok = true;
      for (int l = 0; l < a.L && ok; ++l) {
        const int KP = panels_of(a.dims[l]), NC = chunks_of(a.dims[l + 1]);
        for (int c = 0; c < NC && ok; ++c)
          for (int p = 0; p < KP; ++p) {
            const int s = issued % kRing;
            const uint32_t ph = (issued / kRing) & 1;
            if (*(volatile int*)abort_flag || !mbar_wait(&empty[s], ph ^ 1)) {
              *(volatile int*)abort_flag = 1;
              atomicExch(err_flag, 11);
              ok = false;
              break;
            }
            mbar_expect_tx(&full[s], kTileBytes);
            tma_load_2d(ring + s * kTileBytes, &a.w[l], &full[s], p * kPanel, c * kChunk);
            ++issued;
          }
      }
      // drain: every issued copy must land before the CTA exits (bounded)
      for (int i = (issued > kRing ? issued - kRing : 0); i < issued; ++i)
        if (!mbar_wait(&full[i % kRing], (i / kRing) & 1)) atomicExch(err_flag, 12);
      if (!mbar_wait(a0_full, 0)) atomicExch(err_flag, 13);
    }
  } else if (warp == 1) {
    if (lane == 0) {
      bool ok = mbar_wait(a0_full, 0);
      if (!ok) {
        *(volatile int*)abort_flag = 1;
        atomicExch(err_flag, 14);
      }
      int used = 0;
      for (int l = 0; l < a.L && ok; ++l) {
        if (l > 0 && (*(volatile int*)abort_flag || !mbar_wait(act_ready, (l - 1) & 1))) {
          *(volatile int*)abort_flag = 1;
          atomicExch(err_flag, 15);
          break;
        }
        tc_fence_after();
        const int KP = panels_of(a.dims[l]), N = a.dims[l + 1], NC = chunks_of(N);
        for (int c = 0; c < NC && ok; ++c) {
          const int nc = min(kChunk, N - c * kChunk);  // a multiple of 16 (checked on the host)
          const uint32_t idesc = idesc_bf16(kRows, nc);
          for (int p = 0; p < KP; ++p) {
            const int s = used % kRing;
            const uint32_t ph = (used / kRing) & 1;
            if (*(volatile int*)abort_flag || !mbar_wait(&full[s], ph)) {
              *(volatile int*)abort_flag = 1;
              atomicExch(err_flag, 16);
              ok = false;
              break;
            }
            tc_fence_after();
            const uint32_t aa = smem_u32(act + p * kPanelBytes), bb = smem_u32(ring + s * kTileBytes);
#pragma unroll
            for (int kk = 0; kk < kPanel / 16; ++kk)
              umma_bf16(tmem + c * kChunk, sw128_desc(aa + kk * 32), sw128_desc(bb + kk * 32), idesc, (p | kk) != 0);
            umma_commit(&empty[s]);
            ++used;
          }
        }
        if (ok) umma_commit(mma_done);  // arrives when every MMA of layer l has completed
      }
    }
    __syncwarp();
  } else {
    // epilogue warps 2..5: warp w owns TMEM lanes (rows) 32 (w % 4) .. 32 (w % 4) + 31
    const int quarter = warp % 4;
    const int r = quarter * 32 + lane;
    const int m = m0 + r;
    const uint32_t lane_base = tmem + ((uint32_t)(quarter * 32) << 16);
    for (int l = 0; l < a.L; ++l) {
      // this layer's per-column constants, 16 per lane (lane k holds columns 16k .. 16k+15),
      // loaded while the MMAs run and broadcast with shuffles in the column loop
      const int Nl = a.dims[l + 1];
      const bool last = (l == a.L - 1);
      float cb[16], cs[16], ch[16];
#pragma unroll
      for (int i = 0; i < 16; ++i) {
        const int col = 16 * lane + i;
        cb[i] = col < Nl ? a.bias[l][col] : 0.f;
        cs[i] = (last && a.scale && col < Nl) ? a.scale[col] : 1.f;
        ch[i] = (last && a.shift && col < Nl) ? a.shift[col] : 0.f;
      }
      const bool ok = mbar_wait(mma_done, l & 1);
      if (!ok) {
        *(volatile int*)abort_flag = 1;
        atomicExch(err_flag, 17);
      }
      tc_fence_after();
      // tcgen05.ld is warp-collective: take the decision once per warp
      if (!__all_sync(0xffffffffu, ok && !*(volatile int*)abort_flag)) break;
      const int N = Nl;
      if (!last) {
        // hidden layer: relu(C + b) in bf16 over the activation panels (zero past N)
        const int Np = panels_of(N) * kPanel;
#pragma unroll 1
        for (int c0 = 0; c0 < Np; c0 += 16) {
          float v[16];
          if (c0 < N) tmem_ld16(lane_base + c0, v);
          const int src = c0 / 16;  // lane holding these 16 columns' constants
#pragma unroll
          for (int i = 0; i < 16; ++i) {
            const float b = __shfl_sync(0xffffffffu, cb[i], src);
            v[i] = (c0 + i < N) ? fmaxf(v[i] + b, 0.f) : 0.f;
          }
          uint8_t* pan = act + (c0 / kPanel) * kPanelBytes;
          const int j = (c0 % kPanel) / 8;
          *reinterpret_cast<uint4*>(pan + panel_offset(r, j)) =
              make_uint4(pack_bf16(v[0], v[1]), pack_bf16(v[2], v[3]), pack_bf16(v[4], v[5]), pack_bf16(v[6], v[7]));
          *reinterpret_cast<uint4*>(pan + panel_offset(r, j + 1)) = make_uint4(
              pack_bf16(v[8], v[9]), pack_bf16(v[10], v[11]), pack_bf16(v[12], v[13]), pack_bf16(v[14], v[15]));
        }
        fence_async_smem();  // the panels are the next layer's tensor-core operand
        tc_fence_before();
        __syncwarp();
        if (lane == 0) mbar_arrive(act_ready);
      } else {
        // output layer: (C + b) * scale + shift in FP32 to global memory
#pragma unroll 1
        for (int c0 = 0; c0 < N; c0 += 16) {
          float v[16];
          tmem_ld16(lane_base + c0, v);
          const int src = c0 / 16;
#pragma unroll
          for (int i = 0; i < 16; ++i) {
            const float b = __shfl_sync(0xffffffffu, cb[i], src);
            const float sc = __shfl_sync(0xffffffffu, cs[i], src);
            const float sh = __shfl_sync(0xffffffffu, ch[i], src);
            v[i] = (v[i] + b) * sc + sh;
          }
          if (m < a.rows) {
            float* o = a.out + (size_t)m * a.ldo + c0;
            if (c0 + 16 <= N && (a.ldo % 4) == 0 && (reinterpret_cast<uintptr_t>(a.out) & 15) == 0) {
#pragma unroll
              for (int i = 0; i < 4; ++i)
                reinterpret_cast<float4*>(o)[i] = make_float4(v[4 * i], v[4 * i + 1], v[4 * i + 2], v[4 * i + 3]);
            } else {
              for (int i = 0; i < 16 && c0 + i < N; ++i) o[i] = v[i];
            }
          }
        }
      }
    }
  }
  tc_fence_before();
  __syncthreads();
  if (warp == 1) tmem_dealloc(tmem, kTmemCols);
}

}  // namespace

bool mlp_fused_ok(const int* dims, int L) {
  if (L < 1 || L > kMlpMaxLayers) return false;
  for (int l = 0; l <= L; ++l)
    if (dims[l] < 16 || dims[l] > kMlpMaxWidth || dims[l] % 16) return false;
  return true;
}

int mlp_forward_fused(const __nv_bfloat16* act0, int ld0, const __nv_bfloat16* const* Wb, const int* ldw,
                      const float* const* bias, const int* dims, int L, int rows, const float* scale,
                      const float* shift, float* out, int ldo, int* err, cudaStream_t st) {
  if (!mlp_fused_ok(dims, L) || rows < 1) return fail(DG_ERR_INVALID_ARG, "fused network: unsupported shape");
  MlpArgs a;
  std::memset(&a, 0, sizeof(a));
  int rc = make_map(&a.act0, act0, rows, dims[0], ld0, kRows);
  if (rc) return rc;
  for (int l = 0; l < L; ++l) {
    rc = make_map(&a.w[l], Wb[l], dims[l + 1], dims[l], ldw[l], kChunk);
    if (rc) return rc;
    a.bias[l] = bias[l];
  }
  for (int l = 0; l <= L; ++l) a.dims[l] = dims[l];
  a.L = L;
  a.rows = rows;
  a.scale = scale;
  a.shift = shift;
  a.out = out;
  a.ldo = ldo;
  static bool configured = false;
  if (!configured) {
    DG_CUDA(cudaFuncSetAttribute(k_mlp_fused, cudaFuncAttributeMaxDynamicSharedMemorySize, MlpSmem::kBytes));
    configured = true;
  }
  k_mlp_fused<<<(rows + kRows - 1) / kRows, kThreads, MlpSmem::kBytes, st>>>(a, err);
  DG_CUDA(cudaGetLastError());
  return DG_OK;
}

}  // namespace dgnn

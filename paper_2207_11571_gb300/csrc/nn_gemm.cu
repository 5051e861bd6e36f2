// BF16 GEMM on the 5th-generation tensor cores (tcgen05) of sm_103a.
//
// One CTA computes a 128 x BN tile of C = A B^T.  Six warps:
//   warp 0 (one elected thread): TMA producer, 64-wide K slices of A and B into a
//          4-stage shared-memory ring (128-byte swizzle, K-major), mbarrier-tracked;
//   warp 1: allocates BN TMEM columns; one elected thread issues tcgen05.mma
//          (kind::f16, bf16 x bf16 -> f32, M = 128, N = BN, K = 16 per instruction)
//          and tcgen05.commit to free each stage and to signal the epilogue;
//   warps 2..5: epilogue, each reading its 32-lane quarter of the accumulator with
//          tcgen05.ld and applying bias / ReLU / affine / mask before storing.
// Every mbarrier wait is bounded (about one second of SM clock); on expiry the thread
// sets the error flag, the pipeline drains with bounded waits, TMEM is released and the
// kernel returns.
#include <cudaTypedefs.h>

#include <cstdio>
#include <cstring>
#include <mutex>
#include <unordered_map>

#include "dg_common.h"
#include "nn_gemm.h"
#include "tc_common.cuh"

namespace dgnn {

using namespace tc;

namespace {

constexpr int kBM = 128;
constexpr int kBK = 64;               // 64 bf16 = 128 bytes = one swizzle span
constexpr int kStages = 4;
constexpr int kThreads = 192;

template <int BN>
struct Smem {
  static constexpr int kABytes = kBM * kBK * 2;  // 16 KB
  static constexpr int kBBytes = BN * kBK * 2;
  static constexpr int kStageBytes = kABytes + kBBytes;
  static constexpr int kBarOffset = kStages * kStageBytes;
  static constexpr int kBytes = kBarOffset + 256 + 1024;  // barriers, TMEM slot, alignment slack
};

template <int BN>
__device__ __forceinline__ void epilogue_chunk(const GemmEpilogue& ep, int m, int n, int N, float v[16]) {
  const bool full = (n + 16 <= N);
  if (ep.kind == kGemmBiasReluBf16) {
    __nv_bfloat16* out = static_cast<__nv_bfloat16*>(ep.out) + (size_t)m * ep.ldo + n;
#pragma unroll
    for (int i = 0; i < 16; ++i) {
      float b = (ep.bias && n + i < N) ? ep.bias[n + i] : 0.f;
      v[i] = fmaxf(v[i] + b, 0.f);
    }
    if (full) {
      uint4 lo = make_uint4(pack_bf16(v[0], v[1]), pack_bf16(v[2], v[3]), pack_bf16(v[4], v[5]), pack_bf16(v[6], v[7]));
      uint4 hi = make_uint4(pack_bf16(v[8], v[9]), pack_bf16(v[10], v[11]), pack_bf16(v[12], v[13]),
                            pack_bf16(v[14], v[15]));
      reinterpret_cast<uint4*>(out)[0] = lo;
      reinterpret_cast<uint4*>(out)[1] = hi;
    } else {
      for (int i = 0; i < 16 && n + i < N; ++i) out[i] = __float2bfloat16_rn(v[i]);
    }
    return;
  }
  float* out = static_cast<float*>(ep.out) + (size_t)m * ep.ldo + n;
  if (ep.kind == kGemmMaskF32 && full && (ep.ldm % 8 == 0)) {
    // 16 mask values in two 16-byte loads
    const uint4* mp = reinterpret_cast<const uint4*>(ep.mask + (size_t)m * ep.ldm + n);
    const uint4 lo = mp[0], hi = mp[1];
    const uint32_t w[8] = {lo.x, lo.y, lo.z, lo.w, hi.x, hi.y, hi.z, hi.w};
#pragma unroll
    for (int i = 0; i < 16; ++i) {
      const uint32_t h = (w[i / 2] >> (16 * (i % 2))) & 0xFFFFu;
      // bf16 > 0: sign bit clear and not +0
      v[i] = (h != 0u && (h & 0x8000u) == 0u) ? v[i] : 0.f;
    }
  } else {
#pragma unroll
  for (int i = 0; i < 16; ++i) {
    if (n + i >= N) break;
    float x = v[i];
    if (ep.kind == kGemmMaskF32) {
      x = (__bfloat162float(ep.mask[(size_t)m * ep.ldm + n + i]) > 0.f) ? x : 0.f;
    } else {
      if (ep.bias) x += ep.bias[n + i];
      if (ep.relu) x = fmaxf(x, 0.f);
      if (ep.kind == kGemmAffineF32) {
        if (ep.scale) x *= ep.scale[n + i];
        if (ep.shift) x += ep.shift[n + i];
      }
    }
    v[i] = x;
  }
  }
  if (full && (ep.ldo % 4 == 0)) {
#pragma unroll
    for (int i = 0; i < 4; ++i)
      reinterpret_cast<float4*>(out)[i] = make_float4(v[4 * i], v[4 * i + 1], v[4 * i + 2], v[4 * i + 3]);
  } else {
    for (int i = 0; i < 16 && n + i < N; ++i) out[i] = v[i];
  }
}

template <int BN>
__global__ void __launch_bounds__(kThreads, 1)
k_gemm_bf16(const __grid_constant__ CUtensorMap tmA, const __grid_constant__ CUtensorMap tmB, int M, int N, int K,
            GemmEpilogue ep, int* __restrict__ err_flag) {
  using S = Smem<BN>;
  extern __shared__ uint8_t smem_raw[];
  uint8_t* base = reinterpret_cast<uint8_t*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
  uint64_t* full = reinterpret_cast<uint64_t*>(base + S::kBarOffset);
  uint64_t* empty = full + kStages;
  uint64_t* done = empty + kStages;
  uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(done + 1);
  int* abort_flag = reinterpret_cast<int*>(tmem_slot + 1);

  const int warp = threadIdx.x / 32, lane = threadIdx.x % 32;
  const int m0 = blockIdx.x * kBM, n0 = blockIdx.y * BN;
  // this CTA's run of 64-wide K slices (split-K over gridDim.z)
  const int KBall = (K + kBK - 1) / kBK;
  const int kb0 = (int)((long long)blockIdx.z * KBall / gridDim.z);
  const int KB = (int)((long long)(blockIdx.z + 1) * KBall / gridDim.z) - kb0;
  if (blockIdx.z > 0) ep.out = static_cast<float*>(ep.out) + blockIdx.z * ep.split_stride;

  if (threadIdx.x == 0) {
    for (int s = 0; s < kStages; ++s) {
      mbar_init(&full[s], 1);
      mbar_init(&empty[s], 1);
    }
    mbar_init(done, 1);
    *abort_flag = 0;
    mbar_fence_init();
  }
  if (warp == 1) tmem_alloc(tmem_slot, BN);
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = *tmem_slot;
  // Programmatic dependent launch: the next GEMM of the chain may start its prologue now
  // (it launches once every CTA of this grid is resident); this grid's own operands are
  // read only after the previous grid has completed and its writes are visible.
  asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
  asm volatile("griddepcontrol.wait;" ::: "memory");

  if (warp == 0) {
    if (lane == 0) {
      int issued = 0;
      for (int kb = 0; kb < KB; ++kb) {
        const int s = kb % kStages;
        const uint32_t ph = (kb / kStages) & 1;
        if (*(volatile int*)abort_flag || !mbar_wait(&empty[s], ph ^ 1)) {
          *(volatile int*)abort_flag = 1;
          atomicExch(err_flag, 1);
          break;
        }
        uint8_t* a = base + s * S::kStageBytes;
        uint8_t* b = a + S::kABytes;
        mbar_expect_tx(&full[s], S::kStageBytes);
        tma_load_2d(a, &tmA, &full[s], (kb0 + kb) * kBK, m0);
        tma_load_2d(b, &tmB, &full[s], (kb0 + kb) * kBK, n0);
        issued = kb + 1;
      }
      // drain: every issued copy must land before the CTA exits (bounded)
      for (int kb = (issued > kStages ? issued - kStages : 0); kb < issued; ++kb)
        if (!mbar_wait(&full[kb % kStages], (kb / kStages) & 1)) atomicExch(err_flag, 2);
    }
  } else if (warp == 1) {
    if (lane == 0) {
      constexpr uint32_t idesc = idesc_bf16(kBM, BN);
      for (int kb = 0; kb < KB; ++kb) {
        const int s = kb % kStages;
        const uint32_t ph = (kb / kStages) & 1;
        if (*(volatile int*)abort_flag || !mbar_wait(&full[s], ph)) {
          *(volatile int*)abort_flag = 1;
          atomicExch(err_flag, 3);
          break;
        }
        tc_fence_after();
        const uint32_t a = smem_u32(base + s * S::kStageBytes);
        const uint32_t b = a + S::kABytes;
#pragma unroll
        for (int kk = 0; kk < kBK / 16; ++kk)
          umma_bf16(tmem, sw128_desc(a + kk * 32), sw128_desc(b + kk * 32), idesc, (kb | kk) != 0);
        umma_commit(&empty[s]);
      }
      umma_commit(done);  // fires when every MMA issued above has completed
    }
    __syncwarp();
  } else {
    // epilogue warps 2..5: warp w reads TMEM lanes 32 (w % 4) .. 32 (w % 4) + 31
    const bool ok = mbar_wait(done, 0);
    if (!ok) {
      *(volatile int*)abort_flag = 1;
      atomicExch(err_flag, 4);
    }
    tc_fence_after();
    const int quarter = warp % 4;
    const int row = quarter * 32 + lane;
    const int m = m0 + row;
    // tcgen05.ld is warp-collective: take the decision once per warp
    const bool live = __all_sync(0xffffffffu, ok && !*(volatile int*)abort_flag);
#pragma unroll 1
    for (int c0 = 0; c0 < BN; c0 += 16) {
      float v[16];
      if (live) tmem_ld16(tmem + ((uint32_t)(quarter * 32) << 16) + c0, v);
      if (live && m < M && n0 + c0 < N) epilogue_chunk<BN>(ep, m, n0 + c0, N, v);
    }
  }
  tc_fence_before();
  __syncthreads();
  if (warp == 1) tmem_dealloc(tmem, BN);
}

PFN_cuTensorMapEncodeTiled_v12000 encode_fn() {
  static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
  if (!fn) {
    void* p = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) == cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      fn = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(p);
  }
  return fn;
}

}  // namespace

// A tensor map only encodes an address, a shape, strides and a box, so maps are cached
// on exactly those: a repeated GEMM (every layer of every training step and RK stage)
// skips the driver encode.
struct MapKey {
  uintptr_t ptr;
  long long rows, cols, ld;
  int box_rows;
  bool operator==(const MapKey& o) const {
    return ptr == o.ptr && rows == o.rows && cols == o.cols && ld == o.ld && box_rows == o.box_rows;
  }
};
struct MapKeyHash {
  size_t operator()(const MapKey& k) const {
    size_t h = std::hash<uintptr_t>()(k.ptr);
    for (long long v : {k.rows, k.cols, k.ld, (long long)k.box_rows}) h = h * 1000003u ^ std::hash<long long>()(v);
    return h;
  }
};
std::mutex g_map_mu;
std::unordered_map<MapKey, CUtensorMap, MapKeyHash> g_map_cache;
constexpr size_t kMapCacheMax = 4096;

int encode_map(CUtensorMap* map, const __nv_bfloat16* ptr, long long rows, long long cols, long long ld,
               int box_rows);

int make_map(CUtensorMap* map, const __nv_bfloat16* ptr, long long rows, long long cols, long long ld, int box_rows) {
  const MapKey key{reinterpret_cast<uintptr_t>(ptr), rows, cols, ld, box_rows};
  {
    std::lock_guard<std::mutex> lock(g_map_mu);
    auto it = g_map_cache.find(key);
    if (it != g_map_cache.end()) {
      *map = it->second;
      return DG_OK;
    }
  }
  int rc = encode_map(map, ptr, rows, cols, ld, box_rows);
  if (rc) return rc;
  std::lock_guard<std::mutex> lock(g_map_mu);
  if (g_map_cache.size() >= kMapCacheMax) g_map_cache.clear();
  g_map_cache.emplace(key, *map);
  return DG_OK;
}

int encode_map(CUtensorMap* map, const __nv_bfloat16* ptr, long long rows, long long cols, long long ld,
               int box_rows) {
  auto fn = encode_fn();
  if (!fn) return fail(DG_ERR_CUDA, "cuTensorMapEncodeTiled unavailable");
  if ((reinterpret_cast<uintptr_t>(ptr) & 15) || (ld % 8)) return fail(DG_ERR_INVALID_ARG, "GEMM operand misaligned");
  cuuint64_t dims[2] = {(cuuint64_t)cols, (cuuint64_t)rows};
  cuuint64_t strides[1] = {(cuuint64_t)(ld * 2)};
  cuuint32_t box[2] = {(cuuint32_t)kBK, (cuuint32_t)box_rows};
  cuuint32_t estr[2] = {1, 1};
  CUresult r = fn(map, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2, const_cast<__nv_bfloat16*>(ptr), dims, strides, box, estr,
                  CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                  CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  if (r != CUDA_SUCCESS) return fail(DG_ERR_CUDA, "cuTensorMapEncodeTiled failed (" + std::to_string((int)r) + ")");
  return DG_OK;
}

namespace {

template <int BN>
int launch_gemm(const __nv_bfloat16* A, int lda, const __nv_bfloat16* B, int ldb, int M, int N, int K,
                const GemmEpilogue& ep, int* err, cudaStream_t st) {
  CUtensorMap ma, mb;
  int rc = make_map(&ma, A, M, K, lda, kBM);
  if (rc) return rc;
  rc = make_map(&mb, B, N, K, ldb, BN);
  if (rc) return rc;
  auto kern = k_gemm_bf16<BN>;
  const int smem = Smem<BN>::kBytes;
  static bool configured = false;
  if (!configured) {
    DG_CUDA(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, smem));
    configured = true;
  }
  dim3 grid((M + kBM - 1) / kBM, (N + BN - 1) / BN, ep.splits);
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = grid;
  cfg.blockDim = dim3(kThreads);
  cfg.dynamicSmemBytes = smem;
  cfg.stream = st;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  attr[0].val.programmaticStreamSerializationAllowed = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  DG_CUDA(cudaLaunchKernelEx(&cfg, kern, ma, mb, M, N, K, ep, err));
  DG_CUDA(cudaGetLastError());
  return DG_OK;
}

}  // namespace

int gemm_pick_bn(int M, int N) {
  // enough CTAs to cover the 152 SMs when possible, wider tiles otherwise
  const int mt = (M + kBM - 1) / kBM;
  if (N > 128 && mt * ((N + 255) / 256) >= 152) return 256;
  if (N > 64 && mt * ((N + 127) / 128) >= 152) return 128;
  return 64;
}

int gemm_bf16(const __nv_bfloat16* A, int lda, const __nv_bfloat16* B, int ldb, int M, int N, int K,
              const GemmEpilogue& ep, int* err_flag, cudaStream_t st) {
  if (M <= 0 || N <= 0 || K <= 0) return fail(DG_ERR_INVALID_ARG, "gemm: empty problem");
  if (!ep.out || ep.ldo < N) return fail(DG_ERR_INVALID_ARG, "gemm: bad output");
  if (ep.kind == kGemmBiasReluBf16 && (ep.ldo % 8)) return fail(DG_ERR_INVALID_ARG, "gemm: bf16 output ld % 8");
  if (ep.kind == kGemmMaskF32 && !ep.mask) return fail(DG_ERR_INVALID_ARG, "gemm: mask missing");
  if (ep.splits < 1 || ep.splits > (K + kBK - 1) / kBK || (ep.splits > 1 && ep.kind != kGemmF32))
    return fail(DG_ERR_INVALID_ARG, "gemm: bad split-K");
  switch (gemm_pick_bn(M, N)) {
    case 256: return launch_gemm<256>(A, lda, B, ldb, M, N, K, ep, err_flag, st);
    case 128: return launch_gemm<128>(A, lda, B, ldb, M, N, K, ep, err_flag, st);
    default: return launch_gemm<64>(A, lda, B, ldb, M, N, K, ep, err_flag, st);
  }
}

}  // namespace dgnn

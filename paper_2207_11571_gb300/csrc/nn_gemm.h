// BF16 tensor-core GEMM for sm_103a (tcgen05 + TMA + TMEM), the dense contraction of
// the forcing network (Sec. 2.2, Fig. 2).
#pragma once

#include <cuda.h>
#include <cuda_bf16.h>
#include <cuda_runtime.h>

namespace dgnn {

// Epilogue applied to the FP32 accumulator tile C = A B^T (A: M x K, B: N x K, both
// K-contiguous bf16):
enum GemmKind {
  kGemmBiasReluBf16 = 0,  // out bf16 = relu(C + bias)              (hidden layer)
  kGemmAffineF32 = 1,     // out f32  = (C + bias) * scale + shift   (output layer; scale/shift may be null)
  kGemmF32 = 2,           // out f32  = C (+ bias if given)          (weight gradients)
  kGemmMaskF32 = 3        // out f32  = C * (mask > 0)               (gradient through ReLU)
};

struct GemmEpilogue {
  int kind = kGemmF32;
  const float* bias = nullptr;
  const float* scale = nullptr;
  const float* shift = nullptr;
  const __nv_bfloat16* mask = nullptr;
  int ldm = 0;
  void* out = nullptr;
  int ldo = 0;
  int relu = 0;  // f32 kinds: apply max(., 0) after the bias
  // Split-K (kGemmF32 only): the K range is cut into `splits` equal runs of 64-wide
  // slices; split z writes its partial product to out + z * split_stride (elements).
  int splits = 1;
  long long split_stride = 0;
};

// C[M x N] = A[M x K] B[N x K]^T with the given epilogue.  A and B are row-major bf16
// with leading dimensions lda, ldb (elements, multiples of 8, base 16-byte aligned);
// K is the reduction length: TMA reads columns at or beyond K, and rows beyond M (N),
// as zeros.  err_flag (device int) is set non-zero if a bounded wait inside the kernel
// ran out.  Returns a dg_status.
int gemm_bf16(const __nv_bfloat16* A, int lda, const __nv_bfloat16* B, int ldb, int M, int N, int K,
              const GemmEpilogue& ep, int* err_flag, cudaStream_t st);

// 2D tensor map of a row-major bf16 matrix [rows][cols] (leading dimension ld elements),
// box of 64 columns x box_rows rows with the 128-byte swizzle; cached.  Returns a dg_status.
int make_map(CUtensorMap* map, const __nv_bfloat16* ptr, long long rows, long long cols, long long ld, int box_rows);

// Tile width in N chosen for the problem (64, 128 or 256).
int gemm_pick_bn(int M, int N);

}  // namespace dgnn

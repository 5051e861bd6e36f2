// Fused forward pass of the forcing network on the tensor cores (nn_mlp.cu).
#pragma once

#include <cuda_bf16.h>
#include <cuda_runtime.h>

namespace dgnn {

constexpr int kMlpMaxWidth = 512;   // widest layer (TMEM holds 512 FP32 columns)
constexpr int kMlpMaxLayers = 9;

// True when every width is a multiple of 16 in [16, 512] and 1 <= L <= 9.
bool mlp_fused_ok(const int* dims, int L);

// out[rows][ldo] = scale * (W_L relu(... relu(W_1 x + b_1) ...) + b_L) + shift (scale and
// shift per output column, either may be NULL) for the bf16 inputs act0[rows][ld0]
// (columns dims[0] .. ld0 - 1 ignored), weights Wb[l] [dims[l+1]][ldw[l]] bf16 and biases
// bias[l] (FP32).  128 rows per CTA.  err: device flag set if a bounded wait expired.
int mlp_forward_fused(const __nv_bfloat16* act0, int ld0, const __nv_bfloat16* const* Wb, const int* ldw,
                      const float* const* bias, const int* dims, int L, int rows, const float* scale,
                      const float* shift, float* out, int ldo, int* err, cudaStream_t st);

}  // namespace dgnn

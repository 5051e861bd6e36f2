// The forcing of an RK stage in one cluster launch: every network layer on the tensor
// cores, from the bf16 features to the unscaled forcing (nn_forcing.cu).
#pragma once

#include <cuda_bf16.h>
#include <cuda_runtime.h>

namespace dgnn {

struct ForcingLaunch {
  const __nv_bfloat16* act0;       // features [rows][ld0] bf16 (columns dims[0] .. ld0 - 1 ignored)
  int ld0;
  const __nv_bfloat16* const* Wb;  // Wb[l] [dims[l+1]][ldw[l]] bf16
  const int* ldw;
  const float* const* bias;
  const int* dims;
  int L;
  int rows;             // elements of this launch
  int csize;            // CTAs per cluster (forcing_cluster_size)
  const float* scale;   // output scaling per column (std_out), may be NULL
  const float* shift;   // (mean_out), may be NULL
  float* out;           // [rows][ldo] FP32, 16-byte aligned rows
  int ldo;
  int* err;             // device error flag (bounded waits)
};

// CTAs per cluster (4, 2 or 1) for `rows` elements on `sms` SMs: the largest C whose
// clusters fit one wave and that divides every width into slices of a multiple of 16;
// 0 when the network does not fit the kernel (widths above 512, more than 9 layers).
int forcing_cluster_size(const int* dims, int L, int rows, int sms);

int forcing_fused(const ForcingLaunch& f, cudaStream_t st);

}  // namespace dgnn

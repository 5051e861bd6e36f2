// Corrective-forcing network (Sec. 2.2, Fig. 2): model state, CUDA-core kernels around
// the tensor-core GEMMs (input scaling, loss, gradient preparation, transposes, Adam)
// and the C ABI of include/dgnn_nn.h.
#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <string>
#include <vector>

#include "../../include/dgnn_nn.h"
#include "dg_common.h"
#include "dg_device.cuh"
#include "nn_bridge.h"
#include "nn_forcing.h"
#include "nn_gemm.h"
#include "nn_mlp.h"

using bf16 = __nv_bfloat16;

struct nn_model {
  nn_desc d{};
  int L = 0;                    // dense layers = n_hidden + 1
  int dims[10] = {};            // dims[0] = n_in, dims[1..n_hidden] = width, dims[L] = n_out
  int pad[10] = {};             // round_up(dims[l], 64): leading dimension of bf16 rows
  int bpad = 0;                 // round_up(max_batch, 64)
  float* W[9] = {};             // FP32 master [out][in]
  float* b[9] = {};
  bf16* Wb[9] = {};             // [out][pad(in)]
  bf16* Wt[9] = {};             // [in][pad(out)]
  float *mW[9] = {}, *vW[9] = {}, *mb[9] = {}, *vb[9] = {};
  float *gW[9] = {}, *gb[9] = {};
  float *mean_in = nullptr, *std_in = nullptr, *mean_out = nullptr, *std_out = nullptr;
  int adam_t = 0;
  bf16* act[10] = {};           // act[l]: input of layer l, [max_batch][pad(l)]
  bf16* actT[10] = {};          // [dims[l]][bpad]
  float* y = nullptr;           // [max_batch][n_out], scaled output
  float* dy = nullptr;          // [max_batch][max dim] gradient of the current layer output
  float* dx = nullptr;          // [max_batch][max dim] gradient of the current layer input
  bf16* dyb = nullptr;          // [max_batch][pad(max dim)]
  bf16* dyT = nullptr;          // [max dim][bpad]
  double* loss_part = nullptr;  // reduction partials
  float* gpart = nullptr;       // [bpad / 32][max dim] bias-gradient partial sums
  float* gws = nullptr;         // [kMaxSplits][max dim]^2 split-K partial weight gradients
  double* loss_dev = nullptr;
  double* loss_host = nullptr;  // pinned
  int* err = nullptr;           // device error flag of the tensor-core kernels
  int maxdim = 0;
  int fused = NN_INFER_CLUSTER; // inference path (nn_set_fused)
  // input means for scaling network inputs taken from solver states: in FP64 (FP64 state)
  // and shifted by the reference state of an FP32 context (cached for one reference)
  double* mean_in_d = nullptr;
  float* mean_shift = nullptr;
  double shift_rho = -1.0, shift_E = -1.0;
  std::vector<float> h_mean_in;
};

namespace dgnn {

namespace {

constexpr int kLossBlocks = 1024;
constexpr int kMaxSplits = 8;   // split-K factor bound of the weight-gradient GEMMs
constexpr int kLossThreads = 128;

int round_up(int x, int m) { return (x + m - 1) / m * m; }

// Programmatic dependent launch for the chain of network kernels: each kernel first waits
// until its predecessor has completed and its writes are visible, then lets its own
// successor be launched, so that launch latency overlaps execution.  (A kernel launched
// without the attribute passes the wait at once.)
__device__ __forceinline__ void pdl_enter() {
  asm volatile("griddepcontrol.wait;" ::: "memory");
  asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
}

// ------------------------------------------------------------------------------- kernels

// act0[r][f] = bf16((X[row(r)][f] - mean[f]) / std[f]) for f < n_in, 0 for the padding.
__global__ void k_prep_features(const float* __restrict__ X, const int64_t* __restrict__ idx, int rows, int n_in,
                                int ld, const float* __restrict__ mean, const float* __restrict__ sd,
                                bf16* __restrict__ out) {
  pdl_enter();
  const long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (t >= (long long)rows * ld) return;
  const int r = (int)(t / ld), f = (int)(t - (long long)r * ld);
  float v = 0.f;
  if (f < n_in) {
    const long long src = idx ? idx[r] : r;
    v = (X[src * n_in + f] - mean[f]) / sd[f];
  }
  out[t] = __float2bfloat16_rn(v);
}

// act0[e][slot * np + node] from the FP64 state q[var][elem][node] of elements e0 .. e0 + rows.
__global__ void k_prep_state(const double* __restrict__ q, long long N, int np, int first_var, int n_vars, int e0,
                             int rows, int ld, const double* __restrict__ mean, const float* __restrict__ sd,
                             bf16* __restrict__ out) {
  pdl_enter();
  const long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (t >= (long long)rows * ld) return;
  const int r = (int)(t / ld), f = (int)(t - (long long)r * ld);
  float v = 0.f;
  if (f < n_vars * np) {
    const int slot = f / np, node = f - slot * np;
    const double x = q[(long long)(first_var + slot) * N + (long long)(e0 + r) * np + node];
    v = d2f_rn(x - mean[f]) / sd[f];   // difference before rounding: near-constant features keep their digits
  }
  out[t] = __float2bfloat16_rn(v);
}

// Same from the FP32 reference-shifted stage state qf[var][elem][node] of an FP32 context;
// mshift = mean - reference, formed on the host in FP64.
__global__ void k_prep_state_f32(const float* __restrict__ qf, long long N, int np, int first_var, int n_vars, int e0,
                                 int rows, int ld, const float* __restrict__ mshift, const float* __restrict__ sd,
                                 bf16* __restrict__ out) {
  pdl_enter();
  const long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (t >= (long long)rows * ld) return;
  const int r = (int)(t / ld), f = (int)(t - (long long)r * ld);
  float v = 0.f;
  if (f < n_vars * np) {
    const int slot = f / np, node = f - slot * np;
    const float x = qf[(long long)(first_var + slot) * N + (long long)(e0 + r) * np + node];
    v = (x - mshift[f]) / sd[f];
  }
  out[t] = __float2bfloat16_rn(v);
}

// MSE against scaled targets: dy = 2 (y - t_s) / (rows n), partial sums of (y - t_s)^2.
// dL/dy of the MSE over norm_rows x n values, of which this launch holds rows x n (the
// rest on other ranks of a data-parallel step; norm_rows = rows: the whole batch).
__global__ void k_loss(const float* __restrict__ y, const float* __restrict__ Y, const int64_t* __restrict__ idx,
                       int rows, int norm_rows, int n, const float* __restrict__ mean, const float* __restrict__ sd,
                       float* __restrict__ dy, double* __restrict__ partial) {
  pdl_enter();
  // rows over blocks, features over threads; FP32 sums of a few squares per thread, a
  // warp-shuffle reduction, then the warps' sums added in FP64 in a fixed order
  __shared__ float wsum[kLossThreads / 32];
  float acc = 0.f;
  const float g = 2.f / ((float)norm_rows * (float)n);
  for (int r = blockIdx.x; r < rows; r += gridDim.x) {
    const long long src = idx ? idx[r] : r;
    const float* Yr = Y + src * n;
    const long long o = (long long)r * n;
    for (int f = threadIdx.x; f < n; f += blockDim.x) {
      const float ts = (Yr[f] - mean[f]) / sd[f];
      const float diff = y[o + f] - ts;
      dy[o + f] = g * diff;
      acc += diff * diff;
    }
  }
#pragma unroll
  for (int off = 16; off > 0; off >>= 1) acc += __shfl_down_sync(0xffffffffu, acc, off);
  if ((threadIdx.x & 31) == 0) wsum[threadIdx.x / 32] = acc;
  __syncthreads();
  if (threadIdx.x == 0) {
    double t = 0.0;
    for (int w = 0; w < kLossThreads / 32; ++w) t += (double)wsum[w];
    partial[blockIdx.x] = t;
  }
}
__global__ void k_sum_partials(const double* __restrict__ partial, int n, double scale, double* __restrict__ out) {
  pdl_enter();
  __shared__ double sh[kLossThreads];
  double acc = 0.0;
  for (int i = threadIdx.x; i < n; i += blockDim.x) acc += partial[i];
  sh[threadIdx.x] = acc;
  __syncthreads();
  for (int s = blockDim.x / 2; s > 0; s >>= 1) {
    if (threadIdx.x < s) sh[threadIdx.x] += sh[threadIdx.x + s];
    __syncthreads();
  }
  if (threadIdx.x == 0) *out = sh[0] * scale;
}

// Gradient of one layer's output g[rows][n] (FP32) -> bf16 copies gb[rows][ldb] (columns
// n..ldb-1 zero) and gT[n][ldt] (rows past `rows` zero), and per-tile column sums
// part[tile][n] of the bias gradient.  One 32 x 32 tile per block (2D grid over
// columns and row tiles), so every SM takes part.
__global__ void k_grad_prep(const float* __restrict__ g, int rows, int n, int ldb, int ldt, bf16* __restrict__ gb,
                            bf16* __restrict__ gT, float* __restrict__ part) {
  pdl_enter();
  __shared__ float tile[32][33];
  __shared__ float colsum[8][32];
  const int c0 = blockIdx.x * 32, r0 = blockIdx.y * 32;
  const int tx = threadIdx.x, ty = threadIdx.y;
  float cs = 0.f;
  for (int k = ty; k < 32; k += 8) {
    const int r = r0 + k, c = c0 + tx;
    const float v = (r < rows && c < n) ? g[(long long)r * n + c] : 0.f;
    tile[k][tx] = v;
    if (r < rows && c < ldb) gb[(long long)r * ldb + c] = __float2bfloat16_rn(v);
    cs += v;
  }
  colsum[ty][tx] = cs;
  __syncthreads();
  for (int k = ty; k < 32; k += 8) {
    const int c = c0 + k, r = r0 + tx;
    if (c < n && r < ldt) gT[(long long)c * ldt + r] = __float2bfloat16_rn(tile[tx][k]);
  }
  if (ty == 0 && c0 + tx < n) {
    float t = 0.f;
#pragma unroll
    for (int k = 0; k < 8; ++k) t += colsum[k][tx];
    part[(long long)blockIdx.y * n + c0 + tx] = t;
  }
}

// out[i] = sum over splits z of part[z][i], in split order (deterministic split-K sum).
__global__ void k_split_sum(const float* __restrict__ part, int splits, long long count, float* __restrict__ out) {
  pdl_enter();
  const long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (i >= count) return;
  float s = 0.f;
  for (int z = 0; z < splits; ++z) s += part[z * count + i];
  out[i] = s;
}

// db[c] = sum over row tiles of part[tile][c]: 32 columns per block, each of 32 thread
// rows sums every 32nd tile, then the 32 partial sums are added in row order
// (deterministic).
__global__ void k_col_sum(const float* __restrict__ part, int tiles, int n, float* __restrict__ db) {
  pdl_enter();
  __shared__ float sh[32][33];
  const int c = blockIdx.x * 32 + threadIdx.x;
  float s = 0.f;
  if (c < n)
    for (int t = threadIdx.y; t < tiles; t += 32) s += part[(long long)t * n + c];
  sh[threadIdx.y][threadIdx.x] = s;
  __syncthreads();
  if (threadIdx.y == 0 && c < n) {
    float t = 0.f;
    for (int k = 0; k < 32; ++k) t += sh[k][threadIdx.x];
    db[c] = t;
  }
}

// act[rows][ld] (bf16) -> actT[n][ldt] for the first n columns, rows padded with zeros.
__global__ void k_transpose_bf16(const bf16* __restrict__ a, int rows, int n, int ld, int ldt, bf16* __restrict__ aT) {
  pdl_enter();
  __shared__ bf16 tile[32][34];
  const int c0 = blockIdx.x * 32, r0 = blockIdx.y * 32;
  const int tx = threadIdx.x, ty = threadIdx.y;
  for (int k = ty; k < 32; k += 8) {
    const int r = r0 + k, c = c0 + tx;
    tile[k][tx] = (r < rows && c < n) ? a[(long long)r * ld + c] : __float2bfloat16_rn(0.f);
  }
  __syncthreads();
  for (int k = ty; k < 32; k += 8) {
    const int c = c0 + k, r = r0 + tx;
    if (c < n && r < ldt) aT[(long long)c * ldt + r] = tile[tx][k];
  }
}

// Adam (Kingma & Ba) on every parameter tensor of the network in one launch: segment j
// is a tensor [out][in] (in = 1 for biases); weight segments also refresh their bf16
// copies Wb[out][ldb] and Wt[in][ldt].  Blocks are assigned to segments by prefix counts.
constexpr int kAdamMaxSeg = 18;
struct AdamSeg {
  float *p, *g, *m, *v;
  long long count;
  int in;
  bf16* Wb;
  int ldb;
  bf16* Wt;
  int ldt;
};
struct AdamTable {
  int n;
  int block_start[kAdamMaxSeg + 1];
  AdamSeg seg[kAdamMaxSeg];
  float lr, b1, b2, eps, bc1, bc2;
};

__global__ void k_adam(const __grid_constant__ AdamTable tb) {
  pdl_enter();
  int j = 0;
  while (j + 1 < tb.n && (int)blockIdx.x >= tb.block_start[j + 1]) ++j;
  const AdamSeg& S = tb.seg[j];
  const long long t = (blockIdx.x - tb.block_start[j]) * (long long)blockDim.x + threadIdx.x;
  if (t >= S.count) return;
  const float gi = S.g[t];
  const float mi = tb.b1 * S.m[t] + (1.f - tb.b1) * gi;
  const float vi = tb.b2 * S.v[t] + (1.f - tb.b2) * gi * gi;
  S.m[t] = mi;
  S.v[t] = vi;
  const float mh = mi / tb.bc1, vh = vi / tb.bc2;
  const float w = S.p[t] - tb.lr * mh / (sqrtf(vh) + tb.eps);
  S.p[t] = w;
  if (S.Wb) {
    const int o = (int)(t / S.in), i = (int)(t - (long long)o * S.in);
    const bf16 wb = __float2bfloat16_rn(w);
    S.Wb[(long long)o * S.ldb + i] = wb;
    S.Wt[(long long)i * S.ldt + o] = wb;
  }
}

// bf16 copies of an FP32 weight [out][in].
__global__ void k_refresh_bf16(const float* __restrict__ W, long long count, int in, bf16* __restrict__ Wb, int ldb,
                               bf16* __restrict__ Wt, int ldt) {
  const long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (t >= count) return;
  const int o = (int)(t / in), i = (int)(t - (long long)o * in);
  const bf16 wb = __float2bfloat16_rn(W[t]);
  Wb[(long long)o * ldb + i] = wb;
  Wt[(long long)i * ldt + o] = wb;
}

// Per-feature sums of x and x^2 over rows (FP64), blocks stride over rows.
__global__ void k_moments(const float* __restrict__ X, long long rows, int n, double* __restrict__ s1,
                          double* __restrict__ s2) {
  const int f = blockIdx.x * blockDim.x + threadIdx.x;
  if (f >= n) return;
  double a = 0.0, b = 0.0;
  for (long long r = blockIdx.y; r < rows; r += gridDim.y) {
    const double x = X[r * n + f];
    a += x;
    b += x * x;
  }
  s1[(long long)blockIdx.y * n + f] = a;
  s2[(long long)blockIdx.y * n + f] = b;
}

// ------------------------------------------------------------------------------- helpers

int check_err(const nn_model* m, cudaStream_t st) {
  int h = 0;
  DG_CUDA(cudaMemcpyAsync(&h, m->err, sizeof(int), cudaMemcpyDeviceToHost, st));
  DG_CUDA(cudaStreamSynchronize(st));
  if (h) {
    cudaMemsetAsync(m->err, 0, sizeof(int), st);
    return fail(DG_ERR_TIMEOUT, "tensor-core GEMM: a bounded wait expired (code " + std::to_string(h) + ")");
  }
  return DG_OK;
}

inline unsigned blocks_for(long long n, int t) { return (unsigned)((n + t - 1) / t); }

// Launches a network kernel with programmatic stream serialization (see pdl_enter).
template <typename... KArgs, typename... Args>
cudaError_t pdl_launch(void (*kern)(KArgs...), dim3 grid, dim3 block, cudaStream_t st, Args&&... args) {
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = grid;
  cfg.blockDim = block;
  cfg.dynamicSmemBytes = 0;
  cfg.stream = st;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  attr[0].val.programmaticStreamSerializationAllowed = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  return cudaLaunchKernelEx(&cfg, kern, std::forward<Args>(args)...);
}

// Forward through all layers for `rows` rows whose scaled inputs are in act[0].
// last: if S != null, unscaled forcing into S (ld n_out); else scaled output into m->y.
int forward_layers(const nn_model* m, int rows, float* S, cudaStream_t st) {
  if (S && m->fused == NN_INFER_FUSED && mlp_fused_ok(m->dims, m->L)) {
    // inference: all layers in one kernel, activations kept on the SM
    const bf16* W[kMlpMaxLayers];
    const float* B[kMlpMaxLayers];
    for (int l = 0; l < m->L; ++l) {
      W[l] = m->Wb[l];
      B[l] = m->b[l];
    }
    return mlp_forward_fused(m->act[0], m->pad[0], W, m->pad, B, m->dims, m->L, rows, m->std_out, m->mean_out, S,
                             m->dims[m->L], m->err, st);
  }
  for (int l = 0; l < m->L; ++l) {
    GemmEpilogue ep;
    ep.bias = m->b[l];
    if (l < m->L - 1) {
      ep.kind = kGemmBiasReluBf16;
      ep.out = m->act[l + 1];
      ep.ldo = m->pad[l + 1];
    } else if (S) {
      ep.kind = kGemmAffineF32;
      ep.scale = m->std_out;
      ep.shift = m->mean_out;
      ep.out = S;
      ep.ldo = m->dims[m->L];
    } else {
      ep.kind = kGemmF32;
      ep.out = m->y;
      ep.ldo = m->dims[m->L];
    }
    int rc = gemm_bf16(m->act[l], m->pad[l], m->Wb[l], m->pad[l], rows, m->dims[l + 1], m->dims[l], ep, m->err, st);
    if (rc) return rc;
  }
  return DG_OK;
}

void free_model(nn_model* m) {
  if (!m) return;
  for (int l = 0; l < 9; ++l) {
    cudaFree(m->W[l]); cudaFree(m->b[l]); cudaFree(m->Wb[l]); cudaFree(m->Wt[l]);
    cudaFree(m->mW[l]); cudaFree(m->vW[l]); cudaFree(m->mb[l]); cudaFree(m->vb[l]);
    cudaFree(m->gW[l]); cudaFree(m->gb[l]);
  }
  for (int l = 0; l < 10; ++l) { cudaFree(m->act[l]); cudaFree(m->actT[l]); }
  cudaFree(m->mean_in); cudaFree(m->std_in); cudaFree(m->mean_out); cudaFree(m->std_out);
  cudaFree(m->y); cudaFree(m->dy); cudaFree(m->dx); cudaFree(m->dyb); cudaFree(m->dyT);
  cudaFree(m->loss_part); cudaFree(m->loss_dev); cudaFree(m->err); cudaFree(m->gpart); cudaFree(m->gws);
  cudaFree(m->mean_in_d); cudaFree(m->mean_shift);
  if (m->loss_host) cudaFreeHost(m->loss_host);
  delete m;
}

int validate_desc(const nn_desc* d) {
  if (!d) return fail(DG_ERR_INVALID_ARG, "nn_create: NULL desc");
  if (d->n_in < 1 || d->n_in > 4096 || d->n_out < 1 || d->n_out > 4096)
    return fail(DG_ERR_INVALID_ARG, "nn_create: n_in and n_out must be in [1, 4096]");
  if (d->width < 8 || d->width > 1024 || d->width % 8)
    return fail(DG_ERR_INVALID_ARG, "nn_create: width must be a multiple of 8 in [8, 1024]");
  if (d->n_hidden < 1 || d->n_hidden > 8) return fail(DG_ERR_INVALID_ARG, "nn_create: n_hidden must be in [1, 8]");
  if (d->max_batch < 1 || d->max_batch > (1 << 22)) return fail(DG_ERR_INVALID_ARG, "nn_create: bad max_batch");
  if (!((d->first_var == 0 && d->n_vars == 5) || (d->first_var == 1 && d->n_vars == 3)))
    return fail(DG_ERR_INVALID_ARG, "nn_create: (first_var, n_vars) must be (0, 5) or (1, 3)");
  return DG_OK;
}

int alloc_model(const nn_desc* d, nn_model** out) {
  int rc = validate_desc(d);
  if (rc) return rc;
  nn_model* m = new nn_model();
  m->d = *d;
  m->L = d->n_hidden + 1;
  m->dims[0] = d->n_in;
  for (int l = 1; l <= d->n_hidden; ++l) m->dims[l] = d->width;
  m->dims[m->L] = d->n_out;
  for (int l = 0; l <= m->L; ++l) {
    m->pad[l] = round_up(m->dims[l], 64);
    m->maxdim = std::max(m->maxdim, m->dims[l]);
  }
  m->bpad = round_up(d->max_batch, 64);
  const long long B = d->max_batch;
  cudaError_t e = cudaSuccess;
  auto A = [&](void** p, size_t bytes) {
    if (e == cudaSuccess) e = cudaMalloc(p, bytes);
    if (e == cudaSuccess) e = cudaMemset(*p, 0, bytes);
  };
  for (int l = 0; l < m->L; ++l) {
    const size_t in = m->dims[l], o = m->dims[l + 1];
    A((void**)&m->W[l], in * o * 4); A((void**)&m->b[l], o * 4);
    A((void**)&m->Wb[l], o * m->pad[l] * 2); A((void**)&m->Wt[l], in * m->pad[l + 1] * 2);
    A((void**)&m->mW[l], in * o * 4); A((void**)&m->vW[l], in * o * 4);
    A((void**)&m->mb[l], o * 4); A((void**)&m->vb[l], o * 4);
    A((void**)&m->gW[l], in * o * 4); A((void**)&m->gb[l], o * 4);
  }
  for (int l = 0; l < m->L; ++l) {
    A((void**)&m->act[l], B * m->pad[l] * 2);
    A((void**)&m->actT[l], (size_t)m->dims[l] * m->bpad * 2);
  }
  A((void**)&m->mean_in, d->n_in * 4); A((void**)&m->std_in, d->n_in * 4);
  A((void**)&m->mean_out, d->n_out * 4); A((void**)&m->std_out, d->n_out * 4);
  A((void**)&m->y, B * d->n_out * 4);
  A((void**)&m->dy, B * m->maxdim * 4);
  A((void**)&m->dx, B * m->maxdim * 4);
  A((void**)&m->dyb, B * round_up(m->maxdim, 64) * 2);
  A((void**)&m->dyT, (size_t)m->maxdim * m->bpad * 2);
  A((void**)&m->mean_in_d, d->n_in * 8);
  A((void**)&m->mean_shift, d->n_in * 4);
  A((void**)&m->loss_part, kLossBlocks * 8);
  A((void**)&m->gpart, (size_t)(m->bpad / 32) * m->maxdim * 4);
  A((void**)&m->gws, (size_t)kMaxSplits * m->maxdim * m->maxdim * 4);
  A((void**)&m->loss_dev, 8);
  A((void**)&m->err, 4);
  if (e == cudaSuccess) e = cudaMallocHost(&m->loss_host, 8);
  if (e != cudaSuccess) {
    free_model(m);
    return cuda_fail(e, "nn_create: allocation");
  }
  std::vector<float> ones(std::max(d->n_in, d->n_out), 1.f);
  cudaMemcpy(m->std_in, ones.data(), d->n_in * 4, cudaMemcpyHostToDevice);
  cudaMemcpy(m->std_out, ones.data(), d->n_out * 4, cudaMemcpyHostToDevice);
  m->h_mean_in.assign(d->n_in, 0.f);
  *out = m;
  return DG_OK;
}

// After the input means change: refresh their FP64 device copy and drop the shifted cache.
int means_changed(nn_model* m) {
  m->h_mean_in.resize(m->d.n_in);
  DG_CUDA(cudaMemcpy(m->h_mean_in.data(), m->mean_in, m->d.n_in * 4, cudaMemcpyDeviceToHost));
  std::vector<double> md(m->h_mean_in.begin(), m->h_mean_in.end());
  DG_CUDA(cudaMemcpy(m->mean_in_d, md.data(), m->d.n_in * 8, cudaMemcpyHostToDevice));
  m->shift_rho = m->shift_E = -1.0;
  return DG_OK;
}

// Means shifted by the reference state of an FP32 context (rho - rho_ref, rho e - E_ref).
int ensure_shift(nn_model* m, const dg_ctx* c) {
  if (m->shift_rho == c->phys.rho_ref && m->shift_E == c->phys.E_ref) return DG_OK;
  const int np = c->np;
  std::vector<float> sh(m->d.n_in);
  for (int f = 0; f < m->d.n_in; ++f) {
    const int var = m->d.first_var + f / np;
    const double ref = var == 0 ? c->phys.rho_ref : var == 4 ? c->phys.E_ref : 0.0;
    sh[f] = (float)((double)m->h_mean_in[f] - ref);
  }
  DG_CUDA(cudaMemcpy(m->mean_shift, sh.data(), m->d.n_in * 4, cudaMemcpyHostToDevice));
  m->shift_rho = c->phys.rho_ref;
  m->shift_E = c->phys.E_ref;
  return DG_OK;
}

int refresh_bf16(nn_model* m, int l, cudaStream_t st) {
  const long long cnt = (long long)m->dims[l] * m->dims[l + 1];
  k_refresh_bf16<<<blocks_for(cnt, 256), 256, 0, st>>>(m->W[l], cnt, m->dims[l], m->Wb[l], m->pad[l], m->Wt[l],
                                                        m->pad[l + 1]);
  DG_CUDA(cudaGetLastError());
  return DG_OK;
}

}  // namespace

static int sm_count() {
  static int sms = 0;
  if (!sms) {
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
      sms = 0;
  }
  return sms;
}

bool nn_phase_a_features(const nn_model* m, const dg_ctx* c, FeatureOut* out) {
  const int feat = m->d.n_vars * c->np;
  if (m->fused != NN_INFER_CLUSTER || c->nel > m->d.max_batch || m->d.n_in != feat || feat != m->pad[0]) return false;
  if (forcing_cluster_size(m->dims, m->L, c->nel, sm_count()) <= 0) return false;
  if (c->opts.precision == DG_PREC_FP32 && ensure_shift(const_cast<nn_model*>(m), c) != DG_OK) return false;
  out->out = m->act[0];
  out->ld = m->pad[0];
  out->first_var = m->d.first_var;
  out->n_vars = m->d.n_vars;
  out->shift32 = m->mean_shift;
  out->mean64 = m->mean_in_d;
  out->sd = m->std_in;
  return true;
}

int nn_forcing_on_state(const nn_model* m, const dg_ctx* c, const double* q, float* s, int* first_var, int* n_vars,
                        cudaStream_t st, bool features_ready) {
  if (!m || !c || !q || !s) return fail(DG_ERR_INVALID_ARG, "forcing: NULL argument");
  const int feat = m->d.n_vars * c->np;
  if (m->d.n_in != feat || m->d.n_out != feat)
    return fail(DG_ERR_INVALID_ARG, "forcing: network features do not match n_vars (P+1)^3 of the context");
  const bool f32 = c->opts.precision == DG_PREC_FP32;
  if (f32) {
    // the stage state of the FP32 operator is the reference-shifted copy written by phase A
    int rc = ensure_shift(const_cast<nn_model*>(m), c);
    if (rc) return rc;
  }
  const int sms = sm_count();
  // the one-launch network path writes the forcing rows as 16-byte vectors
  const bool aligned = (reinterpret_cast<uintptr_t>(s) & 15) == 0;
  for (int e0 = 0; e0 < c->nel; e0 += m->d.max_batch) {
    const int rows = std::min(m->d.max_batch, c->nel - e0);
    const long long tot = (long long)rows * m->pad[0];
    if (features_ready && rows == c->nel) {
      // the phase-A launch before this call wrote the features (nn_phase_a_features)
    } else if (f32) {
      DG_CUDA(pdl_launch(k_prep_state_f32, dim3(blocks_for(tot, 256)), dim3(256), st, static_cast<const float*>(c->qf), c->N, c->np,
                                                             m->d.first_var, m->d.n_vars, e0, rows, m->pad[0],
                                                             m->mean_shift, m->std_in, m->act[0]));
    } else {
      DG_CUDA(pdl_launch(k_prep_state, dim3(blocks_for(tot, 256)), dim3(256), st, q, c->N, c->np, m->d.first_var, m->d.n_vars, e0, rows,
                                                         m->pad[0], m->mean_in_d, m->std_in, m->act[0]));
    }
    DG_CUDA(cudaGetLastError());
    const int C = (m->fused == NN_INFER_CLUSTER && aligned) ? forcing_cluster_size(m->dims, m->L, rows, sms) : 0;
    if (C > 0) {
      // every layer in one launch: clusters of C CTAs share the activations on chip
      ForcingLaunch f;
      f.act0 = m->act[0];
      f.ld0 = m->pad[0];
      f.Wb = m->Wb;
      f.ldw = m->pad;
      f.bias = m->b;
      f.dims = m->dims;
      f.L = m->L;
      f.rows = rows;
      f.csize = C;
      f.scale = m->std_out;
      f.shift = m->mean_out;
      f.out = s + (long long)e0 * feat;
      f.ldo = feat;
      f.err = m->err;
      int rc = forcing_fused(f, st);
      if (rc) return rc;
    } else {
      int rc = forward_layers(m, rows, s + (long long)e0 * feat, st);
      if (rc) return rc;
    }
  }
  if (first_var) *first_var = m->d.first_var;
  if (n_vars) *n_vars = m->d.n_vars;
  return DG_OK;
}

}  // namespace dgnn

namespace dgnn {
namespace {

bool adam_ok(const nn_adam& a) {
  return a.lr >= 0.f && std::isfinite(a.lr) && a.beta1 >= 0.f && a.beta1 < 1.f && a.beta2 >= 0.f && a.beta2 < 1.f &&
         a.eps > 0.f && std::isfinite(a.eps);
}

// Forward, MSE and backward of `batch` rows into the model's gradient buffers, normalised
// over norm_batch rows (a data-parallel step's global batch).  The loss share goes to
// m->loss_dev.
int backward_into_grads(nn_model* m, const float* X, const float* Y, const int64_t* idx, int batch, int norm_batch,
                        cudaStream_t st) {
  const int L = m->L, n_out = m->d.n_out;
  // forward, keeping every layer input (bf16) in act[]
  long long tot = (long long)batch * m->pad[0];
  DG_CUDA(pdl_launch(k_prep_features, dim3(blocks_for(tot, 256)), dim3(256), st, X, idx, batch, m->d.n_in, m->pad[0], m->mean_in, m->std_in,
                                                        m->act[0]));
  DG_CUDA(cudaGetLastError());
  int rc = forward_layers(m, batch, nullptr, st);
  if (rc) return rc;
  // loss and dL/dy
  DG_CUDA(pdl_launch(k_loss, dim3(kLossBlocks), dim3(kLossThreads), st, m->y, Y, idx, batch, norm_batch, n_out, m->mean_out,
                     m->std_out, m->dy, m->loss_part));
  DG_CUDA(cudaGetLastError());
  DG_CUDA(pdl_launch(k_sum_partials, dim3(1), dim3(kLossThreads), st, m->loss_part, kLossBlocks,
                     1.0 / ((double)norm_batch * n_out), m->loss_dev));
  DG_CUDA(cudaGetLastError());
  // backward
  float* g = m->dy;   // gradient w.r.t. the output of layer l, [batch][dims[l+1]]
  float* gnext = m->dx;
  for (int l = L - 1; l >= 0; --l) {
    const int o = m->dims[l + 1], in = m->dims[l];
    const int ldb = round_up(o, 64);
    const int tiles = m->bpad / 32;
    dim3 gp(ldb / 32, tiles), bt(32, 8);
    DG_CUDA(pdl_launch(k_grad_prep, dim3(gp), dim3(bt), st, g, batch, o, ldb, m->bpad, m->dyb, m->dyT, m->gpart));
    DG_CUDA(cudaGetLastError());
    DG_CUDA(pdl_launch(k_col_sum, dim3((o + 31) / 32), dim3(dim3(32, 32)), st, m->gpart, tiles, o, m->gb[l]));
    DG_CUDA(cudaGetLastError());
    dim3 gt((in + 31) / 32, (m->bpad + 31) / 32);
    DG_CUDA(pdl_launch(k_transpose_bf16, dim3(gt), dim3(bt), st, m->act[l], batch, in, m->pad[l], m->bpad, m->actT[l]));
    DG_CUDA(cudaGetLastError());
    // dW = g^T act : M = o, N = in, K = batch.  Few output tiles and a long K: split K
    // so that the CTAs cover the SMs, then sum the partial products in a fixed order.
    GemmEpilogue ew;
    ew.kind = kGemmF32;
    ew.ldo = in;
    const int tiles_mn = ((o + 127) / 128) * ((in + gemm_pick_bn(o, in) - 1) / gemm_pick_bn(o, in));
    const int kslices = (batch + 63) / 64;
    const int splits = std::max(1, std::min({kMaxSplits, kslices, 152 / tiles_mn}));
    if (splits > 1) {
      ew.out = m->gws;
      ew.splits = splits;
      ew.split_stride = (long long)o * in;
    } else {
      ew.out = m->gW[l];
    }
    rc = gemm_bf16(m->dyT, m->bpad, m->actT[l], m->bpad, o, in, batch, ew, m->err, st);
    if (rc) return rc;
    if (splits > 1) {
      const long long cnt = (long long)o * in;
      DG_CUDA(pdl_launch(k_split_sum, dim3(blocks_for(cnt, 256)), dim3(256), st, m->gws, splits, cnt, m->gW[l]));
      DG_CUDA(cudaGetLastError());
    }
    if (l > 0) {
      // d act = g W, masked by the ReLU of the layer that produced act[l]
      GemmEpilogue ex;
      ex.kind = kGemmMaskF32;
      ex.mask = m->act[l];
      ex.ldm = m->pad[l];
      ex.out = gnext;
      ex.ldo = in;
      rc = gemm_bf16(m->dyb, ldb, m->Wt[l], m->pad[l + 1], batch, in, o, ex, m->err, st);
      if (rc) return rc;
      std::swap(g, gnext);
    }
  }
  return DG_OK;
}

// One Adam step of every parameter from the gradient buffers (also refreshes the bf16
// copies of the weights).
int adam_apply(nn_model* m, const nn_adam& a, cudaStream_t st) {
  const int L = m->L;
  ++m->adam_t;
  const float bc1 = 1.f - std::pow(a.beta1, (float)m->adam_t);
  const float bc2 = 1.f - std::pow(a.beta2, (float)m->adam_t);
  AdamTable at{};
  at.lr = a.lr;
  at.b1 = a.beta1;
  at.b2 = a.beta2;
  at.eps = a.eps;
  at.bc1 = bc1;
  at.bc2 = bc2;
  int blocks = 0;
  for (int l = 0; l < L; ++l) {
    const long long cw = (long long)m->dims[l] * m->dims[l + 1];
    at.block_start[at.n] = blocks;
    at.seg[at.n++] = AdamSeg{m->W[l], m->gW[l], m->mW[l], m->vW[l], cw, m->dims[l], m->Wb[l], m->pad[l], m->Wt[l],
                             m->pad[l + 1]};
    blocks += (int)blocks_for(cw, 256);
    const long long cb = m->dims[l + 1];
    at.block_start[at.n] = blocks;
    at.seg[at.n++] = AdamSeg{m->b[l], m->gb[l], m->mb[l], m->vb[l], cb, 1, nullptr, 0, nullptr, 0};
    blocks += (int)blocks_for(cb, 256);
  }
  at.block_start[at.n] = blocks;
  DG_CUDA(pdl_launch(k_adam, dim3(blocks), dim3(256), st, at));
  DG_CUDA(cudaGetLastError());
  return DG_OK;
}

int loss_to_host(nn_model* m, float* loss_out, cudaStream_t st) {
  if (!loss_out) return DG_OK;
  DG_CUDA(cudaMemcpyAsync(m->loss_host, m->loss_dev, 8, cudaMemcpyDeviceToHost, st));
  int rc = check_err(m, st);
  if (rc) return rc;
  *loss_out = (float)*m->loss_host;
  return DG_OK;
}

}  // namespace
}  // namespace dgnn

using namespace dgnn;

extern "C" {

int nn_create(const nn_desc* desc, const float* init_uniform, nn_model** out) {
  if (!out) return fail(DG_ERR_INVALID_ARG, "nn_create: out is NULL");
  *out = nullptr;
  nn_model* m = nullptr;
  int rc = alloc_model(desc, &m);
  if (rc) return rc;
  if (init_uniform) {
    size_t off = 0;
    for (int l = 0; l < m->L; ++l) {
      const size_t cnt = (size_t)m->dims[l] * m->dims[l + 1];
      std::vector<float> w(cnt);
      const double s = std::sqrt(6.0 / m->dims[l]);
      for (size_t i = 0; i < cnt; ++i) w[i] = (float)(init_uniform[off + i] * s);
      off += cnt;
      cudaError_t e = cudaMemcpy(m->W[l], w.data(), cnt * 4, cudaMemcpyHostToDevice);
      if (e != cudaSuccess) {
        free_model(m);
        return cuda_fail(e, "nn_create: weight upload");
      }
    }
  }
  for (int l = 0; l < m->L; ++l) {
    rc = refresh_bf16(m, l, 0);
    if (rc) { free_model(m); return rc; }
  }
  cudaError_t e = cudaDeviceSynchronize();
  if (e != cudaSuccess) { free_model(m); return cuda_fail(e, "nn_create"); }
  *out = m;
  return DG_OK;
}

int nn_destroy(nn_model* m) {
  if (!m) return fail(DG_ERR_INVALID_ARG, "nn_destroy: NULL");
  free_model(m);
  return DG_OK;
}

int nn_get_desc(const nn_model* m, nn_desc* d) {
  if (!m || !d) return fail(DG_ERR_INVALID_ARG, "nn_get_desc: NULL");
  *d = m->d;
  return DG_OK;
}

int nn_set_scalers(nn_model* m, const float* mi, const float* si, const float* mo, const float* so) {
  if (!m || !mi || !si || !mo || !so) return fail(DG_ERR_INVALID_ARG, "nn_set_scalers: NULL argument");
  for (int i = 0; i < m->d.n_in; ++i)
    if (!(si[i] > 0) || !std::isfinite(mi[i])) return fail(DG_ERR_INVALID_ARG, "nn_set_scalers: std_in must be > 0");
  for (int i = 0; i < m->d.n_out; ++i)
    if (!(so[i] > 0) || !std::isfinite(mo[i])) return fail(DG_ERR_INVALID_ARG, "nn_set_scalers: std_out must be > 0");
  DG_CUDA(cudaMemcpy(m->mean_in, mi, m->d.n_in * 4, cudaMemcpyHostToDevice));
  DG_CUDA(cudaMemcpy(m->std_in, si, m->d.n_in * 4, cudaMemcpyHostToDevice));
  DG_CUDA(cudaMemcpy(m->mean_out, mo, m->d.n_out * 4, cudaMemcpyHostToDevice));
  DG_CUDA(cudaMemcpy(m->std_out, so, m->d.n_out * 4, cudaMemcpyHostToDevice));
  return means_changed(m);
}

int nn_get_scalers(const nn_model* m, float* mi, float* si, float* mo, float* so) {
  if (!m) return fail(DG_ERR_INVALID_ARG, "nn_get_scalers: NULL");
  if (mi) DG_CUDA(cudaMemcpy(mi, m->mean_in, m->d.n_in * 4, cudaMemcpyDeviceToHost));
  if (si) DG_CUDA(cudaMemcpy(si, m->std_in, m->d.n_in * 4, cudaMemcpyDeviceToHost));
  if (mo) DG_CUDA(cudaMemcpy(mo, m->mean_out, m->d.n_out * 4, cudaMemcpyDeviceToHost));
  if (so) DG_CUDA(cudaMemcpy(so, m->std_out, m->d.n_out * 4, cudaMemcpyDeviceToHost));
  return DG_OK;
}

int nn_compute_scalers(nn_model* m, const float* X, const float* Y, int64_t rows, void* stream) {
  if (!m || !X || !Y || rows < 1) return fail(DG_ERR_INVALID_ARG, "nn_compute_scalers: bad argument");
  cudaStream_t st = (cudaStream_t)stream;
  const int G = 64;
  for (int which = 0; which < 2; ++which) {
    const int n = which ? m->d.n_out : m->d.n_in;
    const float* A = which ? Y : X;
    double* buf = nullptr;
    DG_CUDA(cudaMalloc(&buf, 2 * (size_t)G * n * 8));
    dim3 grid((n + 127) / 128, G);
    k_moments<<<grid, 128, 0, st>>>(A, rows, n, buf, buf + (size_t)G * n);
    cudaError_t e = cudaGetLastError();
    std::vector<double> h(2 * (size_t)G * n);
    if (e == cudaSuccess) e = cudaMemcpyAsync(h.data(), buf, h.size() * 8, cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    cudaFree(buf);
    if (e != cudaSuccess) return cuda_fail(e, "nn_compute_scalers");
    std::vector<float> mean(n), sd(n);
    for (int f = 0; f < n; ++f) {
      double s1 = 0, s2 = 0;
      for (int g = 0; g < G; ++g) {
        s1 += h[(size_t)g * n + f];
        s2 += h[(size_t)G * n + (size_t)g * n + f];
      }
      const double mu = s1 / rows;
      const double var = std::max(s2 / rows - mu * mu, 0.0);
      mean[f] = (float)mu;
      sd[f] = var > 0 ? (float)std::sqrt(var) : 1.f;
      if (!(sd[f] > 0)) sd[f] = 1.f;
    }
    DG_CUDA(cudaMemcpy(which ? m->mean_out : m->mean_in, mean.data(), n * 4, cudaMemcpyHostToDevice));
    DG_CUDA(cudaMemcpy(which ? m->std_out : m->std_in, sd.data(), n * 4, cudaMemcpyHostToDevice));
  }
  return means_changed(m);
}

int nn_set_fused(nn_model* m, int mode) {
  if (!m) return fail(DG_ERR_INVALID_ARG, "nn_set_fused: NULL model");
  if (mode != NN_INFER_LAYERS && mode != NN_INFER_FUSED && mode != NN_INFER_CLUSTER)
    return fail(DG_ERR_INVALID_ARG, "nn_set_fused: unknown mode");
  m->fused = mode;
  return DG_OK;
}

int nn_forward(const nn_model* m, const float* X, float* S, int rows, void* stream) {
  if (!m || !X || !S) return fail(DG_ERR_INVALID_ARG, "nn_forward: NULL argument");
  if (rows < 1 || rows > m->d.max_batch) return fail(DG_ERR_INVALID_ARG, "nn_forward: rows outside [1, max_batch]");
  cudaStream_t st = (cudaStream_t)stream;
  const long long tot = (long long)rows * m->pad[0];
  DG_CUDA(pdl_launch(k_prep_features, dim3(blocks_for(tot, 256)), dim3(256), st, X, nullptr, rows, m->d.n_in, m->pad[0], m->mean_in,
                                                        m->std_in, m->act[0]));
  DG_CUDA(cudaGetLastError());
  return forward_layers(m, rows, S, st);
}

int nn_forcing_infer(const nn_model* m, const dg_ctx* c, const double* q, float* s, void* stream) {
  if (!m || !c || !q || !s) return fail(DG_ERR_INVALID_ARG, "nn_forcing_infer: NULL argument");
  cudaStream_t st = (cudaStream_t)stream;
  // the FP32 operator feeds the network its stage state: build it from q (phase A)
  if (c->opts.precision == DG_PREC_FP32) DG_CUDA(launch_gradient(c, q, 0, st));
  return nn_forcing_on_state(m, c, q, s, nullptr, nullptr, st);
}

int nn_train_step(nn_model* m, const float* X, const float* Y, const int64_t* idx, int batch, const nn_adam* hp,
                  float* loss_out, void* stream) {
  if (!m || !X || !Y) return fail(DG_ERR_INVALID_ARG, "nn_train_step: NULL argument");
  if (batch < 1 || batch > m->d.max_batch) return fail(DG_ERR_INVALID_ARG, "nn_train_step: batch outside [1, max_batch]");
  nn_adam a{1e-3f, 0.9f, 0.999f, 1e-7f};
  if (hp) a = *hp;
  if (!adam_ok(a))
    return fail(DG_ERR_INVALID_ARG, "nn_train_step: Adam needs lr >= 0, beta1 and beta2 in [0, 1), eps > 0 (finite)");
  cudaStream_t st = (cudaStream_t)stream;
  int rc = backward_into_grads(m, X, Y, idx, batch, batch, st);
  if (rc) return rc;
  rc = adam_apply(m, a, st);
  if (rc) return rc;
  return loss_to_host(m, loss_out, st);
}

int nn_backward(nn_model* m, const float* X, const float* Y, const int64_t* idx, int batch, int global_batch,
                float* loss_out, void* stream) {
  if (!m || !X || !Y) return fail(DG_ERR_INVALID_ARG, "nn_backward: NULL argument");
  if (batch < 1 || batch > m->d.max_batch) return fail(DG_ERR_INVALID_ARG, "nn_backward: batch outside [1, max_batch]");
  if (global_batch < batch) return fail(DG_ERR_INVALID_ARG, "nn_backward: global_batch < batch");
  cudaStream_t st = (cudaStream_t)stream;
  int rc = backward_into_grads(m, X, Y, idx, batch, global_batch, st);
  if (rc) return rc;
  return loss_to_host(m, loss_out, st);
}

int nn_grad_buffers(nn_model* m, int l, float** dW, float** db) {
  if (!m || l < 0 || l >= m->L) return fail(DG_ERR_INVALID_ARG, "nn_grad_buffers: bad layer");
  if (dW) *dW = m->gW[l];
  if (db) *db = m->gb[l];
  return DG_OK;
}

int nn_adam_apply(nn_model* m, const nn_adam* hp, void* stream) {
  if (!m) return fail(DG_ERR_INVALID_ARG, "nn_adam_apply: NULL model");
  nn_adam a{1e-3f, 0.9f, 0.999f, 1e-7f};
  if (hp) a = *hp;
  if (!adam_ok(a))
    return fail(DG_ERR_INVALID_ARG, "nn_adam_apply: Adam needs lr >= 0, beta1 and beta2 in [0, 1), eps > 0 (finite)");
  return adam_apply(m, a, (cudaStream_t)stream);
}

int nn_get_params(const nn_model* m, int l, float* W, float* b) {
  if (!m || l < 0 || l >= m->L) return fail(DG_ERR_INVALID_ARG, "nn_get_params: bad layer");
  DG_CUDA(cudaDeviceSynchronize());
  if (W) DG_CUDA(cudaMemcpy(W, m->W[l], (size_t)m->dims[l] * m->dims[l + 1] * 4, cudaMemcpyDeviceToHost));
  if (b) DG_CUDA(cudaMemcpy(b, m->b[l], (size_t)m->dims[l + 1] * 4, cudaMemcpyDeviceToHost));
  return DG_OK;
}

int nn_set_params(nn_model* m, int l, const float* W, const float* b) {
  if (!m || l < 0 || l >= m->L) return fail(DG_ERR_INVALID_ARG, "nn_set_params: bad layer");
  DG_CUDA(cudaDeviceSynchronize());
  if (W) DG_CUDA(cudaMemcpy(m->W[l], W, (size_t)m->dims[l] * m->dims[l + 1] * 4, cudaMemcpyHostToDevice));
  if (b) DG_CUDA(cudaMemcpy(m->b[l], b, (size_t)m->dims[l + 1] * 4, cudaMemcpyHostToDevice));
  int rc = refresh_bf16(m, l, 0);
  if (rc) return rc;
  DG_CUDA(cudaDeviceSynchronize());
  return DG_OK;
}

int nn_get_grads(const nn_model* m, int l, float* dW, float* db) {
  if (!m || l < 0 || l >= m->L) return fail(DG_ERR_INVALID_ARG, "nn_get_grads: bad layer");
  DG_CUDA(cudaDeviceSynchronize());
  if (dW) DG_CUDA(cudaMemcpy(dW, m->gW[l], (size_t)m->dims[l] * m->dims[l + 1] * 4, cudaMemcpyDeviceToHost));
  if (db) DG_CUDA(cudaMemcpy(db, m->gb[l], (size_t)m->dims[l + 1] * 4, cudaMemcpyDeviceToHost));
  return DG_OK;
}

int nn_gemm_bf16(int M, int N, int K, const void* A, int lda, const void* B, int ldb, const float* bias, int relu,
                 float* C, int ldc, void* stream) {
  if (!A || !B || !C) return fail(DG_ERR_INVALID_ARG, "nn_gemm_bf16: NULL argument");
  if (lda < K || ldb < K) return fail(DG_ERR_INVALID_ARG, "nn_gemm_bf16: leading dimension below K");
  // one error flag for the primitive, allocated once (thread-safe static initialisation)
  static int* const err = []() -> int* {
    int* p = nullptr;
    if (cudaMalloc(&p, sizeof(int)) != cudaSuccess) return nullptr;
    if (cudaMemset(p, 0, sizeof(int)) != cudaSuccess) {
      cudaFree(p);
      return nullptr;
    }
    return p;
  }();
  if (!err) return fail(DG_ERR_CUDA, "nn_gemm_bf16: could not allocate the error flag");
  GemmEpilogue ep;
  ep.kind = kGemmF32;
  ep.bias = bias;
  ep.relu = relu;
  ep.out = C;
  ep.ldo = ldc;
  cudaStream_t st = (cudaStream_t)stream;
  int rc = gemm_bf16(static_cast<const bf16*>(A), lda, static_cast<const bf16*>(B), ldb, M, N, K, ep, err, st);
  if (rc) return rc;
  int h = 0;
  DG_CUDA(cudaMemcpyAsync(&h, err, sizeof(int), cudaMemcpyDeviceToHost, st));
  DG_CUDA(cudaStreamSynchronize(st));
  if (h) {
    cudaMemset(err, 0, sizeof(int));
    return fail(DG_ERR_TIMEOUT, "nn_gemm_bf16: a bounded wait expired");
  }
  return DG_OK;
}

}  // extern "C"

// ------------------------------------------------------------------------------- save / load
// File: "DGNNNET1", u32 version, nn_desc, i32 adam step, scalers, then per layer W, b and
// the Adam moments (FP32), then the FNV-1a 64-bit hash of every byte after the magic.

namespace {

struct Blob {
  std::vector<unsigned char> bytes;
  void put(const void* p, size_t n) {
    const unsigned char* c = static_cast<const unsigned char*>(p);
    bytes.insert(bytes.end(), c, c + n);
  }
};

uint64_t fnv1a(const unsigned char* p, size_t n) {
  uint64_t h = 1469598103934665603ull;
  for (size_t i = 0; i < n; ++i) {
    h ^= p[i];
    h *= 1099511628211ull;
  }
  return h;
}

const char kMagic[8] = {'D', 'G', 'N', 'N', 'N', 'E', 'T', '1'};

// Appends n device floats to the blob; false (with the CUDA error in *err) if the copy fails.
bool put_device(Blob& b, const float* d, size_t n, cudaError_t* err) {
  std::vector<float> h(n);
  *err = cudaMemcpy(h.data(), d, n * 4, cudaMemcpyDeviceToHost);
  if (*err != cudaSuccess) return false;
  b.put(h.data(), n * 4);
  return true;
}

}  // namespace

extern "C" int nn_save(const nn_model* m, const char* path) {
  if (!m || !path) return fail(DG_ERR_INVALID_ARG, "nn_save: NULL argument");
  DG_CUDA(cudaDeviceSynchronize());
  Blob b;
  const uint32_t version = 1;
  b.put(&version, 4);
  b.put(&m->d, sizeof(nn_desc));
  b.put(&m->adam_t, 4);
  // every device copy is checked: a failed copy must not be written under a valid checksum
  cudaError_t ce = cudaSuccess;
  bool copied = true;
  for (const float* p : {m->mean_in, m->std_in}) copied = copied && put_device(b, p, m->d.n_in, &ce);
  for (const float* p : {m->mean_out, m->std_out}) copied = copied && put_device(b, p, m->d.n_out, &ce);
  for (int l = 0; copied && l < m->L; ++l) {
    const size_t w = (size_t)m->dims[l] * m->dims[l + 1], o = m->dims[l + 1];
    for (const float* p : {m->W[l], m->mW[l], m->vW[l]}) copied = copied && put_device(b, p, w, &ce);
    for (const float* p : {m->b[l], m->mb[l], m->vb[l]}) copied = copied && put_device(b, p, o, &ce);
  }
  if (!copied) return cuda_fail(ce, "nn_save: device-to-host copy (no file written)");
  const uint64_t h = fnv1a(b.bytes.data(), b.bytes.size());
  FILE* f = std::fopen(path, "wb");
  if (!f) return fail(DG_ERR_IO, std::string("nn_save: cannot open ") + path);
  bool ok = std::fwrite(kMagic, 1, 8, f) == 8 && std::fwrite(b.bytes.data(), 1, b.bytes.size(), f) == b.bytes.size() &&
            std::fwrite(&h, 1, 8, f) == 8;
  ok = (std::fclose(f) == 0) && ok;
  return ok ? DG_OK : fail(DG_ERR_IO, std::string("nn_save: write failed for ") + path);
}

extern "C" int nn_load(const char* path, int max_batch, nn_model** out) {
  if (!path || !out) return fail(DG_ERR_INVALID_ARG, "nn_load: NULL argument");
  *out = nullptr;
  FILE* f = std::fopen(path, "rb");
  if (!f) return fail(DG_ERR_IO, std::string("nn_load: cannot open ") + path);
  std::vector<unsigned char> all;
  unsigned char buf[65536];
  size_t r;
  while ((r = std::fread(buf, 1, sizeof(buf), f)) > 0) all.insert(all.end(), buf, buf + r);
  std::fclose(f);
  const size_t head = 8 + 4 + sizeof(nn_desc) + 4;
  if (all.size() < head + 8 || std::memcmp(all.data(), kMagic, 8) != 0)
    return fail(DG_ERR_IO, "nn_load: not a network file (bad magic or truncated)");
  uint64_t h_file;
  std::memcpy(&h_file, all.data() + all.size() - 8, 8);
  if (fnv1a(all.data() + 8, all.size() - 16) != h_file) return fail(DG_ERR_IO, "nn_load: checksum mismatch");
  size_t off = 8;
  auto get = [&](void* dst, size_t n) -> bool {
    if (off + n > all.size() - 8) return false;
    std::memcpy(dst, all.data() + off, n);
    off += n;
    return true;
  };
  uint32_t version = 0;
  nn_desc d;
  int adam_t = 0;
  get(&version, 4);
  get(&d, sizeof(d));
  get(&adam_t, 4);
  if (version != 1) return fail(DG_ERR_IO, "nn_load: unsupported version");
  d.max_batch = max_batch > 0 ? max_batch : d.max_batch;
  nn_model* m = nullptr;
  int rc = alloc_model(&d, &m);
  if (rc) return rc;
  m->adam_t = adam_t;
  auto upload = [&](float* dst, size_t n) -> bool {
    std::vector<float> h(n);
    if (!get(h.data(), n * 4)) return false;
    return cudaMemcpy(dst, h.data(), n * 4, cudaMemcpyHostToDevice) == cudaSuccess;
  };
  bool ok = upload(m->mean_in, d.n_in) && upload(m->std_in, d.n_in) && upload(m->mean_out, d.n_out) &&
            upload(m->std_out, d.n_out);
  for (int l = 0; ok && l < m->L; ++l) {
    const size_t w = (size_t)m->dims[l] * m->dims[l + 1], o = m->dims[l + 1];
    ok = upload(m->W[l], w) && upload(m->mW[l], w) && upload(m->vW[l], w) && upload(m->b[l], o) &&
         upload(m->mb[l], o) && upload(m->vb[l], o);
  }
  if (!ok || off != all.size() - 8) {
    free_model(m);
    return fail(DG_ERR_IO, "nn_load: truncated or inconsistent file");
  }
  for (int l = 0; l < m->L; ++l) {
    rc = refresh_bf16(m, l, 0);
    if (rc) { free_model(m); return rc; }
  }
  DG_CUDA(cudaDeviceSynchronize());
  rc = means_changed(m);
  if (rc) { free_model(m); return rc; }
  *out = m;
  return DG_OK;
}

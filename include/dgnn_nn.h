/*
 * dgnn_nn.h - C ABI of the corrective-forcing network in libdgnn.so (arXiv
 * 2207.11571, Sec. 2.2 and Fig. 2): a fully connected network, the same for every
 * element, from the element's low-order state to the forcing s at its nodes.
 *
 * Architecture (reading of Sec. 2.2: first and last layers linear, ReLU in between):
 * scaled input -> n_hidden x [Dense(width) + ReLU] -> Dense(n_out) linear.
 * Scaling (Sec. 2.2 "re-scale the values"): per-feature z-scores, x_s = (x - mean_in)
 * / std_in in, s = y * std_out + mean_out out; training minimises the mean squared
 * error of y against the scaled target (Table 1 "Loss Error", MSE).
 *
 * Arithmetic: weights kept in FP32 (master) with a BF16 working copy; every dense
 * layer is a BF16 x BF16 -> FP32 tcgen05 tensor-core GEMM (sm_103a); hidden
 * activations are stored in BF16; bias, ReLU, loss, gradients of the biases and Adam
 * in FP32; the loss is reduced in FP64.
 *
 * Conventions of dgnn.h apply (status codes, dg_last_error, device pointers unless a
 * parameter says HOST, streams as void*).  Feature rows are float32, row-major,
 * n_in (n_out) values per row; used as a forcing, a row is one element and feature
 * v_slot * (P+1)^3 + node holds variable first_var + v_slot at that node.
 */
#ifndef DGNN_NN_H
#define DGNN_NN_H

#include <stdint.h>

#include "dgnn.h"

#ifdef __cplusplus
extern "C" {
#endif

typedef struct {
  int n_in;       /* input features per row (1..4096) */
  int n_out;      /* output features per row (1..4096) */
  int width;      /* hidden width H (8..1024, multiple of 8) */
  int n_hidden;   /* hidden ReLU layers (1..8) */
  int first_var;  /* as a forcing: state variable of feature slot 0 (0: all five, 1: momenta) */
  int n_vars;     /* as a forcing: variables per node (5, or 3 for the momenta of Sec. 2.2) */
  int max_batch;  /* largest number of rows per forward or training call (>= 1) */
} nn_desc;

/* Adam hyperparameters (Kingma & Ba); defaults lr 1e-3, beta1 0.9, beta2 0.999, eps 1e-7. */
typedef struct {
  float lr, beta1, beta2, eps;
} nn_adam;

/* Creates a network.  init_uniform (HOST, may be NULL for all-zero weights) holds U(-1,1)
 * draws for every weight, layer by layer, each layer row-major [out][in]; weights are
 * set to u * sqrt(6 / fan_in) (He uniform), biases to 0, scalers to identity
 * (mean 0, std 1).  Allocates weights, Adam moments and activation buffers for
 * max_batch rows. */
int nn_create(const nn_desc* desc, const float* init_uniform, nn_model** out);
int nn_destroy(nn_model* net);

/* Copies the scalers from HOST arrays (n_in, n_in, n_out, n_out floats). std values must be > 0. */
int nn_set_scalers(nn_model* net, const float* mean_in, const float* std_in, const float* mean_out,
                   const float* std_out);
/* Copies the scalers to HOST arrays (any may be NULL). */
int nn_get_scalers(const nn_model* net, float* mean_in, float* std_in, float* mean_out, float* std_out);
/* Per-feature mean and population standard deviation of X (rows x n_in) and Y (rows x n_out),
 * DEVICE arrays, reduced in FP64; a feature with zero spread gets std 1.  Synchronises. */
int nn_compute_scalers(nn_model* net, const float* X, const float* Y, int64_t rows, void* stream);

/* S = forcing for raw feature rows X: scale, network, unscale.  X: rows x n_in, S: rows x
 * n_out (DEVICE float).  rows <= max_batch. */
int nn_forward(const nn_model* net, const float* X, float* S, int rows, void* stream);

/* Implementation switch of inference, no counterpart in the paper (all modes compute the
 * same network in BF16 with FP32 accumulation):
 *   NN_INFER_CLUSTER (the default): the forcing of a solver state (nn_forcing_infer, and
 *     the forcing inside dg_rhs / dg_rk3_step / dg_diagnostics) runs in one launch that
 *     forms the element features from the stage state, carries 128 elements per cluster of
 *     1, 2 or 4 CTAs through every layer (each CTA owns a slice of every layer's output
 *     columns and shares its activations through distributed shared memory) and writes
 *     the unscaled forcing; it needs every width a multiple of 16 C in [16 C, 512] and
 *     n_hidden <= 8, else (and for nn_forward) one tensor-core GEMM per layer;
 *   NN_INFER_FUSED: nn_forward and the forcing through one fused kernel of 128 rows per
 *     CTA that keeps every layer's activations on the SM (widths multiples of 16 in
 *     [16, 512], n_hidden <= 8);
 *   NN_INFER_LAYERS: one tensor-core GEMM per layer.
 * DG_ERR_INVALID_ARG for another mode. */
enum { NN_INFER_LAYERS = 0, NN_INFER_FUSED = 1, NN_INFER_CLUSTER = 2 };
int nn_set_fused(nn_model* net, int mode);

/* s = forcing of every element of the state q of context ctx (dgnn.h layout), written as
 * rows e = 0 .. K^3 - 1 of n_vars (P+1)^3 floats (DEVICE).  Requires n_in = n_out =
 * n_vars (P+1)^3.  Elements are processed in chunks of max_batch (per-layer paths) or all
 * in one launch (NN_INFER_CLUSTER). */
int nn_forcing_infer(const nn_model* net, const dg_ctx* ctx, const double* q, float* s, void* stream);

/* One optimisation step (Sec. 2.1, "Train corrective forcing"): forward on rows idx[0..batch)
 * of X and Y (idx DEVICE int64, or NULL for rows 0..batch-1), MSE loss against the scaled
 * targets, backward, Adam update of the FP32 weights and refresh of the BF16 copies.
 * hp may be NULL (defaults: lr 1e-3, beta1 0.9, beta2 0.999, eps 1e-7); DG_ERR_INVALID_ARG
 * unless lr >= 0, beta1 and beta2 in [0, 1) and eps > 0, all finite, or batch is outside
 * [1, max_batch].  loss_out (HOST, may be NULL) receives the batch loss; when
 * given the call synchronises the stream.  Returns DG_ERR_TIMEOUT if a bounded wait in a
 * tensor-core kernel expired. */
int nn_train_step(nn_model* net, const float* X, const float* Y, const int64_t* idx, int batch,
                  const nn_adam* hp, float* loss_out, void* stream);

/* The two halves of nn_train_step, for data-parallel training over ranks that each hold
 * part of a batch (the MSE of Sec. 2.2 is a mean over rows, so its gradient is the sum of
 * the ranks' shares):
 *   nn_backward: forward, MSE and backward of rows idx[0..batch) of X and Y (as in
 *     nn_train_step) into the model's gradient buffers, normalised over global_batch rows
 *     (>= batch; = batch: the plain gradient of this batch).  loss_out (HOST, may be
 *     NULL; synchronises the stream) receives this call's share of the loss, the sum of
 *     its squared errors over global_batch x n_out.  No parameter changes.
 *   nn_grad_buffers: DEVICE addresses of layer l's gradient buffers, dW [out][in] and db
 *     [out] FP32, owned by the model and valid until nn_destroy; a caller may all-reduce
 *     them in place between the two calls.
 *   nn_adam_apply: one Adam step of every parameter from the gradient buffers (hp as in
 *     nn_train_step), refreshing the BF16 copies.
 * nn_train_step(batch) is nn_backward(batch, batch) followed by nn_adam_apply, with the
 * same launches in the same order.  Errors as nn_train_step; DG_ERR_INVALID_ARG for
 * global_batch < batch or a bad layer. */
int nn_backward(nn_model* net, const float* X, const float* Y, const int64_t* idx, int batch, int global_batch,
                float* loss_out, void* stream);
int nn_grad_buffers(nn_model* net, int layer, float** dW, float** db);
int nn_adam_apply(nn_model* net, const nn_adam* hp, void* stream);

/* Layer l (0 .. n_hidden) weights [out][in] and biases [out], FP32 master copy (HOST). */
int nn_get_params(const nn_model* net, int layer, float* W, float* b);
int nn_set_params(nn_model* net, int layer, const float* W, const float* b);
/* Gradients of layer l from the last nn_train_step or nn_backward (HOST). */
int nn_get_grads(const nn_model* net, int layer, float* dW, float* db);
/* Description of the network (HOST). */
int nn_get_desc(const nn_model* net, nn_desc* desc);

/* Saves / loads weights, scalers and Adam state to a binary file with a header and an
 * FNV-1a checksum.  Load returns DG_ERR_IO for a missing, truncated or corrupted file. */
int nn_save(const nn_model* net, const char* path);
int nn_load(const char* path, int max_batch, nn_model** out);

/* Library primitive used by the network: C[M x N] = A[M x K] B[N x K]^T on the tensor cores,
 * A, B row-major bf16 (DEVICE, leading dimensions lda, ldb multiples of 8 elements,
 * 16-byte aligned), C row-major float (ldc >= N), optional bias[N] and ReLU.  The operands
 * are read in 16-byte chunks: when K is not a multiple of 8, columns K .. roundup(K, 8) - 1
 * of A and B must hold zeros; columns beyond are never read.  Synchronises the stream and
 * returns DG_ERR_TIMEOUT if a bounded wait of the kernel expired; the flag it reads is one
 * per process, so concurrent calls on several streams may see each other's timeout. */
int nn_gemm_bf16(int M, int N, int K, const void* A, int lda, const void* B, int ldb,
                 const float* bias, int relu, float* C, int ldc, void* stream);

#ifdef __cplusplus
}
#endif

#endif /* DGNN_NN_H */

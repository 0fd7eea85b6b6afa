/*
 * pdqp_ws.h -- C ABI of the learned warm start and of the tensor-core BF16
 * GEMM it runs on (sm_103a).
 *
 * The paper (Lu & Yang, "A Practical and Optimal First-Order Method for
 * Large-Scale Convex Quadratic Programming") has no learned component:
 * Algorithm 1 takes its starting point (x^{0,0}, y^{0,0}) as an input and
 * Section 5 starts from zero.  This network supplies that input for members
 * of a parameterised QP family that share Q, A, l, u and differ in (c, b); the
 * solve itself, its restarts and its termination test are unchanged, so a
 * poor prediction costs iterations but never changes the answer.
 *
 * Network (F = n + m features, all matrices row-major, W of shape (out, in)):
 *   u   = (v - in_mean) * in_scale,   v = [c; b]      per feature, float32, then bf16
 *   h_0 = u P'                       P: d x F, fixed (never trained)
 *   h_j = relu(h_{j-1} W_j' + b_j)    j = 1..depth, width w (layer index j-1)
 *   o   = h_depth W_out' + b_out      W_out: F x w (layer index depth)
 *   [x0; y0] = out_mean + out_std * o                 float64
 * Training minimises mean((o - t)^2) over samples and features with
 * t = (fl32([x*; y*]) - out_mean) * out_inv, by Adam (Kingma & Ba 2015) with
 * bias correction, over minibatches visited in the order
 * i -> (a i + s) mod count, (a, s) from SplitMix64 of (seed, epoch); the last
 * partial minibatch of an epoch is dropped.  Weights and activations are
 * stored in bfloat16 and every product accumulates in float32 (tcgen05 tensor
 * cores, accumulator in tensor memory); master weights, gradients and Adam
 * moments are float32.
 *
 * Data layout of the family arrays (row i = instance i, the stacking of a
 * pdqp_create_batch handle over equal-size instances):
 *   C [count x n], B [count x m], X [count x n], Y [count x m]   float64.
 *
 * Conventions follow pdqp.h (mem_space, stream, ownership, status codes).
 * The handle holds float32/bf16 copies of its parameters and the training set
 * it was last given (its projected inputs and normalised targets).
 */
#ifndef PDQP_WS_H
#define PDQP_WS_H

#include <stdint.h>

#include "pdqp.h"

#ifdef __cplusplus
extern "C" {
#endif

typedef struct pdqp_ws_s *pdqp_ws_handle;

typedef struct {
  int32_t epochs;   /* passes over the training set (>= 0) */
  int32_t batch;    /* minibatch rows: multiple of 8, <= max_batch */
  float lr;         /* Adam step size (> 0) */
  float beta1;      /* first-moment decay, [0, 1) */
  float beta2;      /* second-moment decay, [0, 1) */
  float eps;        /* Adam denominator offset (>= 0) */
  uint64_t seed;    /* visit order */
} pdqp_ws_train_options;

/* Create a network for problems with n variables and m rows: projection width
 * d, `depth` hidden layers of `width` units (d and width multiples of 8), and
 * at most max_batch rows per forward pass (multiple of 8, <= 8192).  All
 * parameters start at zero; set them with pdqp_ws_set_params. */
pdqp_status pdqp_ws_create(pdqp_ws_handle *out, int64_t n, int64_t m, int32_t d, int32_t width, int32_t depth,
                           int32_t max_batch, void *stream);

void pdqp_ws_destroy(pdqp_ws_handle w);

/* Description of the last error of w (or of the last failed create when w is NULL). */
const char *pdqp_ws_last_error(pdqp_ws_handle w);

/* Parameters of one layer, float32 in mem_space: layer -1 is the projection P
 * (W: d x F, b ignored), layers 0..depth-1 the hidden layers (W: width x in,
 * in = d for layer 0), layer depth the output layer (W: F x width).  b may be
 * NULL (zero bias).  Setting parameters keeps the Adam moments. */
pdqp_status pdqp_ws_set_params(pdqp_ws_handle w, int32_t layer, const float *W, const float *b, int32_t mem,
                               void *stream);

/* Read one layer's parameters (what = 0), last gradients (1), or Adam first
 * (2) / second (3) moments into W and/or b (either may be NULL). */
pdqp_status pdqp_ws_get_params(pdqp_ws_handle w, int32_t layer, int32_t what, float *W, float *b, int32_t mem,
                               void *stream);

/* Per-feature normalisation vectors, float32[F] each: inputs u = (v - in_mean)
 * * in_scale; targets t = (y - out_mean) * out_inv; predictions
 * out_mean + out_std * o. */
pdqp_status pdqp_ws_set_normalization(pdqp_ws_handle w, const float *in_mean, const float *in_scale,
                                      const float *out_mean, const float *out_std, const float *out_inv, int32_t mem,
                                      void *stream);
pdqp_status pdqp_ws_get_normalization(pdqp_ws_handle w, float *in_mean, float *in_scale, float *out_mean,
                                      float *out_std, float *out_inv, int32_t mem, void *stream);

/* Fit the normalisation to a training set: per-feature mean and population
 * standard deviation (float64, two passes; a deviation below 1e-8 counts as
 * 1), in_scale = 1/std_in, out_inv = 1/std_out. */
pdqp_status pdqp_ws_fit(pdqp_ws_handle w, const double *C, const double *B, const double *X, const double *Y,
                        int64_t count, int32_t mem, void *stream);

/* One forward and backward pass over `count` <= max_batch samples without an
 * update: the gradients of mean((o - t)^2) are left for pdqp_ws_get_params
 * (what = 1) and the loss is written to *loss (may be NULL). */
pdqp_status pdqp_ws_grad(pdqp_ws_handle w, const double *C, const double *B, const double *X, const double *Y,
                         int64_t count, double *loss, int32_t mem, void *stream);

/* Train on `count` samples (count >= batch): projects and normalises the
 * training set once, then runs opt->epochs epochs of minibatch Adam.  The
 * mean minibatch loss of each epoch goes to losses[epochs] (host, may be
 * NULL).  Adam's step counter continues across calls. */
pdqp_status pdqp_ws_train(pdqp_ws_handle w, const pdqp_ws_train_options *opt, const double *C, const double *B,
                          const double *X, const double *Y, int64_t count, double *losses, int32_t mem,
                          void *stream);

/* Predict warm starts X0 [count x n] and Y0 [count x m] (float64, either may be
 * NULL) for the family members (C, B). */
pdqp_status pdqp_ws_infer(pdqp_ws_handle w, const double *C, const double *B, int64_t count, double *X0,
                          double *Y0, int32_t mem, void *stream);

/* Tensor-core GEMM D = A B' on device arrays: A [M x K] and B [N x K] bf16
 * row-major with leading dimensions lda, ldb (multiples of 8, 16-byte aligned
 * bases), float32 accumulation, then per element (row, col):
 *   r += bias[col] (bias may be NULL); r = max(r, 0) if relu;
 *   r = 0 where mask[row * ldm + col] <= 0 (bf16, mask may be NULL);
 *   D_f32[row * ldd + col] = r and/or D_bf16[row * ldd + col] = bf16(r).
 * splits = 0 picks a split of K over blocks by itself when `workspace`
 * (device, workspace_bytes) has room for its float32 partials, else runs
 * unsplit; splits > 0 asks for that many (then the workspace must hold
 * pdqp_gemm_bf16_splits(M, N, K, splits) * M * N floats).  Asynchronous on
 * `stream`; a device-side wait that gave up is reported by the next
 * pdqp_gemm_bf16_check (which synchronises the stream and clears the flag). */
pdqp_status pdqp_gemm_bf16(int32_t M, int32_t N, int32_t K, const void *A, int32_t lda, const void *B, int32_t ldb,
                           const float *bias, int32_t relu, const void *mask, int32_t ldm, float *D_f32, void *D_bf16,
                           int32_t ldd, int32_t splits, float *workspace, int64_t workspace_bytes, void *stream);
pdqp_status pdqp_gemm_bf16_check(void *stream);

/* Diagnostic of the failure path: runs, in one thread, the bounded wait the
 * tensor-core kernels use on an mbarrier that nothing completes.  The wait
 * gives up after 0.2 s without progress and raises the error flag; the call
 * then returns what pdqp_gemm_bf16_check reads (PDQP_DEVICE_TIMEOUT, the flag
 * cleared; PDQP_ERR_CUDA if the launch failed).  Synchronises the stream.
 * No fault and no hang: the device stays usable. */
pdqp_status pdqp_gemm_bf16_wait_probe(void *stream);

/* The number of K splits pdqp_gemm_bf16 would use (0 on invalid sizes). */
int32_t pdqp_gemm_bf16_splits(int32_t M, int32_t N, int32_t K, int32_t splits);

#ifdef __cplusplus
}
#endif

#endif /* PDQP_WS_H */

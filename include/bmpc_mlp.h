/*
 * bmpc_mlp.h - C ABI of the learned warm start: a multilayer perceptron with BF16 weights and
 * activations and FP32 accumulation (tensor-core GEMMs), its training step (mean squared error,
 * back-propagation, AdamW) and the glue between BMPC batches and the network.
 *
 * The network maps features of a branch-MPC problem (initial state and per-scenario obstacle
 * predictions) to a starting point of the solver (state and control trees, dynamics multipliers
 * and AL multipliers); the solver then starts from it only when its merit is not above that of
 * the fallback start (bmpc_opts.warm_select).  This is an extension of the paper's method (which
 * warm-starts the AL iteration, Sec. IV), not one of its passages.
 *
 * All device memory is caller-owned.  Every width (layer in/out) and the batch size must be
 * multiples of 128; matrices are row-major; bf16 values are passed as uint16_t.  Functions return
 * 0 on success, -1 on a bad argument and -2 on a CUDA error; they are asynchronous on `stream`.
 */
#ifndef BMPC_MLP_H
#define BMPC_MLP_H

#include <stddef.h>
#include <stdint.h>

#include "bmpc.h"

#ifdef __cplusplus
extern "C" {
#endif

#define BMPC_MLP_MAX_LAYERS 8

typedef struct {
    int32_t in, out;            /* widths (multiples of 128) */
    uint16_t *w_bf16;           /* [in][out] bf16 copy used by the GEMMs */
    float *w, *w_m, *w_v;       /* [in][out] fp32 master weights and AdamW moments */
    float *b, *b_m, *b_v;       /* [out] bias and its moments */
    float *dw, *db;             /* gradients written by the training step */
} bmpc_mlp_layer;

typedef struct {
    uint16_t *pre[BMPC_MLP_MAX_LAYERS];   /* hidden layer l: pre-activation [batch][out_l] (bf16) */
    uint16_t *act[BMPC_MLP_MAX_LAYERS];   /* hidden layer l: GELU output [batch][out_l] (bf16) */
    uint16_t *dy0, *dy1;                   /* back-propagated gradients, [batch][widest layer] each */
    float *pred;                           /* network output [batch][out_last] (fp32) */
    float *loss;                           /* device scalar: mean squared error of the last step */
    float *splitk;                         /* split-K workspace (NULL: GEMMs are not split) */
    int64_t splitk_floats;                 /* its size, bmpc_mlp_workspace_floats for this batch */
} bmpc_mlp_work;

/* Weights uniform in [-1/sqrt(in), 1/sqrt(in)) from SplitMix64 of (seed, index); bias and moments 0. */
int bmpc_mlp_init(const bmpc_mlp_layer *layers, int32_t n_layers, uint64_t seed, void *stream);

/* pred = W_L^T ... GELU(W_1^T x + b_1) ... + b_L for a batch of bf16 inputs x [batch][in_1]. */
int bmpc_mlp_forward(const bmpc_mlp_layer *layers, int32_t n_layers, const uint16_t *x, int32_t batch,
                     const bmpc_mlp_work *work, void *stream);

/* One training step on (x, target [batch][out_L] bf16): forward, loss = mean (pred - target)^2,
 * back-propagation, AdamW (beta 0.9 / 0.999, eps 1e-8, decoupled weight decay on weights) with
 * bias correction for step `step` (>= 1). */
int bmpc_mlp_train_step(const bmpc_mlp_layer *layers, int32_t n_layers, const uint16_t *x, const uint16_t *target,
                        int32_t batch, float lr, float weight_decay, int32_t step, const bmpc_mlp_work *work,
                        void *stream);

/* C [M][N] (fp32) = op(A) op(B) with op(A) [M][K], op(B) [K][N]; trans_a: A stored [K][M]; trans_b:
 * B stored [N][K]; lda/ldb/ldc are row lengths of the stored matrices.  M and N must be multiples
 * of 128, K of 64 and the row lengths of 8 (else -1); runs on the tcgen05 tensor cores. */
int bmpc_mlp_gemm(const uint16_t *A, int32_t lda, int32_t trans_a, const uint16_t *B, int32_t ldb, int32_t trans_b,
                  float *C, int32_t ldc, int32_t M, int32_t N, int32_t K, void *stream);

/* Floats of split-K workspace the forward pass and training step need for this batch size: GEMMs
 * with fewer 128 x 128 output tiles than SMs and a long K (the hidden layers, the back-propagation
 * through the output layer) are split along K into partial products that a reduction kernel sums
 * in a fixed order, so results do not depend on the split.  0 when nothing splits, -1 on invalid
 * layers or batch. */
int64_t bmpc_mlp_workspace_floats(const bmpc_mlp_layer *layers, int32_t n_layers, int32_t batch);

/* Waits for `stream`, then reports whether a GEMM gave up waiting for its tensor-core MMAs since the
 * last call (each mbarrier wait is bounded at about 2 s): 0 none, BMPC_ERR_TIMEOUT (-4) one did
 * (its output tile was not written; the flag is cleared), BMPC_ERR_CUDA (-2) on a CUDA error. */
int bmpc_mlp_status(void *stream);

/* Test support for the bounded waits: a one-thread kernel waits for an mbarrier phase that nothing
 * completes, for at most `cycles` SM cycles (1 .. 1e8, about 50 ms at most), then records the
 * timeout exactly as a GEMM does, so that the next bmpc_mlp_status returns BMPC_ERR_TIMEOUT.
 * Nothing faults and the context stays usable.  -1 on cycles out of range, -2 if the launch fails;
 * asynchronous on `stream`. */
int bmpc_mlp_selftest_wait(int64_t cycles, void *stream);

/* ---- glue with a BMPC batch (all problems must share one tree) ----
 * Features of problem k (fp32, feat + k*dim): x0 without its X coordinate (nx - 1 values), then for
 * every scenario s < n_scen and obstacle o < n_obs_max the obstacle's (cx - X0, cy) at the middle
 * node of the scenario's path, (cx - X0, cy, heading) at its leaf (5 values; zeros when absent).
 * dim must be at least nx - 1 + 5 n_scen n_obs_max. */
int bmpc_mlp_features(const bmpc_batch *b, float *feat, int32_t dim, int32_t n_scen, int32_t n_obs_max);
/* Targets of problem k from the batch's current solution (fp32, tgt + k*stride): the packed start
 * x | u | lam | y (node-major) with X0 subtracted from every state's X.  y_sqrt = 1 writes the AL
 * multipliers as sqrt(y) (a variance-stabilising form: the heavy tail of the active keep-out rows'
 * multipliers is compressed and zeros stay zero), 0 as y.  -1 on y_sqrt outside {0, 1} or a stride
 * below a problem's packed size. */
int bmpc_mlp_targets(const bmpc_batch *b, float *tgt, int64_t stride, int32_t y_sqrt);
/* Packed warm starts from network outputs: start[k] = mean + std * pred[k] with X0 added back to
 * every state's X (the inverse of bmpc_mlp_targets after standardisation), the AL multipliers
 * clipped at 0 (and squared when y_sqrt = 1, the inverse of the targets' square-root form), then
 * the states replaced by the rollout of the predicted controls from x0 through the tree, so that
 * the start satisfies the dynamics; feed to bmpc_set_warm_start_device. */
int bmpc_mlp_start(const bmpc_batch *b, const float *pred, int64_t ld_pred, const float *mean, const float *std,
                   float *start, int64_t stride, int32_t y_sqrt);
/* out = bf16((raw - mean) / std) elementwise over rows x dim. */
int bmpc_mlp_standardize(const float *raw, const float *mean, const float *std, uint16_t *out, int64_t rows,
                         int32_t dim, void *stream);

#ifdef __cplusplus
}
#endif
#endif /* BMPC_MLP_H */

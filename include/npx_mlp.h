/* npx_mlp.h -- tensor-core kernels of the learned surrogate (part of libnpx.so).
 *
 * The surrogate is a multilayer perceptron that predicts a scene's next state from its current
 * state, actuator targets and contact flags.  The paper has no counterpart: it is a learned
 * stand-in for the plain step over windows of steps.  Its building block is a BF16 GEMM on the
 * 5th-generation tensor cores with FP32 accumulation:
 *
 *     C[M x N] = A[M x K] . B[N x K]^T        (A, B row-major, K contiguous: "both K-major")
 *
 * followed by a fused epilogue.  All pointers are DEVICE pointers; the call is asynchronous on
 * stream (a cudaStream_t).  Sizes: M a multiple of 128, N a multiple of 128 (tiles of 256 columns
 * when N is a multiple of 256), K a multiple of 64 * splits; A and B 16-byte aligned.  err is a
 * device int that the kernel sets non-zero if a tensor-core or copy barrier stalls for more than
 * two seconds (the kernel then frees its tensor memory and returns without writing C).
 */
#ifndef NPX_MLP_H
#define NPX_MLP_H

#include "npx.h"

#ifdef __cplusplus
extern "C" {
#endif

#define NPX_EPI_BIAS 0       /* y = acc + bias                                        */
#define NPX_EPI_BIAS_GELU 1  /* z = acc + bias (saved to zsave if set), y = gelu(z)    */
#define NPX_EPI_F32 2        /* outf[split] = acc (FP32 partial sums of split K)      */
#define NPX_EPI_DGELU 3      /* y = acc * gelu'(zin): backward through a GELU layer    */

/* Where the epilogue writes; every output is optional unless the mode needs it.
 *   out  [M x ldo] BF16 row-major;  outT [N x ldt] BF16 (the transpose of y);
 *   outf [M x ldf] FP32 row-major (for NPX_EPI_F32: split s at outf + s * split_stride);
 *   zsave [M x ldz] BF16 pre-activations (NPX_EPI_BIAS_GELU); zin [M x ldzi] BF16 (DGELU);
 *   bias [N] FP32 or NULL.
 * bias, out, zsave, zin and outf start on 16-byte boundaries and their row strides (ld * element
 * size, and split_stride * 4) are multiples of 16 bytes; outT is 2-byte aligned. */
typedef struct {
    int mode;
    const float *bias;
    void *out;
    int ldo;
    void *outT;
    int ldt;
    float *outf;
    int ldf;
    long long split_stride;
    void *zsave;
    int ldz;
    const void *zin;
    int ldzi;
} npx_gemm_epilogue;

int npx_gemm_bf16(const void *A, const void *B, int M, int N, int K, int splits,
                  const npx_gemm_epilogue *epilogue, int *err, void *stream);

/* The GEMM's bounded barrier wait on its own, for tests of its failure path: one thread waits on
 * a barrier that nothing completes, until the two-second limit (use_abort = 0) or until a second
 * warp raises the abort flag after 1 ms (use_abort = 1).  Synchronous: *timed_out (host) = 1 if
 * the wait gave up, *elapsed_us (host) = how long it waited; the context stays usable. */
int npx_gemm_wait_selftest(int use_abort, int *timed_out, int *elapsed_us, void *stream);

/* --- the surrogate network --------------------------------------------------------------
 * y = W_L gelu(... gelu(W_1 x + b_1) ...) + b_L with n_hidden_layers GELU layers of width
 * n_hidden (exact GELU, z Phi(z)), trained on the mean over the batch of the squared error summed
 * over outputs, with Adam.  Master weights, gradients and Adam moments are FP32; the GEMMs read
 * BF16 copies of the weights and BF16 activations and accumulate in FP32.  Inputs are zero-padded
 * to a multiple of 128 features and outputs to a multiple of 128 (the padding never reaches the
 * caller).  x, t, y below are DEVICE arrays, row-major, rows = samples; M (rows per call) must be
 * a multiple of 128 and at most max_batch.  Calls are asynchronous on the network's stream unless
 * they return host data. */
typedef struct npx_mlp npx_mlp;

typedef struct {
    int n_in, n_hidden, n_hidden_layers, n_out;
    int max_batch;
    float lr, beta1, beta2, eps;     /* Adam */
    unsigned long long seed;         /* He-normal initial weights, zero biases */
    void *stream;                    /* cudaStream_t; NULL = a stream the network creates */
} npx_mlp_desc;

int npx_mlp_create(const npx_mlp_desc *desc, npx_mlp **out);
int npx_mlp_destroy(npx_mlp *net);
/* Host FP32 parameters, layer by layer: W_l [n_out_l x n_in_l] row-major, b_l [n_out_l]
 * (unpadded sizes), concatenated in layer order (W_1, b_1, W_2, b_2, ...). */
int npx_mlp_params_set(npx_mlp *net, const float *params, size_t n);
int npx_mlp_params_get(npx_mlp *net, float *params, size_t n);
size_t npx_mlp_param_count(const npx_mlp *net);
/* y [M x n_out] = network(x [M x n_in]) */
int npx_mlp_forward(npx_mlp *net, const float *x, float *y, int M);
/* Gradients of the loss on (x, t) into the network's gradient buffers; *loss (device float)
 * receives the batch loss. */
int npx_mlp_backward(npx_mlp *net, const float *x, const float *t, int M, float *loss);
/* Host FP32 copy of the last gradients, same layout as the parameters. */
int npx_mlp_grads_get(npx_mlp *net, float *grads, size_t n);
/* One Adam step with the last gradients. */
int npx_mlp_adam_step(npx_mlp *net);
/* Learning rate of the following Adam steps (a schedule sets it between steps); lr > 0. */
int npx_mlp_set_lr(npx_mlp *net, float lr);

/* --- the surrogate step -----------------------------------------------------------------
 * For worlds whose scenes all have the same number of links NL (NL - 1 joints) and NS contact-
 * sensor bits, a scene's features are, per link: the CoG of the link's points (x, y relative to a
 * horizontal reference, z absolute), the link's orientation quaternion, the velocity of its CoG
 * and the angular velocity (13 numbers), then the NL - 1 joint angles after the current step's
 * joint update and the NS contact bits of the last step: n_features = 14 NL - 1 + NS (271 for
 * the 18-DoF six-sensor hexapod).  The target of a transition is the change of the link part
 * over one window of `stride` steps (n_targets = 13 NL), positions taken relative to the first
 * state's CoG.  A window never holds a joint-update step (n % K == 0): on actuated worlds a
 * window starts at a step n with 1 <= n % K and n % K + stride <= K, so joint-update steps and
 * the (K - 1) mod stride steps left over before them are plain steps.
 * Standardisation (all DEVICE arrays, NULL = raw values): features (x - x_mu) * x_isd, targets
 * (d - t_mu) / t_sd. */
typedef struct {
    const float *x_mu, *x_isd, *t_mu, *t_sd;
} npx_surrogate_norm;

int npx_surrogate_dims(npx_world *w, int *n_features, int *n_targets);
/* Advance the world with the plain step until n_windows windows of `stride` steps (1 <= stride
 * < K on actuated worlds) have been recorded, writing each window's features X (at its first
 * step) and targets T (DEVICE, rows = window * n_scenes + scene, standardised when norm is
 * given).  Steps outside windows are stepped but not recorded.  Worlds with arenas
 * (npx_world_set_arenas) are refused with NPX_EINVAL: the features describe robots alone. */
int npx_surrogate_collect(npx_world *w, const npx_surrogate_norm *norm, int stride, int n_windows,
                          float *X, float *T);
/* Advance the world n_steps steps with the surrogate: at each window start the network predicts
 * every scene's state `stride` steps later from its features; scenes whose contact sensors at
 * the predicted state differ from those at the window's start in more bits than the world's
 * fallback threshold (npx_surrogate_set_fallback; 0 by default: any change) redo the window with
 * the plain step (the fallback); steps outside windows, and a last window that does not fit in n_steps, are
 * plain for every scene.  *fallbacks (host, may be NULL) receives the number of scene-steps that
 * fell back.  The network must have been trained on windows of the same stride, take n_features
 * inputs, give n_targets outputs, and hold at least n_scenes rounded up to 128 rows.  Worlds
 * with arenas are refused (NPX_EINVAL). */
int npx_world_step_surrogate(npx_world *w, npx_mlp *net, const npx_surrogate_norm *norm, int stride,
                             int n_steps, long long *fallbacks);
/* Per-scene fallback windows: counts[s] (HOST, n_scenes ints) receives how many of scene s's
 * surrogate windows fell back to the plain step since the previous call (or since the world's
 * first surrogate call), and the counters restart at zero.  Synchronises the world's stream.
 * This is how a caller tells the scenes that stayed on the network from those the plain step
 * took over, e.g. to state the network's own error apart from the plain step's. */
int npx_surrogate_fallback_counts(npx_world *w, int *counts);
/* The fallback rule of npx_world_step_surrogate: a window falls back when more than
 * max_changed_bits of the scene's contact sensors differ between the window's start and the
 * predicted state.  0 (the default) falls back on any change; -1 never falls back (every window
 * keeps the network's prediction, and its sensors are those read at the predicted state).  A
 * looser rule trades the 50-step state error for throughput; the paper has no counterpart (the
 * surrogate is not part of it).  Values below -1 are refused with NPX_EINVAL. */
int npx_surrogate_set_fallback(npx_world *w, int max_changed_bits);

/* FP64 column statistics of FP32 rows: for X [rows x cols] (DEVICE, row-major), adds the sum and
 * the sum of squares of every column to sum[cols] and sumsq[cols] (DEVICE, FP64; the caller
 * zeroes them first).  Each column is summed in a fixed order, so results repeat bit for bit.
 * Asynchronous on stream (a cudaStream_t).  The surrogate's standardisation statistics and the
 * zero-predictor loss of training rows use it. */
int npx_column_moments(const float *X, long long rows, int cols, double *sum, double *sumsq, void *stream);

#ifdef __cplusplus
}
#endif
#endif

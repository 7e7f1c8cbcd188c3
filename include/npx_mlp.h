/* npx_mlp.h -- tensor-core kernels of the learned surrogate (part of libnpx.so).
 *
 * The surrogate is a multilayer perceptron that predicts a scene's next state from its current
 * state, actuator targets and contact flags.  The paper has no counterpart (it is the batched
 * extension the task asks for beside the plain step).  Its building block is a BF16 GEMM on the
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
 *   bias [N] FP32 or NULL. */
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

#ifdef __cplusplus
}
#endif
#endif

// npx_mlp.cu -- the learned surrogate's network on the tensor cores: forward, backward and Adam.
//
// Layers are GEMMs of npx_gemm.cu with fused epilogues: hidden layers write the pre-activation z
// (kept for the backward pass), the activation gelu(z) and its transpose (the B operand of the
// weight-gradient GEMM); the output layer writes FP32.  Backward: dY = 2 (y - t) / M, then for
// each layer dW = dZ^T X (split-K GEMM over the batch, partial sums reduced in FP32),
// db = column sums of dZ, and dZ_prev = (dZ W) * gelu'(z_prev) (GEMM with the GELU' epilogue,
// also writing its transpose).  Adam updates FP32 master weights and refreshes the BF16 copies
// W and W^T that the GEMMs read.
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include <cmath>
#include <cstdio>
#include <random>
#include <string>
#include <vector>

#include "../../include/npx_mlp.h"
#include "npx_internal.h"

typedef __nv_bfloat16 bf16;

namespace {

int pad_to(int n, int m) { return (n + m - 1) / m * m; }

// Tiles of 32 x 32 elements go through shared memory so that both the row-major output and its
// transpose are written in full lines: block (32, 8), grid (cols / 32, rows / 32).

// X = bf16(x) zero-padded to in_p columns, and optionally X^T [in_p x M]
__global__ void __launch_bounds__(256) pack_input_kernel(const float *__restrict__ x, int M, int n_in, int in_p,
                                                         bf16 *X, bf16 *XT) {
    __shared__ bf16 tile[32][33];
    const int k0 = blockIdx.x * 32, m0 = blockIdx.y * 32, tx = threadIdx.x, ty = threadIdx.y;
#pragma unroll
    for (int i = 0; i < 4; ++i) {
        const int m = m0 + ty + 8 * i, k = k0 + tx;
        const bf16 v = __float2bfloat16_rn(k < n_in ? x[(size_t)m * n_in + k] : 0.f);
        X[(size_t)m * in_p + k] = v;
        tile[ty + 8 * i][tx] = v;
    }
    if (!XT) return;   // block-uniform
    __syncthreads();
#pragma unroll
    for (int i = 0; i < 4; ++i) XT[(size_t)(k0 + ty + 8 * i) * M + m0 + tx] = tile[tx][ty + 8 * i];
}

// dY = 2 (y - t) / M on real outputs, 0 on the padding, and dY^T; loss += sum (y - t)^2 / M
__global__ void __launch_bounds__(256) loss_grad_kernel(const float *__restrict__ Y, const float *__restrict__ T,
                                                        int M, int n_out, int out_p, bf16 *dY, bf16 *dYT,
                                                        float *loss) {
    __shared__ bf16 tile[32][33];
    __shared__ float red[8];
    const int j0 = blockIdx.x * 32, m0 = blockIdx.y * 32, tx = threadIdx.x, ty = threadIdx.y;
    const float inv = 1.f / (float)M;
    float sq = 0.f;
#pragma unroll
    for (int i = 0; i < 4; ++i) {
        const int m = m0 + ty + 8 * i, j = j0 + tx;
        const float d = j < n_out ? Y[(size_t)m * out_p + j] - T[(size_t)m * n_out + j] : 0.f;
        sq += d * d * inv;
        const bf16 g = __float2bfloat16_rn(2.f * d * inv);
        dY[(size_t)m * out_p + j] = g;
        tile[ty + 8 * i][tx] = g;
    }
    __syncthreads();
#pragma unroll
    for (int i = 0; i < 4; ++i) dYT[(size_t)(j0 + ty + 8 * i) * M + m0 + tx] = tile[tx][ty + 8 * i];
    for (int o = 16; o > 0; o >>= 1) sq += __shfl_xor_sync(0xffffffffu, sq, o);
    if (tx == 0) red[ty] = sq;
    __syncthreads();
    if (ty == 0 && tx == 0) {
        float t = 0.f;
        for (int i = 0; i < 8; ++i) t += red[i];
        if (t != 0.f) atomicAdd(loss, t);
    }
}

// out[n] = sum over the M entries of row n of GT [N x M] (the bias gradient: column sums of the
// layer's output gradient, read from its transpose so that every load is a full line)
__global__ void __launch_bounds__(256) rowsum_kernel(const bf16 *__restrict__ GT, int M, float *out) {
    __shared__ float red[8];
    const bf16 *row = GT + (size_t)blockIdx.x * M;
    float s = 0.f;
    for (int m = threadIdx.x * 8; m < M; m += 256 * 8) {
        const uint4 u = *reinterpret_cast<const uint4 *>(row + m);
        const __nv_bfloat162 *h = reinterpret_cast<const __nv_bfloat162 *>(&u);
#pragma unroll
        for (int k = 0; k < 4; ++k) {
            const float2 f = __bfloat1622float2(h[k]);
            s += f.x + f.y;
        }
    }
    for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = s;
    __syncthreads();
    if (threadIdx.x == 0) {
        float t = 0.f;
        for (int i = 0; i < 8; ++i) t += red[i];
        out[blockIdx.x] = t;
    }
}

__global__ void splitk_reduce_kernel(const float *__restrict__ part, int splits, long long n, float *out) {
    const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    float s = 0.f;
    for (int k = 0; k < splits; ++k) s += part[(size_t)k * n + i];
    out[i] = s;
}

// Adam on FP32 master parameters [rows x cols]; refreshes the BF16 copy and its transpose
__global__ void adam_kernel(float *p, const float *g, float *m, float *v, long long n, int cols, float lr,
                            float b1, float b2, float eps, float bc1, float bc2, bf16 *pb, bf16 *pbT, int rows) {
    const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const float gi = g[i];
    const float mi = b1 * m[i] + (1.f - b1) * gi;
    const float vi = b2 * v[i] + (1.f - b2) * gi * gi;
    m[i] = mi;
    v[i] = vi;
    const float pi = p[i] - lr * (mi / bc1) / (sqrtf(vi / bc2) + eps);
    p[i] = pi;
    if (pb) {
        const bf16 b = __float2bfloat16_rn(pi);
        pb[i] = b;
        pbT[(size_t)(i % cols) * rows + (i / cols)] = b;
    }
}

__global__ void to_bf16_kernel(const float *p, long long n, int cols, int rows, bf16 *pb, bf16 *pbT) {
    const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const bf16 b = __float2bfloat16_rn(p[i]);
    pb[i] = b;
    pbT[(size_t)(i % cols) * rows + (i / cols)] = b;
}

__global__ void unpad_kernel(const float *__restrict__ Y, int M, int out_p, int n_out, float *y) {
    const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= (long long)M * n_out) return;
    const int m = (int)(i / n_out), j = (int)(i % n_out);
    y[i] = Y[(size_t)m * out_p + j];
}

inline unsigned blocks_for(long long n, int t = 256) { return (unsigned)((n + t - 1) / t); }

// Column sums and sums of squares in FP64: block x covers 32 columns; thread (tx, ty) sums column
// 32 x + tx over rows ty, ty + 32, ... (in that order), then thread ty = 0 adds the 32 partial sums
// in ty order.  Every column is summed in a fixed order by one block: deterministic, no atomics.
__global__ void __launch_bounds__(1024) column_moments_kernel(const float *__restrict__ X, long long rows, int cols,
                                                              double *sum, double *sumsq) {
    __shared__ double red[2][32][33];
    const int tx = threadIdx.x, ty = threadIdx.y, c = blockIdx.x * 32 + tx;
    double s = 0.0, q = 0.0;
    if (c < cols)
        for (long long r = ty; r < rows; r += 32) {
            const double v = (double)X[r * cols + c];
            s += v;
            q += v * v;
        }
    red[0][ty][tx] = s;
    red[1][ty][tx] = q;
    __syncthreads();
    if (ty == 0 && c < cols) {
        double ts = 0.0, tq = 0.0;
        for (int k = 0; k < 32; ++k) {
            ts += red[0][k][tx];
            tq += red[1][k][tx];
        }
        sum[c] += ts;
        sumsq[c] += tq;
    }
}

}  // namespace

struct npx_mlp {
    npx_mlp_desc d{};
    cudaStream_t stream = nullptr, own = nullptr;
    int L = 0;                                  // layers (hidden + output)
    std::vector<int> din, dout, rin, rout;      // padded and real widths per layer
    std::vector<float *> W, b, mW, vW, mb, vb, dW, db;
    std::vector<bf16 *> Wb, WbT;
    bf16 *X0 = nullptr, *X0T = nullptr, *dY = nullptr, *dYT = nullptr;
    std::vector<bf16 *> Z, X, XT, dZ, dZT;      // hidden layers
    float *Y = nullptr, *part = nullptr, *loss_tmp = nullptr;
    int *err = nullptr;
    size_t part_elems = 0;
    int t = 0;
    std::vector<void *> bufs;
};

namespace {

template <class T>
bool dalloc(npx_mlp *n, T **p, size_t count) {
    void *q = nullptr;
    if (cudaMalloc(&q, std::max<size_t>(count, 1) * sizeof(T)) != cudaSuccess) return false;
    cudaMemset(q, 0, std::max<size_t>(count, 1) * sizeof(T));
    n->bufs.push_back(q);
    *p = static_cast<T *>(q);
    return true;
}

int gemm(npx_mlp *n, const void *A, const void *B, int M, int N, int K, int splits, const npx_gemm_epilogue &ep) {
    return npx_gemm_bf16(A, B, M, N, K, splits, &ep, n->err, n->stream);
}

npx_gemm_epilogue epi(int mode) {
    npx_gemm_epilogue e{};
    e.mode = mode;
    return e;
}

int pick_splits(int Mg, int Ng, int K) {
    const int tiles = (Mg / 128) * (Ng / (Ng % 256 == 0 ? 256 : 128));
    int s = 1;
    while (s * 2 * tiles <= 152 && K % (64 * s * 2) == 0 && s < 64) s *= 2;
    return s;
}

int check(npx_mlp *n, int M) {
    if (!n) return npx::set_last_error(NPX_EINVAL, "null network");
    if (M < 128 || M % 128 || M > n->d.max_batch)
        return npx::set_last_error(NPX_EINVAL, "M must be a multiple of 128 and at most max_batch");
    return NPX_OK;
}

#define CU(call)                                                                                 \
    do {                                                                                         \
        cudaError_t e_ = (call);                                                                 \
        if (e_ != cudaSuccess) return npx::set_last_error(NPX_ECUDA, cudaGetErrorString(e_));    \
    } while (0)
#define RC(call)                    \
    do {                            \
        int r_ = (call);            \
        if (r_) return r_;          \
    } while (0)

// the layers, from the packed BF16 input X0
int forward_layers(npx_mlp *n, int M, bool train) {
    const bf16 *A = n->X0;
    for (int l = 0; l < n->L - 1; ++l) {
        npx_gemm_epilogue e = epi(NPX_EPI_BIAS_GELU);
        e.bias = n->b[l];
        e.out = n->X[l];
        e.ldo = n->dout[l];
        if (train) {
            e.zsave = n->Z[l];
            e.ldz = n->dout[l];
            e.outT = n->XT[l];
            e.ldt = M;
        }
        RC(gemm(n, A, n->Wb[l], M, n->dout[l], n->din[l], 1, e));
        A = n->X[l];
    }
    const int l = n->L - 1;
    npx_gemm_epilogue e = epi(NPX_EPI_BIAS);
    e.bias = n->b[l];
    e.outf = n->Y;
    e.ldf = n->dout[l];
    RC(gemm(n, A, n->Wb[l], M, n->dout[l], n->din[l], 1, e));
    return NPX_OK;
}

int forward_impl(npx_mlp *n, const float *x, int M, bool train) {
    const int in_p = n->din[0];
    pack_input_kernel<<<dim3(in_p / 32, M / 32), dim3(32, 8), 0, n->stream>>>(x, M, n->d.n_in, in_p, n->X0,
                                                                             train ? n->X0T : nullptr);
    CU(cudaGetLastError());
    return forward_layers(n, M, train);
}

}  // namespace

cudaStream_t npx::mlp_stream(const npx_mlp *n) { return n->stream; }
int npx::mlp_max_batch(const npx_mlp *n) { return n->d.max_batch; }
void npx::mlp_dims(const npx_mlp *n, int *n_in, int *n_out) {
    *n_in = n->d.n_in;
    *n_out = n->d.n_out;
}
__nv_bfloat16 *npx::mlp_input(npx_mlp *n, int *ld) {
    *ld = n->din[0];
    return n->X0;
}
int npx::mlp_forward_packed(npx_mlp *n, int M) {
    RC(check(n, M));
    return forward_layers(n, M, false);
}
const float *npx::mlp_output(const npx_mlp *n, int *ld) {
    *ld = n->dout[n->L - 1];
    return n->Y;
}

extern "C" {

int npx_mlp_create(const npx_mlp_desc *d, npx_mlp **out) {
    if (!d || !out) return npx::set_last_error(NPX_EINVAL, "null argument");
    *out = nullptr;
    if (d->n_in < 1 || d->n_out < 1 || d->n_hidden < 128 || d->n_hidden % 128 || d->n_hidden_layers < 1 ||
        d->max_batch < 128 || d->max_batch % 128)
        return npx::set_last_error(NPX_EINVAL, "bad network sizes (hidden width and max_batch multiples of 128)");
    npx_mlp *n = new (std::nothrow) npx_mlp();
    if (!n) return npx::set_last_error(NPX_ENOMEM, "out of host memory");
    n->d = *d;
    n->stream = static_cast<cudaStream_t>(d->stream);
    if (!n->stream) {
        if (cudaStreamCreateWithFlags(&n->own, cudaStreamNonBlocking) != cudaSuccess) {
            delete n;
            return npx::set_last_error(NPX_ECUDA, "stream creation failed");
        }
        n->stream = n->own;
    }
    n->L = d->n_hidden_layers + 1;
    const int H = d->n_hidden, Mx = d->max_batch;
    for (int l = 0; l < n->L; ++l) {
        n->rin.push_back(l == 0 ? d->n_in : H);
        n->rout.push_back(l == n->L - 1 ? d->n_out : H);
        n->din.push_back(l == 0 ? pad_to(d->n_in, 128) : H);
        n->dout.push_back(l == n->L - 1 ? pad_to(d->n_out, 128) : H);
    }
    bool ok = true;
    n->W.resize(n->L); n->b.resize(n->L); n->mW.resize(n->L); n->vW.resize(n->L); n->mb.resize(n->L);
    n->vb.resize(n->L); n->dW.resize(n->L); n->db.resize(n->L); n->Wb.resize(n->L); n->WbT.resize(n->L);
    size_t max_w = 0;
    for (int l = 0; l < n->L && ok; ++l) {
        const size_t nw = (size_t)n->dout[l] * n->din[l];
        max_w = std::max(max_w, nw);
        ok = dalloc(n, &n->W[l], nw) && dalloc(n, &n->mW[l], nw) && dalloc(n, &n->vW[l], nw) &&
             dalloc(n, &n->dW[l], nw) && dalloc(n, &n->Wb[l], nw) && dalloc(n, &n->WbT[l], nw) &&
             dalloc(n, &n->b[l], n->dout[l]) && dalloc(n, &n->mb[l], n->dout[l]) &&
             dalloc(n, &n->vb[l], n->dout[l]) && dalloc(n, &n->db[l], n->dout[l]);
    }
    n->Z.resize(n->L - 1); n->X.resize(n->L - 1); n->XT.resize(n->L - 1); n->dZ.resize(n->L - 1); n->dZT.resize(n->L - 1);
    for (int l = 0; l < n->L - 1 && ok; ++l)
        ok = dalloc(n, &n->Z[l], (size_t)Mx * H) && dalloc(n, &n->X[l], (size_t)Mx * H) &&
             dalloc(n, &n->XT[l], (size_t)Mx * H) && dalloc(n, &n->dZ[l], (size_t)Mx * H) &&
             dalloc(n, &n->dZT[l], (size_t)Mx * H);
    n->part_elems = 64 * max_w;
    ok = ok && dalloc(n, &n->X0, (size_t)Mx * n->din[0]) && dalloc(n, &n->X0T, (size_t)Mx * n->din[0]) &&
         dalloc(n, &n->Y, (size_t)Mx * n->dout[n->L - 1]) && dalloc(n, &n->dY, (size_t)Mx * n->dout[n->L - 1]) &&
         dalloc(n, &n->dYT, (size_t)Mx * n->dout[n->L - 1]) && dalloc(n, &n->part, n->part_elems) &&
         dalloc(n, &n->err, 1) && dalloc(n, &n->loss_tmp, 1);
    if (!ok) {
        npx_mlp_destroy(n);
        return npx::set_last_error(NPX_ENOMEM, "device allocation failed");
    }
    // He-normal initial weights (std sqrt(2 / fan_in)), zero biases
    std::mt19937_64 rng(d->seed);
    std::vector<float> host;
    for (int l = 0; l < n->L; ++l) {
        host.assign((size_t)n->dout[l] * n->din[l], 0.f);
        std::normal_distribution<float> nd(0.f, std::sqrt(2.f / n->rin[l]));
        for (int o = 0; o < n->rout[l]; ++o)
            for (int i = 0; i < n->rin[l]; ++i) host[(size_t)o * n->din[l] + i] = nd(rng);
        CU(cudaMemcpy(n->W[l], host.data(), host.size() * sizeof(float), cudaMemcpyHostToDevice));
        to_bf16_kernel<<<blocks_for((long long)host.size()), 256, 0, n->stream>>>(
            n->W[l], (long long)host.size(), n->din[l], n->dout[l], n->Wb[l], n->WbT[l]);
    }
    CU(cudaStreamSynchronize(n->stream));
    *out = n;
    return NPX_OK;
}

int npx_mlp_destroy(npx_mlp *n) {
    if (!n) return NPX_OK;
    if (n->stream) cudaStreamSynchronize(n->stream);
    for (void *p : n->bufs) cudaFree(p);
    if (n->own) cudaStreamDestroy(n->own);
    delete n;
    return NPX_OK;
}

size_t npx_mlp_param_count(const npx_mlp *n) {
    if (!n) return 0;
    size_t c = 0;
    for (int l = 0; l < n->L; ++l) c += (size_t)n->rout[l] * n->rin[l] + n->rout[l];
    return c;
}

static int copy_params(npx_mlp *n, float *host, size_t count, bool to_device, bool grads) {
    if (!n || !host) return npx::set_last_error(NPX_EINVAL, "null argument");
    if (count != npx_mlp_param_count(n)) return npx::set_last_error(NPX_EINVAL, "parameter count mismatch");
    CU(cudaStreamSynchronize(n->stream));
    int err = 0;
    CU(cudaMemcpy(&err, n->err, sizeof err, cudaMemcpyDeviceToHost));
    if (err) return npx::set_last_error(NPX_ETIMEOUT, "a tensor-core GEMM barrier timed out");
    size_t off = 0;
    for (int l = 0; l < n->L; ++l) {
        float *Wd = grads ? n->dW[l] : n->W[l];
        float *bd = grads ? n->db[l] : n->b[l];
        // rows of W are padded to din[l] columns: copy row by row with a 2D copy
        const size_t sp = (size_t)n->din[l] * sizeof(float), hp = (size_t)n->rin[l] * sizeof(float);
        if (to_device)
            CU(cudaMemcpy2D(Wd, sp, host + off, hp, hp, n->rout[l], cudaMemcpyHostToDevice));
        else
            CU(cudaMemcpy2D(host + off, hp, Wd, sp, hp, n->rout[l], cudaMemcpyDeviceToHost));
        off += (size_t)n->rout[l] * n->rin[l];
        if (to_device)
            CU(cudaMemcpy(bd, host + off, n->rout[l] * sizeof(float), cudaMemcpyHostToDevice));
        else
            CU(cudaMemcpy(host + off, bd, n->rout[l] * sizeof(float), cudaMemcpyDeviceToHost));
        off += n->rout[l];
        if (to_device && !grads) {
            const long long nw = (long long)n->dout[l] * n->din[l];
            to_bf16_kernel<<<blocks_for(nw), 256, 0, n->stream>>>(n->W[l], nw, n->din[l], n->dout[l], n->Wb[l],
                                                                  n->WbT[l]);
            CU(cudaGetLastError());
        }
    }
    CU(cudaStreamSynchronize(n->stream));
    return NPX_OK;
}

int npx_mlp_params_set(npx_mlp *n, const float *p, size_t c) { return copy_params(n, const_cast<float *>(p), c, true, false); }
int npx_mlp_params_get(npx_mlp *n, float *p, size_t c) { return copy_params(n, p, c, false, false); }
int npx_mlp_grads_get(npx_mlp *n, float *g, size_t c) { return copy_params(n, g, c, false, true); }

int npx_mlp_forward(npx_mlp *n, const float *x, float *y, int M) {
    RC(check(n, M));
    if (!x || !y) return npx::set_last_error(NPX_EINVAL, "null array");
    RC(forward_impl(n, x, M, false));
    const int out_p = n->dout[n->L - 1];
    unpad_kernel<<<blocks_for((long long)M * n->d.n_out), 256, 0, n->stream>>>(n->Y, M, out_p, n->d.n_out, y);
    CU(cudaGetLastError());
    return NPX_OK;
}

int npx_mlp_backward(npx_mlp *n, const float *x, const float *t, int M, float *loss) {
    RC(check(n, M));
    if (!x || !t || !loss) return npx::set_last_error(NPX_EINVAL, "null array");
    RC(forward_impl(n, x, M, true));
    const int L = n->L, H = n->d.n_hidden, out_p = n->dout[L - 1];
    CU(cudaMemsetAsync(loss, 0, sizeof(float), n->stream));
    loss_grad_kernel<<<dim3(out_p / 32, M / 32), dim3(32, 8), 0, n->stream>>>(n->Y, t, M, n->d.n_out, out_p, n->dY,
                                                                              n->dYT, loss);
    CU(cudaGetLastError());
    const bf16 *G = n->dY, *GT = n->dYT;     // gradient of the current layer's output
    for (int l = L - 1; l >= 0; --l) {
        const int No = n->dout[l], Ni = n->din[l];
        // dW = G^T X_prev: A = G^T [No x M], B = X_prev^T [Ni x M]
        const bf16 *XprevT = l > 0 ? n->XT[l - 1] : n->X0T;
        const int splits = pick_splits(No, Ni, M);
        npx_gemm_epilogue e = epi(NPX_EPI_F32);
        e.outf = n->part;
        e.ldf = Ni;
        e.split_stride = (long long)No * Ni;
        RC(gemm(n, GT, XprevT, No, Ni, M, splits, e));
        splitk_reduce_kernel<<<blocks_for((long long)No * Ni), 256, 0, n->stream>>>(n->part, splits, (long long)No * Ni,
                                                                                   n->dW[l]);
        rowsum_kernel<<<No, 256, 0, n->stream>>>(GT, M, n->db[l]);
        CU(cudaGetLastError());
        if (l > 0) {
            // dZ_prev = (G W) * gelu'(Z_prev): A = G [M x No], B = W^T [Ni x No]
            npx_gemm_epilogue e2 = epi(NPX_EPI_DGELU);
            e2.zin = n->Z[l - 1];
            e2.ldzi = H;
            e2.out = n->dZ[l - 1];
            e2.ldo = H;
            e2.outT = n->dZT[l - 1];
            e2.ldt = M;
            RC(gemm(n, G, n->WbT[l], M, Ni, No, 1, e2));
            G = n->dZ[l - 1];
            GT = n->dZT[l - 1];
        }
    }
    return NPX_OK;
}

int npx_column_moments(const float *X, long long rows, int cols, double *sum, double *sumsq, void *stream) {
    if (!X || !sum || !sumsq || rows < 0 || cols < 1) return npx::set_last_error(NPX_EINVAL, "npx_column_moments: bad arguments");
    if (rows == 0) return NPX_OK;
    column_moments_kernel<<<(cols + 31) / 32, dim3(32, 32), 0, static_cast<cudaStream_t>(stream)>>>(X, rows, cols, sum,
                                                                                                  sumsq);
    CU(cudaGetLastError());
    return NPX_OK;
}

int npx_mlp_adam_step(npx_mlp *n) {
    if (!n) return npx::set_last_error(NPX_EINVAL, "null network");
    n->t += 1;
    const float b1 = n->d.beta1, b2 = n->d.beta2;
    const float bc1 = 1.f - std::pow(b1, (float)n->t), bc2 = 1.f - std::pow(b2, (float)n->t);
    for (int l = 0; l < n->L; ++l) {
        const long long nw = (long long)n->dout[l] * n->din[l];
        adam_kernel<<<blocks_for(nw), 256, 0, n->stream>>>(n->W[l], n->dW[l], n->mW[l], n->vW[l], nw, n->din[l],
                                                          n->d.lr, b1, b2, n->d.eps, bc1, bc2, n->Wb[l], n->WbT[l],
                                                          n->dout[l]);
        adam_kernel<<<blocks_for(n->dout[l]), 256, 0, n->stream>>>(n->b[l], n->db[l], n->mb[l], n->vb[l], n->dout[l],
                                                                   1, n->d.lr, b1, b2, n->d.eps, bc1, bc2, nullptr,
                                                                   nullptr, 1);
    }
    CU(cudaGetLastError());
    return NPX_OK;
}

int npx_mlp_set_lr(npx_mlp *n, float lr) {
    if (!n) return npx::set_last_error(NPX_EINVAL, "null network");
    if (!(lr > 0.f) || !std::isfinite(lr)) return npx::set_last_error(NPX_EINVAL, "learning rate must be positive");
    n->d.lr = lr;
    return NPX_OK;
}

}  // extern "C"

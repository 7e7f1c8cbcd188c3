// npx_gemm.cu -- BF16 GEMM on the 5th-generation tensor cores (tcgen05 / TMEM / TMA, sm_103a)
// for the learned surrogate: C[M x N] = A[M x K] . B[N x K]^T, both operands K-major (row-major
// with K contiguous), FP32 accumulation in tensor memory, fused epilogues.
//
// One CTA computes a 128 x BN tile.  Thread 0 streams 128 x 64 and BN x 64 operand tiles with TMA
// (128-byte swizzle, the layout the UMMA shared-memory descriptors describe) through a STAGES-deep
// ring of shared-memory buffers and issues one tcgen05.mma (M = 128, N = BN, K = 16) per 32-byte
// step of each 64-wide K block; tcgen05.commit on an mbarrier hands each buffer back to the TMA.
// The four warps then read the accumulator out of tensor memory (warp w owns rows 32w .. 32w+31)
// and apply the epilogue.  Every wait is bounded: a stalled barrier sets an error flag, the
// kernel drains the copies it started, frees its tensor memory and returns.
#include <cuda.h>
#include <cuda_bf16.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include "../../include/npx_mlp.h"
#include "npx_internal.h"

namespace npx {
namespace gemm {

constexpr int BM = 128, BK = 64, STAGES = 4, THREADS = 128;
constexpr unsigned long long WAIT_NS = 2000000000ull;   // 2 s per barrier wait

__device__ __forceinline__ uint32_t smem_u32(const void *p) {
    return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

__device__ __forceinline__ unsigned long long global_ns() {
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

__device__ __forceinline__ void mbar_init(uint64_t *b, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(b)), "r"(count) : "memory");
}

__device__ __forceinline__ void mbar_expect_tx(uint64_t *b, uint32_t bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(b)), "r"(bytes)
                 : "memory");
}

__device__ __forceinline__ bool mbar_try_wait(uint64_t *b, uint32_t parity) {
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(ok)
        : "r"(smem_u32(b)), "r"(parity)
        : "memory");
    return ok != 0;
}

// bounded wait: false after WAIT_NS without the phase completing
__device__ __forceinline__ bool mbar_wait(uint64_t *b, uint32_t parity) {
    if (mbar_try_wait(b, parity)) return true;
    const unsigned long long t0 = global_ns();
    while (!mbar_try_wait(b, parity))
        if (global_ns() - t0 > WAIT_NS) return false;
    return true;
}

__device__ __forceinline__ void tma_load_2d(void *dst, const CUtensorMap *map, int x, int y, uint64_t *bar) {
    asm volatile(
        "cp.async.bulk.tensor.2d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3}], [%4];"
        ::"r"(smem_u32(dst)), "l"(reinterpret_cast<uint64_t>(map)), "r"(x), "r"(y), "r"(smem_u32(bar))
        : "memory");
}

// UMMA shared-memory descriptor of a K-major operand tile in the 128-byte swizzled layout:
// rows of 128 bytes (64 BF16 along K), 8-row groups 1024 bytes apart (stride byte offset),
// descriptor version 1, swizzle mode 2 (128 B).  The leading byte offset is unused here.
__device__ __forceinline__ uint64_t sdesc_k_sw128(uint32_t saddr) {
    uint64_t d = 0;
    d |= (uint64_t)((saddr & 0x3FFFFu) >> 4);
    d |= (uint64_t)1 << 16;
    d |= (uint64_t)(1024 >> 4) << 32;
    d |= (uint64_t)1 << 46;
    d |= (uint64_t)2 << 61;
    return d;
}

// instruction descriptor of kind::f16: FP32 accumulator, BF16 A and B, both K-major, M x N
__host__ __device__ constexpr uint32_t idesc_bf16(int M, int N) {
    return (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(N >> 3) << 17) | ((uint32_t)(M >> 4) << 24);
}

__device__ __forceinline__ void umma_bf16(uint32_t tmem_d, uint64_t a, uint64_t b, uint32_t idesc,
                                          uint32_t accumulate) {
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "setp.ne.b32 p, %4, 0;\n\t"
        "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}"
        ::"r"(tmem_d), "l"(a), "l"(b), "r"(idesc), "r"(accumulate)
        : "memory");
}

__device__ __forceinline__ void umma_commit(uint64_t *bar) {
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(smem_u32(bar))
                 : "memory");
}

__device__ __forceinline__ void tc_fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void tc_fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }

__device__ __forceinline__ void tmem_ld16(uint32_t taddr, float (&v)[16]) {
    uint32_t r[16];
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
          "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
        : "r"(taddr)
        : "memory");
    asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
    for (int i = 0; i < 16; ++i) v[i] = __uint_as_float(r[i]);
}

__device__ __forceinline__ float gelu(float z) { return 0.5f * z * (1.f + erff(z * 0.70710678118654752f)); }
__device__ __forceinline__ float gelu_grad(float z) {
    return 0.5f * (1.f + erff(z * 0.70710678118654752f)) + z * 0.3989422804014327f * expf(-0.5f * z * z);
}

template <int BN>
__global__ void __launch_bounds__(THREADS, 1)
gemm_tn_kernel(const __grid_constant__ CUtensorMap ta, const __grid_constant__ CUtensorMap tb, int M, int N,
               int k_per_split, npx_gemm_epilogue ep, int *err) {
    extern __shared__ uint8_t smem_raw[];
    uint8_t *smem = reinterpret_cast<uint8_t *>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
    constexpr int A_BYTES = BM * BK * 2, B_BYTES = BN * BK * 2;
    uint8_t *sA = smem;
    uint8_t *sB = smem + STAGES * A_BYTES;
    uint64_t *full = reinterpret_cast<uint64_t *>(sB + STAGES * B_BYTES);
    uint64_t *empty = full + STAGES;
    uint64_t *done = empty + STAGES;
    uint32_t *tmem_slot = reinterpret_cast<uint32_t *>(done + 1);

    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int m0 = blockIdx.x * BM, n0 = blockIdx.y * BN;
    const int kbeg = blockIdx.z * k_per_split;
    const int nk = k_per_split / BK;

    if (warp == 0) {   // whole warp: allocate BN accumulator columns of tensor memory
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(tmem_slot)),
                     "r"((uint32_t)BN)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    if (threadIdx.x == 32) {
        for (int s = 0; s < STAGES; ++s) {
            mbar_init(&full[s], 1);
            mbar_init(&empty[s], 1);
        }
        mbar_init(done, 1);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = *tmem_slot;

    __shared__ int s_ok;
    if (threadIdx.x == 0) {
        const uint32_t idesc = idesc_bf16(BM, BN);
        bool ok = true;
        int issued = 0;   // k-blocks whose TMA was started
        auto issue = [&](int kb) {
            const int s = kb % STAGES;
            mbar_expect_tx(&full[s], A_BYTES + B_BYTES);
            tma_load_2d(sA + s * A_BYTES, &ta, kbeg + kb * BK, m0, &full[s]);
            tma_load_2d(sB + s * B_BYTES, &tb, kbeg + kb * BK, n0, &full[s]);
            ++issued;
        };
        for (int kb = 0; kb < nk && kb < STAGES; ++kb) issue(kb);
        int consumed = 0;
        for (int kb = 0; kb < nk; ++kb) {
            const int s = kb % STAGES;
            const uint32_t ph = (uint32_t)((kb / STAGES) & 1);
            if (!mbar_wait(&full[s], ph)) { ok = false; break; }
            ++consumed;
            tc_fence_after();
            const uint64_t da = sdesc_k_sw128(smem_u32(sA + s * A_BYTES));
            const uint64_t db = sdesc_k_sw128(smem_u32(sB + s * B_BYTES));
#pragma unroll
            for (int k = 0; k < BK / 16; ++k)   // 32 bytes along K per instruction
                umma_bf16(tmem, da + (uint64_t)(2 * k), db + (uint64_t)(2 * k), idesc, (kb | k) != 0);
            umma_commit(&empty[s]);
            if (kb + STAGES < nk) {
                if (!mbar_wait(&empty[s], ph)) { ok = false; break; }
                issue(kb + STAGES);
            }
        }
        umma_commit(done);
        if (!ok) {
            // drain the copies still in flight before the CTA's shared memory goes away
            for (int kb = consumed; kb < issued; ++kb) mbar_wait(&full[kb % STAGES], (uint32_t)((kb / STAGES) & 1));
            atomicExch(err, 1);
        }
        s_ok = ok ? 1 : 0;
    }
    __syncthreads();
    const bool fin = mbar_wait(done, 0);
    tc_fence_after();
    if (!fin) atomicExch(err, 2);
    if (fin && s_ok) {
        const int row = m0 + warp * 32 + lane;
        const uint32_t trow = tmem + ((uint32_t)(warp * 32) << 16);
        for (int c0 = 0; c0 < BN; c0 += 16) {
            float v[16];
            tmem_ld16(trow + (uint32_t)c0, v);
            const int col = n0 + c0;
            if (ep.mode == NPX_EPI_F32) {
                float *o = ep.outf + (size_t)blockIdx.z * ep.split_stride + (size_t)row * ep.ldf + col;
#pragma unroll
                for (int i = 0; i < 16; i += 4) *reinterpret_cast<float4 *>(o + i) = make_float4(v[i], v[i + 1], v[i + 2], v[i + 3]);
                continue;
            }
            if (ep.bias) {
#pragma unroll
                for (int i = 0; i < 16; ++i) v[i] += ep.bias[col + i];
            }
            if (ep.mode == NPX_EPI_BIAS_GELU) {
                if (ep.zsave) {
                    __nv_bfloat16 *z = static_cast<__nv_bfloat16 *>(ep.zsave) + (size_t)row * ep.ldz + col;
#pragma unroll
                    for (int i = 0; i < 16; i += 2) *reinterpret_cast<__nv_bfloat162 *>(z + i) = __floats2bfloat162_rn(v[i], v[i + 1]);
                }
#pragma unroll
                for (int i = 0; i < 16; ++i) v[i] = gelu(v[i]);
            } else if (ep.mode == NPX_EPI_DGELU) {
                const __nv_bfloat16 *z = static_cast<const __nv_bfloat16 *>(ep.zin) + (size_t)row * ep.ldzi + col;
#pragma unroll
                for (int i = 0; i < 16; ++i) v[i] *= gelu_grad(__bfloat162float(z[i]));
            }
            if (ep.outf) {
                float *o = ep.outf + (size_t)row * ep.ldf + col;
#pragma unroll
                for (int i = 0; i < 16; i += 4) *reinterpret_cast<float4 *>(o + i) = make_float4(v[i], v[i + 1], v[i + 2], v[i + 3]);
            }
            if (ep.out) {
                __nv_bfloat16 *o = static_cast<__nv_bfloat16 *>(ep.out) + (size_t)row * ep.ldo + col;
#pragma unroll
                for (int i = 0; i < 16; i += 2) *reinterpret_cast<__nv_bfloat162 *>(o + i) = __floats2bfloat162_rn(v[i], v[i + 1]);
            }
            if (ep.outT) {
#pragma unroll
                for (int i = 0; i < 16; ++i)
                    static_cast<__nv_bfloat16 *>(ep.outT)[(size_t)(col + i) * ep.ldt + row] = __float2bfloat16_rn(v[i]);
            }
        }
    }
    tc_fence_before();
    __syncthreads();
    if (warp == 0) {
        tc_fence_after();
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"((uint32_t)BN) : "memory");
    }
}

// ------------------------------------------------------------------------ host side

typedef CUresult (*EncodeTiledFn)(CUtensorMap *, CUtensorMapDataType, cuuint32_t, void *, const cuuint64_t *,
                                  const cuuint64_t *, const cuuint32_t *, const cuuint32_t *, CUtensorMapInterleave,
                                  CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

static EncodeTiledFn encode_fn() {
    static EncodeTiledFn fn = nullptr;
    if (!fn) {
        void *p = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) == cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            fn = reinterpret_cast<EncodeTiledFn>(p);
    }
    return fn;
}

// 2D map of a row-major [rows x cols] BF16 matrix read in boxes of box_rows x 64 (128 B rows)
static bool make_map(CUtensorMap *m, const void *ptr, int rows, int cols, int box_rows) {
    EncodeTiledFn fn = encode_fn();
    if (!fn) return false;
    const cuuint64_t dims[2] = {(cuuint64_t)cols, (cuuint64_t)rows};
    const cuuint64_t strides[1] = {(cuuint64_t)cols * 2};
    const cuuint32_t box[2] = {(cuuint32_t)BK, (cuuint32_t)box_rows};
    const cuuint32_t es[2] = {1, 1};
    return fn(m, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2, const_cast<void *>(ptr), dims, strides, box, es,
              CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
              CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

template <int BN>
static size_t smem_bytes() {
    return 1024 + (size_t)STAGES * (BM * BK * 2 + BN * BK * 2) + (2 * STAGES + 1) * 8 + 16;
}

template <int BN>
static cudaError_t launch(const CUtensorMap &ta, const CUtensorMap &tb, int M, int N, int K, int splits,
                          const npx_gemm_epilogue &ep, int *err, cudaStream_t st) {
    const size_t smem = smem_bytes<BN>();
    cudaError_t e = cudaFuncSetAttribute(gemm_tn_kernel<BN>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    dim3 grid(M / BM, N / BN, splits);
    gemm_tn_kernel<BN><<<grid, THREADS, smem, st>>>(ta, tb, M, N, K / splits, ep, err);
    return cudaGetLastError();
}

}  // namespace gemm
}  // namespace npx

extern "C" int npx_gemm_bf16(const void *A, const void *B, int M, int N, int K, int splits,
                             const npx_gemm_epilogue *ep, int *err, void *stream) {
    using namespace npx::gemm;
    if (!A || !B || !ep || !err) return npx::set_last_error(NPX_EINVAL, "npx_gemm_bf16: null argument");
    if (splits < 1) return npx::set_last_error(NPX_EINVAL, "npx_gemm_bf16: splits must be >= 1");
    const int BN = (N % 256 == 0) ? 256 : 128;
    if (M < BM || M % BM || N < 128 || N % 128 || K < BK || K % (BK * splits))
        return npx::set_last_error(NPX_EINVAL, "npx_gemm_bf16: M must be a multiple of 128, N of 128, K of 64 x splits");
    if ((reinterpret_cast<uintptr_t>(A) | reinterpret_cast<uintptr_t>(B)) & 15)
        return npx::set_last_error(NPX_EINVAL, "npx_gemm_bf16: A and B must be 16-byte aligned");
    if (ep->mode != NPX_EPI_BIAS && ep->mode != NPX_EPI_BIAS_GELU && ep->mode != NPX_EPI_DGELU && ep->mode != NPX_EPI_F32)
        return npx::set_last_error(NPX_EINVAL, "npx_gemm_bf16: unknown epilogue mode");
    if (ep->mode == NPX_EPI_F32 ? !ep->outf : (!ep->out && !ep->outT && !ep->outf))
        return npx::set_last_error(NPX_EINVAL, "npx_gemm_bf16: no output");
    if (ep->mode == NPX_EPI_DGELU && !ep->zin) return npx::set_last_error(NPX_EINVAL, "npx_gemm_bf16: DGELU needs zin");
    if (splits > 1 && ep->mode != NPX_EPI_F32) return npx::set_last_error(NPX_EINVAL, "npx_gemm_bf16: split K needs the F32 epilogue");
    CUtensorMap ta, tb;
    if (!make_map(&ta, A, M, K, BM) || !make_map(&tb, B, N, K, BN))
        return npx::set_last_error(NPX_ECUDA, "npx_gemm_bf16: tensor-map encoding failed");
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    cudaError_t e = BN == 256 ? launch<256>(ta, tb, M, N, K, splits, *ep, err, st)
                              : launch<128>(ta, tb, M, N, K, splits, *ep, err, st);
    if (e != cudaSuccess) return npx::set_last_error(NPX_ECUDA, cudaGetErrorString(e));
    return NPX_OK;
}

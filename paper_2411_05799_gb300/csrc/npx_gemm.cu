// npx_gemm.cu -- BF16 GEMM on the 5th-generation tensor cores (tcgen05 / TMEM / TMA, sm_103a)
// for the learned surrogate: C[M x N] = A[M x K] . B[N x K]^T, both operands K-major (row-major
// with K contiguous), FP32 accumulation in tensor memory, fused epilogues.
//
// A persistent, warp-specialised kernel: each CTA (one per SM) walks tiles of 128 x BN (and, for
// split K, one K range) in a static round-robin.  Warp 0 streams 128 x 64 and BN x 64 operand
// tiles with TMA (128-byte swizzle, the layout the UMMA shared-memory descriptors describe)
// through a STAGES-deep ring of shared-memory buffers; warp 1 issues one tcgen05.mma (M = 128,
// N = BN, K = 16) per 32-byte step of each 64-wide K block into one of two accumulators in tensor
// memory (2 x BN columns) and hands each ring buffer back with tcgen05.commit; sixteen epilogue warps
// read the other accumulator out (warp w owns TMEM lanes 32 (w % 4) .. + 31 and a quarter of
// the columns), apply the epilogue and release it, so a tile's epilogue overlaps the next tile's
// MMAs.  Every wait is bounded and also gives up once another role has failed: the failing role
// sets an error flag, the kernel drains the copies it started, waits for its MMAs, frees its
// tensor memory and returns.
#include <cuda.h>
#include <cuda_bf16.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include <cstring>

#include "../../include/npx_mlp.h"
#include "npx_internal.h"

namespace npx {
namespace gemm {

constexpr int BM = 128, BK = 64, STAGES = 4, EPI_WARPS = 16, THREADS = 32 * (2 + EPI_WARPS);
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

// bounded wait: false after WAIT_NS without the phase completing, or (when abort is given) as
// soon as another role has raised the abort flag
__device__ __forceinline__ bool mbar_wait(uint64_t *b, uint32_t parity, const volatile int *abort = nullptr) {
    if (mbar_try_wait(b, parity)) return true;
    const unsigned long long t0 = global_ns();
    while (!mbar_try_wait(b, parity)) {
        if (abort && *abort) return false;
        if (global_ns() - t0 > WAIT_NS) return false;
    }
    return true;
}

__device__ __forceinline__ void mbar_arrive(uint64_t *b) {
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(b)) : "memory");
}

__device__ __forceinline__ void tma_load_2d(void *dst, const CUtensorMap *map, int x, int y, uint64_t *bar) {
    asm volatile(
        "cp.async.bulk.tensor.2d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3}], [%4];"
        ::"r"(smem_u32(dst)), "l"(reinterpret_cast<uint64_t>(map)), "r"(x), "r"(y), "r"(smem_u32(bar))
        : "memory");
}

// TMA store of a box from shared memory (bulk group), its commit and waits
__device__ __forceinline__ void tma_store_2d(const CUtensorMap *map, int x, int y, const void *src) {
    asm volatile("cp.async.bulk.tensor.2d.global.shared::cta.bulk_group [%0, {%1, %2}], [%3];"
                 ::"l"(reinterpret_cast<uint64_t>(map)), "r"(x), "r"(y), "r"(smem_u32(src))
                 : "memory");
}
__device__ __forceinline__ void tma_store_3d(const CUtensorMap *map, int x, int y, int z, const void *src) {
    asm volatile("cp.async.bulk.tensor.3d.global.shared::cta.bulk_group [%0, {%1, %2, %3}], [%4];"
                 ::"l"(reinterpret_cast<uint64_t>(map)), "r"(x), "r"(y), "r"(z), "r"(smem_u32(src))
                 : "memory");
}
__device__ __forceinline__ void bulk_commit() { asm volatile("cp.async.bulk.commit_group;" ::: "memory"); }
template <int N>
__device__ __forceinline__ void bulk_wait_read() { asm volatile("cp.async.bulk.wait_group.read %0;" ::"n"(N) : "memory"); }
__device__ __forceinline__ void bulk_wait_all() { asm volatile("cp.async.bulk.wait_group 0;" ::: "memory"); }
__device__ __forceinline__ void fence_async_shared() { asm volatile("fence.proxy.async.shared::cta;" ::: "memory"); }

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

// 16 consecutive accumulator columns of this thread's TMEM lane; the values are valid after
// tmem_wait_ld
__device__ __forceinline__ void tmem_ld16_issue(uint32_t taddr, uint32_t (&r)[16]) {
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
          "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
        : "r"(taddr)
        : "memory");
}
__device__ __forceinline__ void tmem_wait_ld() { asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory"); }

// GELU in its tanh form, gelu(z) = z (1 + tanh(u)) / 2 with u = k (z + c z^3), k = sqrt(2 / pi),
// c = 0.044715, and its derivative (1 + t) / 2 + z (1 - t^2) k (1 + 3 c z^2) / 2, t = tanh(u).
// tanh comes from the special-function unit (PTX tanh.approx.f32, relative error about 2^-11):
// one special-function operation and a few FMAs per element, where the epilogue's element rate
// bounds the hidden layers' GEMMs.  The error it leaves is of the order of the BF16 rounding of the
// stored activations.
__device__ __forceinline__ float tanh_approx(float x) {
    float y;
    asm("tanh.approx.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}
__device__ __forceinline__ float gelu(float z) {
    const float t = tanh_approx(z * fmaf(0.035677408136300125f, z * z, 0.7978845608028654f));
    const float h = 0.5f * z;
    return fmaf(h, t, h);
}
__device__ __forceinline__ float gelu_grad(float z) {
    const float z2 = z * z;
    const float t = tanh_approx(z * fmaf(0.035677408136300125f, z2, 0.7978845608028654f));
    const float du = fmaf(0.10703222440890038f, z2, 0.7978845608028654f);   // k (1 + 3 c z^2)
    return fmaf(0.5f * z * du, fmaf(-t, t, 1.f), fmaf(0.5f, t, 0.5f));
}

__device__ __forceinline__ void store_bf16x16(__nv_bfloat16 *o, const float (&v)[16]) {
    uint4 u[2];
    uint32_t *w = reinterpret_cast<uint32_t *>(u);
#pragma unroll
    for (int i = 0; i < 8; ++i) {
        const __nv_bfloat162 h = __floats2bfloat162_rn(v[2 * i], v[2 * i + 1]);
        w[i] = *reinterpret_cast<const uint32_t *>(&h);
    }
    reinterpret_cast<uint4 *>(o)[0] = u[0];
    reinterpret_cast<uint4 *>(o)[1] = u[1];
}

// The epilogue of 16 accumulator values of one row: v = acc[row, col .. col + 15].  With a store
// mode the row-major output goes to this thread's row of the warp's staging box (st: 16 BF16 or
// 16 FP32 values) instead of global memory; the warp then stores the box with TMA.
__device__ __forceinline__ void stage16(void *st, const float (&v)[16], bool f32) {
    if (f32) {
        float4 *o = reinterpret_cast<float4 *>(st);
#pragma unroll
        for (int i = 0; i < 4; ++i) o[i] = make_float4(v[4 * i], v[4 * i + 1], v[4 * i + 2], v[4 * i + 3]);
    } else {
        uint32_t w[8];
#pragma unroll
        for (int i = 0; i < 8; ++i) {
            const __nv_bfloat162 h = __floats2bfloat162_rn(v[2 * i], v[2 * i + 1]);
            w[i] = *reinterpret_cast<const uint32_t *>(&h);
        }
        uint4 *o = reinterpret_cast<uint4 *>(st);
        o[0] = make_uint4(w[0], w[1], w[2], w[3]);
        o[1] = make_uint4(w[4], w[5], w[6], w[7]);
    }
}

__device__ __forceinline__ void epilogue16(const npx_gemm_epilogue &ep, float (&v)[16], int row, int col, int split,
                                           int store_mode, void *st) {
    if (ep.mode == NPX_EPI_F32) {
        if (store_mode == 2) { stage16(st, v, true); return; }
        float4 *o = reinterpret_cast<float4 *>(ep.outf + (size_t)split * ep.split_stride + (size_t)row * ep.ldf + col);
#pragma unroll
        for (int i = 0; i < 4; ++i) o[i] = make_float4(v[4 * i], v[4 * i + 1], v[4 * i + 2], v[4 * i + 3]);
        return;
    }
    if (ep.bias) {
        const float4 *bb = reinterpret_cast<const float4 *>(ep.bias + col);
#pragma unroll
        for (int i = 0; i < 4; ++i) {
            const float4 b = bb[i];
            v[4 * i] += b.x; v[4 * i + 1] += b.y; v[4 * i + 2] += b.z; v[4 * i + 3] += b.w;
        }
    }
    if (ep.mode == NPX_EPI_BIAS_GELU) {
        if (ep.zsave) store_bf16x16(static_cast<__nv_bfloat16 *>(ep.zsave) + (size_t)row * ep.ldz + col, v);
#pragma unroll
        for (int i = 0; i < 16; ++i) v[i] = gelu(v[i]);
    } else if (ep.mode == NPX_EPI_DGELU) {
        const uint4 *zp = reinterpret_cast<const uint4 *>(static_cast<const __nv_bfloat16 *>(ep.zin) + (size_t)row * ep.ldzi + col);
        uint4 u[2] = {zp[0], zp[1]};
        const __nv_bfloat162 *h = reinterpret_cast<const __nv_bfloat162 *>(u);
#pragma unroll
        for (int i = 0; i < 8; ++i) {
            const float2 z = __bfloat1622float2(h[i]);
            v[2 * i] *= gelu_grad(z.x);
            v[2 * i + 1] *= gelu_grad(z.y);
        }
    }
    if (ep.outf) {
        if (store_mode == 2) {
            stage16(st, v, true);
        } else {
            float4 *o = reinterpret_cast<float4 *>(ep.outf + (size_t)row * ep.ldf + col);
#pragma unroll
            for (int i = 0; i < 4; ++i) o[i] = make_float4(v[4 * i], v[4 * i + 1], v[4 * i + 2], v[4 * i + 3]);
        }
    }
    if (ep.out) {
        if (store_mode == 1) stage16(st, v, false);
        else store_bf16x16(static_cast<__nv_bfloat16 *>(ep.out) + (size_t)row * ep.ldo + col, v);
    }
    if (ep.outT) {
        // lanes hold consecutive rows: each store instruction writes 64 contiguous bytes
        __nv_bfloat16 *o = static_cast<__nv_bfloat16 *>(ep.outT) + (size_t)col * ep.ldt + row;
#pragma unroll
        for (int i = 0; i < 16; ++i) o[(size_t)i * ep.ldt] = __float2bfloat16_rn(v[i]);
    }
}

// STORE = 2: the FP32 row-major output (outf) leaves through per-warp shared-memory boxes and TMA
// stores (tout); STORE = 0: every output is stored directly.
template <int BN, int STORE>
__global__ void __launch_bounds__(THREADS, 1)
gemm_tn_kernel(const __grid_constant__ CUtensorMap ta, const __grid_constant__ CUtensorMap tb,
               const __grid_constant__ CUtensorMap tout, int M, int N, int k_per_split, int splits,
               npx_gemm_epilogue ep, int *err) {
    constexpr int store_mode = STORE;
    extern __shared__ uint8_t smem_raw[];
    uint8_t *smem = reinterpret_cast<uint8_t *>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
    constexpr int A_BYTES = BM * BK * 2, B_BYTES = BN * BK * 2;
    uint8_t *sA = smem;
    uint8_t *sB = smem + STAGES * A_BYTES;
    uint64_t *full = reinterpret_cast<uint64_t *>(sB + STAGES * B_BYTES);
    uint64_t *empty = full + STAGES;
    uint64_t *tfull = empty + STAGES;     // accumulator b ready for the epilogue
    uint64_t *tempty = tfull + 2;         // accumulator b drained by the epilogue
    uint64_t *done = tempty + 2;          // every MMA of this CTA complete
    uint32_t *tmem_slot = reinterpret_cast<uint32_t *>(done + 1);
    volatile int *abort = reinterpret_cast<volatile int *>(tmem_slot + 1);
    int *issued = reinterpret_cast<int *>(tmem_slot + 2);      // k-blocks whose copies were started
    int *consumed = reinterpret_cast<int *>(tmem_slot + 3);    // k-blocks whose copies were waited for
    // per epilogue warp, a 2 KB staging area for the TMA store of the row-major output: two
    // 32 x 16 BF16 boxes (double-buffered) or one 32 x 16 FP32 box
    uint8_t *stage_base = sB + STAGES * B_BYTES + 1024;

    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int tiles_m = M / BM, tiles_n = N / BN, total = tiles_m * tiles_n * splits;
    const int nk = k_per_split / BK;

    if (warp == 1) {   // whole warp: allocate two accumulators of BN columns
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(tmem_slot)),
                     "r"((uint32_t)(2 * BN))
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    if (threadIdx.x == 0) {
        for (int s = 0; s < STAGES; ++s) {
            mbar_init(&full[s], 1);
            mbar_init(&empty[s], 1);
        }
        for (int b = 0; b < 2; ++b) {
            mbar_init(&tfull[b], 1);
            mbar_init(&tempty[b], EPI_WARPS);
        }
        mbar_init(done, 1);
        *abort = 0;
        *issued = 0;
        *consumed = 0;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = *tmem_slot;

    if (warp == 0) {
        // ---- TMA producer
        if (lane == 0) {
            int g = 0;
            bool ok = true;
            for (int t = blockIdx.x; t < total && ok; t += gridDim.x) {
                const int split = t % splits, rest = t / splits;
                const int n0 = (rest % tiles_n) * BN, m0 = (rest / tiles_n) * BM;
                const int kbeg = split * k_per_split;
                for (int kb = 0; kb < nk; ++kb, ++g) {
                    const int s = g % STAGES;
                    if (g >= STAGES && !mbar_wait(&empty[s], (uint32_t)(((g / STAGES) - 1) & 1), abort)) {
                        ok = false;
                        break;
                    }
                    mbar_expect_tx(&full[s], A_BYTES + B_BYTES);
                    tma_load_2d(sA + s * A_BYTES, &ta, kbeg + kb * BK, m0, &full[s]);
                    tma_load_2d(sB + s * B_BYTES, &tb, kbeg + kb * BK, n0, &full[s]);
                    *issued = g + 1;
                }
            }
            if (!ok) {
                *abort = 1;
                atomicExch(err, 1);
            }
        }
    } else if (warp == 1) {
        // ---- MMA issuer
        if (lane == 0) {
            const uint32_t idesc = idesc_bf16(BM, BN);
            int g = 0, tl = 0;
            bool ok = true;
            for (int t = blockIdx.x; t < total && ok; t += gridDim.x, ++tl) {
                const int b = tl & 1;
                if (tl >= 2 && !mbar_wait(&tempty[b], (uint32_t)(((tl >> 1) - 1) & 1), abort)) {
                    ok = false;
                    break;
                }
                tc_fence_after();
                const uint32_t d = tmem + (uint32_t)(b * BN);
                for (int kb = 0; kb < nk; ++kb, ++g) {
                    const int s = g % STAGES;
                    if (!mbar_wait(&full[s], (uint32_t)((g / STAGES) & 1), abort)) {
                        ok = false;
                        break;
                    }
                    *consumed = g + 1;
                    tc_fence_after();
                    const uint64_t da = sdesc_k_sw128(smem_u32(sA + s * A_BYTES));
                    const uint64_t db = sdesc_k_sw128(smem_u32(sB + s * B_BYTES));
#pragma unroll
                    for (int k = 0; k < BK / 16; ++k)   // 32 bytes along K per instruction
                        umma_bf16(d, da + (uint64_t)(2 * k), db + (uint64_t)(2 * k), idesc, (kb | k) != 0);
                    umma_commit(&empty[s]);
                }
                if (!ok) break;
                umma_commit(&tfull[b]);
            }
            umma_commit(done);
            if (!ok) {
                *abort = 1;
                atomicExch(err, 2);
            }
        }
    } else {
        // ---- epilogue: warp w reads TMEM lanes 32 (w % 4) .. + 31 and column quarter (w - 2) / 4
        const int q = warp & 3, part = (warp - 2) >> 2;
        constexpr int COLS = BN / (EPI_WARPS / 4);
        uint8_t *stage = stage_base + (warp - 2) * 2048;
        const bool f32 = store_mode == 2;
        int nstore = 0;   // TMA stores issued by this warp
        int tl = 0;
        for (int t = blockIdx.x; t < total; t += gridDim.x, ++tl) {
            const int b = tl & 1;
            const int split = t % splits, rest = t / splits;
            const int n0 = (rest % tiles_n) * BN, m0 = (rest / tiles_n) * BM;
            if (!mbar_wait(&tfull[b], (uint32_t)((tl >> 1) & 1), abort)) {
                if (lane == 0) {
                    *abort = 1;
                    atomicExch(err, 3);
                }
                break;
            }
            tc_fence_after();
            const int row = m0 + q * 32 + lane;
            const uint32_t taddr = tmem + ((uint32_t)(q * 32) << 16) + (uint32_t)(b * BN);
#pragma unroll 1
            for (int c0 = part * COLS; c0 < (part + 1) * COLS; c0 += 16) {
                uint32_t r[16];
                tmem_ld16_issue(taddr + (uint32_t)c0, r);
                tmem_wait_ld();
                float v[16];
#pragma unroll
                for (int i = 0; i < 16; ++i) v[i] = __uint_as_float(r[i]);
                uint8_t *box = nullptr;
                if (store_mode) {
                    // the staging box is free once the store that last read it has read it
                    box = stage + (f32 ? 0 : (nstore & 1) * 1024);
                    if (f32 ? nstore >= 1 : nstore >= 2) {
                        if (lane == 0) {
                            if (f32) bulk_wait_read<0>();
                            else bulk_wait_read<1>();
                        }
                        __syncwarp();
                    }
                }
                epilogue16(ep, v, row, n0 + c0, split, store_mode, box + lane * (f32 ? 64 : 32));
                if (store_mode) {
                    fence_async_shared();
                    __syncwarp();
                    if (lane == 0) {
                        if (f32) tma_store_3d(&tout, n0 + c0, m0 + q * 32, split, box);
                        else tma_store_2d(&tout, n0 + c0, m0 + q * 32, box);
                        bulk_commit();
                    }
                    ++nstore;
                }
            }
            tc_fence_before();
            __syncwarp();
            if (lane == 0) mbar_arrive(&tempty[b]);
        }
        if (store_mode && lane == 0) bulk_wait_all();   // the stores have landed before the CTA ends
        __syncwarp();
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        // after a failure: let the copies still in flight land before the shared memory goes away
        for (int g = *consumed; g < *issued; ++g) mbar_wait(&full[g % STAGES], (uint32_t)((g / STAGES) & 1));
        // every MMA issued by this CTA has completed before its tensor memory is freed
        if (!mbar_wait(done, 0)) atomicExch(err, 4);
    }
    tc_fence_before();
    __syncthreads();
    if (warp == 1) {
        tc_fence_after();
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"((uint32_t)(2 * BN)) : "memory");
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

// map of the row-major output written by the epilogue's TMA stores, in boxes of 32 rows x 16
// columns: BF16 [rows x cols] with row stride ld (2-D), or FP32 split partials
// [splits][rows x cols] with row stride ld and split stride split_stride (3-D)
static bool make_out_map(CUtensorMap *m, void *ptr, bool f32, int rows, int cols, long long ld, int splits,
                         long long split_stride) {
    EncodeTiledFn fn = encode_fn();
    if (!fn) return false;
    const cuuint64_t es = f32 ? 4 : 2;
    const cuuint64_t dims[3] = {(cuuint64_t)cols, (cuuint64_t)rows, (cuuint64_t)splits};
    const cuuint64_t strides[2] = {(cuuint64_t)ld * es, (cuuint64_t)(splits > 1 ? split_stride : ld * rows) * es};
    const cuuint32_t box[3] = {16, 32, 1};
    const cuuint32_t el[3] = {1, 1, 1};
    return fn(m, f32 ? CU_TENSOR_MAP_DATA_TYPE_FLOAT32 : CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, f32 ? 3 : 2, ptr, dims,
              strides, box, el, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE,
              CU_TENSOR_MAP_L2_PROMOTION_NONE, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

template <int BN, int STORE>
static size_t smem_bytes() {
    return 1024 + (size_t)STAGES * (BM * BK * 2 + BN * BK * 2) + 1024 + (STORE ? (size_t)EPI_WARPS * 2048 : 0);
}

static int sm_count() {
    static int n = 0;
    if (!n) {
        int dev = 0;
        if (cudaGetDevice(&dev) != cudaSuccess ||
            cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || n < 1)
            n = 1;
    }
    return n;
}

template <int BN, int STORE>
static cudaError_t launch(const CUtensorMap &ta, const CUtensorMap &tb, const CUtensorMap &tout, int M, int N, int K,
                          int splits, const npx_gemm_epilogue &ep, int *err, cudaStream_t st) {
    const size_t smem = smem_bytes<BN, STORE>();
    cudaError_t e = cudaFuncSetAttribute(gemm_tn_kernel<BN, STORE>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    const int tiles = (M / BM) * (N / BN) * splits;
    const int grid = tiles < sm_count() ? tiles : sm_count();
    gemm_tn_kernel<BN, STORE><<<grid, THREADS, smem, st>>>(ta, tb, tout, M, N, K / splits, splits, ep, err);
    return cudaGetLastError();
}

// The bounded barrier wait on its own: thread 0 waits on a barrier that nothing completes; with
// use_abort, warp 1 raises the abort flag after ABORT_NS.  out[0] = 1 if the wait gave up (0 if
// the phase completed), out[1] = the wait in microseconds.
constexpr unsigned long long ABORT_NS = 1000000ull;   // 1 ms
__global__ void __launch_bounds__(64) wait_selftest_kernel(int use_abort, int *out) {
    __shared__ uint64_t bar;
    __shared__ volatile int abort_flag;
    if (threadIdx.x == 0) {
        mbar_init(&bar, 1);
        abort_flag = 0;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    __syncthreads();
    if (use_abort && threadIdx.x == 32) {
        const unsigned long long t0 = global_ns();
        while (global_ns() - t0 < ABORT_NS) {
        }
        abort_flag = 1;
    }
    if (threadIdx.x == 0) {
        const unsigned long long t0 = global_ns();
        const bool ok = mbar_wait(&bar, 0, use_abort ? &abort_flag : nullptr);
        out[0] = ok ? 0 : 1;
        out[1] = (int)((global_ns() - t0) / 1000ull);
    }
}

}  // namespace gemm
}  // namespace npx

extern "C" int npx_gemm_wait_selftest(int use_abort, int *timed_out, int *elapsed_us, void *stream) {
    if (!timed_out || !elapsed_us) return npx::set_last_error(NPX_EINVAL, "npx_gemm_wait_selftest: null argument");
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    int *d = nullptr;
    cudaError_t e = cudaMalloc(&d, 2 * sizeof(int));
    if (e != cudaSuccess) return npx::set_last_error(NPX_ENOMEM, cudaGetErrorString(e));
    int h[2] = {-1, -1};
    npx::gemm::wait_selftest_kernel<<<1, 64, 0, st>>>(use_abort ? 1 : 0, d);
    e = cudaGetLastError();
    if (e == cudaSuccess) e = cudaMemcpyAsync(h, d, sizeof h, cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    cudaFree(d);
    if (e != cudaSuccess) return npx::set_last_error(NPX_ECUDA, cudaGetErrorString(e));
    *timed_out = h[0];
    *elapsed_us = h[1];
    return NPX_OK;
}

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
    // the epilogue stores 16-byte vectors: 16-byte aligned rows of the row-major outputs
    auto rows16 = [](const void *p, long long ld, int elem) {
        return !p || ((reinterpret_cast<uintptr_t>(p) & 15) == 0 && (ld * elem) % 16 == 0);
    };
    if (!rows16(ep->bias, 0, 4) || !rows16(ep->out, ep->ldo, 2) || !rows16(ep->zsave, ep->ldz, 2) ||
        !rows16(ep->zin, ep->ldzi, 2) || !rows16(ep->outf, ep->ldf, 4) ||
        (ep->outf && splits > 1 && (ep->split_stride * 4) % 16 != 0) ||
        (ep->outT && (reinterpret_cast<uintptr_t>(ep->outT) & 1)))
        return npx::set_last_error(NPX_EINVAL, "npx_gemm_bf16: outputs, bias and zin need 16-byte aligned rows");
    if (splits > 1 && ep->mode != NPX_EPI_F32) return npx::set_last_error(NPX_EINVAL, "npx_gemm_bf16: split K needs the F32 epilogue");
    CUtensorMap ta, tb, tout;
    if (!make_map(&ta, A, M, K, BM) || !make_map(&tb, B, N, K, BN))
        return npx::set_last_error(NPX_ECUDA, "npx_gemm_bf16: tensor-map encoding failed");
    // the row-major output leaves through per-warp staging boxes and TMA stores: FP32 (store
    // mode 2), or BF16 when it is the only row-major output (mode 1)
    memset(&tout, 0, sizeof tout);
    int store_mode = 0;
    if (ep->outf && !(ep->out && ep->mode != NPX_EPI_F32)) {
        if (!make_out_map(&tout, ep->outf, true, M, N, ep->ldf, ep->mode == NPX_EPI_F32 ? splits : 1, ep->split_stride))
            return npx::set_last_error(NPX_ECUDA, "npx_gemm_bf16: output tensor-map encoding failed");
        store_mode = 2;
    } else if (ep->out && !ep->outf && ep->mode != NPX_EPI_F32) {
        if (!make_out_map(&tout, ep->out, false, M, N, ep->ldo, 1, 0))
            return npx::set_last_error(NPX_ECUDA, "npx_gemm_bf16: output tensor-map encoding failed");
        store_mode = 1;
    }
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    cudaError_t e;
    if (store_mode == 2)
        e = BN == 256 ? launch<256, 2>(ta, tb, tout, M, N, K, splits, *ep, err, st)
                      : launch<128, 2>(ta, tb, tout, M, N, K, splits, *ep, err, st);
    else if (store_mode == 1)
        e = BN == 256 ? launch<256, 1>(ta, tb, tout, M, N, K, splits, *ep, err, st)
                      : launch<128, 1>(ta, tb, tout, M, N, K, splits, *ep, err, st);
    else
        e = BN == 256 ? launch<256, 0>(ta, tb, tout, M, N, K, splits, *ep, err, st)
                      : launch<128, 0>(ta, tb, tout, M, N, K, splits, *ep, err, st);
    if (e != cudaSuccess) return npx::set_last_error(NPX_ECUDA, cudaGetErrorString(e));
    return NPX_OK;
}

// eses_mlp_tc.cuh -- the proposer MLP on the fifth-generation tensor cores:
// BF16 weights and activations, FP32 accumulation in tensor memory.
//
// One CTA of 128 threads scores 128 rows (tiles) at a time:
//   layer 1: D1[128 x 64] = A1[128 x 32] . W1   (two MMAs of K = 16)
//   layer 2: D2[128 x 64] = relu(D1 + b1)[128 x 64] . W2   (four MMAs)
//   layer 3: z = relu(D2 + b2) . w3 + b3 on the CUDA cores (FP32)
// tcgen05.mma (cta_group::1, kind::f16, BF16 inputs, F32 accumulator) is
// issued by one thread, with both operands in shared memory in the canonical
// K-major layout without swizzle: 8 x 8 core matrices of 128 contiguous
// bytes, LBO = 128 B between core matrices along K, SBO = K * 16 B between
// 8-row groups; the weights are stored transposed (N x K, K-major), so
// D = A . B^T.  The accumulators live in 128 TMEM columns (64 per layer;
// row r of D in TMEM lane r) and every thread reads its own row back with
// tcgen05.ld (32x32b shape).  Completion is signalled by tcgen05.commit on an
// mbarrier; every wait is bounded: a wait that runs out sets *err and the
// rows it covers score +inf, i.e. "near" (the exact path then runs).
#pragma once

#include <cuda_bf16.h>
#include <stdint.h>

namespace eses {

constexpr int TC_ROWS = 128;
constexpr int TC_COLS = 128;              // TMEM columns allocated per CTA
constexpr long long TC_WAIT_LIMIT = 1LL << 22;

struct TcSmem {
    alignas(128) uint8_t A1[TC_ROWS * MLP_IN * 2];
    alignas(128) uint8_t A2[TC_ROWS * MLP_H * 2];
    alignas(128) uint8_t B1[MLP_H * MLP_IN * 2];
    alignas(128) uint8_t B2[MLP_H * MLP_H * 2];
    float b1[MLP_H], b2[MLP_H], w3[MLP_H];
    float b3;
    alignas(8) unsigned long long mbar;
    uint32_t tmem;
    int dead;  // a wait ran out: no further tensor-core work in this CTA
    long long wait_limit;  // iterations of each scoring wait (tc_teardown always waits TC_WAIT_LIMIT)
};

// byte offset of element (r, k) of a K-major matrix with K columns (canonical, no swizzle)
__device__ __forceinline__ int kmaj_off(int r, int k, int K)
{
    return (r >> 3) * (K * 16) + (k >> 3) * 128 + (r & 7) * 16 + (k & 7) * 2;
}

__device__ __forceinline__ uint32_t smem_u32(const void *p) { return (uint32_t)__cvta_generic_to_shared(p); }

// shared-memory matrix descriptor (version 1, no swizzle)
__device__ __forceinline__ uint64_t smem_desc(const void *p, uint32_t lbo, uint32_t sbo)
{
    uint64_t d = 0;
    d |= (uint64_t)((smem_u32(p) >> 4) & 0x3FFF);
    d |= (uint64_t)((lbo >> 4) & 0x3FFF) << 16;
    d |= (uint64_t)((sbo >> 4) & 0x3FFF) << 32;
    d |= (uint64_t)1 << 46;
    return d;
}

// instruction descriptor: F32 accumulator, BF16 A and B, both K-major, M x N
__host__ __device__ constexpr uint32_t idesc_bf16(int M, int N)
{
    return (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(N >> 3) << 17) | ((uint32_t)(M >> 4) << 24);
}

__device__ __forceinline__ void tc_mma(uint32_t d_tmem, uint64_t a, uint64_t b, uint32_t idesc, int accum)
{
    asm volatile(
        "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
        "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}\n" ::"r"(d_tmem),
        "l"(a), "l"(b), "r"(idesc), "r"(accum));
}

__device__ __forceinline__ void tc_commit(unsigned long long *mbar)
{
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(smem_u32(mbar))
                 : "memory");
}

__device__ __forceinline__ void mbar_init(unsigned long long *mbar, int count)
{
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(mbar)), "r"(count) : "memory");
}

// bounded wait for the phase with the given parity (at most `limit` polls);
// false when the limit ran out
__device__ __forceinline__ bool mbar_wait(unsigned long long *mbar, uint32_t parity, long long limit = TC_WAIT_LIMIT)
{
    const uint32_t a = smem_u32(mbar);
    for (long long it = 0; it < limit; ++it) {
        uint32_t done;
        asm volatile(
            "{\n\t.reg .pred p;\n\tmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
            "selp.u32 %0, 1, 0, p;\n\t}\n"
            : "=r"(done)
            : "r"(a), "r"(parity)
            : "memory");
        if (done) return true;
    }
    return false;
}

__device__ __forceinline__ void tc_fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void tc_fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void fence_async_smem() { asm volatile("fence.proxy.async.shared::cta;" ::: "memory"); }

// 16 consecutive FP32 columns of this thread's TMEM lane
__device__ __forceinline__ void tmem_ld16(uint32_t taddr, float *v)
{
    uint32_t r[16];
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, "
        "%15}, [%16];"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]), "=r"(r[8]),
          "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
        : "r"(taddr));
    asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
    for (int k = 0; k < 16; ++k) v[k] = __uint_as_float(r[k]);
}

// one warp: allocate / free the CTA's TMEM columns
__device__ __forceinline__ void tmem_alloc(uint32_t *dst)
{
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(dst)),
                 "r"(TC_COLS)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
}
__device__ __forceinline__ void tmem_free(uint32_t taddr)
{
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(taddr), "r"(TC_COLS) : "memory");
}

// weights into shared memory (BF16, transposed to N x K, K-major) and biases;
// TMEM allocation and mbarrier set-up.  wait_limit: polls of each scoring wait
// (< 0: TC_WAIT_LIMIT; 0 makes every scoring wait give up at once, which only
// a test of the fallback wants).  Whole CTA (128 threads); ends with a barrier.
__device__ void tc_setup(TcSmem &T, const float *__restrict__ P, long long wait_limit = -1)
{
    for (int e = threadIdx.x; e < MLP_H * MLP_IN; e += blockDim.x) {
        const int n = e / MLP_IN, k = e % MLP_IN;
        *reinterpret_cast<__nv_bfloat16 *>(T.B1 + kmaj_off(n, k, MLP_IN)) = __float2bfloat16_rn(P[P_W1 + k * MLP_H + n]);
    }
    for (int e = threadIdx.x; e < MLP_H * MLP_H; e += blockDim.x) {
        const int n = e / MLP_H, k = e % MLP_H;
        *reinterpret_cast<__nv_bfloat16 *>(T.B2 + kmaj_off(n, k, MLP_H)) = __float2bfloat16_rn(P[P_W2 + k * MLP_H + n]);
    }
    for (int k = threadIdx.x; k < MLP_H; k += blockDim.x) {
        T.b1[k] = P[P_B1 + k];
        T.b2[k] = P[P_B2 + k];
        T.w3[k] = P[P_W3 + k];
    }
    if (threadIdx.x == 0) {
        T.b3 = P[P_B3];
        T.dead = 0;
        T.wait_limit = wait_limit < 0 ? TC_WAIT_LIMIT : wait_limit;
        mbar_init(&T.mbar, 1);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if (threadIdx.x < 32) tmem_alloc(&T.tmem);
    fence_async_smem();
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
}

__device__ __forceinline__ void tc_teardown(TcSmem &T, uint32_t phase)
{
    // after a wait that ran out, give the MMAs in flight one more bounded wait
    if (T.dead && threadIdx.x == 0) mbar_wait(&T.mbar, phase);
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    if (threadIdx.x < 32) tmem_free(T.tmem);
}

// Scores of the CTA's 128 rows: thread t owns row t, whose 32 features are x
// (valid only when `valid`).  phase: the mbarrier parity of the CTA's next
// wait (two waits per call; flipped only after a completed wait).  Returns z
// for row t, +inf when a wait ran out (then the CTA stops using the tensor
// cores and tc_teardown waits once more before freeing TMEM).
__device__ float tc_score(TcSmem &T, const float *x, bool valid, uint32_t &phase, int *err)
{
    const int t = threadIdx.x;
    if (T.dead) return INFINITY;  // uniform: set under a barrier
    // row t of A1 (zeros for an invalid row)
#pragma unroll
    for (int k = 0; k < MLP_IN; k += 8) {
        __nv_bfloat162 v[4];
#pragma unroll
        for (int q = 0; q < 4; ++q)
            v[q] = valid ? __floats2bfloat162_rn(x[k + 2 * q], x[k + 2 * q + 1]) : __floats2bfloat162_rn(0.0f, 0.0f);
        *reinterpret_cast<uint4 *>(T.A1 + kmaj_off(t, k, MLP_IN)) = *reinterpret_cast<uint4 *>(v);
    }
    fence_async_smem();
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t d1 = T.tmem, d2 = T.tmem + MLP_H;
    constexpr uint32_t ID = idesc_bf16(TC_ROWS, MLP_H);
    if (t == 0) {
#pragma unroll
        for (int s = 0; s < MLP_IN / 16; ++s)
            tc_mma(d1, smem_desc(T.A1 + s * 256, 128, MLP_IN * 16), smem_desc(T.B1 + s * 256, 128, MLP_IN * 16), ID,
                   s > 0);
        tc_commit(&T.mbar);
    }
    bool ok = __all_sync(0xffffffffu, mbar_wait(&T.mbar, phase, T.wait_limit));
    tc_fence_after();
    const uint32_t lane_base = (uint32_t)((t >> 5) * 32) << 16;
    // layer 1 epilogue: bias, ReLU, BF16 into row t of A2
    if (ok) {
#pragma unroll
        for (int c = 0; c < MLP_H; c += 16) {
            float v[16];
            tmem_ld16(d1 + lane_base + c, v);
            __nv_bfloat162 o[8];
#pragma unroll
            for (int q = 0; q < 8; ++q)
                o[q] = __floats2bfloat162_rn(fmaxf(v[2 * q] + T.b1[c + 2 * q], 0.0f),
                                             fmaxf(v[2 * q + 1] + T.b1[c + 2 * q + 1], 0.0f));
            *reinterpret_cast<uint4 *>(T.A2 + kmaj_off(t, c, MLP_H)) = *reinterpret_cast<uint4 *>(&o[0]);
            *reinterpret_cast<uint4 *>(T.A2 + kmaj_off(t, c + 8, MLP_H)) = *reinterpret_cast<uint4 *>(&o[4]);
        }
    }
    ok = __syncthreads_and(ok);
    if (!ok) {
        if (t == 0) {
            atomicOr(err, ERR_TIMEOUT);
            T.dead = 1;
        }
        __syncthreads();
        return INFINITY;
    }
    phase ^= 1;
    fence_async_smem();
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    if (t == 0) {
#pragma unroll
        for (int s = 0; s < MLP_H / 16; ++s)
            tc_mma(d2, smem_desc(T.A2 + s * 256, 128, MLP_H * 16), smem_desc(T.B2 + s * 256, 128, MLP_H * 16), ID,
                   s > 0);
        tc_commit(&T.mbar);
    }
    ok = __all_sync(0xffffffffu, mbar_wait(&T.mbar, phase, T.wait_limit));
    tc_fence_after();
    float z = T.b3;
    if (ok) {
#pragma unroll
        for (int c = 0; c < MLP_H; c += 16) {
            float v[16];
            tmem_ld16(d2 + lane_base + c, v);
#pragma unroll
            for (int q = 0; q < 16; ++q) z = fmaf(fmaxf(v[q] + T.b2[c + q], 0.0f), T.w3[c + q], z);
        }
    }
    ok = __syncthreads_and(ok);
    if (!ok) {
        if (t == 0) {
            atomicOr(err, ERR_TIMEOUT);
            T.dead = 1;
        }
        __syncthreads();
        return INFINITY;
    }
    phase ^= 1;
    return z;
}

}  // namespace eses

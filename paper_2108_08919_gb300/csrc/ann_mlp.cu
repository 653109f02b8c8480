// BF16 tensor-core GEMMs for the learned surrogate (5th-generation tensor cores, tcgen05, sm_103a):
//
//   nt:  C[rows x N] = act([A1 | A2][rows x (K1 + K2)] . B[N x K]^T + bias)   (forward, dX)
//   tn:  C[K x N]   += A[rows x K]^T . B[rows x N]                              (weight gradients)
//
// A, B are BF16, accumulation FP32 in tensor memory.  One CTA of 128 threads: thread 0 issues
// tcgen05.mma (M = 128, K = 16 per instruction) from shared-memory descriptors, the completion is
// committed to an mbarrier, and the four warps read the 128 x N accumulator back with tcgen05.ld
// (warp w owns TMEM lanes 32w .. 32w + 31, i.e. tile rows).  Operands are staged into shared memory
// by the threads in the canonical no-swizzle K-major layout: 8-row x 16-byte core matrices, core
// matrix (r, k) at byte k * LBO + r * SBO with LBO = 128 and SBO = 128 * (K / 8).  Every wait on
// the mbarrier is bounded; on time-out the kernel records an error and leaves.
#include "../../include/ann.h"
#include "ann_internal.cuh"

#include <cuda_bf16.h>

namespace ann {
namespace {

constexpr int MT = 128;                 // rows of a tile (the MMA's M)
constexpr unsigned SPIN_LIMIT = 1u << 26;

__device__ __forceinline__ uint32_t smem_u32(const void *p) { return (uint32_t)__cvta_generic_to_shared(p); }

// Shared-memory matrix descriptor: start address, leading (K) and stride (M/N) byte offsets, the
// descriptor version bit of the 5th-generation format, no swizzle.
__device__ __forceinline__ uint64_t smem_desc(uint32_t addr, uint32_t lbo, uint32_t sbo)
{
    uint64_t d = 0;
    d |= (uint64_t)((addr >> 4) & 0x3FFFu);
    d |= (uint64_t)((lbo >> 4) & 0x3FFFu) << 16;
    d |= (uint64_t)((sbo >> 4) & 0x3FFFu) << 32;
    d |= (uint64_t)1 << 46;   // version
    return d;                 // base offset 0, layout SWIZZLE_NONE (0)
}

// Instruction descriptor of kind::f16: D FP32, A and B BF16, both K-major, N >> 3, M >> 4.
__host__ __device__ constexpr uint32_t idesc_bf16(int M, int N)
{
    return (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(N >> 3) << 17) | ((uint32_t)(M >> 4) << 24);
}

__device__ __forceinline__ void tmem_alloc(uint32_t *holder, uint32_t ncols)
{
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(holder)),
                 "r"(ncols));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
}

__device__ __forceinline__ void tmem_dealloc(uint32_t taddr, uint32_t ncols)
{
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(taddr), "r"(ncols));
}

__device__ __forceinline__ void mma_bf16(uint32_t dtmem, uint64_t a, uint64_t b, uint32_t idesc, bool acc)
{
    asm volatile(
        "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
        "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}" ::"r"(dtmem),
        "l"(a), "l"(b), "r"(idesc), "r"((uint32_t)acc));
}

__device__ __forceinline__ void mma_commit(uint64_t *mbar)
{
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
        smem_u32(mbar)));
}

__device__ __forceinline__ void fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void fence_async_smem() { asm volatile("fence.proxy.async.shared::cta;" ::: "memory"); }

__device__ __forceinline__ void mbar_init(uint64_t *mbar, uint32_t count)
{
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(mbar)), "r"(count));
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");   // visible to the async proxy
}

// Bounded wait for the phase `parity` of the mbarrier to complete; false on time-out.
__device__ __forceinline__ bool mbar_wait(uint64_t *mbar, uint32_t parity)
{
    uint32_t a = smem_u32(mbar);
    for (unsigned it = 0; it < SPIN_LIMIT; it++) {
        uint32_t done;
        asm volatile(
            "{\n\t.reg .pred p;\n\tmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\tselp.u32 %0, 1, 0, p;\n\t}"
            : "=r"(done)
            : "r"(a), "r"(parity)
            : "memory");
        if (done) return true;
    }
    return false;
}

// 16 consecutive FP32 columns of this thread's TMEM lane.
__device__ __forceinline__ void tmem_ld16(uint32_t taddr, float *v)
{
    uint32_t r[16];
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
          "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
        : "r"(taddr));
    asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
    for (int k = 0; k < 16; k++) v[k] = __uint_as_float(r[k]);
}

// Byte offset of element (row, k) of a K-major operand with Kt columns in the canonical layout.
__device__ __forceinline__ uint32_t kmaj_off(int row, int k, int Kt)
{
    return (uint32_t)(((k >> 3) * 128) + ((row >> 3) * (Kt >> 3) * 128) + ((row & 7) * 16) + ((k & 7) * 2));
}

__device__ __forceinline__ uint32_t ncols_for(int N) { return N <= 32 ? 32u : (N <= 64 ? 64u : (N <= 128 ? 128u : 256u)); }

// Rows r0 .. r0 + 127 of [A1 | A2] (K = K1 + K2 columns, zero past `rows`) into the canonical layout
// at sA, by the 128 threads of the CTA.  Thread t moves 16-byte chunks t, t + 128, ... of the tile
// (consecutive threads read consecutive chunks of a row: coalesced), loading a batch of 8 chunks
// into registers before storing any, so that 8 loads per thread are in flight at once.
__device__ __forceinline__ void stage_rows(const __nv_bfloat16 *A1, int K1, const __nv_bfloat16 *A2, int K2, int r0,
                                           int rows, unsigned char *sA, int tid)
{
    const int K = K1 + K2, kc = K / 8, c1 = K1 / 8;
    for (int u0 = 0; u0 < kc; u0 += 8) {
        uint4 v[8];
#pragma unroll
        for (int u = 0; u < 8; u++) {
            v[u] = make_uint4(0u, 0u, 0u, 0u);
            const int e = tid + MT * (u0 + u), r = e / kc, c = e - r * kc, gr = r0 + r;
            if (u0 + u < kc && gr < rows) {
                const __nv_bfloat16 *src = c < c1 ? A1 + (size_t)gr * K1 + c * 8 : A2 + (size_t)gr * K2 + (c - c1) * 8;
                v[u] = __ldcs(reinterpret_cast<const uint4 *>(src));
            }
        }
#pragma unroll
        for (int u = 0; u < 8; u++) {
            const int e = tid + MT * (u0 + u), r = e / kc, c = e - r * kc;
            if (u0 + u < kc) *reinterpret_cast<uint4 *>(sA + kmaj_off(r, c * 8, K)) = v[u];
        }
    }
}

// ------------------------------------------------------------------------------------------------
// nt: persistent CTAs keep B (N x K) in shared memory and walk 128-row tiles of A.
// ------------------------------------------------------------------------------------------------

struct NtArgs {
    const __nv_bfloat16 *A1, *A2;   // rows x K1, rows x K2 (row-major), A2 may be null (K2 = 0)
    const __nv_bfloat16 *B;         // N x K (row-major: K-major)
    const float *bias;              // N or null
    void *C;                        // rows x N (row stride ldc): BF16 or FP32
    int rows, K1, K2, N, relu, c_bf16, accumulate, ldc;
    unsigned *err;
};

__global__ void __launch_bounds__(128) k_gemm_nt(NtArgs a)
{
    extern __shared__ __align__(128) unsigned char sm[];
    __shared__ uint64_t mbar;
    __shared__ uint32_t tbase;
    const int K = a.K1 + a.K2, N = a.N;
    unsigned char *sB = sm;                                  // N x K
    unsigned char *sA = sm + (size_t)N * K * 2;              // MT x K
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const uint32_t ncols = ncols_for(N);
    if (warp == 0) tmem_alloc(&tbase, ncols);
    if (tid == 0) mbar_init(&mbar, 1);
    // B once per CTA: 8 BF16 (16 bytes) per copy
    for (int e = tid; e < N * (K / 8); e += blockDim.x) {
        int n = e / (K / 8), k8 = (e % (K / 8)) * 8;
        uint4 v = *reinterpret_cast<const uint4 *>(a.B + (size_t)n * K + k8);
        *reinterpret_cast<uint4 *>(sB + kmaj_off(n, k8, K)) = v;
    }
    fence_before();
    __syncthreads();
    fence_after();
    const uint32_t tmem = tbase;
    const uint32_t idesc = idesc_bf16(MT, N);
    const int ntiles = (a.rows + MT - 1) / MT;
    uint32_t phase = 0;
    bool ok = true;
    for (int t = blockIdx.x; t < ntiles && ok; t += gridDim.x) {
        const int r0 = t * MT;
        stage_rows(a.A1, a.K1, a.A2, a.K2, r0, a.rows, sA, tid);
        fence_async_smem();
        fence_before();
        __syncthreads();
        fence_after();
        if (tid == 0) {
            const uint32_t sbo_a = (uint32_t)(K / 8) * 128, sbo_b = (uint32_t)(K / 8) * 128;
            for (int k = 0; k < K / 16; k++) {
                uint64_t da = smem_desc(smem_u32(sA) + (uint32_t)k * 256, 128, sbo_a);
                uint64_t db = smem_desc(smem_u32(sB) + (uint32_t)k * 256, 128, sbo_b);
                mma_bf16(tmem, da, db, idesc, k > 0);
            }
            mma_commit(&mbar);
        }
        ok = __syncthreads_and(mbar_wait(&mbar, phase)) != 0;   // one decision for the whole CTA
        phase ^= 1u;
        fence_after();
        if (!ok) {
            if (tid == 0) atomicOr(a.err, 1u);
            break;
        }
        const int row = warp * 32 + lane, gr = r0 + row;
        for (int c0 = 0; c0 < N; c0 += 16) {
            float v[16];
            tmem_ld16(tmem + ((uint32_t)(warp * 32) << 16) + (uint32_t)c0, v);
            if (gr < a.rows) {
#pragma unroll
                for (int k = 0; k < 16; k++) {
                    float x = v[k] + (a.bias ? a.bias[c0 + k] : 0.f);
                    if (a.relu) x = fmaxf(x, 0.f);
                    v[k] = x;
                }
                if (a.c_bf16) {   // 32 bytes of the row: two 16-byte stores
                    uint4 w[2];
                    __nv_bfloat162 *h = reinterpret_cast<__nv_bfloat162 *>(w);
#pragma unroll
                    for (int k = 0; k < 8; k++) h[k] = __floats2bfloat162_rn(v[2 * k], v[2 * k + 1]);
                    uint4 *C = reinterpret_cast<uint4 *>(static_cast<__nv_bfloat16 *>(a.C) + (size_t)gr * a.ldc + c0);
                    C[0] = w[0];
                    C[1] = w[1];
                } else {          // 64 bytes: four 16-byte stores
                    float4 *C = reinterpret_cast<float4 *>(static_cast<float *>(a.C) + (size_t)gr * a.ldc + c0);
#pragma unroll
                    for (int k = 0; k < 4; k++) {
                        float4 o = make_float4(v[4 * k], v[4 * k + 1], v[4 * k + 2], v[4 * k + 3]);
                        if (a.accumulate) {
                            float4 c = C[k];
                            o.x += c.x;
                            o.y += c.y;
                            o.z += c.z;
                            o.w += c.w;
                        }
                        C[k] = o;
                    }
                }
            }
        }
        fence_before();
        __syncthreads();   // the next tile's staging overwrites sA; TMEM is rewritten by the next MMA
        fence_after();
    }
    fence_before();
    __syncthreads();
    fence_after();
    if (warp == 0) tmem_dealloc(tmem, ncols);
}

// ------------------------------------------------------------------------------------------------
// tn: C[K x N] += A^T B over all rows.  CTA (x, y): feature block y (128 features of A's K), row
// chunks x, x + gridDim.x, ...; the chunk of 128 rows is staged transposed (features x rows and
// N x rows, both K-major in the rows) and reduced by 8 MMAs of K = 16 rows into TMEM; at the end
// the CTA adds its 128 x N partial to C with FP32 atomics.
// ------------------------------------------------------------------------------------------------

// Columns f0 .. f0 + W - 1 (zero past K) of rows r0 .. r0 + 127 (zero past `rows`) of the row-major
// X (rows x K), transposed into the canonical layout: element (column f, row r) at
// kmaj_off(f - f0, r, 128).  Thread t owns row r0 + t and reads it in 16-byte chunks (batches of 8
// in flight) when K is a multiple of 8 and X 16-byte aligned, element by element otherwise.
__device__ __forceinline__ void stage_rows_T(const __nv_bfloat16 *X, int K, int f0, int r0, int rows, unsigned char *s,
                                             int W, int tid)
{
    const int gr = r0 + tid;
    const bool live = gr < rows;
    if ((K & 7) == 0 && (reinterpret_cast<uintptr_t>(X) & 15) == 0) {
        const uint4 *row = reinterpret_cast<const uint4 *>(X + (size_t)(live ? gr : 0) * K);
        for (int c0 = 0; c0 < W / 8; c0 += 8) {
            uint4 v[8];
#pragma unroll
            for (int u = 0; u < 8; u++) {
                const int f = f0 + (c0 + u) * 8;
                v[u] = make_uint4(0u, 0u, 0u, 0u);
                if (live && c0 + u < W / 8 && f < K) v[u] = __ldg(row + f / 8);
            }
#pragma unroll
            for (int u = 0; u < 8; u++) {
                if (c0 + u >= W / 8) break;
                const __nv_bfloat16 *h = reinterpret_cast<const __nv_bfloat16 *>(&v[u]);
#pragma unroll
                for (int q = 0; q < 8; q++)
                    *reinterpret_cast<__nv_bfloat16 *>(s + kmaj_off((c0 + u) * 8 + q, tid, MT)) = h[q];
            }
        }
    } else {
        for (int f = 0; f < W; f++) {
            __nv_bfloat16 v = __float2bfloat16(0.f);
            if (live && f0 + f < K) v = X[(size_t)gr * K + f0 + f];
            *reinterpret_cast<__nv_bfloat16 *>(s + kmaj_off(f, tid, MT)) = v;
        }
    }
}

struct TnArgs {
    const __nv_bfloat16 *A;   // rows x K
    const __nv_bfloat16 *B;   // rows x N
    float *C;                 // K x N (FP32, accumulated, row stride ldc)
    int rows, K, N, ldc;
    unsigned *err;
};

__global__ void __launch_bounds__(128) k_gemm_tn(TnArgs a)
{
    extern __shared__ __align__(128) unsigned char sm[];
    __shared__ uint64_t mbar;
    __shared__ uint32_t tbase;
    const int N = a.N, f0 = blockIdx.y * MT;
    unsigned char *sA = sm;                        // 128 features x 128 rows
    unsigned char *sB = sm + MT * MT * 2;          // N x 128 rows
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const uint32_t ncols = ncols_for(N);
    if (warp == 0) tmem_alloc(&tbase, ncols);
    if (tid == 0) mbar_init(&mbar, 1);
    fence_before();
    __syncthreads();
    fence_after();
    const uint32_t tmem = tbase;
    const uint32_t idesc = idesc_bf16(MT, N);
    const int nchunks = (a.rows + MT - 1) / MT;
    uint32_t phase = 0;
    bool ok = true, any = false;
    for (int ch = blockIdx.x; ch < nchunks && ok; ch += gridDim.x) {
        const int r0 = ch * MT;
        // A^T: element (feature f, row r) at kmaj_off(f, r, 128); B^T: (n, r) at kmaj_off(n, r, 128)
        stage_rows_T(a.A, a.K, f0, r0, a.rows, sA, MT, tid);
        stage_rows_T(a.B, N, 0, r0, a.rows, sB, N, tid);
        fence_async_smem();
        fence_before();
        __syncthreads();
        fence_after();
        if (tid == 0) {
            const uint32_t sbo = (uint32_t)(MT / 8) * 128;
            for (int k = 0; k < MT / 16; k++) {
                uint64_t da = smem_desc(smem_u32(sA) + (uint32_t)k * 256, 128, sbo);
                uint64_t db = smem_desc(smem_u32(sB) + (uint32_t)k * 256, 128, sbo);
                mma_bf16(tmem, da, db, idesc, any || k > 0);
            }
            mma_commit(&mbar);
        }
        any = true;
        ok = __syncthreads_and(mbar_wait(&mbar, phase)) != 0;
        phase ^= 1u;
        fence_after();
        if (!ok && tid == 0) atomicOr(a.err, 2u);
        fence_before();
        __syncthreads();   // the next chunk's staging overwrites sA, sB
        fence_after();
    }
    if (ok && any) {
        const int f = f0 + warp * 32 + lane;
        for (int c0 = 0; c0 < N; c0 += 16) {
            float v[16];
            tmem_ld16(tmem + ((uint32_t)(warp * 32) << 16) + (uint32_t)c0, v);
            if (f < a.K)
#pragma unroll
                for (int k = 0; k < 16; k++) atomicAdd(&a.C[(size_t)f * a.ldc + c0 + k], v[k]);
        }
    }
    fence_before();
    __syncthreads();
    fence_after();
    if (warp == 0) tmem_dealloc(tmem, ncols);
}

}  // namespace

bool gemm_shape_ok(int K, int N) { return K >= 16 && K <= 256 && K % 16 == 0 && N >= 16 && N <= 256 && N % 16 == 0; }

cudaError_t enqueue_gemm_nt(const void *A1, int K1, const void *A2, int K2, const void *B, int N, int rows,
                            const float *bias, int relu, void *C, int c_bf16, int accumulate, unsigned *err,
                            int max_ctas, cudaStream_t s, int ldc)
{
    NtArgs a{static_cast<const __nv_bfloat16 *>(A1), static_cast<const __nv_bfloat16 *>(A2),
             static_cast<const __nv_bfloat16 *>(B), bias, C, rows, K1, K2, N, relu, c_bf16, accumulate,
             ldc > 0 ? ldc : N, err};
    int K = K1 + K2;
    size_t smem = (size_t)(N + MT) * K * 2;
    cudaError_t e = cudaFuncSetAttribute(k_gemm_nt, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e) return e;
    int tiles = (rows + MT - 1) / MT;
    int g = tiles < max_ctas ? tiles : max_ctas;
    if (g < 1) return cudaSuccess;
    k_gemm_nt<<<g, 128, smem, s>>>(a);
    return cudaGetLastError();
}

cudaError_t enqueue_gemm_tn(const void *A, int K, const void *B, int N, int rows, float *C, unsigned *err,
                            int max_ctas, cudaStream_t s, int ldc)
{
    TnArgs a{static_cast<const __nv_bfloat16 *>(A), static_cast<const __nv_bfloat16 *>(B), C, rows, K, N,
             ldc > 0 ? ldc : N, err};
    size_t smem = (size_t)(MT + N) * MT * 2;
    cudaError_t e = cudaFuncSetAttribute(k_gemm_tn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e) return e;
    int chunks = (rows + MT - 1) / MT;
    int gx = chunks < max_ctas ? chunks : max_ctas;
    if (gx < 1) return cudaSuccess;
    dim3 g(gx, (K + MT - 1) / MT);
    k_gemm_tn<<<g, 128, smem, s>>>(a);
    return cudaGetLastError();
}

}  // namespace ann

namespace {
__device__ unsigned g_gemm_err;   // time-out flags of the stand-alone GEMM entry points
}

extern "C" {

int ann_bf16_gemm(const void *A1, int32_t K1, const void *A2, int32_t K2, const void *B, int32_t N, int64_t rows,
                  const float *bias, int32_t relu, void *C, int32_t c_bf16, int32_t accumulate, void *stream)
{
    if (!A1 || !B || !C || rows < 0 || rows > (1ll << 30) || K1 < 16 || K1 % 16 || K2 < 0 || K2 % 16 ||
        (K2 > 0 && !A2) || !ann::gemm_shape_ok(K1 + K2, N) || (relu != 0 && relu != 1) || (c_bf16 != 0 && c_bf16 != 1) ||
        (accumulate != 0 && accumulate != 1) || (accumulate && c_bf16) ||
        ((reinterpret_cast<uintptr_t>(A1) | reinterpret_cast<uintptr_t>(A2) | reinterpret_cast<uintptr_t>(B) |
          reinterpret_cast<uintptr_t>(C)) & 15))
        return ANN_ERR_INVALID_ARG;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    unsigned *err = nullptr, zero = 0, h = 0;
    cudaError_t e = cudaGetSymbolAddress((void **)&err, g_gemm_err);
    if (!e) e = cudaMemcpyAsync(err, &zero, sizeof zero, cudaMemcpyHostToDevice, s);
    if (!e) e = ann::enqueue_gemm_nt(A1, K1, A2, K2, B, N, (int)rows, bias, relu, C, c_bf16, accumulate, err, 296, s);
    if (!e) e = cudaMemcpyAsync(&h, err, sizeof h, cudaMemcpyDeviceToHost, s);
    if (!e) e = cudaStreamSynchronize(s);
    if (e) return e == cudaErrorMemoryAllocation ? ANN_ERR_OOM : ANN_ERR_CUDA;
    return h ? ANN_ERR_CUDA : ANN_OK;
}

int ann_bf16_gemm_tn(const void *A, int32_t K, const void *B, int32_t N, int64_t rows, float *C, void *stream)
{
    if (!A || !B || !C || rows < 0 || rows > (1ll << 30) || K < 1 || K > 256 || !ann::gemm_shape_ok(16, N))
        return ANN_ERR_INVALID_ARG;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    unsigned *err = nullptr, zero = 0, h = 0;
    cudaError_t e = cudaGetSymbolAddress((void **)&err, g_gemm_err);
    if (!e) e = cudaMemcpyAsync(err, &zero, sizeof zero, cudaMemcpyHostToDevice, s);
    if (!e) e = ann::enqueue_gemm_tn(A, K, B, N, (int)rows, C, err, 296, s);
    if (!e) e = cudaMemcpyAsync(&h, err, sizeof h, cudaMemcpyDeviceToHost, s);
    if (!e) e = cudaStreamSynchronize(s);
    if (e) return e == cudaErrorMemoryAllocation ? ANN_ERR_OOM : ANN_ERR_CUDA;
    return h ? ANN_ERR_CUDA : ANN_OK;
}

}  // extern "C"

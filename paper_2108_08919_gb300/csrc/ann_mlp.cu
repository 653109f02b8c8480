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
#include <cudaTypedefs.h>

#include <cstring>

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

// Descriptor of a K-major operand in a swizzled layout: rows of `span` bytes (128, 64 or 32: one
// TMA box row), 16-byte chunk j of row r stored at chunk j ^ ((r * span / 128) mod (span / 16)),
// 8-row groups `8 span` bytes apart (SBO), the leading offset unused.  Atoms are 1024-byte aligned.
__device__ __forceinline__ uint64_t smem_desc_sw(uint32_t addr, uint32_t span)
{
    const uint64_t mode = span == 128 ? 2u : (span == 64 ? 4u : 6u);   // SWIZZLE_128B / 64B / 32B
    uint64_t d = 0;
    d |= (uint64_t)((addr >> 4) & 0x3FFFu);
    d |= (uint64_t)1 << 16;                                  // LBO (unused): 16 bytes
    d |= (uint64_t)(((8u * span) >> 4) & 0x3FFFu) << 32;     // SBO
    d |= (uint64_t)1 << 46;                                  // version
    d |= mode << 61;
    return d;
}

// Byte offset of 16-byte chunk j of row r in a swizzled box with rows of `span` bytes.
__device__ __forceinline__ uint32_t sw_off(int r, int j, uint32_t span)
{
    const int x = span == 128 ? (r & 7) : (span == 64 ? ((r >> 1) & 3) : ((r >> 2) & 1));
    return (uint32_t)r * span + ((uint32_t)(j ^ x) << 4);
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
__device__ __forceinline__ bool mbar_wait(uint64_t *mbar, uint32_t parity, unsigned limit = SPIN_LIMIT)
{
    uint32_t a = smem_u32(mbar);
    for (unsigned it = 0; it < limit; it++) {
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

// 16 consecutive FP32 columns of this thread's TMEM lane, without waiting: the registers are valid
// after tmem_ld_wait().
__device__ __forceinline__ void tmem_ld16_async(uint32_t taddr, uint32_t *r)
{
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
          "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
        : "r"(taddr));
}

__device__ __forceinline__ void tmem_ld_wait() { asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory"); }

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
// layer: one message-passing layer per 128-row tile, two chained MMAs with the hidden activation
// kept on chip:
//   h = relu([A1 | A2] . W^T + bw)    (128 x 128 FP32 in TMEM; BF16 copy into shared memory as the
//                                      next MMA's A operand, optionally stored to H)
//   z = h . P^T (+ bp)                (128 x Np in TMEM; stored to Z, BF16 or FP32)
// One persistent CTA per SM, warp-specialised: lane 0 of warp 8 loads A tiles by TMA into a ring
// of `stages` buffers and issues the MMAs; warps 0-7 run the epilogues.  The accumulators are
// double-buffered in TMEM (buffer b = tile mod 2 at columns 256 b: h at +0, z at +128), as is the
// z staging tile in shared memory, so that the products of one tile overlap the epilogues of the
// previous one; the h staging tile is single (its space buys a third A stage at K = 160, which
// keeps two tiles' loads in flight).  Hand-offs are mbarriers:
//   full[s]      TMA bytes of stage s landed          -> MMA of h
//   empty[s]     MMA of h has read stage s            -> next TMA into s
//   acc1_full[b] h accumulated                         -> epilogue 1
//   h_full[b]    BF16 h written to shared memory       -> MMA of z
//   acc2_full[b] z accumulated (h no longer read)      -> epilogue 2
//   acc_empty[b] both accumulators of b read           -> MMA of h two tiles later
// TMA boxes are 128 rows high and 128 bytes wide (64 columns), or the whole row where a part is
// only 32 or 64 bytes wide, and land in the matching swizzled K-major layout (16-byte chunks of a
// row XOR-permuted by the row within its 8-row group), which the MMA descriptors name; the epilogue
// writes h and z in the same layouts and TMA stores them.  Rows past the end are zero-filled on
// load and clipped on store.  Epilogue warp w reads TMEM lanes 32 (w mod 4) .. + 31 (tile rows) and half
// of the columns.  Every wait is bounded; the epilogue warps take each wait's outcome together
// (a barrier reduction), so a time-out ends all of them at the same tile.
// ------------------------------------------------------------------------------------------------

struct LayerMaps {
    CUtensorMap a1, a2, h, z;   // A1 rows x K1, A2 rows x K2, H rows x 128, Z rows x Np
};

struct LayerArgs {
    const __nv_bfloat16 *W;   // 128 x K
    const float *bw;          // 128
    const __nv_bfloat16 *P;   // Np x 128
    const float *bp;          // Np or null
    int rows, K1, K2, Np, z_bf16, store_h, stages;
    unsigned *err;
};

constexpr int HW = 128;          // hidden width of a layer
constexpr int EPI = 256;         // epilogue threads (warps 0-7)
constexpr int LT = EPI + 32;     // + the TMA / MMA warp
constexpr int NSMAX = 4;         // A stages at most

// Row span in bytes of the boxes of a part of C BF16 columns (or FP32 when es = 4): 128 (boxes of
// 64 columns) when C is a multiple of 64, else the whole row of 32 or 64 bytes.
__host__ __device__ constexpr uint32_t part_span(int C, int es = 2)
{
    return (uint32_t)(C * es >= 128 ? 128 : C * es);
}

__device__ __forceinline__ void tma_load_2d(uint32_t dst, const CUtensorMap *map, int x, int y, uint32_t mbar)
{
    asm volatile(
        "cp.async.bulk.tensor.2d.shared::cluster.global.tile.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3}], [%4];" ::
            "r"(dst), "l"(reinterpret_cast<uint64_t>(map)), "r"(x), "r"(y), "r"(mbar)
        : "memory");
}

__device__ __forceinline__ void tma_store_2d(const CUtensorMap *map, int x, int y, uint32_t src)
{
    asm volatile("cp.async.bulk.tensor.2d.global.shared::cta.tile.bulk_group [%0, {%1, %2}], [%3];" ::"l"(
                     reinterpret_cast<uint64_t>(map)),
                 "r"(x), "r"(y), "r"(src)
                 : "memory");
}

__device__ __forceinline__ void mbar_expect(uint64_t *mbar, uint32_t bytes)
{
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(mbar)), "r"(bytes) : "memory");
}

__device__ __forceinline__ void mbar_arrive(uint64_t *mbar)
{
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(mbar)) : "memory");
}

// AND of v over the 256 epilogue threads (named barrier 1); also a barrier among them.
__device__ __forceinline__ bool epi_all(bool v)
{
    uint32_t r;
    asm volatile(
        "{\n\t.reg .pred p, q;\n\tsetp.ne.u32 p, %1, 0;\n\tbar.red.and.pred q, 1, 256, p;\n\tselp.u32 %0, 1, 0, q;\n\t}"
        : "=r"(r)
        : "r"((uint32_t)v)
        : "memory");
    return r != 0;
}

__device__ __forceinline__ void epi_sync() { asm volatile("bar.sync 1, 256;" ::: "memory"); }

// The A tile of rows r0.. into stage buffer sA, completing on `full`: part A1 then part A2, each as
// boxes of 128 rows x span bytes (span / 2 columns), one after the other.
__device__ __forceinline__ void layer_load(const LayerMaps &m, int K1, int K2, int r0, uint32_t sA, uint64_t *full)
{
    mbar_expect(full, (uint32_t)MT * (uint32_t)(K1 + K2) * 2u);
    const uint32_t mb = smem_u32(full), s1 = part_span(K1), s2 = part_span(K2);
    uint32_t d = sA;
    for (int c = 0; c < K1; c += (int)s1 / 2, d += MT * s1) tma_load_2d(d, &m.a1, c, r0, mb);
    for (int c = 0; c < K2; c += (int)s2 / 2, d += MT * s2) tma_load_2d(d, &m.a2, c, r0, mb);
}

__global__ void __launch_bounds__(LT, 1) k_layer(const __grid_constant__ LayerMaps maps, LayerArgs a)
{
    extern __shared__ __align__(128) unsigned char sm_raw[];
    __shared__ uint64_t full[NSMAX], empty[NSMAX], acc1_full[2], acc2_full[2], h_full[2], acc_empty[2];
    __shared__ uint32_t tbase;
    __shared__ __align__(16) float sbw[HW], sbp[HW];
    const int K = a.K1 + a.K2, Np = a.Np, NS = a.stages;
    const uint32_t zspan = part_span(Np, a.z_bf16 ? 2 : 4);            // 64 bytes for the widths used here
    const uint32_t zbytes = (uint32_t)MT * (uint32_t)Np * (a.z_bf16 ? 2u : 4u);
    // swizzle atoms want 1024-byte alignment: the launch adds 1 KB of slack
    unsigned char *sm = sm_raw + ((1024u - (smem_u32(sm_raw) & 1023u)) & 1023u);
    unsigned char *sW = sm;                                // 128 x K (no swizzle: LBO 128, SBO 128 K / 8)
    unsigned char *sP = sW + (size_t)HW * K * 2;           // Np x 128 (no swizzle: LBO 128, SBO 2048)
    unsigned char *sH = sP + (size_t)Np * HW * 2;          // 128 x 128: two 128-byte-span boxes
    unsigned char *sZ0 = sH + (size_t)MT * HW * 2;         // 2 x (128 x Np)
    unsigned char *sA0 = sZ0 + (size_t)2 * zbytes;         // NS x (128 x K)
    const size_t abytes = (size_t)MT * K * 2;
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int ntiles = (a.rows + MT - 1) / MT;
    const int mine = (int)blockIdx.x < ntiles ? (ntiles - 1 - (int)blockIdx.x) / (int)gridDim.x + 1 : 0;
    if (warp == 0) tmem_alloc(&tbase, 512);
    if (tid == 0) {
        for (int q = 0; q < NS; q++) {
            mbar_init(&full[q], 1);
            mbar_init(&empty[q], 1);
        }
        for (int b = 0; b < 2; b++) {
            mbar_init(&acc1_full[b], 1);
            mbar_init(&acc2_full[b], 1);
            mbar_init(&h_full[b], EPI);
            mbar_init(&acc_empty[b], EPI);
        }
    }
    for (int e = tid; e < HW * (K / 8); e += LT) {
        int r = e / (K / 8), k8 = (e % (K / 8)) * 8;
        *reinterpret_cast<uint4 *>(sW + kmaj_off(r, k8, K)) = *reinterpret_cast<const uint4 *>(a.W + (size_t)r * K + k8);
    }
    for (int e = tid; e < Np * (HW / 8); e += LT) {
        int r = e / (HW / 8), k8 = (e % (HW / 8)) * 8;
        *reinterpret_cast<uint4 *>(sP + kmaj_off(r, k8, HW)) = *reinterpret_cast<const uint4 *>(a.P + (size_t)r * HW + k8);
    }
    if (tid < HW) {
        sbw[tid] = a.bw[tid];
        sbp[tid] = (a.bp && tid < Np) ? a.bp[tid] : 0.f;
    }
    fence_async_smem();
    fence_before();
    __syncthreads();
    fence_after();
    const uint32_t tmem = tbase;
    if (warp == EPI / 32) {
        if (lane == 0) {
            // TMA and MMA issue.  Order per step i: the product of h for tile i, the load of tile
            // i + NS - 1 (into the stage of tile i - 1), the product of z for tile i - 1.
            const uint32_t idesc1 = idesc_bf16(MT, HW), idesc2 = idesc_bf16(MT, Np);
            const uint32_t sbo_w = (uint32_t)(K / 8) * 128, sbo_p = (uint32_t)(HW / 8) * 128;
            int issued = 0, consumed = 0;
            bool ok = true;
            for (int q = 0; q < NS - 1 && q < mine; q++, issued++)
                layer_load(maps, a.K1, a.K2, (blockIdx.x + q * gridDim.x) * MT, smem_u32(sA0 + (size_t)q * abytes),
                           &full[q]);
            for (int i = 0; i <= mine && ok; i++) {
                if (i < mine) {
                    const int st = i % NS, b = i & 1;
                    ok = mbar_wait(&full[st], (uint32_t)(i / NS) & 1u);
                    if (ok) consumed++;
                    if (ok && i >= 2) ok = mbar_wait(&acc_empty[b], (uint32_t)((i - 2) / 2) & 1u);
                    if (!ok) break;
                    fence_after();
                    // K steps of 16 columns (32 bytes): part A1's boxes, then A2's
                    uint32_t box = smem_u32(sA0 + (size_t)st * abytes);
                    int kk = 0;
                    for (int part = 0; part < 2; part++) {
                        const int C = part ? a.K2 : a.K1;
                        const uint32_t span = part_span(C);
                        for (int c = 0; c < C; c += 16, kk += 16) {
                            const uint32_t in_box = (uint32_t)(c % ((int)span / 2)) * 2;
                            mma_bf16(tmem + (uint32_t)b * 256u, smem_desc_sw(box + in_box, span),
                                     smem_desc(smem_u32(sW) + (uint32_t)(kk / 8) * 128, 128, sbo_w), idesc1, kk > 0);
                            if (in_box + 32 == span) box += MT * span;
                        }
                    }
                    mma_commit(&empty[st]);
                    mma_commit(&acc1_full[b]);
                    const int j = i + NS - 1;
                    if (j < mine) {
                        const int sj = j % NS;
                        if (i >= 1) ok = mbar_wait(&empty[sj], (uint32_t)((i - 1) / NS) & 1u);
                        if (!ok) break;
                        layer_load(maps, a.K1, a.K2, (blockIdx.x + j * gridDim.x) * MT,
                                   smem_u32(sA0 + (size_t)sj * abytes), &full[sj]);
                        issued++;
                    }
                }
                if (i >= 1) {
                    const int j = i - 1, b = j & 1;
                    ok = mbar_wait(&h_full[b], (uint32_t)(j / 2) & 1u);
                    if (!ok) break;
                    fence_after();
                    const uint32_t h0 = smem_u32(sH);
                    for (int k = 0; k < HW / 16; k++)
                        mma_bf16(tmem + (uint32_t)b * 256u + (uint32_t)HW,
                                 smem_desc_sw(h0 + (uint32_t)(k / 4) * MT * 128 + (uint32_t)(k % 4) * 32, 128),
                                 smem_desc(smem_u32(sP) + (uint32_t)k * 256, 128, sbo_p), idesc2, k > 0);
                    mma_commit(&acc2_full[b]);
                }
            }
            if (!ok) atomicOr(a.err, 4u);
            // loads issued for tiles that were not reached (only after a failed wait) land before exit
            for (int q = consumed; q < issued; q++) mbar_wait(&full[q % NS], (uint32_t)(q / NS) & 1u);
        }
        __syncwarp();
    } else {
        const int row = (warp & 3) * 32 + lane, half = warp >> 2;
        const uint32_t lane_base = (uint32_t)((warp & 3) * 32) << 16;
        const bool leader = tid == 0;
        bool ok = true;
        for (int i = 0; i < mine; i++) {
            const int t = blockIdx.x + i * gridDim.x, b = i & 1;
            unsigned char *sZ = sZ0 + (size_t)b * zbytes;
            const uint32_t acc = tmem + (uint32_t)b * 256u + lane_base;
            // stores commit two groups a tile, h then z: once at most the last (z of tile i - 1) is
            // still reading, sH (stored from by tile i - 1) and sZ of buffer b (by tile i - 2) are free
            if (leader && i >= 1) asm volatile("cp.async.bulk.wait_group.read 1;" ::: "memory");
            ok = epi_all(mbar_wait(&acc1_full[b], (uint32_t)(i / 2) & 1u));
            if (!ok) break;
            fence_after();
            // h: bias, relu, BF16 into sH; 64 columns per warp, 32 at a time
            for (int c0 = half * (HW / 2); c0 < (half + 1) * (HW / 2); c0 += 32) {
                uint32_t r[32];
                tmem_ld16_async(acc + (uint32_t)c0, r);
                tmem_ld16_async(acc + (uint32_t)(c0 + 16), r + 16);
                tmem_ld_wait();
                uint4 w[4];
                __nv_bfloat162 *h2 = reinterpret_cast<__nv_bfloat162 *>(w);
#pragma unroll
                for (int k = 0; k < 16; k++) {
                    const float2 bb = *reinterpret_cast<const float2 *>(sbw + c0 + 2 * k);
                    h2[k] = __floats2bfloat162_rn(fmaxf(__uint_as_float(r[2 * k]) + bb.x, 0.f),
                                                  fmaxf(__uint_as_float(r[2 * k + 1]) + bb.y, 0.f));
                }
#pragma unroll
                for (int q = 0; q < 4; q++) {   // chunk j of the 64-column box c0 / 64
                    const int j = (c0 % 64) / 8 + q;
                    *reinterpret_cast<uint4 *>(sH + (size_t)(c0 / 64) * MT * 128 + sw_off(row, j, 128)) = w[q];
                }
            }
            fence_async_smem();
            mbar_arrive(&h_full[b]);
            epi_sync();
            if (leader) {
                if (a.store_h)
                    for (int c = 0; c < HW / 64; c++)
                        tma_store_2d(&maps.h, c * 64, t * MT, smem_u32(sH) + (uint32_t)c * MT * 128);
                asm volatile("cp.async.bulk.commit_group;" ::: "memory");
            }
            ok = epi_all(mbar_wait(&acc2_full[b], (uint32_t)(i / 2) & 1u));
            if (!ok) break;
            fence_after();
            // z (+ bias) into sZ: BF16 blocks of 8 columns or FP32 blocks of 4
            for (int c0 = half * 16; c0 < Np; c0 += 32) {
                uint32_t r[16];
                tmem_ld16_async(acc + (uint32_t)(HW + c0), r);
                tmem_ld_wait();
                float v[16];
#pragma unroll
                for (int k = 0; k < 16; k++) v[k] = __uint_as_float(r[k]) + sbp[c0 + k];
                if (a.z_bf16) {
                    uint4 w[2];
                    __nv_bfloat162 *h2 = reinterpret_cast<__nv_bfloat162 *>(w);
#pragma unroll
                    for (int k = 0; k < 8; k++) h2[k] = __floats2bfloat162_rn(v[2 * k], v[2 * k + 1]);
#pragma unroll
                    for (int q = 0; q < 2; q++)
                        *reinterpret_cast<uint4 *>(sZ + sw_off(row, c0 / 8 + q, zspan)) = w[q];
                } else {
#pragma unroll
                    for (int q = 0; q < 4; q++)
                        *reinterpret_cast<float4 *>(sZ + sw_off(row, c0 / 4 + q, zspan)) =
                            make_float4(v[4 * q], v[4 * q + 1], v[4 * q + 2], v[4 * q + 3]);
                }
            }
            fence_async_smem();
            fence_before();
            mbar_arrive(&acc_empty[b]);
            epi_sync();
            if (leader) {
                tma_store_2d(&maps.z, 0, t * MT, smem_u32(sZ));
                asm volatile("cp.async.bulk.commit_group;" ::: "memory");
            }
        }
        if (!ok && leader) atomicOr(a.err, 4u);
        if (leader) asm volatile("cp.async.bulk.wait_group 0;" ::: "memory");
    }
    fence_before();
    __syncthreads();
    fence_after();
    if (warp == 0) tmem_dealloc(tmem, 512);
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

// Self-test of the bounded wait: one thread polls an mbarrier that nothing completes (a fresh
// barrier's phase 0 never finishes) and, after `limit` polls, raises the flag exactly as an
// expired wait of the tensor-core kernels does.
__global__ void k_wait_probe(unsigned limit, unsigned *err)
{
    __shared__ uint64_t mbar;
    if (threadIdx.x == 0) mbar_init(&mbar, 1);
    __syncthreads();
    if (threadIdx.x == 0 && !mbar_wait(&mbar, 0u, limit)) atomicOr(err, 1u);
}

}  // namespace

cudaError_t enqueue_wait_probe(unsigned limit, unsigned *err, cudaStream_t s)
{
    k_wait_probe<<<1, 32, 0, s>>>(limit, err);
    return cudaGetLastError();
}

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

namespace {

PFN_cuTensorMapEncodeTiled_v12000 tensor_map_encoder()
{
    static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
    if (!fn) {
        void *p = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) ==
                cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            fn = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(p);
    }
    return fn;
}

// 2-D map of a row-major rows x cols matrix with boxes of 128 rows x part_span(cols) bytes, in the
// swizzle mode of that span.
bool row_map(CUtensorMap *m, const void *base, int rows, int cols, bool fp32)
{
    PFN_cuTensorMapEncodeTiled_v12000 enc = tensor_map_encoder();
    if (!enc) return false;
    const int es = fp32 ? 4 : 2;
    const uint32_t span = part_span(cols, es);
    const CUtensorMapSwizzle sw = span == 128 ? CU_TENSOR_MAP_SWIZZLE_128B
                                  : (span == 64 ? CU_TENSOR_MAP_SWIZZLE_64B : CU_TENSOR_MAP_SWIZZLE_32B);
    cuuint64_t dims[2] = {(cuuint64_t)cols, (cuuint64_t)rows};
    cuuint64_t strides[1] = {(cuuint64_t)cols * es};
    cuuint32_t box[2] = {span / (cuuint32_t)es, (cuuint32_t)MT};
    cuuint32_t estr[2] = {1, 1};
    return enc(m, fp32 ? CU_TENSOR_MAP_DATA_TYPE_FLOAT32 : CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2, const_cast<void *>(base),
               dims, strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE, sw, CU_TENSOR_MAP_L2_PROMOTION_L2_128B,
               CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

// Widths a part of a tile may have: whole swizzle rows of 32 or 64 bytes, or 64-column boxes.
bool part_ok(int C, int es = 2) { return C * es == 32 || C * es == 64 || (C * es) % 128 == 0; }

}  // namespace

cudaError_t enqueue_layer(const void *A1, int K1, const void *A2, int K2, const void *W, const float *bw,
                          const void *P, const float *bp, int Np, void *H, void *Z, int z_bf16, int rows,
                          unsigned *err, int max_ctas, cudaStream_t s)
{
    const int K = K1 + K2;
    if (K < 16 || K > 256 || K % 16 || K1 % 16 || K1 < 16 || Np < 16 || Np > 128 || Np % 16 || rows < 0 ||
        (K2 > 0 && !A2) || !part_ok(K1) || (K2 > 0 && !part_ok(K2)) || !part_ok(Np, z_bf16 ? 2 : 4) ||
        (z_bf16 ? 2 : 4) * Np > 128)
        return cudaErrorInvalidValue;
    if (rows == 0) return cudaSuccess;
    LayerMaps maps;
    std::memset(&maps, 0, sizeof maps);
    if (!row_map(&maps.a1, A1, rows, K1, false) || (K2 > 0 && !row_map(&maps.a2, A2, rows, K2, false)) ||
        (H && !row_map(&maps.h, H, rows, HW, false)) || !row_map(&maps.z, Z, rows, Np, !z_bf16))
        return cudaErrorInvalidValue;
    LayerArgs a{static_cast<const __nv_bfloat16 *>(W), bw, static_cast<const __nv_bfloat16 *>(P), bp,
                rows, K1, K2, Np, z_bf16, H ? 1 : 0, 2, err};
    // W, P, an h tile, two z tiles and a ring of 2 to 4 A tiles in at most 216 KB; at least 116 KB,
    // so that one CTA (all 512 TMEM columns) runs per SM
    const size_t zbytes = (size_t)MT * Np * (z_bf16 ? 2 : 4);
    const size_t fixed = ((size_t)HW * K + (size_t)Np * HW + (size_t)MT * HW) * 2 + 2 * zbytes,
                 abytes = (size_t)MT * K * 2;
    size_t room = 216 * 1024 > fixed ? 216 * 1024 - fixed : 0;
    a.stages = (int)(room / abytes);
    if (a.stages > NSMAX) a.stages = NSMAX;
    if (a.stages < 2) a.stages = 2;
    size_t smem = fixed + (size_t)a.stages * abytes + 1024;   // + alignment slack
    if (smem < 116 * 1024) smem = 116 * 1024;
    cudaError_t e = cudaFuncSetAttribute(k_layer, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e) return e;
    static int sms = 0;
    if (!sms) {
        int dev = 0;
        e = cudaGetDevice(&dev);
        if (!e) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
        if (e) return e;
    }
    int tiles = (rows + MT - 1) / MT;
    int g = tiles < sms ? tiles : sms;
    if (max_ctas > 0 && g > max_ctas) g = max_ctas;
    k_layer<<<g, LT, smem, s>>>(maps, a);
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
__device__ unsigned g_gemm_err;    // time-out flags of the stand-alone GEMM entry points
__device__ unsigned g_probe_err;   // flag of ann_check_bounded_wait
}

extern "C" {

int ann_check_bounded_wait(uint32_t spin_limit)
{
    if (spin_limit < 1 || spin_limit > (1u << 20)) return ANN_ERR_INVALID_ARG;
    int ndev = 0;
    if (cudaGetDeviceCount(&ndev) != cudaSuccess || ndev == 0) {
        cudaGetLastError();
        return ANN_ERR_NOT_AVAILABLE;
    }
    unsigned *err = nullptr, zero = 0, h = 0;
    cudaError_t e = cudaGetSymbolAddress((void **)&err, g_probe_err);
    if (!e) e = cudaMemcpy(err, &zero, sizeof zero, cudaMemcpyHostToDevice);
    if (!e) e = ann::enqueue_wait_probe(spin_limit, err, nullptr);
    if (!e) e = cudaMemcpy(&h, err, sizeof h, cudaMemcpyDeviceToHost);
    if (e) return ANN_ERR_CUDA;
    return h ? ANN_ERR_TIMEOUT : ANN_OK;
}

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
    return h ? ANN_ERR_TIMEOUT : ANN_OK;
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
    return h ? ANN_ERR_TIMEOUT : ANN_OK;
}

}  // extern "C"

// sm_103a kernels of the flow diagnostics of the results section (arXiv 2108.08919, §5): fields on
// an M x M grid by Shepard interpolation with the method's kernel (Eq. 18), the kinetic-energy
// spectrum of Eq. 31 by a radix-2 FFT, the vorticity correlation of Eq. 32 along the centre line,
// topological defects as winding numbers of the gridded Q, the mixing of coloured particles, and
// unwrapped positions for pathlines.  None of these run inside a step.
#include "ann_device.cuh"

#include <cmath>

namespace ann {
namespace {

// ------------------------------------------------------------------------------------------------
// Shepard gridding.  Nodes (ix L/M, iy L/M).  Each node gathers from the particles of the 5 x 5
// cells around its own cell in the cell order of the last re-sort: a particle has moved far less
// than one cell since then (a re-sort comes once anything moves half the 0.02 x 3h skin), so every
// particle within 3h of the node is in reach, and the sum runs in a fixed order.
// ------------------------------------------------------------------------------------------------

// Per slot: position relative to the corner of the slot's cell (FP32), and the four fields.
__global__ void k_grid_prep(DevParams P, Bufs b, DiagSrc src, float2 *off, float4 *fld)
{
    int s = blockIdx.x * blockDim.x + threadIdx.x;
    if (s >= P.n) return;
    uint32_t key = b.mkey[s];
    int cx = (int)(key % (uint32_t)P.nc), cy = (int)(key / (uint32_t)P.nc);
    double ox = src.x[s] - b.origin[cx], oy = src.y[s] - b.origin[cy];
    if (ox > 0.5 * P.L) ox -= P.L;   // crossed a face since the re-sort
    else if (ox < -0.5 * P.L) ox += P.L;
    if (oy > 0.5 * P.L) oy -= P.L;
    else if (oy < -0.5 * P.L) oy += P.L;
    off[s] = make_float2((float)ox, (float)oy);
    fld[s] = src.u4 ? src.u4[s] : make_float4(src.ux[s], src.uy[s], src.q11[s], src.q12[s]);
}

constexpr int GRID_TILE = 16;   // a block covers 16 x 16 nodes

__global__ void __launch_bounds__(256) k_grid(DevParams P, Bufs b, int M, const float2 *off, const float4 *fld,
                                              double *grid)
{
    int ix = blockIdx.x * GRID_TILE + (threadIdx.x % GRID_TILE);
    int iy = blockIdx.y * GRID_TILE + (threadIdx.x / GRID_TILE);
    if (ix >= M || iy >= M) return;
    double gx = (double)ix * P.L / M, gy = (double)iy * P.L / M;
    int cx = min((int)(gx * P.inv_cell), P.nc - 1), cy = min((int)(gy * P.inv_cell), P.nc - 1);
    float rx0 = (float)(gx - b.origin[cx]), ry0 = (float)(gy - b.origin[cy]);
    float cellf = (float)P.cell;
    float R2 = (float)P.R2;   // (3h)^2: W vanishes there, so the FP32 test is enough
    float sw = 0.f;
    float4 acc = make_float4(0.f, 0.f, 0.f, 0.f);
    for (int oy = -2; oy <= 2; oy++) {
        int ccy = cy + oy;
        ccy = ccy < 0 ? ccy + P.nc : (ccy >= P.nc ? ccy - P.nc : ccy);
        float ry = ry0 - (float)oy * cellf;
        for (int ox = -2; ox <= 2; ox++) {
            int ccx = cx + ox;
            ccx = ccx < 0 ? ccx + P.nc : (ccx >= P.nc ? ccx - P.nc : ccx);
            float rx = rx0 - (float)ox * cellf;
            int c = ccy * P.nc + ccx;
            uint32_t s0 = b.cell_start[c], s1 = b.cell_start[c + 1];
            for (uint32_t s = s0; s < s1; s++) {
                float2 o = off[s];
                float2 d = make_float2(rx - o.x, ry - o.y);
                float r2 = len2(d);
                if (r2 < R2) {
                    float W = kernel_w<true>(r2, P);
                    float4 f = fld[s];
                    sw += W;
                    acc.x = fmaf(W, f.x, acc.x);
                    acc.y = fmaf(W, f.y, acc.y);
                    acc.z = fmaf(W, f.z, acc.z);
                    acc.w = fmaf(W, f.w, acc.w);
                }
            }
        }
    }
    size_t MM = (size_t)M * M, g = (size_t)iy * M + ix;
    bool any = sw > 0.f;
    grid[g] = any ? (double)acc.x / sw : 0.0;
    grid[MM + g] = any ? (double)acc.y / sw : 0.0;
    grid[2 * MM + g] = any ? (double)acc.z / sw : 0.0;
    grid[3 * MM + g] = any ? (double)acc.w / sw : 0.0;
    grid[4 * MM + g] = (double)sw;
}

// ------------------------------------------------------------------------------------------------
// FFT (FP64, radix 2, M a power of two).  z = ux + i uy is transformed along rows, transposed and
// transformed along rows again; |Z|^2 is symmetric under the transposition as far as the shells
// are concerned (|k| depends on kx^2 + ky^2).  E_n = 1/2 sum_{|k| -> n} |Z(k)|^2 / M^4 equals
// 1/2 sum (|ux_hat|^2 + |uy_hat|^2) with u_hat = fft2(u) / M^2, because Z(k) = Ux(k) + i Uy(k)
// for real ux, uy gives |Z(k)|^2 + |Z(-k)|^2 = 2 (|Ux(k)|^2 + |Uy(k)|^2) and every shell holds
// -k with k.
// ------------------------------------------------------------------------------------------------

__global__ void k_twiddles(int M, double2 *tw)
{
    int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= M / 2) return;
    double s, c;
    sincospi(-2.0 * (double)k / (double)M, &s, &c);   // exp(-2 pi i k / M)
    tw[k] = make_double2(c, s);
}

__device__ __forceinline__ double2 cmul(double2 a, double2 b)
{
    return make_double2(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}

// One row per block: bit-reversed load into shared memory, log2 M butterfly stages, natural store.
// PACK: the input is the real grid pair (ux, uy) packed as ux + i uy.
template <bool PACK>
__global__ void k_fft_rows(int M, int logM, const double2 *in, const double *gx, const double *gy, double2 *out,
                           const double2 *tw)
{
    extern __shared__ double2 row[];
    size_t base = (size_t)blockIdx.x * M;
    for (int i = threadIdx.x; i < M; i += blockDim.x) {
        int r = (int)(__brev((unsigned)i) >> (32 - logM));
        row[r] = PACK ? make_double2(gx[base + i], gy[base + i]) : in[base + i];
    }
    __syncthreads();
    for (int half = 1; half < M; half <<= 1) {
        int stride = M / (2 * half);
        for (int t = threadIdx.x; t < M / 2; t += blockDim.x) {
            int pos = t % half, i = (t / half) * 2 * half + pos, j = i + half;
            double2 a = row[i], w = cmul(row[j], tw[pos * stride]);
            row[i] = make_double2(a.x + w.x, a.y + w.y);
            row[j] = make_double2(a.x - w.x, a.y - w.y);
        }
        __syncthreads();
    }
    for (int i = threadIdx.x; i < M; i += blockDim.x) out[base + i] = row[i];
}

__global__ void k_transpose(int M, const double2 *in, double2 *out)
{
    __shared__ double2 tile[32][33];
    int x = blockIdx.x * 32 + threadIdx.x, y0 = blockIdx.y * 32;
    for (int k = threadIdx.y; k < 32; k += blockDim.y)
        if (x < M && y0 + k < M) tile[k][threadIdx.x] = in[(size_t)(y0 + k) * M + x];
    __syncthreads();
    int xo = blockIdx.y * 32 + threadIdx.x, yo0 = blockIdx.x * 32;
    for (int k = threadIdx.y; k < 32; k += blockDim.y)
        if (xo < M && yo0 + k < M) out[(size_t)(yo0 + k) * M + xo] = tile[threadIdx.x][k];
}

// One block per shell: its modes in increasing index order, a fixed-order tree over the threads.
__global__ void __launch_bounds__(256) k_shell_sum(int M, const double2 *Z, const int *off, const int *modes,
                                                   double *E)
{
    __shared__ double red[256];
    int n = blockIdx.x;
    double acc = 0.0;
    for (int t = off[n] + threadIdx.x; t < off[n + 1]; t += blockDim.x) {
        double2 z = Z[modes[t]];
        acc += z.x * z.x + z.y * z.y;
    }
    red[threadIdx.x] = acc;
    __syncthreads();
    for (int s = 128; s > 0; s >>= 1) {
        if (threadIdx.x < s) red[threadIdx.x] += red[threadIdx.x + s];
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        double m2 = (double)M * (double)M;
        E[n] = 0.5 * red[0] / (m2 * m2);
    }
}

// ------------------------------------------------------------------------------------------------
// Vorticity on the centre row by periodic central differences, and its correlation (Eq. 32).
// ------------------------------------------------------------------------------------------------

__global__ void __launch_bounds__(1024) k_correlation(int M, double L, const double *grid, int all_origins, double *C)
{
    extern __shared__ double om[];
    size_t MM = (size_t)M * M;
    const double *ux = grid, *uy = grid + MM;
    int j0 = M / 2, jm = j0 - 1, jp = (j0 + 1) % M;
    double D2 = 2.0 * (L / M);
    for (int i = threadIdx.x; i < M; i += blockDim.x) {
        int ip = (i + 1) % M, im = (i + M - 1) % M;
        double dvx = (uy[(size_t)j0 * M + ip] - uy[(size_t)j0 * M + im]) / D2;
        double duy = (ux[(size_t)jp * M + i] - ux[(size_t)jm * M + i]) / D2;
        om[i] = dvx - duy;
    }
    __syncthreads();
    for (int k = threadIdx.x; k <= M / 2; k += blockDim.x) {
        if (all_origins) {
            double num = 0.0, den = 0.0;
            for (int i = 0; i < M; i++) {
                num += om[(i + k) % M] * om[i];
                den += om[i] * om[i];
            }
            C[k] = num / den;
        } else {
            int i0 = M / 2;
            C[k] = om[(i0 + k) % M] * om[i0] / (om[i0] * om[i0]);
        }
    }
}

// ------------------------------------------------------------------------------------------------
// Defects: winding number m of (Q11, Q12) around the plaquette with lower-left node (ix, iy), by
// signed crossings of the positive Q11 axis; cross products without fused operations so that the
// integer decision is the plain FP64 one.
// ------------------------------------------------------------------------------------------------

__device__ __forceinline__ int crossing(double a1, double a2, double b1, double b2)
{
    double cr = __dsub_rn(__dmul_rn(a1, b2), __dmul_rn(a2, b1));
    if (a2 <= 0.0 && b2 > 0.0 && cr > 0.0) return 1;
    if (b2 <= 0.0 && a2 > 0.0 && cr < 0.0) return -1;
    return 0;
}

__global__ void k_defects(int M, const double *grid, signed char *map, unsigned long long *counts)
{
    size_t MM = (size_t)M * M;
    size_t g = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (g >= MM) return;
    const double *q1 = grid + 2 * MM, *q2 = grid + 3 * MM;
    int ix = (int)(g % M), iy = (int)(g / M), xp = (ix + 1) % M, yp = (iy + 1) % M;
    size_t v[4] = {(size_t)iy * M + ix, (size_t)iy * M + xp, (size_t)yp * M + xp, (size_t)yp * M + ix};
    int m = 0;
#pragma unroll
    for (int e = 0; e < 4; e++) m += crossing(q1[v[e]], q2[v[e]], q1[v[(e + 1) % 4]], q2[v[(e + 1) % 4]]);
    map[g] = (signed char)m;
    if (m == 1) atomicAdd(&counts[0], 1ull);
    else if (m == -1) atomicAdd(&counts[1], 1ull);
    else if (m != 0) atomicAdd(&counts[2], 1ull);
}

// ------------------------------------------------------------------------------------------------
// Mixing: particles per (bin, colour), bins floor(x G / L) clamped to G - 1 (integer counts, exact).
// Pathlines: unwrapped positions of chosen particle IDs.
// ------------------------------------------------------------------------------------------------

__global__ void k_mix_bins(DevParams P, Bufs b, const unsigned char *colors, int G, int S, unsigned *cnt)
{
    int s = blockIdx.x * blockDim.x + threadIdx.x;
    if (s >= P.n) return;
    int bx = min((int)floor(__ddiv_rn(__dmul_rn(b.sx[s], (double)G), P.L)), G - 1);
    int by = min((int)floor(__ddiv_rn(__dmul_rn(b.sy[s], (double)G), P.L)), G - 1);
    int col = colors[b.sid[s]];
    atomicAdd(&cnt[((size_t)by * G + bx) * S + col], 1u);
}

__global__ void k_inverse(int n, const int *sid, int *inv)
{
    int s = blockIdx.x * blockDim.x + threadIdx.x;
    if (s < n) inv[sid[s]] = s;
}

__global__ void k_unwrap(DevParams P, Bufs b, const int *inv, const long long *ids, int k, double *xy)
{
    int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= k) return;
    long long id = ids[t];
    int s = inv[id];
    int2 im = b.img[id];
    xy[2 * t] = b.sx[s] + (double)im.x * P.L;
    xy[2 * t + 1] = b.sy[s] + (double)im.y * P.L;
}

inline unsigned blocks(size_t n, int t) { return (unsigned)((n + t - 1) / t); }

}  // namespace

cudaError_t enqueue_grid(const DevParams &P, const Bufs &b, DiagSrc src, int M, float2 *off, float4 *fld,
                         double *grid, cudaStream_t s)
{
    k_grid_prep<<<blocks(P.n, 256), 256, 0, s>>>(P, b, src, off, fld);
    dim3 g((M + GRID_TILE - 1) / GRID_TILE, (M + GRID_TILE - 1) / GRID_TILE);
    k_grid<<<g, 256, 0, s>>>(P, b, M, off, fld, grid);
    return cudaGetLastError();
}

cudaError_t enqueue_twiddles(int M, double2 *tw, cudaStream_t s)
{
    k_twiddles<<<blocks(M / 2, 256), 256, 0, s>>>(M, tw);
    return cudaGetLastError();
}

cudaError_t enqueue_spectrum(int M, const double *grid, double2 *z, double2 *zt, const double2 *tw,
                             const int *shell_off, const int *shell_modes, int nshell, double *E, cudaStream_t s)
{
    int logM = 0;
    while ((1 << logM) < M) logM++;
    int th = M / 2 < 512 ? M / 2 : 512;
    size_t smem = sizeof(double2) * (size_t)M;
    cudaError_t e = cudaFuncSetAttribute(k_fft_rows<true>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (!e) e = cudaFuncSetAttribute(k_fft_rows<false>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e) return e;
    size_t MM = (size_t)M * M;
    k_fft_rows<true><<<M, th, smem, s>>>(M, logM, nullptr, grid, grid + MM, z, tw);
    dim3 tb(32, 8), tg((M + 31) / 32, (M + 31) / 32);
    k_transpose<<<tg, tb, 0, s>>>(M, z, zt);
    k_fft_rows<false><<<M, th, smem, s>>>(M, logM, zt, nullptr, nullptr, z, tw);
    k_shell_sum<<<nshell, 256, 0, s>>>(M, z, shell_off, shell_modes, E);
    return cudaGetLastError();
}

cudaError_t enqueue_correlation(int M, double L, const double *grid, int all_origins, double *C, cudaStream_t s)
{
    size_t smem = sizeof(double) * (size_t)M;
    k_correlation<<<1, 1024, smem, s>>>(M, L, grid, all_origins, C);
    return cudaGetLastError();
}

cudaError_t enqueue_defects(int M, const double *grid, signed char *map, unsigned long long *counts, cudaStream_t s)
{
    cudaError_t e = cudaMemsetAsync(counts, 0, 3 * sizeof(unsigned long long), s);
    if (e) return e;
    k_defects<<<blocks((size_t)M * M, 256), 256, 0, s>>>(M, grid, map, counts);
    return cudaGetLastError();
}

cudaError_t enqueue_mixing(const DevParams &P, const Bufs &b, const unsigned char *colors, int G, int S,
                           unsigned *cnt, cudaStream_t s)
{
    cudaError_t e = cudaMemsetAsync(cnt, 0, sizeof(unsigned) * (size_t)G * G * S, s);
    if (e) return e;
    k_mix_bins<<<blocks(P.n, 256), 256, 0, s>>>(P, b, colors, G, S, cnt);
    return cudaGetLastError();
}

cudaError_t enqueue_unwrapped(const DevParams &P, const Bufs &b, int *inv, const long long *ids, int k, double *xy,
                              cudaStream_t s)
{
    k_inverse<<<blocks(P.n, 256), 256, 0, s>>>(P.n, b.sid, inv);
    if (k > 0) k_unwrap<<<blocks(k, 256), 256, 0, s>>>(P, b, inv, ids, k, xy);
    return cudaGetLastError();
}

}  // namespace ann

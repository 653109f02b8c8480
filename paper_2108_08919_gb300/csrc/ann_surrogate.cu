// Learned coarse-step surrogate: a message-passing MLP over the SPH neighbour graph that predicts
// the increments of Q and u over k steps, trained and evaluated on the GPU.  The paper has no
// learned component; the network is the project's.
//
//   features  x_i = (r_i, agg(r)_i - r_i, a k dt / ys_u, m k dt / ys_q, lapQ Gamma K k dt / ys_q,
//             (div u, vort u) k dt), r = (Q11, Q12, ux / us, uy / us), with the tendencies of the
//             last recorded step: acceleration a, projected Q rate m, Laplacian of Q, and the
//             divergence and vorticity of the corrected velocity gradient
//   prediction  (dQ, du) = k dt (m, agg(agg(a))) + (ys_q y0, ys_q y1, ys_u y2, ys_u y3): the
//               explicit increment, with the acceleration SPH-smoothed twice (the mean removes the
//               velocity modes that k dt beyond the explicit viscous limit would amplify), plus
//               the network's correction
//   h1 = relu(W1 [x ; agg(x)] + b1),  z1 = P1 h1,  h2 = relu(W2 [h1 ; agg(z1)] + b2),
//   z2 = P2 h2,  h3 = relu(W3 [h2 ; agg(z2)] + b3),  y = Wo h3 + bo
//   agg(f)_i = (W(0) f_i + sum_j W_ij f_j) / S_i,  S_i = W(0) + sum_j W_ij   (an SPH mean, Eq. 19)
//
// Dense products run on the tensor cores (ann_mlp.cu: BF16 operands, FP32 accumulation);
// activations are stored in BF16, gradients accumulate in FP32, the optimiser (Adam) keeps FP32
// master weights.  On the device the particles are in the cell-sorted order of the context's last
// search, so that neighbour rows gathered by the SPH mean sit close in memory; host inputs and
// outputs are in ID order and are permuted on the way in or out.
#include "../../include/ann.h"
#include "ann_internal.cuh"

#include <cuda_bf16.h>

#include <cmath>
#include <cstring>
#include <string>
#include <vector>

using bf16 = __nv_bfloat16;

namespace ann {
namespace {

constexpr int F0 = 16, WIDTH = 128, MSG = 32, NOUT = 4, NOUTP = 16;
// flat parameter layout: W1 b1 P1 W2 b2 P2 W3 b3 Wo bo
constexpr int O_W1 = 0, O_B1 = O_W1 + WIDTH * 2 * F0, O_P1 = O_B1 + WIDTH, O_W2 = O_P1 + MSG * WIDTH,
              O_B2 = O_W2 + WIDTH * (WIDTH + MSG), O_P2 = O_B2 + WIDTH, O_W3 = O_P2 + MSG * WIDTH,
              O_B3 = O_W3 + WIDTH * (WIDTH + MSG), O_WO = O_B3 + WIDTH, O_BO = O_WO + NOUT * WIDTH,
              NPARAM = O_BO + NOUT;
static_assert(NPARAM == ANN_SG_PARAMS, "parameter count");

struct GraphView {
    const int *nbr;
    const float *W;
    const int *cnt;
    const float *S;
    int n;
    float W0;
};

// The tendencies of the context's last recorded step, into ID order (8 x n, component-major):
// the accelerations are held in the state order (slot g is particle sid[g]), the recorded Q rate
// (2 per slot), Laplacian of Q (2) and velocity gradient (4: xx, xy, yx, yy) in the sorted order of
// that step's search (slot g is particle mid[g]); div u = D_xx + D_yy, vort u = D_yx - D_xy.
__global__ void k_sg_tend_from_ctx(int n, const int *sid, const int *mid, const float *sax, const float *say,
                                   const float *qrate, const float *lap, const float *gu, float *tend)
{
    int g = blockIdx.x * blockDim.x + threadIdx.x;
    if (g >= n) return;
    const size_t N = (size_t)n;
    const int a = sid[g], m = mid[g];
    tend[a] = sax[g];
    tend[N + a] = say[g];
    tend[2 * N + m] = qrate[2 * (size_t)g];
    tend[3 * N + m] = qrate[2 * (size_t)g + 1];
    tend[4 * N + m] = lap[2 * (size_t)g];
    tend[5 * N + m] = lap[2 * (size_t)g + 1];
    const float *d = gu + 4 * (size_t)g;
    tend[6 * N + m] = d[0] + d[3];
    tend[7 * N + m] = d[2] - d[1];
}

// Rows of 4 between the graph's sorted order and ID order: to_id: dst[ids[g]] = src[g] (src row
// stride ld); from_id: dst[g] = src[ids[g]].
__global__ void k_sg_rows_to_id(int n, const int *ids, const float *src, int ld, float *dst)
{
    int g = blockIdx.x * blockDim.x + threadIdx.x;
    if (g >= n) return;
    reinterpret_cast<float4 *>(dst)[ids[g]] = *reinterpret_cast<const float4 *>(src + (size_t)g * ld);
}

__global__ void k_sg_rows_from_id(int n, const int *ids, const float *src, float *dst)
{
    int g = blockIdx.x * blockDim.x + threadIdx.x;
    if (g >= n) return;
    reinterpret_cast<float4 *>(dst)[g] = reinterpret_cast<const float4 *>(src)[ids[g]];
}

__device__ __forceinline__ void fma8_bf16(float *acc, uint4 r, float w)
{
    const __nv_bfloat162 *h = reinterpret_cast<const __nv_bfloat162 *>(&r);
#pragma unroll
    for (int q = 0; q < 4; q++) {
        float2 f = __bfloat1622float2(h[q]);
        acc[2 * q] = fmaf(w, f.x, acc[2 * q]);
        acc[2 * q + 1] = fmaf(w, f.y, acc[2 * q + 1]);
    }
}

__device__ __forceinline__ uint4 pack8_bf16(const float *v, float s)
{
    uint4 r;
    __nv_bfloat162 *h = reinterpret_cast<__nv_bfloat162 *>(&r);
#pragma unroll
    for (int q = 0; q < 4; q++) h[q] = __floats2bfloat162_rn(v[2 * q] * s, v[2 * q + 1] * s);
    return r;
}

// out[i] = agg(in)[i] for rows of C BF16 channels (FP32 sums).  C / (8 V) lanes per particle, each
// gathering V x 16 bytes (8 V channels) of every neighbour row; neighbours are taken four at a time
// so that 4 V row loads per lane are in flight.  Each channel sums in list order whatever V is.
// V = 2 measured best on GB300 at 1M particles (forward 0.76 ms against 0.80 with V = 1 and 0.89
// with V = 4).
#ifndef SG_AGG_V
#define SG_AGG_V 2
#endif
template <int C>
__global__ void __launch_bounds__(256) k_sg_agg(GraphView g, const bf16 *in, bf16 *out)
{
    constexpr int V = (C / 8) % SG_AGG_V == 0 ? SG_AGG_V : 1;   // 16-byte chunks per lane
    constexpr int LP = C / (8 * V);
    const size_t t = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    const int i = (int)(t / LP), q = (int)(t % LP);
    if (i >= g.n) return;
    const uint4 *src = reinterpret_cast<const uint4 *>(in) + q * V;
    const size_t n = (size_t)g.n;
    constexpr int RU = C / 8;   // uint4 per row
    float acc[V][8];
#pragma unroll
    for (int v = 0; v < V; v++)
#pragma unroll
        for (int c = 0; c < 8; c++) acc[v][c] = 0.f;
#pragma unroll
    for (int v = 0; v < V; v++) fma8_bf16(acc[v], __ldg(src + (size_t)i * RU + v), g.W0);
    const int m = g.cnt[i];
    const int *nb = g.nbr + i;
    const float *wp = g.W + i;
    int k = 0;
    for (; k + 4 <= m; k += 4) {
        int j[4];
        float w[4];
        uint4 r[4][V];
#pragma unroll
        for (int u = 0; u < 4; u++) {
            j[u] = __ldg(nb + (k + u) * n);
            w[u] = __ldg(wp + (k + u) * n);
        }
#pragma unroll
        for (int u = 0; u < 4; u++)
#pragma unroll
            for (int v = 0; v < V; v++) r[u][v] = __ldg(src + (size_t)j[u] * RU + v);
#pragma unroll
        for (int u = 0; u < 4; u++)
#pragma unroll
            for (int v = 0; v < V; v++) fma8_bf16(acc[v], r[u][v], w[u]);
    }
    for (; k < m; k++) {
        const int jj = __ldg(nb + k * n);
        const float ww = __ldg(wp + k * n);
#pragma unroll
        for (int v = 0; v < V; v++) fma8_bf16(acc[v], __ldg(src + (size_t)jj * RU + v), ww);
    }
    const float is = 1.f / g.S[i];
#pragma unroll
    for (int v = 0; v < V; v++) reinterpret_cast<uint4 *>(out)[(size_t)i * RU + q * V + v] = pack8_bf16(acc[v], is);
}

// The adjoint of agg: out[j] = W(0)/S_j in[j] + sum_{i in N(j)} W_ij / S_i in[i]; the neighbour
// relation is symmetric, so j's own row lists the i and W_ij.  in: FP32 rows of C channels at row
// stride ld (a multiple of 4, 16-byte aligned rows); C / 8 lanes per particle, 8 channels each.
template <int C>
__global__ void __launch_bounds__(256) k_sg_agg_T(GraphView g, const float *in, int ld, bf16 *out)
{
    constexpr int LP = C / 8;
    const size_t t = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    const int j = (int)(t / LP), q = (int)(t % LP);
    if (j >= g.n) return;
    const size_t n = (size_t)g.n;
    float acc[8];
    auto add = [&](int i, float w) {
        const float4 *p = reinterpret_cast<const float4 *>(in + (size_t)i * ld) + 2 * q;
        float4 a = __ldg(p), b = __ldg(p + 1);
        acc[0] = fmaf(w, a.x, acc[0]);
        acc[1] = fmaf(w, a.y, acc[1]);
        acc[2] = fmaf(w, a.z, acc[2]);
        acc[3] = fmaf(w, a.w, acc[3]);
        acc[4] = fmaf(w, b.x, acc[4]);
        acc[5] = fmaf(w, b.y, acc[5]);
        acc[6] = fmaf(w, b.z, acc[6]);
        acc[7] = fmaf(w, b.w, acc[7]);
    };
#pragma unroll
    for (int c = 0; c < 8; c++) acc[c] = 0.f;
    add(j, g.W0 / g.S[j]);
    const int m = g.cnt[j];
#pragma unroll 4
    for (int k = 0; k < m; k++) {
        const int i = __ldg(g.nbr + k * n + j);
        add(i, __ldg(g.W + k * n + j) / __ldg(g.S + i));
    }
    reinterpret_cast<uint4 *>(out)[(size_t)j * LP + q] = pack8_bf16(acc, 1.f);
}

// dY = 2 (y - t) / (4 n) on the 4 outputs (0 on the padding), and the sum of (y - t)^2.
__global__ void k_sg_loss(int n, const float *Y, const float *T, bf16 *dY, double *loss)
{
    __shared__ double red[256];
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    double s = 0.0;
    if (i < n) {
        float sc = 2.f / (4.f * (float)n);
        for (int c = 0; c < NOUTP; c++) {
            float d = c < NOUT ? Y[(size_t)i * NOUTP + c] - T[(size_t)i * NOUT + c] : 0.f;
            s += (double)d * d;
            dY[(size_t)i * NOUTP + c] = __float2bfloat16(sc * d);
        }
    }
    red[threadIdx.x] = s;
    __syncthreads();
    for (int k = blockDim.x / 2; k > 0; k >>= 1) {
        if (threadIdx.x < k) red[threadIdx.x] += red[threadIdx.x + k];
        __syncthreads();
    }
    if (threadIdx.x == 0) atomicAdd(loss, red[0]);
}

// dA = dH * (H > 0) (relu), dH FP32 with row stride ld, H and dA BF16 with C columns.
__global__ void k_sg_relu_bwd(int n, int C, const float *dH, int ld, const bf16 *H, bf16 *dA)
{
    size_t t = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= (size_t)n * C) return;
    size_t i = t / C, c = t % C;
    float h = __bfloat162float(H[t]);
    dA[t] = __float2bfloat16(h > 0.f ? dH[i * ld + c] : 0.f);
}

// out[c] += sum_i in[i][c] (bias gradients); block: 256 threads over rows, one column per y.
__global__ void k_sg_colsum(int n, int C, const bf16 *in, float *out)
{
    __shared__ float red[256];
    int c = blockIdx.y;
    float s = 0.f;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x)
        s += __bfloat162float(in[(size_t)i * C + c]);
    red[threadIdx.x] = s;
    __syncthreads();
    for (int k = blockDim.x / 2; k > 0; k >>= 1) {
        if (threadIdx.x < k) red[threadIdx.x] += red[threadIdx.x + k];
        __syncthreads();
    }
    if (threadIdx.x == 0) atomicAdd(&out[c], red[0]);
}

// BF16 copies of an R x C FP32 matrix: dst (R x C, rows padded to Rp with zeros) and its
// transpose dstT (C x Rp).
__global__ void k_sg_cast(const float *src, int R, int C, int Rp, bf16 *dst, bf16 *dstT)
{
    int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= Rp * C) return;
    int r = t / C, c = t % C;
    float v = r < R ? src[r * C + c] : 0.f;
    if (dst) dst[r * C + c] = __float2bfloat16(v);
    if (dstT) dstT[c * Rp + r] = __float2bfloat16(v);
}

__global__ void k_sg_adam(float *p, const float *g, float *m, float *v, int count, float lr, float b1, float b2,
                          float eps, float bc1, float bc2)
{
    int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= count) return;
    float gg = g[t];
    float mm = b1 * m[t] + (1.f - b1) * gg, vv = b2 * v[t] + (1.f - b2) * gg * gg;
    m[t] = mm;
    v[t] = vv;
    p[t] -= lr * (mm / bc1) / (sqrtf(vv / bc2) + eps);
}

// The jump: (Q, u) += inc + (ys_q y0, ys_q y1, ys_u y2, ys_u y3), x += k dt (u + u') / 2
// (trapezoid), wrapped with the periodic image count.  Row i is slot i of the context's evaluation
// copy (particle ids[i]); the new state goes straight into the context's state arrays at the same
// slot, with the density unchanged and the accelerations restarting from 0, so the context keeps
// its cell structure and candidate lists.
__global__ void k_sg_jump(int n, const int *ids, const double *x, const double *y, const float4 *u4, const float *dr,
                          const float *Y, const float *inc, float ysq, float ysu, double dtk, double L, Bufs b)
{
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const int id = ids[i];
    float4 s = u4[i];
    const float *yi = Y + (size_t)i * NOUTP;
    const float *ci = inc + (size_t)i * NOUT;
    float ux = s.x + (ci[2] + ysu * yi[2]), uy = s.y + (ci[3] + ysu * yi[3]);
    float q1 = s.z + (ci[0] + ysq * yi[0]);
    float q2 = s.w + (ci[1] + ysq * yi[1]);
    double xn = x[i] + dtk * 0.5 * ((double)s.x + (double)ux);
    double yn = y[i] + dtk * 0.5 * ((double)s.y + (double)uy);
    int kx = (int)floor(xn / L), ky = (int)floor(yn / L);
    xn -= kx * L;
    yn -= ky * L;
    if (xn >= L) xn -= L;   // rounding at the face
    if (yn >= L) yn -= L;
    if (!(xn >= 0.0 && xn < L && yn >= 0.0 && yn < L && isfinite(ux) && isfinite(uy) && isfinite(q1) &&
          isfinite(q2))) {
        atomicOr(b.err, EB_NONFINITE);
        xn = yn = 0.0;
        kx = ky = 0;
    }
    if (kx | ky) {
        b.img[id].x += kx;
        b.img[id].y += ky;
    }
    b.sx[i] = xn;
    b.sy[i] = yn;
    b.sux[i] = ux;
    b.suy[i] = uy;
    b.sq11[i] = q1;
    b.sq12[i] = q2;
    b.sdr[i] = dr[i];
    b.sax[i] = 0.f;
    b.say[i] = 0.f;
    b.sid[i] = id;
}

inline unsigned nb(size_t n, int t = 256) { return (unsigned)((n + t - 1) / t); }

// lanes per particle of k_sg_agg<C>
constexpr int agg_lanes(int C) { return C / (8 * ((C / 8) % SG_AGG_V == 0 ? SG_AGG_V : 1)); }

// Sums over the particles (ID order) of the increments of a checked cycle: |dQ_jump - dQ_plain|^2,
// |dQ_plain|^2, |du_jump - du_plain|^2, |du_plain|^2, one FP64 partial per block (summed on the
// host in block order: deterministic).
__global__ void __launch_bounds__(256) k_sg_guard_sums(int n, const float *const *b, const float *const *j,
                                                       const float *const *p, double *part)
{
    __shared__ double red[4][256];
    const int i = blockIdx.x * 256 + threadIdx.x;
    double v[4] = {0.0, 0.0, 0.0, 0.0};
    if (i < n) {
        for (int c = 0; c < 4; c++) {   // components ux, uy, q11, q12 of the state arrays
            const double b0 = b[c][i], dj = (double)j[c][i] - b0, dp = (double)p[c][i] - b0;
            const int w = c < 2 ? 2 : 0;   // u -> slots 2, 3; Q -> slots 0, 1
            v[w] += (dj - dp) * (dj - dp);
            v[w + 1] += dp * dp;
        }
    }
    for (int q = 0; q < 4; q++) red[q][threadIdx.x] = v[q];
    __syncthreads();
    for (int st = 128; st > 0; st >>= 1) {
        if (threadIdx.x < st)
            for (int q = 0; q < 4; q++) red[q][threadIdx.x] += red[q][threadIdx.x + st];
        __syncthreads();
    }
    if (threadIdx.x < 4) part[4 * blockIdx.x + threadIdx.x] = red[threadIdx.x][0];
}

}  // namespace
}  // namespace ann

using namespace ann;

struct ann_surrogate {
    int64_t nmax = 0;
    int n = 0;
    double us = 1.0, ysq = 1.0, ysu = 1.0;
    int k = 8;                  // steps the network spans
    int vel_corr = 0;           // the jump adds the network's velocity correction
    double gammaK = 0.0;        // Gamma K of the loaded context
    cudaStream_t s = nullptr;
    std::vector<void *> allocs;
    std::string last_err;
    // graph and state in the context's cell-sorted order (row g is particle ids[g]); tend_id and
    // io4 hold ID-ordered tendencies and host rows on their way in or out
    int *nbr = nullptr, *cnt2 = nullptr, *ids = nullptr;
    float *W = nullptr, *S2 = nullptr, *dr = nullptr, *inc = nullptr, *tend_id = nullptr, *io4 = nullptr,
          *agg1 = nullptr;
    double *x = nullptr, *y = nullptr;
    float4 *u4 = nullptr;
    float W0 = 0.f;
    double L = 1.0, dt = 0.0;
    float rho0 = 1.f;
    bool loaded = false;
    // activations (BF16) and outputs
    bf16 *X0, *AX, *H1, *Z1, *AZ1, *H2, *Z2, *AZ2, *H3;
    float *Y, *T;
    // backward scratch
    bf16 *dY, *dA, *dZ;
    float *dH;   // n x 160
    // parameters
    float *p, *g, *m, *v;   // FP32 flat (NPARAM)
    bf16 *W1b, *P1b, *W2b, *P2b, *W3b, *Wob, *W3T, *W2T, *P2T, *P1T, *WoT;
    float *bop;             // bo padded to 16
    double *loss;
    unsigned *err;
    unsigned *ovf;   // the graph export found more than MAXN2H neighbours closer than 2h
    int adam_t = 0;
    // the guard of ann_surrogate_advance (allocated on its first call): three ID-ordered states --
    // before a checked cycle, after its jump, after its plain steps -- and the error partial sums
    struct GuardState {
        double *x = nullptr, *y = nullptr;
        float *f[7] = {};   // ux, uy, q11, q12, drho, ax, ay
    } gs[3];
    double *gpart = nullptr;   // 4 partial sums per block
};

namespace {

template <typename T>
cudaError_t sg_alloc(ann_surrogate *S, T *&ptr, size_t count)
{
    void *p = nullptr;
    cudaError_t e = cudaMalloc(&p, std::max<size_t>(count, 1) * sizeof(T));
    if (e) return e;
    S->allocs.push_back(p);
    ptr = static_cast<T *>(p);
    return cudaMemsetAsync(p, 0, std::max<size_t>(count, 1) * sizeof(T), S->s);
}

int sfail(ann_surrogate *S, int code, const std::string &msg)
{
    if (S) S->last_err = msg;
    return code;
}

int scuda(ann_surrogate *S, cudaError_t e, const char *where)
{
    return sfail(S, e == cudaErrorMemoryAllocation ? ANN_ERR_OOM : ANN_ERR_CUDA,
                 std::string(where) + ": " + cudaGetErrorString(e));
}

// The network's graph (neighbours closer than 2h, the first cnt2 entries of each row).
GraphView view_net(const ann_surrogate *S) { return GraphView{S->nbr, S->W, S->cnt2, S->S2, S->n, S->W0}; }

// BF16 copies (and transposes) of the weights for the next forward / backward pass.
cudaError_t cast_weights(ann_surrogate *S)
{
    cudaStream_t s = S->s;
    k_sg_cast<<<nb(WIDTH * 2 * F0), 256, 0, s>>>(S->p + O_W1, WIDTH, 2 * F0, WIDTH, S->W1b, nullptr);
    k_sg_cast<<<nb(MSG * WIDTH), 256, 0, s>>>(S->p + O_P1, MSG, WIDTH, MSG, S->P1b, S->P1T);
    k_sg_cast<<<nb(WIDTH * (WIDTH + MSG)), 256, 0, s>>>(S->p + O_W2, WIDTH, WIDTH + MSG, WIDTH, S->W2b, S->W2T);
    k_sg_cast<<<nb(MSG * WIDTH), 256, 0, s>>>(S->p + O_P2, MSG, WIDTH, MSG, S->P2b, S->P2T);
    k_sg_cast<<<nb(WIDTH * (WIDTH + MSG)), 256, 0, s>>>(S->p + O_W3, WIDTH, WIDTH + MSG, WIDTH, S->W3b, S->W3T);
    k_sg_cast<<<nb(NOUTP * WIDTH), 256, 0, s>>>(S->p + O_WO, NOUT, WIDTH, NOUTP, S->Wob, S->WoT);
    cudaError_t e = cudaMemsetAsync(S->bop, 0, NOUTP * sizeof(float), s);
    if (!e) e = cudaMemcpyAsync(S->bop, S->p + O_BO, NOUT * sizeof(float), cudaMemcpyDeviceToDevice, s);
    if (!e) e = cudaGetLastError();
    return e;
}

constexpr int GEMM_CTAS = 296;   // two persistent CTAs per SM

// The three layers, each one fused kernel (both products of a layer on the tensor cores, h kept on
// chip), with the SPH means in between; H3 is kept only for a backward pass.
cudaError_t forward(ann_surrogate *S, bool keep_h3)
{
    cudaStream_t s = S->s;
    int n = S->n;
    GraphView g = view_net(S);
    unsigned *err = S->err;
    k_sg_agg<F0><<<nb((size_t)n * agg_lanes(F0)), 256, 0, s>>>(g, S->X0, S->AX);
    cudaError_t e = enqueue_layer(S->X0, F0, S->AX, F0, S->W1b, S->p + O_B1, S->P1b, nullptr, MSG, S->H1, S->Z1, 1,
                                  n, err, GEMM_CTAS, s);
    if (!e) {
        k_sg_agg<MSG><<<nb((size_t)n * agg_lanes(MSG)), 256, 0, s>>>(g, S->Z1, S->AZ1);
        e = enqueue_layer(S->H1, WIDTH, S->AZ1, MSG, S->W2b, S->p + O_B2, S->P2b, nullptr, MSG, S->H2, S->Z2, 1, n,
                          err, GEMM_CTAS, s);
    }
    if (!e) {
        k_sg_agg<MSG><<<nb((size_t)n * agg_lanes(MSG)), 256, 0, s>>>(g, S->Z2, S->AZ2);
        e = enqueue_layer(S->H2, WIDTH, S->AZ2, MSG, S->W3b, S->p + O_B3, S->Wob, S->bop, NOUTP,
                          keep_h3 ? S->H3 : nullptr, S->Y, 0, n, err, GEMM_CTAS, s);
    }
    return e ? e : cudaGetLastError();
}

// Gradients of the mean-squared loss against the targets in S->T (after forward).
cudaError_t backward(ann_surrogate *S)
{
    cudaStream_t s = S->s;
    int n = S->n;
    GraphView g = view_net(S);
    unsigned *err = S->err;
    const int K2 = WIDTH + MSG;
    float *gp = S->g;
    cudaError_t e = cudaMemsetAsync(gp, 0, NPARAM * sizeof(float), s);
    if (!e) e = cudaMemsetAsync(S->loss, 0, sizeof(double), s);
    if (e) return e;
    k_sg_loss<<<nb(n), 256, 0, s>>>(n, S->Y, S->T, S->dY, S->loss);
    // output layer: gWo (rows 0..3 of the 16 x 128 product), gbo
    float *gWo16 = S->dH;   // 16 x 128 scratch, copied below
    e = cudaMemsetAsync(gWo16, 0, NOUTP * WIDTH * sizeof(float), s);
    if (!e) e = enqueue_gemm_tn(S->dY, NOUTP, S->H3, WIDTH, n, gWo16, err, GEMM_CTAS, s);
    if (!e) e = cudaMemcpyAsync(gp + O_WO, gWo16, NOUT * WIDTH * sizeof(float), cudaMemcpyDeviceToDevice, s);
    if (e) return e;
    {
        dim3 gr(64, NOUT);
        k_sg_colsum<<<gr, 256, 0, s>>>(n, NOUTP, S->dY, gp + O_BO);
    }
    // layer 3
    e = enqueue_gemm_nt(S->dY, NOUTP, nullptr, 0, S->WoT, WIDTH, n, nullptr, 0, S->dH, 0, 0, err, GEMM_CTAS, s, K2);
    if (e) return e;
    k_sg_relu_bwd<<<nb((size_t)n * WIDTH), 256, 0, s>>>(n, WIDTH, S->dH, K2, S->H3, S->dA);
    {
        dim3 gr(64, WIDTH);
        k_sg_colsum<<<gr, 256, 0, s>>>(n, WIDTH, S->dA, gp + O_B3);
    }
    e = enqueue_gemm_tn(S->dA, WIDTH, S->H2, WIDTH, n, gp + O_W3, err, GEMM_CTAS, s, K2);
    if (!e) e = enqueue_gemm_tn(S->dA, WIDTH, S->AZ2, MSG, n, gp + O_W3 + WIDTH, err, GEMM_CTAS, s, K2);
    if (!e) e = enqueue_gemm_nt(S->dA, WIDTH, nullptr, 0, S->W3T, K2, n, nullptr, 0, S->dH, 0, 0, err, GEMM_CTAS, s);
    if (e) return e;
    k_sg_agg_T<MSG><<<nb((size_t)n * (MSG / 8)), 256, 0, s>>>(g, S->dH + WIDTH, K2, S->dZ);
    e = enqueue_gemm_tn(S->dZ, MSG, S->H2, WIDTH, n, gp + O_P2, err, GEMM_CTAS, s);
    if (!e) e = enqueue_gemm_nt(S->dZ, MSG, nullptr, 0, S->P2T, WIDTH, n, nullptr, 0, S->dH, 0, 1, err, GEMM_CTAS, s, K2);
    if (e) return e;
    // layer 2
    k_sg_relu_bwd<<<nb((size_t)n * WIDTH), 256, 0, s>>>(n, WIDTH, S->dH, K2, S->H2, S->dA);
    {
        dim3 gr(64, WIDTH);
        k_sg_colsum<<<gr, 256, 0, s>>>(n, WIDTH, S->dA, gp + O_B2);
    }
    e = enqueue_gemm_tn(S->dA, WIDTH, S->H1, WIDTH, n, gp + O_W2, err, GEMM_CTAS, s, K2);
    if (!e) e = enqueue_gemm_tn(S->dA, WIDTH, S->AZ1, MSG, n, gp + O_W2 + WIDTH, err, GEMM_CTAS, s, K2);
    if (!e) e = enqueue_gemm_nt(S->dA, WIDTH, nullptr, 0, S->W2T, K2, n, nullptr, 0, S->dH, 0, 0, err, GEMM_CTAS, s);
    if (e) return e;
    k_sg_agg_T<MSG><<<nb((size_t)n * (MSG / 8)), 256, 0, s>>>(g, S->dH + WIDTH, K2, S->dZ);
    e = enqueue_gemm_tn(S->dZ, MSG, S->H1, WIDTH, n, gp + O_P1, err, GEMM_CTAS, s);
    if (!e) e = enqueue_gemm_nt(S->dZ, MSG, nullptr, 0, S->P1T, WIDTH, n, nullptr, 0, S->dH, 0, 1, err, GEMM_CTAS, s, K2);
    if (e) return e;
    // layer 1
    k_sg_relu_bwd<<<nb((size_t)n * WIDTH), 256, 0, s>>>(n, WIDTH, S->dH, K2, S->H1, S->dA);
    {
        dim3 gr(64, WIDTH);
        k_sg_colsum<<<gr, 256, 0, s>>>(n, WIDTH, S->dA, gp + O_B1);
    }
    e = enqueue_gemm_tn(S->dA, WIDTH, S->X0, F0, n, gp + O_W1, err, GEMM_CTAS, s, 2 * F0);
    if (!e) e = enqueue_gemm_tn(S->dA, WIDTH, S->AX, F0, n, gp + O_W1 + F0, err, GEMM_CTAS, s, 2 * F0);
    return e ? e : cudaGetLastError();
}

int check_err(ann_surrogate *S, const char *where)
{
    unsigned h = 0;
    cudaError_t e = cudaMemcpyAsync(&h, S->err, sizeof h, cudaMemcpyDeviceToHost, S->s);
    if (!e) e = cudaStreamSynchronize(S->s);
    if (e) return scuda(S, e, where);
    if (h) return sfail(S, ANN_ERR_TIMEOUT, std::string(where) + ": a tensor-core wait timed out");
    return ANN_OK;
}

}  // namespace

namespace {

// Copy the state of ctx (ID order) into guard state k.
int guard_get(ann_surrogate *S, ann_ctx *ctx, int k)
{
    auto &g = S->gs[k];
    return ann_get_state(ctx, g.x, g.y, g.f[0], g.f[1], g.f[2], g.f[3], g.f[4], g.f[5], g.f[6], 1);
}

// Give ctx (n particles) the state held in guard state k, with its accelerations.  A context that
// holds no particles or has an error raised is loaded afresh first (ann_set_state clears the
// error bits), then updated.
int guard_put(ann_surrogate *S, ann_ctx *ctx, int k, int64_t n)
{
    auto &g = S->gs[k];
    ann_diag d;
    if (ann_get_diagnostics(ctx, &d) != ANN_OK || d.error_bits != 0u) {
        int st = ann_set_state(ctx, n, g.x, g.y, g.f[0], g.f[1], g.f[2], g.f[3], g.f[4], 1);
        if (st) return st;
    }
    return ann_update_state(ctx, g.x, g.y, g.f[0], g.f[1], g.f[2], g.f[3], g.f[4], g.f[5], g.f[6], 1);
}

}  // namespace

extern "C" {

int ann_surrogate_create(int64_t n_max, ann_surrogate **out)
{
    if (!out || n_max < 1 || n_max > (1ll << 26)) return ANN_ERR_INVALID_ARG;
    *out = nullptr;
    int dev = 0;
    if (cudaGetDeviceCount(&dev) != cudaSuccess || dev == 0) return ANN_ERR_NOT_AVAILABLE;
    ann_surrogate *S = new (std::nothrow) ann_surrogate();
    if (!S) return ANN_ERR_OOM;
    S->nmax = n_max;
    size_t n = (size_t)n_max, K2 = WIDTH + MSG;
    cudaError_t e = cudaStreamCreateWithFlags(&S->s, cudaStreamNonBlocking);
#define SA_(p, c) if (!e) e = sg_alloc(S, S->p, c)
    SA_(nbr, (size_t)MAXN2H * n); SA_(W, (size_t)MAXN2H * n); SA_(dr, n); SA_(cnt2, n); SA_(S2, n);
    SA_(agg1, 2 * n);
    SA_(x, n); SA_(y, n); SA_(u4, n); SA_(inc, 4 * n); SA_(ids, n); SA_(tend_id, 8 * n);
    SA_(io4, 4 * n);
    SA_(X0, n * F0); SA_(AX, n * F0); SA_(H1, n * WIDTH); SA_(Z1, n * MSG); SA_(AZ1, n * MSG);
    SA_(H2, n * WIDTH); SA_(Z2, n * MSG); SA_(AZ2, n * MSG); SA_(H3, n * WIDTH);
    SA_(Y, n * NOUTP); SA_(T, n * NOUT); SA_(dY, n * NOUTP); SA_(dA, n * WIDTH); SA_(dZ, n * MSG);
    SA_(dH, std::max(n * K2, (size_t)NOUTP * WIDTH));
    SA_(p, NPARAM); SA_(g, NPARAM); SA_(m, NPARAM); SA_(v, NPARAM);
    SA_(W1b, WIDTH * 2 * F0); SA_(P1b, MSG * WIDTH); SA_(W2b, WIDTH * K2); SA_(P2b, MSG * WIDTH);
    SA_(W3b, WIDTH * K2); SA_(Wob, NOUTP * WIDTH); SA_(W3T, K2 * WIDTH); SA_(W2T, K2 * WIDTH);
    SA_(P2T, WIDTH * MSG); SA_(P1T, WIDTH * MSG); SA_(WoT, WIDTH * NOUTP); SA_(bop, NOUTP);
    SA_(loss, 1); SA_(err, 1); SA_(ovf, 1);
#undef SA_
    if (!e) e = cudaStreamSynchronize(S->s);
    if (e) {
        int code = e == cudaErrorMemoryAllocation ? ANN_ERR_OOM : ANN_ERR_CUDA;
        ann_surrogate_destroy(S);
        return code;
    }
    *out = S;
    return ANN_OK;
}

void ann_surrogate_destroy(ann_surrogate *S)
{
    if (!S) return;
    if (S->s) cudaStreamSynchronize(S->s);
    for (void *p : S->allocs) cudaFree(p);
    if (S->s) cudaStreamDestroy(S->s);
    delete S;
}

int ann_surrogate_set_params(ann_surrogate *S, const float *params)
{
    if (!S || !params) return ANN_ERR_INVALID_ARG;
    cudaError_t e = cudaMemcpyAsync(S->p, params, NPARAM * sizeof(float), cudaMemcpyHostToDevice, S->s);
    if (!e) e = cudaMemsetAsync(S->m, 0, NPARAM * sizeof(float), S->s);
    if (!e) e = cudaMemsetAsync(S->v, 0, NPARAM * sizeof(float), S->s);
    if (!e) e = cast_weights(S);
    if (!e) e = cudaStreamSynchronize(S->s);
    S->adam_t = 0;
    return e ? scuda(S, e, "ann_surrogate_set_params") : ANN_OK;
}

int ann_surrogate_get_params(ann_surrogate *S, float *params)
{
    if (!S || !params) return ANN_ERR_INVALID_ARG;
    cudaError_t e = cudaMemcpyAsync(params, S->p, NPARAM * sizeof(float), cudaMemcpyDeviceToHost, S->s);
    if (!e) e = cudaStreamSynchronize(S->s);
    return e ? scuda(S, e, "ann_surrogate_get_params") : ANN_OK;
}

int ann_surrogate_set_scales(ann_surrogate *S, double us, double ys_q, double ys_u, int32_t k)
{
    if (!S || !(us > 0.0) || !(ys_q > 0.0) || !(ys_u > 0.0) || !std::isfinite(us) || !std::isfinite(ys_q) ||
        !std::isfinite(ys_u) || k < 1)
        return ANN_ERR_INVALID_ARG;
    S->us = us;
    S->ysq = ys_q;
    S->ysu = ys_u;
    S->k = k;
    return ANN_OK;
}

int ann_surrogate_load(ann_surrogate *S, ann_ctx *ctx, const float *tend)
{
    ann::NvtxRange range("ann_surrogate_load");
    if (!S || !ctx) return ANN_ERR_INVALID_ARG;
    CtxView v;
    int st = ctx_view(ctx, &v);
    if (st) return sfail(S, st, "ann_surrogate_load: context has no particles");
    if (v.P.n > S->nmax) return sfail(S, ANN_ERR_INVALID_ARG, "context has more particles than n_max");
    size_t n = (size_t)v.P.n;
    if (tend) {
        cudaError_t e = cudaMemcpyAsync(S->tend_id, tend, 8 * n * sizeof(float), cudaMemcpyHostToDevice, S->s);
        if (!e) e = cudaStreamSynchronize(S->s);
        if (e) return scuda(S, e, "ann_surrogate_load: tendencies");
    } else {
        if (!v.rec_valid)
            return sfail(S, ANN_ERR_STATE, "the context's last step did not record its tendencies "
                                          "(ann_set_record(ctx, 1), then ann_step)");
        // on the context's stream, ahead of the search that re-sorts the recorded arrays' order
        k_sg_tend_from_ctx<<<nb(n), 256, 0, v.stream>>>((int)n, v.b.sid, v.b.mid, v.b.sax, v.b.say, v.b.rec_qrate,
                                                        v.b.rec_lap, v.b.rec_gu, S->tend_id);
        cudaError_t e = cudaGetLastError();
        if (e) return scuda(S, e, "ann_surrogate_load: tendencies");
    }
    st = ctx_search_present(ctx);
    if (st) return sfail(S, st, "ann_surrogate_load: search");
    ctx_view(ctx, &v);
    S->n = v.P.n;
    S->W0 = v.P.W0;
    S->L = v.P.L;
    S->dt = v.P.dt_d;
    S->rho0 = v.P.rho0;
    S->gammaK = (double)v.P.Gamma * (double)v.P.K;
    const double kdt = S->k * S->dt;
    GraphOut o{S->nbr, S->W, S->ovf, S->cnt2, S->S2, S->x, S->y, S->u4, S->dr, S->ids, S->agg1, S->tend_id, S->X0,
               (float)(1.0 / S->us),
               {(float)(kdt / S->ysu), (float)(kdt / S->ysq), (float)(S->gammaK * kdt / S->ysq), (float)kdt}};
    // the export forms the support means of (u, Q) and a and the network's input rows; its second
    // walk gives the explicit increment k dt (m11, m12, agg(agg(a)))
    cudaError_t e = cudaStreamSynchronize(v.stream);
    if (!e) e = cudaMemsetAsync(S->ovf, 0, sizeof(unsigned), S->s);
    if (!e) e = enqueue_export_graph(v.P, v.b, o, (float)kdt, S->inc, S->s);
    unsigned ovf = 0u;
    if (!e) e = cudaMemcpyAsync(&ovf, S->ovf, sizeof ovf, cudaMemcpyDeviceToHost, S->s);
    if (!e) e = cudaStreamSynchronize(S->s);
    if (e) return scuda(S, e, "ann_surrogate_load");
    if (ovf) return sfail(S, ANN_ERR_NBR_OVERFLOW, "ann_surrogate_load: a particle has more neighbours closer than 2h "
                                                   "than the network's graph holds (64)");
    S->loaded = true;
    return ANN_OK;
}

int ann_surrogate_forward(ann_surrogate *S, float *y)
{
    if (!S) return ANN_ERR_INVALID_ARG;
    if (!S->loaded) return sfail(S, ANN_ERR_STATE, "no graph loaded");
    cudaError_t e = cudaMemsetAsync(S->err, 0, sizeof(unsigned), S->s);
    if (!e) e = forward(S, false);
    if (!e && y) {
        k_sg_rows_to_id<<<nb(S->n), 256, 0, S->s>>>(S->n, S->ids, S->Y, NOUTP, S->io4);
        e = cudaGetLastError();
        if (!e) e = cudaMemcpyAsync(y, S->io4, (size_t)S->n * NOUT * sizeof(float), cudaMemcpyDeviceToHost, S->s);
    }
    if (e) return scuda(S, e, "ann_surrogate_forward");
    return check_err(S, "ann_surrogate_forward");
}

int ann_surrogate_gradients(ann_surrogate *S, const float *target, double *loss, float *grads)
{
    if (!S || !target) return ANN_ERR_INVALID_ARG;
    if (!S->loaded) return sfail(S, ANN_ERR_STATE, "no graph loaded");
    cudaError_t e = cudaMemsetAsync(S->err, 0, sizeof(unsigned), S->s);
    if (!e) e = cudaMemcpyAsync(S->io4, target, (size_t)S->n * NOUT * sizeof(float), cudaMemcpyHostToDevice, S->s);
    if (!e) {
        k_sg_rows_from_id<<<nb(S->n), 256, 0, S->s>>>(S->n, S->ids, S->io4, S->T);
        e = cudaGetLastError();
    }
    if (!e) e = forward(S, true);
    if (!e) e = backward(S);
    double h = 0.0;
    if (!e) e = cudaMemcpyAsync(&h, S->loss, sizeof h, cudaMemcpyDeviceToHost, S->s);
    if (!e && grads) e = cudaMemcpyAsync(grads, S->g, NPARAM * sizeof(float), cudaMemcpyDeviceToHost, S->s);
    if (e) return scuda(S, e, "ann_surrogate_gradients");
    int st = check_err(S, "ann_surrogate_gradients");
    if (loss) *loss = h / (4.0 * S->n);
    return st;
}

int ann_surrogate_adam(ann_surrogate *S, double lr)
{
    if (!S || !(lr > 0.0)) return ANN_ERR_INVALID_ARG;
    S->adam_t++;
    const float b1 = 0.9f, b2 = 0.999f;
    float bc1 = 1.f - std::pow(b1, (float)S->adam_t), bc2 = 1.f - std::pow(b2, (float)S->adam_t);
    k_sg_adam<<<nb(NPARAM), 256, 0, S->s>>>(S->p, S->g, S->m, S->v, NPARAM, (float)lr, b1, b2, 1e-8f, bc1, bc2);
    cudaError_t e = cudaGetLastError();
    if (!e) e = cast_weights(S);
    if (!e) e = cudaStreamSynchronize(S->s);
    return e ? scuda(S, e, "ann_surrogate_adam") : ANN_OK;
}

int ann_surrogate_jump(ann_surrogate *S, ann_ctx *ctx, const float *tend)
{
    ann::NvtxRange range("ann_surrogate_jump");
    if (!S || !ctx) return ANN_ERR_INVALID_ARG;
    const int k = S->k;
    int st = ann_surrogate_load(S, ctx, tend);
    if (st) return st;
    st = ann_surrogate_forward(S, nullptr);
    if (st) return st;
    CtxView v;
    st = ctx_view(ctx, &v);
    if (st) return st;
    k_sg_jump<<<nb(S->n), 256, 0, S->s>>>(S->n, S->ids, S->x, S->y, S->u4, S->dr, S->Y, S->inc, (float)S->ysq,
                                          S->vel_corr ? (float)S->ysu : 0.f, S->dt * k, S->L, v.b);
    cudaError_t e = cudaGetLastError();
    if (!e) e = cudaStreamSynchronize(S->s);
    S->loaded = false;   // the context moves on: the next forward needs a new load
    if (e) return scuda(S, e, "ann_surrogate_jump");
    return ctx_commit_in_place(ctx, k);
}

// He initialisation: every weight matrix drawn N(0, 2 / fan_in) (the output layer at half that
// standard deviation), biases 0.  Normals by Box-Muller from SplitMix64 (Steele, Lea and Flood
// 2014) in counter form: value k of stream `seed` is the mix of seed + (k + 1) * 0x9E3779B97F4A7C15.
int ann_surrogate_init(ann_surrogate *S, uint64_t seed)
{
    if (!S) return ANN_ERR_INVALID_ARG;
    auto mix = [](uint64_t z) {
        z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
        z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
        return z ^ (z >> 31);
    };
    uint64_t ctr = 0;
    auto uni = [&]() {   // uniform in (0, 1], 53 bits
        uint64_t v = mix(seed + (++ctr) * 0x9E3779B97F4A7C15ull);
        return ((v >> 11) + 1) * (1.0 / 9007199254740992.0);
    };
    std::vector<float> p(NPARAM, 0.f);
    struct M { int off, rows, cols; double gain; };
    // the output layer starts at zero: an untrained network predicts the explicit increment, and
    // training moves it only as far as the data pull (a random output layer starts the prediction
    // tens of percent off, and in the developed flow it never came back on held-out trajectories)
    const M ms[] = {{O_W1, WIDTH, 2 * F0, 1.0}, {O_P1, MSG, WIDTH, 1.0}, {O_W2, WIDTH, WIDTH + MSG, 1.0},
                    {O_P2, MSG, WIDTH, 1.0}, {O_W3, WIDTH, WIDTH + MSG, 1.0}};
    for (const M &m : ms) {
        double sd = m.gain * std::sqrt(2.0 / m.cols);
        for (int k = 0; k < m.rows * m.cols; k++) {
            double u1 = uni(), u2 = uni();
            p[(size_t)m.off + k] = (float)(sd * std::sqrt(-2.0 * std::log(u1)) * std::cos(6.283185307179586 * u2));
        }
    }
    return ann_surrogate_set_params(S, p.data());
}

int ann_surrogate_euler(ann_surrogate *S, float *inc)
{
    if (!S || !inc) return ANN_ERR_INVALID_ARG;
    if (!S->loaded) return sfail(S, ANN_ERR_STATE, "no graph loaded");
    k_sg_rows_to_id<<<nb(S->n), 256, 0, S->s>>>(S->n, S->ids, S->inc, NOUT, S->io4);
    cudaError_t e = cudaGetLastError();
    if (!e) e = cudaMemcpyAsync(inc, S->io4, (size_t)S->n * NOUT * sizeof(float), cudaMemcpyDeviceToHost, S->s);
    if (!e) e = cudaStreamSynchronize(S->s);
    return e ? scuda(S, e, "ann_surrogate_euler") : ANN_OK;
}

int ann_surrogate_advance(ann_surrogate *S, ann_ctx *ctx, ann_ctx *shadow, int32_t cycles, int32_t check_every,
                          double tol, ann_guard_report *rep)
{
    ann::NvtxRange range("ann_surrogate_advance");
    if (!S || !ctx || !rep || cycles < 0 || check_every < 0 || !(tol > 0.0)) return ANN_ERR_INVALID_ARG;
    if (check_every > 0 && (!shadow || shadow == ctx)) return ANN_ERR_INVALID_ARG;
    CtxView v;
    int st = ctx_view(ctx, &v);
    if (st) return st;
    const int64_t n = v.P.n;
    const int rec0 = v.P.record;
    if (n > S->nmax) return sfail(S, ANN_ERR_INVALID_ARG, "the context holds more particles than the network's n_max");
    if (check_every > 0) {
        CtxView w;
        st = ctx_view(shadow, &w);
        if (st == ANN_ERR_STATE) st = ANN_OK;   // a shadow without particles is loaded at the first check
        if (st) return st;
    }
    cudaError_t e = cudaSuccess;
    if (!S->gpart) {
        for (int k = 0; k < 3 && !e; k++) {
            e = sg_alloc(S, S->gs[k].x, (size_t)S->nmax);
            if (!e) e = sg_alloc(S, S->gs[k].y, (size_t)S->nmax);
            for (int c = 0; c < 7 && !e; c++) e = sg_alloc(S, S->gs[k].f[c], (size_t)S->nmax);
        }
        if (!e) e = sg_alloc(S, S->gpart, 4 * (size_t)nb((int)S->nmax));
        if (e) return scuda(S, e, "ann_surrogate_advance buffers");
    }
    *rep = ann_guard_report{};
    rep->fallback_cycle = -1;
    const int k = S->k;
    int result = ANN_OK;
    for (int32_t c = 0; c < cycles; c++) {
        const bool check = check_every > 0 && c % check_every == 0;
        if (check) {
            st = guard_get(S, ctx, 0);
            if (!st) st = guard_put(S, shadow, 0, n);
            if (st) { result = st; break; }
        }
        // the cycle: one recorded plain step, then the jump over k steps
        st = ann_set_record(ctx, 1);
        if (!st) st = ann_step(ctx, 1);
        if (st) { result = st; break; }
        st = ann_surrogate_jump(S, ctx, nullptr);
        const bool bad_jump = st == ANN_ERR_NONFINITE;
        if (st && !bad_jump) { result = st; break; }
        if (!check) {
            if (bad_jump) { result = st; break; }
            rep->cycles_done++;
            continue;
        }
        // the same cycle in plain SPH on the shadow, and the relative errors of the increments
        st = ann_step(shadow, 1 + k);
        if (!st) st = guard_get(S, shadow, 2);
        if (st) { result = st; break; }
        double eq = INFINITY, eu = INFINITY;
        if (!bad_jump) {
            st = guard_get(S, ctx, 1);
            if (st) { result = st; break; }
            const float *b[4] = {S->gs[0].f[0], S->gs[0].f[1], S->gs[0].f[2], S->gs[0].f[3]};
            const float *j[4] = {S->gs[1].f[0], S->gs[1].f[1], S->gs[1].f[2], S->gs[1].f[3]};
            const float *pl[4] = {S->gs[2].f[0], S->gs[2].f[1], S->gs[2].f[2], S->gs[2].f[3]};
            const float **dptr = nullptr;
            const int nbk = nb((int)n);
            // the three sets of four component pointers travel as a small device array
            e = cudaMalloc(&dptr, 12 * sizeof(float *));
            if (!e) {
                const float *hp[12] = {b[0], b[1], b[2], b[3], j[0], j[1], j[2], j[3], pl[0], pl[1], pl[2], pl[3]};
                e = cudaMemcpyAsync(dptr, hp, sizeof hp, cudaMemcpyHostToDevice, S->s);
                if (!e) k_sg_guard_sums<<<nbk, 256, 0, S->s>>>((int)n, dptr, dptr + 4, dptr + 8, S->gpart);
                if (!e) e = cudaGetLastError();
                std::vector<double> h(4 * (size_t)nbk);
                if (!e) e = cudaMemcpyAsync(h.data(), S->gpart, sizeof(double) * h.size(), cudaMemcpyDeviceToHost, S->s);
                if (!e) e = cudaStreamSynchronize(S->s);
                cudaFree(dptr);
                if (!e) {
                    double sums[4] = {0.0, 0.0, 0.0, 0.0};
                    for (int q = 0; q < nbk; q++)
                        for (int t = 0; t < 4; t++) sums[t] += h[4 * (size_t)q + t];
                    auto rel = [](double num, double den) { return den > 0.0 ? std::sqrt(num / den) : (num > 0.0 ? INFINITY : 0.0); };
                    eq = rel(sums[0], sums[1]);
                    eu = rel(sums[2], sums[3]);
                }
            }
            if (e) { result = scuda(S, e, "ann_surrogate_advance check"); break; }
        }
        rep->checks++;
        rep->last_err_q = eq;
        rep->last_err_u = eu;
        rep->max_err_q = std::max(rep->max_err_q, eq);
        rep->max_err_u = std::max(rep->max_err_u, eu);
        if (!(eq <= tol && eu <= tol)) {
            // fall back: the context takes the plain result of this cycle, and the remaining cycles
            // run as plain steps
            int64_t steps_before = 0;
            {
                CtxView w;
                if (!ctx_view(ctx, &w)) steps_before = w.steps;
            }
            ann_diag d;
            const bool broken = ann_get_diagnostics(ctx, &d) != ANN_OK || d.error_bits != 0u;
            st = guard_put(S, ctx, 2, n);
            if (!st && broken) st = ctx_commit_in_place(ctx, steps_before);   // ann_set_state restarted t and the count
            if (st) { result = st; break; }
            rep->fell_back = 1;
            rep->fallback_cycle = c;
            const int64_t plain = (int64_t)(cycles - c - 1) * (1 + k);
            st = ann_set_record(ctx, rec0);
            if (!st) st = ann_step(ctx, plain);
            rep->plain_steps = plain;
            return st;
        }
        rep->cycles_done++;
    }
    int st2 = ann_set_record(ctx, rec0);
    return result ? result : st2;
}

int ann_surrogate_set_velocity_correction(ann_surrogate *S, int32_t on)
{
    if (!S || (on != 0 && on != 1)) return ANN_ERR_INVALID_ARG;
    S->vel_corr = on;
    return ANN_OK;
}

const char *ann_surrogate_last_error(ann_surrogate *S) { return S ? S->last_err.c_str() : ""; }

}  // extern "C"

// Three-dimensional variant of the SPH active-nematic step (the paper's equations for d = 3):
// a periodic cube, Q as the symmetric traceless 3x3 tensor (Q11, Q12, Q13, Q22, Q23), the corrected
// SPH operators with a 3x3 correction tensor, the viscous term with 2 (d + 2) nu = 10 nu.
//
// One step (modified Euler, §3.1), all on the device, one thread per particle:
//   predict     u += dt/2 a, r += dt/2 u (wrap), max |u|; the re-sort test (a particle has moved
//               half the skin since the last re-sort)
//   re-sort only: cell keys and counts, scan (one block), scatter, each cell's slots sorted by
//               particle ID (deterministic), gather into the new order (buffer set M), candidate
//               lists: every j within 3h (1 + skin) in the 27 surrounding cells
//   filter      neighbour lists (|r_i - r_j| < 3h among the candidates; FP32 test, FP64 in a band
//               around 3h), sum W, V = 1 / sum W (Eq. 19)
//   pass 1      alpha (Eq. 22) and B = alpha^-1, continuity k (Eq. 25), rho_half, corrected
//               velocity gradient (Eq. 20), corrected Laplacian of Q (Eq. 21), Q rate m (Eqs. 2, 7,
//               24), Q^{n+1}: one walk of the neighbours, B applied to the sums afterwards
//   pass 2      density filter (Eq. 28), equation of state (Eq. 26) with c0 = max(10 max|u|, c0_min)
//   pass 3      momentum (Eq. 23), artificial displacement (Eq. 29), corrector; the new state is
//               written into buffer set S in the new order
// The state lives in S between steps, in the cell order of the last step.  Errors are sticky bits
// set by the kernels' own checks (neighbour overflow, non-finite state, singular alpha).  The pair
// loops read each neighbour through a few 16-byte loads of packed per-particle records, written by
// the kernel that produces them.
#include "../../include/ann.h"

#include <cuda_runtime.h>
#include <nvtx3/nvToolsExt.h>

#include <cmath>
#include <cstring>
#include <new>
#include <string>
#include <vector>

namespace {

constexpr int MAXN3 = ANN3_MAX_NEIGHBORS;
constexpr int MAXC3 = 576;          // candidates: neighbours within 3h (1 + SKIN3) at the last re-sort
static_assert(MAXN3 % 4 == 0 && MAXC3 % 4 == 0, "lists are whole int4 words");
constexpr double SKIN3 = 0.05;      // candidate lists stay valid while no particle moves SKIN3 3h / 2
constexpr uint32_t E3_NBR = 4u, E3_NONFINITE = 8u, E3_ALPHA = 16u;

struct P3 {
    int n, nc, ncell;
    double L, inv_cell, cell, R2d, half_dt_d;
    float h, inv_h, ad, adh, W0, dt, half_dt, cell_f, R2lo, R2hi, R2c;
    double skin_max2;
    float rho0, nu, Gamma, lambda, A, B, C, K, zeta, gamma_eos, beta, c0_min, c_shift;
    int apd;
};

struct Set3 {   // one buffer set of the state
    double *x, *y, *z;
    float *u[3], *q[5], *dr, *a[3];   // dr: density deviation rho / rho0 - 1 (FP32 keeps its digits)
    int *id;
    float4 *xi;   // (gathered set only) position relative to the corner of the particle's cell, FP32;
                  // w holds the bits of cxyz, so one load gives a neighbour's geometry
    int *cxyz;    // (gathered set only) cell coordinates cx | cy << 10 | cz << 20
};

// Neighbour and candidate lists: entry k of particle i is component k % 4 of the int4 word
// list[(k / 4) n + i], so a warp reads 32 consecutive words per load and a thread four entries.
struct Work3 {
    int *key, *slot, *perm, *count, *start, *nnbr, *ncand;
    int4 *nbr, *cand;
    double *xr, *yr, *zr;   // positions at the last re-sort (sorted order)
    unsigned *flag;         // non-zero: this step re-sorts and rebuilds the candidate lists
    unsigned *rebuilds;
    float *sumW, *V, *B, *k, *dh, *dhat, *p, *qn, *an, *gu, *lap, *m;   // dh, dhat: deviations of rho_half, rho_hat
    // what the pair loops read of a neighbour j, packed so that one 16-byte load brings four values:
    float4 *vu;    // (V, u) at the midpoint                                     written by the filter
    float4 *q4;    // (Q11, Q12, Q13, Q22) of the midpoint state (Q23: M.q[4])   written by the filter
    float4 *vpu;   // (V, p / rho_hat^2, u_x, u_y)                               written by pass 2
    float4 *uqn;   // (u_z, Q^{n+1}_11, Q^{n+1}_12, Q^{n+1}_13)                   written by pass 1
    float2 *qn2;   // (Q^{n+1}_22, Q^{n+1}_23)                                   written by pass 1
    unsigned *umax, *err;
};

__device__ __forceinline__ double min_image(double d, double L)
{
    if (d > 0.5 * L) d -= L;
    else if (d < -0.5 * L) d += L;
    return d;
}

__device__ __forceinline__ double wrap(double v, double L)
{
    double w = v - L * floor(v / L);
    if (w >= L) w -= L;
    if (w < 0.0) w = 0.0;
    return w;
}

__device__ __forceinline__ int cell_step(int dc, int nc) { return dc > 1 ? dc - nc : (dc < -1 ? dc + nc : dc); }

struct Here3 {   // particle i's own data for its pair loop
    float4 xi;
    int cx, cy, cz;
};

__device__ __forceinline__ Here3 here_of(const Set3 &M, int i)
{
    Here3 h;
    h.xi = M.xi[i];
    int c = M.cxyz[i];
    h.cx = c & 1023;
    h.cy = (c >> 10) & 1023;
    h.cz = c >> 20;
    return h;
}

// Pair geometry of i and j: d = r_i - r_j, |d|^2, 1/|d| and |d|.  d is taken from the FP32
// positions relative to each particle's cell corner and the (periodic) cell offset, which is -1, 0
// or 1 cell per axis for neighbours: d = xi_i - xi_j + (c_i - c_j) cell.  The cell-local offsets
// carry the FP64 positions to about 1e-9 (cells of side ~0.04 L), so d is good to ~1e-7 relative.
struct Geo3 {
    float d[3], r2, rinv, r;
};

__device__ __forceinline__ Geo3 geo_of(const P3 &P, const Here3 &h, const float4 xj)
{
    Geo3 g;
    const int cj = __float_as_int(xj.w);
    g.d[0] = (h.xi.x - xj.x) + (float)cell_step(h.cx - (cj & 1023), P.nc) * P.cell_f;
    g.d[1] = (h.xi.y - xj.y) + (float)cell_step(h.cy - ((cj >> 10) & 1023), P.nc) * P.cell_f;
    g.d[2] = (h.xi.z - xj.z) + (float)cell_step(h.cz - (cj >> 20), P.nc) * P.cell_f;
    g.r2 = g.d[0] * g.d[0] + g.d[1] * g.d[1] + g.d[2] * g.d[2];
    g.rinv = rsqrtf(g.r2);
    g.r = g.r2 * g.rinv;
    return g;
}

// Quintic kernel (Eq. 18) times the 3D constant: W(r), and F with grad_i W = F d (F = W'(r) / r).
__device__ __forceinline__ float w3(const P3 &P, const Geo3 &g)
{
    const float b = g.r * P.inv_h;
    const float t3 = fmaxf(3.f - b, 0.f), t2 = fmaxf(2.f - b, 0.f), t1 = fmaxf(1.f - b, 0.f);
    const float s3 = t3 * t3, s2 = t2 * t2, s1 = t1 * t1;
    return P.ad * (s3 * s3 * t3 - 6.f * s2 * s2 * t2 + 15.f * s1 * s1 * t1);
}

__device__ __forceinline__ float f3(const P3 &P, const Geo3 &g)
{
    const float b = g.r * P.inv_h;
    const float t3 = fmaxf(3.f - b, 0.f), t2 = fmaxf(2.f - b, 0.f), t1 = fmaxf(1.f - b, 0.f);
    const float s3 = t3 * t3, s2 = t2 * t2, s1 = t1 * t1;
    return P.adh * (30.f * s2 * s2 - 5.f * s3 * s3 - 75.f * s1 * s1) * g.rinv;
}

__device__ __forceinline__ void wf3(const P3 &P, const Geo3 &g, float &W, float &F)
{
    const float b = g.r * P.inv_h;
    const float t3 = fmaxf(3.f - b, 0.f), t2 = fmaxf(2.f - b, 0.f), t1 = fmaxf(1.f - b, 0.f);
    const float s3 = t3 * t3, s2 = t2 * t2, s1 = t1 * t1;
    const float q3 = s3 * s3, q2 = s2 * s2, q1 = s1 * s1;
    W = P.ad * (q3 * t3 - 6.f * q2 * t2 + 15.f * q1 * t1);
    F = P.adh * (30.f * q2 - 5.f * q3 - 75.f * q1) * g.rinv;
}

// out = B d (B row-major, held in registers)
__device__ __forceinline__ void bd_of(const float B[9], const float d[3], float out[3])
{
    for (int a = 0; a < 3; a++) out[a] = B[3 * a] * d[0] + B[3 * a + 1] * d[1] + B[3 * a + 2] * d[2];
}

__device__ __forceinline__ void load_b(const Work3 &w, int i, float B[9])
{
    const float *p = w.B + 9 * (size_t)i;
    for (int c = 0; c < 9; c++) B[c] = p[c];
}

// Occupancy hints of the pair kernels (minimum resident blocks of 256 threads per SM; 0 leaves the
// register budget to the compiler) and the list-word prefetch distance (words of four entries).
// The defaults are the measured best on GB300 at 96^3: passes 1 and 3 keep ~125 registers (two
// blocks per SM), because the four independent neighbours of a list word, loaded together, hide
// the gather latency better than more resident warps with fewer registers each would.
#ifndef ANN3_MINB_F
#define ANN3_MINB_F 4
#endif
#ifndef ANN3_MINB_1
#define ANN3_MINB_1 2
#endif
#ifndef ANN3_MINB_3
#define ANN3_MINB_3 2
#endif
#ifndef ANN3_PF
#define ANN3_PF 1
#endif
#define ANN3_BOUNDS(minb) __launch_bounds__(256, (minb) > 0 ? (minb) : 1)

// Visit entries 0 .. m - 1 of particle i's list in order, fn(entry, k), keeping the next ANN3_PF
// words in flight while the current one is processed; word w is loaded only when 4 w < m.
template <typename Fn>
__device__ __forceinline__ void for_each_entry(const int4 *list, int n, int i, int m, Fn &&fn)
{
    constexpr int PF = ANN3_PF;
    static_assert(PF >= 1 && PF <= 3, "prefetch distance");
    const int4 *p = list + i;
    int4 r[PF + 1];
#pragma unroll
    for (int t = 0; t <= PF; t++) r[t] = (4 * t < m) ? __ldg(p + (size_t)t * n) : make_int4(0, 0, 0, 0);
    p += (size_t)(PF + 1) * n;
    int k = 0;
    for (; k + 3 < m; k += 4) {
        const int4 e = r[0];
#pragma unroll
        for (int t = 0; t < PF; t++) r[t] = r[t + 1];
        r[PF] = (k + 4 * (PF + 1) < m) ? __ldg(p) : make_int4(0, 0, 0, 0);
        p += n;
        fn(e.x, k);
        fn(e.y, k + 1);
        fn(e.z, k + 2);
        fn(e.w, k + 3);
    }
    if (k < m) fn(r[0].x, k);
    if (k + 1 < m) fn(r[0].y, k + 1);
    if (k + 2 < m) fn(r[0].z, k + 2);
}

// Builds a list in the int4 layout one entry at a time: four entries are written as one word.
struct ListWriter {
    int4 *list;
    int n, i, k = 0;
    int4 acc = make_int4(0, 0, 0, 0);
    __device__ ListWriter(int4 *l, int n_, int i_) : list(l), n(n_), i(i_) {}
    __device__ __forceinline__ void push(int j)
    {
        acc = make_int4(acc.y, acc.z, acc.w, j);
        if ((++k & 3) == 0) list[(size_t)(k / 4 - 1) * n + i] = acc;
    }
    __device__ __forceinline__ void finish()   // writes the last, partial word (unused entries 0)
    {
        if (k & 3) {
            for (int t = k & 3; t < 4; t++) acc = make_int4(acc.y, acc.z, acc.w, 0);
            list[(size_t)(k / 4) * n + i] = acc;
        }
    }
};

__device__ __forceinline__ int cell_of(const P3 &P, double x, double y, double z)
{
    int cx = min((int)(x * P.inv_cell), P.nc - 1), cy = min((int)(y * P.inv_cell), P.nc - 1),
        cz = min((int)(z * P.inv_cell), P.nc - 1);
    return (cz * P.nc + cy) * P.nc + max(cx, 0);
}

// ---- predictor, cell counts --------------------------------------------------------------------

__device__ __forceinline__ bool resorting(const Work3 &w) { return *(volatile unsigned *)w.flag != 0u; }

// Predictor on S (in place) and a copy into M in the same order (the order of the last re-sort),
// with the FP32 offset to the particle's assigned cell; a particle that has moved SKIN3 3h / 2 since
// the last re-sort makes this step re-sort (the gated kernels after this one see the flag).
__global__ void k3_predict(P3 P, Set3 S, Set3 M, Work3 w)
{
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    float sp = 0.f;
    const bool rs = resorting(w);
    if (i < P.n) {
        float u[3];
        for (int c = 0; c < 3; c++) {
            u[c] = S.u[c][i] + P.half_dt * S.a[c][i];
            S.u[c][i] = u[c];
            M.u[c][i] = u[c];
        }
        double x = wrap(S.x[i] + P.half_dt_d * (double)u[0], P.L);
        double y = wrap(S.y[i] + P.half_dt_d * (double)u[1], P.L);
        double z = wrap(S.z[i] + P.half_dt_d * (double)u[2], P.L);
        if (!(isfinite(x) && isfinite(y) && isfinite(z) && isfinite(u[0]) && isfinite(u[1]) && isfinite(u[2]))) {
            atomicOr(w.err, E3_NONFINITE);
            x = y = z = 0.0;
        }
        S.x[i] = x;
        S.y[i] = y;
        S.z[i] = z;
        sp = sqrtf(u[0] * u[0] + u[1] * u[1] + u[2] * u[2]);
        if (!isfinite(sp)) sp = 0.f;
        if (!rs) {
            double ex = min_image(x - w.xr[i], P.L), ey = min_image(y - w.yr[i], P.L), ez = min_image(z - w.zr[i], P.L);
            if (ex * ex + ey * ey + ez * ez > P.skin_max2) *(volatile unsigned *)w.flag = 1u;
            M.x[i] = x;
            M.y[i] = y;
            M.z[i] = z;
            for (int c = 0; c < 5; c++) M.q[c][i] = S.q[c][i];
            M.dr[i] = S.dr[i];
            M.id[i] = S.id[i];
            int cc = M.cxyz[i];
            int cx = cc & 1023, cy = (cc >> 10) & 1023, cz = cc >> 20;
            M.xi[i] = make_float4((float)min_image(x - cx * P.cell, P.L), (float)min_image(y - cy * P.cell, P.L),
                                  (float)min_image(z - cz * P.cell, P.L), __int_as_float(cc));
        }
    }
    for (int o = 16; o > 0; o >>= 1) sp = fmaxf(sp, __shfl_xor_sync(0xFFFFFFFFu, sp, o));
    if ((threadIdx.x & 31) == 0) atomicMax(w.umax, __float_as_uint(sp));   // sp >= 0: bits order as values
}

// Cell of each particle and the cell counts (re-sort steps only).
__global__ void k3_keys(P3 P, const Set3 S, Work3 w)
{
    if (!resorting(w)) return;
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= P.n) return;
    int c = cell_of(P, S.x[i], S.y[i], S.z[i]);
    w.key[i] = c;
    w.slot[i] = atomicAdd(&w.count[c], 1);
}

// Exclusive scan of the cell counts by one block of 1024 threads (chunks of 1024 cells).
__global__ void __launch_bounds__(1024) k3_scan(Work3 w, int ncell, const int *count, int *start)
{
    if (!resorting(w)) return;
    __shared__ int s[1024];
    __shared__ int carry;
    if (threadIdx.x == 0) carry = 0;
    __syncthreads();
    for (int base = 0; base < ncell; base += 1024) {
        int c = base + threadIdx.x;
        int v = c < ncell ? count[c] : 0;
        s[threadIdx.x] = v;
        __syncthreads();
        for (int o = 1; o < 1024; o <<= 1) {
            int t = threadIdx.x >= o ? s[threadIdx.x - o] : 0;
            __syncthreads();
            s[threadIdx.x] += t;
            __syncthreads();
        }
        if (c < ncell) start[c] = carry + s[threadIdx.x] - v;
        __syncthreads();
        if (threadIdx.x == 1023) carry += s[1023];
        __syncthreads();
    }
    if (threadIdx.x == 0) start[ncell] = carry;
}

__global__ void k3_scatter(P3 P, Work3 w)
{
    if (!resorting(w)) return;
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < P.n) w.perm[w.start[w.key[i]] + w.slot[i]] = i;
}

// The slots of each cell in particle-ID order (insertion sort; cells hold tens of particles).
__global__ void k3_cellsort(P3 P, const Set3 S, Work3 w)
{
    if (!resorting(w)) return;
    int c = blockIdx.x * blockDim.x + threadIdx.x;
    if (c >= P.ncell) return;
    int b = w.start[c], e = w.start[c + 1];
    for (int s = b + 1; s < e; s++) {
        int v = w.perm[s], iv = S.id[v], t = s - 1;
        while (t >= b && S.id[w.perm[t]] > iv) {
            w.perm[t + 1] = w.perm[t];
            t--;
        }
        w.perm[t + 1] = v;
    }
}

__global__ void k3_gather(P3 P, const Set3 S, Set3 M, Work3 w)
{
    if (!resorting(w)) return;
    int g = blockIdx.x * blockDim.x + threadIdx.x;
    if (g >= P.n) return;
    int i = w.perm[g];
    M.x[g] = S.x[i];
    M.y[g] = S.y[i];
    M.z[g] = S.z[i];
    for (int c = 0; c < 3; c++) {
        M.u[c][g] = S.u[c][i];
        M.a[c][g] = S.a[c][i];
    }
    for (int c = 0; c < 5; c++) M.q[c][g] = S.q[c][i];
    M.dr[g] = S.dr[i];
    M.id[g] = S.id[i];
    const double x = S.x[i], y = S.y[i], z = S.z[i];
    const int c = cell_of(P, x, y, z);
    const int cx = c % P.nc, cy = (c / P.nc) % P.nc, cz = c / (P.nc * P.nc);
    w.key[g] = c;
    M.cxyz[g] = cx | (cy << 10) | (cz << 20);
    M.xi[g] = make_float4((float)(x - cx * P.cell), (float)(y - cy * P.cell), (float)(z - cz * P.cell),
                          __int_as_float(M.cxyz[g]));
}

// ---- neighbours, volumes, correction -------------------------------------------------------------

// Candidate lists (re-sort steps only): every j within 3h (1 + SKIN3) from the 27 surrounding
// cells, and the positions they were taken at.
__global__ void k3_candidates(P3 P, const Set3 M, Work3 w)
{
    if (!resorting(w)) return;
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= P.n) return;
    if (i == 0) atomicAdd(w.rebuilds, 1u);
    const Here3 h = here_of(M, i);
    ListWriter out(w.cand, P.n, i);
    bool over = false;
    for (int oz = -1; oz <= 1; oz++)
        for (int oy = -1; oy <= 1; oy++)
            for (int ox = -1; ox <= 1; ox++) {
                int qx = h.cx + ox, qy = h.cy + oy, qz = h.cz + oz;
                qx += qx < 0 ? P.nc : (qx >= P.nc ? -P.nc : 0);
                qy += qy < 0 ? P.nc : (qy >= P.nc ? -P.nc : 0);
                qz += qz < 0 ? P.nc : (qz >= P.nc ? -P.nc : 0);
                const int q = (qz * P.nc + qy) * P.nc + qx;
                // d = xi_i - xi_j - (offset of cell q) cell
                const float sx = h.xi.x - (float)ox * P.cell_f, sy = h.xi.y - (float)oy * P.cell_f,
                            sz = h.xi.z - (float)oz * P.cell_f;
                const int e = w.start[q + 1];
                for (int j = w.start[q]; j < e; j++) {
                    if (j == i) continue;
                    const float4 xj = __ldg(M.xi + j);
                    const float dx = sx - xj.x, dy = sy - xj.y, dz = sz - xj.z;
                    if (dx * dx + dy * dy + dz * dz < P.R2c) {
                        if (out.k < MAXC3) out.push(j);
                        else over = true;
                    }
                }
            }
    out.finish();
    if (over) atomicOr(w.err, E3_NBR);
    w.ncand[i] = out.k;
    w.xr[i] = M.x[i];
    w.yr[i] = M.y[i];
    w.zr[i] = M.z[i];
}

// Every step: the neighbours (|r_i - r_j| < 3h; FP32 test, FP64 near 3h as the oracle decides)
// among the candidates, sum W and V = 1 / sum W (Eq. 19).  Clears the re-sort flag: the gated
// kernels of this step have run.
__global__ void ANN3_BOUNDS(ANN3_MINB_F) k3_filter(P3 P, const Set3 M, Work3 w)
{
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (blockIdx.x == 0 && threadIdx.x == 0) *(volatile unsigned *)w.flag = 0u;
    if (i >= P.n) return;
    const Here3 hi = here_of(M, i);
    ListWriter out(w.nbr, P.n, i);
    float s = P.W0;
    bool over = false;
    for_each_entry(w.cand, P.n, i, w.ncand[i], [&](int j, int) {
        const Geo3 g = geo_of(P, hi, __ldg(M.xi + j));
        bool in = g.r2 < P.R2lo;
        if (!in && g.r2 < P.R2hi) {
            double ex = min_image(M.x[i] - M.x[j], P.L), ey = min_image(M.y[i] - M.y[j], P.L),
                   ez = min_image(M.z[i] - M.z[j], P.L);
            in = ex * ex + ey * ey + ez * ez < P.R2d;
        }
        if (in) {
            if (out.k < MAXN3) {
                out.push(j);
                s += w3(P, g);
            } else {
                over = true;
            }
        }
    });
    out.finish();
    if (over) atomicOr(w.err, E3_NBR);
    w.nnbr[i] = out.k;
    w.sumW[i] = s;
    const float v = 1.f / s;
    w.V[i] = v;
    w.vu[i] = make_float4(v, M.u[0][i], M.u[1][i], M.u[2][i]);
    w.q4[i] = make_float4(M.q[0][i], M.q[1][i], M.q[2][i], M.q[3][i]);
}

// B = alpha^-1 of a symmetric alpha (Eq. 22); flags a non-positive determinant.
__device__ __forceinline__ void invert_alpha(const float a[3][3], float *B, unsigned *err)
{
    float det = a[0][0] * (a[1][1] * a[2][2] - a[1][2] * a[2][1]) - a[0][1] * (a[1][0] * a[2][2] - a[1][2] * a[2][0]) +
                a[0][2] * (a[1][0] * a[2][1] - a[1][1] * a[2][0]);
    if (!(det > 0.f)) atomicOr(err, E3_ALPHA);
    float id = 1.f / det;
    B[0] = (a[1][1] * a[2][2] - a[1][2] * a[2][1]) * id;
    B[1] = (a[0][2] * a[2][1] - a[0][1] * a[2][2]) * id;
    B[2] = (a[0][1] * a[1][2] - a[0][2] * a[1][1]) * id;
    B[3] = (a[1][2] * a[2][0] - a[1][0] * a[2][2]) * id;
    B[4] = (a[0][0] * a[2][2] - a[0][2] * a[2][0]) * id;
    B[5] = (a[0][2] * a[1][0] - a[0][0] * a[1][2]) * id;
    B[6] = (a[1][0] * a[2][1] - a[1][1] * a[2][0]) * id;
    B[7] = (a[0][1] * a[2][0] - a[0][0] * a[2][1]) * id;
    B[8] = (a[0][0] * a[1][1] - a[0][1] * a[1][0]) * id;
}

// ---- pass 1: continuity, velocity gradient, Laplacian of Q, Q rate ----------------------------------

__device__ __forceinline__ void full_q(const float *q, float Q[3][3])
{
    Q[0][0] = q[0]; Q[0][1] = q[1]; Q[0][2] = q[2];
    Q[1][0] = q[1]; Q[1][1] = q[3]; Q[1][2] = q[4];
    Q[2][0] = q[2]; Q[2][1] = q[4]; Q[2][2] = -q[0] - q[3];
}

// Eq. (24) with Eqs. (2) and (7): m = S + Gamma H, projected onto the symmetric traceless part.
__device__ void q_rate3(const P3 &P, const float *q, const float D[3][3], const float *lq, float *m5)
{
    float Q[3][3], LQ[3][3], M[3][3], E[3][3], Om[3][3];
    full_q(q, Q);
    full_q(lq, LQ);
    float QD = 0.f;
    for (int a = 0; a < 3; a++)
        for (int b = 0; b < 3; b++) {
            E[a][b] = 0.5f * (D[a][b] + D[b][a]);
            Om[a][b] = 0.5f * (D[a][b] - D[b][a]);
            M[a][b] = Q[a][b] + (a == b ? P.c_shift : 0.f);
            QD += Q[a][b] * D[a][b];
        }
    float trQ2 = 0.f, Q2[3][3];
    for (int a = 0; a < 3; a++)
        for (int b = 0; b < 3; b++) {
            Q2[a][b] = Q[a][0] * Q[0][b] + Q[a][1] * Q[1][b] + Q[a][2] * Q[2][b];
        }
    trQ2 = Q2[0][0] + Q2[1][1] + Q2[2][2];
    float m[3][3];
    for (int a = 0; a < 3; a++)
        for (int b = 0; b < 3; b++) {
            // (lambda E + Omega) M + M (lambda E - Omega) - 2 lambda M (Q : grad u)
            float s = 0.f;
            for (int c = 0; c < 3; c++)
                s += (P.lambda * E[a][c] + Om[a][c]) * M[c][b] + M[a][c] * (P.lambda * E[c][b] - Om[c][b]);
            s -= 2.f * P.lambda * M[a][b] * QD;
            float H = -P.A * Q[a][b] + P.B * (Q2[a][b] - (a == b ? trQ2 / 3.f : 0.f)) - P.C * Q[a][b] * trQ2 +
                      P.K * LQ[a][b];
            m[a][b] = s + P.Gamma * H;
        }
    float tr = m[0][0] + m[1][1] + m[2][2];
    m5[0] = m[0][0] - tr / 3.f;
    m5[1] = 0.5f * (m[0][1] + m[1][0]);
    m5[2] = 0.5f * (m[0][2] + m[2][0]);
    m5[3] = m[1][1] - tr / 3.f;
    m5[4] = 0.5f * (m[1][2] + m[2][1]);
}

// One walk of the neighbours gives alpha and every raw sum of pass 1; B enters after the walk,
// since each corrected quantity is a contraction of B with a sum that does not involve it:
//   alpha_ab = -sum_j V_j F d_a d_b                                                   (Eq. 22)
//   grad u   = rhs B,  rhs_cl = sum_j V_j (u_j - u_i)_c F d_l                         (Eq. 20)
//   k / rho  = sum_j V_j F (u_i - u_j) . B d = -sum_ab B_ab rhs_ab                    (Eq. 25)
//   lap Q_c  = 2 sum_j V_j F (Q_i - Q_j)_c (d . B d) / r^2 = 2 sum_ab B_ab L_c,ab,
//              L_c,ab = sum_j V_j F d_a d_b (Q_i - Q_j)_c / r^2 (symmetric in ab)     (Eq. 21)
__global__ void ANN3_BOUNDS(ANN3_MINB_1) k3_pass1(P3 P, const Set3 M, Work3 w)
{
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= P.n) return;
    const Here3 hi = here_of(M, i);
    float ui[3] = {M.u[0][i], M.u[1][i], M.u[2][i]}, qi[5];
    for (int c = 0; c < 5; c++) qi[c] = M.q[c][i];
    float al[6] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f};   // (00, 01, 02, 11, 12, 22) of sum_j V_j F d_a d_b
    float rhs[3][3] = {{0.f, 0.f, 0.f}, {0.f, 0.f, 0.f}, {0.f, 0.f, 0.f}};
    float L[5][6] = {};
    for_each_entry(w.nbr, P.n, i, w.nnbr[i], [&](int j, int) {
        const Geo3 g = geo_of(P, hi, __ldg(M.xi + j));
        const float4 vu = __ldg(w.vu + j), qa = __ldg(w.q4 + j);
        const float qj[5] = {qa.x, qa.y, qa.z, qa.w, __ldg(M.q[4] + j)};
        const float vf = vu.x * f3(P, g);   // V_j F
        const float e0 = vf * g.d[0], e1 = vf * g.d[1], e2 = vf * g.d[2];
        const float pab[6] = {e0 * g.d[0], e0 * g.d[1], e0 * g.d[2], e1 * g.d[1], e1 * g.d[2], e2 * g.d[2]};
        for (int k = 0; k < 6; k++) al[k] += pab[k];
        const float du[3] = {vu.y - ui[0], vu.z - ui[1], vu.w - ui[2]};   // u_j - u_i
        const float ev[3] = {e0, e1, e2};
        for (int c = 0; c < 3; c++)
            for (int l = 0; l < 3; l++) rhs[c][l] = fmaf(du[c], ev[l], rhs[c][l]);
        const float ir2 = g.rinv * g.rinv;
        for (int c = 0; c < 5; c++) {
            const float dq = (qi[c] - qj[c]) * ir2;
            for (int k = 0; k < 6; k++) L[c][k] = fmaf(pab[k], dq, L[c][k]);
        }
    });
    const float a[3][3] = {{-al[0], -al[1], -al[2]}, {-al[1], -al[3], -al[4]}, {-al[2], -al[4], -al[5]}};
    float B[9];
    invert_alpha(a, B, w.err);
    for (int c = 0; c < 9; c++) w.B[9 * (size_t)i + c] = B[c];
    float D[3][3];
    for (int c = 0; c < 3; c++)
        for (int b = 0; b < 3; b++) D[c][b] = rhs[c][0] * B[b] + rhs[c][1] * B[3 + b] + rhs[c][2] * B[6 + b];
    float kc = 0.f;
    for (int a_ = 0; a_ < 3; a_++)
        for (int b = 0; b < 3; b++) kc -= B[3 * a_ + b] * rhs[a_][b];
    // B_ab + B_ba weights of the off-diagonal pairs of the symmetric L
    const float bw[6] = {B[0], B[1] + B[3], B[2] + B[6], B[4], B[5] + B[7], B[8]};
    float lap[5];
    for (int c = 0; c < 5; c++) {
        float sl = 0.f;
        for (int k = 0; k < 6; k++) sl = fmaf(bw[k], L[c][k], sl);
        lap[c] = 2.f * sl;
    }
    float k_i = P.rho0 * (1.f + M.dr[i]) * kc;
    w.k[i] = k_i;
    w.dh[i] = M.dr[i] + P.half_dt * k_i / P.rho0;
    float m5[5], qn[5];
    q_rate3(P, qi, D, lap, m5);
    for (int c = 0; c < 5; c++) {
        qn[c] = qi[c] + P.dt * m5[c];
        w.m[(size_t)c * P.n + i] = m5[c];
        w.lap[(size_t)c * P.n + i] = lap[c];
        w.qn[(size_t)c * P.n + i] = qn[c];
    }
    w.uqn[i] = make_float4(ui[2], qn[0], qn[1], qn[2]);
    w.qn2[i] = make_float2(qn[3], qn[4]);
    for (int c = 0; c < 9; c++) w.gu[(size_t)c * P.n + i] = D[c / 3][c % 3];
}

// ---- pass 2: density filter, equation of state ------------------------------------------------------

__global__ void k3_pass2(P3 P, const Set3 M, Work3 w)
{
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= P.n) return;
    const Here3 hi = here_of(M, i);
    // Eq. (28) on the deviations (rho0 factors out of the filter)
    float di = w.dh[i], num = 0.f, den = P.W0;
    for_each_entry(w.nbr, P.n, i, w.nnbr[i], [&](int j, int) {
        const float W = w3(P, geo_of(P, hi, __ldg(M.xi + j)));
        num = fmaf(di - __ldg(w.dh + j), W, num);
        den += W;
    });
    float dhat = di - P.beta * num / den;
    w.dhat[i] = dhat;
    // Eq. (26): (rho / rho0)^gamma - 1 = expm1(gamma log1p(delta)), accurate for small delta
    float c0 = fmaxf(10.f * __uint_as_float(*w.umax), P.c0_min);
    const float p = P.rho0 * c0 * c0 / P.gamma_eos * expm1f(P.gamma_eos * log1pf(dhat));
    const float rho = P.rho0 * (1.f + dhat);
    w.p[i] = p;
    w.vpu[i] = make_float4(w.V[i], p / (rho * rho), M.u[0][i], M.u[1][i]);
}

// ---- pass 3: momentum, artificial displacement, corrector --------------------------------------------

__global__ void ANN3_BOUNDS(ANN3_MINB_3) k3_pass3(P3 P, const Set3 M, Set3 S, Work3 w)
{
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= P.n) return;
    const Here3 hi = here_of(M, i);
    float B[9];
    load_b(w, i, B);
    float ri = P.rho0 * (1.f + w.dhat[i]), pri = w.p[i] / (ri * ri);
    float ui[3] = {M.u[0][i], M.u[1][i], M.u[2][i]}, qi[5];
    for (int c = 0; c < 5; c++) qi[c] = w.qn[(size_t)c * P.n + i];
    float Qi[3][3];
    full_q(qi, Qi);
    // pressure and viscous terms share B grad_i W = F B d:
    //   fw = sum_j V_j F [ -rho_i (p_i/rho_i^2 + p_j/rho_j^2) + kv (u_ij . d) / r^2 ] B d,  kv = 10 nu rho0 / rho_i
    const float kv = 10.f * P.nu * P.rho0 / ri;
    float fw[3] = {0.f, 0.f, 0.f}, dq[3] = {0.f, 0.f, 0.f};
    float su[3] = {0.f, 0.f, 0.f}, sw = P.W0, sr = 0.f, sd[3] = {0.f, 0.f, 0.f};
    // sum_j d / r^3 of Eq. (29) nearly cancels (terms ~1/r^2, sum ~ their imbalance): compensated
    // (Kahan) summation keeps it to FP32 rounding of the sum rather than of the terms
    float sdc[3] = {0.f, 0.f, 0.f};
    const int m = w.nnbr[i];
    for_each_entry(w.nbr, P.n, i, m, [&](int j, int) {
        const Geo3 g = geo_of(P, hi, __ldg(M.xi + j));
        const float4 vp = __ldg(w.vpu + j), uq = __ldg(w.uqn + j);
        const float2 q2 = __ldg(w.qn2 + j);
        float W, F;
        wf3(P, g, W, F);
        const float vf = vp.x * F;   // V_j F
        float bd[3];
        bd_of(B, g.d, bd);
        const float du[3] = {ui[0] - vp.z, ui[1] - vp.w, ui[2] - uq.x};
        const float ud = du[0] * g.d[0] + du[1] * g.d[1] + du[2] * g.d[2];
        const float rinv2 = g.rinv * g.rinv;
        const float coef = vf * fmaf(kv, ud * rinv2, -ri * (pri + vp.y));
        const float qj[5] = {uq.y, uq.z, uq.w, q2.x, q2.y};
        float Qj[3][3];
        full_q(qj, Qj);
        const float rinv3 = rinv2 * g.rinv;
        for (int c = 0; c < 3; c++) {
            fw[c] = fmaf(coef, bd[c], fw[c]);
            dq[c] = fmaf(vf, (Qj[c][0] - Qi[c][0]) * bd[0] + (Qj[c][1] - Qi[c][1]) * bd[1] + (Qj[c][2] - Qi[c][2]) * bd[2],
                         dq[c]);
            su[c] = fmaf(du[c], W, su[c]);
            const float y = g.d[c] * rinv3 - sdc[c];
            const float t = sd[c] + y;
            sdc[c] = (t - sd[c]) - y;
            sd[c] = t;
        }
        sw += W;
        sr += g.r;
    });
    float an[3], apd[3] = {0.f, 0.f, 0.f};
    for (int c = 0; c < 3; c++) an[c] = fw[c] - P.zeta / ri * dq[c];
    if (P.apd) {
        float uv = sqrtf(su[0] * su[0] + su[1] * su[1] + su[2] * su[2]) / sw;
        float r0 = m > 0 ? sr / (float)m : 0.f;
        for (int c = 0; c < 3; c++) apd[c] = sd[c] * r0 * r0 * uv * P.dt;
    }
    // corrector into S (the new cell order)
    float un[3];
    for (int c = 0; c < 3; c++) {
        un[c] = ui[c] + P.half_dt * an[c];
        S.u[c][i] = un[c];
        S.a[c][i] = an[c];
    }
    double x = wrap(M.x[i] + P.half_dt_d * (double)un[0] + (double)apd[0], P.L);
    double y = wrap(M.y[i] + P.half_dt_d * (double)un[1] + (double)apd[1], P.L);
    double z = wrap(M.z[i] + P.half_dt_d * (double)un[2] + (double)apd[2], P.L);
    float dr = w.dhat[i] + P.half_dt * w.k[i] / P.rho0;
    bool ok = isfinite(x) && isfinite(y) && isfinite(z) && isfinite(un[0]) && isfinite(un[1]) && isfinite(un[2]) &&
              isfinite(dr);
    for (int c = 0; c < 5; c++) ok = ok && isfinite(qi[c]);
    if (!ok) {
        atomicOr(w.err, E3_NONFINITE);
        x = y = z = 0.0;
    }
    S.x[i] = x;
    S.y[i] = y;
    S.z[i] = z;
    S.dr[i] = dr;
    for (int c = 0; c < 5; c++) S.q[c][i] = qi[c];
    S.id[i] = M.id[i];
}

// dst[id[g] * nc + c] = planes[c][g] (ID order, interleaved, FP64)
__global__ void k3_to_id(int n, int ncomp, const float *const *planes, const int *id, double *dst)
{
    int g = blockIdx.x * blockDim.x + threadIdx.x;
    if (g >= n) return;
    for (int c = 0; c < ncomp; c++) dst[(size_t)id[g] * ncomp + c] = (double)planes[c][g];
}

__global__ void k3_pos_to_id(int n, const double *x, const double *y, const double *z, const int *id, double *dst)
{
    int g = blockIdx.x * blockDim.x + threadIdx.x;
    if (g >= n) return;
    dst[3 * (size_t)id[g]] = x[g];
    dst[3 * (size_t)id[g] + 1] = y[g];
    dst[3 * (size_t)id[g] + 2] = z[g];
}

__global__ void k3_int_to_id(int n, const int *v, const int *id, double *dst)
{
    int g = blockIdx.x * blockDim.x + threadIdx.x;
    if (g < n) dst[id[g]] = (double)v[g];
}

inline unsigned nb3(size_t n, int t = 256) { return (unsigned)((n + t - 1) / t); }

// A named NVTX range for the lifetime of the object (profilers show the library's calls).
struct Range3 {
    explicit Range3(const char *name) { nvtxRangePushA(name); }
    ~Range3() { nvtxRangePop(); }
    Range3(const Range3 &) = delete;
    Range3 &operator=(const Range3 &) = delete;
};

}  // namespace

struct ann3_ctx {
    ann3_params prm;
    P3 P;
    Set3 S, M;
    Work3 w;
    std::vector<void *> allocs;
    cudaStream_t s = nullptr;
    bool have = false;
    int64_t steps = 0;
    std::string last_err;
    double *tmp = nullptr;         // device staging for ann3_get_field (9n doubles)
    const float **planes = nullptr;   // device array of plane pointers
};

namespace {

template <typename T>
cudaError_t alloc3(ann3_ctx *c, T *&p, size_t count)
{
    void *v = nullptr;
    cudaError_t e = cudaMalloc(&v, std::max<size_t>(count, 1) * sizeof(T));
    if (e) return e;
    c->allocs.push_back(v);
    p = static_cast<T *>(v);
    return cudaMemsetAsync(v, 0, std::max<size_t>(count, 1) * sizeof(T), c->s);
}

cudaError_t alloc_set(ann3_ctx *c, Set3 &S, size_t n)
{
    cudaError_t e = alloc3(c, S.x, n);
    if (!e) e = alloc3(c, S.y, n);
    if (!e) e = alloc3(c, S.z, n);
    for (int k = 0; k < 3 && !e; k++) e = alloc3(c, S.u[k], n);
    for (int k = 0; k < 3 && !e; k++) e = alloc3(c, S.a[k], n);
    for (int k = 0; k < 5 && !e; k++) e = alloc3(c, S.q[k], n);
    if (!e) e = alloc3(c, S.dr, n);
    if (!e) e = alloc3(c, S.id, n);
    if (!e) e = alloc3(c, S.xi, n);
    if (!e) e = alloc3(c, S.cxyz, n);
    return e;
}

int fail3(ann3_ctx *c, int code, const std::string &m)
{
    if (c) c->last_err = m;
    return code;
}

int cuda3(ann3_ctx *c, cudaError_t e, const char *where)
{
    return fail3(c, e == cudaErrorMemoryAllocation ? ANN_ERR_OOM : ANN_ERR_CUDA, std::string(where) + ": " +
                                                                                  cudaGetErrorString(e));
}

// The first cause wins: truncated neighbour lists can make alpha singular and the state non-finite.
int status_of_bits(uint32_t b)
{
    if (b & E3_NBR) return ANN_ERR_NBR_OVERFLOW;
    if (b & E3_ALPHA) return ANN_ERR_SINGULAR_ALPHA;
    if (b & E3_NONFINITE) return ANN_ERR_NONFINITE;
    return ANN_OK;
}

}  // namespace

extern "C" {

int ann3_default_params(ann3_params *p)
{
    if (!p) return ANN_ERR_INVALID_ARG;
    std::memset(p, 0, sizeof *p);
    p->n = 32 * 32 * 32;
    p->L = 1.0;
    p->h = 1.3 / 32;
    p->dt = 1e-4;
    p->rho0 = 1.0;
    p->eta = 1.0;
    p->Gamma = 0.34;
    p->lambda_ = 0.7;
    p->A = 0.0;
    p->B = 0.0;
    p->C = 1.0;
    p->K = 0.04;
    p->zeta = 0.05;
    p->gamma_eos = 7.0;
    p->beta = 1.0;
    p->c0_min = 0.0;
    p->c_shift = 1.0 / 3.0;
    p->apd = 1;
    return ANN_OK;
}

int ann3_create(const ann3_params *p, ann3_ctx **out)
{
    if (!p || !out) return ANN_ERR_INVALID_ARG;
    *out = nullptr;
    if (p->n < 1 || p->n > (1ll << 26) || !(p->L > 0.0) || !(p->h > 0.0) || !(p->dt > 0.0) || !(p->rho0 > 0.0) ||
        !(p->gamma_eos > 0.0))
        return ANN_ERR_INVALID_ARG;
    int nc = (int)std::floor(p->L / (3.0 * p->h * (1.0 + SKIN3)));
    if (nc < 3 || (int64_t)nc * nc * nc > (1ll << 28)) return ANN_ERR_INVALID_ARG;
    int dev = 0;
    if (cudaGetDeviceCount(&dev) != cudaSuccess || dev == 0) return ANN_ERR_NOT_AVAILABLE;
    ann3_ctx *c = new (std::nothrow) ann3_ctx();
    if (!c) return ANN_ERR_OOM;
    c->prm = *p;
    P3 &P = c->P;
    P.n = (int)p->n;
    P.nc = nc;
    P.ncell = nc * nc * nc;
    P.L = p->L;
    P.inv_cell = nc / p->L;
    P.cell = p->L / nc;
    P.cell_f = (float)P.cell;
    P.R2d = 9.0 * p->h * p->h;
    P.R2lo = (float)(P.R2d * (1.0 - 4e-6));   // FP32 r^2 of a pair is good to ~1e-6 relative
    P.R2hi = (float)(P.R2d * (1.0 + 4e-6));
    P.R2c = (float)(P.R2d * (1.0 + SKIN3) * (1.0 + SKIN3) * (1.0 + 1e-5));   // padded for FP32 rounding
    P.skin_max2 = (0.5 * SKIN3 * 3.0 * p->h) * (0.5 * SKIN3 * 3.0 * p->h);
    P.half_dt_d = 0.5 * p->dt;
    P.h = (float)p->h;
    P.inv_h = (float)(1.0 / p->h);
    P.ad = (float)(3.0 / (359.0 * 3.14159265358979323846 * p->h * p->h * p->h));   // Eq. (18), d = 3
    P.adh = P.ad * P.inv_h;
    P.W0 = P.ad * 66.f;                                           // W(0) = a_d (3^5 - 6 2^5 + 15)
    P.dt = (float)p->dt;
    P.half_dt = (float)(0.5 * p->dt);
    P.rho0 = (float)p->rho0;
    P.nu = (float)(p->eta / p->rho0);
    P.Gamma = (float)p->Gamma;
    P.lambda = (float)p->lambda_;
    P.A = (float)p->A;
    P.B = (float)p->B;
    P.C = (float)p->C;
    P.K = (float)p->K;
    P.zeta = (float)p->zeta;
    P.gamma_eos = (float)p->gamma_eos;
    P.beta = (float)p->beta;
    P.c0_min = (float)p->c0_min;
    P.c_shift = (float)p->c_shift;
    P.apd = p->apd;
    size_t n = (size_t)p->n;
    cudaError_t e = cudaStreamCreateWithFlags(&c->s, cudaStreamNonBlocking);
    if (!e) e = alloc_set(c, c->S, n);
    if (!e) e = alloc_set(c, c->M, n);
    Work3 &w = c->w;
    if (!e) e = alloc3(c, w.key, n);
    if (!e) e = alloc3(c, w.slot, n);
    if (!e) e = alloc3(c, w.perm, n);
    if (!e) e = alloc3(c, w.count, (size_t)P.ncell);
    if (!e) e = alloc3(c, w.start, (size_t)P.ncell + 1);
    if (!e) e = alloc3(c, w.nbr, (size_t)(MAXN3 / 4) * n);
    if (!e) e = alloc3(c, w.cand, (size_t)(MAXC3 / 4) * n);
    if (!e) e = alloc3(c, w.ncand, n);
    if (!e) e = alloc3(c, w.xr, n);
    if (!e) e = alloc3(c, w.yr, n);
    if (!e) e = alloc3(c, w.zr, n);
    if (!e) e = alloc3(c, w.flag, 1);
    if (!e) e = alloc3(c, w.rebuilds, 1);
    if (!e) e = alloc3(c, w.nnbr, n);
    if (!e) e = alloc3(c, w.sumW, n);
    if (!e) e = alloc3(c, w.V, n);
    if (!e) e = alloc3(c, w.B, 9 * n);
    if (!e) e = alloc3(c, w.k, n);
    if (!e) e = alloc3(c, w.dh, n);
    if (!e) e = alloc3(c, w.dhat, n);
    if (!e) e = alloc3(c, w.p, n);
    if (!e) e = alloc3(c, w.qn, 5 * n);
    if (!e) e = alloc3(c, w.an, 3 * n);
    if (!e) e = alloc3(c, w.gu, 9 * n);
    if (!e) e = alloc3(c, w.lap, 5 * n);
    if (!e) e = alloc3(c, w.m, 5 * n);
    if (!e) e = alloc3(c, w.vu, n);
    if (!e) e = alloc3(c, w.q4, n);
    if (!e) e = alloc3(c, w.vpu, n);
    if (!e) e = alloc3(c, w.uqn, n);
    if (!e) e = alloc3(c, w.qn2, n);
    if (!e) e = alloc3(c, w.umax, 1);
    if (!e) e = alloc3(c, w.err, 1);
    if (!e) e = alloc3(c, c->tmp, 9 * n);
    if (!e) e = alloc3(c, c->planes, 9);
    if (!e) e = cudaStreamSynchronize(c->s);
    if (e) {
        int code = e == cudaErrorMemoryAllocation ? ANN_ERR_OOM : ANN_ERR_CUDA;
        ann3_destroy(c);
        return code;
    }
    *out = c;
    return ANN_OK;
}

void ann3_destroy(ann3_ctx *c)
{
    if (!c) return;
    if (c->s) cudaStreamSynchronize(c->s);
    for (void *p : c->allocs) cudaFree(p);
    if (c->s) cudaStreamDestroy(c->s);
    delete c;
}

int ann3_set_particles(ann3_ctx *c, int64_t n, const double *x, const double *y, const double *z, const double *u,
                       const double *q, const double *rho)
{
    if (!c) return ANN_ERR_INVALID_ARG;
    if (n != c->prm.n || !x || !y || !z || !u || !q) return fail3(c, ANN_ERR_INVALID_ARG, "bad arguments");
    const double L = c->prm.L;
    for (int64_t i = 0; i < n; i++) {
        const double r[3] = {x[i], y[i], z[i]};
        for (double v : r)
            if (!(v >= 0.0 && v < L)) return fail3(c, ANN_ERR_INVALID_ARG, "position outside [0, L)");
        for (int k = 0; k < 3; k++)
            if (!std::isfinite(u[3 * i + k])) return fail3(c, ANN_ERR_INVALID_ARG, "non-finite velocity");
        for (int k = 0; k < 5; k++)
            if (!std::isfinite(q[5 * i + k])) return fail3(c, ANN_ERR_INVALID_ARG, "non-finite Q");
        if (rho && !(std::isfinite(rho[i]) && rho[i] > 0.0)) return fail3(c, ANN_ERR_INVALID_ARG, "bad density");
    }
    size_t nn = (size_t)n;
    std::vector<float> f(nn);
    std::vector<int> id(nn);
    cudaError_t e = cudaMemcpyAsync(c->S.x, x, nn * 8, cudaMemcpyHostToDevice, c->s);
    if (!e) e = cudaMemcpyAsync(c->S.y, y, nn * 8, cudaMemcpyHostToDevice, c->s);
    if (!e) e = cudaMemcpyAsync(c->S.z, z, nn * 8, cudaMemcpyHostToDevice, c->s);
    auto plane = [&](float *dst, const double *src, int stride, int comp, double dflt) -> cudaError_t {
        for (size_t i = 0; i < nn; i++) f[i] = (float)(src ? src[i * stride + comp] : dflt);
        if (dst == c->S.dr)   // the deviation, taken in FP64
            for (size_t i = 0; i < nn; i++) f[i] = (float)(src ? src[i] / c->prm.rho0 - 1.0 : 0.0);
        cudaError_t r = cudaMemcpyAsync(dst, f.data(), nn * 4, cudaMemcpyHostToDevice, c->s);
        if (!r) r = cudaStreamSynchronize(c->s);   // f is reused
        return r;
    };
    for (int k = 0; k < 3 && !e; k++) e = plane(c->S.u[k], u, 3, k, 0.0);
    for (int k = 0; k < 5 && !e; k++) e = plane(c->S.q[k], q, 5, k, 0.0);
    if (!e) e = plane(c->S.dr, rho, 1, 0, c->prm.rho0);
    for (int k = 0; k < 3 && !e; k++) e = cudaMemsetAsync(c->S.a[k], 0, nn * 4, c->s);
    for (size_t i = 0; i < nn; i++) id[i] = (int)i;
    if (!e) e = cudaMemcpyAsync(c->S.id, id.data(), nn * 4, cudaMemcpyHostToDevice, c->s);
    if (!e) e = cudaMemsetAsync(c->w.err, 0, 4, c->s);
    const unsigned one = 1u;   // the first step re-sorts
    if (!e) e = cudaMemcpyAsync(c->w.flag, &one, 4, cudaMemcpyHostToDevice, c->s);
    if (!e) e = cudaMemsetAsync(c->w.rebuilds, 0, 4, c->s);
    if (!e) e = cudaStreamSynchronize(c->s);
    if (e) return cuda3(c, e, "ann3_set_particles");
    c->have = true;
    c->steps = 0;
    return ANN_OK;
}

int ann3_step(ann3_ctx *c, int64_t nsteps)
{
    Range3 range("ann3_step");
    if (!c || nsteps < 0) return ANN_ERR_INVALID_ARG;
    if (!c->have) return fail3(c, ANN_ERR_STATE, "ann3_step before ann3_set_particles");
    const P3 &P = c->P;
    cudaStream_t s = c->s;
    const unsigned g = nb3((size_t)P.n);
    cudaError_t e = cudaSuccess;
    for (int64_t t = 0; t < nsteps && !e; t++) {
        e = cudaMemsetAsync(c->w.count, 0, sizeof(int) * (size_t)P.ncell, s);
        if (!e) e = cudaMemsetAsync(c->w.umax, 0, 4, s);
        if (e) break;
        k3_predict<<<g, 256, 0, s>>>(P, c->S, c->M, c->w);
        // re-sort and candidate rebuild: each kernel returns at once unless the flag is set
        k3_keys<<<g, 256, 0, s>>>(P, c->S, c->w);
        k3_scan<<<1, 1024, 0, s>>>(c->w, P.ncell, c->w.count, c->w.start);
        k3_scatter<<<g, 256, 0, s>>>(P, c->w);
        k3_cellsort<<<nb3((size_t)P.ncell), 256, 0, s>>>(P, c->S, c->w);
        k3_gather<<<g, 256, 0, s>>>(P, c->S, c->M, c->w);
        k3_candidates<<<g, 256, 0, s>>>(P, c->M, c->w);
        k3_filter<<<g, 256, 0, s>>>(P, c->M, c->w);
        k3_pass1<<<g, 256, 0, s>>>(P, c->M, c->w);
        k3_pass2<<<g, 256, 0, s>>>(P, c->M, c->w);
        k3_pass3<<<g, 256, 0, s>>>(P, c->M, c->S, c->w);
        e = cudaGetLastError();
    }
    uint32_t bits = 0;
    if (!e) e = cudaMemcpyAsync(&bits, c->w.err, 4, cudaMemcpyDeviceToHost, s);
    if (!e) e = cudaStreamSynchronize(s);
    if (e) return cuda3(c, e, "ann3_step");
    c->steps += nsteps;
    int st = status_of_bits(bits);
    if (st) return fail3(c, st, "ann3_step: device error bits " + std::to_string(bits));
    return ANN_OK;
}

int ann3_get_field(ann3_ctx *c, int32_t field, double *dst)
{
    if (!c || !dst || field < 0 || field >= ANN3_FIELD_COUNT) return ANN_ERR_INVALID_ARG;
    if (!c->have) return fail3(c, ANN_ERR_STATE, "no particles");
    const int n = c->P.n;
    const Work3 &w = c->w;
    const float *pl[9];
    int nc = 0;
    cudaError_t e = cudaSuccess;
    switch (field) {
    case ANN3_FIELD_POS:
        k3_pos_to_id<<<nb3(n), 256, 0, c->s>>>(n, c->S.x, c->S.y, c->S.z, c->S.id, c->tmp);
        nc = -3;
        break;
    case ANN3_FIELD_NNBR:
        k3_int_to_id<<<nb3(n), 256, 0, c->s>>>(n, w.nnbr, c->S.id, c->tmp);
        nc = -1;
        break;
    case ANN3_FIELD_U: for (int k = 0; k < 3; k++) pl[k] = c->S.u[k]; nc = 3; break;
    case ANN3_FIELD_Q: for (int k = 0; k < 5; k++) pl[k] = c->S.q[k]; nc = 5; break;
    case ANN3_FIELD_RHO: pl[0] = c->S.dr; nc = 1; break;
    case ANN3_FIELD_A: for (int k = 0; k < 3; k++) pl[k] = c->S.a[k]; nc = 3; break;
    case ANN3_FIELD_SUMW: pl[0] = w.sumW; nc = 1; break;
    case ANN3_FIELD_GRADU: for (int k = 0; k < 9; k++) pl[k] = w.gu + (size_t)k * n; nc = 9; break;
    case ANN3_FIELD_LAPQ: for (int k = 0; k < 5; k++) pl[k] = w.lap + (size_t)k * n; nc = 5; break;
    case ANN3_FIELD_QRATE: for (int k = 0; k < 5; k++) pl[k] = w.m + (size_t)k * n; nc = 5; break;
    case ANN3_FIELD_P: pl[0] = w.p; nc = 1; break;
    default: return ANN_ERR_INVALID_ARG;
    }
    int comps = nc < 0 ? -nc : nc;
    if (nc > 0) {
        e = cudaMemcpyAsync(c->planes, pl, sizeof(float *) * (size_t)nc, cudaMemcpyHostToDevice, c->s);
        if (!e) k3_to_id<<<nb3(n), 256, 0, c->s>>>(n, nc, c->planes, c->S.id, c->tmp);
    }
    if (!e) e = cudaGetLastError();
    if (!e) e = cudaMemcpyAsync(dst, c->tmp, sizeof(double) * (size_t)n * comps, cudaMemcpyDeviceToHost, c->s);
    if (!e) e = cudaStreamSynchronize(c->s);
    if (e) return cuda3(c, e, "ann3_get_field");
    if (field == ANN3_FIELD_RHO)
        for (int i = 0; i < n; i++) dst[i] = c->prm.rho0 * (1.0 + dst[i]);
    return ANN_OK;
}

int ann3_get_status(ann3_ctx *c, int64_t *steps, uint32_t *error_bits, int64_t *resorts)
{
    if (!c) return ANN_ERR_INVALID_ARG;
    uint32_t b = 0, r = 0;
    cudaError_t e = cudaMemcpyAsync(&b, c->w.err, 4, cudaMemcpyDeviceToHost, c->s);
    if (!e) e = cudaMemcpyAsync(&r, c->w.rebuilds, 4, cudaMemcpyDeviceToHost, c->s);
    if (!e) e = cudaStreamSynchronize(c->s);
    if (e) return cuda3(c, e, "ann3_get_status");
    if (steps) *steps = c->steps;
    if (error_bits) *error_bits = b;
    if (resorts) *resorts = r;
    return ANN_OK;
}

const char *ann3_last_error(ann3_ctx *c) { return c ? c->last_err.c_str() : ""; }

}  // extern "C"

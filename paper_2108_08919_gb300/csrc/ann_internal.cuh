// Internal declarations shared by the kernels and the C-ABI of the SPH active-nematic solver.
#pragma once

#include "../../include/ann.h"

#include <cstdint>
#include <cuda_bf16.h>
#include <cuda_runtime.h>
#include <nvtx3/nvToolsExt.h>

namespace ann {

// A named NVTX range for the lifetime of the object: profilers (Nsight Systems and the like) show
// the library's calls and, in the profiled step, each pass; without a profiler attached it costs
// a check of a function pointer.
struct NvtxRange {
    explicit NvtxRange(const char *name) { nvtxRangePushA(name); }
    ~NvtxRange() { nvtxRangePop(); }
    NvtxRange(const NvtxRange &) = delete;
    NvtxRange &operator=(const NvtxRange &) = delete;
};

// Tiling of the pair passes: one CUDA block per TILE x TILE cells; it stages the particles of the
// (TILE+2) x (TILE+2) cells around them (periodic images included) in shared memory.
constexpr int TILE = 4;
constexpr int HALO = TILE + 2;
constexpr int NHC = HALO * HALO;      // halo cells per tile
constexpr int HCAP = 1024;            // halo particles a tile may stage
constexpr int MAXN = 128;             // neighbours per particle (ANN_MAX_NEIGHBORS)
constexpr int MAXN2H = 64;            // neighbours closer than 2h kept in the surrogate's graph
constexpr int MAXC = 64;              // particles per cell (ANN_MAX_PER_CELL)
constexpr int PT = 256;               // threads per pair-pass block
constexpr int NKERNELS = 10;
// Candidate ("Verlet") lists hold every pair within 3h (1 + SKIN) at the last re-sort; they stay
// valid until some particle has moved SKIN/2 * 3h.  Cells are at least 3h (1 + SKIN) wide.
constexpr double SKIN = 0.02;
constexpr int MAXV = 128;             // candidates per particle (two 64-bit neighbour masks)
constexpr int SCAN_CHUNK = 4096;      // cells per block of the cell-count scan

// Sticky device error bits.
enum : uint32_t {
    EB_CELL = 1u,        // a cell held more than MAXC particles
    EB_HALO = 2u,        // a tile halo held more than HCAP particles
    EB_NBR = 4u,         // a particle had more than MAXN neighbours
    EB_NONFINITE = 8u,   // NaN / infinity in the state
    EB_SINGULAR = 16u,   // det(alpha) <= 0
    EB_CFL = 32u,        // dt above a stability limit of the step (dt_mode ANN_DT_CHECK)
};

// Parameters in the form the kernels use (FP64 where positions are involved).
struct DevParams {
    int n, nc, ncell, tiles;
    int apd, conservative, qnew, record, elastic;
    double L, cell, inv_cell, R2, dt_d, half_dt_d;
    double q;              // power-of-two grid of the "hi" coordinate part: cell / q in [2^12, 2^13)
    long long bitsL;       // bit pattern of L: for x >= +0, x < L iff bits(x) < bits(L)
    float cell_hi, cell_lo;  // cell = cell_hi + cell_lo, cell_hi a multiple of q
    float qf, iqf;           // q and 1/q in FP32 (powers of two: exact)
    float R2lo, R2hi;      // FP32 band around (3h)^2 inside which the support test is redone in FP64
    float R2c;             // coarse (hi-part only) radius^2 of the re-sort scan, padded by the hi-only error
    float R2v;             // candidate-list radius^2: (3h (1 + SKIN))^2
    float skin_max2;       // displacement^2 beyond which a candidate list is no longer valid: (SKIN 3h / 2)^2
    float inv_h, ad, W0, dt, half_dt;
    float kw6, kw15;       // -6 a_d, 15 a_d           (W = a_d t3^5 + kw6 t2^5 + kw15 t1^5)
    float kf5, kf30, kf75; // -5 a_d/h, 30 a_d/h, -75 a_d/h  (F r = kf5 t3^4 + kf30 t2^4 + kf75 t1^4)
    int nsblk;             // blocks of SCAN_CHUNK cells (scan)
    float rho0, nu, mu, Gamma, lambda, A, Bl, C, K, zeta, gamma_eos, beta, c0_min, c_shift, mass;
    int dt_check;          // ANN_DT_CHECK: pass C tests dt against dt_static and 0.25 h / (c0 + max|u|)
    float dt_static;       // min(0.125 h^2 / nu, 0.125 h^2 / (Gamma K)) (infinity where a rate is 0)
};

// One copy of the state of §3.1 at the end of a step, in the particle order of that step's
// evaluation (slot g holds particle id[g]).
struct StateSet {
    double *x, *y;
    float *ux, *uy, *q11, *q12, *dr, *ax, *ay;
    int *id;
};

// Step control words (ctl[]).  The state lives in two StateSets: st[ctl[CTL_CUR]] holds the last
// committed step, and a step writes the other one.  A step commits when the next step begins with
// no error raised (k_commit) or, for the last step of a call, when the host finds no error after it;
// a failed step is never committed, so its input -- the last completed step -- stays intact.
enum : int {
    CTL_CUR = 0,       // index of the committed state set
    CTL_PENDING = 1,   // 1: a step has written st[CUR ^ 1] and is not yet committed
    CTL_COMMITS = 2,   // steps committed on the device (counts up; the host takes differences)
    CTL_XLOG = 3,      // entries in the crossing log of the step in flight
    CTL_WORDS = 4,
};

// Device buffers.  S: the host's view of the committed state (the StateSet st[CUR]: the kernels
// outside the step read and write the state through it).  The step kernels take their input and
// output sets from st[] and ctl[] instead.  M: the current step's cell-sorted copy.  Per-particle
// intermediates are in M order.
struct Bufs {
    double *sx, *sy;
    float *sux, *suy, *sq11, *sq12, *sdr, *sax, *say;
    float4 *sxi;        // split cell-local offset of the predicted position, S order (predictor)
    const double *origin;   // origin[c] = c * cell, c < n_c (cell-corner coordinates)
    int *sid;
    double *mx, *my;
    float4 *mu4;   // (ux, uy, q11, q12) of the evaluation copy, one record per particle
    float *mdr;
    float4 *xi;         // cell-local offset split as (hi_x, hi_y, lo_x, lo_y), hi on the q grid
    float4 *xi_ref;     // split offset at the last re-sort (candidate lists were built from it)
    uint32_t *mkey;     // cell each particle was assigned to at the last re-sort
    int *mid;
    uint32_t *cell_count, *cell_start, *key, *rank, *perm;
    int *nnbr;          // neighbours per particle (exact support test)
    uint2 *vnbr;        // candidate lists: 16-bit slot byte offsets, four per 64-bit word, word m of particle g at [m n + g]
    int *vcnt;
    uint32_t *rebuild;  // non-zero: this step re-sorts and rebuilds the candidate lists
    uint32_t *resorts;  // number of re-sort steps since the particles were loaded
    float *sumW, *V, *p;
    float4 *cr;   // (V, delta_half, Q11^{n+1}, Q12^{n+1}) per particle (pass B): the record pass C stages
    float4 *bk;   // (B11, B12, B22, k) per particle (pass B): the correction tensor and continuity rate
    float4 *cq;   // (div Q x, div Q y, delta_hat, sum W) per particle (pass C), read by pass D
    float4 *rd;   // (V, p / rho_hat^2, ux, uy) per particle (pass C): the record pass D stages
    float *rec_gu, *rec_lap, *rec_apd, *rec_qrate;   // 4n, 2n, 2n, 2n (recording only)
    float4 *pel;        // elastic stress (11, 12, 22, -) of Eq. 12 (elastic_stress only)
    float *delx, *dely; // its corrected divergence (paper momentum only)
    int2 *img;          // by particle ID: net periodic shifts (x, y) since ann_set_particles
    uint32_t *err, *maxu;
    unsigned long long *band;
    StateSet st[2];     // the two state sets (st[0] is the host view's storage at creation)
    uint32_t *ctl;      // CTL_WORDS step control words
    int4 *xlog;         // crossings of the step in flight: (particle ID, dx, dy, -), undone if it fails
    int xlog_cap;       // entries of xlog
};

// Input and output state sets of a step kernel (the step reads the committed set and writes the
// other).  Only the step kernels use these; ctl[CUR] does not change while a step runs.
__device__ __forceinline__ StateSet pick_set(const Bufs &b, bool one)
{
    StateSet s;
    s.x = one ? b.st[1].x : b.st[0].x;
    s.y = one ? b.st[1].y : b.st[0].y;
    s.ux = one ? b.st[1].ux : b.st[0].ux;
    s.uy = one ? b.st[1].uy : b.st[0].uy;
    s.q11 = one ? b.st[1].q11 : b.st[0].q11;
    s.q12 = one ? b.st[1].q12 : b.st[0].q12;
    s.dr = one ? b.st[1].dr : b.st[0].dr;
    s.ax = one ? b.st[1].ax : b.st[0].ax;
    s.ay = one ? b.st[1].ay : b.st[0].ay;
    s.id = one ? b.st[1].id : b.st[0].id;
    return s;
}
// ctl[CTL_CUR] changes only in k_commit, a kernel of its own, so the step kernels may read it through
// the read-only cache (one L2 round trip per SM instead of one per thread).
__device__ __forceinline__ bool cur_set(const Bufs &b) { return __ldg(b.ctl + CTL_CUR) != 0u; }
__device__ __forceinline__ StateSet state_in(const Bufs &b) { return pick_set(b, cur_set(b)); }
__device__ __forceinline__ StateSet state_out(const Bufs &b) { return pick_set(b, !cur_set(b)); }

// Launch-configuration helpers (defined with the kernels).
const char *kernel_name(int k);
cudaError_t prepare_kernels();
// Launch kernel k (0 <= k < NKERNELS, in step order) of the time step on `s`.  Kernels 1-5 are the
// re-sort path and kernel 6 its alternative; each also checks the re-sort flag itself.
cudaError_t launch_kernel(int k, const DevParams &P, const Bufs &b, cudaStream_t s);
// Copy the re-sort flag into a graph conditional handle (one thread).
cudaError_t launch_set_condition(const Bufs &b, cudaGraphConditionalHandle h, cudaStream_t s);
// The first node of every step: commits the previous step if no error was raised since (one thread).
cudaError_t launch_commit(const Bufs &b, cudaStream_t s);
// Undo the crossings logged by a failed step in the image counts (img), n_log entries.
cudaError_t enqueue_undo_crossings(const Bufs &b, int n_log, cudaStream_t s);
// Cell sort and the re-sort pass A only (neighbour lists and volumes) at the positions in S advanced
// by P.half_dt (callers pass 0 to keep them).  Requires *b.rebuild != 0.
cudaError_t enqueue_search(const DevParams &P, const Bufs &b, cudaStream_t s);
// Rebuild the candidate lists from xi_ref (the split positions of the last re-sort), with the
// cell starts of that re-sort: used after a checkpoint is loaded.
cudaError_t enqueue_candidates_from_ref(const DevParams &P, const Bufs &b, cudaStream_t s);
// Load FP64 inputs (ID order) into S; rho may be null.
cudaError_t enqueue_load(const DevParams &P, const Bufs &b, const double *x, const double *y,
                         const double *ux, const double *uy, const double *q11, const double *q12,
                         const double *rho, cudaStream_t s, bool reset_images = true);
// Scatter field f (M or S order, element size es) into out[id[g]].
cudaError_t enqueue_unpermute(const void *f, const int *id, void *out, int n, int es, cudaStream_t s);
// Neighbour export: for each M-order particle g and k < nnbr[g], cols_tmp[k * n + g] = original ID
// of its k-th neighbour.
cudaError_t enqueue_export_nbrs(const DevParams &P, const Bufs &b, int *cols_tmp, cudaStream_t s);
// Diagnostics: deterministic two-level FP64 reductions into out[0..ndiag).
constexpr int NDIAG = 12;
cudaError_t enqueue_diag(const DevParams &P, const Bufs &b, double *partials, int nblocks,
                         double *out, cudaStream_t s);
int diag_blocks(int n);

// Flow diagnostics (ann_diag.cu).  DiagSrc: the state the analysis reads, in the cell order of the
// last re-sort (mkey, cell_start).
struct DiagSrc {
    const double *x, *y;
    const float *ux, *uy, *q11, *q12;   // separate arrays, or
    const float4 *u4;                   // (ux, uy, q11, q12) records when not null
};
// grid: 5 x M x M doubles (ux, uy, q11, q12, Shepard weight sum), [field][iy][ix]
cudaError_t enqueue_grid(const DevParams &P, const Bufs &b, DiagSrc src, int M, float2 *off, float4 *fld,
                         double *grid, cudaStream_t s);
cudaError_t enqueue_twiddles(int M, double2 *tw, cudaStream_t s);
cudaError_t enqueue_spectrum(int M, const double *grid, double2 *z, double2 *zt, const double2 *tw,
                             const int *shell_off, const int *shell_modes, int nshell, double *E, cudaStream_t s);
cudaError_t enqueue_correlation(int M, double L, const double *grid, int all_origins, double *C, cudaStream_t s);
cudaError_t enqueue_defects(int M, const double *grid, signed char *map, unsigned long long *counts, cudaStream_t s);
cudaError_t enqueue_mixing(const DevParams &P, const Bufs &b, const unsigned char *colors, int G, int S,
                           unsigned *cnt, cudaStream_t s);
// Neighbour graph of the present positions in the cell-sorted order of the last search, for the
// learned surrogate (row g is particle ids[g]): the neighbours closer than 2h as ELL rows (entry k
// of row g at k * n + g, neighbours as sorted indices) with W and S2 = W(0) + sum W; and over the
// support (3h) the SPH means of (ux, uy, Q11, Q12) and of the recorded acceleration, and from them
// the network's input rows.
struct GraphOut {
    int *nbr;               // MAXN2H x n neighbour sorted indices (2h)
    float *W;               // MAXN2H x n kernel values W(|x_i - x_j|)
    unsigned *overflow;     // set when a particle has more than MAXN2H neighbours closer than 2h
    int *cnt2;              // n: neighbours closer than 2h
    float *S2;              // n: W(0) + sum_j W over them
    double *x, *y;          // n: positions
    float4 *u4;             // n: (ux, uy, q11, q12)
    float *dr;              // n: rho / rho0 - 1
    int *ids;               // n: particle ID of sorted row g
    float *agg1;            // 2 x n: SPH mean of (ax, ay) over the support
    const float *tend_id;   // 8 x n tendencies by particle ID (ax, ay, m11, m12, lapQ, div, vort)
    __nv_bfloat16 *X;       // n x 16: the network's input rows (BF16)
    float inv_us;           // 1 / velocity scale
    float scale[4];         // tendency scales per pair of channels (a, m, lap Q, div / vort)
};
// The export, then inc (n x 4, sorted order) = kdt (m11, m12, agg(agg1)) with a second walk.
cudaError_t enqueue_export_graph(const DevParams &P, const Bufs &b, const GraphOut &o, float kdt, float *inc,
                                 cudaStream_t s);

// Context hooks for the surrogate (implemented in ann_api.cu; the context itself stays opaque).
struct CtxView {
    DevParams P;
    Bufs b;
    cudaStream_t stream;
    double *tmp;   // staging of at least 7 n doubles
    double t;
    int64_t steps;
    bool rec_valid;   // the last step recorded grad u, lap Q and a
};
int ctx_view(ann_ctx *c, CtxView *v);
int ctx_search_present(ann_ctx *c);                                  // search at the present positions
int ctx_commit_in_place(ann_ctx *c, int64_t add_steps);              // S was rewritten in the order of M

// BF16 tensor-core GEMMs of the surrogate (ann_mlp.cu).  K, N multiples of 16 in [16, 256].
bool gemm_shape_ok(int K, int N);
// ldc: row stride of C in elements (0: N)
cudaError_t enqueue_gemm_nt(const void *A1, int K1, const void *A2, int K2, const void *B, int N, int rows,
                            const float *bias, int relu, void *C, int c_bf16, int accumulate, unsigned *err,
                            int max_ctas, cudaStream_t s, int ldc = 0);
cudaError_t enqueue_gemm_tn(const void *A, int K, const void *B, int N, int rows, float *C, unsigned *err,
                            int max_ctas, cudaStream_t s, int ldc = 0);
// One surrogate layer: h = relu([A1 | A2] W^T + bw) (128 wide; to H unless null), z = h P^T + bp
// (Np wide, bp may be null; BF16 or FP32).  W 128 x (K1 + K2), P Np x 128, BF16, 16-byte aligned.
cudaError_t enqueue_layer(const void *A1, int K1, const void *A2, int K2, const void *W, const float *bw,
                          const void *P, const float *bp, int Np, void *H, void *Z, int z_bf16, int rows,
                          unsigned *err, int max_ctas, cudaStream_t s);
cudaError_t enqueue_unwrapped(const DevParams &P, const Bufs &b, int *inv, const long long *ids, int k, double *xy,
                              cudaStream_t s);

}  // namespace ann

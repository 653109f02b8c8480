// C-ABI of the SPH active-nematic solver: context, device buffers, CUDA-graph step, I/O.
#include "../../include/ann.h"
#include "ann_internal.cuh"

#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <new>
#include <string>
#include <vector>

using namespace ann;

struct ann_ctx {
    ann_params prm{};
    DevParams P{};
    Bufs b{};
    int device = 0;
    cudaStream_t own = nullptr;
    cudaStream_t aux = nullptr;     // captures the bodies of the step graph's conditional node
    cudaStream_t stream = nullptr;
    cudaGraphExec_t exec = nullptr;
    bool have_particles = false;
    int64_t steps = 0;
    double t = 0.0;
    std::string last_err;
    ann_allocator al{};           // device memory provider (alloc == nullptr: cudaMalloc / cudaFree)
    bool al_misaligned = false;   // the provider returned a pointer that is not 16-byte aligned
    std::vector<std::pair<void *, size_t>> allocs;
    void *tmp = nullptr;          // staging: max(7 n doubles, MAXN n ints)
    double *diag_part = nullptr;  // diag_blocks(n) x NDIAG
    double *diag_out = nullptr;   // NDIAG
    uint32_t *h_err = nullptr;    // pinned
    uint32_t *h_ctl = nullptr;    // pinned: step control words and the error word read back, words to write
    int cur = 0;                  // the state set the host view (b.sx, ...) points at: the committed one
    // Which arrays hold the present state in the cell order of the last re-sort (the order the
    // flow diagnostics need): S after a step or a load that kept the cell structure, the
    // evaluation copy M after a neighbour export; neither after ann_set_particles.
    bool s_sorted = false, m_current = false;
    bool rec_valid = false;   // the last step ran with recording on (GRADU, LAPQ, APD and a are its values)
    // flow diagnostics (allocated on first use, sized for the largest request so far)
    unsigned char *colors = nullptr;   // by particle ID (n)
    int ncolors = 1;                   // largest colour + 1
    int *inv = nullptr;                // slot of each particle ID (n)
    struct Scratch {
        void *p = nullptr;
        size_t bytes = 0;
    } d_grid, d_off, d_fld, d_z, d_zt, d_tw, d_shoff, d_shmodes, d_out, d_map, d_cnt, d_ids;
    int grid_M = 0, tw_M = 0, shell_M = 0;
    int64_t grid_step = -1;            // step count of the gridded fields in d_grid (-1: none)
};

namespace {

constexpr double kCellSlack = 1e-9;

const char *status_text(int s)
{
    switch (s) {
    case ANN_OK: return "ok";
    case ANN_ERR_INVALID_ARG: return "invalid argument";
    case ANN_ERR_OOM: return "out of memory";
    case ANN_ERR_CUDA: return "CUDA error";
    case ANN_ERR_CELL_OVERFLOW: return "cell or tile halo overflow";
    case ANN_ERR_NBR_OVERFLOW: return "neighbour list overflow";
    case ANN_ERR_NONFINITE: return "non-finite state";
    case ANN_ERR_SINGULAR_ALPHA: return "singular correction tensor";
    case ANN_ERR_IO: return "checkpoint I/O error";
    case ANN_ERR_STATE: return "call out of order";
    case ANN_ERR_NOT_AVAILABLE: return "no CUDA device";
    case ANN_ERR_TOO_LARGE: return "size beyond the fixed scratch of a no-allocation entry point";
    case ANN_ERR_TIMEOUT: return "a bounded device wait timed out";
    case ANN_ERR_CFL_VIOLATION: return "dt above a stability limit (CFL)";
    default: return "unknown status";
    }
}

int fail(ann_ctx *c, int code, const std::string &msg)
{
    if (c) c->last_err = msg;
    return code;
}

int cuda_fail(ann_ctx *c, cudaError_t e, const char *where)
{
    return fail(c, e == cudaErrorMemoryAllocation ? ANN_ERR_OOM : ANN_ERR_CUDA,
                std::string(where) + ": " + cudaGetErrorString(e));
}

bool finite_pos(double v) { return std::isfinite(v) && v > 0.0; }

// Cells are at least as wide as the candidate radius 3h (1 + SKIN).
int cells_per_side(const ann_params &p)
{
    return (int)std::floor(p.L / (3.0 * p.h * (1.0 + SKIN) * (1.0 + kCellSlack)));
}

double effective_dt(const ann_params &p)
{
    double dt = p.dt;
    if (p.dt_mode == ANN_DT_STABLE) {
        double nu = p.eta / p.rho0;
        if (nu > 0.0) dt = std::min(dt, 0.125 * p.h * p.h / nu);
        if (p.Gamma * p.K > 0.0) dt = std::min(dt, 0.125 * p.h * p.h / (p.Gamma * p.K));
        if (p.c0_min > 0.0) dt = std::min(dt, 0.25 * p.h / p.c0_min);
    }
    return dt;
}

int64_t device_bytes(const ann_params &p)
{
    int64_t n = p.n, nc = cells_per_side(p), ncell = nc * nc;
    int64_t per = 2 * 8 + 7 * 4 + 4 + 16      // S
                  + 2 * 8 + 5 * 4 + 16 + 4    // M
                  + 3 * 4                     // key, rank, perm
                  + 4                         // neighbour counts (the neighbour bits sit in the lists)
                  + (MAXV / 2) * 4 + 4 + 16 + 4   // candidate lists, counts, split at re-sort, cell
                  + 4 * 4 + 3 * 16            // intermediates: sum W, V, delta_half, p; (B, k), (div Q, delta_hat,
                                              // sum W) and pass D's staged record (V, p/rho^2, u) as float4
                  + 10 * 4                    // recording
                  + 16 + 8                    // elastic stress and its divergence
                  + 8 + 1 + 4                 // image counts, colour, inverse order (diagnostics)
                  + 2 * 8 + 7 * 4 + 4         // the second state set (a step writes it, rollback keeps the first)
                  + 2;                        // crossing log (n/8 entries of 16 bytes)
    int64_t tmp = 7 * 8 * n;                  // staging of state and field transfers
    return per * n + tmp + 2 * 4 * (ncell + 1) + 4096;
}

int validate(const ann_params *p, std::string &why)
{
    if (!p) { why = "null parameters"; return ANN_ERR_INVALID_ARG; }
    // 2^29 keeps every per-particle index of the kernels (up to 4 n for the recorded gradient) in
    // int32; at ~663 bytes per particle that is 356 GB, beyond one GPU's memory anyway
    if (p->n < 1 || p->n > (int64_t)1 << 29) { why = "n must be in [1, 2^29]"; return ANN_ERR_INVALID_ARG; }
    if (!finite_pos(p->L) || !finite_pos(p->h) || !finite_pos(p->dt) || !finite_pos(p->rho0)) {
        why = "L, h, dt and rho0 must be finite and positive";
        return ANN_ERR_INVALID_ARG;
    }
    if (cells_per_side(*p) < 3) { why = "need at least three cells of side 3h across the box"; return ANN_ERR_INVALID_ARG; }
    const double nonneg[] = {p->eta, p->Gamma, p->gamma_eos, p->c0_min};
    for (double v : nonneg)
        if (!std::isfinite(v) || v < 0.0) { why = "eta, Gamma, gamma_eos, c0_min must be finite and >= 0"; return ANN_ERR_INVALID_ARG; }
    if (!(p->gamma_eos > 0.0)) { why = "gamma_eos must be > 0"; return ANN_ERR_INVALID_ARG; }
    if (!(p->beta >= 0.0 && p->beta <= 1.0)) { why = "beta must be in [0, 1]"; return ANN_ERR_INVALID_ARG; }
    const double fin[] = {p->lambda, p->A, p->B, p->C, p->K, p->zeta, p->c_shift};
    for (double v : fin)
        if (!std::isfinite(v)) { why = "lambda, A, B, C, K, zeta, c_shift must be finite"; return ANN_ERR_INVALID_ARG; }
    if (p->apd != 0 && p->apd != 1) { why = "apd must be 0 or 1"; return ANN_ERR_INVALID_ARG; }
    if (p->momentum_mode != ANN_MOMENTUM_PAPER && p->momentum_mode != ANN_MOMENTUM_CONSERVATIVE) {
        why = "unknown momentum_mode";
        return ANN_ERR_INVALID_ARG;
    }
    if (p->q_new_in_momentum != 0 && p->q_new_in_momentum != 1) { why = "q_new_in_momentum must be 0 or 1"; return ANN_ERR_INVALID_ARG; }
    if (p->dt_mode != ANN_DT_FIXED && p->dt_mode != ANN_DT_STABLE && p->dt_mode != ANN_DT_CHECK) {
        why = "unknown dt_mode";
        return ANN_ERR_INVALID_ARG;
    }
    if (p->elastic_stress != 0 && p->elastic_stress != 1) { why = "elastic_stress must be 0 or 1"; return ANN_ERR_INVALID_ARG; }
    double R = 3.0 * p->h;
    double expected = M_PI * R * R * (double)p->n / (p->L * p->L);
    if (expected > 0.85 * MAXN) { why = "too many expected neighbours for the list capacity"; return ANN_ERR_INVALID_ARG; }
    // a 4 x 4-cell tile plus halo must fit its staging buffer with room for fluctuations
    double cell = p->L / cells_per_side(*p);
    double per_cell = (double)p->n * cell * cell / (p->L * p->L);
    if (per_cell * NHC > 0.7 * HCAP || per_cell > 0.6 * MAXC) {
        why = "too many particles per cell (3h is large against the particle spacing)";
        return ANN_ERR_INVALID_ARG;
    }
    return ANN_OK;
}

DevParams make_dev(const ann_params &p)
{
    DevParams d{};
    d.n = (int)p.n;
    d.nc = cells_per_side(p);
    d.ncell = d.nc * d.nc;
    d.tiles = (d.nc + TILE - 1) / TILE;
    d.apd = p.apd;
    d.conservative = p.momentum_mode == ANN_MOMENTUM_CONSERVATIVE;
    d.qnew = p.q_new_in_momentum;
    d.record = 0;
    d.elastic = p.elastic_stress;
    d.L = p.L;
    d.cell = p.L / d.nc;
    d.inv_cell = (double)d.nc / p.L;
    d.R2 = (3.0 * p.h) * (3.0 * p.h);
    double dt = effective_dt(p);
    d.dt_d = dt;
    d.half_dt_d = 0.5 * dt;
    // Pair vectors are formed as (hi_i - hi_j) + (lo_i - lo_j): the hi parts lie on a power-of-two
    // grid q = 2^(floor(log2 cell) - 12) with at most 16 significant bits, so their difference is
    // exact in FP32 and d is correctly rounded up to ~2^-33 cell.  |d|^2 is then within
    // 4 * 2^-24 of the FP64 value; pairs within a relative band of 2^-20 of (3h)^2 are decided in
    // FP64 from the positions, exactly as the definition states.
    int ex = 0;
    std::frexp(d.cell, &ex);               // cell = m 2^ex, m in [0.5, 1)
    d.q = std::ldexp(1.0, ex - 13);
    d.qf = (float)d.q;
    d.iqf = (float)(1.0 / d.q);
    {
        double L = p.L;
        std::memcpy(&d.bitsL, &L, sizeof L);
    }
    double chi = std::nearbyint(d.cell / d.q) * d.q;
    d.cell_hi = (float)chi;
    d.cell_lo = (float)(d.cell - chi);
    const double band = 1.0 / 1048576.0;
    d.R2lo = (float)(d.R2 * (1.0 - band));
    d.R2hi = (float)(d.R2 * (1.0 + band));
    d.inv_h = (float)(1.0 / p.h);
    double ad = 7.0 / (478.0 * M_PI * p.h * p.h);
    d.ad = (float)ad;
    d.W0 = (float)(ad * 66.0);   // W(0) = a_d (3^5 - 6 2^5 + 15)
    d.kw6 = (float)(-6.0 * ad);
    d.kw15 = (float)(15.0 * ad);
    d.kf5 = (float)(-5.0 * ad / p.h);
    d.kf30 = (float)(30.0 * ad / p.h);
    d.kf75 = (float)(-75.0 * ad / p.h);
    // Candidates are first tested on the hi parts alone.  |lo| <= q/2 + 5 |cell_lo| <= 3q per
    // coordinate, so the hi-only distance is within 6 sqrt(2) q < 9q of the true one; the coarse
    // radius 3h + 9q (rounded up) keeps every neighbour.
    double Rv = 3.0 * p.h * (1.0 + SKIN);
    d.R2c = (float)((Rv + 9.0 * d.q) * (Rv + 9.0 * d.q) * (1.0 + 1.0 / 1048576.0));
    d.R2v = (float)(Rv * Rv * (1.0 + 1.0 / 262144.0));
    // A pair within 3h at some step was within 3h + 2 * (SKIN 3h / 2) = Rv at the last re-sort as
    // long as no particle has moved SKIN 3h / 2 since; past that the step re-sorts.
    double smax = 0.5 * SKIN * 3.0 * p.h;
    d.skin_max2 = (float)(smax * smax);
    d.nsblk = (d.ncell + SCAN_CHUNK - 1) / SCAN_CHUNK;
    d.dt = (float)dt;
    d.half_dt = (float)(0.5 * dt);
    d.rho0 = (float)p.rho0;
    d.nu = (float)(p.eta / p.rho0);
    d.mu = (float)p.eta;
    d.Gamma = (float)p.Gamma;
    d.lambda = (float)p.lambda;
    d.A = (float)p.A;
    d.Bl = (float)p.B;
    d.C = (float)p.C;
    d.K = (float)p.K;
    d.zeta = (float)p.zeta;
    d.gamma_eos = (float)p.gamma_eos;
    d.beta = (float)p.beta;
    d.c0_min = (float)p.c0_min;
    d.c_shift = (float)p.c_shift;
    d.mass = (float)(p.rho0 * p.L * p.L / (double)p.n);
    d.dt_check = p.dt_mode == ANN_DT_CHECK;
    {
        double lim = INFINITY, nu = p.eta / p.rho0;
        if (nu > 0.0) lim = std::min(lim, 0.125 * p.h * p.h / nu);
        if (p.Gamma * p.K > 0.0) lim = std::min(lim, 0.125 * p.h * p.h / (p.Gamma * p.K));
        d.dt_static = (float)lim;
    }
    return d;
}

// Device memory of a context: from its ann_allocator when it has one, else cudaMalloc.
cudaError_t dev_alloc(ann_ctx *c, void **v, size_t bytes)
{
    *v = nullptr;
    if (!c->al.alloc) return cudaMalloc(v, bytes);
    void *p = c->al.alloc(bytes, (void *)c->own, c->al.user);
    if (!p) return cudaErrorMemoryAllocation;
    if ((uintptr_t)p & 15u) {
        c->al.release(p, bytes, (void *)c->own, c->al.user);
        c->al_misaligned = true;
        return cudaErrorInvalidValue;
    }
    *v = p;
    return cudaSuccess;
}

void dev_free(ann_ctx *c, void *v, size_t bytes)
{
    if (!v) return;
    if (c->al.release) c->al.release(v, bytes, (void *)c->own, c->al.user);
    else cudaFree(v);
}

template <typename T>
cudaError_t dalloc(ann_ctx *c, T *&ptr, size_t count)
{
    void *v = nullptr;
    const size_t bytes = std::max<size_t>(count, 1) * sizeof(T);
    cudaError_t e = dev_alloc(c, &v, bytes);
    if (e) return e;
    c->allocs.emplace_back(v, bytes);
    ptr = static_cast<T *>(v);
    return cudaMemset(v, 0, bytes);
}

cudaError_t alloc_all(ann_ctx *c)
{
    size_t n = (size_t)c->P.n, ncell = (size_t)c->P.ncell;
    Bufs &b = c->b;
    cudaError_t e;
#define A_(p, cnt) if ((e = dalloc(c, b.p, cnt))) return e
    A_(sx, n); A_(sy, n); A_(sux, n); A_(suy, n); A_(sq11, n); A_(sq12, n); A_(sdr, n); A_(sax, n);
    A_(say, n); A_(sid, n); A_(sxi, n);
    A_(mx, n); A_(my, n); A_(mu4, n); A_(mdr, n); A_(xi, n); A_(mid, n);
    A_(cell_count, ncell + 1); A_(cell_start, ncell + 1); A_(key, n); A_(rank, n); A_(perm, n);
    A_(nnbr, n);
    A_(vnbr, n * (MAXV / 4)); A_(vcnt, n); A_(xi_ref, n); A_(mkey, n); A_(rebuild, 1); A_(resorts, 1);
    A_(sumW, n); A_(V, n); A_(bk, n); A_(cr, n);
    A_(p, n); A_(rd, n); A_(cq, n);
    A_(rec_gu, 4 * n); A_(rec_lap, 2 * n); A_(rec_apd, 2 * n); A_(rec_qrate, 2 * n);
    A_(pel, n); A_(delx, n); A_(dely, n); A_(img, n);
    A_(err, 1); A_(maxu, 1); A_(band, 1);
    // the state sets: st[0] is the storage the host view starts on, st[1] the step's other copy
    b.st[0] = StateSet{b.sx, b.sy, b.sux, b.suy, b.sq11, b.sq12, b.sdr, b.sax, b.say, b.sid};
    A_(st[1].x, n); A_(st[1].y, n); A_(st[1].ux, n); A_(st[1].uy, n); A_(st[1].q11, n); A_(st[1].q12, n);
    A_(st[1].dr, n); A_(st[1].ax, n); A_(st[1].ay, n); A_(st[1].id, n);
    A_(ctl, CTL_WORDS);
    b.xlog_cap = (int)std::max<size_t>(1024, n / 8);
    A_(xlog, (size_t)b.xlog_cap);
#undef A_
    double *origin = nullptr;
    if ((e = dalloc(c, origin, (size_t)c->P.nc))) return e;
    {
        std::vector<double> h((size_t)c->P.nc);
        for (int k = 0; k < c->P.nc; k++) h[(size_t)k] = (double)k * c->P.cell;
        if ((e = cudaMemcpy(origin, h.data(), sizeof(double) * h.size(), cudaMemcpyHostToDevice))) return e;
    }
    b.origin = origin;
    unsigned char *tmp = nullptr;
    if ((e = dalloc(c, tmp, (size_t)(7 * 8) * n))) return e;
    c->tmp = tmp;
    if ((e = dalloc(c, c->colors, n))) return e;
    if ((e = dalloc(c, c->inv, n))) return e;
    if ((e = dalloc(c, c->diag_part, (size_t)diag_blocks((int)n) * NDIAG))) return e;
    if ((e = dalloc(c, c->diag_out, NDIAG))) return e;
    return cudaSuccess;
}

// The step graph: predict -> set-condition -> IF (re-sort flag) { keys, scan, scatter, cell order,
// re-sort pass A } ELSE { pass A } -> passes B, C, D.  The branch not taken costs nothing.
// capture_step records one step of context c onto stream s, which is capturing into graph g (the
// context's own graph, or an ensemble graph holding many contexts); the bodies of the conditional
// node are captured on the context's aux stream.
cudaError_t capture_step(ann_ctx *c, cudaStream_t s, cudaGraph_t g)
{
    cudaGraphConditionalHandle h = 0;
    cudaError_t ec = cudaGraphConditionalHandleCreate(&h, g, 0, cudaGraphCondAssignDefault);
    if (!ec) ec = launch_commit(c->b, s);
    if (!ec) ec = launch_kernel(0, c->P, c->b, s);
    if (!ec) ec = launch_set_condition(c->b, h, s);
    cudaGraph_t body[2] = {nullptr, nullptr};
    if (!ec) {
        cudaStreamCaptureStatus st;
        const cudaGraphNode_t *deps = nullptr;
        size_t nd = 0;
        cudaGraph_t capg = nullptr;
        ec = cudaStreamGetCaptureInfo(s, &st, nullptr, &capg, &deps, nullptr, &nd);
        cudaGraphNode_t cn = nullptr;
        if (!ec) {
            // zeroed storage: the parameter struct's union has no default constructor
            alignas(cudaGraphNodeParams) unsigned char raw[sizeof(cudaGraphNodeParams)] = {};
            cudaGraphNodeParams &cp = *reinterpret_cast<cudaGraphNodeParams *>(raw);
            cp.type = cudaGraphNodeTypeConditional;
            cp.conditional.handle = h;
            cp.conditional.type = cudaGraphCondTypeIf;
            cp.conditional.size = 2;
            ec = cudaGraphAddNode(&cn, capg, deps, nullptr, nd, &cp);
            if (!ec) {
                body[0] = cp.conditional.phGraph_out[0];
                body[1] = cp.conditional.phGraph_out[1];
            }
        }
        if (!ec) ec = cudaStreamUpdateCaptureDependencies(s, &cn, nullptr, 1, cudaStreamSetCaptureDependencies);
    }
    for (int k = 0; k < 2 && !ec; k++) {
        ec = cudaStreamBeginCaptureToGraph(c->aux, body[k], nullptr, nullptr, 0, cudaStreamCaptureModeThreadLocal);
        if (ec) break;
        cudaError_t el = cudaSuccess;
        if (k == 0)
            for (int q = 1; q <= 5 && !el; q++) el = launch_kernel(q, c->P, c->b, c->aux);
        else
            el = launch_kernel(6, c->P, c->b, c->aux);
        cudaGraph_t got = body[k];
        ec = cudaStreamEndCapture(c->aux, &got);
        if (!ec) ec = el;
    }
    for (int k = 7; k < NKERNELS && !ec; k++) ec = launch_kernel(k, c->P, c->b, s);
    return ec;
}

cudaError_t capture(ann_ctx *c)
{
    if (c->exec) {
        cudaGraphExecDestroy(c->exec);
        c->exec = nullptr;
    }
    cudaGraph_t g = nullptr;
    cudaError_t e = cudaGraphCreate(&g, 0);
    if (e) return e;
    e = cudaStreamBeginCaptureToGraph(c->own, g, nullptr, nullptr, 0, cudaStreamCaptureModeThreadLocal);
    if (e) {
        cudaGraphDestroy(g);
        return e;
    }
    cudaError_t ec = capture_step(c, c->own, g);
    e = cudaStreamEndCapture(c->own, &g);
    if (ec || e) {
        if (g) cudaGraphDestroy(g);
        return ec ? ec : e;
    }
    e = cudaGraphInstantiate(&c->exec, g, 0);
    cudaGraphDestroy(g);
    return e;
}

// Read and clear nothing: returns the status implied by the sticky device error word.
int device_status(ann_ctx *c)
{
    cudaError_t e = cudaMemcpyAsync(c->h_err, c->b.err, sizeof(uint32_t), cudaMemcpyDeviceToHost, c->stream);
    if (!e) e = cudaStreamSynchronize(c->stream);
    if (e) return cuda_fail(c, e, "reading the device status");
    uint32_t bits = *c->h_err;
    if (!bits) return ANN_OK;
    char buf[160];
    std::snprintf(buf, sizeof buf,
                  "device error bits 0x%x (1 cell, 2 halo, 4 neighbours, 8 non-finite, 16 alpha, 32 CFL)", bits);
    c->last_err = buf;
    if (bits & EB_NONFINITE) return ANN_ERR_NONFINITE;
    if (bits & (EB_CELL | EB_HALO)) return ANN_ERR_CELL_OVERFLOW;
    if (bits & EB_NBR) return ANN_ERR_NBR_OVERFLOW;
    if (bits & EB_CFL) return ANN_ERR_CFL_VIOLATION;
    return ANN_ERR_SINGULAR_ALPHA;
}

// Clears the sticky error bits and counters and schedules a re-sort for the next step.
cudaError_t clear_flags(ann_ctx *c)
{
    cudaError_t e = cudaMemsetAsync(c->b.err, 0, sizeof(uint32_t), c->stream);
    if (!e) e = cudaMemsetAsync(c->b.rebuild, 1, sizeof(uint32_t), c->stream);
    if (!e) e = cudaMemsetAsync(c->b.maxu, 0, sizeof(uint32_t), c->stream);
    if (!e) e = cudaMemsetAsync(c->b.cell_count, 0, sizeof(uint32_t) * (c->P.ncell + 1), c->stream);
    // no step pending, counters cleared; the committed set (ctl[CTL_CUR]) stays the host view's
    if (!e) e = cudaMemsetAsync(c->b.ctl + CTL_PENDING, 0, sizeof(uint32_t) * (CTL_WORDS - CTL_PENDING), c->stream);
    return e;
}

// Point the host view of the state (b.sx, ...) at state set k.
void set_view(ann_ctx *c, int k)
{
    c->cur = k;
    const StateSet &t = c->b.st[k];
    Bufs &b = c->b;
    b.sx = t.x;
    b.sy = t.y;
    b.sux = t.ux;
    b.suy = t.uy;
    b.sq11 = t.q11;
    b.sq12 = t.q12;
    b.sdr = t.dr;
    b.sax = t.ax;
    b.say = t.ay;
    b.sid = t.id;
}

// After a batch of `launched` steps (graph replays or the profiled loop): with no error raised the
// last step is committed here (the next step's k_commit would do it); after an error the failed
// step is rolled back -- its output set is dropped, so the committed set is the state of the last
// completed step, the image counts it changed are restored from its crossing log, and the next
// step re-sorts, as the failed step may have re-sorted the cell structure.  Adds the completed
// steps to the step count and time; returns the status of the device error word.
int settle_steps(ann_ctx *c, int64_t launched)
{
    uint32_t *h = c->h_ctl;   // [0, CTL_WORDS) read back, [CTL_WORDS] the error word, then the words to write
    cudaError_t e = cudaMemcpyAsync(h, c->b.ctl, sizeof(uint32_t) * CTL_WORDS, cudaMemcpyDeviceToHost, c->stream);
    if (!e) e = cudaMemcpyAsync(h + CTL_WORDS, c->b.err, sizeof(uint32_t), cudaMemcpyDeviceToHost, c->stream);
    if (!e) e = cudaStreamSynchronize(c->stream);
    if (e) return cuda_fail(c, e, "reading the step status");
    const bool failed = h[CTL_WORDS] != 0u;
    uint32_t cur = h[CTL_CUR] & 1u;
    int64_t done = launched;
    bool log_lost = false;
    if (!failed) {
        if (h[CTL_PENDING]) cur ^= 1u;
    } else {
        done = std::min<int64_t>(launched, h[CTL_COMMITS]);
        const uint32_t nlog = h[CTL_XLOG];
        log_lost = nlog > (uint32_t)c->b.xlog_cap;
        e = enqueue_undo_crossings(c->b, (int)std::min<uint32_t>(nlog, (uint32_t)c->b.xlog_cap), c->stream);
        if (!e) e = cudaMemsetAsync(c->b.rebuild, 1, sizeof(uint32_t), c->stream);
    }
    uint32_t *w = h + CTL_WORDS + 1;
    w[CTL_CUR] = cur;
    w[CTL_PENDING] = 0u;
    w[CTL_COMMITS] = 0u;
    w[CTL_XLOG] = 0u;
    if (!e) e = cudaMemcpyAsync(c->b.ctl, w, sizeof(uint32_t) * CTL_WORDS, cudaMemcpyHostToDevice, c->stream);
    if (e) return cuda_fail(c, e, "settling the steps");
    set_view(c, (int)cur);
    c->steps += done;
    c->t += done * c->P.dt_d;
    if (done > 0 || failed) {
        c->s_sorted = !failed;   // after a rollback the cell structure may not follow the state
        c->m_current = false;
        c->grid_step = -1;
        c->rec_valid = !failed && c->P.record != 0;
    }
    int st = device_status(c);   // synchronises: the words above are written when this returns
    if (failed) {
        c->last_err += "; the state is that of the last completed step (" + std::to_string(c->steps) + ")";
        if (log_lost) c->last_err += "; more crossings than the log holds: image counts not restored";
    }
    return st;
}

struct Field {
    const void *ptr;
    int es;
    bool state;   // in S order (else M order)
    int stride;   // interleaved component count
    int comp;
};

bool field_of(ann_ctx *c, int f, Field &out)
{
    const Bufs &b = c->b;
    out = Field{nullptr, 4, false, 1, 0};
    switch (f) {
    case ANN_FIELD_X: out = {b.sx, 8, true, 1, 0}; return true;
    case ANN_FIELD_Y: out = {b.sy, 8, true, 1, 0}; return true;
    case ANN_FIELD_UX: out = {b.sux, 4, true, 1, 0}; return true;
    case ANN_FIELD_UY: out = {b.suy, 4, true, 1, 0}; return true;
    case ANN_FIELD_Q11: out = {b.sq11, 4, true, 1, 0}; return true;
    case ANN_FIELD_Q12: out = {b.sq12, 4, true, 1, 0}; return true;
    case ANN_FIELD_DRHO: out = {b.sdr, 4, true, 1, 0}; return true;
    case ANN_FIELD_AX: out = {b.sax, 4, true, 1, 0}; return true;
    case ANN_FIELD_AY: out = {b.say, 4, true, 1, 0}; return true;
    case ANN_FIELD_SUMW: out.ptr = b.sumW; return true;
    case ANN_FIELD_V: out.ptr = b.V; return true;
    case ANN_FIELD_B11: case ANN_FIELD_B12: case ANN_FIELD_B22: case ANN_FIELD_K:
        out = {b.bk, 4, false, 4, f - ANN_FIELD_B11}; return true;
    case ANN_FIELD_DRHO_HALF: out = {b.cr, 4, false, 4, 1}; return true;
    case ANN_FIELD_DRHO_HAT: out = {b.cq, 4, false, 4, 2}; return true;
    case ANN_FIELD_P: out.ptr = b.p; return true;
    case ANN_FIELD_DIVQX: case ANN_FIELD_DIVQY:
        out = {b.cq, 4, false, 4, f - ANN_FIELD_DIVQX}; return true;
    case ANN_FIELD_NNBR: out.ptr = b.nnbr; return true;
    case ANN_FIELD_GRADU_XX: case ANN_FIELD_GRADU_XY: case ANN_FIELD_GRADU_YX: case ANN_FIELD_GRADU_YY:
        out = {b.rec_gu, 4, false, 4, f - ANN_FIELD_GRADU_XX}; return true;
    case ANN_FIELD_LAPQ11: case ANN_FIELD_LAPQ12:
        out = {b.rec_lap, 4, false, 2, f - ANN_FIELD_LAPQ11}; return true;
    case ANN_FIELD_APDX: case ANN_FIELD_APDY:
        out = {b.rec_apd, 4, false, 2, f - ANN_FIELD_APDX}; return true;
    case ANN_FIELD_QRATE11: case ANN_FIELD_QRATE12:
        out = {b.rec_qrate, 4, false, 2, f - ANN_FIELD_QRATE11}; return true;
    default: return false;
    }
}

// ann_set_state's load: the state as the context stores it (FP64 positions, FP32 fields, the
// density as its deviation), re-inserted into the box as ann_set_particles does.
__global__ void k_load_state(DevParams P, Bufs b, const double *x, const double *y, const float *ux,
                             const float *uy, const float *q11, const float *q12, const float *drho)
{
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= P.n) return;
    double xx = x[i], yy = y[i];
    const float d = drho ? drho[i] : 0.f;
    if (!(isfinite(xx) && isfinite(yy) && isfinite(ux[i]) && isfinite(uy[i]) && isfinite(q11[i]) &&
          isfinite(q12[i]) && isfinite(d) && d > -1.f)) {
        atomicOr(b.err, EB_NONFINITE);
        xx = 0.0;
        yy = 0.0;
    }
    if (xx < -P.L || xx >= 2.0 * P.L) xx = xx - floor(xx / P.L) * P.L;
    if (yy < -P.L || yy >= 2.0 * P.L) yy = yy - floor(yy / P.L) * P.L;
    if (xx < 0.0) xx += P.L;
    if (xx >= P.L) xx -= P.L;
    if (yy < 0.0) yy += P.L;
    if (yy >= P.L) yy -= P.L;
    b.sx[i] = xx + 0.0;
    b.sy[i] = yy + 0.0;
    b.sux[i] = ux[i];
    b.suy[i] = uy[i];
    b.sq11[i] = q11[i];
    b.sq12[i] = q12[i];
    b.sdr[i] = d;
    b.sax[i] = 0.f;
    b.say[i] = 0.f;
    b.sid[i] = i;
    b.img[i] = make_int2(0, 0);
}

// Slot g of the state takes particle id's values, checked and re-inserted into the box.
__device__ __forceinline__ void store_slot(const DevParams &P, const Bufs &b, int g, int id, double xx, double yy,
                                          float ux, float uy, float q11, float q12, float d, float a0, float a1)
{
    if (!(isfinite(xx) && isfinite(yy) && isfinite(ux) && isfinite(uy) && isfinite(q11) && isfinite(q12) &&
          isfinite(d) && d > -1.f && isfinite(a0) && isfinite(a1))) {
        atomicOr(b.err, EB_NONFINITE);
        xx = 0.0;
        yy = 0.0;
    }
    if (xx < -P.L || xx >= 2.0 * P.L) xx = xx - floor(xx / P.L) * P.L;
    if (yy < -P.L || yy >= 2.0 * P.L) yy = yy - floor(yy / P.L) * P.L;
    if (xx < 0.0) xx += P.L;
    if (xx >= P.L) xx -= P.L;
    if (yy < 0.0) yy += P.L;
    if (yy >= P.L) yy -= P.L;
    b.sx[g] = xx + 0.0;
    b.sy[g] = yy + 0.0;
    b.sux[g] = ux;
    b.suy[g] = uy;
    b.sq11[g] = q11;
    b.sq12[g] = q12;
    b.sdr[g] = d;
    b.sax[g] = a0;
    b.say[g] = a1;
    b.sid[g] = id;
}

// ann_update_state from device arrays: slot g takes particle ids[g]'s values (ids: the particle at
// each slot in the order of the last re-sort), so the cell structure and candidate lists stay valid.
__global__ void k_update_state(DevParams P, Bufs b, const int *ids, const double *x, const double *y,
                               const float *ux, const float *uy, const float *q11, const float *q12,
                               const float *drho, const float *ax, const float *ay)
{
    int g = blockIdx.x * blockDim.x + threadIdx.x;
    if (g >= P.n) return;
    const int id = ids[g];
    store_slot(P, b, g, id, x[id], y[id], ux[id], uy[id], q11[id], q12[id], drho ? drho[id] : 0.f,
               ax ? ax[id] : 0.f, ay ? ay[id] : 0.f);
}

// inv[ids[g]] = g: the slot of each particle.
__global__ void k_invert(const int *ids, int *inv, int n)
{
    int g = blockIdx.x * blockDim.x + threadIdx.x;
    if (g < n) inv[ids[g]] = g;
}

// ann_update_state from page-locked host arrays that the device maps: thread i reads particle i
// (a warp reads whole consecutive lines over the host link) and writes its slot inv[i].
__global__ void k_update_state_mapped(DevParams P, Bufs b, const int *inv, const double *x, const double *y,
                                      const float *ux, const float *uy, const float *q11, const float *q12,
                                      const float *drho, const float *ax, const float *ay)
{
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= P.n) return;
    store_slot(P, b, inv[i], i, x[i], y[i], ux[i], uy[i], q11[i], q12[i], drho ? drho[i] : 0.f,
               ax ? ax[i] : 0.f, ay ? ay[i] : 0.f);
}

// ann_get_state into page-locked host arrays that the device maps: particle i's values from its
// slot inv[i], written in particle order (NULL destinations skipped).
__global__ void k_get_state_mapped(Bufs b, int n, const int *inv, double *x, double *y, float *ux, float *uy,
                                   float *q11, float *q12, float *drho, float *ax, float *ay)
{
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const int g = inv[i];
    if (x) x[i] = b.sx[g];
    if (y) y[i] = b.sy[g];
    if (ux) ux[i] = b.sux[g];
    if (uy) uy[i] = b.suy[g];
    if (q11) q11[i] = b.sq11[g];
    if (q12) q12[i] = b.sq12[g];
    if (drho) drho[i] = b.sdr[g];
    if (ax) ax[i] = b.sax[g];
    if (ay) ay[i] = b.say[g];
}

// Device address of a page-locked host array that the device maps (nullptr if p is not one).
void *mapped_host(const void *p)
{
    cudaPointerAttributes a;
    if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
        cudaGetLastError();
        return nullptr;
    }
    return a.type == cudaMemoryTypeHost ? a.devicePointer : nullptr;
}

// Device addresses of the non-null host arrays p[0..k) if every one is mapped (false otherwise).
bool all_mapped(const void *const *p, void **d, int k)
{
    for (int j = 0; j < k; j++) {
        d[j] = nullptr;
        if (p[j] && !(d[j] = mapped_host(p[j]))) return false;
    }
    return true;
}

__global__ void k_deinterleave(const float *src, float *dst, int n, int stride, int comp)
{
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) dst[i] = src[(size_t)i * stride + comp];
}

const char kMagic[8] = {'A', 'N', 'N', 'S', 'T', 'A', 'T', '3'};
const char kMagicV2[8] = {'A', 'N', 'N', 'S', 'T', 'A', 'T', '2'};   // read: no image counts, colours

}  // namespace

extern "C" {

int ann_version(void) { return ANN_ABI_VERSION; }

const char *ann_status_string(int status) { return status_text(status); }

int ann_default_params(ann_params *p)
{
    if (!p) return ANN_ERR_INVALID_ARG;
    std::memset(p, 0, sizeof *p);
    p->n = 64 * 64;
    p->L = 1.0;
    p->h = 1.3 / 64.0;
    p->dt = 1e-4;
    p->rho0 = 1.0;
    p->eta = 1.0;
    p->Gamma = 0.34;
    p->lambda = 0.7;
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
    p->momentum_mode = ANN_MOMENTUM_PAPER;
    p->q_new_in_momentum = 1;
    p->dt_mode = ANN_DT_FIXED;
    return ANN_OK;
}

int ann_validate_params(const ann_params *p)
{
    std::string why;
    return validate(p, why);
}

int ann_grid_info(const ann_params *p, ann_grid *out)
{
    std::string why;
    int s = validate(p, why);
    if (s) return s;
    if (!out) return ANN_ERR_INVALID_ARG;
    out->cells_per_side = cells_per_side(*p);
    out->tiles_per_side = (out->cells_per_side + TILE - 1) / TILE;
    out->cell_size = p->L / out->cells_per_side;
    out->dt_effective = effective_dt(*p);
    out->expected_neighbors = M_PI * 9.0 * p->h * p->h * (double)p->n / (p->L * p->L);
    out->device_bytes = device_bytes(*p);
    return ANN_OK;
}

int ann_create(const ann_params *p, ann_ctx **out) { return ann_create_with_allocator(p, nullptr, out); }

int ann_create_with_allocator(const ann_params *p, const ann_allocator *a, ann_ctx **out)
{
    if (!out) return ANN_ERR_INVALID_ARG;
    *out = nullptr;
    std::string why;
    int s = validate(p, why);
    if (s) return s;
    if (a && (!a->alloc || !a->release)) return ANN_ERR_INVALID_ARG;
    int ndev = 0;
    if (cudaGetDeviceCount(&ndev) != cudaSuccess || ndev == 0) {
        cudaGetLastError();
        return ANN_ERR_NOT_AVAILABLE;
    }
    ann_ctx *c = new (std::nothrow) ann_ctx();
    if (!c) return ANN_ERR_OOM;
    c->prm = *p;
    c->P = make_dev(*p);
    if (a) c->al = *a;
    cudaError_t e = cudaGetDevice(&c->device);
    if (!e) e = prepare_kernels();
    if (!e) e = cudaStreamCreateWithFlags(&c->own, cudaStreamNonBlocking);
    if (!e) e = cudaStreamCreateWithFlags(&c->aux, cudaStreamNonBlocking);
    if (!e) { c->stream = c->own; e = alloc_all(c); }
    if (!e) e = cudaMallocHost(&c->h_err, sizeof(uint32_t));
    if (!e) e = cudaMallocHost(&c->h_ctl, sizeof(uint32_t) * (2 * CTL_WORDS + 1));
    if (!e) e = capture(c);
    if (!e) e = cudaStreamSynchronize(c->own);
    if (e) {
        int code = c->al_misaligned ? fail(c, ANN_ERR_INVALID_ARG, "ann_create: allocator returned a misaligned pointer")
                                    : cuda_fail(c, e, "ann_create");
        ann_destroy(c);
        return code;
    }
    *out = c;
    return ANN_OK;
}

void ann_destroy(ann_ctx *c)
{
    if (!c) return;
    if (c->stream) cudaStreamSynchronize(c->stream);
    if (c->exec) cudaGraphExecDestroy(c->exec);
    for (auto &v : c->allocs) dev_free(c, v.first, v.second);
    for (ann_ctx::Scratch *sc : {&c->d_grid, &c->d_off, &c->d_fld, &c->d_z, &c->d_zt, &c->d_tw, &c->d_shoff,
                                 &c->d_shmodes, &c->d_out, &c->d_map, &c->d_cnt, &c->d_ids})
        dev_free(c, sc->p, sc->bytes);
    if (c->h_err) cudaFreeHost(c->h_err);
    if (c->h_ctl) cudaFreeHost(c->h_ctl);
    if (c->own) cudaStreamDestroy(c->own);
    if (c->aux) cudaStreamDestroy(c->aux);
    delete c;
}

int ann_set_stream(ann_ctx *c, void *stream)
{
    if (!c) return ANN_ERR_INVALID_ARG;
    cudaStreamSynchronize(c->stream);
    c->stream = static_cast<cudaStream_t>(stream);
    return ANN_OK;
}

int ann_set_particles(ann_ctx *c, int64_t n, const double *x, const double *y, const double *ux,
                      const double *uy, const double *q11, const double *q12, const double *rho,
                      int is_device)
{
    NvtxRange range("ann_set_particles");
    if (!c) return ANN_ERR_INVALID_ARG;
    if (n != c->prm.n) return fail(c, ANN_ERR_INVALID_ARG, "n differs from the n of ann_create");
    if (!x || !y || !ux || !uy || !q11 || !q12) return fail(c, ANN_ERR_INVALID_ARG, "null input array");
    cudaError_t e = clear_flags(c);
    if (!e) e = cudaMemsetAsync(c->b.resorts, 0, sizeof(uint32_t), c->stream);
    if (e) return cuda_fail(c, e, "ann_set_particles");
    const double *src[7] = {x, y, ux, uy, q11, q12, rho};
    const double *dev[7] = {x, y, ux, uy, q11, q12, rho};
    if (!is_device) {
        double *t = static_cast<double *>(c->tmp);
        for (int k = 0; k < 7; k++) {
            if (!src[k]) { dev[k] = nullptr; continue; }
            e = cudaMemcpyAsync(t + (size_t)k * n, src[k], sizeof(double) * n, cudaMemcpyHostToDevice, c->stream);
            if (e) return cuda_fail(c, e, "ann_set_particles copy");
            dev[k] = t + (size_t)k * n;
        }
    }
    e = enqueue_load(c->P, c->b, dev[0], dev[1], dev[2], dev[3], dev[4], dev[5], dev[6], c->stream);
    if (e) return cuda_fail(c, e, "ann_set_particles load");
    c->have_particles = true;
    c->steps = 0;
    c->t = 0.0;
    c->s_sorted = c->m_current = false;
    c->rec_valid = false;
    c->grid_step = -1;
    int s = device_status(c);
    if (s) {
        c->have_particles = false;
        clear_flags(c);
        cudaStreamSynchronize(c->stream);
    }
    return s;
}

int ann_set_state(ann_ctx *c, int64_t n, const double *x, const double *y, const float *ux, const float *uy,
                  const float *q11, const float *q12, const float *drho, int is_device)
{
    NvtxRange range("ann_set_state");
    if (!c) return ANN_ERR_INVALID_ARG;
    if (n != c->prm.n) return fail(c, ANN_ERR_INVALID_ARG, "n differs from the n of ann_create");
    if (!x || !y || !ux || !uy || !q11 || !q12) return fail(c, ANN_ERR_INVALID_ARG, "null input array");
    cudaError_t e = clear_flags(c);
    if (!e) e = cudaMemsetAsync(c->b.resorts, 0, sizeof(uint32_t), c->stream);
    if (e) return cuda_fail(c, e, "ann_set_state");
    const void *dev[7] = {x, y, ux, uy, q11, q12, drho};
    if (!is_device) {
        unsigned char *t = static_cast<unsigned char *>(c->tmp);   // 36 of its 56 bytes per particle
        size_t off = 0;
        for (int k = 0; k < 7; k++) {
            const size_t bytes = (k < 2 ? 8 : 4) * (size_t)n;
            if (dev[k]) {
                e = cudaMemcpyAsync(t + off, dev[k], bytes, cudaMemcpyHostToDevice, c->stream);
                if (e) return cuda_fail(c, e, "ann_set_state copy");
                dev[k] = t + off;
            }
            off += bytes;
        }
    }
    k_load_state<<<(unsigned)((n + 255) / 256), 256, 0, c->stream>>>(
        c->P, c->b, (const double *)dev[0], (const double *)dev[1], (const float *)dev[2], (const float *)dev[3],
        (const float *)dev[4], (const float *)dev[5], (const float *)dev[6]);
    e = cudaGetLastError();
    if (e) return cuda_fail(c, e, "ann_set_state load");
    c->have_particles = true;
    c->steps = 0;
    c->t = 0.0;
    c->s_sorted = c->m_current = false;
    c->rec_valid = false;
    c->grid_step = -1;
    int s = device_status(c);
    if (s) {
        c->have_particles = false;
        clear_flags(c);
        cudaStreamSynchronize(c->stream);
    }
    return s;
}

int ann_update_state(ann_ctx *c, const double *x, const double *y, const float *ux, const float *uy,
                     const float *q11, const float *q12, const float *drho, const float *ax, const float *ay,
                     int is_device)
{
    NvtxRange range("ann_update_state");
    if (!c) return ANN_ERR_INVALID_ARG;
    if (!c->have_particles) return fail(c, ANN_ERR_STATE, "ann_update_state before ann_set_particles");
    if (!x || !y || !ux || !uy || !q11 || !q12) return fail(c, ANN_ERR_INVALID_ARG, "null input array");
    const size_t n = (size_t)c->P.n;
    const void *dev[9] = {x, y, ux, uy, q11, q12, drho, ax, ay};
    // the particle at each slot of the last re-sort: M's order when M holds the present state (a
    // search may have re-sorted into it), else S's
    const int *ids = c->m_current ? c->b.mid : c->b.sid;
    const unsigned nb = (unsigned)((n + 255) / 256);
    cudaError_t e = cudaSuccess;
    void *hd[9];
    if (!is_device && all_mapped(dev, hd, 9)) {
        // page-locked host arrays: one kernel reads them over the host link, no staging copy
        int *inv = static_cast<int *>(c->tmp);
        k_invert<<<nb, 256, 0, c->stream>>>(ids, inv, (int)n);
        k_update_state_mapped<<<nb, 256, 0, c->stream>>>(
            c->P, c->b, inv, (const double *)hd[0], (const double *)hd[1], (const float *)hd[2], (const float *)hd[3],
            (const float *)hd[4], (const float *)hd[5], (const float *)hd[6], (const float *)hd[7],
            (const float *)hd[8]);
        e = cudaGetLastError();
        if (e) return cuda_fail(c, e, "ann_update_state");
        c->s_sorted = c->m_current = false;
        c->rec_valid = false;
        c->grid_step = -1;
        return device_status(c);
    }
    if (!is_device) {
        unsigned char *t = static_cast<unsigned char *>(c->tmp);   // 44 of its 56 bytes per particle
        size_t off = 0;
        for (int k = 0; k < 9 && !e; k++) {
            const size_t bytes = (k < 2 ? 8 : 4) * n;
            if (dev[k]) {
                e = cudaMemcpyAsync(t + off, dev[k], bytes, cudaMemcpyHostToDevice, c->stream);
                dev[k] = t + off;
            }
            off += bytes;
        }
        if (e) return cuda_fail(c, e, "ann_update_state copy");
    }
    k_update_state<<<nb, 256, 0, c->stream>>>(
        c->P, c->b, ids, (const double *)dev[0], (const double *)dev[1], (const float *)dev[2], (const float *)dev[3],
        (const float *)dev[4], (const float *)dev[5], (const float *)dev[6], (const float *)dev[7],
        (const float *)dev[8]);
    e = cudaGetLastError();
    if (e) return cuda_fail(c, e, "ann_update_state");
    c->s_sorted = c->m_current = false;
    c->rec_valid = false;
    c->grid_step = -1;
    return device_status(c);
}

int ann_step(ann_ctx *c, int64_t nsteps)
{
    NvtxRange range("ann_step");
    if (!c || nsteps < 0) return ANN_ERR_INVALID_ARG;
    if (!c->have_particles) return fail(c, ANN_ERR_STATE, "ann_step before ann_set_particles");
    for (int64_t s = 0; s < nsteps; s++) {
        cudaError_t e = cudaGraphLaunch(c->exec, c->stream);
        if (e) return cuda_fail(c, e, "ann_step graph launch");
    }
    return settle_steps(c, nsteps);
}

int ann_step_profile(ann_ctx *c, int64_t nsteps, double *kernel_ms)
{
    NvtxRange range("ann_step_profile");
    if (!c || nsteps < 0 || !kernel_ms) return ANN_ERR_INVALID_ARG;
    if (!c->have_particles) return fail(c, ANN_ERR_STATE, "ann_step_profile before ann_set_particles");
    // The same kernels as the step graph, launched one by one between CUDA events.  The host reads
    // the re-sort decision after each predictor (one synchronisation per step) and launches only the
    // branch the graph would take, so each kernel's time is what it costs inside the graph.
    // Events per step: E[0] before the predictor, E[1] after it, E[2] after the host has read the
    // decision, E[k + 2] after kernel k >= 1 (or where it would have run).
    const size_t per = NKERNELS + 2;
    std::vector<cudaEvent_t> ev(per * (size_t)nsteps);
    std::vector<char> resorted((size_t)nsteps, 0);
    cudaError_t e = cudaSuccess;
    size_t made = 0;
    for (; made < ev.size() && !e; made++) e = cudaEventCreate(&ev[made]);
    for (int64_t s = 0; s < nsteps && !e; s++) {
        cudaEvent_t *E = &ev[(size_t)s * per];
        e = launch_commit(c->b, c->stream);   // as the graph's first node (not timed)
        if (!e) e = cudaEventRecord(E[0], c->stream);
        if (!e) e = launch_kernel(0, c->P, c->b, c->stream);
        if (!e) e = cudaEventRecord(E[1], c->stream);
        if (!e) e = cudaMemcpyAsync(c->h_err, c->b.rebuild, sizeof(uint32_t), cudaMemcpyDeviceToHost, c->stream);
        if (!e) e = cudaStreamSynchronize(c->stream);
        bool rs = !e && *c->h_err != 0u;
        resorted[(size_t)s] = rs;
        if (!e) e = cudaEventRecord(E[2], c->stream);
        for (int k = 1; k < NKERNELS && !e; k++) {
            bool run = (k <= 5) ? rs : (k == 6 ? !rs : true);
            if (run) {
                NvtxRange r(kernel_name(k));
                e = launch_kernel(k, c->P, c->b, c->stream);
            }
            if (!e) e = cudaEventRecord(E[k + 2], c->stream);
        }
    }
    if (!e) e = cudaStreamSynchronize(c->stream);
    for (int64_t s = 0; s < nsteps && !e; s++) {
        cudaEvent_t *E = &ev[(size_t)s * per];
        bool rs = resorted[(size_t)s];
        for (int k = 0; k < NKERNELS && !e; k++) {
            bool ran = (k >= 1 && k <= 5) ? rs : (k == 6 ? !rs : true);
            if (!ran) continue;   // a skipped branch adds nothing (only the events' own gap)
            float ms = 0.f;
            e = (k == 0) ? cudaEventElapsedTime(&ms, E[0], E[1]) : cudaEventElapsedTime(&ms, E[k + 1], E[k + 2]);
            kernel_ms[k] += ms;
        }
    }
    for (size_t k = 0; k < made; k++)
        if (ev[k]) cudaEventDestroy(ev[k]);
    if (e) return cuda_fail(c, e, "ann_step_profile");
    return settle_steps(c, nsteps);
}

int ann_kernel_count(void) { return NKERNELS; }

const char *ann_kernel_name(int k) { return kernel_name(k); }

int ann_set_record(ann_ctx *c, int on)
{
    if (!c || (on != 0 && on != 1)) return ANN_ERR_INVALID_ARG;
    if (c->P.record == on) return ANN_OK;
    cudaStreamSynchronize(c->stream);
    c->P.record = on;
    cudaError_t e = capture(c);
    if (e) return cuda_fail(c, e, "ann_set_record");
    return ANN_OK;
}

int ann_get_field(ann_ctx *c, int field, void *dst, int64_t bytes, int dst_is_device)
{
    if (!c || !dst) return ANN_ERR_INVALID_ARG;
    if (!c->have_particles) return fail(c, ANN_ERR_STATE, "no particles");
    Field f;
    if (!field_of(c, field, f)) return fail(c, ANN_ERR_INVALID_ARG, "unknown field");
    int n = c->P.n;
    if (bytes < (int64_t)n * f.es) return fail(c, ANN_ERR_INVALID_ARG, "destination too small");
    cudaError_t e = cudaSuccess;
    const void *src = f.ptr;
    unsigned char *tmp = static_cast<unsigned char *>(c->tmp);
    if (f.stride > 1) {
        float *d = reinterpret_cast<float *>(tmp + (size_t)8 * n);
        k_deinterleave<<<(n + 255) / 256, 256, 0, c->stream>>>(static_cast<const float *>(f.ptr), d, n, f.stride, f.comp);
        e = cudaGetLastError();
        src = d;
    }
    if (!e) e = enqueue_unpermute(src, f.state ? c->b.sid : c->b.mid, tmp, n, f.es, c->stream);
    if (!e) e = cudaMemcpyAsync(dst, tmp, (size_t)n * f.es,
                                dst_is_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost, c->stream);
    if (!e) e = cudaStreamSynchronize(c->stream);
    if (e) return cuda_fail(c, e, "ann_get_field");
    return ANN_OK;
}

int ann_get_state(ann_ctx *c, double *x, double *y, float *ux, float *uy, float *q11, float *q12, float *drho,
                  float *ax, float *ay, int dst_is_device)
{
    NvtxRange range("ann_get_state");
    if (!c) return ANN_ERR_INVALID_ARG;
    if (!c->have_particles) return fail(c, ANN_ERR_STATE, "no particles");
    const size_t n = (size_t)c->P.n;
    const Bufs &b = c->b;
    // each field is un-permuted into its own part of the staging buffer (44 bytes per particle of
    // the 56 it holds), so all copies are in flight before the one synchronisation
    unsigned char *tmp = static_cast<unsigned char *>(c->tmp);
    struct Part { const void *src; void *dst; int es; } parts[9] = {
        {b.sx, x, 8}, {b.sy, y, 8}, {b.sux, ux, 4}, {b.suy, uy, 4}, {b.sq11, q11, 4}, {b.sq12, q12, 4}, {b.sdr, drho, 4},
        {b.sax, ax, 4}, {b.say, ay, 4}};
    const cudaMemcpyKind kind = dst_is_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost;
    cudaError_t e = cudaSuccess;
    const void *dst[9] = {x, y, ux, uy, q11, q12, drho, ax, ay};
    void *hd[9];
    if (!dst_is_device && all_mapped(dst, hd, 9)) {
        // page-locked host arrays: one kernel gathers each particle's slot and writes them in
        // particle order over the host link, no staging copy
        const unsigned nb = (unsigned)((n + 255) / 256);
        int *inv = reinterpret_cast<int *>(tmp);
        k_invert<<<nb, 256, 0, c->stream>>>(b.sid, inv, (int)n);
        k_get_state_mapped<<<nb, 256, 0, c->stream>>>(
            b, (int)n, inv, (double *)hd[0], (double *)hd[1], (float *)hd[2], (float *)hd[3], (float *)hd[4],
            (float *)hd[5], (float *)hd[6], (float *)hd[7], (float *)hd[8]);
        e = cudaGetLastError();
        if (!e) e = cudaStreamSynchronize(c->stream);
        return e ? cuda_fail(c, e, "ann_get_state") : ANN_OK;
    }
    size_t off = 0;
    for (const Part &p : parts) {
        unsigned char *stage = tmp + off;
        off += (size_t)p.es * n;
        if (!p.dst) continue;
        e = enqueue_unpermute(p.src, b.sid, stage, (int)n, p.es, c->stream);
        if (!e) e = cudaMemcpyAsync(p.dst, stage, (size_t)p.es * n, kind, c->stream);
        if (e) break;
    }
    if (!e) e = cudaStreamSynchronize(c->stream);
    return e ? cuda_fail(c, e, "ann_get_state") : ANN_OK;
}

int ann_get_diagnostics(ann_ctx *c, ann_diag *out)
{
    if (!c || !out) return ANN_ERR_INVALID_ARG;
    if (!c->have_particles) return fail(c, ANN_ERR_STATE, "no particles");
    int nb = diag_blocks(c->P.n);
    double h[NDIAG];
    uint32_t bits = 0;
    unsigned long long band = 0;
    uint32_t resorts = 0;
    cudaError_t e = enqueue_diag(c->P, c->b, c->diag_part, nb, c->diag_out, c->stream);
    if (!e) e = cudaMemcpyAsync(&resorts, c->b.resorts, sizeof resorts, cudaMemcpyDeviceToHost, c->stream);
    if (!e) e = cudaMemcpyAsync(h, c->diag_out, sizeof h, cudaMemcpyDeviceToHost, c->stream);
    if (!e) e = cudaMemcpyAsync(&bits, c->b.err, sizeof bits, cudaMemcpyDeviceToHost, c->stream);
    if (!e) e = cudaMemcpyAsync(&band, c->b.band, sizeof band, cudaMemcpyDeviceToHost, c->stream);
    if (!e) e = cudaStreamSynchronize(c->stream);
    if (e) return cuda_fail(c, e, "ann_get_diagnostics");
    std::memset(out, 0, sizeof *out);
    int n = c->P.n;
    out->t = c->t;
    out->step = c->steps;
    out->momentum[0] = h[0];
    out->momentum[1] = h[1];
    out->kinetic_energy = h[2] / n;
    out->max_speed = h[3];
    // c0 of the last step is not kept on the device; report the bound it obeys now
    out->c0 = std::max(10.0 * h[3], c->prm.c0_min);
    out->mass = h[4];
    out->mean_q = h[5] / n;
    out->nbr_mean = h[6] / n;
    out->nbr_min = (int32_t)h[7];
    out->nbr_max = (int32_t)h[8];
    out->min_det_alpha = h[9];
    out->error_bits = bits;
    out->band_checks = band;
    out->resorts = (int32_t)resorts;
    return ANN_OK;
}

int ann_get_neighbors(ann_ctx *c, int64_t *rowptr, int32_t *cols, int64_t cap)
{
    if (!c || !rowptr) return ANN_ERR_INVALID_ARG;
    if (!c->have_particles) return fail(c, ANN_ERR_STATE, "no particles");
    int n = c->P.n;
    DevParams Q = c->P;
    Q.half_dt = 0.f;
    Q.half_dt_d = 0.0;
    // the search re-sorts at the present positions; S keeps its order, so the next step re-sorts too
    cudaError_t e = cudaMemsetAsync(c->b.rebuild, 1, sizeof(uint32_t), c->stream);
    if (!e) e = enqueue_search(Q, c->b, c->stream);
    if (e) return cuda_fail(c, e, "ann_get_neighbors search");
    int s = device_status(c);
    if (s) return s;
    c->s_sorted = false;   // the cell structure now follows M, which holds the present state
    c->m_current = true;
    std::vector<int> nn(n), mid(n);
    e = cudaMemcpyAsync(nn.data(), c->b.nnbr, sizeof(int) * n, cudaMemcpyDeviceToHost, c->stream);
    if (!e) e = cudaMemcpyAsync(mid.data(), c->b.mid, sizeof(int) * n, cudaMemcpyDeviceToHost, c->stream);
    if (!e) e = cudaStreamSynchronize(c->stream);
    if (e) return cuda_fail(c, e, "ann_get_neighbors counts");
    std::vector<int64_t> cnt(n + 1, 0);
    for (int g = 0; g < n; g++) cnt[mid[g] + 1] = nn[g];
    rowptr[0] = 0;
    for (int i = 0; i < n; i++) rowptr[i + 1] = rowptr[i] + cnt[i + 1];
    if (!cols) return ANN_OK;
    if (cap < rowptr[n]) return fail(c, ANN_ERR_INVALID_ARG, "cols capacity below rowptr[n]");
    // the export (MAXN entries per particle, column-major) takes a device buffer of its own for the
    // duration of the call, so a context does not hold 4 MAXN bytes per particle between calls
    std::vector<int> hc;
    try {
        hc.resize((size_t)MAXN * n);
    } catch (...) {
        return fail(c, ANN_ERR_OOM, "host allocation");
    }
    const size_t dbytes = sizeof(int) * (size_t)MAXN * n;
    void *dv = nullptr;
    if (dev_alloc(c, &dv, dbytes) != cudaSuccess) {
        cudaGetLastError();
        return fail(c, ANN_ERR_OOM, "ann_get_neighbors: device buffer of the export");
    }
    int *dcols = static_cast<int *>(dv);
    e = enqueue_export_nbrs(c->P, c->b, dcols, c->stream);
    if (!e) e = cudaMemcpyAsync(hc.data(), dcols, dbytes, cudaMemcpyDeviceToHost, c->stream);
    const cudaError_t es = cudaStreamSynchronize(c->stream);
    if (!e) e = es;
    dev_free(c, dv, dbytes);
    if (e) return cuda_fail(c, e, "ann_get_neighbors export");
    for (int g = 0; g < n; g++) {
        int i = mid[g];
        int32_t *row = cols + rowptr[i];
        for (int k = 0; k < nn[g]; k++) row[k] = hc[(size_t)k * n + g];
        std::sort(row, row + nn[g]);
    }
    return ANN_OK;
}

// File layout: magic, n, parameters, t, step count, re-sort flag, then per particle in the internal
// order: x, y (FP64); ux, uy, q11, q12, delta, ax, ay (FP32); ID; cell of the last re-sort; split
// position of the last re-sort (4 x FP32).  The last three reproduce the candidate lists exactly.
// Then per particle ID: periodic image counts (2 x int32) and colour (uint8).  Files of the
// previous layout ("ANNSTAT2", without the last two) load with zero counts and colour 0.
int ann_save_state(ann_ctx *c, const char *path)
{
    if (!c || !path) return ANN_ERR_INVALID_ARG;
    if (!c->have_particles) return fail(c, ANN_ERR_STATE, "no particles");
    size_t n = (size_t)c->P.n;
    std::vector<double> d(2 * n);
    std::vector<float> f(7 * n), xr(4 * n);
    std::vector<int> id(n);
    std::vector<uint32_t> mk(n);
    uint32_t rb = 1;
    const Bufs &b = c->b;
    const float *fs[7] = {b.sux, b.suy, b.sq11, b.sq12, b.sdr, b.sax, b.say};
    cudaError_t e = cudaMemcpyAsync(d.data(), b.sx, 8 * n, cudaMemcpyDeviceToHost, c->stream);
    if (!e) e = cudaMemcpyAsync(d.data() + n, b.sy, 8 * n, cudaMemcpyDeviceToHost, c->stream);
    for (int k = 0; k < 7 && !e; k++) e = cudaMemcpyAsync(f.data() + k * n, fs[k], 4 * n, cudaMemcpyDeviceToHost, c->stream);
    if (!e) e = cudaMemcpyAsync(id.data(), b.sid, 4 * n, cudaMemcpyDeviceToHost, c->stream);
    if (!e) e = cudaMemcpyAsync(mk.data(), b.mkey, 4 * n, cudaMemcpyDeviceToHost, c->stream);
    if (!e) e = cudaMemcpyAsync(xr.data(), b.xi_ref, 16 * n, cudaMemcpyDeviceToHost, c->stream);
    if (!e) e = cudaMemcpyAsync(&rb, b.rebuild, 4, cudaMemcpyDeviceToHost, c->stream);
    std::vector<int> img(2 * n);
    std::vector<unsigned char> col(n);
    if (!e) e = cudaMemcpyAsync(img.data(), b.img, 8 * n, cudaMemcpyDeviceToHost, c->stream);
    if (!e) e = cudaMemcpyAsync(col.data(), c->colors, n, cudaMemcpyDeviceToHost, c->stream);
    if (!e) e = cudaStreamSynchronize(c->stream);
    if (e) return cuda_fail(c, e, "ann_save_state");
    if (c->steps == 0) rb = 1;   // nothing evaluated yet: the next step re-sorts
    FILE *fp = std::fopen(path, "wb");
    if (!fp) return fail(c, ANN_ERR_IO, std::string("cannot open ") + path);
    int64_t nn = (int64_t)n;
    bool ok = std::fwrite(kMagic, 1, 8, fp) == 8 && std::fwrite(&nn, 8, 1, fp) == 1 &&
              std::fwrite(&c->prm, sizeof c->prm, 1, fp) == 1 && std::fwrite(&c->t, 8, 1, fp) == 1 &&
              std::fwrite(&c->steps, 8, 1, fp) == 1 && std::fwrite(&rb, 4, 1, fp) == 1 &&
              std::fwrite(d.data(), 8, 2 * n, fp) == 2 * n && std::fwrite(f.data(), 4, 7 * n, fp) == 7 * n &&
              std::fwrite(id.data(), 4, n, fp) == n && std::fwrite(mk.data(), 4, n, fp) == n &&
              std::fwrite(xr.data(), 4, 4 * n, fp) == 4 * n && std::fwrite(img.data(), 4, 2 * n, fp) == 2 * n &&
              std::fwrite(col.data(), 1, n, fp) == n;
    ok = (std::fclose(fp) == 0) && ok;
    return ok ? ANN_OK : fail(c, ANN_ERR_IO, "short write");
}

int ann_load_state(ann_ctx *c, const char *path)
{
    if (!c || !path) return ANN_ERR_INVALID_ARG;
    FILE *fp = std::fopen(path, "rb");
    if (!fp) return fail(c, ANN_ERR_IO, std::string("cannot open ") + path);
    char magic[8];
    int64_t nn = 0;
    ann_params prm;
    double t = 0.0;
    int64_t steps = 0;
    uint32_t rb = 1;
    bool ok = std::fread(magic, 1, 8, fp) == 8;
    bool v3 = ok && std::memcmp(magic, kMagic, 8) == 0;
    ok = ok && (v3 || std::memcmp(magic, kMagicV2, 8) == 0) &&
              std::fread(&nn, 8, 1, fp) == 1 && std::fread(&prm, sizeof prm, 1, fp) == 1 &&
              std::fread(&t, 8, 1, fp) == 1 && std::fread(&steps, 8, 1, fp) == 1 &&
              std::fread(&rb, 4, 1, fp) == 1;
    if (!ok) { std::fclose(fp); return fail(c, ANN_ERR_INVALID_ARG, "not a state file"); }
    if (nn != c->prm.n) { std::fclose(fp); return fail(c, ANN_ERR_INVALID_ARG, "state file n differs"); }
    size_t n = (size_t)nn;
    std::vector<double> d(2 * n);
    std::vector<float> f(7 * n), xr(4 * n);
    std::vector<int> id(n);
    std::vector<uint32_t> mk(n);
    ok = std::fread(d.data(), 8, 2 * n, fp) == 2 * n && std::fread(f.data(), 4, 7 * n, fp) == 7 * n &&
         std::fread(id.data(), 4, n, fp) == n && std::fread(mk.data(), 4, n, fp) == n &&
         std::fread(xr.data(), 4, 4 * n, fp) == 4 * n;
    std::vector<int> img(2 * n, 0);
    std::vector<unsigned char> col(n, 0);
    if (ok && v3) ok = std::fread(img.data(), 4, 2 * n, fp) == 2 * n && std::fread(col.data(), 1, n, fp) == n;
    std::fclose(fp);
    for (unsigned char v : col)
        if (v >= ANN_MAX_COLORS) return fail(c, ANN_ERR_INVALID_ARG, "state file colour out of range");
    if (!ok) return fail(c, ANN_ERR_IO, "short read");
    // cell starts of the last re-sort, from the cell of each particle (nondecreasing in this order)
    std::vector<uint32_t> start((size_t)c->P.ncell + 1, 0);
    if (!rb) {
        for (size_t i = 0; i < n; i++) {
            if (mk[i] >= (uint32_t)c->P.ncell || (i > 0 && mk[i] < mk[i - 1]))
                return fail(c, ANN_ERR_INVALID_ARG, "state file cell assignment is not sorted");
            start[mk[i] + 1]++;
        }
        for (int k = 0; k < c->P.ncell; k++) start[k + 1] += start[k];
    }
    const Bufs &b = c->b;
    float *fs[7] = {b.sux, b.suy, b.sq11, b.sq12, b.sdr, b.sax, b.say};
    cudaError_t e = clear_flags(c);
    if (!e) e = cudaMemcpyAsync(b.sx, d.data(), 8 * n, cudaMemcpyHostToDevice, c->stream);
    if (!e) e = cudaMemcpyAsync(b.sy, d.data() + n, 8 * n, cudaMemcpyHostToDevice, c->stream);
    for (int k = 0; k < 7 && !e; k++) e = cudaMemcpyAsync(fs[k], f.data() + k * n, 4 * n, cudaMemcpyHostToDevice, c->stream);
    if (!e) e = cudaMemcpyAsync(b.sid, id.data(), 4 * n, cudaMemcpyHostToDevice, c->stream);
    if (!e) e = cudaMemcpyAsync(b.mkey, mk.data(), 4 * n, cudaMemcpyHostToDevice, c->stream);
    if (!e) e = cudaMemcpyAsync(b.xi_ref, xr.data(), 16 * n, cudaMemcpyHostToDevice, c->stream);
    if (!e) e = cudaMemcpyAsync(b.img, img.data(), 8 * n, cudaMemcpyHostToDevice, c->stream);
    if (!e) e = cudaMemcpyAsync(c->colors, col.data(), n, cudaMemcpyHostToDevice, c->stream);
    if (!e && !rb) {
        e = cudaMemcpyAsync(b.cell_start, start.data(), 4 * start.size(), cudaMemcpyHostToDevice, c->stream);
        if (!e) e = enqueue_candidates_from_ref(c->P, b, c->stream);
        if (!e) e = cudaMemsetAsync(b.rebuild, 0, sizeof(uint32_t), c->stream);
    }
    if (!e) e = cudaStreamSynchronize(c->stream);
    if (e) return cuda_fail(c, e, "ann_load_state");
    c->have_particles = true;
    c->t = t;
    c->steps = steps;
    c->s_sorted = !rb;
    c->m_current = false;
    c->rec_valid = false;
    c->grid_step = -1;
    c->ncolors = 1;
    for (unsigned char v : col) c->ncolors = std::max(c->ncolors, (int)v + 1);
    return device_status(c);
}

const char *ann_last_error(ann_ctx *c) { return c ? c->last_err.c_str() : ""; }

}  // extern "C"

// ------------------------------------------------------------------------------------------------
// Flow diagnostics of the results section
// ------------------------------------------------------------------------------------------------

namespace {

// Grows a scratch buffer to at least `bytes` (contents are not kept).  The context's stream is
// synchronised before an old buffer is released.
cudaError_t ensure(ann_ctx *c, ann_ctx::Scratch &sc, size_t bytes)
{
    if (sc.p && sc.bytes >= bytes) return cudaSuccess;
    if (sc.p) {
        cudaError_t e = cudaStreamSynchronize(c->stream);
        if (e) return e;
        dev_free(c, sc.p, sc.bytes);
    }
    sc.p = nullptr;
    sc.bytes = 0;
    const size_t cap = std::max<size_t>(bytes, 16);
    cudaError_t e = dev_alloc(c, &sc.p, cap);
    if (!e) sc.bytes = cap;
    return e;
}

bool grid_size_ok(int M) { return M >= 8 && M <= ANN_GRID_MAX && (M & (M - 1)) == 0; }

int nshell_of(int M) { return (int)std::lround((double)M / std::sqrt(2.0)) + 1; }

// The present state in the cell order of the last re-sort: S or M, else a search at the present
// positions (the next step re-sorts in that case anyway, so the trajectory is unchanged).
int diag_source(ann_ctx *c, DiagSrc &src)
{
    const Bufs &b = c->b;
    if (!c->s_sorted && !c->m_current) {
        DevParams Q = c->P;
        Q.half_dt = 0.f;
        Q.half_dt_d = 0.0;
        cudaError_t e = cudaMemsetAsync(c->b.rebuild, 1, sizeof(uint32_t), c->stream);
        if (!e) e = enqueue_search(Q, c->b, c->stream);
        if (e) return cuda_fail(c, e, "diagnostics search");
        int st = device_status(c);
        if (st) return st;
        c->m_current = true;
    }
    if (c->s_sorted) src = DiagSrc{b.sx, b.sy, b.sux, b.suy, b.sq11, b.sq12, nullptr};
    else src = DiagSrc{b.mx, b.my, nullptr, nullptr, nullptr, nullptr, b.mu4};
    return ANN_OK;
}

// Gridded fields of the present state in d_grid (computed once per step and grid size).
int diag_grid(ann_ctx *c, int M)
{
    if (!c->have_particles) return fail(c, ANN_ERR_STATE, "no particles");
    if (!grid_size_ok(M)) return fail(c, ANN_ERR_INVALID_ARG, "grid size must be a power of two in [8, ANN_GRID_MAX]");
    if (c->P.nc < 5) return fail(c, ANN_ERR_INVALID_ARG, "gridding needs at least 5 cells per side");
    if (c->grid_M == M && c->grid_step == c->steps) return ANN_OK;
    DiagSrc src;
    int st = diag_source(c, src);
    if (st) return st;
    size_t n = (size_t)c->P.n, MM = (size_t)M * M;
    cudaError_t e = ensure(c, c->d_grid, 5 * MM * sizeof(double));
    if (!e) e = ensure(c, c->d_off, n * sizeof(float2));
    if (!e) e = ensure(c, c->d_fld, n * sizeof(float4));
    if (!e) e = enqueue_grid(c->P, c->b, src, M, (float2 *)c->d_off.p, (float4 *)c->d_fld.p, (double *)c->d_grid.p,
                             c->stream);
    if (!e) e = cudaStreamSynchronize(c->stream);
    if (e) return cuda_fail(c, e, "gridding");
    c->grid_M = M;
    c->grid_step = c->steps;
    return ANN_OK;
}

// Shells of the FFT modes (index a M + b, a and b FFT indices): CSR in increasing mode index.
cudaError_t shell_table(ann_ctx *c, int M)
{
    if (c->shell_M == M) return cudaSuccess;
    int ns = nshell_of(M);
    size_t MM = (size_t)M * M;
    std::vector<int> cnt((size_t)ns + 1, 0), modes(MM), which(MM);
    for (int a = 0; a < M; a++) {
        long long ka = a < M / 2 ? a : a - M;
        for (int bb = 0; bb < M; bb++) {
            long long kb = bb < M / 2 ? bb : bb - M;
            int sh = (int)std::llround(std::sqrt((double)(ka * ka + kb * kb)));
            which[(size_t)a * M + bb] = sh;
            cnt[(size_t)sh + 1]++;
        }
    }
    for (int k = 0; k < ns; k++) cnt[(size_t)k + 1] += cnt[(size_t)k];
    std::vector<int> fill(cnt.begin(), cnt.end() - 1);
    for (size_t i = 0; i < MM; i++) modes[(size_t)fill[(size_t)which[i]]++] = (int)i;
    cudaError_t e = ensure(c, c->d_shoff, cnt.size() * sizeof(int));
    if (!e) e = ensure(c, c->d_shmodes, MM * sizeof(int));
    if (!e) e = cudaMemcpy(c->d_shoff.p, cnt.data(), cnt.size() * sizeof(int), cudaMemcpyHostToDevice);
    if (!e) e = cudaMemcpy(c->d_shmodes.p, modes.data(), MM * sizeof(int), cudaMemcpyHostToDevice);
    if (!e) c->shell_M = M;
    return e;
}

double crossing_length(const double *C, int M, double L, double level)
{
    for (int k = 0; k < M / 2; k++)
        if (C[k] > level && level >= C[k + 1]) return (k + (C[k] - level) / (C[k] - C[k + 1])) * L / M;
    return NAN;
}

}  // namespace

extern "C" {

int ann_spectrum_shells(int32_t M) { return grid_size_ok(M) ? nshell_of(M) : ANN_ERR_INVALID_ARG; }

int ann_grid_fields(ann_ctx *c, int32_t M, double *dst, int dst_is_device)
{
    if (!c || !dst) return ANN_ERR_INVALID_ARG;
    int st = diag_grid(c, M);
    if (st) return st;
    cudaError_t e = cudaMemcpyAsync(dst, c->d_grid.p, 5 * (size_t)M * M * sizeof(double),
                                    dst_is_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost, c->stream);
    if (!e) e = cudaStreamSynchronize(c->stream);
    return e ? cuda_fail(c, e, "ann_grid_fields") : ANN_OK;
}

int ann_energy_spectrum(ann_ctx *c, int32_t M, double *E, int32_t nshell)
{
    if (!c || !E) return ANN_ERR_INVALID_ARG;
    int st = diag_grid(c, M);
    if (st) return st;
    int ns = nshell_of(M);
    if (nshell < ns) return fail(c, ANN_ERR_INVALID_ARG, "E holds fewer than ann_spectrum_shells(M) values");
    size_t MM = (size_t)M * M;
    cudaError_t e = ensure(c, c->d_z, MM * sizeof(double2));
    if (!e) e = ensure(c, c->d_zt, MM * sizeof(double2));
    if (!e) e = ensure(c, c->d_tw, (size_t)(M / 2) * sizeof(double2));
    if (!e) e = ensure(c, c->d_out, (size_t)std::max(ns, M / 2 + 1) * sizeof(double));
    if (!e && c->tw_M != M) {
        e = enqueue_twiddles(M, (double2 *)c->d_tw.p, c->stream);
        if (!e) c->tw_M = M;
    }
    if (!e) e = shell_table(c, M);
    if (!e) e = enqueue_spectrum(M, (const double *)c->d_grid.p, (double2 *)c->d_z.p, (double2 *)c->d_zt.p,
                                 (const double2 *)c->d_tw.p, (const int *)c->d_shoff.p, (const int *)c->d_shmodes.p,
                                 ns, (double *)c->d_out.p, c->stream);
    if (!e) e = cudaMemcpyAsync(E, c->d_out.p, (size_t)ns * sizeof(double), cudaMemcpyDeviceToHost, c->stream);
    if (!e) e = cudaStreamSynchronize(c->stream);
    return e ? cuda_fail(c, e, "ann_energy_spectrum") : ANN_OK;
}

int ann_spectrum_slope(const double *E, int32_t nshell, double L, double w1, double w2, double *slope)
{
    if (!E || !slope || nshell < 1 || !(L > 0.0)) return ANN_ERR_INVALID_ARG;
    double sx = 0, sy = 0, sxx = 0, sxy = 0;
    int m = 0;
    for (int k = 1; k < nshell; k++) {
        double w = 2.0 * M_PI * k / L;
        if (w < w1 || w > w2 || !(E[k] > 0.0)) continue;
        double x = std::log(w), y = std::log(E[k]);
        sx += x;
        sy += y;
        sxx += x * x;
        sxy += x * y;
        m++;
    }
    if (m < 2) {
        *slope = NAN;
        return ANN_OK;
    }
    *slope = (m * sxy - sx * sy) / (m * sxx - sx * sx);
    return ANN_OK;
}

int ann_vorticity_correlation(ann_ctx *c, int32_t M, int32_t all_origins, double *C, double *lengths)
{
    if (!c || !C || (all_origins != 0 && all_origins != 1)) return ANN_ERR_INVALID_ARG;
    int st = diag_grid(c, M);
    if (st) return st;
    cudaError_t e = ensure(c, c->d_out, (size_t)std::max(nshell_of(M), M / 2 + 1) * sizeof(double));
    if (!e) e = enqueue_correlation(M, c->prm.L, (const double *)c->d_grid.p, all_origins, (double *)c->d_out.p,
                                    c->stream);
    if (!e) e = cudaMemcpyAsync(C, c->d_out.p, (size_t)(M / 2 + 1) * sizeof(double), cudaMemcpyDeviceToHost, c->stream);
    if (!e) e = cudaStreamSynchronize(c->stream);
    if (e) return cuda_fail(c, e, "ann_vorticity_correlation");
    if (lengths) {
        double mx = C[0];
        for (int k = 1; k <= M / 2; k++) mx = std::max(mx, C[k]);
        lengths[0] = crossing_length(C, M, c->prm.L, 0.0);
        lengths[1] = crossing_length(C, M, c->prm.L, 0.2 * mx);
    }
    return ANN_OK;
}

int ann_defects(ann_ctx *c, int32_t M, int64_t *counts, int8_t *map)
{
    if (!c || !counts) return ANN_ERR_INVALID_ARG;
    int st = diag_grid(c, M);
    if (st) return st;
    size_t MM = (size_t)M * M;
    unsigned long long h[3];
    cudaError_t e = ensure(c, c->d_map, MM);
    if (!e) e = ensure(c, c->d_cnt, std::max<size_t>(3 * sizeof(unsigned long long), c->d_cnt.bytes));
    if (!e) e = enqueue_defects(M, (const double *)c->d_grid.p, (signed char *)c->d_map.p,
                                (unsigned long long *)c->d_cnt.p, c->stream);
    if (!e) e = cudaMemcpyAsync(h, c->d_cnt.p, sizeof h, cudaMemcpyDeviceToHost, c->stream);
    if (!e && map) e = cudaMemcpyAsync(map, c->d_map.p, MM, cudaMemcpyDeviceToHost, c->stream);
    if (!e) e = cudaStreamSynchronize(c->stream);
    if (e) return cuda_fail(c, e, "ann_defects");
    for (int k = 0; k < 3; k++) counts[k] = (int64_t)h[k];
    return ANN_OK;
}

int ann_set_colors(ann_ctx *c, const uint8_t *colors, int64_t n, int is_device)
{
    if (!c || !colors) return ANN_ERR_INVALID_ARG;
    if (n != c->prm.n) return fail(c, ANN_ERR_INVALID_ARG, "n differs from the n of ann_create");
    std::vector<uint8_t> h((size_t)n);
    cudaError_t e = cudaMemcpyAsync(h.data(), colors, (size_t)n, is_device ? cudaMemcpyDeviceToHost : cudaMemcpyHostToHost,
                                    c->stream);
    if (!e) e = cudaStreamSynchronize(c->stream);
    if (e) return cuda_fail(c, e, "ann_set_colors");
    int mx = 0;
    for (uint8_t v : h) mx = std::max(mx, (int)v);
    if (mx >= ANN_MAX_COLORS) return fail(c, ANN_ERR_INVALID_ARG, "colour beyond ANN_MAX_COLORS - 1");
    e = cudaMemcpyAsync(c->colors, h.data(), (size_t)n, cudaMemcpyHostToDevice, c->stream);
    if (!e) e = cudaStreamSynchronize(c->stream);
    if (e) return cuda_fail(c, e, "ann_set_colors");
    c->ncolors = mx + 1;
    return ANN_OK;
}

int ann_mixing_index(ann_ctx *c, int32_t G, double *index, double *per_species)
{
    if (!c || !index || G < 1 || G > ANN_MIX_BINS_MAX) return ANN_ERR_INVALID_ARG;
    if (!c->have_particles) return fail(c, ANN_ERR_STATE, "no particles");
    int S = c->ncolors;
    size_t nb = (size_t)G * G, bytes = nb * S * sizeof(unsigned);
    cudaError_t e = ensure(c, c->d_cnt, std::max<size_t>(bytes, 3 * sizeof(unsigned long long)));
    if (!e) e = enqueue_mixing(c->P, c->b, c->colors, G, S, (unsigned *)c->d_cnt.p, c->stream);
    std::vector<unsigned> cnt(nb * S);
    if (!e) e = cudaMemcpyAsync(cnt.data(), c->d_cnt.p, bytes, cudaMemcpyDeviceToHost, c->stream);
    if (!e) e = cudaStreamSynchronize(c->stream);
    if (e) return cuda_fail(c, e, "ann_mixing_index");
    std::vector<double> Ns((size_t)S, 0.0);
    std::vector<double> Nb(nb, 0.0);
    double N = 0.0;
    for (size_t k = 0; k < nb; k++)
        for (int s2 = 0; s2 < S; s2++) {
            double v = cnt[k * S + s2];
            Ns[(size_t)s2] += v;
            Nb[k] += v;
            N += v;
        }
    double sum = 0.0;
    int used = 0;
    for (int s2 = 0; s2 < S; s2++) {
        double a = N > 0 ? Ns[(size_t)s2] / N : 0.0, Is = NAN;
        if (a > 0.0 && a < 1.0) {
            double acc = 0.0;
            int full = 0;
            for (size_t k = 0; k < nb; k++) {
                if (Nb[k] <= 0.0) continue;
                double f = cnt[k * S + s2] / Nb[k] - a;
                acc += f * f;
                full++;
            }
            Is = acc / full / (a * (1.0 - a));
            sum += Is;
            used++;
        }
        if (per_species) per_species[s2] = Is;
    }
    if (per_species)
        for (int s2 = S; s2 < ANN_MAX_COLORS; s2++) per_species[s2] = NAN;
    *index = used ? sum / used : 0.0;
    return ANN_OK;
}

int ann_get_unwrapped(ann_ctx *c, const int64_t *ids, int64_t k, double *xy)
{
    if (!c || (k > 0 && (!ids || !xy)) || k < 0 || k > c->prm.n) return ANN_ERR_INVALID_ARG;
    if (!c->have_particles) return fail(c, ANN_ERR_STATE, "no particles");
    for (int64_t t = 0; t < k; t++)
        if (ids[t] < 0 || ids[t] >= c->prm.n) return fail(c, ANN_ERR_INVALID_ARG, "particle ID out of range");
    if (k == 0) return ANN_OK;
    size_t kk = (size_t)k;
    cudaError_t e = ensure(c, c->d_ids, kk * (sizeof(long long) + 2 * sizeof(double)));
    long long *dids = (long long *)c->d_ids.p;
    double *dxy = (double *)(dids + kk);
    if (!e) e = cudaMemcpyAsync(dids, ids, kk * sizeof(long long), cudaMemcpyHostToDevice, c->stream);
    if (!e) e = enqueue_unwrapped(c->P, c->b, c->inv, dids, (int)k, dxy, c->stream);
    if (!e) e = cudaMemcpyAsync(xy, dxy, 2 * kk * sizeof(double), cudaMemcpyDeviceToHost, c->stream);
    if (!e) e = cudaStreamSynchronize(c->stream);
    return e ? cuda_fail(c, e, "ann_get_unwrapped") : ANN_OK;
}

}  // extern "C"

// ------------------------------------------------------------------------------------------------
// Batched ensemble: independent contexts stepped by one graph launch per step
// ------------------------------------------------------------------------------------------------

struct ann_ensemble {
    std::vector<ann_ctx *> m;
    cudaStream_t s0 = nullptr;                 // origin stream of the ensemble graph
    std::vector<cudaStream_t> br;              // branch streams used while capturing
    cudaGraphExec_t exec = nullptr;
    int groups = 0;                            // members are dealt round-robin to this many branches
    std::string last_err;
};

namespace {

int efail(ann_ensemble *e, int code, const std::string &msg)
{
    if (e) e->last_err = msg;
    return code;
}

// One graph: the origin forks `groups` branches; branch j steps members j, j + groups, ... one
// after the other; the branches join the origin at the end.
cudaError_t build_ensemble_graph(ann_ensemble *E, int groups)
{
    if (E->exec) {
        cudaGraphExecDestroy(E->exec);
        E->exec = nullptr;
    }
    cudaGraph_t g = nullptr;
    cudaError_t e = cudaGraphCreate(&g, 0);
    if (e) return e;
    e = cudaStreamBeginCaptureToGraph(E->s0, g, nullptr, nullptr, 0, cudaStreamCaptureModeThreadLocal);
    if (e) {
        cudaGraphDestroy(g);
        return e;
    }
    std::vector<cudaEvent_t> ev((size_t)groups + 1, nullptr);
    cudaError_t ec = cudaSuccess;
    for (auto &x : ev)
        if (!ec) ec = cudaEventCreateWithFlags(&x, cudaEventDisableTiming);
    if (!ec) ec = cudaEventRecord(ev[0], E->s0);
    for (int j = 0; j < groups && !ec; j++) {
        cudaStream_t s = E->br[(size_t)j];
        ec = cudaStreamWaitEvent(s, ev[0], 0);
        for (size_t k = (size_t)j; k < E->m.size() && !ec; k += (size_t)groups) ec = capture_step(E->m[k], s, g);
        if (!ec) ec = cudaEventRecord(ev[(size_t)j + 1], s);
        if (!ec) ec = cudaStreamWaitEvent(E->s0, ev[(size_t)j + 1], 0);
    }
    e = cudaStreamEndCapture(E->s0, &g);
    for (auto &x : ev)
        if (x) cudaEventDestroy(x);
    if (ec || e) {
        if (g) cudaGraphDestroy(g);
        return ec ? ec : e;
    }
    e = cudaGraphInstantiate(&E->exec, g, 0);
    cudaGraphDestroy(g);
    if (!e) E->groups = groups;
    return e;
}

}  // namespace

extern "C" {

int ann_ensemble_create(const ann_params *params, int32_t members, ann_ensemble **out)
{
    if (!params || !out || members < 1 || members > ANN_ENSEMBLE_MAX) return ANN_ERR_INVALID_ARG;
    *out = nullptr;
    ann_ensemble *E = new (std::nothrow) ann_ensemble();
    if (!E) return ANN_ERR_OOM;
    int st = ANN_OK;
    for (int k = 0; k < members && !st; k++) {
        ann_ctx *c = nullptr;
        st = ann_create(&params[k], &c);
        if (!st) E->m.push_back(c);
    }
    cudaError_t e = cudaSuccess;
    if (!st) e = cudaStreamCreateWithFlags(&E->s0, cudaStreamNonBlocking);
    for (int k = 0; k < members && !st && !e; k++) {
        cudaStream_t s = nullptr;
        e = cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking);
        if (!e) E->br.push_back(s);
    }
    if (!st && !e) e = build_ensemble_graph(E, members);
    if (st || e) {
        if (!st) st = e == cudaErrorMemoryAllocation ? ANN_ERR_OOM : ANN_ERR_CUDA;
        ann_ensemble_destroy(E);
        return st;
    }
    *out = E;
    return ANN_OK;
}

void ann_ensemble_destroy(ann_ensemble *E)
{
    if (!E) return;
    if (E->s0) cudaStreamSynchronize(E->s0);
    if (E->exec) cudaGraphExecDestroy(E->exec);
    for (cudaStream_t s : E->br) cudaStreamDestroy(s);
    if (E->s0) cudaStreamDestroy(E->s0);
    for (ann_ctx *c : E->m) ann_destroy(c);
    delete E;
}

int ann_ensemble_member(ann_ensemble *E, int32_t k, ann_ctx **ctx)
{
    if (!E || !ctx || k < 0 || k >= (int32_t)E->m.size()) return ANN_ERR_INVALID_ARG;
    *ctx = E->m[(size_t)k];
    return ANN_OK;
}

// Settle every member after a batch of ensemble steps (settle_steps); the first failing member's
// status is returned and named.
static int ensemble_settle(ann_ensemble *E, int64_t launched)
{
    int first = ANN_OK;
    for (size_t k = 0; k < E->m.size(); k++) {
        ann_ctx *c = E->m[k];
        int st = settle_steps(c, launched);
        if (st && first == ANN_OK) {
            first = st;
            E->last_err = "member " + std::to_string(k) + ": " + c->last_err;
        }
    }
    return first;
}

int ann_ensemble_set_groups(ann_ensemble *E, int32_t groups)
{
    if (!E || groups < 1 || groups > (int32_t)E->m.size()) return ANN_ERR_INVALID_ARG;
    if (groups == E->groups) return ANN_OK;
    cudaError_t e = build_ensemble_graph(E, groups);
    return e ? efail(E, ANN_ERR_CUDA, std::string("ensemble graph: ") + cudaGetErrorString(e)) : ANN_OK;
}

int ann_ensemble_step(ann_ensemble *E, int64_t nsteps)
{
    ann::NvtxRange range("ann_ensemble_step");
    if (!E || nsteps < 0) return ANN_ERR_INVALID_ARG;
    for (size_t k = 0; k < E->m.size(); k++)
        if (!E->m[k]->have_particles)
            return efail(E, ANN_ERR_STATE, "member " + std::to_string(k) + " has no particles");
    for (int64_t s = 0; s < nsteps; s++) {
        cudaError_t e = cudaGraphLaunch(E->exec, E->s0);
        if (e) return efail(E, ANN_ERR_CUDA, std::string("ensemble graph launch: ") + cudaGetErrorString(e));
    }
    cudaError_t e = cudaStreamSynchronize(E->s0);
    if (e) return efail(E, ANN_ERR_CUDA, std::string("ensemble step: ") + cudaGetErrorString(e));
    return ensemble_settle(E, nsteps);
}

int ann_ensemble_autotune(ann_ensemble *E, int32_t trial_steps, int32_t *groups_out, double *ms_per_step)
{
    if (!E || trial_steps < 1) return ANN_ERR_INVALID_ARG;
    int nm = (int)E->m.size();
    std::vector<int> cand;
    for (int g = 1; g < nm; g *= 4) cand.push_back(g);
    cand.push_back(nm);
    cudaEvent_t a = nullptr, b = nullptr;
    cudaError_t e = cudaEventCreate(&a);
    if (!e) e = cudaEventCreate(&b);
    int best = E->groups;
    float best_ms = -1.f;
    int st = ANN_OK;
    for (int g : cand) {
        if (e || st) break;
        e = build_ensemble_graph(E, g);
        if (e) break;
        st = ann_ensemble_step(E, 1);   // warm-up (and the first re-sort of fresh members)
        if (st) break;
        e = cudaEventRecord(a, E->s0);
        for (int s2 = 0; s2 < trial_steps && !e; s2++) e = cudaGraphLaunch(E->exec, E->s0);
        if (!e) e = cudaEventRecord(b, E->s0);
        if (!e) e = cudaEventSynchronize(b);
        float ms = 0.f;
        if (!e) e = cudaEventElapsedTime(&ms, a, b);
        if (!e) st = ensemble_settle(E, trial_steps);   // commit (or roll back) the trial steps
        if (!e && (best_ms < 0.f || ms < best_ms)) {
            best_ms = ms;
            best = g;
        }
    }
    if (a) cudaEventDestroy(a);
    if (b) cudaEventDestroy(b);
    if (e) return efail(E, ANN_ERR_CUDA, std::string("ensemble autotune: ") + cudaGetErrorString(e));
    if (st) return st;
    e = build_ensemble_graph(E, best);
    if (e) return efail(E, ANN_ERR_CUDA, std::string("ensemble graph: ") + cudaGetErrorString(e));
    if (groups_out) *groups_out = best;
    if (ms_per_step) *ms_per_step = best_ms / trial_steps;
    return ANN_OK;
}

const char *ann_ensemble_last_error(ann_ensemble *E) { return E ? E->last_err.c_str() : ""; }

}  // extern "C"

// ------------------------------------------------------------------------------------------------
// Hooks for the learned surrogate
// ------------------------------------------------------------------------------------------------

namespace ann {

int ctx_view(ann_ctx *c, CtxView *v)
{
    if (!c || !v) return ANN_ERR_INVALID_ARG;
    if (!c->have_particles) return fail(c, ANN_ERR_STATE, "no particles");
    v->P = c->P;
    v->b = c->b;
    v->stream = c->stream;
    v->tmp = static_cast<double *>(c->tmp);
    v->t = c->t;
    v->steps = c->steps;
    v->rec_valid = c->rec_valid;
    return ANN_OK;
}

int ctx_search_present(ann_ctx *c)
{
    if (!c->have_particles) return fail(c, ANN_ERR_STATE, "no particles");
    if (c->m_current) return ANN_OK;
    DevParams Q = c->P;
    Q.half_dt = 0.f;
    Q.half_dt_d = 0.0;
    // re-sorts only if the lists of the last re-sort no longer cover the present positions: the
    // host reads the predictor's decision and launches only the branch that does work
    cudaError_t e = launch_kernel(0, Q, c->b, c->stream);
    if (!e) e = cudaMemcpyAsync(c->h_err, c->b.rebuild, sizeof(uint32_t), cudaMemcpyDeviceToHost, c->stream);
    if (!e) e = cudaStreamSynchronize(c->stream);
    const bool rs = !e && *c->h_err != 0u;
    for (int k = rs ? 1 : 6; k <= (rs ? 5 : 6) && !e; k++) e = launch_kernel(k, Q, c->b, c->stream);
    if (!e) e = cudaMemsetAsync(c->b.maxu, 0, sizeof(uint32_t), c->stream);
    if (e) return cuda_fail(c, e, "search");
    int st = device_status(c);
    if (st) return st;
    c->s_sorted = false;
    c->m_current = true;
    return ANN_OK;
}

// The state arrays S were rewritten in place, in the order of the evaluation copy M (the order of
// the last re-sort), with accelerations 0: t and the step count advance by add_steps.  The cell
// structure is kept: the next step re-sorts only if a particle has moved half the skin since the
// last re-sort, as after any step.
int ctx_commit_in_place(ann_ctx *c, int64_t add_steps)
{
    int st = device_status(c);
    c->t += add_steps * c->P.dt_d;
    c->steps += add_steps;
    c->s_sorted = c->m_current = false;   // diagnostics search the present positions first
    c->rec_valid = false;
    c->grid_step = -1;
    return st;
}

}  // namespace ann

// sm_103a kernels of one SPH active-nematic time step (arXiv 2108.08919, §3 and §3.1).
//
// Layout: particles live in structure-of-arrays form, sorted by square cells of side >= 3h (§4);
// cells are numbered row-major.  A pair pass runs one block per 4 x 4 cells ("tile"): the block
// stages the particles of the surrounding 6 x 6 cells in shared memory -- periodic images of the
// cells on the far side of the box take the place of the paper's ghost particles (Eq. 30) -- and
// each thread accumulates the sums of one particle over its neighbours.  Positions are FP64; the pair
// passes use a split tile-local coordinate hi + lo in FP32 whose hi parts lie on a power-of-two grid,
// so d = (hi_i - hi_j) + (lo_i - lo_j) is the correctly rounded FP32 pair vector.  The support test
// |d|^2 < (3h)^2 is decided in FP32 unless it falls within a rounding band of the cutoff, where it is
// redone in FP64 from the FP64 positions exactly as the definition states.
#include "ann_device.cuh"

#include <cmath>

namespace ann {
namespace {

constexpr unsigned FULL = 0xffffffffu;

__device__ __forceinline__ int wrapc(int c, int nc) { return c < 0 ? c + nc : (c >= nc ? c - nc : c); }

__device__ __forceinline__ bool stopped(const Bufs &b) { return *(volatile uint32_t *)b.err != 0u; }

// FP64 support test of the definition for particles gi and gj: d = minimum image of x_i - x_j
// (x_i - x_j, then -L or +L when beyond L/2), |d|^2 = d_x*d_x + d_y*d_y, no fused operations.
__device__ __noinline__ bool support64(const DevParams &P, const Bufs &b, int gi, int gj)
{
    double hL = 0.5 * P.L;
    double dx = __dsub_rn(b.mx[gi], b.mx[gj]);
    if (dx > hL) dx = __dsub_rn(dx, P.L);
    else if (dx < -hL) dx = __dadd_rn(dx, P.L);
    double dy = __dsub_rn(b.my[gi], b.my[gj]);
    if (dy > hL) dy = __dsub_rn(dy, P.L);
    else if (dy < -hL) dy = __dadd_rn(dy, P.L);
    double r2 = __dadd_rn(__dmul_rn(dx, dx), __dmul_rn(dy, dy));
    return r2 < P.R2;
}

__device__ __forceinline__ bool resorting(const Bufs &b) { return *(volatile uint32_t *)b.rebuild != 0u; }

// A particle crossed the box (Eq. 30): update its periodic image count (one thread per particle)
// and log the crossing, so that the host can undo it if this step fails.  Crossings are rare.
__device__ __forceinline__ void add_crossing(const Bufs &b, int id, int kx, int ky)
{
    int2 &im = b.img[id];
    im.x += kx;
    im.y += ky;
    const unsigned k = atomicAdd(b.ctl + CTL_XLOG, 1u);
    if (k < (unsigned)b.xlog_cap) b.xlog[k] = make_int4(id, kx, ky, 0);
}

// ---------------------------------------------------------------------------------------------
// Tile bookkeeping shared by the pair passes
// ---------------------------------------------------------------------------------------------

struct TileShared {
    int off[NHC + 1];      // exclusive prefix of halo-cell particle counts (slots)
    int start[NHC];        // first sorted index of each halo cell
    int rowpre[TILE + 1];  // prefix of inner-row slot counts
};

struct Tile {
    int cx0, cy0, wx, wy, HX, NH, H, Ni;
};

__device__ __forceinline__ bool tile_begin(const DevParams &P, const Bufs &b, TileShared &ts, Tile &T)
{
    int tx = blockIdx.x % P.tiles, ty = blockIdx.x / P.tiles;
    T.cx0 = tx * TILE;
    T.cy0 = ty * TILE;
    T.wx = min(TILE, P.nc - T.cx0);
    T.wy = min(TILE, P.nc - T.cy0);
    T.HX = T.wx + 2;
    T.NH = T.HX * (T.wy + 2);
    int t = threadIdx.x;
    if (t < T.NH) {
        int hx = t % T.HX, hy = t / T.HX;
        int c = wrapc(T.cy0 - 1 + hy, P.nc) * P.nc + wrapc(T.cx0 - 1 + hx, P.nc);
        uint32_t s0 = b.cell_start[c], s1 = b.cell_start[c + 1];
        ts.start[t] = (int)s0;
        ts.off[t + 1] = (int)(s1 - s0);
    }
    __syncthreads();
    if (t == 0) {
        ts.off[0] = 0;
        for (int h = 0; h < T.NH; h++) ts.off[h + 1] += ts.off[h];
        int acc = 0;
        ts.rowpre[0] = 0;
        for (int r = 0; r < T.wy; r++) {
            int row = (r + 1) * T.HX;
            acc += ts.off[row + T.wx + 1] - ts.off[row + 1];
            ts.rowpre[r + 1] = acc;
        }
    }
    __syncthreads();
    T.H = ts.off[T.NH];
    T.Ni = ts.rowpre[T.wy];
    return T.H <= HCAP;
}

// Halo cell holding slot t (largest h with off[h] <= t).
__device__ __forceinline__ int slot_cell(const TileShared &ts, int NH, int t)
{
    int lo = 0, hi = NH - 1;
    while (lo < hi) {
        int mid = (lo + hi + 1) >> 1;
        if (ts.off[mid] <= t) lo = mid;
        else hi = mid - 1;
    }
    return lo;
}

// Slot of the q-th particle of the tile's inner cells.
__device__ __forceinline__ int inner_slot(const TileShared &ts, const Tile &T, int q)
{
    int r = 0;
    while (r + 1 < T.wy && ts.rowpre[r + 1] <= q) r++;
    return ts.off[(r + 1) * T.HX + 1] + (q - ts.rowpre[r]);
}

// Sorted index and tile-local position (hi_x, hi_y, lo_x, lo_y) of slot t.  The halo cell offset
// hx * cell is added as hx * cell_hi (exact on the q grid) plus hx * cell_lo.
struct SlotInfo {
    int g, h;
    float4 e;
};

__device__ __forceinline__ SlotInfo slot_info(const DevParams &P, const Bufs &b, const TileShared &ts,
                                              const Tile &T, int t)
{
    SlotInfo s;
    s.h = slot_cell(ts, T.NH, t);
    s.g = ts.start[s.h] + (t - ts.off[s.h]);
    float hx = (float)(s.h % T.HX), hy = (float)(s.h / T.HX);
    float4 o = b.xi[s.g];
    s.e = make_float4(o.x + hx * P.cell_hi, o.y + hy * P.cell_hi, o.z + hx * P.cell_lo, o.w + hy * P.cell_lo);
    return s;
}

// Pair vector d_ij from two split tile-local positions: (hi_i - hi_j) + (lo_i - lo_j) per lane.
__device__ __forceinline__ float2 pair_d(const float4 &a, const float4 &b)
{
    return add2(sub2(f2(a.x, a.y), f2(b.x, b.y)), sub2(f2(a.z, a.w), f2(b.z, b.w)));
}


// Element of a staged shared-memory array at byte offset o of a 16-byte slot (candidate lists
// store o = 16 * slot): o / (16 / sizeof(T)) for narrower element types.
template <typename T>
__device__ __forceinline__ const T &slot_at(const T *base, int o)
{
    static_assert(sizeof(T) == 16 || sizeof(T) == 8 || sizeof(T) == 4, "staged element size");
    constexpr int sh = sizeof(T) == 16 ? 0 : (sizeof(T) == 8 ? 1 : 2);
    return *reinterpret_cast<const T *>(reinterpret_cast<const char *>(base) + (o >> sh));
}

// ---------------------------------------------------------------------------------------------
// Kernel 0: predictor, re-insertion, max |u'|, re-sort decision                   (§3.1, Eq. 30)
// ---------------------------------------------------------------------------------------------

// Split of the offset o of a position from a cell corner: hi = o rounded (in FP32) to the q grid,
// exact in both precisions; lo = o - hi, exact in FP64, then rounded to FP32.
__device__ __forceinline__ float2 split_offset(double o, const DevParams &P)
{
    float hi = rintf((float)o * P.iqf) * P.qf;
    return make_float2(hi, (float)(o - (double)hi));
}

__global__ void __launch_bounds__(256, 8) k_predict(DevParams P, Bufs b)
{
    if (stopped(b)) return;
    __shared__ float wmax[8];
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    bool rs = resorting(b);
    float sp = 0.f;
    int moved = 0;   // this particle left half the skin: the step re-sorts
    if (i < P.n) {
        // the committed state in, the predicted positions and velocities into the other set
        const StateSet in = state_in(b), out = state_out(b);
        float ux = in.ux[i] + P.half_dt * in.ax[i];
        float uy = in.uy[i] + P.half_dt * in.ay[i];
        // FP64 work is kept to what the positions need: GB300 issues FP64 at 1/64 of FP32.
        double x = in.x[i] + (double)(P.half_dt * ux);
        double y = in.y[i] + (double)(P.half_dt * uy);
        if (!(in_box(x, P.bitsL) && in_box(y, P.bitsL))) {   // rare: crossed a face, or not finite
            int kx = wrap_count(x, P.L), ky = wrap_count(y, P.L);
            x = x + 0.0;
            y = y + 0.0;
            if (kx | ky) add_crossing(b, in.id[i], kx, ky);   // periodic image count (pathlines)
            if (!(in_box(x, P.bitsL) && in_box(y, P.bitsL) && isfinite(ux) && isfinite(uy))) {
                atomicOr(b.err, EB_NONFINITE);
                x = 0.0;
                y = 0.0;
                ux = 0.f;
                uy = 0.f;
            }
        }
        sp = sqrtf(ux * ux + uy * uy);
        out.ux[i] = ux;
        out.uy[i] = uy;
        out.x[i] = x;
        out.y[i] = y;
        if (!rs) {
            // The order is that of the last re-sort: write the evaluation copy directly, split
            // against the cell the particle was assigned to then.  A particle that has moved half
            // the skin since makes this step re-sort (the kernels after this one see the flag).
            uint32_t mk = b.mkey[i];
            int cx = (int)(mk % (uint32_t)P.nc), cy = (int)(mk / (uint32_t)P.nc);
            double ox = x - __ldg(&b.origin[cx]), oy = y - __ldg(&b.origin[cy]);
            if (cx == 0 || cx == P.nc - 1) {   // the particle may have crossed the face since
                if (ox > 0.5 * P.L) ox -= P.L;
                else if (ox < -0.5 * P.L) ox += P.L;
            }
            if (cy == 0 || cy == P.nc - 1) {
                if (oy > 0.5 * P.L) oy -= P.L;
                else if (oy < -0.5 * P.L) oy += P.L;
            }
            float2 sx_ = split_offset(ox, P), sy_ = split_offset(oy, P);
            float4 xi = make_float4(sx_.x, sy_.x, sx_.y, sy_.y);
            float4 rf = b.xi_ref[i];
            float ddx = (xi.x - rf.x) + (xi.z - rf.z), ddy = (xi.y - rf.y) + (xi.w - rf.w);
            moved = ddx * ddx + ddy * ddy > P.skin_max2;
            b.mx[i] = x;
            b.my[i] = y;
            b.xi[i] = xi;
            b.mu4[i] = make_float4(ux, uy, in.q11[i], in.q12[i]);
            b.mdr[i] = in.dr[i];
            b.mid[i] = in.id[i];
        }
    }
    for (int o = 16; o > 0; o >>= 1) sp = fmaxf(sp, __shfl_xor_sync(FULL, sp, o));
    if ((threadIdx.x & 31) == 0) wmax[threadIdx.x >> 5] = sp;
    // one flag store per block (a store from every particle that moved would queue on one address
    // when many move at once, e.g. after ann_update_state)
    if (__syncthreads_or(moved) && threadIdx.x == 0) *(volatile uint32_t *)b.rebuild = 1u;
    if (threadIdx.x < 32) {
        sp = threadIdx.x < (blockDim.x >> 5) ? wmax[threadIdx.x] : 0.f;
        for (int o = 16; o > 0; o >>= 1) sp = fmaxf(sp, __shfl_xor_sync(FULL, sp, o));
        if (threadIdx.x == 0 && sp > 0.f) atomicMax(b.maxu, __float_as_uint(sp));
    }
}

// ---------------------------------------------------------------------------------------------
// Kernel 1 (re-sort steps only): cell key of each predicted position, its split against that
// cell, and its rank in the cell
// ---------------------------------------------------------------------------------------------

__global__ void __launch_bounds__(256) k_keys(DevParams P, Bufs b)
{
    if (stopped(b) || !resorting(b)) return;
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    int lane = threadIdx.x & 31;
    uint32_t key = 0xffffffffu;
    if (i < P.n) {
        const StateSet out = state_out(b);   // the predicted positions
        double x = out.x[i], y = out.y[i];
        int cx = min((int)(x * P.inv_cell), P.nc - 1);
        int cy = min((int)(y * P.inv_cell), P.nc - 1);
        key = (uint32_t)(cy * P.nc + cx);
        b.key[i] = key;
        float2 sx_ = split_offset(x - __ldg(&b.origin[cx]), P);
        float2 sy_ = split_offset(y - __ldg(&b.origin[cy]), P);
        b.sxi[i] = make_float4(sx_.x, sy_.x, sx_.y, sy_.y);
    }
    // Particles arrive in the previous cell order, so a warp holds a few runs of equal keys: one
    // atomic per run instead of one per particle.
    unsigned grp = __match_any_sync(FULL, key);
    int leader = __ffs(grp) - 1;
    uint32_t base = 0;
    if (lane == leader && key != 0xffffffffu) base = atomicAdd(&b.cell_count[key], (uint32_t)__popc(grp));
    base = __shfl_sync(FULL, base, leader);
    if (i < P.n) b.rank[i] = base + (uint32_t)__popc(grp & ((1u << lane) - 1u));
}

// ---------------------------------------------------------------------------------------------
// Kernel 2: exclusive scan of cell counts -> cell starts, one block per SCAN_CHUNK cells.  Each
// block first sums the counts of all cells before its chunk (coalesced, L2-resident reads), so no
// block waits on another; then it scans its own chunk.  The counts are cleared by the scatter
// kernel, after every block has read them.
// ---------------------------------------------------------------------------------------------

__global__ void __launch_bounds__(1024) k_scan(DevParams P, Bufs b)
{
    if (stopped(b) || !resorting(b)) return;
    __shared__ uint32_t wsum[32];
    __shared__ uint32_t s_base, s_max;
    int t = threadIdx.x, lane = t & 31, w = t >> 5;
    {
        uint32_t acc = 0;
        int end = blockIdx.x * SCAN_CHUNK;
        for (int c = t; c < end; c += 1024) acc += b.cell_count[c];
        for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(FULL, acc, o);
        if (t == 0) {
            s_base = 0;
            s_max = 0;
        }
        __syncthreads();
        if (lane == 0) atomicAdd(&s_base, acc);
    }
    int c0 = blockIdx.x * SCAN_CHUNK + 4 * t;
    uint32_t v[4], sum = 0, mx = 0;
#pragma unroll
    for (int k = 0; k < 4; k++) {
        v[k] = (c0 + k < P.ncell) ? b.cell_count[c0 + k] : 0u;
        sum += v[k];
        mx = max(mx, v[k]);
    }
    uint32_t inc = sum;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        uint32_t u = __shfl_up_sync(FULL, inc, o);
        if (lane >= o) inc += u;
    }
    if (lane == 31) wsum[w] = inc;
    __syncthreads();
    if (w == 0) {
        uint32_t x = wsum[lane], xi = x;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            uint32_t u = __shfl_up_sync(FULL, xi, o);
            if (lane >= o) xi += u;
        }
        wsum[lane] = xi - x;
    }
    __syncthreads();
    uint32_t run = s_base + wsum[w] + inc - sum;
#pragma unroll
    for (int k = 0; k < 4; k++) {
        if (c0 + k < P.ncell) b.cell_start[c0 + k] = run;
        run += v[k];
    }
    atomicMax(&s_max, mx);
    __syncthreads();
    if (t == 0) {
        if (blockIdx.x == gridDim.x - 1) b.cell_start[P.ncell] = (uint32_t)P.n;
        if (s_max > (uint32_t)MAXC) atomicOr(b.err, EB_CELL);
    }
}

// ---------------------------------------------------------------------------------------------
// Kernel 3: scatter particle indices into their cells
// ---------------------------------------------------------------------------------------------

__global__ void __launch_bounds__(256) k_scatter(DevParams P, Bufs b)
{
    if (stopped(b) || !resorting(b)) return;
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < P.n) b.perm[b.cell_start[b.key[i]] + b.rank[i]] = (uint32_t)i;
    // every scan block has read the cell counts: clear them for the next step
    for (int c = i; c < P.ncell; c += gridDim.x * blockDim.x) b.cell_count[c] = 0u;
}

// ---------------------------------------------------------------------------------------------
// Kernel 4: order each cell by previous index (a stable sort overall) and gather the state into
// cell order; FP32 offsets from the cell corner.  One warp per cell.
// ---------------------------------------------------------------------------------------------

__global__ void __launch_bounds__(256) k_cell_order(DevParams P, Bufs b)
{
    if (stopped(b) || !resorting(b)) return;
    __shared__ uint32_t srt[8][MAXC];
    int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
    int c = blockIdx.x * 8 + w;
    if (c >= P.ncell) return;
    uint32_t start = b.cell_start[c];
    int cnt = (int)(b.cell_start[c + 1] - start);   // <= MAXC: k_scan raised EB_CELL otherwise
    uint32_t v0 = lane < cnt ? b.perm[start + lane] : 0xffffffffu;
    uint32_t v1 = lane + 32 < cnt ? b.perm[start + 32 + lane] : 0xffffffffu;
    // rank of each entry among the cell's entries (all distinct); a cell already in ascending
    // order (entries scattered by one warp, or by warps that happened to run in order) skips it
    int r0 = lane, r1 = lane + 32;
    uint32_t nxt = __shfl_down_sync(FULL, v0, 1);
    bool ordered = cnt <= 32 && (lane + 1 >= cnt || v0 < nxt);
    if (!__all_sync(FULL, ordered)) {
        r0 = 0;
        r1 = 0;
        int lim = min(cnt, 32);
        for (int k = 0; k < lim; k++) {
            uint32_t a = __shfl_sync(FULL, v0, k);
            r0 += (a < v0);
            r1 += (a < v1);
        }
        for (int k = 0; k < cnt - 32; k++) {
            uint32_t d = __shfl_sync(FULL, v1, k);
            r0 += (d < v0);
            r1 += (d < v1);
        }
    }
    if (lane < cnt) srt[w][r0] = v0;
    if (lane + 32 < cnt) srt[w][r1] = v1;
    __syncwarp();
    // predicted positions and velocities from the output set, the rest of the state from the input
    const StateSet in = state_in(b), out = state_out(b);
    for (int s = lane; s < cnt; s += 32) {
        uint32_t old = srt[w][s], g = start + (uint32_t)s;
        b.mx[g] = out.x[old];
        b.my[g] = out.y[old];
        b.xi[g] = b.sxi[old];
        b.mkey[g] = (uint32_t)c;
        b.mu4[g] = make_float4(out.ux[old], out.uy[old], in.q11[old], in.q12[old]);
        b.mdr[g] = in.dr[old];
        b.mid[g] = in.id[old];
    }
}

// Exact support test of a candidate at FP32 squared distance r2: FP32 outside the rounding band,
// the FP64 definition inside it.
__device__ __forceinline__ bool in_support(float r2, const DevParams &P, const Bufs &b, int gi, int gj)
{
    bool in = r2 < P.R2lo;
    if (!in && r2 < P.R2hi) {
        in = support64(P, b, gi, gj);
        atomicAdd(b.band, 1ull);
    }
    return in;
}

// ---------------------------------------------------------------------------------------------
// Kernel 5 (re-sort steps only): pass A -- candidate lists, neighbour counts, sum_j W_ij (self
// included) and V = 1/sum  (Eqs. 18, 19)
//
// Two levels.  The coarse scan runs over the 3 x 3 cell stencil (three contiguous slot ranges, one
// per stencil row) on the hi parts alone against a padded radius, appending candidates without a
// branch.  The fine pass forms the correctly rounded pair vector of each candidate and keeps those
// within 3h (1 + SKIN): the candidate list of this and the following steps.  For this step it also
// counts the neighbours (exact support test) and sums W, which is zero beyond the support.
// With FROM_REF the positions are those of the last re-sort (xi_ref) and only the candidate lists
// are rebuilt (used after a checkpoint is loaded).
// ---------------------------------------------------------------------------------------------

// Candidate lists hold the byte offset 16 * slot of each candidate's 16-byte staging slot, two
// 16-bit entries per 32-bit half of a 64-bit word; the mask keeps every offset inside the HCAP
// staged slots.  Bit 0 of an entry (free: offsets are multiples of 16) is the candidate's neighbour
// bit of the present step (within 3h by the exact test), set by pass A; bits 1..3 are zero.
constexpr uint32_t SLOT_OFF_MASK = (HCAP - 1) << 4;
static_assert(((HCAP - 1) << 4) <= 0xffff, "slot offsets must fit 16 bits");

constexpr int SMEM_A = HCAP * (16 + 4 + 1) + MAXV * PT * 2;

template <bool FROM_REF>
__global__ void __launch_bounds__(PT) k_pass_a_resort(DevParams P, Bufs b)
{
    if (stopped(b) || (!FROM_REF && !resorting(b))) return;
    __shared__ TileShared ts;
    extern __shared__ __align__(16) unsigned char dsm[];
    float4 *pos = reinterpret_cast<float4 *>(dsm);
    const float2 *phi = reinterpret_cast<const float2 *>(dsm);   // hi parts: phi[2 j] = pos[j].xy
    int *sg = reinterpret_cast<int *>(pos + HCAP);
    uint16_t *lst = reinterpret_cast<uint16_t *>(sg + HCAP);
    unsigned char *shc = reinterpret_cast<unsigned char *>(lst + MAXV * PT);
    Tile T;
    if (!tile_begin(P, b, ts, T)) {
        if (threadIdx.x == 0) atomicOr(b.err, EB_HALO);
        return;
    }
    for (int t = threadIdx.x; t < T.H; t += PT) {
        int h = slot_cell(ts, T.NH, t);
        int g = ts.start[h] + (t - ts.off[h]);
        float hx = (float)(h % T.HX), hy = (float)(h / T.HX);
        float4 o = FROM_REF ? b.xi_ref[g] : b.xi[g];
        pos[t] = make_float4(o.x + hx * P.cell_hi, o.y + hy * P.cell_hi, o.z + hx * P.cell_lo, o.w + hy * P.cell_lo);
        sg[t] = g;
        shc[t] = (unsigned char)h;
    }
    __syncthreads();
    if (!FROM_REF && blockIdx.x == 0 && threadIdx.x == 0) atomicAdd(b.resorts, 1u);
    uint16_t *my = lst + threadIdx.x;   // this thread's list column, stride PT
    for (int q = threadIdx.x; q < T.Ni; q += PT) {
        int si = inner_slot(ts, T, q);
        int h = shc[si], hx = h % T.HX, hy = h / T.HX;
        float4 pi = pos[si];
        int gi = sg[si];
        int cnt = 0;
        for (int oy = -1; oy <= 1; oy++) {
            int row = (hy + oy) * T.HX + hx;
            int j0 = ts.off[row - 1], j1 = ts.off[row + 2];
            for (int j = j0; j < j1; j++) {
                float2 pj = phi[2 * j];
                float dx = pi.x - pj.x, dy = pi.y - pj.y;
                bool in = (dx * dx + dy * dy < P.R2c) & (j != si);
                my[min(cnt, MAXV - 1) * PT] = (uint16_t)j;
                cnt += in;
            }
        }
        if (cnt > MAXV) {
            atomicOr(b.err, EB_NBR);
            cnt = MAXV;
        }
        float sw = P.W0;
        int cv = 0, nn = 0, nlow = 0;
        for (int k = 0; k < cnt; k++) {
            int j = my[k * PT];   // slot (the coarse scan stores slots)
            float2 d = pair_d(pi, pos[j]);
            float r2 = len2(d);
            bool cand = r2 < P.R2v;
            bool in = false;
            if (!FROM_REF && cand) {
                sw += kernel_w<true>(r2, P);
                in = in_support(r2, P, b, gi, sg[j]);
                nn += in;
            }
            // byte offset of the slot; bit 0 (free: offsets are multiples of 16) carries the support bit
            my[cv * PT] = (uint16_t)((j << 4) | (int)in);
            nlow += cand & (j < si);
            cv += cand;
        }
        // The kept candidates are in ascending slot order; the list starts at the first slot after
        // si and wraps around.  The threads of a warp hold consecutive slots, so at each step of
        // their walks they load mostly distinct, consecutive slots, which spreads the staged loads
        // of the pair passes over the shared-memory banks (ascending order: ~2x the bank conflicts).
        auto at = [&](int k) { return (uint32_t)my[(k + nlow < cv ? k + nlow : k + nlow - cv) * PT]; };
        uint2 *out = b.vnbr + gi;
        for (int k = 0; k < cv; k += 4) {
            uint32_t s0 = at(k);
            uint32_t s1 = (k + 1 < cv) ? at(k + 1) : 0u;
            uint32_t s2 = (k + 2 < cv) ? at(k + 2) : 0u;
            uint32_t s3 = (k + 3 < cv) ? at(k + 3) : 0u;
            *out = make_uint2(s0 | (s1 << 16), s2 | (s3 << 16));
            out += P.n;
        }
        b.vcnt[gi] = cv;
        if (!FROM_REF) {
            b.nnbr[gi] = nn;
            b.sumW[gi] = sw;
            b.V[gi] = 1.0f / sw;
            b.xi_ref[gi] = b.xi[gi];   // the split positions this re-sort used
        }
    }
}

// Occupancy hints of the pair passes (minimum resident blocks of PT threads per SM; 0 leaves the
// register budget to the compiler) and the list-word prefetch distance of each (1 to 3 words of
// four candidates).
// The defaults are the measured best on GB300 at 1M and 16M particles: the register caps they
// imply (32, 48, 48, 48; pass C takes 46 and runs without spills) keep the resident warps
// near what the staged shared memory allows, which hides the latency of the list and gather loads
// better than the instruction savings of more registers (pass D at 4 blocks per SM, 64 registers
// and no spills, is 8 % slower than at 5).
#ifndef ANN_MINB_A
#define ANN_MINB_A 8
#endif
#ifndef ANN_MINB_B
#define ANN_MINB_B 5
#endif
#ifndef ANN_MINB_C
#define ANN_MINB_C 5
#endif
#ifndef ANN_MINB_D
#define ANN_MINB_D 5
#endif
#ifndef ANN_PF_A
#define ANN_PF_A 1
#endif
#ifndef ANN_PF_B
#define ANN_PF_B 1
#endif
#ifndef ANN_PF_C
#define ANN_PF_C 1
#endif
#ifndef ANN_PF_D
#define ANN_PF_D 1
#endif
#define ANN_BOUNDS(minb) __launch_bounds__(PT, (minb) > 0 ? (minb) : 1)
#if ANN_MINB_A > 0
#define BOUNDS_A ANN_BOUNDS(ANN_MINB_A)
#else
#define BOUNDS_A __launch_bounds__(PT)
#endif
#if ANN_MINB_B > 0
#define BOUNDS_B ANN_BOUNDS(ANN_MINB_B)
#else
#define BOUNDS_B __launch_bounds__(PT)
#endif
#if ANN_MINB_C > 0
#define BOUNDS_C ANN_BOUNDS(ANN_MINB_C)
#else
#define BOUNDS_C __launch_bounds__(PT)
#endif
#if ANN_MINB_D > 0
#define BOUNDS_D ANN_BOUNDS(ANN_MINB_D)
#else
#define BOUNDS_D __launch_bounds__(PT)
#endif

// Visit the candidates of particle gi (c of them, four per 64-bit list word) in order, keeping the
// next PF words in flight while the current ones are processed: fn(byte offset of the slot,
// candidate index, bit), bit = the entry's neighbour bit (nonzero iff the candidate is a neighbour).
// Word m (candidates 4m .. 4m + 3) is loaded only when 4m < c.
template <int PF, typename Fn>
__device__ __forceinline__ void for_each_slot(const uint2 *list, int n, int gi, int c, Fn &&fn)
{
    static_assert(PF >= 1 && PF <= 3, "prefetch distance");
    const uint2 *p = list + gi;
    uint2 r[PF + 1];   // r[0]: the current word, r[m]: word k/4 + m
#pragma unroll
    for (int m = 0; m <= PF; m++) r[m] = (4 * m < c) ? __ldg(p + (size_t)m * n) : make_uint2(0u, 0u);
    p += (size_t)(PF + 1) * n;
    int k = 0;
    for (; k + 3 < c; k += 4) {
        uint2 w = r[0];
#pragma unroll
        for (int m = 0; m < PF; m++) r[m] = r[m + 1];
        r[PF] = (k + 4 * (PF + 1) < c) ? __ldg(p) : make_uint2(0u, 0u);   // word k/4 + PF + 1
        p += n;
        fn((int)(w.x & SLOT_OFF_MASK), k, w.x & 1u);
        fn((int)((w.x >> 16) & SLOT_OFF_MASK), k + 1, w.x & 0x10000u);
        fn((int)(w.y & SLOT_OFF_MASK), k + 2, w.y & 1u);
        fn((int)((w.y >> 16) & SLOT_OFF_MASK), k + 3, w.y & 0x10000u);
    }
    unsigned long long w64 = ((unsigned long long)r[0].y << 32) | r[0].x;
    for (int t = 0; k < c; k++, t++) {   // the last 0 to 3 candidates
        const unsigned e = (unsigned)(w64 >> (16 * t));
        fn((int)(e & SLOT_OFF_MASK), k, e & 1u);
    }
}

// Candidates of particle gi.  Beyond the support the clamped kernel gives W = F = 0 exactly, and
// adding +0 or -0 leaves an FP32 sum unchanged, so sums over candidates equal sums over neighbours.
template <int PF, typename Fn>
__device__ __forceinline__ void for_each_candidate(const DevParams &P, const Bufs &b, int gi, Fn &&fn)
{
    for_each_slot<PF>(b.vnbr, P.n, gi, b.vcnt[gi], fn);
}

// ---------------------------------------------------------------------------------------------
// Kernel 6: pass A -- neighbour counts (exact support test on the candidates), sum_j W_ij (self
// included) and V = 1/sum  (Eqs. 18, 19).  Skipped on re-sort steps, which do this in kernel 5.
// ---------------------------------------------------------------------------------------------

constexpr int SMEM_AF = HCAP * (16 + 4);

__global__ void BOUNDS_A k_pass_a_filter(DevParams P, Bufs b)
{
    if (stopped(b) || resorting(b)) return;
    __shared__ TileShared ts;
    extern __shared__ __align__(16) unsigned char dsm[];
    float4 *pos = reinterpret_cast<float4 *>(dsm);
    int *sg = reinterpret_cast<int *>(pos + HCAP);
    Tile T;
    if (!tile_begin(P, b, ts, T)) {
        if (threadIdx.x == 0) atomicOr(b.err, EB_HALO);
        return;
    }
    for (int t = threadIdx.x; t < T.H; t += PT) {
        SlotInfo s = slot_info(P, b, ts, T, t);
        pos[t] = s.e;
        sg[t] = s.g;
    }
    __syncthreads();
    for (int q = threadIdx.x; q < T.Ni; q += PT) {
        int si = inner_slot(ts, T, q);
        int gi = sg[si];
        float4 pi = pos[si];
        float sw = P.W0;
        int c = b.vcnt[gi];
        // one walk over the list words, setting each candidate's neighbour bit by the FP32 test;
        // a candidate inside the rounding band around (3h)^2 (rare) is only noted here and decided
        // in FP64 by a second walk.  A word is stored only when a bit changed (a pair crossed 3h).
        int nn = 0;
        bool band = false;
        auto test = [&](uint32_t e) {
            const uint32_t o = e & SLOT_OFF_MASK;
            float r2 = len2(pair_d(pi, slot_at(pos, (int)o)));
            sw += kernel_w<true>(r2, P);
            const uint32_t in = r2 < P.R2lo;
            band |= (r2 >= P.R2lo) & (r2 < P.R2hi);
            nn += (int)in;
            return o | in;
        };
        uint2 *p = b.vnbr + gi;
        uint2 nxt = c > 0 ? *p : make_uint2(0u, 0u);   // plain loads: this kernel writes the words
        int k = 0;
        for (; k + 3 < c; k += 4, p += P.n) {
            const uint2 w = nxt;
            if (k + 4 < c) nxt = p[P.n];   // the next word, in flight while this one is done
            const uint32_t e0 = test(w.x & 0xffffu), e1 = test(w.x >> 16), e2 = test(w.y & 0xffffu),
                           e3 = test(w.y >> 16);
            const uint2 v = make_uint2(e0 | (e1 << 16), e2 | (e3 << 16));
            if (v.x != w.x || v.y != w.y) *p = v;
        }
        if (k < c) {   // the last word, 1 to 3 candidates (the rest of it is zero)
            const uint2 w = nxt;
            uint32_t e[4] = {w.x & 0xffffu, w.x >> 16, w.y & 0xffffu, w.y >> 16};
            for (int t = 0; t < c - k; t++) e[t] = test(e[t]);
            const uint2 v = make_uint2(e[0] | (e[1] << 16), e[2] | (e[3] << 16));
            if (v.x != w.x || v.y != w.y) *p = v;
        }
        if (band) {   // the band's candidates, decided in FP64 (the FP32 test left their bit 0)
            uint2 *q = b.vnbr + gi;
            for (int k0 = 0; k0 < c; k0 += 4, q += P.n) {
                uint2 w = *q;
                uint32_t e[4] = {w.x & 0xffffu, w.x >> 16, w.y & 0xffffu, w.y >> 16};
                for (int t = 0; t < 4 && k0 + t < c; t++) {
                    const int o = (int)(e[t] & SLOT_OFF_MASK);
                    float r2 = len2(pair_d(pi, slot_at(pos, o)));
                    if (r2 >= P.R2lo && in_support(r2, P, b, gi, slot_at(sg, o))) {
                        e[t] |= 1u;
                        nn++;
                    }
                }
                *q = make_uint2(e[0] | (e[1] << 16), e[2] | (e[3] << 16));
            }
        }
        b.nnbr[gi] = nn;
        b.sumW[gi] = sw;
        b.V[gi] = 1.0f / sw;
    }
}

// ---------------------------------------------------------------------------------------------
// Kernel 7: pass B -- correction tensor alpha and B = alpha^-1 (Eq. 22), corrected velocity
// gradient (Eq. 20), continuity (Eq. 25) and half-step density, Q Laplacian (Eq. 21), molecular
// field (Eq. 7), co-rotation term (Eq. 2) and the Q update of Eq. (24).
// ---------------------------------------------------------------------------------------------

constexpr int SMEM_B = HCAP * (16 + 16 + 4 + 4);

template <bool QOLD>
__global__ void BOUNDS_B k_pass_b(DevParams P, Bufs b)
{
    if (stopped(b)) return;
    if (blockIdx.x == 0 && threadIdx.x == 0) *b.rebuild = 0u;   // both pass A kernels have run
    __shared__ TileShared ts;
    extern __shared__ __align__(16) unsigned char dsm[];
    float4 *sp = reinterpret_cast<float4 *>(dsm);     // split position
    float4 *sb = sp + HCAP;                           // (ux, uy, q11, q12): two-lane pairs in place
    float *sv = reinterpret_cast<float *>(sb + HCAP); // V
    int *sg = reinterpret_cast<int *>(sv + HCAP);
    Tile T;
    if (!tile_begin(P, b, ts, T)) {
        if (threadIdx.x == 0) atomicOr(b.err, EB_HALO);
        return;
    }
    for (int t = threadIdx.x; t < T.H; t += PT) {
        SlotInfo s = slot_info(P, b, ts, T, t);
        sp[t] = s.e;
        sb[t] = b.mu4[s.g];
        sv[t] = b.V[s.g];
        sg[t] = s.g;
    }
    __syncthreads();
    for (int q = threadIdx.x; q < T.Ni; q += PT) {
        int si = inner_slot(ts, T, q);
        int gi = sg[si];
        float4 pi = sp[si], bi = sb[si];
        // two-lane accumulators: (a11, a12), a22; L rows (l00, l01), (l10, l11); Laplacian sums
        // per tensor entry for (q11, q12): (r1xx, r2xx), (r1xy, r2xy), (r1yy, r2yy); div Q rows
        float2 a1 = f2(0.f, 0.f), l0 = f2(0.f, 0.f), l1 = f2(0.f, 0.f);
        float2 rxx = f2(0.f, 0.f), rxy = f2(0.f, 0.f), ryy = f2(0.f, 0.f);
        float2 gq1 = f2(0.f, 0.f), gq2 = f2(0.f, 0.f);
        float a22 = 0.f;
        float di = b.mdr[gi];   // loaded ahead of the neighbour loop
        const float2 ui = f2(bi.x, bi.y), qi = f2(bi.z, bi.w);
        for_each_candidate<ANN_PF_B>(P, b, gi, [&](int o, int, unsigned) {
            float4 bj = slot_at(sb, o);
            float2 d = pair_d(pi, slot_at(sp, o));
            KernelPowers kp = kernel_powers<true>(len2(d), P);
            float F = kernel_f_of(kp, P);
            float2 g = mul2(bc(slot_at(sv, o) * F), d);  // V_j grad_i W = (gx, gy)
            float2 mx = mul2(bc(g.x), d);                 // (mxx, mxy)
            float myy = g.y * d.y;
            a1 = sub2(a1, mx);
            a22 -= myy;
            float2 du = sub2(f2(bj.x, bj.y), ui);         // u_j - u_i
            l0 = fma2(bc(du.x), g, l0);
            l1 = fma2(bc(du.y), g, l1);
            float2 dq = sub2(f2(bj.z, bj.w), qi);         // Q_j - Q_i per component
            float2 e = mul2(dq, bc(-(kp.rinv * kp.rinv)));
            rxx = fma2(e, bc(mx.x), rxx);
            rxy = fma2(e, bc(mx.y), rxy);
            ryy = fma2(e, bc(myy), ryy);
            if (QOLD) {
                gq1 = fma2(bc(dq.x), g, gq1);
                gq2 = fma2(bc(dq.y), g, gq2);
            }
        });
        float a11 = a1.x, a12 = a1.y;
        float l00 = l0.x, l01 = l0.y, l10 = l1.x, l11 = l1.y;
        float r1xx = rxx.x, r2xx = rxx.y, r1xy = rxy.x, r2xy = rxy.y, r1yy = ryy.x, r2yy = ryy.y;
        float g1x = gq1.x, g1y = gq1.y, g2x = gq2.x, g2y = gq2.y;
        float det = a11 * a22 - a12 * a12;
        if (!(det > 0.f)) atomicOr(b.err, EB_SINGULAR);
        float idet = 1.f / det;
        float B11 = a22 * idet, B12 = -a12 * idet, B22 = a11 * idet;
        // D[a][b] = du_a/dx_b = sum_l L[a][l] B[l][b]
        float D00 = l00 * B11 + l01 * B12, D01 = l00 * B12 + l01 * B22;
        float D10 = l10 * B11 + l11 * B12, D11 = l10 * B12 + l11 * B22;
        float divu = D00 + D11;
        float kr = -(1.f + di) * divu;
        float lap1 = 2.f * (B11 * r1xx + 2.f * B12 * r1xy + B22 * r1yy);
        float lap2 = 2.f * (B11 * r2xx + 2.f * B12 * r2xy + B22 * r2yy);
        // Q rate, projected on symmetric traceless tensors.  With E = sym(D), w = (D10 - D01)/2:
        //   S_tl = lambda tr(E) Q + 2 c lambda E_tl + (Omega Q - Q Omega) - 2 lambda (Q:E) Q
        //   H_tl = -A Q - C tr(Q^2) Q + K lap Q        (the B term of Eq. 7 is isotropic in 2D)
        float q1 = bi.z, q2 = bi.w;
        float E12 = 0.5f * (D01 + D10), om = 0.5f * (D10 - D01);
        float QE = q1 * (D00 - D11) + 2.f * q2 * E12;
        float trQ2 = 2.f * (q1 * q1 + q2 * q2);
        float lam = P.lambda, cl = P.c_shift * lam;
        float hb = -P.A - P.C * trQ2;
        float m1 = lam * divu * q1 + cl * (D00 - D11) - 2.f * om * q2 - 2.f * lam * QE * q1 +
                   P.Gamma * (hb * q1 + P.K * lap1);
        float m2 = lam * divu * q2 + 2.f * cl * E12 + 2.f * om * q1 - 2.f * lam * QE * q2 +
                   P.Gamma * (hb * q2 + P.K * lap2);
        const float q1n = q1 + P.dt * m1, q2n = q2 + P.dt * m2;
        {
            const StateSet out = state_out(b);   // Q^{n+1} into the step's output set
            out.q11[gi] = q1n;
            out.q12[gi] = q2n;
        }
        if (P.elastic) {
            // Elastic stress of Eq. (12) without -p I: with H = H_tl + h0 I (h0 from the B term),
            // M = Q + c I and the 2D identity A B + B A = (A:B) I for symmetric traceless A, B:
            //   Pi = 2 lambda M (Q:H) - lambda [(Q:H) I + 2c H_tl + 2 h0 Q + 2c h0 I]
            float h1 = hb * q1 + P.K * lap1, h2 = hb * q2 + P.K * lap2;
            float h0 = P.Bl * trQ2 * (1.f / 6.f);
            float c = P.c_shift, QH = 2.f * (q1 * h1 + q2 * h2);
            float iso = QH + 2.f * c * h0;
            float p11 = 2.f * lam * (q1 + c) * QH - lam * (iso + 2.f * c * h1 + 2.f * h0 * q1);
            float p22 = 2.f * lam * (c - q1) * QH - lam * (iso - 2.f * c * h1 - 2.f * h0 * q1);
            float p12 = 2.f * lam * q2 * QH - lam * (2.f * c * h2 + 2.f * h0 * q2);
            b.pel[gi] = make_float4(p11, p12, p22, 0.f);
        }
        b.bk[gi] = make_float4(B11, B12, B22, kr);
        b.cr[gi] = make_float4(sv[si], di + P.half_dt * kr, q1n, q2n);   // pass C's staged record
        if (QOLD) {   // div Q^n for pass D (pass C then leaves the divergence part of cq alone)
            float q1x = g1x * B11 + g1y * B12, q1y = g1x * B12 + g1y * B22;
            float q2x = g2x * B11 + g2y * B12, q2y = g2x * B12 + g2y * B22;
            float2 *dq = reinterpret_cast<float2 *>(b.cq + gi);
            *dq = make_float2(q1x + q2y, q2x - q1y);
        }
        if (P.record) {
            b.rec_gu[4 * gi + 0] = D00;
            b.rec_gu[4 * gi + 1] = D01;
            b.rec_gu[4 * gi + 2] = D10;
            b.rec_gu[4 * gi + 3] = D11;
            b.rec_lap[2 * gi + 0] = lap1;
            b.rec_lap[2 * gi + 1] = lap2;
            b.rec_qrate[2 * gi + 0] = m1;
            b.rec_qrate[2 * gi + 1] = m2;
        }
    }
}

// ---------------------------------------------------------------------------------------------
// Kernel 8: pass C -- density filter (Eq. 28), equation of state (Eq. 26), div Q^{n+1}
// ---------------------------------------------------------------------------------------------

// the elastic stress tile exists only in the instantiations that read it
constexpr int smem_c(bool el) { return HCAP * (16 + 16 + (el ? 16 : 0) + 4); }

template <bool QNEW, bool EL>
__global__ void BOUNDS_C k_pass_c(DevParams P, Bufs b)
{
    if (stopped(b)) return;
    __shared__ TileShared ts;
    extern __shared__ __align__(16) unsigned char dsm[];
    float4 *sp = reinterpret_cast<float4 *>(dsm);      // split position
    float4 *sb = sp + HCAP;                            // (V, drho_half, q11^{n+1}, q12^{n+1})
    float4 *se = sb + HCAP;                            // elastic stress (11, 12, 22, -)
    int *sg = reinterpret_cast<int *>(se + (EL ? HCAP : 0));
    Tile T;
    if (!tile_begin(P, b, ts, T)) {
        if (threadIdx.x == 0) atomicOr(b.err, EB_HALO);
        return;
    }
    const StateSet out = state_out(b);   // Q^{n+1} (pass B)
    for (int t = threadIdx.x; t < T.H; t += PT) {
        SlotInfo s = slot_info(P, b, ts, T, t);
        sp[t] = s.e;
        sb[t] = b.cr[s.g];   // (V, delta_half, Q^{n+1}); pass C reads Q^{n+1} only with QNEW
        if (EL) se[t] = b.pel[s.g];
        sg[t] = s.g;
    }
    __syncthreads();
    const float umax = __uint_as_float(*b.maxu);
    float c0 = fmaxf(10.f * umax, P.c0_min);
    float pref = P.rho0 * c0 * c0 / P.gamma_eos;
    // stability limits of this step's dt (a zero speed gives an infinite limit); pass D then stops
    if (P.dt_check && blockIdx.x == 0 && threadIdx.x == 0 &&
        (P.dt > P.dt_static || P.dt * (c0 + umax) * P.inv_h > 0.25f))
        atomicOr(b.err, EB_CFL);
    for (int q = threadIdx.x; q < T.Ni; q += PT) {
        int si = inner_slot(ts, T, q);
        int gi = sg[si];
        float4 pi = sp[si], bi = sb[si];
        float shep = 0.f;
        float swi = b.sumW[gi];   // loaded ahead of the neighbour loop
        float B11 = 0.f, B12 = 0.f, B22 = 0.f;
        if (QNEW || EL) {
            const float4 bb = b.bk[gi];
            B11 = bb.x;
            B12 = bb.y;
            B22 = bb.z;
        }
        float4 ei = EL ? se[si] : make_float4(0.f, 0.f, 0.f, 0.f);
        // two-lane accumulators: corrected-gradient raw sums of q11, q12 and of Pi11, Pi12, Pi22
        float2 gq1 = f2(0.f, 0.f), gq2 = f2(0.f, 0.f), ge1 = f2(0.f, 0.f), ge2 = f2(0.f, 0.f),
               ge3 = f2(0.f, 0.f);
        const float2 qi = f2(bi.z, bi.w);
        for_each_candidate<ANN_PF_C>(P, b, gi, [&](int o, int, unsigned) {
            float4 bj = slot_at(sb, o);
            float2 d = pair_d(pi, slot_at(sp, o));
            KernelPowers kp = kernel_powers<true>(len2(d), P);
            float Wv = kernel_w_of(kp, P);
            shep += (bi.y - bj.y) * Wv;
            if (QNEW || EL) {
                float2 g = mul2(bc(bj.x * kernel_f_of(kp, P)), d);
                if (QNEW) {
                    float2 dq = sub2(f2(bj.z, bj.w), qi);
                    gq1 = fma2(bc(dq.x), g, gq1);
                    gq2 = fma2(bc(dq.y), g, gq2);
                }
                if (EL) {
                    float4 ej = slot_at(se, o);
                    ge1 = fma2(bc(ej.x - ei.x), g, ge1);
                    ge2 = fma2(bc(ej.y - ei.y), g, ge2);
                    ge3 = fma2(bc(ej.z - ei.z), g, ge3);
                }
            }
        });
        float g1x = gq1.x, g1y = gq1.y, g2x = gq2.x, g2y = gq2.y;
        float e1x = ge1.x, e1y = ge1.y, e2x = ge2.x, e2y = ge2.y, e3x = ge3.x, e3y = ge3.y;
        float dhat = bi.y - P.beta * shep / swi;
        const float pg = pref * expm1f(P.gamma_eos * log1pf(dhat));
        b.p[gi] = pg;
        {   // pass D's staged record (V, p / rho_hat^2, u): one 16-byte load per staged slot there
            float rho = P.rho0 * (1.f + dhat);
            float irho = 1.f / rho;
            const float2 u = *reinterpret_cast<const float2 *>(b.mu4 + gi);
            b.rd[gi] = make_float4(bi.x, pg * irho * irho, u.x, u.y);
        }
        if (QNEW) {
            float q1x = g1x * B11 + g1y * B12, q1y = g1x * B12 + g1y * B22;
            float q2x = g2x * B11 + g2y * B12, q2y = g2x * B12 + g2y * B22;
            b.cq[gi] = make_float4(q1x + q2y, q2x - q1y, dhat, swi);
        } else {   // div Q^n came from pass B
            float2 *hs = reinterpret_cast<float2 *>(b.cq + gi) + 1;
            *hs = make_float2(dhat, swi);
        }
        if (EL) {   // div Pi = (d_x Pi11 + d_y Pi12, d_x Pi12 + d_y Pi22), corrected gradients
            float p11x = e1x * B11 + e1y * B12;
            float p12x = e2x * B11 + e2y * B12, p12y = e2x * B12 + e2y * B22;
            float p22y = e3x * B12 + e3y * B22;
            b.delx[gi] = p11x + p12y;
            b.dely[gi] = p12x + p22y;
        }
    }
}

// ---------------------------------------------------------------------------------------------
// Kernel 9: pass D -- momentum (Eq. 23), corrector (§3.1), APD (Eq. 29), re-insertion (Eq. 30)
// ---------------------------------------------------------------------------------------------

// (the (q11, q12)/rho^2 tile exists in the conservative mode only, Pi/rho^2 with the elastic stress)
constexpr int smem_d(bool cons, bool el) { return HCAP * (16 + 16 + (cons ? 8 : 0) + (cons && el ? 16 : 0) + 4); }

template <bool CONS, bool EL>
__global__ void BOUNDS_D k_pass_d(DevParams P, Bufs b)
{
    if (stopped(b)) return;
    __shared__ TileShared ts;
    extern __shared__ __align__(16) unsigned char dsm[];
    float4 *sp = reinterpret_cast<float4 *>(dsm);       // split position
    float4 *sb = sp + HCAP;                             // paper: (V, p/rho^2, ux, uy)  cons: (p/rho^2, 1/rho, ux, uy)
    float2 *sc = reinterpret_cast<float2 *>(sb + HCAP); // cons: (q11/rho^2, q12/rho^2)
    float4 *se = reinterpret_cast<float4 *>(sc + (CONS ? HCAP : 0)); // cons + elastic: Pi/rho^2
    int *sg = reinterpret_cast<int *>(se + ((CONS && EL) ? HCAP : 0));
    // the step's output set: Q^{n+1} (pass B) in, the new state out; k_commit of the next step (or
    // the host) commits it if no error has been raised by then
    if (blockIdx.x == 0 && threadIdx.x == 0) b.ctl[CTL_PENDING] = 1u;
    Tile T;
    if (!tile_begin(P, b, ts, T)) {
        if (threadIdx.x == 0) atomicOr(b.err, EB_HALO);
        return;
    }
    const StateSet out = state_out(b);
    for (int t = threadIdx.x; t < T.H; t += PT) {
        SlotInfo s = slot_info(P, b, ts, T, t);
        sp[t] = s.e;
        if (CONS) {
            float rho = P.rho0 * (1.f + reinterpret_cast<const float *>(b.cq + s.g)[2]);
            float irho = 1.f / rho;
            float pr = b.p[s.g] * irho * irho;
            const float4 m4 = b.mu4[s.g];
            float q1 = P.qnew ? out.q11[s.g] : m4.z;
            float q2 = P.qnew ? out.q12[s.g] : m4.w;
            sb[t] = make_float4(pr, irho, m4.x, m4.y);
            sc[t] = make_float2(q1 * irho * irho, q2 * irho * irho);
            if (EL) {
                float4 pe = b.pel[s.g];
                float ir2 = irho * irho;
                se[t] = make_float4(pe.x * ir2, pe.y * ir2, pe.z * ir2, 0.f);
            }
        } else {
            sb[t] = b.rd[s.g];
        }
        sg[t] = s.g;
    }
    __syncthreads();
    if (blockIdx.x == 0 && threadIdx.x == 0) *b.maxu = 0u;   // pass C has consumed it
    for (int q = threadIdx.x; q < T.Ni; q += PT) {
        int si = inner_slot(ts, T, q);
        int gi = sg[si];
        float4 pi = sp[si], bi = sb[si];
        float2 ci = CONS ? sc[si] : make_float2(0.f, 0.f);
        float4 eci = (CONS && EL) ? se[si] : make_float4(0.f, 0.f, 0.f, 0.f);
        int c = b.nnbr[gi];
        // the epilogue's other per-particle inputs are loaded after the neighbour loop: held across
        // it they would take 11 registers (and spill), while other warps hide their latency there
        float dhat = reinterpret_cast<const float *>(b.cq + gi)[2];
        float rho = P.rho0 * (1.f + dhat);
        // paper mode: pressure and viscous sums share grad_i W, so they accumulate as one vector
        //   w = sum_j V_j F [ -rho_i (p_i/rho_i^2 + p_j/rho_j^2) + kv (u_ij . d) / r^2 ] d,
        // with kv = 8 nu rho0 / rho_i, and a = B w + (active and elastic terms)
        float irho = 1.f / rho;
        float nrho = -rho, kv = 8.f * P.nu * P.rho0 * irho;
        float pci = nrho * bi.y;        // paper: -rho_i p_i / rho_i^2
        float k8 = 8.f * P.mu * bi.y;   // conservative: 8 mu / rho_i
        const float2 ui = f2(bi.z, bi.w);
        float2 w = f2(0.f, 0.f), su = f2(0.f, 0.f), sd = f2(0.f, 0.f);
        float sr = 0.f;
        for_each_candidate<ANN_PF_D>(P, b, gi, [&](int o, int, unsigned in) {
            float4 bj = slot_at(sb, o);
            float2 d = pair_d(pi, slot_at(sp, o));
            float r2 = len2(d);
            KernelPowers kp = kernel_powers<true>(r2, P);
            float Wv = kernel_w_of(kp, P), F = kernel_f_of(kp, P);
            float2 du = sub2(ui, f2(bj.z, bj.w));   // u_i - u_j
            float ud = fmaf(du.x, d.x, du.y * d.y);
            float rinv2 = kp.rinv * kp.rinv;
            if (CONS) {
                float2 cj = slot_at(sc, o);
                float2 g = mul2(bc(F), d);
                float visc = k8 * bj.y * ud * rinv2;
                w = fma2(bc(visc - (bi.x + bj.x)), g, w);
                float2 qs = add2(ci, cj);   // (Q11_i/rho_i^2 + Q11_j/rho_j^2, same for Q12)
                // Q.g = (qa gx + qb gy, qb gx - qa gy)
                float2 act = fma2(qs, bc(g.x), mul2(f2(qs.y, -qs.x), bc(g.y)));
                w = fma2(bc(-P.zeta), act, w);
                if (EL) {   // + sum_j m (Pi_i/rho_i^2 + Pi_j/rho_j^2) . grad_i W
                    float4 ecj = slot_at(se, o);
                    float2 e1 = add2(f2(eci.x, eci.y), f2(ecj.x, ecj.y));   // (Pi11, Pi12)
                    float e22 = eci.z + ecj.z;
                    w = fma2(e1, bc(g.x), fma2(f2(e1.y, e22), bc(g.y), w));
                }
            } else {
                float coef = fmaf(kv, ud * rinv2, fmaf(nrho, bj.y, pci));
                w = fma2(bc(bj.x * F * coef), d, w);
            }
            su = fma2(du, bc(Wv), su);
            // APD sums run over the neighbours only (their terms do not vanish at the support
            // edge): `in` is the candidate's bit of the neighbour mask
            if (in) {
                sr += kp.r;
                sd = fma2(d, bc(rinv2 * kp.rinv), sd);
            }
        });
        const float4 bb = b.bk[gi], cc = b.cq[gi];
        float kri = bb.w, swi = cc.w;
        float B11 = 0.f, B12 = 0.f, B22 = 0.f, dvx = 0.f, dvy = 0.f;
        if (!CONS) {
            B11 = bb.x;
            B12 = bb.y;
            B22 = bb.z;
            dvx = cc.x;
            dvy = cc.y;
        }
        const double mxi = b.mx[gi], myi = b.my[gi];
        float elx = 0.f, ely = 0.f;
        if (EL && !CONS) {
            elx = b.delx[gi];
            ely = b.dely[gi];
        }
        float ax, ay;
        if (CONS) {
            ax = P.mass * w.x;
            ay = P.mass * w.y;
        } else {
            ax = fmaf(B11, w.x, B12 * w.y) - P.zeta * irho * dvx + irho * elx;
            ay = fmaf(B12, w.x, B22 * w.y) - P.zeta * irho * dvy + irho * ely;
        }
        float sux = su.x, suy = su.y, sdx = sd.x, sdy = sd.y;
        float unx = bi.z + P.half_dt * ax, uny = bi.w + P.half_dt * ay;
        float apx = 0.f, apy = 0.f;
        if (P.apd && c > 0) {
            float uv = sqrtf(sux * sux + suy * suy) / swi;
            float r0 = sr / (float)c;
            float sc_ = P.dt * uv * r0 * r0;
            apx = sc_ * sdx;
            apy = sc_ * sdy;
        }
        float stepx = P.half_dt * unx + apx, stepy = P.half_dt * uny + apy;
        double xn = mxi + (double)stepx;
        double yn = myi + (double)stepy;
        if (!(in_box(xn, P.bitsL) && in_box(yn, P.bitsL))) {   // rare: re-insert (Eq. 30)
            int kx = wrap_count(xn, P.L), ky = wrap_count(yn, P.L);
            xn = xn + 0.0;
            yn = yn + 0.0;
            if (kx | ky) add_crossing(b, b.mid[gi], kx, ky);   // periodic image count (pathlines)
        }
        float dn = dhat + P.half_dt * kri;
        if (!(isfinite(unx) && isfinite(uny) && isfinite(dn) && in_box(xn, P.bitsL) &&
              in_box(yn, P.bitsL) && isfinite(out.q11[gi]) && isfinite(out.q12[gi])))
            atomicOr(b.err, EB_NONFINITE);
        out.x[gi] = xn;
        out.y[gi] = yn;
        out.ux[gi] = unx;
        out.uy[gi] = uny;
        out.dr[gi] = dn;
        out.ax[gi] = ax;
        out.ay[gi] = ay;
        out.id[gi] = b.mid[gi];
        if (P.record) {
            b.rec_apd[2 * gi + 0] = apx;
            b.rec_apd[2 * gi + 1] = apy;
        }
    }
}

// First node of every step: the previous step is complete -- commit its output set -- unless an
// error has been raised since it began (then nothing here changes: the host rolls back).  Also
// starts this step's crossing log.  One thread.
__global__ void k_commit(Bufs b)
{
    if (*(volatile uint32_t *)b.err != 0u) return;
    volatile uint32_t *c = b.ctl;
    if (c[CTL_PENDING]) {
        c[CTL_CUR] ^= 1u;
        c[CTL_PENDING] = 0u;
        c[CTL_COMMITS] += 1u;
    }
    c[CTL_XLOG] = 0u;
}

// Takes back the image-count changes of a failed step's logged crossings.
__global__ void k_undo_crossings(Bufs b, int n_log)
{
    int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= n_log) return;
    const int4 e = b.xlog[k];
    atomicSub(&b.img[e.x].x, e.y);
    atomicSub(&b.img[e.x].y, e.z);
}

// Copies the re-sort decision into the condition of the step graph's IF / ELSE node.
__global__ void k_set_condition(Bufs b, cudaGraphConditionalHandle h)
{
    cudaGraphSetConditional(h, *(volatile uint32_t *)b.rebuild != 0u ? 1u : 0u);
}

// ---------------------------------------------------------------------------------------------
// Utility kernels (outside the time step)
// ---------------------------------------------------------------------------------------------

__global__ void k_load(DevParams P, Bufs b, const double *x, const double *y, const double *ux,
                       const double *uy, const double *q11, const double *q12, const double *rho,
                       bool reset_images)
{
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= P.n) return;
    double xx = x[i], yy = y[i];
    double r = rho ? rho[i] : (double)P.rho0;
    bool ok = isfinite(xx) && isfinite(yy) && isfinite(ux[i]) && isfinite(uy[i]) &&
              isfinite(q11[i]) && isfinite(q12[i]) && isfinite(r) && r > 0.0;
    if (!ok) {
        atomicOr(b.err, EB_NONFINITE);
        xx = 0.0;
        yy = 0.0;
    }
    if (xx < -P.L || xx >= 2.0 * P.L) xx = xx - floor(xx / P.L) * P.L;
    if (yy < -P.L || yy >= 2.0 * P.L) yy = yy - floor(yy / P.L) * P.L;
    b.sx[i] = wrap_d(xx, P.L) + 0.0;
    b.sy[i] = wrap_d(yy, P.L) + 0.0;
    b.sux[i] = (float)ux[i];
    b.suy[i] = (float)uy[i];
    b.sq11[i] = (float)q11[i];
    b.sq12[i] = (float)q12[i];
    b.sdr[i] = rho ? (float)(r / (double)P.rho0 - 1.0) : 0.f;
    b.sax[i] = 0.f;
    b.say[i] = 0.f;
    b.sid[i] = i;
    if (reset_images) b.img[i] = make_int2(0, 0);   // pathlines start at the loaded (wrapped) positions
}

template <typename T>
__global__ void k_unpermute(const T *f, const int *id, T *out, int n)
{
    int g = blockIdx.x * blockDim.x + threadIdx.x;
    if (g < n) out[id[g]] = f[g];
}

__global__ void __launch_bounds__(PT) k_export_nbrs(DevParams P, Bufs b, int *cols)
{
    __shared__ TileShared ts;
    extern __shared__ __align__(16) unsigned char dsm[];
    float4 *pos = reinterpret_cast<float4 *>(dsm);
    int *sg = reinterpret_cast<int *>(pos + HCAP);
    Tile T;
    if (!tile_begin(P, b, ts, T)) return;
    for (int t = threadIdx.x; t < T.H; t += PT) {
        SlotInfo s = slot_info(P, b, ts, T, t);
        pos[t] = s.e;
        sg[t] = s.g;
    }
    __syncthreads();
    for (int q = threadIdx.x; q < T.Ni; q += PT) {
        int si = inner_slot(ts, T, q);
        int gi = sg[si];
        int k = 0;
        for_each_candidate<1>(P, b, gi, [&](int o, int, unsigned in) {
            int j = o >> 4;
            if (in && j < T.H && k < MAXN) {
                cols[(size_t)k * P.n + gi] = b.mid[sg[j]];
                k++;
            }
        });
    }
}

// The neighbour graph of the present positions in particle-ID order, for the learned surrogate:
// row id = mid[g] of particle g holds its neighbours' IDs and kernel values W(|d|) (the exact
// support test's neighbours, from the mask), the count, and S = sum_j W + W(0) of the search;
// the state is gathered by ID too.  Runs after a search at the present positions.
constexpr int SMEM_EX = HCAP * (16 + 4 + 16 + 8);   // position, slot, (u, Q), a

// Graph export for the surrogate, one walk of each particle's candidates at the present
// positions: the neighbours closer than 2h (the network's graph) into the ELL rows with W and their
// normalisation S2, and over the whole support (3h) the SPH means (Eq. 19 weights W / sum W, self
// term included) of (ux, uy, Q11, Q12) and of the recorded acceleration (o.tend_id planes 0, 1 by
// particle ID).
__global__ void __launch_bounds__(PT) k_export_graph(DevParams P, Bufs b, GraphOut o)
{
    __shared__ TileShared ts;
    extern __shared__ __align__(16) unsigned char dsm[];
    float4 *pos = reinterpret_cast<float4 *>(dsm);
    float4 *su = pos + HCAP;                                  // (ux, uy, q11, q12)
    float2 *sa = reinterpret_cast<float2 *>(su + HCAP);       // (ax, ay)
    int *sg = reinterpret_cast<int *>(sa + HCAP);
    Tile T;
    if (!tile_begin(P, b, ts, T)) return;
    for (int t = threadIdx.x; t < T.H; t += PT) {
        SlotInfo s = slot_info(P, b, ts, T, t);
        pos[t] = s.e;
        sg[t] = s.g;
        su[t] = b.mu4[s.g];
        const int id = b.mid[s.g];
        sa[t] = make_float2(o.tend_id[id], o.tend_id[(size_t)P.n + id]);
    }
    __syncthreads();
    const float r2net = 4.f / (P.inv_h * P.inv_h);
    for (int q = threadIdx.x; q < T.Ni; q += PT) {
        int si = inner_slot(ts, T, q);
        int gi = sg[si];
        float4 pi = pos[si], ui = su[si];
        float2 ai = sa[si];
        int k = 0;
        float s2 = P.W0;
        float4 m4 = make_float4(P.W0 * ui.x, P.W0 * ui.y, P.W0 * ui.z, P.W0 * ui.w);
        float2 m2 = make_float2(P.W0 * ai.x, P.W0 * ai.y);
        for_each_candidate<1>(P, b, gi, [&](int off, int, unsigned in) {
            int j = off >> 4;
            if (in && j < T.H) {
                float r2 = len2(pair_d(pi, slot_at(pos, off)));
                float w = kernel_w<true>(r2, P);
                float4 uj = slot_at(su, off);
                float2 aj = slot_at(sa, off);
                m4.x = fmaf(w, uj.x, m4.x);
                m4.y = fmaf(w, uj.y, m4.y);
                m4.z = fmaf(w, uj.z, m4.z);
                m4.w = fmaf(w, uj.w, m4.w);
                m2.x = fmaf(w, aj.x, m2.x);
                m2.y = fmaf(w, aj.y, m2.y);
                if (r2 < r2net) {
                    if (k < MAXN2H) {
                        o.nbr[(size_t)k * P.n + gi] = sg[j];
                        o.W[(size_t)k * P.n + gi] = w;
                        s2 += w;
                        k++;
                    } else {
                        *o.overflow = 1u;   // the graph cannot hold this particle's neighbours
                    }
                }
            }
        });
        const float is = 1.f / b.sumW[gi];
        o.cnt2[gi] = k;
        o.S2[gi] = s2;
        o.agg1[gi] = m2.x * is;
        o.agg1[(size_t)P.n + gi] = m2.y * is;
        // the network's input row (16 BF16): (Q11, Q12, ux/us, uy/us), their deviation from the
        // support mean, and the 8 tendencies scaled to increments over k dt
        {
            const int id = b.mid[gi];
            const float r[4] = {ui.z, ui.w, ui.x * o.inv_us, ui.y * o.inv_us};
            const float mr[4] = {m4.z * is, m4.w * is, m4.x * is * o.inv_us, m4.y * is * o.inv_us};
            float f[16];
            for (int c = 0; c < 4; c++) {
                f[c] = r[c];
                f[4 + c] = mr[c] - r[c];
            }
            for (int c = 0; c < 8; c++) f[8 + c] = o.tend_id[(size_t)c * P.n + id] * o.scale[c >> 1];
            uint4 w[2];
            __nv_bfloat162 *h2 = reinterpret_cast<__nv_bfloat162 *>(w);
            for (int c = 0; c < 8; c++) h2[c] = __floats2bfloat162_rn(f[2 * c], f[2 * c + 1]);
            uint4 *row = reinterpret_cast<uint4 *>(o.X + 16 * (size_t)gi);
            row[0] = w[0];
            row[1] = w[1];
        }
        o.x[gi] = b.mx[gi];
        o.y[gi] = b.my[gi];
        o.u4[gi] = make_float4(ui.x, ui.y, ui.z, ui.w);
        o.dr[gi] = b.mdr[gi];
        o.ids[gi] = b.mid[gi];
    }
}

// The second support mean of the acceleration and the explicit increment of the surrogate:
// inc[g] = kdt (m11, m12, agg(agg1)x, agg(agg1)y), with m the recorded Q rate (tend_id planes 2, 3
// by particle ID); the same walk as the export (run right after it, on the same candidate lists).
__global__ void __launch_bounds__(PT) k_export_increment(DevParams P, Bufs b, const float *agg1,
                                                         const float *tend_id, float kdt, float *inc)
{
    __shared__ TileShared ts;
    extern __shared__ __align__(16) unsigned char dsm[];
    float4 *pos = reinterpret_cast<float4 *>(dsm);
    float2 *sa = reinterpret_cast<float2 *>(pos + HCAP);
    int *sg = reinterpret_cast<int *>(sa + HCAP);
    Tile T;
    if (!tile_begin(P, b, ts, T)) return;
    for (int t = threadIdx.x; t < T.H; t += PT) {
        SlotInfo s = slot_info(P, b, ts, T, t);
        pos[t] = s.e;
        sg[t] = s.g;
        sa[t] = make_float2(agg1[s.g], agg1[(size_t)P.n + s.g]);
    }
    __syncthreads();
    for (int q = threadIdx.x; q < T.Ni; q += PT) {
        int si = inner_slot(ts, T, q);
        int gi = sg[si];
        float4 pi = pos[si];
        float2 ai = sa[si];
        float2 m2 = make_float2(P.W0 * ai.x, P.W0 * ai.y);
        for_each_candidate<1>(P, b, gi, [&](int off, int, unsigned in) {
            int j = off >> 4;
            if (in && j < T.H) {
                float w = kernel_w<true>(len2(pair_d(pi, slot_at(pos, off))), P);
                float2 aj = slot_at(sa, off);
                m2.x = fmaf(w, aj.x, m2.x);
                m2.y = fmaf(w, aj.y, m2.y);
            }
        });
        const float is = 1.f / b.sumW[gi];
        const int id = b.mid[gi];
        *reinterpret_cast<float4 *>(inc + 4 * (size_t)gi) =
            make_float4(kdt * tend_id[2 * (size_t)P.n + id], kdt * tend_id[3 * (size_t)P.n + id], kdt * m2.x * is,
                        kdt * m2.y * is);
    }
}

// Per-block partial sums in FP64: out[blk * NDIAG + q].
__global__ void __launch_bounds__(256) k_diag_partial(DevParams P, Bufs b, double *part)
{
    __shared__ double red[256];
    double v[NDIAG];
    for (int q = 0; q < NDIAG; q++) v[q] = 0.0;
    v[3] = 0.0;
    v[7] = 1e300;
    v[8] = -1e300;
    v[9] = 1e300;
    for (int g = blockIdx.x * blockDim.x + threadIdx.x; g < P.n; g += gridDim.x * blockDim.x) {
        double ux = b.sux[g], uy = b.suy[g];
        double rho = (double)P.rho0 * (1.0 + (double)b.sdr[g]);
        double m = P.conservative ? (double)P.mass : rho * (double)b.V[g];
        v[0] += m * ux;
        v[1] += m * uy;
        double u2 = ux * ux + uy * uy;
        v[2] += 0.5 * u2;
        v[3] = fmax(v[3], u2);   // max |u|^2; the square root is taken once, at the end
        v[4] += m;
        float q1 = b.sq11[g], q2 = b.sq12[g];
        v[5] += (double)sqrtf(q1 * q1 + q2 * q2);   // FP32 state: q in FP32, summed in FP64
        double nn = (double)b.nnbr[g];
        v[6] += nn;
        v[7] = fmin(v[7], nn);
        v[8] = fmax(v[8], nn);
        const float4 bb = b.bk[g];
        double b11 = bb.x, b12 = bb.y, b22 = bb.z;
        double detb = b11 * b22 - b12 * b12;
        v[9] = fmin(v[9], detb != 0.0 ? (double)(1.0f / (float)detb) : 1e300);
    }
    for (int q = 0; q < NDIAG; q++) {
        red[threadIdx.x] = v[q];
        __syncthreads();
        for (int s = 128; s > 0; s >>= 1) {
            if (threadIdx.x < s) {
                double a = red[threadIdx.x], c = red[threadIdx.x + s];
                red[threadIdx.x] = (q == 3 || q == 8) ? fmax(a, c) : ((q == 7 || q == 9) ? fmin(a, c) : a + c);
            }
            __syncthreads();
        }
        if (threadIdx.x == 0) part[blockIdx.x * NDIAG + q] = red[0];
        __syncthreads();
    }
}

// One block per quantity: a strided pass over the block partials, then a fixed-order tree.
__global__ void __launch_bounds__(256) k_diag_final(const double *part, int nblocks, double *out)
{
    __shared__ double red[256];
    int q = blockIdx.x;
    bool mx = (q == 3 || q == 8), mn = (q == 7 || q == 9);
    double acc = mn ? 1e300 : (mx ? -1e300 : 0.0);
    for (int k = threadIdx.x; k < nblocks; k += blockDim.x) {
        double a = part[k * NDIAG + q];
        acc = mx ? fmax(acc, a) : (mn ? fmin(acc, a) : acc + a);
    }
    red[threadIdx.x] = acc;
    __syncthreads();
    for (int s = 128; s > 0; s >>= 1) {
        if (threadIdx.x < s) {
            double a = red[threadIdx.x], c = red[threadIdx.x + s];
            red[threadIdx.x] = mx ? fmax(a, c) : (mn ? fmin(a, c) : a + c);
        }
        __syncthreads();
    }
    if (threadIdx.x == 0) out[q] = (q == 3) ? sqrt(red[0]) : red[0];
}

const char *const kNames[NKERNELS] = {"predict", "cell_keys", "cell_scan", "cell_scatter", "cell_order",
                                      "pass_a_resort", "pass_a", "pass_b", "pass_c", "pass_d"};

inline int blocks_for(int n, int t) { return (n + t - 1) / t; }

}  // namespace

const char *kernel_name(int k) { return (k >= 0 && k < NKERNELS) ? kNames[k] : nullptr; }

cudaError_t prepare_kernels()
{
    cudaError_t e;
    if ((e = cudaFuncSetAttribute(k_pass_a_resort<false>, cudaFuncAttributeMaxDynamicSharedMemorySize, SMEM_A))) return e;
    if ((e = cudaFuncSetAttribute(k_pass_a_resort<true>, cudaFuncAttributeMaxDynamicSharedMemorySize, SMEM_A))) return e;
    if ((e = cudaFuncSetAttribute(k_pass_a_filter, cudaFuncAttributeMaxDynamicSharedMemorySize, SMEM_AF))) return e;
    if ((e = cudaFuncSetAttribute(k_pass_b<false>, cudaFuncAttributeMaxDynamicSharedMemorySize, SMEM_B))) return e;
    if ((e = cudaFuncSetAttribute(k_pass_b<true>, cudaFuncAttributeMaxDynamicSharedMemorySize, SMEM_B))) return e;
    if ((e = cudaFuncSetAttribute(k_pass_c<false, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem_c(false)))) return e;
    if ((e = cudaFuncSetAttribute(k_pass_c<true, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem_c(false)))) return e;
    if ((e = cudaFuncSetAttribute(k_pass_c<false, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem_c(true)))) return e;
    if ((e = cudaFuncSetAttribute(k_pass_c<true, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem_c(true)))) return e;
    if ((e = cudaFuncSetAttribute(k_pass_d<false, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem_d(false, false)))) return e;
    if ((e = cudaFuncSetAttribute(k_pass_d<true, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem_d(true, false)))) return e;
    if ((e = cudaFuncSetAttribute(k_pass_d<false, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem_d(false, true)))) return e;
    if ((e = cudaFuncSetAttribute(k_pass_d<true, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem_d(true, true)))) return e;
    return cudaSuccess;
}

// Kernel k of the step on stream s (see kNames).
cudaError_t launch_kernel(int k, const DevParams &P, const Bufs &b, cudaStream_t s)
{
    int nb = blocks_for(P.n, 256), nt = P.tiles * P.tiles;
    switch (k) {
    case 0: k_predict<<<nb, 256, 0, s>>>(P, b); break;
    case 1: k_keys<<<nb, 256, 0, s>>>(P, b); break;
    case 2: k_scan<<<P.nsblk, 1024, 0, s>>>(P, b); break;
    case 3: k_scatter<<<nb, 256, 0, s>>>(P, b); break;
    case 4: k_cell_order<<<blocks_for(P.ncell, 8), 256, 0, s>>>(P, b); break;
    case 5: k_pass_a_resort<false><<<nt, PT, SMEM_A, s>>>(P, b); break;
    case 6: k_pass_a_filter<<<nt, PT, SMEM_AF, s>>>(P, b); break;
    case 7:
        if (P.qnew) k_pass_b<false><<<nt, PT, SMEM_B, s>>>(P, b);
        else k_pass_b<true><<<nt, PT, SMEM_B, s>>>(P, b);
        break;
    case 8: {
        bool el = P.elastic && !P.conservative;   // the paper momentum takes div Pi from here
        if (P.qnew && el) k_pass_c<true, true><<<nt, PT, smem_c(true), s>>>(P, b);
        else if (P.qnew) k_pass_c<true, false><<<nt, PT, smem_c(false), s>>>(P, b);
        else if (el) k_pass_c<false, true><<<nt, PT, smem_c(true), s>>>(P, b);
        else k_pass_c<false, false><<<nt, PT, smem_c(false), s>>>(P, b);
        break;
    }
    case 9:
        if (P.conservative && P.elastic) k_pass_d<true, true><<<nt, PT, smem_d(true, true), s>>>(P, b);
        else if (P.conservative) k_pass_d<true, false><<<nt, PT, smem_d(true, false), s>>>(P, b);
        else if (P.elastic) k_pass_d<false, true><<<nt, PT, smem_d(false, true), s>>>(P, b);
        else k_pass_d<false, false><<<nt, PT, smem_d(false, false), s>>>(P, b);
        break;
    default: return cudaErrorInvalidValue;
    }
    return cudaGetLastError();
}

cudaError_t launch_set_condition(const Bufs &b, cudaGraphConditionalHandle h, cudaStream_t s)
{
    k_set_condition<<<1, 1, 0, s>>>(b, h);
    return cudaGetLastError();
}

cudaError_t launch_commit(const Bufs &b, cudaStream_t s)
{
    k_commit<<<1, 1, 0, s>>>(b);
    return cudaGetLastError();
}

cudaError_t enqueue_undo_crossings(const Bufs &b, int n_log, cudaStream_t s)
{
    if (n_log <= 0) return cudaSuccess;
    k_undo_crossings<<<blocks_for(n_log, 256), 256, 0, s>>>(b, n_log);
    return cudaGetLastError();
}

cudaError_t enqueue_search(const DevParams &P, const Bufs &b, cudaStream_t s)
{
    cudaError_t e = cudaSuccess;
    for (int k = 0; k <= 5 && !e; k++) e = launch_kernel(k, P, b, s);
    if (e) return e;
    return cudaMemsetAsync(b.maxu, 0, sizeof(uint32_t), s);
}

cudaError_t enqueue_candidates_from_ref(const DevParams &P, const Bufs &b, cudaStream_t s)
{
    k_pass_a_resort<true><<<P.tiles * P.tiles, PT, SMEM_A, s>>>(P, b);
    return cudaGetLastError();
}

cudaError_t enqueue_load(const DevParams &P, const Bufs &b, const double *x, const double *y,
                         const double *ux, const double *uy, const double *q11, const double *q12,
                         const double *rho, cudaStream_t s, bool reset_images)
{
    k_load<<<blocks_for(P.n, 256), 256, 0, s>>>(P, b, x, y, ux, uy, q11, q12, rho, reset_images);
    return cudaGetLastError();
}

cudaError_t enqueue_unpermute(const void *f, const int *id, void *out, int n, int es, cudaStream_t s)
{
    if (es == 8)
        k_unpermute<unsigned long long><<<blocks_for(n, 256), 256, 0, s>>>(
            (const unsigned long long *)f, id, (unsigned long long *)out, n);
    else
        k_unpermute<uint32_t><<<blocks_for(n, 256), 256, 0, s>>>((const uint32_t *)f, id, (uint32_t *)out, n);
    return cudaGetLastError();
}

cudaError_t enqueue_export_graph(const DevParams &P, const Bufs &b, const GraphOut &o, float kdt, float *inc,
                                 cudaStream_t s)
{
    cudaError_t e = cudaFuncSetAttribute(k_export_graph, cudaFuncAttributeMaxDynamicSharedMemorySize, SMEM_EX);
    if (!e) e = cudaFuncSetAttribute(k_export_increment, cudaFuncAttributeMaxDynamicSharedMemorySize, SMEM_EX);
    if (e) return e;
    k_export_graph<<<P.tiles * P.tiles, PT, SMEM_EX, s>>>(P, b, o);
    k_export_increment<<<P.tiles * P.tiles, PT, HCAP * (16 + 8 + 4), s>>>(P, b, o.agg1, o.tend_id, kdt, inc);
    return cudaGetLastError();
}

cudaError_t enqueue_export_nbrs(const DevParams &P, const Bufs &b, int *cols_tmp, cudaStream_t s)
{
    k_export_nbrs<<<P.tiles * P.tiles, PT, SMEM_AF, s>>>(P, b, cols_tmp);
    return cudaGetLastError();
}

int diag_blocks(int n) { return std::min(std::max(blocks_for(n, 256), 1), 1024); }

cudaError_t enqueue_diag(const DevParams &P, const Bufs &b, double *partials, int nblocks, double *out,
                         cudaStream_t s)
{
    k_diag_partial<<<nblocks, 256, 0, s>>>(P, b, partials);
    k_diag_final<<<NDIAG, 256, 0, s>>>(partials, nblocks, out);
    return cudaGetLastError();
}

}  // namespace ann

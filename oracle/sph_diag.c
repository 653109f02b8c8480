/*
 * FP64 CPU oracle of the flow diagnostics of the paper's results section -- TEST INFRASTRUCTURE.
 *
 * Only tests/, __graft_entry__.smoke() and bench.py's CPU legs may load this code (through
 * oracle/diagnostics.py).  It shares nothing with the CUDA path.
 *
 * What the paper measures on the particle state, and the plain definitions taken here:
 *   - gridded fields: the spectrum, the vorticity correlation and the defects are analyses of
 *     continuous fields, while the state lives on particles.  The oracle samples a field f at the
 *     nodes (ix L/M, iy L/M) of an M x M grid by Shepard interpolation with the method's own
 *     kernel (Eq. 18):  f(x_g) = sum_j f_j W(|x_g - x_j|) / sum_j W(|x_g - x_j|), minimum-image
 *     distances, strict support r < 3h; a node with no particle in reach gets 0 and weight 0.
 *     Brute force over all particles, a cell-list form (same sums, other order) for larger
 *     cases, and a per-node form for sampled nodes of a full-size state.
 *   - topological defects: the paper labels a particle a defect when its neighbours' alignments
 *     match the +1/2 or -1/2 pattern.  The oracle counts, on the gridded Q, the winding number m
 *     of the vector (Q11, Q12) (the doubled director angle) around each grid plaquette
 *     (ix, iy) -> (ix+1, iy) -> (ix+1, iy+1) -> (ix, iy+1); the director's charge is m / 2.
 *     The winding number is computed exactly by counting signed crossings of the positive Q11
 *     axis (no angles): an edge a -> b with a12 <= 0 < b12 and cross(a, b) > 0 counts +1, one with
 *     b12 <= 0 < a12 and cross(a, b) < 0 counts -1, cross(a, b) = a11 b12 - a12 b11.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>

double orc_W(double b, double h);   /* quintic kernel of Eq. (18) at b = r/h, sph_oracle.c */

static double min_image(double d, double L)
{
    if (d > 0.5 * L) return d - L;
    if (d < -0.5 * L) return d + L;
    return d;
}

/* Contribution of particle j to node (gx, gy): W, or 0 beyond the support. */
static double node_weight(double gx, double gy, double xj, double yj, double L, double h)
{
    double dx = min_image(gx - xj, L), dy = min_image(gy - yj, L);
    double r2 = dx * dx + dy * dy;
    if (!(r2 < (3.0 * h) * (3.0 * h))) return 0.0;
    return orc_W(sqrt(r2) / h, h);
}

/* f is field-major: f[q * n + j].  out[q * M * M + iy * M + ix], wsum[iy * M + ix]. */
void orc_grid_shepard_brute(int64_t n, const double *x, const double *y, int32_t nf, const double *f,
                            double L, double h, int32_t M, double *out, double *wsum)
{
    int64_t MM = (int64_t)M * M;
#pragma omp parallel for schedule(static)
    for (int64_t g = 0; g < MM; g++) {
        double gx = (double)(g % M) * L / M, gy = (double)(g / M) * L / M;
        double sw = 0.0, acc[16] = {0};
        for (int64_t j = 0; j < n; j++) {
            double w = node_weight(gx, gy, x[j], y[j], L, h);
            if (w == 0.0) continue;
            sw += w;
            for (int q = 0; q < nf; q++) acc[q] += w * f[(int64_t)q * n + j];
        }
        wsum[g] = sw;
        for (int q = 0; q < nf; q++) out[(int64_t)q * MM + g] = sw > 0.0 ? acc[q] / sw : 0.0;
    }
}

/* The same sums over the particles of the 3 x 3 cells (side >= 3h) around the node's cell. */
void orc_grid_shepard_cells(int64_t n, const double *x, const double *y, int32_t nf, const double *f,
                            double L, double h, int32_t M, double *out, double *wsum)
{
    int nc = (int)floor(L / (3.0 * h));
    if (nc < 3) {   /* fewer than 3 cells: the stencil would visit a cell twice */
        orc_grid_shepard_brute(n, x, y, nf, f, L, h, M, out, wsum);
        return;
    }
    double cs = L / nc;
    int64_t ncell = (int64_t)nc * nc;
    int64_t *start = calloc((size_t)ncell + 1, sizeof(int64_t));
    int64_t *fill = calloc((size_t)ncell, sizeof(int64_t));
    int64_t *idx = malloc((size_t)(n > 0 ? n : 1) * sizeof(int64_t));
    int *key = malloc((size_t)(n > 0 ? n : 1) * sizeof(int));
    for (int64_t j = 0; j < n; j++) {
        int cx = (int)(x[j] / cs), cy = (int)(y[j] / cs);
        if (cx >= nc) cx = nc - 1;
        if (cy >= nc) cy = nc - 1;
        key[j] = cy * nc + cx;
        start[key[j] + 1]++;
    }
    for (int64_t c = 0; c < ncell; c++) start[c + 1] += start[c];
    for (int64_t j = 0; j < n; j++) idx[start[key[j]] + fill[key[j]]++] = j;
    int64_t MM = (int64_t)M * M;
#pragma omp parallel for schedule(static)
    for (int64_t g = 0; g < MM; g++) {
        double gx = (double)(g % M) * L / M, gy = (double)(g / M) * L / M;
        int cx = (int)(gx / cs), cy = (int)(gy / cs);
        if (cx >= nc) cx = nc - 1;
        if (cy >= nc) cy = nc - 1;
        double sw = 0.0, acc[16] = {0};
        for (int oy = -1; oy <= 1; oy++)
            for (int ox = -1; ox <= 1; ox++) {
                int c = ((cy + oy + nc) % nc) * nc + (cx + ox + nc) % nc;
                for (int64_t s = start[c]; s < start[c + 1]; s++) {
                    int64_t j = idx[s];
                    double w = node_weight(gx, gy, x[j], y[j], L, h);
                    if (w == 0.0) continue;
                    sw += w;
                    for (int q = 0; q < nf; q++) acc[q] += w * f[(int64_t)q * n + j];
                }
            }
        wsum[g] = sw;
        for (int q = 0; q < nf; q++) out[(int64_t)q * MM + g] = sw > 0.0 ? acc[q] / sw : 0.0;
    }
    free(start);
    free(fill);
    free(idx);
    free(key);
}

/* Selected nodes only (node index iy * M + ix), brute force: out[k * nf + q], wsum[k]. */
void orc_grid_nodes(int64_t n, const double *x, const double *y, int32_t nf, const double *f, double L,
                    double h, int32_t M, int64_t k, const int64_t *nodes, double *out, double *wsum)
{
#pragma omp parallel for schedule(static)
    for (int64_t t = 0; t < k; t++) {
        int64_t g = nodes[t];
        double gx = (double)(g % M) * L / M, gy = (double)(g / M) * L / M;
        double sw = 0.0, acc[16] = {0};
        for (int64_t j = 0; j < n; j++) {
            double w = node_weight(gx, gy, x[j], y[j], L, h);
            if (w == 0.0) continue;
            sw += w;
            for (int q = 0; q < nf; q++) acc[q] += w * f[(int64_t)q * n + j];
        }
        wsum[t] = sw;
        for (int q = 0; q < nf; q++) out[t * nf + q] = sw > 0.0 ? acc[q] / sw : 0.0;
    }
}

/* Signed crossing of the positive first axis by the edge a -> b (see the header). */
static int crossing(double a1, double a2, double b1, double b2)
{
    double cr = a1 * b2 - a2 * b1;
    if (a2 <= 0.0 && b2 > 0.0 && cr > 0.0) return 1;
    if (b2 <= 0.0 && a2 > 0.0 && cr < 0.0) return -1;
    return 0;
}

/* Winding number m of (q11, q12) around every plaquette of the periodic M x M grid (grids
 * row-major [iy * M + ix]); m_out[iy * M + ix] for the plaquette whose lower-left node is
 * (ix, iy).  counts[0] = plaquettes with m = +1 (+1/2 defects), counts[1] = m = -1 (-1/2),
 * counts[2] = |m| >= 2. */
void orc_defects(int32_t M, const double *q11, const double *q12, int8_t *m_out, int64_t *counts)
{
    counts[0] = counts[1] = counts[2] = 0;
    for (int iy = 0; iy < M; iy++)
        for (int ix = 0; ix < M; ix++) {
            int xp = (ix + 1) % M, yp = (iy + 1) % M;
            int64_t v[4] = {(int64_t)iy * M + ix, (int64_t)iy * M + xp, (int64_t)yp * M + xp,
                            (int64_t)yp * M + ix};
            int m = 0;
            for (int e = 0; e < 4; e++) {
                int64_t a = v[e], b = v[(e + 1) % 4];
                m += crossing(q11[a], q12[a], q11[b], q12[b]);
            }
            m_out[(int64_t)iy * M + ix] = (int8_t)m;
            if (m == 1) counts[0]++;
            else if (m == -1) counts[1]++;
            else if (m != 0) counts[2]++;
        }
}

/* W(b_k) of Eq. (18) for an array of b = r/h (the surrogate oracle's neighbour weights). */
void orc_W_array(int64_t n, const double *b, double h, double *out)
{
    for (int64_t k = 0; k < n; k++) out[k] = orc_W(b[k], h);
}

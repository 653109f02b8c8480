/*
 * FP64 CPU oracle for the SPH active-nematic time step of Saghatchi, Kolukisa and Yildiz,
 * "Development of Smoothed Particle Hydrodynamics Method for Modeling Active Nematics"
 * (arXiv 2108.08919).
 *
 * TEST INFRASTRUCTURE ONLY.  This file is the plain, slow reference that the CUDA path is checked
 * against.  Only the test suite, the smoke check and the benchmark's CPU-baseline leg may load it.
 * It shares no code, header, table or constant with the CUDA library: every formula below is
 * written from the paper's equations (cited per function) in the paper's order and notation.
 *
 * Conventions (the paper's equations are numbered in order of appearance):
 *   Eq. (1)  nematodynamic equation          Eq. (2)  co-rotation term S
 *   Eq. (7)  molecular field H               Eq. (18) quintic kernel
 *   Eq. (19) SPH sum and particle volume     Eq. (20) corrected first derivative
 *   Eq. (21) corrected Laplacian             Eq. (22) correction tensor alpha
 *   Eq. (23) SPH momentum                    Eq. (24) SPH Q rate
 *   Eq. (25) SPH continuity                  Eq. (26) equation of state
 *   Eq. (27) time-integration derivatives    Eq. (28) density filter
 *   Eq. (29) artificial particle displacement Eq. (30) periodic boundary conditions
 *
 *   d_ij = r_i - r_j (minimum image), r = |d_ij|, b = r/h, support 3h.
 *   dW_ij/dx_i^l = W'(b) / h * d_ij^l / r.
 *   Tensor index order: D[s][k] = d f^s / d x^k.
 *
 * Readings of ambiguous passages (all selectable where the paper admits two readings):
 *   - neighbour set N(i) = { j != i : |d_ij|^2 < (3h)^2 }, decided in FP64 with no fused
 *     multiply-add (the file is compiled with -ffp-contract=off);
 *   - sums that define V, the Shepard filter and u_v include the self term j = i;
 *     gradient, Laplacian, momentum and APD sums exclude it (their r = 0 term is undefined);
 *   - Laplacian (Eq. 21, whose indices are garbled): the scalar corrected form
 *     lap f_i = 2 sum_j V_j (f_i - f_j) (d_ij . B_i grad_i W_ij) / r^2, applied per tensor
 *     component (the factor 8/(d+2) = 2 in two dimensions);
 *   - velocity gradient W_ab = d u_a / d x_b, E = (W + W^T)/2, Omega = (W - W^T)/2;
 *   - S uses M = Q + c I with c = c_shift (1/3 as printed in Eq. 2, or 1/2);
 *   - m = S + Gamma H is projected onto the symmetric traceless subspace before Q is advanced;
 *   - H keeps both the C and the K terms (Eq. 7 drops C's coefficient, Eq. 24 drops K);
 *   - the Q term of Eq. (23) is multiplied by -zeta / rho_i (active stress -zeta Q, Eq. 13);
 *   - momentum uses Q^{n+1} (text order of §3.1) unless q_new_in_momentum = 0;
 *   - corrector u^{n+1} = u^{n+1/2} + dt/2 a^{n+1/2}; rho^{n+1} = rho_hat + dt/2 k^{n+1/2};
 *   - c0 = max(10 max|u^{n+1/2}|, c0_min);
 *   - APD uses the midpoint pair data and u^{n+1/2}; r0 averages over the N_i neighbours;
 *   - elastic stress (Eq. 12, off by default as in the paper): Pi_el = 2 lambda M (Q:H)
 *     - lambda (H M + M H), M = Q + c I, from Q^n and the H of the Q rate; it enters the momentum
 *     through the corrected divergence (paper mode) or the pair-antisymmetric form.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#ifdef _OPENMP
#include <omp.h>
#endif

#ifndef M_PI
#define M_PI 3.14159265358979323846
#endif

/* ------------------------------------------------------------------------------------------ */
/* Parameters                                                                                  */
/* ------------------------------------------------------------------------------------------ */

typedef struct {
    double L;          /* periodic box side */
    double h;          /* smoothing length */
    double dt;         /* time step */
    double rho0;       /* reference density */
    double eta;        /* dynamic viscosity mu; nu = eta / rho0 */
    double Gamma;      /* rotational diffusivity */
    double lambda;     /* tumbling / flow-alignment parameter */
    double A, B, C;    /* Landau-de Gennes coefficients */
    double K;          /* elastic constant */
    double zeta;       /* activity (> 0 extensile) */
    double gamma_eos;  /* EoS exponent (7) */
    double beta;       /* density filter coefficient (1 = Shepard) */
    double c0_min;     /* floor of the sound speed */
    double c_shift;    /* c in M = Q + c I */
    int32_t apd;               /* 1: apply artificial particle displacement */
    int32_t conservative;      /* 1: pair-antisymmetric momentum with fixed masses */
    int32_t q_new_in_momentum; /* 1: Q^{n+1} in the active force, 0: Q^n */
    int32_t nbr_mode;          /* 0 brute force, 1 ghost layer, 2 cell grid */
    int32_t elastic;           /* 1: add the elastic stress of Eq. (12) */
} orc_params;

/* Intermediates of the last step (each pointer may be NULL). */
typedef struct {
    double *sumW, *V;
    double *B11, *B12, *B22;
    double *gradu;          /* 4 per particle: du_x/dx, du_x/dy, du_y/dx, du_y/dy */
    double *lapQ11, *lapQ12;
    double *k, *rho_half, *rho_hat, *p;
    double *divQx, *divQy;
    double *ax, *ay;
    double *apdx, *apdy;
    double *trace_m;        /* trace of m = S + Gamma H before projection */
    double *qrate11, *qrate12;  /* the projected Q rate m of Eq. (24) (dQ/dt of the step) */
    int32_t *nnbr;
    double *c0;             /* scalar */
} orc_record;

/* ------------------------------------------------------------------------------------------ */
/* Quintic kernel, §3 Eq. (18)                                                                 */
/* ------------------------------------------------------------------------------------------ */

static double p4(double t) { return t * t * t * t; }
static double p5(double t) { return t * t * t * t * t; }

/* 2D normalisation a_d = 7 / (478 pi h^2) (§3, text under Eq. 18). */
double orc_kernel_ad(double h) { return 7.0 / (478.0 * M_PI * h * h); }

/* W(b) for b = r/h, piecewise on [0,1], [1,2], [2,3], zero beyond 3. */
double orc_W(double b, double h)
{
    double ad = orc_kernel_ad(h);
    if (b < 0.0) return NAN;
    if (b <= 1.0) return ad * (p5(3.0 - b) - 6.0 * p5(2.0 - b) + 15.0 * p5(1.0 - b));
    if (b <= 2.0) return ad * (p5(3.0 - b) - 6.0 * p5(2.0 - b));
    if (b <= 3.0) return ad * p5(3.0 - b);
    return 0.0;
}

/* dW/db, the derivative of each piece of Eq. (18). */
double orc_dWdb(double b, double h)
{
    double ad = orc_kernel_ad(h);
    if (b < 0.0) return NAN;
    if (b <= 1.0) return ad * (-5.0 * p4(3.0 - b) + 30.0 * p4(2.0 - b) - 75.0 * p4(1.0 - b));
    if (b <= 2.0) return ad * (-5.0 * p4(3.0 - b) + 30.0 * p4(2.0 - b));
    if (b <= 3.0) return ad * (-5.0 * p4(3.0 - b));
    return 0.0;
}

/* ------------------------------------------------------------------------------------------ */
/* Periodic geometry, §3.1 Eq. (30)                                                            */
/* ------------------------------------------------------------------------------------------ */

/* Minimum-image component of r_i - r_j; both coordinates lie in [0, L). */
static double min_image(double a, double b, double L)
{
    double d = a - b;
    if (d > 0.5 * L) d = d - L;
    else if (d < -0.5 * L) d = d + L;
    return d;
}

/* Re-insert a coordinate that left [0, L) by +-L. */
static double wrap(double a, double L)
{
    if (a < 0.0) a = a + L;
    if (a >= L) a = a - L;
    return a;
}

/* ------------------------------------------------------------------------------------------ */
/* Neighbour search                                                                            */
/* ------------------------------------------------------------------------------------------ */

static int in_support(double dx, double dy, double R2)
{
    double r2 = dx * dx + dy * dy;
    return r2 < R2;
}

static double support_R2(double h) { return (3.0 * h) * (3.0 * h); }

/* Definition: all j != i within the support, minimum image, O(N^2).
 * Two calls: with cols == NULL only rowptr is filled (counts), else cols too.  Rows are in
 * ascending j.  Returns the total pair count. */
int64_t orc_neighbors_brute(int64_t n, const double *x, const double *y, double L, double h,
                            int64_t *rowptr, int32_t *cols)
{
    double R2 = support_R2(h);
    if (cols == NULL) {
        #pragma omp parallel for schedule(dynamic, 64)
        for (int64_t i = 0; i < n; i++) {
            int64_t c = 0;
            for (int64_t j = 0; j < n; j++) {
                if (j == i) continue;
                if (in_support(min_image(x[i], x[j], L), min_image(y[i], y[j], L), R2)) c++;
            }
            rowptr[i + 1] = c;
        }
        rowptr[0] = 0;
        for (int64_t i = 0; i < n; i++) rowptr[i + 1] += rowptr[i];
        return rowptr[n];
    }
    #pragma omp parallel for schedule(dynamic, 64)
    for (int64_t i = 0; i < n; i++) {
        int64_t c = rowptr[i];
        for (int64_t j = 0; j < n; j++) {
            if (j == i) continue;
            if (in_support(min_image(x[i], x[j], L), min_image(y[i], y[j], L), R2))
                cols[c++] = (int32_t)j;
        }
    }
    return rowptr[n];
}

/* The paper's periodic treatment taken literally (§3.1, Eq. 30 and the ghost-particle figure):
 * every particle within 3h of a face is copied and displaced by +-L across it (corner copies
 * included); fluid particles then search fluid and ghost particles with plain differences.
 * A ghost reports its source ID.  Same two-call protocol as orc_neighbors_brute. */
int64_t orc_neighbors_ghost(int64_t n, const double *x, const double *y, double L, double h,
                            int64_t *rowptr, int32_t *cols)
{
    double R = 3.0 * h, R2 = support_R2(h);
    int64_t cap = 9 * n + 1, ng = 0;
    double *gx = (double *)malloc(sizeof(double) * (size_t)cap);
    double *gy = (double *)malloc(sizeof(double) * (size_t)cap);
    int32_t *gs = (int32_t *)malloc(sizeof(int32_t) * (size_t)cap);
    if (!gx || !gy || !gs) { free(gx); free(gy); free(gs); return -1; }
    for (int64_t j = 0; j < n; j++) {
        gx[ng] = x[j]; gy[ng] = y[j]; gs[ng] = (int32_t)j; ng++;       /* the fluid particle */
        for (int sx = -1; sx <= 1; sx++) {
            for (int sy = -1; sy <= 1; sy++) {
                if (sx == 0 && sy == 0) continue;
                if (sx == 1 && !(x[j] < R)) continue;        /* near x = 0: copy to x + L */
                if (sx == -1 && !(x[j] >= L - R)) continue;  /* near x = L: copy to x - L */
                if (sy == 1 && !(y[j] < R)) continue;
                if (sy == -1 && !(y[j] >= L - R)) continue;
                gx[ng] = x[j] + sx * L; gy[ng] = y[j] + sy * L; gs[ng] = (int32_t)j; ng++;
            }
        }
    }
    int fill = cols != NULL;
    if (!fill) rowptr[0] = 0;
    #pragma omp parallel for schedule(dynamic, 64)
    for (int64_t i = 0; i < n; i++) {
        int64_t c = fill ? rowptr[i] : 0;
        int64_t start = c;
        for (int64_t g = 0; g < ng; g++) {
            if (gs[g] == i) continue;
            if (in_support(x[i] - gx[g], y[i] - gy[g], R2)) {
                if (fill) cols[c] = gs[g];
                c++;
            }
        }
        if (fill) {
            /* ascending source ID */
            for (int64_t a = start + 1; a < c; a++) {
                int32_t v = cols[a];
                int64_t b = a - 1;
                while (b >= start && cols[b] > v) { cols[b + 1] = cols[b]; b--; }
                cols[b + 1] = v;
            }
        } else {
            rowptr[i + 1] = c;
        }
    }
    if (!fill)
        for (int64_t i = 0; i < n; i++) rowptr[i + 1] += rowptr[i];
    free(gx); free(gy); free(gs);
    return rowptr[n];
}

/* The paper's search structure (§4): square cells of side >= 3h, particles binned per cell, each
 * particle scanning the 3x3 block of cells around its own (periodic).  Candidates are accepted
 * with the same minimum-image test as the brute-force definition.  Falls back to brute force when
 * fewer than 3 cells fit across the box. */
int64_t orc_neighbors_cells(int64_t n, const double *x, const double *y, double L, double h,
                            int64_t *rowptr, int32_t *cols)
{
    double R2 = support_R2(h);
    int64_t nc = (int64_t)floor(L / (3.0 * h));
    if (nc < 3) return orc_neighbors_brute(n, x, y, L, h, rowptr, cols);
    int64_t ncell = nc * nc;
    int64_t *head = (int64_t *)calloc((size_t)(ncell + 1), sizeof(int64_t));
    int64_t *cellof = (int64_t *)malloc(sizeof(int64_t) * (size_t)(n > 0 ? n : 1));
    int64_t *members = (int64_t *)malloc(sizeof(int64_t) * (size_t)(n > 0 ? n : 1));
    int64_t *fillp = (int64_t *)malloc(sizeof(int64_t) * (size_t)(ncell + 1));
    if (!head || !cellof || !members || !fillp) {
        free(head); free(cellof); free(members); free(fillp);
        return -1;
    }
    for (int64_t i = 0; i < n; i++) {
        int64_t cx = (int64_t)(x[i] / L * (double)nc);
        int64_t cy = (int64_t)(y[i] / L * (double)nc);
        if (cx > nc - 1) cx = nc - 1;
        if (cy > nc - 1) cy = nc - 1;
        if (cx < 0) cx = 0;
        if (cy < 0) cy = 0;
        cellof[i] = cy * nc + cx;
        head[cellof[i] + 1]++;
    }
    for (int64_t c = 0; c < ncell; c++) head[c + 1] += head[c];
    memcpy(fillp, head, sizeof(int64_t) * (size_t)(ncell + 1));
    for (int64_t i = 0; i < n; i++) members[fillp[cellof[i]]++] = i;

    int fill = cols != NULL;
    if (!fill) rowptr[0] = 0;
    #pragma omp parallel for schedule(dynamic, 256)
    for (int64_t i = 0; i < n; i++) {
        int64_t cx = cellof[i] % nc, cy = cellof[i] / nc;
        int64_t c = fill ? rowptr[i] : 0, start = c;
        for (int64_t oy = -1; oy <= 1; oy++) {
            for (int64_t ox = -1; ox <= 1; ox++) {
                int64_t qx = (cx + ox + nc) % nc, qy = (cy + oy + nc) % nc;
                int64_t q = qy * nc + qx;
                for (int64_t m = head[q]; m < head[q + 1]; m++) {
                    int64_t j = members[m];
                    if (j == i) continue;
                    if (in_support(min_image(x[i], x[j], L), min_image(y[i], y[j], L), R2)) {
                        if (fill) cols[c] = (int32_t)j;
                        c++;
                    }
                }
            }
        }
        if (fill) {
            for (int64_t a = start + 1; a < c; a++) {
                int32_t v = cols[a];
                int64_t b = a - 1;
                while (b >= start && cols[b] > v) { cols[b + 1] = cols[b]; b--; }
                cols[b + 1] = v;
            }
        } else {
            rowptr[i + 1] = c;
        }
    }
    if (!fill)
        for (int64_t i = 0; i < n; i++) rowptr[i + 1] += rowptr[i];
    free(head); free(cellof); free(members); free(fillp);
    return rowptr[n];
}

static int64_t search(int mode, int64_t n, const double *x, const double *y, double L, double h,
                      int64_t *rowptr, int32_t *cols)
{
    if (mode == 1) return orc_neighbors_ghost(n, x, y, L, h, rowptr, cols);
    if (mode == 2) return orc_neighbors_cells(n, x, y, L, h, rowptr, cols);
    return orc_neighbors_brute(n, x, y, L, h, rowptr, cols);
}

/* ------------------------------------------------------------------------------------------ */
/* Pair geometry                                                                               */
/* ------------------------------------------------------------------------------------------ */

typedef struct {
    double dx, dy;    /* d_ij = r_i - r_j */
    double r;         /* |d_ij| */
    double W;         /* W_ij */
    double gx, gy;    /* grad_i W_ij */
} pair_t;

static pair_t pair_of(const double *x, const double *y, int64_t i, int64_t j, double L, double h)
{
    pair_t p;
    p.dx = min_image(x[i], x[j], L);
    p.dy = min_image(y[i], y[j], L);
    p.r = sqrt(p.dx * p.dx + p.dy * p.dy);
    double b = p.r / h;
    p.W = orc_W(b, h);
    double dWdb = orc_dWdb(b, h);
    p.gx = dWdb / h * p.dx / p.r;
    p.gy = dWdb / h * p.dy / p.r;
    return p;
}

/* ------------------------------------------------------------------------------------------ */
/* SPH operators (§3), one function per equation                                                */
/* ------------------------------------------------------------------------------------------ */

/* Eq. (19): V_i = 1 / sum_j W_ij, the sum including j = i (W(0)). */
void orc_volumes(int64_t n, const double *x, const double *y, double L, double h,
                 const int64_t *rowptr, const int32_t *cols, double *sumW, double *V)
{
    #pragma omp parallel for schedule(static)
    for (int64_t i = 0; i < n; i++) {
        double s = orc_W(0.0, h);
        for (int64_t e = rowptr[i]; e < rowptr[i + 1]; e++) s += pair_of(x, y, i, cols[e], L, h).W;
        if (sumW) sumW[i] = s;
        V[i] = 1.0 / s;
    }
}

/* Eq. (22): alpha_i^{sl} = sum_j r_ji^s V_j dW_ij/dx_i^l; B_i = alpha_i^{-1} (text under Eq. 23).
 * B is returned as its three independent entries (alpha is symmetric for a radial kernel; the
 * inverse is formed from the full matrix). Returns the number of particles with det(alpha) <= 0. */
int64_t orc_correction(int64_t n, const double *x, const double *y, double L, double h,
                       const int64_t *rowptr, const int32_t *cols, const double *V,
                       double *B11, double *B12, double *B22)
{
    int64_t bad = 0;
    #pragma omp parallel for schedule(static) reduction(+ : bad)
    for (int64_t i = 0; i < n; i++) {
        double a[2][2] = {{0.0, 0.0}, {0.0, 0.0}};
        for (int64_t e = rowptr[i]; e < rowptr[i + 1]; e++) {
            int64_t j = cols[e];
            pair_t p = pair_of(x, y, i, j, L, h);
            double rji[2] = {-p.dx, -p.dy};
            double g[2] = {p.gx, p.gy};
            for (int s = 0; s < 2; s++)
                for (int l = 0; l < 2; l++) a[s][l] += rji[s] * V[j] * g[l];
        }
        double det = a[0][0] * a[1][1] - a[0][1] * a[1][0];
        if (!(det > 0.0)) bad++;
        B11[i] = a[1][1] / det;
        B12[i] = -a[0][1] / det;   /* (B)_{01}; (B)_{10} = -a[1][0]/det equals it for symmetric alpha */
        B22[i] = a[0][0] / det;
    }
    return bad;
}

/* Eq. (20): corrected gradient of a scalar field f: (df/dx^k) alpha^{kl} = sum_j V_j (f_j - f_i)
 * dW_ij/dx_i^l, solved with B = alpha^{-1}.  out[2*i + k] = df/dx^k at particle i. */
void orc_gradient(int64_t n, const double *x, const double *y, double L, double h,
                  const int64_t *rowptr, const int32_t *cols, const double *V,
                  const double *B11, const double *B12, const double *B22,
                  const double *f, double *out)
{
    #pragma omp parallel for schedule(static)
    for (int64_t i = 0; i < n; i++) {
        double rhs[2] = {0.0, 0.0};
        for (int64_t e = rowptr[i]; e < rowptr[i + 1]; e++) {
            int64_t j = cols[e];
            pair_t p = pair_of(x, y, i, j, L, h);
            rhs[0] += V[j] * (f[j] - f[i]) * p.gx;
            rhs[1] += V[j] * (f[j] - f[i]) * p.gy;
        }
        double B[2][2] = {{B11[i], B12[i]}, {B12[i], B22[i]}};
        for (int k = 0; k < 2; k++) out[2 * i + k] = rhs[0] * B[0][k] + rhs[1] * B[1][k];
    }
}

/* Eq. (21) read as the scalar corrected Laplacian:
 * lap f_i = 2 sum_j V_j (f_i - f_j) (d_ij . B_i grad_i W_ij) / |d_ij|^2. */
void orc_laplacian(int64_t n, const double *x, const double *y, double L, double h,
                   const int64_t *rowptr, const int32_t *cols, const double *V,
                   const double *B11, const double *B12, const double *B22,
                   const double *f, double *out)
{
    #pragma omp parallel for schedule(static)
    for (int64_t i = 0; i < n; i++) {
        double B[2][2] = {{B11[i], B12[i]}, {B12[i], B22[i]}};
        double s = 0.0;
        for (int64_t e = rowptr[i]; e < rowptr[i + 1]; e++) {
            int64_t j = cols[e];
            pair_t p = pair_of(x, y, i, j, L, h);
            double Bg[2] = {B[0][0] * p.gx + B[0][1] * p.gy, B[1][0] * p.gx + B[1][1] * p.gy};
            double dBg = p.dx * Bg[0] + p.dy * Bg[1];
            s += V[j] * (f[i] - f[j]) * dBg / (p.r * p.r);
        }
        out[i] = 2.0 * s;
    }
}

/* Eq. (28): rho_hat_i = rho_i - beta sum_j (rho_i - rho_j) W_ij / sum_j W_ij, sums over N(i) and
 * the particle itself. */
void orc_density_filter(int64_t n, const double *x, const double *y, double L, double h,
                        const int64_t *rowptr, const int32_t *cols, double beta,
                        const double *rho, double *rho_hat)
{
    #pragma omp parallel for schedule(static)
    for (int64_t i = 0; i < n; i++) {
        double W0 = orc_W(0.0, h);
        double num = (rho[i] - rho[i]) * W0, den = W0;
        for (int64_t e = rowptr[i]; e < rowptr[i + 1]; e++) {
            int64_t j = cols[e];
            pair_t p = pair_of(x, y, i, j, L, h);
            num += (rho[i] - rho[j]) * p.W;
            den += p.W;
        }
        rho_hat[i] = rho[i] - beta * num / den;
    }
}

/* Eq. (26): p = rho0 c0^2 / gamma [ (rho/rho0)^gamma - 1 ]. */
double orc_eos(double rho, double rho0, double c0, double gamma_eos)
{
    return rho0 * c0 * c0 / gamma_eos * (pow(rho / rho0, gamma_eos) - 1.0);
}

/* Eq. (25): k_i = rho_i sum_j V_j (u_i - u_j) . (B_i grad_i W_ij). */
void orc_continuity(int64_t n, const double *x, const double *y, double L, double h,
                    const int64_t *rowptr, const int32_t *cols, const double *V,
                    const double *B11, const double *B12, const double *B22,
                    const double *ux, const double *uy, const double *rho, double *k)
{
    #pragma omp parallel for schedule(static)
    for (int64_t i = 0; i < n; i++) {
        double B[2][2] = {{B11[i], B12[i]}, {B12[i], B22[i]}};
        double s = 0.0;
        for (int64_t e = rowptr[i]; e < rowptr[i + 1]; e++) {
            int64_t j = cols[e];
            pair_t p = pair_of(x, y, i, j, L, h);
            double Bg[2] = {B[0][0] * p.gx + B[0][1] * p.gy, B[1][0] * p.gx + B[1][1] * p.gy};
            s += V[j] * ((ux[i] - ux[j]) * Bg[0] + (uy[i] - uy[j]) * Bg[1]);
        }
        k[i] = rho[i] * s;
    }
}

/* Q as a full 2x2 tensor from its two independent entries (symmetric, traceless). */
static void q_tensor(double q11, double q12, double Q[2][2])
{
    Q[0][0] = q11; Q[0][1] = q12; Q[1][0] = q12; Q[1][1] = -q11;
}

static void mat_mul(const double A[2][2], const double B[2][2], double Cm[2][2])
{
    for (int a = 0; a < 2; a++)
        for (int b = 0; b < 2; b++) Cm[a][b] = A[a][0] * B[0][b] + A[a][1] * B[1][b];
}

/* Eq. (24) with Eqs. (2) and (7): the Q rate m for one particle.
 *   D     : velocity gradient, D[a][b] = du_a/dx_b (corrected, Eq. 20)
 *   lapQ  : corrected Laplacian of each entry of Q (Eq. 21)
 * Writes the projected rate (m11, m12) and the trace of the unprojected m. */
void orc_q_rate(const orc_params *P, double q11, double q12, const double D[2][2],
                const double lapQ[2][2], double *m11, double *m12, double *trace_m, double Hout[2][2])
{
    double Q[2][2], I[2][2] = {{1.0, 0.0}, {0.0, 1.0}};
    q_tensor(q11, q12, Q);
    double E[2][2], Om[2][2], M[2][2];
    for (int a = 0; a < 2; a++)
        for (int b = 0; b < 2; b++) {
            E[a][b] = 0.5 * (D[a][b] + D[b][a]);
            Om[a][b] = 0.5 * (D[a][b] - D[b][a]);
            M[a][b] = Q[a][b] + P->c_shift * I[a][b];
        }
    double QddD = 0.0;                                   /* Q : grad u */
    for (int a = 0; a < 2; a++)
        for (int b = 0; b < 2; b++) QddD += Q[a][b] * D[a][b];
    double L1[2][2], L2[2][2], T1[2][2], T2[2][2];
    for (int a = 0; a < 2; a++)
        for (int b = 0; b < 2; b++) {
            L1[a][b] = P->lambda * E[a][b] + Om[a][b];
            L2[a][b] = P->lambda * E[a][b] - Om[a][b];
        }
    mat_mul(L1, M, T1);
    mat_mul(M, L2, T2);
    double S[2][2];
    for (int a = 0; a < 2; a++)
        for (int b = 0; b < 2; b++) S[a][b] = T1[a][b] + T2[a][b] - 2.0 * P->lambda * M[a][b] * QddD;

    double Q2[2][2];
    mat_mul(Q, Q, Q2);
    double trQ2 = Q2[0][0] + Q2[1][1];
    double H[2][2];
    for (int a = 0; a < 2; a++)
        for (int b = 0; b < 2; b++)
            H[a][b] = -P->A * Q[a][b] + P->B * (Q2[a][b] - I[a][b] / 3.0 * trQ2)
                      - P->C * Q[a][b] * trQ2 + P->K * lapQ[a][b];

    if (Hout)
        for (int a = 0; a < 2; a++)
            for (int b = 0; b < 2; b++) Hout[a][b] = H[a][b];
    double m[2][2];
    for (int a = 0; a < 2; a++)
        for (int b = 0; b < 2; b++) m[a][b] = S[a][b] + P->Gamma * H[a][b];
    double tr = m[0][0] + m[1][1];
    if (trace_m) *trace_m = tr;
    /* symmetric traceless part */
    double ms[2][2];
    for (int a = 0; a < 2; a++)
        for (int b = 0; b < 2; b++) ms[a][b] = 0.5 * (m[a][b] + m[b][a]) - 0.5 * tr * I[a][b];
    *m11 = ms[0][0];
    *m12 = ms[0][1];
}

/* Eq. (12) without its -p I (the pressure enters separately):
 * Pi_el = 2 lambda M (Q:H) - lambda H M - lambda M H with M = Q + c I. */
void orc_elastic_stress(const orc_params *P, double q11, double q12, const double H[2][2],
                        double Pi[2][2])
{
    double Q[2][2], M[2][2], HM[2][2], MH[2][2];
    q_tensor(q11, q12, Q);
    for (int a = 0; a < 2; a++)
        for (int b = 0; b < 2; b++) M[a][b] = Q[a][b] + (a == b ? P->c_shift : 0.0);
    double QH = 0.0;
    for (int a = 0; a < 2; a++)
        for (int b = 0; b < 2; b++) QH += Q[a][b] * H[a][b];
    mat_mul(H, M, HM);
    mat_mul(M, H, MH);
    for (int a = 0; a < 2; a++)
        for (int b = 0; b < 2; b++)
            Pi[a][b] = 2.0 * P->lambda * M[a][b] * QH - P->lambda * HM[a][b] - P->lambda * MH[a][b];
}

/* The active-force sum of Eq. (23): sum_j V_j (Q_j - Q_i) (B_i grad_i W_ij), a vector. */
static void active_sum(int64_t i, const double *x, const double *y, double L, double h,
                       const int64_t *rowptr, const int32_t *cols, const double *V,
                       const double B[2][2], const double *q11, const double *q12, double out[2])
{
    double Qi[2][2];
    q_tensor(q11[i], q12[i], Qi);
    out[0] = out[1] = 0.0;
    for (int64_t e = rowptr[i]; e < rowptr[i + 1]; e++) {
        int64_t j = cols[e];
        pair_t p = pair_of(x, y, i, j, L, h);
        double Qj[2][2];
        q_tensor(q11[j], q12[j], Qj);
        double Bg[2] = {B[0][0] * p.gx + B[0][1] * p.gy, B[1][0] * p.gx + B[1][1] * p.gy};
        for (int a = 0; a < 2; a++)
            out[a] += V[j] * ((Qj[a][0] - Qi[a][0]) * Bg[0] + (Qj[a][1] - Qi[a][1]) * Bg[1]);
    }
}

/* Eq. (23), the corrected momentum equation, with the Q term scaled by -zeta/rho_i. */
void orc_momentum_paper(const orc_params *P, int64_t n, const double *x, const double *y,
                        const int64_t *rowptr, const int32_t *cols, const double *V,
                        const double *B11, const double *B12, const double *B22,
                        const double *rho, const double *p, const double *ux, const double *uy,
                        const double *q11, const double *q12,
                        double *ax, double *ay, double *divQx, double *divQy, const double *pel)
{
    double L = P->L, h = P->h, nu = P->eta / P->rho0;
    #pragma omp parallel for schedule(static)
    for (int64_t i = 0; i < n; i++) {
        double B[2][2] = {{B11[i], B12[i]}, {B12[i], B22[i]}};
        double fp[2] = {0.0, 0.0}, fv[2] = {0.0, 0.0};
        for (int64_t e = rowptr[i]; e < rowptr[i + 1]; e++) {
            int64_t j = cols[e];
            pair_t pr = pair_of(x, y, i, j, L, h);
            double Bg[2] = {B[0][0] * pr.gx + B[0][1] * pr.gy, B[1][0] * pr.gx + B[1][1] * pr.gy};
            double cp = p[i] / (rho[i] * rho[i]) + p[j] / (rho[j] * rho[j]);
            double uijd = (ux[i] - ux[j]) * pr.dx + (uy[i] - uy[j]) * pr.dy;
            double r2 = pr.r * pr.r;
            for (int a = 0; a < 2; a++) {
                fp[a] += V[j] * cp * Bg[a];
                fv[a] += V[j] * uijd / r2 * Bg[a];
            }
        }
        double dq[2];
        active_sum(i, x, y, L, h, rowptr, cols, V, B, q11, q12, dq);
        double del[2] = {0.0, 0.0};   /* sum_j V_j (Pi_j - Pi_i) . (B_i grad_i W_ij): div Pi_el */
        if (P->elastic && pel) {
            for (int64_t e = rowptr[i]; e < rowptr[i + 1]; e++) {
                int64_t j = cols[e];
                pair_t pr = pair_of(x, y, i, j, L, h);
                double Bg[2] = {B[0][0] * pr.gx + B[0][1] * pr.gy, B[1][0] * pr.gx + B[1][1] * pr.gy};
                double Pj[2][2] = {{pel[3 * j], pel[3 * j + 1]}, {pel[3 * j + 1], pel[3 * j + 2]}};
                double Pi[2][2] = {{pel[3 * i], pel[3 * i + 1]}, {pel[3 * i + 1], pel[3 * i + 2]}};
                for (int a = 0; a < 2; a++)
                    del[a] += V[j] * ((Pj[a][0] - Pi[a][0]) * Bg[0] + (Pj[a][1] - Pi[a][1]) * Bg[1]);
            }
        }
        double a_[2];
        for (int a = 0; a < 2; a++)
            a_[a] = -rho[i] * fp[a] + 8.0 * nu * P->rho0 / rho[i] * fv[a] - P->zeta / rho[i] * dq[a]
                    + del[a] / rho[i];
        ax[i] = a_[0];
        ay[i] = a_[1];
        if (divQx) divQx[i] = dq[0];
        if (divQy) divQy[i] = dq[1];
    }
}

/* Pair-antisymmetric momentum with fixed particle masses m = rho0 L^2 / N and no correction
 * tensor: each pair term changes sign under i <-> j, so sum_i m_i a_i = 0 up to rounding.
 *   a_i = - sum_j m (p_i/rho_i^2 + p_j/rho_j^2) grad_i W
 *         + sum_j m 8 mu / (rho_i rho_j) (u_ij . d_ij) / r^2 grad_i W
 *         - zeta sum_j m (Q_i/rho_i^2 + Q_j/rho_j^2) . grad_i W */
void orc_momentum_conservative(const orc_params *P, int64_t n, const double *x, const double *y,
                               const int64_t *rowptr, const int32_t *cols, const double *rho,
                               const double *p, const double *ux, const double *uy,
                               const double *q11, const double *q12, double *ax, double *ay,
                               const double *pel)
{
    double L = P->L, h = P->h, mass = P->rho0 * P->L * P->L / (double)n, mu = P->eta;
    #pragma omp parallel for schedule(static)
    for (int64_t i = 0; i < n; i++) {
        double Qi[2][2];
        q_tensor(q11[i], q12[i], Qi);
        double a_[2] = {0.0, 0.0};
        for (int64_t e = rowptr[i]; e < rowptr[i + 1]; e++) {
            int64_t j = cols[e];
            pair_t pr = pair_of(x, y, i, j, L, h);
            double g[2] = {pr.gx, pr.gy};
            double Qj[2][2];
            q_tensor(q11[j], q12[j], Qj);
            double cp = p[i] / (rho[i] * rho[i]) + p[j] / (rho[j] * rho[j]);
            double uijd = (ux[i] - ux[j]) * pr.dx + (uy[i] - uy[j]) * pr.dy;
            double r2 = pr.r * pr.r;
            for (int a = 0; a < 2; a++) {
                double act = 0.0;
                for (int b = 0; b < 2; b++)
                    act += (Qi[a][b] / (rho[i] * rho[i]) + Qj[a][b] / (rho[j] * rho[j])) * g[b];
                double el = 0.0;   /* + sum_j m (Pi_i/rho_i^2 + Pi_j/rho_j^2) . grad_i W */
                if (P->elastic && pel) {
                    double Pi_[2][2] = {{pel[3 * i], pel[3 * i + 1]}, {pel[3 * i + 1], pel[3 * i + 2]}};
                    double Pj_[2][2] = {{pel[3 * j], pel[3 * j + 1]}, {pel[3 * j + 1], pel[3 * j + 2]}};
                    for (int b = 0; b < 2; b++)
                        el += (Pi_[a][b] / (rho[i] * rho[i]) + Pj_[a][b] / (rho[j] * rho[j])) * g[b];
                }
                a_[a] += -mass * cp * g[a] + mass * 8.0 * mu / (rho[i] * rho[j]) * uijd / r2 * g[a]
                         - P->zeta * mass * act + mass * el;
            }
        }
        ax[i] = a_[0];
        ay[i] = a_[1];
    }
}

/* Eq. (29): delta r_i = sum_j d_ij / r^3 r0^2 u_v dt with
 * u_v = |sum_j (u_i - u_j) W_ij| / sum_j W_ij (self term included) and r0 = sum_j r_ij / N_i. */
void orc_apd(int64_t n, const double *x, const double *y, double L, double h, double dt,
             const int64_t *rowptr, const int32_t *cols, const double *ux, const double *uy,
             double *dxo, double *dyo)
{
    #pragma omp parallel for schedule(static)
    for (int64_t i = 0; i < n; i++) {
        double W0 = orc_W(0.0, h);
        double su[2] = {0.0, 0.0}, sw = W0, sr = 0.0, sd[2] = {0.0, 0.0};
        int64_t N = rowptr[i + 1] - rowptr[i];
        for (int64_t e = rowptr[i]; e < rowptr[i + 1]; e++) {
            int64_t j = cols[e];
            pair_t p = pair_of(x, y, i, j, L, h);
            su[0] += (ux[i] - ux[j]) * p.W;
            su[1] += (uy[i] - uy[j]) * p.W;
            sw += p.W;
            sr += p.r;
            double r3 = p.r * p.r * p.r;
            sd[0] += p.dx / r3;
            sd[1] += p.dy / r3;
        }
        double uv = sqrt(su[0] * su[0] + su[1] * su[1]) / sw;
        double r0 = N > 0 ? sr / (double)N : 0.0;
        dxo[i] = sd[0] * r0 * r0 * uv * dt;
        dyo[i] = sd[1] * r0 * r0 * uv * dt;
    }
}

/* ------------------------------------------------------------------------------------------ */
/* One time step, §3.1: modified-Euler predictor-corrector                                     */
/* ------------------------------------------------------------------------------------------ */

static void *xalloc(size_t bytes) { return malloc(bytes > 0 ? bytes : 1); }

/* Advances the state (arrays of length n, updated in place) by nsteps steps.
 * rho is the density (not its deviation); ax, ay carry a^n between steps (a^0 = 0).
 * rec (nullable) receives the intermediates of the last step.
 * Returns 0, or -1 on allocation failure, -2 if some alpha was singular. */
int orc_step(const orc_params *P, int64_t n, double *x, double *y, double *ux, double *uy,
             double *q11, double *q12, double *rho, double *ax, double *ay, int64_t nsteps,
             orc_record *rec)
{
    if (n <= 0) return 0;
    double L = P->L, h = P->h, dt = P->dt;
    size_t nd = sizeof(double) * (size_t)n;
    double *sumW = xalloc(nd), *V = xalloc(nd), *B11 = xalloc(nd), *B12 = xalloc(nd),
           *B22 = xalloc(nd), *k = xalloc(nd), *rh = xalloc(nd), *rhat = xalloc(nd),
           *p = xalloc(nd), *gux = xalloc(2 * nd), *guy = xalloc(2 * nd), *lap = xalloc(4 * nd),
           *qn11 = xalloc(nd), *qn12 = xalloc(nd), *an_x = xalloc(nd), *an_y = xalloc(nd),
           *divx = xalloc(nd), *divy = xalloc(nd), *apx = xalloc(nd), *apy = xalloc(nd),
           *trm = xalloc(nd), *f = xalloc(nd), *pel = xalloc(3 * nd);
    int64_t *rowptr = (int64_t *)xalloc(sizeof(int64_t) * (size_t)(n + 1));
    int32_t *cols = NULL;
    int rc = 0;
    if (!sumW || !V || !B11 || !B12 || !B22 || !k || !rh || !rhat || !p || !gux || !guy || !lap ||
        !qn11 || !qn12 || !an_x || !an_y || !divx || !divy || !apx || !apy || !trm || !f || !pel ||
        !rowptr) {
        rc = -1;
        goto done;
    }
    for (int64_t s = 0; s < nsteps; s++) {
        /* predictor: u^{n+1/2} = u^n + dt/2 a^n, r^{n+1/2} = r^n + dt/2 u^{n+1/2}, re-insert */
        double umax = 0.0;
        for (int64_t i = 0; i < n; i++) {
            ux[i] = ux[i] + 0.5 * dt * ax[i];
            uy[i] = uy[i] + 0.5 * dt * ay[i];
            x[i] = wrap(x[i] + 0.5 * dt * ux[i], L);
            y[i] = wrap(y[i] + 0.5 * dt * uy[i], L);
            double um = sqrt(ux[i] * ux[i] + uy[i] * uy[i]);
            if (um > umax) umax = um;
        }
        double c0 = 10.0 * umax;
        if (c0 < P->c0_min) c0 = P->c0_min;

        /* one neighbour search at the projected configuration */
        search(P->nbr_mode, n, x, y, L, h, rowptr, NULL);
        free(cols);
        cols = (int32_t *)xalloc(sizeof(int32_t) * (size_t)rowptr[n]);
        if (!cols) { rc = -1; goto done; }
        search(P->nbr_mode, n, x, y, L, h, rowptr, cols);

        /* kernel sums, volumes, correction tensor */
        orc_volumes(n, x, y, L, h, rowptr, cols, sumW, V);
        if (orc_correction(n, x, y, L, h, rowptr, cols, V, B11, B12, B22) > 0) rc = -2;

        /* continuity and half-step density */
        orc_continuity(n, x, y, L, h, rowptr, cols, V, B11, B12, B22, ux, uy, rho, k);
        for (int64_t i = 0; i < n; i++) rh[i] = rho[i] + 0.5 * dt * k[i];

        /* density filter and equation of state */
        orc_density_filter(n, x, y, L, h, rowptr, cols, P->beta, rh, rhat);
        for (int64_t i = 0; i < n; i++) p[i] = orc_eos(rhat[i], P->rho0, c0, P->gamma_eos);

        /* Q rate and Q^{n+1} */
        orc_gradient(n, x, y, L, h, rowptr, cols, V, B11, B12, B22, ux, gux);
        orc_gradient(n, x, y, L, h, rowptr, cols, V, B11, B12, B22, uy, guy);
        double *Qc[4] = {q11, q12, q12, NULL};
        for (int64_t i = 0; i < n; i++) f[i] = -q11[i];  /* Q22 */
        Qc[3] = f;
        for (int c = 0; c < 4; c++)
            orc_laplacian(n, x, y, L, h, rowptr, cols, V, B11, B12, B22, Qc[c], lap + (size_t)c * n);
        for (int64_t i = 0; i < n; i++) {
            double D[2][2] = {{gux[2 * i], gux[2 * i + 1]}, {guy[2 * i], guy[2 * i + 1]}};
            double lQ[2][2] = {{lap[i], lap[n + i]}, {lap[2 * n + i], lap[3 * n + i]}};
            double m11, m12, H[2][2], Pe[2][2];
            orc_q_rate(P, q11[i], q12[i], D, lQ, &m11, &m12, &trm[i], H);
            qn11[i] = q11[i] + dt * m11;
            qn12[i] = q12[i] + dt * m12;
            if (rec && rec->qrate11) rec->qrate11[i] = m11;   /* the last step's values remain */
            if (rec && rec->qrate12) rec->qrate12[i] = m12;
            orc_elastic_stress(P, q11[i], q12[i], H, Pe);
            pel[3 * i] = Pe[0][0];
            pel[3 * i + 1] = Pe[0][1];
            pel[3 * i + 2] = Pe[1][1];
        }

        /* momentum at the midpoint */
        const double *qa = P->q_new_in_momentum ? qn11 : q11;
        const double *qb = P->q_new_in_momentum ? qn12 : q12;
        if (P->conservative) {
            orc_momentum_conservative(P, n, x, y, rowptr, cols, rhat, p, ux, uy, qa, qb, an_x, an_y, pel);
            for (int64_t i = 0; i < n; i++) {
                double B[2][2] = {{B11[i], B12[i]}, {B12[i], B22[i]}}, dq[2];
                active_sum(i, x, y, L, h, rowptr, cols, V, B, qa, qb, dq);
                divx[i] = dq[0];
                divy[i] = dq[1];
            }
        } else {
            orc_momentum_paper(P, n, x, y, rowptr, cols, V, B11, B12, B22, rhat, p, ux, uy, qa, qb,
                               an_x, an_y, divx, divy, pel);
        }

        /* artificial particle displacement from the midpoint configuration */
        if (P->apd) orc_apd(n, x, y, L, h, dt, rowptr, cols, ux, uy, apx, apy);
        else
            for (int64_t i = 0; i < n; i++) apx[i] = apy[i] = 0.0;

        if (rec && s == nsteps - 1) {
            for (int64_t i = 0; i < n; i++) {
                if (rec->sumW) rec->sumW[i] = sumW[i];
                if (rec->V) rec->V[i] = V[i];
                if (rec->B11) rec->B11[i] = B11[i];
                if (rec->B12) rec->B12[i] = B12[i];
                if (rec->B22) rec->B22[i] = B22[i];
                if (rec->gradu) {
                    rec->gradu[4 * i + 0] = gux[2 * i];
                    rec->gradu[4 * i + 1] = gux[2 * i + 1];
                    rec->gradu[4 * i + 2] = guy[2 * i];
                    rec->gradu[4 * i + 3] = guy[2 * i + 1];
                }
                if (rec->lapQ11) rec->lapQ11[i] = lap[i];
                if (rec->lapQ12) rec->lapQ12[i] = lap[n + i];
                if (rec->k) rec->k[i] = k[i];
                if (rec->rho_half) rec->rho_half[i] = rh[i];
                if (rec->rho_hat) rec->rho_hat[i] = rhat[i];
                if (rec->p) rec->p[i] = p[i];
                if (rec->divQx) rec->divQx[i] = divx[i];
                if (rec->divQy) rec->divQy[i] = divy[i];
                if (rec->ax) rec->ax[i] = an_x[i];
                if (rec->ay) rec->ay[i] = an_y[i];
                if (rec->apdx) rec->apdx[i] = apx[i];
                if (rec->apdy) rec->apdy[i] = apy[i];
                if (rec->trace_m) rec->trace_m[i] = trm[i];
                if (rec->nnbr) rec->nnbr[i] = (int32_t)(rowptr[i + 1] - rowptr[i]);
            }
            if (rec->c0) *rec->c0 = c0;
        }

        /* corrector, then APD and re-insertion */
        for (int64_t i = 0; i < n; i++) {
            ux[i] = ux[i] + 0.5 * dt * an_x[i];
            uy[i] = uy[i] + 0.5 * dt * an_y[i];
            double xn = x[i] + 0.5 * dt * ux[i] + apx[i];
            double yn = y[i] + 0.5 * dt * uy[i] + apy[i];
            x[i] = wrap(xn, L);
            y[i] = wrap(yn, L);
            rho[i] = rhat[i] + 0.5 * dt * k[i];
            q11[i] = qn11[i];
            q12[i] = qn12[i];
            ax[i] = an_x[i];
            ay[i] = an_y[i];
        }
    }
done:
    free(sumW); free(V); free(B11); free(B12); free(B22); free(k); free(rh); free(rhat); free(p);
    free(gux); free(guy); free(lap); free(qn11); free(qn12); free(an_x); free(an_y);
    free(divx); free(divy); free(apx); free(apy); free(trm); free(f); free(pel); free(rowptr); free(cols);
    return rc;
}

int orc_num_threads(void)
{
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}

void orc_set_num_threads(int t)
{
#ifdef _OPENMP
    if (t > 0) omp_set_num_threads(t);
#else
    (void)t;
#endif
}

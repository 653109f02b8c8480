/*
 * FP64 CPU oracle of the three-dimensional SPH active-nematic time step (arXiv 2108.08919, the
 * paper's formulation written for d = 3).
 *
 * TEST INFRASTRUCTURE ONLY.  The plain, slow reference that the CUDA 3D path is checked against;
 * only the test suite and the benchmark's CPU-baseline leg may load it.  It shares no code,
 * header, table or constant with the CUDA library.
 *
 * The paper's runs are two-dimensional; its equations are written for vectors and tensors of any
 * dimension, and Eq. (18) gives the 3D normalisation of the quintic kernel, a_d = 3 / (359 pi h^3).
 * This file takes the 2D oracle's readings over to d = 3:
 *   - Q is the symmetric traceless 3x3 tensor, stored as (Q11, Q12, Q13, Q22, Q23), Q33 =
 *     -Q11 - Q22; m = S + Gamma H is projected onto the symmetric traceless subspace (minus tr/3 I);
 *   - H = -A Q + B (Q^2 - tr(Q^2) I / 3) - C tr(Q^2) Q + K lap Q (Eq. 7; the B term is the one
 *     that survives in 3D);
 *   - the corrected Laplacian keeps the dimension-free factor 2 of the scalar form
 *     lap f_i = 2 sum_j V_j (f_i - f_j) (d_ij . B_i grad_i W_ij) / r^2, applied per component;
 *   - the viscous term of Eq. (23) carries 2 (d + 2) nu = 10 nu (the printed 8 nu is the d = 2
 *     value of the same factor: it makes sum_j V_j (u_ij . d_ij) / r^2 B grad W equal lap u for a
 *     divergence-free field);
 *   - everything else (volumes, correction tensor, continuity, density filter, equation of state,
 *     momentum, artificial displacement, modified Euler) as in the 2D oracle, with x, y, z;
 *   - the elastic stress and the conservative momentum mode are not part of the 3D path.
 * Conventions: d_ij = r_i - r_j (minimum image), r = |d_ij|, b = r/h, support 3h, neighbours
 * j != i with |d_ij|^2 < (3h)^2 in FP64 (no fused multiply-add: -ffp-contract=off);
 * dW_ij/dx_i^l = W'(b)/h d_ij^l / r; D[a][b] = du_a/dx_b.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#ifndef M_PI
#define M_PI 3.14159265358979323846
#endif

typedef struct {
    double L, h, dt, rho0, eta, Gamma, lambda, A, B, C, K, zeta, gamma_eos, beta, c0_min, c_shift;
    int32_t apd;
} orc3_params;

/* Intermediates of the last step (each pointer may be NULL). */
typedef struct {
    double *sumW, *V;
    double *Bm;      /* 9 per particle, row-major */
    double *gradu;   /* 9 per particle: D[a][b] = du_a/dx_b */
    double *lapQ;    /* 5 per particle */
    double *qrate;   /* 5 per particle: the projected rate m */
    double *k, *rho_half, *rho_hat, *p;
    double *a;       /* 3 per particle */
    double *apd;     /* 3 per particle */
    int32_t *nnbr;
    double *c0;
} orc3_record;

/* ---- Quintic kernel, Eq. (18), d = 3 ----------------------------------------------------- */

double orc3_kernel_ad(double h) { return 3.0 / (359.0 * M_PI * h * h * h); }

static double p4(double t) { return t * t * t * t; }
static double p5(double t) { return t * t * t * t * t; }

double orc3_W(double b, double h)
{
    if (b >= 3.0) return 0.0;
    double w = p5(3.0 - b);
    if (b < 2.0) w -= 6.0 * p5(2.0 - b);
    if (b < 1.0) w += 15.0 * p5(1.0 - b);
    return orc3_kernel_ad(h) * w;
}

double orc3_dWdb(double b, double h)
{
    if (b >= 3.0) return 0.0;
    double w = -5.0 * p4(3.0 - b);
    if (b < 2.0) w += 30.0 * p4(2.0 - b);
    if (b < 1.0) w -= 75.0 * p4(1.0 - b);
    return orc3_kernel_ad(h) * w;
}

/* ---- Geometry ----------------------------------------------------------------------------- */

static double min_image(double a, double b, double L)
{
    double d = a - b;
    if (d > 0.5 * L) d -= L;
    else if (d < -0.5 * L) d += L;
    return d;
}

static double wrap(double a, double L)
{
    double w = a - L * floor(a / L);
    if (w >= L) w -= L;
    if (w < 0.0) w = 0.0;
    return w;
}

typedef struct {
    double d[3];   /* d_ij */
    double r, W;
    double g[3];   /* grad_i W_ij */
} pair3_t;

static pair3_t pair3(const double *x, const double *y, const double *z, int64_t i, int64_t j, double L, double h)
{
    pair3_t p;
    p.d[0] = min_image(x[i], x[j], L);
    p.d[1] = min_image(y[i], y[j], L);
    p.d[2] = min_image(z[i], z[j], L);
    p.r = sqrt(p.d[0] * p.d[0] + p.d[1] * p.d[1] + p.d[2] * p.d[2]);
    double b = p.r / h;
    p.W = orc3_W(b, h);
    double f = orc3_dWdb(b, h) / (h * p.r);
    for (int a = 0; a < 3; a++) p.g[a] = f * p.d[a];
    return p;
}

/* Neighbour lists by a cell grid (cells of side >= 3h; all pairs of the 27 surrounding cells are
 * tested, so the set equals the brute-force one).  rowptr[n + 1]; cols (may be NULL to count). */
int64_t orc3_neighbors(int64_t n, const double *x, const double *y, const double *z, double L, double h,
                       int64_t *rowptr, int32_t *cols)
{
    double R2 = 9.0 * h * h;
    int nc = (int)floor(L / (3.0 * h));
    if (nc < 3) {   /* brute force */
        int64_t e = 0;
        for (int64_t i = 0; i < n; i++) {
            rowptr[i] = e;
            for (int64_t j = 0; j < n; j++) {
                if (j == i) continue;
                double dx = min_image(x[i], x[j], L), dy = min_image(y[i], y[j], L), dz = min_image(z[i], z[j], L);
                if (dx * dx + dy * dy + dz * dz < R2) {
                    if (cols) cols[e] = (int32_t)j;
                    e++;
                }
            }
        }
        rowptr[n] = e;
        return e;
    }
    double cs = L / nc;
    int64_t ncell = (int64_t)nc * nc * nc;
    int64_t *start = calloc((size_t)ncell + 1, sizeof(int64_t));
    int64_t *order = malloc(sizeof(int64_t) * (size_t)(n > 0 ? n : 1));
    int64_t *cell = malloc(sizeof(int64_t) * (size_t)(n > 0 ? n : 1));
    for (int64_t i = 0; i < n; i++) {
        int cx = (int)(x[i] / cs), cy = (int)(y[i] / cs), cz = (int)(z[i] / cs);
        if (cx >= nc) cx = nc - 1;
        if (cy >= nc) cy = nc - 1;
        if (cz >= nc) cz = nc - 1;
        cell[i] = ((int64_t)cz * nc + cy) * nc + cx;
        start[cell[i] + 1]++;
    }
    for (int64_t c = 0; c < ncell; c++) start[c + 1] += start[c];
    int64_t *fill = malloc(sizeof(int64_t) * (size_t)ncell);
    memcpy(fill, start, sizeof(int64_t) * (size_t)ncell);
    for (int64_t i = 0; i < n; i++) order[fill[cell[i]]++] = i;
    /* per particle: neighbours in increasing j (sorted), for a reproducible order */
    int64_t e = 0;
    int64_t *tmp = malloc(sizeof(int64_t) * (size_t)(n > 0 ? n : 1));
    for (int64_t i = 0; i < n; i++) {
        rowptr[i] = e;
        int64_t c = cell[i];
        int cx = (int)(c % nc), cy = (int)((c / nc) % nc), cz = (int)(c / ((int64_t)nc * nc));
        int64_t m = 0;
        for (int oz = -1; oz <= 1; oz++)
            for (int oy = -1; oy <= 1; oy++)
                for (int ox = -1; ox <= 1; ox++) {
                    int qx = (cx + ox + nc) % nc, qy = (cy + oy + nc) % nc, qz = (cz + oz + nc) % nc;
                    int64_t q = ((int64_t)qz * nc + qy) * nc + qx;
                    for (int64_t s = start[q]; s < start[q + 1]; s++) {
                        int64_t j = order[s];
                        if (j == i) continue;
                        double dx = min_image(x[i], x[j], L), dy = min_image(y[i], y[j], L),
                               dz = min_image(z[i], z[j], L);
                        if (dx * dx + dy * dy + dz * dz < R2) tmp[m++] = j;
                    }
                }
        /* insertion sort (rows are short) */
        for (int64_t a = 1; a < m; a++) {
            int64_t v = tmp[a], b = a - 1;
            while (b >= 0 && tmp[b] > v) { tmp[b + 1] = tmp[b]; b--; }
            tmp[b + 1] = v;
        }
        if (cols)
            for (int64_t a = 0; a < m; a++) cols[e + a] = (int32_t)tmp[a];
        e += m;
    }
    rowptr[n] = e;
    free(start); free(order); free(cell); free(fill); free(tmp);
    return e;
}

/* ---- The step's operators (Eqs. 19-29 for d = 3) ------------------------------------------ */

typedef struct {
    int64_t n;
    const double *x, *y, *z;
    double L, h;
    const int64_t *rp;
    const int32_t *cols;
} nb3_t;

/* Eq. (19) with the self term: S_i = W(0) + sum_j W_ij, V_i = 1 / S_i. */
void orc3_volumes(const nb3_t *nb, double *sumW, double *V)
{
    #pragma omp parallel for schedule(static)
    for (int64_t i = 0; i < nb->n; i++) {
        double s = orc3_W(0.0, nb->h);
        for (int64_t e = nb->rp[i]; e < nb->rp[i + 1]; e++) s += pair3(nb->x, nb->y, nb->z, i, nb->cols[e], nb->L, nb->h).W;
        if (sumW) sumW[i] = s;
        V[i] = 1.0 / s;
    }
}

static double det3(const double a[3][3])
{
    return a[0][0] * (a[1][1] * a[2][2] - a[1][2] * a[2][1]) - a[0][1] * (a[1][0] * a[2][2] - a[1][2] * a[2][0]) +
           a[0][2] * (a[1][0] * a[2][1] - a[1][1] * a[2][0]);
}

/* Eq. (22): alpha_i^{sl} = sum_j r_ji^s V_j dW_ij/dx_i^l; B_i = alpha_i^{-1} (adjugate / det).
 * Bm: 9 per particle.  Returns the number of particles with det(alpha) <= 0. */
int64_t orc3_correction(const nb3_t *nb, const double *V, double *Bm)
{
    int64_t bad = 0;
    #pragma omp parallel for schedule(static) reduction(+ : bad)
    for (int64_t i = 0; i < nb->n; i++) {
        double a[3][3] = {{0}};
        for (int64_t e = nb->rp[i]; e < nb->rp[i + 1]; e++) {
            int64_t j = nb->cols[e];
            pair3_t p = pair3(nb->x, nb->y, nb->z, i, j, nb->L, nb->h);
            for (int s = 0; s < 3; s++)
                for (int l = 0; l < 3; l++) a[s][l] += (-p.d[s]) * V[j] * p.g[l];
        }
        double det = det3(a);
        if (!(det > 0.0)) bad++;
        double *B = Bm + 9 * i;
        B[0] = (a[1][1] * a[2][2] - a[1][2] * a[2][1]) / det;
        B[1] = (a[0][2] * a[2][1] - a[0][1] * a[2][2]) / det;
        B[2] = (a[0][1] * a[1][2] - a[0][2] * a[1][1]) / det;
        B[3] = (a[1][2] * a[2][0] - a[1][0] * a[2][2]) / det;
        B[4] = (a[0][0] * a[2][2] - a[0][2] * a[2][0]) / det;
        B[5] = (a[0][2] * a[1][0] - a[0][0] * a[1][2]) / det;
        B[6] = (a[1][0] * a[2][1] - a[1][1] * a[2][0]) / det;
        B[7] = (a[0][1] * a[2][0] - a[0][0] * a[2][1]) / det;
        B[8] = (a[0][0] * a[1][1] - a[0][1] * a[1][0]) / det;
    }
    return bad;
}

/* B_i grad_i W_ij as in the 2D oracle: (B g)_a = sum_b B[a][b] g_b. */
static void Bg3(const double *B, const double g[3], double out[3])
{
    for (int a = 0; a < 3; a++) out[a] = B[3 * a] * g[0] + B[3 * a + 1] * g[1] + B[3 * a + 2] * g[2];
}

/* Eq. (20): corrected gradient of a scalar field: (df/dx^k) alpha^{kl} = sum_j V_j (f_j - f_i)
 * dW_ij/dx_i^l, i.e. grad f = rhs B (row vector times B).  out: 3 per particle. */
void orc3_gradient(const nb3_t *nb, const double *V, const double *Bm, const double *f, double *out)
{
    #pragma omp parallel for schedule(static)
    for (int64_t i = 0; i < nb->n; i++) {
        double rhs[3] = {0, 0, 0};
        for (int64_t e = nb->rp[i]; e < nb->rp[i + 1]; e++) {
            int64_t j = nb->cols[e];
            pair3_t p = pair3(nb->x, nb->y, nb->z, i, j, nb->L, nb->h);
            for (int l = 0; l < 3; l++) rhs[l] += V[j] * (f[j] - f[i]) * p.g[l];
        }
        const double *B = Bm + 9 * i;
        for (int k = 0; k < 3; k++) out[3 * i + k] = rhs[0] * B[k] + rhs[1] * B[3 + k] + rhs[2] * B[6 + k];
    }
}

/* Eq. (21), scalar corrected reading: lap f_i = 2 sum_j V_j (f_i - f_j) (d_ij . B_i grad W) / r^2. */
void orc3_laplacian(const nb3_t *nb, const double *V, const double *Bm, const double *f, double *out)
{
    #pragma omp parallel for schedule(static)
    for (int64_t i = 0; i < nb->n; i++) {
        double s = 0.0;
        for (int64_t e = nb->rp[i]; e < nb->rp[i + 1]; e++) {
            int64_t j = nb->cols[e];
            pair3_t p = pair3(nb->x, nb->y, nb->z, i, j, nb->L, nb->h);
            double bg[3];
            Bg3(Bm + 9 * i, p.g, bg);
            s += V[j] * (f[i] - f[j]) * (p.d[0] * bg[0] + p.d[1] * bg[1] + p.d[2] * bg[2]) / (p.r * p.r);
        }
        out[i] = 2.0 * s;
    }
}

/* Eq. (25): k_i = rho_i sum_j V_j (u_i - u_j) . (B_i grad_i W_ij). */
void orc3_continuity(const nb3_t *nb, const double *V, const double *Bm, const double *u3, const double *rho, double *k)
{
    #pragma omp parallel for schedule(static)
    for (int64_t i = 0; i < nb->n; i++) {
        double s = 0.0;
        for (int64_t e = nb->rp[i]; e < nb->rp[i + 1]; e++) {
            int64_t j = nb->cols[e];
            pair3_t p = pair3(nb->x, nb->y, nb->z, i, j, nb->L, nb->h);
            double bg[3];
            Bg3(Bm + 9 * i, p.g, bg);
            for (int a = 0; a < 3; a++) s += V[j] * (u3[3 * i + a] - u3[3 * j + a]) * bg[a];
        }
        k[i] = rho[i] * s;
    }
}

/* Eq. (28): rho_hat_i = rho_i - beta sum_j (rho_i - rho_j) W_ij / sum_j W_ij (self term in both). */
void orc3_density_filter(const nb3_t *nb, double beta, const double *rho, double *rho_hat)
{
    #pragma omp parallel for schedule(static)
    for (int64_t i = 0; i < nb->n; i++) {
        double W0 = orc3_W(0.0, nb->h), num = 0.0, den = W0;
        for (int64_t e = nb->rp[i]; e < nb->rp[i + 1]; e++) {
            int64_t j = nb->cols[e];
            pair3_t p = pair3(nb->x, nb->y, nb->z, i, j, nb->L, nb->h);
            num += (rho[i] - rho[j]) * p.W;
            den += p.W;
        }
        rho_hat[i] = rho[i] - beta * num / den;
    }
}

/* Eq. (26). */
double orc3_eos(double rho, double rho0, double c0, double gamma_eos)
{
    return rho0 * c0 * c0 / gamma_eos * (pow(rho / rho0, gamma_eos) - 1.0);
}

static void q3_full(const double *q, double Q[3][3])
{
    Q[0][0] = q[0]; Q[0][1] = q[1]; Q[0][2] = q[2];
    Q[1][0] = q[1]; Q[1][1] = q[3]; Q[1][2] = q[4];
    Q[2][0] = q[2]; Q[2][1] = q[4]; Q[2][2] = -q[0] - q[3];
}

static void mm3(const double A[3][3], const double B[3][3], double C[3][3])
{
    for (int a = 0; a < 3; a++)
        for (int b = 0; b < 3; b++) C[a][b] = A[a][0] * B[0][b] + A[a][1] * B[1][b] + A[a][2] * B[2][b];
}

/* Eq. (24) with Eqs. (2) and (7) for one particle: the projected rate m (5 components) and the
 * trace of the unprojected m.  D[a][b] = du_a/dx_b; lapQ: 5 components of the corrected Laplacian
 * of Q (lap Q33 = -lap Q11 - lap Q22). */
void orc3_q_rate(const orc3_params *P, const double *q, const double D[3][3], const double *lapq, double *m5,
                 double *trace_m)
{
    double Q[3][3], LQ[3][3], E[3][3], Om[3][3], M[3][3];
    q3_full(q, Q);
    q3_full(lapq, LQ);
    for (int a = 0; a < 3; a++)
        for (int b = 0; b < 3; b++) {
            E[a][b] = 0.5 * (D[a][b] + D[b][a]);
            Om[a][b] = 0.5 * (D[a][b] - D[b][a]);
            M[a][b] = Q[a][b] + (a == b ? P->c_shift : 0.0);
        }
    double QddD = 0.0;
    for (int a = 0; a < 3; a++)
        for (int b = 0; b < 3; b++) QddD += Q[a][b] * D[a][b];
    double L1[3][3], L2[3][3], T1[3][3], T2[3][3], S[3][3];
    for (int a = 0; a < 3; a++)
        for (int b = 0; b < 3; b++) {
            L1[a][b] = P->lambda * E[a][b] + Om[a][b];
            L2[a][b] = P->lambda * E[a][b] - Om[a][b];
        }
    mm3(L1, M, T1);
    mm3(M, L2, T2);
    for (int a = 0; a < 3; a++)
        for (int b = 0; b < 3; b++) S[a][b] = T1[a][b] + T2[a][b] - 2.0 * P->lambda * M[a][b] * QddD;
    double Q2[3][3];
    mm3(Q, Q, Q2);
    double trQ2 = Q2[0][0] + Q2[1][1] + Q2[2][2];
    double m[3][3];
    for (int a = 0; a < 3; a++)
        for (int b = 0; b < 3; b++) {
            double H = -P->A * Q[a][b] + P->B * (Q2[a][b] - (a == b ? trQ2 / 3.0 : 0.0)) - P->C * Q[a][b] * trQ2 +
                       P->K * LQ[a][b];
            m[a][b] = S[a][b] + P->Gamma * H;
        }
    double tr = m[0][0] + m[1][1] + m[2][2];
    if (trace_m) *trace_m = tr;
    double ms[3][3];
    for (int a = 0; a < 3; a++)
        for (int b = 0; b < 3; b++) ms[a][b] = 0.5 * (m[a][b] + m[b][a]) - (a == b ? tr / 3.0 : 0.0);
    m5[0] = ms[0][0]; m5[1] = ms[0][1]; m5[2] = ms[0][2]; m5[3] = ms[1][1]; m5[4] = ms[1][2];
}

/* Eq. (23) for d = 3: a_i = -rho_i sum_j V_j (p_i/rho_i^2 + p_j/rho_j^2) B grad W
 *   + 10 nu rho0/rho_i sum_j V_j (u_ij . d_ij) / r^2 B grad W - zeta/rho_i sum_j V_j (Q_j - Q_i) B grad W.
 * a: 3 per particle; divQ (may be NULL): the active sum. */
void orc3_momentum(const orc3_params *P, const nb3_t *nb, const double *V, const double *Bm, const double *rho,
                   const double *p, const double *u3, const double *q5, double *a, double *divQ)
{
    double nu = P->eta / P->rho0;
    #pragma omp parallel for schedule(static)
    for (int64_t i = 0; i < nb->n; i++) {
        double fp[3] = {0, 0, 0}, fv[3] = {0, 0, 0}, dq[3] = {0, 0, 0}, Qi[3][3];
        q3_full(q5 + 5 * i, Qi);
        for (int64_t e = nb->rp[i]; e < nb->rp[i + 1]; e++) {
            int64_t j = nb->cols[e];
            pair3_t pr = pair3(nb->x, nb->y, nb->z, i, j, nb->L, nb->h);
            double bg[3], Qj[3][3];
            Bg3(Bm + 9 * i, pr.g, bg);
            q3_full(q5 + 5 * j, Qj);
            double cp = p[i] / (rho[i] * rho[i]) + p[j] / (rho[j] * rho[j]);
            double uijd = 0.0;
            for (int c = 0; c < 3; c++) uijd += (u3[3 * i + c] - u3[3 * j + c]) * pr.d[c];
            double r2 = pr.r * pr.r;
            for (int c = 0; c < 3; c++) {
                fp[c] += V[j] * cp * bg[c];
                fv[c] += V[j] * uijd / r2 * bg[c];
                dq[c] += V[j] * ((Qj[c][0] - Qi[c][0]) * bg[0] + (Qj[c][1] - Qi[c][1]) * bg[1] +
                                 (Qj[c][2] - Qi[c][2]) * bg[2]);
            }
        }
        for (int c = 0; c < 3; c++)
            a[3 * i + c] = -rho[i] * fp[c] + 10.0 * nu * P->rho0 / rho[i] * fv[c] - P->zeta / rho[i] * dq[c];
        if (divQ)
            for (int c = 0; c < 3; c++) divQ[3 * i + c] = dq[c];
    }
}

/* Eq. (29): delta r_i = sum_j d_ij / r^3 r0^2 u_v dt, u_v = |sum_j (u_i - u_j) W_ij| / sum_j W_ij
 * (self term in the denominator), r0 = sum_j r_ij / N_i. */
void orc3_apd(const nb3_t *nb, double dt, const double *u3, double *dr)
{
    #pragma omp parallel for schedule(static)
    for (int64_t i = 0; i < nb->n; i++) {
        double su[3] = {0, 0, 0}, sw = orc3_W(0.0, nb->h), sr = 0.0, sd[3] = {0, 0, 0};
        int64_t N = nb->rp[i + 1] - nb->rp[i];
        for (int64_t e = nb->rp[i]; e < nb->rp[i + 1]; e++) {
            int64_t j = nb->cols[e];
            pair3_t p = pair3(nb->x, nb->y, nb->z, i, j, nb->L, nb->h);
            for (int c = 0; c < 3; c++) su[c] += (u3[3 * i + c] - u3[3 * j + c]) * p.W;
            sw += p.W;
            sr += p.r;
            double r3 = p.r * p.r * p.r;
            for (int c = 0; c < 3; c++) sd[c] += p.d[c] / r3;
        }
        double uv = sqrt(su[0] * su[0] + su[1] * su[1] + su[2] * su[2]) / sw;
        double r0 = N > 0 ? sr / (double)N : 0.0;
        for (int c = 0; c < 3; c++) dr[3 * i + c] = sd[c] * r0 * r0 * uv * dt;
    }
}

/* ---- One step, §3.1 (modified Euler) ------------------------------------------------------- */

/* State arrays of length n (x, y, z, rho) and 3n (u, a), 5n (q), updated in place.  Returns 0,
 * -1 on allocation failure, -2 if some alpha was singular. */
int orc3_step(const orc3_params *P, int64_t n, double *x, double *y, double *z, double *u, double *q, double *rho,
              double *a, int64_t nsteps, orc3_record *rec)
{
    if (n <= 0) return 0;
    double L = P->L, h = P->h, dt = P->dt;
    size_t nd = sizeof(double) * (size_t)n;
    double *sumW = malloc(nd), *V = malloc(nd), *Bm = malloc(9 * nd), *k = malloc(nd), *rh = malloc(nd),
           *rhat = malloc(nd), *p = malloc(nd), *gu = malloc(9 * nd), *lap = malloc(5 * nd), *qn = malloc(5 * nd),
           *an = malloc(3 * nd), *ap = malloc(3 * nd), *f = malloc(nd), *g3 = malloc(3 * nd), *lf = malloc(nd),
           *m5 = malloc(5 * nd);
    int64_t *rowptr = malloc(sizeof(int64_t) * (size_t)(n + 1));
    int32_t *cols = NULL;
    int rc = 0;
    if (!sumW || !V || !Bm || !k || !rh || !rhat || !p || !gu || !lap || !qn || !an || !ap || !f || !g3 || !lf ||
        !m5 || !rowptr) {
        rc = -1;
        goto done;
    }
    for (int64_t s = 0; s < nsteps; s++) {
        double umax = 0.0;
        for (int64_t i = 0; i < n; i++) {
            for (int c = 0; c < 3; c++) u[3 * i + c] += 0.5 * dt * a[3 * i + c];
            x[i] = wrap(x[i] + 0.5 * dt * u[3 * i], L);
            y[i] = wrap(y[i] + 0.5 * dt * u[3 * i + 1], L);
            z[i] = wrap(z[i] + 0.5 * dt * u[3 * i + 2], L);
            double um = sqrt(u[3 * i] * u[3 * i] + u[3 * i + 1] * u[3 * i + 1] + u[3 * i + 2] * u[3 * i + 2]);
            if (um > umax) umax = um;
        }
        double c0 = 10.0 * umax;
        if (c0 < P->c0_min) c0 = P->c0_min;
        int64_t ne = orc3_neighbors(n, x, y, z, L, h, rowptr, NULL);
        free(cols);
        cols = malloc(sizeof(int32_t) * (size_t)(ne > 0 ? ne : 1));
        if (!cols) { rc = -1; goto done; }
        orc3_neighbors(n, x, y, z, L, h, rowptr, cols);
        nb3_t nb = {n, x, y, z, L, h, rowptr, cols};
        orc3_volumes(&nb, sumW, V);
        if (orc3_correction(&nb, V, Bm) > 0) rc = -2;
        orc3_continuity(&nb, V, Bm, u, rho, k);
        for (int64_t i = 0; i < n; i++) rh[i] = rho[i] + 0.5 * dt * k[i];
        orc3_density_filter(&nb, P->beta, rh, rhat);
        for (int64_t i = 0; i < n; i++) p[i] = orc3_eos(rhat[i], P->rho0, c0, P->gamma_eos);
        for (int c = 0; c < 3; c++) {   /* row c of the velocity gradient */
            for (int64_t i = 0; i < n; i++) f[i] = u[3 * i + c];
            orc3_gradient(&nb, V, Bm, f, g3);
            for (int64_t i = 0; i < n; i++)
                for (int b = 0; b < 3; b++) gu[9 * i + 3 * c + b] = g3[3 * i + b];
        }
        for (int c = 0; c < 5; c++) {
            for (int64_t i = 0; i < n; i++) f[i] = q[5 * i + c];
            orc3_laplacian(&nb, V, Bm, f, lf);
            for (int64_t i = 0; i < n; i++) lap[5 * i + c] = lf[i];
        }
        for (int64_t i = 0; i < n; i++) {
            double D[3][3];
            for (int r = 0; r < 3; r++)
                for (int c = 0; c < 3; c++) D[r][c] = gu[9 * i + 3 * r + c];
            orc3_q_rate(P, q + 5 * i, D, lap + 5 * i, m5 + 5 * i, NULL);
            for (int c = 0; c < 5; c++) qn[5 * i + c] = q[5 * i + c] + dt * m5[5 * i + c];
        }
        orc3_momentum(P, &nb, V, Bm, rhat, p, u, qn, an, NULL);
        if (P->apd) orc3_apd(&nb, dt, u, ap);
        else memset(ap, 0, 3 * nd);
        if (rec && s == nsteps - 1) {
            for (int64_t i = 0; i < n; i++) {
                if (rec->sumW) rec->sumW[i] = sumW[i];
                if (rec->V) rec->V[i] = V[i];
                if (rec->k) rec->k[i] = k[i];
                if (rec->rho_half) rec->rho_half[i] = rh[i];
                if (rec->rho_hat) rec->rho_hat[i] = rhat[i];
                if (rec->p) rec->p[i] = p[i];
                if (rec->nnbr) rec->nnbr[i] = (int32_t)(rowptr[i + 1] - rowptr[i]);
                for (int c = 0; c < 9; c++) {
                    if (rec->Bm) rec->Bm[9 * i + c] = Bm[9 * i + c];
                    if (rec->gradu) rec->gradu[9 * i + c] = gu[9 * i + c];
                }
                for (int c = 0; c < 5; c++) {
                    if (rec->lapQ) rec->lapQ[5 * i + c] = lap[5 * i + c];
                    if (rec->qrate) rec->qrate[5 * i + c] = m5[5 * i + c];
                }
                for (int c = 0; c < 3; c++) {
                    if (rec->a) rec->a[3 * i + c] = an[3 * i + c];
                    if (rec->apd) rec->apd[3 * i + c] = ap[3 * i + c];
                }
            }
            if (rec->c0) *rec->c0 = c0;
        }
        for (int64_t i = 0; i < n; i++) {
            for (int c = 0; c < 3; c++) u[3 * i + c] += 0.5 * dt * an[3 * i + c];
            x[i] = wrap(x[i] + 0.5 * dt * u[3 * i] + ap[3 * i], L);
            y[i] = wrap(y[i] + 0.5 * dt * u[3 * i + 1] + ap[3 * i + 1], L);
            z[i] = wrap(z[i] + 0.5 * dt * u[3 * i + 2] + ap[3 * i + 2], L);
            rho[i] = rhat[i] + 0.5 * dt * k[i];
            for (int c = 0; c < 5; c++) q[5 * i + c] = qn[5 * i + c];
            for (int c = 0; c < 3; c++) a[3 * i + c] = an[3 * i + c];
        }
    }
done:
    free(sumW); free(V); free(Bm); free(k); free(rh); free(rhat); free(p); free(gu); free(lap); free(qn);
    free(an); free(ap); free(f); free(g3); free(lf); free(m5); free(rowptr); free(cols);
    return rc;
}

/*
 * rp.c -- rectangular-polar (RP) singular / near-singular correction for
 * cube-sphere surfaces, FP64 (TEST INFRASTRUCTURE ONLY, like oracle.c).
 *
 * For each target x_l and each patch Gamma^q within distance delta of it
 * (Eq. SingGridPts), the patch integral of K(x_l, y) phi(y) is evaluated as
 * sum_{n,m} a^q_{nm} beta^{q,l}_{nm} (Eq. IntOpAtSing) with
 *   a^q_{nm}       Chebyshev coefficients of phi on the patch (Eq. ChebyCoeff),
 *   beta^{q,l}_{nm} = int K(x_l, y^q(u,v)) T_n(u) T_m(v) J^q(u,v) du dv (Eq. BetaAtSing),
 * computed with Fejer's first rule after the clustering change of variables
 * xi_alpha (Eq. CoV) built on the Kress map w(tau; d) (Eq. wMap, Eq. vMap) and
 * centred at the closest patch point (u_bar, v_bar) (Eq. MinNode, golden-section
 * search; exact when x_l is a node of the patch).  Kernel values closer than
 * 1e-14 L are dropped (end of Section 4.2).
 *
 * The output is the correction C = (RP rows) - (regular rows on the same
 * patches), as CSR over the point order: the regular part (Eq.
 * ReguIntOpQuadrature with m != l) is what the accelerated sum already
 * contains, so y = c_I phi + (regular sum) + C phi uses RP on near patches.
 *
 * Geometry: equiangular cube-sphere of radius R; face f (axis f/2, sign +-1),
 * sub-patch (pu, pv) of P x P per face, m x m Chebyshev-Gauss nodes per patch.
 * Unspecified RP constants (delta, d, N_beta, golden tolerance) are parameters.
 */
#include <complex.h>
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

typedef double complex cplx;
#define RP_PI 3.14159265358979323846

typedef struct {
    double R;
    int P, m;
} rp_sphere;

/* face frames: face point = X eX + Y eY + en */
static void face_frame(int f, double *eX, double *eY, double *en) {
    int ax = f / 2;
    double sg = (f % 2 == 0) ? 1.0 : -1.0;
    int o1 = (ax + 1) % 3, o2 = (ax + 2) % 3;
    for (int a = 0; a < 3; a++) eX[a] = eY[a] = en[a] = 0.0;
    eX[o1] = 1.0;
    eY[o2] = sg;
    en[ax] = sg;
}

/* y^q(u, v), Jacobian J^q and unit normal for patch q, local (u, v) in [-1, 1]^2 */
static void patch_map(const rp_sphere *S, int q, double u, double v, double *y, double *J, double *nu) {
    int P = S->P;
    int f = q / (P * P), pu = (q / P) % P, pv = q % P;
    double eX[3], eY[3], en[3];
    face_frame(f, eX, eY, en);
    double U = -1.0 + (2.0 * pu + 1.0 + u) / P, V = -1.0 + (2.0 * pv + 1.0 + v) / P;
    double X = tan(RP_PI * U / 4.0), Y = tan(RP_PI * V / 4.0);
    double p[3];
    for (int a = 0; a < 3; a++) p[a] = X * eX[a] + Y * eY[a] + en[a];
    double rho = sqrt(1.0 + X * X + Y * Y);
    for (int a = 0; a < 3; a++) {
        nu[a] = p[a] / rho;
        y[a] = S->R * nu[a];
    }
    *J = S->R * S->R * (RP_PI / 4.0) * (RP_PI / 4.0) * (1.0 + X * X) * (1.0 + Y * Y) / (rho * rho * rho) / (P * P);
}

static double dist2_to(const rp_sphere *S, int q, const double *x, double u, double v) {
    double y[3], J, nu[3];
    patch_map(S, q, u, v, y, &J, nu);
    double d0 = x[0] - y[0], d1 = x[1] - y[1], d2 = x[2] - y[2];
    return d0 * d0 + d1 * d1 + d2 * d2;
}

/* golden-section search of a unimodal function on [a, b] */
typedef double (*fn1)(void *ctx, double t);
static double golden(fn1 f, void *ctx, double a, double b, double tol, double *fmin) {
    const double g = (sqrt(5.0) - 1.0) / 2.0;
    double c = b - g * (b - a), d = a + g * (b - a);
    double fc = f(ctx, c), fd = f(ctx, d);
    while (b - a > tol) {
        if (fc < fd) {
            b = d; d = c; fd = fc;
            c = b - g * (b - a); fc = f(ctx, c);
        } else {
            a = c; c = d; fc = fd;
            d = a + g * (b - a); fd = f(ctx, d);
        }
    }
    double t = 0.5 * (a + b);
    if (fmin) *fmin = f(ctx, t);
    return t;
}

typedef struct {
    const rp_sphere *S;
    int q;
    const double *x;
    double u;
    double tol;
} gs_ctx;

static double f_inner(void *c, double v) {
    gs_ctx *g = (gs_ctx *)c;
    return dist2_to(g->S, g->q, g->x, g->u, v);
}
static double f_outer(void *c, double u) {
    gs_ctx *g = (gs_ctx *)c;
    g->u = u;
    double fm;
    golden(f_inner, c, -1.0, 1.0, g->tol, &fm);
    return fm;
}

/* closest point (Eq. MinNode) by nested golden-section searches */
static double closest_point(const rp_sphere *S, int q, const double *x, double tol, double *ub, double *vb) {
    gs_ctx g = {S, q, x, 0.0, tol};
    double u = golden(f_outer, &g, -1.0, 1.0, tol, NULL);
    g.u = u;
    double fm;
    double v = golden(f_inner, &g, -1.0, 1.0, tol, &fm);
    *ub = u;
    *vb = v;
    return sqrt(fm);
}

/* Kress-type grading: nu(tau; d) (Eq. vMap), w(tau; d) (Eq. wMap) and w'(tau) */
static double vmap(double t, double d) {
    double a = (RP_PI - t) / RP_PI;
    return (1.0 / d - 0.5) * a * a * a + (1.0 / d) * ((t - RP_PI) / RP_PI) + 0.5;
}
static double vmap_d(double t, double d) {
    double a = (RP_PI - t) / RP_PI;
    return (1.0 / d - 0.5) * 3.0 * a * a * (-1.0 / RP_PI) + (1.0 / d) / RP_PI;
}
static double wmap(double t, double d) {
    double A = pow(vmap(t, d), d), B = pow(vmap(2.0 * RP_PI - t, d), d);
    return 2.0 * RP_PI * A / (A + B);
}
static double wmap_d(double t, double d) {
    double va = vmap(t, d), vb = vmap(2.0 * RP_PI - t, d);
    double A = pow(va, d), B = pow(vb, d);
    double dA = d * pow(va, d - 1.0) * vmap_d(t, d);
    double dB = -d * pow(vb, d - 1.0) * vmap_d(2.0 * RP_PI - t, d);
    return 2.0 * RP_PI * (dA * B - A * dB) / ((A + B) * (A + B));
}

/* clustering change of variables xi_alpha(tau; d) of Eq. CoV and its derivative */
static void cov(double alpha, double tau, double d, double *xi, double *dxi) {
    if (alpha >= 1.0) {
        double s = RP_PI * fabs((tau - 1.0) / 2.0);
        *xi = alpha - ((1.0 + alpha) / RP_PI) * wmap(s, d);
        *dxi = wmap_d(s, d) * ((1.0 + alpha) / RP_PI) * (RP_PI / 2.0);
    } else if (alpha <= -1.0) {
        double s = RP_PI * fabs((tau + 1.0) / 2.0);
        *xi = alpha + ((1.0 - alpha) / RP_PI) * wmap(s, d);
        *dxi = wmap_d(s, d) * ((1.0 - alpha) / RP_PI) * (RP_PI / 2.0);
    } else {
        double sg = (tau > 0) - (tau < 0);
        double s = RP_PI * fabs(tau);
        *xi = alpha + ((sg - alpha) / RP_PI) * wmap(s, d);
        *dxi = ((sg - alpha) / RP_PI) * wmap_d(s, d) * RP_PI * sg;
    }
}

static cplx cfie_k(double k, double eta, const double *x, const double *y, const double *ny) {
    double d0 = x[0] - y[0], d1 = x[1] - y[1], d2 = x[2] - y[2];
    double r = sqrt(d0 * d0 + d1 * d1 + d2 * d2);
    cplx e = cexp(I * k * r);
    double dn = d0 * ny[0] + d1 * ny[1] + d2 * ny[2];
    return e * (1.0 - I * k * r) * dn / (4.0 * RP_PI * r * r * r) - I * eta * e / (4.0 * RP_PI * r);
}

static void cheb_T(double t, int n, double *T) {
    T[0] = 1.0;
    if (n > 1) T[1] = t;
    for (int i = 2; i < n; i++) T[i] = 2.0 * t * T[i - 1] - T[i - 2];
}

/*
 * Build the correction.  Points are indexed by the caller; for point g,
 * patch[g] = q and node[g] = i * m + j (its Chebyshev-Gauss node (i, j) on patch q),
 * node_of[q * m * m + i * m + j] = g.  xyz / nrm / w are the points, normals and
 * quadrature weights used by the regular sum.  Output arrays are allocated with
 * malloc and returned through the pointers (free with oracle_rp_free).
 * Returns 0 on success.
 */
int oracle_rp_correction(int64_t N, const double *xyz, const double *nrm, const double *w, const int *patch,
                         const int *node, const int *node_of, double R, int P, int m, double k, double eta,
                         double delta, int Nbeta, double dgrade, double tol_zero, int64_t **rowptr_out,
                         int32_t **col_out, double **val_out) {
    if (m > 32 || Nbeta > 128 || N <= 0) return -1;
    rp_sphere S = {R, P, m};
    const int Q = 6 * P * P;
    const int m2 = m * m;
    /* patch centres and radii for a quick rejection */
    double *pc = (double *)malloc(sizeof(double) * 3 * Q), *prad = (double *)malloc(sizeof(double) * Q);
    for (int q = 0; q < Q; q++) {
        double y[3], J, nu[3];
        patch_map(&S, q, 0.0, 0.0, y, &J, nu);
        memcpy(pc + 3 * q, y, sizeof(y));
        double rmax = 0;
        for (int c = 0; c < 4; c++) {
            double yc[3];
            patch_map(&S, q, (c & 1) ? 1.0 : -1.0, (c & 2) ? 1.0 : -1.0, yc, &J, nu);
            double dd = sqrt((yc[0] - y[0]) * (yc[0] - y[0]) + (yc[1] - y[1]) * (yc[1] - y[1]) +
                             (yc[2] - y[2]) * (yc[2] - y[2]));
            if (dd > rmax) rmax = dd;
        }
        prad[q] = rmax;
    }
    /* Fejer nodes/weights for beta, Chebyshev-Gauss nodes of the patches and alpha_n / (m^2) */
    double sb[128], wb[128], tn[32];
    for (int i = 0; i < Nbeta; i++) {
        sb[i] = cos(RP_PI * (2.0 * i + 1.0) / (2.0 * Nbeta));
        double acc = 0.0;
        for (int l = 1; l <= Nbeta / 2; l++) acc += cos(l * RP_PI * (2.0 * i + 1.0) / Nbeta) / (4.0 * l * l - 1.0);
        wb[i] = (2.0 / Nbeta) * (1.0 - 2.0 * acc);
    }
    for (int i = 0; i < m; i++) tn[i] = cos(RP_PI * (2.0 * i + 1.0) / (2.0 * m));
    /* Tnode[n][i] = alpha_n T_n(t_i) / m (Eq. ChebyCoeff, one factor per direction) */
    double *Tnode = (double *)malloc(sizeof(double) * m * m);
    for (int i = 0; i < m; i++) {
        double T[32];
        cheb_T(tn[i], m, T);
        for (int n = 0; n < m; n++) Tnode[n * m + i] = (n == 0 ? 1.0 : 2.0) * T[n] / m;
    }
    /* per target rows (variable length), assembled afterwards */
    int64_t *cnt = (int64_t *)calloc(N, sizeof(int64_t));
    int32_t **rcol = (int32_t **)calloc(N, sizeof(int32_t *));
    cplx **rval = (cplx **)calloc(N, sizeof(cplx *));
    int err = 0;
#pragma omp parallel for schedule(dynamic, 4)
    for (int64_t l = 0; l < N; l++) {
        const double *x = xyz + 3 * l;
        int cap = 16 * m2, nn = 0;
        int32_t *cl = (int32_t *)malloc(sizeof(int32_t) * cap);
        cplx *vl = (cplx *)malloc(sizeof(cplx) * cap);
        cplx beta[32 * 32], Wn[32 * 32];
        double Tu[128][32], Tv[128][32], uq[128], vq[128], wu[128], wv[128];
        for (int q = 0; q < Q; q++) {
            double dc = sqrt((x[0] - pc[3 * q]) * (x[0] - pc[3 * q]) + (x[1] - pc[3 * q + 1]) * (x[1] - pc[3 * q + 1]) +
                             (x[2] - pc[3 * q + 2]) * (x[2] - pc[3 * q + 2]));
            if (dc - prad[q] > delta) continue;
            double ub, vb, dist;
            if (patch[l] == q) {
                ub = tn[node[l] / m];
                vb = tn[node[l] % m];
                dist = 0.0;
            } else {
                dist = closest_point(&S, q, x, 1e-12, &ub, &vb);
                if (ub > 1.0 - 1e-10) ub = 1.0;
                if (ub < -1.0 + 1e-10) ub = -1.0;
                if (vb > 1.0 - 1e-10) vb = 1.0;
                if (vb < -1.0 + 1e-10) vb = -1.0;
            }
            if (dist > delta) continue;
            /* graded Fejer rule (Eq. BetaCov, Eq. CovNodesWeights) */
            for (int a = 0; a < Nbeta; a++) {
                double xi, dxi;
                cov(ub, sb[a], dgrade, &xi, &dxi);
                uq[a] = xi;
                wu[a] = dxi * wb[a];
                cheb_T(xi, m, Tu[a]);
                cov(vb, sb[a], dgrade, &xi, &dxi);
                vq[a] = xi;
                wv[a] = dxi * wb[a];
                cheb_T(xi, m, Tv[a]);
            }
            for (int i = 0; i < m2; i++) beta[i] = 0.0;
            for (int a = 0; a < Nbeta; a++)
                for (int b = 0; b < Nbeta; b++) {
                    double y[3], J, nu[3];
                    patch_map(&S, q, uq[a], vq[b], y, &J, nu);
                    double d0 = x[0] - y[0], d1 = x[1] - y[1], d2 = x[2] - y[2];
                    if (sqrt(d0 * d0 + d1 * d1 + d2 * d2) < tol_zero) continue;
                    cplx Kv = cfie_k(k, eta, x, y, nu) * J * wu[a] * wv[b];
                    for (int n = 0; n < m; n++) {
                        cplx kn = Kv * Tu[a][n];
                        for (int mm = 0; mm < m; mm++) beta[n * m + mm] += kn * Tv[b][mm];
                    }
                }
            /* RP weight of node (i, j): sum_{n,m} beta_nm alpha_n alpha_m T_n(t_i) T_m(t_j) / m^2 */
            for (int i = 0; i < m; i++) {
                cplx tmp[32];
                for (int mm = 0; mm < m; mm++) {
                    cplx s = 0.0;
                    for (int n = 0; n < m; n++) s += beta[n * m + mm] * Tnode[n * m + i];
                    tmp[mm] = s;
                }
                for (int j = 0; j < m; j++) {
                    cplx s = 0.0;
                    for (int mm = 0; mm < m; mm++) s += tmp[mm] * Tnode[mm * m + j];
                    Wn[i * m + j] = s;
                }
            }
            if (nn + m2 > cap) {
                cap = 2 * (nn + m2);
                cl = (int32_t *)realloc(cl, sizeof(int32_t) * cap);
                vl = (cplx *)realloc(vl, sizeof(cplx) * cap);
            }
            for (int ij = 0; ij < m2; ij++) {
                int g = node_of[q * m2 + ij];
                cplx v = Wn[ij];
                if (g != l) {
                    const double *yg = xyz + 3 * g;
                    double d0 = x[0] - yg[0], d1 = x[1] - yg[1], d2 = x[2] - yg[2];
                    if (sqrt(d0 * d0 + d1 * d1 + d2 * d2) >= tol_zero) v -= cfie_k(k, eta, x, yg, nrm + 3 * g) * w[g];
                }
                cl[nn] = g;
                vl[nn] = v;
                nn++;
            }
        }
        cnt[l] = nn;
        rcol[l] = cl;
        rval[l] = vl;
    }
    int64_t *rowptr = (int64_t *)malloc(sizeof(int64_t) * (N + 1));
    rowptr[0] = 0;
    for (int64_t l = 0; l < N; l++) rowptr[l + 1] = rowptr[l] + cnt[l];
    int64_t nnz = rowptr[N];
    int32_t *col = (int32_t *)malloc(sizeof(int32_t) * (nnz > 0 ? nnz : 1));
    double *val = (double *)malloc(sizeof(double) * 2 * (nnz > 0 ? nnz : 1));
    for (int64_t l = 0; l < N; l++) {
        for (int64_t j = 0; j < cnt[l]; j++) {
            col[rowptr[l] + j] = rcol[l][j];
            val[2 * (rowptr[l] + j)] = creal(rval[l][j]);
            val[2 * (rowptr[l] + j) + 1] = cimag(rval[l][j]);
        }
        free(rcol[l]);
        free(rval[l]);
    }
    free(rcol); free(rval); free(cnt); free(pc); free(prad); free(Tnode);
    *rowptr_out = rowptr;
    *col_out = col;
    *val_out = val;
    return err;
}

void oracle_rp_free(void *p) { free(p); }

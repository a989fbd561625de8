/*
 * oracle.c -- plain FP64 CPU reference for the IFGF-accelerated CFIE apply.
 *
 * TEST INFRASTRUCTURE ONLY.  Only the tests, the smoke check and the bench's
 * CPU-baseline leg may load this library.  It shares no code, header, table or
 * constant generator with the CUDA library; the two only see the same seeded
 * inputs (points, normals, weights, densities).
 *
 * What it computes (all FP64):
 *   oracle_direct_rows:   y_l = cI s_l + sum_{m != l} K(x_l, x_m) w_m s_m   (Eq. field1 with
 *                         the combined-field kernel of Eq. CombinedLayer, Eq. GreenFunction,
 *                         Eq. double_layer; the 1/2 identity term of Eq. CombLayIE is cI);
 *                         the *_layer variants and oracle_params.layer take the double layer
 *                         dPhi/dnu or the single layer Phi alone instead
 *   oracle_direct_adjoint_rows: (A^H g)_m = conj(cI) g_m + w_m sum_{l != m} conj(K(x_l, x_m)) g_l
 *   oracle_ifgf:          the same sum accelerated by the IFGF method of Section 3.4, in stages:
 *                         the leaf expansions of the analytic factor at the cone-segment
 *                         interpolation points, then for d = D..3 interpolation onto the cousin
 *                         points and, for d > 3, onto the parent's interpolation points with
 *                         re-centring (Eq. cent_fact); the level-D neighbour interactions by
 *                         direct summation (Remark level_D_neighboring).
 *                         With oracle_params.leaf_max > 0 the octree is adaptive: a box of at most
 *                         leaf_max points is a leaf at its level (leaf expansions there, no boxes
 *                         below it), cousin interpolations reach only points that still have a box at
 *                         that level, and the near field pairs points whose boxes neighbour at the
 *                         coarser of their two leaf levels.
 *   oracle_ifgf_far_field: the far-field pattern (Eq. FarField) from the level-3 interpolants:
 *                         the s -> 0 limit of E(x; y_B) F_B(x) summed over the level-3 boxes.
 *
 * Readings of the paper taken here (each also listed in the design notes):
 *   - Chebyshev interpolation uses first-kind nodes cos((2k+1)pi/(2n)) with the discrete-
 *     orthogonality coefficients a_i = (2 / (n b_i)) sum_k u(x_k) T_i(x_k), b_0 = 2, b_i = 1
 *     (Eq. ChebyNodes; the printed Eq. ChebyCoeffs has Lobatto-type factors that do not
 *     interpolate at first-kind nodes).
 *   - Cone counts (Remark cone_seg_size): cone_rule 0 doubles (n_s, n_C) each time H_d exceeds
 *     lambda/2 * 2^e; cone_rule 1 is the literal remark (leaf level at (nS0, nC0), doubling
 *     from level d to d-1 when k H_d > 1/2).
 *   - Propagation factor (Section 3.4, child to parent): the ratio of centred factors E(x; y_child) / E(x; y_parent)
 *     of Eq. cent_fact.
 *   - Interpolated factors: combined W_C = W~2 - i k W3 - i eta W1 (q = 1) on levels with
 *     H >= lambda/2 and the split pair {W2 (q = 2), W13 = -i k W3 - i eta W1 (q = 1)} below
 *     (Section 3.3's hybrid recommendation applied to the combined-field kernel); factor_mode
 *     1 / 2 force combined / split everywhere.
 *   - The phase k (h/s)(|u - v s| - 1) of Eq. V3 is evaluated in the algebraically identical
 *     cancellation-free form k (s |y - y0|^2 / h - 2 u.(y - y0)) / (|u - v s| + 1).
 *   - Cone indices are clamped (min(floor(.), n - 1)); phi in [0, 2 pi); theta from atan2.
 *     A point on a cone boundary (within 1e-12 relative) belongs to the upper interval.
 *   - Pairs closer than 1e-14 L (L the root box side) are dropped (Section 4.2 end).
 *   - Root box: centre = AABB midpoint, side = max AABB extent * (1 + 2^-30).
 *   - Automatic level count: D = argmin_{d >= 3} |log(N / #relevant level-d boxes / leaf_target)|.
 */
#include <complex.h>
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

typedef double complex cplx;

#define OR_MAXD 20
#define OR_PI 3.14159265358979323846

typedef struct {
    double k, eta;
    int Ps, Pang, nC0, nS0, levels;
    double leaf_target;
    int cone_rule, factor_mode;
    double identity_coef;
    double root_center[3], root_side;
    int far_field; /* 1: level 3 also keeps every segment with is = 0 (oracle_ifgf_far_field) */
    int layer;     /* 0 combined field, 1 double layer, 2 single layer (layer_kernel) */
    int leaf_max;  /* 0: uniform tree; > 0: a box of level 3..D-1 with at most leaf_max points is a leaf */
} oracle_params;

typedef struct {
    int D;
    double root_center[3], root_side;
    int nbox[OR_MAXD + 1], ns[OR_MAXD + 1], nC[OR_MAXD + 1], split[OR_MAXD + 1];
    int64_t nrc[OR_MAXD + 1];
    int64_t cousin_evals[OR_MAXD + 1];
    int64_t prop_evals[OR_MAXD + 1];
    int64_t leaf_evals, near_pairs;
} oracle_info;

int oracle_num_threads(void) {
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}

/* ------------------------------------------------------------------------- */
/* kernels (Eq. GreenFunction, Eq. double_layer): layer 0 the combined field K = dPhi/dnu(y) - i eta Phi
 * (Eq. CombinedLayer), layer 1 the double layer dPhi/dnu(y), layer 2 the single layer Phi */

static cplx layer_kernel(int layer, double k, double eta, const double *x, const double *y, const double *ny) {
    double d0 = x[0] - y[0], d1 = x[1] - y[1], d2 = x[2] - y[2];
    double r = sqrt(d0 * d0 + d1 * d1 + d2 * d2);
    cplx e = cexp(I * k * r);
    cplx Phi = e / (4.0 * OR_PI * r);
    double dn = d0 * ny[0] + d1 * ny[1] + d2 * ny[2];
    cplx dPhi = e * (1.0 - I * k * r) * dn / (4.0 * OR_PI * r * r * r);
    if (layer == 2) return Phi;
    if (layer == 1) return dPhi;
    return dPhi - I * eta * Phi;
}

static cplx cfie_kernel(double k, double eta, const double *x, const double *y, const double *ny) {
    return layer_kernel(0, k, eta, x, y, ny);
}

void oracle_kernel(double k, double eta, const double *x, const double *y, const double *ny, double *out) {
    cplx v = cfie_kernel(k, eta, x, y, ny);
    out[0] = creal(v);
    out[1] = cimag(v);
}

/* single-layer Phi and double-layer dPhi/dnu(y) separately (for the tests' pins) */
void oracle_layer_kernels(double k, const double *x, const double *y, const double *ny, double *out) {
    double d0 = x[0] - y[0], d1 = x[1] - y[1], d2 = x[2] - y[2];
    double r = sqrt(d0 * d0 + d1 * d1 + d2 * d2);
    cplx e = cexp(I * k * r);
    cplx Phi = e / (4.0 * OR_PI * r);
    double dn = d0 * ny[0] + d1 * ny[1] + d2 * ny[2];
    cplx dPhi = e * (1.0 - I * k * r) * dn / (4.0 * OR_PI * r * r * r);
    out[0] = creal(Phi); out[1] = cimag(Phi);
    out[2] = creal(dPhi); out[3] = cimag(dPhi);
}

static double root_side_of(int64_t N, const double *xyz, double *center) {
    double lo[3] = {INFINITY, INFINITY, INFINITY}, hi[3] = {-INFINITY, -INFINITY, -INFINITY};
    for (int64_t i = 0; i < N; i++)
        for (int a = 0; a < 3; a++) {
            double v = xyz[3 * i + a];
            if (v < lo[a]) lo[a] = v;
            if (v > hi[a]) hi[a] = v;
        }
    double ext = 0.0;
    for (int a = 0; a < 3; a++) {
        center[a] = 0.5 * (lo[a] + hi[a]);
        if (hi[a] - lo[a] > ext) ext = hi[a] - lo[a];
    }
    if (!(ext > 0.0)) ext = 1.0;
    return ext * (1.0 + ldexp(1.0, -30));
}

/* ------------------------------------------------------------------------- */
/* direct sums (Eq. field1)                                                   */

int oracle_direct_rows_layer(int layer, int64_t N, const double *xyz, const double *nrm, const double *w,
                             double k, double eta, double cI_re, double cI_im, int nrhs, const double *sigma,
                             int64_t nrows, const int64_t *rows, double *out) {
    if (N <= 0 || nrhs <= 0 || nrhs > 64) return -1;
    double c[3];
    double tol = 1e-14 * root_side_of(N, xyz, c);
    const cplx *sg = (const cplx *)sigma;
    cplx *o = (cplx *)out;
    cplx cI = cI_re + I * cI_im;
#pragma omp parallel for schedule(dynamic, 16)
    for (int64_t t = 0; t < nrows; t++) {
        int64_t l = rows ? rows[t] : t;
        cplx acc[64];
        for (int q = 0; q < nrhs; q++) acc[q] = 0.0;
        for (int64_t m = 0; m < N; m++) {
            if (m == l) continue;
            const double *x = xyz + 3 * l, *y = xyz + 3 * m;
            double d0 = x[0] - y[0], d1 = x[1] - y[1], d2 = x[2] - y[2];
            if (sqrt(d0 * d0 + d1 * d1 + d2 * d2) < tol) continue;
            cplx K = layer_kernel(layer, k, eta, x, y, nrm + 3 * m) * w[m];
            for (int q = 0; q < nrhs; q++) acc[q] += K * sg[(int64_t)q * N + m];
        }
        for (int q = 0; q < nrhs; q++) o[(int64_t)q * nrows + t] = cI * sg[(int64_t)q * N + l] + acc[q];
    }
    return 0;
}

int oracle_direct_rows(int64_t N, const double *xyz, const double *nrm, const double *w, double k, double eta,
                       double cI_re, double cI_im, int nrhs, const double *sigma, int64_t nrows,
                       const int64_t *rows, double *out) {
    return oracle_direct_rows_layer(0, N, xyz, nrm, w, k, eta, cI_re, cI_im, nrhs, sigma, nrows, rows, out);
}

int oracle_direct_adjoint_rows_layer(int layer, int64_t N, const double *xyz, const double *nrm, const double *w,
                                     double k, double eta, double cI_re, double cI_im, int nrhs, const double *g,
                                     int64_t nrows, const int64_t *rows, double *out) {
    if (N <= 0 || nrhs <= 0 || nrhs > 64) return -1;
    double c[3];
    double tol = 1e-14 * root_side_of(N, xyz, c);
    const cplx *gg = (const cplx *)g;
    cplx *o = (cplx *)out;
    cplx cI = cI_re + I * cI_im;
#pragma omp parallel for schedule(dynamic, 16)
    for (int64_t t = 0; t < nrows; t++) {
        int64_t m = rows ? rows[t] : t;
        cplx acc[64];
        for (int q = 0; q < nrhs; q++) acc[q] = 0.0;
        for (int64_t l = 0; l < N; l++) {
            if (l == m) continue;
            const double *x = xyz + 3 * l, *y = xyz + 3 * m;
            double d0 = x[0] - y[0], d1 = x[1] - y[1], d2 = x[2] - y[2];
            if (sqrt(d0 * d0 + d1 * d1 + d2 * d2) < tol) continue;
            cplx K = conj(layer_kernel(layer, k, eta, x, y, nrm + 3 * m)) * w[m];
            for (int q = 0; q < nrhs; q++) acc[q] += K * gg[(int64_t)q * N + l];
        }
        for (int q = 0; q < nrhs; q++) o[(int64_t)q * nrows + t] = conj(cI) * gg[(int64_t)q * N + m] + acc[q];
    }
    return 0;
}

int oracle_direct_adjoint_rows(int64_t N, const double *xyz, const double *nrm, const double *w, double k,
                               double eta, double cI_re, double cI_im, int nrhs, const double *g, int64_t nrows,
                               const int64_t *rows, double *out) {
    return oracle_direct_adjoint_rows_layer(0, N, xyz, nrm, w, k, eta, cI_re, cI_im, nrhs, g, nrows, rows, out);
}

/* ------------------------------------------------------------------------- */
/* Chebyshev interpolation (Eq. ChebyPoly, Eq. ChebyNodes; coefficients per the
 * first-kind discrete orthogonality)                                          */

static double cheb_node(int kk, int n) { return cos((2.0 * kk + 1.0) * OR_PI / (2.0 * n)); }

/* T_0..T_{n-1}(t) by the three-term recurrence T_{i+1} = 2 t T_i - T_{i-1} */
static void cheb_T(double t, int n, double *T) {
    T[0] = 1.0;
    if (n > 1) T[1] = t;
    for (int i = 2; i < n; i++) T[i] = 2.0 * t * T[i - 1] - T[i - 2];
}

/* A[i][k] = 2 / (n b_i) T_i(x_k) */
static void cheb_coeff_matrix(int n, double *A) {
    double T[32];
    for (int kk = 0; kk < n; kk++) {
        cheb_T(cheb_node(kk, n), n, T);
        for (int i = 0; i < n; i++) A[i * n + kk] = (2.0 / n) * (i == 0 ? 0.5 : 1.0) * T[i];
    }
}

/* 1-D interpolation of values v at the n first-kind nodes, evaluated at t (tests' pin). */
double oracle_cheb_interp_1d(int n, const double *v, double t) {
    double A[32 * 32], T[32], s = 0.0;
    cheb_coeff_matrix(n, A);
    cheb_T(t, n, T);
    for (int i = 0; i < n; i++) {
        double ci = 0.0;
        for (int kk = 0; kk < n; kk++) ci += A[i * n + kk] * v[kk];
        s += ci * T[i];
    }
    return s;
}

/* ------------------------------------------------------------------------- */
/* octree levels                                                              */

typedef struct {
    int64_t key;
    int idx;
} keyidx;

static int cmp_keyidx(const void *a, const void *b) {
    const keyidx *x = (const keyidx *)a, *y = (const keyidx *)b;
    if (x->key < y->key) return -1;
    if (x->key > y->key) return 1;
    return (x->idx > y->idx) - (x->idx < y->idx);
}

static int cmp_int(const void *a, const void *b) {
    int x = *(const int *)a, y = *(const int *)b;
    return (x > y) - (x < y);
}

static int64_t make_key(int i, int j, int k) { return ((int64_t)i << 42) | ((int64_t)j << 21) | (int64_t)k; }

typedef struct {
    int nbox;
    double H, h;
    int64_t *key;
    int *ijk;
    int *pstart, *pcount, *perm;
    int *parent;
    int *co_start, *co_list;
    int ns, nC, nph, ncone;
    double ds, dth, dph;
    int split, nfac;
    int *rc_start, *rc_ids;
    int64_t nrc;
    cplx *F, *C;
    unsigned char *alive, *leaf; /* adaptive tree: a box exists (alive) when every ancestor is subdivided;
                                    a leaf is alive and not subdivided (always at level D) */
} olevel;

typedef struct {
    int D, P, Ps, Pang, nrhs, far_field, layer, leaf_max;
    double k, eta, L, c0[3];
    const double *xyz, *nrm, *w;
    int64_t N;
    olevel lv[OR_MAXD + 1];
    double As[32 * 32], Aa[32 * 32];
    double ts[32], ta[32];
} otree;

static int find_box(const olevel *L, int i, int j, int k) {
    int n = 1 << 20;
    if (i < 0 || j < 0 || k < 0 || i >= n || j >= n || k >= n) return -1;
    int64_t key = make_key(i, j, k);
    int lo = 0, hi = L->nbox - 1;
    while (lo <= hi) {
        int mid = (lo + hi) / 2;
        if (L->key[mid] == key) return mid;
        if (L->key[mid] < key) lo = mid + 1; else hi = mid - 1;
    }
    return -1;
}

/* boxes of level d: B(y0, H_d) half-open cubes (Eq. box), relevant boxes only (Eq. RelevantBoxes) */
static void build_level(otree *T, int d) {
    olevel *L = &T->lv[d];
    int64_t N = T->N;
    L->H = ldexp(T->L, -(d - 1));
    L->h = sqrt(3.0) / 2.0 * L->H;
    int nside = 1 << (d - 1);
    keyidx *ki = (keyidx *)malloc(sizeof(keyidx) * N);
    for (int64_t i = 0; i < N; i++) {
        int b[3];
        for (int a = 0; a < 3; a++) {
            double f = floor((T->xyz[3 * i + a] - (T->c0[a] - 0.5 * T->L)) / L->H);
            int v = (int)f;
            if (v < 0) v = 0;
            if (v > nside - 1) v = nside - 1;
            b[a] = v;
        }
        ki[i].key = make_key(b[0], b[1], b[2]);
        ki[i].idx = (int)i;
    }
    qsort(ki, N, sizeof(keyidx), cmp_keyidx);
    int nb = 0;
    for (int64_t i = 0; i < N; i++)
        if (i == 0 || ki[i].key != ki[i - 1].key) nb++;
    L->nbox = nb;
    L->key = (int64_t *)malloc(sizeof(int64_t) * nb);
    L->ijk = (int *)malloc(sizeof(int) * 3 * nb);
    L->pstart = (int *)malloc(sizeof(int) * nb);
    L->pcount = (int *)calloc(nb, sizeof(int));
    L->perm = (int *)malloc(sizeof(int) * N);
    int b = -1;
    for (int64_t i = 0; i < N; i++) {
        if (i == 0 || ki[i].key != ki[i - 1].key) {
            b++;
            L->key[b] = ki[i].key;
            L->ijk[3 * b + 0] = (int)(ki[i].key >> 42);
            L->ijk[3 * b + 1] = (int)((ki[i].key >> 21) & ((1 << 21) - 1));
            L->ijk[3 * b + 2] = (int)(ki[i].key & ((1 << 21) - 1));
            L->pstart[b] = (int)i;
        }
        L->pcount[b]++;
        L->perm[i] = ki[i].idx;
    }
    free(ki);
}

static void box_center(const otree *T, int d, int b, double *y0) {
    const olevel *L = &T->lv[d];
    for (int a = 0; a < 3; a++) y0[a] = T->c0[a] - 0.5 * T->L + (L->ijk[3 * b + a] + 0.5) * L->H;
}

/* cousins M B (Eq. NeighborsCousins): relevant non-neighbours whose parent neighbours B's parent */
static void build_cousins(otree *T, int d) {
    olevel *L = &T->lv[d];
    L->co_start = (int *)malloc(sizeof(int) * (L->nbox + 1));
    int cap = L->nbox * 216 + 1;
    int *tmp = (int *)malloc(sizeof(int) * cap);
    int n = 0;
    for (int b = 0; b < L->nbox; b++) {
        L->co_start[b] = n;
        const int *q = L->ijk + 3 * b;
        int p[3] = {q[0] >> 1, q[1] >> 1, q[2] >> 1};
        for (int o0 = -1; o0 <= 1; o0++)
            for (int o1 = -1; o1 <= 1; o1++)
                for (int o2 = -1; o2 <= 1; o2++)
                    for (int ch = 0; ch < 8; ch++) {
                        int j0 = 2 * (p[0] + o0) + (ch & 1), j1 = 2 * (p[1] + o1) + ((ch >> 1) & 1),
                            j2 = 2 * (p[2] + o2) + ((ch >> 2) & 1);
                        int dm = abs(j0 - q[0]);
                        if (abs(j1 - q[1]) > dm) dm = abs(j1 - q[1]);
                        if (abs(j2 - q[2]) > dm) dm = abs(j2 - q[2]);
                        if (dm <= 1) continue; /* neighbour */
                        int c = find_box(L, j0, j1, j2);
                        if (c >= 0) tmp[n++] = c;
                    }
    }
    L->co_start[L->nbox] = n;
    L->co_list = (int *)malloc(sizeof(int) * (n > 0 ? n : 1));
    memcpy(L->co_list, tmp, sizeof(int) * n);
    free(tmp);
}

/* ------------------------------------------------------------------------- */
/* cone segments (Eq. deltas, Eq. ConeIntervals, Eq. ConeSegmentSet)          */

static double snap_boundary(double u) {
    double r = nearbyint(u);
    return fabs(u - r) <= 1e-12 * (fabs(u) > 1.0 ? fabs(u) : 1.0) ? r : u;
}

/* Classify x in the cone grid of box b (level d): returns cone id and the local
 * interpolation coordinates t in [-1, 1]^3 (s, theta, phi). */
static int classify(const otree *T, int d, int b, const double *x, double *t3) {
    const olevel *L = &T->lv[d];
    double y0[3];
    box_center(T, d, b, y0);
    double dx = x[0] - y0[0], dy = x[1] - y0[1], dz = x[2] - y0[2];
    double r = sqrt(dx * dx + dy * dy + dz * dz);
    double s = L->h / r;
    double th = atan2(sqrt(dx * dx + dy * dy), dz);
    double ph = atan2(dy, dx);
    if (ph < 0) ph += 2.0 * OR_PI;
    if (ph >= 2.0 * OR_PI) ph = 0.0;
    /* a coordinate within 1e-12 (relative) of a cone boundary is placed on it, so the
     * interval owning a boundary point (the upper one) does not depend on last-bit rounding */
    double us = snap_boundary(s / L->ds), ut = snap_boundary(th / L->dth), up = snap_boundary(ph / L->dph);
    int is = (int)floor(us), it = (int)floor(ut), ip = (int)floor(up);
    if (is > L->ns - 1) is = L->ns - 1;
    if (it > L->nC - 1) it = L->nC - 1;
    if (ip > L->nph - 1) ip = L->nph - 1;
    if (is < 0) is = 0;
    if (it < 0) it = 0;
    if (ip < 0) ip = 0;
    if (t3) {
        t3[0] = 2.0 * (us - is) - 1.0;
        t3[1] = 2.0 * (ut - it) - 1.0;
        t3[2] = 2.0 * (up - ip) - 1.0;
    }
    return (is * L->nC + it) * L->nph + ip;
}

/* Position of interpolation node n of cone `cone` of box b at level d
 * (Eq. defparametrizationins / Eq. defparametrizationr). */
static void node_position(const otree *T, int d, int b, int cone, int n, double *x) {
    const olevel *L = &T->lv[d];
    int ip = cone % L->nph, it = (cone / L->nph) % L->nC, is = cone / (L->nph * L->nC);
    int na = T->Pang;
    int a = n / (na * na), bb = (n / na) % na, c = n % na;
    double s = (is + 0.5 * (T->ts[a] + 1.0)) * L->ds;
    double th = (it + 0.5 * (T->ta[bb] + 1.0)) * L->dth;
    double ph = (ip + 0.5 * (T->ta[c] + 1.0)) * L->dph;
    double y0[3];
    box_center(T, d, b, y0);
    double r = L->h / s;
    x[0] = y0[0] + r * sin(th) * cos(ph);
    x[1] = y0[1] + r * sin(th) * sin(ph);
    x[2] = y0[2] + r * cos(th);
}

static int rc_find(const olevel *L, int b, int cone) {
    int lo = L->rc_start[b], hi = L->rc_start[b + 1] - 1;
    while (lo <= hi) {
        int mid = (lo + hi) / 2;
        if (L->rc_ids[mid] == cone) return mid;
        if (L->rc_ids[mid] < cone) lo = mid + 1; else hi = mid - 1;
    }
    return -1;
}

/* relevant cone segments R_C B (Eq. RelevantCones), built from d = 3 towards D */
static void build_relevant_cones(otree *T, int d) {
    olevel *L = &T->lv[d];
    int P = T->P;
    int **ids = (int **)malloc(sizeof(int *) * L->nbox);
    int *cnt = (int *)calloc(L->nbox, sizeof(int));
#pragma omp parallel for schedule(dynamic, 1)
    for (int b = 0; b < L->nbox; b++) {
        if (!L->alive[b]) { /* below a leaf: no factor, no cones */
            ids[b] = (int *)malloc(sizeof(int));
            cnt[b] = 0;
            continue;
        }
        int64_t cap = 0;
        for (int c = L->co_start[b]; c < L->co_start[b + 1]; c++) cap += L->pcount[L->co_list[c]];
        int pb = -1;
        if (d > 3) {
            pb = L->parent[b];
            const olevel *PL = &T->lv[d - 1];
            cap += (int64_t)(PL->rc_start[pb + 1] - PL->rc_start[pb]) * P;
        }
        const int ffar = d == 3 && T->far_field;
        if (ffar) cap += (int64_t)L->nC * L->nph;
        int *v = (int *)malloc(sizeof(int) * (cap > 0 ? cap : 1));
        int64_t n = 0;
        /* far field: s = h / r -> 0 lies in the segments with is = 0, in every direction */
        if (ffar)
            for (int c = 0; c < L->nC * L->nph; c++) v[n++] = c;
        for (int c = L->co_start[b]; c < L->co_start[b + 1]; c++) {
            int cb = L->co_list[c];
            if (!L->alive[cb]) continue; /* points below a coarser leaf take no level-d interpolation */
            for (int i = 0; i < L->pcount[cb]; i++) {
                int pt = L->perm[L->pstart[cb] + i];
                v[n++] = classify(T, d, b, T->xyz + 3 * pt, NULL);
            }
        }
        if (d > 3) {
            const olevel *PL = &T->lv[d - 1];
            for (int rc = PL->rc_start[pb]; rc < PL->rc_start[pb + 1]; rc++)
                for (int nn = 0; nn < P; nn++) {
                    double x[3];
                    node_position(T, d - 1, pb, PL->rc_ids[rc], nn, x);
                    v[n++] = classify(T, d, b, x, NULL);
                }
        }
        qsort(v, n, sizeof(int), cmp_int);
        int u = 0;
        for (int64_t i = 0; i < n; i++)
            if (i == 0 || v[i] != v[i - 1]) v[u++] = v[i];
        ids[b] = v;
        cnt[b] = u;
    }
    L->rc_start = (int *)malloc(sizeof(int) * (L->nbox + 1));
    int64_t tot = 0;
    for (int b = 0; b < L->nbox; b++) {
        L->rc_start[b] = (int)tot;
        tot += cnt[b];
    }
    L->rc_start[L->nbox] = (int)tot;
    L->nrc = tot;
    L->rc_ids = (int *)malloc(sizeof(int) * (tot > 0 ? tot : 1));
    for (int b = 0; b < L->nbox; b++) {
        memcpy(L->rc_ids + L->rc_start[b], ids[b], sizeof(int) * cnt[b]);
        free(ids[b]);
    }
    free(ids);
    free(cnt);
}

/* ------------------------------------------------------------------------- */
/* analytic factors (Eq. V3, Eq. W2W2, Eq. w23)                               */

/* Factors at target x for source y (normal ny) in the box with centre y0 and
 * half-diagonal h, for the kernel of `layer`: the double layer dPhi/dnu = E_2 W2 + E_1 (-i k W3) with
 * E_1 W~2 = E_2 W2 (W~2 = (s/h) W2), the single layer Phi = E_1 W1 (Eq. V3, Eq. W2W2, Eq. w23).
 * split = 0: out[0] is the one q = 1 factor (combined field W~2 - i k W3 - i eta W1, double layer
 * W~2 - i k W3, single layer W1); split = 1: out[0] the q = 2 factor (W2, W2, 0) and out[1] the q = 1
 * factor (-i k W3 - i eta W1, -i k W3, W1). */
static void wfactors_layer(int layer, double k, double eta, const double *x, const double *y0, double h,
                           const double *y, const double *ny, int split, cplx *out) {
    double dx[3] = {x[0] - y0[0], x[1] - y0[1], x[2] - y0[2]};
    double r = sqrt(dx[0] * dx[0] + dx[1] * dx[1] + dx[2] * dx[2]);
    double s = h / r;
    double u[3] = {dx[0] / r, dx[1] / r, dx[2] / r};
    double yv[3] = {y[0] - y0[0], y[1] - y0[1], y[2] - y0[2]};
    double dv[3] = {u[0] - yv[0] / r, u[1] - yv[1] / r, u[2] - yv[2] / r}; /* u - v s */
    double a = sqrt(dv[0] * dv[0] + dv[1] * dv[1] + dv[2] * dv[2]);
    double yy = yv[0] * yv[0] + yv[1] * yv[1] + yv[2] * yv[2];
    double uy = u[0] * yv[0] + u[1] * yv[1] + u[2] * yv[2];
    double psi = k * (s * yy / h - 2.0 * uy) / (a + 1.0);
    cplx e = cexp(I * psi);
    double dn = dv[0] * ny[0] + dv[1] * ny[1] + dv[2] * ny[2];
    cplx W1 = e / a, W3 = e * dn / (a * a), W2 = e * dn / (a * a * a);
    const cplx sl = W1;                       /* single layer, q = 1 */
    const cplx dl2 = W2, dl1 = -I * k * W3;   /* double layer: q = 2 and q = 1 parts */
    cplx q2, q1;
    if (layer == 2) {
        q2 = 0.0;
        q1 = sl;
    } else if (layer == 1) {
        q2 = dl2;
        q1 = dl1;
    } else {
        q2 = dl2;
        q1 = dl1 - I * eta * sl;
    }
    if (split) {
        out[0] = q2;
        out[1] = q1;
    } else {
        out[0] = (s / h) * q2 + q1;
    }
}

static void wfactors(double k, double eta, const double *x, const double *y0, double h, const double *y,
                     const double *ny, int split, cplx *out) {
    wfactors_layer(0, k, eta, x, y0, h, y, ny, split, out);
}

/* Same factors with the literal phase k (h/s)(|u - v s| - 1) (tests compare the two forms). */
void oracle_wfactors(double k, double eta, const double *x, const double *y0, double h, const double *y,
                     const double *ny, int split, int literal, double *out) {
    cplx o[2] = {0, 0};
    if (!literal) {
        wfactors(k, eta, x, y0, h, y, ny, split, o);
    } else {
        double dx[3] = {x[0] - y0[0], x[1] - y0[1], x[2] - y0[2]};
        double r = sqrt(dx[0] * dx[0] + dx[1] * dx[1] + dx[2] * dx[2]);
        double s = h / r;
        double dv[3];
        for (int a = 0; a < 3; a++) dv[a] = dx[a] / r - (y[a] - y0[a]) / h * s;
        double a = sqrt(dv[0] * dv[0] + dv[1] * dv[1] + dv[2] * dv[2]);
        cplx e = cexp(I * k * (h / s) * (a - 1.0));
        double dn = dv[0] * ny[0] + dv[1] * ny[1] + dv[2] * ny[2];
        cplx W1 = e / a, W3 = e * dn / (a * a), W2 = e * dn / (a * a * a);
        if (split) {
            o[0] = W2;
            o[1] = -I * k * W3 - I * eta * W1;
        } else {
            o[0] = (s / h) * W2 - I * k * W3 - I * eta * W1;
        }
    }
    out[0] = creal(o[0]); out[1] = cimag(o[0]);
    out[2] = creal(o[1]); out[3] = cimag(o[1]);
}

/* centred factor E_q(x; y0) = e^{i k r} / (4 pi r^q) (Eq. cent_fact) */
static cplx centred(double k, const double *x, const double *y0, int q) {
    double d0 = x[0] - y0[0], d1 = x[1] - y0[1], d2 = x[2] - y0[2];
    double r = sqrt(d0 * d0 + d1 * d1 + d2 * d2);
    return cexp(I * k * r) / (4.0 * OR_PI * (q == 2 ? r * r : r));
}

/* ------------------------------------------------------------------------- */

static int nfac_of(const olevel *L) { return L->split ? 2 : 1; }

/* F / C layout: [rc][fac][rhs][P] */
static int64_t fidx(const otree *T, const olevel *L, int64_t rc, int fac, int q) {
    return ((rc * L->nfac + fac) * T->nrhs + q) * T->P;
}

/* Chebyshev coefficients of all relevant cones of level d (tensor-product transform) */
static void level_coefficients(otree *T, int d) {
    olevel *L = &T->lv[d];
    int Ps = T->Ps, Pa = T->Pang, P = T->P;
    int64_t nv = L->nrc * L->nfac * T->nrhs;
#pragma omp parallel for schedule(static)
    for (int64_t v = 0; v < nv; v++) {
        const cplx *f = L->F + v * P;
        cplx *c = L->C + v * P;
        for (int i = 0; i < Ps; i++)
            for (int j = 0; j < Pa; j++)
                for (int l = 0; l < Pa; l++) {
                    cplx acc = 0.0;
                    for (int a = 0; a < Ps; a++)
                        for (int b = 0; b < Pa; b++)
                            for (int cc = 0; cc < Pa; cc++)
                                acc += T->As[i * Ps + a] * T->Aa[j * Pa + b] * T->Aa[l * Pa + cc] *
                                       f[(a * Pa + b) * Pa + cc];
                    c[(i * Pa + j) * Pa + l] = acc;
                }
    }
}

static cplx cheb_eval3(const otree *T, const cplx *c, const double *t3) {
    double Ts[32], Tt[32], Tp[32];
    cheb_T(t3[0], T->Ps, Ts);
    cheb_T(t3[1], T->Pang, Tt);
    cheb_T(t3[2], T->Pang, Tp);
    int Pa = T->Pang;
    cplx acc = 0.0;
    for (int i = 0; i < T->Ps; i++)
        for (int j = 0; j < Pa; j++)
            for (int l = 0; l < Pa; l++) acc += c[(i * Pa + j) * Pa + l] * Ts[i] * Tt[j] * Tp[l];
    return acc;
}

/* Interpolated field of box b (level d) at x, multiplied by its centred factors:
 * sum_j E_j(x; y_b) Interp(F_{b,j})(x), one value per rhs.  Returns 0 on success. */
static int field_from_box(const otree *T, int d, int b, const double *x, cplx *res) {
    const olevel *L = &T->lv[d];
    double t3[3];
    int cone = classify(T, d, b, x, t3);
    int rc = rc_find(L, b, cone);
    if (rc < 0) return -1;
    double y0[3];
    box_center(T, d, b, y0);
    for (int q = 0; q < T->nrhs; q++) {
        if (L->split) {
            cplx v2 = cheb_eval3(T, L->C + fidx(T, L, rc, 0, q), t3);
            cplx v13 = cheb_eval3(T, L->C + fidx(T, L, rc, 1, q), t3);
            res[q] = centred(T->k, x, y0, 2) * v2 + centred(T->k, x, y0, 1) * v13;
        } else {
            res[q] = centred(T->k, x, y0, 1) * cheb_eval3(T, L->C + fidx(T, L, rc, 0, q), t3);
        }
    }
    return 0;
}

static void free_tree(otree *T) {
    for (int d = 1; d <= T->D; d++) {
        olevel *L = &T->lv[d];
        free(L->key); free(L->ijk); free(L->pstart); free(L->pcount); free(L->perm); free(L->parent);
        free(L->alive); free(L->leaf);
        free(L->co_start); free(L->co_list); free(L->rc_start); free(L->rc_ids); free(L->F); free(L->C);
    }
}

static int count_boxes(const double *xyz, int64_t N, const double *c0, double L, int d) {
    double H = ldexp(L, -(d - 1));
    int nside = 1 << (d - 1);
    int64_t *keys = (int64_t *)malloc(sizeof(int64_t) * N);
    for (int64_t i = 0; i < N; i++) {
        int b[3];
        for (int a = 0; a < 3; a++) {
            int v = (int)floor((xyz[3 * i + a] - (c0[a] - 0.5 * L)) / H);
            if (v < 0) v = 0;
            if (v > nside - 1) v = nside - 1;
            b[a] = v;
        }
        keys[i] = make_key(b[0], b[1], b[2]);
    }
    keyidx *ki = (keyidx *)malloc(sizeof(keyidx) * N);
    for (int64_t i = 0; i < N; i++) { ki[i].key = keys[i]; ki[i].idx = 0; }
    qsort(ki, N, sizeof(keyidx), cmp_keyidx);
    int nb = 0;
    for (int64_t i = 0; i < N; i++)
        if (i == 0 || ki[i].key != ki[i - 1].key) nb++;
    free(ki);
    free(keys);
    return nb;
}

/* automatic level count: argmin_{d >= 3} |log(N / #relevant level-d boxes / leaf_target)| */
int oracle_auto_levels(int64_t N, const double *xyz, double leaf_target) {
    double c0[3];
    double L = root_side_of(N, xyz, c0);
    double lt = leaf_target > 0 ? leaf_target : 64.0;
    double best = INFINITY;
    int D = 3;
    for (int d = 3; d <= 16; d++) {
        int nb = count_boxes(xyz, N, c0, L, d);
        double m = fabs(log((double)N / nb / lt));
        if (m < best) { best = m; D = d; }
        if ((double)N / nb < lt / 16.0) break;
    }
    return D;
}

/* ------------------------------------------------------------------------- */
/* IFGF apply (Section 3.4)                                                   */
/*                                                                           */
/* The method splits the sum of Eq. field1 into level-D neighbour pairs,     */
/* summed directly, and, for every level d = D..3, pairs (x, B) of a box B   */
/* and a point x in one of B's cousin boxes (Eq. NeighborsCousins).  For the  */
/* latter the field of B's sources at x is the centred factor E(x; y_B)      */
/* (Eq. cent_fact) times an analytic factor F_B that is interpolated in the  */
/* spherical cone segment around y_B containing x (Section 3.2, Eq.          */
/* ChebyPoly).  F_B is known exactly only at the leaf level; coarser boxes   */
/* obtain it at their interpolation points from their children's             */
/* interpolants, re-centred from child to parent.  The stages below follow   */
/* that order: structure, leaf expansions, one pass per level from the       */
/* finest to level 3, near field, identity term.                              */

/* Octree, cone grids (Remark cone_seg_size) and relevant cone segments (Eq.
 * RelevantCones) for the given parameters; allocates the per-level F and C. */
static int setup_tree(otree *T, const oracle_params *prm, int64_t N, const double *xyz, const double *nrm,
                      const double *w, int nrhs) {
    T->N = N; T->xyz = xyz; T->nrm = nrm; T->w = w; T->nrhs = nrhs;
    T->k = prm->k; T->eta = prm->eta; T->Ps = prm->Ps; T->Pang = prm->Pang; T->P = prm->Ps * prm->Pang * prm->Pang;
    T->far_field = prm->far_field != 0;
    T->layer = prm->layer;
    T->leaf_max = prm->leaf_max > 0 ? prm->leaf_max : 0;
    if (prm->root_side > 0) {
        T->L = prm->root_side;
        for (int a = 0; a < 3; a++) T->c0[a] = prm->root_center[a];
    } else {
        T->L = root_side_of(N, xyz, T->c0);
    }
    /* level count */
    int D = prm->levels;
    if (D <= 0) {
        double lt = prm->leaf_target > 0 ? prm->leaf_target : 64.0;
        double best = INFINITY;
        D = 3;
        for (int d = 3; d <= 16; d++) {
            int nb = count_boxes(xyz, N, T->c0, T->L, d);
            double m = fabs(log((double)N / nb / lt));
            if (m < best) { best = m; D = d; }
            if ((double)N / nb < lt / 16.0) break;
        }
    }
    if (D < 3 || D > 16) return -1;
    T->D = D;
    for (int i = 0; i < T->Ps; i++) T->ts[i] = cheb_node(i, T->Ps);
    for (int i = 0; i < T->Pang; i++) T->ta[i] = cheb_node(i, T->Pang);
    cheb_coeff_matrix(T->Ps, T->As);
    cheb_coeff_matrix(T->Pang, T->Aa);

    double lam = 2.0 * OR_PI / T->k;
    for (int d = 1; d <= D; d++) build_level(T, d);
    for (int d = 2; d <= D; d++) {
        olevel *L = &T->lv[d];
        L->parent = (int *)malloc(sizeof(int) * L->nbox);
        for (int b = 0; b < L->nbox; b++)
            L->parent[b] = find_box(&T->lv[d - 1], L->ijk[3 * b] >> 1, L->ijk[3 * b + 1] >> 1, L->ijk[3 * b + 2] >> 1);
    }
    /* adaptive octree: level-3 boxes exist; a box with at most leaf_max points (or at level D) is a
     * leaf; the boxes below a leaf do not exist */
    for (int d = 3; d <= D; d++) {
        olevel *L = &T->lv[d];
        L->alive = (unsigned char *)malloc(L->nbox > 0 ? L->nbox : 1);
        L->leaf = (unsigned char *)malloc(L->nbox > 0 ? L->nbox : 1);
        for (int b = 0; b < L->nbox; b++) {
            const olevel *PL = &T->lv[d - 1];
            L->alive[b] = d == 3 ? 1 : (PL->alive[L->parent[b]] && !PL->leaf[L->parent[b]]);
            L->leaf[b] = L->alive[b] && (d == D || (T->leaf_max > 0 && L->pcount[b] <= T->leaf_max));
        }
    }
    /* cone grid per level (Remark cone_seg_size) */
    int e_lit = 0;
    for (int d = D; d >= 3; d--) {
        olevel *L = &T->lv[d];
        int e = 0;
        if (prm->cone_rule == 0) {
            while (L->H > ldexp(0.5 * lam, e)) e++;
        } else {
            if (d < D && T->k * T->lv[d + 1].H > 0.5) e_lit++;
            e = e_lit;
        }
        L->ns = prm->nS0 << e;
        L->nC = prm->nC0 << e;
        L->nph = 2 * L->nC;
        L->ncone = L->ns * L->nC * L->nph;
        L->ds = (sqrt(3.0) / 3.0) / L->ns;
        L->dth = OR_PI / L->nC;
        L->dph = OR_PI / L->nC;
        if (prm->factor_mode == 1) L->split = 0;
        else if (prm->factor_mode == 2) L->split = 1;
        else L->split = (L->H < 0.5 * lam) ? 1 : 0;
        L->nfac = nfac_of(L);
    }
    for (int d = 3; d <= D; d++) build_cousins(T, d);
    for (int d = 3; d <= D; d++) build_relevant_cones(T, d);
    for (int d = 3; d <= D; d++) {
        olevel *L = &T->lv[d];
        int64_t sz = L->nrc * L->nfac * nrhs * T->P;
        L->F = (cplx *)calloc(sz > 0 ? sz : 1, sizeof(cplx));
        L->C = (cplx *)calloc(sz > 0 ? sz : 1, sizeof(cplx));
    }
    return 0;
}

/* Leaf expansions: at every interpolation point x of every relevant cone segment of every
 * level-D box, F(x) = sum over the box's sources y of w_y sigma_y W(x, y) with the analytic
 * factor W of Eq. V3 / Eq. W2W2 / Eq. w23 (the combined factor or the split pair). */
static int64_t stage_leaf_expansions(otree *T, const cplx *sg) {
    const int64_t N = T->N;
    const int nrhs = T->nrhs;
    int64_t leaf_evals = 0;
    for (int D = 3; D <= T->D; D++) { /* every level's leaf boxes (only level D in a uniform tree) */
    olevel *L = &T->lv[D];
#pragma omp parallel for schedule(dynamic, 1) reduction(+ : leaf_evals)
    for (int b = 0; b < L->nbox; b++) {
        if (!L->leaf[b]) continue;
        double y0[3];
        box_center(T, D, b, y0);
        for (int rc = L->rc_start[b]; rc < L->rc_start[b + 1]; rc++)
            for (int nn = 0; nn < T->P; nn++) {
                double x[3];
                node_position(T, D, b, L->rc_ids[rc], nn, x);
                for (int i = 0; i < L->pcount[b]; i++) {
                    int m = L->perm[L->pstart[b] + i];
                    cplx W[2];
                    wfactors_layer(T->layer, T->k, T->eta, x, y0, L->h, T->xyz + 3 * m, T->nrm + 3 * m, L->split, W);
                    for (int fc = 0; fc < L->nfac; fc++)
                        for (int q = 0; q < nrhs; q++)
                            L->F[fidx(T, L, rc, fc, q) + nn] += T->w[m] * sg[(int64_t)q * N + m] * W[fc];
                    leaf_evals++;
                }
            }
    }
    }
    return leaf_evals;
}

/* Re-centre the child box's interpolated factor at point x (a parent interpolation point)
 * onto the parent: ratio of centred factors E(x; y_child) / E(x; y_parent) of Eq. cent_fact,
 * per factor when both levels store the split pair, through the child's field otherwise. */
static void recentre_to_parent(const otree *T, const olevel *CL, olevel *PL, int crc, const double *t3,
                               const double *x, const double *yc, const double *yp, int rc, int nn) {
    for (int q = 0; q < T->nrhs; q++) {
        if (CL->split && PL->split) {
            cplx v2 = cheb_eval3(T, CL->C + fidx(T, CL, crc, 0, q), t3);
            cplx v13 = cheb_eval3(T, CL->C + fidx(T, CL, crc, 1, q), t3);
            PL->F[fidx(T, PL, rc, 0, q) + nn] += v2 * centred(T->k, x, yc, 2) / centred(T->k, x, yp, 2);
            PL->F[fidx(T, PL, rc, 1, q) + nn] += v13 * centred(T->k, x, yc, 1) / centred(T->k, x, yp, 1);
        } else if (CL->split) {
            cplx v2 = cheb_eval3(T, CL->C + fidx(T, CL, crc, 0, q), t3);
            cplx v13 = cheb_eval3(T, CL->C + fidx(T, CL, crc, 1, q), t3);
            PL->F[fidx(T, PL, rc, 0, q) + nn] +=
                (centred(T->k, x, yc, 2) * v2 + centred(T->k, x, yc, 1) * v13) / centred(T->k, x, yp, 1);
        } else {
            cplx v = cheb_eval3(T, CL->C + fidx(T, CL, crc, 0, q), t3);
            PL->F[fidx(T, PL, rc, 0, q) + nn] += v * centred(T->k, x, yc, 1) / centred(T->k, x, yp, 1);
        }
    }
}

/* One level d of the recursion, for every box B of the level: (a) the factor's interpolant
 * (Chebyshev coefficients of Eq. ChebyCoeffs per cone segment) evaluated at each point x in
 * B's cousin boxes and multiplied by E(x; y_B), added to the field u at x; (b) above level 3,
 * the same interpolant evaluated at every interpolation point of the parent's relevant cone
 * segments and re-centred onto the parent (recentre_to_parent), accumulated into the parent's
 * F.  Returns nonzero if a point falls outside the relevant segments (cannot happen for a
 * consistent tree). */
static int stage_level(otree *T, int d, cplx *u, int64_t *n_cousin, int64_t *n_parent) {
    const int64_t N = T->N;
    const int nrhs = T->nrhs;
    olevel *L = &T->lv[d];
    level_coefficients(T, d);
    int64_t nce = 0, npe = 0;
    int err = 0;
    int *plist = (int *)malloc(sizeof(int) * N);
    for (int b = 0; b < L->nbox && !err; b++) {
        if (!L->alive[b]) continue;
        /* (a) cousin points of B (Eq. NeighborsCousins) that have a level-d box; skipped when u is NULL */
        int np = 0;
        for (int c = L->co_start[b]; u && c < L->co_start[b + 1]; c++) {
            int cb = L->co_list[c];
            if (!L->alive[cb]) continue;
            for (int i = 0; i < L->pcount[cb]; i++) plist[np++] = L->perm[L->pstart[cb] + i];
        }
        int lerr = 0;
#pragma omp parallel for schedule(static) reduction(| : lerr)
        for (int i = 0; i < np; i++) {
            int pt = plist[i];
            cplx res[64];
            if (field_from_box(T, d, b, T->xyz + 3 * pt, res)) { lerr |= 1; continue; }
            for (int q = 0; q < nrhs; q++) u[(int64_t)q * N + pt] += res[q];
        }
        nce += np;
        if (lerr) err = 1;
        /* (b) the parent's interpolation points */
        if (d > 3 && !err) {
            olevel *PL = &T->lv[d - 1];
            int pb = L->parent[b];
            double yp[3], yc[3];
            box_center(T, d - 1, pb, yp);
            box_center(T, d, b, yc);
            int r0 = PL->rc_start[pb], r1 = PL->rc_start[pb + 1];
            int64_t nw = (int64_t)(r1 - r0) * T->P;
#pragma omp parallel for schedule(static) reduction(| : lerr)
            for (int64_t wi = 0; wi < nw; wi++) {
                int rc = r0 + (int)(wi / T->P), nn = (int)(wi % T->P);
                double x[3], t3[3];
                node_position(T, d - 1, pb, PL->rc_ids[rc], nn, x);
                int crc = rc_find(L, b, classify(T, d, b, x, t3));
                if (crc < 0) { lerr |= 1; continue; }
                recentre_to_parent(T, L, PL, crc, t3, x, yc, yp, rc, nn);
            }
            npe += nw;
            if (lerr) err = 1;
        }
    }
    free(plist);
    *n_cousin = nce;
    *n_parent = npe;
    return err;
}

/* Near field of the adaptive octree.  A target in a leaf of level d_t and a source in a leaf of
 * level d_s interact directly when their boxes at level m = min(d_t, d_s) are neighbours (or the
 * same box); every other pair is carried by exactly one cousin interpolation (the level at which
 * their boxes stop being neighbours is at most m).  In a uniform tree m = D and this is the
 * 27-neighbourhood rule of stage_near_field.  Direct summation as there. */
static int64_t stage_near_field_adaptive(const otree *T, const cplx *sg, cplx *u) {
    const int D = T->D;
    const int64_t N = T->N;
    const int nrhs = T->nrhs;
    const double tol = 1e-14 * T->L;
    /* per point: level-D cell and leaf level */
    int *cell = (int *)malloc(sizeof(int) * 3 * N), *lev = (int *)malloc(sizeof(int) * N);
    const olevel *LD = &T->lv[D];
    for (int b = 0; b < LD->nbox; b++)
        for (int i = 0; i < LD->pcount[b]; i++) {
            const int pt = LD->perm[LD->pstart[b] + i];
            for (int a = 0; a < 3; a++) cell[3 * pt + a] = LD->ijk[3 * b + a];
        }
    for (int d = 3; d <= D; d++) {
        const olevel *L = &T->lv[d];
        for (int b = 0; b < L->nbox; b++)
            if (L->leaf[b])
                for (int i = 0; i < L->pcount[b]; i++) lev[L->perm[L->pstart[b] + i]] = d;
    }
    int64_t near_pairs = 0;
#pragma omp parallel for schedule(dynamic, 64) reduction(+ : near_pairs)
    for (int64_t l = 0; l < N; l++) {
        for (int64_t m = 0; m < N; m++) {
            if (m == l) continue;
            const int lv = lev[l] < lev[m] ? lev[l] : lev[m], sh = D - lv;
            int nbr = 1;
            for (int a = 0; a < 3; a++) {
                const int dd = (cell[3 * l + a] >> sh) - (cell[3 * m + a] >> sh);
                if (dd < -1 || dd > 1) nbr = 0;
            }
            if (!nbr) continue;
            const double *x = T->xyz + 3 * l, *y = T->xyz + 3 * m;
            double d0 = x[0] - y[0], d1 = x[1] - y[1], d2 = x[2] - y[2];
            near_pairs++;
            if (sqrt(d0 * d0 + d1 * d1 + d2 * d2) < tol) continue;
            cplx K = layer_kernel(T->layer, T->k, T->eta, x, y, T->nrm + 3 * m) * T->w[m];
            for (int qq = 0; qq < nrhs; qq++) u[(int64_t)qq * N + l] += K * sg[(int64_t)qq * N + m];
        }
    }
    free(cell);
    free(lev);
    return near_pairs;
}

/* Level-D neighbour pairs (own box and the 26 adjacent ones) by direct summation of the
 * combined-field kernel (Remark level_D_neighboring), m != l, pairs closer than 1e-14 L
 * dropped.  Returns the number of pairs visited. */
static int64_t stage_near_field(const otree *T, const cplx *sg, cplx *u) {
    if (T->leaf_max > 0) return stage_near_field_adaptive(T, sg, u);
    const int D = T->D;
    const int64_t N = T->N;
    const int nrhs = T->nrhs;
    const olevel *L = &T->lv[D];
    const double tol = 1e-14 * T->L;
    int64_t near_pairs = 0;
#pragma omp parallel for schedule(dynamic, 1) reduction(+ : near_pairs)
    for (int b = 0; b < L->nbox; b++) {
        const int *q3 = L->ijk + 3 * b;
        int nbl[27], nn = 0;
        for (int o0 = -1; o0 <= 1; o0++)
            for (int o1 = -1; o1 <= 1; o1++)
                for (int o2 = -1; o2 <= 1; o2++) {
                    int c = find_box(L, q3[0] + o0, q3[1] + o1, q3[2] + o2);
                    if (c >= 0) nbl[nn++] = c;
                }
        for (int i = 0; i < L->pcount[b]; i++) {
            int l = L->perm[L->pstart[b] + i];
            for (int j = 0; j < nn; j++) {
                int c = nbl[j];
                for (int s = 0; s < L->pcount[c]; s++) {
                    int m = L->perm[L->pstart[c] + s];
                    if (m == l) continue;
                    const double *x = T->xyz + 3 * l, *y = T->xyz + 3 * m;
                    double d0 = x[0] - y[0], d1 = x[1] - y[1], d2 = x[2] - y[2];
                    near_pairs++;
                    if (sqrt(d0 * d0 + d1 * d1 + d2 * d2) < tol) continue;
                    cplx K = layer_kernel(T->layer, T->k, T->eta, x, y, T->nrm + 3 * m) * T->w[m];
                    for (int qq = 0; qq < nrhs; qq++) u[(int64_t)qq * N + l] += K * sg[(int64_t)qq * N + m];
                }
            }
        }
    }
    return near_pairs;
}

/* structural part of oracle_info */
static void tree_info(const otree *T, oracle_info *info) {
    info->D = T->D;
    info->root_side = T->L;
    for (int a = 0; a < 3; a++) info->root_center[a] = T->c0[a];
    for (int d = 1; d <= T->D; d++) {
        info->nbox[d] = T->lv[d].nbox;
        if (d >= 3) {
            info->ns[d] = T->lv[d].ns;
            info->nC[d] = T->lv[d].nC;
            info->split[d] = T->lv[d].split;
            info->nrc[d] = T->lv[d].nrc;
        }
    }
}

int oracle_ifgf(const oracle_params *prm, int64_t N, const double *xyz, const double *nrm, const double *w,
                int nrhs, const double *sigma, double *out, oracle_info *info) {
    if (N <= 0 || nrhs <= 0 || nrhs > 64 || !(prm->k > 0) || prm->Ps < 1 || prm->Pang < 1 || prm->Ps > 31 ||
        prm->Pang > 31)
        return -1;
    otree T;
    memset(&T, 0, sizeof(T));
    if (setup_tree(&T, prm, N, xyz, nrm, w, nrhs)) {
        free_tree(&T);
        return -1;
    }
    const int D = T.D;
    const cplx *sg = (const cplx *)sigma;
    cplx *u = (cplx *)calloc((size_t)N * nrhs, sizeof(cplx));
    int err = 0;
    const int64_t leaf_evals = stage_leaf_expansions(&T, sg);
    for (int d = D; d >= 3 && !err; d--) {
        int64_t nce = 0, npe = 0;
        err = stage_level(&T, d, u, &nce, &npe);
        if (info) {
            info->cousin_evals[d] = nce;
            if (d > 3) info->prop_evals[d - 1] = npe;
        }
    }
    int64_t near_pairs = 0;
    if (!err) near_pairs = stage_near_field(&T, sg, u);
    if (!err) {  /* identity term of Eq. CombLayIE */
        cplx *o = (cplx *)out;
        for (int64_t i = 0; i < N * nrhs; i++) o[i] = prm->identity_coef * sg[i] + u[i];
    }
    if (info) {
        tree_info(&T, info);
        info->leaf_evals = leaf_evals;
        info->near_pairs = near_pairs;
    }
    free(u);
    free_tree(&T);
    return err ? -2 : 0;
}

/* Far-field pattern (Eq. FarField) from the level-3 interpolants.  With x = R xhat the
 * centred factors of Eq. cent_fact satisfy R e^{-ikR} E_1(x; y_B) -> e^{-ik xhat.y_B} / (4 pi)
 * and R e^{-ikR} E_2(x; y_B) -> 0 as R -> infinity, while s = h / |x - y_B| -> 0 and the
 * direction of x - y_B tends to xhat.  The level-3 boxes partition the sources, so
 *   u_inf(xhat) = sum_B e^{-ik xhat.y_B} / (4 pi) Interp(F_B)(s = 0, theta(xhat), phi(xhat)),
 * with F_B the combined factor, or the q = 1 member W13 of the split pair (its W2 member
 * carries E_2 and drops out).  The point s = 0 is the lower end of segment is = 0 (local
 * coordinate -1), which the far-field option keeps relevant at level 3 in every direction.
 * The factors come from the leaf expansions and the propagation of Section 3.4 exactly as
 * in oracle_ifgf; the cousin interpolations and the near field are not needed. */
int oracle_ifgf_far_field(const oracle_params *prm, int64_t N, const double *xyz, const double *nrm,
                          const double *w, int nrhs, const double *sigma, int64_t M, const double *xhat,
                          double *out, oracle_info *info) {
    if (N <= 0 || M < 0 || nrhs <= 0 || nrhs > 64 || !(prm->k > 0) || prm->Ps < 1 || prm->Pang < 1 ||
        prm->Ps > 31 || prm->Pang > 31)
        return -1;
    oracle_params q = *prm;
    q.far_field = 1;
    otree T;
    memset(&T, 0, sizeof(T));
    if (setup_tree(&T, &q, N, xyz, nrm, w, nrhs)) {
        free_tree(&T);
        return -1;
    }
    const cplx *sg = (const cplx *)sigma;
    const int64_t leaf_evals = stage_leaf_expansions(&T, sg);
    int err = 0;
    for (int d = T.D; d >= 3 && !err; d--) {
        int64_t nce = 0, npe = 0;
        err = stage_level(&T, d, NULL, &nce, &npe);
        if (info && d > 3) info->prop_evals[d - 1] = npe;
    }
    const olevel *L = &T.lv[3];
    const int fac = L->split ? 1 : 0;
    cplx *o = (cplx *)out;
    int lerr = 0;
#pragma omp parallel for schedule(static) reduction(| : lerr)
    for (int64_t j = 0; j < (err ? 0 : M); j++) {
        const double *e = xhat + 3 * j;
        /* direction only: theta, phi of xhat on the cone grid, s = 0 */
        double th = atan2(sqrt(e[0] * e[0] + e[1] * e[1]), e[2]);
        double ph = atan2(e[1], e[0]);
        if (ph < 0) ph += 2.0 * OR_PI;
        if (ph >= 2.0 * OR_PI) ph = 0.0;
        double ut = snap_boundary(th / L->dth), up = snap_boundary(ph / L->dph);
        int it = (int)floor(ut), ip = (int)floor(up);
        if (it > L->nC - 1) it = L->nC - 1;
        if (ip > L->nph - 1) ip = L->nph - 1;
        if (it < 0) it = 0;
        if (ip < 0) ip = 0;
        const double t3[3] = {-1.0, 2.0 * (ut - it) - 1.0, 2.0 * (up - ip) - 1.0};
        const int cone = it * L->nph + ip; /* is = 0 */
        cplx acc[64];
        for (int qq = 0; qq < nrhs; qq++) acc[qq] = 0.0;
        for (int b = 0; b < L->nbox; b++) {
            int rc = rc_find(L, b, cone);
            if (rc < 0) { lerr |= 1; continue; }
            double y0[3];
            box_center(&T, 3, b, y0);
            const cplx ph0 = cexp(-I * T.k * (e[0] * y0[0] + e[1] * y0[1] + e[2] * y0[2])) / (4.0 * OR_PI);
            for (int qq = 0; qq < nrhs; qq++) acc[qq] += ph0 * cheb_eval3(&T, L->C + fidx(&T, L, rc, fac, qq), t3);
        }
        for (int qq = 0; qq < nrhs; qq++) o[(int64_t)qq * M + j] = acc[qq];
    }
    if (info) {
        tree_info(&T, info);
        info->leaf_evals = leaf_evals;
    }
    free_tree(&T);
    return (err || lerr) ? -2 : 0;
}

// Rectangular-polar (RP) singular / near-singular correction, host side (Section 4.2).
//
// The surface is the union of Q patches, each carrying the m x m Chebyshev-Gauss nodes of
// Eq. FejersNodes.  For a target x_l and a patch Gamma^q within the proximity distance delta
// of it (Eq. SingGridPts), the patch integral of K(x_l, y) phi(y) is
//   sum_{n,m} a^q_{nm} beta^{q,l}_{nm}                                   (Eq. IntOpAtSing)
// with a^q the Chebyshev coefficients of phi on the patch (Eq. ChebyCoeff) and beta the
// integrals of K T_n T_m J (Eq. BetaAtSing), computed with Fejer's first rule after the
// clustering change of variables xi_alpha (Eq. CoV, Kress map Eq. wMap / Eq. vMap) centred at
// the patch point closest to x_l (Eq. MinNode).  Folding Eq. ChebyCoeff into Eq. IntOpAtSing
// makes the result linear in the nodal values of phi: row l gets, for node (i, j) of the
// patch, c_ij = sum over the graded quadrature of K J l_i(u) l_j(v) w_u w_v, l_i the Lagrange
// basis of the nodes.  The regular Fejer row (Eq. ReguIntOpQuadrature, m != l) that the
// accelerated operator already sums is subtracted, so that
//   y = c_I phi + (regular sum) + C phi
// uses the RP value on the near patches.
//
// The patch map y^q(u, v) is not passed in: it is the tensor Chebyshev interpolant of the
// patch's node positions (degree m - 1 per direction, the representation Section 4.1 uses
// for densities), its normal the normalised y_u x y_v oriented like the caller's normals.
// The closest patch point is found by projected Gauss-Newton from the nearest node.
#include <algorithm>
#include <cmath>
#include <complex>
#include <cstdlib>
#include <cstring>
#include <vector>

#include "ifgf_internal.h"

namespace ifgf {

void clear_error();

namespace {

using cd = std::complex<double>;
constexpr double kPiD = 3.14159265358979323846;

// T_0..T_{n-1}(t) and their derivatives (three-term recurrence).
inline void cheb_vals(int n, double t, double *T, double *dT) {
    T[0] = 1.0;
    dT[0] = 0.0;
    if (n > 1) {
        T[1] = t;
        dT[1] = 1.0;
    }
    for (int k = 2; k < n; k++) {
        T[k] = 2.0 * t * T[k - 1] - T[k - 2];
        dT[k] = 2.0 * T[k - 1] + 2.0 * t * dT[k - 1] - dT[k - 2];
    }
}

// Chebyshev-Gauss nodes (Eq. FejersNodes) and Fejer first-rule weights (Eq. FejersWeights).
void fejer_rule(int J, std::vector<double> &s, std::vector<double> &w) {
    s.resize(J);
    w.resize(J);
    for (int j = 0; j < J; j++) {
        s[j] = std::cos(kPiD * (2.0 * j + 1.0) / (2.0 * J));
        double acc = 0.0;
        for (int l = 1; l <= J / 2; l++) acc += std::cos(l * kPiD * (2.0 * j + 1.0) / J) / (4.0 * l * l - 1.0);
        w[j] = 2.0 / J * (1.0 - 2.0 * acc);
    }
}

// Kress map w(tau; d) of Eq. wMap / Eq. vMap on [0, 2 pi] and its derivative.
inline double kress_nu(double t, double d) {
    const double a = (kPiD - t) / kPiD;
    return (1.0 / d - 0.5) * a * a * a + (1.0 / d) * (t - kPiD) / kPiD + 0.5;
}
inline double kress_dnu(double t, double d) {
    const double a = (kPiD - t) / kPiD;
    return -3.0 / kPiD * (1.0 / d - 0.5) * a * a + 1.0 / (d * kPiD);
}
inline void kress_w(double t, double d, double &w, double &dw) {
    const double n1 = kress_nu(t, d), n2 = kress_nu(2.0 * kPiD - t, d);
    const double A = std::pow(n1, d), B = std::pow(n2, d);
    const double dA = d * std::pow(n1, d - 1.0) * kress_dnu(t, d);
    const double dB = -d * std::pow(n2, d - 1.0) * kress_dnu(2.0 * kPiD - t, d);
    const double S = A + B;
    w = 2.0 * kPiD * A / S;
    dw = 2.0 * kPiD * (dA * B - A * dB) / (S * S);
}

// Change of variables xi_alpha(tau; d) of Eq. CoV, clustering at alpha, and d xi / d tau.
inline void cov(double alpha, double tau, double d, double &xi, double &dxi) {
    double w, dw;
    if (alpha >= 1.0) {
        kress_w(kPiD * std::fabs((tau - 1.0) / 2.0), d, w, dw);
        xi = 1.0 - (2.0 / kPiD) * w;
        dxi = dw;  // d/dtau of -(2/pi) w(pi (1 - tau) / 2)
    } else if (alpha <= -1.0) {
        kress_w(kPiD * std::fabs((tau + 1.0) / 2.0), d, w, dw);
        xi = -1.0 + (2.0 / kPiD) * w;
        dxi = dw;
    } else {
        const double sg = tau > 0 ? 1.0 : (tau < 0 ? -1.0 : 0.0);
        kress_w(kPiD * std::fabs(tau), d, w, dw);
        xi = alpha + (sg - alpha) / kPiD * w;
        dxi = (1.0 - alpha * sg) * dw;
    }
}

// Tensor Chebyshev interpolant of one patch's node positions:
// y_a(u, v) = sum_{n,p} c[(a * m + n) * m + p] T_n(u) T_p(v).
struct PatchMap {
    int m = 0;
    std::vector<double> c;  // 3 m m
    double ctr[3] = {0, 0, 0}, rad = 0;
    double orient = 1.0;    // +-1: sign that makes y_u x y_v point like the caller's normals

    void eval(double u, double v, double *y, double *yu, double *yv, std::vector<double> &tmp) const {
        tmp.resize(4 * (size_t)m);
        double *Tu = tmp.data(), *dTu = Tu + m, *Tv = dTu + m, *dTv = Tv + m;
        cheb_vals(m, u, Tu, dTu);
        cheb_vals(m, v, Tv, dTv);
        for (int a = 0; a < 3; a++) {
            double s = 0, su = 0, sv = 0;
            for (int n = 0; n < m; n++) {
                const double *cr = &c[((size_t)a * m + n) * m];
                double r = 0, rv = 0;
                for (int p = 0; p < m; p++) {
                    r += cr[p] * Tv[p];
                    rv += cr[p] * dTv[p];
                }
                s += Tu[n] * r;
                su += dTu[n] * r;
                sv += Tu[n] * rv;
            }
            y[a] = s;
            yu[a] = su;
            yv[a] = sv;
        }
    }
};

inline void cross(const double *a, const double *b, double *c) {
    c[0] = a[1] * b[2] - a[2] * b[1];
    c[1] = a[2] * b[0] - a[0] * b[2];
    c[2] = a[0] * b[1] - a[1] * b[0];
}
inline double dot3(const double *a, const double *b) { return a[0] * b[0] + a[1] * b[1] + a[2] * b[2]; }

// Combined-field kernel dPhi/dnu(y) - i eta Phi at (x, y, nu) (Eq. GreenFunction, Eq. double_layer);
// zero closer than tol.
inline cd cfie_kernel(double k, double eta, const double *x, const double *y, const double *nu, double tol) {
    const double d[3] = {x[0] - y[0], x[1] - y[1], x[2] - y[2]};
    const double r = std::sqrt(dot3(d, d));
    if (!(r >= tol)) return cd(0.0, 0.0);
    const double a = 1.0 / (4.0 * kPiD * r);
    double sn, cs;
    ::sincos(k * r, &sn, &cs);
    const cd e(a * cs, a * sn);
    return e * (cd(1.0, -k * r) * dot3(d, nu) / (r * r) - cd(0.0, eta));
}

}  // namespace

namespace {

// Closest point of patch P to x (Eq. MinNode): projected Gauss-Newton on |x - y(u, v)|^2
// started at (u0, v0), with coordinates held at the parameter-square boundary while the
// gradient pushes outward.
void closest_point(const PatchMap &P, const double *x, double &u, double &v, std::vector<double> &tmp) {
    double y[3], yu[3], yv[3];
    for (int it = 0; it < 60; it++) {
        P.eval(u, v, y, yu, yv, tmp);
        const double r[3] = {x[0] - y[0], x[1] - y[1], x[2] - y[2]};
        const double gu = dot3(yu, r), gv = dot3(yv, r);
        const double a = dot3(yu, yu), b = dot3(yu, yv), c = dot3(yv, yv);
        const bool fu = (u >= 1.0 && gu > 0) || (u <= -1.0 && gu < 0);  // u held at the boundary
        const bool fv = (v >= 1.0 && gv > 0) || (v <= -1.0 && gv < 0);
        double du = 0, dv = 0;
        if (!fu && !fv) {
            const double det = a * c - b * b;
            if (!(det > 0)) break;
            du = (c * gu - b * gv) / det;
            dv = (a * gv - b * gu) / det;
        } else if (!fu) {
            du = gu / a;
        } else if (!fv) {
            dv = gv / c;
        }
        const double un = std::min(1.0, std::max(-1.0, u + du)), vn = std::min(1.0, std::max(-1.0, v + dv));
        const double step = std::max(std::fabs(un - u), std::fabs(vn - v));
        u = un;
        v = vn;
        if (step < 1e-15) break;
    }
}

}  // namespace

// device quadrature of the (target, near patch) pairs (rp_gpu.cu)
ifgf_status rp_quadrature_device(int m, int nbeta, double k, double eta, double tol, double dgrade,
                                 const std::vector<double> &coef, const std::vector<double> &orient, const double *xyz,
                                 const double *nrm, const double *w, int64_t N, const std::vector<int64_t> &node_pt,
                                 const std::vector<double> &sb, const std::vector<double> &wb,
                                 const std::vector<double> &lag, const std::vector<int64_t> &pl,
                                 const std::vector<int> &pq, const std::vector<double> &puv, cudaStream_t s,
                                 std::vector<double> &out);

// Builds C (CSR over the caller's point order; values complex128 interleaved).  With `device`
// the host finds the near patches and closest points only, and the quadrature of every pair runs
// on the current GPU (rp_quadrature_device) with the same formulas.
static ifgf_status build_rp(const double *xyz, const double *nrm, const double *w, int64_t N, const int32_t *patch_node,
                            int m, double k, double eta, double delta, int nbeta, double dgrade,
                            int64_t **rowptr_out, int32_t **col_out, double **val_out, bool device = false,
                            cudaStream_t stream = nullptr) {
    const int mm = m * m;
    const int64_t Q = N / mm;
    std::vector<int64_t> node_pt((size_t)N, -1);  // (q, i, j) -> caller index
    for (int64_t l = 0; l < N; l++) {
        const int32_t t = patch_node[l];
        if (t < 0 || t >= N || node_pt[t] >= 0) {
            set_error("patch_node must be a permutation of 0..N-1 (entry %lld = %d)", (long long)l, (int)t);
            return IFGF_EINVAL;
        }
        node_pt[t] = l;
    }
    std::vector<double> sm, wm, sb, wb;
    fejer_rule(m, sm, wm);
    fejer_rule(nbeta, sb, wb);
    // alpha_n T_n(s_i) / m: l_i(u) = sum_n lag[i * m + n] T_n(u) (Eq. ChebyCoeff folded in)
    std::vector<double> lag((size_t)mm), Tn(m), dTn(m);
    for (int i = 0; i < m; i++) {
        cheb_vals(m, sm[i], Tn.data(), dTn.data());
        for (int n = 0; n < m; n++) lag[(size_t)i * m + n] = (n == 0 ? 1.0 : 2.0) * Tn[n] / m;
    }
    // root-box side (AABB max extent (1 + 2^-30)) for the kernel cut-off
    double lo[3] = {INFINITY, INFINITY, INFINITY}, hi[3] = {-INFINITY, -INFINITY, -INFINITY};
    for (int64_t l = 0; l < N; l++)
        for (int a = 0; a < 3; a++) {
            lo[a] = std::min(lo[a], xyz[3 * l + a]);
            hi[a] = std::max(hi[a], xyz[3 * l + a]);
        }
    const double L = std::max({hi[0] - lo[0], hi[1] - lo[1], hi[2] - lo[2]}) * (1.0 + std::ldexp(1.0, -30));
    const double tol = 1e-14 * L;

    // patch interpolants (coefficients from the node positions, Eq. ChebyCoeff per coordinate)
    std::vector<PatchMap> P((size_t)Q);
#pragma omp parallel
    {
        std::vector<double> tmp;
        std::vector<double> T(m), dT(m);
#pragma omp for schedule(static)
        for (int64_t q = 0; q < Q; q++) {
            PatchMap &pm = P[q];
            pm.m = m;
            pm.c.assign(3 * (size_t)mm, 0.0);
            for (int i = 0; i < m; i++)
                for (int j = 0; j < m; j++) {
                    const double *y = xyz + 3 * node_pt[q * mm + i * m + j];
                    for (int a = 0; a < 3; a++)
                        for (int n = 0; n < m; n++) {
                            const double li = lag[(size_t)i * m + n];
                            for (int p = 0; p < m; p++) pm.c[((size_t)a * m + n) * m + p] += y[a] * li * lag[(size_t)j * m + p];
                        }
                }
            double cx[3] = {0, 0, 0};
            for (int t = 0; t < mm; t++)
                for (int a = 0; a < 3; a++) cx[a] += xyz[3 * node_pt[q * mm + t] + a] / mm;
            double rad = 0;
            for (int t = 0; t < mm; t++) {
                const double *y = xyz + 3 * node_pt[q * mm + t];
                rad = std::max(rad, std::sqrt((y[0] - cx[0]) * (y[0] - cx[0]) + (y[1] - cx[1]) * (y[1] - cx[1]) +
                                              (y[2] - cx[2]) * (y[2] - cx[2])));
            }
            for (int a = 0; a < 3; a++) pm.ctr[a] = cx[a];
            pm.rad = 1.25 * rad;  // the interpolant's patch between and just beyond the nodes
            // orientation from the node nearest the patch centre
            const int ic = m / 2, jc = m / 2;
            const int64_t lc = node_pt[q * mm + ic * m + jc];
            double y[3], yu[3], yv[3], nn[3];
            pm.eval(sm[ic], sm[jc], y, yu, yv, tmp);
            cross(yu, yv, nn);
            pm.orient = dot3(nn, nrm + 3 * lc) >= 0 ? 1.0 : -1.0;
        }
    }

    // Uniform grid over the patch centres with cells no smaller than max radius + delta: a patch
    // that can lie within delta of x has its centre in x's cell or one of the 26 around it.
    double rmax = 0, clo[3] = {INFINITY, INFINITY, INFINITY}, chi[3] = {-INFINITY, -INFINITY, -INFINITY};
    for (int64_t q = 0; q < Q; q++) {
        rmax = std::max(rmax, P[q].rad);
        for (int a = 0; a < 3; a++) {
            clo[a] = std::min(clo[a], P[q].ctr[a]);
            chi[a] = std::max(chi[a], P[q].ctr[a]);
        }
    }
    double hc = std::max(rmax + delta, 1e-300);
    int64_t gd[3];
    for (;;) {
        for (int a = 0; a < 3; a++) gd[a] = (int64_t)std::floor((chi[a] - clo[a]) / hc) + 1;
        if (gd[0] * gd[1] * gd[2] <= 8 * Q + 4096) break;
        hc *= 1.5;  // coarser cells keep the grid within a few entries per patch
    }
    auto cell_of = [&](const double *c, int64_t *ijk) {
        for (int a = 0; a < 3; a++)
            ijk[a] = std::min(gd[a] - 1, std::max<int64_t>(0, (int64_t)std::floor((c[a] - clo[a]) / hc)));
    };
    std::vector<int64_t> cstart((size_t)(gd[0] * gd[1] * gd[2]) + 1, 0);
    std::vector<int64_t> clist((size_t)Q);
    {
        std::vector<int64_t> cq((size_t)Q);
        for (int64_t q = 0; q < Q; q++) {
            int64_t ijk[3];
            cell_of(P[q].ctr, ijk);
            cq[q] = (ijk[0] * gd[1] + ijk[1]) * gd[2] + ijk[2];
            cstart[cq[q] + 1]++;
        }
        for (size_t c = 0; c + 1 < cstart.size(); c++) cstart[c + 1] += cstart[c];
        std::vector<int64_t> fill(cstart.begin(), cstart.end() - 1);
        for (int64_t q = 0; q < Q; q++) clist[fill[cq[q]]++] = q;
    }

    std::vector<std::vector<std::pair<int32_t, cd>>> rows(device ? 0 : (size_t)N);
    // device mode: per target, the near patches and their closest-point parameters
    std::vector<std::vector<std::pair<int64_t, std::pair<double, double>>>> near(device ? (size_t)N : 0);
    int bad = 0;
#pragma omp parallel
    {
        std::vector<int64_t> cand;
        std::vector<double> tmp, ua(nbeta), wua(nbeta), vb(nbeta), wvb(nbeta);
        std::vector<double> Tu((size_t)nbeta * m), dTu((size_t)nbeta * m), Tv((size_t)nbeta * m), dTv((size_t)nbeta * m);
        std::vector<double> E((size_t)3 * m * nbeta), Ev((size_t)3 * m * nbeta);
        std::vector<double> Lu((size_t)nbeta * m), Lv((size_t)nbeta * m);
        std::vector<cd> G((size_t)nbeta * nbeta), H((size_t)m * nbeta);
        std::vector<double> Yg((size_t)9 * nbeta * nbeta);
#pragma omp for schedule(dynamic, 16)
        for (int64_t l = 0; l < N; l++) {
            const double *x = xyz + 3 * l;
            const int64_t ql = patch_node[l] / mm;
            std::vector<std::pair<int32_t, cd>> dummy;
            auto &row = device ? dummy : rows[l];
            // candidate patches from the 27 cells around x (ascending patch order)
            cand.clear();
            {
                int64_t ijk[3];
                cell_of(x, ijk);
                for (int64_t i0 = std::max<int64_t>(0, ijk[0] - 1); i0 <= std::min(gd[0] - 1, ijk[0] + 1); i0++)
                    for (int64_t i1 = std::max<int64_t>(0, ijk[1] - 1); i1 <= std::min(gd[1] - 1, ijk[1] + 1); i1++)
                        for (int64_t i2 = std::max<int64_t>(0, ijk[2] - 1); i2 <= std::min(gd[2] - 1, ijk[2] + 1); i2++) {
                            const int64_t c = (i0 * gd[1] + i1) * gd[2] + i2;
                            for (int64_t t = cstart[c]; t < cstart[c + 1]; t++) cand.push_back(clist[t]);
                        }
                bool own = false;
                for (int64_t q : cand) own = own || q == ql;
                if (!own) cand.push_back(ql);
                std::sort(cand.begin(), cand.end());
            }
            for (int64_t q : cand) {
                const PatchMap &pm = P[q];
                const double dc = std::sqrt((x[0] - pm.ctr[0]) * (x[0] - pm.ctr[0]) + (x[1] - pm.ctr[1]) * (x[1] - pm.ctr[1]) +
                                            (x[2] - pm.ctr[2]) * (x[2] - pm.ctr[2]));
                if (q != ql && dc > pm.rad + delta) continue;
                // closest patch point (Eq. MinNode): exact for the target's own patch
                double ub, vb_;
                if (q == ql) {
                    const int t = patch_node[l] % mm;
                    ub = sm[t / m];
                    vb_ = sm[t % m];
                } else {
                    double best = INFINITY;
                    int tb = 0;
                    for (int t = 0; t < mm; t++) {
                        const double *y = xyz + 3 * node_pt[q * mm + t];
                        const double d2 = (x[0] - y[0]) * (x[0] - y[0]) + (x[1] - y[1]) * (x[1] - y[1]) + (x[2] - y[2]) * (x[2] - y[2]);
                        if (d2 < best) {
                            best = d2;
                            tb = t;
                        }
                    }
                    ub = sm[tb / m];
                    vb_ = sm[tb % m];
                    closest_point(pm, x, ub, vb_, tmp);
                    double y[3], yu[3], yv[3];
                    pm.eval(ub, vb_, y, yu, yv, tmp);
                    const double dd = std::sqrt((x[0] - y[0]) * (x[0] - y[0]) + (x[1] - y[1]) * (x[1] - y[1]) + (x[2] - y[2]) * (x[2] - y[2]));
                    if (!(dd <= delta)) continue;  // regular interaction (Eq. ReguGridPts)
                }
                if (device) {
                    near[l].push_back({q, {ub, vb_}});
                    continue;
                }
                // graded Fejer nodes (Eq. CovNodesWeights)
                for (int a = 0; a < nbeta; a++) {
                    double xi, dxi;
                    cov(ub, sb[a], dgrade, xi, dxi);
                    ua[a] = xi;
                    wua[a] = dxi * wb[a];
                    cov(vb_, sb[a], dgrade, xi, dxi);
                    vb[a] = xi;
                    wvb[a] = dxi * wb[a];
                    cheb_vals(m, ua[a], &Tu[(size_t)a * m], &dTu[(size_t)a * m]);
                    cheb_vals(m, vb[a], &Tv[(size_t)a * m], &dTv[(size_t)a * m]);
                }
                // patch map on the graded grid: E[c][n][b] = sum_p coef T_p(v_b), Ev with T_p'
                for (int c = 0; c < 3; c++)
                    for (int n = 0; n < m; n++) {
                        const double *cr = &pm.c[((size_t)c * m + n) * m];
                        for (int b = 0; b < nbeta; b++) {
                            double s = 0, sv = 0;
                            for (int p = 0; p < m; p++) {
                                s += cr[p] * Tv[(size_t)b * m + p];
                                sv += cr[p] * dTv[(size_t)b * m + p];
                            }
                            E[((size_t)c * m + n) * nbeta + b] = s;
                            Ev[((size_t)c * m + n) * nbeta + b] = sv;
                        }
                    }
                // y, y_u, y_v on the grid, coordinate-major rows over b (contiguous, vectorisable)
                std::fill(Yg.begin(), Yg.end(), 0.0);
                for (int c = 0; c < 3; c++)
                    for (int a = 0; a < nbeta; a++) {
                        double *yr = &Yg[((size_t)(3 * c + 0) * nbeta + a) * nbeta];
                        double *yur = &Yg[((size_t)(3 * c + 1) * nbeta + a) * nbeta];
                        double *yvr = &Yg[((size_t)(3 * c + 2) * nbeta + a) * nbeta];
                        for (int n = 0; n < m; n++) {
                            const double tu = Tu[(size_t)a * m + n], dtu = dTu[(size_t)a * m + n];
                            const double *e = &E[((size_t)c * m + n) * nbeta], *ev = &Ev[((size_t)c * m + n) * nbeta];
                            for (int b = 0; b < nbeta; b++) {
                                yr[b] += tu * e[b];
                                yur[b] += dtu * e[b];
                                yvr[b] += tu * ev[b];
                            }
                        }
                    }
                for (int a = 0; a < nbeta; a++)
                    for (int b = 0; b < nbeta; b++) {
                        double y[3], yu[3], yv[3];
                        for (int c = 0; c < 3; c++) {
                            y[c] = Yg[((size_t)(3 * c + 0) * nbeta + a) * nbeta + b];
                            yu[c] = Yg[((size_t)(3 * c + 1) * nbeta + a) * nbeta + b];
                            yv[c] = Yg[((size_t)(3 * c + 2) * nbeta + a) * nbeta + b];
                        }
                        double nn[3];
                        cross(yu, yv, nn);
                        const double J = std::sqrt(dot3(nn, nn));
                        const double nu[3] = {pm.orient * nn[0] / J, pm.orient * nn[1] / J, pm.orient * nn[2] / J};
                        G[(size_t)a * nbeta + b] = cfie_kernel(k, eta, x, y, nu, tol) * (J * wua[a] * wvb[b]);
                    }
                // c_ij = sum_ab G_ab l_i(u_a) l_j(v_b)
                for (int a = 0; a < nbeta; a++)
                    for (int i = 0; i < m; i++) {
                        double su = 0, sv = 0;
                        for (int n = 0; n < m; n++) {
                            su += lag[(size_t)i * m + n] * Tu[(size_t)a * m + n];
                            sv += lag[(size_t)i * m + n] * Tv[(size_t)a * m + n];
                        }
                        Lu[(size_t)a * m + i] = su;
                        Lv[(size_t)a * m + i] = sv;
                    }
                for (int i = 0; i < m; i++)
                    for (int b = 0; b < nbeta; b++) {
                        cd s = 0;
                        for (int a = 0; a < nbeta; a++) s += Lu[(size_t)a * m + i] * G[(size_t)a * nbeta + b];
                        H[(size_t)i * nbeta + b] = s;
                    }
                for (int i = 0; i < m; i++)
                    for (int j = 0; j < m; j++) {
                        cd s = 0;
                        for (int b = 0; b < nbeta; b++) s += H[(size_t)i * nbeta + b] * Lv[(size_t)b * m + j];
                        const int64_t lp = node_pt[q * mm + i * m + j];
                        if (lp != l) s -= cfie_kernel(k, eta, x, xyz + 3 * lp, nrm + 3 * lp, tol) * w[lp];
                        if (!std::isfinite(s.real()) || !std::isfinite(s.imag())) {
#pragma omp atomic write
                            bad = 1;
                        }
                        row.emplace_back((int32_t)lp, s);
                    }
            }
        }
    }
    if (bad) {
        set_error("non-finite correction entry (degenerate patch geometry?)");
        return IFGF_EINVAL;
    }
    if (device) {  // the quadrature on the GPU, then the CSR in target order
        std::vector<int64_t> pl;
        std::vector<int> pq;
        std::vector<double> puv, coef((size_t)Q * 3 * mm), orient((size_t)Q);
        for (int64_t l = 0; l < N; l++)
            for (const auto &e : near[l]) {
                pl.push_back(l);
                pq.push_back((int)e.first);
                puv.push_back(e.second.first);
                puv.push_back(e.second.second);
            }
        for (int64_t q = 0; q < Q; q++) {
            std::copy(P[q].c.begin(), P[q].c.end(), coef.begin() + q * 3 * mm);
            orient[q] = P[q].orient;
        }
        std::vector<double> vals;
        ifgf_status st = rp_quadrature_device(m, nbeta, k, eta, tol, dgrade, coef, orient, xyz, nrm, w, N, node_pt, sb,
                                              wb, lag, pl, pq, puv, stream, vals);
        if (st != IFGF_OK) return st;
        for (double v : vals)
            if (!std::isfinite(v)) {
                set_error("non-finite correction entry (degenerate patch geometry?)");
                return IFGF_EINVAL;
            }
        const size_t nnz = pl.size() * (size_t)mm;
        int64_t *rowptr = (int64_t *)std::malloc(sizeof(int64_t) * ((size_t)N + 1));
        int32_t *col = (int32_t *)std::malloc(sizeof(int32_t) * std::max<size_t>(nnz, 1));
        double *val = (double *)std::malloc(sizeof(double) * 2 * std::max<size_t>(nnz, 1));
        if (!rowptr || !col || !val) {
            std::free(rowptr);
            std::free(col);
            std::free(val);
            set_error("host allocation failed (%zu correction entries)", nnz);
            return IFGF_ENOMEM;
        }
        rowptr[0] = 0;
        for (int64_t l = 0; l < N; l++) rowptr[l + 1] = rowptr[l] + (int64_t)near[l].size() * mm;
        for (size_t pr = 0; pr < pl.size(); pr++)
            for (int t = 0; t < mm; t++) col[pr * mm + t] = (int32_t)node_pt[(size_t)pq[pr] * mm + t];
        std::memcpy(val, vals.data(), sizeof(double) * 2 * nnz);
        *rowptr_out = rowptr;
        *col_out = col;
        *val_out = val;
        return IFGF_OK;
    }
    // CSR straight into the caller's arrays, each row released once copied (bounds the peak)
    int64_t *rowptr = (int64_t *)std::malloc(sizeof(int64_t) * ((size_t)N + 1));
    if (!rowptr) {
        set_error("host allocation failed");
        return IFGF_ENOMEM;
    }
    rowptr[0] = 0;
    for (int64_t l = 0; l < N; l++) rowptr[l + 1] = rowptr[l] + (int64_t)rows[l].size();
    const size_t nnz = (size_t)rowptr[N];
    int32_t *col = (int32_t *)std::malloc(sizeof(int32_t) * std::max<size_t>(nnz, 1));
    double *val = (double *)std::malloc(sizeof(double) * 2 * std::max<size_t>(nnz, 1));
    if (!col || !val) {
        std::free(rowptr);
        std::free(col);
        std::free(val);
        set_error("host allocation failed (%zu correction entries)", nnz);
        return IFGF_ENOMEM;
    }
    for (int64_t l = 0; l < N; l++) {
        int64_t o = rowptr[l];
        for (const auto &e : rows[l]) {
            col[o] = e.first;
            val[2 * o] = e.second.real();
            val[2 * o + 1] = e.second.imag();
            o++;
        }
        std::vector<std::pair<int32_t, cd>>().swap(rows[l]);
    }
    *rowptr_out = rowptr;
    *col_out = col;
    *val_out = val;
    return IFGF_OK;
}

}  // namespace ifgf

using namespace ifgf;

extern "C" {

static ifgf_status rp_entry(const double *xyz, const double *normals, const double *weights, int64_t N,
                            const int32_t *patch_node, int32_t m, double k, double eta, double delta, int32_t n_beta,
                            double d_grade, int64_t **rowptr_out, int32_t **col_out, double **val_out, bool device,
                            void *stream) {
    clear_error();
    if (!rowptr_out || !col_out || !val_out) {
        set_error("null output pointer");
        return IFGF_EINVAL;
    }
    *rowptr_out = nullptr;
    *col_out = nullptr;
    *val_out = nullptr;
    if (!xyz || !normals || !weights || !patch_node) {
        set_error("null input array");
        return IFGF_EINVAL;
    }
    if (m < 2 || m > 64 || N < (int64_t)m * m || N % ((int64_t)m * m) != 0 || N > (int64_t)0x7fffffff) {
        set_error("N (%lld) must be a positive multiple of m * m with 2 <= m <= 64 (m = %d)", (long long)N, (int)m);
        return IFGF_EINVAL;
    }
    if (!(k > 0) || !std::isfinite(k) || !std::isfinite(eta) || !(delta >= 0) || !std::isfinite(delta) ||
        n_beta < 2 || n_beta > 512 || !(d_grade >= 2) || !std::isfinite(d_grade)) {
        set_error("invalid k, eta, delta, n_beta or d_grade");
        return IFGF_EINVAL;
    }
    if (device && (m > 16 || n_beta > 64)) {
        set_error("the device quadrature takes m <= 16 and n_beta <= 64 (m = %d, n_beta = %d); use ifgf_rp_correction",
                  (int)m, (int)n_beta);
        return IFGF_EUNSUPPORTED;
    }
    for (int64_t i = 0; i < 3 * N; i++)
        if (!std::isfinite(xyz[i]) || !std::isfinite(normals[i])) {
            set_error("non-finite point or normal");
            return IFGF_EINVAL;
        }
    try {
        return build_rp(xyz, normals, weights, N, patch_node, m, k, eta, delta, n_beta, d_grade, rowptr_out, col_out,
                        val_out, device, (cudaStream_t)stream);
    } catch (const std::bad_alloc &) {
        set_error("host allocation failed");
        return IFGF_ENOMEM;
    }
}

ifgf_status ifgf_rp_correction(const double *xyz, const double *normals, const double *weights, int64_t N,
                               const int32_t *patch_node, int32_t m, double k, double eta, double delta,
                               int32_t n_beta, double d_grade, int64_t **rowptr_out, int32_t **col_out,
                               double **val_out) {
    return rp_entry(xyz, normals, weights, N, patch_node, m, k, eta, delta, n_beta, d_grade, rowptr_out, col_out,
                    val_out, false, nullptr);
}

ifgf_status ifgf_rp_correction_gpu(const double *xyz, const double *normals, const double *weights, int64_t N,
                                   const int32_t *patch_node, int32_t m, double k, double eta, double delta,
                                   int32_t n_beta, double d_grade, void *stream, int64_t **rowptr_out,
                                   int32_t **col_out, double **val_out) {
    return rp_entry(xyz, normals, weights, N, patch_node, m, k, eta, delta, n_beta, d_grade, rowptr_out, col_out,
                    val_out, true, stream);
}

void ifgf_free(void *ptr) { std::free(ptr); }

}  // extern "C"

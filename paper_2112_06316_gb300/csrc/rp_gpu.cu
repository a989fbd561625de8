// Rectangular-polar correction, device quadrature (Section 4.2).
//
// The host (rp.cpp) builds the patch maps, finds for every target the patches within the
// proximity distance and the closest patch point (Eq. MinNode), and hands the flat list of
// (target, patch, closest-point parameters) pairs to rp_quadrature_device.  One block per pair
// then evaluates, in FP64, the graded Fejer quadrature of Eq. BetaCov after the change of
// variables of Eq. CoV (Kress map, Eq. wMap / Eq. vMap) centred at the closest point, folds the
// Chebyshev coefficients of Eq. ChebyCoeff into nodal weights, and subtracts the regular row
// (Eq. ReguIntOpQuadrature) -- the same arithmetic as the host builder, in a different order.
#include <cmath>
#include <vector>

#include "ifgf_internal.h"

namespace ifgf {

namespace {

constexpr int kRpThreads = 64;
constexpr double kPiRp = 3.14159265358979323846;

__device__ __forceinline__ void rp_cheb(int n, double t, double *T, double *dT) {
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

__device__ __forceinline__ double rp_nu(double t, double d) {
    const double a = (kPiRp - t) / kPiRp;
    return (1.0 / d - 0.5) * a * a * a + (1.0 / d) * (t - kPiRp) / kPiRp + 0.5;
}
__device__ __forceinline__ double rp_dnu(double t, double d) {
    const double a = (kPiRp - t) / kPiRp;
    return -3.0 / kPiRp * (1.0 / d - 0.5) * a * a + 1.0 / (d * kPiRp);
}
// Kress map w(tau; d) on [0, 2 pi] and its derivative (Eq. wMap, Eq. vMap)
__device__ __forceinline__ void rp_kress(double t, double d, double &w, double &dw) {
    const double n1 = rp_nu(t, d), n2 = rp_nu(2.0 * kPiRp - t, d);
    const double A = pow(n1, d), B = pow(n2, d);
    const double dA = d * pow(n1, d - 1.0) * rp_dnu(t, d);
    const double dB = -d * pow(n2, d - 1.0) * rp_dnu(2.0 * kPiRp - t, d);
    const double S = A + B;
    w = 2.0 * kPiRp * A / S;
    dw = 2.0 * kPiRp * (dA * B - A * dB) / (S * S);
}
// xi_alpha(tau; d) of Eq. CoV, clustering at alpha, and d xi / d tau
__device__ __forceinline__ void rp_cov(double alpha, double tau, double d, double &xi, double &dxi) {
    double w, dw;
    if (alpha >= 1.0) {
        rp_kress(kPiRp * fabs((tau - 1.0) / 2.0), d, w, dw);
        xi = 1.0 - (2.0 / kPiRp) * w;
        dxi = dw;
    } else if (alpha <= -1.0) {
        rp_kress(kPiRp * fabs((tau + 1.0) / 2.0), d, w, dw);
        xi = -1.0 + (2.0 / kPiRp) * w;
        dxi = dw;
    } else {
        const double sg = tau > 0 ? 1.0 : (tau < 0 ? -1.0 : 0.0);
        rp_kress(kPiRp * fabs(tau), d, w, dw);
        xi = alpha + (sg - alpha) / kPiRp * w;
        dxi = (1.0 - alpha * sg) * dw;
    }
}

// combined-field kernel dPhi/dnu(y) - i eta Phi (Eq. GreenFunction, Eq. double_layer), zero closer than tol
__device__ __forceinline__ double2 rp_kernel(double k, double eta, const double *x, const double *y, const double *nu,
                                             double tol) {
    const double d0 = x[0] - y[0], d1 = x[1] - y[1], d2 = x[2] - y[2];
    const double r = sqrt(d0 * d0 + d1 * d1 + d2 * d2);
    if (!(r >= tol)) return make_double2(0.0, 0.0);
    const double a = 1.0 / (4.0 * kPiRp * r);
    double sn, cs;
    sincos(k * r, &sn, &cs);
    const double dn = (d0 * nu[0] + d1 * nu[1] + d2 * nu[2]) / (r * r);
    // e (1 - i k r) dn - i eta e,  e = a (cs + i sn)
    const double br = dn, bi = -k * r * dn - eta;
    return make_double2(a * (cs * br - sn * bi), a * (sn * br + cs * bi));
}

struct RpDev {
    int m, nbeta;
    double k, eta, tol, dgrade;
    const double *coef;      // Q x 3 m m patch-map coefficients
    const double *orient;    // Q
    const double *xyz, *nrm, *w;  // caller order
    const int *node_pt;      // Q m m -> caller index
    const double *sb, *wb;   // Fejer nodes / weights of the graded rule (nbeta)
    const double *lag;       // m x m: l_i(u) = sum_n lag[i m + n] T_n(u)
    const long long *pl;     // per pair: target
    const int *pq;           // per pair: patch
    const double2 *puv;      // per pair: closest point (u, v)
    double2 *out;            // per pair: m m values
};

__global__ void __launch_bounds__(kRpThreads) k_rp_pair(RpDev a) {
    extern __shared__ double rp_sm[];
    const int m = a.m, nb = a.nbeta, mm = m * m;
    const long long pr = blockIdx.x;
    const long long l = a.pl[pr];
    const int q = a.pq[pr];
    const double2 uv = a.puv[pr];
    double *Tu = rp_sm, *dTu = Tu + nb * m, *Tv = dTu + nb * m, *dTv = Tv + nb * m;
    double *E = dTv + nb * m, *Ev = E + 3 * m * nb;        // [c][n][b]
    double *Lu = Ev + 3 * m * nb, *Lv = Lu + nb * m;        // [a][i]
    double *wu = Lv + nb * m, *wv = wu + nb;                 // graded weights
    double2 *H = reinterpret_cast<double2 *>(wv + nb);       // [i][b]
    const double *cf = a.coef + (size_t)q * 3 * mm;
    const double x[3] = {a.xyz[3 * l], a.xyz[3 * l + 1], a.xyz[3 * l + 2]};
    // graded nodes and weights, Chebyshev values and nodal bases on them
    for (int t = threadIdx.x; t < nb; t += blockDim.x) {
        double xi, dxi;
        rp_cov(uv.x, a.sb[t], a.dgrade, xi, dxi);
        wu[t] = dxi * a.wb[t];
        rp_cheb(m, xi, Tu + t * m, dTu + t * m);
        rp_cov(uv.y, a.sb[t], a.dgrade, xi, dxi);
        wv[t] = dxi * a.wb[t];
        rp_cheb(m, xi, Tv + t * m, dTv + t * m);
    }
    __syncthreads();
    for (int t = threadIdx.x; t < nb * m; t += blockDim.x) {
        const int aa = t / m, i = t % m;
        double su = 0, sv = 0;
        for (int n = 0; n < m; n++) {
            su += a.lag[i * m + n] * Tu[aa * m + n];
            sv += a.lag[i * m + n] * Tv[aa * m + n];
        }
        Lu[t] = su;
        Lv[t] = sv;
    }
    // patch map contracted along v: E[c][n][b] = sum_p coef T_p(v_b), Ev with T_p'
    for (int t = threadIdx.x; t < 3 * m * nb; t += blockDim.x) {
        const int c = t / (m * nb), n = (t / nb) % m, b = t % nb;
        const double *cr = cf + (c * m + n) * m;
        double s = 0, sv = 0;
        for (int p = 0; p < m; p++) {
            s += cr[p] * Tv[b * m + p];
            sv += cr[p] * dTv[b * m + p];
        }
        E[t] = s;
        Ev[t] = sv;
    }
    __syncthreads();
    // one graded column b per thread: G(a, b) = K(x, y) J w_u w_v on the fly, H[i][b] = sum_a Lu[a][i] G
    const double orient = a.orient[q];
    for (int b = threadIdx.x; b < nb; b += blockDim.x) {
        double2 h[16];
        for (int i = 0; i < m; i++) h[i] = make_double2(0.0, 0.0);
        for (int aa = 0; aa < nb; aa++) {
            double y[3], yu[3], yv[3];
            for (int c = 0; c < 3; c++) {
                double s = 0, su = 0, sv = 0;
                for (int n = 0; n < m; n++) {
                    const double e = E[(c * m + n) * nb + b], ev = Ev[(c * m + n) * nb + b];
                    s += Tu[aa * m + n] * e;
                    su += dTu[aa * m + n] * e;
                    sv += Tu[aa * m + n] * ev;
                }
                y[c] = s;
                yu[c] = su;
                yv[c] = sv;
            }
            const double n0 = yu[1] * yv[2] - yu[2] * yv[1], n1 = yu[2] * yv[0] - yu[0] * yv[2],
                         n2 = yu[0] * yv[1] - yu[1] * yv[0];
            const double J = sqrt(n0 * n0 + n1 * n1 + n2 * n2);
            const double nu[3] = {orient * n0 / J, orient * n1 / J, orient * n2 / J};
            const double2 K = rp_kernel(a.k, a.eta, x, y, nu, a.tol);
            const double sc = J * wu[aa] * wv[b];
            const double gr = K.x * sc, gi = K.y * sc;
            for (int i = 0; i < m; i++) {
                const double lu = Lu[aa * m + i];
                h[i].x += lu * gr;
                h[i].y += lu * gi;
            }
        }
        for (int i = 0; i < m; i++) H[i * nb + b] = h[i];
    }
    __syncthreads();
    // c_ij = sum_b H[i][b] Lv[b][j], minus the regular row's entry for node (i, j)
    for (int t = threadIdx.x; t < mm; t += blockDim.x) {
        const int i = t / m, j = t % m;
        double sr = 0, si = 0;
        for (int b = 0; b < nb; b++) {
            const double2 hv = H[i * nb + b];
            const double lv = Lv[b * m + j];
            sr += hv.x * lv;
            si += hv.y * lv;
        }
        const int lp = a.node_pt[(size_t)q * mm + t];
        if (lp != l) {
            const double2 K = rp_kernel(a.k, a.eta, x, a.xyz + 3 * (size_t)lp, a.nrm + 3 * (size_t)lp, a.tol);
            sr -= K.x * a.w[lp];
            si -= K.y * a.w[lp];
        }
        a.out[pr * mm + t] = make_double2(sr, si);
    }
}

}  // namespace

// Quadrature of every (target, near patch) pair on the current device: `out` receives, pair by
// pair, the m * m complex128 entries (interleaved re, im) of the correction row block.  Pairs go
// in batches (bounded device memory); synchronous on stream s.
ifgf_status rp_quadrature_device(int m, int nbeta, double k, double eta, double tol, double dgrade,
                                 const std::vector<double> &coef, const std::vector<double> &orient, const double *xyz,
                                 const double *nrm, const double *w, int64_t N, const std::vector<int64_t> &node_pt,
                                 const std::vector<double> &sb, const std::vector<double> &wb,
                                 const std::vector<double> &lag, const std::vector<int64_t> &pl,
                                 const std::vector<int> &pq, const std::vector<double> &puv, cudaStream_t s,
                                 std::vector<double> &out) {
    const int mm = m * m;
    const size_t np = pl.size();
    out.assign(2 * np * (size_t)mm, 0.0);
    if (np == 0) return IFGF_OK;
    constexpr size_t kBatch = size_t(1) << 17;
    const size_t nb = std::min(np, kBatch);
    std::vector<void *> mem;
    auto alloc = [&](size_t bytes) -> void * {
        void *ptr = nullptr;
        if (cudaMalloc(&ptr, bytes > 0 ? bytes : 16) != cudaSuccess) return nullptr;
        mem.push_back(ptr);
        return ptr;
    };
    auto release = [&]() {
        for (void *ptr : mem) cudaFree(ptr);
        mem.clear();
    };
    std::vector<int> npt((size_t)N);
    for (int64_t i = 0; i < N; i++) npt[i] = (int)node_pt[i];
    RpDev a;
    a.m = m;
    a.nbeta = nbeta;
    a.k = k;
    a.eta = eta;
    a.tol = tol;
    a.dgrade = dgrade;
    double *d_coef = (double *)alloc(sizeof(double) * coef.size());
    double *d_or = (double *)alloc(sizeof(double) * orient.size());
    double *d_x = (double *)alloc(sizeof(double) * 3 * N);
    double *d_n = (double *)alloc(sizeof(double) * 3 * N);
    double *d_w = (double *)alloc(sizeof(double) * N);
    int *d_np = (int *)alloc(sizeof(int) * N);
    double *d_sb = (double *)alloc(sizeof(double) * nbeta);
    double *d_wb = (double *)alloc(sizeof(double) * nbeta);
    double *d_lag = (double *)alloc(sizeof(double) * lag.size());
    long long *d_pl = (long long *)alloc(sizeof(long long) * nb);
    int *d_pq = (int *)alloc(sizeof(int) * nb);
    double2 *d_uv = (double2 *)alloc(sizeof(double2) * nb);
    double2 *d_out = (double2 *)alloc(sizeof(double2) * nb * mm);
    if (mem.size() != 13) {
        release();
        set_error("device allocation for the correction quadrature failed");
        return IFGF_ENOMEM;
    }
    cudaError_t e = cudaSuccess;
    auto h2d = [&](void *dst, const void *src, size_t bytes) {
        if (e == cudaSuccess && bytes) e = cudaMemcpyAsync(dst, src, bytes, cudaMemcpyHostToDevice, s);
    };
    h2d(d_coef, coef.data(), sizeof(double) * coef.size());
    h2d(d_or, orient.data(), sizeof(double) * orient.size());
    h2d(d_x, xyz, sizeof(double) * 3 * N);
    h2d(d_n, nrm, sizeof(double) * 3 * N);
    h2d(d_w, w, sizeof(double) * N);
    h2d(d_np, npt.data(), sizeof(int) * N);
    h2d(d_sb, sb.data(), sizeof(double) * nbeta);
    h2d(d_wb, wb.data(), sizeof(double) * nbeta);
    h2d(d_lag, lag.data(), sizeof(double) * lag.size());
    a.coef = d_coef;
    a.orient = d_or;
    a.xyz = d_x;
    a.nrm = d_n;
    a.w = d_w;
    a.node_pt = d_np;
    a.sb = d_sb;
    a.wb = d_wb;
    a.lag = d_lag;
    a.pl = d_pl;
    a.pq = d_pq;
    a.puv = d_uv;
    a.out = d_out;
    const size_t smem = sizeof(double) * (14 * (size_t)nbeta * m + 2 * (size_t)nbeta);
    if (e == cudaSuccess) e = cudaFuncSetAttribute(k_rp_pair, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    for (size_t p0 = 0; p0 < np && e == cudaSuccess; p0 += nb) {
        const size_t cnt = std::min(nb, np - p0);
        h2d(d_pl, pl.data() + p0, sizeof(long long) * cnt);
        h2d(d_pq, pq.data() + p0, sizeof(int) * cnt);
        h2d(d_uv, puv.data() + 2 * p0, sizeof(double2) * cnt);
        if (e != cudaSuccess) break;
        k_rp_pair<<<(unsigned)cnt, kRpThreads, smem, s>>>(a);
        e = cudaGetLastError();
        if (e == cudaSuccess)
            e = cudaMemcpyAsync(out.data() + 2 * p0 * mm, d_out, sizeof(double2) * cnt * mm, cudaMemcpyDeviceToHost, s);
        if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    }
    release();
    if (e != cudaSuccess) {
        set_error("correction quadrature on the device: %s", cudaGetErrorString(e));
        return e == cudaErrorMemoryAllocation ? IFGF_ENOMEM : IFGF_ECUDA;
    }
    return IFGF_OK;
}

}  // namespace ifgf

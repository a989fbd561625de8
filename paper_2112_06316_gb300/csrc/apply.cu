// Forward apply of the IFGF-accelerated CFIE operator on sm_103a.
//
// Pipeline of one apply (Algorithm 1 + Remark level_D_neighboring):
//   gather   a = w * sigma in Morton order
//   K1 leaf  F^D at every relevant level-D cone node (Algorithm 1, first loop nest)
//   K3 prop  for d = D..4: F^{d-1}(x) = sum_children Interp(F^d_child)(x) E(x;y_c)/E(x;y_p)
//   K4 near  u = level-D neighbour interactions by direct summation
//   K2 cous  for d = D..3: u(x) += sum_cousin-boxes E(x;y_k) Interp(F^d_k)(x)
//   scatter  y = c_I sigma + u (+ C sigma) in the caller's order
// Every kernel is output-stationary (one thread owns one output value), so no
// atomics are needed and FP64 results are bitwise reproducible run to run.
#include <algorithm>
#include <cstdio>

#include "ifgf_internal.h"
#include "kernels.cuh"

namespace ifgf {

#define CK(call)                                                                                  \
    do {                                                                                          \
        cudaError_t e_ = (call);                                                                  \
        if (e_ != cudaSuccess) {                                                                  \
            set_error("%s failed: %s", #call, cudaGetErrorString(e_));                            \
            return IFGF_ECUDA;                                                                    \
        }                                                                                         \
    } while (0)

static constexpr int kBlock = 128;
static constexpr int kRB = 4;  // right-hand sides per register block

__device__ __forceinline__ double2 cmul(double2 a, double2 b) {
    return make_double2(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}

// ============================================================================
// gather / scatter
// ============================================================================
template <typename T>
__global__ void k_gather(int N, int nrhs, const int *__restrict__ perm, const T *__restrict__ w,
                         const typename C2T<T>::type *__restrict__ sigma, typename C2T<T>::type *__restrict__ a) {
    long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (i >= (long long)N * nrhs) return;
    int q = (int)(i / N), s = (int)(i % N);
    typename C2T<T>::type v = sigma[(long long)q * N + perm[s]];
    T ww = w[s];
    v.x *= ww;
    v.y *= ww;
    a[i] = v;
}

template <typename T>
__global__ void k_scatter(int N, int nrhs, const int *__restrict__ perm, double cI,
                          const typename C2T<T>::type *__restrict__ sigma, const typename C2T<T>::type *__restrict__ u,
                          typename C2T<T>::type *__restrict__ y) {
    long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (i >= (long long)N * nrhs) return;
    int q = (int)(i / N), s = (int)(i % N);
    long long o = (long long)q * N + perm[s];
    typename C2T<T>::type sg = sigma[o], uu = u[i], r;
    r.x = (T)cI * sg.x + uu.x;
    r.y = (T)cI * sg.y + uu.y;
    y[o] = r;
}

// ============================================================================
// FP64 kernels (absolute coordinates)
// ============================================================================
__device__ __forceinline__ void center64(const CommonArgs &ca, const LevelArgs &L, int b, double *y0) {
    y0[0] = ca.c0[0] + (L.ijk[3 * b] + 0.5) * L.H;
    y0[1] = ca.c0[1] + (L.ijk[3 * b + 1] + 0.5) * L.H;
    y0[2] = ca.c0[2] + (L.ijk[3 * b + 2] + 0.5) * L.H;
}

// Boundary points (within 1e-12 relative of an integer multiple of the interval)
// are placed exactly on the boundary: the upper interval owns them whatever the
// last-bit rounding of atan2 / sqrt.
__device__ __forceinline__ double snap64(double u) {
    double r = rint(u);
    return fabs(u - r) <= 1e-12 * fmax(fabs(u), 1.0) ? r : u;
}

// cone id and local coordinates of the point at offset (dx, dy, dz) from a box centre
__device__ __forceinline__ int classify64(const LevelArgs &L, double dx, double dy, double dz, double &r, double *t3) {
    double rho = sqrt(dx * dx + dy * dy);
    r = sqrt(dx * dx + dy * dy + dz * dz);
    double s = L.h / r;
    double th = atan2(rho, dz);
    double ph = atan2(dy, dx);
    if (ph < 0) ph += 2.0 * kPi;
    if (ph >= 2.0 * kPi) ph = 0.0;
    double us = snap64(s / L.ds), ut = snap64(th / L.dth), up = snap64(ph / L.dph);
    int is = min((int)floor(us), L.ns - 1), it = min((int)floor(ut), L.nC - 1), ip = min((int)floor(up), L.nph - 1);
    is = max(is, 0);
    it = max(it, 0);
    ip = max(ip, 0);
    t3[0] = 2.0 * (us - is) - 1.0;
    t3[1] = 2.0 * (ut - it) - 1.0;
    t3[2] = 2.0 * (up - ip) - 1.0;
    return (is * L.nC + it) * L.nph + ip;
}

// node n of cone `cone`: (s, unit direction)
template <int PS, int PA>
__device__ __forceinline__ void node64(const LevelArgs &L, const ChebTab &tb, int cone, int n, double &s, double *u) {
    int ip = cone % L.nph, it = (cone / L.nph) % L.nC, is = cone / (L.nph * L.nC);
    int ia = n / (PA * PA), ib = (n / PA) % PA, ic = n % PA;
    s = (is + 0.5 * (tb.xs[ia] + 1.0)) * L.ds;
    double th = (it + 0.5 * (tb.xa[ib] + 1.0)) * L.dth;
    double ph = (ip + 0.5 * (tb.xa[ic] + 1.0)) * L.dph;
    double st, ct, sp, cp;
    sincos(th, &st, &ct);
    sincos(ph, &sp, &cp);
    u[0] = st * cp;
    u[1] = st * sp;
    u[2] = ct;
}

// K1 (FP64): F at the relevant leaf cone nodes.
template <int PS, int PA>
__global__ void __launch_bounds__(kBlock) k_leaf64(CommonArgs ca, LevelArgs L, ChebTab tb, const double2 *__restrict__ a) {
    constexpr int P = PS * PA * PA;
    long long tid = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (tid >= L.nrc * P) return;
    int rc = (int)(tid / P), n = (int)(tid % P);
    int b = L.rc_box[rc];
    double s, u[3];
    node64<PS, PA>(L, tb, L.rc_cone[rc], n, s, u);
    double y0[3];
    center64(ca, L, b, y0);
    const double r = L.h / s, k = ca.k, eta = ca.eta, soh = s / L.h;
    const int j0 = L.start[b], j1 = L.start[b + 1];
    double2 *F = (double2 *)L.F;
    for (int q0 = 0; q0 < ca.nrhs; q0 += kRB) {
        double2 acc0[kRB], acc1[kRB];
#pragma unroll
        for (int qq = 0; qq < kRB; qq++) acc0[qq] = acc1[qq] = make_double2(0, 0);
        for (int j = j0; j < j1; j++) {
            double yv[3] = {ca.x64[3 * j] - y0[0], ca.x64[3 * j + 1] - y0[1], ca.x64[3 * j + 2] - y0[2]};
            double dv[3] = {u[0] - yv[0] / r, u[1] - yv[1] / r, u[2] - yv[2] / r};
            double a2 = dv[0] * dv[0] + dv[1] * dv[1] + dv[2] * dv[2];
            double am = sqrt(a2);
            double yy = yv[0] * yv[0] + yv[1] * yv[1] + yv[2] * yv[2];
            double uy = u[0] * yv[0] + u[1] * yv[1] + u[2] * yv[2];
            double psi = k * (s * yy / L.h - 2.0 * uy) / (am + 1.0);
            double sn, cs;
            sincos(psi, &sn, &cs);
            double dn = dv[0] * ca.n64[3 * j] + dv[1] * ca.n64[3 * j + 1] + dv[2] * ca.n64[3 * j + 2];
            double ia = 1.0 / am;
            double w1 = ia, w3 = dn * ia * ia, w2 = w3 * ia;
            double2 W0, W1;
            if (L.split) {
                W0 = make_double2(cs * w2, sn * w2);
                // -i k W3 - i eta W1 = -i e (k w3 + eta w1)
                double g = k * w3 + eta * w1;
                W1 = make_double2(sn * g, -cs * g);
            } else {
                double g = k * w3 + eta * w1;
                W0 = make_double2(cs * soh * w2 + sn * g, sn * soh * w2 - cs * g);
            }
#pragma unroll
            for (int qq = 0; qq < kRB; qq++) {
                if (q0 + qq < ca.nrhs) {
                    double2 aj = a[(long long)(q0 + qq) * ca.N + j];
                    double2 t0 = cmul(aj, W0);
                    acc0[qq].x += t0.x;
                    acc0[qq].y += t0.y;
                    if (L.split) {
                        double2 t1 = cmul(aj, W1);
                        acc1[qq].x += t1.x;
                        acc1[qq].y += t1.y;
                    }
                }
            }
        }
#pragma unroll
        for (int qq = 0; qq < kRB; qq++) {
            if (q0 + qq < ca.nrhs) {
                long long base = ((long long)(q0 + qq) * L.nrc + rc) * L.nfac;
                F[base * ca.Pstride + n] = acc0[qq];
                if (L.split) F[(base + 1) * ca.Pstride + n] = acc1[qq];
            }
        }
    }
}

// K3 (FP64): F^{d-1} at the parent's relevant cone nodes from the children's interpolants.
template <int PS, int PA>
__global__ void __launch_bounds__(kBlock) k_prop64(CommonArgs ca, LevelArgs C, LevelArgs Pl, ChebTab tb) {
    constexpr int P = PS * PA * PA;
    long long tid = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (tid >= Pl.nrc * P) return;
    int rc = (int)(tid / P), n = (int)(tid % P);
    int pb = Pl.rc_box[rc];
    double s, u[3];
    node64<PS, PA>(Pl, tb, Pl.rc_cone[rc], n, s, u);
    double yp[3];
    center64(ca, Pl, pb, yp);
    const double rp = Pl.h / s;
    const double x[3] = {yp[0] + rp * u[0], yp[1] + rp * u[1], yp[2] + rp * u[2]};
    const double2 *FC = (const double2 *)C.F;
    double2 *FP = (double2 *)Pl.F;
    for (int q0 = 0; q0 < ca.nrhs; q0 += kRB) {
        double2 acc0[kRB], acc1[kRB];
#pragma unroll
        for (int qq = 0; qq < kRB; qq++) acc0[qq] = acc1[qq] = make_double2(0, 0);
        for (int ci = Pl.ch_start[pb]; ci < Pl.ch_start[pb + 1]; ci++) {
            int cb = Pl.ch_list[ci];
            double yc[3];
            center64(ca, C, cb, yc);
            double rc_, t3[3];
            int cone = classify64(C, x[0] - yc[0], x[1] - yc[1], x[2] - yc[2], rc_, t3);
            int crc = C.cone_map[(long long)cb * C.ncone + cone];
            if (crc < 0) {
                if (q0 == 0) atomicAdd(ca.missed, 1ULL);
                continue;
            }
            double Ls[PS], Lt[PA], Lp[PA];
            lagrange<PS, double>(t3[0], tb.xs, tb.cs, Ls);
            lagrange<PA, double>(t3[1], tb.xa, tb.ca, Lt);
            lagrange<PA, double>(t3[2], tb.xa, tb.ca, Lp);
            double sn, cs;
            sincos(ca.k * (rc_ - rp), &sn, &cs);
            double g1 = rp / rc_;
            double2 ratio1 = make_double2(cs * g1, sn * g1);
            double2 ratio2 = make_double2(ratio1.x * g1, ratio1.y * g1);
#pragma unroll
            for (int qq = 0; qq < kRB; qq++) {
                if (q0 + qq >= ca.nrhs) continue;
                long long base = ((long long)(q0 + qq) * C.nrc + crc) * C.nfac;
                double vr, vi;
                interp3<PS, PA, double>(FC + base * ca.Pstride, Ls, Lt, Lp, vr, vi);
                if (C.split) {
                    double wr, wi;
                    interp3<PS, PA, double>(FC + (base + 1) * ca.Pstride, Ls, Lt, Lp, wr, wi);
                    if (Pl.split) {
                        double2 t0 = cmul(make_double2(vr, vi), ratio2), t1 = cmul(make_double2(wr, wi), ratio1);
                        acc0[qq].x += t0.x; acc0[qq].y += t0.y;
                        acc1[qq].x += t1.x; acc1[qq].y += t1.y;
                    } else {
                        double ir = 1.0 / rc_;
                        double2 t0 = cmul(make_double2(vr * ir + wr, vi * ir + wi), ratio1);
                        acc0[qq].x += t0.x; acc0[qq].y += t0.y;
                    }
                } else {
                    double2 t0 = cmul(make_double2(vr, vi), ratio1);
                    acc0[qq].x += t0.x; acc0[qq].y += t0.y;
                }
            }
        }
#pragma unroll
        for (int qq = 0; qq < kRB; qq++) {
            if (q0 + qq < ca.nrhs) {
                long long base = ((long long)(q0 + qq) * Pl.nrc + rc) * Pl.nfac;
                FP[base * ca.Pstride + n] = acc0[qq];
                if (Pl.split) FP[(base + 1) * ca.Pstride + n] = acc1[qq];
            }
        }
    }
}

// K4 (FP64): level-D neighbour interactions by direct summation.
__global__ void __launch_bounds__(kBlock) k_near64(CommonArgs ca, LevelArgs L, const double2 *__restrict__ a,
                                                   double2 *__restrict__ u) {
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= ca.N) return;
    int b = ca.leaf_of[i];
    const double x0 = ca.x64[3 * i], x1 = ca.x64[3 * i + 1], x2 = ca.x64[3 * i + 2];
    const double k = ca.k, eta = ca.eta, c4 = 1.0 / (4.0 * kPi);
    for (int q0 = 0; q0 < ca.nrhs; q0 += kRB) {
        double2 acc[kRB];
#pragma unroll
        for (int qq = 0; qq < kRB; qq++) acc[qq] = make_double2(0, 0);
        for (int nb = ca.nb_start[b]; nb < ca.nb_start[b + 1]; nb++) {
            int c = ca.nb_list[nb];
            for (int j = L.start[c]; j < L.start[c + 1]; j++) {
                if (j == i) continue;
                double d0 = x0 - ca.x64[3 * j], d1 = x1 - ca.x64[3 * j + 1], d2 = x2 - ca.x64[3 * j + 2];
                double r = sqrt(d0 * d0 + d1 * d1 + d2 * d2);
                if (r < ca.tol) continue;
                double sn, cs;
                sincos(k * r, &sn, &cs);
                double ir = 1.0 / r;
                double dn = d0 * ca.n64[3 * j] + d1 * ca.n64[3 * j + 1] + d2 * ca.n64[3 * j + 2];
                // K = e^{ikr}/(4 pi r) [ (1 - i k r) dn / r^2 - i eta ]
                double A = dn * ir * ir, B = -(k * dn * ir + eta);
                double2 K = make_double2(c4 * ir * (cs * A - sn * B), c4 * ir * (sn * A + cs * B));
#pragma unroll
                for (int qq = 0; qq < kRB; qq++) {
                    if (q0 + qq < ca.nrhs) {
                        double2 t = cmul(K, a[(long long)(q0 + qq) * ca.N + j]);
                        acc[qq].x += t.x;
                        acc[qq].y += t.y;
                    }
                }
            }
        }
#pragma unroll
        for (int qq = 0; qq < kRB; qq++)
            if (q0 + qq < ca.nrhs) u[(long long)(q0 + qq) * ca.N + i] = acc[qq];
    }
}

// K2 (FP64): u(x) += sum over cousin boxes of level d of E(x;y_k) Interp(F_k)(x).
template <int PS, int PA>
__global__ void __launch_bounds__(kBlock) k_cousin64(CommonArgs ca, LevelArgs L, const int *__restrict__ box_of,
                                                     ChebTab tb, double2 *__restrict__ u) {
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= ca.N) return;
    int b = box_of[i];
    const double x0 = ca.x64[3 * i], x1 = ca.x64[3 * i + 1], x2 = ca.x64[3 * i + 2];
    const double2 *F = (const double2 *)L.F;
    const double c4 = 1.0 / (4.0 * kPi);
    for (int q0 = 0; q0 < ca.nrhs; q0 += kRB) {
        double2 acc[kRB];
#pragma unroll
        for (int qq = 0; qq < kRB; qq++) acc[qq] = make_double2(0, 0);
        for (int ci = L.co_start[b]; ci < L.co_start[b + 1]; ci++) {
            int c = L.co_list[ci];
            double y0[3];
            center64(ca, L, c, y0);
            double r, t3[3];
            int cone = classify64(L, x0 - y0[0], x1 - y0[1], x2 - y0[2], r, t3);
            int rc = L.cone_map[(long long)c * L.ncone + cone];
            if (rc < 0) {
                if (q0 == 0) atomicAdd(ca.missed, 1ULL);
                continue;
            }
            double Ls[PS], Lt[PA], Lp[PA];
            lagrange<PS, double>(t3[0], tb.xs, tb.cs, Ls);
            lagrange<PA, double>(t3[1], tb.xa, tb.ca, Lt);
            lagrange<PA, double>(t3[2], tb.xa, tb.ca, Lp);
            double sn, cs;
            sincos(ca.k * r, &sn, &cs);
            double ir = 1.0 / r;
            double2 E1 = make_double2(c4 * ir * cs, c4 * ir * sn);
#pragma unroll
            for (int qq = 0; qq < kRB; qq++) {
                if (q0 + qq >= ca.nrhs) continue;
                long long base = ((long long)(q0 + qq) * L.nrc + rc) * L.nfac;
                double vr, vi;
                interp3<PS, PA, double>(F + base * ca.Pstride, Ls, Lt, Lp, vr, vi);
                if (L.split) {
                    double wr, wi;
                    interp3<PS, PA, double>(F + (base + 1) * ca.Pstride, Ls, Lt, Lp, wr, wi);
                    vr = vr * ir + wr;
                    vi = vi * ir + wi;
                }
                double2 t = cmul(E1, make_double2(vr, vi));
                acc[qq].x += t.x;
                acc[qq].y += t.y;
            }
        }
#pragma unroll
        for (int qq = 0; qq < kRB; qq++) {
            if (q0 + qq < ca.nrhs) {
                long long o = (long long)(q0 + qq) * ca.N + i;
                double2 v = u[o];
                v.x += acc[qq].x;
                v.y += acc[qq].y;
                u[o] = v;
            }
        }
    }
}

// ============================================================================
// Mixed kernels: FP32 arithmetic in leaf-box units, exact phase reduction,
// compensated FP32 accumulation.
// ============================================================================
struct CAcc {
    float sr, cr, si, ci;
    __device__ __forceinline__ void zero() { sr = cr = si = ci = 0.f; }
    __device__ __forceinline__ void add(float re, float im) {
        comp_add(sr, cr, re);
        comp_add(si, ci, im);
    }
    __device__ __forceinline__ float2 get() const { return make_float2(sr + cr, si + ci); }
};

template <int PS, int PA>
__device__ __forceinline__ void node32(const LevelArgs &L, const ChebTab &tb, int cone, int n, float &s, float *u) {
    int ip = cone % L.nph, it = (cone / L.nph) % L.nC, is = cone / (L.nph * L.nC);
    int ia = n / (PA * PA), ib = (n / PA) % PA, ic = n % PA;
    s = (is + 0.5f * (tb.fxs[ia] + 1.f)) * L.fds;
    float th = (it + 0.5f * (tb.fxa[ib] + 1.f)) * L.fdth;
    float ph = (ip + 0.5f * (tb.fxa[ic] + 1.f)) * L.fdph;
    float st, ct, sp, cp;
    sincosf(th, &st, &ct);
    sincosf(ph, &sp, &cp);
    u[0] = st * cp;
    u[1] = st * sp;
    u[2] = ct;
}

// cone id and local coordinates of the point at leaf-unit offset p from a box centre
__device__ __forceinline__ int classify32(const LevelArgs &L, float px, float py, float pz, float r, float *t3) {
    float rho = sqrtf(px * px + py * py);
    float s = L.hu / r;
    float th = atan2f(rho, pz);
    float ph = atan2f(py, px);
    if (ph < 0.f) ph += 2.f * kPiF;
    float us = s * L.inv_ds, ut = th * L.inv_dth, up = ph * L.inv_dph;
    int is = min((int)us, L.ns - 1), it = min((int)ut, L.nC - 1), ip = min((int)up, L.nph - 1);
    is = max(is, 0);
    it = max(it, 0);
    ip = max(ip, 0);
    t3[0] = 2.f * (us - is) - 1.f;
    t3[1] = 2.f * (ut - it) - 1.f;
    t3[2] = 2.f * (up - ip) - 1.f;
    return (is * L.nC + it) * L.nph + ip;
}

// e^{2 pi i t} for |t| <= 1/2 (t already reduced)
__device__ __forceinline__ void cis_cycles(float t, float &sn, float &cs) { __sincosf(2.f * kPiF * t, &sn, &cs); }

// K1 (mixed)
template <int PS, int PA>
__global__ void __launch_bounds__(kBlock) k_leaf32(CommonArgs ca, LevelArgs L, ChebTab tb, const float2 *__restrict__ a) {
    constexpr int P = PS * PA * PA;
    long long tid = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (tid >= L.nrc * P) return;
    int rc = (int)(tid / P), n = (int)(tid % P);
    int b = L.rc_box[rc];
    float s, u[3];
    node32<PS, PA>(L, tb, L.rc_cone[rc], n, s, u);
    const float hu = L.hu;                 // h in leaf units
    const float ir = s / hu;               // 1 / r (leaf units)
    const float kap = ca.kappa_hi;         // k HD / (2 pi)
    const float soh = s / (hu * ca.HDf);   // s / h (absolute)
    const float kf = ca.kf, etaf = ca.etaf;
    const int j0 = L.start[b], j1 = L.start[b + 1];
    float2 *F = (float2 *)L.F;
    for (int q0 = 0; q0 < ca.nrhs; q0 += kRB) {
        CAcc acc0[kRB], acc1[kRB];
#pragma unroll
        for (int qq = 0; qq < kRB; qq++) {
            acc0[qq].zero();
            acc1[qq].zero();
        }
        for (int j = j0; j < j1; j++) {
            const float f0 = ca.f32[3 * j], f1 = ca.f32[3 * j + 1], f2 = ca.f32[3 * j + 2];
            float dv0 = u[0] - f0 * ir, dv1 = u[1] - f1 * ir, dv2 = u[2] - f2 * ir;
            float a2 = dv0 * dv0 + dv1 * dv1 + dv2 * dv2;
            float ia = rsqrtf(a2);
            float am = a2 * ia;
            float yy = f0 * f0 + f1 * f1 + f2 * f2;
            float uy = u[0] * f0 + u[1] * f1 + u[2] * f2;
            float t = kap * (s * yy / hu - 2.f * uy) / (am + 1.f);
            t -= rintf(t);
            float sn, cs;
            cis_cycles(t, sn, cs);
            float dn = dv0 * ca.n32[3 * j] + dv1 * ca.n32[3 * j + 1] + dv2 * ca.n32[3 * j + 2];
            float w3 = dn * ia * ia, w2 = w3 * ia;
            float g = kf * w3 + etaf * ia;
            float W0r, W0i, W1r = 0.f, W1i = 0.f;
            if (L.split) {
                W0r = cs * w2;
                W0i = sn * w2;
                W1r = sn * g;
                W1i = -cs * g;
            } else {
                W0r = cs * soh * w2 + sn * g;
                W0i = sn * soh * w2 - cs * g;
            }
#pragma unroll
            for (int qq = 0; qq < kRB; qq++) {
                if (q0 + qq < ca.nrhs) {
                    float2 aj = a[(long long)(q0 + qq) * ca.N + j];
                    acc0[qq].add(aj.x * W0r - aj.y * W0i, aj.x * W0i + aj.y * W0r);
                    if (L.split) acc1[qq].add(aj.x * W1r - aj.y * W1i, aj.x * W1i + aj.y * W1r);
                }
            }
        }
#pragma unroll
        for (int qq = 0; qq < kRB; qq++) {
            if (q0 + qq < ca.nrhs) {
                long long base = ((long long)(q0 + qq) * L.nrc + rc) * L.nfac;
                F[base * ca.Pstride + n] = acc0[qq].get();
                if (L.split) F[(base + 1) * ca.Pstride + n] = acc1[qq].get();
            }
        }
    }
}

// K3 (mixed)
template <int PS, int PA>
__global__ void __launch_bounds__(kBlock) k_prop32(CommonArgs ca, LevelArgs C, LevelArgs Pl, ChebTab tb) {
    constexpr int P = PS * PA * PA;
    long long tid = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (tid >= Pl.nrc * P) return;
    int rc = (int)(tid / P), n = (int)(tid % P);
    int pb = Pl.rc_box[rc];
    float s, u[3];
    node32<PS, PA>(Pl, tb, Pl.rc_cone[rc], n, s, u);
    const float rp = Pl.hu / s;  // leaf units
    const float nv[3] = {rp * u[0], rp * u[1], rp * u[2]};
    const float pc[3] = {(Pl.ijk[3 * pb] + 0.5f) * Pl.scale, (Pl.ijk[3 * pb + 1] + 0.5f) * Pl.scale,
                         (Pl.ijk[3 * pb + 2] + 0.5f) * Pl.scale};
    const float2 *FC = (const float2 *)C.F;
    float2 *FP = (float2 *)Pl.F;
    for (int q0 = 0; q0 < ca.nrhs; q0 += kRB) {
        CAcc acc0[kRB], acc1[kRB];
#pragma unroll
        for (int qq = 0; qq < kRB; qq++) {
            acc0[qq].zero();
            acc1[qq].zero();
        }
        for (int ci = Pl.ch_start[pb]; ci < Pl.ch_start[pb + 1]; ci++) {
            int cb = Pl.ch_list[ci];
            // child centre minus parent centre, exact in leaf units
            float o0 = (C.ijk[3 * cb] + 0.5f) * C.scale - pc[0];
            float o1 = (C.ijk[3 * cb + 1] + 0.5f) * C.scale - pc[1];
            float o2 = (C.ijk[3 * cb + 2] + 0.5f) * C.scale - pc[2];
            float p0 = nv[0] - o0, p1 = nv[1] - o1, p2 = nv[2] - o2;
            float rc_ = sqrtf(p0 * p0 + p1 * p1 + p2 * p2);
            float t3[3];
            int cone = classify32(C, p0, p1, p2, rc_, t3);
            int crc = C.cone_map[(long long)cb * C.ncone + cone];
            if (crc < 0) {
                if (q0 == 0) atomicAdd(ca.missed, 1ULL);
                continue;
            }
            float Ls[PS], Lt[PA], Lp[PA];
            lagrange<PS, float>(t3[0], tb.fxs, tb.fcs, Ls);
            lagrange<PA, float>(t3[1], tb.fxa, tb.fca, Lt);
            lagrange<PA, float>(t3[2], tb.fxa, tb.fca, Lp);
            // r_c - r_p = (|o|^2 - 2 n.o) / (r_c + r_p), free of cancellation
            float oo = o0 * o0 + o1 * o1 + o2 * o2;
            float no = nv[0] * o0 + nv[1] * o1 + nv[2] * o2;
            float dr = (oo - 2.f * no) / (rc_ + rp);
            float t = ca.kappa_hi * dr;
            t -= rintf(t);
            float sn, cs;
            cis_cycles(t, sn, cs);
            float g1 = rp / rc_;
            float r1r = cs * g1, r1i = sn * g1;
            float r2r = r1r * g1, r2i = r1i * g1;
            float irabs = 1.f / (rc_ * ca.HDf);
#pragma unroll
            for (int qq = 0; qq < kRB; qq++) {
                if (q0 + qq >= ca.nrhs) continue;
                long long base = ((long long)(q0 + qq) * C.nrc + crc) * C.nfac;
                float vr, vi;
                interp3<PS, PA, float>(FC + base * ca.Pstride, Ls, Lt, Lp, vr, vi);
                if (C.split) {
                    float wr, wi;
                    interp3<PS, PA, float>(FC + (base + 1) * ca.Pstride, Ls, Lt, Lp, wr, wi);
                    if (Pl.split) {
                        acc0[qq].add(vr * r2r - vi * r2i, vr * r2i + vi * r2r);
                        acc1[qq].add(wr * r1r - wi * r1i, wr * r1i + wi * r1r);
                    } else {
                        float zr = vr * irabs + wr, zi = vi * irabs + wi;
                        acc0[qq].add(zr * r1r - zi * r1i, zr * r1i + zi * r1r);
                    }
                } else {
                    acc0[qq].add(vr * r1r - vi * r1i, vr * r1i + vi * r1r);
                }
            }
        }
#pragma unroll
        for (int qq = 0; qq < kRB; qq++) {
            if (q0 + qq < ca.nrhs) {
                long long base = ((long long)(q0 + qq) * Pl.nrc + rc) * Pl.nfac;
                FP[base * ca.Pstride + n] = acc0[qq].get();
                if (Pl.split) FP[(base + 1) * ca.Pstride + n] = acc1[qq].get();
            }
        }
    }
}

// K4 (mixed)
__global__ void __launch_bounds__(kBlock) k_near32(CommonArgs ca, LevelArgs L, const float2 *__restrict__ a,
                                                   float2 *__restrict__ u) {
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= ca.N) return;
    int b = ca.leaf_of[i];
    const int bi0 = L.ijk[3 * b], bi1 = L.ijk[3 * b + 1], bi2 = L.ijk[3 * b + 2];
    const float fx0 = ca.f32[3 * i], fx1 = ca.f32[3 * i + 1], fx2 = ca.f32[3 * i + 2];
    const float kf = ca.kf, etaf = ca.etaf, kap = ca.kappa_hi;
    const float c4 = 1.f / (4.f * kPiF * ca.HDf), iHD = 1.f / ca.HDf;
    const float tolu = (float)(ca.tol / ca.HD);
    for (int q0 = 0; q0 < ca.nrhs; q0 += kRB) {
        CAcc acc[kRB];
#pragma unroll
        for (int qq = 0; qq < kRB; qq++) acc[qq].zero();
        for (int nb = ca.nb_start[b]; nb < ca.nb_start[b + 1]; nb++) {
            int c = ca.nb_list[nb];
            const float D0 = (float)(bi0 - L.ijk[3 * c]) + fx0, D1 = (float)(bi1 - L.ijk[3 * c + 1]) + fx1,
                        D2 = (float)(bi2 - L.ijk[3 * c + 2]) + fx2;
            for (int j = L.start[c]; j < L.start[c + 1]; j++) {
                if (j == i) continue;
                float d0 = D0 - ca.f32[3 * j], d1 = D1 - ca.f32[3 * j + 1], d2 = D2 - ca.f32[3 * j + 2];
                float r2 = d0 * d0 + d1 * d1 + d2 * d2;
                float ir = rsqrtf(r2);
                float r = r2 * ir;
                if (!(r >= tolu)) continue;
                float t = kap * r;
                t -= rintf(t);
                float sn, cs;
                cis_cycles(t, sn, cs);
                float dn = d0 * ca.n32[3 * j] + d1 * ca.n32[3 * j + 1] + d2 * ca.n32[3 * j + 2];
                // K = e^{ikR}/(4 pi R) [ dn_u / (r^2 HD) - i (k dn_u / r + eta) ],  R = r HD
                float A = dn * ir * ir * iHD, B = -(kf * dn * ir + etaf);
                float amp = c4 * ir;
                float Kr = amp * (cs * A - sn * B), Ki = amp * (sn * A + cs * B);
#pragma unroll
                for (int qq = 0; qq < kRB; qq++) {
                    if (q0 + qq < ca.nrhs) {
                        float2 aj = a[(long long)(q0 + qq) * ca.N + j];
                        acc[qq].add(Kr * aj.x - Ki * aj.y, Kr * aj.y + Ki * aj.x);
                    }
                }
            }
        }
#pragma unroll
        for (int qq = 0; qq < kRB; qq++)
            if (q0 + qq < ca.nrhs) u[(long long)(q0 + qq) * ca.N + i] = acc[qq].get();
    }
}

// K2 (mixed)
template <int PS, int PA>
__global__ void __launch_bounds__(kBlock) k_cousin32(CommonArgs ca, LevelArgs L, LevelArgs LD, const int *__restrict__ box_of,
                                                     ChebTab tb, float2 *__restrict__ u) {
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= ca.N) return;
    int b = box_of[i];
    int bl = ca.leaf_of[i];
    const float I0 = LD.ijk[3 * bl] + 0.5f, I1 = LD.ijk[3 * bl + 1] + 0.5f, I2 = LD.ijk[3 * bl + 2] + 0.5f;
    const float f0 = ca.f32[3 * i], f1 = ca.f32[3 * i + 1], f2 = ca.f32[3 * i + 2];
    const float2 *F = (const float2 *)L.F;
    const float c4 = 1.f / (4.f * kPiF * ca.HDf), iHD = 1.f / ca.HDf;
    const float sc = (float)L.scale;
    for (int q0 = 0; q0 < ca.nrhs; q0 += kRB) {
        CAcc acc[kRB];
#pragma unroll
        for (int qq = 0; qq < kRB; qq++) acc[qq].zero();
        for (int ci = L.co_start[b]; ci < L.co_start[b + 1]; ci++) {
            int c = L.co_list[ci];
            float M0 = I0 - (L.ijk[3 * c] + 0.5f) * sc, M1 = I1 - (L.ijk[3 * c + 1] + 0.5f) * sc,
                  M2 = I2 - (L.ijk[3 * c + 2] + 0.5f) * sc;
            float r;
            float t = phase_cycles_exact(M0, M1, M2, f0, f1, f2, ca.kappa_hi, ca.kappa_lo, r);
            float t3[3];
            int cone = classify32(L, M0 + f0, M1 + f1, M2 + f2, r, t3);
            int rc = L.cone_map[(long long)c * L.ncone + cone];
            if (rc < 0) {
                if (q0 == 0) atomicAdd(ca.missed, 1ULL);
                continue;
            }
            float Ls[PS], Lt[PA], Lp[PA];
            lagrange<PS, float>(t3[0], tb.fxs, tb.fcs, Ls);
            lagrange<PA, float>(t3[1], tb.fxa, tb.fca, Lt);
            lagrange<PA, float>(t3[2], tb.fxa, tb.fca, Lp);
            float sn, cs;
            cis_cycles(t, sn, cs);
            float ir = 1.f / r;
            float E1r = c4 * ir * cs, E1i = c4 * ir * sn;
            float irabs = ir * iHD;
#pragma unroll
            for (int qq = 0; qq < kRB; qq++) {
                if (q0 + qq >= ca.nrhs) continue;
                long long base = ((long long)(q0 + qq) * L.nrc + rc) * L.nfac;
                float vr, vi;
                interp3<PS, PA, float>(F + base * ca.Pstride, Ls, Lt, Lp, vr, vi);
                if (L.split) {
                    float wr, wi;
                    interp3<PS, PA, float>(F + (base + 1) * ca.Pstride, Ls, Lt, Lp, wr, wi);
                    vr = vr * irabs + wr;
                    vi = vi * irabs + wi;
                }
                acc[qq].add(E1r * vr - E1i * vi, E1r * vi + E1i * vr);
            }
        }
#pragma unroll
        for (int qq = 0; qq < kRB; qq++) {
            if (q0 + qq < ca.nrhs) {
                long long o = (long long)(q0 + qq) * ca.N + i;
                float2 v = u[o], w = acc[qq].get();
                v.x += w.x;
                v.y += w.y;
                u[o] = v;
            }
        }
    }
}

// ============================================================================
// host side
// ============================================================================
template <typename T>
static T *dalloc(Plan &p, size_t n, cudaError_t &err) {
    void *ptr = nullptr;
    err = cudaMalloc(&ptr, n * sizeof(T) + 16);
    if (err != cudaSuccess) return nullptr;
    p.allocs.push_back(ptr);
    p.device_bytes += (int64_t)(n * sizeof(T) + 16);
    return (T *)ptr;
}

template <typename T>
static ifgf_status upload(Plan &p, T *&dst, const T *src, size_t n, cudaStream_t s) {
    cudaError_t err;
    dst = dalloc<T>(p, n > 0 ? n : 1, err);
    if (!dst) {
        set_error("cudaMalloc(%zu bytes) failed: %s", n * sizeof(T), cudaGetErrorString(err));
        return err == cudaErrorMemoryAllocation ? IFGF_ENOMEM : IFGF_ECUDA;
    }
    if (n) CK(cudaMemcpyAsync(dst, src, n * sizeof(T), cudaMemcpyHostToDevice, s));
    return IFGF_OK;
}

#define UP(dst, vec)                                                               \
    do {                                                                           \
        ifgf_status st_ = upload(p, dst, (vec).data(), (vec).size(), s);           \
        if (st_ != IFGF_OK) return st_;                                            \
    } while (0)

ifgf_status upload_plan(Plan &p, const double *xyz, const double *nrm, const double *w, cudaStream_t s) {
    CK(cudaGetDevice(&p.device));
    const int64_t N = p.N;
    const int D = p.D;
    std::vector<double> x64(3 * N), n64(3 * N), w64(N);
    std::vector<float> f32(3 * N), n32(3 * N), w32(N);
    const HostLevel &LD = p.lv[D];
    for (int64_t si = 0; si < N; si++) {
        int o = p.perm[si];
        int b = p.leaf_of[si];
        for (int a = 0; a < 3; a++) {
            x64[3 * si + a] = xyz[3 * o + a];
            n64[3 * si + a] = nrm[3 * o + a];
            double cen = p.c0[a] + (LD.ijk[3 * b + a] + 0.5) * p.HD;
            f32[3 * si + a] = (float)((xyz[3 * o + a] - cen) / p.HD);
            n32[3 * si + a] = (float)nrm[3 * o + a];
        }
        w64[si] = w[o];
        w32[si] = (float)w[o];
    }
    UP(p.d_x64, x64);
    UP(p.d_n64, n64);
    UP(p.d_w64, w64);
    UP(p.d_f32, f32);
    UP(p.d_n32, n32);
    UP(p.d_w32, w32);
    UP(p.d_perm, p.perm);
    UP(p.d_leaf_of, p.leaf_of);
    UP(p.d_nb_start, p.nb_start);
    UP(p.d_nb_list, p.nb_list);
    for (int d = 3; d <= D; d++) {
        const HostLevel &L = p.lv[d];
        DevLevel &dl = p.dl[d];
        dl.nbox = L.nbox; dl.ns = L.ns; dl.nC = L.nC; dl.nph = L.nph; dl.ncone = L.ncone;
        dl.split = L.split; dl.nfac = L.nfac; dl.scale = L.scale; dl.nrc = L.nrc;
        dl.H = L.H; dl.h = L.h; dl.ds = L.ds; dl.dth = L.dth; dl.dph = L.dph;
        UP(dl.ijk, L.ijk);
        UP(dl.start, L.start);
        UP(dl.parent, L.parent);
        UP(dl.ch_start, L.ch_start);
        UP(dl.ch_list, L.ch_list);
        UP(dl.co_start, L.co_start);
        UP(dl.co_list, L.co_list);
        UP(dl.rc_start, L.rc_start);
        UP(dl.rc_cone, L.rc_cone);
        UP(dl.rc_box, L.rc_box);
        UP(dl.cone_map, L.cone_map);
        std::vector<int> box_of(N);
        for (int b = 0; b < L.nbox; b++)
            for (int si = L.start[b]; si < L.start[b + 1]; si++) box_of[si] = b;
        UP(p.d_box_of[d], box_of);
    }
    {
        cudaError_t err;
        p.d_missed = dalloc<unsigned long long>(p, 1, err);
        if (!p.d_missed) {
            set_error("cudaMalloc failed: %s", cudaGetErrorString(err));
            return IFGF_ENOMEM;
        }
        CK(cudaMemsetAsync(p.d_missed, 0, sizeof(unsigned long long), s));
    }
    CK(cudaStreamSynchronize(s));
    return IFGF_OK;
}

void free_plan_device(Plan &p) {
    for (int i = 0; i < Plan::kMaxEv; i++)
        if (p.ev[i]) {
            cudaEventDestroy(p.ev[i]);
            p.ev[i] = nullptr;
        }
    for (void *a : p.allocs) cudaFree(a);
    p.allocs.clear();
    if (p.ws.base) cudaFree(p.ws.base);
    p.ws = Workspace();
}

ifgf_status ensure_workspace(Plan &p, int nrhs, int prec) {
    if (p.ws.base && p.ws.nrhs >= nrhs && p.ws.prec == prec) return IFGF_OK;
    const size_t cb = prec == IFGF_FP64 ? 16 : 8;  // bytes per complex
    auto al = [](size_t x) { return (x + 255) & ~(size_t)255; };
    size_t off = 0;
    size_t oa = off; off += al(cb * p.N * nrhs);
    size_t ou = off; off += al(cb * p.N * nrhs);
    size_t oF[IFGF_MAXD + 1] = {};
    for (int d = 3; d <= p.D; d++) {
        oF[d] = off;
        off += al(cb * (size_t)nrhs * p.lv[d].nrc * p.lv[d].nfac * p.Pstride);
    }
    if (p.ws.base) cudaFree(p.ws.base);
    p.ws = Workspace();
    void *base = nullptr;
    cudaError_t e = cudaMalloc(&base, off);
    if (e != cudaSuccess) {
        set_error("workspace cudaMalloc(%zu bytes) failed: %s", off, cudaGetErrorString(e));
        return e == cudaErrorMemoryAllocation ? IFGF_ENOMEM : IFGF_ECUDA;
    }
    p.ws.base = base;
    p.ws.bytes = off;
    p.ws.nrhs = nrhs;
    p.ws.prec = prec;
    char *c = (char *)base;
    p.ws.a = c + oa;
    p.ws.u = c + ou;
    for (int d = 3; d <= p.D; d++) p.ws.F[d] = c + oF[d];
    return IFGF_OK;
}

static LevelArgs level_args(const Plan &p, int d, void *F) {
    const DevLevel &dl = p.dl[d];
    LevelArgs a;
    a.nbox = dl.nbox; a.ns = dl.ns; a.nC = dl.nC; a.nph = dl.nph; a.ncone = dl.ncone;
    a.split = dl.split; a.nfac = dl.nfac; a.scale = dl.scale; a.nrc = dl.nrc;
    a.H = dl.H; a.h = dl.h; a.ds = dl.ds; a.dth = dl.dth; a.dph = dl.dph;
    a.hu = (float)(std::sqrt(3.0) / 2.0 * dl.scale);
    a.inv_ds = (float)(1.0 / dl.ds); a.inv_dth = (float)(1.0 / dl.dth); a.inv_dph = (float)(1.0 / dl.dph);
    a.fds = (float)dl.ds; a.fdth = (float)dl.dth; a.fdph = (float)dl.dph;
    a.ijk = dl.ijk; a.start = dl.start; a.ch_start = dl.ch_start; a.ch_list = dl.ch_list;
    a.co_start = dl.co_start; a.co_list = dl.co_list; a.rc_start = dl.rc_start; a.rc_cone = dl.rc_cone;
    a.rc_box = dl.rc_box; a.cone_map = dl.cone_map;
    a.F = F;
    return a;
}

static CommonArgs common_args(const Plan &p, int nrhs) {
    CommonArgs c;
    c.N = (int)p.N; c.nrhs = nrhs; c.D = p.D; c.Pstride = p.Pstride;
    c.k = p.prm.k; c.eta = p.prm.eta; c.HD = p.HD; c.L = p.L; c.tol = 1e-14 * p.L;
    for (int a = 0; a < 3; a++) c.c0[a] = p.c0[a];
    c.kf = (float)p.prm.k; c.etaf = (float)p.prm.eta; c.HDf = (float)p.HD;
    double kap = p.prm.k * p.HD / (2.0 * kPi);
    c.kappa_hi = (float)kap;
    c.kappa_lo = (float)(kap - (double)c.kappa_hi);
    c.leaf_of = p.d_leaf_of; c.nb_start = p.d_nb_start; c.nb_list = p.d_nb_list;
    c.x64 = p.d_x64; c.n64 = p.d_n64; c.w64 = p.d_w64;
    c.f32 = p.d_f32; c.n32 = p.d_n32; c.w32 = p.d_w32;
    c.missed = p.d_missed;
    return c;
}

static ChebTab cheb_tab(const Plan &p) {
    ChebTab t;
    for (int j = 0; j < 12; j++) {
        t.xs[j] = j < p.Ps ? p.cs.x[j] : 0; t.cs[j] = j < p.Ps ? p.cs.c[j] : 0;
        t.xa[j] = j < p.Pang ? p.ca.x[j] : 0; t.ca[j] = j < p.Pang ? p.ca.c[j] : 0;
        t.fxs[j] = (float)t.xs[j]; t.fcs[j] = (float)t.cs[j]; t.fxa[j] = (float)t.xa[j]; t.fca[j] = (float)t.ca[j];
    }
    return t;
}

static unsigned nblk(long long n) { return (unsigned)((n + kBlock - 1) / kBlock); }

template <int PS, int PA>
static ifgf_status run_apply_t(Plan &p, const void *sigma, void *y, int nrhs, int prec, cudaStream_t s) {
    constexpr int P = PS * PA * PA;
    const int D = p.D;
    const int N = (int)p.N;
    CommonArgs ca = common_args(p, nrhs);
    ChebTab tb = cheb_tab(p);
    LevelArgs L[IFGF_MAXD + 1];
    for (int d = 3; d <= D; d++) L[d] = level_args(p, d, p.ws.F[d]);
    const long long NT = (long long)N * nrhs;
    prof_begin(p, s);
    if (prec == IFGF_FP64) {
        k_gather<double><<<nblk(NT), kBlock, 0, s>>>(N, nrhs, p.d_perm, p.d_w64, (const double2 *)sigma, (double2 *)p.ws.a);
        prof_mark(p, s, kStGather, 0);
        if (L[D].nrc) {
            k_leaf64<PS, PA><<<nblk(L[D].nrc * P), kBlock, 0, s>>>(ca, L[D], tb, (const double2 *)p.ws.a);
            prof_mark(p, s, kStLeaf, D);
        }
        for (int d = D; d >= 4; d--)
            if (L[d - 1].nrc) {
                k_prop64<PS, PA><<<nblk(L[d - 1].nrc * P), kBlock, 0, s>>>(ca, L[d], L[d - 1], tb);
                prof_mark(p, s, kStProp, d - 1);
            }
        k_near64<<<nblk(N), kBlock, 0, s>>>(ca, L[D], (const double2 *)p.ws.a, (double2 *)p.ws.u);
        prof_mark(p, s, kStNear, D);
        for (int d = D; d >= 3; d--) {
            k_cousin64<PS, PA><<<nblk(N), kBlock, 0, s>>>(ca, L[d], p.d_box_of[d], tb, (double2 *)p.ws.u);
            prof_mark(p, s, kStCousin, d);
        }
        k_scatter<double><<<nblk(NT), kBlock, 0, s>>>(N, nrhs, p.d_perm, p.prm.identity_coef, (const double2 *)sigma,
                                                       (const double2 *)p.ws.u, (double2 *)y);
        prof_mark(p, s, kStScatter, 0);
    } else {
        k_gather<float><<<nblk(NT), kBlock, 0, s>>>(N, nrhs, p.d_perm, p.d_w32, (const float2 *)sigma, (float2 *)p.ws.a);
        prof_mark(p, s, kStGather, 0);
        if (L[D].nrc) {
            k_leaf32<PS, PA><<<nblk(L[D].nrc * P), kBlock, 0, s>>>(ca, L[D], tb, (const float2 *)p.ws.a);
            prof_mark(p, s, kStLeaf, D);
        }
        for (int d = D; d >= 4; d--)
            if (L[d - 1].nrc) {
                k_prop32<PS, PA><<<nblk(L[d - 1].nrc * P), kBlock, 0, s>>>(ca, L[d], L[d - 1], tb);
                prof_mark(p, s, kStProp, d - 1);
            }
        k_near32<<<nblk(N), kBlock, 0, s>>>(ca, L[D], (const float2 *)p.ws.a, (float2 *)p.ws.u);
        prof_mark(p, s, kStNear, D);
        for (int d = D; d >= 3; d--) {
            k_cousin32<PS, PA><<<nblk(N), kBlock, 0, s>>>(ca, L[d], L[D], p.d_box_of[d], tb, (float2 *)p.ws.u);
            prof_mark(p, s, kStCousin, d);
        }
        k_scatter<float><<<nblk(NT), kBlock, 0, s>>>(N, nrhs, p.d_perm, p.prm.identity_coef, (const float2 *)sigma,
                                                      (const float2 *)p.ws.u, (float2 *)y);
        prof_mark(p, s, kStScatter, 0);
    }
    CK(cudaGetLastError());
    return IFGF_OK;
}

ifgf_status run_apply(Plan &p, const void *sigma, void *y, int nrhs, int prec, cudaStream_t s) {
    ifgf_status st = ensure_workspace(p, nrhs, prec);
    if (st != IFGF_OK) return st;
#define IFGF_CASE(a, b) \
    if (p.Ps == a && p.Pang == b) return run_apply_t<a, b>(p, sigma, y, nrhs, prec, s);
    IFGF_CASE(3, 5)
    IFGF_CASE(4, 6)
    IFGF_CASE(5, 7)
    IFGF_CASE(6, 8)
#undef IFGF_CASE
    set_error("orders Ps=%d Pang=%d not compiled", p.Ps, p.Pang);
    return IFGF_EUNSUPPORTED;
}

// Same launches as run_apply on a caller-provided workspace view (no allocation).
ifgf_status run_apply_on(Plan &p, const Workspace &ws, const void *sigma, void *y, int nrhs, int prec,
                         cudaStream_t s) {
    Workspace saved = p.ws;
    p.ws = ws;
    ifgf_status st = IFGF_EUNSUPPORTED;
    if (p.Ps == 3 && p.Pang == 5) st = run_apply_t<3, 5>(p, sigma, y, nrhs, prec, s);
    else if (p.Ps == 4 && p.Pang == 6) st = run_apply_t<4, 6>(p, sigma, y, nrhs, prec, s);
    else if (p.Ps == 5 && p.Pang == 7) st = run_apply_t<5, 7>(p, sigma, y, nrhs, prec, s);
    else if (p.Ps == 6 && p.Pang == 8) st = run_apply_t<6, 8>(p, sigma, y, nrhs, prec, s);
    else set_error("orders Ps=%d Pang=%d not compiled", p.Ps, p.Pang);
    p.ws = saved;
    return st;
}

}  // namespace ifgf

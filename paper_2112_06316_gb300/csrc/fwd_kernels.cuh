// Forward-apply kernels of the IFGF-accelerated CFIE operator on sm_103a
// (included by one instantiation unit per interpolation-order pair).
//
// Pipeline of one apply (Algorithm 1 + Remark level_D_neighboring):
//   gather   a = w * sigma in Morton order
//   K1 leaf  F^D at every relevant level-D cone node (Section 3.4, leaf expansions)
//   K3 prop  for d = D..4: F^{d-1}(x) = sum_children Interp(F^d_child)(x) E(x;y_c)/E(x;y_p)
//   K4 near  u = level-D neighbour interactions by direct summation
//   K2 cous  for d = D..3: u(x) += sum_cousin-boxes E(x;y_k) Interp(F^d_k)(x)
//   scatter  y = c_I sigma + u (+ C sigma) in the caller's order
// Every kernel is output-stationary (one thread owns one output value), so no
// atomics are needed and FP64 results are bitwise reproducible run to run.
#pragma once
#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <type_traits>

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

namespace {  // kernels get internal linkage in each instantiation unit

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

// K1 (FP64): F at the relevant leaf cone nodes.  rc_list: the relevant cones of the leaves of a
// coarser level of an adaptive tree (nlist of them); nullptr: every relevant cone of the level.
template <int PS, int PA>
__global__ void __launch_bounds__(kBlock) k_leaf64(CommonArgs ca, LevelArgs L, ChebTab tb, const double2 *__restrict__ a,
                                                   const int *__restrict__ rc_list, long long nlist) {
    constexpr int P = PS * PA * PA;
    long long tid = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (tid >= nlist * P) return;
    int rc = rc_list ? rc_list[tid / P] : (int)(tid / P), n = (int)(tid % P);
    int b = L.rc_box[rc];
    double s, u[3];
    node64<PS, PA>(L, tb, L.rc_cone[rc], n, s, u);
    double y0[3];
    center64(ca, L, b, y0);
    const double r = L.h / s, k = ca.k, eta = ca.eta, etai = ca.etai, soh = s / L.h;
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
            // -i k W3 - i (eta + i etai) W1 = e (etai w1 - i g),  g = k w3 + eta w1
            const double g = k * w3 + eta * w1, hr = etai * w1;
            if (L.split) {
                W0 = make_double2(cs * w2, sn * w2);
                W1 = make_double2(cs * hr + sn * g, sn * hr - cs * g);
            } else {
                const double a = soh * w2 + hr;
                W0 = make_double2(cs * a + sn * g, sn * a - cs * g);
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
    const double k = ca.k, eta = ca.eta, etai = ca.etai, c4 = 1.0 / (4.0 * kPi);
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
                // K = e^{ikr}/(4 pi r) [ (1 - i k r) dn / r^2 - i (eta + i etai) ]
                double A = dn * ir * ir + etai, B = -(k * dn * ir + eta);
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
                                                     const uint8_t *__restrict__ alive, ChebTab tb,
                                                     double2 *__restrict__ u) {
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= ca.N) return;
    int b = box_of[i];
    if (!alive[b]) return;  // below a coarser leaf: no level-d box for this point
    const double x0 = ca.x64[3 * i], x1 = ca.x64[3 * i + 1], x2 = ca.x64[3 * i + 2];
    const double2 *F = (const double2 *)L.F;
    const double c4 = 1.0 / (4.0 * kPi);
    for (int q0 = 0; q0 < ca.nrhs; q0 += kRB) {
        double2 acc[kRB];
#pragma unroll
        for (int qq = 0; qq < kRB; qq++) acc[qq] = make_double2(0, 0);
        for (int ci = L.co_start[b]; ci < L.co_start[b + 1]; ci++) {
            int c = L.co_list[ci];
            if (L.rc_start[c] == L.rc_start[c + 1]) continue;  // no sources in c
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
// Kahan-compensated complex accumulator (four adds per component, no compare):
// the running correction c holds the negated low part lost by the last add.
__device__ __forceinline__ void kahan_add(float &s, float &c, float x) {
    const float y = __fsub_rn(x, c);
    const float t = __fadd_rn(s, y);
    c = __fsub_rn(__fsub_rn(t, s), y);
    s = t;
}

// plain FP32 complex sum (random-phase sums of comparable terms: the rounding error stays at the
// level of one rounding of the result)
struct PAcc {
    float sr, si;
    __device__ __forceinline__ void zero() { sr = si = 0.f; }
    __device__ __forceinline__ void add(float re, float im) {
        sr += re;
        si += im;
    }
    __device__ __forceinline__ float2 get() const { return make_float2(sr, si); }
};

struct CAcc {
    float sr, cr, si, ci;
    __device__ __forceinline__ void zero() { sr = cr = si = ci = 0.f; }
    __device__ __forceinline__ void add(float re, float im) {
        kahan_add(sr, cr, re);
        kahan_add(si, ci, im);
    }
    __device__ __forceinline__ float2 get() const { return make_float2(sr - cr, si - ci); }
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

// K1 (mixed).  RB right-hand sides per pass; SPLIT = the level stores the two
// factors {W2, W13} instead of the combined one.
template <int PS, int PA, int RB, bool SPLIT>
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
    const float kf = ca.kf, etaf = ca.etaf, etaif = ca.etaif;
    const int j0 = L.start[b], j1 = L.start[b + 1];
    const float4 *pn = ca.pn32;
    float2 *F = (float2 *)L.F;
    for (int q0 = 0; q0 < ca.nrhs; q0 += RB) {
        PAcc acc0[RB], acc1[RB];
#pragma unroll
        for (int qq = 0; qq < RB; qq++) {
            acc0[qq].zero();
            acc1[qq].zero();
        }
        for (int j = j0; j < j1; j++) {
            const float4 fj = __ldg(pn + 2 * j), nj = __ldg(pn + 2 * j + 1);
            float dv0 = u[0] - fj.x * ir, dv1 = u[1] - fj.y * ir, dv2 = u[2] - fj.z * ir;
            float a2 = dv0 * dv0 + dv1 * dv1 + dv2 * dv2;
            float ia = rsqrtf(a2);
            float am = a2 * ia;
            const float yy = fj.w;  // |f|^2
            float uy = u[0] * fj.x + u[1] * fj.y + u[2] * fj.z;
            // (|x - y| - |x|) / (h / s) in leaf units; am + 1 lies in [1, 3]: the fast divide is exact to 2 ulp
            float t = kap * __fdividef(ir * yy - 2.f * uy, am + 1.f);
            t -= rintf(t);
            float sn, cs;
            cis_cycles(t, sn, cs);
            float dn = dv0 * nj.x + dv1 * nj.y + dv2 * nj.z;
            float w3 = dn * ia * ia, w2 = w3 * ia;
            float g = kf * w3 + etaf * ia, hr = etaif * ia;
            float W0r, W0i, W1r = 0.f, W1i = 0.f;
            if (SPLIT) {
                W0r = cs * w2;
                W0i = sn * w2;
                W1r = cs * hr + sn * g;
                W1i = sn * hr - cs * g;
            } else {
                const float w2s = soh * w2 + hr;
                W0r = cs * w2s + sn * g;
                W0i = sn * w2s - cs * g;
            }
#pragma unroll
            for (int qq = 0; qq < RB; qq++) {
                if (RB == 1 || q0 + qq < ca.nrhs) {
                    float2 aj = a[(long long)(q0 + qq) * ca.N + j];
                    acc0[qq].add(aj.x * W0r - aj.y * W0i, aj.x * W0i + aj.y * W0r);
                    if (SPLIT) acc1[qq].add(aj.x * W1r - aj.y * W1i, aj.x * W1i + aj.y * W1r);
                }
            }
        }
#pragma unroll
        for (int qq = 0; qq < RB; qq++) {
            if (RB == 1 || q0 + qq < ca.nrhs) {
                long long base = ((long long)(q0 + qq) * L.nrc + rc) * L.nfac;
                F[base * ca.Pstride + n] = acc0[qq].get();
                if (SPLIT) F[(base + 1) * ca.Pstride + n] = acc1[qq].get();
            }
        }
    }
}

// K1 (mixed) for the leaves of a coarser level d of an adaptive tree: the arithmetic of k_leaf32 with
// one thread per (listed relevant cone, node).  A source's offset from the leaf's centre is its
// offset from its level-D box centre plus the difference of the two centres, exact in leaf units
// (integer box coordinates times powers of two).
template <int PS, int PA, bool SPLIT>
__global__ void __launch_bounds__(kBlock) k_leaf32a(CommonArgs ca, LevelArgs L, LevelArgs LD, ChebTab tb,
                                                    const float2 *__restrict__ a, const int *__restrict__ rc_list,
                                                    long long nlist) {
    constexpr int P = PS * PA * PA;
    const long long tid = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (tid >= nlist * P) return;
    const int rc = rc_list[tid / P], n = (int)(tid % P);
    const int b = L.rc_box[rc];
    float s, u[3];
    node32<PS, PA>(L, tb, L.rc_cone[rc], n, s, u);
    const float ir = s / L.hu, kap = ca.kappa_hi, soh = s / (L.hu * ca.HDf);
    const float kf = ca.kf, etaf = ca.etaf, etaif = ca.etaif;
    const float cb0 = (L.ijk[3 * b] + 0.5f) * L.scale, cb1 = (L.ijk[3 * b + 1] + 0.5f) * L.scale,
                cb2 = (L.ijk[3 * b + 2] + 0.5f) * L.scale;
    const int j0 = L.start[b], j1 = L.start[b + 1];
    float2 *F = (float2 *)L.F;
    for (int q = 0; q < ca.nrhs; q++) {
        PAcc acc0, acc1;
        acc0.zero();
        acc1.zero();
        for (int j = j0; j < j1; j++) {
            const int e = ca.leaf_of[j];
            const float4 fj = __ldg(ca.pn32 + 2 * j), nj = __ldg(ca.pn32 + 2 * j + 1);
            const float f0 = fj.x + ((LD.ijk[3 * e] + 0.5f) - cb0), f1 = fj.y + ((LD.ijk[3 * e + 1] + 0.5f) - cb1),
                        f2 = fj.z + ((LD.ijk[3 * e + 2] + 0.5f) - cb2);
            const float dv0 = u[0] - f0 * ir, dv1 = u[1] - f1 * ir, dv2 = u[2] - f2 * ir;
            const float a2 = dv0 * dv0 + dv1 * dv1 + dv2 * dv2;
            const float ia = rsqrtf(a2), am = a2 * ia;
            const float yy = f0 * f0 + f1 * f1 + f2 * f2, uy = u[0] * f0 + u[1] * f1 + u[2] * f2;
            float t = kap * __fdividef(ir * yy - 2.f * uy, am + 1.f);
            t -= rintf(t);
            float sn, cs;
            cis_cycles(t, sn, cs);
            const float dn = dv0 * nj.x + dv1 * nj.y + dv2 * nj.z;
            const float w3 = dn * ia * ia, w2 = w3 * ia;
            const float g = kf * w3 + etaf * ia, hr = etaif * ia;
            float W0r, W0i, W1r = 0.f, W1i = 0.f;
            if (SPLIT) {
                W0r = cs * w2;
                W0i = sn * w2;
                W1r = cs * hr + sn * g;
                W1i = sn * hr - cs * g;
            } else {
                const float w2s = soh * w2 + hr;
                W0r = cs * w2s + sn * g;
                W0i = sn * w2s - cs * g;
            }
            const float2 aj = a[(long long)q * ca.N + j];
            acc0.add(aj.x * W0r - aj.y * W0i, aj.x * W0i + aj.y * W0r);
            if (SPLIT) acc1.add(aj.x * W1r - aj.y * W1i, aj.x * W1i + aj.y * W1r);
        }
        const long long base = ((long long)q * L.nrc + rc) * L.nfac;
        F[base * ca.Pstride + n] = acc0.get();
        if (SPLIT) F[(base + 1) * ca.Pstride + n] = acc1.get();
    }
}

// Packed two-lane FP32 arithmetic (fma.rn.f32x2, sm_100 and later): one instruction
// performs the real and imaginary FMAs of a complex value times a real weight, each
// lane rounded exactly as fmaf.  Halves the issue slots of the interpolation sums.
__device__ __forceinline__ unsigned long long f2pack(float x, float y) {
    unsigned long long r;
    asm("mov.b64 %0, {%1, %2};" : "=l"(r) : "f"(x), "f"(y));
    return r;
}
__device__ __forceinline__ void f2unpack(unsigned long long v, float &x, float &y) {
    asm("mov.b64 {%0, %1}, %2;" : "=f"(x), "=f"(y) : "l"(v));
}
// acc += (w, w) * v, lane by lane
__device__ __forceinline__ void f2fma(unsigned long long &acc, unsigned long long w, unsigned long long v) {
    asm("fma.rn.f32x2 %0, %1, %2, %0;" : "+l"(acc) : "l"(w), "l"(v));
}
using u64 = unsigned long long;
__device__ __forceinline__ u64 f2add(u64 a, u64 b) {
    u64 r;
    asm("add.rn.f32x2 %0, %1, %2;" : "=l"(r) : "l"(a), "l"(b));
    return r;
}
__device__ __forceinline__ u64 f2sub(u64 a, u64 b) {
    u64 r;
    asm("sub.rn.f32x2 %0, %1, %2;" : "=l"(r) : "l"(a), "l"(b));
    return r;
}
__device__ __forceinline__ u64 f2mul(u64 a, u64 b) {
    u64 r;
    asm("mul.rn.f32x2 %0, %1, %2;" : "=l"(r) : "l"(a), "l"(b));
    return r;
}
__device__ __forceinline__ u64 f2fma3(u64 a, u64 b, u64 c) {  // a * b + c, lane by lane
    u64 r;
    asm("fma.rn.f32x2 %0, %1, %2, %3;" : "=l"(r) : "l"(a), "l"(b), "l"(c));
    return r;
}
__device__ __forceinline__ u64 f2dup(float x) {
    u64 r;
    asm("mov.b64 %0, {%1, %1};" : "=l"(r) : "f"(x));
    return r;
}

// ap[q][m] = (a[s0].x, a[s1].x, a[s0].y, a[s1].y) for the pair (s0, s1) (s1 < 0: the padding zero)
__global__ void __launch_bounds__(kBlock) k_pack_pairs(int N, int npairs, int nrhs, const int2 *__restrict__ src,
                                                       const float2 *__restrict__ a, float4 *__restrict__ ap) {
    const long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (i >= (long long)npairs * nrhs) return;
    const int q = (int)(i / npairs), m = (int)(i % npairs);
    const int2 sp = src[m];
    const float2 a0 = a[(long long)q * N + sp.x];
    const float2 a1 = sp.y >= 0 ? a[(long long)q * N + sp.y] : make_float2(0.f, 0.f);
    ap[i] = make_float4(a0.x, a1.x, a0.y, a1.y);
}

// K1 (mixed), one right-hand side, two adjacent cone nodes per thread and two sources per
// instruction (the pair layout above): per (node, source pair) the factor of Eq. V3 / Eq. W2W2 /
// Eq. w23 with the arithmetic of k_leaf32 (every source record loaded once for both nodes), the
// sums of the even and odd sources kept apart and added at the end.
template <int PS, int PA, bool SPLIT>
__global__ void __launch_bounds__(kBlock) k_leaf32p(CommonArgs ca, LevelArgs L, ChebTab tb,
                                                    const ulonglong2 *__restrict__ pp, const int *__restrict__ pstart,
                                                    const ulonglong2 *__restrict__ ap) {
    constexpr int P = PS * PA * PA, PH = (P + 1) / 2;
    const long long tid = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (tid >= L.nrc * PH) return;
    const int rc = (int)(tid / PH), m = (int)(tid % PH);
    const int n0 = 2 * m, n1 = 2 * m + 1;
    const bool has1 = n1 < P;
    const int b = L.rc_box[rc];
    float s0, u0[3], s1, u1[3];
    node32<PS, PA>(L, tb, L.rc_cone[rc], n0, s0, u0);
    node32<PS, PA>(L, tb, L.rc_cone[rc], has1 ? n1 : n0, s1, u1);
    const float hu = L.hu;
    const float ir0 = s0 / hu, ir1 = s1 / hu;  // 1 / r (leaf units)
    const float soh0 = s0 / (hu * ca.HDf), soh1 = s1 / (hu * ca.HDf);
    const u64 kap2 = f2dup(ca.kappa_hi), kf2 = f2dup(ca.kf), eta2 = f2dup(ca.etaf), etai2 = f2dup(ca.etaif);
    const u64 one2 = f2dup(1.f), mtwo2 = f2dup(-2.f);
    struct Node {
        u64 ux, uy, uz, mir, ir, soh;
    };
    const Node nd[2] = {{f2dup(u0[0]), f2dup(u0[1]), f2dup(u0[2]), f2dup(-ir0), f2dup(ir0), f2dup(soh0)},
                        {f2dup(u1[0]), f2dup(u1[1]), f2dup(u1[2]), f2dup(-ir1), f2dup(ir1), f2dup(soh1)}};
    // accumulators per node: re = sum W0r ax - sum W0i ay (kept as two sums), im = sum W0r ay + W0i ax
    u64 r0a[2] = {0ull, 0ull}, r0b[2] = {0ull, 0ull}, i0[2] = {0ull, 0ull};
    u64 r1a[2] = {0ull, 0ull}, r1b[2] = {0ull, 0ull}, i1[2] = {0ull, 0ull};
    const int p0 = pstart[b], p1 = pstart[b + 1];
    for (int pm = p0; pm < p1; pm++) {
        const ulonglong2 R0 = __ldg(pp + 4 * pm), R1 = __ldg(pp + 4 * pm + 1), R2 = __ldg(pp + 4 * pm + 2),
                         R3 = __ldg(pp + 4 * pm + 3), A = __ldg(ap + pm);
        const u64 fx = R0.x, fy = R0.y, fz = R1.x, yy = R1.y, nx = R2.x, ny = R2.y, nz = R3.x, fn = R3.y;
        const u64 ax = A.x, ay = A.y;
#pragma unroll
        for (int k = 0; k < 2; k++) {
            const Node &v = nd[k];
            // with u a unit vector and v = u - ir f:  |v|^2 = 1 + ir (ir |f|^2 - 2 u.f)  (>= (1 - s)^2, no
            // cancellation: ir |f| <= s <= 1/sqrt(3)) and v.n = u.n - ir f.n (f.n stored per source)
            const u64 uy = f2fma3(fz, v.uz, f2fma3(fy, v.uy, f2mul(fx, v.ux)));
            const u64 num = f2fma3(uy, mtwo2, f2mul(v.ir, yy));  // ir |f|^2 - 2 u.f
            const u64 a2 = f2fma3(v.ir, num, one2);
            float a2l, a2h;
            f2unpack(a2, a2l, a2h);
            const u64 ia = f2pack(rsqrtf(a2l), rsqrtf(a2h));
            float dl, dh;
            f2unpack(f2fma3(a2, ia, one2), dl, dh);  // |v| + 1 in [1, 3]: the fast reciprocal is exact to 2 ulp
            u64 t = f2mul(kap2, f2mul(num, f2pack(__fdividef(1.f, dl), __fdividef(1.f, dh))));
            float tl, th;
            f2unpack(t, tl, th);
            t = f2sub(t, f2pack(rintf(tl), rintf(th)));
            f2unpack(t, tl, th);
            float snl, csl, snh, csh;
            cis_cycles(tl, snl, csl);
            cis_cycles(th, snh, csh);
            const u64 sn = f2pack(snl, snh), cs = f2pack(csl, csh), ncs = f2pack(-csl, -csh);
            const u64 dn = f2fma3(v.mir, fn, f2fma3(nz, v.uz, f2fma3(ny, v.uy, f2mul(nx, v.ux))));
            const u64 w3 = f2mul(dn, f2mul(ia, ia)), w2 = f2mul(w3, ia);
            const u64 g = f2fma3(kf2, w3, f2mul(eta2, ia)), hr = f2mul(etai2, ia);
            if (SPLIT) {
                const u64 W0r = f2mul(cs, w2), W0i = f2mul(sn, w2);
                const u64 W1r = f2fma3(sn, g, f2mul(cs, hr)), W1i = f2fma3(ncs, g, f2mul(sn, hr));
                r0a[k] = f2fma3(W0r, ax, r0a[k]);
                r0b[k] = f2fma3(W0i, ay, r0b[k]);
                i0[k] = f2fma3(W0i, ax, f2fma3(W0r, ay, i0[k]));
                r1a[k] = f2fma3(W1r, ax, r1a[k]);
                r1b[k] = f2fma3(W1i, ay, r1b[k]);
                i1[k] = f2fma3(W1i, ax, f2fma3(W1r, ay, i1[k]));
            } else {
                const u64 w2s = f2fma3(v.soh, w2, hr);
                const u64 W0r = f2fma3(sn, g, f2mul(cs, w2s)), W0i = f2fma3(ncs, g, f2mul(sn, w2s));
                r0a[k] = f2fma3(W0r, ax, r0a[k]);
                r0b[k] = f2fma3(W0i, ay, r0b[k]);
                i0[k] = f2fma3(W0i, ax, f2fma3(W0r, ay, i0[k]));
            }
        }
    }
    auto fold = [](u64 ra, u64 rb, u64 im) {  // (even + odd sources)
        float ral, rah, rbl, rbh, iml, imh;
        f2unpack(ra, ral, rah);
        f2unpack(rb, rbl, rbh);
        f2unpack(im, iml, imh);
        return make_float2((ral - rbl) + (rah - rbh), iml + imh);
    };
    float2 *F = (float2 *)L.F;
    const long long base = (long long)rc * L.nfac;
    F[base * ca.Pstride + n0] = fold(r0a[0], r0b[0], i0[0]);
    if (SPLIT) F[(base + 1) * ca.Pstride + n0] = fold(r1a[0], r1b[0], i1[0]);
    if (has1) {
        F[base * ca.Pstride + n1] = fold(r0a[1], r0b[1], i0[1]);
        if (SPLIT) F[(base + 1) * ca.Pstride + n1] = fold(r1a[1], r1b[1], i1[1]);
    }
}

// K3 (mixed): geometry of one (parent node, child box) pair.
struct PropGeo {
    int crc;
    float t3[3];
    float r1r, r1i, g1, irabs;  // e^{ik(r_c - r_p)} r_p / r_c, r_p / r_c, 1 / |x - y_c| (absolute)
};

__device__ __forceinline__ void prop_geo32(const CommonArgs &ca, const LevelArgs &C, int cb, const float *nv, float rp,
                                           float o0, float o1, float o2, PropGeo &g) {
    float p0 = nv[0] - o0, p1 = nv[1] - o1, p2 = nv[2] - o2;
    float rc_ = sqrtf(p0 * p0 + p1 * p1 + p2 * p2);
    int cone = classify32(C, p0, p1, p2, rc_, g.t3);
    g.crc = C.cone_map[(long long)cb * C.ncone + cone];
    // r_c - r_p = (|o|^2 - 2 n.o) / (r_c + r_p), free of cancellation
    float oo = o0 * o0 + o1 * o1 + o2 * o2;
    float no = nv[0] * o0 + nv[1] * o1 + nv[2] * o2;
    float dr = (oo - 2.f * no) / (rc_ + rp);
    float t = ca.kappa_hi * dr;
    t -= rintf(t);
    float sn, cs;
    cis_cycles(t, sn, cs);
    g.g1 = rp / rc_;
    g.r1r = cs * g.g1;
    g.r1i = sn * g.g1;
    g.irabs = 1.f / (rc_ * ca.HDf);
}

// add one node's contribution from a child given the interpolated factor values
__device__ __forceinline__ void prop_add(CAcc &a0, CAcc &a1, bool csplit, bool psplit, const PropGeo &g, float vr,
                                         float vi, float wr, float wi) {
    if (csplit) {
        if (psplit) {
            float r2r = g.r1r * g.g1, r2i = g.r1i * g.g1;
            a0.add(vr * r2r - vi * r2i, vr * r2i + vi * r2r);
            a1.add(wr * g.r1r - wi * g.r1i, wr * g.r1i + wi * g.r1r);
        } else {
            float zr = vr * g.irabs + wr, zi = vi * g.irabs + wi;
            a0.add(zr * g.r1r - zi * g.r1i, zr * g.r1i + zi * g.r1r);
        }
    } else {
        a0.add(vr * g.r1r - vi * g.r1i, vr * g.r1i + vi * g.r1r);
    }
}

// K4 (mixed), RB right-hand sides per pass.  One warp per chunk of at most 64 targets of one
// leaf box, two per lane: every lane walks the same neighbour boxes and sources (no divergence),
// each source record (a 32-byte broadcast load) feeds two pairs, and the two independent sums
// keep the FMA and MUFU pipes busy while the next record is in flight.  Per target the sources
// are summed in neighbour-list order, as in the oracle's near-field stage.
constexpr int kNearWarps = 4;

// contribution of source j (offset fj, normal nj from the target's box offset D) to one target:
// K = e^{ikR}/(4 pi R) [ dn_u / (r^2 HD) + etai - i (k dn_u / r + eta) ],  R = r HD, times `keep` (1, or 0
// for the target itself and for coincident points: no branch, r^2 floored so that the zeroed
// terms stay finite)
__device__ __forceinline__ void near_pair32(const CommonArgs &ca, float D0, float D1, float D2, const float4 &fj,
                                            const float4 &nj, float c4, float iHD, float tolu2, bool keep,
                                            float &Kr, float &Ki) {
    const float d0 = D0 - fj.x, d1 = D1 - fj.y, d2 = D2 - fj.z;
    const float r2 = d0 * d0 + d1 * d1 + d2 * d2;
    const bool k2 = keep && r2 >= tolu2;
    const float ir = rsqrtf(fmaxf(r2, 1e-30f));
    const float r = r2 * ir;
    float t = ca.kappa_hi * r;
    t -= rintf(t);
    float sn, cs;
    cis_cycles(t, sn, cs);
    const float dn = d0 * nj.x + d1 * nj.y + d2 * nj.z;
    const float amp = k2 ? c4 * ir : 0.f;
    const float A = amp * fmaf(dn * ir * ir, iHD, ca.etaif), Bv = -amp * (ca.kf * dn * ir + ca.etaf);
    Kr = cs * A - sn * Bv;
    Ki = sn * A + cs * Bv;
}

template <int RB>
__global__ void __launch_bounds__(kNearWarps * 32) k_near32(CommonArgs ca, LevelArgs L, const int4 *__restrict__ chunks,
                                                           int nchunk, const float2 *__restrict__ a,
                                                           float2 *__restrict__ u) {
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int ch = blockIdx.x * kNearWarps + warp;
    if (ch >= nchunk) return;  // warp-uniform
    const int4 cw = chunks[ch];
    const int b = cw.x;
    const bool v0 = lane < cw.z, v1 = lane + 32 < cw.z;
    const int i0 = cw.y + (v0 ? lane : 0), i1 = cw.y + (v1 ? lane + 32 : 0);
    const int bi0 = L.ijk[3 * b], bi1 = L.ijk[3 * b + 1], bi2 = L.ijk[3 * b + 2];
    const float4 *pn = ca.pn32;
    const float4 f0 = __ldg(pn + 2 * i0), f1 = __ldg(pn + 2 * i1);
    const float c4 = 1.f / (4.f * kPiF * ca.HDf), iHD = 1.f / ca.HDf;
    const float tolu = (float)(ca.tol / ca.HD), tolu2 = tolu * tolu;
    const int nb0 = ca.nb_start[b], nb1 = ca.nb_start[b + 1];
    for (int q0 = 0; q0 < ca.nrhs; q0 += RB) {
        PAcc A0[RB], A1[RB];
#pragma unroll
        for (int qq = 0; qq < RB; qq++) {
            A0[qq].zero();
            A1[qq].zero();
        }
        for (int nb = nb0; nb < nb1; nb++) {
            const int c = ca.nb_list[nb];
            const float E0 = (float)(bi0 - L.ijk[3 * c]), E1 = (float)(bi1 - L.ijk[3 * c + 1]),
                        E2 = (float)(bi2 - L.ijk[3 * c + 2]);
            const float D00 = E0 + f0.x, D01 = E1 + f0.y, D02 = E2 + f0.z;
            const float D10 = E0 + f1.x, D11 = E1 + f1.y, D12 = E2 + f1.z;
            const int j1 = L.start[c + 1];
#pragma unroll 2
            for (int j = L.start[c]; j < j1; j++) {
                const float4 fj = __ldg(pn + 2 * j), nj = __ldg(pn + 2 * j + 1);
                float K0r, K0i, K1r, K1i;
                near_pair32(ca, D00, D01, D02, fj, nj, c4, iHD, tolu2, j != i0, K0r, K0i);
                near_pair32(ca, D10, D11, D12, fj, nj, c4, iHD, tolu2, j != i1, K1r, K1i);
#pragma unroll
                for (int qq = 0; qq < RB; qq++) {
                    if (RB == 1 || q0 + qq < ca.nrhs) {
                        const float2 aj = a[(long long)(q0 + qq) * ca.N + j];
                        A0[qq].add(K0r * aj.x - K0i * aj.y, K0r * aj.y + K0i * aj.x);
                        A1[qq].add(K1r * aj.x - K1i * aj.y, K1r * aj.y + K1i * aj.x);
                    }
                }
            }
        }
#pragma unroll
        for (int qq = 0; qq < RB; qq++)
            if (RB == 1 || q0 + qq < ca.nrhs) {
                if (v0) u[(long long)(q0 + qq) * ca.N + i0] = A0[qq].get();
                if (v1) u[(long long)(q0 + qq) * ca.N + i1] = A1[qq].get();
            }
    }
}

// K4 (mixed), one right-hand side, on the source pairs: the chunks and neighbour walk of k_near32,
// each target against two sources per instruction (near_pair32's arithmetic, lane by lane); the
// even and odd sources are summed apart and added at the end.
__global__ void __launch_bounds__(kNearWarps * 32) k_near32p(CommonArgs ca, LevelArgs L, const int4 *__restrict__ chunks,
                                                            int nchunk, const ulonglong2 *__restrict__ pp,
                                                            const int *__restrict__ pstart,
                                                            const ulonglong2 *__restrict__ ap, float2 *__restrict__ u) {
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int ch = blockIdx.x * kNearWarps + warp;
    if (ch >= nchunk) return;  // warp-uniform
    const int4 cw = chunks[ch];
    const int b = cw.x;
    const bool v0 = lane < cw.z, v1 = lane + 32 < cw.z;
    const int i0 = cw.y + (v0 ? lane : 0), i1 = cw.y + (v1 ? lane + 32 : 0);
    const int bi0 = L.ijk[3 * b], bi1 = L.ijk[3 * b + 1], bi2 = L.ijk[3 * b + 2];
    const float4 f0 = __ldg(ca.pn32 + 2 * i0), f1 = __ldg(ca.pn32 + 2 * i1);
    const float c4 = 1.f / (4.f * kPiF * ca.HDf);
    const float tolu = (float)(ca.tol / ca.HD), tolu2 = tolu * tolu;
    const u64 kap2 = f2dup(ca.kappa_hi), kf2 = f2dup(ca.kf), eta2 = f2dup(ca.etaf), etai2 = f2dup(ca.etaif);
    const u64 iHD2 = f2dup(1.f / ca.HDf);
    u64 ra[2] = {0ull, 0ull}, rb[2] = {0ull, 0ull}, im[2] = {0ull, 0ull};
    const int fi[2] = {i0, i1};
    for (int nb = ca.nb_start[b]; nb < ca.nb_start[b + 1]; nb++) {
        const int c = ca.nb_list[nb];
        const float E0 = (float)(bi0 - L.ijk[3 * c]), E1 = (float)(bi1 - L.ijk[3 * c + 1]),
                    E2 = (float)(bi2 - L.ijk[3 * c + 2]);
        const u64 Dx[2] = {f2dup(E0 + f0.x), f2dup(E0 + f1.x)}, Dy[2] = {f2dup(E1 + f0.y), f2dup(E1 + f1.y)},
                  Dz[2] = {f2dup(E2 + f0.z), f2dup(E2 + f1.z)};
        const int js = L.start[c];
        for (int pm = pstart[c]; pm < pstart[c + 1]; pm++) {
            const ulonglong2 R0 = __ldg(pp + 4 * pm), R1 = __ldg(pp + 4 * pm + 1), R2 = __ldg(pp + 4 * pm + 2),
                             R3 = __ldg(pp + 4 * pm + 3), A = __ldg(ap + pm);
            const int jl = js + 2 * (pm - pstart[c]);  // sorted index of the even source
#pragma unroll
            for (int k = 0; k < 2; k++) {
                const u64 dx = f2sub(Dx[k], R0.x), dy = f2sub(Dy[k], R0.y), dz = f2sub(Dz[k], R1.x);
                const u64 r2 = f2fma3(dz, dz, f2fma3(dy, dy, f2mul(dx, dx)));
                float r2l, r2h;
                f2unpack(r2, r2l, r2h);
                const bool kl = fi[k] != jl && r2l >= tolu2, kh = fi[k] != jl + 1 && r2h >= tolu2;
                const float irl = rsqrtf(fmaxf(r2l, 1e-30f)), irh = rsqrtf(fmaxf(r2h, 1e-30f));
                const u64 ir = f2pack(irl, irh);
                u64 t = f2mul(kap2, f2mul(r2, ir));
                float tl, th;
                f2unpack(t, tl, th);
                t = f2sub(t, f2pack(rintf(tl), rintf(th)));
                f2unpack(t, tl, th);
                float snl, csl, snh, csh;
                cis_cycles(tl, snl, csl);
                cis_cycles(th, snh, csh);
                const u64 dn = f2fma3(dz, R3.x, f2fma3(dy, R2.y, f2mul(dx, R2.x)));
                const u64 amp = f2pack(kl ? c4 * irl : 0.f, kh ? c4 * irh : 0.f);
                const u64 dnir = f2mul(dn, ir);
                // K = amp e^{i 2 pi t} (A' - i B'),  A' = dn / (r^2 HD) + etai, B' = k dn / r + eta
                const u64 Ar = f2mul(amp, f2fma3(f2mul(dnir, ir), iHD2, etai2));
                const u64 nB = f2mul(amp, f2fma3(kf2, dnir, eta2));
                const u64 Kr = f2fma3(f2pack(snl, snh), nB, f2mul(f2pack(csl, csh), Ar));
                const u64 Ki = f2fma3(f2pack(-csl, -csh), nB, f2mul(f2pack(snl, snh), Ar));
                ra[k] = f2fma3(Kr, A.x, ra[k]);
                rb[k] = f2fma3(Ki, A.y, rb[k]);
                im[k] = f2fma3(Ki, A.x, f2fma3(Kr, A.y, im[k]));
            }
        }
    }
    auto fold = [](u64 a, u64 bb, u64 c) {
        float al, ah, bl, bh, cl, chh;
        f2unpack(a, al, ah);
        f2unpack(bb, bl, bh);
        f2unpack(c, cl, chh);
        return make_float2((al - bl) + (ah - bh), cl + chh);
    };
    if (v0) u[i0] = fold(ra[0], rb[0], im[0]);
    if (v1) u[i1] = fold(ra[1], rb[1], im[1]);
}

// ---- near field of an adaptive tree -------------------------------------------------------------
// A chunk holds at most 64 targets of one leaf (of any level); the leaf's near sources are a list of
// contiguous point ranges (every level-D box under an existing box is contiguous in point order) with
// the matching pair ranges.  A source's level-D box differs from pair to pair, so its integer box
// coordinates travel with it, packed 21 bits per axis (depth <= 20); the target-source offset is the
// exact integer box difference plus the two leaf-unit offsets, as in k_near32.  The source itself is
// dropped by the distance test (its offset is exactly zero), like any pair closer than the tolerance.
// Chunks of leaves with long lists (a small leaf of a coarse level beside dense boxes) run as one
// block whose warps split the sources, summed in warp order in shared memory.
constexpr int kNearBlkWarps = 16;

__device__ __forceinline__ void unpack_ijk(unsigned long long k, int &c0, int &c1, int &c2) {
    c0 = (int)(k & 0x1fffffULL);
    c1 = (int)((k >> 21) & 0x1fffffULL);
    c2 = (int)((k >> 42) & 0x1fffffULL);
}

// the two targets of a lane: level-D box coordinates and leaf-unit offsets
struct NearTargets {
    int ai[2][3];
    float4 fv[2];
};

__device__ __forceinline__ NearTargets near_targets(const CommonArgs &ca, const unsigned long long *__restrict__ pt_ijk,
                                                    int i0, int i1) {
    NearTargets t;
    unpack_ijk(__ldg(pt_ijk + i0), t.ai[0][0], t.ai[0][1], t.ai[0][2]);
    unpack_ijk(__ldg(pt_ijk + i1), t.ai[1][0], t.ai[1][1], t.ai[1][2]);
    t.fv[0] = __ldg(ca.pn32 + 2 * i0);
    t.fv[1] = __ldg(ca.pn32 + 2 * i1);
    return t;
}

// one right-hand side: the lane's two targets against the source pairs p0, p0 + step, ... < p1
// (k_near32p's arithmetic with per-pair box coordinates); accumulates (Re Kr a, Im Ki a, imag) per target
__device__ __forceinline__ void near_pairs_acc(const CommonArgs &ca, const NearTargets &t, int p0, int p1, int step,
                                               const ulonglong2 *__restrict__ pp, const ulonglong2 *__restrict__ ap,
                                               const unsigned long long *__restrict__ pair_ijk,
                                               u64 (&ra)[2], u64 (&rb)[2], u64 (&im)[2]) {
    const float c4 = 1.f / (4.f * kPiF * ca.HDf);
    const float tolu = (float)(ca.tol / ca.HD), tolu2 = tolu * tolu;
    const u64 kap2 = f2dup(ca.kappa_hi), kf2 = f2dup(ca.kf), eta2 = f2dup(ca.etaf), etai2 = f2dup(ca.etaif);
    const u64 iHD2 = f2dup(1.f / ca.HDf);
    for (int pm = p0; pm < p1; pm += step) {
        const ulonglong2 R0 = __ldg(pp + 4 * pm), R1 = __ldg(pp + 4 * pm + 1), R2 = __ldg(pp + 4 * pm + 2),
                         R3 = __ldg(pp + 4 * pm + 3), A = __ldg(ap + pm);
        int c0, c1, c2;
        unpack_ijk(__ldg(pair_ijk + pm), c0, c1, c2);
#pragma unroll
        for (int k = 0; k < 2; k++) {
            const u64 dx = f2sub(f2dup((float)(t.ai[k][0] - c0) + t.fv[k].x), R0.x),
                      dy = f2sub(f2dup((float)(t.ai[k][1] - c1) + t.fv[k].y), R0.y),
                      dz = f2sub(f2dup((float)(t.ai[k][2] - c2) + t.fv[k].z), R1.x);
            const u64 r2 = f2fma3(dz, dz, f2fma3(dy, dy, f2mul(dx, dx)));
            float r2l, r2h;
            f2unpack(r2, r2l, r2h);
            const bool kl = r2l >= tolu2, kh = r2h >= tolu2;
            const float irl = rsqrtf(fmaxf(r2l, 1e-30f)), irh = rsqrtf(fmaxf(r2h, 1e-30f));
            const u64 ir = f2pack(irl, irh);
            u64 tt = f2mul(kap2, f2mul(r2, ir));
            float tl, th;
            f2unpack(tt, tl, th);
            tt = f2sub(tt, f2pack(rintf(tl), rintf(th)));
            f2unpack(tt, tl, th);
            float snl, csl, snh, csh;
            cis_cycles(tl, snl, csl);
            cis_cycles(th, snh, csh);
            const u64 dn = f2fma3(dz, R3.x, f2fma3(dy, R2.y, f2mul(dx, R2.x)));
            const u64 amp = f2pack(kl ? c4 * irl : 0.f, kh ? c4 * irh : 0.f);
            const u64 dnir = f2mul(dn, ir);
            const u64 Ar = f2mul(amp, f2fma3(f2mul(dnir, ir), iHD2, etai2));
            const u64 nB = f2mul(amp, f2fma3(kf2, dnir, eta2));
            const u64 Kr = f2fma3(f2pack(snl, snh), nB, f2mul(f2pack(csl, csh), Ar));
            const u64 Ki = f2fma3(f2pack(-csl, -csh), nB, f2mul(f2pack(snl, snh), Ar));
            ra[k] = f2fma3(Kr, A.x, ra[k]);
            rb[k] = f2fma3(Ki, A.y, rb[k]);
            im[k] = f2fma3(Ki, A.x, f2fma3(Kr, A.y, im[k]));
        }
    }
}

__device__ __forceinline__ float2 near_fold(u64 x, u64 y, u64 z) {
    float xl, xh, yl, yh, zl, zh;
    f2unpack(x, xl, xh);
    f2unpack(y, yl, yh);
    f2unpack(z, zl, zh);
    return make_float2((xl - yl) + (xh - yh), zl + zh);
}

// several right-hand sides, RB at a time from q0: the lane's two targets against the sources
// j0, j0 + step, ... < j1 (near_pair32's arithmetic)
template <int RB>
__device__ __forceinline__ void near_points_acc(const CommonArgs &ca, const NearTargets &t, int j0, int j1, int step,
                                                const unsigned long long *__restrict__ pt_ijk, int q0,
                                                const float2 *__restrict__ a, PAcc (&A0)[RB], PAcc (&A1)[RB]) {
    const float c4 = 1.f / (4.f * kPiF * ca.HDf), iHD = 1.f / ca.HDf;
    const float tolu = (float)(ca.tol / ca.HD), tolu2 = tolu * tolu;
    for (int j = j0; j < j1; j += step) {
        const float4 fj = __ldg(ca.pn32 + 2 * j), nj = __ldg(ca.pn32 + 2 * j + 1);
        int c0, c1, c2;
        unpack_ijk(__ldg(pt_ijk + j), c0, c1, c2);
        float K0r, K0i, K1r, K1i;
        near_pair32(ca, (float)(t.ai[0][0] - c0) + t.fv[0].x, (float)(t.ai[0][1] - c1) + t.fv[0].y,
                    (float)(t.ai[0][2] - c2) + t.fv[0].z, fj, nj, c4, iHD, tolu2, true, K0r, K0i);
        near_pair32(ca, (float)(t.ai[1][0] - c0) + t.fv[1].x, (float)(t.ai[1][1] - c1) + t.fv[1].y,
                    (float)(t.ai[1][2] - c2) + t.fv[1].z, fj, nj, c4, iHD, tolu2, true, K1r, K1i);
#pragma unroll
        for (int qq = 0; qq < RB; qq++) {
            if (RB == 1 || q0 + qq < ca.nrhs) {
                const float2 aj = a[(long long)(q0 + qq) * ca.N + j];
                A0[qq].add(K0r * aj.x - K0i * aj.y, K0r * aj.y + K0i * aj.x);
                A1[qq].add(K1r * aj.x - K1i * aj.y, K1r * aj.y + K1i * aj.x);
            }
        }
    }
}

// one warp per chunk (at most 64 targets), several right-hand sides
template <int RB>
__global__ void __launch_bounds__(kNearWarps * 32) k_near32r(CommonArgs ca, const int4 *__restrict__ chunks, int nchunk,
                                                            const int *__restrict__ nr_start,
                                                            const int4 *__restrict__ nr,
                                                            const unsigned long long *__restrict__ pt_ijk,
                                                            const float2 *__restrict__ a, float2 *__restrict__ u) {
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int ch = blockIdx.x * kNearWarps + warp;
    if (ch >= nchunk) return;  // warp-uniform
    const int4 cw = chunks[ch];
    const bool v0 = lane < cw.z, v1 = lane + 32 < cw.z;
    const int i0 = cw.y + (v0 ? lane : 0), i1 = cw.y + (v1 ? lane + 32 : 0);
    const NearTargets t = near_targets(ca, pt_ijk, i0, i1);
    const int r0 = nr_start[cw.w], r1 = nr_start[cw.w + 1];
    for (int q0 = 0; q0 < ca.nrhs; q0 += RB) {
        PAcc A0[RB], A1[RB];
#pragma unroll
        for (int qq = 0; qq < RB; qq++) {
            A0[qq].zero();
            A1[qq].zero();
        }
        for (int r = r0; r < r1; r++) {
            const int4 rg = __ldg(nr + r);
            near_points_acc<RB>(ca, t, rg.x, rg.y, 1, pt_ijk, q0, a, A0, A1);
        }
#pragma unroll
        for (int qq = 0; qq < RB; qq++)
            if (RB == 1 || q0 + qq < ca.nrhs) {
                if (v0) u[(long long)(q0 + qq) * ca.N + i0] = A0[qq].get();
                if (v1) u[(long long)(q0 + qq) * ca.N + i1] = A1[qq].get();
            }
    }
}

// one warp per chunk, one right-hand side on the source pairs (pair_ijk: the packed coordinates of each
// pair's level-D box; both sources of a pair share it)
__global__ void __launch_bounds__(kNearWarps * 32) k_near32pr(CommonArgs ca, const int4 *__restrict__ chunks, int nchunk,
                                                             const int *__restrict__ nr_start,
                                                             const int4 *__restrict__ nr,
                                                             const unsigned long long *__restrict__ pt_ijk,
                                                             const unsigned long long *__restrict__ pair_ijk,
                                                             const ulonglong2 *__restrict__ pp,
                                                             const ulonglong2 *__restrict__ ap, float2 *__restrict__ u) {
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int ch = blockIdx.x * kNearWarps + warp;
    if (ch >= nchunk) return;  // warp-uniform
    const int4 cw = chunks[ch];
    const bool v0 = lane < cw.z, v1 = lane + 32 < cw.z;
    const int i0 = cw.y + (v0 ? lane : 0), i1 = cw.y + (v1 ? lane + 32 : 0);
    const NearTargets t = near_targets(ca, pt_ijk, i0, i1);
    u64 ra[2] = {0ull, 0ull}, rb[2] = {0ull, 0ull}, im[2] = {0ull, 0ull};
    for (int r = nr_start[cw.w]; r < nr_start[cw.w + 1]; r++) {
        const int4 rg = __ldg(nr + r);
        near_pairs_acc(ca, t, rg.z, rg.w, 1, pp, ap, pair_ijk, ra, rb, im);
    }
    if (v0) u[i0] = near_fold(ra[0], rb[0], im[0]);
    if (v1) u[i1] = near_fold(ra[1], rb[1], im[1]);
}

// one block per chunk of a leaf with a long source list: warp w takes every kNearBlkWarps-th source
// (pair) of each range; the warps' partial sums are added in warp order
__global__ void __launch_bounds__(kNearBlkWarps * 32) k_near32pr_blk(CommonArgs ca, const int4 *__restrict__ chunks,
                                                                    const int *__restrict__ nr_start,
                                                                    const int4 *__restrict__ nr,
                                                                    const unsigned long long *__restrict__ pt_ijk,
                                                                    const unsigned long long *__restrict__ pair_ijk,
                                                                    const ulonglong2 *__restrict__ pp,
                                                                    const ulonglong2 *__restrict__ ap,
                                                                    float2 *__restrict__ u) {
    __shared__ float2 part[kNearBlkWarps][64];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int4 cw = chunks[blockIdx.x];
    const bool v0 = lane < cw.z, v1 = lane + 32 < cw.z;
    const int i0 = cw.y + (v0 ? lane : 0), i1 = cw.y + (v1 ? lane + 32 : 0);
    const NearTargets t = near_targets(ca, pt_ijk, i0, i1);
    u64 ra[2] = {0ull, 0ull}, rb[2] = {0ull, 0ull}, im[2] = {0ull, 0ull};
    for (int r = nr_start[cw.w]; r < nr_start[cw.w + 1]; r++) {
        const int4 rg = __ldg(nr + r);
        near_pairs_acc(ca, t, rg.z + warp, rg.w, kNearBlkWarps, pp, ap, pair_ijk, ra, rb, im);
    }
    part[warp][lane] = near_fold(ra[0], rb[0], im[0]);
    part[warp][lane + 32] = near_fold(ra[1], rb[1], im[1]);
    __syncthreads();
    if (threadIdx.x < cw.z) {
        float2 z = make_float2(0.f, 0.f);
#pragma unroll
        for (int w = 0; w < kNearBlkWarps; w++) {
            z.x += part[w][threadIdx.x].x;
            z.y += part[w][threadIdx.x].y;
        }
        u[cw.y + threadIdx.x] = z;
    }
}

// the same for several right-hand sides, one at a time
__global__ void __launch_bounds__(kNearBlkWarps * 32) k_near32r_blk(CommonArgs ca, const int4 *__restrict__ chunks,
                                                                   const int *__restrict__ nr_start,
                                                                   const int4 *__restrict__ nr,
                                                                   const unsigned long long *__restrict__ pt_ijk,
                                                                   const float2 *__restrict__ a,
                                                                   float2 *__restrict__ u) {
    __shared__ float2 part[kNearBlkWarps][64];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int4 cw = chunks[blockIdx.x];
    const bool v0 = lane < cw.z, v1 = lane + 32 < cw.z;
    const int i0 = cw.y + (v0 ? lane : 0), i1 = cw.y + (v1 ? lane + 32 : 0);
    const NearTargets t = near_targets(ca, pt_ijk, i0, i1);
    for (int q = 0; q < ca.nrhs; q++) {
        PAcc A0[1], A1[1];
        A0[0].zero();
        A1[0].zero();
        for (int r = nr_start[cw.w]; r < nr_start[cw.w + 1]; r++) {
            const int4 rg = __ldg(nr + r);
            near_points_acc<1>(ca, t, rg.x + warp, rg.y, kNearBlkWarps, pt_ijk, q, a, A0, A1);
        }
        part[warp][lane] = A0[0].get();
        part[warp][lane + 32] = A1[0].get();
        __syncthreads();
        if (threadIdx.x < cw.z) {
            float2 z = make_float2(0.f, 0.f);
#pragma unroll
            for (int w = 0; w < kNearBlkWarps; w++) {
                z.x += part[w][threadIdx.x].x;
                z.y += part[w][threadIdx.x].y;
            }
            u[(long long)q * ca.N + cw.y + threadIdx.x] = z;
        }
        __syncthreads();  // part is rewritten by the next right-hand side
    }
}

// K2 (mixed): geometry of one (target, cousin box) pair.
struct CousGeo {
    int rc;
    float t3[3];
    float E1r, E1i, irabs;  // e^{ikr} / (4 pi r), 1 / r (absolute)
};

__device__ __forceinline__ void cousin_geo32(const CommonArgs &ca, const LevelArgs &L, int c, const float *I,
                                             const float *f, CousGeo &g) {
    const float sc = (float)L.scale;
    const float M0 = I[0] - (L.ijk[3 * c] + 0.5f) * sc, M1 = I[1] - (L.ijk[3 * c + 1] + 0.5f) * sc,
                M2 = I[2] - (L.ijk[3 * c + 2] + 0.5f) * sc;
    float r;
    const float t = phase_cycles_exact(M0, M1, M2, f[0], f[1], f[2], ca.kappa_hi, ca.kappa_lo, r);
    const int cone = classify32(L, M0 + f[0], M1 + f[1], M2 + f[2], r, g.t3);
    g.rc = L.cone_map[(long long)c * L.ncone + cone];
    float sn, cs;
    cis_cycles(t, sn, cs);
    const float ir = 1.f / r;
    const float c4 = 1.f / (4.f * kPiF * ca.HDf);
    g.E1r = c4 * ir * cs;
    g.E1i = c4 * ir * sn;
    g.irabs = ir / ca.HDf;
}

__device__ __forceinline__ void cousin_add(CAcc &a, bool split, const CousGeo &g, float vr, float vi, float wr,
                                           float wi) {
    if (split) {
        vr = vr * g.irabs + wr;
        vi = vi * g.irabs + wi;
    }
    a.add(g.E1r * vr - g.E1i * vi, g.E1r * vi + g.E1i * vr);
}

// K2 (mixed), staged.  One warp owns a chunk of at most 32 targets of one level-d
// box (one per lane) and walks the box's cousin list.  For every cousin, the
// distinct cones its lanes fall into are taken one at a time: the warp copies that
// cone's node values (all factors) into its shared-memory buffer with coalesced
// 16-byte loads, and the lanes of that cone interpolate from shared memory (every
// lane reads the same address: broadcasts).
constexpr int kCwWarps = 4;

// 16-byte global -> shared copy that bypasses the registers (cp.async, L2 only)
__device__ __forceinline__ void cp_async16(void *smem, const void *gmem) {
    const unsigned sa = (unsigned)__cvta_generic_to_shared(smem);
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(sa), "l"(gmem) : "memory");
}
__device__ __forceinline__ void cp_async_wait_all() { asm volatile("cp.async.wait_all;\n" ::: "memory"); }


template <int PS, int PA>
__device__ __forceinline__ void interp3f_one(const float2 *f, const float *Ls, const float *Lt, const float *Lp,
                                             float &r, float &i) {
    unsigned long long lp2[PA], lt2[PA];
#pragma unroll
    for (int c = 0; c < PA; c++) {
        lp2[c] = f2pack(Lp[c], Lp[c]);
        lt2[c] = f2pack(Lt[c], Lt[c]);
    }
    unsigned long long acc = 0ull;  // (0.f, 0.f)
#pragma unroll 1
    for (int a = 0; a < PS; a++) {
        const float2 *fa = f + a * PA * PA;
        unsigned long long acc_a = 0ull;
#pragma unroll
        for (int b = 0; b < PA; b++) {
            unsigned long long acc_b = 0ull;
            const float2 *row = fa + b * PA;
            if constexpr (PA % 2 == 0) {
#pragma unroll
                for (int c = 0; c < PA; c += 2) {
                    const float4 v = *reinterpret_cast<const float4 *>(row + c);
                    f2fma(acc_b, lp2[c], f2pack(v.x, v.y));
                    f2fma(acc_b, lp2[c + 1], f2pack(v.z, v.w));
                }
            } else {
#pragma unroll
                for (int c = 0; c < PA; c++) {
                    const float2 v = row[c];
                    f2fma(acc_b, lp2[c], f2pack(v.x, v.y));
                }
            }
            f2fma(acc_a, lt2[b], acc_b);
        }
        const float la = pick<PS>(Ls, a);
        f2fma(acc, f2pack(la, la), acc_a);
    }
    f2unpack(acc, r, i);
}

template <int PS, int PA, int RB>
__global__ void __launch_bounds__(kCwWarps * 32) k_cousin_w(CommonArgs ca, LevelArgs L, LevelArgs LD,
                                                            const int4 *__restrict__ chunks, int nchunk, ChebTab tb,
                                                            float2 *__restrict__ u) {
    constexpr int P = PS * PA * PA, PST = P + (P & 1);  // PST = node stride of one factor (the plan's Pstride)
    constexpr int NL = (PST + 31) / 32;                  // float4 per lane to copy two factors
    // four slots of one factor each (slot k at k (PST + 2): 16 bytes of stagger per slot, so that lanes
    // reading different cones at the same offset hit different bank groups); a pass stages up to
    // 4 / nfac distinct cones, cone k in slots nfac k .. nfac k + nfac - 1
    constexpr int SLOT = PST + 2;
    __shared__ __align__(16) float2 sF[kCwWarps][4 * SLOT];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int ch = blockIdx.x * kCwWarps + warp;
    if (ch >= nchunk) return;  // warp-uniform: no block-wide barrier below
    const int4 cw = chunks[ch];
    const int b = cw.x;
    const bool act = lane < cw.z;
    const int i = cw.y + (act ? lane : 0);
    const int l = ca.leaf_of[i];
    const float I[3] = {LD.ijk[3 * l] + 0.5f, LD.ijk[3 * l + 1] + 0.5f, LD.ijk[3 * l + 2] + 0.5f};
    const float4 fi = __ldg(ca.pn32 + 2 * i);
    const float f[3] = {fi.x, fi.y, fi.z};
    const float2 *F = (const float2 *)L.F;
    const bool sp = L.split != 0;
    const int nv4 = PST / 2;  // float4 of one factor of a relevant cone
    const int nfac = L.nfac, kmax = 4 / nfac;  // cones per pass
    float2 *buf = sF[warp];
    const int c0 = L.co_start[b], c1 = L.co_start[b + 1];
    for (int q0 = 0; q0 < ca.nrhs; q0 += RB) {
        CAcc acc[RB];
#pragma unroll
        for (int qq = 0; qq < RB; qq++) acc[qq].zero();
        for (int ci = c0; ci < c1; ci++) {
            const int c = L.co_list[ci];
            if (L.rc_start[c] == L.rc_start[c + 1]) continue;  // no sources in c (warp-uniform)
            CousGeo g;
            cousin_geo32(ca, L, c, I, f, g);
            if (!act) g.rc = -2;
            if (q0 == 0 && g.rc == -1) atomicAdd(ca.missed, 1ULL);
            float Ls[PS], Lt[PA], Lp[PA];
            lagrange<PS, float>(g.t3[0], tb.fxs, tb.fcs, Ls);
            lagrange<PA, float>(g.t3[1], tb.fxa, tb.fca, Lt);
            lagrange<PA, float>(g.t3[2], tb.fxa, tb.fca, Lp);
            bool pend = g.rc >= 0;
            while (__any_sync(0xffffffffu, pend)) {
                // up to kmax distinct cones of the pending lanes (leaders in lane order)
                int rcs[4] = {-1, -1, -1, -1};
                int nk = 0, myk = -1;
                bool left = pend;
                for (int k = 0; k < kmax; k++) {
                    const unsigned mk = __ballot_sync(0xffffffffu, left);
                    if (!mk) break;
                    const int rk = __shfl_sync(0xffffffffu, g.rc, __ffs(mk) - 1);
                    if (left && g.rc == rk) {
                        myk = k;
                        left = false;
                    }
                    rcs[k] = rk;
                    nk = k + 1;
                }
                const bool mine = myk >= 0;
                const float2 *mybuf = buf + (mine ? myk * nfac : 0) * SLOT;
#pragma unroll
                for (int qq = 0; qq < RB; qq++) {
                    if (RB > 1 && q0 + qq >= ca.nrhs) break;  // warp-uniform
                    __syncwarp();  // the previous cones' readers are done
                    for (int k = 0; k < nk; k++)
                        for (int fc = 0; fc < nfac; fc++) {
                            const float4 *src = reinterpret_cast<const float4 *>(
                                F + (((long long)(q0 + qq) * L.nrc + rcs[k]) * nfac + fc) * ca.Pstride);
                            float4 *dk = reinterpret_cast<float4 *>(buf + (k * nfac + fc) * SLOT);
#pragma unroll
                            for (int v = 0; v < NL; v++)
                                if (lane + 32 * v < nv4) cp_async16(dk + lane + 32 * v, src + lane + 32 * v);
                        }
                    cp_async_wait_all();
                    __syncwarp();
                    if (mine) {
                        float vr, vi, wr = 0.f, wi = 0.f;
                        interp3f_one<PS, PA>(mybuf, Ls, Lt, Lp, vr, vi);
                        if (sp) interp3f_one<PS, PA>(mybuf + SLOT, Ls, Lt, Lp, wr, wi);
                        cousin_add(acc[qq], sp, g, vr, vi, wr, wi);
                    }
                }
                pend = pend && !mine;
            }
        }
        if (act) {
#pragma unroll
            for (int qq = 0; qq < RB; qq++) {
                if (RB == 1 || q0 + qq < ca.nrhs) {
                    const long long o = (long long)(q0 + qq) * ca.N + i;
                    float2 v = u[o];
                    const float2 w = acc[qq].get();
                    v.x += w.x;
                    v.y += w.y;
                    u[o] = v;
                }
            }
        }
    }
}


// ---------------------------------------------------------------------------
// K2 (mixed), cone-stationary.  The host lists, for every relevant cone of level d, the
// cousin targets that fall in it (FP64 classification); once per plan, k_cousin_geo stores
// each entry's local coordinates in the cone, its centred factor and its output slot.
// Phase 1: one warp per work item (one cone, <= 64 of its targets) copies the cone's node
// values into shared memory once; each lane interpolates two targets, so every 16-byte
// shared load is a broadcast that feeds four packed FMAs, and writes E(x; y_c)
// Interp(F_c)(x) to the value buffer at the target's (box, cousin slot) position.  Phase 2 (k_cousin_sum): one thread per target adds
// its slots in cousin-list order with compensation, so the field stays deterministic.
constexpr int kCsWarps = 4;

// per-target interpolation weights and centred factor of one (target, cone) pair
template <int PS, int PA>
struct CsTgt {
    unsigned long long lt2[PA], lp2[PA];  // (L, L) pairs of the angular bases
    float Ls[PS];
    float Er, Ei, irabs;  // E(x; y_c) = e^{ikr} / (4 pi r); 1 / r (absolute)
    int dest;             // slot in the value buffer, -1 for an idle lane
};

// Interpolation weights of entry e from its plan-time geometry: local coordinates in the list's
// cone segment and the centred factor, both computed once per plan in FP64 (k_cousin_geo).
template <int PS, int PA>
__device__ __forceinline__ void cs_load(const ChebTab &tb, const float4 *__restrict__ geo4,
                                        const float2 *__restrict__ geo2, int e, CsTgt<PS, PA> &g) {
    const float4 a = __ldg(geo4 + e);
    const float2 b = __ldg(geo2 + e);
    float Lt[PA], Lp[PA];
    lagrange<PS, float>(a.x, tb.fxs, tb.fcs, g.Ls);
    lagrange<PA, float>(a.y, tb.fxa, tb.fca, Lt);
    lagrange<PA, float>(a.z, tb.fxa, tb.fca, Lp);
#pragma unroll
    for (int k = 0; k < PA; k++) {
        g.lt2[k] = f2pack(Lt[k], Lt[k]);
        g.lp2[k] = f2pack(Lp[k], Lp[k]);
    }
    g.Er = a.w;
    g.Ei = b.x;
    g.irabs = 4.f * kPiF * sqrtf(a.w * a.w + b.x * b.x);  // |E| = 1 / (4 pi r)
    g.dest = __float_as_int(b.y);
}

// interpolation of one factor's node values f (shared memory) for two targets at once; W holds a
// target's packed angular weights lt2, lp2 and radial weights Ls
template <int PS, int PA, typename W>
__device__ __forceinline__ void cs_interp2(const float2 *f, const W &g0, const W &g1, unsigned long long &v0,
                                           unsigned long long &v1) {
    v0 = 0ull;
    v1 = 0ull;
#pragma unroll 1
    for (int a = 0; a < PS; a++) {
        const float2 *fa = f + a * PA * PA;
        unsigned long long a0 = 0ull, a1 = 0ull;
#pragma unroll
        for (int b = 0; b < PA; b++) {
            unsigned long long b0 = 0ull, b1 = 0ull;
            const float2 *row = fa + b * PA;
            if constexpr (PA % 2 == 0) {
#pragma unroll
                for (int k = 0; k < PA; k += 2) {
                    const float4 v = *reinterpret_cast<const float4 *>(row + k);
                    const unsigned long long x = f2pack(v.x, v.y), y = f2pack(v.z, v.w);
                    f2fma(b0, g0.lp2[k], x);
                    f2fma(b1, g1.lp2[k], x);
                    f2fma(b0, g0.lp2[k + 1], y);
                    f2fma(b1, g1.lp2[k + 1], y);
                }
            } else {
#pragma unroll
                for (int k = 0; k < PA; k++) {
                    const float2 v = row[k];
                    const unsigned long long x = f2pack(v.x, v.y);
                    f2fma(b0, g0.lp2[k], x);
                    f2fma(b1, g1.lp2[k], x);
                }
            }
            f2fma(a0, g0.lt2[b], b0);
            f2fma(a1, g1.lt2[b], b1);
        }
        const float l0 = pick<PS>(g0.Ls, a), l1 = pick<PS>(g1.Ls, a);
        f2fma(v0, f2pack(l0, l0), a0);
        f2fma(v1, f2pack(l1, l1), a1);
    }
}

template <int PS, int PA, bool SPLIT>
__global__ void __launch_bounds__(kCsWarps * 32) k_cousin_cs(CommonArgs ca, LevelArgs L, const int4 *__restrict__ items,
                                                             int nitems, const float4 *__restrict__ geo4,
                                                             const float2 *__restrict__ geo2, ChebTab tb,
                                                             float2 *__restrict__ pv, long long pv_stride) {
    constexpr int P = PS * PA * PA, PST = P + (P & 1), NF = SPLIT ? 2 : 1;
    constexpr int NV4 = NF * PST / 2;  // float4 of one cone's values (all factors, contiguous)
    __shared__ __align__(16) float2 sF[kCsWarps][NF * PST];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int item = blockIdx.x * kCsWarps + warp;
    if (item >= nitems) return;  // warp-uniform: no block-wide barrier below
    const int4 w = items[item];
    const int rc = w.x, e0 = w.y, cnt = w.z;
    CsTgt<PS, PA> g0, g1;
    const bool has0 = lane < cnt, has1 = lane + 32 < cnt;
    cs_load<PS, PA>(tb, geo4, geo2, e0 + (has0 ? lane : 0), g0);
    cs_load<PS, PA>(tb, geo4, geo2, e0 + (has1 ? lane + 32 : 0), g1);
    const float2 *F = (const float2 *)L.F;
    float2 *buf = sF[warp];
    for (int q = 0; q < ca.nrhs; q++) {
        __syncwarp();  // the previous right-hand side's readers are done
        const float4 *src = reinterpret_cast<const float4 *>(F + ((long long)q * L.nrc + rc) * NF * PST);
        float4 *dst = reinterpret_cast<float4 *>(buf);
        for (int v = lane; v < NV4; v += 32) cp_async16(dst + v, src + v);
        cp_async_wait_all();
        __syncwarp();
        unsigned long long v0, v1;
        cs_interp2<PS, PA>(buf, g0, g1, v0, v1);
        float vr0, vi0, vr1, vi1;
        f2unpack(v0, vr0, vi0);
        f2unpack(v1, vr1, vi1);
        if constexpr (SPLIT) {  // E (W2 / r + W13) with the second factor's interpolant
            unsigned long long w0, w1;
            cs_interp2<PS, PA>(buf + PST, g0, g1, w0, w1);
            float wr0, wi0, wr1, wi1;
            f2unpack(w0, wr0, wi0);
            f2unpack(w1, wr1, wi1);
            vr0 = vr0 * g0.irabs + wr0;
            vi0 = vi0 * g0.irabs + wi0;
            vr1 = vr1 * g1.irabs + wr1;
            vi1 = vi1 * g1.irabs + wi1;
        }
        float2 *out = pv + (long long)q * pv_stride;
        if (has0) out[g0.dest] = make_float2(g0.Er * vr0 - g0.Ei * vi0, g0.Er * vi0 + g0.Ei * vr0);
        if (has1) out[g1.dest] = make_float2(g1.Er * vr1 - g1.Ei * vi1, g1.Er * vi1 + g1.Ei * vr1);
    }
}

// Phase 2: u(x) += sum over the cousin slots of x's level-d box of the phase-1 values, in
// slot order with Kahan compensation (one thread per target; the slots of a box's targets
// are contiguous, so consecutive threads read consecutive values).
__global__ void __launch_bounds__(kBlock) k_cousin_sum(CommonArgs ca, LevelArgs L, const int *__restrict__ box_of,
                                                       const uint8_t *__restrict__ alive, const int *__restrict__ pvoff,
                                                       const float2 *__restrict__ pv, long long pv_stride,
                                                       float2 *__restrict__ u) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= ca.N) return;
    const int b = box_of[i];
    if (!alive[b]) return;  // below a coarser leaf: no level-d box for this point
    const int s0 = L.start[b], nt = L.start[b + 1] - s0;
    const int ncous = L.co_start[b + 1] - L.co_start[b];
    const long long base = (long long)pvoff[b] + (i - s0);
    for (int q = 0; q < ca.nrhs; q++) {
        const float2 *src = pv + (long long)q * pv_stride + base;
        CAcc acc;
        acc.zero();
        for (int j = 0; j < ncous; j++) {
            const float2 v = __ldg(src + (long long)j * nt);
            acc.add(v.x, v.y);
        }
        const long long o = (long long)q * ca.N + i;
        float2 x = u[o];
        const float2 z = acc.get();
        x.x += z.x;
        x.y += z.y;
        u[o] = x;
    }
}

// K3 (mixed), staged: one warp owns 32 nodes of one parent relevant cone and walks the
// parent box's children; for every distinct child cone its lanes fall into, the warp
// copies that cone's node values (all factors) into shared memory with cp.async and the
// lanes of that cone interpolate from there (the pattern of k_cousin_w).
template <int PS, int PA, int RB>
__global__ void __launch_bounds__(kCwWarps * 32) k_prop_w(CommonArgs ca, LevelArgs C, LevelArgs Pl, ChebTab tb) {
    constexpr int P = PS * PA * PA, PST = P + (P & 1), NCH = (P + 31) / 32;
    constexpr int NL = (PST + 31) / 32;
    constexpr int SLOT = PST + 2;  // four 16-byte-staggered one-factor slots, as in k_cousin_w
    __shared__ __align__(16) float2 sF[kCwWarps][4 * SLOT];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const long long unit = (long long)blockIdx.x * kCwWarps + warp;
    if (unit >= Pl.nrc * (long long)NCH) return;  // warp-uniform: no block-wide barrier below
    const int rc = (int)(unit / NCH), n = (int)(unit % NCH) * 32 + lane;
    const bool act = n < P;
    const int pb = Pl.rc_box[rc];
    float s, uu[3];
    node32<PS, PA>(Pl, tb, Pl.rc_cone[rc], act ? n : 0, s, uu);
    const float rp = Pl.hu / s;  // leaf units
    const float nv[3] = {rp * uu[0], rp * uu[1], rp * uu[2]};
    const float pc[3] = {(Pl.ijk[3 * pb] + 0.5f) * Pl.scale, (Pl.ijk[3 * pb + 1] + 0.5f) * Pl.scale,
                         (Pl.ijk[3 * pb + 2] + 0.5f) * Pl.scale};
    const float2 *FC = (const float2 *)C.F;
    float2 *FP = (float2 *)Pl.F;
    const bool cs_ = C.split != 0, ps_ = Pl.split != 0;
    const int nv4 = PST / 2;  // float4 of one factor of a child cone
    const int nfac = C.nfac, kmax = 4 / nfac;  // child cones per pass
    float2 *buf = sF[warp];
    const int c0 = Pl.ch_start[pb], c1 = Pl.ch_start[pb + 1];
    for (int q0 = 0; q0 < ca.nrhs; q0 += RB) {
        CAcc a0[RB], a1[RB];  // parent factors
#pragma unroll
        for (int qq = 0; qq < RB; qq++) {
            a0[qq].zero();
            a1[qq].zero();
        }
        for (int ci = c0; ci < c1; ci++) {
            const int cb = Pl.ch_list[ci];
            const float o0 = (C.ijk[3 * cb] + 0.5f) * C.scale - pc[0];
            const float o1 = (C.ijk[3 * cb + 1] + 0.5f) * C.scale - pc[1];
            const float o2 = (C.ijk[3 * cb + 2] + 0.5f) * C.scale - pc[2];
            PropGeo g;
            prop_geo32(ca, C, cb, nv, rp, o0, o1, o2, g);
            if (!act) g.crc = -2;
            if (q0 == 0 && g.crc == -1) atomicAdd(ca.missed, 1ULL);
            float Ls[PS], Lt[PA], Lp[PA];
            lagrange<PS, float>(g.t3[0], tb.fxs, tb.fcs, Ls);
            lagrange<PA, float>(g.t3[1], tb.fxa, tb.fca, Lt);
            lagrange<PA, float>(g.t3[2], tb.fxa, tb.fca, Lp);
            bool pend = g.crc >= 0;
            while (__any_sync(0xffffffffu, pend)) {
                // up to kmax distinct child cones of the pending lanes (leaders in lane order)
                int crcs[4] = {-1, -1, -1, -1};
                int nk = 0, myk = -1;
                bool left = pend;
                for (int k = 0; k < kmax; k++) {
                    const unsigned mk = __ballot_sync(0xffffffffu, left);
                    if (!mk) break;
                    const int ck = __shfl_sync(0xffffffffu, g.crc, __ffs(mk) - 1);
                    if (left && g.crc == ck) {
                        myk = k;
                        left = false;
                    }
                    crcs[k] = ck;
                    nk = k + 1;
                }
                const bool mine = myk >= 0;
                const float2 *mybuf = buf + (mine ? myk * nfac : 0) * SLOT;
#pragma unroll
                for (int qq = 0; qq < RB; qq++) {
                    if (RB > 1 && q0 + qq >= ca.nrhs) break;  // warp-uniform
                    __syncwarp();  // the previous cones' readers are done
                    for (int k = 0; k < nk; k++)
                        for (int fc = 0; fc < nfac; fc++) {
                            const float4 *src = reinterpret_cast<const float4 *>(
                                FC + (((long long)(q0 + qq) * C.nrc + crcs[k]) * nfac + fc) * ca.Pstride);
                            float4 *dk = reinterpret_cast<float4 *>(buf + (k * nfac + fc) * SLOT);
#pragma unroll
                            for (int v = 0; v < NL; v++)
                                if (lane + 32 * v < nv4) cp_async16(dk + lane + 32 * v, src + lane + 32 * v);
                        }
                    cp_async_wait_all();
                    __syncwarp();
                    if (mine) {
                        float vr, vi, wr = 0.f, wi = 0.f;
                        interp3f_one<PS, PA>(mybuf, Ls, Lt, Lp, vr, vi);
                        if (cs_) interp3f_one<PS, PA>(mybuf + SLOT, Ls, Lt, Lp, wr, wi);
                        prop_add(a0[qq], a1[qq], cs_, ps_, g, vr, vi, wr, wi);
                    }
                }
                pend = pend && !mine;
            }
        }
        if (act) {
#pragma unroll
            for (int qq = 0; qq < RB; qq++) {
                if (RB == 1 || q0 + qq < ca.nrhs) {
                    const long long base = ((long long)(q0 + qq) * Pl.nrc + rc) * Pl.nfac;
                    FP[base * ca.Pstride + n] = a0[qq].get();
                    if (ps_) FP[(base + 1) * ca.Pstride + n] = a1[qq].get();
                }
            }
        }
    }
}


// ============================================================================
// Adjoint (conjugate transpose) kernels.  Same geometry as the forward kernels,
// stages transposed and run in reverse order (all output-stationary).
// ============================================================================
template <typename T> struct CT;
template <> struct CT<double> { typedef double2 c; };
template <> struct CT<float> { typedef float2 c; };

template <typename C>
__device__ __forceinline__ C cconj_mul(C a, C b) {  // conj(a) * b
    C r;
    r.x = a.x * b.x + a.y * b.y;
    r.y = a.x * b.y - a.y * b.x;
    return r;
}

// Sum of one double per thread of the block, written to partials[blockIdx.x] (the
// k-derivative reductions; every thread of the block must call it).
__device__ __forceinline__ void block_sum_store(double v, double *partials) {
    __shared__ double sh[32];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    if (lane == 0) sh[wid] = v;
    __syncthreads();
    if (wid == 0) {
        v = lane < (int)(blockDim.x >> 5) ? sh[lane] : 0.0;
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
        if (lane == 0) partials[blockIdx.x] = v;
    }
}

// Re(conj(a) * b)
template <typename C>
__device__ __forceinline__ double re_conj_mul(C a, C b) {
    return (double)a.x * (double)b.x + (double)a.y * (double)b.y;
}

// Per-entry data staged in shared memory by the anterpolation kernel: the angular
// basis values and, per factor, the radial basis values times the entry's complex
// weight (sv[f][a] = Ls[a] v_f).  Rows padded so that vector loads stay aligned.
template <typename T, int PS, int PA, int NSV>
struct __align__(16) AntEntry {
    static constexpr int PAP = (PA + 3) & ~3, PSP = (PS + 1) & ~1;
    T Lt[PAP], Lp[PAP];
    typename CT<T>::c sv[NSV][PSP];  // [factor] weights; FP32 with the k-derivative also [2 + factor]
    T rho;                           // k-derivative factor of the entry (FP64 with the k-derivative)
};

// FP32 anterpolation accumulates with the packed two-lane FMA (f2fma).
constexpr bool kAntPacked = true;

// Columns c of one output row (factor, b) that an anterpolation thread owns: four or
// two consecutive ones in FP32 when Pang allows it, one otherwise.
template <int PA, bool MX>
struct AntCols {
    static constexpr int CQ = !MX ? 1 : (PA % 4 == 0 ? 4 : (PA % 2 == 0 ? 2 : 1));
};

// Anterpolation into the relevant cones of level d (transpose of K2 and K3):
// G_d[rc] = sum over its cousin targets of L(t) conj(E) g  +  sum over parent
// nodes propagated from it of L(t) conj(ratio) G_{d-1}.  One block per rc.
// With FUSE the block also accumulates H_d[rc], the same sum with every entry's
// weight scaled by -i rho, rho = r (cousin target) or r_c - r_p (parent node) --
// the k-derivatives of E and of the ratio -- and adds Re <H_d[rc], F_d[rc]> (F_d
// the forward cone values) to dk_partials[rc]: the k-derivative of the level's
// cousin and propagation terms, without storing H.  Each thread dots its own
// entry group's share of H (the shares sum to H by linearity).  The FP32 adjoint
// keeps six blocks per SM (at most 80 registers): the entry set-up chases
// dependent loads, and that occupancy hides them better than the extra registers
// of an uncapped build would pay back.
template <int PS, int PA, bool MX, bool FUSE>
__global__ void __launch_bounds__(128, MX ? (FUSE ? 4 : 6) : 4) k_ant(CommonArgs ca, LevelArgs L, LevelArgs Pl, LevelArgs LD,
                                              int has_parent, const long long *__restrict__ ad_start,
                                              const int *__restrict__ ad_list, ChebTab tb, const void *gs_,
                                              const void *Gp_, void *Gc_, const void *Fd_, double *dk_partials,
                                              const int *__restrict__ cs_first, const float4 *__restrict__ cs_geo4,
                                              const float2 *__restrict__ cs_geo2) {
    typedef typename std::conditional<MX, float, double>::type T;
    typedef typename CT<T>::c C;
    constexpr int P = PS * PA * PA, PA2 = PA * PA;
    const C *gs = (const C *)gs_;
    const C *Gp = (const C *)Gp_;
    C *Gc = (C *)Gc_;
    constexpr int CQ = AntCols<PA, MX>::CQ, PAQ = PA / CQ;
    // the k-derivative weights (-i rho) sv: staged as two more rows in FP32 (packed FMAs), formed
    // from rho in the accumulation in FP64 (same FMA count; keeps the stage within 48 KB)
    constexpr int NSV = (FUSE && MX) ? 4 : 2;
    typedef AntEntry<T, PS, PA, NSV> Ent;
    const C *Fd = (const C *)Fd_;
    double dk = 0.0;  // FUSE: this thread's share of Re <H_d[rc], F_d[rc]> over all right-hand sides
    // the entries of one batch, and after the last batch the partial sums of the entry groups
    union Stage {
        Ent ent[128];
        C part[128][CQ * PS];
    };
    __shared__ Stage sh;
    const int rc = blockIdx.x;
    const int cbox = L.rc_box[rc];
    const long long e0 = ad_start[rc], e1 = ad_start[rc + 1];
    const int nfac = L.nfac;
    const bool csplit = L.split != 0, psplit = has_parent && Pl.split != 0;
    // accumulation: thread = (factor, b, CQ consecutive c) of the output cone, all PS radial nodes
    // (a, b, c); the ng = 128 / (nfac PA PA / CQ) groups of such threads take every ng-th entry and
    // are summed at the end
    const int unit = threadIdx.x, nout = nfac * PA * PAQ, ng = 128 / nout;
    const int eg = unit / nout, uo = unit % nout;
    const bool active = eg < ng;
    const int fac = uo / (PA * PAQ), rb = uo % (PA * PAQ);
    const int ub = rb / PAQ, uc0 = (rb % PAQ) * CQ;
    for (int q = 0; q < ca.nrhs; q++) {
        C acc[CQ][PS], acck[FUSE ? CQ : 1][PS];
        unsigned long long acc2[CQ][PS], acck2[FUSE ? CQ : 1][PS];  // FP32: packed (re, im) accumulators of f2fma
#pragma unroll
        for (int j = 0; j < CQ; j++)
#pragma unroll
            for (int a = 0; a < PS; a++) {
                acc[j][a].x = acc[j][a].y = T(0);
                acc2[j][a] = 0ull;
                if constexpr (FUSE) {
                    acck[j][a].x = acck[j][a].y = T(0);
                    acck2[j][a] = 0ull;
                }
            }
        int ev_next = e0 + threadIdx.x < e1 ? ad_list[e0 + threadIdx.x] : 0;
        for (long long base = e0; base < e1; base += 128) {
            const long long e = base + threadIdx.x;
            const int ev = ev_next;
            if (e + 128 < e1) ev_next = ad_list[e + 128];  // next batch's entry, in flight during this one
            Ent &me = sh.ent[threadIdx.x];
            T t3[3] = {T(0), T(0), T(0)};
            C v0, v1;
            v0.x = v0.y = v1.x = v1.y = T(0);
            int cone_got = L.rc_cone[rc];
            T rho = T(0);  // k-derivative factor of the entry's weight (FUSE)
            if (e < e1) {
                if (ev < ca.N) {  // cousin target
                    const int i = ev;
                    const C g = gs[(long long)q * ca.N + i];
                    T Er, Ei, ir_abs;
                    if (MX && cs_first) {
                        // the forward lists hold this cone's cousin targets in the same order, with their
                        // local coordinates and centred factor from FP64 (|E| = 1 / (4 pi r))
                        const long long ge = (long long)cs_first[rc] + (e - e0);
                        const float4 g4 = __ldg(cs_geo4 + ge);
                        const float2 g2 = __ldg(cs_geo2 + ge);
                        t3[0] = (T)g4.x; t3[1] = (T)g4.y; t3[2] = (T)g4.z;
                        Er = (T)g4.w;
                        Ei = (T)g2.x;
                        ir_abs = (T)(4.f * kPiF * sqrtf(g4.w * g4.w + g2.x * g2.x));
                        rho = (T)1 / ir_abs;
                    } else if constexpr (MX) {
                        const int bl = ca.leaf_of[i];
                        const float sc = (float)L.scale;
                        const float M0 = LD.ijk[3 * bl] + 0.5f - (L.ijk[3 * cbox] + 0.5f) * sc;
                        const float M1 = LD.ijk[3 * bl + 1] + 0.5f - (L.ijk[3 * cbox + 1] + 0.5f) * sc;
                        const float M2 = LD.ijk[3 * bl + 2] + 0.5f - (L.ijk[3 * cbox + 2] + 0.5f) * sc;
                        const float f0 = ca.f32[3 * i], f1 = ca.f32[3 * i + 1], f2 = ca.f32[3 * i + 2];
                        float r;
                        const float tph = phase_cycles_exact(M0, M1, M2, f0, f1, f2, ca.kappa_hi, ca.kappa_lo, r);
                        float tt[3];
                        cone_got = classify32(L, M0 + f0, M1 + f1, M2 + f2, r, tt);
                        t3[0] = tt[0]; t3[1] = tt[1]; t3[2] = tt[2];
                        float sn, cs;
                        cis_cycles(tph, sn, cs);
                        const float c4 = 1.f / (4.f * kPiF * ca.HDf * r);
                        Er = c4 * cs;
                        Ei = c4 * sn;
                        ir_abs = 1.f / (r * ca.HDf);
                        rho = r * ca.HDf;
                    } else {
                        double y0[3];
                        center64(ca, L, cbox, y0);
                        double r, tt[3];
                        cone_got = classify64(L, ca.x64[3 * i] - y0[0], ca.x64[3 * i + 1] - y0[1], ca.x64[3 * i + 2] - y0[2],
                                              r, tt);
                        t3[0] = tt[0]; t3[1] = tt[1]; t3[2] = tt[2];
                        double sn, cs;
                        sincos(ca.k * r, &sn, &cs);
                        const double c4 = 1.0 / (4.0 * kPi * r);
                        Er = c4 * cs;
                        Ei = c4 * sn;
                        ir_abs = 1.0 / r;
                        rho = r;
                    }
                    C E;
                    E.x = Er;
                    E.y = Ei;
                    if (csplit) {
                        C E2;
                        E2.x = Er * ir_abs;
                        E2.y = Ei * ir_abs;
                        v0 = cconj_mul(E2, g);
                        v1 = cconj_mul(E, g);
                    } else {
                        v0 = cconj_mul(E, g);
                    }
                } else {  // parent cone node
                    const int idx = ev - ca.N;
                    const int rcp = idx / P, n = idx % P;
                    const int pb = Pl.rc_box[rcp];
                    T r1r, r1i, g1, irabs;
                    if constexpr (MX) {
                        float s, u[3];
                        node32<PS, PA>(Pl, tb, Pl.rc_cone[rcp], n, s, u);
                        const float rp = Pl.hu / s;
                        const float nv[3] = {rp * u[0], rp * u[1], rp * u[2]};
                        const float o0 = (L.ijk[3 * cbox] + 0.5f) * L.scale - (Pl.ijk[3 * pb] + 0.5f) * Pl.scale;
                        const float o1 = (L.ijk[3 * cbox + 1] + 0.5f) * L.scale - (Pl.ijk[3 * pb + 1] + 0.5f) * Pl.scale;
                        const float o2 = (L.ijk[3 * cbox + 2] + 0.5f) * L.scale - (Pl.ijk[3 * pb + 2] + 0.5f) * Pl.scale;
                        const float p0 = nv[0] - o0, p1 = nv[1] - o1, p2 = nv[2] - o2;
                        const float rcv = sqrtf(p0 * p0 + p1 * p1 + p2 * p2);
                        float tt[3];
                        cone_got = classify32(L, p0, p1, p2, rcv, tt);
                        t3[0] = tt[0]; t3[1] = tt[1]; t3[2] = tt[2];
                        const float oo = o0 * o0 + o1 * o1 + o2 * o2;
                        const float no = nv[0] * o0 + nv[1] * o1 + nv[2] * o2;
                        const float dr = (oo - 2.f * no) / (rcv + rp);
                        float t = ca.kappa_hi * dr;
                        t -= rintf(t);
                        float sn, cs;
                        cis_cycles(t, sn, cs);
                        g1 = rp / rcv;
                        r1r = cs * g1;
                        r1i = sn * g1;
                        irabs = 1.f / (rcv * ca.HDf);
                        rho = dr * ca.HDf;
                    } else {
                        double s, u[3];
                        node64<PS, PA>(Pl, tb, Pl.rc_cone[rcp], n, s, u);
                        double yp[3], yc[3];
                        center64(ca, Pl, pb, yp);
                        center64(ca, L, cbox, yc);
                        const double rp = Pl.h / s;
                        const double x[3] = {yp[0] + rp * u[0], yp[1] + rp * u[1], yp[2] + rp * u[2]};
                        double rcv, tt[3];
                        cone_got = classify64(L, x[0] - yc[0], x[1] - yc[1], x[2] - yc[2], rcv, tt);
                        t3[0] = tt[0]; t3[1] = tt[1]; t3[2] = tt[2];
                        double sn, cs;
                        sincos(ca.k * (rcv - rp), &sn, &cs);
                        g1 = rp / rcv;
                        r1r = cs * g1;
                        r1i = sn * g1;
                        irabs = 1.0 / rcv;
                        rho = rcv - rp;
                    }
                    C ratio1;
                    ratio1.x = r1r;
                    ratio1.y = r1i;
                    const long long pbase = ((long long)q * Pl.nrc + rcp) * Pl.nfac;
                    const C gp0 = Gp[pbase * ca.Pstride + n];
                    if (csplit) {
                        if (psplit) {
                            C ratio2;
                            ratio2.x = r1r * g1;
                            ratio2.y = r1i * g1;
                            const C gp1 = Gp[(pbase + 1) * ca.Pstride + n];
                            v0 = cconj_mul(ratio2, gp0);
                            v1 = cconj_mul(ratio1, gp1);
                        } else {
                            C rr;
                            rr.x = r1r * irabs;
                            rr.y = r1i * irabs;
                            v0 = cconj_mul(rr, gp0);
                            v1 = cconj_mul(ratio1, gp0);
                        }
                    } else {
                        v0 = cconj_mul(ratio1, gp0);
                    }
                }
                // express the local coordinates in the list's cone (an FP32 classification can land
                // in a neighbouring cone near a boundary): t' = t + 2 (i_got - i_list), phi wrapping
                const int cl = L.rc_cone[rc];
                if (cone_got != cl) {
                    const int ipg = cone_got % L.nph, itg = (cone_got / L.nph) % L.nC, isg = cone_got / (L.nph * L.nC);
                    const int ipl = cl % L.nph, itl = (cl / L.nph) % L.nC, isl = cl / (L.nph * L.nC);
                    int dp = ipg - ipl;
                    if (dp > L.nph / 2) dp -= L.nph;
                    if (dp < -L.nph / 2) dp += L.nph;
                    t3[0] += T(2 * (isg - isl));
                    t3[1] += T(2 * (itg - itl));
                    t3[2] += T(2 * dp);
                    const T lim = T(1.02);
                    if (q == 0 && (fabs(t3[0]) > lim || fabs(t3[1]) > lim || fabs(t3[2]) > lim)) atomicAdd(ca.missed, 1ULL);
                }
            }
            {
                T Ls[PS];
                lagrange<PS, T>(t3[0], MX ? (const T *)tb.fxs : (const T *)tb.xs,
                                MX ? (const T *)tb.fcs : (const T *)tb.cs, Ls);
                lagrange<PA, T>(t3[1], MX ? (const T *)tb.fxa : (const T *)tb.xa,
                                MX ? (const T *)tb.fca : (const T *)tb.ca, me.Lt);
                lagrange<PA, T>(t3[2], MX ? (const T *)tb.fxa : (const T *)tb.xa,
                                MX ? (const T *)tb.fca : (const T *)tb.ca, me.Lp);
#pragma unroll
                for (int a = 0; a < PS; a++) {
                    C z;
                    z.x = Ls[a] * v0.x;
                    z.y = Ls[a] * v0.y;
                    me.sv[0][a] = z;
                }
                if (csplit) {
#pragma unroll
                    for (int a = 0; a < PS; a++) {
                        C z;
                        z.x = Ls[a] * v1.x;
                        z.y = Ls[a] * v1.y;
                        me.sv[1][a] = z;
                    }
                }
                me.rho = rho;
                if constexpr (FUSE && MX) {  // (-i rho) times the weights
#pragma unroll
                    for (int f = 0; f < 2; f++) {
                        if (f == 1 && !csplit) break;
#pragma unroll
                        for (int a = 0; a < PS; a++) {
                            const C z = me.sv[f][a];
                            C zk;
                            zk.x = rho * z.y;
                            zk.y = -rho * z.x;
                            me.sv[NSV - 2 + f][a] = zk;
                        }
                    }
                }
            }
            __syncthreads();
            if (active) {
                const int cnt = (int)min((long long)128, e1 - base);
                for (int t = eg; t < cnt; t += ng) {
                    const Ent &en = sh.ent[t];
                    const T lt = en.Lt[ub];
                    T lp[CQ];
                    if constexpr (CQ == 4) {
                        const float4 l4 = *reinterpret_cast<const float4 *>(&en.Lp[uc0]);
                        lp[0] = l4.x; lp[1] = l4.y; lp[2] = l4.z; lp[3] = l4.w;
                    } else if constexpr (CQ == 2) {
                        const float2 l2 = *reinterpret_cast<const float2 *>(&en.Lp[uc0]);
                        lp[0] = l2.x; lp[1] = l2.y;
                    } else {
                        lp[0] = en.Lp[uc0];
                    }
                    if constexpr (MX && kAntPacked) {
                        unsigned long long sv[PS], svk[FUSE ? PS : 1];
                        const unsigned long long *row = reinterpret_cast<const unsigned long long *>(en.sv[fac]);
#pragma unroll
                        for (int a = 0; a < PS; a++) sv[a] = row[a];
                        if constexpr (FUSE) {
                            const unsigned long long *rowk = reinterpret_cast<const unsigned long long *>(en.sv[NSV - 2 + fac]);
#pragma unroll
                            for (int a = 0; a < PS; a++) svk[a] = rowk[a];
                        }
#pragma unroll
                        for (int j = 0; j < CQ; j++) {
                            const float w = lt * lp[j];
                            const unsigned long long w2 = f2pack(w, w);
#pragma unroll
                            for (int a = 0; a < PS; a++) {
                                f2fma(acc2[j][a], w2, sv[a]);
                                if constexpr (FUSE) f2fma(acck2[j][a], w2, svk[a]);
                            }
                        }
                    } else {
                        C sv[PS];
#pragma unroll
                        for (int a = 0; a < PS; a++) sv[a] = en.sv[fac][a];
                        const T rho = FUSE ? en.rho : T(0);
#pragma unroll
                        for (int j = 0; j < CQ; j++) {
                            const T w = lt * lp[j], wr = w * rho;
#pragma unroll
                            for (int a = 0; a < PS; a++) {
                                acc[j][a].x = fma(w, sv[a].x, acc[j][a].x);
                                acc[j][a].y = fma(w, sv[a].y, acc[j][a].y);
                                if constexpr (FUSE) {  // (-i rho) w sv
                                    acck[j][a].x = fma(wr, sv[a].y, acck[j][a].x);
                                    acck[j][a].y = fma(-wr, sv[a].x, acck[j][a].y);
                                }
                            }
                        }
                    }
                }
            }
            __syncthreads();
        }
        if constexpr (MX && kAntPacked) {
#pragma unroll
            for (int j = 0; j < CQ; j++)
#pragma unroll
                for (int a = 0; a < PS; a++) {
                    float x, y;
                    f2unpack(acc2[j][a], x, y);
                    acc[j][a].x = x;
                    acc[j][a].y = y;
                    if constexpr (FUSE) {
                        f2unpack(acck2[j][a], x, y);
                        acck[j][a].x = x;
                        acck[j][a].y = y;
                    }
                }
        }
        if constexpr (FUSE) {  // this entry group's share of H dotted with the forward values
            if (active) {
                const C *fo = Fd + (((long long)q * L.nrc + rc) * nfac + fac) * ca.Pstride + ub * PA + uc0;
#pragma unroll
                for (int j = 0; j < CQ; j++)
#pragma unroll
                    for (int a = 0; a < PS; a++) dk += re_conj_mul(acck[j][a], fo[a * PA2 + j]);
            }
        }
        // the loop's last barrier ends every read of the entries: the union's partial sums reuse them
        if (active && eg > 0) {
#pragma unroll
            for (int j = 0; j < CQ; j++)
#pragma unroll
                for (int a = 0; a < PS; a++) sh.part[unit][j * PS + a] = acc[j][a];
        }
        __syncthreads();
        if (active && eg == 0) {
            for (int g2 = 1; g2 < ng; g2++)
#pragma unroll
                for (int j = 0; j < CQ; j++)
#pragma unroll
                    for (int a = 0; a < PS; a++) {
                        acc[j][a].x += sh.part[g2 * nout + uo][j * PS + a].x;
                        acc[j][a].y += sh.part[g2 * nout + uo][j * PS + a].y;
                    }
            C *out = Gc + (((long long)q * L.nrc + rc) * nfac + fac) * ca.Pstride + ub * PA + uc0;
#pragma unroll
            for (int j = 0; j < CQ; j++)
#pragma unroll
                for (int a = 0; a < PS; a++) out[a * PA2 + j] = acc[j][a];
        }
        __syncthreads();
    }
    if constexpr (FUSE) block_sum_store(dk, dk_partials);
}

// Transposed leaf evaluation: b_j += sum over the cone nodes of j's leaf box of
// conj(W(x_n, y_j)) G (transpose of K1).  box_of == nullptr: the leaves of level D (L = LD); else the
// level of L, for the points whose level-L box is a leaf (leaf flags), as in an adaptive tree.
// With DK (mixed only) the same evaluations also give the leaf's part of Re <g, dA/dk sigma>
// (conj(dW/dk) G against the forward w sigma, as in k_leaf_adj_w), one double per block in dk_partials.
template <int PS, int PA, bool MX, bool DK = false>
__global__ void __launch_bounds__(128) k_leaf_adj(CommonArgs ca, LevelArgs L, ChebTab tb, const void *G_, void *b_,
                                                  const int *__restrict__ box_of, const uint8_t *__restrict__ leaf,
                                                  LevelArgs LD, const float2 *__restrict__ a_fwd = nullptr,
                                                  double *dk_partials = nullptr) {
    typedef typename std::conditional<MX, float, double>::type T;
    typedef typename CT<T>::c C;
    static_assert(!DK || MX, "the FP64 k-derivative of the leaf has its own pass (k_dk_leaf)");
    constexpr int P = PS * PA * PA;
    const C *G = (const C *)G_;
    C *bo = (C *)b_;
    const int jt = blockIdx.x * blockDim.x + threadIdx.x;
    double dk = 0.0;
    const int b = jt < ca.N ? (box_of ? box_of[jt] : ca.leaf_of[jt]) : 0;
    const bool act = jt < ca.N && !(leaf && !leaf[b]);
    if (!DK && !act) return;
    const int j = act ? jt : 0;
    const bool split = L.split != 0;
    // mixed: the source's offset from the box centre in leaf units (its level-D box offset plus the exact
    // difference of the two centres; zero at level D)
    float f0 = 0.f, f1 = 0.f, f2 = 0.f;
    if constexpr (MX) {
        const int e = ca.leaf_of[j];
        f0 = ca.f32[3 * j] + ((LD.ijk[3 * e] + 0.5f) - (L.ijk[3 * b] + 0.5f) * L.scale);
        f1 = ca.f32[3 * j + 1] + ((LD.ijk[3 * e + 1] + 0.5f) - (L.ijk[3 * b + 1] + 0.5f) * L.scale);
        f2 = ca.f32[3 * j + 2] + ((LD.ijk[3 * e + 2] + 0.5f) - (L.ijk[3 * b + 2] + 0.5f) * L.scale);
    }
    for (int q = 0; q < ca.nrhs && act; q++) {
        T ar = T(0), ai = T(0);
        float dr = 0.f, di = 0.f;  // DK: sum of conj(dW/dk) G
        for (int rc = L.rc_start[b]; rc < L.rc_start[b + 1]; rc++) {
            const int cone = L.rc_cone[rc];
            const long long gb = ((long long)q * L.nrc + rc) * L.nfac;
            for (int n = 0; n < P; n++) {
                T W0r, W0i, W1r = T(0), W1i = T(0);
                T D0r = T(0), D0i = T(0), D1r = T(0), D1i = T(0);  // DK: dW/dk
                if constexpr (MX) {
                    float s, u[3];
                    node32<PS, PA>(L, tb, cone, n, s, u);
                    const float hu = L.hu, ir = s / hu, kap = ca.kappa_hi, soh = s / (hu * ca.HDf);
                    const float dv0 = u[0] - f0 * ir, dv1 = u[1] - f1 * ir, dv2 = u[2] - f2 * ir;
                    const float a2 = dv0 * dv0 + dv1 * dv1 + dv2 * dv2;
                    const float ia = rsqrtf(a2), am = a2 * ia;
                    const float yy = f0 * f0 + f1 * f1 + f2 * f2, uy = u[0] * f0 + u[1] * f1 + u[2] * f2;
                    const float phl = (s * yy / hu - 2.f * uy) / (am + 1.f);  // phase distance, leaf units
                    float t = kap * phl;
                    t -= rintf(t);
                    float sn, cs;
                    cis_cycles(t, sn, cs);
                    const float dn = dv0 * ca.n32[3 * j] + dv1 * ca.n32[3 * j + 1] + dv2 * ca.n32[3 * j + 2];
                    const float w3 = dn * ia * ia, w2 = w3 * ia, g = ca.kf * w3 + ca.etaf * ia,
                                hr = ca.etaif * ia;
                    const float ph0 = phl * ca.HDf;  // absolute: dW/dk = i ph0 W - i e w3 (combined, W13), i ph0 W2
                    if (split) {
                        W0r = cs * w2; W0i = sn * w2; W1r = cs * hr + sn * g; W1i = sn * hr - cs * g;
                        if constexpr (DK) {
                            D0r = -ph0 * W0i; D0i = ph0 * W0r;
                            D1r = -ph0 * W1i + sn * w3; D1i = ph0 * W1r - cs * w3;
                        }
                    } else {
                        const float a = soh * w2 + hr;
                        W0r = cs * a + sn * g; W0i = sn * a - cs * g;
                        if constexpr (DK) {
                            D0r = -ph0 * W0i + sn * w3; D0i = ph0 * W0r - cs * w3;
                        }
                    }
                } else {
                    double s, u[3], y0[3];
                    node64<PS, PA>(L, tb, cone, n, s, u);
                    center64(ca, L, b, y0);
                    const double r = L.h / s, soh = s / L.h;
                    const double yv[3] = {ca.x64[3 * j] - y0[0], ca.x64[3 * j + 1] - y0[1], ca.x64[3 * j + 2] - y0[2]};
                    const double dv[3] = {u[0] - yv[0] / r, u[1] - yv[1] / r, u[2] - yv[2] / r};
                    const double am = sqrt(dv[0] * dv[0] + dv[1] * dv[1] + dv[2] * dv[2]);
                    const double yy = yv[0] * yv[0] + yv[1] * yv[1] + yv[2] * yv[2];
                    const double uy = u[0] * yv[0] + u[1] * yv[1] + u[2] * yv[2];
                    const double psi = ca.k * (s * yy / L.h - 2.0 * uy) / (am + 1.0);
                    double sn, cs;
                    sincos(psi, &sn, &cs);
                    const double dn = dv[0] * ca.n64[3 * j] + dv[1] * ca.n64[3 * j + 1] + dv[2] * ca.n64[3 * j + 2];
                    const double ia = 1.0 / am, w3 = dn * ia * ia, w2 = w3 * ia, g = ca.k * w3 + ca.eta * ia,
                                 hr = ca.etai * ia;
                    if (split) {
                        W0r = cs * w2; W0i = sn * w2; W1r = cs * hr + sn * g; W1i = sn * hr - cs * g;
                    } else {
                        const double a = soh * w2 + hr;
                        W0r = cs * a + sn * g; W0i = sn * a - cs * g;
                    }
                }
                const C g0 = G[gb * ca.Pstride + n];
                ar += W0r * g0.x + W0i * g0.y;  // conj(W) * G
                ai += W0r * g0.y - W0i * g0.x;
                if constexpr (DK) {
                    dr += D0r * g0.x + D0i * g0.y;
                    di += D0r * g0.y - D0i * g0.x;
                }
                if (split) {
                    const C g1 = G[(gb + 1) * ca.Pstride + n];
                    ar += W1r * g1.x + W1i * g1.y;
                    ai += W1r * g1.y - W1i * g1.x;
                    if constexpr (DK) {
                        dr += D1r * g1.x + D1i * g1.y;
                        di += D1r * g1.y - D1i * g1.x;
                    }
                }
            }
        }
        C v = bo[(long long)q * ca.N + j];
        v.x += ar;
        v.y += ai;
        bo[(long long)q * ca.N + j] = v;
        if constexpr (DK) {  // Re(conj(T) a_j), T = sum conj(dW) G
            const float2 aj = a_fwd[(long long)q * ca.N + j];
            dk += (double)dr * aj.x + (double)di * aj.y;
        }
    }
    if constexpr (DK) block_sum_store(dk, dk_partials);
}

// Transposed leaf evaluation (mixed), warp-cooperative: one warp per chunk of at
// most 32 sources of one leaf box (the level-D cousin chunks).  For 32 nodes of a
// relevant cone at a time each lane computes one node's direction, 1/r and scale
// and loads its cone values once into the warp's shared-memory slots; the warp
// then walks the 32 nodes with broadcast loads, every lane evaluating
// conj(W(x_node, y_j)) G for its source.
template <int PS, int PA, bool SPLIT, bool DK>
__global__ void __launch_bounds__(128) k_leaf_adj_w(CommonArgs ca, LevelArgs L, const int4 *__restrict__ chunks,
                                                    int nchunk, ChebTab tb, const float2 *__restrict__ G,
                                                    float2 *__restrict__ bo, const float2 *__restrict__ a_fwd,
                                                    double *dk_partials) {
    constexpr int P = PS * PA * PA;
    __shared__ float4 s_dir[4][32];  // (u0, u1, u2, 1/r) per node, r in leaf units
    __shared__ float4 s_g[4][32];    // (G0, G1) per node; G1 = (s/h, 0) when the factor is combined
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int ch = blockIdx.x * (blockDim.x >> 5) + warp;
    double dk = 0.0;  // DK: this thread's share of the leaf part of Re <g, dA/dk sigma>
    const bool live = ch < nchunk;  // warp-uniform
    const int4 cw = chunks[live ? ch : 0];
    const int b = cw.x;
    const bool act = live && lane < cw.z;
    const int j = cw.y + (act ? lane : 0);
    const float4 fj = __ldg(ca.pn32 + 2 * j), nj = __ldg(ca.pn32 + 2 * j + 1);
    const float hu = L.hu, kap = ca.kappa_hi, kf = ca.kf, etaf = ca.etaf, etaif = ca.etaif, hd = ca.HDf;
    const float yy = fj.w;  // |f|^2
    const int r0 = L.rc_start[b], r1 = L.rc_start[b + 1];
    for (int q = 0; q < ca.nrhs && live; q++) {
        PAcc acc, dacc;
        acc.zero();
        dacc.zero();
        for (int rc = r0; rc < r1; rc++) {
            const int cone = L.rc_cone[rc];
            const long long gb = ((long long)q * L.nrc + rc) * L.nfac;
            for (int n0 = 0; n0 < P; n0 += 32) {
                const int n = min(n0 + lane, P - 1);
                {
                    float sl, ul[3];
                    node32<PS, PA>(L, tb, cone, n, sl, ul);
                    const float2 gl0 = G[gb * ca.Pstride + n];
                    const float irl = sl / hu;  // 1 / r (leaf units)
                    float2 gl1;
                    if (SPLIT)
                        gl1 = G[(gb + 1) * ca.Pstride + n];
                    else
                        gl1 = make_float2(irl / hd, 0.f);  // s / h (absolute)
                    __syncwarp();  // the previous batch's reads are done
                    s_dir[warp][lane] = make_float4(ul[0], ul[1], ul[2], irl);
                    s_g[warp][lane] = make_float4(gl0.x, gl0.y, gl1.x, gl1.y);
                    __syncwarp();
                }
                const int cnt = min(32, P - n0);
                for (int k = 0; k < cnt; k++) {
                    const float4 dk = s_dir[warp][k], gk = s_g[warp][k];
                    const float u0 = dk.x, u1 = dk.y, u2 = dk.z, ir = dk.w;
                    const float g0x = gk.x, g0y = gk.y;
                    const float dv0 = u0 - fj.x * ir, dv1 = u1 - fj.y * ir, dv2 = u2 - fj.z * ir;
                    const float a2 = dv0 * dv0 + dv1 * dv1 + dv2 * dv2;
                    const float ia = rsqrtf(a2), am = a2 * ia;
                    const float uy = u0 * fj.x + u1 * fj.y + u2 * fj.z;
                    const float phl = __fdividef(ir * yy - 2.f * uy, am + 1.f);  // phase distance, leaf units
                    float t = kap * phl;
                    t -= rintf(t);
                    float sn, cs;
                    cis_cycles(t, sn, cs);
                    const float dn = dv0 * nj.x + dv1 * nj.y + dv2 * nj.z;
                    const float w3 = dn * ia * ia, w2 = w3 * ia, g = kf * w3 + etaf * ia, hr = etaif * ia;
                    const float ph0 = phl * hd;  // absolute: dW/dk = i ph0 W - i e w3 (combined, W13), i ph0 W2
                    if (SPLIT) {
                        const float g1x = gk.z, g1y = gk.w;
                        const float W0r = cs * w2, W0i = sn * w2, W1r = cs * hr + sn * g, W1i = sn * hr - cs * g;
                        acc.add(W0r * g0x + W0i * g0y + W1r * g1x + W1i * g1y,
                                W0r * g0y - W0i * g0x + W1r * g1y - W1i * g1x);
                        if constexpr (DK) {  // conj(dW) G
                            const float d0r = -ph0 * W0i, d0i = ph0 * W0r;
                            const float d1r = -ph0 * W1i + sn * w3, d1i = ph0 * W1r - cs * w3;
                            dacc.add(d0r * g0x + d0i * g0y + d1r * g1x + d1i * g1y,
                                     d0r * g0y - d0i * g0x + d1r * g1y - d1i * g1x);
                        }
                    } else {
                        const float a = gk.z * w2 + hr;  // gk.z = s / h
                        const float W0r = cs * a + sn * g, W0i = sn * a - cs * g;
                        acc.add(W0r * g0x + W0i * g0y, W0r * g0y - W0i * g0x);  // conj(W) G
                        if constexpr (DK) {
                            const float d0r = -ph0 * W0i + sn * w3, d0i = ph0 * W0r - cs * w3;
                            dacc.add(d0r * g0x + d0i * g0y, d0r * g0y - d0i * g0x);
                        }
                    }
                }
            }
        }
        if (act) {
            const float2 w = acc.get();
            float2 v = bo[(long long)q * ca.N + j];
            v.x += w.x;
            v.y += w.y;
            bo[(long long)q * ca.N + j] = v;
            if constexpr (DK) {  // Re(conj(T) a_j), T = sum conj(dW) G
                const float2 z = dacc.get(), aj = a_fwd[(long long)q * ca.N + j];
                dk += (double)z.x * aj.x + (double)z.y * aj.y;
            }
        }
    }
    if constexpr (DK) block_sum_store(dk, dk_partials);
}

// Transposed near field (mixed): b_j = sum_{i in the 27-neighbourhood, i != j} conj(K(x_i, x_j)) g_i,
// packed point records, constants hoisted.  With DK the same pairs also give the near-field part of
// Re <g, dA/dk sigma> = sum_j Re( a_j sum_i conj(g_i) dK/dk(x_i, x_j) ), dK/dk = i R K - i E dn / r
// (a = w sigma of the forward state), one double per block in dk_partials.
template <bool DK>
__global__ void __launch_bounds__(128) k_near_adj32(CommonArgs ca, LevelArgs L, const float2 *__restrict__ gs,
                                                    float2 *__restrict__ bo, const float2 *__restrict__ a_fwd,
                                                    double *dk_partials) {
    const int jt = blockIdx.x * blockDim.x + threadIdx.x;
    double dk = 0.0;
    const bool live = jt < ca.N;
    const int j = live ? jt : 0;
    const int b = ca.leaf_of[j];
    const int bi0 = L.ijk[3 * b], bi1 = L.ijk[3 * b + 1], bi2 = L.ijk[3 * b + 2];
    const float4 *pn = ca.pn32;
    const float4 fj = __ldg(pn + 2 * j), nj = __ldg(pn + 2 * j + 1);
    const float kf = ca.kf, etaf = ca.etaf, etaif = ca.etaif, kap = ca.kappa_hi;
    const float c4 = 1.f / (4.f * kPiF * ca.HDf), iHD = 1.f / ca.HDf;
    const float tolu = (float)(ca.tol / ca.HD);
    for (int q = 0; q < ca.nrhs && live; q++) {
        PAcc acc, dacc;
        acc.zero();
        dacc.zero();
        for (int nb = ca.nb_start[b]; nb < ca.nb_start[b + 1]; nb++) {
            const int c = ca.nb_list[nb];
            const float D0 = (float)(L.ijk[3 * c] - bi0) - fj.x, D1 = (float)(L.ijk[3 * c + 1] - bi1) - fj.y,
                        D2 = (float)(L.ijk[3 * c + 2] - bi2) - fj.z;
            for (int i = L.start[c]; i < L.start[c + 1]; i++) {
                if (i == j) continue;
                const float4 fi = __ldg(pn + 2 * i);
                const float d0 = D0 + fi.x, d1 = D1 + fi.y, d2 = D2 + fi.z;  // x_i - x_j (leaf units)
                const float r2 = d0 * d0 + d1 * d1 + d2 * d2, ir = rsqrtf(r2), r = r2 * ir;
                if (!(r >= tolu)) continue;
                float t = kap * r;
                t -= rintf(t);
                float sn, cs;
                cis_cycles(t, sn, cs);
                const float dn = d0 * nj.x + d1 * nj.y + d2 * nj.z;
                const float A = dn * ir * ir * iHD + etaif, Bv = -(kf * dn * ir + etaf);
                const float amp = c4 * ir;
                const float Kr = amp * (cs * A - sn * Bv), Ki = amp * (sn * A + cs * Bv);
                const float2 g = gs[(long long)q * ca.N + i];
                acc.add(Kr * g.x + Ki * g.y, Kr * g.y - Ki * g.x);  // conj(K) g
                if constexpr (DK) {  // conj(g) dK/dk
                    const float R = r * ca.HDf, dnr = dn * ir;
                    const float dKr = -R * Ki + amp * sn * dnr, dKi = R * Kr - amp * cs * dnr;
                    dacc.add(g.x * dKr + g.y * dKi, g.x * dKi - g.y * dKr);
                }
            }
        }
        bo[(long long)q * ca.N + j] = acc.get();
        if constexpr (DK) {
            const float2 z = dacc.get(), aj = a_fwd[(long long)q * ca.N + j];
            dk += (double)z.x * aj.x - (double)z.y * aj.y;  // Re(z a_j)
        }
    }
    if constexpr (DK) block_sum_store(dk, dk_partials);
}

// Transposed near field: b_j = sum_{i in the 27-neighbourhood, i != j} conj(K(x_i, x_j)) g_i.
template <bool MX>
__global__ void __launch_bounds__(128) k_near_adj(CommonArgs ca, LevelArgs L, const void *gs_, void *b_) {
    typedef typename std::conditional<MX, float, double>::type T;
    typedef typename CT<T>::c C;
    const C *gs = (const C *)gs_;
    C *bo = (C *)b_;
    const int j = blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= ca.N) return;
    const int b = ca.leaf_of[j];
    for (int q = 0; q < ca.nrhs; q++) {
        T ar = T(0), ai = T(0);
        for (int nb = ca.nb_start[b]; nb < ca.nb_start[b + 1]; nb++) {
            const int c = ca.nb_list[nb];
            for (int i = L.start[c]; i < L.start[c + 1]; i++) {
                if (i == j) continue;
                T Kr, Ki;
                if constexpr (MX) {
                    const float d0 = (float)(L.ijk[3 * c] - L.ijk[3 * b]) + ca.f32[3 * i] - ca.f32[3 * j];
                    const float d1 = (float)(L.ijk[3 * c + 1] - L.ijk[3 * b + 1]) + ca.f32[3 * i + 1] - ca.f32[3 * j + 1];
                    const float d2 = (float)(L.ijk[3 * c + 2] - L.ijk[3 * b + 2]) + ca.f32[3 * i + 2] - ca.f32[3 * j + 2];
                    const float r2 = d0 * d0 + d1 * d1 + d2 * d2, ir = rsqrtf(r2), r = r2 * ir;
                    if (!(r >= (float)(ca.tol / ca.HD))) continue;
                    float t = ca.kappa_hi * r;
                    t -= rintf(t);
                    float sn, cs;
                    cis_cycles(t, sn, cs);
                    const float dn = d0 * ca.n32[3 * j] + d1 * ca.n32[3 * j + 1] + d2 * ca.n32[3 * j + 2];
                    const float A = dn * ir * ir / ca.HDf + ca.etaif, Bv = -(ca.kf * dn * ir + ca.etaf);
                    const float amp = ir / (4.f * kPiF * ca.HDf);
                    Kr = amp * (cs * A - sn * Bv);
                    Ki = amp * (sn * A + cs * Bv);
                } else {
                    const double d0 = ca.x64[3 * i] - ca.x64[3 * j], d1 = ca.x64[3 * i + 1] - ca.x64[3 * j + 1],
                                 d2 = ca.x64[3 * i + 2] - ca.x64[3 * j + 2];
                    const double r = sqrt(d0 * d0 + d1 * d1 + d2 * d2);
                    if (r < ca.tol) continue;
                    double sn, cs;
                    sincos(ca.k * r, &sn, &cs);
                    const double ir = 1.0 / r;
                    const double dn = d0 * ca.n64[3 * j] + d1 * ca.n64[3 * j + 1] + d2 * ca.n64[3 * j + 2];
                    const double A = dn * ir * ir + ca.etai, Bv = -(ca.k * dn * ir + ca.eta);
                    const double amp = ir / (4.0 * kPi);
                    Kr = amp * (cs * A - sn * Bv);
                    Ki = amp * (sn * A + cs * Bv);
                }
                const C g = gs[(long long)q * ca.N + i];
                ar += Kr * g.x + Ki * g.y;
                ai += Kr * g.y - Ki * g.x;
            }
        }
        C v;
        v.x = ar;
        v.y = ai;
        bo[(long long)q * ca.N + j] = v;
    }
}

// gs[q][s] = g[q][perm[s]]
template <typename C>
__global__ void k_gather_plain(int N, int nrhs, const int *__restrict__ perm, const C *__restrict__ g, C *__restrict__ gs) {
    long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (i >= (long long)N * nrhs) return;
    const int q = (int)(i / N), s = (int)(i % N);
    gs[i] = g[(long long)q * N + perm[s]];
}

// out[q][perm[s]] = conj(cI) g[q][perm[s]] + w_s b[q][s]   (cI real)
template <typename T>
__global__ void k_scatter_adj(int N, int nrhs, const int *__restrict__ perm, double cI, const T *__restrict__ w,
                              const typename CT<T>::c *__restrict__ g, const typename CT<T>::c *__restrict__ b,
                              typename CT<T>::c *__restrict__ out) {
    long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (i >= (long long)N * nrhs) return;
    const int q = (int)(i / N), s = (int)(i % N);
    const long long o = (long long)q * N + perm[s];
    typename CT<T>::c gg = g[o], bb = b[i], r;
    r.x = (T)cI * gg.x + w[s] * bb.x;
    r.y = (T)cI * gg.y + w[s] * bb.y;
    out[o] = r;
}


// ============================================================================
// k-derivative reductions:  Re <g, (dA/dk) sigma>  with the plan frozen and eta
// fixed.  Each kernel mirrors a forward stage and reduces conj(cotangent) times
// the k-derivative of that stage's output, using the forward state (w sigma, the
// cone values F) and the adjoint state (gathered g, the cone values G).  One
// double per block is written to `partials`.  The cousin and propagation terms
// are reduced inside the anterpolation (k_ant with FUSE).
// ============================================================================
// near field: sum_i conj(g_i) sum_j dK/dk(x_i, x_j) a_j,  dK/dk = i r K - i E1 dn / r
template <bool MX>
__global__ void __launch_bounds__(128) k_dk_near(CommonArgs ca, LevelArgs L, const void *a_, const void *gs_,
                                                 double *partials) {
    typedef typename std::conditional<MX, float, double>::type T;
    typedef typename CT<T>::c C;
    const C *a = (const C *)a_;
    const C *gs = (const C *)gs_;
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    double acc = 0.0;
    if (i < ca.N) {
        const int b = ca.leaf_of[i];
        for (int q = 0; q < ca.nrhs; q++) {
            T sr = T(0), si = T(0);
            for (int nb = ca.nb_start[b]; nb < ca.nb_start[b + 1]; nb++) {
                const int c = ca.nb_list[nb];
                for (int j = L.start[c]; j < L.start[c + 1]; j++) {
                    if (j == i) continue;
                    T Er, Ei, Br, Bi, R, dnr;
                    if constexpr (MX) {
                        const float4 fi = __ldg(ca.pn32 + 2 * i), fj = __ldg(ca.pn32 + 2 * j);
                        const float d0 = (float)(L.ijk[3 * b] - L.ijk[3 * c]) + fi.x - fj.x;
                        const float d1 = (float)(L.ijk[3 * b + 1] - L.ijk[3 * c + 1]) + fi.y - fj.y;
                        const float d2 = (float)(L.ijk[3 * b + 2] - L.ijk[3 * c + 2]) + fi.z - fj.z;
                        const float r2 = d0 * d0 + d1 * d1 + d2 * d2, ir = rsqrtf(r2), r = r2 * ir;
                        if (!(r >= (float)(ca.tol / ca.HD))) continue;
                        float t = ca.kappa_hi * r;
                        t -= rintf(t);
                        float sn, cs;
                        cis_cycles(t, sn, cs);
                        const float4 nj = __ldg(ca.pn32 + 2 * j + 1);
                        const float dn = d0 * nj.x + d1 * nj.y + d2 * nj.z;
                        const float amp = ir / (4.f * kPiF * ca.HDf);
                        Er = amp * cs; Ei = amp * sn;
                        Br = dn * ir * ir / ca.HDf + ca.etaif; Bi = -(ca.kf * dn * ir + ca.etaf);
                        R = r * ca.HDf;
                        dnr = dn * ir;
                    } else {
                        const double d0 = ca.x64[3 * i] - ca.x64[3 * j], d1 = ca.x64[3 * i + 1] - ca.x64[3 * j + 1],
                                     d2 = ca.x64[3 * i + 2] - ca.x64[3 * j + 2];
                        const double r = sqrt(d0 * d0 + d1 * d1 + d2 * d2);
                        if (r < ca.tol) continue;
                        double sn, cs;
                        sincos(ca.k * r, &sn, &cs);
                        const double ir = 1.0 / r, dn = d0 * ca.n64[3 * j] + d1 * ca.n64[3 * j + 1] + d2 * ca.n64[3 * j + 2];
                        Er = cs * ir / (4.0 * kPi); Ei = sn * ir / (4.0 * kPi);
                        Br = dn * ir * ir + ca.etai; Bi = -(ca.k * dn * ir + ca.eta);
                        R = r;
                        dnr = dn * ir;
                    }
                    // K = E B; dK/dk = i R E B - i E dn/r
                    const T Kr = Er * Br - Ei * Bi, Ki = Er * Bi + Ei * Br;
                    const T dKr = -R * Ki + Ei * dnr, dKi = R * Kr - Er * dnr;
                    const C aj = a[(long long)q * ca.N + j];
                    sr += dKr * aj.x - dKi * aj.y;
                    si += dKr * aj.y + dKi * aj.x;
                }
            }
            C z;
            z.x = sr;
            z.y = si;
            acc += re_conj_mul(gs[(long long)q * ca.N + i], z);
        }
    }
    block_sum_store(acc, partials);
}

// leaf evaluation: sum_{rc,n} conj(G_D[n]) sum_j dW/dk(x_n, y_j) a_j,
// dW/dk = i phi0 W - i e w3 (combined or W13),  i phi0 W2 (split W2)
// (rc_list: the relevant cones of the leaves of a coarser level of an adaptive tree, nlist of them, FP64
// only; nullptr: every relevant cone of the level)
template <int PS, int PA, bool MX>
__global__ void __launch_bounds__(128) k_dk_leaf(CommonArgs ca, LevelArgs L, ChebTab tb, const void *a_, const void *G_,
                                                 double *partials, const int *__restrict__ rc_list, long long nlist) {
    typedef typename std::conditional<MX, float, double>::type T;
    typedef typename CT<T>::c C;
    constexpr int P = PS * PA * PA;
    const C *a = (const C *)a_;
    const C *G = (const C *)G_;
    const long long tid = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    double acc = 0.0;
    if (tid < nlist * P) {
        const int rc = rc_list ? rc_list[tid / P] : (int)(tid / P), n = (int)(tid % P);
        const int b = L.rc_box[rc];
        // the node's geometry, once (FP32 in leaf units, FP64 absolute)
        float s32 = 0.f, u32[3] = {0.f, 0.f, 0.f};
        double s64 = 0.0, u64[3] = {0.0, 0.0, 0.0}, y0[3] = {0.0, 0.0, 0.0};
        if constexpr (MX) node32<PS, PA>(L, tb, L.rc_cone[rc], n, s32, u32);
        else {
            node64<PS, PA>(L, tb, L.rc_cone[rc], n, s64, u64);
            center64(ca, L, b, y0);
        }
        for (int q = 0; q < ca.nrhs; q++) {
            T s0r = T(0), s0i = T(0), s1r = T(0), s1i = T(0);
            for (int j = L.start[b]; j < L.start[b + 1]; j++) {
                T cs, sn, w1, w2, w3, soh, ph0;
                if constexpr (MX) {
                    const float s = s32, *u = u32;
                    const float hu = L.hu, ir = s / hu;
                    const float4 fj = __ldg(ca.pn32 + 2 * j), nj = __ldg(ca.pn32 + 2 * j + 1);
                    const float f0 = fj.x, f1 = fj.y, f2 = fj.z;
                    const float dv0 = u[0] - f0 * ir, dv1 = u[1] - f1 * ir, dv2 = u[2] - f2 * ir;
                    const float a2 = dv0 * dv0 + dv1 * dv1 + dv2 * dv2, ia = rsqrtf(a2), am = a2 * ia;
                    const float yy = fj.w, uy = u[0] * f0 + u[1] * f1 + u[2] * f2;
                    const float phl = __fdividef(s * yy / hu - 2.f * uy, am + 1.f);  // leaf units; am + 1 in [1, 3]
                    float t = ca.kappa_hi * phl;
                    t -= rintf(t);
                    float snf, csf;
                    cis_cycles(t, snf, csf);
                    sn = snf; cs = csf;
                    const float dn = dv0 * nj.x + dv1 * nj.y + dv2 * nj.z;
                    w1 = ia; w3 = dn * ia * ia; w2 = w3 * ia;
                    soh = s / (hu * ca.HDf);
                    ph0 = phl * ca.HDf;
                } else {
                    const double s = s64, *u = u64;
                    const double r = L.h / s;
                    const double yv[3] = {ca.x64[3 * j] - y0[0], ca.x64[3 * j + 1] - y0[1], ca.x64[3 * j + 2] - y0[2]};
                    const double dv[3] = {u[0] - yv[0] / r, u[1] - yv[1] / r, u[2] - yv[2] / r};
                    const double am = sqrt(dv[0] * dv[0] + dv[1] * dv[1] + dv[2] * dv[2]);
                    const double yy = yv[0] * yv[0] + yv[1] * yv[1] + yv[2] * yv[2];
                    const double uy = u[0] * yv[0] + u[1] * yv[1] + u[2] * yv[2];
                    ph0 = (s * yy / L.h - 2.0 * uy) / (am + 1.0);
                    sincos(ca.k * ph0, &sn, &cs);
                    const double dn = dv[0] * ca.n64[3 * j] + dv[1] * ca.n64[3 * j + 1] + dv[2] * ca.n64[3 * j + 2];
                    const double ia = 1.0 / am;
                    w1 = ia; w3 = dn * ia * ia; w2 = w3 * ia;
                    soh = s / L.h;
                }
                const T kk = MX ? (T)ca.kf : (T)ca.k, ee = MX ? (T)ca.etaf : (T)ca.eta,
                        ei = MX ? (T)ca.etaif : (T)ca.etai;
                // W = e (A + i B): combined A = soh w2 + etai w1, B = -(k w3 + eta w1); split: W2 = e w2,
                // W13 = e (etai w1 - i (k w3 + eta w1))
                T d0r, d0i, d1r = T(0), d1i = T(0);
                const T g = kk * w3 + ee * w1, hr = ei * w1;
                if (L.split) {
                    // dW2/dk = i ph0 e w2
                    d0r = -ph0 * sn * w2; d0i = ph0 * cs * w2;
                    // dW13 = i ph0 W13 - i e w3
                    const T W13r = cs * hr + sn * g, W13i = sn * hr - cs * g;
                    d1r = -ph0 * W13i + sn * w3;
                    d1i = ph0 * W13r - cs * w3;
                } else {
                    const T a0 = soh * w2 + hr;
                    const T Wr = cs * a0 + sn * g, Wi = sn * a0 - cs * g;
                    d0r = -ph0 * Wi + sn * w3;
                    d0i = ph0 * Wr - cs * w3;
                }
                const C aj = a[(long long)q * ca.N + j];
                s0r += d0r * aj.x - d0i * aj.y; s0i += d0r * aj.y + d0i * aj.x;
                s1r += d1r * aj.x - d1i * aj.y; s1i += d1r * aj.y + d1i * aj.x;
            }
            const long long gb = ((long long)q * L.nrc + rc) * L.nfac;
            C z0, z1;
            z0.x = s0r; z0.y = s0i; z1.x = s1r; z1.y = s1i;
            acc += re_conj_mul(G[gb * ca.Pstride + n], z0);
            if (L.split) acc += re_conj_mul(G[(gb + 1) * ca.Pstride + n], z1);
        }
    }
    block_sum_store(acc, partials);
}


// ============================================================================
// Tensor-core propagation (mixed path, Pang = 8).  For one group key (child
// octant, parent cone id) the map from a child cone's node values to the parent
// cone's node values is the same for every (parent cone, child box) pair of the
// key, so a block evaluates it as a dense contraction
//     D[node, pair] = sum_k W[node, k] F_child(pair)[k]      (M = P, K = P, N = pairs)
// with warp-level mma.sync m16n8k8 TF32 and a three-term split (hi*hi + hi*lo +
// lo*hi) that keeps FP32 accuracy; W[node, (a,b,c)] = Ls[a] Lt[b] Lp[c] at the
// node's child coordinates is generated in the A fragments from per-node basis
// values staged in shared memory.  The epilogue multiplies by the centred-factor
// ratio and adds into the parent cone values (the caller zeroes them and launches
// one octant at a time, so no parent cone is written twice by one launch).
// ============================================================================
__device__ __forceinline__ unsigned f2tf32(float x) {
    unsigned r;
    asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(r) : "f"(x));
    return r;
}

__device__ __forceinline__ void split_tf32(float x, unsigned &hi, unsigned &lo) {
    hi = f2tf32(x);
    lo = f2tf32(x - __uint_as_float(hi));
}

__device__ __forceinline__ void mma_tf32(float *d, const unsigned *a, const unsigned *b) {
    asm volatile(
        "mma.sync.aligned.m16n8k8.row.col.f32.tf32.tf32.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, "
        "{%0,%1,%2,%3};\n"
        : "+f"(d[0]), "+f"(d[1]), "+f"(d[2]), "+f"(d[3])
        : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b[0]), "r"(b[1]));
}

// four 8x8 b16 tiles from shared memory; with 32-bit elements, lane l receives word (l % 4)
// of row (l / 4) of each tile — the m16n8k8 TF32 B fragment layout for an n-major tile
__device__ __forceinline__ void ldmatrix_x4(const void *smem_row, unsigned &r0, unsigned &r1, unsigned &r2,
                                            unsigned &r3) {
    const unsigned a = (unsigned)__cvta_generic_to_shared(smem_row);
    asm volatile("ldmatrix.sync.aligned.m8n8.x4.shared.b16 {%0,%1,%2,%3}, [%4];\n"
                 : "=r"(r0), "=r"(r1), "=r"(r2), "=r"(r3)
                 : "r"(a));
}

constexpr int kTcRows = 64;  // parent nodes per block (one m16 tile per warp)

template <int PS>
struct TcSmem {
    float Ls[kTcRows][PS];
    float Lt[kTcRows][12];  // row stride 12: the 32 lanes' (row, tig) reads hit 32 distinct banks
    float Lp[kTcRows][12];
    float rr[kTcRows], ri[kTcRows], g1[kTcRows], ir[kTcRows];
    short perm[kTcRows];        // parent node of each block row (nodes sorted by child cone)
    signed char slot[kTcRows];  // index of the row's child cone in `cones`, -1 if absent
    int cones[16];
    int ncones;
    int present[16];
    int jlist[16];  // slots present among the block's rows, ascending
    int njp;
    int crc[16][kTcPairs];
    int rcp[kTcPairs], cb[kTcPairs];
    // one K-chunk (64 child nodes) of the pairs' child values, split into TF32 hi (bt[0]) and
    // lo (bt[1]), stored n-major: bt[h][n][k] with n = 2 * pair + (re, im).  The row stride of
    // 68 words (272 bytes) puts the 8 rows of an ldmatrix tile in 8 distinct 16-byte bank groups.
    // Before the first chunk, bt holds the child cone of every parent node (P ints).
    alignas(16) unsigned bt[2][64][68];
};

// Parent node n of cone gamma seen from the child: position relative to the child
// centre (p), its distance (rcv) and the node's distance to the parent centre (rp).
template <int PS>
__device__ __forceinline__ int tc_child_cone(const LevelArgs &C, const LevelArgs &Pl, const ChebTab &tb, int gamma,
                                             int n, float o0, float o1, float o2, float *nv, float &rp, float &rcv,
                                             float *t3) {
    float s, u[3];
    node32<PS, 8>(Pl, tb, gamma, n, s, u);
    rp = Pl.hu / s;
    nv[0] = rp * u[0];
    nv[1] = rp * u[1];
    nv[2] = rp * u[2];
    const float p0 = nv[0] - o0, p1 = nv[1] - o1, p2 = nv[2] - o2;
    rcv = sqrtf(p0 * p0 + p1 * p1 + p2 * p2);
    return classify32(C, p0, p1, p2, rcv, t3);
}

// grid: (tiles of this octant) x (P / 64 row slices).  The parent nodes of the group
// key are ordered by the child cone they fall in (ascending cone id, then node index),
// so the 16 rows of a warp mostly share one child cone and the masked work of rows in
// other cones stays small; block y takes rows [64 y, 64 y + 64) of that order.
template <int PS>
__global__ void __launch_bounds__(128, 4) k_prop_tc(CommonArgs ca, LevelArgs C, LevelArgs Pl, ChebTab tb, TcLevel T,
                                                 int tile0) {
    constexpr int P = PS * 64, NT = kTcPairs / 4;
    __shared__ TcSmem<PS> sm;
    static_assert(P <= 2 * 64 * 68, "child cone table must fit in the staging buffer");
    int *ccone = reinterpret_cast<int *>(&sm.bt[0][0][0]);
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31, g = lane >> 2, tig = lane & 3;
    const int tile = tile0 + (blockIdx.x >> 1), half = blockIdx.x & 1;  // a tile is two blocks of 32 pairs
    const int row0 = blockIdx.y * kTcRows;  // first sorted row of this block
    const int grp = T.tile_group[tile], p0 = T.tile_start[tile] + kTcPairs * half;
    const int np = min(kTcPairs, T.tile_count[tile] - kTcPairs * half);
    if (np <= 0) return;  // block-uniform, before any barrier
    const int gamma = T.grp_gamma[grp], pb = T.grp_pb[grp], cb0 = T.grp_cb[grp];
    if (tid < kTcPairs) {
        sm.rcp[tid] = tid < np ? T.pair_rcp[p0 + tid] : -1;
        sm.cb[tid] = tid < np ? T.pair_cb[p0 + tid] : -1;
    }
    if (tid < 16) sm.present[tid] = 0;
    // node geometry relative to the child (the same for every pair of the group)
    const float o0 = (C.ijk[3 * cb0] + 0.5f) * C.scale - (Pl.ijk[3 * pb] + 0.5f) * Pl.scale;
    const float o1 = (C.ijk[3 * cb0 + 1] + 0.5f) * C.scale - (Pl.ijk[3 * pb + 1] + 0.5f) * Pl.scale;
    const float o2 = (C.ijk[3 * cb0 + 2] + 0.5f) * C.scale - (Pl.ijk[3 * pb + 2] + 0.5f) * Pl.scale;
    for (int n = tid; n < P; n += blockDim.x) {
        float nv[3], rp, rcv, t3[3];
        ccone[n] = tc_child_cone<PS>(C, Pl, tb, gamma, n, o0, o1, o2, nv, rp, rcv, t3);
    }
    __syncthreads();
    if (warp == 0) {
        // distinct child cones, ascending (deterministic order)
        int nc = 0;
        for (int base = 0; base < P; base += 32) {
            const int c = ccone[base + lane];
            unsigned todo = 0xffffffffu;
            while (todo) {
                const int leader = __ffs(todo) - 1;
                const int cl = __shfl_sync(0xffffffffu, c, leader);
                const unsigned same = __ballot_sync(0xffffffffu, c == cl);
                todo &= ~same;
                bool seen = false;
                for (int j = 0; j < nc; j++) seen |= sm.cones[j] == cl;
                if (!seen && nc < 16) {
                    if (lane == 0) sm.cones[nc] = cl;
                    nc++;
                }
                __syncwarp();
            }
        }
        if (lane == 0) {
            for (int i = 1; i < nc; i++)
                for (int j = i; j > 0 && sm.cones[j - 1] > sm.cones[j]; j--) {
                    const int t = sm.cones[j];
                    sm.cones[j] = sm.cones[j - 1];
                    sm.cones[j - 1] = t;
                }
            sm.ncones = nc;
        }
        __syncwarp();
        // stable counting sort of the nodes by slot (slot nc collects nodes of no listed cone)
        int cnt = 0;  // lane j: nodes in slot j
        for (int base = 0; base < P; base += 32) {
            const int c = ccone[base + lane];
            int sl = 0;
            while (sl < nc && sm.cones[sl] != c) sl++;
            for (int j = 0; j <= nc; j++) {
                const unsigned m = __ballot_sync(0xffffffffu, sl == j);
                if (lane == j) cnt += __popc(m);
            }
        }
        int start = cnt;  // exclusive prefix over lanes 0..nc
        for (int o = 1; o < 32; o <<= 1) {
            const int v = __shfl_up_sync(0xffffffffu, start, o);
            if (lane >= o) start += v;
        }
        start -= cnt;
        for (int base = 0; base < P; base += 32) {
            const int c = ccone[base + lane];
            int sl = 0;
            while (sl < nc && sm.cones[sl] != c) sl++;
            for (int j = 0; j <= nc; j++) {
                const unsigned m = __ballot_sync(0xffffffffu, sl == j);
                const int sj = __shfl_sync(0xffffffffu, start, j);
                if (sl == j) {
                    const int pos = sj + __popc(m & ((1u << lane) - 1u)) - row0;
                    if (pos >= 0 && pos < kTcRows) sm.perm[pos] = (short)(base + lane);
                }
                if (lane == j) start += __popc(m);
            }
        }
    }
    __syncthreads();
    const int nc = sm.ncones;
    if (tid < kTcRows) {
        const int n = sm.perm[tid];
        float nv[3], rp, rcv, t3[3];
        const int cone = tc_child_cone<PS>(C, Pl, tb, gamma, n, o0, o1, o2, nv, rp, rcv, t3);
        int j = 0;
        while (j < nc && sm.cones[j] != cone) j++;
        sm.slot[tid] = (signed char)(j < nc ? j : -1);
        if (j < nc) sm.present[j] = 1;
        else atomicAdd(ca.missed, 1ULL);
        const float oo = o0 * o0 + o1 * o1 + o2 * o2, no = nv[0] * o0 + nv[1] * o1 + nv[2] * o2;
        float t = ca.kappa_hi * ((oo - 2.f * no) / (rcv + rp));
        t -= rintf(t);
        float sn, cs;
        cis_cycles(t, sn, cs);
        const float g1 = rp / rcv;
        sm.rr[tid] = cs * g1;
        sm.ri[tid] = sn * g1;
        sm.g1[tid] = g1;
        sm.ir[tid] = 1.f / (rcv * ca.HDf);
        lagrange<PS, float>(t3[0], tb.fxs, tb.fcs, sm.Ls[tid]);
        lagrange<8, float>(t3[1], tb.fxa, tb.fca, sm.Lt[tid]);
        lagrange<8, float>(t3[2], tb.fxa, tb.fca, sm.Lp[tid]);
    }
    for (int idx = tid; idx < nc * kTcPairs; idx += blockDim.x) {
        const int j = idx / kTcPairs, q = idx % kTcPairs;
        const int cb = sm.cb[q];
        int crc = -1;
        if (cb >= 0) {
            crc = C.cone_map[(long long)cb * C.ncone + sm.cones[j]];
            if (crc < 0) atomicAdd(ca.missed, 1ULL);
        }
        sm.crc[j][q] = crc;
    }
    __syncthreads();
    if (tid == 0) {
        int m = 0;
        for (int j = 0; j < nc; j++)
            if (sm.present[j]) sm.jlist[m++] = j;
        sm.njp = m;
    }
    __syncthreads();
    const bool csplit = C.split != 0, psplit = Pl.split != 0;
    const int npass = (csplit && psplit) ? 2 : 1;
    const float *FC = (const float *)C.F;
    float2 *FP = (float2 *)Pl.F;
    const int r0 = warp * 16 + g, r1 = r0 + 8;  // block-local rows of this lane
    constexpr int NKC = P / 64;                  // K-chunks of 64 child nodes
    constexpr int NIT = kTcPairs * 16 / 128;     // staging items per thread
    const int njp = sm.njp;
    for (int q = 0; q < ca.nrhs; q++) {
        for (int pass = 0; pass < npass; pass++) {
            const int cf_lo = (csplit && psplit) ? pass : 0, cf_hi = (csplit && psplit) ? pass : (csplit ? 1 : 0);
            const int fp = (csplit && psplit) ? pass : 0;
            const bool use_g1 = csplit && psplit && pass == 0;
            const int ncf = cf_hi - cf_lo + 1;
            const int nsteps = njp * ncf * NKC;  // flattened (cone slot, factor, K-chunk) steps
            float d[NT][4];
#pragma unroll
            for (int nt = 0; nt < NT; nt++) d[nt][0] = d[nt][1] = d[nt][2] = d[nt][3] = 0.f;
            float4 pre[NIT][2];  // next step's child values, fetched while the current step computes
            auto fetch = [&](int st) {
                const int kc = (st % NKC) * 64, t = st / NKC;
                const int cf = cf_lo + t % ncf, j = sm.jlist[t / ncf];
#pragma unroll
                for (int i = 0; i < NIT; i++) {
                    const int it = tid + 128 * i;
                    const int pr = it >> 4, k4 = (it & 15) * 4;
                    const int crc = sm.crc[j][pr];
                    pre[i][0] = pre[i][1] = make_float4(0.f, 0.f, 0.f, 0.f);
                    if (crc >= 0) {
                        const float4 *src = reinterpret_cast<const float4 *>(
                            FC + 2 * ((((long long)q * C.nrc + crc) * C.nfac + cf) * ca.Pstride + kc + k4));
                        pre[i][0] = __ldg(src);
                        pre[i][1] = __ldg(src + 1);
                    }
                }
            };
            if (nsteps > 0) fetch(0);
            for (int st = 0; st < nsteps; st++) {
                const int kc = (st % NKC) * 64, t = st / NKC;
                const int cf = cf_lo + t % ncf, j = sm.jlist[t / ncf];
                __syncthreads();  // the previous step's fragment reads are done
#pragma unroll
                for (int i = 0; i < NIT; i++) {
                    // item = (pair, 4 consecutive nodes), nodes fastest: 8 threads store 128 contiguous bytes
                    const int it = tid + 128 * i;
                    const int pr = it >> 4, k4 = (it & 15) * 4;
                    uint4 hr, lr, hi_, li;
                    split_tf32(pre[i][0].x, hr.x, lr.x);
                    split_tf32(pre[i][0].z, hr.y, lr.y);
                    split_tf32(pre[i][1].x, hr.z, lr.z);
                    split_tf32(pre[i][1].z, hr.w, lr.w);
                    split_tf32(pre[i][0].y, hi_.x, li.x);
                    split_tf32(pre[i][0].w, hi_.y, li.y);
                    split_tf32(pre[i][1].y, hi_.z, li.z);
                    split_tf32(pre[i][1].w, hi_.w, li.w);
                    *reinterpret_cast<uint4 *>(&sm.bt[0][2 * pr][k4]) = hr;
                    *reinterpret_cast<uint4 *>(&sm.bt[1][2 * pr][k4]) = lr;
                    *reinterpret_cast<uint4 *>(&sm.bt[0][2 * pr + 1][k4]) = hi_;
                    *reinterpret_cast<uint4 *>(&sm.bt[1][2 * pr + 1][k4]) = li;
                }
                __syncthreads();
                if (st + 1 < nsteps) fetch(st + 1);
                const bool on0 = sm.slot[r0] == j, on1 = sm.slot[r1] == j;
                if (!__any_sync(0xffffffffu, on0 || on1)) continue;  // every lane votes: warp-uniform
                const float sc0 = (csplit && !psplit && cf == 0) ? sm.ir[r0] : 1.f;
                const float sc1 = (csplit && !psplit && cf == 0) ? sm.ir[r1] : 1.f;
                // a chunk of 64 nodes is one radial index a = kc / 64; node k = kc + 8 b + c
                const int a = kc >> 6;
                const float s0 = on0 ? sc0 * sm.Ls[r0][a] : 0.f, s1 = on1 ? sc1 * sm.Ls[r1][a] : 0.f;
                const float p00 = sm.Lp[r0][tig], p04 = sm.Lp[r0][tig + 4];
                const float p10 = sm.Lp[r1][tig], p14 = sm.Lp[r1][tig + 4];
#pragma unroll 2
                for (int kk = 0; kk < 64; kk += 8) {
                    const int b = kk >> 3;
                    const float w0 = s0 * sm.Lt[r0][b];
                    const float w1 = s1 * sm.Lt[r1][b];
                    unsigned ah[4], al[4];
                    split_tf32(w0 * p00, ah[0], al[0]);
                    split_tf32(w1 * p10, ah[1], al[1]);
                    split_tf32(w0 * p04, ah[2], al[2]);
                    split_tf32(w1 * p14, ah[3], al[3]);
                    unsigned bh[NT][2], bl[NT][2];
#pragma unroll
                    for (int nt = 0; nt < NT; nt++) {
                        // lane supplies the row address of tile (lane / 8): hi k0-3, hi k4-7, lo k0-3, lo k4-7
                        const int tl = lane >> 3;
                        const unsigned *row = &sm.bt[tl >> 1][8 * nt + (lane & 7)][kk + 4 * (tl & 1)];
                        ldmatrix_x4(row, bh[nt][0], bh[nt][1], bl[nt][0], bl[nt][1]);
                    }
                    // the three split terms as three sweeps over the n-tiles: dependent MMAs are NT apart
#pragma unroll
                    for (int nt = 0; nt < NT; nt++) mma_tf32(d[nt], ah, bh[nt]);
#pragma unroll
                    for (int nt = 0; nt < NT; nt++) mma_tf32(d[nt], ah, bl[nt]);
#pragma unroll
                    for (int nt = 0; nt < NT; nt++) mma_tf32(d[nt], al, bh[nt]);
                }
            }
            // epilogue: rows r0, r1; this lane holds pair 4 nt + tig (re, im)
            // the pairs of a tile have distinct parent cones: all loads before any store
            long long oo[NT][2];
            float2 vv[NT][2];
#pragma unroll
            for (int nt = 0; nt < NT; nt++) {
                const int rcp = sm.rcp[nt * 4 + tig];
                const long long base = (((long long)q * Pl.nrc + rcp) * Pl.nfac + fp) * ca.Pstride;
#pragma unroll
                for (int h = 0; h < 2; h++) {
                    oo[nt][h] = rcp < 0 ? -1 : base + sm.perm[h ? r1 : r0];
                    vv[nt][h] = rcp < 0 ? make_float2(0.f, 0.f) : FP[oo[nt][h]];
                }
            }
#pragma unroll
            for (int nt = 0; nt < NT; nt++) {
#pragma unroll
                for (int h = 0; h < 2; h++) {
                    if (oo[nt][h] < 0) continue;
                    const int r = h ? r1 : r0;
                    const float dr = d[nt][2 * h], di = d[nt][2 * h + 1];
                    float rr = sm.rr[r], ri = sm.ri[r];
                    if (use_g1) {
                        rr *= sm.g1[r];
                        ri *= sm.g1[r];
                    }
                    vv[nt][h].x += rr * dr - ri * di;
                    vv[nt][h].y += rr * di + ri * dr;
                    FP[oo[nt][h]] = vv[nt][h];
                }
            }
        }
    }
}

// ============================================================================
// Tensor-core propagation on the 5th-generation tensor cores (tcgen05, TMEM).
// The interpolation from a child cone is a tensor product; its two angular
// contractions form one GEMM with K = 64 (node index (b, c) within a radial
// index a):
//     D[node, (a, pair, re/im)] = sum_{b,c} Lt[node][b] Lp[node][c] F_pair[a, b, c]
// with A[node][(b, c)] = Lt[b] Lp[c] the same for every pair, radial index and
// child cone (kept in tensor memory as TF32 hi / lo), and the radial factor
// Ls[node][a] applied when D is read back.
// A block owns 128 parent nodes (TMEM lanes) in the plan's child-cone order and
// one half of a tile (up to 32 of its 64 pairs; two blocks per tile), so that two
// blocks share an SM and each one's start-up, node geometry and epilogue overlap
// the other's MMAs.  Each step (child cone, factor, radial index a) stages B (32
// pairs x re/im = 64 columns, K = 64) in shared memory as TF32 hi / lo and runs 8
// k-slices x 3 split terms (hi*hi + hi*lo + lo*hi) of tcgen05.mma 128 x 64 x 8 (A
// from tensor memory, B from shared memory) into one of two 64-column TMEM
// buffers.  TMEM columns (256 per block): D0 0-63, D1 64-127, A hi 128-191,
// A lo 192-255.
// Warp-specialised: warps 0-3 stage operands and read D back (one thread per
// node), warp 4 only issues MMAs.  mbarriers hand the work over: full (per B
// stage: B staged), done and empty (per D buffer: MMAs complete via
// tcgen05.commit; D read back).  The workers stage step s + 2 as soon as the MMAs
// of step s are done (its B stage is then free) and before reading D(s) back, so
// the MMAs of s + 1 run during both.  Every wait is bounded; a timeout sets a
// block flag that ends the remaining waits early and is reported in the missed
// counter (high word).
// ============================================================================
constexpr int kT5Rows = 128;     // parent nodes per block (TMEM lanes)
constexpr int kT5Pairs = 32;     // pairs per block (half a tile)
constexpr int kT5Cols = 2 * kT5Pairs;  // TMEM columns of one step's D (two buffers); the MMA's N
constexpr int kT5Work = 128;     // staging / readback threads (warps 0-3)
constexpr int kT5Threads = kT5Work + 32;  // + the MMA-issuing warp
constexpr int kT5K = 64;         // contraction length (b, c)
constexpr int kT5TileBytes = kT5Cols * kT5K * 4;  // one 64 x 64 TF32 operand tile (B of one step)
constexpr uint32_t kT5ColA = 2 * kT5Cols;  // TMEM column of A hi (A lo at + 64)
constexpr uint32_t kT5TmemCols = 256;

__device__ __forceinline__ uint32_t smem_u32(const void *p) { return (uint32_t)__cvta_generic_to_shared(p); }

// byte offset of (row, k) in a K-major, non-swizzled tcgen05 operand tile of 128 rows x K = 64 TF32,
// stored as 8 contiguous k-slices of 8 values (4 KB each, one MMA's K): within a slice, 8-row x
// 16-byte core matrices, the two k-halves 128 bytes apart (LBO) and 8-row groups 256 bytes apart
// (SBO), so that the rows an MMA reads together fall in distinct banks
__device__ __forceinline__ int t5_off(int r, int k) {
    return (k >> 3) * 4096 + (r >> 3) * 256 + ((k >> 2) & 1) * 128 + (r & 7) * 16 + (k & 3) * 4;
}

// the same layout for the 64-row B tile of k_prop_t5 (k-slices of 2 KB)
__device__ __forceinline__ int t5h_off(int r, int k) {
    return (k >> 3) * 2048 + (r >> 3) * 256 + ((k >> 2) & 1) * 128 + (r & 7) * 16 + (k & 3) * 4;
}

__device__ __forceinline__ uint64_t t5_desc(uint32_t addr) {
    return (uint64_t)((addr >> 4) & 0x3FFF) | ((uint64_t)(128 >> 4) << 16) | ((uint64_t)(256 >> 4) << 32) |
           ((uint64_t)1 << 46);
}

// D (TMEM) += A (TMEM, lane = row, 8 consecutive columns) x B (shared memory descriptor)
__device__ __forceinline__ void t5_mma(uint32_t d_tmem, uint32_t a_tmem, uint64_t b, uint32_t idesc, uint32_t acc) {
    asm volatile(
        "{\n.reg .pred p;\nsetp.ne.b32 p, %4, 0;\n"
        "tcgen05.mma.cta_group::1.kind::tf32 [%0], [%1], %2, %3, p;\n}\n" ::"r"(d_tmem),
        "r"(a_tmem), "l"(b), "r"(idesc), "r"(acc)
        : "memory");
}

__device__ __forceinline__ void t5_st32(uint32_t taddr, const uint32_t *r) {
    asm volatile(
        "tcgen05.st.sync.aligned.32x32b.x32.b32 [%0], {%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,%16,"
        "%17,%18,%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31,%32};\n" ::"r"(taddr),
        "r"(r[0]), "r"(r[1]), "r"(r[2]), "r"(r[3]), "r"(r[4]), "r"(r[5]), "r"(r[6]), "r"(r[7]), "r"(r[8]),
        "r"(r[9]), "r"(r[10]), "r"(r[11]), "r"(r[12]), "r"(r[13]), "r"(r[14]), "r"(r[15]), "r"(r[16]),
        "r"(r[17]), "r"(r[18]), "r"(r[19]), "r"(r[20]), "r"(r[21]), "r"(r[22]), "r"(r[23]), "r"(r[24]),
        "r"(r[25]), "r"(r[26]), "r"(r[27]), "r"(r[28]), "r"(r[29]), "r"(r[30]), "r"(r[31])
        : "memory");
}

__device__ __forceinline__ void t5_arrive(uint32_t mbar) {
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];\n" ::"r"(mbar) : "memory");
}

// bounded wait for the completion of the phase with the given parity; gives up early once the
// block's abort flag is set
__device__ __forceinline__ bool t5_wait(uint32_t mbar, uint32_t parity, volatile int *abort_flag) {
    uint32_t done = 0;
    for (int it = 0; it < (1 << 20) && !done; it++) {
        asm volatile(
            "{\n.reg .pred p;\nmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\nselp.u32 %0, 1, 0, p;\n}\n"
            : "=r"(done)
            : "r"(mbar), "r"(parity)
            : "memory");
        if (!done && (it & 255) == 255 && *abort_flag) break;
    }
    if (!done) *abort_flag = 1;
    return done != 0;
}

__device__ __forceinline__ void t5_ld32(uint32_t taddr, uint32_t *r) {
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,"
        "%16,%17,%18,%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31}, [%32];\n"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
          "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15]),
          "=r"(r[16]), "=r"(r[17]), "=r"(r[18]), "=r"(r[19]), "=r"(r[20]), "=r"(r[21]), "=r"(r[22]), "=r"(r[23]),
          "=r"(r[24]), "=r"(r[25]), "=r"(r[26]), "=r"(r[27]), "=r"(r[28]), "=r"(r[29]), "=r"(r[30]), "=r"(r[31])
        : "r"(taddr));
}

__device__ __forceinline__ void t5_ld_wait() { asm volatile("tcgen05.wait::ld.sync.aligned;\n" ::: "memory"); }

// TMEM address of lane 32 * quadrant, column 0 (a warp reaches the lanes of quadrant warp % 4)
__device__ __forceinline__ uint32_t tmem_row_base(uint32_t tmem, int quadrant) {
    return tmem + ((uint32_t)(32 * quadrant) << 16);
}

struct T5Misc {
    short perm[kT5Rows];
    int crc[kT5Pairs];
    int rcp[kT5Pairs];
    unsigned long long full[2], done[2], empty[2];
    uint32_t tmem;
    int abort_;
};

// dynamic shared memory: B[stage][hi / lo], misc; padded so that at most two blocks fit on an SM
// (their 2 x 256 TMEM columns are then always free for tcgen05.alloc)
constexpr size_t kT5SmemUsed = 4 * (size_t)kT5TileBytes + sizeof(T5Misc) + 1024;
constexpr size_t kT5Smem = 80 * 1024;
static_assert(kT5SmemUsed <= kT5Smem, "k_prop_t5 shared memory");

template <int PS>
__global__ void __launch_bounds__(kT5Threads, 2) k_prop_t5(CommonArgs ca, LevelArgs C, LevelArgs Pl, ChebTab tb,
                                                           TcLevel T, int item0) {
    constexpr int P = PS * 64, NH = kT5Pairs;
    extern __shared__ unsigned char t5_dyn[];
    unsigned char *base = (unsigned char *)(((uintptr_t)t5_dyn + 1023) & ~(uintptr_t)1023);
    unsigned char *sB = base;  // buffer b: sB + (2 * b + hl) * kT5TileBytes
    T5Misc &sm = *reinterpret_cast<T5Misc *>(base + 4 * kT5TileBytes);
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const bool worker = warp < 4;
    const int qd = warp & 3;  // TMEM lane quadrant
    const int row = 32 * qd + lane;
    // item header (filled once per plan): nodes, group, child cone, pairs, child-centre offset; this
    // block takes the pairs [32 half, 32 half + 32) of the item's tile
    const long long it = item0 + (blockIdx.x >> 1);
    const int half = blockIdx.x & 1;
    const int4 h0 = T.item_hdr[3 * it], h1 = T.item_hdr[3 * it + 1], h2 = T.item_hdr[3 * it + 2];
    const int row0 = h0.x, nrows = h0.y, grp = h0.z, gamma = h0.w;
    const int ccone = h1.x, p0 = h1.y + kT5Pairs * half, np = h1.z - kT5Pairs * half;
    if (np <= 0) return;  // block-uniform: the tile has no second half
    const float o0 = __int_as_float(h2.x), o1 = __int_as_float(h2.y), o2 = __int_as_float(h2.z);
    if (tid < kT5Pairs) {
        sm.rcp[tid] = tid < np ? T.pair_rcp[p0 + tid] : -1;
        sm.crc[tid] = T.item_crc[kTcTile * it + kT5Pairs * half + tid];
    }
    if (tid == 0) {
        sm.abort_ = 0;
        for (int b = 0; b < 2; b++) {
            asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;\n" ::"r"(smem_u32(&sm.full[b])), "r"(kT5Work));
            asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;\n" ::"r"(smem_u32(&sm.empty[b])), "r"(kT5Work));
            asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;\n" ::"r"(smem_u32(&sm.done[b])));
        }
        asm volatile("fence.mbarrier_init.release.cluster;\n" ::: "memory");
    }
    if (warp == 4) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;\n" ::"r"(smem_u32(&sm.tmem)),
                     "r"(kT5TmemCols));
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;\n");
    }
    // the item's nodes (one child cone) in the plan's node order (k_tc_order)
    if (tid < kT5Rows) sm.perm[tid] = tid < nrows ? T.grp_perm[(long long)grp * P + row0 + tid] : (short)-1;
    asm volatile("tcgen05.fence::before_thread_sync;\n" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory");
    const uint32_t tmem = sm.tmem;
    const bool csplit = C.split != 0, psplit = Pl.split != 0;
    const float *FC = (const float *)C.F;
    // staging item: pair = 8 warp + (lane & 7), nodes [16 qn, 16 qn + 16) of the step's radial index with
    // qn = lane >> 3.  16-byte shared stores are serviced 8 lanes at a time: lanes 0-3 and 4-7 of each
    // group of 8 store the re / im rows in opposite order, so the 8 lanes cover all 8 bank groups
    const int s_pair = 8 * (warp & 3) + (lane & 7), s_qn = lane >> 3;
    // child values of step st (factor cf_lo + st / PS, radial index st % PS) of right-hand side q
    auto fetch_to = [&](int q, int cf_lo, int st, float4 *dst) {
        const int a = st % PS, cf = cf_lo + st / PS;
        const int crc = sm.crc[s_pair];
#pragma unroll
        for (int e = 0; e < 8; e++) dst[e] = make_float4(0.f, 0.f, 0.f, 0.f);
        if (crc >= 0) {
            const float4 *src = reinterpret_cast<const float4 *>(
                FC + 2 * ((((long long)q * C.nrc + crc) * C.nfac + cf) * ca.Pstride + a * 64 + 16 * s_qn));
#pragma unroll
            for (int e = 0; e < 8; e++) dst[e] = __ldg(src + e);
        }
    };
    // the first pipeline's first step is in flight while the node geometry is computed
    float4 pre[8];
    if (worker) fetch_to(0, 0, 0, pre);  // right-hand side 0, pass 0 (factor 0), step 0
    // this thread's node: geometry, cone slot, Lagrange factors
    const int node = worker ? sm.perm[row] : -1;
    int slot = -1;
    float Ls[PS], rr = 0.f, ri = 0.f, g1 = 0.f, irs = 0.f;
#pragma unroll
    for (int e = 0; e < PS; e++) Ls[e] = 0.f;
    if (worker) {
        float Lt[8], Lp[8];
#pragma unroll
        for (int e = 0; e < 8; e++) Lp[e] = Lt[e] = 0.f;
        if (node >= 0) {
            float nv[3], rp, rcv, t3[3];
            const int cone = tc_child_cone<PS>(C, Pl, tb, gamma, node, o0, o1, o2, nv, rp, rcv, t3);
            if (cone == ccone) slot = 0;
            else if (half == 0) atomicAdd(ca.missed, 1ULL);  // the plan's order puts every node in its cone
            const float oo = o0 * o0 + o1 * o1 + o2 * o2, no = nv[0] * o0 + nv[1] * o1 + nv[2] * o2;
            float t = ca.kappa_hi * ((oo - 2.f * no) / (rcv + rp));
            t -= rintf(t);
            float sn, cs;
            cis_cycles(t, sn, cs);
            g1 = rp / rcv;
            rr = cs * g1;
            ri = sn * g1;
            irs = 1.f / (rcv * ca.HDf);
            lagrange<PS, float>(t3[0], tb.fxs, tb.fcs, Ls);
            lagrange<8, float>(t3[1], tb.fxa, tb.fca, Lt);
            lagrange<8, float>(t3[2], tb.fxa, tb.fca, Lp);
        }
        // A[row][(b, c)] = Lt[b] Lp[c] into TMEM lane `row`, b in [0, 4) then [4, 8)
        const uint32_t lane_base = tmem_row_base(sm.tmem, qd);
#pragma unroll
        for (int hb = 0; hb < 2; hb++) {
            uint32_t ah[32], al[32];
#pragma unroll
            for (int bb = 0; bb < 4; bb++)
#pragma unroll
                for (int c = 0; c < 8; c++) split_tf32(Lt[4 * hb + bb] * Lp[c], ah[8 * bb + c], al[8 * bb + c]);
            t5_st32(lane_base + kT5ColA + 32u * hb, ah);
            t5_st32(lane_base + kT5ColA + 64u + 32u * hb, al);
        }
        asm volatile("tcgen05.wait::st.sync.aligned;\n" ::: "memory");
    }
    if (tid < kT5Pairs && tid < np && sm.crc[tid] < 0) atomicAdd(ca.missed, 1ULL);
    asm volatile("tcgen05.fence::before_thread_sync;\n" ::: "memory");  // A in TMEM, for the MMAs
    __syncthreads();
    const int npass = (csplit && psplit) ? 2 : 1;
    float2 *FP = (float2 *)Pl.F;
    volatile int *abort_flag = &sm.abort_;
    const int first_ri = (lane >> 2) & 1;
    const uint32_t idesc_base = (1u << 4) | (2u << 7) | (2u << 10) | ((uint32_t)(kT5Rows >> 4) << 24);
    const uint32_t aH = tmem + kT5ColA, aL = tmem + kT5ColA + 64u;
    const uint32_t my_taddr = tmem + ((uint32_t)(32 * qd) << 16);  // this node's row, the block's 32 pairs
    // global step index G: B stage and D buffer G & 1 (use G >> 1); a barrier's phase parity is its
    // use count & 1
    int G = 0;
    for (int q = 0; q < ca.nrhs; q++) {
        for (int pass = 0; pass < npass; pass++) {
            const int cf_lo = (csplit && psplit) ? pass : 0, cf_hi = (csplit && psplit) ? pass : (csplit ? 1 : 0);
            const int fp = (csplit && psplit) ? pass : 0;
            const bool use_g1 = csplit && psplit && pass == 0;
            const int ncf = cf_hi - cf_lo + 1;
            const int nsteps = ncf * PS;  // (factor, radial index)
            float E[NH][2];
#pragma unroll
            for (int pr = 0; pr < NH; pr++) E[pr][0] = E[pr][1] = 0.f;
            if (worker) {
                auto fetch = [&](int st) { fetch_to(q, cf_lo, st, pre); };
                auto stage = [&](int gs) {  // into buffer gs & 1, then signal full
                    unsigned char *bh = sB + (2 * (gs & 1)) * kT5TileBytes, *bl = bh + kT5TileBytes;
                    const int nre = s_pair * 2;
#pragma unroll
                    for (int o = 0; o < 2; o++) {
                        const bool im = (o ^ first_ri) != 0;
                        const int n = nre + (im ? 1 : 0);
#pragma unroll
                        for (int kq = 0; kq < 4; kq++) {
                            // nodes 16 qn + 4 kq .. + 3: pre[2 kq] = (n0, n1), pre[2 kq + 1] = (n2, n3)
                            const float4 u0 = pre[2 * kq], u1 = pre[2 * kq + 1];
                            uint4 h, l;
                            split_tf32(im ? u0.y : u0.x, h.x, l.x);
                            split_tf32(im ? u0.w : u0.z, h.y, l.y);
                            split_tf32(im ? u1.y : u1.x, h.z, l.z);
                            split_tf32(im ? u1.w : u1.z, h.w, l.w);
                            const int k = 16 * s_qn + 4 * kq;
                            *reinterpret_cast<uint4 *>(bh + t5h_off(n, k)) = h;
                            *reinterpret_cast<uint4 *>(bl + t5h_off(n, k)) = l;
                        }
                    }
                    asm volatile("fence.proxy.async.shared::cta;\n" ::: "memory");
                    t5_arrive(smem_u32(&sm.full[gs & 1]));
                };
                // prologue: the first two steps' loads in flight together (step 0 of the block's
                // first pipeline was issued before the node geometry)
                float4 pre2[8];
                if ((q > 0 || pass > 0) && nsteps > 0) fetch(0);
                if (nsteps > 1) fetch_to(q, cf_lo, 1, pre2);
                if (nsteps > 0) stage(G);
                if (nsteps > 1) {
#pragma unroll
                    for (int e = 0; e < 8; e++) pre[e] = pre2[e];
                    stage(G + 1);
                }
                if (nsteps > 2) fetch(2);
                for (int st = 0; st < nsteps; st++) {
                    const int gs = G + st, dsel = gs & 1;
                    const int a = st % PS, cf = cf_lo + st / PS;
                    const bool ok = t5_wait(smem_u32(&sm.done[dsel]), (gs >> 1) & 1, abort_flag);
                    asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory");
                    if (st + 2 < nsteps) {  // B stage gs & 1 was consumed by the MMAs just waited for
                        stage(gs + 2);
                        if (st + 3 < nsteps) fetch(st + 3);
                    }
                    // D row of this node: columns 2 i + re/im for the block's pairs i
                    const float sc = (csplit && !psplit && cf == 0) ? irs : 1.f;
                    const float w = (slot == 0 && ok) ? sc * pick<PS>(Ls, a) : 0.f;
                    const uint32_t dcol = my_taddr + (uint32_t)(dsel * kT5Cols);
                    uint32_t v0[32], v1[32];
                    t5_ld32(dcol, v0);
                    t5_ld32(dcol + 32u, v1);
                    t5_ld_wait();
                    asm volatile("tcgen05.fence::before_thread_sync;\n" ::: "memory");
                    t5_arrive(smem_u32(&sm.empty[dsel]));
#pragma unroll
                    for (int i = 0; i < 16; i++) {
                        E[i][0] = fmaf(w, __uint_as_float(v0[2 * i]), E[i][0]);
                        E[i][1] = fmaf(w, __uint_as_float(v0[2 * i + 1]), E[i][1]);
                        E[16 + i][0] = fmaf(w, __uint_as_float(v1[2 * i]), E[16 + i][0]);
                        E[16 + i][1] = fmaf(w, __uint_as_float(v1[2 * i + 1]), E[16 + i][1]);
                    }
                }
            } else if (lane == 0) {
                // MMA issuer
                for (int st = 0; st < nsteps; st++) {
                    const int gs = G + st, sel = gs & 1;
                    t5_wait(smem_u32(&sm.full[sel]), (gs >> 1) & 1, abort_flag);
                    if (gs >= 2) t5_wait(smem_u32(&sm.empty[sel]), ((gs >> 1) - 1) & 1, abort_flag);
                    asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory");
                    const uint32_t idesc = idesc_base | ((uint32_t)(kT5Cols >> 3) << 17);
                    const uint32_t d = tmem + (uint32_t)(sel * kT5Cols);
                    const uint32_t bH = smem_u32(sB + (2 * sel) * kT5TileBytes), bL = bH + kT5TileBytes;
                    if (!*abort_flag) {
#pragma unroll 1
                        for (int kk = 0; kk < 8; kk++) {
                            const uint32_t ko = 2048u * kk, ka = 8u * kk;
                            t5_mma(d, aH + ka, t5_desc(bH + ko), idesc, kk > 0 ? 1u : 0u);
                            t5_mma(d, aH + ka, t5_desc(bL + ko), idesc, 1u);
                            t5_mma(d, aL + ka, t5_desc(bH + ko), idesc, 1u);
                        }
                        asm volatile(
                            "tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];\n" ::"r"(
                                smem_u32(&sm.done[sel]))
                            : "memory");
                    }
                }
            }
            G += nsteps;
            __syncwarp();
            __syncthreads();
            // epilogue: times the centred-factor ratio, added into the parent cone values
            if (worker && slot >= 0) {
                float prr = rr, pri = ri;
                if (use_g1) {
                    prr *= g1;
                    pri *= g1;
                }
                // the pairs of a tile have distinct parent cones (one child per octant), so every
                // parent value has one writer in this launch: reduction stores (no read round trip)
#pragma unroll
                for (int i = 0; i < NH; i++) {
                    const int rcp = sm.rcp[i];
                    if (rcp < 0) continue;
                    const long long o = (((long long)q * Pl.nrc + rcp) * Pl.nfac + fp) * ca.Pstride + node;
                    atomicAdd(FP + o, make_float2(prr * E[i][0] - pri * E[i][1], prr * E[i][1] + pri * E[i][0]));
                }
            }
        }
    }
    asm volatile("tcgen05.fence::before_thread_sync;\n" ::: "memory");
    __syncthreads();
    if (tid == 0 && sm.abort_) atomicAdd(ca.missed, 1ULL << 32);
    if (warp == 4) {
        asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory");
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;\n" ::"r"(tmem), "r"(kT5TmemCols));
    }
}

// K3 (mixed), cone-stationary, on the grouping of the tensor-core tables (Pang = 8): within a
// group (child octant, parent cone id) the parent nodes are ordered by the child cone they fall
// in, and every (parent cone, child box) pair of a tile maps the same nodes to the same child
// cone id.  One warp per item (<= 64 nodes of one child cone, two per lane, and one tile of <= 64
// pairs): the nodes' geometry and basis weights are computed once, then for every pair the warp
// stages that pair's child cone (double-buffered cp.async) and interpolates it for its nodes with
// broadcast shared reads, times the centred-factor ratio, adding into the parent cone values.
// The caller zeroes F_{d-1} and launches one octant at a time, so each parent value has one
// writer per launch and the result is deterministic.
template <int PS, int PA>
struct PcNode {
    unsigned long long lt2[PA], lp2[PA];
    float Ls[PS];
    float rr, ri, g1, irs;  // ratio e^{ik(r_c - r_p)} r_p / r_c, r_p / r_c, 1 / r_c (absolute)
    int node;               // parent node index, -1 for an idle slot
};

template <int PS>
__device__ __forceinline__ void pc_node(const CommonArgs &ca, const LevelArgs &C, const LevelArgs &Pl,
                                        const ChebTab &tb, int gamma, int node, float o0, float o1, float o2,
                                        PcNode<PS, 8> &g) {
    g.node = node;
    float nv[3], rp, rcv, t3[3];
    tc_child_cone<PS>(C, Pl, tb, gamma, node >= 0 ? node : 0, o0, o1, o2, nv, rp, rcv, t3);
    const float oo = o0 * o0 + o1 * o1 + o2 * o2, no = nv[0] * o0 + nv[1] * o1 + nv[2] * o2;
    float t = ca.kappa_hi * ((oo - 2.f * no) / (rcv + rp));
    t -= rintf(t);
    float sn, cs;
    cis_cycles(t, sn, cs);
    g.g1 = rp / rcv;
    g.rr = cs * g.g1;
    g.ri = sn * g.g1;
    g.irs = 1.f / (rcv * ca.HDf);
    float Lt[8], Lp[8];
    lagrange<PS, float>(t3[0], tb.fxs, tb.fcs, g.Ls);
    lagrange<8, float>(t3[1], tb.fxa, tb.fca, Lt);
    lagrange<8, float>(t3[2], tb.fxa, tb.fca, Lp);
#pragma unroll
    for (int k = 0; k < 8; k++) {
        g.lt2[k] = f2pack(Lt[k], Lt[k]);
        g.lp2[k] = f2pack(Lp[k], Lp[k]);
    }
}

// add one parent node's share from one child (interpolated factor values v, and w for a split
// child) into the parent cone values at FP[base + fac * pstride + node]: with both levels split,
// each factor re-centred with its own power of r (ratio g1 for W2, ratio for W13); a split child
// into a combined parent through the child's field (W2 / r_c + W13); otherwise the ratio
template <bool CSPLIT, bool PSPLIT, typename N>
__device__ __forceinline__ void pc_store(float2 *FP, long long base, int pstride, const N &g,
                                         unsigned long long v, unsigned long long w) {
    if (g.node < 0) return;
    float vr, vi, wr, wi;
    f2unpack(v, vr, vi);
    f2unpack(w, wr, wi);
    if (CSPLIT && PSPLIT) {
        const float r2r = g.rr * g.g1, r2i = g.ri * g.g1;
        atomicAdd(FP + base + g.node, make_float2(vr * r2r - vi * r2i, vr * r2i + vi * r2r));
        atomicAdd(FP + base + pstride + g.node, make_float2(wr * g.rr - wi * g.ri, wr * g.ri + wi * g.rr));
    } else {
        if (CSPLIT) {
            vr = vr * g.irs + wr;
            vi = vi * g.irs + wi;
        }
        atomicAdd(FP + base + g.node, make_float2(vr * g.rr - vi * g.ri, vr * g.ri + vi * g.rr));
    }
}

template <int PS, bool CSPLIT, bool PSPLIT>
__global__ void __launch_bounds__(kCsWarps * 32) k_prop_cs(CommonArgs ca, LevelArgs C, LevelArgs Pl, ChebTab tb,
                                                           TcLevel T, int item0, int nitem) {
    constexpr int P = PS * 64, PST = P, NF = CSPLIT ? 2 : 1;
    constexpr int NV4 = NF * PST / 2;  // float4 of one child cone's values (all factors, contiguous)
    __shared__ __align__(16) float2 sF[kCsWarps][2][NF * PST];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int it = blockIdx.x * kCsWarps + warp;
    if (it >= nitem) return;  // warp-uniform: no block-wide barrier below
    const int4 w = T.cs_items[item0 + it];
    const int tile = w.x, row0 = w.y, rows = w.z, slot = w.w;
    const int g = T.tile_group[tile];
    const int gamma = T.grp_gamma[g], pb = T.grp_pb[g], cb0 = T.grp_cb[g];
    const int cc = T.grp_cones[16 * g + slot];
    const int ts = T.tile_start[tile], np = T.tile_count[tile];
    // child-centre offset from the parent centre (leaf units; exact: integers times powers of two)
    const float o0 = (C.ijk[3 * cb0] + 0.5f) * C.scale - (Pl.ijk[3 * pb] + 0.5f) * Pl.scale;
    const float o1 = (C.ijk[3 * cb0 + 1] + 0.5f) * C.scale - (Pl.ijk[3 * pb + 1] + 0.5f) * Pl.scale;
    const float o2 = (C.ijk[3 * cb0 + 2] + 0.5f) * C.scale - (Pl.ijk[3 * pb + 2] + 0.5f) * Pl.scale;
    // every lane looks up the child cone storage index of pairs lane and lane + 32
    int crc_a = -1, crc_b = -1, rcp_a = -1, rcp_b = -1;
    if (lane < np) {
        crc_a = C.cone_map[(long long)T.pair_cb[ts + lane] * C.ncone + cc];
        rcp_a = T.pair_rcp[ts + lane];
    }
    if (lane + 32 < np) {
        crc_b = C.cone_map[(long long)T.pair_cb[ts + lane + 32] * C.ncone + cc];
        rcp_b = T.pair_rcp[ts + lane + 32];
    }
    PcNode<PS, 8> n0, n1;
    pc_node<PS>(ca, C, Pl, tb, gamma, lane < rows ? (int)T.grp_perm[(long long)g * P + row0 + lane] : -1, o0, o1, o2,
                n0);
    pc_node<PS>(ca, C, Pl, tb, gamma, lane + 32 < rows ? (int)T.grp_perm[(long long)g * P + row0 + lane + 32] : -1,
                o0, o1, o2, n1);
    const float2 *FC = (const float2 *)C.F;
    float2 *FP = (float2 *)Pl.F;
    for (int q = 0; q < ca.nrhs; q++) {
        auto crc_of = [&](int pr) { return __shfl_sync(0xffffffffu, pr < 32 ? crc_a : crc_b, pr & 31); };
        auto rcp_of = [&](int pr) { return __shfl_sync(0xffffffffu, pr < 32 ? rcp_a : rcp_b, pr & 31); };
        auto stage = [&](int pr, int bsel) {
            const int crc = crc_of(pr);
            if (crc < 0) return;
            const float4 *src = reinterpret_cast<const float4 *>(FC + ((long long)q * C.nrc + crc) * NF * PST);
            float4 *dst = reinterpret_cast<float4 *>(sF[warp][bsel]);
            for (int v = lane; v < NV4; v += 32) cp_async16(dst + v, src + v);
        };
        __syncwarp();  // the previous right-hand side's readers are done
        stage(0, 0);
        asm volatile("cp.async.commit_group;\n" ::: "memory");
        for (int pr = 0; pr < np; pr++) {
            const int bsel = pr & 1;
            if (pr + 1 < np) stage(pr + 1, bsel ^ 1);  // the buffer last read at pair pr - 1
            asm volatile("cp.async.commit_group;\n" ::: "memory");
            asm volatile("cp.async.wait_group 1;\n" ::: "memory");  // pair pr's copy has landed
            __syncwarp();
            const int crc = crc_of(pr), rcp = rcp_of(pr);
            if (crc < 0) atomicAdd(ca.missed, 1ULL);  // warp-uniform
            else {
                const float2 *buf = sF[warp][bsel];
                unsigned long long v0, v1, w0 = 0ull, w1 = 0ull;
                cs_interp2<PS, 8>(buf, n0, n1, v0, v1);
                if constexpr (CSPLIT) cs_interp2<PS, 8>(buf + PST, n0, n1, w0, w1);
                pc_store<CSPLIT, PSPLIT>(FP, ((long long)q * Pl.nrc + rcp) * Pl.nfac * ca.Pstride, ca.Pstride, n0, v0, w0);
                pc_store<CSPLIT, PSPLIT>(FP, ((long long)q * Pl.nrc + rcp) * Pl.nfac * ca.Pstride, ca.Pstride, n1, v1, w1);
            }
            __syncwarp();  // buffer bsel may be overwritten by the stage of pair pr + 2
        }
        cp_async_wait_all();
    }
}

// ---------------------------------------------------------------------------
// K3 (mixed, Pang = 8) on tcgen05, c-axis contraction.  For one work item (<= 128 parent nodes
// that fall in one child cone, TMEM lane = node) and one tile of (parent cone, child box) pairs
// of the same group key, the interpolant of every pair's child cone at the nodes is
//     sum_a Ls[a] sum_b Lt[b] D[node, (a, b)],   D[node, (a, b, re/im)] = sum_c Lp[node][c] F_pair[a, b, c]
// The c-contraction runs on the tensor cores per pair: M = 128 nodes, N = NF x PS x 16 ((factor,
// a, b, re/im)), K = 8, three TF32 split terms (hi hi + hi lo + lo hi) with A = Lp (hi / lo) in tensor
// memory, B = the pair's child cone values (hi / lo) in shared memory (K-major, no swizzle), and
// FP32 accumulators in tensor memory.  The threads (one per node) then do the b- and
// a-contractions (45 packed FMAs per factor), the centred-factor ratio and a reduction store into
// the parent values.  The readback of step p - 2 overlaps the MMAs of steps p - 1 and p (three D
// buffers and three B buffers; the child values are fetched into registers two steps ahead).  With
// one factor at orders (5, 8) two blocks fit per SM (256 TMEM columns each).  The caller zeroes
// F_{d-1} and launches one octant at a time: one writer per parent value per launch.
// Every wait is bounded; a timeout sets a block flag that skips the remaining MMAs and is
// reported through the missed counter (high word).
// ---------------------------------------------------------------------------
constexpr int kT6Threads = 128;

template <int PS, int NF>
struct T6Cfg {
    static constexpr int kNF = PS * 16;                    // (a, b, re/im) columns of one factor
    static constexpr int kN = NF * kNF;                    // MMA N (a multiple of 16, at most 192)
    static constexpr int kTileBytes = kN * 8 * 4;          // one B tile (kN rows x K = 8 TF32)
    static constexpr int kTileStride = (kTileBytes + 1023) & ~1023;
    // D and B buffers: three (readback two steps behind) when they and A fit in the 512 tensor-memory
    // columns of an SM, else two (readback one step behind)
    static constexpr int kBuf = 3 * kN + 16 <= 512 ? 3 : 2;
    static constexpr uint32_t kColA = kBuf * kN;           // A hi at kColA, A lo at kColA + 8
    static constexpr uint32_t kCols = kBuf * kN + 16 <= 256 ? 256 : 512;  // TMEM allocation
    static_assert(kBuf * kN + 16 <= (int)kCols && kCols <= 512, "tensor memory budget");
};

// 32 consecutive TMEM columns of this warp's 32 lanes, wait included (see t6_ld16)
__device__ __forceinline__ void t6_ld32w(uint32_t taddr, uint32_t *r) {
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,"
        "%16,%17,%18,%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31}, [%32];\n"
        "tcgen05.wait::ld.sync.aligned;\n"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
          "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15]),
          "=r"(r[16]), "=r"(r[17]), "=r"(r[18]), "=r"(r[19]), "=r"(r[20]), "=r"(r[21]), "=r"(r[22]), "=r"(r[23]),
          "=r"(r[24]), "=r"(r[25]), "=r"(r[26]), "=r"(r[27]), "=r"(r[28]), "=r"(r[29]), "=r"(r[30]), "=r"(r[31])
        : "r"(taddr));
}

// 16 consecutive TMEM columns of this warp's 32 lanes; the wait is in the same statement, so the
// outputs cannot be used before the load has completed
__device__ __forceinline__ void t6_ld16(uint32_t taddr, uint32_t *r) {
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];\n"
        "tcgen05.wait::ld.sync.aligned;\n"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]), "=r"(r[8]),
          "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
        : "r"(taddr));
}

struct T6Misc {
    unsigned long long done[3];
    uint32_t tmem;
    int abort_;
};

template <int PS, bool CSPLIT, bool PSPLIT>
__global__ void __launch_bounds__(kT6Threads) k_prop_t6(CommonArgs ca, LevelArgs C, LevelArgs Pl, ChebTab tb,
                                                       TcLevel T, int item0, int nitem) {
    constexpr int P = PS * 64, NF = CSPLIT ? 2 : 1;
    typedef T6Cfg<PS, NF> Cfg;
    __shared__ __align__(1024) unsigned char sB[Cfg::kBuf][2][Cfg::kTileStride];  // [buffer][hi / lo]
    __shared__ T6Misc sm;
    __shared__ int s_crc[kTcTile], s_rcp[kTcTile];
    const int tid = threadIdx.x, warp = tid >> 5;
    if (tid == 0) {
        sm.abort_ = 0;
        for (int b = 0; b < Cfg::kBuf; b++)
            asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;\n" ::"r"(smem_u32(&sm.done[b])));
        asm volatile("fence.mbarrier_init.release.cluster;\n" ::: "memory");
    }
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;\n" ::"r"(smem_u32(&sm.tmem)),
                     "r"(Cfg::kCols));
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;\n");
    }
    asm volatile("tcgen05.fence::before_thread_sync;\n" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory");
    const uint32_t tmem = sm.tmem;
    volatile int *abort_flag = &sm.abort_;
    const uint32_t lane_base = tmem + ((uint32_t)(32 * warp) << 16);
    // instruction descriptor: F32 accumulate, TF32 A and B, K-major, N / 8, M / 16
    const uint32_t idesc = (1u << 4) | (2u << 7) | (2u << 10) | ((uint32_t)(Cfg::kN >> 3) << 17) |
                           ((uint32_t)(128 >> 4) << 24);
    const float2 *FC = (const float2 *)C.F;
    float2 *FP = (float2 *)Pl.F;
    int G = 0;  // steps issued by this block so far: D / B buffer G % 3, mbarrier parity (G / 3) & 1
    for (int it = blockIdx.x; it < nitem; it += gridDim.x) {
        const long long item = item0 + it;
        const int4 h0 = T.item_hdr[3 * item], h1 = T.item_hdr[3 * item + 1], h2 = T.item_hdr[3 * item + 2];
        const int row0 = h0.x, nrows = h0.y, grp = h0.z, gamma = h0.w;
        const int ccone = h1.x, p0 = h1.y, np = h1.z;
        const float o0 = __int_as_float(h2.x), o1 = __int_as_float(h2.y), o2 = __int_as_float(h2.z);
        __syncthreads();  // the previous item's readers of s_crc / s_rcp are done
        if (tid < kTcTile) {
            s_crc[tid] = T.item_crc[kTcTile * item + tid];
            s_rcp[tid] = tid < np ? T.pair_rcp[p0 + tid] : -1;
            if (tid < np && s_crc[tid] < 0) atomicAdd(ca.missed, 1ULL);  // a child cone outside the relevant set
        }
        // this thread's node: geometry, basis weights, centred-factor ratio; A row = Lp (hi / lo)
        const int node = tid < nrows ? (int)T.grp_perm[(long long)grp * P + row0 + tid] : -1;
        float Ls[PS], rr = 0.f, ri = 0.f, g1 = 0.f, irs = 0.f;
        unsigned long long lt2[8];
        uint32_t ah[8], al[8];
        {
            float Lt[8], Lp[8];
#pragma unroll
            for (int e = 0; e < 8; e++) Lt[e] = Lp[e] = 0.f;
#pragma unroll
            for (int e = 0; e < PS; e++) Ls[e] = 0.f;
            if (node >= 0) {
                float nv[3], rp, rcv, t3[3];
                const int cone = tc_child_cone<PS>(C, Pl, tb, gamma, node, o0, o1, o2, nv, rp, rcv, t3);
                if (cone != ccone) atomicAdd(ca.missed, 1ULL);  // the plan's order puts every node in its cone
                const float oo = o0 * o0 + o1 * o1 + o2 * o2, no = nv[0] * o0 + nv[1] * o1 + nv[2] * o2;
                float t = ca.kappa_hi * ((oo - 2.f * no) / (rcv + rp));
                t -= rintf(t);
                float sn, cs;
                cis_cycles(t, sn, cs);
                g1 = rp / rcv;
                rr = cs * g1;
                ri = sn * g1;
                irs = 1.f / (rcv * ca.HDf);
                lagrange<PS, float>(t3[0], tb.fxs, tb.fcs, Ls);
                lagrange<8, float>(t3[1], tb.fxa, tb.fca, Lt);
                lagrange<8, float>(t3[2], tb.fxa, tb.fca, Lp);
            }
#pragma unroll
            for (int e = 0; e < 8; e++) {
                lt2[e] = f2pack(Lt[e], Lt[e]);
                split_tf32(Lp[e], ah[e], al[e]);
            }
        }
        asm volatile(
            "tcgen05.st.sync.aligned.32x32b.x8.b32 [%0], {%1,%2,%3,%4,%5,%6,%7,%8};\n" ::"r"(lane_base + Cfg::kColA),
            "r"(ah[0]), "r"(ah[1]), "r"(ah[2]), "r"(ah[3]), "r"(ah[4]), "r"(ah[5]), "r"(ah[6]), "r"(ah[7])
            : "memory");
        asm volatile(
            "tcgen05.st.sync.aligned.32x32b.x8.b32 [%0], {%1,%2,%3,%4,%5,%6,%7,%8};\n" ::"r"(lane_base + Cfg::kColA + 8u),
            "r"(al[0]), "r"(al[1]), "r"(al[2]), "r"(al[3]), "r"(al[4]), "r"(al[5]), "r"(al[6]), "r"(al[7])
            : "memory");
        asm volatile("tcgen05.wait::st.sync.aligned;\n" ::: "memory");
        __syncthreads();  // the item's pair tables are in shared memory
        const int nsteps = ca.nrhs * np;  // (right-hand side, pair)
        // B staging: unit u = (factor, a, b, half) holds 4 complex child values (one row half for the
        // re and the im row); each thread owns units tid + 128 r, fetched two steps ahead into registers
        constexpr int NU = NF * PS * 16, R = (NU + kT6Threads - 1) / kT6Threads;
        float4 pre[2][R][2];
        auto fetch = [&](int step, int slot) {
            const int q = step / np, pr = step % np;
            const int crc = s_crc[pr];
#pragma unroll
            for (int r = 0; r < R; r++) {
                const int u = tid + kT6Threads * r;
                pre[slot][r][0] = pre[slot][r][1] = make_float4(0.f, 0.f, 0.f, 0.f);
                if (u < NU && crc >= 0) {
                    const int half = u & 1, rab = u >> 1, f = rab / (PS * 8), ab = rab % (PS * 8);
                    const float4 *src = reinterpret_cast<const float4 *>(
                        FC + (((long long)q * C.nrc + crc) * C.nfac + f) * ca.Pstride + ab * 8 + 4 * half);
                    pre[slot][r][0] = __ldg(src);
                    pre[slot][r][1] = __ldg(src + 1);
                }
            }
        };
        if (nsteps > 0) fetch(0, 0);
        if (nsteps > 1) fetch(1, 1);
        // step st uses prefetch slot st & 1 (a compile-time index: the loop runs two steps per pass)
        auto step = [&](const int st, auto slot_c) {
            constexpr int slot = decltype(slot_c)::value;
            const int gs = G + st;
            const int bsel = gs % Cfg::kBuf;
            if (st < nsteps) {  // stage B of step st: rows (factor, a, b, re/im), K = c, hi / lo
                unsigned char *bh = sB[bsel][0], *bl = sB[bsel][1];
#pragma unroll
                for (int r = 0; r < R; r++) {
                    const int u = tid + kT6Threads * r;
                    if (u >= NU) continue;
                    const float4 v0 = pre[slot][r][0], v1 = pre[slot][r][1];
                    uint4 hr, lr, hi, li;
                    split_tf32(v0.x, hr.x, lr.x);
                    split_tf32(v0.z, hr.y, lr.y);
                    split_tf32(v1.x, hr.z, lr.z);
                    split_tf32(v1.z, hr.w, lr.w);
                    split_tf32(v0.y, hi.x, li.x);
                    split_tf32(v0.w, hi.y, li.y);
                    split_tf32(v1.y, hi.z, li.z);
                    split_tf32(v1.w, hi.w, li.w);
                    const int nre = 2 * (u >> 1), k = 4 * (u & 1);
                    *reinterpret_cast<uint4 *>(bh + t5_off(nre, k)) = hr;
                    *reinterpret_cast<uint4 *>(bl + t5_off(nre, k)) = lr;
                    *reinterpret_cast<uint4 *>(bh + t5_off(nre + 1, k)) = hi;
                    *reinterpret_cast<uint4 *>(bl + t5_off(nre + 1, k)) = li;
                }
                if (st + 2 < nsteps) fetch(st + 2, slot);  // in flight during this step and the next
                asm volatile("fence.proxy.async.shared::cta;\n" ::: "memory");
            }
            asm volatile("tcgen05.fence::before_thread_sync;\n" ::: "memory");
            __syncthreads();  // B staged; the readers of D buffer gs % kBuf (step st - kBuf) are done
            asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory");
            if (st < nsteps && tid == 0 && !*abort_flag) {
                const uint32_t d = tmem + (uint32_t)(bsel * Cfg::kN);
                const uint32_t bH = smem_u32(sB[bsel][0]), bL = smem_u32(sB[bsel][1]);
                const uint32_t aH = tmem + Cfg::kColA, aL = aH + 8u;
                t5_mma(d, aH, t5_desc(bH), idesc, 0u);
                t5_mma(d, aH, t5_desc(bL), idesc, 1u);
                t5_mma(d, aL, t5_desc(bH), idesc, 1u);
                asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];\n" ::"r"(
                                 smem_u32(&sm.done[bsel]))
                             : "memory");
            }
            constexpr int LAG = Cfg::kBuf - 1;  // steps between an MMA and its readback
            if (st >= LAG) {  // read back step st - LAG and add it into the parent values
                const int gp = gs - LAG, q = (st - LAG) / np, pr = (st - LAG) % np;
                const bool ok = t5_wait(smem_u32(&sm.done[gp % Cfg::kBuf]), (gp / Cfg::kBuf) & 1, abort_flag);
                asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory");
                const uint32_t dcol = lane_base + (uint32_t)((gp % Cfg::kBuf) * Cfg::kN);
                unsigned long long acc[NF];
#pragma unroll
                for (int f = 0; f < NF; f++) {
                    unsigned long long s = 0ull;
#pragma unroll
                    for (int a0 = 0; a0 < PS; a0 += 2) {  // columns 16 a .. 16 a + 15: (b, re/im) of radial index a
                        uint32_t v[32];
                        if (a0 + 1 < PS) t6_ld32w(dcol + (uint32_t)(f * Cfg::kNF + 16 * a0), v);
                        else t6_ld16(dcol + (uint32_t)(f * Cfg::kNF + 16 * a0), v);
#pragma unroll
                        for (int a = a0; a < a0 + 2 && a < PS; a++) {
                            const uint32_t *va = v + 16 * (a - a0);
                            unsigned long long sa = 0ull;
#pragma unroll
                            for (int b = 0; b < 8; b++)
                                f2fma(sa, lt2[b], f2pack(__uint_as_float(va[2 * b]), __uint_as_float(va[2 * b + 1])));
                            f2fma(s, f2pack(Ls[a], Ls[a]), sa);
                        }
                    }
                    acc[f] = ok ? s : 0ull;
                }
                const int rcp = s_rcp[pr];
                if (node >= 0 && rcp >= 0 && s_crc[pr] >= 0) {
                    const long long base = ((long long)q * Pl.nrc + rcp) * Pl.nfac * ca.Pstride;
                    float vr, vi, wr = 0.f, wi = 0.f;
                    f2unpack(acc[0], vr, vi);
                    if constexpr (CSPLIT) f2unpack(acc[NF - 1], wr, wi);
                    if (CSPLIT && PSPLIT) {
                        const float r2r = rr * g1, r2i = ri * g1;
                        atomicAdd(FP + base + node, make_float2(vr * r2r - vi * r2i, vr * r2i + vi * r2r));
                        atomicAdd(FP + base + ca.Pstride + node, make_float2(wr * rr - wi * ri, wr * ri + wi * rr));
                    } else {
                        if (CSPLIT) {
                            vr = vr * irs + wr;
                            vi = vi * irs + wi;
                        }
                        atomicAdd(FP + base + node, make_float2(vr * rr - vi * ri, vr * ri + vi * rr));
                    }
                }
            }
        };
        const int last = nsteps + Cfg::kBuf - 2;  // drain steps read back the last pairs
        for (int st = 0; st <= last; st += 2) {
            step(st, std::integral_constant<int, 0>{});
            if (st + 1 <= last) step(st + 1, std::integral_constant<int, 1>{});
        }
        G += nsteps;
    }
    if (tid == 0 && sm.abort_) atomicAdd(ca.missed, 1ULL << 32);
    asm volatile("tcgen05.fence::before_thread_sync;\n" ::: "memory");
    __syncthreads();
    if (warp == 0) {
        asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory");
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;\n" ::"r"(tmem), "r"(Cfg::kCols));
    }
}

// Once per plan: for every group key (child octant, parent cone), the child cone of each of the P
// parent nodes (FP32, the classification the propagation kernels use), the distinct cones in
// ascending order (at most 16; nodes of further cones go last and are counted as missed when
// propagated), and the nodes in stable order of their cone.  One warp per group.
template <int PS>
__global__ void __launch_bounds__(32) k_tc_order(LevelArgs C, LevelArgs Pl, ChebTab tb, TcLevel T) {
    constexpr int P = PS * 64;
    __shared__ int ccone[P];
    __shared__ int cones[16];
    const int g = blockIdx.x, lane = threadIdx.x;
    const int gamma = T.grp_gamma[g], pb = T.grp_pb[g], cb0 = T.grp_cb[g];
    const float o0 = (C.ijk[3 * cb0] + 0.5f) * C.scale - (Pl.ijk[3 * pb] + 0.5f) * Pl.scale;
    const float o1 = (C.ijk[3 * cb0 + 1] + 0.5f) * C.scale - (Pl.ijk[3 * pb + 1] + 0.5f) * Pl.scale;
    const float o2 = (C.ijk[3 * cb0 + 2] + 0.5f) * C.scale - (Pl.ijk[3 * pb + 2] + 0.5f) * Pl.scale;
    for (int n = lane; n < P; n += 32) {
        float nv[3], rp, rcv, t3[3];
        ccone[n] = tc_child_cone<PS>(C, Pl, tb, gamma, n, o0, o1, o2, nv, rp, rcv, t3);
    }
    __syncwarp();
    int nc = 0;
    for (int b0 = 0; b0 < P; b0 += 32) {
        const int c = ccone[b0 + lane];
        unsigned todo = 0xffffffffu;
        while (todo) {
            const int leader = __ffs(todo) - 1;
            const int cl = __shfl_sync(0xffffffffu, c, leader);
            const unsigned same = __ballot_sync(0xffffffffu, c == cl);
            todo &= ~same;
            bool seen = false;
            for (int j = 0; j < nc; j++) seen |= cones[j] == cl;
            if (!seen && nc < 16) {
                if (lane == 0) cones[nc] = cl;
                nc++;
            }
            __syncwarp();
        }
    }
    if (lane == 0) {
        for (int i = 1; i < nc; i++)
            for (int j = i; j > 0 && cones[j - 1] > cones[j]; j--) {
                const int t = cones[j];
                cones[j] = cones[j - 1];
                cones[j - 1] = t;
            }
    }
    __syncwarp();
    if (lane < 16) T.grp_cones[16 * g + lane] = lane < nc ? cones[lane] : -1;
    if (lane == 0) T.grp_nc[g] = nc;
    int cnt = 0;
    for (int b0 = 0; b0 < P; b0 += 32) {
        const int c = ccone[b0 + lane];
        int sl = 0;
        while (sl < nc && cones[sl] != c) sl++;
        for (int j = 0; j <= nc; j++) {
            const unsigned m = __ballot_sync(0xffffffffu, sl == j);
            if (lane == j) cnt += __popc(m);
        }
    }
    // lane j holds the nodes of slot j; slot nc (cones beyond the first 16) is empty unless nc = 16
    if (lane <= 16) T.grp_cnt[17 * g + lane] = cnt;
    int start = cnt;
    for (int o = 1; o < 32; o <<= 1) {
        const int v = __shfl_up_sync(0xffffffffu, start, o);
        if (lane >= o) start += v;
    }
    start -= cnt;
    for (int b0 = 0; b0 < P; b0 += 32) {
        const int c = ccone[b0 + lane];
        int sl = 0;
        while (sl < nc && cones[sl] != c) sl++;
        for (int j = 0; j <= nc; j++) {
            const unsigned m = __ballot_sync(0xffffffffu, sl == j);
            const int sj = __shfl_sync(0xffffffffu, start, j);
            if (sl == j) T.grp_perm[(long long)g * P + sj + __popc(m & ((1u << lane) - 1u))] = (short)(b0 + lane);
            if (lane == j) start += __popc(m);
        }
    }
}


}  // namespace

// ============================================================================
// launch sequence of one apply
// ============================================================================
static inline LevelArgs level_args(const Plan &p, int d, void *F) {
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

static inline CommonArgs common_args(const Plan &p, int nrhs) {
    CommonArgs c;
    c.N = (int)p.N; c.nrhs = nrhs; c.D = p.D; c.Pstride = p.Pstride;
    c.k = p.prm.k; c.HD = p.HD; c.L = p.L; c.tol = 1e-14 * p.L;
    coupling(p.prm, c.eta, c.etai);
    for (int a = 0; a < 3; a++) c.c0[a] = p.c0[a];
    c.kf = (float)p.prm.k; c.etaf = (float)c.eta; c.etaif = (float)c.etai; c.HDf = (float)p.HD;
    double kap = p.prm.k * p.HD / (2.0 * kPi);
    c.kappa_hi = (float)kap;
    c.kappa_lo = (float)(kap - (double)c.kappa_hi);
    c.leaf_of = p.d_leaf_of; c.nb_start = p.d_nb_start; c.nb_list = p.d_nb_list;
    c.x64 = p.d_x64; c.n64 = p.d_n64; c.w64 = p.d_w64;
    c.f32 = p.d_f32; c.n32 = p.d_n32; c.w32 = p.d_w32; c.pn32 = p.d_pn32;
    c.missed = p.d_missed;
    return c;
}

static inline ChebTab cheb_tab(const Plan &p) {
    ChebTab t;
    for (int j = 0; j < 12; j++) {
        t.xs[j] = j < p.Ps ? p.cs.x[j] : 0; t.cs[j] = j < p.Ps ? p.cs.c[j] : 0;
        t.xa[j] = j < p.Pang ? p.ca.x[j] : 0; t.ca[j] = j < p.Pang ? p.ca.c[j] : 0;
        t.fxs[j] = (float)t.xs[j]; t.fcs[j] = (float)t.cs[j]; t.fxa[j] = (float)t.xa[j]; t.fca[j] = (float)t.ca[j];
    }
    return t;
}

static inline unsigned nblk(long long n) { return (unsigned)((n + kBlock - 1) / kBlock); }

static inline int __float_as_int_host(float f) {
    int i;
    std::memcpy(&i, &f, sizeof i);
    return i;
}

template <int PS>
ifgf_status t5_prepare(Plan &p, cudaStream_t s) {
    cudaError_t e = cudaFuncSetAttribute(k_prop_t5<PS>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kT5Smem);
    if (e != cudaSuccess) {
        set_error("cudaFuncSetAttribute(k_prop_t5): %s", cudaGetErrorString(e));
        return IFGF_ECUDA;
    }
    const ChebTab tb = cheb_tab(p);
    for (int d = p.D; d >= 4; d--) {
        const TcLevel &T = p.tc[d];
        if (T.ngroups == 0 || !T.grp_perm) continue;
        k_tc_order<PS><<<T.ngroups, 32, 0, s>>>(level_args(p, d, nullptr), level_args(p, d - 1, nullptr), tb, T);
    }
    e = cudaStreamSynchronize(s);
    if (e == cudaSuccess) e = cudaGetLastError();
    if (e != cudaSuccess) {
        set_error("k_tc_order: %s", cudaGetErrorString(e));
        return IFGF_ECUDA;
    }
    // work items of the tcgen05 engine: each tile's nodes split by child cone into runs of <= 128
    for (int d = p.D; d >= 4; d--) {
        TcLevel &T = p.tc[d];
        if (T.ngroups == 0 || !T.grp_perm) continue;
        std::vector<int> tg(T.ntiles), cnt(17 * (size_t)T.ngroups), nc(T.ngroups);
        e = cudaMemcpy(tg.data(), T.tile_group, sizeof(int) * tg.size(), cudaMemcpyDeviceToHost);
        if (e == cudaSuccess) e = cudaMemcpy(cnt.data(), T.grp_cnt, sizeof(int) * cnt.size(), cudaMemcpyDeviceToHost);
        if (e == cudaSuccess) e = cudaMemcpy(nc.data(), T.grp_nc, sizeof(int) * nc.size(), cudaMemcpyDeviceToHost);
        if (e != cudaSuccess) {
            set_error("tensor-core items: %s", cudaGetErrorString(e));
            return IFGF_ECUDA;
        }
        bool ok = true;
        std::vector<int4> items;
        for (int o = 0; o < 8; o++) {
            T.oct_item_start[o] = (int)items.size();
            for (int t = T.oct_tile_start[o]; t < T.oct_tile_start[o + 1]; t++) {
                const int g = tg[t];
                ok = ok && cnt[17 * (size_t)g + 16] == 0;
                int off = 0;
                for (int j = 0; j < nc[g]; j++) {
                    const int n = cnt[17 * (size_t)g + j];
                    for (int r = 0; r < n; r += kT5Rows) items.push_back(make_int4(t, off + r, std::min(kT5Rows, n - r), j));
                    off += n;
                }
            }
        }
        T.oct_item_start[8] = (int)items.size();
        T.nitems = (int)items.size();
        T.items_ok = ok;
        {  // the cone-stationary CUDA-core engine: runs of one child cone in chunks of <= 64 nodes
            std::vector<int4> cs;
            for (int o = 0; o < 8; o++) {
                T.oct_cs_start[o] = (int)cs.size();
                for (int t = T.oct_tile_start[o]; t < T.oct_tile_start[o + 1]; t++) {
                    const int g = tg[t];
                    int off = 0;
                    for (int j = 0; j < nc[g]; j++) {
                        const int n = cnt[17 * (size_t)g + j];
                        for (int r = 0; r < n; r += 64) cs.push_back(make_int4(t, off + r, std::min(64, n - r), j));
                        off += n;
                    }
                }
            }
            T.oct_cs_start[8] = (int)cs.size();
            T.ncs_items = (int)cs.size();
            void *ptr = nullptr;
            e = cudaMalloc(&ptr, sizeof(int4) * (cs.size() + 1));
            if (e == cudaSuccess && !cs.empty())
                e = cudaMemcpy(ptr, cs.data(), sizeof(int4) * cs.size(), cudaMemcpyHostToDevice);
            if (e != cudaSuccess) {
                if (ptr) cudaFree(ptr);
                set_error("propagation items: %s", cudaGetErrorString(e));
                return e == cudaErrorMemoryAllocation ? IFGF_ENOMEM : IFGF_ECUDA;
            }
            p.allocs.push_back(ptr);
            p.device_bytes += (int64_t)(sizeof(int4) * (cs.size() + 1));
            T.cs_items = (int4 *)ptr;
        }
        // item headers and child-cone storage indices (host copies of the tile and group tables)
        std::vector<int> ts(T.ntiles), tcn(T.ntiles), gg(T.ngroups), gpb(T.ngroups), gcb(T.ngroups),
            gcones(16 * (size_t)T.ngroups), pcb;
        int npairs = 0;
        e = cudaMemcpy(ts.data(), T.tile_start, sizeof(int) * ts.size(), cudaMemcpyDeviceToHost);
        if (e == cudaSuccess) e = cudaMemcpy(tcn.data(), T.tile_count, sizeof(int) * tcn.size(), cudaMemcpyDeviceToHost);
        if (e == cudaSuccess) e = cudaMemcpy(gg.data(), T.grp_gamma, sizeof(int) * gg.size(), cudaMemcpyDeviceToHost);
        if (e == cudaSuccess) e = cudaMemcpy(gpb.data(), T.grp_pb, sizeof(int) * gpb.size(), cudaMemcpyDeviceToHost);
        if (e == cudaSuccess) e = cudaMemcpy(gcb.data(), T.grp_cb, sizeof(int) * gcb.size(), cudaMemcpyDeviceToHost);
        if (e == cudaSuccess)
            e = cudaMemcpy(gcones.data(), T.grp_cones, sizeof(int) * gcones.size(), cudaMemcpyDeviceToHost);
        for (int t = 0; t < T.ntiles; t++) npairs = std::max(npairs, ts[t] + tcn[t]);
        pcb.resize(npairs > 0 ? npairs : 1);
        if (e == cudaSuccess && npairs > 0)
            e = cudaMemcpy(pcb.data(), T.pair_cb, sizeof(int) * npairs, cudaMemcpyDeviceToHost);
        if (e != cudaSuccess) {
            set_error("tensor-core items: %s", cudaGetErrorString(e));
            return IFGF_ECUDA;
        }
        const HostLevel &HC = p.lv[d], &HP = p.lv[d - 1];
        std::vector<int4> hdr(3 * items.size() + 1);
        std::vector<int> icrc(kTcTile * items.size() + 1, -1);
        for (size_t i = 0; i < items.size(); i++) {
            const int t = items[i].x, g = tg[t], cc = gcones[16 * (size_t)g + items[i].w];
            const int pb = gpb[g], cb0 = gcb[g];
            float o[3];
            for (int a = 0; a < 3; a++)  // exact: integer box coordinates, power-of-two scales
                o[a] = ((float)HC.ijk[3 * cb0 + a] + 0.5f) * (float)HC.scale -
                       ((float)HP.ijk[3 * pb + a] + 0.5f) * (float)HP.scale;
            hdr[3 * i] = make_int4(items[i].y, items[i].z, g, gg[g]);
            hdr[3 * i + 1] = make_int4(cc, ts[t], tcn[t], 0);
            hdr[3 * i + 2] = make_int4(__float_as_int_host(o[0]), __float_as_int_host(o[1]),
                                       __float_as_int_host(o[2]), 0);
            for (int q = 0; q < tcn[t]; q++) {
                const int cb = pcb[ts[t] + q];
                icrc[kTcTile * i + q] = HC.cone_map[(size_t)cb * HC.ncone + cc];
            }
        }
        void *ph = nullptr, *pc = nullptr;
        e = cudaMalloc(&ph, sizeof(int4) * hdr.size());
        if (e == cudaSuccess) e = cudaMalloc(&pc, sizeof(int) * icrc.size());
        if (e == cudaSuccess) e = cudaMemcpy(ph, hdr.data(), sizeof(int4) * hdr.size(), cudaMemcpyHostToDevice);
        if (e == cudaSuccess) e = cudaMemcpy(pc, icrc.data(), sizeof(int) * icrc.size(), cudaMemcpyHostToDevice);
        if (e != cudaSuccess) {
            if (ph) cudaFree(ph);
            if (pc) cudaFree(pc);
            set_error("tensor-core items: %s", cudaGetErrorString(e));
            return e == cudaErrorMemoryAllocation ? IFGF_ENOMEM : IFGF_ECUDA;
        }
        p.allocs.push_back(ph);
        p.allocs.push_back(pc);
        p.device_bytes += (int64_t)(sizeof(int4) * hdr.size() + sizeof(int) * icrc.size());
        T.item_hdr = (int4 *)ph;
        T.item_crc = (int *)pc;
        void *ptr = nullptr;
        e = cudaMalloc(&ptr, sizeof(int4) * (items.size() + 1));
        if (e == cudaSuccess && !items.empty())
            e = cudaMemcpy(ptr, items.data(), sizeof(int4) * items.size(), cudaMemcpyHostToDevice);
        if (e != cudaSuccess) {
            if (ptr) cudaFree(ptr);
            set_error("tensor-core items: %s", cudaGetErrorString(e));
            return e == cudaErrorMemoryAllocation ? IFGF_ENOMEM : IFGF_ECUDA;
        }
        p.allocs.push_back(ptr);
        p.device_bytes += (int64_t)(sizeof(int4) * (items.size() + 1));
        T.items = (int4 *)ptr;
    }
    return IFGF_OK;
}

// one-time launch attributes of this order's kernels (the tcgen05 propagation takes more than
// 48 KB of dynamic shared memory)
template <int PS, int PA>
ifgf_status prepare_t(Plan &p, cudaStream_t s) {
    if constexpr (PA == 8) return t5_prepare<PS>(p, s);
    (void)p;
    (void)s;
    return IFGF_OK;
}

template <int PS, int PA>
ifgf_status run_apply_t(Plan &p, const void *sigma, void *y, int nrhs, int prec, cudaStream_t s) {
    constexpr int P = PS * PA * PA;
    const int D = p.D;
    const int N = (int)p.N;
    CommonArgs ca = common_args(p, nrhs);
    ChebTab tb = cheb_tab(p);
    LevelArgs L[IFGF_MAXD + 1];
    for (int d = 3; d <= D; d++) L[d] = level_args(p, d, p.ws.F[d]);
    const long long NT = (long long)N * nrhs;
    prof_begin(p, s);
    // The near field and the cousin interpolation of level d depend only on the gathered density and
    // on F_d: they run on the plan's auxiliary stream beside the leaf / propagation chain (fork after
    // the gather, one event per finished level, join before the scatter).  The auxiliary stream runs
    // near, then cousin D, ..., 3 in order, so the field u has one writer at a time.
    // upward pass only (far-field evaluation): leaf expansions and propagation, nothing that writes u
    const bool down = !p.upward_only;
    const bool par = !p.profile && p.aux && down;
    const cudaStream_t sb = par ? p.aux : s;
    // fork / join (and the cousin launches' buffer clearing) record the first failure of their
    // calls (checked after the join); they return nothing, so that every path through them is well
    // defined
    cudaError_t dep_err = cudaSuccess;
    auto fork = [&](int slot) {
        if (par && dep_err == cudaSuccess) {
            dep_err = cudaEventRecord(p.dep[slot], s);
            if (dep_err == cudaSuccess) dep_err = cudaStreamWaitEvent(sb, p.dep[slot], 0);
        }
    };
    auto join = [&]() {
        if (par && dep_err == cudaSuccess) {
            dep_err = cudaEventRecord(p.dep[Plan::kMaxDep - 1], sb);
            if (dep_err == cudaSuccess) dep_err = cudaStreamWaitEvent(s, p.dep[Plan::kMaxDep - 1], 0);
        }
    };
    if (prec == IFGF_FP64) {
        k_gather<double><<<nblk(NT), kBlock, 0, s>>>(N, nrhs, p.d_perm, p.d_w64, (const double2 *)sigma, (double2 *)p.ws.a);
        prof_mark(p, s, kStGather, 0);
        fork(0);
        if (down) {
            k_near64<<<nblk(N), kBlock, 0, sb>>>(ca, L[D], (const double2 *)p.ws.a, (double2 *)p.ws.u);
            prof_mark(p, sb, kStNear, D);
        }
        if (L[D].nrc) {
            k_leaf64<PS, PA><<<nblk(L[D].nrc * P), kBlock, 0, s>>>(ca, L[D], tb, (const double2 *)p.ws.a, nullptr,
                                                                   L[D].nrc);
            prof_mark(p, s, kStLeaf, D);
        }
        fork(1);
        if (down) {
            k_cousin64<PS, PA><<<nblk(N), kBlock, 0, sb>>>(ca, L[D], p.d_box_of[D], p.d_alive[D], tb,
                                                           (double2 *)p.ws.u);
            prof_mark(p, sb, kStCousin, D);
        }
        for (int d = D; d >= 4; d--) {
            if (L[d - 1].nrc) {
                k_prop64<PS, PA><<<nblk(L[d - 1].nrc * P), kBlock, 0, s>>>(ca, L[d], L[d - 1], tb);
                prof_mark(p, s, kStProp, d - 1);
            }
            if (p.nleaf_rc[d - 1]) {  // adaptive tree: the leaves of level d-1 (no children, F from sources)
                const long long nl = p.nleaf_rc[d - 1];
                k_leaf64<PS, PA><<<nblk(nl * P), kBlock, 0, s>>>(ca, L[d - 1], tb, (const double2 *)p.ws.a,
                                                                 p.d_leaf_rc[d - 1], nl);
                prof_mark(p, s, kStLeaf, d - 1);
            }
            fork(2 + D - d);
            if (down) {
                k_cousin64<PS, PA><<<nblk(N), kBlock, 0, sb>>>(ca, L[d - 1], p.d_box_of[d - 1], p.d_alive[d - 1], tb,
                                                               (double2 *)p.ws.u);
                prof_mark(p, sb, kStCousin, d - 1);
            }
        }
        join();
        CK(dep_err);
        if (down) {
            k_scatter<double><<<nblk(NT), kBlock, 0, s>>>(N, nrhs, p.d_perm, p.prm.identity_coef,
                                                           (const double2 *)sigma, (const double2 *)p.ws.u,
                                                           (double2 *)y);
            prof_mark(p, s, kStScatter, 0);
        }
    } else {
        const bool rb1 = nrhs == 1 || p.rhs_block == 1;
        float2 *u32 = (float2 *)p.ws.u;
        auto cousin = [&](int d) {
            if (!down) return;
            const int nch = p.ncchunk[d];
            if (p.cs_ok && p.interp_engine == 1) {
                const int ni = p.ncs_item[d];
                const long long stride = p.cs_max_entries;
                float2 *pv = (float2 *)p.ws.pv;
                if (ni > 0) {
                    const unsigned g = (unsigned)((ni + kCsWarps - 1) / kCsWarps);
                    // slots of cousins without sources are never written: zero them first
                    if (p.has_inactive && dep_err == cudaSuccess)
                        dep_err = cudaMemsetAsync(pv, 0, sizeof(float2) * (size_t)nrhs * stride, sb);
                    if (L[d].split)
                        k_cousin_cs<PS, PA, true><<<g, kCsWarps * 32, 0, sb>>>(
                            ca, L[d], p.d_cs_item[d], ni, p.d_cs_geo4[d], p.d_cs_geo2[d], tb, pv, stride);
                    else
                        k_cousin_cs<PS, PA, false><<<g, kCsWarps * 32, 0, sb>>>(
                            ca, L[d], p.d_cs_item[d], ni, p.d_cs_geo4[d], p.d_cs_geo2[d], tb, pv, stride);
                    prof_mark(p, sb, kStCousin, d);
                    k_cousin_sum<<<nblk(N), kBlock, 0, sb>>>(ca, L[d], p.d_box_of[d], p.d_alive[d], p.d_cs_pvoff[d], pv,
                                                             stride, u32);
                    prof_mark(p, sb, kStCousinSum, d);
                }
                return;
            } else if (nch > 0) {
                const unsigned g = (unsigned)((nch + kCwWarps - 1) / kCwWarps);
                if (rb1) k_cousin_w<PS, PA, 1><<<g, kCwWarps * 32, 0, sb>>>(ca, L[d], L[D], p.d_cchunk[d], nch, tb, u32);
                else k_cousin_w<PS, PA, kRB><<<g, kCwWarps * 32, 0, sb>>>(ca, L[d], L[D], p.d_cchunk[d], nch, tb, u32);
            }
            prof_mark(p, sb, kStCousin, d);
        };
        k_gather<float><<<nblk(NT), kBlock, 0, s>>>(N, nrhs, p.d_perm, p.d_w32, (const float2 *)sigma, (float2 *)p.ws.a);
        const ulonglong2 *pp = (const ulonglong2 *)p.d_pp32, *ap = (const ulonglong2 *)p.ws.ap;
        if (nrhs == 1)  // one right-hand side: the leaf and the near field run on source pairs
            k_pack_pairs<<<nblk(p.npairs), kBlock, 0, s>>>(N, p.npairs, 1, p.d_pair_src, (const float2 *)p.ws.a,
                                                           (float4 *)p.ws.ap);
        prof_mark(p, s, kStGather, 0);
        fork(0);
        if (down) {
            const unsigned gn = (unsigned)((p.nnchunk + kNearWarps - 1) / kNearWarps);
            if (p.adaptive) {  // leaves of several levels: ranges of near sources per leaf
                const unsigned gl = (unsigned)((p.nnchunk_light + kNearWarps - 1) / kNearWarps);
                const int4 *hv = p.d_nchunk + p.nnchunk_light;
                const int nh = p.nnchunk - p.nnchunk_light;
                if (nrhs == 1) {
                    if (gl)
                        k_near32pr<<<gl, kNearWarps * 32, 0, sb>>>(ca, p.d_nchunk, p.nnchunk_light, p.d_nr_start, p.d_nr,
                                                                   p.d_pt_ijk, p.d_pair_ijk, pp, ap, u32);
                    if (nh)
                        k_near32pr_blk<<<nh, kNearBlkWarps * 32, 0, sb>>>(ca, hv, p.d_nr_start, p.d_nr, p.d_pt_ijk,
                                                                          p.d_pair_ijk, pp, ap, u32);
                } else {
                    const float2 *a32 = (const float2 *)p.ws.a;
                    if (gl && rb1)
                        k_near32r<1><<<gl, kNearWarps * 32, 0, sb>>>(ca, p.d_nchunk, p.nnchunk_light, p.d_nr_start,
                                                                     p.d_nr, p.d_pt_ijk, a32, u32);
                    else if (gl)
                        k_near32r<kRB><<<gl, kNearWarps * 32, 0, sb>>>(ca, p.d_nchunk, p.nnchunk_light, p.d_nr_start,
                                                                       p.d_nr, p.d_pt_ijk, a32, u32);
                    if (nh)
                        k_near32r_blk<<<nh, kNearBlkWarps * 32, 0, sb>>>(ca, hv, p.d_nr_start, p.d_nr, p.d_pt_ijk, a32,
                                                                         u32);
                }
            }
            else if (nrhs == 1)
                k_near32p<<<gn, kNearWarps * 32, 0, sb>>>(ca, L[D], p.d_nchunk, p.nnchunk, pp, p.d_pstart, ap, u32);
            else if (rb1)
                k_near32<1><<<gn, kNearWarps * 32, 0, sb>>>(ca, L[D], p.d_nchunk, p.nnchunk, (const float2 *)p.ws.a, u32);
            else
                k_near32<kRB><<<gn, kNearWarps * 32, 0, sb>>>(ca, L[D], p.d_nchunk, p.nnchunk, (const float2 *)p.ws.a, u32);
        }
        if (down) prof_mark(p, sb, kStNear, D);
        if (L[D].nrc) {
            const unsigned g = nblk(L[D].nrc * P);
            const float2 *a32 = (const float2 *)p.ws.a;
            const unsigned g2 = nblk(L[D].nrc * ((P + 1) / 2));
            if (nrhs == 1) {  // source pairs (packed after the gather): two sources per instruction
                if (L[D].split) k_leaf32p<PS, PA, true><<<g2, kBlock, 0, s>>>(ca, L[D], tb, pp, p.d_pstart, ap);
                else k_leaf32p<PS, PA, false><<<g2, kBlock, 0, s>>>(ca, L[D], tb, pp, p.d_pstart, ap);
            } else if (L[D].split) {
                if (rb1) k_leaf32<PS, PA, 1, true><<<g, kBlock, 0, s>>>(ca, L[D], tb, a32);
                else k_leaf32<PS, PA, kRB, true><<<g, kBlock, 0, s>>>(ca, L[D], tb, a32);
            } else {
                if (rb1) k_leaf32<PS, PA, 1, false><<<g, kBlock, 0, s>>>(ca, L[D], tb, a32);
                else k_leaf32<PS, PA, kRB, false><<<g, kBlock, 0, s>>>(ca, L[D], tb, a32);
            }
            prof_mark(p, s, kStLeaf, D);
        }
        fork(1);
        cousin(D);
        for (int d = D; d >= 4; d--) {
            if (L[d - 1].nrc && PA == 8 && p.use_tc && p.tc[d].fill >= p.tc_min_fill &&
                (p.tc_engine == 0 || p.tc[d].items_ok)) {
                if constexpr (PA == 8) {
                    const size_t bytes = sizeof(float2) * (size_t)nrhs * L[d - 1].nrc * L[d - 1].nfac * p.Pstride;
                    CK(cudaMemsetAsync(L[d - 1].F, 0, bytes, s));
                    const TcLevel &T = p.tc[d];
                    for (int o = 0; o < 8; o++) {
                        const int t0 = T.oct_tile_start[o], nt = T.oct_tile_start[o + 1] - t0;
                        if (nt <= 0) continue;
                        if (p.tc_engine == 1) {
                            const int i0 = T.oct_item_start[o], ni = T.oct_item_start[o + 1] - i0;
                            if (ni > 0)
                                k_prop_t5<PS><<<2 * ni, kT5Threads, kT5Smem, s>>>(ca, L[d], L[d - 1], tb, T, i0);
                        } else if (p.tc_engine == 2) {
                            const int i0 = T.oct_item_start[o], ni = T.oct_item_start[o + 1] - i0;
                            // persistent: as many blocks per SM as their tensor memory allows
                            auto grid = [&](uint32_t cols) { return std::min(ni, (cols <= 256 ? 2 : 1) * p.num_sms); };
                            if (ni > 0) {
                                if (L[d].split && L[d - 1].split)
                                    k_prop_t6<PS, true, true><<<grid(T6Cfg<PS, 2>::kCols), kT6Threads, 0, s>>>(
                                        ca, L[d], L[d - 1], tb, T, i0, ni);
                                else if (L[d].split)
                                    k_prop_t6<PS, true, false><<<grid(T6Cfg<PS, 2>::kCols), kT6Threads, 0, s>>>(
                                        ca, L[d], L[d - 1], tb, T, i0, ni);
                                else
                                    k_prop_t6<PS, false, false><<<grid(T6Cfg<PS, 1>::kCols), kT6Threads, 0, s>>>(
                                        ca, L[d], L[d - 1], tb, T, i0, ni);
                            }
                        } else {
                            k_prop_tc<PS><<<dim3(2 * nt, P / kTcRows), 128, 0, s>>>(ca, L[d], L[d - 1], tb, T, t0);
                        }
                    }
                    prof_mark(p, s, kStPropTc, d - 1);
                }
            } else if (L[d - 1].nrc && PA == 8 && p.use_tc && p.tc[d].items_ok && p.interp_engine == 1) {
                if constexpr (PA == 8) {
                    const size_t bytes = sizeof(float2) * (size_t)nrhs * L[d - 1].nrc * L[d - 1].nfac * p.Pstride;
                    CK(cudaMemsetAsync(L[d - 1].F, 0, bytes, s));
                    const TcLevel &T = p.tc[d];
                    for (int o = 0; o < 8; o++) {
                        const int i0 = T.oct_cs_start[o], ni = T.oct_cs_start[o + 1] - i0;
                        if (ni <= 0) continue;
                        const unsigned gc = (unsigned)((ni + kCsWarps - 1) / kCsWarps);
                        if (L[d].split && L[d - 1].split)
                            k_prop_cs<PS, true, true><<<gc, kCsWarps * 32, 0, s>>>(ca, L[d], L[d - 1], tb, T, i0, ni);
                        else if (L[d].split)
                            k_prop_cs<PS, true, false><<<gc, kCsWarps * 32, 0, s>>>(ca, L[d], L[d - 1], tb, T, i0, ni);
                        else
                            k_prop_cs<PS, false, false><<<gc, kCsWarps * 32, 0, s>>>(ca, L[d], L[d - 1], tb, T, i0, ni);
                    }
                    prof_mark(p, s, kStPropCs, d - 1);
                }
            } else if (L[d - 1].nrc) {
                const long long nw = L[d - 1].nrc * (long long)((P + 31) / 32);
                const unsigned gw = (unsigned)((nw + kCwWarps - 1) / kCwWarps);
                if (rb1) k_prop_w<PS, PA, 1><<<gw, kCwWarps * 32, 0, s>>>(ca, L[d], L[d - 1], tb);
                else k_prop_w<PS, PA, kRB><<<gw, kCwWarps * 32, 0, s>>>(ca, L[d], L[d - 1], tb);
                prof_mark(p, s, kStProp, d - 1);
            }
            if (p.nleaf_rc[d - 1]) {  // adaptive tree: the leaves of level d-1 (no children, F from sources)
                const long long nl = p.nleaf_rc[d - 1];
                const float2 *a32 = (const float2 *)p.ws.a;
                if (L[d - 1].split)
                    k_leaf32a<PS, PA, true><<<nblk(nl * P), kBlock, 0, s>>>(ca, L[d - 1], L[D], tb, a32,
                                                                            p.d_leaf_rc[d - 1], nl);
                else
                    k_leaf32a<PS, PA, false><<<nblk(nl * P), kBlock, 0, s>>>(ca, L[d - 1], L[D], tb, a32,
                                                                             p.d_leaf_rc[d - 1], nl);
                prof_mark(p, s, kStLeaf, d - 1);
            }
            fork(2 + D - d);
            cousin(d - 1);
        }
        join();
        CK(dep_err);
        if (down) {
            k_scatter<float><<<nblk(NT), kBlock, 0, s>>>(N, nrhs, p.d_perm, p.prm.identity_coef,
                                                          (const float2 *)sigma, (const float2 *)p.ws.u, (float2 *)y);
            prof_mark(p, s, kStScatter, 0);
        }
    }
    CK(cudaGetLastError());
    return IFGF_OK;
}


// ============================================================================
// launch sequence of one adjoint apply (workspace prepared by the caller)
// ============================================================================
template <int PS, int PA>
ifgf_status run_adjoint_t(Plan &p, const void *g, void *out, int nrhs, int prec, cudaStream_t s, void *gs, void *bws,
                          void **G, void *const *Fd, double *dk_partials) {
    const int D = p.D;
    const int N = (int)p.N;
    CommonArgs ca = common_args(p, nrhs);
    ChebTab tb = cheb_tab(p);
    LevelArgs L[IFGF_MAXD + 1];
    for (int d = 3; d <= D; d++) L[d] = level_args(p, d, nullptr);
    const long long NT = (long long)N * nrhs;
    prof_begin(p, s);
    if (prec == IFGF_FP64) {
        k_gather_plain<double2><<<nblk(NT), kBlock, 0, s>>>(N, nrhs, p.d_perm, (const double2 *)g, (double2 *)gs);
        prof_mark(p, s, kStGather, 0);
        for (int d = 3; d <= D; d++)
            if (L[d].nrc) {
                const Plan::AntArgs aa = {(const long long *)p.d_ad_start[d], p.d_ad_list[d]};
                if (Fd)
                    k_ant<PS, PA, false, true><<<(unsigned)L[d].nrc, 128, 0, s>>>(
                        ca, L[d], d > 3 ? L[d - 1] : L[d], L[D], d > 3, aa.start, aa.list, tb, gs,
                        d > 3 ? G[d - 1] : nullptr, G[d], Fd[d], dk_partials, nullptr, nullptr, nullptr);
                else
                    k_ant<PS, PA, false, false><<<(unsigned)L[d].nrc, 128, 0, s>>>(
                        ca, L[d], d > 3 ? L[d - 1] : L[d], L[D], d > 3, aa.start, aa.list, tb, gs,
                        d > 3 ? G[d - 1] : nullptr, G[d], nullptr, nullptr, nullptr, nullptr, nullptr);
                if (Fd) dk_partials += L[d].nrc;
                prof_mark(p, s, kStCousin, d);
            }
        k_near_adj<false><<<nblk(N), kBlock, 0, s>>>(ca, L[D], gs, bws);
        prof_mark(p, s, kStNear, D);
        if (L[D].nrc) {
            k_leaf_adj<PS, PA, false><<<nblk(N), kBlock, 0, s>>>(ca, L[D], tb, G[D], bws, nullptr, nullptr, L[D]);
            prof_mark(p, s, kStLeaf, D);
        }
        for (int d = 3; d < D; d++)  // adaptive tree: the leaves of the coarser levels
            if (p.nleaf_rc[d]) {
                k_leaf_adj<PS, PA, false><<<nblk(N), kBlock, 0, s>>>(ca, L[d], tb, G[d], bws, p.d_box_of[d],
                                                                     p.d_leaf[d], L[D]);
                prof_mark(p, s, kStLeaf, d);
            }
        k_scatter_adj<double><<<nblk(NT), kBlock, 0, s>>>(N, nrhs, p.d_perm, p.prm.identity_coef, p.d_w64,
                                                           (const double2 *)g, (const double2 *)bws, (double2 *)out);
        prof_mark(p, s, kStScatter, 0);
    } else {
        k_gather_plain<float2><<<nblk(NT), kBlock, 0, s>>>(N, nrhs, p.d_perm, (const float2 *)g, (float2 *)gs);
        prof_mark(p, s, kStGather, 0);
        for (int d = 3; d <= D; d++)
            if (L[d].nrc) {
                const Plan::AntArgs aa = {(const long long *)p.d_ad_start[d], p.d_ad_list[d]};
                // the cone-stationary forward lists' geometry serves the cousin entries
                const bool cg = p.cs_ok && p.d_cs_first[d];
                const int *csf = cg ? p.d_cs_first[d] : nullptr;
                const float4 *cg4 = cg ? p.d_cs_geo4[d] : nullptr;
                const float2 *cg2 = cg ? p.d_cs_geo2[d] : nullptr;
                if (Fd)
                    k_ant<PS, PA, true, true><<<(unsigned)L[d].nrc, 128, 0, s>>>(
                        ca, L[d], d > 3 ? L[d - 1] : L[d], L[D], d > 3, aa.start, aa.list, tb, gs,
                        d > 3 ? G[d - 1] : nullptr, G[d], Fd[d], dk_partials, csf, cg4, cg2);
                else
                    k_ant<PS, PA, true, false><<<(unsigned)L[d].nrc, 128, 0, s>>>(
                        ca, L[d], d > 3 ? L[d - 1] : L[d], L[D], d > 3, aa.start, aa.list, tb, gs,
                        d > 3 ? G[d - 1] : nullptr, G[d], nullptr, nullptr, csf, cg4, cg2);
                if (Fd) dk_partials += L[d].nrc;
                prof_mark(p, s, kStCousin, d);
            }
        // with the k-derivative (Fd given), the near-field and leaf parts of Re <g, dA/dk sigma> come from
        // the same pair loops: one double per block after the anterpolation's per-cone partials
        const float2 *afw = (const float2 *)p.ws.a;
        if (Fd) k_near_adj32<true><<<nblk(N), kBlock, 0, s>>>(ca, L[D], (const float2 *)gs, (float2 *)bws, afw, dk_partials);
        else k_near_adj32<false><<<nblk(N), kBlock, 0, s>>>(ca, L[D], (const float2 *)gs, (float2 *)bws, nullptr, nullptr);
        if (Fd) dk_partials += nblk(N);
        prof_mark(p, s, kStNear, D);
        if (L[D].nrc) {
            const int nch = p.ncchunk[D];
            const unsigned gw = (unsigned)((nch + 3) / 4);
            const float2 *GD = (const float2 *)G[D];
            if (L[D].split) {
                if (Fd) k_leaf_adj_w<PS, PA, true, true><<<gw, 128, 0, s>>>(ca, L[D], p.d_cchunk[D], nch, tb, GD, (float2 *)bws, afw, dk_partials);
                else k_leaf_adj_w<PS, PA, true, false><<<gw, 128, 0, s>>>(ca, L[D], p.d_cchunk[D], nch, tb, GD, (float2 *)bws, nullptr, nullptr);
            } else {
                if (Fd) k_leaf_adj_w<PS, PA, false, true><<<gw, 128, 0, s>>>(ca, L[D], p.d_cchunk[D], nch, tb, GD, (float2 *)bws, afw, dk_partials);
                else k_leaf_adj_w<PS, PA, false, false><<<gw, 128, 0, s>>>(ca, L[D], p.d_cchunk[D], nch, tb, GD, (float2 *)bws, nullptr, nullptr);
            }
            if (Fd) dk_partials += gw;
            prof_mark(p, s, kStLeaf, D);
        }
        for (int d = 3; d < D; d++)  // adaptive tree: the leaves of the coarser levels
            if (p.nleaf_rc[d]) {
                if (Fd) {
                    k_leaf_adj<PS, PA, true, true><<<nblk(N), kBlock, 0, s>>>(ca, L[d], tb, G[d], bws, p.d_box_of[d],
                                                                              p.d_leaf[d], L[D], afw, dk_partials);
                    dk_partials += nblk(N);
                } else {
                    k_leaf_adj<PS, PA, true><<<nblk(N), kBlock, 0, s>>>(ca, L[d], tb, G[d], bws, p.d_box_of[d],
                                                                        p.d_leaf[d], L[D]);
                }
                prof_mark(p, s, kStLeaf, d);
            }
        k_scatter_adj<float><<<nblk(NT), kBlock, 0, s>>>(N, nrhs, p.d_perm, p.prm.identity_coef, p.d_w32,
                                                          (const float2 *)g, (const float2 *)bws, (float2 *)out);
        prof_mark(p, s, kStScatter, 0);
    }
    CK(cudaGetLastError());
    return IFGF_OK;
}


// ============================================================================
// k-derivative reductions (forward state in p.ws, adjoint state gs / G)
// ============================================================================
template <int PS, int PA>
ifgf_status run_dk_t(Plan &p, int nrhs, int prec, cudaStream_t s, const void *gs, void **G, double *partials,
                     long long *nparts) {
    constexpr int P = PS * PA * PA;
    const int D = p.D;
    const int N = (int)p.N;
    CommonArgs ca = common_args(p, nrhs);
    ChebTab tb = cheb_tab(p);
    LevelArgs LD = level_args(p, D, p.ws.F[D]);
    long long off = 0;
    const bool mx = prec == IFGF_MIXED;
    if (mx) k_dk_near<true><<<nblk(N), kBlock, 0, s>>>(ca, LD, p.ws.a, gs, partials + off);
    else k_dk_near<false><<<nblk(N), kBlock, 0, s>>>(ca, LD, p.ws.a, gs, partials + off);
    off += nblk(N);
    const long long nt = LD.nrc * P;
    if (nt) {
        if (mx)
            k_dk_leaf<PS, PA, true><<<nblk(nt), kBlock, 0, s>>>(ca, LD, tb, p.ws.a, G[D], partials + off, nullptr,
                                                                LD.nrc);
        else
            k_dk_leaf<PS, PA, false><<<nblk(nt), kBlock, 0, s>>>(ca, LD, tb, p.ws.a, G[D], partials + off, nullptr,
                                                                 LD.nrc);
        off += nblk(nt);
    }
    for (int d = 3; d < D && !mx; d++)  // adaptive tree: the leaves of the coarser levels (FP64)
        if (p.nleaf_rc[d]) {
            const long long nl = p.nleaf_rc[d];
            LevelArgs Ld = level_args(p, d, p.ws.F[d]);
            k_dk_leaf<PS, PA, false><<<nblk(nl * P), kBlock, 0, s>>>(ca, Ld, tb, p.ws.a, G[d], partials + off,
                                                                     p.d_leaf_rc[d], nl);
            off += nblk(nl * P);
        }
    *nparts = off;
    CK(cudaGetLastError());
    return IFGF_OK;
}

// number of partial sums a vector-Jacobian product writes: one per relevant cone (the fused
// anterpolation), then the near-field and leaf reductions of run_dk_t
inline long long dk_partials_needed(const Plan &p) {
    long long n = nblk(p.N) + nblk(p.lv[p.D].nrc * p.P);
    for (int d = 3; d <= p.D; d++) n += p.lv[d].nrc;
    for (int d = 3; d < p.D; d++) n += std::max<long long>(nblk(p.N), nblk((long long)p.nleaf_rc[d] * p.P));
    return n;
}

// ============================================================================
// far-field pattern from the level-3 interpolants (Eq. FarField, Section 3.4)
// ============================================================================
// With x = R xhat, R e^{-ikR} times the centred factor e^{ik|x - y_B|} / (4 pi |x - y_B|) of a
// level-3 box tends to e^{-ik xhat.y_B} / (4 pi), s = h_3 / |x - y_B| tends to 0 and the
// direction of x - y_B to xhat, so u_inf(xhat) = sum_B e^{-ik xhat.y_B} / (4 pi) F_B(0, xhat).
// Every box shares the cone (is = 0, it, ip) of xhat and the interpolation weights (local s
// coordinate -1), so the sum over boxes is one weighted reduction of the boxes' node values.
// One warp per direction: lane l holds the weights of nodes l, l + 32, ... and reads those
// nodes of each box (coalesced), scales its partial by the box's phase (from shared memory),
// and the warp adds its lanes at the end.  FP64 path: FP64 throughout; mixed path: the phases
// are formed in FP64 and rounded to FP32, the sums run in FP32 (the stored values are FP32).
constexpr int kFarWarps = 4;
constexpr int kFarMaxBox = 64;  // level 3 has 4^3 boxes (side L / 4)

template <int PS, int PA, typename TF>
__global__ void __launch_bounds__(kFarWarps * 32)
    k_far_ifgf(CommonArgs ca, LevelArgs L, ChebTab tb, const typename C2T<TF>::type *__restrict__ F,
               const double *__restrict__ xhat, long long M, int fac, typename C2T<TF>::type *__restrict__ out) {
    constexpr int P = PS * PA * PA, NJ = (P + 31) / 32;
    using C2 = typename C2T<TF>::type;
    __shared__ C2 s_ph[kFarWarps][kFarMaxBox];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const long long j = (long long)blockIdx.x * kFarWarps + warp;
    if (j >= M) return;  // whole warp
    const double e0 = xhat[3 * j], e1 = xhat[3 * j + 1], e2 = xhat[3 * j + 2];
    // direction of xhat on the cone grid (theta, phi as in classify64), segment is = 0
    double th = atan2(sqrt(e0 * e0 + e1 * e1), e2);
    double ph = atan2(e1, e0);
    if (ph < 0) ph += 2.0 * kPi;
    if (ph >= 2.0 * kPi) ph = 0.0;
    const double ut = snap64(th / L.dth), up = snap64(ph / L.dph);
    const int it = max(min((int)floor(ut), L.nC - 1), 0), ip = max(min((int)floor(up), L.nph - 1), 0);
    const int cone = it * L.nph + ip;
    double Ls[PS], Lt[PA], Lp[PA];
    lagrange<PS, double>(-1.0, tb.xs, tb.cs, Ls);
    lagrange<PA, double>(2.0 * (ut - it) - 1.0, tb.xa, tb.ca, Lt);
    lagrange<PA, double>(2.0 * (up - ip) - 1.0, tb.xa, tb.ca, Lp);
    TF w[NJ];
#pragma unroll
    for (int jj = 0; jj < NJ; jj++) {
        const int n = lane + 32 * jj;
        w[jj] = n < P ? (TF)(Ls[n / (PA * PA)] * Lt[(n / PA) % PA] * Lp[n % PA]) : TF(0);
    }
    const double c4 = 1.0 / (4.0 * kPi);
    for (int b = lane; b < L.nbox; b += 32) {
        double y0[3];
        center64(ca, L, b, y0);
        double sn, cs;
        sincos(-ca.k * (e0 * y0[0] + e1 * y0[1] + e2 * y0[2]), &sn, &cs);
        C2 e;
        e.x = (TF)(c4 * cs);
        e.y = (TF)(c4 * sn);
        s_ph[warp][b] = e;
    }
    __syncwarp();
    for (int q = 0; q < ca.nrhs; q++) {
        TF ar = TF(0), ai = TF(0);
        for (int b = 0; b < L.nbox; b++) {
            if (L.rc_start[b] == L.rc_start[b + 1]) continue;  // no sources in b
            const int rc = L.cone_map[(long long)b * L.ncone + cone];
            if (rc < 0) {  // outside the relevant set: the plan lacks the far-field segments
                if (lane == 0 && q == 0) atomicAdd(ca.missed, 1ULL);
                continue;
            }
            const C2 *f = F + (((long long)q * L.nrc + rc) * L.nfac + fac) * ca.Pstride;
            TF vr = TF(0), vi = TF(0);
#pragma unroll
            for (int jj = 0; jj < NJ; jj++) {
                const int n = lane + 32 * jj;
                if (n < P) {
                    const C2 v = f[n];
                    vr += w[jj] * v.x;
                    vi += w[jj] * v.y;
                }
            }
            const C2 e = s_ph[warp][b];
            ar += e.x * vr - e.y * vi;
            ai += e.x * vi + e.y * vr;
        }
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            ar += __shfl_xor_sync(0xffffffffu, ar, o);
            ai += __shfl_xor_sync(0xffffffffu, ai, o);
        }
        if (lane == 0) {
            C2 r;
            r.x = ar;
            r.y = ai;
            out[(long long)q * M + j] = r;
        }
    }
}

// launch of the far-field evaluation on the level-3 cone values that the upward pass left in
// the plan's workspace
template <int PS, int PA>
ifgf_status run_far_t(Plan &p, const double *xhat, long long M, void *out, int nrhs, int prec, cudaStream_t s) {
    if (p.lv[3].nbox > kFarMaxBox) {
        set_error("far field: %d level-3 boxes (at most %d)", p.lv[3].nbox, kFarMaxBox);
        return IFGF_EINTERNAL;
    }
    CommonArgs ca = common_args(p, nrhs);
    ChebTab tb = cheb_tab(p);
    LevelArgs L3 = level_args(p, 3, p.ws.F[3]);
    const int fac = L3.split ? 1 : 0;  // the W13 member of a split pair; W2 drops out
    const unsigned g = (unsigned)((M + kFarWarps - 1) / kFarWarps);
    if (prec == IFGF_FP64)
        k_far_ifgf<PS, PA, double><<<g, kFarWarps * 32, 0, s>>>(ca, L3, tb, (const double2 *)p.ws.F[3], xhat, M, fac,
                                                                (double2 *)out);
    else
        k_far_ifgf<PS, PA, float><<<g, kFarWarps * 32, 0, s>>>(ca, L3, tb, (const float2 *)p.ws.F[3], xhat, M, fac,
                                                               (float2 *)out);
    CK(cudaGetLastError());
    return IFGF_OK;
}

}  // namespace ifgf

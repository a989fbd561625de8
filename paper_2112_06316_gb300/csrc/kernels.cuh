// Device helpers shared by the forward kernels (sm_103a).
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

namespace ifgf {

constexpr double kPi = 3.14159265358979323846;
constexpr float kPiF = 3.14159265358979323846f;

// Chebyshev tables passed by value (kernel parameter space is constant memory).
struct ChebTab {
    double xs[12], cs[12], xa[12], ca[12];
    float fxs[12], fcs[12], fxa[12], fca[12];
};

// Per-level arrays and cone-grid scalars, passed by value.
struct LevelArgs {
    int nbox, ns, nC, nph, ncone, split, nfac, scale;
    long long nrc;
    double H, h, ds, dth, dph;
    float hu, inv_ds, inv_dth, inv_dph, fds, fdth, fdph;
    const int *ijk, *start, *ch_start, *ch_list, *co_start, *co_list, *rc_start, *rc_cone, *rc_box, *cone_map;
    void *F;
};

struct CommonArgs {
    int N, nrhs, D, Pstride;
    // the kernel is alpha dPhi/dnu(y) + beta Phi with beta = -i (eta + i etai): alpha enters through the
    // normals (zero for the single layer alone), eta / etai are the real and imaginary parts of the
    // coupling (combined field: (eta, 0); double layer: (0, 0); single layer: (0, 1), beta = 1)
    double k, eta, etai, HD, L, tol;
    double c0[3];
    float kf, etaf, etaif, HDf, kappa_hi, kappa_lo;  // kappa = k HD / (2 pi) split in two floats
    const int *leaf_of, *nb_start, *nb_list;
    const double *x64, *n64, *w64;
    const float *f32, *n32, *w32;
    const float4 *pn32;  // per point: (leaf offset f, |f|^2), (normal, 0) — one 32-byte record
    unsigned long long *missed;
};

// ---- complex helpers -------------------------------------------------------
template <typename T> struct C2T;
template <> struct C2T<double> { typedef double2 type; };
template <> struct C2T<float> { typedef float2 type; };

// Neumaier-compensated accumulation of x into (s, c).
__device__ __forceinline__ void comp_add(float &s, float &c, float x) {
    float t = __fadd_rn(s, x);
    float e = (fabsf(s) >= fabsf(x)) ? __fadd_rn(__fsub_rn(s, t), x) : __fadd_rn(__fsub_rn(x, t), s);
    s = t;
    c = __fadd_rn(c, e);
}

// ---- Lagrange basis at first-kind Chebyshev nodes (product form) ----------
template <int n, typename T>
__device__ __forceinline__ void lagrange(T t, const T *x, const T *c, T *Lv) {
    T d[n];
#pragma unroll
    for (int j = 0; j < n; j++) d[j] = t - x[j];
    T pre = T(1);
    T prefix[n];
#pragma unroll
    for (int j = 0; j < n; j++) {
        prefix[j] = pre;
        pre *= d[j];
    }
    T suf = T(1);
#pragma unroll
    for (int j = n - 1; j >= 0; j--) {
        Lv[j] = c[j] * prefix[j] * suf;
        suf *= d[j];
    }
}

// Tensor-product interpolation of one cone's PS*PA*PA complex node values
// (node index (a*PA + b)*PA + c: a along s, b along theta, c along phi).
template <int PS, int PA, typename T>
__device__ __forceinline__ void interp3(const typename C2T<T>::type *__restrict__ f, const T *Ls, const T *Lt,
                                        const T *Lp, T &re, T &im) {
    re = T(0);
    im = T(0);
#pragma unroll
    for (int a = 0; a < PS; a++) {
        T ra = T(0), ia = T(0);
#pragma unroll
        for (int b = 0; b < PA; b++) {
            T rb = T(0), ib = T(0);
#pragma unroll
            for (int c = 0; c < PA; c++) {
                typename C2T<T>::type v = __ldg(f + (a * PA + b) * PA + c);
                rb = fma(Lp[c], v.x, rb);
                ib = fma(Lp[c], v.y, ib);
            }
            ra = fma(Lt[b], rb, ra);
            ia = fma(Lt[b], ib, ia);
        }
        re = fma(Ls[a], ra, re);
        im = fma(Ls[a], ia, im);
    }
}

// Value of L[a] for a runtime index a (select chain; keeps L in registers).
template <int n>
__device__ __forceinline__ float pick(const float *L, int a) {
    float v = L[0];
#pragma unroll
    for (int j = 1; j < n; j++) v = (a == j) ? L[j] : v;
    return v;
}

// Phase (in cycles, reduced to [-1/2, 1/2]) of kappa * |M + f| where M has
// half-integer components with |2M|^2 < 2^24 (so |M|^2 is exact in FP32) and f is
// a small FP32 offset; kappa = kappa_hi + kappa_lo.  |M + f| = sqrt(S) + T / (r + sqrt(S))
// with S = |M|^2 exact and T = 2 M.f + |f|^2; sqrt(S) is carried as a two-float value.
// Also returns r = |M + f| (FP32).
__device__ __forceinline__ float phase_cycles_exact(float Mx, float My, float Mz, float fx, float fy, float fz,
                                                    float khi, float klo, float &r) {
    float S = __fmaf_rn(Mx, Mx, __fmaf_rn(My, My, __fmul_rn(Mz, Mz)));
    float T = __fmaf_rn(2.f * Mx, fx, __fmaf_rn(2.f * My, fy, __fmaf_rn(2.f * Mz, fz,
              __fmaf_rn(fx, fx, __fmaf_rn(fy, fy, __fmul_rn(fz, fz))))));
    r = sqrtf(S + T);
    float r0 = sqrtf(S);
    float e0 = __fmaf_rn(-r0, r0, S);
    float r0l = (r0 > 0.f) ? e0 / (2.f * r0) : 0.f;
    float dlt = (r + r0 > 0.f) ? T / (r + r0) : 0.f;
    float p = __fmul_rn(khi, r0);
    float pe = __fmaf_rn(khi, r0, -p);
    float n = rintf(p);
    float t = __fsub_rn(p, n) + (pe + __fmaf_rn(khi, r0l + dlt, klo * r0));
    t -= rintf(t);
    return t;
}

}  // namespace ifgf

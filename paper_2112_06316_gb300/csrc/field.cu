// Off-surface evaluation from a density on the plan's surface (the paper's
// post-processing of a solved density, Section 5):
//   * the combined-layer potential of Eq. CombinedLayer at arbitrary targets x
//     (the near-field planes of Eq. PlanarGrid are such target sets),
//       u(x) = sum_m [dPhi(x, y_m)/dnu(y_m) - i eta Phi(x, y_m)] w_m sigma_m
//     (with the plan's layer: the double layer alone is eta = 0, the single layer alone has no
//     normal term and Phi's coefficient 1, carried as eta = i);
//   * its far-field pattern of Eq. FarField at directions xhat,
//       u_inf(xhat) = (1/4pi) sum_m [-i k xhat.nu_m - i eta] e^{-i k xhat.y_m} w_m sigma_m.
// Both are direct sums over every quadrature point (no octree acceleration),
// one thread per target and the sources walked leaf box by leaf box in Morton
// order, so that all threads of a warp read the same source record (broadcast
// loads).  When the targets alone do not fill the GPU, the leaf boxes are split
// into chunks (blockIdx.y) whose partial sums a second kernel adds in a fixed
// order, so results are deterministic.
//
// ifgf_far_field_ifgf instead takes the far-field pattern from the IFGF level-3 interpolants
// (the s -> 0 limit of the factorisation; kernel k_far_ifgf beside the forward kernels), and
// ifgf_field_ifgf the potential at targets that were part of the plan's octree (zero-weight points:
// their rows of the apply are the off-surface potential, accelerated like any other row).
//
// Mixed precision keeps the phase exact to ~1e-7 cycles without FP64 per pair:
// per (target, leaf box) the box part of the phase is formed once (far field:
// a two-float product with the exact half-integer box offset; potential: FP64
// distance to the box centre), and per source only a small FP32 correction is
// added (far field: xhat.f for the in-box offset f; potential: |D - f| - |D| =
// (|f|^2 - 2 D.f) / (|D - f| + |D|)).
#include <algorithm>
#include <cmath>

#include "ifgf_internal.h"
#include "kernels.cuh"

namespace ifgf {

void clear_error();

constexpr int kFieldBlock = 128;
constexpr int kFieldMaxSplit = 256;
constexpr int kFieldRB = 4;  // right-hand sides per register block when nrhs > 1

struct FieldArgs {
    int N, M, nrhs, nbox, split;
    double k, eta, etai, HD, tol;  // coupling eta + i etai (the kernel's Phi coefficient is -i (eta + i etai))
    double c0[3];                          // root box corner
    double kap;                            // k HD / (2 pi): phase cycles per leaf unit
    float kf, etaf, etaif, kapf, c4, iHD, tolu;  // c4 = 1 / (4 pi HD); tolu = tol / HD
    const int *ijk, *start;                // leaf boxes (level D): integer coordinates, point ranges
    const double *x64, *n64;               // sorted absolute positions / normals
    const float4 *pn32;                    // sorted (leaf offset f, |f|^2), (normal, 0)
    const double *tgt;                     // M x 3 targets (points or directions)
};

template <typename T>
__global__ void k_field_gather(int N, int nrhs, const int *__restrict__ perm, const T *__restrict__ w,
                               const typename C2T<T>::type *__restrict__ sigma, typename C2T<T>::type *__restrict__ a) {
    const long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (i >= (long long)N * nrhs) return;
    const int q = (int)(i / N), s = (int)(i % N);
    typename C2T<T>::type v = sigma[(long long)q * N + perm[s]];
    const T ww = w[s];
    v.x *= ww;
    v.y *= ww;
    a[i] = v;
}

// Chunk c of `split` near-equal ranges of leaf boxes.
__device__ __forceinline__ void box_range(const FieldArgs &fa, int c, int &b0, int &b1) {
    b0 = (int)((long long)fa.nbox * c / fa.split);
    b1 = (int)((long long)fa.nbox * (c + 1) / fa.split);
}

// (gh + gl) * m reduced to about [-1/2, 1/2] (+ a small remainder) for an exact FP32 m:
// gh * m = p + pe exactly, p - rint(p) is exact for |p| < 2^23.
__device__ __forceinline__ float cycles_of(float gh, float gl, float m) {
    const float p = __fmul_rn(gh, m);
    const float pe = __fmaf_rn(gh, m, -p);
    return __fsub_rn(p, rintf(p)) + __fmaf_rn(gl, m, pe);
}

// ---- far field, mixed ------------------------------------------------------------------
// Source y = c_b + HD f with c_b = c0 + HD (ijk_b + 1/2); the phase (in cycles) of
// e^{-ik xhat.y} is a0 + g.(ijk_b + 1/2) + g.f with g = k HD xhat / (2 pi).
template <int RB>
__global__ void __launch_bounds__(kFieldBlock) k_far32(FieldArgs fa, const float2 *__restrict__ a,
                                                       float2 *__restrict__ out) {
    const long long j = blockIdx.x * (long long)kFieldBlock + threadIdx.x;
    if (j >= fa.M) return;
    int b0, b1;
    box_range(fa, blockIdx.y, b0, b1);
    const double ux = fa.tgt[3 * j], uy = fa.tgt[3 * j + 1], uz = fa.tgt[3 * j + 2];
    const double gx = fa.kap * ux, gy = fa.kap * uy, gz = fa.kap * uz;
    const float ghx = (float)gx, ghy = (float)gy, ghz = (float)gz;
    const float glx = (float)(gx - (double)ghx), gly = (float)(gy - (double)ghy), glz = (float)(gz - (double)ghz);
    double a0d = fa.k / (2.0 * kPi) * (ux * fa.c0[0] + uy * fa.c0[1] + uz * fa.c0[2]);
    a0d -= rint(a0d);
    const float a0 = (float)a0d;
    const float kx = (float)(fa.k * ux), ky = (float)(fa.k * uy), kz = (float)(fa.k * uz);
    const float inv4pi = 1.f / (4.f * kPiF);
    for (int q0 = 0; q0 < fa.nrhs; q0 += RB) {
        float sr[RB], cr[RB], si[RB], ci[RB];
#pragma unroll
        for (int qq = 0; qq < RB; qq++) sr[qq] = cr[qq] = si[qq] = ci[qq] = 0.f;
        for (int b = b0; b < b1; b++) {
            const float mx = (float)__ldg(fa.ijk + 3 * b) + 0.5f, my = (float)__ldg(fa.ijk + 3 * b + 1) + 0.5f,
                        mz = (float)__ldg(fa.ijk + 3 * b + 2) + 0.5f;
            float t = a0 + cycles_of(ghx, glx, mx) + cycles_of(ghy, gly, my) + cycles_of(ghz, glz, mz);
            t -= rintf(t);
            float sb, cb;
            __sincosf(2.f * kPiF * t, &sb, &cb);
            float pr[RB], pi[RB];
#pragma unroll
            for (int qq = 0; qq < RB; qq++) pr[qq] = pi[qq] = 0.f;
            const int m1 = __ldg(fa.start + b + 1);
            for (int m = __ldg(fa.start + b); m < m1; m++) {
                const float4 f = __ldg(fa.pn32 + 2 * m), nu = __ldg(fa.pn32 + 2 * m + 1);
                float tt = __fmaf_rn(ghx, f.x, __fmaf_rn(ghy, f.y, __fmul_rn(ghz, f.z)));
                tt -= rintf(tt);
                float sn, cs;
                __sincosf(2.f * kPiF * tt, &sn, &cs);
                const float tau = __fmaf_rn(kx, nu.x, __fmaf_rn(ky, nu.y, __fmaf_rn(kz, nu.z, fa.etaf)));
                // (etai - i tau) e^{-i 2 pi tt} = (etai cs - tau sn, -etai sn - tau cs)
                const float wr = __fmaf_rn(fa.etaif, cs, -tau * sn), wi = -__fmaf_rn(fa.etaif, sn, tau * cs);
#pragma unroll
                for (int qq = 0; qq < RB; qq++) {
                    if (RB == 1 || q0 + qq < fa.nrhs) {
                        const float2 am = __ldg(a + (long long)(q0 + qq) * fa.N + m);
                        pr[qq] = __fmaf_rn(wr, am.x, __fmaf_rn(-wi, am.y, pr[qq]));
                        pi[qq] = __fmaf_rn(wr, am.y, __fmaf_rn(wi, am.x, pi[qq]));
                    }
                }
            }
            // times the box phase e^{-i 2 pi t} = (cb, -sb)
#pragma unroll
            for (int qq = 0; qq < RB; qq++) {
                comp_add(sr[qq], cr[qq], __fmaf_rn(cb, pr[qq], sb * pi[qq]));
                comp_add(si[qq], ci[qq], __fmaf_rn(cb, pi[qq], -sb * pr[qq]));
            }
        }
#pragma unroll
        for (int qq = 0; qq < RB; qq++)
            if (RB == 1 || q0 + qq < fa.nrhs)
                out[((long long)blockIdx.y * fa.nrhs + q0 + qq) * fa.M + j] =
                    make_float2((sr[qq] + cr[qq]) * inv4pi, (si[qq] + ci[qq]) * inv4pi);
    }
}

// ---- combined-layer potential, mixed ---------------------------------------------------
// Target in leaf units D = (x - c_b) / HD per box (FP64 once per box), source offset f:
// x - y = HD (D - f); the phase k HD |D - f| / (2 pi) = kap |D| + kap (|D - f| - |D|).
template <int RB>
__global__ void __launch_bounds__(kFieldBlock) k_pot32(FieldArgs fa, const float2 *__restrict__ a,
                                                       float2 *__restrict__ out) {
    const long long j = blockIdx.x * (long long)kFieldBlock + threadIdx.x;
    if (j >= fa.M) return;
    int b0, b1;
    box_range(fa, blockIdx.y, b0, b1);
    const double iH = 1.0 / fa.HD;
    const double X = (fa.tgt[3 * j] - fa.c0[0]) * iH, Y = (fa.tgt[3 * j + 1] - fa.c0[1]) * iH,
                 Z = (fa.tgt[3 * j + 2] - fa.c0[2]) * iH;
    const float kf = fa.kf, etaf = fa.etaf, etaif = fa.etaif, kapf = fa.kapf, c4 = fa.c4, iHD = fa.iHD,
                tolu = fa.tolu;
    for (int q0 = 0; q0 < fa.nrhs; q0 += RB) {
        float sr[RB], cr[RB], si[RB], ci[RB];
#pragma unroll
        for (int qq = 0; qq < RB; qq++) sr[qq] = cr[qq] = si[qq] = ci[qq] = 0.f;
        for (int b = b0; b < b1; b++) {
            const double Dx = X - ((double)__ldg(fa.ijk + 3 * b) + 0.5), Dy = Y - ((double)__ldg(fa.ijk + 3 * b + 1) + 0.5),
                         Dz = Z - ((double)__ldg(fa.ijk + 3 * b + 2) + 0.5);
            const double R = sqrt(Dx * Dx + Dy * Dy + Dz * Dz);
            double pc = fa.kap * R;
            pc -= rint(pc);
            const float psi = (float)pc, Rf = (float)R;
            const float dx = (float)Dx, dy = (float)Dy, dz = (float)Dz;
            float pr[RB], pi[RB];
#pragma unroll
            for (int qq = 0; qq < RB; qq++) pr[qq] = pi[qq] = 0.f;
            const int m1 = __ldg(fa.start + b + 1);
            for (int m = __ldg(fa.start + b); m < m1; m++) {
                const float4 f = __ldg(fa.pn32 + 2 * m), nu = __ldg(fa.pn32 + 2 * m + 1);
                const float d0 = dx - f.x, d1 = dy - f.y, d2 = dz - f.z;
                const float r2 = __fmaf_rn(d0, d0, __fmaf_rn(d1, d1, d2 * d2));
                const float ir = rsqrtf(r2);
                const float r = r2 * ir;
                if (!(r >= tolu)) continue;  // coincident pair (or r2 = 0): kernel set to 0
                const float num = __fmaf_rn(-2.f * dx, f.x, __fmaf_rn(-2.f * dy, f.y, __fmaf_rn(-2.f * dz, f.z, f.w)));
                float t = __fmaf_rn(kapf, __fdividef(num, r + Rf), psi);
                t -= rintf(t);
                float sn, cs;
                __sincosf(2.f * kPiF * t, &sn, &cs);
                const float dn = __fmaf_rn(d0, nu.x, __fmaf_rn(d1, nu.y, d2 * nu.z));
                // K = e^{ikR} / (4 pi R) [dn / (r^2 HD) + etai - i (k dn / r + eta)],  R = r HD
                const float A = __fmaf_rn(dn * ir * ir, iHD, etaif), B = -__fmaf_rn(kf * dn, ir, etaf);
                const float amp = c4 * ir;
                const float Kr = amp * __fmaf_rn(cs, A, -sn * B), Ki = amp * __fmaf_rn(sn, A, cs * B);
#pragma unroll
                for (int qq = 0; qq < RB; qq++) {
                    if (RB == 1 || q0 + qq < fa.nrhs) {
                        const float2 am = __ldg(a + (long long)(q0 + qq) * fa.N + m);
                        pr[qq] = __fmaf_rn(Kr, am.x, __fmaf_rn(-Ki, am.y, pr[qq]));
                        pi[qq] = __fmaf_rn(Kr, am.y, __fmaf_rn(Ki, am.x, pi[qq]));
                    }
                }
            }
#pragma unroll
            for (int qq = 0; qq < RB; qq++) {
                comp_add(sr[qq], cr[qq], pr[qq]);
                comp_add(si[qq], ci[qq], pi[qq]);
            }
        }
#pragma unroll
        for (int qq = 0; qq < RB; qq++)
            if (RB == 1 || q0 + qq < fa.nrhs)
                out[((long long)blockIdx.y * fa.nrhs + q0 + qq) * fa.M + j] =
                    make_float2(sr[qq] + cr[qq], si[qq] + ci[qq]);
    }
}

// ---- FP64 forms: absolute coordinates, FP64 phase and accumulation ---------------------
template <bool FAR>
__global__ void __launch_bounds__(kFieldBlock) k_field64(FieldArgs fa, const double2 *__restrict__ a,
                                                         double2 *__restrict__ out) {
    const long long j = blockIdx.x * (long long)kFieldBlock + threadIdx.x;
    if (j >= fa.M) return;
    int b0, b1;
    box_range(fa, blockIdx.y, b0, b1);
    const int m0 = __ldg(fa.start + b0), m1 = __ldg(fa.start + b1);
    const double tx = fa.tgt[3 * j], ty = fa.tgt[3 * j + 1], tz = fa.tgt[3 * j + 2];
    const double k = fa.k, eta = fa.eta, etai = fa.etai, inv4pi = 1.0 / (4.0 * kPi);
    for (int q = 0; q < fa.nrhs; q++) {
        const double2 *aq = a + (long long)q * fa.N;
        double ar = 0.0, ai = 0.0;
        for (int m = m0; m < m1; m++) {
            const double yx = __ldg(fa.x64 + 3 * m), yy = __ldg(fa.x64 + 3 * m + 1), yz = __ldg(fa.x64 + 3 * m + 2);
            const double nx = __ldg(fa.n64 + 3 * m), ny = __ldg(fa.n64 + 3 * m + 1), nz = __ldg(fa.n64 + 3 * m + 2);
            double Kr, Ki;
            if (FAR) {
                // (etai - i (k xhat.nu + eta)) e^{-i k xhat.y} / (4 pi)
                const double tau = k * (tx * nx + ty * ny + tz * nz) + eta;
                double sn, cs;
                sincos(k * (tx * yx + ty * yy + tz * yz), &sn, &cs);
                Kr = (etai * cs - tau * sn) * inv4pi;
                Ki = -(etai * sn + tau * cs) * inv4pi;
            } else {
                const double dx = tx - yx, dy = ty - yy, dz = tz - yz;
                const double r = sqrt(dx * dx + dy * dy + dz * dz);
                if (!(r >= fa.tol)) continue;
                const double dn = dx * nx + dy * ny + dz * nz;
                double sn, cs;
                sincos(k * r, &sn, &cs);
                // e^{ikr} / (4 pi r) [(1 - ikr) dn / r^2 + etai - i eta]
                const double A = dn / (r * r) + etai, B = -(k * dn / r + eta);
                const double amp = inv4pi / r;
                Kr = amp * (cs * A - sn * B);
                Ki = amp * (sn * A + cs * B);
            }
            const double2 am = __ldg(aq + m);
            ar += Kr * am.x - Ki * am.y;
            ai += Kr * am.y + Ki * am.x;
        }
        out[((long long)blockIdx.y * fa.nrhs + q) * fa.M + j] = make_double2(ar, ai);
    }
}

// out[i] = sum over chunks c (in order) of part[c][i], i over nrhs * M (compensated in FP32).
template <typename T>
__global__ void k_field_reduce(long long n, int split, const typename C2T<T>::type *__restrict__ part,
                               typename C2T<T>::type *__restrict__ out) {
    const long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (i >= n) return;
    T sr = 0, cr = 0, si = 0, ci = 0;
    for (int c = 0; c < split; c++) {
        const typename C2T<T>::type v = part[(long long)c * n + i];
        if constexpr (sizeof(T) == 4) {
            comp_add(sr, cr, v.x);
            comp_add(si, ci, v.y);
        } else {
            sr += v.x;
            si += v.y;
        }
    }
    typename C2T<T>::type r;
    r.x = sr + cr;
    r.y = si + ci;
    out[i] = r;
}

// ---- host ------------------------------------------------------------------------------
#define FCK(call)                                                                                 \
    do {                                                                                          \
        cudaError_t e_ = (call);                                                                  \
        if (e_ != cudaSuccess) {                                                                  \
            set_error("%s failed: %s", #call, cudaGetErrorString(e_));                            \
            return IFGF_ECUDA;                                                                    \
        }                                                                                         \
    } while (0)

static ifgf_status field_workspace(Plan &p, size_t bytes) {
    if (p.field_ws && p.field_ws_bytes >= bytes) return IFGF_OK;
    if (p.field_ws) cudaFree(p.field_ws);
    p.field_ws = nullptr;
    p.field_ws_bytes = 0;
    cudaError_t e = cudaMalloc(&p.field_ws, bytes);
    if (e != cudaSuccess) {
        p.field_ws = nullptr;
        set_error("field workspace cudaMalloc(%zu bytes) failed: %s", bytes, cudaGetErrorString(e));
        return e == cudaErrorMemoryAllocation ? IFGF_ENOMEM : IFGF_ECUDA;
    }
    p.field_ws_bytes = bytes;
    return IFGF_OK;
}

// Leaf-box chunks so that about 8 blocks per SM are in flight (at most one chunk per box).
static int field_split(const Plan &p, int64_t M) {
    int sms = 152;
    int dev = 0;
    if (cudaGetDevice(&dev) == cudaSuccess) cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    const int64_t nbm = (M + kFieldBlock - 1) / kFieldBlock;
    const int64_t want = (8LL * sms + nbm - 1) / nbm;
    return (int)std::max<int64_t>(1, std::min<int64_t>({want, (int64_t)kFieldMaxSplit, (int64_t)p.lv[p.D].nbox}));
}

static ifgf_status field_run(ifgf_plan *plan, const void *sigma, const double *tgt, int64_t M, void *out, int nrhs,
                             ifgf_precision prec, void *stream, bool far) {
    clear_error();
    if (!plan) {
        set_error("null plan");
        return IFGF_EINVAL;
    }
    if (nrhs < 0 || M < 0 || M > (int64_t)0x7fffffff - kFieldBlock) {
        set_error("invalid nrhs (%d) or target count (%lld)", nrhs, (long long)M);
        return IFGF_EINVAL;
    }
    if (prec != IFGF_FP64 && prec != IFGF_MIXED) {
        set_error("unknown precision %d", (int)prec);
        return IFGF_EINVAL;
    }
    if (nrhs == 0 || M == 0) return IFGF_OK;
    if (!sigma || !tgt || !out) {
        set_error("null device pointer");
        return IFGF_EINVAL;
    }
    if (out == sigma || (const void *)tgt == out) {
        set_error("out must not alias sigma or the targets");
        return IFGF_EINVAL;
    }
    Plan &p = plan->p;
    cudaStream_t s = (cudaStream_t)stream;
    const int N = (int)p.N, D = p.D;
    const HostLevel &LD = p.lv[D];
    const size_t cb = prec == IFGF_FP64 ? 16 : 8;
    const int split = field_split(p, M);
    auto al = [](size_t x) { return (x + 255) & ~(size_t)255; };
    const size_t abytes = al(cb * (size_t)N * nrhs);
    const size_t pbytes = split > 1 ? cb * (size_t)split * nrhs * (size_t)M : 0;
    ifgf_status st = field_workspace(p, abytes + pbytes);
    if (st != IFGF_OK) return st;
    char *ws = (char *)p.field_ws;
    void *a = ws, *part = split > 1 ? (void *)(ws + abytes) : out;

    FieldArgs fa;
    fa.N = N;
    fa.M = (int)M;
    fa.nrhs = nrhs;
    fa.nbox = LD.nbox;
    fa.split = split;
    fa.k = p.prm.k;
    coupling(p.prm, fa.eta, fa.etai);
    fa.HD = p.HD;
    fa.tol = 1e-14 * p.L;
    for (int i = 0; i < 3; i++) fa.c0[i] = p.c0[i];
    fa.kap = p.prm.k * p.HD / (2.0 * kPi);
    fa.kf = (float)p.prm.k;
    fa.etaf = (float)fa.eta;
    fa.etaif = (float)fa.etai;
    fa.kapf = (float)fa.kap;
    fa.c4 = (float)(1.0 / (4.0 * kPi * p.HD));
    fa.iHD = (float)(1.0 / p.HD);
    fa.tolu = (float)(fa.tol / p.HD);
    fa.ijk = p.dl[D].ijk;
    fa.start = p.dl[D].start;
    fa.x64 = p.d_x64;
    fa.n64 = p.d_n64;
    fa.pn32 = p.d_pn32;
    fa.tgt = tgt;

    const long long NT = (long long)N * nrhs;
    const unsigned gg = (unsigned)((NT + kFieldBlock - 1) / kFieldBlock);
    const dim3 grid((unsigned)((M + kFieldBlock - 1) / kFieldBlock), (unsigned)split);
    if (prec == IFGF_FP64) {
        k_field_gather<double><<<gg, kFieldBlock, 0, s>>>(N, nrhs, p.d_perm, p.d_w64, (const double2 *)sigma,
                                                          (double2 *)a);
        if (far) k_field64<true><<<grid, kFieldBlock, 0, s>>>(fa, (const double2 *)a, (double2 *)part);
        else k_field64<false><<<grid, kFieldBlock, 0, s>>>(fa, (const double2 *)a, (double2 *)part);
    } else {
        k_field_gather<float><<<gg, kFieldBlock, 0, s>>>(N, nrhs, p.d_perm, p.d_w32, (const float2 *)sigma,
                                                         (float2 *)a);
        const float2 *a32 = (const float2 *)a;
        float2 *o32 = (float2 *)part;
        if (far) {
            if (nrhs == 1) k_far32<1><<<grid, kFieldBlock, 0, s>>>(fa, a32, o32);
            else k_far32<kFieldRB><<<grid, kFieldBlock, 0, s>>>(fa, a32, o32);
        } else {
            if (nrhs == 1) k_pot32<1><<<grid, kFieldBlock, 0, s>>>(fa, a32, o32);
            else k_pot32<kFieldRB><<<grid, kFieldBlock, 0, s>>>(fa, a32, o32);
        }
    }
    if (split > 1) {
        const long long n = (long long)nrhs * M;
        const unsigned gr = (unsigned)((n + kFieldBlock - 1) / kFieldBlock);
        if (prec == IFGF_FP64)
            k_field_reduce<double><<<gr, kFieldBlock, 0, s>>>(n, split, (const double2 *)part, (double2 *)out);
        else
            k_field_reduce<float><<<gr, kFieldBlock, 0, s>>>(n, split, (const float2 *)part, (float2 *)out);
    }
    FCK(cudaGetLastError());
    return IFGF_OK;
}

ifgf_status run_apply(Plan &p, const void *sigma, void *y, int nrhs, int prec, cudaStream_t s);
template <int PS, int PA>
ifgf_status run_far_t(Plan &p, const double *xhat, long long M, void *out, int nrhs, int prec, cudaStream_t s);
extern template ifgf_status run_far_t<3, 5>(Plan &, const double *, long long, void *, int, int, cudaStream_t);
extern template ifgf_status run_far_t<4, 6>(Plan &, const double *, long long, void *, int, int, cudaStream_t);
extern template ifgf_status run_far_t<5, 7>(Plan &, const double *, long long, void *, int, int, cudaStream_t);
extern template ifgf_status run_far_t<5, 8>(Plan &, const double *, long long, void *, int, int, cudaStream_t);
extern template ifgf_status run_far_t<6, 8>(Plan &, const double *, long long, void *, int, int, cudaStream_t);

// Far-field pattern through the IFGF factorisation: the upward pass of an apply (leaf
// expansions and propagation into the level-3 cone values), then the s -> 0 evaluation.
static ifgf_status far_ifgf_run(ifgf_plan *plan, const void *sigma, const double *xhat, int64_t M, void *out,
                                int nrhs, ifgf_precision prec, void *stream) {
    clear_error();
    if (!plan) {
        set_error("null plan");
        return IFGF_EINVAL;
    }
    if (nrhs < 0 || M < 0 || M > (int64_t)0x7fffffff) {
        set_error("invalid nrhs (%d) or direction count (%lld)", nrhs, (long long)M);
        return IFGF_EINVAL;
    }
    if (prec != IFGF_FP64 && prec != IFGF_MIXED) {
        set_error("unknown precision %d", (int)prec);
        return IFGF_EINVAL;
    }
    Plan &p = plan->p;
    if (!p.prm.far_field) {
        set_error("the plan was created without params.far_field = 1: its level-3 cone values do not reach s = 0");
        return IFGF_EINVAL;
    }
    if (nrhs == 0 || M == 0) return IFGF_OK;
    if (!sigma || !xhat || !out) {
        set_error("null device pointer");
        return IFGF_EINVAL;
    }
    if (out == sigma || (const void *)xhat == out) {
        set_error("out must not alias sigma or the directions");
        return IFGF_EINVAL;
    }
    cudaStream_t s = (cudaStream_t)stream;
    p.upward_only = true;
    ifgf_status st = run_apply(p, sigma, nullptr, nrhs, (int)prec, s);
    p.upward_only = false;
    if (st != IFGF_OK) return st;
#define IFGF_CASE(a, b) \
    if (p.Ps == a && p.Pang == b) return run_far_t<a, b>(p, xhat, M, out, nrhs, (int)prec, s);
    IFGF_CASE(3, 5)
    IFGF_CASE(4, 6)
    IFGF_CASE(5, 7)
    IFGF_CASE(5, 8)
    IFGF_CASE(6, 8)
#undef IFGF_CASE
    set_error("orders Ps=%d Pang=%d not compiled", p.Ps, p.Pang);
    return IFGF_EUNSUPPORTED;
}

// Potential at the targets of a plan built with targets: the apply over sources and targets with the
// density padded by zeros at the targets (weight 0: they are no sources), the targets' rows copied out.
static ifgf_status field_ifgf_run(ifgf_plan *plan, const void *sigma, void *out, int nrhs, ifgf_precision prec,
                                  void *stream) {
    clear_error();
    if (!plan) {
        set_error("null plan");
        return IFGF_EINVAL;
    }
    if (nrhs < 0) {
        set_error("invalid nrhs (%d)", nrhs);
        return IFGF_EINVAL;
    }
    if (prec != IFGF_FP64 && prec != IFGF_MIXED) {
        set_error("unknown precision %d", (int)prec);
        return IFGF_EINVAL;
    }
    Plan &p = plan->p;
    if (p.n_tgt <= 0) {
        set_error("the plan has no targets: create it with ifgf_plan_create_with_targets");
        return IFGF_EINVAL;
    }
    if (nrhs == 0) return IFGF_OK;
    if (!sigma || !out || sigma == out) {
        set_error("null or aliasing device pointer");
        return IFGF_EINVAL;
    }
    const size_t cb = prec == IFGF_FP64 ? 16 : 8;
    const size_t ns = (size_t)p.n_src, nt = (size_t)p.n_tgt, nall = ns + nt;
    auto al = [](size_t x) { return (x + 255) & ~(size_t)255; };
    const size_t half = al(cb * nall * (size_t)nrhs);
    ifgf_status st = field_workspace(p, 2 * half);
    if (st != IFGF_OK) return st;
    char *pad = (char *)p.field_ws, *yall = pad + half;
    cudaStream_t s = (cudaStream_t)stream;
    cudaError_t e = cudaMemcpy2DAsync(pad, cb * nall, sigma, cb * ns, cb * ns, (size_t)nrhs, cudaMemcpyDeviceToDevice, s);
    if (e == cudaSuccess) e = cudaMemset2DAsync(pad + cb * ns, cb * nall, 0, cb * nt, (size_t)nrhs, s);
    if (e != cudaSuccess) {
        set_error("target density padding: %s", cudaGetErrorString(e));
        return IFGF_ECUDA;
    }
    st = run_apply(p, pad, yall, nrhs, (int)prec, s);
    if (st != IFGF_OK) return st;
    e = cudaMemcpy2DAsync(out, cb * nt, yall + cb * ns, cb * nall, cb * nt, (size_t)nrhs, cudaMemcpyDeviceToDevice, s);
    if (e != cudaSuccess) {
        set_error("target rows: %s", cudaGetErrorString(e));
        return IFGF_ECUDA;
    }
    return IFGF_OK;
}

}  // namespace ifgf

using namespace ifgf;

extern "C" {

ifgf_status ifgf_field(ifgf_plan *plan, const void *sigma_dev, const double *x_dev, int64_t M, void *out_dev,
                       int nrhs, ifgf_precision prec, void *stream) {
    return field_run(plan, sigma_dev, x_dev, M, out_dev, nrhs, prec, stream, false);
}

ifgf_status ifgf_far_field(ifgf_plan *plan, const void *sigma_dev, const double *xhat_dev, int64_t M,
                           void *out_dev, int nrhs, ifgf_precision prec, void *stream) {
    return field_run(plan, sigma_dev, xhat_dev, M, out_dev, nrhs, prec, stream, true);
}

ifgf_status ifgf_field_ifgf(ifgf_plan *plan, const void *sigma_dev, void *out_dev, int nrhs, ifgf_precision prec,
                            void *stream) {
    return field_ifgf_run(plan, sigma_dev, out_dev, nrhs, prec, stream);
}

ifgf_status ifgf_far_field_ifgf(ifgf_plan *plan, const void *sigma_dev, const double *xhat_dev, int64_t M,
                                void *out_dev, int nrhs, ifgf_precision prec, void *stream) {
    return far_ifgf_run(plan, sigma_dev, xhat_dev, M, out_dev, nrhs, prec, stream);
}

}  // extern "C"

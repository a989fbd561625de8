// K8: restarted GMRES(m) for A x = b with the plan's operator (Section 5: the
// complex-arithmetic GMRES of Saad & Schultz used to solve Eq. CombLayIE).
//
// Arnoldi runs on the device in FP64 with classical Gram-Schmidt applied twice
// (CGS2): one batched inner-product kernel and one batched update kernel per
// pass.  The (m+1) x m Hessenberg matrix, its Givens rotations and the small
// triangular solve live on the host in FP64 (a few hundred flops per iteration).
// The operator apply inside is FP64 or mixed; for the mixed apply the Krylov
// vector is rounded to complex64 and the result widened back to complex128.
// Inner products use a fixed grid and a two-stage reduction, so results are
// deterministic run to run.
#include <cmath>
#include <complex>
#include <vector>

#include "ifgf_internal.h"

namespace ifgf {

ifgf_status run_apply(Plan &p, const void *sigma, void *y, int nrhs, int prec, cudaStream_t s);
ifgf_status apply_correction(Plan &p, const void *sigma, void *y, int nrhs, int prec, cudaStream_t s);
void clear_error();

namespace {

constexpr int kDotBlocks = 304;  // 2 x 152 SMs
constexpr int kDotThreads = 256;

// partial[i * kDotBlocks + b] = sum over this block's slice of conj(V_i) w, i = 0..nv-1
__global__ void k_dots_partial(const double2 *__restrict__ V, long long ldv, int nv, const double2 *__restrict__ w,
                               int N, double2 *__restrict__ partial) {
    __shared__ double sr[kDotThreads], si[kDotThreads];
    const int i = blockIdx.y;
    const double2 *v = V + (long long)i * ldv;
    double ar = 0.0, ai = 0.0;
    for (long long n = blockIdx.x * (long long)blockDim.x + threadIdx.x; n < N; n += (long long)gridDim.x * blockDim.x) {
        double2 a = v[n], b = w[n];
        ar += a.x * b.x + a.y * b.y;  // conj(a) * b
        ai += a.x * b.y - a.y * b.x;
    }
    sr[threadIdx.x] = ar;
    si[threadIdx.x] = ai;
    __syncthreads();
    for (int o = blockDim.x / 2; o > 0; o >>= 1) {
        if (threadIdx.x < o) {
            sr[threadIdx.x] += sr[threadIdx.x + o];
            si[threadIdx.x] += si[threadIdx.x + o];
        }
        __syncthreads();
    }
    if (threadIdx.x == 0) partial[(long long)i * gridDim.x + blockIdx.x] = make_double2(sr[0], si[0]);
}

__global__ void k_dots_final(const double2 *__restrict__ partial, int nblocks, int nv, double2 *__restrict__ out) {
    const int i = blockIdx.x;
    if (i >= nv) return;
    __shared__ double sr[kDotThreads], si[kDotThreads];
    double ar = 0.0, ai = 0.0;
    for (int b = threadIdx.x; b < nblocks; b += blockDim.x) {
        double2 p = partial[(long long)i * nblocks + b];
        ar += p.x;
        ai += p.y;
    }
    sr[threadIdx.x] = ar;
    si[threadIdx.x] = ai;
    __syncthreads();
    for (int o = blockDim.x / 2; o > 0; o >>= 1) {
        if (threadIdx.x < o) {
            sr[threadIdx.x] += sr[threadIdx.x + o];
            si[threadIdx.x] += si[threadIdx.x + o];
        }
        __syncthreads();
    }
    if (threadIdx.x == 0) out[i] = make_double2(sr[0], si[0]);
}

// w -= sum_i V_i h_i   (h on the device)
__global__ void k_sub_combination(const double2 *__restrict__ V, long long ldv, int nv, const double2 *__restrict__ h,
                                  double2 *__restrict__ w, int N) {
    long long n = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (n >= N) return;
    double2 acc = w[n];
    for (int i = 0; i < nv; i++) {
        double2 v = V[(long long)i * ldv + n], c = h[i];
        acc.x -= v.x * c.x - v.y * c.y;
        acc.y -= v.x * c.y + v.y * c.x;
    }
    w[n] = acc;
}

// x += sum_i V_i y_i
__global__ void k_add_combination(const double2 *__restrict__ V, long long ldv, int nv, const double2 *__restrict__ y,
                                  double2 *__restrict__ x, int N) {
    long long n = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (n >= N) return;
    double2 acc = x[n];
    for (int i = 0; i < nv; i++) {
        double2 v = V[(long long)i * ldv + n], c = y[i];
        acc.x += v.x * c.x - v.y * c.y;
        acc.y += v.x * c.y + v.y * c.x;
    }
    x[n] = acc;
}

// out = a * x + b * y (complex scalars a, b real here)
__global__ void k_axpby(double a, const double2 *__restrict__ x, double b, const double2 *__restrict__ y,
                        double2 *__restrict__ out, int N) {
    long long n = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (n >= N) return;
    double2 u = x[n], v = y ? y[n] : make_double2(0, 0);
    out[n] = make_double2(a * u.x + b * v.x, a * u.y + b * v.y);
}

__global__ void k_narrow(const double2 *__restrict__ x, float2 *__restrict__ y, int N) {
    long long n = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (n < N) y[n] = make_float2((float)x[n].x, (float)x[n].y);
}

__global__ void k_widen(const float2 *__restrict__ x, double2 *__restrict__ y, int N) {
    long long n = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (n < N) y[n] = make_double2((double)x[n].x, (double)x[n].y);
}

unsigned blocks_for(long long n) { return (unsigned)((n + 255) / 256); }

struct Gm {
    Plan &p;
    cudaStream_t s;
    int N;
    int prec;
    double2 *V = nullptr, *w = nullptr, *partial = nullptr, *hd = nullptr, *tmp = nullptr;
    float2 *v32 = nullptr, *y32 = nullptr;
    long long ldv = 0;
    ifgf_status st = IFGF_OK;

    Gm(Plan &pl, cudaStream_t st_, int prec_) : p(pl), s(st_), N((int)pl.N), prec(prec_) {}

    bool ok(cudaError_t e, const char *what) {
        if (e != cudaSuccess) {
            set_error("%s: %s", what, cudaGetErrorString(e));
            st = e == cudaErrorMemoryAllocation ? IFGF_ENOMEM : IFGF_ECUDA;
            return false;
        }
        return true;
    }

    // y = A x (complex128 in and out)
    bool apply(const double2 *x, double2 *y) {
        if (prec == IFGF_FP64) {
            st = run_apply(p, x, y, 1, IFGF_FP64, s);
            if (st == IFGF_OK) st = apply_correction(p, x, y, 1, IFGF_FP64, s);
        } else {
            k_narrow<<<blocks_for(N), 256, 0, s>>>(x, v32, N);
            st = run_apply(p, v32, y32, 1, IFGF_MIXED, s);
            if (st == IFGF_OK) st = apply_correction(p, v32, y32, 1, IFGF_MIXED, s);
            k_widen<<<blocks_for(N), 256, 0, s>>>(y32, y, N);
        }
        return st == IFGF_OK;
    }

    // h[0..nv-1] = V[0..nv-1]^H w (host copy in hh)
    bool dots(const double2 *Vb, long long ld, int nv, const double2 *x, std::vector<std::complex<double>> &hh) {
        dim3 g(kDotBlocks, nv);
        k_dots_partial<<<g, kDotThreads, 0, s>>>(Vb, ld, nv, x, N, partial);
        k_dots_final<<<nv, kDotThreads, 0, s>>>(partial, kDotBlocks, nv, hd);
        hh.resize(nv);
        if (!ok(cudaMemcpyAsync(hh.data(), hd, sizeof(double2) * nv, cudaMemcpyDeviceToHost, s), "gmres dot copy"))
            return false;
        return ok(cudaStreamSynchronize(s), "gmres sync");
    }

    double norm(const double2 *x) {
        std::vector<std::complex<double>> h;
        if (!dots(x, 0, 1, x, h)) return -1.0;
        return std::sqrt(std::max(h[0].real(), 0.0));
    }
};

}  // namespace
}  // namespace ifgf

using namespace ifgf;

extern "C" ifgf_status ifgf_gmres(ifgf_plan *plan, const void *rhs_dev, void *x_dev, int restart, int maxit, double tol,
                                  ifgf_precision apply_prec, int *iters, double *resid_hist, void *stream) {
    clear_error();
    if (!plan || !rhs_dev || !x_dev || restart < 1 || maxit < 0 || !(tol >= 0)) {
        set_error("invalid GMRES arguments");
        return IFGF_EINVAL;
    }
    if (apply_prec != IFGF_FP64 && apply_prec != IFGF_MIXED) {
        set_error("unknown precision %d", (int)apply_prec);
        return IFGF_EINVAL;
    }
    if (rhs_dev == x_dev) {
        set_error("rhs and x must not alias");
        return IFGF_EINVAL;
    }
    Plan &p = plan->p;
    cudaStream_t s = (cudaStream_t)stream;
    Gm g(p, s, (int)apply_prec);
    const int N = g.N;
    const int m = restart;
    g.ldv = N + (N & 1);
    void *mem = nullptr;
    const size_t vbytes = sizeof(double2) * (size_t)g.ldv * (m + 1);
    const size_t total = vbytes + sizeof(double2) * (size_t)g.ldv * 2 + sizeof(double2) * kDotBlocks * (m + 1) +
                         sizeof(double2) * (m + 1) + sizeof(float2) * (size_t)g.ldv * 2 + 1024;
    if (!g.ok(cudaMalloc(&mem, total), "gmres workspace")) return g.st;
    char *c = (char *)mem;
    g.V = (double2 *)c; c += vbytes;
    g.w = (double2 *)c; c += sizeof(double2) * g.ldv;
    g.tmp = (double2 *)c; c += sizeof(double2) * g.ldv;
    g.partial = (double2 *)c; c += sizeof(double2) * kDotBlocks * (m + 1);
    g.hd = (double2 *)c; c += sizeof(double2) * (m + 1);
    g.v32 = (float2 *)c; c += sizeof(float2) * g.ldv;
    g.y32 = (float2 *)c;
    const double2 *b = (const double2 *)rhs_dev;
    double2 *x = (double2 *)x_dev;
    int it = 0;
    bool converged = false;
    ifgf_status result = IFGF_OK;
    auto fail = [&](ifgf_status stt) {
        cudaFree(mem);
        if (iters) *iters = it;
        return stt;
    };
    const double bnorm = g.norm(b);
    if (bnorm < 0) return fail(g.st);
    if (bnorm == 0.0) {
        k_axpby<<<blocks_for(N), 256, 0, s>>>(0.0, b, 0.0, nullptr, x, N);
        if (resid_hist) resid_hist[0] = 0.0;
        cudaStreamSynchronize(s);
        return fail(IFGF_OK);
    }
    // r = b - A x
    if (!g.apply(x, g.tmp)) return fail(g.st);
    k_axpby<<<blocks_for(N), 256, 0, s>>>(1.0, b, -1.0, g.tmp, g.w, N);
    double beta = g.norm(g.w);
    if (beta < 0) return fail(g.st);
    if (resid_hist) resid_hist[0] = beta / bnorm;
    if (beta / bnorm <= tol) converged = true;
    std::vector<std::complex<double>> H((size_t)(m + 1) * m), gv(m + 1), cs(m), sn(m), h, h2;
    while (!converged && it < maxit) {
        k_axpby<<<blocks_for(N), 256, 0, s>>>(1.0 / beta, g.w, 0.0, nullptr, g.V, N);
        std::fill(gv.begin(), gv.end(), std::complex<double>(0.0));
        gv[0] = beta;
        int j = 0;
        for (; j < m && it < maxit; j++) {
            double2 *vj = g.V + (long long)j * g.ldv;
            if (!g.apply(vj, g.w)) return fail(g.st);
            it++;
            // classical Gram-Schmidt, twice
            if (!g.dots(g.V, g.ldv, j + 1, g.w, h)) return fail(g.st);
            if (!g.ok(cudaMemcpyAsync(g.hd, h.data(), sizeof(double2) * (j + 1), cudaMemcpyHostToDevice, s), "h copy"))
                return fail(g.st);
            k_sub_combination<<<blocks_for(N), 256, 0, s>>>(g.V, g.ldv, j + 1, g.hd, g.w, N);
            if (!g.dots(g.V, g.ldv, j + 1, g.w, h2)) return fail(g.st);
            if (!g.ok(cudaMemcpyAsync(g.hd, h2.data(), sizeof(double2) * (j + 1), cudaMemcpyHostToDevice, s), "h copy"))
                return fail(g.st);
            k_sub_combination<<<blocks_for(N), 256, 0, s>>>(g.V, g.ldv, j + 1, g.hd, g.w, N);
            for (int i = 0; i <= j; i++) H[(size_t)i * m + j] = h[i] + h2[i];
            double hn = g.norm(g.w);
            if (hn < 0) return fail(g.st);
            H[(size_t)(j + 1) * m + j] = hn;
            // previous rotations, then a new one zeroing H[j+1][j]
            for (int i = 0; i < j; i++) {
                std::complex<double> a = H[(size_t)i * m + j], bb = H[(size_t)(i + 1) * m + j];
                H[(size_t)i * m + j] = std::conj(cs[i]) * a + std::conj(sn[i]) * bb;
                H[(size_t)(i + 1) * m + j] = -sn[i] * a + cs[i] * bb;
            }
            std::complex<double> a = H[(size_t)j * m + j], bb = H[(size_t)(j + 1) * m + j];
            double den = std::sqrt(std::norm(a) + std::norm(bb));
            if (den == 0.0) {
                cs[j] = 1.0;
                sn[j] = 0.0;
            } else {
                cs[j] = a / den;
                sn[j] = bb / den;
            }
            H[(size_t)j * m + j] = den;
            H[(size_t)(j + 1) * m + j] = 0.0;
            gv[j + 1] = -sn[j] * gv[j];
            gv[j] = std::conj(cs[j]) * gv[j];
            const double res = std::abs(gv[j + 1]) / bnorm;
            if (resid_hist) resid_hist[it] = res;
            if (res <= tol) converged = true;
            if (converged || hn == 0.0) {
                j++;
                break;
            }
            k_axpby<<<blocks_for(N), 256, 0, s>>>(1.0 / hn, g.w, 0.0, nullptr, g.V + (long long)(j + 1) * g.ldv, N);
        }
        // y = H^{-1} g (upper triangular j x j); x += V y
        std::vector<std::complex<double>> y(j);
        for (int i = j - 1; i >= 0; i--) {
            std::complex<double> acc = gv[i];
            for (int l = i + 1; l < j; l++) acc -= H[(size_t)i * m + l] * y[l];
            y[i] = acc / H[(size_t)i * m + i];
        }
        if (j > 0) {
            if (!g.ok(cudaMemcpyAsync(g.hd, y.data(), sizeof(double2) * j, cudaMemcpyHostToDevice, s), "y copy"))
                return fail(g.st);
            k_add_combination<<<blocks_for(N), 256, 0, s>>>(g.V, g.ldv, j, g.hd, x, N);
        }
        if (converged || it >= maxit) break;
        // restart from the true residual
        if (!g.apply(x, g.tmp)) return fail(g.st);
        k_axpby<<<blocks_for(N), 256, 0, s>>>(1.0, b, -1.0, g.tmp, g.w, N);
        beta = g.norm(g.w);
        if (beta < 0) return fail(g.st);
        if (beta / bnorm <= tol) converged = true;
    }
    if (!g.ok(cudaStreamSynchronize(s), "gmres final sync")) return fail(g.st);
    if (!g.ok(cudaGetLastError(), "gmres kernels")) return fail(g.st);
    if (!converged) {
        set_error("GMRES: relative residual above %.3g after %d iterations", tol, it);
        result = IFGF_ENOTCONVERGED;
    }
    return fail(result);
}

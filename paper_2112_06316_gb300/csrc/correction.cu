// K5: sparse singular / near-singular correction y += C sigma (Eq. IntOpAtSing).
//
// The host precomputes C (rectangular-polar rows minus the regular-quadrature
// rows they replace); the GPU applies it as a complex CSR product over the
// caller's point order.  One warp per row: lanes stride over the row's
// entries (coalesced col/val reads), then a shuffle reduction.
#include <cmath>
#include <vector>

#include "ifgf_internal.h"
#include "kernels.cuh"

namespace ifgf {

template <typename T>
__global__ void k_spmv(int N, int nrhs, const long long *__restrict__ rowptr, const int *__restrict__ col,
                       const typename C2T<T>::type *__restrict__ val, const typename C2T<T>::type *__restrict__ sigma,
                       typename C2T<T>::type *__restrict__ y) {
    long long gw = (blockIdx.x * (long long)blockDim.x + threadIdx.x) >> 5;
    int lane = threadIdx.x & 31;
    if (gw >= N) return;
    const long long j0 = rowptr[gw], j1 = rowptr[gw + 1];
    for (int q = 0; q < nrhs; q++) {
        const typename C2T<T>::type *sq = sigma + (long long)q * N;
        T ar = 0, ai = 0;
        // four entries per lane in flight: the value and column loads of all four are issued before
        // the dependent density loads (the row is ~600 entries long, bound by memory latency)
        long long j = j0 + lane;
        for (; j + 96 < j1; j += 128) {
            typename C2T<T>::type v[4], sv[4];
            int cl[4];
#pragma unroll
            for (int u = 0; u < 4; u++) {
                v[u] = __ldg(val + j + 32 * u);
                cl[u] = __ldg(col + j + 32 * u);
            }
#pragma unroll
            for (int u = 0; u < 4; u++) sv[u] = __ldg(sq + cl[u]);
#pragma unroll
            for (int u = 0; u < 4; u++) {
                ar += v[u].x * sv[u].x - v[u].y * sv[u].y;
                ai += v[u].x * sv[u].y + v[u].y * sv[u].x;
            }
        }
        for (; j < j1; j += 32) {
            const typename C2T<T>::type v = __ldg(val + j), sv = __ldg(sq + __ldg(col + j));
            ar += v.x * sv.x - v.y * sv.y;
            ai += v.x * sv.y + v.y * sv.x;
        }
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            ar += __shfl_down_sync(0xffffffffu, ar, o);
            ai += __shfl_down_sync(0xffffffffu, ai, o);
        }
        if (lane == 0) {
            typename C2T<T>::type yy = y[(long long)q * N + gw];
            yy.x += ar;
            yy.y += ai;
            y[(long long)q * N + gw] = yy;
        }
    }
}

static void free_correction(Plan &p) {
    for (void *q : {(void *)p.d_corrT_rowptr, (void *)p.d_corrT_col, (void *)p.d_corrT_val64, (void *)p.d_corrT_val32})
        if (q) cudaFree(q);
    p.d_corrT_rowptr = nullptr;
    p.d_corrT_col = nullptr;
    p.d_corrT_val64 = nullptr;
    p.d_corrT_val32 = nullptr;
    if (p.d_corr_rowptr) cudaFree(p.d_corr_rowptr);
    if (p.d_corr_col) cudaFree(p.d_corr_col);
    if (p.d_corr_val64) cudaFree(p.d_corr_val64);
    if (p.d_corr_val32) cudaFree(p.d_corr_val32);
    p.d_corr_rowptr = nullptr;
    p.d_corr_col = nullptr;
    p.d_corr_val64 = nullptr;
    p.d_corr_val32 = nullptr;
    p.corr_nnz = 0;
}

ifgf_status set_correction(Plan &p, const int64_t *rowptr, const int32_t *col, const double *val, int64_t nnz) {
    p.gen++;
    if (nnz == 0) {
        free_correction(p);
        return IFGF_OK;
    }
    if (nnz < 0 || !rowptr || !col || !val) {
        set_error("invalid correction arrays");
        return IFGF_EINVAL;
    }
    const int64_t N = p.N;
    if (rowptr[0] != 0 || rowptr[N] != nnz) {
        set_error("rowptr[0] must be 0 and rowptr[N] == nnz");
        return IFGF_EINVAL;
    }
    for (int64_t i = 0; i < N; i++)
        if (rowptr[i + 1] < rowptr[i]) {
            set_error("rowptr not monotone at row %lld", (long long)i);
            return IFGF_EINVAL;
        }
    std::vector<float> v32(2 * nnz);
    for (int64_t j = 0; j < nnz; j++) {
        if (col[j] < 0 || col[j] >= N) {
            set_error("correction column %d out of range at entry %lld", col[j], (long long)j);
            return IFGF_EINVAL;
        }
        if (!std::isfinite(val[2 * j]) || !std::isfinite(val[2 * j + 1])) {
            set_error("non-finite correction value at entry %lld", (long long)j);
            return IFGF_EINVAL;
        }
        v32[2 * j] = (float)val[2 * j];
        v32[2 * j + 1] = (float)val[2 * j + 1];
    }
    free_correction(p);
    cudaError_t e = cudaMalloc(&p.d_corr_rowptr, sizeof(int64_t) * (N + 1));
    if (e == cudaSuccess) e = cudaMalloc(&p.d_corr_col, sizeof(int) * nnz);
    if (e == cudaSuccess) e = cudaMalloc(&p.d_corr_val64, sizeof(double) * 2 * nnz);
    if (e == cudaSuccess) e = cudaMalloc(&p.d_corr_val32, sizeof(float) * 2 * nnz);
    if (e == cudaSuccess) e = cudaMemcpy(p.d_corr_rowptr, rowptr, sizeof(int64_t) * (N + 1), cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemcpy(p.d_corr_col, col, sizeof(int) * nnz, cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemcpy(p.d_corr_val64, val, sizeof(double) * 2 * nnz, cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemcpy(p.d_corr_val32, v32.data(), sizeof(float) * 2 * nnz, cudaMemcpyHostToDevice);
    // conjugate transpose for the adjoint: row j of C^H holds conj(C[i][j]) at column i
    std::vector<int64_t> trp(N + 1, 0);
    for (int64_t j = 0; j < nnz; j++) trp[col[j] + 1]++;
    for (int64_t i = 0; i < N; i++) trp[i + 1] += trp[i];
    std::vector<int> tcol(nnz);
    std::vector<double> tv64(2 * nnz);
    std::vector<float> tv32(2 * nnz);
    {
        std::vector<int64_t> fill(trp.begin(), trp.end() - 1);
        for (int64_t i = 0; i < N; i++)
            for (int64_t j = rowptr[i]; j < rowptr[i + 1]; j++) {
                int64_t o = fill[col[j]]++;
                tcol[o] = (int)i;
                tv64[2 * o] = val[2 * j];
                tv64[2 * o + 1] = -val[2 * j + 1];
                tv32[2 * o] = (float)val[2 * j];
                tv32[2 * o + 1] = -(float)val[2 * j + 1];
            }
    }
    if (e == cudaSuccess) e = cudaMalloc(&p.d_corrT_rowptr, sizeof(int64_t) * (N + 1));
    if (e == cudaSuccess) e = cudaMalloc(&p.d_corrT_col, sizeof(int) * nnz);
    if (e == cudaSuccess) e = cudaMalloc(&p.d_corrT_val64, sizeof(double) * 2 * nnz);
    if (e == cudaSuccess) e = cudaMalloc(&p.d_corrT_val32, sizeof(float) * 2 * nnz);
    if (e == cudaSuccess) e = cudaMemcpy(p.d_corrT_rowptr, trp.data(), sizeof(int64_t) * (N + 1), cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemcpy(p.d_corrT_col, tcol.data(), sizeof(int) * nnz, cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemcpy(p.d_corrT_val64, tv64.data(), sizeof(double) * 2 * nnz, cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemcpy(p.d_corrT_val32, tv32.data(), sizeof(float) * 2 * nnz, cudaMemcpyHostToDevice);
    if (e != cudaSuccess) {
        free_correction(p);
        set_error("correction upload failed: %s", cudaGetErrorString(e));
        return e == cudaErrorMemoryAllocation ? IFGF_ENOMEM : IFGF_ECUDA;
    }
    p.corr_nnz = nnz;
    return IFGF_OK;
}

// y += C^H g (conjugate-transposed correction)
ifgf_status apply_correction_adjoint(Plan &p, const void *g, void *y, int nrhs, int prec, cudaStream_t s) {
    if (p.corr_nnz == 0) return IFGF_OK;
    const int N = (int)p.N;
    const unsigned blocks = (unsigned)(((long long)N * 32 + 127) / 128);
    if (prec == IFGF_FP64)
        k_spmv<double><<<blocks, 128, 0, s>>>(N, nrhs, (const long long *)p.d_corrT_rowptr, p.d_corrT_col,
                                              (const double2 *)p.d_corrT_val64, (const double2 *)g, (double2 *)y);
    else
        k_spmv<float><<<blocks, 128, 0, s>>>(N, nrhs, (const long long *)p.d_corrT_rowptr, p.d_corrT_col,
                                             (const float2 *)p.d_corrT_val32, (const float2 *)g, (float2 *)y);
    prof_mark(p, s, kStCorr, 0);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) {
        set_error("correction-adjoint kernel launch failed: %s", cudaGetErrorString(e));
        return IFGF_ECUDA;
    }
    return IFGF_OK;
}

ifgf_status apply_correction(Plan &p, const void *sigma, void *y, int nrhs, int prec, cudaStream_t s) {
    if (p.corr_nnz == 0) return IFGF_OK;
    const int N = (int)p.N;
    const unsigned blocks = (unsigned)(((long long)N * 32 + 127) / 128);
    if (prec == IFGF_FP64)
        k_spmv<double><<<blocks, 128, 0, s>>>(N, nrhs, (const long long *)p.d_corr_rowptr, p.d_corr_col,
                                              (const double2 *)p.d_corr_val64, (const double2 *)sigma, (double2 *)y);
    else
        k_spmv<float><<<blocks, 128, 0, s>>>(N, nrhs, (const long long *)p.d_corr_rowptr, p.d_corr_col,
                                             (const float2 *)p.d_corr_val32, (const float2 *)sigma, (float2 *)y);
    prof_mark(p, s, kStCorr, 0);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) {
        set_error("correction kernel launch failed: %s", cudaGetErrorString(e));
        return IFGF_ECUDA;
    }
    return IFGF_OK;
}

}  // namespace ifgf

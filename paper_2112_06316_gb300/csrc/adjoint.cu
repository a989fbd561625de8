// Host side of the adjoint apply A^H g (conjugate transpose of the discrete
// operator, including the correction): builds the anterpolation lists on the
// first call, manages the adjoint workspace and dispatches over the compiled
// interpolation orders (kernels in fwd_kernels.cuh).
#include <cmath>
#include <vector>

#include "ifgf_internal.h"

namespace ifgf {

template <int PS, int PA>
ifgf_status run_adjoint_t(Plan &p, const void *g, void *out, int nrhs, int prec, cudaStream_t s, void *gs, void *bws,
                          void **G);
extern template ifgf_status run_adjoint_t<3, 5>(Plan &, const void *, void *, int, int, cudaStream_t, void *, void *, void **);
extern template ifgf_status run_adjoint_t<4, 6>(Plan &, const void *, void *, int, int, cudaStream_t, void *, void *, void **);
extern template ifgf_status run_adjoint_t<5, 7>(Plan &, const void *, void *, int, int, cudaStream_t, void *, void *, void **);
extern template ifgf_status run_adjoint_t<5, 8>(Plan &, const void *, void *, int, int, cudaStream_t, void *, void *, void **);
extern template ifgf_status run_adjoint_t<6, 8>(Plan &, const void *, void *, int, int, cudaStream_t, void *, void *, void **);
ifgf_status apply_correction_adjoint(Plan &p, const void *g, void *y, int nrhs, int prec, cudaStream_t s);
void clear_error();

static ifgf_status cuda_fail(cudaError_t e, const char *what) {
    set_error("%s: %s", what, cudaGetErrorString(e));
    return e == cudaErrorMemoryAllocation ? IFGF_ENOMEM : IFGF_ECUDA;
}

// Anterpolation lists per level (host build, then upload); once per plan.
static ifgf_status ensure_adjoint_lists(Plan &p, cudaStream_t s) {
    if (p.adj_ready) return IFGF_OK;
    if ((int64_t)p.N + (int64_t)p.lv[p.D].nrc * p.P >= (int64_t)0x7fffffff) {
        set_error("adjoint lists exceed 32-bit entry range");
        return IFGF_EUNSUPPORTED;
    }
    ifgf_status st = build_adjoint_lists(p, p.xs.data());
    if (st != IFGF_OK) return st;
    for (int d = 3; d <= p.D; d++) {
        HostLevel &L = p.lv[d];
        void *a = nullptr, *b = nullptr;
        cudaError_t e = cudaMalloc(&a, sizeof(int64_t) * L.ad_start.size());
        if (e == cudaSuccess) e = cudaMalloc(&b, sizeof(int) * (L.ad_list.size() + 1));
        if (e != cudaSuccess) return cuda_fail(e, "adjoint list allocation");
        p.allocs.push_back(a);
        p.allocs.push_back(b);
        p.device_bytes += (int64_t)(sizeof(int64_t) * L.ad_start.size() + sizeof(int) * (L.ad_list.size() + 1));
        e = cudaMemcpyAsync(a, L.ad_start.data(), sizeof(int64_t) * L.ad_start.size(), cudaMemcpyHostToDevice, s);
        if (e == cudaSuccess && !L.ad_list.empty())
            e = cudaMemcpyAsync(b, L.ad_list.data(), sizeof(int) * L.ad_list.size(), cudaMemcpyHostToDevice, s);
        if (e == cudaSuccess) e = cudaStreamSynchronize(s);
        if (e != cudaSuccess) return cuda_fail(e, "adjoint list upload");
        p.d_ad_start[d] = (int64_t *)a;
        p.d_ad_list[d] = (int *)b;
        std::vector<int64_t>().swap(L.ad_start);
        std::vector<int>().swap(L.ad_list);
    }
    p.adj_ready = true;
    return IFGF_OK;
}

}  // namespace ifgf

using namespace ifgf;

extern "C" ifgf_status ifgf_apply_adjoint(ifgf_plan *plan, const void *g_dev, void *out_dev, int nrhs,
                                          ifgf_precision prec, void *stream) {
    clear_error();
    if (!plan) {
        set_error("null plan");
        return IFGF_EINVAL;
    }
    if (nrhs < 0 || (nrhs > 0 && (!g_dev || !out_dev))) {
        set_error("invalid nrhs or null device pointer");
        return IFGF_EINVAL;
    }
    if (prec != IFGF_FP64 && prec != IFGF_MIXED) {
        set_error("unknown precision %d", (int)prec);
        return IFGF_EINVAL;
    }
    if (nrhs == 0) return IFGF_OK;
    if (g_dev == out_dev) {
        set_error("g and out must not alias");
        return IFGF_EINVAL;
    }
    Plan &p = plan->p;
    cudaStream_t s = (cudaStream_t)stream;
    ifgf_status st = ensure_adjoint_lists(p, s);
    if (st != IFGF_OK) return st;
    // workspace: gs [nrhs][N], b [nrhs][N], G of levels 3..D
    const size_t cb = prec == IFGF_FP64 ? 16 : 8;
    auto al = [](size_t x) { return (x + 255) & ~(size_t)255; };
    size_t off = 0, ogs = 0, ob = 0, oG[IFGF_MAXD + 1] = {};
    ogs = off; off += al(cb * p.N * nrhs);
    ob = off; off += al(cb * p.N * nrhs);
    for (int d = 3; d <= p.D; d++) {
        oG[d] = off;
        off += al(cb * (size_t)nrhs * p.lv[d].nrc * p.lv[d].nfac * p.Pstride);
    }
    if (off > p.adj_ws_bytes) {
        if (p.adj_ws) cudaFree(p.adj_ws);
        p.adj_ws = nullptr;
        p.adj_ws_bytes = 0;
        cudaError_t e = cudaMalloc(&p.adj_ws, off);
        if (e != cudaSuccess) return cuda_fail(e, "adjoint workspace");
        p.adj_ws_bytes = off;
    }
    char *c = (char *)p.adj_ws;
    void *G[IFGF_MAXD + 1] = {};
    for (int d = 3; d <= p.D; d++) G[d] = c + oG[d];
#define IFGF_ADJ(a, b)                                                                                  \
    else if (p.Ps == a && p.Pang == b) st = run_adjoint_t<a, b>(p, g_dev, out_dev, nrhs, (int)prec, s, c + ogs, c + ob, G);
    if (false) {
    }
    IFGF_ADJ(3, 5) IFGF_ADJ(4, 6) IFGF_ADJ(5, 7) IFGF_ADJ(5, 8) IFGF_ADJ(6, 8)
    else {
        set_error("orders Ps=%d Pang=%d not compiled", p.Ps, p.Pang);
        return IFGF_EUNSUPPORTED;
    }
#undef IFGF_ADJ
    if (st != IFGF_OK) return st;
    return apply_correction_adjoint(p, g_dev, out_dev, nrhs, (int)prec, s);
}

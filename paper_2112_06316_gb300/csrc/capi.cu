// C ABI entry points (declared in include/ifgf.h).
#include <algorithm>
#include <cmath>
#include <cstring>
#include <new>
#include <vector>

#include "ifgf_internal.h"

namespace ifgf {
const char *last_error_str();
void clear_error();
ifgf_status apply_correction(Plan &p, const void *sigma, void *y, int nrhs, int prec, cudaStream_t s);
ifgf_status set_correction(Plan &p, const int64_t *rowptr, const int32_t *col, const double *val, int64_t nnz);
}  // namespace ifgf

using namespace ifgf;

static bool supported_pair(int ps, int pa) {
    return (ps == 3 && pa == 5) || (ps == 4 && pa == 6) || (ps == 5 && pa == 7) || (ps == 5 && pa == 8) || (ps == 6 && pa == 8);
}

extern "C" {

void ifgf_params_default(ifgf_params *p, double k) {
    std::memset(p, 0, sizeof(*p));
    p->k = k;
    p->eta = k;
    p->Ps = 3;
    p->Pang = 5;
    p->nC0 = 2;
    p->nS0 = 1;
    p->levels = 0;
    p->leaf_target = 64.0;
    p->cone_rule = 0;
    p->factor_mode = 0;
    p->identity_coef = 0.5;
    p->root_side = 0.0;
    p->cone_band = 1e-4;
    p->far_field = 0;
    p->layer = IFGF_LAYER_COMBINED;
    p->leaf_max = 0;
}

const char *ifgf_supported_orders(void) { return "3x5,4x6,5x7,5x8,6x8"; }

const char *ifgf_last_error(void) { return last_error_str(); }

static ifgf_status validate(const double *xyz, const double *normals, const double *weights, int64_t N,
                            const ifgf_params *params) {
    if (!params) {
        set_error("null params pointer");
        return IFGF_EINVAL;
    }
    if (N < 1 || N > (int64_t)0x7fffffff) {
        set_error("N must be in 1..2^31-1 (got %lld)", (long long)N);
        return IFGF_EINVAL;
    }
    if (!xyz || !normals || !weights) {
        set_error("null input array");
        return IFGF_EINVAL;
    }
    const ifgf_params &pr = *params;
    if (!(pr.k > 0) || !std::isfinite(pr.k) || !std::isfinite(pr.eta)) {
        set_error("k must be finite and > 0, eta finite");
        return IFGF_EINVAL;
    }
    if (pr.levels != 0 && (pr.levels < 3 || pr.levels > 16)) {
        set_error("levels must be 0 (auto) or in 3..16");
        return IFGF_EINVAL;
    }
    if (pr.nC0 < 1 || pr.nS0 < 1 || pr.nC0 > 64 || pr.nS0 > 64 || pr.cone_rule < 0 || pr.cone_rule > 1 ||
        pr.factor_mode < 0 || pr.factor_mode > 2 || !(pr.cone_band >= 0) || !std::isfinite(pr.identity_coef) ||
        pr.far_field < 0 || pr.far_field > 1 || pr.layer < IFGF_LAYER_COMBINED || pr.layer > IFGF_LAYER_SINGLE ||
        pr.leaf_max < 0) {
        set_error("invalid cone, factor, far-field, layer or leaf_max parameters");
        return IFGF_EINVAL;
    }
    if (!supported_pair(pr.Ps, pr.Pang)) {
        set_error("interpolation orders Ps=%d Pang=%d not compiled (supported: %s)", pr.Ps, pr.Pang,
                  ifgf_supported_orders());
        return IFGF_EUNSUPPORTED;
    }
    for (int64_t i = 0; i < N; i++) {
        double nn = 0;
        for (int a = 0; a < 3; a++) {
            if (!std::isfinite(xyz[3 * i + a]) || !std::isfinite(normals[3 * i + a])) {
                set_error("non-finite point or normal at index %lld", (long long)i);
                return IFGF_EINVAL;
            }
            nn += normals[3 * i + a] * normals[3 * i + a];
        }
        if (std::fabs(std::sqrt(nn) - 1.0) > 1e-6) {
            set_error("normal %lld is not unit length (|n| = %.17g)", (long long)i, std::sqrt(nn));
            return IFGF_EINVAL;
        }
        if (!(weights[i] > 0) || !std::isfinite(weights[i])) {
            set_error("weight %lld must be finite and > 0", (long long)i);
            return IFGF_EINVAL;
        }
    }
    return IFGF_OK;
}

static void init_plan(Plan &p, const ifgf_params &pr, int64_t N) {
    p.prm = pr;
    p.N = N;
    p.Ps = pr.Ps;
    p.Pang = pr.Pang;
    p.P = pr.Ps * pr.Pang * pr.Pang;
    p.Pstride = p.P + (p.P & 1);
}

static void fill_info(const Plan &p, ifgf_info *out) {
    std::memset(out, 0, sizeof(*out));
    out->N = p.N;
    out->D = p.D;
    for (int a = 0; a < 3; a++) out->root_center[a] = p.center[a];
    out->root_side = p.L;
    for (int d = 1; d <= p.D; d++) {
        const HostLevel &L = p.lv[d];
        out->nbox[d] = L.nbox;
        out->ns[d] = L.ns;
        out->nC[d] = L.nC;
        out->split[d] = L.split;
        out->nrc[d] = L.nrc;
        out->cousin_evals[d] = L.cousin_evals;
        out->prop_evals[d] = L.prop_evals;
    }
    out->leaf_evals = p.leaf_evals;
    out->near_pairs = p.near_pairs;
    out->correction_nnz = p.corr_nnz;
    out->device_bytes = p.device_bytes;
    out->near_block_chunks = p.adaptive ? p.nnchunk - p.nnchunk_light : 0;
}

ifgf_status ifgf_plan_dry_run(const double *xyz, const double *normals, const double *weights, int64_t N,
                              const ifgf_params *params, ifgf_info *out) {
    clear_error();
    if (!out) {
        set_error("null output pointer");
        return IFGF_EINVAL;
    }
    ifgf_status st = validate(xyz, normals, weights, N, params);
    if (st != IFGF_OK) return st;
    Plan p;
    init_plan(p, *params, N);
    try {
        st = build_host_plan(p, xyz, normals, weights);
    } catch (const std::bad_alloc &) {
        set_error("host allocation failed while building the plan");
        st = IFGF_ENOMEM;
    }
    if (st == IFGF_OK) fill_info(p, out);
    return st;
}

// Octree, cone structure and device upload of a validated point set.
static ifgf_status create_plan(const double *xyz, const double *normals, const double *weights, int64_t N,
                               const ifgf_params &pr, void *stream, ifgf_plan **out, int64_t n_src = 0) {
    ifgf_plan *pl = new (std::nothrow) ifgf_plan();
    if (!pl) {
        set_error("host allocation failed");
        return IFGF_ENOMEM;
    }
    Plan &p = pl->p;
    init_plan(p, pr, N);
    p.n_src = n_src;
    p.n_tgt = n_src > 0 ? N - n_src : 0;
    ifgf_status st;
    try {
        st = build_host_plan(p, xyz, normals, weights);
        if (st == IFGF_OK) st = build_cousin_lists(p);
    } catch (const std::bad_alloc &) {
        set_error("host allocation failed while building the plan");
        st = IFGF_ENOMEM;
    }
    if (st == IFGF_OK) st = upload_plan(p, xyz, normals, weights, (cudaStream_t)stream);
    if (st != IFGF_OK) {
        free_plan_device(p);
        delete pl;
        return st;
    }
    *out = pl;
    return IFGF_OK;
}

ifgf_status ifgf_plan_create(const double *xyz, const double *normals, const double *weights, int64_t N,
                             const ifgf_params *params, void *stream, ifgf_plan **out) {
    clear_error();
    if (out) *out = nullptr;
    if (!out) {
        set_error("null output pointer");
        return IFGF_EINVAL;
    }
    ifgf_status vst = validate(xyz, normals, weights, N, params);
    if (vst != IFGF_OK) return vst;
    return create_plan(xyz, normals, weights, N, *params, stream, out);
}

ifgf_status ifgf_plan_create_with_targets(const double *xyz, const double *normals, const double *weights, int64_t N,
                                          const double *targets, int64_t M, const ifgf_params *params, void *stream,
                                          ifgf_plan **out) {
    clear_error();
    if (out) *out = nullptr;
    if (!out) {
        set_error("null output pointer");
        return IFGF_EINVAL;
    }
    ifgf_status vst = validate(xyz, normals, weights, N, params);
    if (vst != IFGF_OK) return vst;
    if (M < 1 || !targets || N + M > (int64_t)0x7fffffff) {
        set_error("targets: need 1 <= M and N + M <= 2^31 - 1, and a target array (M = %lld)", (long long)M);
        return IFGF_EINVAL;
    }
    for (int64_t i = 0; i < 3 * M; i++)
        if (!std::isfinite(targets[i])) {
            set_error("non-finite target coordinate at index %lld", (long long)(i / 3));
            return IFGF_EINVAL;
        }
    std::vector<double> x, n, w;
    try {
        x.resize(3 * (size_t)(N + M));
        n.assign(3 * (size_t)(N + M), 0.0);
        w.assign((size_t)(N + M), 0.0);
    } catch (const std::bad_alloc &) {
        set_error("host allocation failed");
        return IFGF_ENOMEM;
    }
    std::copy(xyz, xyz + 3 * N, x.begin());
    std::copy(targets, targets + 3 * M, x.begin() + 3 * N);
    std::copy(normals, normals + 3 * N, n.begin());
    std::copy(weights, weights + N, w.begin());
    return create_plan(x.data(), n.data(), w.data(), N + M, *params, stream, out, N);
}

void ifgf_plan_destroy(ifgf_plan *plan) {
    if (!plan) return;
    set_correction(plan->p, nullptr, nullptr, nullptr, 0);
    free_plan_device(plan->p);
    delete plan;
}

ifgf_status ifgf_apply(ifgf_plan *plan, const void *sigma_dev, void *y_dev, int nrhs, ifgf_precision prec,
                       void *stream) {
    clear_error();
    if (!plan) {
        set_error("null plan");
        return IFGF_EINVAL;
    }
    if (nrhs < 0 || (nrhs > 0 && (!sigma_dev || !y_dev))) {
        set_error("invalid nrhs or null device pointer");
        return IFGF_EINVAL;
    }
    if (prec != IFGF_FP64 && prec != IFGF_MIXED) {
        set_error("unknown precision %d", (int)prec);
        return IFGF_EINVAL;
    }
    if (nrhs == 0) return IFGF_OK;
    if (sigma_dev == y_dev) {
        set_error("sigma and y must not alias");
        return IFGF_EINVAL;
    }
    Plan &p = plan->p;
    cudaStream_t s = (cudaStream_t)stream;
    ifgf_status st = run_apply(p, sigma_dev, y_dev, nrhs, (int)prec, s);
    if (st != IFGF_OK) return st;
    return apply_correction(p, sigma_dev, y_dev, nrhs, (int)prec, s);
}

ifgf_status ifgf_plan_set_correction(ifgf_plan *plan, const int64_t *rowptr, const int32_t *col, const double *val,
                                     int64_t nnz) {
    clear_error();
    if (!plan) {
        set_error("null plan");
        return IFGF_EINVAL;
    }
    return set_correction(plan->p, rowptr, col, val, nnz);
}

ifgf_status ifgf_plan_info(const ifgf_plan *plan, ifgf_info *out) {
    clear_error();
    if (!plan || !out) {
        set_error("null plan or output");
        return IFGF_EINVAL;
    }
    fill_info(plan->p, out);
    return IFGF_OK;
}

ifgf_status ifgf_plan_check(ifgf_plan *plan, void *stream, int64_t *missed_lookups) {
    clear_error();
    if (!plan || !missed_lookups) {
        set_error("null plan or output");
        return IFGF_EINVAL;
    }
    unsigned long long h = 0;
    cudaStream_t s = (cudaStream_t)stream;
    cudaError_t e = cudaMemcpyAsync(&h, plan->p.d_missed, sizeof(h), cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaMemsetAsync(plan->p.d_missed, 0, sizeof(h), s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) {
        set_error("ifgf_plan_check: %s", cudaGetErrorString(e));
        return IFGF_ECUDA;
    }
    *missed_lookups = (int64_t)h;
    return IFGF_OK;
}

ifgf_status ifgf_plan_set_rhs_block(ifgf_plan *plan, int rhs_block) {
    clear_error();
    if (!plan || (rhs_block != 1 && rhs_block != 4)) {
        set_error("rhs_block must be 1 or 4");
        return IFGF_EINVAL;
    }
    // the setting decides which kernels a captured group graph holds: a change forces a recapture
    if (plan->p.rhs_block != rhs_block) plan->p.gen++;
    plan->p.rhs_block = rhs_block;
    return IFGF_OK;
}

ifgf_status ifgf_plan_set_tc_fill(ifgf_plan *plan, double min_fill) {
    clear_error();
    if (!plan || !(min_fill >= 0)) {
        set_error("min_fill must be >= 0");
        return IFGF_EINVAL;
    }
    if (plan->p.tc_min_fill != min_fill) plan->p.gen++;
    plan->p.tc_min_fill = min_fill;
    return IFGF_OK;
}

ifgf_status ifgf_plan_set_tc_engine(ifgf_plan *plan, int engine) {
    clear_error();
    if (!plan || engine < 0 || engine > 2) {
        set_error("engine must be 0 (mma.sync), 1 (tcgen05, angular contraction) or 2 (tcgen05, c contraction)");
        return IFGF_EINVAL;
    }
    if (plan->p.tc_engine != engine) plan->p.gen++;
    plan->p.tc_engine = engine;
    return IFGF_OK;
}

ifgf_status ifgf_plan_set_interp_engine(ifgf_plan *plan, int engine) {
    clear_error();
    if (!plan || (engine != 0 && engine != 1)) {
        set_error("engine must be 0 (point-stationary) or 1 (cone-stationary)");
        return IFGF_EINVAL;
    }
    if (plan->p.interp_engine != engine) plan->p.gen++;
    plan->p.interp_engine = engine;
    return IFGF_OK;
}

ifgf_status ifgf_plan_set_profiling(ifgf_plan *plan, int enable) {
    clear_error();
    if (!plan) {
        set_error("null plan");
        return IFGF_EINVAL;
    }
    Plan &p = plan->p;
    if (enable && !p.ev[0]) {
        for (int i = 0; i < Plan::kMaxEv; i++) {
            cudaError_t e = cudaEventCreate(&p.ev[i]);
            if (e != cudaSuccess) {
                set_error("cudaEventCreate: %s", cudaGetErrorString(e));
                return IFGF_ECUDA;
            }
        }
    }
    p.profile = enable != 0;
    p.nev = 0;
    return IFGF_OK;
}

int ifgf_plan_stage_times(ifgf_plan *plan, int cap, int *kind, int *level, double *ms) {
    clear_error();
    if (!plan || cap < 0) {
        set_error("null plan or negative capacity");
        return IFGF_EINVAL;
    }
    Plan &p = plan->p;
    if (!p.profile || p.nev < 2) return 0;
    cudaError_t e = cudaEventSynchronize(p.ev[p.nev - 1]);
    if (e != cudaSuccess) {
        set_error("cudaEventSynchronize: %s", cudaGetErrorString(e));
        return IFGF_ECUDA;
    }
    int n = p.nev - 1 < cap ? p.nev - 1 : cap;
    for (int i = 0; i < n; i++) {
        float t = 0.f;
        cudaEventElapsedTime(&t, p.ev[i], p.ev[i + 1]);
        if (kind) kind[i] = p.ev_kind[i];
        if (level) level[i] = p.ev_level[i];
        if (ms) ms[i] = t;
    }
    return n;
}

}  // extern "C"

// Host side of the forward apply: plan upload, workspace, dispatch over the
// compiled interpolation orders (kernels in fwd_kernels.cuh, instantiated per
// order pair in inst_<Ps>x<Pang>.cu).
#include <algorithm>
#include <cmath>
#include <cstdio>

#include "ifgf_internal.h"

namespace ifgf {

// level-D box coordinates packed 21 bits per axis (depth <= 20: coordinates below 2^19)
static inline uint64_t pack_ijk(const int *q) {
    return (uint64_t)q[0] | ((uint64_t)q[1] << 21) | ((uint64_t)q[2] << 42);
}

#define CK(call)                                                                                  \
    do {                                                                                          \
        cudaError_t e_ = (call);                                                                  \
        if (e_ != cudaSuccess) {                                                                  \
            set_error("%s failed: %s", #call, cudaGetErrorString(e_));                            \
            return IFGF_ECUDA;                                                                    \
        }                                                                                         \
    } while (0)

template <int PS, int PA>
ifgf_status run_apply_t(Plan &p, const void *sigma, void *y, int nrhs, int prec, cudaStream_t s);
template <int PS, int PA>
ifgf_status prepare_t(Plan &p, cudaStream_t s);
extern template ifgf_status prepare_t<3, 5>(Plan &, cudaStream_t);
extern template ifgf_status prepare_t<4, 6>(Plan &, cudaStream_t);
extern template ifgf_status prepare_t<5, 7>(Plan &, cudaStream_t);
extern template ifgf_status prepare_t<5, 8>(Plan &, cudaStream_t);
extern template ifgf_status prepare_t<6, 8>(Plan &, cudaStream_t);
extern template ifgf_status run_apply_t<3, 5>(Plan &, const void *, void *, int, int, cudaStream_t);
extern template ifgf_status run_apply_t<4, 6>(Plan &, const void *, void *, int, int, cudaStream_t);
extern template ifgf_status run_apply_t<5, 7>(Plan &, const void *, void *, int, int, cudaStream_t);
extern template ifgf_status run_apply_t<5, 8>(Plan &, const void *, void *, int, int, cudaStream_t);
extern template ifgf_status run_apply_t<6, 8>(Plan &, const void *, void *, int, int, cudaStream_t);

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

// Plan-time geometry of the cone-stationary cousin interpolation, in FP64, once per plan: for
// every entry (target x, relevant cone (box c, segment (is, it, ip))) the local coordinates of x
// in that segment (Eq. ConeIntervals mapped to [-1, 1] per axis: s = h / r, theta, phi about the
// centre y_c) and the centred factor E(x; y_c) = e^{ik r} / (4 pi r) of Eq. cent_fact, rounded to
// FP32, and the entry's slot in the value buffer (box of x, cousin slot, position in the box).
// One warp per work item (one cone, <= kCsItem entries), as in the apply kernel.
__global__ void __launch_bounds__(128) k_cousin_geo(int nitems, const int4 *__restrict__ items,
                                                    const uint32_t *__restrict__ ent, const int *__restrict__ rc_box,
                                                    const int *__restrict__ rc_cone, const int *__restrict__ ijk,
                                                    const int *__restrict__ start, const int *__restrict__ box_of,
                                                    const int *__restrict__ pvoff, const double *__restrict__ x64,
                                                    double c00, double c01, double c02, double H, double h, double ds,
                                                    double dth, double dph, int nC, int nph, double k,
                                                    float4 *__restrict__ geo4, float2 *__restrict__ geo2) {
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int item = blockIdx.x * 4 + warp;
    if (item >= nitems) return;
    const int4 w = items[item];
    const int rc = w.x, c = rc_box[rc], cone = rc_cone[rc];
    const int ip = cone % nph, it = (cone / nph) % nC, is = cone / (nph * nC);
    const double y0 = c00 + (ijk[3 * c] + 0.5) * H, y1 = c01 + (ijk[3 * c + 1] + 0.5) * H,
                 y2 = c02 + (ijk[3 * c + 2] + 0.5) * H;
    const double twopi = 2.0 * 3.14159265358979323846;
    for (int m = lane; m < w.z; m += 32) {
        const int e = w.y + m;
        const uint32_t en = ent[e];
        const int i = (int)(en & 0xFFFFFFu), slot = (int)(en >> 24);
        const double dx = x64[3 * i] - y0, dy = x64[3 * i + 1] - y1, dz = x64[3 * i + 2] - y2;
        const double rho = sqrt(dx * dx + dy * dy);
        const double r = sqrt(dx * dx + dy * dy + dz * dz);
        double ph = atan2(dy, dx);
        if (ph < 0) ph += twopi;
        if (ph >= twopi) ph = 0.0;
        const double us = (h / r) / ds - is, ut = atan2(rho, dz) / dth - it;
        double up = ph / dph - ip;
        if (up > 0.5 * nph) up -= nph;  // phi wrapped across 2 pi relative to the segment
        else if (up < -0.5 * nph) up += nph;
        double sn, cs;
        sincos(k * r, &sn, &cs);
        const double a = 1.0 / (4.0 * 3.14159265358979323846 * r);
        const int b = box_of[i], s0 = start[b];
        const int dest = pvoff[b] + slot * (start[b + 1] - s0) + (i - s0);
        geo4[e] = make_float4((float)(2.0 * us - 1.0), (float)(2.0 * ut - 1.0), (float)(2.0 * up - 1.0), (float)(a * cs));
        geo2[e] = make_float2((float)(a * sn), __int_as_float(dest));
    }
}

#define UP(dst, vec)                                                               \
    do {                                                                           \
        ifgf_status st_ = upload(p, dst, (vec).data(), (vec).size(), s);           \
        if (st_ != IFGF_OK) return st_;                                            \
    } while (0)

ifgf_status upload_plan(Plan &p, const double *xyz, const double *nrm, const double *w, cudaStream_t s) {
    CK(cudaGetDevice(&p.device));
    CK(cudaDeviceGetAttribute(&p.num_sms, cudaDevAttrMultiProcessorCount, p.device));
    const int64_t N = p.N;
    const int D = p.D;
    std::vector<double> x64(3 * N), n64(3 * N), w64(N);
    std::vector<float> f32(3 * N), n32(3 * N), w32(N);
    const HostLevel &LD = p.lv[D];
    // the kernels take the double-layer coefficient from the normals: the device copies are the
    // normals times that coefficient (0 for the single layer alone, else 1)
    const double alpha = p.prm.layer == IFGF_LAYER_SINGLE ? 0.0 : 1.0;
    for (int64_t si = 0; si < N; si++) {
        int o = p.perm[si];
        int b = p.leaf_of[si];
        for (int a = 0; a < 3; a++) {
            x64[3 * si + a] = xyz[3 * o + a];
            n64[3 * si + a] = alpha * nrm[3 * o + a];
            double cen = p.c0[a] + (LD.ijk[3 * b + a] + 0.5) * p.HD;
            f32[3 * si + a] = (float)((xyz[3 * o + a] - cen) / p.HD);
            n32[3 * si + a] = (float)(alpha * nrm[3 * o + a]);
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
    std::vector<int> pstart_h;  // first source pair of each level-D box
    {
        std::vector<float4> pn(2 * (size_t)N);
        for (int64_t i = 0; i < N; i++) {
            const float fx = f32[3 * i], fy = f32[3 * i + 1], fz = f32[3 * i + 2];
            pn[2 * i] = make_float4(fx, fy, fz, fx * fx + fy * fy + fz * fz);
            pn[2 * i + 1] = make_float4(n32[3 * i], n32[3 * i + 1], n32[3 * i + 2], 0.f);
        }
        UP(p.d_pn32, pn);
        // the same records in source pairs per leaf box (an odd box ends with a zero source)
        const HostLevel &LDb = p.lv[D];
        std::vector<int> &pstart = pstart_h;
        pstart.assign(LDb.nbox + 1, 0);
        for (int b = 0; b < LDb.nbox; b++) pstart[b + 1] = pstart[b] + (LDb.start[b + 1] - LDb.start[b] + 1) / 2;
        p.npairs = pstart[LDb.nbox];
        std::vector<float4> pp(4 * (size_t)p.npairs);
        std::vector<int2> psrc(p.npairs);
        std::vector<unsigned long long> pair_ijk(p.npairs);
        for (int b = 0; b < LDb.nbox; b++)
            for (int j = LDb.start[b], m = pstart[b]; j < LDb.start[b + 1]; j += 2, m++) {
                const bool two = j + 1 < LDb.start[b + 1];
                const float4 z = make_float4(0.f, 0.f, 0.f, 0.f);
                const float4 a0 = pn[2 * j], b0 = pn[2 * j + 1];
                const float4 a1 = two ? pn[2 * j + 2] : z, b1 = two ? pn[2 * j + 3] : z;
                pp[4 * (size_t)m] = make_float4(a0.x, a1.x, a0.y, a1.y);
                pp[4 * (size_t)m + 1] = make_float4(a0.z, a1.z, a0.w, a1.w);
                pp[4 * (size_t)m + 2] = make_float4(b0.x, b1.x, b0.y, b1.y);
                // last slot: f.n of each source (the leaf's |u - ir f| and (u - ir f).n from u.f and u.n)
                auto fdotn = [](float4 f, float4 nn) {
                    return (float)((double)f.x * nn.x + (double)f.y * nn.y + (double)f.z * nn.z);
                };
                pp[4 * (size_t)m + 3] = make_float4(b0.z, b1.z, fdotn(a0, b0), two ? fdotn(a1, b1) : 0.f);
                pair_ijk[m] = pack_ijk(&LDb.ijk[3 * b]);  // read by the adaptive near field
                psrc[m] = make_int2(j, two ? j + 1 : -1);
            }
        UP(p.d_pp32, pp);
        if (p.adaptive) UP(p.d_pair_ijk, pair_ijk);
        UP(p.d_pstart, pstart);
        UP(p.d_pair_src, psrc);
    }
    UP(p.d_perm, p.perm);
    UP(p.d_leaf_of, p.leaf_of);
    UP(p.d_nb_start, p.nb_start);
    UP(p.d_nb_list, p.nb_list);
    {
        // near-field chunks (.x the level-D box of the first target, .y the first target, .z the count,
        // .w the leaf's index): at most 64 targets of one leaf box (level-D boxes, or leaves of any level
        // in an adaptive tree), in point order; an adaptive tree's chunks with long source lists last
        std::vector<int2> leaves;  // point ranges of the leaves
        for (int d = 3; d <= D; d++) {
            const HostLevel &L = p.lv[d];
            for (int b = 0; b < L.nbox; b++)
                if (L.leaf[b]) leaves.push_back(make_int2(L.start[b], L.start[b + 1]));
        }
        std::sort(leaves.begin(), leaves.end(), [](int2 a, int2 b) { return a.x < b.x; });
        std::vector<int64_t> leaf_pairs(leaves.size(), 0);  // near source pairs of each leaf (adaptive)
        if (p.adaptive) {
            // per leaf: its near sources (the level-D boxes of its first level-D box's list, which every
            // level-D box under the leaf shares) as merged point / pair ranges
            const HostLevel &LD = p.lv[D];
            std::vector<int> nr_start(leaves.size() + 1, 0);
            std::vector<int4> nr;
            std::vector<int4> tmp;
            for (size_t li = 0; li < leaves.size(); li++) {
                const int e = p.leaf_of[leaves[li].x];
                tmp.clear();
                for (int q = p.nb_start[e]; q < p.nb_start[e + 1]; q++) {
                    const int c = p.nb_list[q];
                    tmp.push_back(make_int4(LD.start[c], LD.start[c + 1], pstart_h[c], pstart_h[c + 1]));
                }
                std::sort(tmp.begin(), tmp.end(), [](const int4 &a, const int4 &b) { return a.x < b.x; });
                for (size_t t = 0; t < tmp.size(); t++) {
                    leaf_pairs[li] += tmp[t].w - tmp[t].z;
                    if ((int)nr.size() > nr_start[li] && nr.back().y == tmp[t].x) {
                        nr.back().y = tmp[t].y;  // consecutive level-D boxes: one range
                        nr.back().w = tmp[t].w;
                    } else {
                        nr.push_back(tmp[t]);
                    }
                }
                nr_start[li + 1] = (int)nr.size();
            }
            if (nr.empty()) nr.push_back(make_int4(0, 0, 0, 0));
            UP(p.d_nr_start, nr_start);
            UP(p.d_nr, nr);
            std::vector<unsigned long long> pk(N);
            for (int b = 0; b < LD.nbox; b++)
                for (int si = LD.start[b]; si < LD.start[b + 1]; si++) pk[si] = pack_ijk(&LD.ijk[3 * b]);
            UP(p.d_pt_ijk, pk);
        }
        // chunks of leaves with long source lists (adaptive trees) go last: one block each
        constexpr int64_t kHeavyPairs = 2048;
        std::vector<int4> ch, heavy;
        for (size_t li = 0; li < leaves.size(); li++) {
            const int2 r = leaves[li];
            const int n = r.y - r.x;
            const int nch = (n + 63) / 64;
            for (int k = 0; k < nch; k++) {
                const int s0 = r.x + (int)((int64_t)n * k / nch);
                const int s1 = r.x + (int)((int64_t)n * (k + 1) / nch);
                (leaf_pairs[li] > kHeavyPairs ? heavy : ch).push_back(make_int4(p.leaf_of[s0], s0, s1 - s0, (int)li));
            }
        }
        p.nnchunk_light = (int)ch.size();
        ch.insert(ch.end(), heavy.begin(), heavy.end());
        p.nnchunk = (int)ch.size();
        UP(p.d_nchunk, ch);
    }
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
        UP(p.d_alive[d], L.alive);
        UP(p.d_leaf[d], L.leaf);
        p.nleaf_rc[d] = (int)L.leaf_rc.size();
        if (!L.leaf_rc.empty()) UP(p.d_leaf_rc[d], L.leaf_rc);
        std::vector<int4> ch;
        for (int b = 0; b < L.nbox; b++) {
            if (!L.alive[b]) continue;  // below a coarser leaf: no level-d interpolation for these points
            const int n = L.start[b + 1] - L.start[b];
            const int nch = (n + 31) / 32;
            for (int k = 0; k < nch; k++) {
                const int s0 = L.start[b] + (int)((int64_t)n * k / nch);
                const int s1 = L.start[b] + (int)((int64_t)n * (k + 1) / nch);
                ch.push_back(make_int4(b, s0, s1 - s0, 0));
            }
        }
        p.ncchunk[d] = (int)ch.size();
        UP(p.d_cchunk[d], ch);
    }
    // cone-stationary cousin interpolation: work items of at most kCsItem entries of one cone
    if (p.cs_ok) {
        for (int d = 3; d <= D; d++) {
            HostLevel &L = p.lv[d];
            std::vector<int4> items;
            for (int64_t rc = 0; rc < L.nrc; rc++)
                for (int64_t e = L.cs_start[rc]; e < L.cs_start[rc + 1]; e += kCsItem)
                    items.push_back(make_int4((int)rc, (int)e, (int)std::min<int64_t>(kCsItem, L.cs_start[rc + 1] - e), 0));
            p.ncs_item[d] = (int)items.size();
            UP(p.d_cs_item[d], items);
            {
                std::vector<int> first(L.nrc > 0 ? L.nrc : 1, 0);
                for (int64_t rc = 0; rc < L.nrc; rc++) first[rc] = (int)L.cs_start[rc];
                UP(p.d_cs_first[d], first);
            }
            UP(p.d_cs_pvoff[d], L.cs_pvoff);
            {
                const size_t ne = L.cs_ent.size() > 0 ? L.cs_ent.size() : 1;
                cudaError_t err;
                p.d_cs_geo4[d] = dalloc<float4>(p, ne, err);
                if (p.d_cs_geo4[d]) p.d_cs_geo2[d] = dalloc<float2>(p, ne, err);
                if (!p.d_cs_geo2[d]) {
                    set_error("cudaMalloc failed: %s", cudaGetErrorString(err));
                    return IFGF_ENOMEM;
                }
                uint32_t *ent = nullptr;
                CK(cudaMalloc(&ent, sizeof(uint32_t) * ne));
                cudaError_t e2 = cudaMemcpyAsync(ent, L.cs_ent.data(), sizeof(uint32_t) * L.cs_ent.size(),
                                                 cudaMemcpyHostToDevice, s);
                const DevLevel &dl = p.dl[d];
                if (e2 == cudaSuccess && !items.empty()) {
                    k_cousin_geo<<<(unsigned)((items.size() + 3) / 4), 128, 0, s>>>(
                        (int)items.size(), p.d_cs_item[d], ent, dl.rc_box, dl.rc_cone, dl.ijk, dl.start,
                        p.d_box_of[d], p.d_cs_pvoff[d], p.d_x64, p.c0[0], p.c0[1], p.c0[2], L.H, L.h, L.ds, L.dth,
                        L.dph, L.nC, L.nph, p.prm.k, p.d_cs_geo4[d], p.d_cs_geo2[d]);
                    e2 = cudaGetLastError();
                }
                if (e2 == cudaSuccess) e2 = cudaStreamSynchronize(s);
                cudaFree(ent);
                if (e2 != cudaSuccess) {
                    set_error("cousin geometry: %s", cudaGetErrorString(e2));
                    return IFGF_ECUDA;
                }
            }
            std::vector<int64_t>().swap(L.cs_start);
            std::vector<uint32_t>().swap(L.cs_ent);
            std::vector<int>().swap(L.cs_pvoff);
        }
    }
    // tensor-core propagation tables (orders with Pang = 8)
    if (p.Pang == 8) {
        p.use_tc = true;
        for (int d = D; d >= 4; d--) {
            const HostLevel &Cl = p.lv[d], &Pl = p.lv[d - 1];
            // key = octant * ncone_parent + parent cone id
            std::vector<std::pair<long long, std::pair<int, int>>> pairs;  // (key, (rcp, cb))
            for (int pb = 0; pb < Pl.nbox; pb++)
                for (int ci = Pl.ch_start[pb]; ci < Pl.ch_start[pb + 1]; ci++) {
                    const int cb = Pl.ch_list[ci];
                    const int o = (Cl.ijk[3 * cb] & 1) + 2 * (Cl.ijk[3 * cb + 1] & 1) + 4 * (Cl.ijk[3 * cb + 2] & 1);
                    for (int rc = Pl.rc_start[pb]; rc < Pl.rc_start[pb + 1]; rc++)
                        pairs.push_back({(long long)o * Pl.ncone + Pl.rc_cone[rc], {rc, cb}});
                }
            std::stable_sort(pairs.begin(), pairs.end(),
                             [](const auto &a, const auto &b) { return a.first < b.first; });
            std::vector<int> tg, ts, tcnt, gg, gpb, gcb, prc, pcb;
            TcLevel &T = p.tc[d];
            int cur_oct = -1;
            for (size_t i = 0; i < pairs.size();) {
                size_t j = i;
                while (j < pairs.size() && pairs[j].first == pairs[i].first) j++;
                const int g = (int)gg.size();
                const int oct = (int)(pairs[i].first / Pl.ncone);
                while (cur_oct < oct) T.oct_tile_start[++cur_oct] = (int)tg.size();
                gg.push_back((int)(pairs[i].first % Pl.ncone));
                gpb.push_back(Pl.rc_box[pairs[i].second.first]);
                gcb.push_back(pairs[i].second.second);
                for (size_t t = i; t < j; t += kTcTile) {
                    tg.push_back(g);
                    ts.push_back((int)(prc.size() + (t - i)));
                    tcnt.push_back((int)std::min<size_t>(kTcTile, j - t));
                }
                for (size_t t = i; t < j; t++) {
                    prc.push_back(pairs[t].second.first);
                    pcb.push_back(pairs[t].second.second);
                }
                i = j;
            }
            while (cur_oct < 8) T.oct_tile_start[++cur_oct] = (int)tg.size();
            T.ntiles = (int)tg.size();
            T.ngroups = (int)gg.size();
            T.fill = T.ntiles ? (double)prc.size() / ((double)T.ntiles * kTcTile) : 0.0;
            UP(T.tile_group, tg);
            UP(T.tile_start, ts);
            UP(T.tile_count, tcnt);
            UP(T.grp_gamma, gg);
            UP(T.grp_pb, gpb);
            UP(T.grp_cb, gcb);
            UP(T.pair_rcp, prc);
            UP(T.pair_cb, pcb);
            {
                cudaError_t err;
                const size_t ng = gg.size() > 0 ? gg.size() : 1;
                T.grp_perm = dalloc<short>(p, ng * (size_t)p.P, err);
                if (T.grp_perm) T.grp_cones = dalloc<int>(p, ng * 16, err);
                if (T.grp_cones) T.grp_nc = dalloc<int>(p, ng, err);
                if (T.grp_nc) T.grp_cnt = dalloc<int>(p, ng * 17, err);
                if (!T.grp_cnt) {
                    set_error("cudaMalloc failed: %s", cudaGetErrorString(err));
                    return IFGF_ENOMEM;
                }
            }
        }
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
    CK(cudaStreamCreateWithFlags(&p.aux, cudaStreamNonBlocking));
    for (int i = 0; i < Plan::kMaxDep; i++) CK(cudaEventCreateWithFlags(&p.dep[i], cudaEventDisableTiming));
    ifgf_status st = IFGF_EUNSUPPORTED;
    if (p.Ps == 3 && p.Pang == 5) st = prepare_t<3, 5>(p, s);
    else if (p.Ps == 4 && p.Pang == 6) st = prepare_t<4, 6>(p, s);
    else if (p.Ps == 5 && p.Pang == 7) st = prepare_t<5, 7>(p, s);
    else if (p.Ps == 5 && p.Pang == 8) st = prepare_t<5, 8>(p, s);
    else if (p.Ps == 6 && p.Pang == 8) st = prepare_t<6, 8>(p, s);
    else set_error("orders Ps=%d Pang=%d not compiled", p.Ps, p.Pang);
    return st;
}

void free_plan_device(Plan &p) {
    for (int i = 0; i < Plan::kMaxDep; i++)
        if (p.dep[i]) {
            cudaEventDestroy(p.dep[i]);
            p.dep[i] = nullptr;
        }
    if (p.aux) cudaStreamDestroy(p.aux);
    p.aux = nullptr;
    if (p.adj_ws) cudaFree(p.adj_ws);
    p.adj_ws = nullptr;
    p.adj_ws_bytes = 0;
    if (p.dk_ws) cudaFree(p.dk_ws);
    p.dk_ws = nullptr;
    p.dk_ws_bytes = 0;
    if (p.field_ws) cudaFree(p.field_ws);
    p.field_ws = nullptr;
    p.field_ws_bytes = 0;
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

// Byte offsets of the workspace parts for nrhs right-hand sides in one precision: a, u, then F of
// levels 3..D, each 256-byte aligned; returns the total.  ensure_workspace and the allocation-free
// apply share this layout.
size_t workspace_layout(const Plan &p, int nrhs, int prec, WorkspaceLayout &lay) {
    const size_t cb = prec == IFGF_FP64 ? 16 : 8;  // bytes per complex
    auto al = [](size_t x) { return (x + 255) & ~(size_t)255; };
    size_t off = 0;
    lay = WorkspaceLayout();
    lay.a = off; off += al(cb * (size_t)p.N * nrhs);
    lay.u = off; off += al(cb * (size_t)p.N * nrhs);
    for (int d = 3; d <= p.D; d++) {
        lay.F[d] = off;
        off += al(cb * (size_t)nrhs * p.lv[d].nrc * p.lv[d].nfac * p.Pstride);
    }
    lay.pv = off;
    if (prec == IFGF_MIXED && p.cs_ok && p.interp_engine == 1) off += al(8 * (size_t)nrhs * p.cs_max_entries);
    lay.ap = off;
    if (prec == IFGF_MIXED) off += al(16 * (size_t)nrhs * p.npairs);
    lay.total = off;
    return off;
}

void workspace_bind(Workspace &ws, const Plan &p, void *base, const WorkspaceLayout &lay, int nrhs, int prec) {
    char *c = static_cast<char *>(base);
    ws.base = base;
    ws.bytes = lay.total;
    ws.nrhs = nrhs;
    ws.prec = prec;
    ws.a = c + lay.a;
    ws.u = c + lay.u;
    for (int d = 3; d <= p.D; d++) ws.F[d] = c + lay.F[d];
    ws.pv = c + lay.pv;
    ws.ap = c + lay.ap;
}

ifgf_status ensure_workspace(Plan &p, int nrhs, int prec) {
    WorkspaceLayout lay;
    const size_t off = workspace_layout(p, nrhs, prec, lay);
    if (p.ws.base && p.ws.nrhs >= nrhs && p.ws.prec == prec && p.ws.bytes >= off) return IFGF_OK;
    if (p.ws.base) cudaFree(p.ws.base);
    p.ws = Workspace();
    p.gen++;
    void *base = nullptr;
    cudaError_t e = cudaMalloc(&base, off);
    if (e != cudaSuccess) {
        set_error("workspace cudaMalloc(%zu bytes) failed: %s", off, cudaGetErrorString(e));
        return e == cudaErrorMemoryAllocation ? IFGF_ENOMEM : IFGF_ECUDA;
    }
    workspace_bind(p.ws, p, base, lay, nrhs, prec);
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
    IFGF_CASE(5, 8)
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
    else if (p.Ps == 5 && p.Pang == 8) st = run_apply_t<5, 8>(p, sigma, y, nrhs, prec, s);
    else if (p.Ps == 6 && p.Pang == 8) st = run_apply_t<6, 8>(p, sigma, y, nrhs, prec, s);
    else set_error("orders Ps=%d Pang=%d not compiled", p.Ps, p.Pang);
    p.ws = saved;
    return st;
}

}  // namespace ifgf

// Host plan builder: octree, relevant boxes, neighbours/cousins, cone grids and
// relevant cone segments (Section 3.4; Eq. box, Eq. RelevantBoxes,
// Eq. NeighborsCousins, Eq. deltas, Eq. ConeIntervals, Eq. RelevantCones).
//
// Points are sorted along a Morton (Z) curve of their leaf boxes (the ordering
// Section 3.5 uses for its task vectors); every octree box then owns a
// contiguous range of sorted points at every level.
#include <algorithm>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <numeric>

#include "ifgf_internal.h"

namespace ifgf {

static thread_local std::string g_err;

void set_error(const char *fmt, ...) {
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof(buf), fmt, ap);
    va_end(ap);
    g_err = buf;
}

const char *last_error_str() { return g_err.c_str(); }
void clear_error() { g_err.clear(); }

void cheb_axis(int n, ChebAxis *a) {
    a->n = n;
    for (int j = 0; j < n; j++) a->x[j] = std::cos((2.0 * j + 1.0) * M_PI / (2.0 * n));
    for (int j = 0; j < n; j++) {
        double prod = 1.0;
        for (int m = 0; m < n; m++)
            if (m != j) prod *= (a->x[j] - a->x[m]);
        a->c[j] = 1.0 / prod;
    }
}

static uint64_t spread3(uint64_t v) {
    // spread the low 21 bits of v to every third bit
    v &= 0x1fffffULL;
    v = (v | (v << 32)) & 0x1f00000000ffffULL;
    v = (v | (v << 16)) & 0x1f0000ff0000ffULL;
    v = (v | (v << 8)) & 0x100f00f00f00f00fULL;
    v = (v | (v << 4)) & 0x10c30c30c30c30c3ULL;
    v = (v | (v << 2)) & 0x1249249249249249ULL;
    return v;
}
static uint64_t morton(int i, int j, int k) { return (spread3(i) << 2) | (spread3(j) << 1) | spread3(k); }

static int leaf_coord(double x, double corner, double H, int nside) {
    double f = std::floor((x - corner) / H);
    int v = (int)f;
    if (f < 0) v = 0;
    if (f > nside - 1) v = nside - 1;
    return v;
}

int morton_levels_auto(const double *xyz, int64_t N, const double *c0, double L, double leaf_target) {
    double lt = leaf_target > 0 ? leaf_target : 64.0;
    double best = INFINITY;
    int D = 3;
    // keys at the finest candidate level; the level-d key is the prefix key >> 3 (16 - d)
    // (box sides are powers of two apart, so the floors nest exactly)
    std::vector<uint64_t> keys(N);
    {
        const double H = std::ldexp(L, -15);
        const int nside = 1 << 15;
        for (int64_t i = 0; i < N; i++)
            keys[i] = morton(leaf_coord(xyz[3 * i], c0[0], H, nside), leaf_coord(xyz[3 * i + 1], c0[1], H, nside),
                             leaf_coord(xyz[3 * i + 2], c0[2], H, nside));
        std::sort(keys.begin(), keys.end());
    }
    for (int d = 3; d <= 16; d++) {
        const int sh = 3 * (16 - d);
        int64_t nb = 0;
        for (int64_t i = 0; i < N; i++)
            if (i == 0 || (keys[i] >> sh) != (keys[i - 1] >> sh)) nb++;
        double m = std::fabs(std::log((double)N / nb / lt));
        if (m < best) {
            best = m;
            D = d;
        }
        if ((double)N / nb < lt / 16.0) break;
    }
    return D;
}

static int find_box(const HostLevel &L, int i, int j, int k) {
    int n = 1 << (L.d - 1);
    if (i < 0 || j < 0 || k < 0 || i >= n || j >= n || k >= n) return -1;
    uint64_t key = morton(i, j, k);
    auto it = std::lower_bound(L.mkey.begin(), L.mkey.end(), key);
    if (it == L.mkey.end() || *it != key) return -1;
    return (int)(it - L.mkey.begin());
}

namespace {

struct Ctx {
    const Plan *p;
    const double *xs;  // sorted absolute positions
};

inline void box_center(const Plan &p, const HostLevel &L, int b, double *y0) {
    for (int a = 0; a < 3; a++) y0[a] = p.c0[a] + (L.ijk[3 * b + a] + 0.5) * L.H;
}

// Candidate indices along one axis: the clamped floor plus neighbours within `band`
// (in units of the interval) of a boundary.  Returns the count (1..3), or -1 when the
// position is too uncertain and every index 0..n-1 is a candidate.
inline int axis_candidates(double u, int n, double band, bool wrap, int *out) {
    int i = (int)std::floor(u);
    if (i > n - 1) i = n - 1;
    if (i < 0) i = 0;
    int c = 0;
    out[c++] = i;
    if (band <= 0) return 1;
    if (band >= 0.5) return -1;
    double fr = u - i;
    if (fr < band) {
        if (i > 0) out[c++] = i - 1;
        else if (wrap) out[c++] = n - 1;
    }
    if (fr > 1.0 - band) {
        if (i < n - 1) out[c++] = i + 1;
        else if (wrap) out[c++] = 0;
    }
    return c;
}

// Boundary points (within 1e-12 relative) are placed on the boundary, so the upper
// interval owns them independently of last-bit rounding (same rule as the kernels).
inline double snap(double u) {
    double r = std::nearbyint(u);
    return std::fabs(u - r) <= 1e-12 * std::max(std::fabs(u), 1.0) ? r : u;
}

// Mark in `bits` every cone (level L) that the point at offset (dx, dy, dz) from a box
// centre may fall into (Eq. ConeIntervals with clamped indices; phi in [0, 2 pi)).
inline void mark_offset(const HostLevel &L, double dx, double dy, double dz, double tau, uint64_t *bits,
                        std::vector<int> *touched = nullptr) {
    double rho = std::sqrt(dx * dx + dy * dy);
    double r = std::sqrt(dx * dx + dy * dy + dz * dz);
    double s = L.h / r;
    double th = std::atan2(rho, dz);
    double ph = std::atan2(dy, dx);
    if (ph < 0) ph += 2.0 * M_PI;
    if (ph >= 2.0 * M_PI) ph = 0.0;
    double us = snap(s / L.ds), ut = snap(th / L.dth), up = snap(ph / L.dph);
    int cs[3] = {0, 0, 0}, ct[3] = {0, 0, 0}, cp[3] = {0, 0, 0};
    double bs = 0, bt = 0, bp = 0;
    if (tau > 0) {
        // tau plus the reach of FP32 rounding of the geometry (relative 4e-7 of r)
        bs = tau + 4e-7 * us;
        bt = tau + 4e-7 / L.dth;
        bp = (rho > 0) ? tau + 4e-7 * (r / rho) / L.dph : 1.0;
    }
    int ns = axis_candidates(us, L.ns, bs, false, cs);
    int nt = axis_candidates(ut, L.nC, bt, false, ct);
    int np = axis_candidates(up, L.nph, bp, true, cp);
    int ns_n = ns < 0 ? L.ns : ns, nt_n = nt < 0 ? L.nC : nt, np_n = np < 0 ? L.nph : np;
    for (int a = 0; a < ns_n; a++)
        for (int c = 0; c < nt_n; c++)
            for (int e = 0; e < np_n; e++) {
                int is = ns < 0 ? a : cs[a], it = nt < 0 ? c : ct[c], ip = np < 0 ? e : cp[e];
                int cone = (is * L.nC + it) * L.nph + ip;
                const uint64_t m = 1ULL << (cone & 63);
                if (touched && !(bits[cone >> 6] & m)) touched->push_back(cone);
                bits[cone >> 6] |= m;
            }
}

// The same for an absolute position x and box b of level L.
inline void mark_point(const Plan &p, const HostLevel &L, int b, const double *x, double tau, uint64_t *bits) {
    double y0[3];
    box_center(p, L, b, y0);
    mark_offset(L, x[0] - y0[0], x[1] - y0[1], x[2] - y0[2], tau, bits);
}

// Offset of interpolation node n of cone `cone` (level L) from its box centre:
// (h / s) (sin theta cos phi, sin theta sin phi, cos theta) (Eq. defparametrizationins).
inline void node_offset(const Plan &p, const HostLevel &L, int cone, int n, double *v) {
    int ip = cone % L.nph, it = (cone / L.nph) % L.nC, is = cone / (L.nph * L.nC);
    int na = p.Pang;
    int a = n / (na * na), bb = (n / na) % na, c = n % na;
    double s = (is + 0.5 * (p.cs.x[a] + 1.0)) * L.ds;
    double th = (it + 0.5 * (p.ca.x[bb] + 1.0)) * L.dth;
    double ph = (ip + 0.5 * (p.ca.x[c] + 1.0)) * L.dph;
    double r = L.h / s;
    v[0] = r * std::sin(th) * std::cos(ph);
    v[1] = r * std::sin(th) * std::sin(ph);
    v[2] = r * std::cos(th);
}

}  // namespace

ifgf_status build_host_plan(Plan &p, const double *xyz, const double *nrm, const double *w) {
    const ifgf_params &prm = p.prm;
    const int64_t N = p.N;
    // ---- root box (centre = AABB midpoint, side = max extent (1 + 2^-30)) ----
    if (prm.root_side > 0) {
        p.L = prm.root_side;
        for (int a = 0; a < 3; a++) p.center[a] = prm.root_center[a];
    } else {
        double lo[3] = {INFINITY, INFINITY, INFINITY}, hi[3] = {-INFINITY, -INFINITY, -INFINITY};
        for (int64_t i = 0; i < N; i++)
            for (int a = 0; a < 3; a++) {
                lo[a] = std::min(lo[a], xyz[3 * i + a]);
                hi[a] = std::max(hi[a], xyz[3 * i + a]);
            }
        double ext = 0;
        for (int a = 0; a < 3; a++) {
            p.center[a] = 0.5 * (lo[a] + hi[a]);
            ext = std::max(ext, hi[a] - lo[a]);
        }
        if (!(ext > 0)) ext = 1.0;
        p.L = ext * (1.0 + std::ldexp(1.0, -30));
    }
    for (int a = 0; a < 3; a++) p.c0[a] = p.center[a] - 0.5 * p.L;
    // ---- level count ----
    // the automatic level count follows the sources (the first n_src points of a plan with targets)
    int D = prm.levels > 0 ? prm.levels
                           : morton_levels_auto(xyz, p.n_src > 0 ? p.n_src : N, p.c0, p.L, prm.leaf_target);
    if (D < 3 || D > 16) {
        set_error("levels must be in 3..16 (got %d)", D);
        return IFGF_EINVAL;
    }
    p.D = D;
    p.HD = std::ldexp(p.L, -(D - 1));
    cheb_axis(p.Ps, &p.cs);
    cheb_axis(p.Pang, &p.ca);
    const double lam = 2.0 * M_PI / prm.k;

    // ---- leaf coordinates and Morton sort ----
    const int nside = 1 << (D - 1);
    std::vector<int> I(3 * N);
    std::vector<uint64_t> key(N);
    for (int64_t i = 0; i < N; i++) {
        for (int a = 0; a < 3; a++) I[3 * i + a] = leaf_coord(xyz[3 * i + a], p.c0[a], p.HD, nside);
        key[i] = morton(I[3 * i], I[3 * i + 1], I[3 * i + 2]);
    }
    p.perm.resize(N);
    std::iota(p.perm.begin(), p.perm.end(), 0);
    std::stable_sort(p.perm.begin(), p.perm.end(), [&](int a, int b) { return key[a] < key[b]; });
    p.lv.assign(D + 1, HostLevel());
    for (int d = 1; d <= D; d++) {
        HostLevel &L = p.lv[d];
        L.d = d;
        L.H = std::ldexp(p.L, -(d - 1));
        L.h = std::sqrt(3.0) / 2.0 * L.H;
        L.scale = 1 << (D - d);
        const int sh = 3 * (D - d);
        for (int64_t s = 0; s < N; s++) {
            uint64_t kk = key[p.perm[s]] >> sh;
            if (s == 0 || kk != L.mkey.back()) {
                L.mkey.push_back(kk);
                L.start.push_back((int)s);
                int pi = p.perm[s];
                L.ijk.push_back(I[3 * pi] >> (D - d));
                L.ijk.push_back(I[3 * pi + 1] >> (D - d));
                L.ijk.push_back(I[3 * pi + 2] >> (D - d));
            }
        }
        L.nbox = (int)L.mkey.size();
        L.start.push_back((int)N);
    }
    p.leaf_of.resize(N);
    {
        const HostLevel &L = p.lv[D];
        for (int b = 0; b < L.nbox; b++)
            for (int s = L.start[b]; s < L.start[b + 1]; s++) p.leaf_of[s] = b;
    }
    // parents and children
    for (int d = 1; d <= D; d++) {
        HostLevel &L = p.lv[d];
        L.parent.assign(L.nbox, -1);
        if (d > 1) {
            for (int b = 0; b < L.nbox; b++)
                L.parent[b] = find_box(p.lv[d - 1], L.ijk[3 * b] >> 1, L.ijk[3 * b + 1] >> 1, L.ijk[3 * b + 2] >> 1);
        }
    }
    // adaptive octree (leaf_max > 0): a box of level 3..D-1 holding at most leaf_max points is a leaf
    // and the boxes below it do not exist; otherwise every box exists and the leaves are at level D
    p.adaptive = prm.leaf_max > 0;
    p.has_inactive = false;
    for (int d = 1; d <= D; d++) {
        HostLevel &L = p.lv[d];
        L.alive.assign(L.nbox, 1);
        L.leaf.assign(L.nbox, d == D ? 1 : 0);
        if (d < 3) continue;
        for (int b = 0; b < L.nbox; b++) {
            if (d > 3) {
                const HostLevel &PL = p.lv[d - 1];
                L.alive[b] = PL.alive[L.parent[b]] && !PL.leaf[L.parent[b]];
            }
            L.leaf[b] = L.alive[b] && (d == D || (p.adaptive && L.start[b + 1] - L.start[b] <= prm.leaf_max));
            p.has_inactive = p.has_inactive || !L.alive[b];
        }
    }
    // source boxes: existing boxes holding a point of positive weight (a plan with targets has boxes
    // without any)
    for (int d = 1; d <= D; d++) {
        HostLevel &L = p.lv[d];
        L.active.assign(L.nbox, 0);
        for (int b = 0; b < L.nbox; b++) {
            for (int s = L.start[b]; s < L.start[b + 1] && !L.active[b] && L.alive[b]; s++)
                L.active[b] = w[p.perm[s]] > 0;
            p.has_inactive = p.has_inactive || !L.active[b];
        }
    }
    // children lists hold the source children only: propagation reads nothing from the others
    for (int d = 1; d < D; d++) {
        HostLevel &L = p.lv[d];
        const HostLevel &C = p.lv[d + 1];
        L.ch_start.assign(L.nbox + 1, 0);
        for (int b = 0; b < C.nbox; b++)
            if (C.active[b]) L.ch_start[C.parent[b] + 1]++;
        for (int b = 0; b < L.nbox; b++) L.ch_start[b + 1] += L.ch_start[b];
        L.ch_list.assign(L.ch_start[L.nbox], 0);
        std::vector<int> fill(L.ch_start.begin(), L.ch_start.end() - 1);
        for (int b = 0; b < C.nbox; b++)
            if (C.active[b]) L.ch_list[fill[C.parent[b]]++] = b;
    }
    p.lv[D].ch_start.assign(p.lv[D].nbox + 1, 0);
    // near-field lists per level-D box (the 27-neighbourhood including the box itself).  In an adaptive
    // tree a point of a leaf at level d_t and one of a leaf at level d_s are near when their boxes at
    // level min(d_t, d_s) neighbour: for the level-D box b below the leaf B (level d_B) that is every
    // level-D box below an existing neighbour of B, and every level-D box below a leaf of a coarser
    // level m that neighbours B's ancestor there (each source box exactly once).
    {
        const HostLevel &L = p.lv[D];
        p.nb_start.assign(L.nbox + 1, 0);
        p.nb_list.clear();
        int64_t pairs = 0;
        std::vector<int> anc(D + 1);
        for (int b = 0; b < L.nbox; b++) {
            p.nb_start[b] = (int)p.nb_list.size();
            int64_t cnt = 0;
            anc[D] = b;
            for (int d = D; d > 3; d--) anc[d - 1] = p.lv[d].parent[anc[d]];
            int dB = 3;
            while (!p.lv[dB].leaf[anc[dB]]) dB++;
            for (int m = p.adaptive ? 3 : D; m <= dB; m++) {
                const HostLevel &M = p.lv[m];
                const int *q = &M.ijk[3 * anc[m]];
                for (int o0 = -1; o0 <= 1; o0++)
                    for (int o1 = -1; o1 <= 1; o1++)
                        for (int o2 = -1; o2 <= 1; o2++) {
                            const int c = find_box(M, q[0] + o0, q[1] + o1, q[2] + o2);
                            if (c < 0 || !M.alive[c] || (m < dB && !M.leaf[c])) continue;
                            const int f0 = p.leaf_of[M.start[c]], f1 = p.leaf_of[M.start[c + 1] - 1];
                            for (int e = f0; e <= f1; e++) {
                                p.nb_list.push_back(e);
                                cnt += L.start[e + 1] - L.start[e];
                            }
                        }
            }
            pairs += cnt * (L.start[b + 1] - L.start[b]);
        }
        p.nb_start[L.nbox] = (int)p.nb_list.size();
        p.near_pairs = pairs;
    }
    // cousins (Eq. NeighborsCousins): non-neighbours whose parent neighbours the parent
    for (int d = 3; d <= D; d++) {
        HostLevel &L = p.lv[d];
        L.co_start.assign(L.nbox + 1, 0);
        L.co_list.clear();
        for (int b = 0; b < L.nbox; b++) {
            L.co_start[b] = (int)L.co_list.size();
            const int *q = &L.ijk[3 * b];
            int pp[3] = {q[0] >> 1, q[1] >> 1, q[2] >> 1};
            for (int o0 = -1; o0 <= 1; o0++)
                for (int o1 = -1; o1 <= 1; o1++)
                    for (int o2 = -1; o2 <= 1; o2++)
                        for (int ch = 0; ch < 8; ch++) {
                            int j0 = 2 * (pp[0] + o0) + (ch & 1), j1 = 2 * (pp[1] + o1) + ((ch >> 1) & 1),
                                j2 = 2 * (pp[2] + o2) + ((ch >> 2) & 1);
                            int dm = std::max(std::abs(j0 - q[0]), std::max(std::abs(j1 - q[1]), std::abs(j2 - q[2])));
                            if (dm <= 1) continue;
                            int c = find_box(L, j0, j1, j2);
                            if (c >= 0) L.co_list.push_back(c);
                        }
        }
        L.co_start[L.nbox] = (int)L.co_list.size();
        int64_t ev = 0;  // (source box, point in one of its existing cousins) pairs
        for (int b = 0; b < L.nbox; b++)
            for (int c = L.co_start[b]; c < L.co_start[b + 1] && L.active[b]; c++)
                if (L.alive[L.co_list[c]]) ev += L.start[L.co_list[c] + 1] - L.start[L.co_list[c]];
        L.cousin_evals = ev;
    }
    // cone grids (Remark cone_seg_size) and factor split (Section 3.3)
    int e_lit = 0;
    for (int d = D; d >= 3; d--) {
        HostLevel &L = p.lv[d];
        int e = 0;
        if (prm.cone_rule == 0) {
            while (L.H > std::ldexp(0.5 * lam, e) && e < 24) e++;
        } else {
            if (d < D && prm.k * p.lv[d + 1].H > 0.5) e_lit++;
            e = e_lit;
        }
        L.ns = prm.nS0 << e;
        L.nC = prm.nC0 << e;
        L.nph = 2 * L.nC;
        int64_t nc = (int64_t)L.ns * L.nC * L.nph;
        if (nc > (1LL << 28)) {
            set_error("cone grid too fine at level %d (%lld cones per box)", d, (long long)nc);
            return IFGF_EUNSUPPORTED;
        }
        L.ncone = (int)nc;
        L.ds = (std::sqrt(3.0) / 3.0) / L.ns;
        L.dth = M_PI / L.nC;
        L.dph = M_PI / L.nC;
        L.split = prm.factor_mode == 1 ? 0 : prm.factor_mode == 2 ? 1 : (L.H < 0.5 * lam ? 1 : 0);
        L.nfac = L.split ? 2 : 1;
    }
    // sorted absolute positions (for classification; kept for the adjoint lists)
    p.xs.resize(3 * N);
    std::vector<double> &xs = p.xs;
    for (int64_t s = 0; s < N; s++)
        for (int a = 0; a < 3; a++) xs[3 * s + a] = xyz[3 * p.perm[s] + a];
    // relevant cone segments (Eq. RelevantCones), from d = 3 towards D
    const double tau = prm.cone_band;
    for (int d = 3; d <= D; d++) {
        HostLevel &L = p.lv[d];
        const int words = (L.ncone + 63) / 64;
        std::vector<std::vector<int>> lists(L.nbox);
        const HostLevel *PL = d > 3 ? &p.lv[d - 1] : nullptr;
        // The cones that the parent's cone nodes mark in a child depend only on (parent cone id,
        // child octant): a node's offset from the child centre is its offset from the parent
        // centre plus (1/2 - bit) H_d per axis.  Each used pair is classified once (CSR by key
        // = compact parent cone index * 8 + octant).
        std::vector<int> key_of;
        std::vector<int64_t> mk_start;
        std::vector<int> mk_list;
        if (PL) {
            key_of.assign(PL->ncone, -1);
            std::vector<int> used;
            for (int64_t rc = 0; rc < PL->nrc; rc++) {
                const int g = PL->rc_cone[rc];
                if (key_of[g] < 0) {
                    key_of[g] = 0;
                    used.push_back(g);
                }
            }
            std::sort(used.begin(), used.end());
            for (size_t i = 0; i < used.size(); i++) key_of[used[i]] = (int)i;
            const int64_t nkey = (int64_t)used.size() * 8;
            std::vector<std::vector<int>> kl(nkey);
            std::vector<unsigned char> need(nkey, 0);  // keys some (child box, parent cone) pair uses
            for (int b = 0; b < L.nbox; b++) {
                if (!L.active[b]) continue;
                const int pb = L.parent[b];
                const int o = (L.ijk[3 * b] & 1) + 2 * (L.ijk[3 * b + 1] & 1) + 4 * (L.ijk[3 * b + 2] & 1);
                for (int rc = PL->rc_start[pb]; rc < PL->rc_start[pb + 1]; rc++)
                    need[(int64_t)key_of[PL->rc_cone[rc]] * 8 + o] = 1;
            }
#pragma omp parallel
            {
                std::vector<uint64_t> kb(words, 0ULL);
                std::vector<int> touched;
                std::vector<double> off(3 * (size_t)p.P);
#pragma omp for schedule(dynamic, 4)
                for (int64_t gi = 0; gi < (int64_t)used.size(); gi++) {
                    bool any = false;
                    for (int o = 0; o < 8; o++) any = any || need[gi * 8 + o];
                    if (!any) continue;
                    for (int n = 0; n < p.P; n++) node_offset(p, *PL, used[gi], n, &off[3 * n]);
                    for (int o = 0; o < 8; o++) {
                        if (!need[gi * 8 + o]) continue;
                        const double sx = (0.5 - (o & 1)) * L.H, sy = (0.5 - ((o >> 1) & 1)) * L.H,
                                     sz = (0.5 - ((o >> 2) & 1)) * L.H;
                        touched.clear();
                        for (int n = 0; n < p.P; n++)
                            mark_offset(L, off[3 * n] + sx, off[3 * n + 1] + sy, off[3 * n + 2] + sz, tau, kb.data(),
                                        &touched);
                        std::sort(touched.begin(), touched.end());
                        for (int c : touched) kb[c >> 6] = 0ULL;
                        kl[gi * 8 + o] = touched;
                    }
                }
            }
            mk_start.assign(nkey + 1, 0);
            for (int64_t kk = 0; kk < nkey; kk++) mk_start[kk + 1] = mk_start[kk] + (int64_t)kl[kk].size();
            mk_list.resize(mk_start[nkey]);
            for (int64_t kk = 0; kk < nkey; kk++) std::copy(kl[kk].begin(), kl[kk].end(), mk_list.begin() + mk_start[kk]);
        }
#pragma omp parallel
        {
            std::vector<uint64_t> bits(words);
#pragma omp for schedule(dynamic, 1)
            for (int b = 0; b < L.nbox; b++) {
                if (!L.active[b]) continue;  // no sources: no factor to interpolate
                std::fill(bits.begin(), bits.end(), 0ULL);
                // far-field option: s = h / r -> 0 lies in the segments with is = 0 (cone ids
                // 0 .. nC nph - 1), kept in every direction at level 3
                if (d == 3 && prm.far_field)
                    for (int c = 0; c < L.nC * L.nph; c++) bits[c >> 6] |= 1ULL << (c & 63);
                for (int c = L.co_start[b]; c < L.co_start[b + 1]; c++) {
                    int cb = L.co_list[c];
                    if (!L.alive[cb]) continue;  // points below a coarser leaf take no level-d interpolation
                    for (int s = L.start[cb]; s < L.start[cb + 1]; s++) mark_point(p, L, b, &xs[3 * s], tau, bits.data());
                }
                if (PL) {
                    const int pb = L.parent[b];
                    const int o = (L.ijk[3 * b] & 1) + 2 * (L.ijk[3 * b + 1] & 1) + 4 * (L.ijk[3 * b + 2] & 1);
                    for (int rc = PL->rc_start[pb]; rc < PL->rc_start[pb + 1]; rc++) {
                        const int64_t kk = (int64_t)key_of[PL->rc_cone[rc]] * 8 + o;
                        for (int64_t j = mk_start[kk]; j < mk_start[kk + 1]; j++) {
                            const int c = mk_list[j];
                            bits[c >> 6] |= 1ULL << (c & 63);
                        }
                    }
                }
                std::vector<int> &v = lists[b];
                for (int wi = 0; wi < words; wi++) {
                    uint64_t m = bits[wi];
                    while (m) {
                        int t = __builtin_ctzll(m);
                        v.push_back(wi * 64 + t);
                        m &= m - 1;
                    }
                }
            }
        }
        L.rc_start.assign(L.nbox + 1, 0);
        for (int b = 0; b < L.nbox; b++) L.rc_start[b + 1] = L.rc_start[b] + (int)lists[b].size();
        L.nrc = L.rc_start[L.nbox];
        L.rc_cone.resize(L.nrc);
        L.rc_box.resize(L.nrc);
        L.cone_map.assign((size_t)L.nbox * L.ncone, -1);
        for (int b = 0; b < L.nbox; b++)
            for (size_t j = 0; j < lists[b].size(); j++) {
                int rc = L.rc_start[b] + (int)j;
                L.rc_cone[rc] = lists[b][j];
                L.rc_box[rc] = b;
                L.cone_map[(size_t)b * L.ncone + lists[b][j]] = rc;
            }
        if (PL) {
            int64_t pe = 0;
            for (int b = 0; b < L.nbox; b++)
                if (L.active[b]) pe += (int64_t)(PL->rc_start[L.parent[b] + 1] - PL->rc_start[L.parent[b]]) * p.P;
            p.lv[d - 1].prop_evals = pe;
        }
    }
    // leaf expansions: every level's source leaves (level D: all of its source boxes)
    int64_t le = 0;
    for (int d = 3; d <= D; d++) {
        HostLevel &L = p.lv[d];
        L.leaf_rc.clear();
        for (int b = 0; b < L.nbox; b++) {
            if (!L.leaf[b] || !L.active[b]) continue;
            le += (int64_t)(L.rc_start[b + 1] - L.rc_start[b]) * p.P * (L.start[b + 1] - L.start[b]);
            if (d < D)
                for (int rc = L.rc_start[b]; rc < L.rc_start[b + 1]; rc++) L.leaf_rc.push_back(rc);
        }
    }
    p.leaf_evals = le;
    return IFGF_OK;
}

// Adjoint lists: for every relevant cone of level d, the cousin targets and parent
// cone nodes that the forward apply interpolates from it, classified with the same
// rule as the kernels (no margin band).  Entry order is deterministic.
static int classify_offset(const HostLevel &L, double dx, double dy, double dz) {
    double rho = std::sqrt(dx * dx + dy * dy);
    double r = std::sqrt(dx * dx + dy * dy + dz * dz);
    double s = L.h / r;
    double th = std::atan2(rho, dz);
    double ph = std::atan2(dy, dx);
    if (ph < 0) ph += 2.0 * M_PI;
    if (ph >= 2.0 * M_PI) ph = 0.0;
    double us = snap(s / L.ds), ut = snap(th / L.dth), up = snap(ph / L.dph);
    int is = std::min(std::max((int)std::floor(us), 0), L.ns - 1);
    int it = std::min(std::max((int)std::floor(ut), 0), L.nC - 1);
    int ip = std::min(std::max((int)std::floor(up), 0), L.nph - 1);
    return (is * L.nC + it) * L.nph + ip;
}

static int classify_exact(const Plan &p, const HostLevel &L, int b, const double *x) {
    double y0[3];
    box_center(p, L, b, y0);
    return classify_offset(L, x[0] - y0[0], x[1] - y0[1], x[2] - y0[2]);
}

ifgf_status build_adjoint_lists(Plan &p, const double *xs) {
    const int64_t N = p.N;
    for (int d = 3; d <= p.D; d++) {
        HostLevel &L = p.lv[d];
        const HostLevel *PL = d > 3 ? &p.lv[d - 1] : nullptr;
        // Child cone of every parent cone node, per (parent cone id, child octant) used at this
        // level (translation invariant, as in build_host_plan): node_cone[idx * P + n], idx from
        // key_idx[compact parent cone index * 8 + octant].
        std::vector<int> key_of, key_idx, node_cone;
        if (PL) {
            key_of.assign(PL->ncone, -1);
            std::vector<int> used;
            for (int64_t rc = 0; rc < PL->nrc; rc++) {
                const int g = PL->rc_cone[rc];
                if (key_of[g] < 0) {
                    key_of[g] = 0;
                    used.push_back(g);
                }
            }
            std::sort(used.begin(), used.end());
            for (size_t i = 0; i < used.size(); i++) key_of[used[i]] = (int)i;
            key_idx.assign(used.size() * 8, -1);
            for (int b = 0; b < L.nbox; b++) {
                const int pb = L.parent[b];
                const int o = (L.ijk[3 * b] & 1) + 2 * (L.ijk[3 * b + 1] & 1) + 4 * (L.ijk[3 * b + 2] & 1);
                for (int rc = PL->rc_start[pb]; rc < PL->rc_start[pb + 1]; rc++)
                    key_idx[(size_t)key_of[PL->rc_cone[rc]] * 8 + o] = 0;
            }
            std::vector<int64_t> keys;  // needed (compact cone index * 8 + octant), ascending
            for (size_t kk = 0; kk < key_idx.size(); kk++)
                if (key_idx[kk] == 0) {
                    key_idx[kk] = (int)keys.size();
                    keys.push_back((int64_t)kk);
                }
            node_cone.resize(keys.size() * (size_t)p.P);
#pragma omp parallel
            {
                std::vector<double> off(3 * (size_t)p.P);
                int last = -1;
#pragma omp for schedule(dynamic, 16)
                for (int64_t i = 0; i < (int64_t)keys.size(); i++) {
                    const int gi = (int)(keys[i] / 8), o = (int)(keys[i] % 8);
                    if (gi != last) {
                        for (int n = 0; n < p.P; n++) node_offset(p, *PL, used[gi], n, &off[3 * n]);
                        last = gi;
                    }
                    const double sx = (0.5 - (o & 1)) * L.H, sy = (0.5 - ((o >> 1) & 1)) * L.H,
                                 sz = (0.5 - ((o >> 2) & 1)) * L.H;
                    for (int n = 0; n < p.P; n++)
                        node_cone[i * p.P + n] = classify_offset(L, off[3 * n] + sx, off[3 * n + 1] + sy, off[3 * n + 2] + sz);
                }
            }
        }
        std::vector<std::vector<std::vector<int>>> per_box(L.nbox);
#pragma omp parallel for schedule(dynamic, 1)
        for (int b = 0; b < L.nbox; b++) {
            const int r0 = L.rc_start[b], nr = L.rc_start[b + 1] - r0;
            std::vector<std::vector<int>> &lists = per_box[b];
            lists.assign(nr, std::vector<int>());
            if (nr == 0) continue;
            for (int c = L.co_start[b]; c < L.co_start[b + 1]; c++) {
                int cb = L.co_list[c];
                if (!L.alive[cb]) continue;
                for (int si = L.start[cb]; si < L.start[cb + 1]; si++) {
                    int rc = L.cone_map[(size_t)b * L.ncone + classify_exact(p, L, b, xs + 3 * si)];
                    if (rc >= 0) lists[rc - r0].push_back(si);
                }
            }
            if (PL) {
                const int pb = L.parent[b];
                const int o = (L.ijk[3 * b] & 1) + 2 * (L.ijk[3 * b + 1] & 1) + 4 * (L.ijk[3 * b + 2] & 1);
                for (int rcp = PL->rc_start[pb]; rcp < PL->rc_start[pb + 1]; rcp++) {
                    const int *nc = &node_cone[(size_t)key_idx[(size_t)key_of[PL->rc_cone[rcp]] * 8 + o] * p.P];
                    for (int n = 0; n < p.P; n++) {
                        int rc = L.cone_map[(size_t)b * L.ncone + nc[n]];
                        if (rc >= 0) lists[rc - r0].push_back((int)(N + (int64_t)rcp * p.P + n));
                    }
                }
            }
        }
        L.ad_start.assign(L.nrc + 1, 0);
        for (int b = 0; b < L.nbox; b++)
            for (size_t j = 0; j < per_box[b].size(); j++) L.ad_start[L.rc_start[b] + j + 1] = per_box[b][j].size();
        for (int64_t r = 0; r < L.nrc; r++) L.ad_start[r + 1] += L.ad_start[r];
        L.ad_list.resize(L.ad_start[L.nrc]);
        for (int b = 0; b < L.nbox; b++)
            for (size_t j = 0; j < per_box[b].size(); j++)
                std::copy(per_box[b][j].begin(), per_box[b][j].end(), L.ad_list.begin() + L.ad_start[L.rc_start[b] + j]);
    }
    return IFGF_OK;
}

// Forward cousin lists of the mixed path: for every relevant cone (box c, cone gamma) of level d,
// the targets x in c's cousin boxes that fall in gamma (Eq. NeighborsCousins is symmetric: x is
// a cousin point of c iff c is a cousin of x's box), classified in FP64 with the rule of the
// adjoint lists, in cousin-list then Morton order.  Each entry packs x's sorted position and
// the slot of c in the cousin list of x's box; cs_pvoff gives the value-buffer block of each box.
ifgf_status build_cousin_lists(Plan &p) {
    const int64_t N = p.N;
    p.cs_ok = N < (int64_t(1) << 24);
    p.cs_max_entries = 0;
    for (int d = 3; d <= p.D && p.cs_ok; d++) p.cs_ok = p.lv[d].cousin_evals < (int64_t(1) << 31);
    if (!p.cs_ok) return IFGF_OK;  // the kernels fall back to the target-stationary cousin interpolation
    const double *xs = p.xs.data();
    for (int d = 3; d <= p.D; d++) {
        HostLevel &L = p.lv[d];
        // slot of box c in the cousin list of each of its cousins
        std::vector<uint8_t> rev(L.co_list.size());
        int bad = 0;
#pragma omp parallel for schedule(dynamic, 16) reduction(| : bad)
        for (int c = 0; c < L.nbox; c++)
            for (int ci = L.co_start[c]; ci < L.co_start[c + 1]; ci++) {
                const int cb = L.co_list[ci];
                int j = -1;
                for (int k = L.co_start[cb]; k < L.co_start[cb + 1]; k++)
                    if (L.co_list[k] == c) {
                        j = k - L.co_start[cb];
                        break;
                    }
                if (j < 0 || j > 255) bad |= 1;
                else rev[ci] = (uint8_t)j;
            }
        if (bad) {  // more than 256 cousins or an asymmetric relation: keep the other kernel
            p.cs_ok = false;
            return IFGF_OK;
        }
        std::vector<std::vector<std::vector<uint32_t>>> per_box(L.nbox);
        int miss = 0;
#pragma omp parallel for schedule(dynamic, 1) reduction(| : miss)
        for (int c = 0; c < L.nbox; c++) {
            const int r0 = L.rc_start[c], nr = L.rc_start[c + 1] - r0;
            std::vector<std::vector<uint32_t>> &lists = per_box[c];
            lists.assign(nr, std::vector<uint32_t>());
            for (int ci = L.co_start[c]; ci < L.co_start[c + 1] && nr > 0; ci++) {
                const int cb = L.co_list[ci];
                if (!L.alive[cb]) continue;  // no level-d box for these points
                const uint32_t slot = (uint32_t)rev[ci] << 24;
                for (int si = L.start[cb]; si < L.start[cb + 1]; si++) {
                    const int rc = L.cone_map[(size_t)c * L.ncone + classify_exact(p, L, c, xs + 3 * si)];
                    if (rc < 0) {
                        miss |= 1;
                        continue;
                    }
                    lists[rc - r0].push_back((uint32_t)si | slot);
                }
            }
        }
        if (miss) {
            set_error("cousin lists: a cousin target falls outside the relevant cone segments");
            return IFGF_EINVAL;
        }
        L.cs_start.assign(L.nrc + 1, 0);
        for (int c = 0; c < L.nbox; c++)
            for (size_t j = 0; j < per_box[c].size(); j++) L.cs_start[L.rc_start[c] + j + 1] = per_box[c][j].size();
        for (int64_t r = 0; r < L.nrc; r++) L.cs_start[r + 1] += L.cs_start[r];
        L.cs_ent.resize(L.cs_start[L.nrc]);
        for (int c = 0; c < L.nbox; c++) {
            for (size_t j = 0; j < per_box[c].size(); j++)
                std::copy(per_box[c][j].begin(), per_box[c][j].end(), L.cs_ent.begin() + L.cs_start[L.rc_start[c] + j]);
            std::vector<std::vector<uint32_t>>().swap(per_box[c]);
        }
        L.cs_pvoff.assign(L.nbox + 1, 0);
        int64_t off = 0;
        for (int b = 0; b < L.nbox; b++) {
            L.cs_pvoff[b] = (int)off;
            off += (int64_t)(L.co_start[b + 1] - L.co_start[b]) * (L.start[b + 1] - L.start[b]);
        }
        L.cs_pvoff[L.nbox] = (int)off;
        // the value buffer has a slot for every cousin (those without sources stay zero); the entries
        // cover the (source box, cousin point) pairs
        if ((int64_t)L.cs_ent.size() != L.cousin_evals || (!p.has_inactive && off != L.cousin_evals)) {
            set_error("cousin lists: %lld entries for %lld cousin pairs", (long long)L.cs_ent.size(),
                      (long long)L.cousin_evals);
            return IFGF_EINVAL;
        }
        p.cs_max_entries = std::max(p.cs_max_entries, off);
    }
    return IFGF_OK;
}

}  // namespace ifgf

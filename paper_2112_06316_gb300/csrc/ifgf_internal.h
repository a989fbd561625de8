// Internal structures of the GB300 IFGF library (not part of the C ABI).
#pragma once
#include <cstdint>
#include <string>
#include <vector>

#include <cuda_runtime.h>

#include "../../include/ifgf.h"

namespace ifgf {

constexpr int kMaxP = 12;  // largest supported points per axis

void set_error(const char *fmt, ...);

// Chebyshev first-kind nodes x_j = cos((2j+1) pi / (2n)) and Lagrange product
// weights c_j = 1 / prod_{m != j} (x_j - x_m) for one axis (Section 3.2).
struct ChebAxis {
    int n;
    double x[kMaxP], c[kMaxP];
};
void cheb_axis(int n, ChebAxis *a);

// Host-side description of one octree level (Section 3.4).
struct HostLevel {
    int d = 0;
    int nbox = 0;
    double H = 0, h = 0;      // box side and half diagonal sqrt(3)/2 H (Eq. def_eps)
    int scale = 1;            // box side in leaf units, 2^(D-d)
    std::vector<int> ijk;     // 3 * nbox integer coordinates at this level
    std::vector<int> start;   // nbox + 1 ranges into the Morton-sorted points
    std::vector<int> parent;  // index of the parent box (level d-1), -1 at d = 1
    std::vector<int> ch_start, ch_list;  // children (level d+1) CSR
    std::vector<int> co_start, co_list;  // cousins CSR (Eq. NeighborsCousins)
    std::vector<uint64_t> mkey;          // Morton key of each box (sorted)
    int ns = 0, nC = 0, nph = 0, ncone = 0;
    double ds = 0, dth = 0, dph = 0;
    int split = 0, nfac = 1;
    // source boxes: boxes holding a point of positive weight (all boxes unless the plan has targets);
    // the others have no relevant cones, no children in ch_list and act on nothing
    std::vector<uint8_t> active;
    // adaptive octree: a box exists (alive) when every ancestor is subdivided; a leaf is alive and not
    // subdivided.  Uniform trees: all boxes alive, leaves at level D.  `active` implies alive.
    std::vector<uint8_t> alive, leaf;
    std::vector<int> leaf_rc;  // relevant cones of the source leaf boxes of this level (levels < D)
    std::vector<int> rc_start, rc_cone, rc_box;  // relevant cones (Eq. RelevantCones)
    std::vector<int> cone_map;                   // nbox * ncone -> rc index or -1
    int64_t nrc = 0;
    // adjoint: for every relevant cone, the forward interpolations that read it:
    // entries e < N are cousin targets (sorted positions); e >= N are parent cone
    // nodes (e - N = parent rc * P + node)
    std::vector<int64_t> ad_start;
    std::vector<int> ad_list;
    int64_t cousin_evals = 0, prop_evals = 0;
    // forward cousin lists of the mixed path (host copies, released after upload): for every
    // relevant cone, the cousin targets it serves as (sorted position | slot << 24), where slot is
    // the cone owner's index in the target box's cousin list; cs_pvoff[b] = first entry of box b
    // in the per-(box, slot, target) value buffer ([slot][target in b] blocks)
    std::vector<int64_t> cs_start;
    std::vector<uint32_t> cs_ent;
    std::vector<int> cs_pvoff;
};

// Tensor-core propagation into level d-1 (mixed path, Pang = 8): pairs (parent
// relevant cone, child box) grouped by (child octant, parent cone id) — the
// propagation weights depend only on that key — and cut into tiles of up to
// kTcTile pairs; tiles are ordered by octant so one launch per octant never
// writes the same parent cone twice.
constexpr int kTcTile = 64;   // pairs per tile
constexpr int kCsItem = 64;   // cousin targets per work item of the cone-stationary interpolation (two per lane)
constexpr int kTcPairs = 32;  // pairs per block of the warp-level (mma.sync) engine: a tile is two blocks
struct TcLevel {
    int ntiles = 0, ngroups = 0;
    double fill = 0.0;  // pairs / (tiles * kTcTile)
    int oct_tile_start[9] = {};
    int *tile_group = nullptr, *tile_start = nullptr, *tile_count = nullptr;
    int *grp_gamma = nullptr, *grp_pb = nullptr, *grp_cb = nullptr;
    int *pair_rcp = nullptr, *pair_cb = nullptr;
    // per group, filled once per plan on the device: the P parent nodes ordered by the child
    // cone they fall in (ascending cone id, then node), and the distinct child cones (<= 16)
    short *grp_perm = nullptr;
    int *grp_cones = nullptr, *grp_nc = nullptr;
    int *grp_cnt = nullptr;  // 17 per group: nodes per cone slot (slot 16: nodes of further cones)
    // work items of the tcgen05 engine, ordered by octant: (tile, first row in the group's node
    // order, rows <= 128, cone slot) -- every item's rows fall in one child cone
    int4 *items = nullptr;
    int nitems = 0;
    // per item, filled once per plan: header (row0, rows, group, gamma), (child cone id, first pair,
    // pairs, 0), (child-centre offset from the parent centre, 0) and the pairs' child-cone storage
    // indices (kTcTile ints, -1 beyond the tile's pairs)
    int4 *item_hdr = nullptr;
    int *item_crc = nullptr;
    int oct_item_start[9] = {};
    bool items_ok = false;  // every group has at most 16 child cones
    // work items of the cone-stationary CUDA-core propagation, ordered by octant: (tile, first row
    // in the group's node order, rows <= 64, cone slot) -- one warp each
    int4 *cs_items = nullptr;
    int ncs_items = 0;
    int oct_cs_start[9] = {};
};

// Device arrays of one level.
struct DevLevel {
    int nbox, ns, nC, nph, ncone, split, nfac, scale;
    int64_t nrc;
    double H, h, ds, dth, dph;
    int *ijk, *start, *parent, *ch_start, *ch_list, *co_start, *co_list;
    int *rc_start, *rc_cone, *rc_box, *cone_map;
};

struct Workspace {
    int nrhs = 0;
    int prec = -1;
    size_t bytes = 0;
    void *base = nullptr;
    void *a = nullptr;   // w * sigma in sorted order, [nrhs][N]
    void *u = nullptr;   // accumulated field in sorted order, [nrhs][N]
    void *F[IFGF_MAXD + 1] = {};  // cone values per level, [nrhs][nrc][nfac][Pstride]
    void *pv = nullptr;  // mixed path: one level's cousin-interpolation values, [nrhs][pairs]
    void *ap = nullptr;  // mixed path: weighted densities of the source pairs, [nrhs][npairs] float4
};

// byte offsets of the workspace parts (workspace_layout)
struct WorkspaceLayout {
    size_t a = 0, u = 0, F[IFGF_MAXD + 1] = {}, pv = 0, ap = 0, total = 0;
};

struct Plan {
    ifgf_params prm;
    int64_t N = 0;
    int D = 0;
    int Ps = 3, Pang = 5, P = 75, Pstride = 76;
    double c0[3] = {0, 0, 0};  // root box corner (centre - L/2)
    double center[3] = {0, 0, 0};
    double L = 0, HD = 0;
    ChebAxis cs, ca;
    std::vector<HostLevel> lv;  // index d = 0..D
    std::vector<int> perm;      // sorted position -> caller index
    std::vector<double> xs;     // sorted absolute positions (host copy)
    std::vector<int> leaf_of;   // sorted position -> leaf box
    int64_t leaf_evals = 0, near_pairs = 0;
    std::vector<int> nb_start, nb_list;  // leaf neighbours (27-neighbourhood incl. self)

    // device copies
    int device = 0;
    DevLevel dl[IFGF_MAXD + 1] = {};
    int *d_perm = nullptr;
    int *d_leaf_of = nullptr;
    int *d_box_of[IFGF_MAXD + 1] = {};  // sorted position -> box index at level d
    // cousin-interpolation work chunks of level d: (box, first sorted target, count <= 32, 0);
    // the targets of every box split into near-equal runs of at most 32
    int4 *d_cchunk[IFGF_MAXD + 1] = {};
    int ncchunk[IFGF_MAXD + 1] = {};
    // cone-stationary cousin interpolation (mixed path; needs N < 2^24 and fewer than 2^31
    // (target, cousin) pairs per level): work items (relevant cone, first entry, count <= 64),
    // packed entries and per-box offsets of the value buffer (HostLevel::cs_*)
    bool cs_ok = false;
    // CUDA-core interpolation kernels: 1 = cone-stationary (cousin lists; grouped propagation where
    // the tensor-core tables exist and the tensor cores do not take the level), 0 = point-stationary
    // (k_cousin_w, k_prop_w)
    int interp_engine = 1;
    int4 *d_cs_item[IFGF_MAXD + 1] = {};
    int ncs_item[IFGF_MAXD + 1] = {};
    // per entry, FP64-computed once per plan: (local coordinates t_s, t_theta, t_phi, Re E) and
    // (Im E, value-buffer slot as int bits)
    float4 *d_cs_geo4[IFGF_MAXD + 1] = {};
    int *d_cs_first[IFGF_MAXD + 1] = {};  // per relevant cone: its first entry (the adjoint reuses the geometry)
    uint8_t *d_alive[IFGF_MAXD + 1] = {};  // per box: it exists (adaptive octree; all 1 otherwise)
    uint8_t *d_leaf[IFGF_MAXD + 1] = {};   // per box: it is a leaf (level D: every existing box)
    int *d_leaf_rc[IFGF_MAXD + 1] = {};    // relevant cones of the level's source leaves (levels < D)
    int nleaf_rc[IFGF_MAXD + 1] = {};
    float2 *d_cs_geo2[IFGF_MAXD + 1] = {};
    int *d_cs_pvoff[IFGF_MAXD + 1] = {};
    int64_t cs_max_entries = 0;  // largest per-level pair count (size of the value buffer per rhs)
    int *d_nb_start = nullptr, *d_nb_list = nullptr;
    // near-field work chunks: (leaf box, first sorted target, count <= 64, 0), the targets of every
    // leaf box in near-equal runs of at most 64
    int4 *d_nchunk = nullptr;
    int nnchunk = 0;
    int nnchunk_light = 0;  // adaptive trees: the chunks before it run one warp each, the rest one block each
    double *d_x64 = nullptr, *d_n64 = nullptr, *d_w64 = nullptr;  // sorted, absolute FP64
    float *d_f32 = nullptr, *d_n32 = nullptr, *d_w32 = nullptr;   // sorted, leaf offsets / normals / weights
    float4 *d_pn32 = nullptr;                                      // sorted, (offset, |offset|^2), (normal, 0)
    // sources of every leaf box in pairs (the packed leaf kernel): 4 float4 records per pair, the first
    // pair of box b at pstart[b], (sorted index, sorted index or -1) per pair
    float4 *d_pp32 = nullptr;
    int *d_pstart = nullptr;
    int2 *d_pair_src = nullptr;
    // adaptive trees: per leaf (in point order) its near sources as (point start, point end, pair start,
    // pair end) ranges; per point its level-D box coordinates packed 21 bits per axis
    int *d_nr_start = nullptr;
    int4 *d_nr = nullptr;
    unsigned long long *d_pt_ijk = nullptr;
    unsigned long long *d_pair_ijk = nullptr;  // per source pair: its level-D box, packed the same way
    int npairs = 0;
    unsigned long long *d_missed = nullptr;
    TcLevel tc[IFGF_MAXD + 1];  // tc[d]: propagation from level d into level d-1
    bool use_tc = false;
    // a level uses the tensor-core propagation when its tile fill reaches this value
    double tc_min_fill = 0.4;
    // tensor-core propagation engine: 1 = tcgen05 (TMEM accumulators), 0 = warp-level mma.sync
    int tc_engine = 1;
    int num_sms = 152;  // multiprocessors of the plan's device
    std::vector<void *> allocs;
    int64_t device_bytes = 0;

    // sparse correction (CSR in sorted order)
    int64_t corr_nnz = 0;
    int64_t *d_corr_rowptr = nullptr;
    int *d_corr_col = nullptr;
    double *d_corr_val64 = nullptr;
    float *d_corr_val32 = nullptr;

    Workspace ws;

    // adjoint structures (built on the first adjoint apply)
    bool adj_ready = false;
    int64_t *d_ad_start[IFGF_MAXD + 1] = {};
    int *d_ad_list[IFGF_MAXD + 1] = {};
    int64_t *d_corrT_rowptr = nullptr;
    int *d_corrT_col = nullptr;
    double *d_corrT_val64 = nullptr;
    float *d_corrT_val32 = nullptr;
    void *adj_ws = nullptr;      // [nrhs][N] gathered g and accumulated b, plus per-level G
    size_t adj_ws_bytes = 0;
    void *dk_ws = nullptr;       // k-gradient: one level's anterpolated H plus the partial sums
    size_t dk_ws_bytes = 0;
    // plans built with off-surface targets (ifgf_plan_create_with_targets): the points are the n_src
    // sources followed by the n_tgt targets (weight 0); N = n_src + n_tgt.  0, 0 for an ordinary plan.
    int64_t n_src = 0, n_tgt = 0;
    bool has_inactive = false;  // some box holds targets only or lies below a leaf (see HostLevel)
    bool adaptive = false;      // leaves at several levels (params.leaf_max > 0)
    void *field_ws = nullptr;    // off-surface / far-field evaluation: gathered w*sigma and per-chunk partial sums
    size_t field_ws_bytes = 0;

    // bumped whenever device buffers baked into a captured graph may change
    uint64_t gen = 0;
    // tunable: right-hand sides per register block in the mixed interpolation kernels (1 or 4)
    int rhs_block = 4;

    // concurrent stages: the near field and the cousin interpolation run on an auxiliary stream,
    // ordered after the gather, the leaf evaluation and each propagation by the dep events
    cudaStream_t aux = nullptr;
    static constexpr int kMaxDep = IFGF_MAXD + 3;
    cudaEvent_t dep[kMaxDep] = {};

    // anterpolation list pointers of one level (device)
    struct AntArgs {
        const long long *start;
        const int *list;
    };

    // set for the duration of ifgf_far_field_ifgf: the forward launch sequence stops after the
    // leaf expansions and the propagation (no near field, cousin interpolation or scatter)
    bool upward_only = false;

    // optional per-launch timing (events recorded on the apply stream; the apply then runs on
    // that stream alone so that every launch has its own interval)
    bool profile = false;
    static constexpr int kMaxEv = 80;
    cudaEvent_t ev[kMaxEv] = {};
    int nev = 0;                 // events recorded by the last apply
    int ev_kind[kMaxEv] = {};    // stage kind of launch i (between event i and i+1)
    int ev_level[kMaxEv] = {};
};

// stage kinds reported by ifgf_plan_stage_times
enum StageKind {
    kStGather = 0, kStLeaf = 1, kStProp = 2, kStNear = 3, kStCousin = 4, kStScatter = 5, kStCorr = 6,
    kStPropTc = 7,    // propagation on the tensor cores
    kStCousinSum = 8,  // second pass of the cone-stationary cousin interpolation
    kStPropCs = 9      // cone-stationary propagation on CUDA cores (all its octant launches)
};

// Coupling of the kernel alpha dPhi/dnu(y) + beta Phi written as beta = -i (eta + i etai): the combined
// field of Eq. CombinedLayer is (eta, 0), the double layer alone (0, 0), the single layer alone (0, 1)
// (beta = 1; its alpha = 0 is carried by zero device normals).
inline void coupling(const ifgf_params &pr, double &eta, double &etai) {
    eta = pr.layer == IFGF_LAYER_COMBINED ? pr.eta : 0.0;
    etai = pr.layer == IFGF_LAYER_SINGLE ? 1.0 : 0.0;
}

inline void prof_begin(Plan &p, cudaStream_t s) {
    p.nev = 0;
    if (p.profile) cudaEventRecord(p.ev[p.nev++], s);
}
inline void prof_mark(Plan &p, cudaStream_t s, int kind, int level) {
    if (p.profile && p.nev < Plan::kMaxEv) {
        p.ev_kind[p.nev - 1] = kind;
        p.ev_level[p.nev - 1] = level;
        cudaEventRecord(p.ev[p.nev++], s);
    }
}

// plan.cpp
ifgf_status build_host_plan(Plan &p, const double *xyz, const double *nrm, const double *w);
ifgf_status build_adjoint_lists(Plan &p, const double *xs_sorted);
ifgf_status build_cousin_lists(Plan &p);
int morton_levels_auto(const double *xyz, int64_t N, const double *c0, double L, double leaf_target);

// apply.cu
ifgf_status upload_plan(Plan &p, const double *xyz, const double *nrm, const double *w, cudaStream_t s);
size_t workspace_layout(const Plan &p, int nrhs, int prec, WorkspaceLayout &lay);
void workspace_bind(Workspace &ws, const Plan &p, void *base, const WorkspaceLayout &lay, int nrhs, int prec);
ifgf_status ensure_workspace(Plan &p, int nrhs, int prec);
ifgf_status run_apply(Plan &p, const void *sigma, void *y, int nrhs, int prec, cudaStream_t s);
void free_plan_device(Plan &p);

}  // namespace ifgf

// The opaque handle of the C ABI.
struct ifgf_plan {
    ifgf::Plan p;
};

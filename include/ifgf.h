/*
 * ifgf.h -- C ABI of the GB300 IFGF-accelerated combined-field (CFIE) operator.
 *
 * The library applies the discrete combined-field boundary operator of a
 * sound-soft scatterer (Jimenez, Bauinger, Bruno, "IFGF-accelerated high-order
 * integral equation solver for acoustic wave scattering"):
 *
 *   y_l = c_I sigma_l + sum_{m != l} K(x_l, x_m) w_m sigma_m  (+ (C sigma)_l),
 *   K(x, y) = dPhi(x,y)/dnu(y) - i eta Phi(x,y),  Phi = e^{ik|x-y|} / (4 pi |x-y|)
 *
 * i.e. the regular-quadrature discretisation (Eq. ReguIntOpQuadrature) of the
 * combined-field equation (Eq. CombLayIE, c_I = 1/2, eta the coupling
 * parameter gamma) written as the discrete sum of Eq. field1, plus an optional
 * sparse singular/near-singular correction C (Eq. IntOpAtSing minus the regular
 * rows it replaces).  The far interactions are evaluated by the interpolated
 * factored Green function (IFGF) recursion of Algorithm 1 (Section 3.4); the
 * level-D neighbour interactions by direct summation (Remark level_D_neighboring).
 *
 * Conventions shared by every call:
 *  - Status: every call returns IFGF_OK (0) or a negative ifgf_status and, on
 *    error, records a message readable with ifgf_last_error() (thread-local).
 *    Outputs are unspecified after an error.
 *  - Host inputs (points, normals, weights, correction arrays) are copied; the
 *    caller keeps ownership.  Device buffers passed to apply-type calls belong to
 *    the caller, are never freed by the library and must not alias each other.
 *  - Densities are complex, stored column-major N x nrhs (right-hand side j is
 *    the contiguous block [j*N, (j+1)*N)), interleaved (re, im): complex128
 *    (double2) for IFGF_FP64, complex64 (float2) for IFGF_MIXED.  Points keep
 *    the caller's order; the library permutes internally.
 *  - Streams: `stream` is a cudaStream_t (NULL = legacy default stream).  Apply
 *    calls are asynchronous on it; plan creation and GMRES synchronise.  A plan
 *    serves one stream at a time.  Inside a forward apply the near field and the
 *    cousin interpolation run on a stream owned by the plan, forked from and
 *    joined back into `stream` by events, so every effect of the call is ordered
 *    on `stream` (this also holds inside CUDA graph capture).
 */
#ifndef IFGF_H
#define IFGF_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    IFGF_OK = 0,
    IFGF_EINVAL = -1,        /* invalid argument (sizes, NaN/Inf, non-unit normal, ...) */
    IFGF_ENOMEM = -2,        /* host or device allocation failed */
    IFGF_ECUDA = -3,         /* a CUDA runtime call failed */
    IFGF_ENOTCONVERGED = -4, /* GMRES reached maxit above the tolerance */
    IFGF_EUNSUPPORTED = -5,  /* valid request this build does not implement (e.g. Ps/Pang pair) */
    IFGF_EINTERNAL = -6      /* consistency check failed inside the library */
} ifgf_status;

typedef enum {
    IFGF_FP64 = 0,  /* all arithmetic in FP64, densities complex128 */
    IFGF_MIXED = 1  /* FP32 kernel evaluation and interpolation with compensated FP32
                       accumulation; the phase k|x - y| is reduced exactly from integer box
                       offsets plus an FP32 fraction; densities complex64 */
} ifgf_precision;

/* Parameters of the plan.  Fill with ifgf_params_default() and override. */
typedef struct {
    double k;             /* wavenumber (> 0), Eq. ScalarHelmholtz */
    double eta;           /* coupling parameter gamma of Eq. CombinedLayer (default k) */
    int Ps, Pang;         /* Chebyshev points per cone segment in s and in each angle
                             (Section 3.2; paper: 3 and 5); supported pairs listed by
                             ifgf_supported_orders() */
    int nC0, nS0;         /* cone counts of the coarsest cone grid (Remark cone_seg_size; 2, 1) */
    int levels;           /* octree levels D >= 3; 0 = automatic (mean points per leaf closest
                             to leaf_target on a log scale) */
    double leaf_target;   /* target mean points per relevant leaf for automatic D (64) */
    int cone_rule;        /* 0: (n_s, n_C) doubled each time H_d exceeds lambda/2 * 2^e;
                             1: literal Remark cone_seg_size (doubling from level d to d-1 when
                             k H_d > 1/2, leaf level at (nS0, nC0)) */
    int factor_mode;      /* 0: hybrid - split factors {W2, -ikW3 - i eta W1} on levels with
                             H < lambda/2, combined W~2 - ikW3 - i eta W1 above (Section 3.3);
                             1: combined everywhere; 2: split everywhere */
    double identity_coef; /* c_I: 0.5 for Eq. CombLayIE, 0.0 for the bare sum of Eq. field1 */
    double root_center[3];/* root box centre; used only when root_side > 0 */
    double root_side;     /* <= 0: centre = AABB midpoint, side = max extent * (1 + 2^-30) */
    double cone_band;     /* relative margin used when marking relevant cone segments
                             (Eq. RelevantCones) so that a point within this fraction of a cone
                             boundary marks both neighbours; keeps the FP32 classification
                             inside the relevant set.  Default 1e-4; 0 = exact marking. */
    int far_field;        /* 1: also keep every level-3 cone segment with is = 0 (all directions
                             of the s -> 0 end of the cone grid) relevant, and the segments of
                             the finer levels that feed them, so that ifgf_far_field_ifgf can
                             evaluate the far-field pattern from the level-3 interpolants.
                             Adds work to every apply of the plan.  Default 0. */
    int layer;            /* kernel of the operator (ifgf_layer): IFGF_LAYER_COMBINED (default) the
                             combined field dPhi/dnu(y) - i eta Phi of Eq. CombinedLayer;
                             IFGF_LAYER_DOUBLE the double layer dPhi/dnu(y) alone (Eq. double_layer);
                             IFGF_LAYER_SINGLE the single layer Phi alone (Eq. GreenFunction), for
                             other formulations (Section 2).  eta is ignored by the last two.  Applies
                             to every evaluation of the plan: apply, adjoint, k-gradient, off-surface
                             potential and far fields.  The rectangular-polar correction
                             (ifgf_rp_correction*) is built for the combined kernel; it is linear in eta,
                             so the double layer's is C(eta = 0) and the single layer's
                             i (C(eta = 1) - C(eta = 0)). */
    int leaf_max;         /* 0 (default): uniform octree, every leaf at level `levels`.  > 0: adaptive
                             octree for non-uniform point densities: a box of level 3..D-1 holding at
                             most leaf_max points is a leaf (its factor comes from its points directly
                             and no boxes exist below it), `levels` is the maximum depth.  Points of
                             two leaves interact directly when their boxes neighbour at the coarser
                             of the two leaf levels; every other pair goes through one cousin
                             interpolation.  The adjoint and the k-gradient cover adaptive
                             plans (the transposed leaf evaluation at every level's leaves). */
} ifgf_params;

/* Values of ifgf_params.layer. */
typedef enum { IFGF_LAYER_COMBINED = 0, IFGF_LAYER_DOUBLE = 1, IFGF_LAYER_SINGLE = 2 } ifgf_layer;

/* Plan statistics (ifgf_plan_info). Arrays are indexed by level d (0..IFGF_MAXD). */
#define IFGF_MAXD 20
typedef struct {
    int64_t N;
    int D;
    double root_center[3], root_side;
    int nbox[IFGF_MAXD + 1];      /* relevant boxes per level (Eq. RelevantBoxes) */
    int ns[IFGF_MAXD + 1];        /* cone counts per level */
    int nC[IFGF_MAXD + 1];
    int split[IFGF_MAXD + 1];     /* 1 when the level interpolates the split factor pair */
    int64_t nrc[IFGF_MAXD + 1];   /* relevant cone segments per level */
    int64_t cousin_evals[IFGF_MAXD + 1]; /* target interpolations per level */
    int64_t prop_evals[IFGF_MAXD + 1];   /* interpolations into this level's cone nodes */
    int64_t leaf_evals;           /* factor evaluations at leaf cone nodes (level D; every level's
                                     leaves in an adaptive tree) */
    int64_t near_pairs;           /* near-field pairs (including l == m slots) */
    int64_t correction_nnz;       /* stored correction entries (0 if none) */
    int64_t device_bytes;         /* device memory held by the plan (excluding workspaces) */
    int64_t near_block_chunks;    /* adaptive trees: near-field chunks (at most 64 targets of one leaf)
                                     whose long source lists run as one thread block each; 0 for
                                     uniform trees and from ifgf_plan_dry_run */
} ifgf_info;

typedef struct ifgf_plan ifgf_plan;

/* Default parameters for wavenumber k: eta = k, Ps = 3, Pang = 5, nC0 = 2, nS0 = 1,
 * levels = 0, leaf_target = 64, cone_rule = 0, factor_mode = 0, identity_coef = 0.5,
 * root_side = 0, cone_band = 1e-4. */
void ifgf_params_default(ifgf_params *p, double k);

/* Comma-separated list of compiled (Ps, Pang) pairs, e.g. "3x5,4x6". Static string. */
const char *ifgf_supported_orders(void);

/* Build the plan (Section 3.4 octree, Eq. RelevantBoxes, Eq. NeighborsCousins,
 * Eq. RelevantCones) for N points on the current CUDA device and upload it.
 *   xyz, normals: host, N x 3 row-major (x0,y0,z0,x1,...), FP64; normals unit length.
 *   weights: host, N quadrature area weights (> 0).
 *   stream: used for the uploads; the call synchronises it before returning.
 *   out: receives the plan (NULL on error).
 * Errors: IFGF_EINVAL (N < 1, non-finite input, |normal| not 1 within 1e-6, weight <= 0,
 * k <= 0, levels in 1..2 or > 16), IFGF_EUNSUPPORTED (Ps/Pang pair not compiled),
 * IFGF_ENOMEM, IFGF_ECUDA. */
ifgf_status ifgf_plan_create(const double *xyz, const double *normals, const double *weights, int64_t N,
                             const ifgf_params *params, void *stream, ifgf_plan **out);

/* Host-only dry run of ifgf_plan_create: builds the octree and relevant cone
 * segments on the host and fills `out` (device_bytes = 0) without touching any
 * GPU.  Same arguments and errors as ifgf_plan_create (no CUDA errors). */
ifgf_status ifgf_plan_dry_run(const double *xyz, const double *normals, const double *weights, int64_t N,
                              const ifgf_params *params, ifgf_info *out);

/* Attach a sparse correction C (CSR over the caller's point order): row l holds the
 * entries (col[j], val[j]) for j in rowptr[l]..rowptr[l+1]-1; val interleaved complex128.
 * Host arrays, copied.  nnz = rowptr[N].  Passing nnz = 0 removes the correction.
 * Errors: IFGF_EINVAL (rowptr not monotone, col out of range, non-finite value). */
ifgf_status ifgf_plan_set_correction(ifgf_plan *plan, const int64_t *rowptr, const int32_t *col,
                                     const double *val, int64_t nnz);

/* y = A sigma for nrhs right-hand sides (Algorithm 1 + near field + c_I sigma + C sigma).
 * sigma_dev, y_dev: device, N x nrhs complex (see precision).  Asynchronous on stream.
 * The plan's workspace grows on first use for a given nrhs (device allocation).
 * Errors: IFGF_EINVAL (nrhs < 0, null pointers with nrhs > 0), IFGF_ENOMEM, IFGF_ECUDA. */
ifgf_status ifgf_apply(ifgf_plan *plan, const void *sigma_dev, void *y_dev, int nrhs, ifgf_precision prec,
                       void *stream);

/* out = A^H g: the conjugate transpose of the operator applied by ifgf_apply
 * (every stage of Algorithm 1 transposed and run in reverse order: anterpolation
 * from cousin targets and parent cone nodes into each level's cone values, level
 * by level from d = 3 down to D, then the transposed leaf evaluation, the
 * transposed near field, conj(c_I) g and C^H g).  The paper has no adjoint; it is
 * the exact transpose of the discrete FP64 operator (up to rounding) and of the
 * mixed operator up to FP32 rounding of the cone assignment near cone boundaries.
 * Same layout, precision and error conventions as ifgf_apply.  The first call
 * builds the anterpolation lists on the host (synchronous; memory ~ 4 bytes per
 * cousin interpolation and per propagation evaluation); its workspace grows like
 * ifgf_apply's. */
ifgf_status ifgf_apply_adjoint(ifgf_plan *plan, const void *g_dev, void *out_dev, int nrhs, ifgf_precision prec,
                               void *stream);

/* Vector-Jacobian product of y = A(k) sigma for reverse-mode differentiation:
 *   gsigma = A^H g                        (device, N x nrhs, same precision as sigma)
 *   *dk    = Re sum_rhs <g, (dA/dk) sigma> (host double; may be NULL to skip)
 * dA/dk is the derivative with the plan frozen (octree, cone grids and relevant
 * cones fixed, which the piecewise-constant cone rule makes exact for small k
 * changes), the coupling eta held fixed, and the correction C treated as a
 * constant.  It is assembled from four fused reductions that pair the forward
 * cone values with the adjoint cone values (near field, cousin interpolation,
 * propagation ratios, leaf factors).  The paper has no adjoint or k-derivative.
 * Runs one forward apply and one adjoint apply internally (gsigma is used as
 * scratch for the forward output); the k-derivative of the cousin and propagation
 * stages is reduced inside the adjoint's anterpolation, that of the leaf
 * evaluation and the near field by two more passes.  Synchronises `stream` when
 * dk is requested.
 * Errors as ifgf_apply; sigma, g and gsigma must be distinct. */
ifgf_status ifgf_apply_vjp(ifgf_plan *plan, const void *sigma_dev, const void *g_dev, void *gsigma_dev, int nrhs,
                           double *dk_host, ifgf_precision prec, void *stream);

/* Bytes of the workspace that an apply with nrhs right-hand sides in precision prec
 * uses: w*sigma and the field in Morton order, every level's cone values and, on
 * the mixed path, the cousin-interpolation value buffer.  Host-only, synchronous.
 * Errors: IFGF_EINVAL. */
ifgf_status ifgf_plan_workspace_bytes(const ifgf_plan *plan, int nrhs, ifgf_precision prec, int64_t *bytes);

/* ifgf_apply on a caller-owned workspace: ws_dev is device memory of at least
 * ifgf_plan_workspace_bytes(nrhs, prec) bytes, 256-byte aligned, not aliasing
 * sigma or y; the library neither keeps nor frees it.  After the call (in stream
 * order) ws_dev holds the forward state of this sigma -- w*sigma in Morton order
 * and every level's cone values -- which ifgf_apply_vjp_ws reads, so a caller
 * (an autograd forward, for instance) can keep it for the backward pass without a
 * second forward apply.  Arguments, results and errors otherwise as ifgf_apply;
 * IFGF_EINVAL for a missing, small or misaligned workspace.  The paper has no
 * counterpart (no derivatives). */
ifgf_status ifgf_apply_ws(ifgf_plan *plan, const void *sigma_dev, void *y_dev, int nrhs, ifgf_precision prec,
                          void *ws_dev, int64_t ws_bytes, void *stream);

/* ifgf_apply_vjp on the forward state that ifgf_apply_ws left in ws_dev (same
 * plan, nrhs and precision, and the sigma whose gradient is wanted): gsigma =
 * A^H g and, if dk_host is not NULL, *dk_host = Re <g, dA/dk sigma>, without
 * re-running the forward apply.  ws_dev is read only.  Synchronises `stream`
 * when dk is requested.  Errors as ifgf_apply_vjp, IFGF_EINVAL for a missing,
 * small or misaligned workspace. */
ifgf_status ifgf_apply_vjp_ws(ifgf_plan *plan, const void *ws_dev, int64_t ws_bytes, const void *g_dev,
                              void *gsigma_dev, int nrhs, double *dk_host, ifgf_precision prec, void *stream);

/* ifgf_apply without any device allocation.  The paper has no counterpart: this
 * entry point exists for callers that cannot call cudaMalloc at apply time -- for
 * example code whose device memory is reserved up front by a host application or
 * pool that must not be bypassed, or code on a path where the implicit device
 * synchronisation of cudaMalloc/cudaFree would stall other work.  The plan must
 * already exist (ifgf_plan_create allocates); this call allocates and frees nothing.
 *
 * The apply's workspace (w*sigma and the field in Morton order, and the cone
 * values of every level) lives in one fixed 64 MiB device array inside the
 * library.  Every GPU that loads the library holds that array until the process
 * exits.  Requests whose workspace exceeds it are rejected with IFGF_EINVAL and a
 * message giving the required size; the workspace grows with N, nrhs, the
 * precision (complex128 needs twice complex64) and the number of relevant cone
 * segments.  The first call on a device looks the array's address up with that
 * device current (once per device and CUDA context: again after cudaDeviceReset);
 * make that first call before any stream capture begins.  All calls share the one array and it keeps the last call's
 * contents (every value an apply reads is written earlier in the same apply, so
 * nothing needs clearing).  Calls that overlap on the GPU -- on different streams,
 * or with ifgf_apply_noalloc of another plan -- race on the array and must be
 * serialised by the caller.  Arguments, results and errors are otherwise those of
 * ifgf_apply. */
ifgf_status ifgf_apply_noalloc(ifgf_plan *plan, const void *sigma_dev, void *y_dev, int nrhs, ifgf_precision prec,
                               void *stream);

/* Restarted GMRES(restart) for A x = b with the plan's operator (Section 5: GMRES
 * of Saad & Schultz applied to Eq. CombLayIE).  Arnoldi in FP64 with classical
 * Gram-Schmidt applied twice on the device; the operator apply inside runs in
 * `apply_prec` (IFGF_MIXED rounds each Krylov vector to complex64 for the apply).
 *   rhs_dev: device, N complex128.  x_dev: device, N complex128; initial guess on
 *            entry, solution on exit (must not alias rhs_dev).
 *   restart >= 1, maxit >= 0 (operator applies inside the Arnoldi loops), tol >= 0
 *   on the relative residual |b - A x| / |b|.
 *   iters: receives the iterations done; resid_hist: host array of maxit + 1
 *   doubles receiving the relative residual before each iteration (entry 0 = the
 *   initial guess's true residual; later entries are the Arnoldi estimates).
 * Allocates its Krylov basis ((restart + 1) x N complex128) for the duration of the
 * call and synchronises `stream` every iteration.
 * Returns IFGF_OK when converged, IFGF_ENOTCONVERGED when maxit is reached (x holds
 * the last iterate), or IFGF_EINVAL / IFGF_ENOMEM / IFGF_ECUDA. */
ifgf_status ifgf_gmres(ifgf_plan *plan, const void *rhs_dev, void *x_dev, int restart, int maxit, double tol,
                       ifgf_precision apply_prec, int *iters, double *resid_hist, void *stream);

/* ---- rectangular-polar singular / near-singular correction (Section 4.2) ------
 * Builds, on the host, the sparse correction C that ifgf_plan_set_correction takes:
 * for every target x_l and every patch within the proximity distance `delta` of it
 * (Eq. SingGridPts), the patch integral of K(x_l, y) phi(y) by the rectangular-polar
 * method (Eq. IntOpAtSing with Eq. BetaCov: Fejer's first rule with N_beta points per
 * direction after the change of variables of Eq. CoV with Kress exponent d_grade,
 * centred at the closest patch point of Eq. MinNode), minus the regular Fejer row
 * (Eq. ReguIntOpQuadrature, m != l) that the accelerated operator already sums.
 * The surface is Q = N / m^2 patches of m x m Chebyshev-Gauss nodes (Eq. FejersNodes):
 *   xyz, normals, weights: host, the points as given to ifgf_plan_create (N x 3, N x 3, N).
 *   patch_node: host, N int32: point l is node (i, j) of patch q where
 *               patch_node[l] = q * m * m + i * m + j, (u_i, v_j) = (cos(pi (2i+1)/(2m)),
 *               cos(pi (2j+1)/(2m))); a permutation of 0..N-1.
 *   k, eta: the operator's wavenumber and coupling; delta >= 0: proximity distance;
 *   n_beta in 2..512 (e.g. 48); d_grade >= 2 (e.g. 5).
 * Each patch's map y(u, v) is the tensor Chebyshev interpolant of its node positions,
 * oriented like the given normals.  Outputs: *rowptr_out (N + 1 int64), *col_out
 * (nnz int32, caller point indices) and *val_out (nnz complex128, interleaved re, im),
 * allocated by the library and released with ifgf_free.  Synchronous, host only (no
 * GPU is touched; OpenMP threads).  Errors: IFGF_EINVAL (null pointers, N not a
 * multiple of m^2, m outside 2..64, patch_node not a permutation, non-finite input,
 * invalid k, eta, delta, n_beta or d_grade), IFGF_ENOMEM; outputs are NULL on error. */
ifgf_status ifgf_rp_correction(const double *xyz, const double *normals, const double *weights, int64_t N,
                               const int32_t *patch_node, int32_t m, double k, double eta, double delta,
                               int32_t n_beta, double d_grade, int64_t **rowptr_out, int32_t **col_out,
                               double **val_out);

/* ifgf_rp_correction with the quadrature on the current GPU: the host builds the
 * patch maps, finds the patches within `delta` of every target and their closest
 * points (as ifgf_rp_correction does), and one CUDA block per (target, patch)
 * pair evaluates the graded Fejer quadrature, the kernel and the two nodal
 * contractions in FP64 and subtracts the regular row.  Same arguments, outputs
 * (host arrays released with ifgf_free), sparsity and entry order as
 * ifgf_rp_correction; the values agree to FP64 rounding.  Requires m <= 16 and
 * n_beta <= 64 (IFGF_EUNSUPPORTED otherwise).  Allocates device memory for the
 * duration of the call; synchronous on `stream`.  Errors as ifgf_rp_correction,
 * plus IFGF_ECUDA. */
ifgf_status ifgf_rp_correction_gpu(const double *xyz, const double *normals, const double *weights, int64_t N,
                                   const int32_t *patch_node, int32_t m, double k, double eta, double delta,
                                   int32_t n_beta, double d_grade, void *stream, int64_t **rowptr_out,
                                   int32_t **col_out, double **val_out);

/* Releases an array returned by ifgf_rp_correction (NULL is a no-op). */
void ifgf_free(void *ptr);

/* ---- evaluation off the surface (Section 5: fields from a solved density) ----
 * Direct sums over every quadrature point of the plan (all N sources, in
 * O(N * M) work), one GPU thread per target; the interpolation orders of the plan
 * play no part.  sigma_dev is the density in the caller's point order, as for
 * ifgf_apply (device, N x nrhs column-major: complex128 for IFGF_FP64, complex64
 * for IFGF_MIXED); out_dev receives M x nrhs values column-major (out[q*M + j]),
 * same complex type.  Targets are device FP64 arrays of M x 3 (x0,y0,z0,x1,...)
 * and are used as given (non-finite values give non-finite results).
 * Asynchronous on `stream`.  The first call for a given (M, nrhs, precision)
 * size may grow a plan-owned device scratch buffer (w*sigma in Morton order and,
 * when the targets alone do not fill the GPU, per-chunk partial sums that a
 * second kernel adds in a fixed order, so results are deterministic).
 * Errors: IFGF_EINVAL (null plan, nrhs < 0, M < 0 or M >= 2^31 - 128, null or
 * aliasing pointers with M, nrhs > 0, unknown precision), IFGF_ENOMEM, IFGF_ECUDA.
 * M = 0 or nrhs = 0 returns IFGF_OK without work. */

/* Combined-layer potential of Eq. CombinedLayer at targets x_j off the surface
 * (for example the planar grids of Eq. PlanarGrid):
 *   u(x) = sum_m [dPhi(x, y_m)/dnu(y_m) - i eta Phi(x, y_m)] w_m sigma_m
 * with Phi of Eq. GreenFunction and dPhi/dnu of Eq. double_layer, eta = the plan's
 * coupling.  Targets are meant to lie off the surface: in FP64 a pair closer than
 * 1e-14 times the root-box side contributes 0 (the rule of the on-surface sum),
 * while the mixed form resolves distances only to about 1e-7 of a leaf box, so a
 * target placed exactly on a source point gives no meaningful value there.  With
 * the solved density this is the scattered field u^s; its accuracy near the
 * surface (closer than about one quadrature patch) is that of the plain surface
 * quadrature, no singular correction is applied. */
ifgf_status ifgf_field(ifgf_plan *plan, const void *sigma_dev, const double *x_dev, int64_t M, void *out_dev,
                       int nrhs, ifgf_precision prec, void *stream);

/* Far-field pattern of Eq. FarField at directions xhat_j (unit vectors, e.g. the
 * spherical grid of Eq. SphereGrid):
 *   u_inf(xhat) = (1/4pi) sum_m [-i k <xhat, nu_m> - i eta] e^{-i k <xhat, y_m>} w_m sigma_m,
 * the limit of u(R xhat) R e^{-ikR} as R grows.  Arguments as ifgf_field. */
ifgf_status ifgf_far_field(ifgf_plan *plan, const void *sigma_dev, const double *xhat_dev, int64_t M,
                           void *out_dev, int nrhs, ifgf_precision prec, void *stream);

/* Plan over N surface points (as ifgf_plan_create) plus M off-surface targets (targets [M][3]
 * host FP64, finite; anywhere, inside or outside the surface's bounding box).  The targets join
 * the octree as points with weight 0 and no normal, so they act on nothing, and their rows of the
 * apply are the potential of Eq. CombinedLayer at the targets (ifgf_field_ifgf): the same
 * leaf expansions, propagation, cousin interpolation and near field as every other row, accelerated
 * instead of the N M direct sum of ifgf_field.  The plan's own applies (ifgf_apply and the rest)
 * act on all N + M points; sizes: 1 <= M, N + M <= 2^31 - 1.  IFGF_EINVAL on invalid input. */
ifgf_status ifgf_plan_create_with_targets(const double *xyz, const double *normals, const double *weights,
                                          int64_t N, const double *targets, int64_t M, const ifgf_params *params,
                                          void *stream, ifgf_plan **out);

/* Potential at the M targets of a plan made by ifgf_plan_create_with_targets (the off-surface
 * counterpart of Eq. field1, with the plan's layer): out[q][t] = sum_m K(x_t, y_m) w_m sigma[q][m].
 * sigma_dev [nrhs][N] (the surface densities), out_dev [nrhs][M]; complex128 for IFGF_FP64,
 * complex64 for IFGF_MIXED.  Pads the density with zeros at the targets (a plan-owned scratch of
 * 2 (N + M) nrhs complex values), runs the apply and copies the targets' rows.  No sparse correction
 * is added (it belongs to on-surface rows).  IFGF_EINVAL for a plan without targets. */
ifgf_status ifgf_field_ifgf(ifgf_plan *plan, const void *sigma_dev, void *out_dev, int nrhs, ifgf_precision prec,
                            void *stream);

/* Far-field pattern of Eq. FarField through the IFGF factorisation (Section 3.4 with the
 * limit s -> 0 of Eq. defparametrizationins).  For x = R xhat the centred factor of a level-3
 * box B satisfies R e^{-ikR} e^{ik|x - y_B|} / (4 pi |x - y_B|) -> e^{-ik xhat.y_B} / (4 pi),
 * while s = h_3 / |x - y_B| -> 0 and the direction of x - y_B tends to xhat, so
 *   u_inf(xhat) = sum over level-3 boxes B of e^{-ik xhat.y_B} / (4 pi) F_B(s = 0, xhat),
 * where F_B is B's interpolated analytic factor (the combined factor, or the W13 member of the
 * split pair on a split level; the W2 member decays one order faster and drops out).  Runs the
 * leaf expansions and the propagation of an apply (not the cousin interpolation, the near
 * field or the sparse correction), then one warp per direction sums the level-3 interpolants
 * at local coordinate s = -1 of segment is = 0.  Cost: the upward pass plus M x (level-3 boxes)
 * x Ps Pang^2 per right-hand side, against N M for ifgf_far_field.
 *   plan:     created with params.far_field = 1 (IFGF_EINVAL otherwise)
 *   sigma_dev, xhat_dev, M, out_dev, nrhs, prec, stream: as ifgf_far_field (xhat unit vectors,
 *             [M][3] FP64; out [nrhs][M] complex128 for IFGF_FP64, complex64 for IFGF_MIXED).
 * Uses (and may grow) the plan's own workspace, like ifgf_apply. */
ifgf_status ifgf_far_field_ifgf(ifgf_plan *plan, const void *sigma_dev, const double *xhat_dev, int64_t M,
                                void *out_dev, int nrhs, ifgf_precision prec, void *stream);

/* ---- batched applies over many plans (one CUDA graph) ----------------------
 * A group applies several plans (e.g. many scatterers of uneven size, each with
 * its own right-hand sides) as one captured CUDA graph.  The first
 * ifgf_group_apply captures the launch sequences of all plans (largest first,
 * round-robin over `nstreams` forked capture streams so that independent plans
 * overlap), instantiates the graph and launches it on `stream`; later calls with
 * the same buffers, nrhs and precision replay it with one cudaGraphLaunch.  A
 * change of buffers, nrhs, precision, stream count, of a plan's workspace or
 * correction, or of a plan's kernel choice (ifgf_plan_set_rhs_block,
 * ifgf_plan_set_tc_fill, ifgf_plan_set_tc_engine) triggers a new capture.  The group references the plans (they must
 * outlive it) and each plan may appear once.  The paper has no batched apply. */
typedef struct ifgf_group ifgf_group;

/* Create a group over nplans >= 1 distinct plans.  Errors: IFGF_EINVAL. */
ifgf_status ifgf_group_create(ifgf_plan *const *plans, int nplans, ifgf_group **out);

/* Number of concurrent capture streams (1..64, default 4). */
ifgf_status ifgf_group_set_streams(ifgf_group *group, int nstreams);

/* y[i] = A_i sigma[i] for every plan i (device buffers as in ifgf_apply, nrhs[i] >= 0
 * right-hand sides each, one precision for all).  Asynchronous on `stream`.  Errors
 * as ifgf_apply; capture failures return IFGF_ECUDA. */
ifgf_status ifgf_group_apply(ifgf_group *group, const void *const *sigma, void *const *y, const int *nrhs,
                             ifgf_precision prec, void *stream);

/* Number of graphs the group has captured so far (each recapture adds one);
 * a replay adds nothing.  Errors: IFGF_EINVAL (null group or output). */
ifgf_status ifgf_group_captures(const ifgf_group *group, int64_t *captures);

/* Release the group and its graph (not the plans). NULL is a no-op. */
void ifgf_group_destroy(ifgf_group *group);

/* Tunable: right-hand sides per register block in the mixed interpolation kernels
 * (4 = share geometry and basis weights across 4 right-hand sides, 1 = recompute
 * them per right-hand side with fewer registers).  Errors: IFGF_EINVAL. */
ifgf_status ifgf_plan_set_rhs_block(ifgf_plan *plan, int rhs_block);

/* Tunable: the mixed propagation from a level uses the tensor-core contraction
 * (orders with Pang = 8) when the fraction of filled pair slots in its tiles is at
 * least min_fill (default 0.4; 0 = always, > 1 = never), else the CUDA-core kernel.
 * Errors: IFGF_EINVAL. */
ifgf_status ifgf_plan_set_tc_fill(ifgf_plan *plan, double min_fill);

/* Tunable: engine of the tensor-core propagation.  1 (default) = 5th-generation
 * tensor cores: the two angular contractions of the tensor-product Chebyshev
 * interpolant (Eq. ChebyPoly; K = 64) run as tcgen05.mma with TF32 hi/lo operands
 * (A in tensor memory, B in shared memory) and FP32 accumulators in tensor
 * memory, the radial one in registers; 0 = warp-level mma.sync over the full
 * K = P contraction.  Both keep FP32-level accuracy (three-term TF32 split).
 * Errors: IFGF_EINVAL for any other value. */
ifgf_status ifgf_plan_set_tc_engine(ifgf_plan *plan, int engine);

/* Tunable: engine of the mixed CUDA-core interpolation kernels (Section 3.4: each
 * box's cone interpolants evaluated at the points of its cousin boxes, and at the
 * parent's cone-segment nodes).  1 (default) = cone-stationary: for the cousin
 * interpolation, plan-time lists give, for every relevant cone segment, the
 * cousin points inside it, with their local coordinates and centred factor
 * computed once in FP64; a warp stages one cone's values once and interpolates 64
 * of its points (two per lane), writing each value to its (box, cousin, point)
 * slot, and a second pass adds each point's slots in fixed order.  For the
 * propagation of levels that do not run on the tensor cores (orders with Pang =
 * 8), a warp takes up to 64 parent nodes that fall in one child cone and walks
 * the (parent cone, child box) pairs that share that geometry, staging each
 * pair's child cone once.  0 = point-stationary: a warp owns up to 32 points
 * (parent nodes) of one box and walks its cousin boxes (children), staging the
 * cones its lanes fall in.  Plans with N >= 2^24 points always use 0 for the
 * cousin interpolation.  Errors: IFGF_EINVAL for any other value. */
ifgf_status ifgf_plan_set_interp_engine(ifgf_plan *plan, int engine);

/* Plan statistics (host struct filled synchronously). */
ifgf_status ifgf_plan_info(const ifgf_plan *plan, ifgf_info *out);

/* Number of failed relevant-cone lookups recorded by applies since the last call
 * (should be 0; a non-zero count means a point fell outside the relevant set and
 * its contribution was skipped).  A tensor-core propagation block whose bounded
 * wait for its MMAs timed out adds 2^32 (its results are invalid).  Synchronises
 * `stream` and resets the counter. */
ifgf_status ifgf_plan_check(ifgf_plan *plan, void *stream, int64_t *missed_lookups);

/* Enable (1) or disable (0) per-launch timing: each later apply records a CUDA
 * event on its stream after every kernel launch.  Errors: IFGF_EINVAL, IFGF_ECUDA. */
ifgf_status ifgf_plan_set_profiling(ifgf_plan *plan, int enable);

/* Per-launch device times of the last apply with profiling on: fills up to `cap`
 * entries of kind (0 gather, 1 leaf evaluation, 2 propagation, 3 near field,
 * 4 cousin interpolation, 5 scatter, 6 correction, 7 propagation on the tensor
 * cores: one entry per level, all its octant launches, 8 second pass of the
 * cone-stationary cousin interpolation, 9 cone-stationary propagation on CUDA
 * cores: one entry per level), level (octree level or 0) and
 * ms (milliseconds); any output pointer may be NULL.  Waits for the last event.
 * Returns the number of entries (0 if profiling is off), or a negative ifgf_status. */
int ifgf_plan_stage_times(ifgf_plan *plan, int cap, int *kind, int *level, double *ms);

/* Release the plan and its device memory (NULL is a no-op). */
void ifgf_plan_destroy(ifgf_plan *plan);

/* Message of the last error on the calling thread ("" if none). */
const char *ifgf_last_error(void);

#ifdef __cplusplus
}
#endif
#endif /* IFGF_H */

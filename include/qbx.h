/*
 * qbx.h -- C ABI of the GB300 (sm_103a) implementation of FMM-accelerated
 * Global QBX for 2D Helmholtz layer potentials (Rachh, Kloeckner, O'Neil,
 * "Fast algorithms for Quadrature by Expansion I: Globally valid expansions").
 *
 * The problem (Sec. 1, Eq. (dlp), Eq. (helmholtz-ker); Sec. 2.2; Sec. 7):
 * given closed curves cut into Gauss-Legendre panels, a wavenumber k, complex
 * densities and targets anywhere in the plane, return
 *     u(t) = cS * S[sigma_S](t) + cD * D[sigma_D](t),
 *     S[s](t) = int (i/4) H_0(k|t-y|) s(y) ds(y),
 *     D[s](t) = int n_y . grad_y (i/4) H_0(k|t-y|) s(y) ds(y),   n outward,
 * at every target: by QBX (Sec. 2.1, Eq. (jexp)-(phiapprox)) with the globally
 * valid expansion of its associated centre (Sec. 6.1) where the target is
 * associated, by smooth Gauss quadrature (Sec. 3.2, Eq. (gauss-layerpot))
 * elsewhere. Targets on the curve receive the one-sided limit of the side they
 * request (Sec. 2, Eq. (oneside)).
 *
 * Conventions
 *  - Complex numbers are interleaved (re, im) doubles.
 *  - Points and normals are [n][2] doubles (x, y).
 *  - Every pointer argument may be host or device memory; the library asks
 *    the CUDA runtime which it is. Device pointers must live on the current
 *    device. Host outputs are written before the call returns.
 *  - The caller owns every buffer it passes; the library copies what it keeps
 *    and never frees caller memory. The handle owns all memory it allocates.
 *  - No C++ exception crosses this boundary. Every call returns a status; on a
 *    non-OK status qbx_last_error() holds a message (thread-local).
 *  - One handle must not be used from two threads at once; distinct handles
 *    are independent.
 */
#ifndef QBX_GB300_H
#define QBX_GB300_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct qbx_handle qbx_handle;

typedef enum {
  QBX_OK = 0,
  QBX_ERR_ARG = 1,          /* invalid argument (NULL, size, order out of range)      */
  QBX_ERR_OOM = 2,          /* device or pinned host allocation failed                */
  QBX_ERR_CUDA = 3,         /* a CUDA runtime call or kernel launch failed            */
  QBX_ERR_CONDITION = 4,    /* Condition 4 (k * max h <= 5, Sec. 3.2) is violated     */
  QBX_ERR_ASSOCIATION = 5,  /* a target in Gamma_near found no centre (Sec. 6.1)      */
  QBX_ERR_TIMEOUT = 6,      /* a bounded device-side wait gave up                     */
  QBX_ERR_STATE = 7         /* call out of order (e.g. eval before tree build)        */
} qbx_status;

enum { QBX_FP64 = 0, QBX_MIXED = 1 };          /* arithmetic of the evaluation   */
enum { QBX_DIRECT = 0, QBX_FMM = 1 };          /* how the sums are computed      */

/* Maximum QBX order p accepted (expansions l = -p..p). */
#define QBX_MAX_P 16

/*
 * Geometry (Sec. 2.2). The density grid carries the expansion centres
 *     c = s + side * (h_k / 2) * n    (side +1: exterior, -1: interior),
 * one per density node and requested side. Centre numbering: the exterior
 * centre of node j is j; with center_sides == 2 the interior centre of node j
 * is n_nodes + j. The source grid carries the quadrature (Sec. 3.2 and
 * Sec. 7, Eq. (QBXFMMpot)). Three ways to give it:
 *  - q_src == 0: the density grid is the source grid and `weight` gives its
 *    weights; densities passed to eval live on it.
 *  - q_src > 0 with src_xy, src_normal_xy, src_weight: the caller's source grid
 *    (q_src nodes per panel, same panels); densities passed to eval live on it.
 *  - q_src > 0 (<= 256) with src_xy, src_normal_xy, src_weight all NULL: the
 *    library makes the source grid (Sec. 2.2): on each panel the density
 *    nodes are read as Gauss-Legendre nodes of the panel's reference variable
 *    u in [-1, 1], positions are interpolated by the degree q-1 polynomial
 *    through them at q_src Gauss-Legendre nodes, normals are the rotated unit
 *    tangents of that polynomial (sign of the interpolated caller normals) and
 *    weights w_j^src |dx/du|. Densities passed to eval then live on the
 *    DENSITY grid ([n_nodes]) and are interpolated to the source nodes the same
 *    way before every evaluation. `weight` is not needed. qbx_table1_q_src
 *    gives the paper's choice of q_src; qbx_get_source_grid exports the grid.
 *
 * All curves of one geometry share the wavenumber k (they form one problem).
 */
typedef struct {
  int64_t n_panels;
  int32_t q;                     /* density nodes per panel (n_nodes = n_panels * q)      */
  const double *node_xy;         /* [n_nodes][2]                                          */
  const double *normal_xy;       /* [n_nodes][2] outward unit normals                      */
  const double *weight;          /* [n_nodes] arclength weights (used if src_xy == NULL)   */
  const double *panel_h;         /* [n_panels] panel arclengths h_k                        */
  int32_t q_src;                 /* source nodes per panel (0 => the density grid)         */
  const double *src_xy;          /* [n_panels * q_src][2] or NULL                          */
  const double *src_normal_xy;   /* [n_panels * q_src][2] or NULL                          */
  const double *src_weight;      /* [n_panels * q_src] or NULL                             */
  double k;                      /* wavenumber, real, > 0                                  */
  int32_t p_qbx;                 /* QBX order p, 0 <= p <= QBX_MAX_P                        */
  int32_t center_sides;          /* 1: exterior centres only, 2: both sides                */
  int32_t n_curves;              /* closed curves; 0 or 1: all panels form one curve       */
  const int64_t *curve_panel_offset; /* [n_curves + 1] first panel of each curve, or NULL   */
  int32_t defer_conditions;      /* 1: accept a geometry breaking Condition 4 (to refine)   */
} qbx_geometry_desc;

/*
 * Copies the geometry to the device and places the centres. The panels of a
 * curve are consecutive and run counter-clockwise around it (outward normals);
 * curve_panel_offset says where each curve starts, which decides which panels
 * are adjacent (Sec. 3.2, Conditions 2 and 3). With defer_conditions == 1 a
 * geometry that breaks Condition 4 is accepted, for qbx_refine to mend;
 * qbx_tree_build then refuses it while the condition is still broken.
 * Errors: QBX_ERR_ARG on NULL/invalid sizes, QBX_ERR_CONDITION if
 * k * max_k h_k > 5 (Condition 4) and defer_conditions == 0,
 * QBX_ERR_OOM / QBX_ERR_CUDA. On success *out owns the new handle (free with
 * qbx_destroy).
 */
qbx_status qbx_geometry_create(const qbx_geometry_desc *desc, qbx_handle **out);

/*
 * Targets and evaluation plan (Sec. 6.1 association, Sec. 7 tree and lists).
 * on_surface_node[t] = j >= 0 marks target t as lying on density node j; it
 * then uses the centre of node j on side on_surface_side[t]: +1 the exterior
 * one-sided limit, -1 the interior one, 0 the on-surface value, the mean of
 * the two limits (Sec. 2, Eq. (oneside): S* and the principal value D*,
 * computed from the node's two centres). The interior side and the mean need
 * center_sides == 2; assoc_out reports the exterior centre for a mean. Other targets take
 * the nearest centre c with |t - c| <= (1 + eps_assoc) h/2 (ties: smaller
 * centre index); a target with no such centre whose distance to some density
 * node of panel k is <= h_k/4 is an association failure; the rest use direct
 * quadrature.
 * mode: QBX_DIRECT (all pairs) or QBX_FMM (quadtree, Sec. 7).
 * p_fmm, p_add: box expansion orders (Sec. 7.1): p_fmm on the finest tree
 * level, larger orders on coarser levels whose boxes span wavelengths (see
 * qbx_fmm_level_orders), each plus p_add; p_add < 0 selects
 * qbx_default_p_add(p).
 * n_max: particles per leaf (sources + centres + targets), 0 => 64.
 * assoc_out (optional, [n_targets] int32) receives the centre of every target
 * (-1: direct quadrature).
 * m2l_engine: the M2L translations of FMM mode (Sec. 7.2, Stage 4): 0 the
 * default (FP64 on tensor cores for levels whose bf16 split is exact, mixed
 * precision on the FP32 CUDA-core GEMM), 1 tensor cores in both precisions,
 * 2 CUDA cores in both; every engine meets the precision's tolerance.
 * Errors: QBX_ERR_ASSOCIATION (count and first target in qbx_last_error()),
 * QBX_ERR_ARG, QBX_ERR_OOM, QBX_ERR_CUDA. Synchronous.
 */
typedef struct {
  int64_t n_targets;
  const double *target_xy;         /* [n_targets][2]                                     */
  const int64_t *on_surface_node;  /* [n_targets] or NULL (no on-surface targets)        */
  const int8_t *on_surface_side;   /* [n_targets] or NULL (all +1)                       */
  int32_t mode;                    /* QBX_DIRECT | QBX_FMM                               */
  int32_t p_fmm;
  int32_t p_add;
  int32_t n_max;
  double eps_assoc;                /* <= 0 => 0.1                                        */
  int32_t *assoc_out;              /* optional                                           */
  int32_t m2l_engine;              /* 0 default, 1 tensor cores, 2 CUDA cores            */
} qbx_tree_desc;

qbx_status qbx_tree_build(qbx_handle *h, const qbx_tree_desc *desc);

/*
 * Evaluates u = cS S[sigma_S] + cD D[sigma_D] at every target (Sec. 7,
 * Stages 2-8 in FMM mode, then QBX evaluation at associated targets, Sec. 2.4
 * step 3). sigma_S / sigma_D: complex [n_src] on the source grid; either may be
 * NULL (that layer is absent). out: complex [n_targets]. alpha_out (optional):
 * complex [n_centres][2p+1], l = -p..p, the QBX coefficients of every centre.
 * Without alpha_out, FMM mode forms the coefficients only at the centres that
 * some target is associated with (the only ones the evaluation reads); with
 * it, at every centre. The potential at the targets is the same either way.
 * precision: QBX_FP64 or QBX_MIXED. cuda_stream: a cudaStream_t (NULL: the
 * legacy default stream). With device buffers the call is asynchronous on the
 * stream; with any host buffer it copies through the stream and returns after
 * the result is in host memory.
 */
qbx_status qbx_layer_potential_eval(qbx_handle *h, double cS_re, double cS_im,
                                    const double *sigma_S, double cD_re, double cD_im,
                                    const double *sigma_D, double *out, double *alpha_out,
                                    int32_t precision, void *cuda_stream);

/* Frees every resource of the handle. NULL-safe. Synchronises the device work
 * of the handle first. */
void qbx_destroy(qbx_handle *h);

/* Message of the last non-OK status on this thread ("" if none). */
const char *qbx_last_error(void);

/*
 * Plan statistics after qbx_tree_build (for logging and benchmarks):
 * stats[0] n_sources, [1] n_centres, [2] n_targets, [3] n_qbx_targets,
 * [4] n_boxes, [5] n_leaves, [6] tree depth, [7] box order on the finest
 * level (p_fmm + p_add), [8] U-list pairs
 * (leaf, leaf), [9] V-list pairs, [10] W-list pairs, [11] X-list pairs,
 * [12] source-centre pairs evaluated directly (P2QBXL), [13] source-target
 * pairs evaluated directly (P2P), [14] (box, centre) pairs of M2QBXL,
 * [15] (box, target) pairs of M2P, [16] kernel launches of the last eval,
 * [17] sources in X-list boxes summed over boxes (P2L pairs), [18] M2M plus
 * L2L translations, [19] largest box order over the levels. Unused entries
 * are 0. n_stats >= 20.
 */
qbx_status qbx_get_stats(const qbx_handle *h, int64_t *stats, int32_t n_stats);

/*
 * Device time of each kernel class of the last eval, in milliseconds, when
 * timing was enabled with qbx_set_timing(h, 1) before that eval (events are
 * recorded on the eval stream; reading them synchronises it).
 * times[i] for i < n_times follows enum qbx_stage; returns the number filled.
 */
enum qbx_stage {
  QBX_STAGE_STRENGTHS = 0, QBX_STAGE_P2M, QBX_STAGE_M2M, QBX_STAGE_P2P, QBX_STAGE_P2QBXL,
  QBX_STAGE_M2L, QBX_STAGE_M2P, QBX_STAGE_M2QBXL, QBX_STAGE_P2L, QBX_STAGE_L2L,
  QBX_STAGE_L2P, QBX_STAGE_L2QBXL, QBX_STAGE_QBXL2P, QBX_STAGE_COUNT
};
qbx_status qbx_set_timing(qbx_handle *h, int32_t enable);
int32_t qbx_get_stage_times(qbx_handle *h, double *times_ms, int32_t n_times);

/*
 * Tree inspection after qbx_tree_build in QBX_FMM mode (the quadtree of Sec. 4
 * and Sec. 7.2, Stage 1, and its U, V, W, X lists). All outputs are HOST
 * memory; any pointer may be NULL (skipped).
 *   info[8]: [0] n_boxes, [1] n_levels, [2..5] entries of the U, V, W, X
 *            lists, [6] box order on the finest level, [7] n_leaves.
 *   root[3]: x0, y0, side of the root square [x0, x0+side] x [y0, y0+side].
 *   box_level [n_boxes]; box_ij [n_boxes][2] integer position at the box's
 *   level; box_child [n_boxes][4] (-1: none; quadrant q = ix&1 + 2(iy&1));
 *   box_range [n_boxes][4][2]: [start, end) of the box's sources, centres,
 *   targets and density nodes in the sorted orders perm_src [n_src],
 *   perm_ctr [n_centres], perm_tgt [n_targets] (original indices).
 *   lists_off [4][n_boxes + 1] and lists_idx [info[2]+...+info[5]]: CSR of
 *   the U, V, W, X lists, concatenated in that order (offsets are local to
 *   each list).
 * Errors: QBX_ERR_STATE if no FMM plan exists.
 */
qbx_status qbx_export_tree(const qbx_handle *h, int64_t *info, double *root, int32_t *box_level,
                           int32_t *box_ij, int32_t *box_child, int32_t *box_range,
                           int32_t *lists_off, int32_t *lists_idx, int32_t *perm_src,
                           int32_t *perm_ctr, int32_t *perm_tgt);

/*
 * The box order of every level of the handle's FMM plan (as computed by
 * qbx_fmm_level_orders for its tree): pb_out int32 [n], entries past the
 * tree's depth set to 0. Errors: QBX_ERR_STATE if no FMM plan exists.
 */
qbx_status qbx_get_box_orders(const qbx_handle *h, int32_t *pb_out, int32_t n);

/*
 * Box expansion orders of a quadtree level by level (Sec. 7.1, "Maintaining
 * Expansion Accuracy"). Level l has boxes of side root_side / 2^l and
 * half-side R_l; its outgoing order is the smallest p with
 *   max_{n > p} |H_n(3 k R_l)| max_{y <= sqrt2 k R_l} |J_n(y)| <= eps,
 * the bound the paper states for sources within sqrt2 R of a box centre and
 * targets beyond 3R. eps is the value of that bound for n > p_fmm at
 * k R = min(k R_finest, 1) (R_finest: half-side on level n_levels - 1), so
 * the finest level gets p_fmm itself unless its boxes exceed k R = 1.
 * pb_out[l] (int32 [n_levels]) receives that order plus p_add for levels
 * l >= 2 and 0 for levels 0 and 1 (no well-separated boxes there).
 * Host computation only. Errors: QBX_ERR_ARG for k <= 0, root_side <= 0,
 * n_levels outside 1..25, p_fmm < 1, p_add < 0, or a level needing an order
 * above 1200 (boxes spanning too many wavelengths).
 */
qbx_status qbx_fmm_level_orders(double k, double root_side, int32_t n_levels, int32_t p_fmm,
                                int32_t p_add, int32_t *pb_out);

/*
 * The p_add used when a tree descriptor asks for the default (p_add < 0),
 * for QBX order p (Sec. 7.1, "Maintaining Expansion Accuracy", and Table 2).
 * The paper sets the box order to p_FMM^l + p_add and finds p_add by
 * experiment: random curves r = 5 + sum_{j<=12} delta_j sin jt at k = 5,
 * Green's identity at targets near the boundary, the smallest p' for which
 * the FMM-accelerated error stays below eps. This library repeats that
 * experiment with its own orders p_FMM^l (qbx_fmm_level_orders) and returns
 * the measured values (0, 0, 0, 3, 3, 7, 7, 9, 9, 9, 9, 10, 10, 11, 11, 11, 11
 * for p = 0..16; Table 2 prints 5, 5, 15, 20 for p = 2, 4, 6, 8 with the
 * paper's point-FMM orders). Orders above 16 take the value of 16. Host
 * computation only; returns -1 for p < 0.
 */
int32_t qbx_default_p_add(int32_t p);

/*
 * The four sufficient conditions of Sec. 3.3 on the handle's geometry
 * (Sec. 3.1-3.2), checked with the panel attribution of Sec. 5:
 *   QBX_COND1 (Condition 1, Eq. (dcgam_perpanel)): some centre of panel n lies
 *     closer than h_n / 2 to another panel m; panel n is flagged (its disks
 *     are too large; Sec. 5.1).
 *   QBX_COND2 (Condition 2): adjacent panels of a curve whose lengths differ by
 *     more than a factor 2; the longer one is flagged.
 *   QBX_COND3 (Condition 3): a centre of panel n lies closer than h_m / 4 to a
 *     panel m that is neither n nor adjacent to n; the source panel m is
 *     flagged (its quadrature is too coarse there; Sec. 5.2 and its figure).
 *   QBX_COND4 (Condition 4): k h_k > 5; panel k is flagged.
 * Distances to a panel are to the curve through its nodes (the interpolating
 * polynomial of degree q - 1 in the panel's reference variable). Candidate
 * (centre, panel) pairs come from area queries in a hierarchy of panel
 * bounding squares (Sec. 4, with a Morton-ordered bounding-volume tree in
 * place of the paper's peer boxes).
 * panel_flags (optional, [n_panels] int32, host or device) receives the OR of
 * the QBX_COND* bits of each panel; counts (optional, [4] int64, host) the
 * number of panels flagged for each condition. Synchronous.
 * Errors: QBX_ERR_ARG, QBX_ERR_OOM, QBX_ERR_CUDA.
 */
enum { QBX_COND1 = 1, QBX_COND2 = 2, QBX_COND3 = 4, QBX_COND4 = 8 };
qbx_status qbx_check_conditions(qbx_handle *h, int32_t *panel_flags, int64_t *counts);

/*
 * Refinement (Sec. 5): checks the conditions and bisects every flagged panel
 * into two panels of equal arclength (the split point from the panel's
 * Legendre expansion; new nodes, normals and weights from the same expansion),
 * rechecks, and repeats until no panel is flagged or max_rounds rounds have
 * run. The handle's geometry is replaced: centres are placed anew, any plan is
 * dropped (build it again with qbx_tree_build), a library-made source grid is
 * made anew. Handles with a caller-supplied source grid cannot be refined
 * (QBX_ERR_STATE). *rounds (optional) receives the rounds run, *n_panels
 * (optional) the new panel count. Returns QBX_ERR_CONDITION if panels are
 * still flagged after max_rounds. Synchronous.
 */
qbx_status qbx_refine(qbx_handle *h, int32_t max_rounds, int32_t *rounds, int64_t *n_panels);

/*
 * The handle's density geometry, e.g. after qbx_refine: *n_panels (required)
 * receives the panel count; the optional host or device arrays node_xy
 * [n_panels q][2], normal_xy [n_panels q][2], weight [n_panels q], panel_h
 * [n_panels], panel_origin [n_panels] (the panel of the geometry given to
 * qbx_geometry_create that the panel lies on), panel_interval [n_panels][2]
 * (the panel's part of that original panel, in its reference variable
 * u in [-1, 1], so that a caller can sample its density there) and
 * curve_panel_offset [n_curves + 1] are filled. Call first with NULL arrays to
 * learn n_panels. Synchronous.
 */
qbx_status qbx_get_geometry(const qbx_handle *h, int64_t *n_panels, double *node_xy,
                            double *normal_xy, double *weight, double *panel_h,
                            int64_t *panel_origin, double *panel_interval,
                            int64_t *curve_panel_offset);

/*
 * The exterior Dirichlet (sound-soft scattering) problem of Sec. 1 and
 * Sec. 8.3: with u = D[sigma] + i k S[sigma] the boundary condition u = f on
 * the curves is the second-kind equation (Eq. (extdir), Eq. (int_eq))
 *     (1/2) sigma + D*[sigma] + i k S*[sigma] = f,
 * whose left side is the exterior one-sided limit that Global QBX evaluates at
 * each density node. Solves it by restarted GMRES (restart vectors, relative
 * residual tol, at most max_iter matrix-vector products), each product one
 * qbx_layer_potential_eval in the given mode (QBX_DIRECT or QBX_FMM with box
 * order p_fmm plus the default p_add) and precision. The call builds its own
 * plan (targets: every density node, exterior side), replacing any plan of
 * the handle.
 * rhs: f, complex [n_nodes] at the density nodes (host or device);
 * sigma_out: complex [n_nodes] (host or device); *iters_out, *resid_out
 * (optional): the products used and the final true relative residual
 * ||f - A sigma|| / ||f||, which the caller compares with tol (the call
 * returns QBX_OK also when max_iter ends it first). Synchronous on
 * cuda_stream. Handles with a caller-supplied source grid are refused
 * (QBX_ERR_STATE): the unknowns live on the density nodes.
 */
qbx_status qbx_solve_dirichlet(qbx_handle *h, const double *rhs, double *sigma_out, int32_t mode,
                               int32_t p_fmm, int32_t precision, double tol, int32_t max_iter,
                               int32_t restart, int32_t *iters_out, double *resid_out,
                               void *cuda_stream);

/*
 * The source grid of the handle (Sec. 2.2): src_xy [n_src][2], src_normal_xy
 * [n_src][2], src_weight [n_src], n_src = n_panels * q_src (the density grid
 * when q_src was 0). Host or device outputs; any may be NULL (skipped).
 * Synchronous. Errors: QBX_ERR_ARG (NULL handle), QBX_ERR_CUDA.
 */
qbx_status qbx_get_source_grid(const qbx_handle *h, double *src_xy, double *src_normal_xy,
                               double *src_weight);

/*
 * Waits for all device work and reports device-side failures that an
 * asynchronous call could not return: QBX_ERR_TIMEOUT if a bounded wait of a
 * kernel (the mbarrier waits of the tensor-core M2L of Sec. 7.2, Stage 4: a
 * deadline of 1 s each) gave up since the last check; the results of the
 * evaluations since then are invalid, and the flag is cleared. An evaluation
 * with host buffers makes the same check before it returns. Errors:
 * QBX_ERR_ARG (NULL handle), QBX_ERR_CUDA.
 */
qbx_status qbx_sync(qbx_handle *h);

/*
 * Self-test of the failure path above: one warp waits, with the bounded wait
 * of the tensor-core kernels and a deadline of limit_us microseconds, on an
 * mbarrier that nothing completes, and sets the handle's wait flag when the
 * wait runs out. The next qbx_sync (or evaluation with host buffers) then
 * returns QBX_ERR_TIMEOUT, and the handle stays usable. Synchronous. Errors:
 * QBX_ERR_ARG (NULL handle, limit_us outside 1..1e6), QBX_ERR_STATE (no FMM
 * plan), QBX_ERR_CUDA.
 */
qbx_status qbx_selftest_wait_timeout(qbx_handle *h, int32_t limit_us);

/*
 * H_0(x) and H_1(x) of the first kind, as every kernel of the library
 * evaluates them on the device (the Hankel values that start the recurrences
 * of Sec. 7.2's translations and the kernel G = (i/4) H_0(k|x - y|) of Sec. 1):
 * below x = 8 piecewise polynomials (Chebyshev fits on eight intervals per
 * octave from 2^-9; below that the ascending series, DLMF 10.2.2 and 10.8.1,
 * economised), the CUDA math library's j0/y0/j1/y1 above. variant 0: the FP64
 * path (degree 10, relative error below 1e-15 of |H_0|, |H_1|); 1: the
 * mixed-precision path (degree 8, below 1e-13). x: host [n], positive and
 * finite; out: host [n][4] =
 * (Re H_0, Im H_0, Re H_1, Im H_1). Synchronous. Errors: QBX_ERR_ARG (NULL
 * pointer with n > 0, n < 0, x[i] <= 0 or not finite, unknown variant),
 * QBX_ERR_OOM / QBX_ERR_CUDA.
 */
qbx_status qbx_hankel01(const double *x, int64_t n, int32_t variant, double *out);

/*
 * The FP64 -> FP32 rounding of the mixed-precision kernels (Sec. 7.2 Stages
 * 3, 5 in mixed precision: Hankel values from the FP64 recurrences), done
 * with integer instructions: round to nearest (ties away from zero), results
 * below 2^-126 in magnitude flushed to zero, overflow to infinity, NaN kept.
 * x: host [n]; out: host float [n]. Synchronous. Errors: QBX_ERR_ARG (NULL
 * pointer with n > 0, n < 0), QBX_ERR_OOM / QBX_ERR_CUDA.
 */
qbx_status qbx_f32_from_f64(const double *x, int64_t n, float *out);

/*
 * Measured FMA rates of this GPU, the denominators of the arithmetic
 * rooflines of the FP64 and mixed paths: 8 independent FMA chains per thread,
 * 8 blocks of 256 threads per SM, best of three timed launches (CUDA events)
 * after a warm-up; flops = 2 per FMA. Takes about 0.1 s. Synchronous. Errors:
 * QBX_ERR_ARG (NULL output), QBX_ERR_CUDA.
 */
qbx_status qbx_measure_fma_rates(double *fp64_tflops, double *fp32_tflops);

/*
 * Table 1 of the paper (Sec. 3.2): source nodes per panel q_src for q density
 * nodes and precision eps, as printed for q = 2, 4, 8, 16 and eps = 1e-3,
 * 1e-6, 1e-9, 1e-12. Other q take the row of the next tabulated q, other eps
 * the column of the next tabulated eps at least as strict. Returns -1 for
 * q outside 1..16 or eps outside [1e-12, inf). Host computation only.
 */
int32_t qbx_table1_q_src(int32_t q, double eps);

/*
 * Measured plan selection. Builds the plan of `desc` (targets, association)
 * for each candidate -- QBX_DIRECT, and QBX_FMM with n_max in {32, 64, 128}
 * -- times `reps` evaluations of each with CUDA events (random unit
 * densities, the given precision and layers: has_S / has_D 0 or 1) and
 * leaves the fastest plan built in the handle. times_ms (optional, [4])
 * receives the median time of each candidate in that order (0 for a
 * candidate that is skipped: FMM plans are skipped for fewer than 512
 * sources); *chosen receives the index of the winner. Decisions are cached
 * per (sources rounded to a power of two, k * mean panel length rounded to
 * 1/8, p, precision) so that similar problems of a batch are timed once.
 * desc->mode, desc->n_max are ignored. Synchronous.
 */
qbx_status qbx_autotune(qbx_handle *h, const qbx_tree_desc *desc, int32_t precision,
                        int32_t has_S, int32_t has_D, int32_t reps, double *times_ms,
                        int32_t *chosen);

/*
 * Accuracy-aware plan selection, the autotuner of batched evaluation. Builds
 * candidate plans of `desc` (its targets and association), times `reps`
 * evaluations of each (CUDA events, random unit densities, the given
 * precision and layers) and keeps the fastest whose result is within tol
 * (relative l2) of the most accurate plan (QBX_DIRECT below 512 sources, else
 * QBX_FMM at desc->p_fmm; both FP64). The search is greedy:
 *  1. plan kind and leaf size: QBX_DIRECT, QBX_FMM with n_max 16, 32, 64, 128;
 *  2. for an FMM winner, box orders p_fmm lowered by 4 at a time while the
 *     result stays within tol (the per-curve order schedule);
 *  3. the M2L engine: the default (FP64 path on tensor cores where the bf16
 *     split is exact, mixed path on the FP32 CUDA-core GEMM), tensor cores for
 *     both precisions, or CUDA cores for both;
 *  4. the centres per warp of L2QBXL (4, 8, 16, 32).
 * Decisions are cached per (sources rounded to a power of two, k * mean panel
 * length rounded to 1/8, p, precision, sides, layers, tol rounded to a power of
 * ten), so similar curves of a batch are tuned once. The winner's plan is left
 * built in the handle.
 * plan_out (optional, int32 [5]): mode, n_max, p_fmm, M2L engine (0 default,
 * 1 tensor cores for both precisions, 2 CUDA cores), L2QBXL centres per warp
 * (0 automatic);
 * report (optional, double [3]): its median time in ms and its error (0 when
 * the decision came from the cache), and the candidates tried.
 * Errors: QBX_ERR_CONDITION if no candidate meets tol; those of
 * qbx_tree_build and qbx_layer_potential_eval. Synchronous.
 */
qbx_status qbx_autotune_tol(qbx_handle *h, const qbx_tree_desc *desc, int32_t precision,
                            int32_t has_S, int32_t has_D, double tol, int32_t reps,
                            int32_t *plan_out, double *report);

/*
 * Batched evaluation of many independent problems (for example curves with
 * their own wavenumbers and densities), each a handle after qbx_tree_build.
 * The evaluations of all handles are captured once into one CUDA graph whose
 * branches run concurrently (handles are dealt round-robin onto n_streams
 * streams), so that many small problems fill the GPU; later calls replay the
 * graph. Densities and results are concatenated in handle order:
 * sigma_S / sigma_D complex [sum n_src_i] (either may be NULL for all
 * handles), out complex [sum n_targets_i]; cS, cD complex [n] per handle.
 * Pointers may be host or device memory; the batch owns device staging
 * buffers whose addresses the graph uses. A change of precision, layers or
 * coefficients re-captures the graph. Synchronous when any pointer is host
 * memory, else asynchronous on cuda_stream. While a handle belongs to a batch
 * (until qbx_batch_destroy), its evaluations favour throughput over the
 * latency of one problem (one stream per handle, wider tiles and more centres
 * per warp); results are unchanged.
 */
typedef struct qbx_batch qbx_batch;
qbx_status qbx_batch_create(int32_t n, qbx_handle *const *handles, int32_t n_streams,
                            qbx_batch **out);
qbx_status qbx_batch_eval(qbx_batch *b, const double *cS, const double *sigma_S,
                          const double *cD, const double *sigma_D, double *out,
                          int32_t precision, void *cuda_stream);
void qbx_batch_destroy(qbx_batch *b);

/*
 * Allocation-free direct QBX evaluation. The paper has no counterpart: this is
 * an interface addition for callers that must not allocate device memory, for
 * example an application whose HBM is entirely handed out up front by its own
 * pool allocator, or a time-critical loop that cannot afford the device-wide
 * synchronisation that cudaMalloc/cudaFree may cause. It performs no
 * allocation of any kind: the caller passes every input and output, and the
 * intermediate strengths and QBX coefficients live in one fixed array of
 * 2^19 complex doubles (8 MiB) that the library reserves on every GPU where it
 * is loaded, held until the process exits.
 *
 * What it computes: for every centre, the local-expansion coefficients
 * l = -p..p of u = cS S[sigma_S] + cD D[sigma_D] summed directly over ALL
 * sources (no tree, no far-field approximation); then, at every target t, the
 * truncated Bessel (J) expansion about centre tgt_centre[t] evaluated at t.
 * This is the same arithmetic as qbx_layer_potential_eval in QBX_DIRECT mode
 * at associated targets. No association is done here; an out-of-range centre
 * index gives NaN at that target.
 *  - All pointers are DEVICE memory on the current device; host memory and
 *    memory of another GPU are rejected with QBX_ERR_ARG, the message naming
 *    the argument: src_xy [n_src][2], src_normal_xy [n_src][2], src_weight
 *    [n_src], sigma_S / sigma_D complex [n_src] (either may be NULL, not
 *    both), ctr_xy [n_ctr][2], tgt_xy [n_tgt][2], tgt_centre int32 [n_tgt],
 *    out complex [n_tgt].
 *  - Limit: 2 * n_src + n_ctr * (2p + 1) <= 2^19; larger problems return
 *    QBX_ERR_ARG with the required size in qbx_last_error(). 0 <= p <= 16.
 *  - Asynchronous on cuda_stream (NULL: legacy default stream).
 *  - The first call on a device looks up the device address of the scratch
 *    array (cudaGetSymbolAddress) and caches it for the life of the process;
 *    make that first call before any stream capture begins. After
 *    cudaDeviceReset (or anything else that destroys the device's primary
 *    context) the cached address is stale: do not call this function again
 *    in that process.
 *  - Every call on a device shares the one scratch array and leaves its last
 *    contents there; calls whose GPU work overlaps (different streams, no
 *    ordering between them) race on it and must be serialised by the caller.
 */
qbx_status qbx_direct_qbx_eval_noalloc(int64_t n_src, const double *src_xy,
                                       const double *src_normal_xy, const double *src_weight,
                                       double k, double cS_re, double cS_im,
                                       const double *sigma_S, double cD_re, double cD_im,
                                       const double *sigma_D, int64_t n_ctr,
                                       const double *ctr_xy, int32_t p, int64_t n_tgt,
                                       const double *tgt_xy, const int32_t *tgt_centre,
                                       double *out, void *cuda_stream);

#ifdef __cplusplus
}
#endif
#endif /* QBX_GB300_H */

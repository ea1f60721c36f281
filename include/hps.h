/*
 * hps.h -- C ABI of libhps, batched HPS leaf static condensation on B300.
 *
 * Method: Yesypenko & Martinsson, "GPU Optimizations for the Hierarchical
 * Poincare-Steklov Scheme" (arXiv 2211.14969).  The BVP is Eq. (bvp) with the
 * variable-coefficient Helmholtz operator of Eq. (var_helm), written on a
 * reference square in the general second-order form of Eq. (chain_rule):
 *
 *   A u = -(c11 u_xx + 2 c12 u_xy + c22 u_yy + c1 u_x + c2 u_y) - kappa^2 b u = f,
 *
 * discretized per Section 2: each leaf box carries a p x p tensor mesh of
 * Chebyshev points, the PDE is collocated at the (p-2)^2 interior nodes, and
 * the flux (outward normal derivative) is continuous across leaf edges.  The
 * four leaf corners are not unknowns.  Static condensation (Section 2)
 * eliminates the interior nodes of every leaf, leaving the reduced system of
 * Eq. (hps_reduced) on the 4(p-2) edge nodes of each leaf.
 *
 * Conventions shared by every call
 * --------------------------------
 *  - Leaf box (x0, y0, hx, hy); node (i, j), i the x index, has id i*p + j
 *    and coordinates x0 + (1 - cos(i pi/(p-1))) hx/2, y0 + (1 - cos(j pi/(p-1))) hy/2.
 *  - Interior nodes (1 <= i, j <= p-2) in lexicographic order, i major:
 *    n_i = (p-2)^2 of them.  Edge nodes in the order [W, E, S, N], each edge
 *    by increasing coordinate: n_b = 4(p-2).
 *  - Per-leaf arrays are packed leaf after leaf: leaf l starts at the sum of
 *    the sizes of leaves 0..l-1 (for one p everywhere, l times the size).
 *    Every matrix is row-major inside its leaf block.
 *  - All pointers named d_* are device pointers on the current CUDA device,
 *    owned by the caller, and must stay valid until the stream reaches the
 *    work that reads or writes them.  Host pointers are read before the call
 *    returns, except the h_* buffers of hps_condense_host, which are copied
 *    asynchronously and must stay valid until the stream reaches the end of
 *    that call.  Every call is asynchronous on the given stream (NULL =
 *    legacy default stream) and reports argument and launch errors
 *    synchronously.
 *  - No call allocates or frees a caller buffer.  A plan owns its device
 *    workspace (allocated at build time, grown on demand by hps_condense,
 *    hps_condense_host and hps_merge, freed by hps_destroy).
 *  - A plan is not thread-safe; use one plan per host thread or serialise.
 */
#ifndef HPS_H
#define HPS_H

#ifdef __cplusplus
extern "C" {
#endif

typedef struct hps_plan hps_plan;
typedef struct CUstream_st *hps_stream; /* a cudaStream_t */

typedef enum {
    HPS_OK = 0,
    HPS_ERR_ARG = 1,      /* invalid argument; nothing was enqueued */
    HPS_ERR_CUDA = 2,     /* a CUDA runtime call failed (message in hps_last_error) */
    HPS_ERR_OOM = 3,      /* device workspace could not be allocated */
    HPS_ERR_SINGULAR = 4, /* an exact zero pivot: hps_check_info on a leaf's info > 0,
                             hps_merge / hps_merge_boxes on a merge's Z */
    HPS_ERR_NOCONV = 5,   /* hps_check_info: a mixed-precision leaf did not converge */
    HPS_ERR_STATE = 6     /* call out of order (e.g. hps_solve before hps_merge) */
} hps_status;

typedef enum {
    HPS_FP64 = 0,        /* everything in FP64 */
    HPS_MIXED_FP32 = 1,  /* FP32 LU/TRSM, FP64-accurate residual + iterative refinement */
    HPS_MIXED_TF32 = 2,  /* as HPS_MIXED_FP32, the LU's trailing updates on the tensor
                            cores (tcgen05, TF32 inputs split hi + lo, FP32 accumulation) */
    HPS_MIXED_BF16 = 3   /* as HPS_MIXED_TF32 with BF16 inputs split hi + lo */
} hps_prec;

/* info code of a leaf whose tensor-core wait timed out (HPS_MIXED_TF32/BF16) */
#define HPS_INFO_TC_TIMEOUT (-1073741824)

#define HPS_PMIN 4
#define HPS_PMAX 42

typedef struct {
    int n_leaves;        /* >= 1 */
    const int *p;        /* host [n_leaves]: points per direction, HPS_PMIN..HPS_PMAX */
    const double *box;   /* host [n_leaves][4]: x0, y0, hx, hy (hx, hy > 0) */
    double kappa;        /* wavenumber of Eq. (var_helm) */
} hps_leaf_desc;

/* Build a plan for a batch of leaves (Section 2: leaf boxes with p x p
 * Chebyshev meshes).  Validates the description, forms the Chebyshev
 * differentiation matrices of every order present in FP64, sorts the leaves
 * into a longest-first work queue and allocates the per-CTA workspace.
 * Returns HPS_ERR_ARG for a bad description (*out is set to NULL),
 * HPS_ERR_OOM / HPS_ERR_CUDA on device failures. */
hps_status hps_build_leaves(const hps_leaf_desc *desc, hps_plan **out, hps_stream stream);

/* Node coordinates of every leaf, so the caller can sample coefficients:
 * d_xy per leaf [2][p*p] (all x, then all y), packed.  Section 2 mesh. */
hps_status hps_leaf_nodes(const hps_plan *plan, double *d_xy, hps_stream stream);

/* Leaf static condensation (Section 2; steps: assemble the collocation
 * operator, factor the interior block with partial pivoting, solve, form the
 * DtN map).  For every leaf:
 *   S = -A_ii^{-1} A_ib         (n_i x n_b)   solution operator
 *   T = N_b + N_i S             (n_b x n_b)   Dirichlet-to-Neumann map
 *   W = A_ii^{-1} f_I           (n_i x m)     particular interior solution
 *   h = N_i W                   (n_b x m)     its outgoing flux
 * where N = [N_b N_i] are the outward-normal-derivative rows at the edge nodes.
 * Inputs:  d_coef per leaf [6][p*p]: c11, c12, c22, c1, c2, b at the nodes.
 *          d_f per leaf [p*p][m] body loads at the nodes (interior used), or
 *          NULL when m == 0.
 * Outputs: d_S (may be NULL: not stored), d_T (required), d_W and d_h
 *          (required when m > 0), d_info per leaf (required):
 *            0     success,
 *            k > 0 exact zero pivot at elimination step k (the leaf's S, T
 *                  hold inf/NaN),
 *            -k    mixed precision: refinement did not reach tol in k steps.
 * prec: HPS_FP64, or the mixed paths HPS_MIXED_FP32 (FP32 LU on the FP32
 *       pipe), HPS_MIXED_TF32 / HPS_MIXED_BF16 (the factorization's trailing
 *       updates on the tensor cores as hi*hi + hi*lo + lo*hi splits); all
 *       mixed paths refine to the same tolerance and need 4(p-2) + m <= 256
 *       for the largest p.
 * tol, kmax: iterative refinement with FP64 residuals.  Per right-hand column
 *            let eta_k = max|correction_k| / max|X| (eta_0 = 1); the error
 *            left after correction k is estimated as eta_k^2 / eta_{k-1}
 *            (linear convergence; hps_set_refine_stop(plan, 1) estimates it
 *            after the first correction from the true residuals instead).
 *            Refinement stops once every column's estimate is <= tol while
 *            still contracting, or after kmax corrections.  kmax = 0
 *            returns the FP32 solution unrefined.
 *            A leaf that does not converge (typically cond(A_ii) u_fp32
 *            near 1, e.g. close to an interior Dirichlet resonance) is
 *            condensed again in FP64 inside the same launch and gets the
 *            FP64 info code; hps_set_fp64_fallback(plan, 0) turns that off,
 *            and such a leaf then reports info = -kmax with the last
 *            iterate.  Ignored for HPS_FP64.
 * Corners: with c12 != 0 the interior rows touch the leaf corners, which are
 * not unknowns; a corner's value is taken as the mean of the polynomial
 * extrapolations (degree p-3) along its two edges from their p-2 edge
 * nodes, so its column is folded into the edge columns (A_ib + A_ic E).
 * Exact for tensor polynomials of degree <= p-3; with c12 == 0 no row
 * touches a corner. */
hps_status hps_condense(hps_plan *plan, hps_prec prec, const double *d_coef, const double *d_f,
                        int m, double tol, int kmax, double *d_S, double *d_T, double *d_h,
                        double *d_W, int *d_info, hps_stream stream);

/* Impedance-to-impedance (ItI) leaf maps, in place of the DtN maps of
 * hps_condense where a leaf may sit at an interior Dirichlet resonance
 * (kappa^2 an eigenvalue of its Dirichlet problem: A_ii singular, no DtN
 * map).  Not in the paper; the impedance formulation of Gillman, Barnett
 * and Martinsson (BIT 2015), from its definitions: on a box boundary the
 * incoming data is f = u_n + i eta u and the outgoing data g = u_n - i eta u
 * (u_n the outward normal derivative, eta > 0, typically kappa).  Per leaf
 * the collocation system with the impedance condition on every edge node
 * (the PDE rows at the interior nodes as in hps_condense, corner columns
 * folded in the same way) is solved in FP64 (complex, assembled in real
 * form of twice the size): with Y the values for unit incoming data and uf
 * those for the body loads with zero incoming data,
 *   R = I - 2 i eta Y_b   (n_b x n_b),   h = -2 i eta uf_b   (n_b x m),
 * so g = R f + h, and the interior values are u_i = Y_i f + uf_i.
 * Outputs are complex, interleaved (re, im), packed as hps_condense's with
 * twice the element count: d_R like T, d_h like h (required when m > 0),
 * d_Y like S (may be NULL), d_uf like W (may be NULL); d_info as
 * hps_condense (k > 0: exact zero pivot at step k of the real-form LU).
 * d_coef, d_f as hps_condense.  HPS_ERR_ARG for eta <= 0. */
hps_status hps_iti_condense(hps_plan *plan, double eta, const double *d_coef, const double *d_f, int m, double *d_R,
                            double *d_h, double *d_Y, double *d_uf, int *d_info, hps_stream stream);

/* Maximum pipeline depth of hps_condense_host. */
#define HPS_HOST_MAX_CHUNKS 64

/* hps_condense with every input and output in HOST memory: the same leaf
 * condensation (Section 2, static condensation of the leaf interiors) and
 * the same arguments, packing and info codes as hps_condense, with h_*
 * host pointers in place of d_*.  The leaves are split into `chunks`
 * contiguous ranges of about equal work (0: 8; at most
 * HPS_HOST_MAX_CHUNKS and n_leaves); each range's inputs are copied to the
 * device on one copy stream, condensed by one launch (ranges alternate
 * between the given stream and a second compute stream, each with half of
 * a doubled workspace), and its outputs copied back on another copy
 * stream, so transfers overlap the condensation.  The results are the
 * ones hps_condense computes (each leaf is condensed by the same code).
 * Host buffers should be page-locked (cudaHostAlloc / pinned): pageable
 * memory gives correct results but the copies then do not overlap.
 * The call returns once everything is enqueued; it completes on `stream`
 * (synchronize it before reading the host outputs).  The plan keeps device
 * copies of all inputs and outputs (allocated on first use, about the size
 * of the caller's arrays), two more streams and their events until
 * hps_destroy.  Successive calls on one plan must be issued on the same
 * stream (or be ordered by the caller).  Errors as hps_condense;
 * HPS_ERR_ARG also for chunks outside 0..HPS_HOST_MAX_CHUNKS. */
hps_status hps_condense_host(hps_plan *plan, hps_prec prec, const double *h_coef, const double *h_f,
                             int m, double tol, int kmax, double *h_S, double *h_T, double *h_h,
                             double *h_W, int *h_info, int chunks, hps_stream stream);

/* Upward merges over a uniform-p nx x ny grid of leaves tiling a rectangle
 * (leaf l = ix*ny + iy), nx and ny powers of two.  Each merge of boxes
 * alpha, beta across their shared edge 3 (1, 2 their other edges) forms
 *   Z = Ta33 + Tb33,  S3 = -Z^{-1}[Ta31 Tb32],  w3 = -Z^{-1}(ha3 + hb3),
 *   T = diag(Ta11, Tb22) + [Ta13; Tb23] S3,  h = [ha1; hb2] + [Ta13; Tb23] w3,
 * the Schur complement the paper takes from its HPS references (Section 2).
 * Merges alternate x then y; box boundaries are ordered [W, E, S, N], each
 * side by increasing coordinate.  d_T, d_h as written by hps_condense.  The
 * plan stores S3, w3 of every merge; the root's T is not formed. */
hps_status hps_merge(hps_plan *plan, int nx, int ny, const double *d_T, const double *d_h, int m,
                     hps_stream stream);

/* hps_merge over a grid of unit BOXES instead of leaves: an nx x ny grid
 * (box b = bx*ny + by) of boxes of wx0 x wy0 leaves each, tiling an
 * (nx wx0) x (ny wy0) leaf grid, with DtN maps and fluxes already formed for
 * every box (d_T packed [nx*ny][nbc0][nbc0], d_h [nx*ny][nbc0][m], nbc0 =
 * 2 (wx0 + wy0)(p - 2), boundary order [W, E, S, N] as for merged boxes).
 * The merges are the levels of the whole grid's merge tree above the boxes
 * (the same schedule as hps_merge, so a box must be a box of that tree:
 * one the schedule reaches from the leaves).  wx0 = wy0 = 1 is hps_merge
 * on condensed leaves.  With d_root_Th != NULL the root's own map is formed
 * there as [T | h], row-major n_root x (n_root + m), n_root = 2 (nx wx0 +
 * ny wy0)(p - 2) (hps_merge stops before it).  This is what distributing
 * the merge tree needs (Section 2 merges, one subtree per GPU): each rank
 * merges its own subtree of leaves up to the subtree's root box and
 * forms the root's map; one rank merges the grid of those root boxes.
 * The plan provides p (uniform) and workspace; its n_leaves must equal
 * nx*ny (for boxes, one plan "leaf" per box: hps_build_leaves with the
 * boxes' geometry).  Errors as hps_merge. */
hps_status hps_merge_boxes(hps_plan *plan, int nx, int ny, int wx0, int wy0, const double *d_T, const double *d_h,
                           int m, double *d_root_Th, hps_stream stream);

/* Top-down pass after hps_merge_boxes: from the Dirichlet data d_g on the
 * root's boundary (n_root x m, order [W, E, S, N]) to the boundary values
 * of every unit box, d_ub [nx*ny][nbc0][m] in each box's [W, E, S, N]
 * order (u3 = S3 [u1; u2] + w3 level by level, Section 2 Remark), which
 * hps_solve of a box's own leaf plan then takes as its d_g.  m >= 1 and
 * equal to the merge's m.  HPS_ERR_STATE before a merge. */
hps_status hps_solve_boxes(hps_plan *plan, const double *d_g, int m, double *d_ub, hps_stream stream);

/* SlabLU, the paper's second solver for the reduced system of
 * Eq. (hps_reduced) (Section 2, the block form of Eq. (dell1)), on a
 * uniform-p nx x ny grid of condensed leaves (leaf l = ix*ny + iy, nx and
 * ny powers of two).  The grid is cut into S = nx / s slabs of s leaf
 * columns (s a power of two, 2 <= s <= nx).  Factor: the nodes interior to
 * every slab are eliminated (by the merges inside the slab, which leave the
 * slab's DtN map on its boundary; the Schur complement is the one the
 * paper's per-slab sparse factorization gives), and the block-tridiagonal
 * system on the S - 1 interfaces (nodes on the vertical lines between
 * slabs, ny (p-2) each) is factored by dense block LU in FP64 (one
 * interface after the other, each step a dense LU over many CTAs).  The
 * factorization keeps explicit operators, so hps_slab_solve for new
 * Dirichlet data is matrix-vector products plus the downward pass inside
 * the slabs and the leaf recovery.  d_T, d_h as written by hps_condense;
 * m >= 1.  The plan's merge state is replaced (hps_solve then needs a new
 * hps_merge).  Errors: HPS_ERR_ARG (sizes), HPS_ERR_CUDA / HPS_ERR_OOM. */
hps_status hps_slab_factor(hps_plan *plan, int nx, int ny, int s, const double *d_T, const double *d_h, int m,
                           hps_stream stream);

/* The solve after hps_slab_factor: d_g Dirichlet data on the grid's outer
 * boundary (order [W, E, S, N], n_outer x m, as hps_solve), d_S and d_W as
 * written by hps_condense; d_u per leaf [p*p][m] as hps_solve.
 * HPS_ERR_STATE before hps_slab_factor, HPS_ERR_ARG for another m. */
hps_status hps_slab_solve(hps_plan *plan, const double *d_g, const double *d_S, const double *d_W, int m, double *d_u,
                          hps_stream stream);

/* Where the large dense products of the merge (Section 2 above) run.
 * enable = 1 (default): on the BF16 tensor cores, FP64-accurate, for
 *   - the parents' maps [T | h] = gather + [Ta13; Tb23] [S3 | w3] of the
 *     levels whose shared edge has 16 to 8192 nodes and whose parent
 *     boundary at least 64 (hps_merge, hps_merge_boxes, the merges inside
 *     hps_slab_factor's slabs), and
 *   - the right-hand-side updates of the merge tree's solves over many CTAs
 *     with shared edges of 256 to 8192 nodes: the right-hand side is
 *     eliminated in blocks of 128 rows, each block's rows below (forward)
 *     and above (backward) updated in one product.
 *   Each row of the left factor and each column of the right one is scaled
 *   by a power of two and cut into eight 7-bit integer slices (exact in
 *   BF16); the 36 slice products of order s + t < 8 accumulate in FP32 in
 *   tensor memory (exactly for s + t <= 5, folded into int64) and are added
 *   to the FP64 data they update.  The error of one product is a few
 *   2^-56 K max_k|a_ik| max_k|b_kj|: FP64's where a row / column is of even
 *   magnitude, larger where it spans many orders of magnitude.
 * enable = 2: as 1, and also SlabLU's interface solves (hps_slab_factor),
 *   whose right-hand sides [-U_k | I] have such columns (measured: 4 x 128
 *   leaves, p = 20, one interface of 2304 nodes, a flux mismatch of 6e-12
 *   against 3e-13 on the FP64 pipe).
 * enable = 0: every product on the FP64 pipe.
 * A tensor-core wait that times out makes the call return HPS_ERR_CUDA.
 * HPS_ERR_ARG for other values. */
hps_status hps_set_merge_tensor(hps_plan *plan, int enable);

/* How hps_merge solves Z [S3 | w3] = -[Ta31 Tb32 | ha3 + hb3] (the merge
 * of Section 2 above) on each level.  A level with fewer than `below`
 * merges runs a blocked LU with partial pivoting whose every step is spread
 * over many CTAs (the few large merges near the root); the others run one
 * CTA per merge.  below = -1 (default): the device's SM count; 0: one CTA
 * per merge everywhere.  Levels whose shared edge exceeds 1599 nodes always
 * run one CTA per merge.  Both give the same result up to rounding.
 * Takes effect at the next hps_merge.  HPS_ERR_ARG for below < -1. */
hps_status hps_set_merge_split(hps_plan *plan, int below);

/* Top-down solve after hps_merge (Section 2 Remark: leaf values from the
 * reduced solution).  d_g: Dirichlet data at the outer edge nodes in the
 * root box order [W, E, S, N] (n_outer x m).  Shared-edge values come from
 * u3 = S3 [u1; u2] + w3, leaf interiors from u_i = S u_b + W.
 * d_u per leaf [p*p][m]: the solution at every node; the four corners are
 * written as 0.  d_S and d_W as written by hps_condense (d_W may be NULL
 * when the merge had m body loads of zero).  HPS_ERR_STATE when the last
 * merge was an hps_merge_boxes over boxes larger than one leaf. */
hps_status hps_solve(hps_plan *plan, const double *d_g, const double *d_S, const double *d_W,
                     int m, double *d_u, hps_stream stream);

/* Leaf solve by re-forming and re-factoring: the paper stores no leaf
 * factorization; after the reduced system is solved it assembles and
 * factors every leaf's interior block again and solves for the interior
 * values (Section 2, the remark on leaf factorizations; Section 4, the leaf
 * solve after the reduced solve).  For every leaf, with its edge values
 * u_b given:
 *   u_i = A_ii^{-1} (f_I - A_ib u_b)      (n_i x m)
 * one elimination with m right-hand columns (not the 4(p-2) + m of
 * hps_condense), FP64 or mixed (FP32 factors and the same refinement and
 * FP64 fallback as hps_condense; HPS_MIXED_TF32 / BF16 run the FP32 path).
 * Inputs:  d_coef, d_f as for hps_condense (d_f NULL: no body load);
 *          d_ub per leaf [n_b][m] edge values in the [W, E, S, N] order,
 *          packed like h.
 * Outputs: d_u per leaf [p*p][m] at every node (edge nodes copied from
 *          d_ub, corners 0), packed like the body loads; d_info per leaf
 *          with the codes of hps_condense.
 * m >= 1.  The mixed paths need 4(p-2) + m <= 256 for the largest p. */
hps_status hps_leaf_resolve(hps_plan *plan, hps_prec prec, const double *d_coef, const double *d_f, int m,
                            const double *d_ub, double tol, int kmax, double *d_u, int *d_info,
                            hps_stream stream);

/* The stored-operator leaf solve it replaces: u_i = S u_b + W per leaf,
 * from the S (required) and W (NULL: no body load) of hps_condense, in FP64;
 * d_ub and d_u as for hps_leaf_resolve; leaves of any orders. */
hps_status hps_leaf_recover(hps_plan *plan, const double *d_S, const double *d_W, int m, const double *d_ub,
                            double *d_u, hps_stream stream);

/* Panel width of the blocked LU for one precision path of this plan:
 * nb_panel = 0 restores the automatic choice (the widest panel whose shared
 * memory leaves three CTAs per SM, widened for the mixed path until its
 * refinement staging fits).  Allowed widths: 4, 8, 16 for HPS_FP64 and 8,
 * 16, 32 for HPS_MIXED_FP32; a width whose shared memory does not fit an SM
 * makes the next hps_condense return HPS_ERR_ARG.  Used by autotuners.
 *
 * CUDA graphs: hps_condense enqueues one memset and one kernel on the
 * stream and allocates only when its workspace must grow, so after one
 * call with the same plan, precision and m it can be captured into a graph
 * (with timing off) and replayed. */
hps_status hps_set_blocking(hps_plan *plan, hps_prec prec, int nb_panel);

/* Mixed path: re-condense leaves whose refinement did not converge in FP64
 * (enable = 1, the default) or report them with info = -kmax (enable = 0). */
hps_status hps_set_fp64_fallback(hps_plan *plan, int enable);

/* Mixed path: how refinement decides after the FIRST correction.
 * residual = 0 (default): on the correction alone, the estimate eta_1^2
 * (which reads the error several times low after one correction, so with
 * the default tol = 1e-12 no leaf stops there).  residual = 1: on the true
 * residuals, estimating X_1's error per column as eta_1 r_1 / r_0 (r_k the
 * column max |R_k| of the k-th double-float residual); this runs its own
 * kernel instantiation with one more pass over each of the first two
 * residuals, and lets leaves stop after one correction at tol >= 1e-11.
 * From the second correction on both use eta_k^2 / eta_{k-1}.  The FP32
 * CUDA-core path only (HPS_MIXED_TF32 / BF16 ignore it).  HPS_ERR_ARG for
 * other values. */
hps_status hps_set_refine_stop(hps_plan *plan, int residual);

/* Number of leaves the last HPS_MIXED_FP32 hps_condense call re-condensed in
 * FP64; waits for the stream of that call. */
hps_status hps_fallback_count(hps_plan *plan, int *count);

/* Host-side check of a device info[] array of n entries (as hps_condense,
 * hps_iti_condense and hps_leaf_resolve write it), after the stream that
 * wrote it (synchronous copy on the legacy stream).  Returns HPS_OK when
 * every entry is 0, HPS_ERR_SINGULAR when some entry is > 0 (exact zero
 * pivot), else HPS_ERR_NOCONV when some entry is < 0 (refinement did not
 * reach tol); *first (may be NULL) receives the index of the first entry
 * of that kind, -1 for HPS_OK.  plan may be NULL (the message then goes to
 * hps_last_error(NULL)).  HPS_ERR_ARG for n < 0 or a NULL array with n > 0. */
hps_status hps_check_info(hps_plan *plan, const int *d_info, int n, int *first);

/* Kernel timing with CUDA events recorded on the launch stream around the
 * condensation kernel of every hps_condense call.  hps_set_timing(plan, 1)
 * enables it and clears the record; hps_phase_times fills up to n values:
 *   ms[0] total kernel time of the recorded calls (milliseconds),
 *   ms[1] number of recorded calls,
 *   ms[2] kernel time of the last recorded call.
 * It waits for the recorded events.  HPS_ERR_STATE if timing is off or no
 * call was recorded.  At most 4096 calls are recorded; later calls are not. */
hps_status hps_set_timing(hps_plan *plan, int enable);
hps_status hps_phase_times(hps_plan *plan, float *ms, int n);

/* FP64 condensation of a batch of leaves of one order p, with no device
 * allocation at all.  There is no counterpart in the paper: this entry point
 * serves callers that cannot call cudaMalloc when they condense -- code
 * inside a host framework that owns all device memory through its own pool
 * and forbids outside allocations, or a latency-critical loop where an
 * allocation could block on device synchronisation or fail under memory
 * pressure.  It computes exactly what hps_condense(HPS_FP64) computes for a
 * plan of n_leaves leaves of order p (same layouts, same info codes).
 * Inputs: d_box device [n_leaves][4] (x0, y0, hx, hy); d_coef, d_f, m as in
 *         hps_condense.  Outputs: d_S (may be NULL), d_T, d_h, d_W, d_info.
 * Scratch: the tables and elimination workspace live in a fixed 32 MiB
 * device array inside the library, held by every GPU that loads the library
 * until the process exits.  A call whose tables plus one leaf's workspace
 * ((p-2)^2 x (round4((p-2)^2) + 4(p-2) + m) doubles) do not fit is rejected
 * with HPS_ERR_ARG; a smaller fit means fewer leaves in flight.  Every call
 * looks up the array's device address in the current context
 * (cudaGetSymbolAddress), so the entry point stays valid after
 * cudaDeviceReset; the first call on a device also loads the library's
 * device code there and should come before any stream capture.  All
 * calls on a device share the array: calls that overlap on the GPU (on
 * different streams, or from different host threads without ordering) race
 * and corrupt each other's results.  Errors: HPS_ERR_ARG / HPS_ERR_CUDA, with
 * the message in hps_last_error(NULL) of the calling thread. */
hps_status hps_condense_noalloc(int n_leaves, int p, double kappa, const double *d_box,
                                const double *d_coef, const double *d_f, int m, double *d_S,
                                double *d_T, double *d_h, double *d_W, int *d_info, hps_stream stream);

/* Number of kernel launches enqueued by the last hps_condense call. */
int hps_last_launch_count(const hps_plan *plan);

/* Last error message of this plan, or, when plan is NULL, of the last
 * failed call without a plan (hps_build_leaves, hps_condense_noalloc) made
 * by the calling host thread (the message is kept per thread); never NULL. */
const char *hps_last_error(const hps_plan *plan);

/* Free the plan and its workspace (synchronises the device first). */
void hps_destroy(hps_plan *plan);

/* ABI version: major * 100 + minor (1.01: hps_merge_boxes, hps_solve_boxes;
 * 1.02: hps_slab_factor, hps_slab_solve; 1.03: hps_iti_condense;
 * 1.04: hps_set_merge_tensor; 1.05: hps_check_info). */
int hps_version(void);

#ifdef __cplusplus
}
#endif
#endif /* HPS_H */

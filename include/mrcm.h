/*
 * mrcm.h -- C ABI of the GB300 Recursive MRCM library (libmrcm.so).
 *
 * Method: the Multiscale Robin Coupled Method for Darcy flow
 *     div u = f,  u = -K grad p  in Omega,  p = g_D / u.n = g_N on the boundary
 * (arXiv 2009.07965, Eqs. ellip.1-ellip.3), discretised with lowest-order
 * Raviart-Thomas elements in their lumped (two-point flux) form on a
 * Cartesian grid, with the global interface problem replaced by the binary
 * hierarchy of two-subdomain interface systems of the Recursive MRCM
 * (Section 3, Algorithm 1), in the MuMM specialisation of Section 4:
 * piecewise-constant interface unknowns on segments of H-bar fine faces and
 * one Robin coefficient per segment, beta = alpha * H-bar / K_eff
 * (Eqs. robin.beta, permeff).
 *
 * Every computation behind these calls runs in CUDA kernels on the calling
 * process's current device; there is no CPU fallback.
 *
 * Conventions shared by all calls
 *   - Arrays are float64, x fastest (cell (i, j) at i + nx*j).
 *   - *_dev arguments are device pointers owned by the caller; the library
 *     never frees them.  Host arguments are read before the call returns.
 *   - Face fluxes are integrated over the face (per unit depth in 2D) and
 *     positive in the +axis direction.  Fx has (nx+1)*ny entries, face i of
 *     row j at i + (nx+1)*j; Fy has nx*(ny+1) entries, face j of column i at
 *     i + nx*j.
 *   - Boundary values bc_val: x- faces (ny, by j), x+ faces (ny), y- faces
 *     (nx, by i), y+ faces (nx).  A Dirichlet side holds g_D, a Neumann side
 *     the outward normal flux density g_N.
 *   - Sources q are integrated per cell (q_c = f_c |c|).
 *   - Calls are asynchronous on the stream given to mrcm_setup, except that
 *     each call ends with one stream synchronisation to read the device
 *     status word, so errors are returned by the call that raised them.
 *   - Return value: MRCM_OK or a negative MRCM_ERR_* code; after an error
 *     the context stays valid unless mrcm_setup itself failed.
 */
#ifndef MRCM_H
#define MRCM_H

#ifdef __cplusplus
extern "C" {
#endif

typedef struct mrcm_ctx mrcm_ctx; /* opaque, owned by the library */

typedef struct {
    int dim;       /* 2 or 3 */
    int n[3];      /* cells per axis (n[2] ignored in 2D) */
    double L[3];   /* domain extent per axis; h_d = L[d] / n[d] */
} mrcm_grid;

enum { MRCM_BC_NEUMANN = 0, MRCM_BC_DIRICHLET = 1 };
enum { MRCM_FP64 = 0, MRCM_MIXED = 1, MRCM_SURROGATE = 2 };

enum {
    MRCM_OK = 0,
    MRCM_ERR_INVALID_ARG = -1, /* null pointer, bad size, alpha <= 0, ...  */
    MRCM_ERR_SHAPE = -2,       /* segment does not divide the leaf side, or
                                  leaf larger than 16x16 cells; in 3D: the
                                  patch shape does not tile the leaves or
                                  the leaves the grid, or a patch-shaped
                                  block exceeds 64 cells or 16 faces a side */
    MRCM_ERR_BAD_K = -3,       /* a permeability is <= 0 or not finite      */
    MRCM_ERR_NOT_BUILT = -4,   /* mrcm_solve before mrcm_build_basis         */
    MRCM_ERR_SINGULAR = -5,    /* zero / tiny pivot, or a pivot of the wrong
                                  sign for the quasi-definite interface form,
                                  in a local or interface factorisation     */
    MRCM_ERR_CUDA = -6,        /* a CUDA runtime call failed                 */
    MRCM_ERR_OOM = -7,         /* device allocation failed                   */
    MRCM_ERR_TIMEOUT = -8,     /* a bounded device wait gave up              */
    MRCM_ERR_UNSUPPORTED = -9  /* valid request not implemented (surrogate,
                                  single-leaf pure Neumann; in 3D: batches,
                                  FP32 leaves, double-double residuals)     */
};

/*
 * mrcm_setup -- plan the decomposition and copy the permeability.
 *
 * Section 2 (Eqs. decomp.1-2) and Section 3.1 (Eqs. dd.l, dd.2,
 * interface.1): the grid is cut into leaves of sub_cells[0] x sub_cells[1]
 * cells (the last leaf of a row / column is truncated when n is not a
 * multiple); every leaf side shared with another leaf is cut into segments
 * of seg_cells[1] cells (x-normal sides) or seg_cells[0] cells (y-normal
 * sides), the last one shorter on truncated sides (Section 4, intermediate
 * scale H-bar).  The hierarchy bisects the box of leaves along the axis with
 * more leaves (x on ties), the lower half taking ceil(count/2).
 *
 * 3D (g->dim = 3; Section 5.1 runs its experiments on boxes): the leaves
 * are sub_cells boxes that must tile the grid, every interface between two
 * leaves is cut into patches of seg_cells[t1] x seg_cells[t2] faces (t1 <
 * t2 the tangential axes), each with beta_t = alpha sqrt(|t|) / Keff_t
 * (sqrt(|t|) the patch side, Eqs. robin.beta / permeff).  The leaves' local
 * Robin problems are solved by the same recursive merges: the grid is tiled
 * by blocks of the patch shape (at most 64 cells, at most 16 faces a side),
 * every face between two blocks of one leaf is a segment of its own (on
 * which the Robin coupling is exact for any beta) and the side between
 * blocks of two leaves is one patch; one tree bisects the box of blocks
 * along the axis with the most blocks (x, y, z on ties).  One problem per
 * context.
 *
 *   out        receives the new context (NULL on failure)
 *   g          grid; g->dim 2 or 3
 *   K_dev      device array, n[0]*n[1] (3D: n[0]*n[1]*n[2]) permeabilities
 *              (> 0), x fastest; copied, the caller may free it when the
 *              call returns
 *   sub_cells  leaf shape in cells, each in [1, 16] (3D: any multiple of the
 *              patch shape that divides n)
 *   seg_cells  segment length in cells; must divide sub_cells per axis
 *   alpha      dimensionless Robin parameter of Eq. (robin.beta), > 0
 *   bc_type    per side (x-, x+, y-, y+, z-, z+): MRCM_BC_NEUMANN or
 *              MRCM_BC_DIRICHLET (z entries ignored in 2D).  All-Neumann
 *              problems are solved with zero-mean pressure.
 *   precision  MRCM_FP64: every step in FP64.  MRCM_MIXED: the merges
 *              (their blocked eliminations and products; by default every
 *              one, mrcm_set_mixed_split) in FP32, and optionally the leaf
 *              factorisations and basis solves (mrcm_set_mixed_leaves; FP64
 *              by default); the coefficients, the solve passes, the
 *              residuals and the fluxes in FP64; mrcm_solve
 *              then refines 3 times by default (2 in 3D; mrcm_set_refinement) with
 *              FP64 residuals (mrcm_set_residual), which brings the result
 *              near the FP64 form's accuracy when the FP32 factors contract
 *              the error (Wilkinson's iterative refinement).  In 3D the
 *              blocks are always factored in FP64.
 *              MRCM_SURROGATE returns MRCM_ERR_UNSUPPORTED.
 *   cuda_stream  cudaStream_t to run on (NULL = legacy default stream)
 * The context allocates and owns all device workspace.
 */
int mrcm_setup(mrcm_ctx** out, const mrcm_grid* g, const double* K_dev,
               const int sub_cells[3], const int seg_cells[3], double alpha,
               const int bc_type[6], int precision, void* cuda_stream);

/*
 * mrcm_setup_batch -- one context for `count` independent problems (an
 * ensemble of realisations, Section 5's permeability studies run many at
 * once), each on its own grid: grids[k] and bc_types[6 k .. 6 k + 5] as in
 * mrcm_setup; sub_cells, seg_cells, alpha and precision shared.  Every grid
 * gets its own leaves (truncated at its own edges), segments and merge
 * tree; the build and solve then run all of them together, one launch per
 * tree height over every tree (the Recursive MRCM of Algorithm 1 applied to
 * each problem), so small problems fill the GPU as one large one would.
 * The paper solves one problem at a time; batching is this library's.
 *
 * Arrays of a batched context are the problems' arrays concatenated in
 * grid order: K_dev, q, p (sum of n[0] n[1]), Fx (sum of (n[0]+1) n[1]),
 * Fy (sum of n[0] (n[1]+1)), bc_val (sum of 2 (n[0] + n[1])), and the
 * one-sided fluxes [Fa_x | Fb_x | Fa_y | Fb_y], each part concatenated in
 * grid order.  mrcm_setup is mrcm_setup_batch with count 1.
 *
 * Errors as mrcm_setup; MRCM_ERR_UNSUPPORTED when count > 1 and a problem
 * has no Dirichlet side (the zero-mean all-Neumann form is single-problem
 * only); MRCM_ERR_INVALID_ARG beyond 2^31 cells or faces in total.
 */
int mrcm_setup_batch(mrcm_ctx** out, int count, const mrcm_grid* grids, const int* bc_types,
                     const double* K_dev, const int sub_cells[3], const int seg_cells[3], double alpha,
                     int precision, void* cuda_stream);

/*
 * mrcm_set_permeability -- replace K (same grid), invalidating the basis.
 * K_dev: device array of n[0]*n[1] values > 0, copied.
 */
int mrcm_set_permeability(mrcm_ctx* ctx, const double* K_dev);

/*
 * mrcm_build_basis -- the data-dependent part that depends only on K, alpha
 * and the boundary-condition types.
 *
 *   1. Robin coefficients per segment, Eqs. (robin.beta) and (permeff).
 *   2. Every leaf's local Robin problem, Eqs. (11.2)-(12.2) with the MMBF
 *      data of Eqs. (11Hhatbasisa)/(11Hhatbasisb): the leaf's pressure
 *      matrix is factored (LDL^T) and its Robin-to-flux map R (one response
 *      per interface segment) is formed.
 *   3. The recursive merge of Algorithm 1, one batched step per tree height:
 *      each pair of siblings solves its interface system on gamma (Eq.
 *      linsys restricted to gamma, rows from Eqs. 13.2 and 14.2) and passes
 *      the merged map up (Eqs. new_bfs.1-2, coefficient tracking remark of
 *      Section 3.2).
 * Errors: MRCM_ERR_BAD_K, MRCM_ERR_SINGULAR, MRCM_ERR_CUDA.
 */
int mrcm_build_basis(mrcm_ctx* ctx);

/*
 * mrcm_solve -- sources and boundary values -> pressures and fluxes.
 *
 *   1. Each leaf's particular solution (Eqs. addu/addp) and its interface
 *      flux traces; up-sweep of the particular data (Eqs. particular.1-2).
 *   2. Root interface system, then top-down recovery of every interface
 *      unknown (Algorithm 1).
 *   3. Final local solutions, Eq. (final): cell pressures.
 *   4. Iterative refinement (mrcm_set_refinement), then the zero-mean shift
 *      of all-Neumann problems and the face fluxes from the cell pressures
 *      and the interface unknowns.
 *
 *   q_dev      n[0]*n[1] integrated sources.  All-Neumann problems need
 *              compatible data: |sum q - sum |e| g_N| <= 1e-14 (sum |q| +
 *              sum |e| |g_N|), both sums evaluated in double-double on the
 *              device; otherwise the call returns MRCM_ERR_INVALID_ARG
 *   bc_val_dev 2*(n[0]+n[1]) boundary values (layout in the header comment);
 *              3D: the six sides x-, x+, y-, y+, z-, z+ concatenated, the x
 *              sides n[2]*n[1] values, the y sides n[2]*n[0], the z sides
 *              n[1]*n[0], each with its first listed index slowest
 *   p_dev      out: n[0]*n[1] (3D: n[0]*n[1]*n[2]) cell pressures
 *   Fx_dev     out: (n[0]+1)*n[1] x-face fluxes (3D: (n[0]+1)*n[1]*n[2]);
 *              skeleton faces hold the mean of the two one-sided values
 *   Fy_dev     out: n[0]*(n[1]+1) y-face fluxes (3D: n[0]*(n[1]+1)*n[2])
 *   Fz_dev     must be NULL in 2D; in 3D required, n[0]*n[1]*(n[2]+1)
 *              z-face fluxes
 *   iface_dev  optional out (NULL to skip): one-sided fluxes, 2*((n[0]+1)*n[1]
 *              + n[0]*(n[1]+1)) values laid out as [Fa_x, Fb_x, Fa_y, Fb_y],
 *              each face-shaped like Fx / Fy; side a is the lower-coordinate
 *              leaf, side b the upper one, both in the +axis direction; off
 *              the skeleton both equal the face flux.  3D: 2*(number of x-,
 *              y- and z-faces) values, [Fa_x, Fb_x, Fa_y, Fb_y, Fa_z, Fb_z].
 * Errors: MRCM_ERR_NOT_BUILT, MRCM_ERR_INVALID_ARG, MRCM_ERR_TIMEOUT,
 * MRCM_ERR_CUDA.
 */
int mrcm_solve(mrcm_ctx* ctx, const double* q_dev, const double* bc_val_dev,
               double* p_dev, double* Fx_dev, double* Fy_dev, double* Fz_dev,
               double* iface_dev);

/* Keys of mrcm_query. */
enum {
    MRCM_Q_LEAVES = 0,        /* number of leaves (3D: patch-shaped blocks)   */
    MRCM_Q_SEGMENTS = 1,      /* number of interface segments                */
    MRCM_Q_LEVELS = 2,        /* tree height (merge steps from leaf to root) */
    MRCM_Q_NODES = 3,         /* tree nodes, leaves included                 */
    MRCM_Q_WORKSPACE_BYTES = 4,
    MRCM_Q_MAX_GAMMA = 5,     /* largest interface system size 2g            */
    MRCM_Q_BUILD_FLOPS = 6,   /* algorithmic FP64 flops of mrcm_build_basis  */
    MRCM_Q_SOLVE_FLOPS = 7,   /* algorithmic FP64 flops of mrcm_solve        */
    MRCM_Q_LEAF_FLOPS = 8,    /* part of BUILD_FLOPS in the leaf kernel      */
    MRCM_Q_KERNEL_LAUNCHES_BUILD = 9, /* kernels launched by one build call  */
    MRCM_Q_KERNEL_LAUNCHES_SOLVE = 10, /* kernels launched by one solve call */
    MRCM_Q_GRAPH_REPLAYS = 11, /* build and solve calls so far that replayed a
                                 captured CUDA graph (see mrcm_use_graphs)   */
    /* reference flop model of a direct method, independent of this
       library's algorithms: banded Cholesky leaves n b^2 + 2 n b m +
       m (m + 1) n + 4 n b (n cells, bandwidth b, m segments), LU-based
       merges (2/3) N^3 + 2 N^2 (m + 1) + 2 m g (m + 1) (N = 2g) */
    MRCM_Q_MODEL_BUILD_FLOPS = 12, /* the whole build under that model        */
    MRCM_Q_MODEL_SWEEP_FLOPS = 13, /* (2/3) N^3 of the merges that run in the
                                     blocked sweep (MRCM_PHASE_GJ_SWEEP)     */
    MRCM_Q_GRIDS = 14,        /* problems in the context (mrcm_setup_batch)   */
    MRCM_Q_CELLS = 15         /* cells over all of them                       */
};

/* mrcm_query -- integer facts about a context.  value: host out pointer. */
int mrcm_query(const mrcm_ctx* ctx, int what, long long* value);

/*
 * mrcm_plan_query -- the same integer facts as mrcm_query (keys
 * MRCM_Q_LEAVES .. MRCM_Q_LEAF_FLOPS and the two MODEL keys; WORKSPACE_BYTES
 * is 0),
 * computed from the decomposition alone on the host: no device, no CUDA
 * call.  Arguments as in mrcm_setup; value: host out pointer.
 */
int mrcm_plan_query(const mrcm_grid* g, const int sub_cells[3], const int seg_cells[3],
                    const int bc_type[6], int what, long long* value);

/* Phases timed by mrcm_phase_times: each groups the launches of one kernel
 * family, so a phase time is the time of that family's kernels. */
enum {
    MRCM_PHASE_COEF = 0,           /* permeability check, Robin and face coefficients */
    MRCM_PHASE_LEAF_BUILD = 1,     /* leaf factorisation and Robin-to-flux maps     */
    MRCM_PHASE_MERGE_SMALL = 2,    /* whole merges of small interface systems       */
    MRCM_PHASE_GJ_SWEEP = 3,       /* blocked merges: Gauss-Jordan inversion of the
                                      quasi-definite form (the cooperative sweep, or
                                      one system per CTA for many mid-sized ones)  */
    MRCM_PHASE_MERGE_FORM = 4,     /* blocked merges: the quasi-definite form of the
                                      interface matrix and its back transform; now
                                      done inside the sweep's launch (timed as
                                      MRCM_PHASE_GJ_SWEEP, this phase reports 0)   */
    MRCM_PHASE_MERGE_X = 5,        /* blocked merges: X = -W C                      */
    MRCM_PHASE_MERGE_R = 6,        /* blocked merges: merged R = R_oo + C^T X       */
    MRCM_PHASE_LEAF_PART = 7,      /* leaf particular solutions (solve)             */
    MRCM_PHASE_TREE_UP = 8,        /* up-sweep of the particular fluxes (solve)     */
    MRCM_PHASE_TREE_DOWN = 9,      /* down-sweep of the Robin data (solve)          */
    MRCM_PHASE_LEAF_PRESSURE = 10, /* leaf pressures, interface unknowns (solve)    */
    MRCM_PHASE_RESIDUAL = 11,      /* refinement residuals (solve)                  */
    MRCM_PHASE_FINISH = 12,        /* mean shift and face fluxes (solve)            */
    MRCM_PHASE_ROOT_FACTOR = 13,   /* blocked merges of a root level in the factor
                                      form: block LDL^T of the quasi-definite form
                                      (mrcm_set_root_form)                         */
    MRCM_PHASE_COUNT = 14
};

/*
 * mrcm_set_refinement -- iterative refinement of mrcm_solve (default 1 step).
 *
 * The discrete MRCM solution is the exact solution of Eqs. (11.2)-(14.2)
 * (lumped RT0); a direct FP64 solve meets it only to the conditioning of the
 * problem times the rounding unit.  Each step evaluates the residual of
 * those equations in double-double arithmetic and solves for the
 * correction with the factored basis (Wilkinson's iterative refinement);
 * the result then matches the discrete solution to near FP64 accuracy when
 * the conditioning is below 1/u.  (With the quasi-definite interface
 * inverses the unrefined solve of a sigma^2 = 4 log-normal field at 1024^2
 * is already within 1e-11 of it; one step reaches the rounding level.)
 *   steps  0..16 refinement steps per mrcm_solve; with 0 (the paper's single
 *          pass) the outputs are formed in plain FP64, otherwise from the
 *          double-double state, rounded once
 *   check  != 0: evaluate the residual once more after the last step (for
 *          mrcm_residual_history)
 *
 * mrcm_residual_history -- out[k] (host) = max |residual| of the k-th
 * evaluation in the last mrcm_solve (cell balances, Eq. 13.2 and 14.2 rows,
 * unscaled); returns the number of evaluations (>= 0) or an error code.
 *
 * mrcm_set_residual -- dd = 1: the refinement residuals in double-double
 * (the FP64 form's default: refinement to the FP64 rounding level); dd = 0:
 * in plain FP64, about six times fewer FP64 operations (the mixed form's
 * default: enough for its 1e-8 target, the refined result then stalls near
 * the plain FP64 solve's accuracy; the only choice in 3D).  Takes effect at
 * the next mrcm_solve.
 * Errors: MRCM_ERR_INVALID_ARG, MRCM_ERR_UNSUPPORTED (dd = 1 in 3D).
 */
int mrcm_set_refinement(mrcm_ctx* ctx, int steps, int check);
int mrcm_set_residual(mrcm_ctx* ctx, int dd);

/*
 * mrcm_set_wait_limit -- polls after which a bounded wait between the CTAs
 * of one cooperative launch (the blocked interface sweeps and the solve's
 * tree sweeps) gives up; the paper has no counterpart.  polls < 0 restores
 * the default (about a second of polling); 0 gives up at the first check
 * that finds the awaited condition unmet.  A wait that gives up makes the
 * call return MRCM_ERR_TIMEOUT; every CTA then leaves the launch at its
 * next wait, nothing is left running, and the context stays usable (a later
 * call with a sufficient limit recomputes everything it needs).  A very
 * small limit is how failure handling is exercised without a fault.
 * Synchronises the context's stream and drops its captured graphs when the
 * limit changes.
 */
int mrcm_set_wait_limit(mrcm_ctx* ctx, long long polls);

/*
 * mrcm_set_mixed_split -- mixed form only: merges whose interface system
 * has 2g <= max_g2_fp32 run in FP32, larger ones in FP64 (default 2^30,
 * every merge in FP32; 0: every merge in FP64).  The paper has no counterpart (its arithmetic is FP64 throughout).
 * Invalidates the basis (call mrcm_build_basis again).  Errors:
 * MRCM_ERR_INVALID_ARG (negative), MRCM_ERR_UNSUPPORTED (not a mixed
 * context), MRCM_ERR_CUDA.
 */
int mrcm_set_mixed_split(mrcm_ctx* ctx, int max_g2_fp32);

/*
 * mrcm_set_mixed_leaves -- mixed form only: fp32 = 1 keeps the leaf
 * factorisations and their stored factors in FP32, fp32 = 0 (the default)
 * in FP64 (then only the merges up to the split run in FP32; their errors
 * are not amplified by the interface systems above as much as the leaf
 * maps' are, and the refinement converges in fewer steps).  The paper has no
 * counterpart.  A mixed context holds both sets of leaf arrays.  Invalidates
 * the basis (call mrcm_build_basis again).  Errors: MRCM_ERR_INVALID_ARG
 * (fp32 not 0 or 1), MRCM_ERR_UNSUPPORTED (not a mixed context, or fp32 = 1
 * in 3D), MRCM_ERR_CUDA.
 */
int mrcm_set_mixed_leaves(mrcm_ctx* ctx, int fp32);

/*
 * mrcm_set_root_form -- how the interface system of a tree's root is kept
 * (Algorithm 1's top merge: the root has no outer segments, so the build
 * needs neither X nor a merged map there, only the means to solve for
 * lambda_gamma in every solve pass, Section 3.2).
 * MRCM_ROOT_FACTOR: the block LDL^T factor T = Lt Dt Lt^T of the
 * quasi-definite form (16-wide diagonal blocks, inverted with the same
 * sign-checked elimination as the inverse), about a third of the
 * inversion's flops; each solve pass then runs two block triangular sweeps
 * on it (64-row blocks, each waiting only for the blocks it depends on).
 * MRCM_ROOT_INVERSE: the explicit inverse, as at every other blocked height;
 * each solve pass then applies it as a matrix-vector product.
 * MRCM_ROOT_AUTO (the default): the factor for root systems of 2g >= 1024,
 * the inverse below (there both eliminations are bound by the same chain of
 * pivot blocks and the product is the shorter solve).
 * Applies to tree heights with 2g > 32 whose nodes all lack outer segments.
 * Both forms solve the same equations (to rounding).  Invalidates the basis
 * (call mrcm_build_basis again).  Errors: MRCM_ERR_INVALID_ARG,
 * MRCM_ERR_CUDA.
 */
enum { MRCM_ROOT_FACTOR = 0, MRCM_ROOT_INVERSE = 1, MRCM_ROOT_AUTO = 2 };
int mrcm_set_root_form(mrcm_ctx* ctx, int form);

/*
 * mrcm_autotune -- picks the launch shapes of every blocked merge level by
 * timing them on this device: CTAs per SM of the cooperative Gauss-Jordan
 * sweep (1 to 4), rows of X per CTA (32 or 64), side of an R tile (16 or
 * 32); each candidate is run `reps` times (1..100) on the context's stream
 * and the fastest kept per launch and tree height.  Every shape computes the
 * same numbers, so the basis stays valid; later builds use the choices (the
 * captured build graph is dropped).  The paper has no counterpart.  Needs a
 * built basis (MRCM_ERR_NOT_BUILT otherwise).  Errors: MRCM_ERR_INVALID_ARG,
 * MRCM_ERR_NOT_BUILT, MRCM_ERR_TIMEOUT, MRCM_ERR_CUDA.
 *
 * mrcm_tune_info -- the choices for tree height `height` (1 = the leaves'
 * parents): out[0] CTAs per SM of the sweep, out[1] X rows, out[2] R tile;
 * 0 where the built-in heuristic applies (before mrcm_autotune, and on
 * heights merged by the small-system kernel); out[0] is also 0 on heights
 * inverted one system per CTA (2g <= 128 with at least one node per two
 * SMs: a fixed rule, no launch shape to choose).
 */
int mrcm_autotune(mrcm_ctx* ctx, int reps);
int mrcm_tune_info(const mrcm_ctx* ctx, int height, int out[3]);
int mrcm_residual_history(mrcm_ctx* ctx, double* out, int cap);

/*
 * mrcm_enable_timing -- on != 0: record a CUDA event pair around every launch
 * group of a phase in the following build / solve calls (on the context's
 * stream).
 * mrcm_phase_times -- ms[MRCM_PHASE_COUNT] (host) receives, per phase, the
 * summed durations of its launch groups in the most recent build and solve
 * (0 where not run).  Only valid after a call made with timing enabled.
 */
int mrcm_enable_timing(mrcm_ctx* ctx, int on);
int mrcm_phase_times(mrcm_ctx* ctx, double* ms);

/*
 * mrcm_use_graphs -- on != 0 (the default): mrcm_build_basis and mrcm_solve
 * capture their launch sequence into a CUDA graph on the first call and
 * replay it on later calls; the solve graph is captured again when its
 * buffer pointers, the refinement settings or timing change.  The results
 * are those of the direct launches, bit for bit.  A context created on the
 * legacy default stream (stream NULL), or whose stream refuses capture,
 * launches directly.  on == 0 launches directly and frees the graphs (after
 * synchronising the context's stream).  The graph replays the buffers given
 * at capture, so their contents may change between calls but they must
 * stay allocated while the graph may run again.
 */
int mrcm_use_graphs(mrcm_ctx* ctx, int on);

/*
 * mrcm_check_reciprocal -- self-check of the reciprocal the interface and
 * leaf kernels use on their sequential pivot chains (a single-precision seed
 * refined by one third-order step of the Newton-Raphson family, within an
 * ulp of 1/x); the paper has no counterpart.  r_dev[i] = 1/x_dev[i] for i < n, both device arrays of n
 * doubles owned by the caller, on cuda_stream (NULL: legacy default
 * stream); synchronises the stream.  Returns MRCM_OK, MRCM_ERR_INVALID_ARG
 * (null pointer, n < 0) or MRCM_ERR_CUDA.
 */
int mrcm_check_reciprocal(const double* x_dev, double* r_dev, long long n, void* cuda_stream);

/*
 * mrcm_group_times -- the timed launch groups of the most recent build and
 * solve in launch order: phase[k] (host) its phase id, ms[k] (host) its
 * duration, for k < min(count, cap).  Returns the number of groups recorded
 * (>= 0) or an error code.  A merge level contributes one group per phase
 * it launches, so the groups of the build resolve the tree height by height.
 */
int mrcm_group_times(mrcm_ctx* ctx, int* phase, double* ms, int cap);

/*
 * mrcm_phase_flops -- flops[MRCM_PHASE_COUNT] (host) receives the algorithmic
 * FP64 flop count of each phase for one mrcm_build_basis (build phases) and
 * one mrcm_solve with the current refinement setting (solve phases): the
 * arithmetic the algorithm needs (a fused multiply-add counts 2), not the
 * instructions a kernel issues.  Host only, no device call.
 */
int mrcm_phase_flops(const mrcm_ctx* ctx, double* flops);

/*
 * Introspection for tests (host buffers, synchronous).
 *
 * mrcm_node_info: info[0] = height (0 for leaves), info[1] = m (outer
 * segments), info[2] = g (segments on the node's internal interface gamma,
 * 0 for leaves), info[3], info[4] = children (-1 for leaves), info[5] =
 * parent (-1 for a root), info[6] = leaf index or -1, info[7..10] = leaf
 * box I0, I1, J0, J1 (half-open, in the leaf grid of the node's own
 * problem).  Nodes 0..leaves-1 are the leaves (problem after problem).
 *
 * mrcm_node_segments: seg_ids[m] = the node's outer segments in the order
 * its R uses.
 *
 * mrcm_segment_info: info[0] = axis of the normal, info[1] = face line
 * (x-face index for axis 0, y-face index for axis 1), info[2] = first cell
 * along the segment, info[3] = number of faces, info[4] = leaf on side a,
 * info[5] = leaf on side b.
 *
 * mrcm_node_operator: R_host[m*m] (row-major) = the node's Robin-to-flux
 * map (outward segment fluxes per unit Robin datum) after mrcm_build_basis;
 * rbar_host[m] (may be NULL) = its particular fluxes after mrcm_solve.
 */
int mrcm_node_info(const mrcm_ctx* ctx, int node, int info[11]);
int mrcm_node_segments(const mrcm_ctx* ctx, int node, int* seg_ids);
int mrcm_segment_info(const mrcm_ctx* ctx, int seg, int info[6]);
int mrcm_node_operator(mrcm_ctx* ctx, int node, double* R_host, double* rbar_host);

/*
 * mrcm_merge_pair_noalloc -- merge two Robin-to-flux maps along their common
 * interface without allocating device memory.
 *
 * The paper has no counterpart to this call; it exists for callers that
 * cannot call cudaMalloc where they need a merge: code running inside
 * another framework's execution step (an inference-engine plugin's enqueue,
 * a solver callback) whose framework owns all device memory, and
 * latency-bound loops that cannot absorb the device synchronisation an
 * allocation implies.  It computes what one merge of mrcm_build_basis
 * computes for one node, from caller-owned buffers only:
 *     M = [[R1_gg + D, -D], [-D, R2_gg + D]]  (2g x 2g, partial-pivot LU),
 *     X = -M^-1 blockdiag(R1_go, R2_go),
 *     R = blockdiag(R1_oo, R2_oo) + blockdiag(R1_og, R2_og) X.
 *
 *   R1_dev, R2_dev  children's maps, m1 x m1 and m2 x m2, row-major (device)
 *   map_dev   device ints, 2g + m values: gpos1[g], gpos2[g] (positions of
 *             the gamma segments in child 1 / child 2, same gamma order),
 *             opos1[m1-g], opos2[m2-g] (the children's other positions, in
 *             the order the merged map uses); out-of-range entries make the
 *             call return MRCM_ERR_INVALID_ARG without touching R or X
 *   g         gamma segments, 1 <= 2g <= MRCM_NOALLOC_MAX_G2
 *   D_dev     g values |t| / (2 beta_t) of the gamma segments (device)
 *   R_dev     out: merged map, m x m with m = m1 + m2 - 2g (device)
 *   X_dev     out: coefficients, 2g x m (device)
 *   cuda_stream  stream to run on
 *
 * Workspace: the LU factors, pivots and a status word live in one
 * file-scope device array sized for 2g = MRCM_NOALLOC_MAX_G2 (about 513 KB),
 * which every GPU that loads the library holds until the process exits.
 * Every call looks up that array's device address for the current device
 * and context (a host-side query that allocates nothing).  Every call
 * reuses the same array and clears the status word itself, so calls that
 * overlap on the GPU (different streams or devices sharing a context) race:
 * serialise them.  The call synchronises its stream once to read the
 * status.  Larger systems return MRCM_ERR_INVALID_ARG.  The interface
 * matrix is factored by LU with partial pivoting (not by the build's
 * quasi-definite inversion, which gives the same maps); MRCM_ERR_SINGULAR
 * here means a pivot of magnitude <= 1e-14 max|M| (no sign test).
 * Errors: MRCM_ERR_INVALID_ARG, MRCM_ERR_SINGULAR, MRCM_ERR_CUDA.
 */
#define MRCM_NOALLOC_MAX_G2 256
int mrcm_merge_pair_noalloc(const double* R1_dev, int m1, const double* R2_dev, int m2,
                            const int* map_dev, int g, const double* D_dev,
                            double* R_dev, double* X_dev, void* cuda_stream);

/*
 * mrcm_probe_peak -- measured throughput ceiling of one arithmetic pipe of
 * the current device, the denominator of the kernels' roofline figures; the
 * paper has no counterpart.  Every scheduler of every SM runs independent
 * chains of one instruction kind for about `seconds` (0 < seconds <= 10) in
 * three timed runs on cuda_stream (NULL: legacy default stream); *tflops
 * (host) receives the fastest run's rate in TFLOP/s (an FMA counts 2
 * flops, an m x n x k MMA 2mnk).  Synchronises the stream.  Errors:
 * MRCM_ERR_INVALID_ARG (unknown kind, bad seconds, NULL tflops),
 * MRCM_ERR_CUDA.
 */
enum {
    MRCM_PROBE_DFMA = 0,   /* FP64 fused multiply-add                        */
    MRCM_PROBE_DMMA = 1,   /* FP64 mma.sync m8n8k4                           */
    MRCM_PROBE_FFMA = 2,   /* FP32 fused multiply-add                        */
    MRCM_PROBE_TF32 = 3,   /* mma.sync m16n8k8, TF32 inputs, FP32 accumulate */
    MRCM_PROBE_BF16 = 4,   /* mma.sync m16n8k16, BF16 inputs, FP32 accumulate */
    MRCM_PROBE_DFMA_DMMA = 5  /* half the warps FP64 FMA, half FP64 MMA      */
};
int mrcm_probe_peak(int kind, double seconds, double* tflops, void* cuda_stream);

/*
 * Learned basis surrogate (the learned part of the grown form; the paper
 * computes every basis by a local solve).  A leaf's basis responses, Eqs.
 * (11Hhatbasisa)/(11Hhatbasisb), are the fields psi_s = A^-1 B e_s (cell
 * pressures for a unit Robin datum on segment s, local Robin problem of Eq.
 * 11.2-12.2), and its Robin-to-flux map is R = B^T psi - W.  A small
 * convolutional network predicts the 16 fields of a full interior 16 x 16
 * leaf from its permeability patch; a residual gate keeps a prediction only
 * where ||A psi_s - B e_s|| / ||B e_s|| <= tau for every s, and the plain
 * local solve stands for every other leaf.
 *
 * Leaf lists are device int arrays of leaf ids (out-of-range ids, and leaves
 * with more than 16 segments, make the call return MRCM_ERR_INVALID_ARG);
 * contexts whose leaves have more than 16 segments return
 * MRCM_ERR_UNSUPPORTED.  Every call synchronises the context's stream.
 *
 * mrcm_interior_leaves -- ids (host, up to cap) of the full interior leaves
 *   (16 x 16 cells, 4 segments per side, no side on the domain boundary);
 *   returns their number (host only).
 * mrcm_leaf_fields -- psi_dev[item][256][16] (float; cell i + 16 j, then
 *   segment: the network's output layout) of the listed leaves from the
 *   built basis (training targets).
 * mrcm_leaf_patches -- x_dev[item][18][18][16] (bf16, NHWC): channel 0 =
 *   (log K - its mean over the leaf) / 2 on the leaf and a one-cell halo,
 *   channel 1 = log10(alpha) / 3, others 0 (network inputs).
 * mrcm_leaf_gate -- res_dev[item] (double) = max over s of the relative
 *   residual of predicted fields psi_dev (float, layout of
 *   mrcm_leaf_fields), in FP64.
 * mrcm_leaf_apply -- for the items with res <= tau: R = B^T psi - W
 *   (symmetrised) replaces the leaf's map; accepted_dev[item] = 1 for them,
 *   0 for the others; then the merges are rebuilt (mrcm_solve uses the new
 *   maps, the leaf factors are unchanged).
 */
int mrcm_interior_leaves(const mrcm_ctx* ctx, int* ids, int cap);
int mrcm_leaf_fields(mrcm_ctx* ctx, const int* ids_dev, int count, float* psi_dev);
int mrcm_leaf_patches(mrcm_ctx* ctx, const int* ids_dev, int count, void* x_dev);
int mrcm_leaf_gate(mrcm_ctx* ctx, const int* ids_dev, int count, const float* psi_dev, double* res_dev);
int mrcm_leaf_apply(mrcm_ctx* ctx, const int* ids_dev, int count, const float* psi_dev, const double* res_dev,
                    double tau, int* accepted_dev);

/*
 * The network's kernels (no context; device buffers; asynchronous on
 * `stream`).  Activations are bf16 NHWC [item][y][x][c], weights bf16
 * [cout][ky][kx][cin], biases and gradients float.  Every output is 16 x 16.
 *
 * mrcm_cnn_conv_forward -- y = act(conv3x3(x, w) + b) on the tensor cores
 *   (mma.sync m16n8k16, BF16 operands, FP32 accumulation): pad = 0 takes an
 *   18 x 18 input ('valid'), pad = 1 a 16 x 16 input with a zero border
 *   ('same'); relu != 0 applies max(., 0); writes y_bf16 and / or y_f32
 *   (either may be NULL, not both); b may be NULL.  Shapes (cin, cout, pad):
 *   (16, 32, 0), (16, 32, 1), (32, 32, 1), (32, 16, 1); others return
 *   MRCM_ERR_UNSUPPORTED.
 * mrcm_cnn_conv_wgrad -- dw[cout][9 cin] += sum over items and pixels of
 *   dy x im2col(x), db[cout] += sum of dy (db may be NULL); shapes (16, 32,
 *   0), (32, 32, 1), (32, 16, 1).
 * mrcm_cnn_flip_weights -- w2[cin][ky][kx][cout] = w[cout][2-ky][2-kx][cin]:
 *   the forward kernel on w2 (cin and cout swapped, pad 1) computes the
 *   input gradient of a 'same' convolution.
 * mrcm_cnn_relu_grad -- dpre (bf16) = dpost (float) where y > 0 (mask != 0;
 *   y the layer's bf16 output), else 0; mask == 0 copies.
 * mrcm_cnn_mse_grad -- loss 0.5 sum (pred - target)^2 / count added into
 *   *loss (device float); dpred = (pred - target) / count.  pred and target
 *   float [count][16][16][16] (NHWC).
 * mrcm_cnn_adam -- one Adam step (step >= 1) on float parameters p with
 *   gradient g and moments m1, m2; p_bf16 (may be NULL) receives the bf16
 *   copy.
 */
int mrcm_cnn_conv_forward(const void* x, int count, int cin, int cout, int pad, int relu, const void* w,
                          const float* b, void* y_bf16, float* y_f32, void* stream);
int mrcm_cnn_conv_wgrad(const void* x, const void* dy, int count, int cin, int cout, int pad, float* dw,
                        float* db, void* stream);
int mrcm_cnn_flip_weights(const void* w, int cout, int cin, void* w2, void* stream);
int mrcm_cnn_relu_grad(const float* dpost, const void* y, long long n, int mask, void* dpre, void* stream);
int mrcm_cnn_mse_grad(const float* pred, const float* target, int count, float* dpred, float* loss,
                      void* stream);
int mrcm_cnn_adam(float* p, const float* g, float* m1, float* m2, void* p_bf16, long long n, float lr,
                  float beta1, float beta2, float eps, int step, void* stream);

/* mrcm_destroy -- free all device and host resources (NULL is a no-op). */
void mrcm_destroy(mrcm_ctx* ctx);

/* mrcm_error_string -- static text for an MRCM_* code. */
const char* mrcm_error_string(int code);

/*
 * mrcm_last_cuda_error -- the cudaError_t behind the last MRCM_ERR_CUDA or
 * MRCM_ERR_OOM returned on the calling thread (0 if none); its name is
 * copied into name[cap] (host, NUL-terminated, may be NULL).
 */
int mrcm_last_cuda_error(char* name, int cap);

#ifdef __cplusplus
}
#endif
#endif /* MRCM_H */

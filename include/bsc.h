/*
 * bsc.h - C ABI of the GB300 (sm_103a) hot path of quadratic B-spline cloth
 * FEM ("Efficient B-Spline Finite Elements for Cloth Simulation",
 * arXiv 2506.18867).
 *
 * One Newton iteration of the paper's implicit-Euler incremental potential
 * (Sec. 3.2, Eq. incremental_potential) evaluates FBW membrane energy
 * (Sec. 4.1) and quadratic bending energy (Sec. 4.2) at the reduced
 * quadrature points of every knot span, projects each span's 27x27 Hessian
 * to PSD (projected Newton, Sec. 5.1), assembles the global Hessian (each
 * control point couples to its 5x5 neighbourhood in 3x3 blocks, Sec. 5.2),
 * and solves with preconditioned CG on that matrix.
 *
 * Conventions shared by every call
 * --------------------------------
 *  - Patch: nu x nv control points (nu, nv >= 5) on open uniform quadratic
 *    knot vectors (0,0,0,1,...,S,S,S), S = n - 2 spans per axis (Sec. 3.1.2:
 *    open, integer lattice, starting at 0).  Control point alpha = j*nu + i.
 *  - Element type: double when the context was created with BSC_FP64, float
 *    with BSC_FP32 ("T" below).  Energies are always double.
 *  - Vectors of control-point data (positions C, gradients, x, y): three
 *    contiguous planes of N = nu*nv elements of T (x plane, then y, then z);
 *    component c of control point alpha is at index c*N + alpha.
 *  - Global Hessian K (the "stencil"): 225 planes of N elements of T.  Entry
 *    (r, c) of the 3x3 block coupling alpha = (i, j) to beta = (i+du, j+dv),
 *    du, dv in [-2, 2], is at index ((slot*9) + 3*r + c)*N + alpha with
 *    slot = (dv+2)*5 + (du+2).  Blocks reaching outside the grid are zero.
 *  - Device pointers come from the caller (e.g. PyTorch tensors) and stay
 *    owned by the caller; they must be 16-byte aligned.  The context owns
 *    its quadrature tables, lumped masses, span workspace, internal K and
 *    solver vectors (allocated once in bsc_create, freed in bsc_destroy).
 *  - Every call is ordered on the context's CUDA stream.  Calls that return
 *    a host value (energy, reports) synchronise that stream.
 *  - Errors: every call returns a bsc_status; no exception or abort crosses
 *    the ABI.  bsc_last_error() gives a message for the context (or, with a
 *    NULL context, for the last failed bsc_create of this thread).
 */
#ifndef BSC_H
#define BSC_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum bsc_status {
  BSC_OK = 0,
  BSC_ERR_INVALID_ARG = 1,   /* bad size, pointer, knot vector or option */
  BSC_ERR_CUDA = 2,          /* a CUDA runtime call failed */
  BSC_ERR_OOM = 3,           /* device allocation failed in bsc_create */
  BSC_ERR_NUMERIC = 4,       /* NaN/Inf in an energy, norm or projection */
  BSC_ERR_NOT_CONVERGED = 5, /* PCG hit its iteration limit */
  BSC_ERR_LINESEARCH = 6,    /* no decrease after max_line_search halvings */
  BSC_ERR_TIMEOUT = 7        /* a bounded device-side wait ran out */
} bsc_status;

enum { BSC_FP64 = 0, BSC_FP32 = 1 };

/* Quadrature rules: the paper's reduced rules (Sec. 4.1 membrane: dual-grid
 * alternating 1x2 / 2x1 Gauss in the interior, 3x3 corner spans, 3x2 / 2x3
 * side spans; Sec. 4.2 bending: one point per boundary span centre and per
 * interior knot intersection, Fig. 3); the baseline of the paper's ablation
 * (Sec. 6.5, case A): 2x2 Gauss on every interior span for both energies,
 * with the reduced rules' boundary-span placements (BSC_QUAD_STANDARD); or
 * full per-span Gauss rules everywhere, used by tests. */
enum { BSC_QUAD_REDUCED = 0, BSC_QUAD_GAUSS2 = 2, BSC_QUAD_GAUSS3 = 3, BSC_QUAD_STANDARD = 4 };

/* PSD projection of the elastic Hessian (projected Newton, Sec. 5.1):
 * NONE  - the Hessian as it is (indefinite in compression);
 * SPAN  - each span's summed membrane + bending 27x27 Hessian replaced by
 *         V max(Lambda, 0) V^T, computed in FP64;
 * POINT - at every membrane quadrature point each FBW term's Hessian w.r.t.
 *         (f_1, f_2) (the two stretch terms and the shear term of Sec. 4.1)
 *         replaced by its PSD projection in closed form before the chain
 *         rule, the eigenanalysis FBW admits; the bending Hessian is PSD
 *         already.  Computed in the precision T of the span evaluation. */
enum { BSC_PROJECT_NONE = 0, BSC_PROJECT_SPAN = 1, BSC_PROJECT_POINT = 2 };

/* Knot grid (Sec. 3.1.2).  knots_u / knots_v may be NULL; if given they must
 * hold the open uniform integer knot vector of length nu+3 / nv+3. */
typedef struct bsc_knot_grid {
  int nu, nv;
  const double* knots_u;
  const double* knots_v;
} bsc_knot_grid;

/* FBW membrane stiffnesses mu_st1, mu_st2, mu_sh [N/m] (Eq. FBW stretching and
 * shearing energy), bending stiffness mu_bd [N m] (Eq. general bending
 * energy) and areal density rho_area [kg/m^2] for the lumped mass (Eq. lumped
 * mass matrix). */
typedef struct bsc_material {
  double mu_st1, mu_st2, mu_sh, mu_bd, rho_area;
} bsc_material;

typedef struct bsc_quadrature {
  int membrane; /* BSC_QUAD_* */
  int bending;  /* BSC_QUAD_* */
} bsc_quadrature;

typedef struct bsc_options {
  int precision;        /* BSC_FP64 or BSC_FP32: element type T of buffers and
                           of span evaluation, assembly and SpMV; the SPD
                           projection, energy sums and norms are FP64 always */
  double dt;            /* > 0: implicit Euler step (inertia M/dt^2, Sec. 3.2);
                           <= 0: static problem (no inertia; Chat ignored) */
  double gravity[3];    /* m/s^2; body force m_alpha * gravity */
  const int32_t* pinned; /* host array of Dirichlet control points (copied) */
  int n_pinned;
  int project;          /* BSC_PROJECT_*: the projection bsc_newton_step uses */
  double pcg_rel_tol;   /* PCG stops when ||r|| <= tol * ||b|| (<= 0: 1e-8) */
  int pcg_max_iter;     /* <= 0: 10000 */
  int max_line_search;  /* halvings of alpha before BSC_ERR_LINESEARCH (<= 0: 30) */
} bsc_options;

typedef struct bsc_newton_report {
  double E0;            /* incremental potential at the input C */
  double E1;            /* at the accepted C + alpha d */
  double alpha;         /* accepted step length (1, 1/2, 1/4, ...) */
  double dir_inf;       /* ||d||_inf (the paper's stopping residual is dir_inf / dt) */
  double pcg_rel_res;   /* final ||r|| / ||b|| of the linear solve */
  int pcg_iters;
  int ls_halvings;
  int status;           /* bsc_status of the step */
  int spans_projected;  /* spans whose Hessian had a negative eigenvalue
                           (BSC_PROJECT_SPAN; 0 otherwise) */
  int fcg_iters;        /* with a learned solver (bsc_set_learned_solver): the
                           flexible-CG iterations, which pcg_iters includes; 0 otherwise */
  int fell_back;        /* 1 when the learned solve stalled and block-Jacobi
                           PCG finished it */
} bsc_newton_report;

typedef struct bsc_ctx bsc_ctx;

/* Build a context for one patch: copies the rest control points, builds the
 * quadrature tables (basis values and derivatives, |det J|, dN/dX and the
 * Laplacian coefficients at every quadrature point; Sec. 4.1, Eq. deformation
 * gradient, Eq. Laplacian in parametric space) and the lumped masses on the
 * device, and allocates all workspace.
 *   g        knot grid, nu, nv >= 5
 *   rest_xy  host, (nu*nv) x 2 doubles, row-major [alpha][X1, X2]; material
 *            coordinates of the control points (Sec. 3.2); must give a
 *            regular map (det dX/d(u,v) != 0 at every quadrature point)
 *   m, q, o  see the structs above (o may not be NULL)
 *   cuda_stream  cudaStream_t for every call (NULL = legacy default stream)
 *   out      receives the context; NULL on failure. */
bsc_status bsc_create(const bsc_knot_grid* g, const double* rest_xy, const bsc_material* m,
                      const bsc_quadrature* q, const bsc_options* o, void* cuda_stream,
                      bsc_ctx** out);

/* Frees every device and host resource of the context (NULL is a no-op). */
void bsc_destroy(bsc_ctx* ctx);

/* Message of the last error of ctx; with ctx == NULL, of the last failed
 * bsc_create on this thread.  Valid until the next call on ctx. */
const char* bsc_last_error(const bsc_ctx* ctx);

/* Change the stream the context launches on (NULL = legacy default). */
bsc_status bsc_set_stream(bsc_ctx* ctx, void* cuda_stream);

/* Incremental potential (Eq. incremental_potential with the lumped mass):
 *   E(C) = sum_alpha m/(2 dt^2) |C - Chat|^2 - sum_alpha m g.C
 *          + sum_spans (membrane + bending energy at the quadrature points).
 * C_dev, Chat_dev: device, 3 planes of N (T); Chat ignored when dt <= 0.
 * E_out: host double.  Synchronises the stream. */
bsc_status bsc_energy(bsc_ctx* ctx, const void* C_dev, const void* Chat_dev, double* E_out);

/* Gradient of E(C) into g_dev (device, 3 planes of N, T); entries of pinned
 * control points are zero (Dirichlet elimination). */
bsc_status bsc_gradient(bsc_ctx* ctx, const void* C_dev, const void* Chat_dev, void* g_dev);

/* Global Hessian of E(C): sum over spans of the 27x27 span Hessian (projected
 * to PSD per project, one of BSC_PROJECT_*), gathered into the 5x5 block
 * stencil in a fixed order without atomics, plus m/dt^2 I on the diagonal;
 * rows and columns of pinned control points are replaced by the identity.
 * K_dev: device, 225 planes of N (T), or NULL to keep K inside the context.
 * The context remembers the matrix for bsc_spmv / bsc_solve.  A project
 * value outside BSC_PROJECT_* returns BSC_ERR_INVALID_ARG. */
bsc_status bsc_assemble_hessian(bsc_ctx* ctx, const void* C_dev, int project, void* K_dev);

/* y = K x with K_dev (NULL = the last matrix assembled by this context).
 * x_dev, y_dev: device, 3 planes of N (T), must not alias. */
bsc_status bsc_spmv(bsc_ctx* ctx, const void* K_dev, const void* x_dev, void* y_dev);

/* Solve K x = b with 3x3 block-Jacobi preconditioned CG (persistent
 * cooperative kernel, FP64 dot products), starting from x = 0, until
 * ||r|| <= rel_tol ||b|| or max_iter.  K_dev NULL = last assembled matrix.
 * iters / rel_res (host, may be NULL) receive the iteration count and the
 * final relative residual.  Synchronises the stream. */
bsc_status bsc_solve(bsc_ctx* ctx, const void* K_dev, const void* b_dev, void* x_dev,
                     double rel_tol, int max_iter, int* iters, double* rel_res);

/* One projected Newton iteration (Sec. 5.1): gradient g and Hessian K (span
 * projection per options.project) at C, d from K d = -g by PCG, then
 * backtracking: alpha = 1, halved until E(C + alpha d) <= E(C), and
 * C <- C + alpha d in place.  rep (host, may be NULL) receives the report.
 * Synchronises the stream. */
bsc_status bsc_newton_step(bsc_ctx* ctx, void* C_dev, const void* Chat_dev, bsc_newton_report* rep);

/* ---- batched patches: many garments in one context ------------------------
 * A context may hold several independent patches with their own grids,
 * materials, rest maps, time steps, gravity and pinned sets (the garment
 * panels of one scene).  Every entry point above then works on all patches
 * at once - one launch per phase, the PCG as one persistent cooperative
 * launch whose co-resident blocks are split into one group per patch - and
 * the patches never interact.
 *  - Layout: the patches' control points are concatenated in patch order;
 *    patch p owns entries [cp_offset[p], cp_offset[p+1]) of every plane of a
 *    control-point vector (3 planes of N = total control points) and of the
 *    225 planes of K.  Its spans likewise follow in patch order
 *    (span_offset).  Within a patch the single-patch numbering holds.
 *  - bsc_energy returns the sum of the patches' energies (added in patch
 *    order); bsc_solve solves every patch's system to rel_tol (iters =
 *    the largest count, rel_res = the largest residual); bsc_newton_step
 *    runs an independent Newton iteration with its own line search per patch
 *    and reports the aggregate (E0, E1: sums; alpha: smallest; dir_inf,
 *    pcg_rel_res, pcg_iters, ls_halvings: largest; spans_projected: sum;
 *    status: the first patch's non-OK status) - bsc_patch_reports gives the
 *    per-patch reports.
 *  - A single-patch context is the one-patch case of the same code. */

/* Build a context for `count` patches (1 <= count <= 304; more than the
 * persistent PCG's co-resident block capacity is refused).
 *   grids, materials, options: arrays of count entries (options[p].pinned
 *   holds patch-local control-point indices); precision, project,
 *   pcg_rel_tol, pcg_max_iter and max_line_search are taken from
 *   options[0];  rest_xy: count host pointers, patch p's (nu*nv) x 2 doubles;
 *   q: the quadrature rules of every patch.  Other arguments as bsc_create. */
bsc_status bsc_create_batch(int count, const bsc_knot_grid* grids, const double* const* rest_xy,
                            const bsc_material* materials, const bsc_quadrature* q,
                            const bsc_options* options, void* cuda_stream, bsc_ctx** out);

/* Patch count and offsets (host arrays of count + 1 ints, either may be NULL). */
bsc_status bsc_batch_layout(const bsc_ctx* ctx, int* count, int* cp_offset, int* span_offset);

/* Per-patch reports of the last bsc_newton_step (host array of count). */
bsc_status bsc_patch_reports(const bsc_ctx* ctx, bsc_newton_report* reps);

/* Per-patch incremental potential (host array of count doubles). */
bsc_status bsc_patch_energies(bsc_ctx* ctx, const void* C_dev, const void* Chat_dev, double* E_out);

/* Autotuner.  Span evaluation runs on work items - a patch and either a run
 * of consecutive spans or a tile of tile_tu x (block / tile_tu) spans - with
 * one tile width per patch-size class (class k: spans per row < 32, < 64,
 * < 128, >= 128); width 0 means runs.  bsc_autotune times the Hessian
 * evaluation of each class present for each candidate width {0, 8, 16, 32}
 * (CUDA events, best of 3) and keeps the fastest, times the SPD projection
 * (interior and border spans together) with each of the three paths of
 * the border spans (at or next to a patch border) and keeps the fastest, likewise the two occupancy variants of the interior
 * projection's eigenpair phase, then assembles K at C,
 * runs one PCG solve per patch to measure its iteration count, and splits
 * the PCG's co-resident blocks in proportion to control points x
 * iterations (bsc_plan_blocks).  C is not modified.  The choices change
 * only the launch shape and the PCG's reduction grouping, not what is
 * computed: span terms and K are bitwise the same for every tile width.
 * out (host, may be NULL) receives the choices and timings. */
typedef struct bsc_tuning {
  int tile_tu[4];          /* chosen width per class (-1: class absent) */
  double tile_ms[4][4];    /* measured ms per class x candidate {0, 8, 16, 32} */
  int pcg_grid;            /* co-resident blocks of the persistent PCG */
  int border_path;         /* SPD projection of the border spans: 0 one warp per
                              span, 1 one thread per span, 2 one warp per span
                              to the tridiagonal form, then one thread per
                              eigenpair, 3 one warp per span for the PSD test,
                              then one warp per failing span (chosen by time) */
  double border_ms[4];     /* measured ms of the whole projection per border path */
  int p2_variant;          /* phase 2 of the interior projection: 0 two, 1 three
                              resident blocks per SM (fewer registers; chosen by time) */
  double p2_ms[2];         /* measured ms of that phase per variant */
  int pcg_grid_cand[4];    /* PCG grids tried: a block per two SMs, one and two
                              per SM, a thread per control point (each clamped
                              to [patches, usable blocks]) */
  double pcg_ms[4];        /* measured ms of the solve per candidate (-1: duplicate) */
  int pcg_form;            /* PCG form chosen at that grid (see bsc_set_pcg_form) */
  double pcg_form_ms[3];   /* measured ms of the solve per form (1e30: did not converge) */
  int psd_test;            /* PSD test mode before the interior eigendecomposition (bsc_set_psd_test) */
  double psd_ms[3];        /* measured ms of the whole projection in modes 0, 1, 2 */
} bsc_tuning;
bsc_status bsc_autotune(bsc_ctx* ctx, const void* C_dev, const void* Chat_dev, bsc_tuning* out);

/* Replace patch p's material (stiffnesses and density; the lumped masses
 * are recomputed when the density changes).  Ordered on the context's
 * stream; synchronises it.  Captured Newton graphs stay valid. */
bsc_status bsc_set_material(bsc_ctx* ctx, int patch, const bsc_material* m);

/* Set the grid of the persistent PCG by hand: grid in [number of patches,
 * usable blocks] (usable: the co-resident capacity, at most one block per 256
 * control points of each patch; BSC_ERR_INVALID_ARG otherwise); the blocks
 * are split over the patches by the current work estimates.  Results are
 * independent of the grid up to the order of the FP64 reductions. */
bsc_status bsc_set_pcg_grid(bsc_ctx* ctx, int grid);

/* Set the tile widths by hand (4 entries, each 0, 8, 16 or 32). */
bsc_status bsc_set_tiles(bsc_ctx* ctx, const int* tile_tu);

/* Set the border projection path by hand (0, 1, 2 or 3, see bsc_tuning); all
 * compute the same projection up to rounding. */
bsc_status bsc_set_border_path(bsc_ctx* ctx, int path);

/* Set the occupancy variant of the interior projection's eigenpair phase by
 * hand (0 or 1, see bsc_tuning); both compute bitwise the same result. */
bsc_status bsc_set_p2_variant(bsc_ctx* ctx, int variant);

/* PSD test of the SPD projection (BSC_PROJECT_SPAN), mode:
 * 0 - every interior span goes through the eigendecomposition;
 * 1 - every interior span's reduced Hessian H_r (order n) first goes
 *     through an FP64 LDL^T factorisation of H_r + tau I, tau = 1e-14
 *     tr(H_r) / n (a span with tr(H_r) <= 0 fails outright); a span whose
 *     pivots are all positive has no eigenvalue below -tau and keeps its
 *     Hessian, and only the spans that fail go on to the eigendecomposition
 *     (gathered into one list, so that it runs with full warps);
 * 2 (the default) - before that, an FP32 certificate: H_r formed and
 *     Cholesky-factored in FP32 with a shift sigma that bounds the rounding
 *     of both (a few 1e-6 of tr(H_r) and of the size of H_r's terms); a
 *     factorisation that completes proves H_r positive definite with every
 *     eigenvalue above sigma / 2, so the span keeps its Hessian without the
 *     FP64 test, which would have passed it too.  Only the spans the
 *     certificate leaves open go through the FP64 test.
 * The border spans (order 24) are tested too whenever the mode is not 0:
 * the warp-per-span paths (bsc_set_border_path 0, 2, 3) form H_r with one
 * column per lane and, in mode 2, certify in FP32 first (the same argument
 * with n = 24), then run the FP64 test; path 1 runs the FP64 test alone.
 * The "FP64 test" of the thread-per-span kernels runs in double-float when
 * bsc_set_proj_arith selects it (the default of FP32 contexts).
 * The projected matrix is the same in modes 1 and 2 bit for bit, and the
 * same as in mode 0 up to eigenvalues of size tau.  bsc_autotune keeps the
 * fastest mode for the state it is given.  Errors: BSC_ERR_INVALID_ARG for
 * another mode. */
bsc_status bsc_set_psd_test(bsc_ctx* ctx, int mode);

/* Arithmetic of the projection's PSD test and of its phase 1 (formation of
 * the reduced Hessian, Householder tridiagonal form) on the thread-per-span
 * kernels: 0 FP64; 1 double-float, pairs of FP32 numbers with about 48
 * significant bits, which GB300's FP32 pipe runs several times faster than
 * its FP64 pipe runs FP64 (backward errors about 2^-47 ||H_r|| instead of
 * 2^-53, so eigenvalues are projected below -1e-12 ||T|| instead of -1e-14;
 * the eigenpair phase stays FP64).  Default: 1 in FP32 contexts, 0 in
 * FP64 contexts (Sec. 5.1 projection, unchanged up to rounding).  Errors:
 * BSC_ERR_INVALID_ARG for another mode. */
bsc_status bsc_set_proj_arith(bsc_ctx* ctx, int mode);

/* Span counts of the last projection (host array of 6 ints): the interior
 * spans, those the FP64 PSD test ran on (all of them in mode 1, the
 * certificate's open ones in mode 2, none in mode 0), those that went on to
 * the eigendecomposition; the border spans, those of them that went on to
 * the eigendecomposition (all of them with the PSD test off), and those the
 * FP64 test ran on (in mode 2 on the warp border paths 0, 2 and 3 the ones
 * the warp's FP32 certificate left open; all of them in mode 1 or on border
 * path 1, read under the current border path; none in mode 0). */
bsc_status bsc_psd_counts(bsc_ctx* ctx, int* out);

/* Form of the persistent block-Jacobi PCG (the same iterates up to rounding):
 * 0 - the textbook recurrences, three group barriers per iteration (one
 *     per reduction, one before the product reads the new direction);
 * 1 - the pipelined recurrences of Ghysels & Vanroose (2014), which carry
 *     K u and M K u so that an iteration's three dot products form in one
 *     pass behind a single group barrier, at the cost of six more vectors
 *     and a recursively updated residual that drifts a little further from
 *     b - K x;
 * 2 - two passes and two group barriers per iteration: since K p = K z +
 *     beta K p_old, the product pass forms K z and updates q = K z + beta q
 *     and p = z + beta p in place, and the direction needs no pass of its
 *     own (q is carried by a recurrence, like r).
 * bsc_autotune picks the fastest form that reaches the tolerance; the
 * default is 0. */
bsc_status bsc_set_pcg_form(bsc_ctx* ctx, int form);

/* Layout of the matrix the Newton step assembles and its block-Jacobi PCG
 * reads (bsc_newton_step, bsc_autotune): symmetric != 0 (the default) keeps
 * only the diagonal block and the 12 blocks that couple a control point to
 * the neighbours after it (dv > 0, or dv = 0 and du > 0) - 13 slots, plane
 * (s' * 9 + 3 r + c) with s' = stencil slot - 12 - and reads each block
 * before a row as the transpose of the neighbour's (K is symmetric: the
 * gathers of (alpha, beta) and (beta, alpha) add the same span entries in the
 * same order).  The product accumulates the same entries in the same order
 * as with the full 25 slots, so both layouts give the same Newton step bit
 * for bit, with half the matrix bytes to write and to stream per PCG
 * iteration.  The learned solver always uses the full layout.  After a
 * Newton step, bsc_spmv and bsc_solve with K_dev NULL use its matrix in
 * whichever layout it has; bsc_assemble_hessian always writes the full one. */
bsc_status bsc_set_k_storage(bsc_ctx* ctx, int symmetric);

/* Current split of the PCG's blocks (host array of count ints). */
bsc_status bsc_pcg_split(const bsc_ctx* ctx, int* blocks_per_patch);

/* The split rule itself, a pure host function: `total` blocks over `count`
 * patches with n_cp[p] control points and work estimates work[p] > 0; each
 * patch gets >= 1 and <= ceil(n_cp / 256) blocks, the rest go one at a time
 * to the patch with the largest work / blocks (ties to the lower index).
 * Writes blocks[count]; returns the number handed out, -1 if total < count. */
int bsc_plan_blocks(int count, const int* n_cp, const double* work, int total, int* blocks);

/* CUDA graph of the Newton iteration.  With on != 0 (the default)
 * bsc_newton_step captures its launches - evaluation, projection, assembly,
 * the persistent PCG and the first line-search round - into a CUDA graph
 * the first time it sees a pair (C_dev, Chat_dev) and replays the graph for
 * later calls with the same pointers; further line-search rounds, needed
 * only by patches that reject alpha = 1, are launched directly.  The graph
 * runs on an internal stream that is ordered after, and before, the
 * context's stream.  bsc_graph_state (host ints, may be NULL): on = the
 * setting, captured = 1 while an executable graph is held, replays = graph
 * launches so far. */
bsc_status bsc_set_graph(bsc_ctx* ctx, int on);
bsc_status bsc_graph_state(const bsc_ctx* ctx, int* on, int* captured, long long* replays);

/* ---- learned preconditioner and flexible CG -------------------------------
 * A 4-layer 3x3 convolutional network on the control grid of a single-patch
 * FP32 context (channels 32 -> 32 -> 32 -> 32 -> 16, ReLU after the first
 * three layers, zero padding), BF16 weights and activations with FP32
 * accumulation on the tensor cores.  It reads the matrix and writes a local
 * linear preconditioner:
 *   features per control point alpha (32): the diagonal block K_aa / d
 *     (entries 00 01 02 11 12 22), the traces of the 24 off-diagonal blocks
 *     / d in slot order, the pin mask and 1 (d = mean diagonal entry of K
 *     over unpinned points);
 *   output channels 0..8 (o_t): tap coefficients a_t(alpha) = o_t / (2 (1 +
 *     sum_s |o_s|)), t = 3 (dy + 1) + (dx + 1) for the neighbour (i + dx,
 *     j + dy) - sum_t |a_t| < 1/2, so cond(B^T B) <= 9 for any weights;
 *   M = P L^-T B^T B L^-1 P,  D_aa = L_a L_a^T (Cholesky of each diagonal
 *     block), (B y)(alpha) = y(alpha) + sum_t a_t(alpha) y(alpha + off_t) for
 *     each component (zero outside the grid), P zeroing pinned entries.
 * M is symmetric positive semidefinite for any weights, and all-zero weights
 * give the block-Jacobi preconditioner.  The network runs once per matrix
 * (bsc_cnn_prepare); each application of M costs two 9-tap stencils and two
 * block triangular solves per control point.
 * Parameters (FP32, bsc_cnn_param_count() of them) in layer order; per layer
 * the weights W[dy][dx][c_in][c_out] (dy, dx in {-1, 0, 1}, the offset of
 * the input pixel (i + dx, j + dy)) then the bias [c_out].
 * Training minimises the energy-norm error of the preconditioned vector of
 * pairs (r = K x, x),
 *   L = (M r - x)^T K (M r - x) / (x^T K x),
 * with Adam on the FP32 master parameters.  Errors go to bsc_last_error(ctx). */
typedef struct bsc_cnn bsc_cnn;
typedef struct bsc_fcg_report {
  int fcg_iters;        /* flexible-CG iterations */
  int pcg_iters;        /* plain PCG iterations after a stall (fallback) */
  int fell_back;        /* 1 when the flexible CG stalled and PCG finished the solve */
  double rel_res;       /* final ||b - K x|| / ||b|| (recursive residual) */
} bsc_fcg_report;

int bsc_cnn_param_count(void);
bsc_status bsc_cnn_create(bsc_ctx* ctx, bsc_cnn** out);   /* all parameters zero */
void bsc_cnn_destroy(bsc_cnn* cnn);
/* host FP32 parameters in; which = 0 parameters / 1 the last gradient out */
bsc_status bsc_cnn_set_params(bsc_cnn* cnn, const float* params, int count);
bsc_status bsc_cnn_get_params(bsc_cnn* cnn, float* out, int count, int which);
/* binds the network to a matrix K_dev (stencil layout): features, block
 * Cholesky factors, and one forward pass of the network */
bsc_status bsc_cnn_prepare(bsc_cnn* cnn, const void* K_dev);
/* z_dev = M r_dev for the prepared matrix (3 planes of N, FP32) */
bsc_status bsc_cnn_apply(bsc_cnn* cnn, const void* r_dev, void* z_dev);
/* loss L at the pair (r, x) (r = K x) with the current weights (the network
 * is re-run on the prepared matrix) and its gradient (kept on the device for
 * the optimizer) */
bsc_status bsc_cnn_loss_grad(bsc_cnn* cnn, const void* r_dev, const void* xstar_dev, double* loss);
bsc_status bsc_cnn_adam_step(bsc_cnn* cnn, double lr, double beta1, double beta2, double eps);
/* activations of the last forward pass as host FP32 [N][channels]: which = 0
 * features (32), 1..3 layer outputs (32), 4 network output (16: o_0..o_8 and 7 unused) */
bsc_status bsc_cnn_activations(bsc_cnn* cnn, int which, float* out);
/* Solve K x = b (x from 0) by flexible CG with z = M r (the call prepares the network on K_dev):
 *   q = K p, a = p.r / p.q, x += a p, r -= a q, z = M r, b = -z.q / p.q, p = z + b p,
 * until ||r|| <= rel_tol ||b||; when r.r has not dropped by 4x in 24
 * iterations (or a curvature p.q <= 0 appears) plain block-Jacobi PCG finishes
 * the solve from the current x. */
bsc_status bsc_solve_fcg(bsc_ctx* ctx, bsc_cnn* cnn, const void* K_dev, const void* b_dev, void* x_dev,
                         double rel_tol, int max_iter, bsc_fcg_report* rep);

/* Linear solver of bsc_newton_step.  With cnn != NULL (a network created on
 * this single-patch FP32 context) every Newton step solves K d = -g by the
 * flexible CG of bsc_solve_fcg - the network runs once on the step's K, the
 * flexible CG iterates with z = M r, and block-Jacobi PCG finishes the solve
 * from the current iterate when it stalls - to the same relative residual
 * (options.pcg_rel_tol), inside the step's CUDA graph.  cnn == NULL returns
 * to plain block-Jacobi PCG.  The report's pcg_iters then counts both
 * solvers' iterations, fcg_iters the flexible CG's, fell_back the fallback.
 * This is the learned preconditioner on the Newton path of Sec. 5.1 (the
 * paper solves with a direct Cholesky factorisation instead).  Destroying the
 * network detaches it. */
bsc_status bsc_set_learned_solver(bsc_ctx* ctx, bsc_cnn* cnn);

/* Stall window of the flexible CG (iterations in which r.r must drop by 4x
 * before the solve falls back to PCG; default 24, range [1, 100000]). */
bsc_status bsc_cnn_set_stall_window(bsc_cnn* cnn, int window);

/* Bounded device waits of the context's persistent solvers (the group
 * barriers of the PCG and of the learned flexible CG): spins = sleeps of
 * about 64 ns before a barrier gives up, raises BSC_ERR_TIMEOUT and returns
 * (default 2^25, about 2 s; range [1, 2^40]).  extra_blocks (0 or 1) makes
 * every barrier wait for that many blocks beyond those launched, so that no
 * barrier can complete: a test hook for the timeout path, which needs no
 * fault.  Normal use leaves it 0.  The solvers' results are undefined after a
 * timeout; the context stays usable. */
bsc_status bsc_set_wait_limit(bsc_ctx* ctx, long long spins, int extra_blocks);

/* ---- contact with a static obstacle (Sec. 4.3) ----------------------------
 * A triangle mesh embedded in the B-spline surface of a single-patch context
 * meets a static obstacle triangle mesh through the log barrier of
 * incremental potential contact.
 *  - Contact mesh: mu x mv vertices at parametric points u_i = S_u i /
 *    (mu - 1), v_j = S_v j / (mv - 1) (vertex k = j mu + i), each moving with
 *    the nine control points of its span, x_k = sum_l N_l(u, v) C_l (Eq. trig
 *    mesh node from control points); cells split into two triangles along
 *    alternating diagonals; weight A_k = a third of the rest areas of its
 *    triangles.  mu, mv <= 0 choose about twice the control points in all
 *    (sqrt(2) (n - 1) + 1 per side).
 *  - Potential: kappa sum_k A_k sum beta(d / dhat), beta(x) = -(x - 1)^2 ln x
 *    for 0 < x < 1, over the (vertex, obstacle triangle) pairs closer than
 *    dhat [m]; a pair whose closest point lies on an edge or a corner counts
 *    once, for the lowest-index triangle holding that feature.  kappa [Pa].
 *  - Every energy, gradient and Hessian of the context then includes it:
 *    per pair the gradient and the PSD projection of the Hessian w.r.t. the
 *    vertex (kappa A beta'' / dhat^2 u u^T, u the unit vector from the
 *    closest point), chained onto the span's control points (Eq. gradient and
 *    hessian of contact barrier) and gathered into the stencil with the
 *    elastic terms (after their projection).
 *  - bsc_newton_step starts its line search at min(1, step bound): the
 *    largest step that keeps every vertex at least 0.1 of its distance from
 *    every obstacle triangle it could reach, from the convexity of the
 *    distance along the step.
 *  - No self-contact of the cloth, no edge-edge or obstacle-vertex-cloth-
 *    triangle pairs, no friction.
 *   obs_xyz  host, n_obs_vertices x 3 doubles [m];  obs_tris  host,
 *            n_obs_tris x 3 vertex indices (distinct, in range).
 * Copies everything; BSC_ERR_INVALID_ARG on bad input; replaces an earlier
 * obstacle.  Drops the captured Newton graph. */
bsc_status bsc_contact_attach(bsc_ctx* ctx, const double* obs_xyz, int n_obs_vertices, const int32_t* obs_tris,
                              int n_obs_tris, int mu, int mv, double dhat, double kappa);
bsc_status bsc_contact_detach(bsc_ctx* ctx);
/* Contact-mesh vertex positions at C (host, nvert x 3 doubles; cap >= nvert),
 * or only the count with x_out == NULL. */
bsc_status bsc_contact_vertices(bsc_ctx* ctx, const void* C_dev, double* x_out, int cap, int* nvert);
/* The line search's step bound of direction D_dev (3 planes of N) from C_dev. */
bsc_status bsc_contact_step_bound(bsc_ctx* ctx, const void* C_dev, const void* D_dev, double* alpha);
/* Contact-mesh vertex count and pairs counted by the last evaluation. */
bsc_status bsc_contact_stats(bsc_ctx* ctx, int* nvert, int* npairs);

/* ---- inspection entry points (parity tests, profiling) ------------------- */

/* Per-span results of the last evaluation path: E_span (device, Nsp doubles),
 * g_span (device, Nsp x 27 T, row-major [span][3*l + c]) and H_span (device,
 * Nsp x 27 x 27 T, row-major) at C, projected per project (BSC_PROJECT_*).  Span
 * s = b*(nu-2) + a; local control point l = lj*3 + li.  Any output may be
 * NULL. */
bsc_status bsc_span_terms(bsc_ctx* ctx, const void* C_dev, int project, double* E_span,
                          void* g_span, void* H_span);

/* Quadrature tables, copied to host in FP64.  which = 0 membrane, 1 bending.
 * Returns the point count through count; if out != NULL writes up to cap
 * records of 25 doubles: [u, v, w, owner_a, owner_b, W = w |det J|, then for
 * membrane g[9][2] = dN_l/dX_beta (18 values), for bending L[9] (the
 * Laplacian coefficient of each control point, 9 values)], zero padded,
 * and record[24] = the owning span's context-wide index (owner_a, owner_b
 * are patch-local). */
bsc_status bsc_quadrature_tables(bsc_ctx* ctx, int which, double* out, int cap, int* count);

/* Lumped masses m_alpha (host, N doubles). */
bsc_status bsc_lumped_mass(bsc_ctx* ctx, double* m_out);

/* Sizes: N control points, Nsp spans, membrane / bending point counts. */
bsc_status bsc_sizes(const bsc_ctx* ctx, int* n_cp, int* n_spans, int* n_mem, int* n_bend);

/* Phase timing of bsc_newton_step.  With on != 0 the step records CUDA
 * events on the context's stream at its phase boundaries; bsc_phase_times
 * (synchronising) writes the durations of the last step in ms to ms_out[6]:
 * [span evaluation, SPD projection, energy + gradient + assembly, linear
 * solve, line search, whole step]. */
bsc_status bsc_set_profiling(bsc_ctx* ctx, int on);
bsc_status bsc_phase_times(bsc_ctx* ctx, double* ms_out);

/* Number of CUDA kernels this context has launched since bsc_create. */
bsc_status bsc_launch_count(const bsc_ctx* ctx, unsigned long long* launches);

/* Per-span statistics of the last SPD projection (host arrays of Nsp ints,
 * either may be NULL): nneg = eigenvalues projected away, nred = dimension
 * of the span's reduced eigenproblem: 15 for interior spans (3 x the rank
 * of their five derivative vectors), 24 for spans at or next to the border
 * (the 3 x 8 mean-free subspace). */
bsc_status bsc_projection_stats(bsc_ctx* ctx, int* nneg, int* nred);

/* ---- solve without device allocation ----------------------------------------
 * The paper has no counterpart of this entry point.
 *
 * Same preconditioned CG as bsc_solve, for callers that cannot allocate
 * device memory themselves: host code whose memory manager owns all of the
 * device memory and forbids cudaMalloc, or a loop that cannot afford the
 * device-wide synchronisation cudaMalloc / cudaFree bring.  It needs no
 * context: K_dev (225 planes of nu*nv, the stencil layout above), b_dev and
 * x_dev (3 planes each) are the caller's device buffers of the element type
 * given by precision; nothing is allocated.  The working set (block-Jacobi
 * inverses, CG vectors, reductions, barrier words) lives in one fixed
 * file-scope device array sized for BSC_STATIC_SOLVE_MAX_CP control points
 * (about 2.8 MB, held on every device that loads the library until the
 * process exits); larger grids return BSC_ERR_INVALID_ARG with a message.
 *   - The first call on a device looks up the array's device address (with
 *     that device current) and caches it; make that first call before any
 *     stream capture on the device.
 *   - Every call on a device uses the same array and leaves its contents
 *     behind (the barrier words are cleared at the start of each call).  Calls
 *     that may overlap on the GPU - issued on two streams, or from two host
 *     threads driving the same device - race and must be serialised by the
 *     caller.
 *   - The call synchronises cuda_stream (NULL = legacy default stream) to
 *     read back iters / rel_res (host, may be NULL).  Errors: the status, and
 *     a message through bsc_last_error(NULL). */
#define BSC_STATIC_SOLVE_MAX_CP 16384
bsc_status bsc_solve_static(int nu, int nv, int precision, const void* K_dev, const void* b_dev, void* x_dev,
                            double rel_tol, int max_iter, void* cuda_stream, int* iters, double* rel_res);

/* ---- strip decomposition of one patch over ranks ----------------------------
 * A patch too large for one GPU splits into strips of whole control-point
 * rows (v direction), one per rank.  Rank r owns the rows [own0, own1) and
 * holds a window of them plus two halo rows on each side (clipped to the
 * grid): rows [row0, row1), row0 = own0 - min(2, own0), row1 = own1 +
 * min(2, nv - own1).  The spans touching an owned row (span b covers rows
 * b .. b + 2) all lie in the window, so with the halo rows of C current the
 * window's gradient and Hessian rows of its owned rows are exactly the
 * patch's, bit for bit (same spans, same gather order).  A span belongs to
 * the rank owning its middle row b + 1.
 *
 * One Newton iteration then needs these exchanges between neighbouring
 * ranks: the halo rows of the search direction p before every product
 * y = K p (the product reads p two rows beyond the owned ones), the halo rows
 * of the solution d before the line search, and sums over ranks of per-row
 * partial sums (the PCG's dot products, the energy of a trial point).  The
 * calls below return those partial sums one per owned row, each computed
 * from that row alone in a fixed order; adding them up in the global row
 * order (after an all-gather) gives every decomposition of a patch - one
 * window of all rows included - the same sums bit for bit.  The exchanges
 * and the all-gather are the caller's (host copies, NCCL, gloo ...): no
 * kernel here waits for another rank. */
typedef struct {
  int row0, row1;  /* global control-point rows held: [row0, row1) */
  int own0, own1;  /* global rows owned: [own0, own1), own0 < own1 */
} bsc_window;

/* Context of one strip window of the patch (g, rest_xy, m, q, o as for
 * bsc_create, describing the WHOLE patch; the pinned list holds whole-patch
 * indices).  Vectors of the window (C, Chat, g, d, ...) are 3 planes of
 * nu * (row1 - row0) values, local row k being global row row0 + k; K holds
 * 225 planes of that length.  Every single-patch call works on it
 * (bsc_gradient, bsc_assemble_hessian, bsc_spmv: rows outside [own0, own1)
 * hold partial sums and are to be ignored; bsc_energy: the owned span rows'
 * and owned control points' share of the incremental potential), except the
 * ones that solve over the whole window (bsc_newton_step, bsc_solve,
 * bsc_autotune) and contact, which return BSC_ERR_INVALID_ARG.
 * Errors: BSC_ERR_INVALID_ARG for a window other than the one defined above
 * or fewer than 3 rows, otherwise as bsc_create. */
bsc_status bsc_create_window(const bsc_knot_grid* g, const double* rest_xy, const bsc_material* m,
                             const bsc_quadrature* q, const bsc_options* o, const bsc_window* w,
                             void* cuda_stream, bsc_ctx** out);

/* Per-row partial sums of the incremental potential at C (Eq. incremental
 * potential): out[0 .. ns) the energies of the owned span rows (global
 * rows max(own0 - 1, 0) .. min(own1 - 1, nv - 2) - 1, each the sum of its
 * spans' energies), then out[ns .. ns + (own1 - own0)) the inertia and
 * gravity terms of the owned control-point rows.  *count = ns + own1 - own0;
 * cap is out's length (out may be NULL to query the count).  Synchronises
 * the context's stream. */
bsc_status bsc_window_energy_rows(bsc_ctx* ctx, const void* C_dev, const void* Chat_dev, double* out, int cap,
                                  int* count);

/* Block-Jacobi PCG of K d = -g over the ranks, one step at a time (Sec. 5.1
 * solve; the iteration of bsc_solve with the reductions left to the caller).
 * x_dev, p_dev: caller-owned window vectors (3 planes) that hold the solution
 * and the search direction from bsc_window_pcg_begin to the end of the solve;
 * the caller fills p's halo rows from the neighbours (their owned rows)
 * before each bsc_window_pcg_product, and reads x's owned rows at the end.
 * Each call works on the owned rows only and writes per-owned-row partial
 * sums to rows (host, n = own1 - own0 per quantity), then synchronises the
 * context's stream.
 *   begin:     block-Jacobi inverses of K; x = 0, r = -g, z = M^-1 r, p = z;
 *              rows[0..n) = r.z, rows[n..2n) = r.r
 *   product:   q = K p; rows[0..n) = p.q
 *   update:    x += alpha p, r -= alpha q, z = M^-1 r; rows = r.z, then r.r
 *   direction: p = z + beta p (no sums)
 * With rz, pq, rr the sums over all rows: alpha = rz / pq, beta = rz_new /
 * rz; stop when rr <= tol^2 rr_0.  K_dev is the window's assembled Hessian
 * (bsc_assemble_hessian). */
bsc_status bsc_window_pcg_begin(bsc_ctx* ctx, const void* K_dev, const void* g_dev, void* x_dev, void* p_dev,
                                double* rows);
bsc_status bsc_window_pcg_product(bsc_ctx* ctx, const void* K_dev, double* rows);
bsc_status bsc_window_pcg_update(bsc_ctx* ctx, double alpha, double* rows);
bsc_status bsc_window_pcg_direction(bsc_ctx* ctx, double beta);

/* out = a + alpha d over all of the context's vector entries (3 planes of
 * N): the trial point C + alpha d of a line search.  Device pointers of the
 * context's element type; out may alias a. */
bsc_status bsc_axpy(bsc_ctx* ctx, const void* a_dev, const void* d_dev, double alpha, void* out_dev);

#ifdef __cplusplus
}
#endif
#endif /* BSC_H */

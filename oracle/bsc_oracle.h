/*
 * Plain FP64 CPU oracle for quadratic B-spline cloth FEM (Efficient B-Spline
 * Finite Elements for Cloth Simulation, arXiv 2506.18867).
 *
 * TEST INFRASTRUCTURE ONLY.  Only the test suite, the smoke check and the
 * bench's CPU-baseline leg may load this library.  It shares no code with
 * the CUDA path; the two meet only on the seeded inputs.
 *
 * Conventions (all arrays are caller-owned host memory):
 *   - nu x nv control points, open uniform quadratic knots (0,0,0,1,..,S,S,S),
 *     S = n - 2 spans per axis; control point alpha = j*nu + i.
 *   - rest: double[nu*nv][2]; C, Chat, gradients: double[nu*nv][3].
 *   - span s = b*Su + a covers [a,a+1]x[b,b+1]; its 9 control points are
 *     local l = lj*3 + li (global (a+li, b+lj)); span DOF 3*l + c.
 *   - stencil Hessian: K[alpha][slot][3][3], slot = (dv+2)*5 + (du+2) couples
 *     alpha = (i,j) with beta = (i+du, j+dv); blocks outside the grid are 0.
 */
#ifndef BSC_ORACLE_H
#define BSC_ORACLE_H

#ifdef __cplusplus
extern "C" {
#endif

/* Quadrature rules: the reduced rules of Sec. 4.1 / 4.2 (Fig. 3); 2x2 or
 * 3x3 Gauss on every span; or the ablation baseline of Sec. 6.5 (case A):
 * 2x2 Gauss on interior spans for both energies, the reduced rules'
 * placements on the boundary spans. */
enum { OR_RULE_REDUCED = 0, OR_RULE_GAUSS2 = 2, OR_RULE_GAUSS3 = 3, OR_RULE_STANDARD = 4 };

typedef struct {
  int nu, nv;
  const double* rest;
  double mu_st1, mu_st2, mu_sh, mu_bd, rho;
  int mem_rule, bend_rule;
} or_problem;

typedef struct {
  double dt;            /* > 0: implicit Euler inertia term; <= 0: static problem */
  double gravity[3];
  const int* pinned;    /* control-point indices fixed by Dirichlet conditions */
  int n_pinned;
  int project;          /* OR_PROJECT_*: PSD projection of the elastic Hessian */
} or_scene;

/* Projection of the elastic Hessian (projected Newton, Sec. 5.1): none; per
 * span (eigenvalues of the summed 27x27 span Hessian clamped at 0); or per
 * membrane point and FBW term (Sec. 4.1: each stretch term's and the shear
 * term's Hessian w.r.t. (f_1, f_2) clamped separately before the chain rule). */
enum { OR_PROJECT_NONE = 0, OR_PROJECT_SPAN = 1, OR_PROJECT_POINT = 2 };

/* Quadrature points (Sec. 4.1 reduced membrane rule, Sec. 4.2 one-point
 * bending rule, Fig. 3).  which = 0 membrane, 1 bending.  Record layout:
 * [u, v, w, owner_a, owner_b].  Returns the count; writes at most cap. */
int or_quad_points(const or_problem* p, int which, double* out, int cap);

/* Per-point geometric tables.  Membrane record (20 doubles):
 *   [W = w|det J|, g[9][2]] with g_{l,beta} = dN_l/dX_beta.
 * Bending record (16 doubles):
 *   [W, L[9], c_uu, c_vv, c_u, c_v, c_uv, |det J|] with L_l the coefficient
 *   of C_l in the Laplacian of Eq. (Laplacian in parametric space). */
int or_point_tables(const or_problem* p, int which, double* out, int cap);

/* Tensor-product basis at (u, v) evaluated in owner span (a, b): 9 values of
 * N, N_u, N_v, N_uu, N_uv, N_vv (out[6][9]). */
void or_basis9(const or_problem* p, double u, double v, int a, int b, double* out);

/* Lumped mass m_alpha = rho * int N_alpha dX (Eq. lumped mass matrix). */
void or_lumped_mass(const or_problem* p, double* m);

/* Elastic (membrane + bending) energy, gradient and Hessian per span.
 * E_span[Nsp], g_span[Nsp][27], H_span[Nsp][27][27] (each may be NULL). */
void or_span_eval(const or_problem* p, const double* C, double* E_span,
                  double* g_span, double* H_span);

/* d^2 Psi / d f d f of the FBW density at one point (Sec. 4.1), f6 = (f_1,
 * f_2), A6 row-major 6x6 with index 3 beta + c, with the material of p; with
 * ptproj each term's Hessian is projected to PSD before they are summed. */
void or_fbw_hessian6(const or_problem* p, const double* f6, int ptproj, double* A6);

/* or_span_eval with the Hessian projected per project (OR_PROJECT_*). */
void or_span_eval_projected(const or_problem* p, const double* C, int project, double* E_span,
                            double* g_span, double* H_span);

/* Span terms of selected spans only (same definitions as or_span_eval):
 * E[n], g[n][27], H[n][27][27] for spans[0..n); H projected per project
 * (OR_PROJECT_*). */
void or_span_terms_subset(const or_problem* p, const double* C, int n, const int* spans, int project,
                          double* E, double* g, double* H);

/* Gradient entries g[n][3] and stencil rows K[n][25][3][3] of selected
 * control points (same definition as or_eval). */
void or_eval_rows(const or_problem* p, const or_scene* sc, const double* C, const double* Chat, int n,
                  const int* rows, double* g, double* K);

/* PSD projection of one symmetric n x n matrix: V max(Lambda, 0) V^T, with
 * the eigensystem from cyclic Jacobi.  Returns the number of sweeps. */
int or_project_psd(int n, const double* H, double* P, double* eig_out);

/* Incremental potential (Eq. incremental_potential) with lumped mass,
 * gravity and Dirichlet conditions: energy, gradient and the stencil
 * Hessian (K may be NULL; grad may be NULL). */
double or_eval(const or_problem* p, const or_scene* sc, const double* C,
               const double* Chat, double* grad, double* K);

/* Energy only. */
double or_energy(const or_problem* p, const or_scene* sc, const double* C,
                 const double* Chat);

/* y = K x with the stencil Hessian. */
void or_stencil_matvec(int nu, int nv, const double* K, const double* x, double* y);

/* Solve K x = b: banded Cholesky (exact up to rounding).  Returns 0 on
 * success, -1 if K is not positive definite. */
int or_solve_banded(int nu, int nv, const double* K, const double* b, double* x);

/* Solve K x = b by 3x3 block-Jacobi preconditioned CG to rel_tol.  Returns
 * the iteration count (negative if not converged). */
int or_solve_pcg(int nu, int nv, const double* K, const double* b, double* x,
                 double rel_tol, int max_iter);

typedef struct {
  double E0, E1, alpha, dir_inf, grad_inf;
  int ls_halvings, solver_iters, status;
} or_newton_report;

/* One projected Newton iteration with backtracking line search (Sec. 5.1):
 * solve K d = -g, alpha = 1, halve until E(C + alpha d) <= E(C) (at most
 * max_halvings), then C += alpha d.  solver: 0 banded Cholesky, 1 PCG. */
int or_newton_step(const or_problem* p, const or_scene* sc, double* C,
                   const double* Chat, int solver, double pcg_tol,
                   int max_halvings, or_newton_report* rep);

/* The backtracking line search of or_newton_step on its own, along a given
 * direction dC from C (energy E0): C <- C + alpha dC for the first alpha in
 * 1, 1/2, ... with E(C + alpha dC) <= E0 (returns 0), or C unchanged and -3
 * after max_halvings halvings.  Ct: workspace of 3N doubles. */
int or_line_search(const or_problem* p, const or_scene* sc, double* C, const double* Chat, const double* dC,
                   double E0, int max_halvings, double* Ct, or_newton_report* rep);

#ifdef __cplusplus
}
#endif
#endif

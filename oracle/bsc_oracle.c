/*
 * Plain FP64 CPU oracle for quadratic B-spline cloth FEM
 * (Efficient B-Spline Finite Elements for Cloth Simulation, arXiv 2506.18867).
 *
 * TEST INFRASTRUCTURE ONLY: loaded by the test suite, the smoke check and the
 * bench's CPU-baseline leg, never by the product path.  It is deliberately
 * slow and literal: every quantity is computed from its definition in the
 * paper, in the paper's order, in double precision, with no blocking, fusion
 * or reuse beyond what the definitions state.  It shares no code with the
 * CUDA path.
 *
 * Readings of points the paper leaves open (each is pinned by a test where a
 * pin exists):
 *   R1 rest control points are inputs (flat patches use Greville placement);
 *   R2 reduced-rule layout for general S extrapolated from Fig. 3 (5x5 spans):
 *      checkerboard with (k_u + k_v) even => the two points lie on u = k_u;
 *      weights = clipped dual-cell area shared equally by the cell's points;
 *   R3 a point on a knot line is owned by span floor(x), clamped to the
 *      interior range [1, S-2] for interior-region points; basis functions are
 *      evaluated one-sided within the owner span (second derivatives jump at
 *      knots);
 *   R4 boundary spans put 3 Gauss points along the direction normal to the
 *      boundary, 2 along it (Fig. 3 red / blue reference cells);
 *   R6 lumped mass integrates rho * N_alpha with 3x3 Gauss per span;
 *   R7 projection clamps the eigenvalues of each span's summed 27x27
 *      elastic Hessian at zero (OR_PROJECT_SPAN); the per-point variant
 *      (OR_PROJECT_POINT) clamps, at every membrane point, the eigenvalues
 *      of each FBW term's own Hessian w.r.t. (f_1, f_2) separately (the two
 *      stretch terms and the shear term), then applies the chain rule; the
 *      bending Hessian is PSD by construction and is kept;
 *   R8 Dirichlet control points are eliminated: zero rows/columns, identity
 *      diagonal block, zero gradient;
 *   R9 line search accepts plain decrease E(C + alpha d) <= E(C).
 */
#include "bsc_oracle.h"

#include <math.h>
#include <stdlib.h>
#include <string.h>

/* ------------------------------------------------------------------------ */
/* Knot vectors and basis functions (Sec. 3.1.1, Eq. B-spline basis)         */
/* ------------------------------------------------------------------------ */

/* Open uniform quadratic knot vector with n control points: xi_k, k = 0..n+2,
 * is (0, 0, 0, 1, 2, ..., S, S, S) with S = n - 2 (integer lattice from 0). */
static double knot(int n, int k) {
  int S = n - 2;
  int v = k - 2;
  if (v < 0) v = 0;
  if (v > S) v = S;
  return (double)v;
}

/* 1/(x) with the paper's convention that a term dividing by zero (repeated
 * knots) is zero. */
static double inv_or_zero(double x) { return x == 0.0 ? 0.0 : 1.0 / x; }

/* Cox-de Boor recursion (Eq. B-spline basis) up to degree 2 with first and
 * second derivatives obtained by differentiating the recursion, evaluated at
 * t within the owner span [a, a+1] (knot interval xi_{a+2}..xi_{a+3}).
 * Degree-0 functions are the indicator of the owner span, so values at knots
 * are one-sided from the owner span.  Only functions a..a+4 (degree 0) can
 * be non-zero on the span; the recursion runs over that window.
 * Outputs the three degree-2 functions a, a+1, a+2: N[k], dN[k], d2N[k]. */
static void basis1d(int n, double t, int a, double N[3], double dN[3], double d2N[3]) {
  double B[3][5], D1[3][5], D2[3][5];
  int o = a + 2;
  for (int k = 0; k < 5; ++k) {
    int i = a + k;
    B[0][k] = (i == o) ? 1.0 : 0.0;
    D1[0][k] = 0.0;
    D2[0][k] = 0.0;
  }
  for (int p = 1; p <= 2; ++p) {
    for (int k = 0; k + p < 5; ++k) {
      int i = a + k;
      double xi_i = knot(n, i), xi_ip = knot(n, i + p);
      double xi_i1 = knot(n, i + 1), xi_ip1 = knot(n, i + p + 1);
      double A = inv_or_zero(xi_ip - xi_i);
      double Bc = inv_or_zero(xi_ip1 - xi_i1);
      B[p][k] = A * (t - xi_i) * B[p - 1][k] + Bc * (xi_ip1 - t) * B[p - 1][k + 1];
      D1[p][k] = A * (B[p - 1][k] + (t - xi_i) * D1[p - 1][k]) +
                 Bc * (-B[p - 1][k + 1] + (xi_ip1 - t) * D1[p - 1][k + 1]);
      D2[p][k] = A * (2.0 * D1[p - 1][k] + (t - xi_i) * D2[p - 1][k]) +
                 Bc * (-2.0 * D1[p - 1][k + 1] + (xi_ip1 - t) * D2[p - 1][k + 1]);
    }
  }
  for (int k = 0; k < 3; ++k) {
    N[k] = B[2][k];
    dN[k] = D1[2][k];
    d2N[k] = D2[2][k];
  }
}

/* Tensor-product basis (Eq. tensor product of B-spline basis): local l =
 * lj*3 + li.  out rows: N, N_u, N_v, N_uu, N_uv, N_vv. */
void or_basis9(const or_problem* p, double u, double v, int a, int b, double* out) {
  double Nu[3], dNu[3], d2Nu[3], Nv[3], dNv[3], d2Nv[3];
  basis1d(p->nu, u, a, Nu, dNu, d2Nu);
  basis1d(p->nv, v, b, Nv, dNv, d2Nv);
  for (int lj = 0; lj < 3; ++lj)
    for (int li = 0; li < 3; ++li) {
      int l = lj * 3 + li;
      out[0 * 9 + l] = Nu[li] * Nv[lj];
      out[1 * 9 + l] = dNu[li] * Nv[lj];
      out[2 * 9 + l] = Nu[li] * dNv[lj];
      out[3 * 9 + l] = d2Nu[li] * Nv[lj];
      out[4 * 9 + l] = dNu[li] * dNv[lj];
      out[5 * 9 + l] = Nu[li] * d2Nv[lj];
    }
}

/* ------------------------------------------------------------------------ */
/* Quadrature rules (Sec. 4.1 Reduced Integration, Sec. 4.2, Fig. 3)         */
/* ------------------------------------------------------------------------ */

typedef struct { double u, v, w; int a, b; } qpoint;
typedef struct { qpoint* pts; int n, cap; } qlist;

static void qpush(qlist* L, double u, double v, double w, int a, int b) {
  if (L->n == L->cap) {
    L->cap = L->cap ? 2 * L->cap : 256;
    L->pts = (qpoint*)realloc(L->pts, (size_t)L->cap * sizeof(qpoint));
  }
  qpoint q = {u, v, w, a, b};
  L->pts[L->n++] = q;
}

static int clampi(int x, int lo, int hi) { return x < lo ? lo : (x > hi ? hi : x); }

/* Owner span of an interior-region coordinate x along an axis with S spans:
 * floor(x), and for a point exactly on knot line k the interior span
 * clamp(k, 1, S-2) (reading R3). */
static int interior_owner(double x, int S) {
  double f = floor(x);
  if (x == f) return clampi((int)f, 1, S - 2);
  return (int)f;
}

/* Gauss-Legendre nodes and weights on [0, 1]. */
static void gauss01(int n, double* x, double* w) {
  if (n == 1) {
    x[0] = 0.5; w[0] = 1.0;
  } else if (n == 2) {
    double d = 0.5 / sqrt(3.0);
    x[0] = 0.5 - d; x[1] = 0.5 + d; w[0] = w[1] = 0.5;
  } else {
    double d = 0.5 * sqrt(0.6);
    x[0] = 0.5 - d; x[1] = 0.5; x[2] = 0.5 + d;
    w[0] = 5.0 / 18.0; w[1] = 8.0 / 18.0; w[2] = 5.0 / 18.0;
  }
}

static void push_gauss_span(qlist* L, int a, int b, int nqu, int nqv) {
  double xu[3], wu[3], xv[3], wv[3];
  gauss01(nqu, xu, wu);
  gauss01(nqv, xv, wv);
  for (int jv = 0; jv < nqv; ++jv)
    for (int iu = 0; iu < nqu; ++iu) qpush(L, a + xu[iu], b + xv[jv], wu[iu] * wv[jv], a, b);
}

static void build_rule(const or_problem* p, int which, qlist* L) {
  int Su = p->nu - 2, Sv = p->nv - 2;
  int rule = which == 0 ? p->mem_rule : p->bend_rule;
  L->n = 0;
  if (rule == OR_RULE_GAUSS2 || rule == OR_RULE_GAUSS3) {
    for (int b = 0; b < Sv; ++b)
      for (int a = 0; a < Su; ++a) push_gauss_span(L, a, b, rule, rule);
    return;
  }
  /* Boundary (ring) spans. */
  for (int b = 0; b < Sv; ++b)
    for (int a = 0; a < Su; ++a) {
      int ring_u = (a == 0 || a == Su - 1), ring_v = (b == 0 || b == Sv - 1);
      if (!ring_u && !ring_v) continue;
      if (which == 0)
        push_gauss_span(L, a, b, ring_u ? 3 : 2, ring_v ? 3 : 2);
      else
        qpush(L, a + 0.5, b + 0.5, 1.0, a, b); /* span centre */
    }
  if (rule == OR_RULE_STANDARD) {
    /* Sec. 6.5 case A: standard 2x2 Gauss on every interior span */
    for (int b = 1; b < Sv - 1; ++b)
      for (int a = 1; a < Su - 1; ++a) push_gauss_span(L, a, b, 2, 2);
    return;
  }
  /* Interior region [1, Su-1] x [1, Sv-1]: dual-grid cells centred on knots
   * (k_u, k_v), edges at k +- 1/2, clipped to the region. */
  double d = 0.5 / sqrt(3.0);
  for (int kv = 1; kv <= Sv - 1; ++kv)
    for (int ku = 1; ku <= Su - 1; ++ku) {
      int bu = (ku == 1 || ku == Su - 1), bv = (kv == 1 || kv == Sv - 1);
      double pu[2], pv[2], w;
      int np;
      if (which == 1) {
        /* one point at the cell centre (the knot), weight = clipped area */
        pu[0] = ku; pv[0] = kv; np = 1;
        w = (bu ? 0.5 : 1.0) * (bv ? 0.5 : 1.0);
      } else if (bu && bv) {
        pu[0] = ku; pv[0] = kv; np = 1; w = 0.25;
      } else if (bu) {
        pu[0] = pu[1] = ku; pv[0] = kv - d; pv[1] = kv + d; np = 2; w = 0.25;
      } else if (bv) {
        pu[0] = ku - d; pu[1] = ku + d; pv[0] = pv[1] = kv; np = 2; w = 0.25;
      } else if (((ku + kv) & 1) == 0) {
        pu[0] = pu[1] = ku; pv[0] = kv - d; pv[1] = kv + d; np = 2; w = 0.5;
      } else {
        pu[0] = ku - d; pu[1] = ku + d; pv[0] = pv[1] = kv; np = 2; w = 0.5;
      }
      for (int k = 0; k < np; ++k)
        qpush(L, pu[k], pv[k], w, interior_owner(pu[k], Su), interior_owner(pv[k], Sv));
    }
}

int or_quad_points(const or_problem* p, int which, double* out, int cap) {
  qlist L = {0, 0, 0};
  build_rule(p, which, &L);
  for (int k = 0; k < L.n && k < cap; ++k) {
    out[5 * k + 0] = L.pts[k].u;
    out[5 * k + 1] = L.pts[k].v;
    out[5 * k + 2] = L.pts[k].w;
    out[5 * k + 3] = L.pts[k].a;
    out[5 * k + 4] = L.pts[k].b;
  }
  int n = L.n;
  free(L.pts);
  return n;
}

/* ------------------------------------------------------------------------ */
/* Rest geometry at a point (Eq. deformation gradient; inverse function      */
/* theorem for the parametric derivatives, Sec. 4.1 and Sec. 4.2)            */
/* ------------------------------------------------------------------------ */

typedef struct {
  double N[6][9];     /* N, N_u, N_v, N_uu, N_uv, N_vv */
  double detJ;        /* det dX/d(u,v) */
  double Jinv[2][2];  /* Jinv[a][beta] = d u_a / d X_beta, u_0 = u, u_1 = v */
  double g[9][2];     /* dN_l / dX_beta */
  double c_uu, c_vv, c_u, c_v, c_uv; /* coefficients of Eq. (Laplacian ...) */
  double L[9];        /* Laplacian coefficient of control point l */
} pgeom;

static void point_geometry(const or_problem* p, const qpoint* q, pgeom* G) {
  or_basis9(p, q->u, q->v, q->a, q->b, &G->N[0][0]);
  /* first and second derivatives of the rest map X(u, v) = sum N_l X^l */
  double Xu[2] = {0, 0}, Xv[2] = {0, 0}, Xuu[2] = {0, 0}, Xuv[2] = {0, 0}, Xvv[2] = {0, 0};
  for (int l = 0; l < 9; ++l) {
    int i = q->a + l % 3, j = q->b + l / 3;
    const double* X = p->rest + 2 * (j * p->nu + i);
    for (int d = 0; d < 2; ++d) {
      Xu[d] += G->N[1][l] * X[d];
      Xv[d] += G->N[2][l] * X[d];
      Xuu[d] += G->N[3][l] * X[d];
      Xuv[d] += G->N[4][l] * X[d];
      Xvv[d] += G->N[5][l] * X[d];
    }
  }
  /* J[d][e] = dX_d / du_e */
  double J[2][2] = {{Xu[0], Xv[0]}, {Xu[1], Xv[1]}};
  double det = J[0][0] * J[1][1] - J[0][1] * J[1][0];
  G->detJ = det;
  G->Jinv[0][0] = J[1][1] / det;
  G->Jinv[0][1] = -J[0][1] / det;
  G->Jinv[1][0] = -J[1][0] / det;
  G->Jinv[1][1] = J[0][0] / det;
  /* X2[d][e][f] = d^2 X_d / du_e du_f */
  double X2[2][2][2];
  for (int d = 0; d < 2; ++d) {
    X2[d][0][0] = Xuu[d];
    X2[d][0][1] = X2[d][1][0] = Xuv[d];
    X2[d][1][1] = Xvv[d];
  }
  /* d^2 u_a / dX_b dX_c = -Jinv[a][d] X2[d][e][f] Jinv[e][b] Jinv[f][c] */
  double U2[2][2][2];
  for (int a = 0; a < 2; ++a)
    for (int b = 0; b < 2; ++b)
      for (int c = 0; c < 2; ++c) {
        double s = 0.0;
        for (int d = 0; d < 2; ++d)
          for (int e = 0; e < 2; ++e)
            for (int f = 0; f < 2; ++f) s += G->Jinv[a][d] * X2[d][e][f] * G->Jinv[e][b] * G->Jinv[f][c];
        U2[a][b][c] = -s;
      }
  double u1 = G->Jinv[0][0], u2 = G->Jinv[0][1], v1 = G->Jinv[1][0], v2 = G->Jinv[1][1];
  G->c_uu = u1 * u1 + u2 * u2;
  G->c_vv = v1 * v1 + v2 * v2;
  G->c_u = U2[0][0][0] + U2[0][1][1];
  G->c_v = U2[1][0][0] + U2[1][1][1];
  G->c_uv = 2.0 * (u1 * v1 + u2 * v2);
  for (int l = 0; l < 9; ++l) {
    for (int beta = 0; beta < 2; ++beta)
      G->g[l][beta] = G->N[1][l] * G->Jinv[0][beta] + G->N[2][l] * G->Jinv[1][beta];
    G->L[l] = G->c_uu * G->N[3][l] + G->c_vv * G->N[5][l] + G->c_u * G->N[1][l] +
              G->c_v * G->N[2][l] + G->c_uv * G->N[4][l];
  }
}

int or_point_tables(const or_problem* p, int which, double* out, int cap) {
  qlist L = {0, 0, 0};
  build_rule(p, which, &L);
  for (int k = 0; k < L.n && k < cap; ++k) {
    pgeom G;
    point_geometry(p, &L.pts[k], &G);
    double W = L.pts[k].w * fabs(G.detJ);
    if (which == 0) {
      double* r = out + 20 * k;
      r[0] = W;
      for (int l = 0; l < 9; ++l) {
        r[1 + 2 * l] = G.g[l][0];
        r[2 + 2 * l] = G.g[l][1];
      }
      r[19] = fabs(G.detJ);
    } else {
      double* r = out + 16 * k;
      r[0] = W;
      for (int l = 0; l < 9; ++l) r[1 + l] = G.L[l];
      r[10] = G.c_uu; r[11] = G.c_vv; r[12] = G.c_u; r[13] = G.c_v; r[14] = G.c_uv;
      r[15] = fabs(G.detJ);
    }
  }
  int n = L.n;
  free(L.pts);
  return n;
}

/* ------------------------------------------------------------------------ */
/* Lumped mass (Eq. lumped mass matrix): m_alpha = rho int N_alpha dX        */
/* ------------------------------------------------------------------------ */

void or_lumped_mass(const or_problem* p, double* m) {
  int Su = p->nu - 2, Sv = p->nv - 2;
  memset(m, 0, sizeof(double) * (size_t)p->nu * p->nv);
  double x[3], w[3];
  gauss01(3, x, w);
  for (int b = 0; b < Sv; ++b)
    for (int a = 0; a < Su; ++a)
      for (int jv = 0; jv < 3; ++jv)
        for (int iu = 0; iu < 3; ++iu) {
          qpoint q = {a + x[iu], b + x[jv], w[iu] * w[jv], a, b};
          pgeom G;
          point_geometry(p, &q, &G);
          for (int l = 0; l < 9; ++l) {
            int i = a + l % 3, j = b + l / 3;
            m[j * p->nu + i] += p->rho * q.w * fabs(G.detJ) * G.N[0][l];
          }
        }
}

/* ------------------------------------------------------------------------ */
/* Membrane: FBW stretching and shearing (Eqs. anisotropic invariants, FBW)  */
/* Bending: quadratic model, Psi = 1/2 mu_bd |Laplacian phi|^2                */
/* ------------------------------------------------------------------------ */

static void gather9(const or_problem* p, const double* C, int a, int b, double Cl[9][3]) {
  for (int l = 0; l < 9; ++l) {
    int i = a + l % 3, j = b + l / 3;
    for (int c = 0; c < 3; ++c) Cl[l][c] = C[3 * (j * p->nu + i) + c];
  }
}

/* Adds the PSD projection of the symmetric 6x6 T to A (both row-major). */
static void add_projected6(const double* T, double* A) {
  double P[36];
  or_project_psd(6, T, P, NULL);
  for (int i = 0; i < 36; ++i) A[i] += P[i];
}

/* d^2 Psi / df_beta,c df_delta,d of the FBW density (row/column index
 * 3 beta + c) as the sum of the three terms' Hessians, each projected to PSD
 * first when ptproj. */
static void fbw_hessian6(const or_problem* p, double f[2][3], int ptproj, double* A6) {
  double I5a = f[0][0] * f[0][0] + f[0][1] * f[0][1] + f[0][2] * f[0][2];
  double I5b = f[1][0] * f[1][0] + f[1][1] * f[1][1] + f[1][2] * f[1][2];
  double I6 = f[0][0] * f[1][0] + f[0][1] * f[1][1] + f[0][2] * f[1][2];
  double s1 = sqrt(I5a), s2 = sqrt(I5b);
  double Hst1[6][6], Hst2[6][6], Hsh[6][6];
  memset(Hst1, 0, sizeof(Hst1));
  memset(Hst2, 0, sizeof(Hst2));
  for (int c = 0; c < 3; ++c)
    for (int d = 0; d < 3; ++d) {
      double del = (c == d) ? 1.0 : 0.0;
      Hst1[c][d] = 2.0 * p->mu_st1 * ((1.0 - 1.0 / s1) * del + f[0][c] * f[0][d] / (s1 * s1 * s1));
      Hst2[3 + c][3 + d] = 2.0 * p->mu_st2 * ((1.0 - 1.0 / s2) * del + f[1][c] * f[1][d] / (s2 * s2 * s2));
      Hsh[c][d] = 2.0 * p->mu_sh * f[1][c] * f[1][d];
      Hsh[3 + c][3 + d] = 2.0 * p->mu_sh * f[0][c] * f[0][d];
      Hsh[c][3 + d] = 2.0 * p->mu_sh * (f[1][c] * f[0][d] + I6 * del);
      Hsh[3 + c][d] = 2.0 * p->mu_sh * (f[0][c] * f[1][d] + I6 * del);
    }
  memset(A6, 0, sizeof(double) * 36);
  if (ptproj) {
    add_projected6(&Hst1[0][0], A6);
    add_projected6(&Hst2[0][0], A6);
    add_projected6(&Hsh[0][0], A6);
  } else {
    for (int i = 0; i < 36; ++i) A6[i] = (&Hst1[0][0])[i] + (&Hst2[0][0])[i] + (&Hsh[0][0])[i];
  }
}

void or_fbw_hessian6(const or_problem* p, const double* f6, int ptproj, double* A6) {
  double f[2][3] = {{f6[0], f6[1], f6[2]}, {f6[3], f6[4], f6[5]}};
  fbw_hessian6(p, f, ptproj, A6);
}

/* Adds W * Psi_membrane and its derivatives w.r.t. the 27 span DOFs.  With
 * ptproj the Hessian of each FBW term is projected before the chain rule. */
static void membrane_point(const or_problem* p, const pgeom* G, double W, double Cl[9][3],
                           double* E, double* g27, double* H27, int ptproj) {
  double f[2][3] = {{0, 0, 0}, {0, 0, 0}}; /* f_beta = F e_beta */
  for (int beta = 0; beta < 2; ++beta)
    for (int c = 0; c < 3; ++c)
      for (int l = 0; l < 9; ++l) f[beta][c] += Cl[l][c] * G->g[l][beta];
  double I5a = f[0][0] * f[0][0] + f[0][1] * f[0][1] + f[0][2] * f[0][2];
  double I5b = f[1][0] * f[1][0] + f[1][1] * f[1][1] + f[1][2] * f[1][2];
  double I6 = f[0][0] * f[1][0] + f[0][1] * f[1][1] + f[0][2] * f[1][2];
  double s1 = sqrt(I5a), s2 = sqrt(I5b);
  double psi = p->mu_st1 * (s1 - 1.0) * (s1 - 1.0) + p->mu_st2 * (s2 - 1.0) * (s2 - 1.0) +
               p->mu_sh * I6 * I6;
  *E += W * psi;
  /* dPsi/df_beta */
  double dP[2][3];
  for (int c = 0; c < 3; ++c) {
    dP[0][c] = 2.0 * p->mu_st1 * (1.0 - 1.0 / s1) * f[0][c] + 2.0 * p->mu_sh * I6 * f[1][c];
    dP[1][c] = 2.0 * p->mu_st2 * (1.0 - 1.0 / s2) * f[1][c] + 2.0 * p->mu_sh * I6 * f[0][c];
  }
  if (g27)
    for (int l = 0; l < 9; ++l)
      for (int c = 0; c < 3; ++c)
        g27[3 * l + c] += W * (G->g[l][0] * dP[0][c] + G->g[l][1] * dP[1][c]);
  if (!H27) return;
  double A6[36];
  fbw_hessian6(p, f, ptproj, A6);
  double A[2][3][2][3];
  for (int be = 0; be < 2; ++be)
    for (int c = 0; c < 3; ++c)
      for (int de = 0; de < 2; ++de)
        for (int d = 0; d < 3; ++d) A[be][c][de][d] = A6[(3 * be + c) * 6 + 3 * de + d];
  /* chain rule: H_(l c)(m d) = sum_{beta, delta} g_l,beta g_m,delta A */
  for (int l = 0; l < 9; ++l)
    for (int c = 0; c < 3; ++c)
      for (int m = 0; m < 9; ++m)
        for (int d = 0; d < 3; ++d) {
          double s = 0.0;
          for (int beta = 0; beta < 2; ++beta)
            for (int delta = 0; delta < 2; ++delta)
              s += G->g[l][beta] * G->g[m][delta] * A[beta][c][delta][d];
          H27[(3 * l + c) * 27 + 3 * m + d] += W * s;
        }
}

static void bending_point(const or_problem* p, const pgeom* G, double W, double Cl[9][3],
                          double* E, double* g27, double* H27) {
  double lap[3] = {0, 0, 0};
  for (int c = 0; c < 3; ++c)
    for (int l = 0; l < 9; ++l) lap[c] += G->L[l] * Cl[l][c];
  *E += W * 0.5 * p->mu_bd * (lap[0] * lap[0] + lap[1] * lap[1] + lap[2] * lap[2]);
  if (g27)
    for (int l = 0; l < 9; ++l)
      for (int c = 0; c < 3; ++c) g27[3 * l + c] += W * p->mu_bd * G->L[l] * lap[c];
  if (H27)
    for (int l = 0; l < 9; ++l)
      for (int m = 0; m < 9; ++m)
        for (int c = 0; c < 3; ++c) H27[(3 * l + c) * 27 + 3 * m + c] += W * p->mu_bd * G->L[l] * G->L[m];
}

static void span_eval_impl(const or_problem* p, const double* C, int ptproj, double* E_span, double* g_span,
                           double* H_span) {
  int Su = p->nu - 2, Sv = p->nv - 2, Nsp = Su * Sv;
  double* E = (double*)calloc((size_t)Nsp, sizeof(double));
  if (g_span) memset(g_span, 0, sizeof(double) * 27 * (size_t)Nsp);
  if (H_span) memset(H_span, 0, sizeof(double) * 729 * (size_t)Nsp);
  for (int which = 0; which < 2; ++which) {
    qlist L = {0, 0, 0};
    build_rule(p, which, &L);
    for (int k = 0; k < L.n; ++k) {
      const qpoint* q = &L.pts[k];
      int s = q->b * Su + q->a;
      pgeom G;
      point_geometry(p, q, &G);
      double W = q->w * fabs(G.detJ);
      double Cl[9][3];
      gather9(p, C, q->a, q->b, Cl);
      double* g27 = g_span ? g_span + 27 * (size_t)s : NULL;
      double* H27 = H_span ? H_span + 729 * (size_t)s : NULL;
      if (which == 0)
        membrane_point(p, &G, W, Cl, &E[s], g27, H27, ptproj);
      else
        bending_point(p, &G, W, Cl, &E[s], g27, H27);
    }
    free(L.pts);
  }
  if (E_span) memcpy(E_span, E, sizeof(double) * (size_t)Nsp);
  free(E);
}

void or_span_eval(const or_problem* p, const double* C, double* E_span, double* g_span,
                  double* H_span) {
  span_eval_impl(p, C, 0, E_span, g_span, H_span);
}

void or_span_eval_projected(const or_problem* p, const double* C, int project, double* E_span,
                            double* g_span, double* H_span) {
  int Nsp = (p->nu - 2) * (p->nv - 2);
  span_eval_impl(p, C, project == OR_PROJECT_POINT, E_span, g_span, H_span);
  if (project == OR_PROJECT_SPAN && H_span) {
    double P[729];
    for (int s = 0; s < Nsp; ++s) {
      or_project_psd(27, H_span + 729 * (size_t)s, P, NULL);
      memcpy(H_span + 729 * (size_t)s, P, sizeof(P));
    }
  }
}

/* Selected spans only: points are enumerated as in or_span_eval and those
 * whose owner span is not selected are skipped. */
void or_span_terms_subset(const or_problem* p, const double* C, int n, const int* spans, int project,
                          double* E, double* g, double* H) {
  int Su = p->nu - 2, Sv = p->nv - 2, Nsp = Su * Sv;
  int* sel = (int*)malloc(sizeof(int) * Nsp);
  for (int s = 0; s < Nsp; ++s) sel[s] = -1;
  for (int k = 0; k < n; ++k) sel[spans[k]] = k;
  memset(E, 0, sizeof(double) * n);
  memset(g, 0, sizeof(double) * 27 * (size_t)n);
  memset(H, 0, sizeof(double) * 729 * (size_t)n);
  for (int which = 0; which < 2; ++which) {
    qlist L = {0, 0, 0};
    build_rule(p, which, &L);
    for (int k = 0; k < L.n; ++k) {
      const qpoint* q = &L.pts[k];
      int j = sel[q->b * Su + q->a];
      if (j < 0) continue;
      pgeom G;
      point_geometry(p, q, &G);
      double W = q->w * fabs(G.detJ);
      double Cl[9][3];
      gather9(p, C, q->a, q->b, Cl);
      if (which == 0)
        membrane_point(p, &G, W, Cl, &E[j], g + 27 * (size_t)j, H + 729 * (size_t)j,
                       project == OR_PROJECT_POINT);
      else
        bending_point(p, &G, W, Cl, &E[j], g + 27 * (size_t)j, H + 729 * (size_t)j);
    }
    free(L.pts);
  }
  if (project == OR_PROJECT_SPAN) {
    double P[729];
    for (int j = 0; j < n; ++j) {
      or_project_psd(27, H + 729 * (size_t)j, P, NULL);
      memcpy(H + 729 * (size_t)j, P, sizeof(P));
    }
  }
  free(sel);
}

/* ------------------------------------------------------------------------ */
/* PSD projection (projected Newton, Sec. 5.1): cyclic Jacobi eigensystem    */
/* ------------------------------------------------------------------------ */

int or_project_psd(int n, const double* H, double* P, double* eig_out) {
  double* A = (double*)malloc(sizeof(double) * n * n);
  double* V = (double*)calloc((size_t)n * n, sizeof(double));
  memcpy(A, H, sizeof(double) * n * n);
  for (int i = 0; i < n; ++i) V[i * n + i] = 1.0;
  double fro = 0.0;
  for (int i = 0; i < n * n; ++i) fro += A[i] * A[i];
  int sweep = 0;
  for (; sweep < 100; ++sweep) {
    double off = 0.0;
    for (int i = 0; i < n; ++i)
      for (int j = 0; j < n; ++j)
        if (i != j) off += A[i * n + j] * A[i * n + j];
    /* converged once the off-diagonal norm is 1e-14 of the Frobenius norm
     * (the rounding floor of the rotations is about n * eps) */
    if (off <= 1e-28 * fro || off == 0.0) break;
    for (int pi = 0; pi < n - 1; ++pi)
      for (int qi = pi + 1; qi < n; ++qi) {
        double apq = A[pi * n + qi];
        if (apq == 0.0) continue;
        double app = A[pi * n + pi], aqq = A[qi * n + qi];
        /* 2x2 symmetric Schur decomposition that zeroes a_pq */
        double tau = (aqq - app) / (2.0 * apq);
        double t = (tau >= 0.0 ? 1.0 : -1.0) / (fabs(tau) + sqrt(1.0 + tau * tau));
        double c = 1.0 / sqrt(1.0 + t * t), s = t * c;
        for (int k = 0; k < n; ++k) { /* A <- A J */
          double akp = A[k * n + pi], akq = A[k * n + qi];
          A[k * n + pi] = c * akp - s * akq;
          A[k * n + qi] = s * akp + c * akq;
        }
        for (int k = 0; k < n; ++k) { /* A <- J^T A */
          double apk = A[pi * n + k], aqk = A[qi * n + k];
          A[pi * n + k] = c * apk - s * aqk;
          A[qi * n + k] = s * apk + c * aqk;
        }
        for (int k = 0; k < n; ++k) { /* V <- V J */
          double vkp = V[k * n + pi], vkq = V[k * n + qi];
          V[k * n + pi] = c * vkp - s * vkq;
          V[k * n + qi] = s * vkp + c * vkq;
        }
      }
  }
  for (int i = 0; i < n; ++i)
    for (int j = 0; j < n; ++j) {
      double s = 0.0;
      for (int k = 0; k < n; ++k) {
        double lam = A[k * n + k];
        if (lam > 0.0) s += V[i * n + k] * lam * V[j * n + k];
      }
      P[i * n + j] = s;
    }
  if (eig_out)
    for (int k = 0; k < n; ++k) eig_out[k] = A[k * n + k];
  free(A);
  free(V);
  return sweep;
}

/* ------------------------------------------------------------------------ */
/* Incremental potential, gradient and stencil Hessian (Sec. 3.2, Sec. 5.1)  */
/* ------------------------------------------------------------------------ */

static int slot_of(int du, int dv) { return (dv + 2) * 5 + (du + 2); }

static double eval_impl(const or_problem* p, const or_scene* sc, const double* C,
                        const double* Chat, double* grad, double* K) {
  int nu = p->nu, nv = p->nv, N = nu * nv;
  int Su = nu - 2, Sv = nv - 2, Nsp = Su * Sv;
  double* E_s = (double*)malloc(sizeof(double) * Nsp);
  double* g_s = grad ? (double*)malloc(sizeof(double) * 27 * (size_t)Nsp) : NULL;
  double* H_s = K ? (double*)malloc(sizeof(double) * 729 * (size_t)Nsp) : NULL;
  span_eval_impl(p, C, sc->project == OR_PROJECT_POINT, E_s, g_s, H_s);
  double* m = (double*)malloc(sizeof(double) * N);
  or_lumped_mass(p, m);

  double E = 0.0;
  for (int s = 0; s < Nsp; ++s) E += E_s[s];
  if (grad) memset(grad, 0, sizeof(double) * 3 * (size_t)N);
  if (K) memset(K, 0, sizeof(double) * 225 * (size_t)N);
  double P[729];
  for (int s = 0; s < Nsp; ++s) {
    int a = s % Su, b = s / Su;
    if (K) {
      if (sc->project == OR_PROJECT_SPAN)
        or_project_psd(27, H_s + 729 * (size_t)s, P, NULL);
      else
        memcpy(P, H_s + 729 * (size_t)s, sizeof(P));
    }
    for (int l = 0; l < 9; ++l) {
      int alpha = (b + l / 3) * nu + a + l % 3;
      if (grad)
        for (int c = 0; c < 3; ++c) grad[3 * alpha + c] += g_s[27 * (size_t)s + 3 * l + c];
      if (K)
        for (int mm = 0; mm < 9; ++mm) {
          int du = mm % 3 - l % 3, dv = mm / 3 - l / 3;
          double* blk = K + 225 * (size_t)alpha + 9 * slot_of(du, dv);
          for (int c = 0; c < 3; ++c)
            for (int d = 0; d < 3; ++d) blk[3 * c + d] += P[(3 * l + c) * 27 + 3 * mm + d];
        }
    }
  }
  /* inertia (implicit Euler) and gravity with the lumped mass */
  for (int al = 0; al < N; ++al) {
    const double* x = C + 3 * al;
    if (sc->dt > 0.0) {
      double k = m[al] / (sc->dt * sc->dt);
      const double* xh = Chat + 3 * al;
      for (int c = 0; c < 3; ++c) {
        E += 0.5 * k * (x[c] - xh[c]) * (x[c] - xh[c]);
        if (grad) grad[3 * al + c] += k * (x[c] - xh[c]);
        if (K) K[225 * (size_t)al + 9 * slot_of(0, 0) + 4 * c] += k;
      }
    }
    for (int c = 0; c < 3; ++c) {
      E -= m[al] * sc->gravity[c] * x[c];
      if (grad) grad[3 * al + c] -= m[al] * sc->gravity[c];
    }
  }
  /* Dirichlet control points: eliminated */
  if (sc->n_pinned > 0) {
    char* pin = (char*)calloc((size_t)N, 1);
    for (int k = 0; k < sc->n_pinned; ++k) pin[sc->pinned[k]] = 1;
    for (int al = 0; al < N; ++al) {
      int i = al % nu, j = al / nu;
      if (grad && pin[al])
        for (int c = 0; c < 3; ++c) grad[3 * al + c] = 0.0;
      if (!K) continue;
      for (int dv = -2; dv <= 2; ++dv)
        for (int du = -2; du <= 2; ++du) {
          int ii = i + du, jj = j + dv;
          if (ii < 0 || ii >= nu || jj < 0 || jj >= nv) continue;
          int be = jj * nu + ii;
          if (pin[al] || pin[be]) {
            double* blk = K + 225 * (size_t)al + 9 * slot_of(du, dv);
            for (int e = 0; e < 9; ++e) blk[e] = 0.0;
            if (al == be) blk[0] = blk[4] = blk[8] = 1.0;
          }
        }
    }
    free(pin);
  }
  free(E_s);
  free(g_s);
  free(H_s);
  free(m);
  return E;
}

double or_eval(const or_problem* p, const or_scene* sc, const double* C, const double* Chat,
               double* grad, double* K) {
  return eval_impl(p, sc, C, Chat, grad, K);
}

double or_energy(const or_problem* p, const or_scene* sc, const double* C, const double* Chat) {
  return eval_impl(p, sc, C, Chat, NULL, NULL);
}

/* Rows of eval_impl for selected control points: the spans touching each
 * row are evaluated (and projected when sc->project), then gathered. */
void or_eval_rows(const or_problem* p, const or_scene* sc, const double* C, const double* Chat, int n,
                  const int* rows, double* g, double* K) {
  int nu = p->nu, nv = p->nv, N = nu * nv, Su = nu - 2, Sv = nv - 2, Nsp = Su * Sv;
  char* need = (char*)calloc((size_t)Nsp, 1);
  for (int k = 0; k < n; ++k) {
    int i = rows[k] % nu, j = rows[k] / nu;
    for (int b = j - 2; b <= j; ++b)
      for (int a = i - 2; a <= i; ++a)
        if (a >= 0 && a < Su && b >= 0 && b < Sv) need[b * Su + a] = 1;
  }
  int ns = 0;
  for (int s = 0; s < Nsp; ++s) ns += need[s];
  int* list = (int*)malloc(sizeof(int) * (ns ? ns : 1));
  int* pos = (int*)malloc(sizeof(int) * Nsp);
  ns = 0;
  for (int s = 0; s < Nsp; ++s) {
    pos[s] = need[s] ? ns : -1;
    if (need[s]) list[ns++] = s;
  }
  double* Es = (double*)malloc(sizeof(double) * (ns ? ns : 1));
  double* gs = (double*)malloc(sizeof(double) * 27 * (size_t)(ns ? ns : 1));
  double* Hs = (double*)malloc(sizeof(double) * 729 * (size_t)(ns ? ns : 1));
  or_span_terms_subset(p, C, ns, list, sc->project, Es, gs, Hs);
  double* m = (double*)malloc(sizeof(double) * N);
  or_lumped_mass(p, m);
  char* pin = (char*)calloc((size_t)N, 1);
  for (int k = 0; k < sc->n_pinned; ++k) pin[sc->pinned[k]] = 1;
  memset(g, 0, sizeof(double) * 3 * (size_t)n);
  memset(K, 0, sizeof(double) * 225 * (size_t)n);
  for (int k = 0; k < n; ++k) {
    int al = rows[k], i = al % nu, j = al / nu;
    double* gk = g + 3 * (size_t)k;
    double* Kk = K + 225 * (size_t)k;
    for (int b = j - 2; b <= j; ++b)
      for (int a = i - 2; a <= i; ++a) {
        if (a < 0 || a >= Su || b < 0 || b >= Sv) continue;
        int jj = pos[b * Su + a], l = (j - b) * 3 + (i - a);
        for (int c = 0; c < 3; ++c) gk[c] += gs[27 * (size_t)jj + 3 * l + c];
        for (int mm = 0; mm < 9; ++mm) {
          int du = a + mm % 3 - i, dv = b + mm / 3 - j;
          double* blk = Kk + 9 * slot_of(du, dv);
          for (int c = 0; c < 3; ++c)
            for (int d = 0; d < 3; ++d) blk[3 * c + d] += Hs[729 * (size_t)jj + (3 * l + c) * 27 + 3 * mm + d];
        }
      }
    const double* x = C + 3 * al;
    for (int c = 0; c < 3; ++c) {
      if (sc->dt > 0.0) {
        double kk = m[al] / (sc->dt * sc->dt);
        gk[c] += kk * (x[c] - Chat[3 * al + c]);
        Kk[9 * slot_of(0, 0) + 4 * c] += kk;
      }
      gk[c] -= m[al] * sc->gravity[c];
    }
    for (int dv = -2; dv <= 2; ++dv)
      for (int du = -2; du <= 2; ++du) {
        int ii = i + du, jj2 = j + dv;
        if (ii < 0 || ii >= nu || jj2 < 0 || jj2 >= nv) continue;
        int be = jj2 * nu + ii;
        if (pin[al] || pin[be]) {
          double* blk = Kk + 9 * slot_of(du, dv);
          for (int e = 0; e < 9; ++e) blk[e] = 0.0;
          if (al == be) blk[0] = blk[4] = blk[8] = 1.0;
        }
      }
    if (pin[al])
      for (int c = 0; c < 3; ++c) gk[c] = 0.0;
  }
  free(need); free(list); free(pos); free(Es); free(gs); free(Hs); free(m); free(pin);
}

/* ------------------------------------------------------------------------ */
/* Linear algebra on the stencil Hessian                                     */
/* ------------------------------------------------------------------------ */

void or_stencil_matvec(int nu, int nv, const double* K, const double* x, double* y) {
  for (int j = 0; j < nv; ++j)
    for (int i = 0; i < nu; ++i) {
      int al = j * nu + i;
      double acc[3] = {0, 0, 0};
      for (int dv = -2; dv <= 2; ++dv)
        for (int du = -2; du <= 2; ++du) {
          int ii = i + du, jj = j + dv;
          if (ii < 0 || ii >= nu || jj < 0 || jj >= nv) continue;
          const double* blk = K + 225 * (size_t)al + 9 * slot_of(du, dv);
          const double* xb = x + 3 * (jj * nu + ii);
          for (int c = 0; c < 3; ++c)
            for (int d = 0; d < 3; ++d) acc[c] += blk[3 * c + d] * xb[d];
        }
      for (int c = 0; c < 3; ++c) y[3 * al + c] = acc[c];
    }
}

int or_solve_banded(int nu, int nv, const double* K, const double* b, double* x) {
  int N = nu * nv, n = 3 * N;
  int bw = 3 * (2 * nu + 2) + 2; /* max |row - col| of a non-zero */
  /* L stored by rows: Lb[i*(bw+1) + (i - j)] = L[i][j], j in [i-bw, i] */
  double* Lb = (double*)calloc((size_t)n * (bw + 1), sizeof(double));
  if (!Lb) return -2;
  /* copy the lower band of K */
  for (int al = 0; al < N; ++al) {
    int i = al % nu, j = al / nu;
    for (int dv = -2; dv <= 2; ++dv)
      for (int du = -2; du <= 2; ++du) {
        int ii = i + du, jj = j + dv;
        if (ii < 0 || ii >= nu || jj < 0 || jj >= nv) continue;
        int be = jj * nu + ii;
        const double* blk = K + 225 * (size_t)al + 9 * slot_of(du, dv);
        for (int c = 0; c < 3; ++c)
          for (int d = 0; d < 3; ++d) {
            int r = 3 * al + c, col = 3 * be + d;
            if (col <= r) Lb[(size_t)r * (bw + 1) + (r - col)] = blk[3 * c + d];
          }
      }
  }
  /* Cholesky A = L L^T within the band */
  for (int r = 0; r < n; ++r) {
    int j0 = r - bw < 0 ? 0 : r - bw;
    for (int col = j0; col <= r; ++col) {
      double s = Lb[(size_t)r * (bw + 1) + (r - col)];
      int k0 = (col - bw < 0 ? 0 : col - bw);
      if (k0 < j0) k0 = j0;
      for (int k = k0; k < col; ++k)
        s -= Lb[(size_t)r * (bw + 1) + (r - k)] * Lb[(size_t)col * (bw + 1) + (col - k)];
      if (col == r) {
        if (!(s > 0.0)) { free(Lb); return -1; }
        Lb[(size_t)r * (bw + 1)] = sqrt(s);
      } else {
        Lb[(size_t)r * (bw + 1) + (r - col)] = s / Lb[(size_t)col * (bw + 1)];
      }
    }
  }
  /* forward and back substitution */
  for (int r = 0; r < n; ++r) {
    double s = b[r];
    int j0 = r - bw < 0 ? 0 : r - bw;
    for (int k = j0; k < r; ++k) s -= Lb[(size_t)r * (bw + 1) + (r - k)] * x[k];
    x[r] = s / Lb[(size_t)r * (bw + 1)];
  }
  for (int r = n - 1; r >= 0; --r) {
    double s = x[r];
    int k1 = r + bw >= n ? n - 1 : r + bw;
    for (int k = r + 1; k <= k1; ++k) s -= Lb[(size_t)k * (bw + 1) + (k - r)] * x[k];
    x[r] = s / Lb[(size_t)r * (bw + 1)];
  }
  free(Lb);
  return 0;
}

/* inverse of a symmetric 3x3 block by the adjugate */
static void inv3(const double* A, double* B) {
  double c00 = A[4] * A[8] - A[5] * A[7], c01 = A[5] * A[6] - A[3] * A[8], c02 = A[3] * A[7] - A[4] * A[6];
  double det = A[0] * c00 + A[1] * c01 + A[2] * c02;
  B[0] = c00 / det;
  B[1] = (A[2] * A[7] - A[1] * A[8]) / det;
  B[2] = (A[1] * A[5] - A[2] * A[4]) / det;
  B[3] = c01 / det;
  B[4] = (A[0] * A[8] - A[2] * A[6]) / det;
  B[5] = (A[2] * A[3] - A[0] * A[5]) / det;
  B[6] = c02 / det;
  B[7] = (A[1] * A[6] - A[0] * A[7]) / det;
  B[8] = (A[0] * A[4] - A[1] * A[3]) / det;
}

static double dot(int n, const double* a, const double* b) {
  double s = 0.0;
  for (int i = 0; i < n; ++i) s += a[i] * b[i];
  return s;
}

int or_solve_pcg(int nu, int nv, const double* K, const double* b, double* x, double rel_tol,
                 int max_iter) {
  int N = nu * nv, n = 3 * N;
  double* Dinv = (double*)malloc(sizeof(double) * 9 * N);
  double *r = (double*)malloc(sizeof(double) * n), *z = (double*)malloc(sizeof(double) * n);
  double *pp = (double*)malloc(sizeof(double) * n), *q = (double*)malloc(sizeof(double) * n);
  for (int al = 0; al < N; ++al) inv3(K + 225 * (size_t)al + 9 * slot_of(0, 0), Dinv + 9 * al);
  memset(x, 0, sizeof(double) * n);
  memcpy(r, b, sizeof(double) * n);
  double bn = sqrt(dot(n, b, b));
  int it = 0, conv = 0;
  if (bn == 0.0) conv = 1;
  for (int al = 0; al < N; ++al)
    for (int c = 0; c < 3; ++c) z[3 * al + c] = dot(3, Dinv + 9 * al + 3 * c, r + 3 * al);
  memcpy(pp, z, sizeof(double) * n);
  double rz = dot(n, r, z);
  while (!conv && it < max_iter) {
    or_stencil_matvec(nu, nv, K, pp, q);
    double alpha = rz / dot(n, pp, q);
    for (int i = 0; i < n; ++i) {
      x[i] += alpha * pp[i];
      r[i] -= alpha * q[i];
    }
    ++it;
    if (sqrt(dot(n, r, r)) <= rel_tol * bn) { conv = 1; break; }
    for (int al = 0; al < N; ++al)
      for (int c = 0; c < 3; ++c) z[3 * al + c] = dot(3, Dinv + 9 * al + 3 * c, r + 3 * al);
    double rz1 = dot(n, r, z);
    double beta = rz1 / rz;
    rz = rz1;
    for (int i = 0; i < n; ++i) pp[i] = z[i] + beta * pp[i];
  }
  free(Dinv); free(r); free(z); free(pp); free(q);
  return conv ? it : -it;
}

/* ------------------------------------------------------------------------ */
/* Projected Newton iteration with backtracking line search (Sec. 5.1)       */
/* ------------------------------------------------------------------------ */

int or_newton_step(const or_problem* p, const or_scene* sc, double* C, const double* Chat,
                   int solver, double pcg_tol, int max_halvings, or_newton_report* rep) {
  int N = p->nu * p->nv, n = 3 * N;
  double* g = (double*)malloc(sizeof(double) * n);
  double* K = (double*)malloc(sizeof(double) * 225 * (size_t)N);
  double* rhs = (double*)malloc(sizeof(double) * n);
  double* dC = (double*)malloc(sizeof(double) * n);
  double* Ct = (double*)malloc(sizeof(double) * n);
  memset(rep, 0, sizeof(*rep));
  double E0 = or_eval(p, sc, C, Chat, g, K);
  for (int i = 0; i < n; ++i) rhs[i] = -g[i];
  int st;
  if (solver == 0) {
    st = or_solve_banded(p->nu, p->nv, K, rhs, dC);
    rep->solver_iters = 0;
  } else {
    st = or_solve_pcg(p->nu, p->nv, K, rhs, dC, pcg_tol, 100000);
    rep->solver_iters = st;
    st = st < 0 ? -1 : 0;
  }
  double ginf = 0.0, dinf = 0.0;
  for (int i = 0; i < n; ++i) {
    if (fabs(g[i]) > ginf) ginf = fabs(g[i]);
    if (fabs(dC[i]) > dinf) dinf = fabs(dC[i]);
  }
  rep->E0 = E0;
  rep->grad_inf = ginf;
  rep->dir_inf = dinf;
  int status = st;
  if (st == 0) status = or_line_search(p, sc, C, Chat, dC, E0, max_halvings, Ct, rep);
  rep->status = status;
  free(g); free(K); free(rhs); free(dC); free(Ct);
  return status;
}

/* Backtracking along dC from C, whose energy is E0 (Sec. 5.1: the step
 * length starts at 1 and is halved until the incremental potential does not
 * increase, plain decrease without an Armijo constant): C <- C + alpha dC
 * for the first alpha in 1, 1/2, 1/4, ... with E(C + alpha dC) <= E0; after
 * max_halvings halvings without one, C is left unchanged and -3 returned.
 * Ct: caller's workspace of 3N doubles.  Fills E1, alpha, ls_halvings. */
int or_line_search(const or_problem* p, const or_scene* sc, double* C, const double* Chat, const double* dC,
                   double E0, int max_halvings, double* Ct, or_newton_report* rep) {
  const int n = 3 * p->nu * p->nv;
  double alpha = 1.0;
  int h = 0;
  for (;;) {
    for (int i = 0; i < n; ++i) Ct[i] = C[i] + alpha * dC[i];
    double E1 = or_energy(p, sc, Ct, Chat);
    if (E1 <= E0) {
      memcpy(C, Ct, sizeof(double) * n);
      rep->E1 = E1;
      rep->alpha = alpha;
      rep->ls_halvings = h;
      return 0;
    }
    if (h == max_halvings) {
      rep->E1 = E1;
      rep->alpha = 0.0;
      rep->ls_halvings = h;
      return -3;
    }
    alpha *= 0.5;
    ++h;
  }
}

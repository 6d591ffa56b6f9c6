// K3: per-span PSD projection of the 27x27 elastic Hessian in FP64
// (projected Newton, Sec. 5.1): P = V max(Lambda, 0) V^T = H - sum_{lam<0}
// lam w w^T.
//
// One thread per span.  The span Hessian is
//   H = sum_q (G_q (x) I3) A_q (G_q (x) I3)^T + sum_b W_b mu_bd (L_b L_b^T) (x) I3,
// so its range lies in R (x) R^3 with R = span{g_q,1, g_q,2, L_b} in R^9;
// every such vector sums to zero over the 9 control points (derivatives of a
// partition of unity), so dim R <= min(8, 2 n_mem + n_bd) =: D.  With an
// orthonormal basis Q of R, H = (Q (x) I3) H_r (Q (x) I3)^T and H_r (3D x 3D)
// has the same non-zero spectrum.  H_r is built directly from the per-point
// d^2 Psi/df^2 (kept by the span evaluator) in FP64, reduced to tridiagonal
// form, its negative eigenvalues are found by Sturm bisection and their
// eigenvectors by inverse iteration; the span Hessian in HBM is then
// corrected in place.  Spans with no negative eigenvalue are left untouched.
#include "bsc_internal.cuh"
#include "eig_small.cuh"

namespace {

template <typename T>
struct ProjArgs {
  int Nsp, Nm, Nb;
  double mubd;
  const int* __restrict__ moff;
  const int* __restrict__ boff;
  const T* __restrict__ tabm;
  const T* __restrict__ tabb;
  const T* __restrict__ A;
  T* __restrict__ H;
  int* __restrict__ nneg;
  int* __restrict__ status;
};

// Eigenvalues below -NEG_REL * ||T|| are projected; above that they are
// rounding noise of exact zeros (their contribution is below 1e-14 ||H||).
constexpr double NEG_REL = 1e-14;
// A basis candidate whose residual after orthogonalisation is below
// RANK_REL of its norm lies in the span of the previous ones.
constexpr double RANK_REL = 1e-13;

template <int D>
__device__ __forceinline__ void add_basis_vector(double (&v)[9], double (&Q)[D][9], int& d) {
  // remove the constant vector (exactly orthogonal in exact arithmetic)
  double mean = 0.0;
#pragma unroll
  for (int l = 0; l < 9; ++l) mean += v[l];
  mean *= (1.0 / 9.0);
  double n0 = 0.0;
#pragma unroll
  for (int l = 0; l < 9; ++l) {
    v[l] -= mean;
    n0 += v[l] * v[l];
  }
  if (n0 == 0.0 || d >= D) return;
  // modified Gram-Schmidt, two passes
  for (int pass = 0; pass < 2; ++pass)
#pragma unroll
    for (int k = 0; k < D; ++k) {
      if (k >= d) break;
      double dot = 0.0;
#pragma unroll
      for (int l = 0; l < 9; ++l) dot += Q[k][l] * v[l];
#pragma unroll
      for (int l = 0; l < 9; ++l) v[l] -= dot * Q[k][l];
    }
  double n1 = 0.0;
#pragma unroll
  for (int l = 0; l < 9; ++l) n1 += v[l] * v[l];
  if (n1 <= RANK_REL * RANK_REL * n0) return;
  const double inv = 1.0 / sqrt(n1);
#pragma unroll
  for (int k = 0; k < D; ++k)
    if (k == d) {
#pragma unroll
      for (int l = 0; l < 9; ++l) Q[k][l] = v[l] * inv;
    }
  ++d;
}

template <typename T, int D, int BLOCK>
__global__ void __launch_bounds__(BLOCK) k_project(ProjArgs<T> P, const int* __restrict__ list,
                                                   int count) {
  constexpr int n = 3 * D;
  constexpr int NP = n * (n + 1) / 2;
  extern __shared__ __align__(16) double smd[];
  const int t = blockIdx.x * BLOCK + threadIdx.x;
  if (t >= count) return;
  const int s = list[t];
  const eig::Packed A{smd + threadIdx.x, BLOCK};
#pragma unroll 1
  for (int k = 0; k < NP; ++k) A.base[k * BLOCK] = 0.0;

  const int q0 = P.moff[s], q1 = P.moff[s + 1];
  const int b0 = P.boff[s], b1 = P.boff[s + 1];

  // 1. orthonormal basis of R = span{g_q,beta, L_b} (mean-free)
  double Q[D][9];
#pragma unroll
  for (int k = 0; k < D; ++k)
#pragma unroll
    for (int l = 0; l < 9; ++l) Q[k][l] = 0.0;
  int d = 0;
  for (int q = q0; q < q1; ++q)
    for (int be = 0; be < 2; ++be) {
      double v[9];
#pragma unroll
      for (int l = 0; l < 9; ++l) v[l] = (double)P.tabm[(1 + 2 * l + be) * P.Nm + q];
      add_basis_vector<D>(v, Q, d);
    }
  for (int q = b0; q < b1; ++q) {
    double v[9];
#pragma unroll
    for (int l = 0; l < 9; ++l) v[l] = (double)P.tabb[(1 + l) * P.Nb + q];
    add_basis_vector<D>(v, Q, d);
  }

  // 2. reduced Hessian H_r(3k+c, 3k'+d) (lower triangle)
  for (int q = q0; q < q1; ++q) {
    double gr[D][2];
#pragma unroll
    for (int k = 0; k < D; ++k) gr[k][0] = gr[k][1] = 0.0;
#pragma unroll
    for (int l = 0; l < 9; ++l) {
      const double g0 = (double)P.tabm[(1 + 2 * l) * P.Nm + q];
      const double g1 = (double)P.tabm[(2 + 2 * l) * P.Nm + q];
#pragma unroll
      for (int k = 0; k < D; ++k) {
        gr[k][0] += Q[k][l] * g0;
        gr[k][1] += Q[k][l] * g1;
      }
    }
    double A6[6][6];
    {
      int e = 0;
#pragma unroll
      for (int r = 0; r < 6; ++r)
#pragma unroll
        for (int c = r; c < 6; ++c) {
          A6[r][c] = (double)P.A[(e++) * P.Nm + q];
          A6[c][r] = A6[r][c];
        }
    }
#pragma unroll
    for (int k = 0; k < D; ++k) {
      double Tk[3][6];
#pragma unroll
      for (int c = 0; c < 3; ++c)
#pragma unroll
        for (int j = 0; j < 6; ++j) Tk[c][j] = gr[k][0] * A6[c][j] + gr[k][1] * A6[3 + c][j];
#pragma unroll
      for (int k2 = 0; k2 <= k; ++k2)
#pragma unroll
        for (int c = 0; c < 3; ++c)
#pragma unroll
          for (int dd = 0; dd < 3; ++dd) {
            if (k2 == k && dd > c) continue;
            A.at(3 * k + c, 3 * k2 + dd) += Tk[c][dd] * gr[k2][0] + Tk[c][3 + dd] * gr[k2][1];
          }
    }
  }
  for (int q = b0; q < b1; ++q) {
    const double WB = (double)P.tabb[q] * P.mubd;
    double Lr[D];
#pragma unroll
    for (int k = 0; k < D; ++k) Lr[k] = 0.0;
#pragma unroll
    for (int l = 0; l < 9; ++l) {
      const double L = (double)P.tabb[(1 + l) * P.Nb + q];
#pragma unroll
      for (int k = 0; k < D; ++k) Lr[k] += Q[k][l] * L;
    }
#pragma unroll
    for (int k = 0; k < D; ++k)
#pragma unroll
      for (int k2 = 0; k2 <= k; ++k2) {
        const double h = WB * Lr[k] * Lr[k2];
#pragma unroll
        for (int c = 0; c < 3; ++c) A.at(3 * k + c, 3 * k2 + c) += h;
      }
  }

  // 3. tridiagonal form and the negative part of the spectrum
  double dg[n], ed[n], tau[n];
  eig::tridiagonalize<n>(A, dg, ed, tau);
  double tn = 0.0;
#pragma unroll
  for (int i = 0; i < n; ++i) {
    const double r = fabs(dg[i]) + fabs(ed[i]) + (i > 0 ? fabs(ed[i - 1]) : 0.0);
    tn = fmax(tn, r);
  }
  if (!(tn > 0.0)) {
    P.nneg[s] = 0;
    if (!isfinite(tn)) atomicOr(P.status, BSC_STATUS_NUMERIC_FLAG);
    return;
  }
  const double itn = 1.0 / tn;
  double ds[n], es[n], e2[n];
#pragma unroll
  for (int i = 0; i < n; ++i) {
    ds[i] = dg[i] * itn;
    es[i] = ed[i] * itn;
    e2[i] = es[i] * es[i];
  }
  const int kneg = eig::sturm_count<n>(ds, e2, -NEG_REL);
  P.nneg[s] = kneg;
  if (kneg == 0) return;

  // 4. eigenpairs of the negative eigenvalues; w = (Q (x) I3) x in span DOFs
  double Y[n][n];    // tridiagonal-basis eigenvectors found so far
  double Wv[n][27];  // their span-DOF images
  double lam[n];
  double lo = -1.0 - 1e-12;
  for (int k = 0; k < kneg; ++k) {
    const double lk = eig::bisect<n>(ds, e2, k, lo, -NEG_REL);
    eig::TriLU<n> lu;
    lu.factor(ds, es, lk, 2.3e-16);
    double y[n];
#pragma unroll
    for (int i = 0; i < n; ++i) y[i] = 1.0 + 0.125 * (double)((7 * i + 3 * k) % 5);
    for (int it = 0; it < 3; ++it) {
      for (int j = 0; j < k; ++j) {
        double dot = 0.0;
#pragma unroll
        for (int i = 0; i < n; ++i) dot += Y[j][i] * y[i];
#pragma unroll
        for (int i = 0; i < n; ++i) y[i] -= dot * Y[j][i];
      }
      if (it < 2) lu.solve(y);
      double nn = 0.0;
#pragma unroll
      for (int i = 0; i < n; ++i) nn += y[i] * y[i];
      const double inv = 1.0 / sqrt(nn);
#pragma unroll
      for (int i = 0; i < n; ++i) y[i] *= inv;
    }
    // Rayleigh quotient on the scaled tridiagonal
    double rq = 0.0;
#pragma unroll
    for (int i = 0; i < n; ++i) {
      double ty = ds[i] * y[i];
      if (i > 0) ty += es[i - 1] * y[i - 1];
      if (i + 1 < n) ty += es[i] * y[i + 1];
      rq += y[i] * ty;
    }
#pragma unroll
    for (int i = 0; i < n; ++i) Y[k][i] = y[i];
    lam[k] = fmin(rq, 0.0) * tn;
    lo = lk - 1e-12;
    eig::back_transform<n>(A, tau, y);
#pragma unroll
    for (int l = 0; l < 9; ++l)
#pragma unroll
      for (int c = 0; c < 3; ++c) {
        double acc = 0.0;
#pragma unroll
        for (int kk = 0; kk < D; ++kk) acc += Q[kk][l] * y[3 * kk + c];
        Wv[k][3 * l + c] = acc;
      }
  }

  // 5. P = H - sum_k lam_k w_k w_k^T on the packed upper 27x27 in HBM
  int e = 0;
#pragma unroll 1
  for (int r = 0; r < 27; ++r)
#pragma unroll 1
    for (int c = r; c < 27; ++c, ++e) {
      double corr = 0.0;
      for (int k = 0; k < kneg; ++k) corr += lam[k] * Wv[k][r] * Wv[k][c];
      T* h = P.H + (size_t)e * P.Nsp + s;
      *h = (T)((double)(*h) - corr);
    }
}

template <typename T, int D, int BLOCK>
cudaError_t run_bucket(bsc_ctx* c, int b) {
  const int count = c->bucket_off[b + 1] - c->bucket_off[b];
  if (count <= 0) return cudaSuccess;
  ProjArgs<T> P;
  P.Nsp = c->Nsp; P.Nm = c->Nmem; P.Nb = c->Nbd; P.mubd = c->mu_bd;
  P.moff = c->mem_off; P.boff = c->bd_off;
  P.tabm = (const T*)c->tab_mem; P.tabb = (const T*)c->tab_bd;
  P.A = (const T*)c->A_mem; P.H = (T*)c->H_span;
  P.nneg = c->nneg; P.status = c->dstatus;
  constexpr int n = 3 * D;
  const size_t sm = sizeof(double) * (n * (n + 1) / 2) * BLOCK;
  auto k = k_project<T, D, BLOCK>;
  cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
  if (e != cudaSuccess) return e;
  k<<<(count + BLOCK - 1) / BLOCK, BLOCK, sm, c->stream>>>(P, c->bucket_list + c->bucket_off[b], count);
  return cudaGetLastError();
}

template <typename T>
cudaError_t run_all(bsc_ctx* c) {
  cudaError_t e;
  if ((e = run_bucket<T, 5, 128>(c, 0)) != cudaSuccess) return e;
  if ((e = run_bucket<T, 7, 64>(c, 1)) != cudaSuccess) return e;
  return run_bucket<T, 8, 64>(c, 2);
}

}  // namespace

cudaError_t launch_project(bsc_ctx* c) {
  if (c->precision == BSC_FP64) return run_all<double>(c);
  return run_all<float>(c);
}

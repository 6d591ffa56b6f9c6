// FP64 building blocks of the per-span SPD projection (projected Newton,
// Sec. 5.1): a symmetric n x n matrix (n = 3 D, D <= 8) held packed in a
// strided store, reduced to tridiagonal form by Householder similarity
// transforms, the negative part of its spectrum located by Sturm-sequence
// bisection, and the matching eigenvectors recovered by inverse iteration on
// the tridiagonal matrix, then mapped back through the reflectors.
//
// All routines are __host__ __device__ so that they run unchanged in one
// GPU thread per span (store = interleaved shared memory) or on the host.
#pragma once

#include <math.h>

#ifndef BSC_HD
#ifdef __CUDACC__
#define BSC_HD __host__ __device__ __forceinline__
#else
#define BSC_HD inline
#endif
#endif

namespace eig {

// Packed lower triangle (row i holds columns 0..i), element stride `stride`.
struct Packed {
  double* base;
  int stride;
  BSC_HD double& at(int i, int j) const {
    return i >= j ? base[(i * (i + 1) / 2 + j) * stride] : base[(j * (j + 1) / 2 + i) * stride];
  }
};

// Householder tridiagonalisation A = Q T Q^T, Q = H_0 H_1 ... H_{n-3},
// H_k = I - tau_k v_k v_k^T acting on rows/cols k+1..n-1.  On return d[], e[]
// hold T (e[i] couples i and i+1), v_k is stored in A(k+1.., k) and tau[k]
// in tau.  Only the lower triangle of A is read and written.
template <int n>
BSC_HD void tridiagonalize(const Packed& A, double* d, double* e, double* tau) {
#pragma unroll
  for (int k = 0; k < n - 2; ++k) {
    d[k] = A.at(k, k);
    const double x0 = A.at(k + 1, k);
    double sigma = 0.0;
#pragma unroll
    for (int i = k + 2; i < n; ++i) sigma += A.at(i, k) * A.at(i, k);
    if (sigma == 0.0) {
      e[k] = x0;
      tau[k] = 0.0;
      continue;
    }
    const double nrm = sqrt(x0 * x0 + sigma);
    const double alpha = x0 >= 0.0 ? -nrm : nrm;
    const double v0 = x0 - alpha;
    const double t = 2.0 / (v0 * v0 + sigma);
    tau[k] = t;
    e[k] = alpha;
    A.at(k + 1, k) = v0;
    double v[n], p[n];
#pragma unroll
    for (int i = k + 1; i < n; ++i) {
      v[i] = A.at(i, k);
      p[i] = 0.0;
    }
    // p = A_sub v (one pass over the lower triangle)
#pragma unroll
    for (int i = k + 1; i < n; ++i) {
#pragma unroll
      for (int j = k + 1; j < i; ++j) {
        const double a = A.at(i, j);
        p[i] += a * v[j];
        p[j] += a * v[i];
      }
      p[i] += A.at(i, i) * v[i];
    }
    double vp = 0.0;
#pragma unroll
    for (int i = k + 1; i < n; ++i) {
      p[i] *= t;
      vp += v[i] * p[i];
    }
    const double K = 0.5 * t * vp;
#pragma unroll
    for (int i = k + 1; i < n; ++i) p[i] -= K * v[i];  // p := w
#pragma unroll
    for (int i = k + 1; i < n; ++i)
#pragma unroll
      for (int j = k + 1; j <= i; ++j) A.at(i, j) -= v[i] * p[j] + p[i] * v[j];
  }
  d[n - 2] = A.at(n - 2, n - 2);
  e[n - 2] = A.at(n - 1, n - 2);
  d[n - 1] = A.at(n - 1, n - 1);
  tau[n - 2] = 0.0;
  e[n - 1] = 0.0;
}

// Number of eigenvalues of the tridiagonal (d, e2 = e^2) that are < x, from
// the signs of the leading principal minors of T - x I (Sturm sequence,
// Sylvester's law of inertia).  Division free; the minors are rescaled by
// powers of two to stay in range (d, e scaled so |entries| <= 1).
template <int n>
BSC_HD int sturm_count(const double* d, const double* e2, double x) {
  double pm = 1.0, p = d[0] - x;
  int cnt = p < 0.0 ? 1 : 0;
  if (p == 0.0) p = -1e-300;
#pragma unroll
  for (int i = 1; i < n; ++i) {
    double pn = (d[i] - x) * p - e2[i - 1] * pm;
    if (pn == 0.0) pn = p < 0.0 ? 1e-300 : -1e-300;
    cnt += ((pn < 0.0) != (p < 0.0)) ? 1 : 0;
    const double ap = fabs(pn);
    if (ap > 1e150 || ap < 1e-150) {
      const double sc = ap > 1e150 ? 1e-150 : 1e150;
      pn *= sc;
      p *= sc;
    }
    pm = p;
    p = pn;
  }
  return cnt;
}

// k-th smallest eigenvalue (0-based) of the tridiagonal in [lo, hi], where
// count(lo) <= k < count(hi), by bisection to full precision.
template <int n>
BSC_HD double bisect(const double* d, const double* e2, int k, double lo, double hi) {
  for (int it = 0; it < 64; ++it) {
    const double mid = 0.5 * (lo + hi);
    if (!(mid > lo && mid < hi)) break;
    if (sturm_count<n>(d, e2, mid) > k)
      hi = mid;
    else
      lo = mid;
  }
  return 0.5 * (lo + hi);
}

// Gaussian elimination with partial pivoting of the tridiagonal T - lam I
// (bands u0 diagonal, u1, u2 superdiagonals; multipliers m; swap flags sw),
// tiny pivots replaced by `tiny`.  Stores reciprocals of the pivots.
template <int n>
struct TriLU {
  double u0r[n], u1[n], u2[n], m[n];
  bool sw[n];
  BSC_HD void factor(const double* d, const double* e, double lam, double tiny) {
    double c0 = d[0] - lam, c1 = e[0], c2 = 0.0;
#pragma unroll
    for (int i = 0; i < n - 1; ++i) {
      const double a1 = d[i + 1] - lam, e1 = (i + 1 < n - 1) ? e[i + 1] : 0.0;
      if (fabs(e[i]) > fabs(c0)) {
        sw[i] = true;
        const double mu = c0 / e[i];
        m[i] = mu;
        u0r[i] = 1.0 / e[i];
        u1[i] = a1;
        u2[i] = e1;
        const double n0 = c1 - mu * a1, n1 = c2 - mu * e1;
        c0 = n0; c1 = n1; c2 = 0.0;
      } else {
        sw[i] = false;
        if (fabs(c0) < tiny) c0 = c0 < 0.0 ? -tiny : tiny;
        const double mu = e[i] / c0;
        m[i] = mu;
        u0r[i] = 1.0 / c0;
        u1[i] = c1;
        u2[i] = c2;
        const double n0 = a1 - mu * c1, n1 = e1 - mu * c2;
        c0 = n0; c1 = n1; c2 = 0.0;
      }
    }
    if (fabs(c0) < tiny) c0 = c0 < 0.0 ? -tiny : tiny;
    u0r[n - 1] = 1.0 / c0;
    u1[n - 1] = 0.0;
    u2[n - 1] = 0.0;
  }
  // solves in place
  BSC_HD void solve(double* b) const {
#pragma unroll
    for (int i = 0; i < n - 1; ++i) {
      if (sw[i]) {
        const double t = b[i];
        b[i] = b[i + 1];
        b[i + 1] = t - m[i] * b[i + 1];
      } else {
        b[i + 1] -= m[i] * b[i];
      }
    }
#pragma unroll
    for (int i = n - 1; i >= 0; --i) {
      double s = b[i];
      if (i + 1 < n) s -= u1[i] * b[i + 1];
      if (i + 2 < n) s -= u2[i] * b[i + 2];
      b[i] = s * u0r[i];
    }
  }
};

// x <- H_0 ... H_{n-3} x (maps a tridiagonal-basis vector back).
template <int n>
BSC_HD void back_transform(const Packed& A, const double* tau, double* x) {
#pragma unroll
  for (int k = n - 3; k >= 0; --k) {
    if (tau[k] == 0.0) continue;
    double s = 0.0;
#pragma unroll
    for (int i = k + 1; i < n; ++i) s += A.at(i, k) * x[i];
    s *= tau[k];
#pragma unroll
    for (int i = k + 1; i < n; ++i) x[i] -= s * A.at(i, k);
  }
}

}  // namespace eig

// Per-span SPD projection (projected Newton, Sec. 5.1) in FP64, written for
// one GPU thread per span with a small on-chip working set:
//   A  packed lower triangle of the reduced Hessian (3D x 3D), then the
//      Householder vectors, with tau_k kept in the freed diagonal slot;
//   R  3n doubles: the scaled tridiagonal (d, e, e^2);
//   Qs  the span's orthonormal basis Q (9 x D) of its derivative vectors,
//      and the derivative vectors in that basis, computed once per context
//      from the rest geometry (span_basis, by the caller);
//   Ys  per-thread scratch slot (global memory): the eigenvectors found so
//      far (for re-orthogonalisation inside clusters).
// The span Hessian in HBM is corrected in place, P = H - sum lam w w^T over
// the negative eigenpairs.  __host__ __device__ so the same code runs on the
// host for checks.  The PSD test and phase 1 also come in double-float
// versions (device only: span_form_df, ldlt_psd_df, span_tridiag_df), pairs
// of FP32 numbers on the FP32 pipe, which GB300 runs many times faster than
// its FP64 pipe; phase 2 stays FP64.
#pragma once

#include <math.h>

#ifndef BSC_HD
#ifdef __CUDACC__
#define BSC_HD __host__ __device__ __forceinline__
#else
#define BSC_HD inline
#endif
#endif
// The large phases are separate calls on the GPU, so that each gets its own
// register allocation instead of one allocation for the whole kernel.
#ifdef __CUDACC__
#define BSC_PHASE __host__ __device__ __noinline__
#else
#define BSC_PHASE inline
#endif

namespace proj {

// Strided view (interleaved shared memory on the GPU, plain arrays on the host).
struct View {
  double* p;
  int s;
  BSC_HD double& operator[](int i) const { return p[(long)i * s]; }
};

BSC_HD int lp(int i, int j) { return i >= j ? i * (i + 1) / 2 + j : j * (j + 1) / 2 + i; }

// Sign bit and biased exponent of a double without FP64 pipe instructions.
BSC_HD int sign_of(double x) {
#ifdef __CUDA_ARCH__
  return (unsigned)__double2hiint(x) >> 31;
#else
  return signbit(x) ? 1 : 0;
#endif
}
BSC_HD int expo_of(double x) {
#ifdef __CUDA_ARCH__
  return (__double2hiint(x) >> 20) & 0x7ff;
#else
  int e;
  if (x == 0.0) return 0;
  frexp(x, &e);
  return e + 1022;
#endif
}

// det(T - x I) of a scaled tridiagonal (d[0..n), e^2[0..n-1)) by the
// three-term recurrence of the leading principal minors, with the Sturm
// count (sign changes of the minors = eigenvalues below x, by Sylvester's
// law of inertia).  An exact zero minor is replaced by a tiny value of the
// sign opposite to its predecessor.  The recurrence is homogeneous in
// (p_i, p_i-1): char_poly_scaled rescales the pair by a power of two
// whenever the larger of the two leaves [2^-500, 2^500].  *exact is false
// when a replacement or a rescaling made the value's scale differ from the
// determinant's.
template <int n>
BSC_PHASE double char_poly_scaled(const double* d, int ds, const double* e2, int es, double x, int* cnt_out,
                                  bool* exact) {
  double pm = 1.0, p = d[0] - x;
  int cnt = sign_of(p);
  bool ok = true;
#pragma unroll 1
  for (int i = 1; i < n; ++i) {
    double pn = (d[(long)i * ds] - x) * p - e2[(long)(i - 1) * es] * pm;
    if (expo_of(pn) == 0) {
      pn = sign_of(p) ? 1e-300 : -1e-300;
      ok = false;
    }
    cnt += sign_of(pn) ^ sign_of(p);
    const int ea = expo_of(pn), eb = expo_of(p), mx = ea > eb ? ea : eb;
    if (mx > 1023 + 500 || mx < 1023 - 500) {
      const double sc = mx > 1023 ? 0x1p-500 : 0x1p500;
      pn *= sc;
      p *= sc;
      ok = false;
    }
    pm = p;
    p = pn;
  }
  *cnt_out = cnt;
  *exact = ok;
  return p;
}

// The same value and count.  With ||T|| <= 1 the minors of the sizes used
// here (n <= 24) stay far inside that range, so this pass runs the
// recurrence without rescaling and tracks the exponents with integer
// operations only; the rare pair that leaves the range sends the call to
// char_poly_scaled, which then gives the identical result.  Each step is
// three FP64 operations; the rescaling multiplications leave the loop.
template <int n, class DA, class EA>
BSC_HD double char_poly(const DA& d, const EA& e2, double x, int* cnt_out, bool* exact) {
  double pm = 1.0, p = d[0] - x;
  int cnt = sign_of(p), eb = expo_of(p);
  bool ok = true, in_range = true;
#pragma unroll
  for (int i = 1; i < n; ++i) {
    double pn = (d[i] - x) * p - e2[i - 1] * pm;
    const bool z = expo_of(pn) == 0;
    pn = z ? (sign_of(p) ? 1e-300 : -1e-300) : pn;
    ok = ok && !z;
    cnt += sign_of(pn) ^ sign_of(p);
    const int ea = expo_of(pn), mx = ea > eb ? ea : eb;
    in_range = in_range && mx <= 1023 + 500 && mx >= 1023 - 500;
    pm = p;
    p = pn;
    eb = ea;
  }
  if (!in_range) {
    // rare: copy the operands out (the fast pass keeps them in registers)
    double buf[2 * n];
#pragma unroll
    for (int i = 0; i < n; ++i) {
      buf[i] = d[i];
      buf[n + i] = e2[i];
    }
    return char_poly_scaled<n>(buf, 1, buf + n, 1, x, cnt_out, exact);
  }
  *cnt_out = cnt;
  *exact = ok;
  return p;
}

// Offset accessor of a strided view (e^2 of the tridiagonal kept in R).
struct ViewAt {
  View v;
  int o;
  BSC_HD double operator[](int i) const { return v[o + i]; }
};

// Eigenvalues of the scaled tridiagonal below x; d at R[0..n), e^2 at
// R[2n..3n).
template <int n>
BSC_HD int sturm(const View& R, double x) {
  int cnt;
  bool ex;
  char_poly<n>(ViewAt{R, 0}, ViewAt{R, 2 * n}, x, &cnt, &ex);
  return cnt;
}

// The same count in FP32 on a copy of the scaled tridiagonal: the FP32 pipe
// is 64x the FP64 one, so the bracket of each eigenvalue is narrowed here
// first and only validated and refined in FP64.  The FP32 count is exact for
// a tridiagonal within a few FP32 ulps of T, so its brackets are widened
// before the FP64 check.  With ||T|| <= 1 and n <= 24 the minors stay below
// (1 + sqrt 2)^24 < 2e9, so only a pair near underflow (next to a multiple
// root, e.g. the exact zero eigenvalues of a rank-deficient span) is
// rescaled.
BSC_HD int sign_of_f(float x) {
#ifdef __CUDA_ARCH__
  return (unsigned)__float_as_int(x) >> 31;
#else
  return signbit(x) ? 1 : 0;
#endif
}

template <int n>
BSC_HD int sturm32(const float (&d)[n], const float (&e2)[n], float x) {
  float pm = 1.0f, p = d[0] - x;
  int cnt = sign_of_f(p);
#pragma unroll
  for (int i = 1; i < n; ++i) {
    float pn = (d[i] - x) * p - e2[i - 1] * pm;
    if (pn == 0.0f) pn = sign_of_f(p) ? 1e-30f : -1e-30f;
    cnt += sign_of_f(pn) ^ sign_of_f(p);
    if (fmaxf(fabsf(pn), fabsf(p)) < 1e-30f) {  // a pair near underflow (a multiple root nearby)
      pn *= 1e30f;
      p *= 1e30f;
    }
    pm = p;
    p = pn;
  }
  return cnt;
}

// FP32 bracket of eigenvalue k in [*a, *b] to 2^-22 of its width by
// quadrisection: each step counts at the three quarter points, which are
// independent (three dependent chains in flight instead of one).
template <int n>
BSC_HD void bracket32(const float (&d)[n], const float (&e2)[n], int k, float* a, float* b) {
  float lo = *a, hi = *b;
#pragma unroll 1
  for (int it = 0; it < 11; ++it) {
    const float h = 0.25f * (hi - lo);
    const float m1 = lo + h, m2 = lo + 2.0f * h, m3 = lo + 3.0f * h;
    const bool c1 = sturm32<n>(d, e2, m1) > k, c2 = sturm32<n>(d, e2, m2) > k, c3 = sturm32<n>(d, e2, m3) > k;
    if (c1) {
      hi = m1;
    } else if (c2) {
      lo = m1;
      hi = m2;
    } else if (c3) {
      lo = m2;
      hi = m3;
    } else {
      lo = m3;
    }
  }
  *a = lo;
  *b = hi;
}

// Householder vectors in A(i, k), i > k; tau_k in A(k, k).  x <- H_0 ... H_{n-3} x.
template <int n>
BSC_HD void back_transform(const View& A, double (&x)[n]) {
#pragma unroll
  for (int k = n - 3; k >= 0; --k) {
    const double t = A[lp(k, k)];
    double s = 0.0;
#pragma unroll
    for (int i = k + 1; i < n; ++i) s += A[lp(i, k)] * x[i];
    s *= t;
#pragma unroll
    for (int i = k + 1; i < n; ++i) x[i] -= s * A[lp(i, k)];
  }
}

// Orthonormal basis Q (rows Q[9 k + l], k < D) of the span of a span's
// derivative vectors {g_q,beta, L_b} with the constant vector removed (it
// lies in the kernel of every one): modified Gram-Schmidt with one
// re-orthogonalisation pass; a candidate whose residual is below rank_rel of
// its norm is dependent and skipped, unused rows are zero.  Depends on the
// rest geometry only.  Returns the rank.
template <int D, class Tab, class QView>
BSC_HD int span_basis(const Tab& tab, const QView& Q, double rank_rel) {
  int d = 0;
  const int nm = tab.nm(), nb = tab.nb(), nvec = 2 * nm + nb;
  for (int iv = 0; iv < nvec; ++iv) {
    double v[9];
    if (iv < 2 * nm) {
#pragma unroll
      for (int l = 0; l < 9; ++l) v[l] = tab.g(iv >> 1, l, iv & 1);
    } else {
#pragma unroll
      for (int l = 0; l < 9; ++l) v[l] = tab.L(iv - 2 * nm, l);
    }
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
    if (d >= D || n0 == 0.0) continue;
#pragma unroll
    for (int pass = 0; pass < 2; ++pass)
#pragma unroll
      for (int k = 0; k < D; ++k) {
        if (k >= d) break;
        double dt = 0.0;
#pragma unroll
        for (int l = 0; l < 9; ++l) dt += Q[9 * k + l] * v[l];
#pragma unroll
        for (int l = 0; l < 9; ++l) v[l] -= dt * Q[9 * k + l];
      }
    double n1 = 0.0;
#pragma unroll
    for (int l = 0; l < 9; ++l) n1 += v[l] * v[l];
    if (n1 <= rank_rel * rank_rel * n0) continue;
    const double inv = 1.0 / sqrt(n1);
#pragma unroll
    for (int l = 0; l < 9; ++l) Q[9 * d + l] = v[l] * inv;
    ++d;
  }
  for (int k = d; k < D; ++k)
#pragma unroll
    for (int l = 0; l < 9; ++l) Q[9 * k + l] = 0.0;
  return d;
}

// The reduced Hessian H_r of a span into A (packed lower triangle, index
// 3k + c for reduced vector k and component c).  Tab: nm(), nb(), wb(q) =
// W mu_bd, a6(q, e) (packed upper 6x6), gr(q, k, beta) and lr(q, k): the
// derivative vectors g_q,beta and L_q in the span's reduced basis.
template <int D, class Tab>
BSC_PHASE void span_form(const Tab& tab, const View& A) {
  constexpr int n = 3 * D;
  constexpr int NP = n * (n + 1) / 2;
#pragma unroll 1
  for (int k = 0; k < NP; ++k) A[k] = 0.0;
  const int nm = tab.nm(), nb = tab.nb();

  // 1. reduced Hessian, lower triangle, index 3k + c
  for (int q = 0; q < nm; ++q) {
    double gr[D][2];
#pragma unroll
    for (int k = 0; k < D; ++k) {
      gr[k][0] = tab.gr(q, k, 0);
      gr[k][1] = tab.gr(q, k, 1);
    }
    double A6[6][6];
    {
      int e = 0;
#pragma unroll
      for (int r = 0; r < 6; ++r)
#pragma unroll
        for (int c = r; c < 6; ++c) {
          A6[r][c] = tab.a6(q, e++);
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
            // two FMAs into the accumulator (a separate product and sum would
            // cost the FP64 pipe a DMUL and a DADD more per entry)
            const int ix = lp(3 * k + c, 3 * k2 + dd);
            A[ix] = fma(Tk[c][3 + dd], gr[k2][1], fma(Tk[c][dd], gr[k2][0], A[ix]));
          }
    }
  }
  for (int q = 0; q < nb; ++q) {
    const double WB = tab.wb(q);
    double Lr[D];
#pragma unroll
    for (int k = 0; k < D; ++k) Lr[k] = tab.lr(q, k);
#pragma unroll
    for (int k = 0; k < D; ++k) {
      const double wl = WB * Lr[k];
#pragma unroll
      for (int k2 = 0; k2 <= k; ++k2)
#pragma unroll
        for (int c = 0; c < 3; ++c) {
          const int ix = lp(3 * k + c, 3 * k2 + c);
          A[ix] = fma(wl, Lr[k2], A[ix]);
        }
    }
  }
}

// The PSD test that precedes the eigendecomposition: an LDL^T factorisation
// of H_r + tau I in FP64, tau = neg_rel tr(H_r) / n, in place in A.  For a
// PSD matrix tr / n lies between ||H_r||_2 / n and ||H_r||_2, so tau is at
// most the eigendecomposition's own threshold (neg_rel on the same scale).
// Every pivot positive means H_r + tau I is positive definite (the
// factorisation's backward error, about n eps ||H_r||, is below tau), so no
// eigenvalue of H_r lies below -tau and the span needs no projection.  A
// non-positive trace, or a non-positive or non-finite pivot, fails the test;
// the span then goes through the eigendecomposition, which decides which
// eigenvalues to clamp.  Destroys A.  Returns true when the test passes.
template <int D>
BSC_PHASE bool ldlt_psd(const View& A, double neg_rel) {
  constexpr int n = 3 * D;
  double tr = 0.0;
#pragma unroll
  for (int i = 0; i < n; ++i) tr += A[lp(i, i)];
  if (!(tr > 0.0) || !isfinite(tr)) return false;
  const double tau = neg_rel * tr * (1.0 / n);
#pragma unroll 1
  for (int i = 0; i < n; ++i) A[lp(i, i)] += tau;
  // right-looking LDL^T: A(i, j) -= l_ik A(j, k) over the trailing block,
  // l_ik = A(i, k) / d_k; the multipliers are not kept
#pragma unroll 1
  for (int k = 0; k < n; ++k) {
    const double dk = A[lp(k, k)];
    if (!(dk > 0.0) || !isfinite(dk)) return false;
    const double r = 1.0 / dk;
#pragma unroll 1
    for (int i = k + 1; i < n; ++i) {
      const int ri = i * (i + 1) / 2;
      const double l = A[ri + k] * r;
#pragma unroll 1
      for (int j = k + 1; j <= i; ++j) A[ri + j] = fma(-l, A[j * (j + 1) / 2 + k], A[ri + j]);
    }
  }
  return true;
}

#ifdef __CUDACC__
// ---------------------------------------------------------------------------
// Double-float arithmetic: a value is an unevaluated sum hi + lo of two FP32
// numbers (|lo| <= ulp(hi) / 2 once normalised), about 48 significant bits.
// GB300 retires 64 times as many FP32 as FP64 operations per clock, so the
// ~15 FP32 operations of a double-float multiply-add cost a quarter of the
// FP64 instruction they replace.  The error-free transformations are Knuth's
// two-sum, Dekker's fast two-sum (|a| >= |b|) and the FMA two-product; every
// operation is an explicitly rounded intrinsic, so no contraction or
// reassociation can change them.
// ---------------------------------------------------------------------------
struct DF {
  float h, l;
};
__device__ __forceinline__ DF df_two_sum(float a, float b) {
  const float s = __fadd_rn(a, b), bb = __fsub_rn(s, a);
  return {s, __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb))};
}
__device__ __forceinline__ DF df_fast_two_sum(float a, float b) {
  const float s = __fadd_rn(a, b);
  return {s, __fsub_rn(b, __fsub_rn(s, a))};
}
// x * a with a in FP32 (exact product of the high parts plus the low part's)
__device__ __forceinline__ DF df_mul_f(DF x, float a) {
  const float p = __fmul_rn(x.h, a);
  return {p, __fmaf_rn(x.l, a, __fmaf_rn(x.h, a, -p))};
}
// x * y (the lo * lo term, below 2^-48 of the product, is dropped)
__device__ __forceinline__ DF df_mul(DF x, DF y) {
  const float p = __fmul_rn(x.h, y.h);
  return {p, __fmaf_rn(x.h, y.l, __fmaf_rn(x.l, y.h, __fmaf_rn(x.h, y.h, -p)))};
}
// x + y for unnormalised x, y, normalised result
__device__ __forceinline__ DF df_add(DF x, DF y) {
  const DF s = df_two_sum(x.h, y.h);
  return df_fast_two_sum(s.h, __fadd_rn(__fadd_rn(x.l, y.l), s.l));
}
__device__ __forceinline__ DF df_norm(DF x) { return df_fast_two_sum(x.h, x.l); }
__device__ __forceinline__ DF df_neg(DF x) { return {-x.h, -x.l}; }
// 1 / x by one Newton step from the FP32 reciprocal
__device__ __forceinline__ DF df_rcp(DF x) {
  const float r = __frcp_rn(x.h);
  const float p = __fmul_rn(x.h, r);
  const float e = __fmaf_rn(-x.l, r, __fsub_rn(__fsub_rn(1.0f, p), __fmaf_rn(x.h, r, -p)));  // 1 - x r
  return df_fast_two_sum(r, __fmul_rn(r, e));
}
__device__ __forceinline__ DF df_split(double v) {
  const float h = __double2float_rn(v);
  return {h, __double2float_rn(v - (double)h)};
}
// a slot of a double View holds a double-float during the double-float phases
__device__ __forceinline__ DF& df_at(const View& A, int i) { return *reinterpret_cast<DF*>(&A[i]); }

// Scales the NP double-float entries of A by the power of two that brings the
// largest to [1, 2) (exact; FP32's exponent range is that of the scaled
// problem, so squares and reciprocals of small entries stay normal) and
// returns the inverse scale (1 when it leaves A unscaled).
template <int NP>
__device__ __forceinline__ float df_scale_unit(const View& A) {
  float mx = 0.0f;
#pragma unroll 1
  for (int e = 0; e < NP; ++e) mx = fmaxf(mx, fabsf(df_at(A, e).h));
  // a zero, non-finite or vanishing matrix (largest entry below 2^-100,
  // whose scale factor could overflow FP32) stays as it is: its columns fall
  // below the no-reflection threshold, as exact zeros do in FP64
  if (!(mx >= 7.8886091e-31f) || !isfinite(mx)) return 1.0f;
  const int ex = ilogbf(mx);
  const float sc = ldexpf(1.0f, -ex);
#pragma unroll 1
  for (int e = 0; e < NP; ++e) {
    DF& a = df_at(A, e);
    a = DF{__fmul_rn(a.h, sc), __fmul_rn(a.l, sc)};
  }
  return ldexpf(1.0f, ex);
}


// span_form in double-float arithmetic: Tab gives the reduced vectors as
// double-float splits (gr2, lr2), d^2 Psi / df^2 (a6, exact floats when
// Tab::kFloatA6) and the bending weights (wb2) as double-floats; each entry's accumulation
// carries about 2^-47 of the sum of its terms' magnitudes, some 30 times the
// FP64 formation's rounding and far below the PSD test's threshold.  A
// holds the double-float entries (df_at) on return.
template <int D, class Tab>
__device__ __noinline__ void span_form_df(const Tab& tab, const View& A) {
  constexpr int n = 3 * D;
  constexpr int NP = n * (n + 1) / 2;
#pragma unroll 1
  for (int k = 0; k < NP; ++k) df_at(A, k) = DF{0.0f, 0.0f};
  const int nm = tab.nm(), nb = tab.nb();
  for (int q = 0; q < nm; ++q) {
    DF g[D][2];
#pragma unroll
    for (int k = 0; k < D; ++k) {
      g[k][0] = tab.gr2(q, k, 0);
      g[k][1] = tab.gr2(q, k, 1);
    }
    DF A6[6][6];
    {
      int e = 0;
#pragma unroll
      for (int r = 0; r < 6; ++r)
#pragma unroll
        for (int c = r; c < 6; ++c) {
          A6[r][c] = tab.a6(q, e++);
          A6[c][r] = A6[r][c];
        }
    }
#pragma unroll 1
    for (int k = 0; k < D; ++k) {
      DF gk0 = g[0][0], gk1 = g[0][1];
#pragma unroll
      for (int z = 1; z < D; ++z)
        if (z == k) { gk0 = g[z][0]; gk1 = g[z][1]; }
      DF Tk[3][6];
#pragma unroll
      for (int c = 0; c < 3; ++c)
#pragma unroll
        for (int j = 0; j < 6; ++j) {
          if constexpr (Tab::kFloatA6)  // FP32 tables: the entries are exact floats
            Tk[c][j] = df_add(df_mul_f(gk0, A6[c][j].h), df_mul_f(gk1, A6[3 + c][j].h));
          else
            Tk[c][j] = df_add(df_mul(gk0, A6[c][j]), df_mul(gk1, A6[3 + c][j]));
        }
#pragma unroll
      for (int k2 = 0; k2 < D; ++k2) {
        if (k2 > k) break;
#pragma unroll
        for (int c = 0; c < 3; ++c)
#pragma unroll
          for (int dd = 0; dd < 3; ++dd) {
            if (k2 == k && dd > c) continue;
            DF& a = df_at(A, lp(3 * k + c, 3 * k2 + dd));
            const DF t = df_add(df_mul(Tk[c][dd], g[k2][0]), df_mul(Tk[c][3 + dd], g[k2][1]));
            a = df_add(a, t);
          }
      }
    }
  }
  for (int q = 0; q < nb; ++q) {
    const DF WB = tab.wb2(q);
    DF Lr[D];
#pragma unroll
    for (int k = 0; k < D; ++k) Lr[k] = tab.lr2(q, k);
#pragma unroll
    for (int k = 0; k < D; ++k) {
      const DF wl = df_norm(df_mul(WB, Lr[k]));
#pragma unroll
      for (int k2 = 0; k2 <= k; ++k2)
#pragma unroll
        for (int c = 0; c < 3; ++c) {
          DF& a = df_at(A, lp(3 * k + c, 3 * k2 + c));
          a = df_add(a, df_mul(wl, Lr[k2]));
        }
    }
  }
}

// ldlt_psd in double-float on the double-float H_r that span_form_df left in
// A: the same test (H_r + tau I positive definite, tau = neg_rel tr / n), its
// backward error about n 2^-46 tr(H_r) instead of n 2^-53 tr(H_r) - both far
// inside the projection's accuracy.  Destroys A.
template <int D>
__device__ __noinline__ bool ldlt_psd_df(const View& A, double neg_rel) {
  constexpr int n = 3 * D;
  DF tr{0.0f, 0.0f};
#pragma unroll
  for (int i = 0; i < n; ++i) tr = df_add(tr, df_at(A, lp(i, i)));
  // the factorisation forms no squares: only a trace far from 1 (2^+-60) is
  // brought to [1, 2) first, so that pivots and reciprocals stay normal (the
  // test does not depend on the scale)
  if (tr.h > 0.0f && isfinite(tr.h) && abs(ilogbf(tr.h)) > 60) {
    df_scale_unit<n * (n + 1) / 2>(A);
    tr = DF{0.0f, 0.0f};
#pragma unroll
    for (int i = 0; i < n; ++i) tr = df_add(tr, df_at(A, lp(i, i)));
  }
  if (!(tr.h > 0.0f) || !isfinite(tr.h)) return false;
  const float tau = (float)(neg_rel / n) * tr.h;
#pragma unroll 1
  for (int i = 0; i < n; ++i) {
    DF& a = df_at(A, lp(i, i));
    a = df_add(a, DF{tau, 0.0f});
  }
#pragma unroll 1
  for (int k = 0; k < n; ++k) {
    const DF dk = df_at(A, lp(k, k));
    if (!(dk.h > 0.0f) || !isfinite(dk.h)) return false;
    const DF r = df_rcp(dk);
#pragma unroll 1
    for (int i = k + 1; i < n; ++i) {
      const int ri = i * (i + 1) / 2;
      const DF l = df_neg(df_norm(df_mul(df_at(A, ri + k), r)));
#pragma unroll 1
      for (int j = k + 1; j <= i; ++j) {
        DF& a = df_at(A, ri + j);
        a = df_add(a, df_mul(l, df_at(A, j * (j + 1) / 2 + k)));
      }
    }
  }
  return true;
}
__device__ __forceinline__ double df_to_double(DF x) { return (double)x.h + (double)x.l; }
// sqrt(x), x > 0: the FP32 root corrected by its exact remainder (FMA)
__device__ __forceinline__ DF df_sqrt(DF x) {
  const float r = __fsqrt_rn(x.h);
  const float rem = __fadd_rn(__fmaf_rn(-r, r, x.h), x.l);
  return df_fast_two_sum(r, __fmul_rn(rem, __fmul_rn(0.5f, __frcp_rn(r))));
}

// Cascaded double-float sum (Ogita, Rump & Oishi, "Accurate sum and dot
// product", Sum2 / Dot2): the high parts add with one FP32 addition per term,
// the two-sum errors and the terms' low parts collect in a second FP32
// accumulator; one normalisation at the end.  As accurate as a double-float
// sum, with one dependent addition per term on the critical path.
struct DFAcc {
  float h = 0.0f, l = 0.0f;
  __device__ __forceinline__ void add(DF x) {
    const float s = __fadd_rn(h, x.h), bb = __fsub_rn(s, h);
    const float err = __fadd_rn(__fsub_rn(h, __fsub_rn(s, bb)), __fsub_rn(x.h, bb));
    l = __fadd_rn(l, __fadd_rn(err, x.l));
    h = s;
  }
  __device__ __forceinline__ DF result() const {
    const DF r = df_two_sum(h, l);
    return df_fast_two_sum(r.h, r.l);
  }
};

// span_tridiag in double-float on the double-float H_r that span_form_df left
// in A: the same Householder steps, the reflectors, tau and the tridiagonal
// then converted to FP64 (A and R as span_tridiag leaves them), so phase 2
// runs unchanged.  Each step is backward stable with unit roundoff about
// 2^-47, so the tridiagonal's eigenvalues lie within about n 2^-47 ||H_r||
// of H_r's.  The scaling and the inertia count run in FP64 as before.
template <int D>
__device__ __noinline__ int span_tridiag_df(const View& A, const View& R, double* tn_out, double neg_rel) {
  constexpr int n = 3 * D;
  constexpr int NP = n * (n + 1) / 2;
  // largest entry in [1, 2); the reflector pairs (v, tau) do not depend on
  // the scale, the tridiagonal is scaled back as it is stored
  const double unscale = (double)df_scale_unit<NP>(A);
#pragma unroll 1
  for (int k = 0; k < n - 2; ++k) {
    R[k] = df_to_double(df_at(A, lp(k, k))) * unscale;
    const DF x0 = df_at(A, lp(k + 1, k));
    DFAcc sacc;
#pragma unroll 2
    for (int i = k + 2; i < n; ++i) {
      const DF a = df_at(A, lp(i, k));
      sacc.add(df_mul(a, a));
    }
    const DF sigma = sacc.result();
    // a column below the subdiagonal at 2^-50 of the largest entry or less
    // (below the double-float rounding) is taken as zero, as the FP64
    // version takes an exact zero: no reflection
    if (sigma.h < 7.8886091e-31f /* 2^-100 */) {
      R[n + k] = df_to_double(x0) * unscale;
      df_at(A, lp(k, k)) = DF{0.0f, 0.0f};
      continue;
    }
    const DF nrm = df_sqrt(df_add(df_mul(x0, x0), sigma));
    const DF alpha = x0.h >= 0.0f ? df_neg(nrm) : nrm;
    const DF v0 = df_add(x0, df_neg(alpha));
    const DF r2 = df_rcp(df_add(df_mul(v0, v0), sigma));
    const DF t{2.0f * r2.h, 2.0f * r2.l};
    R[n + k] = df_to_double(alpha) * unscale;
    df_at(A, lp(k, k)) = t;
    df_at(A, lp(k + 1, k)) = v0;
    // p_i = t sum_j A(i, j) v_j over the trailing block, into R[2n + i]
#pragma unroll 1
    for (int i = k + 1; i < n; ++i) {
      DFAcc acc;
      const int ri = i * (i + 1) / 2;
#pragma unroll 2
      for (int j = k + 1; j <= i; ++j) acc.add(df_mul(df_at(A, ri + j), df_at(A, j * (j + 1) / 2 + k)));
#pragma unroll 2
      for (int j = i + 1; j < n; ++j) acc.add(df_mul(df_at(A, j * (j + 1) / 2 + i), df_at(A, j * (j + 1) / 2 + k)));
      df_at(R, 2 * n + i) = df_norm(df_mul(t, acc.result()));
    }
    DFAcc vacc;
#pragma unroll 2
    for (int i = k + 1; i < n; ++i) vacc.add(df_mul(df_at(A, i * (i + 1) / 2 + k), df_at(R, 2 * n + i)));
    const DF vp = vacc.result();
    const DF K = df_norm(df_mul(DF{0.5f * t.h, 0.5f * t.l}, vp));
#pragma unroll 1
    for (int i = k + 1; i < n; ++i) {  // w = p - K v
      DF& w = df_at(R, 2 * n + i);
      w = df_add(w, df_neg(df_mul(K, df_at(A, i * (i + 1) / 2 + k))));
    }
#pragma unroll 1
    for (int i = k + 1; i < n; ++i) {  // A -= v w^T + w v^T
      const DF vi = df_at(A, i * (i + 1) / 2 + k), wi = df_at(R, 2 * n + i);
      const int ri = i * (i + 1) / 2;
#pragma unroll 2
      for (int j = k + 1; j <= i; ++j) {
        DF& a = df_at(A, ri + j);
        DFAcc u;
        u.h = a.h;
        u.l = a.l;
        u.add(df_neg(df_mul(vi, df_at(R, 2 * n + j))));
        u.add(df_neg(df_mul(wi, df_at(A, j * (j + 1) / 2 + k))));
        a = u.result();
      }
    }
  }
  R[n - 2] = df_to_double(df_at(A, lp(n - 2, n - 2))) * unscale;
  R[n + n - 2] = df_to_double(df_at(A, lp(n - 1, n - 2))) * unscale;
  R[n - 1] = df_to_double(df_at(A, lp(n - 1, n - 1))) * unscale;
  R[2 * n - 1] = 0.0;
  // the reflectors and tau to FP64 in place (the other entries are not read again)
#pragma unroll 1
  for (int e = 0; e < NP; ++e) A[e] = df_to_double(df_at(A, e));

  // scale to ||T|| <= 1; e^2 -> R[2n..3n)
  double tn = 0.0;
#pragma unroll
  for (int i = 0; i < n; ++i) {
    const double r = fabs(R[i]) + fabs(R[n + i]) + (i > 0 ? fabs(R[n + i - 1]) : 0.0);
    tn = fmax(tn, r);
  }
  *tn_out = tn;
  if (!(tn > 0.0) || !isfinite(tn)) return isfinite(tn) ? 0 : -1;
  const double itn = 1.0 / tn;
#pragma unroll
  for (int i = 0; i < n; ++i) {
    const double ds = R[i] * itn, es = R[n + i] * itn;
    R[i] = ds;
    R[n + i] = es;
    R[2 * n + i] = es * es;
  }
  return sturm<n>(R, -neg_rel);
}

template <int D, class Tab>
__device__ __noinline__ int span_phase1_df(const Tab& tab, const View& A, const View& R, double* tn_out,
                                           double neg_rel) {
  span_form_df<D>(tab, A);
  return span_tridiag_df<D>(A, R, tn_out, neg_rel);
}
#endif  // __CUDACC__

// Phase 1 of a span: reduced Hessian (span_form), then span_tridiag.
template <int D, class Tab>
BSC_PHASE int span_phase1(const Tab& tab, const View& A, const View& R, double* tn_out, double neg_rel);

// Tridiagonal form and inertia of the reduced Hessian in A.  On return R
// holds the scaled tridiagonal (d, e, e^2), A the reflectors, *tn the
// scale; returns the number of eigenvalues below -neg_rel ||T|| (-1 on a
// non-finite matrix).
template <int D>
BSC_PHASE int span_tridiag(const View& A, const View& R, double* tn_out, double neg_rel) {
  constexpr int n = 3 * D;
  // 2. Householder tridiagonalisation: d -> R[0..n), e -> R[n..2n); the
  //    reflector v_k stays in column k of A, p = tau A v in R[2n..3n).
  //    Operands come from shared memory: the FP64 pipe, not the loads, is
  //    the limit, and no per-thread arrays compete for registers.
#pragma unroll 1
  for (int k = 0; k < n - 2; ++k) {
    R[k] = A[lp(k, k)];
    const double x0 = A[lp(k + 1, k)];
    double sigma = 0.0;
#pragma unroll 1
    for (int i = k + 2; i < n; ++i) {
      const double a = A[lp(i, k)];
      sigma += a * a;
    }
    if (sigma == 0.0) {
      R[n + k] = x0;
      A[lp(k, k)] = 0.0;
      continue;
    }
    const double nrm = sqrt(x0 * x0 + sigma);
    const double alpha = x0 >= 0.0 ? -nrm : nrm;
    const double v0 = x0 - alpha;
    const double t = 2.0 / (v0 * v0 + sigma);
    R[n + k] = alpha;
    A[lp(k, k)] = t;
    A[lp(k + 1, k)] = v0;
    // p_i = t sum_j A(i, j) v_j over the trailing block (rows of the lower triangle)
#pragma unroll 1
    for (int i = k + 1; i < n; ++i) {
      double acc = 0.0;
      const int ri = i * (i + 1) / 2;
#pragma unroll 1
      for (int j = k + 1; j <= i; ++j) acc += A[ri + j] * A[j * (j + 1) / 2 + k];
#pragma unroll 1
      for (int j = i + 1; j < n; ++j) acc += A[j * (j + 1) / 2 + i] * A[j * (j + 1) / 2 + k];
      R[2 * n + i] = t * acc;
    }
    double vp = 0.0;
#pragma unroll 1
    for (int i = k + 1; i < n; ++i) vp += A[i * (i + 1) / 2 + k] * R[2 * n + i];
    const double K = 0.5 * t * vp;
#pragma unroll 1
    for (int i = k + 1; i < n; ++i) R[2 * n + i] -= K * A[i * (i + 1) / 2 + k];  // w
#pragma unroll 1
    for (int i = k + 1; i < n; ++i) {
      const double vi = A[i * (i + 1) / 2 + k], wi = R[2 * n + i];
      const int ri = i * (i + 1) / 2;
#pragma unroll 1
      for (int j = k + 1; j <= i; ++j)  // A -= v w^T + w v^T as two FMAs per entry
        A[ri + j] = fma(-wi, A[j * (j + 1) / 2 + k], fma(-vi, R[2 * n + j], A[ri + j]));
    }
  }
  R[n - 2] = A[lp(n - 2, n - 2)];
  R[n + n - 2] = A[lp(n - 1, n - 2)];
  R[n - 1] = A[lp(n - 1, n - 1)];
  R[2 * n - 1] = 0.0;

  // 3. scale to ||T|| <= 1; e^2 -> R[2n..3n)
  double tn = 0.0;
#pragma unroll
  for (int i = 0; i < n; ++i) {
    const double r = fabs(R[i]) + fabs(R[n + i]) + (i > 0 ? fabs(R[n + i - 1]) : 0.0);
    tn = fmax(tn, r);
  }
  *tn_out = tn;
  if (!(tn > 0.0) || !isfinite(tn)) return isfinite(tn) ? 0 : -1;
  const double itn = 1.0 / tn;
#pragma unroll
  for (int i = 0; i < n; ++i) {
    const double ds = R[i] * itn, es = R[n + i] * itn;
    R[i] = ds;
    R[n + i] = es;
    R[2 * n + i] = es * es;
  }
  return sturm<n>(R, -neg_rel);
}

template <int D, class Tab>
BSC_PHASE int span_phase1(const Tab& tab, const View& A, const View& R, double* tn_out, double neg_rel) {
  span_form<D>(tab, A);
  return span_tridiag<D>(A, R, tn_out, neg_rel);
}

// ---------------------------------------------------------------------------
// Phase-2 items with the tridiagonal in registers (no shared memory needed):
// the span's scaled (d, e, e^2) are loaded once per item.
// ---------------------------------------------------------------------------

// Eigenvalue k (scaled) of the tridiagonal stored in R (d at R[0..n), e^2 at
// R[2n..3n)), loaded into registers.  After the FP32 bracket and its FP64
// check, a bracket that isolates eigenvalue k is refined by the Illinois
// variant of regula falsi on det(T - x I) (superlinear, bracketing), a
// bracket holding several eigenvalues by bisection.  Regula falsi stalls
// when an end of the bracket sits next to a multiple root of det(T - x I)
// (a padded basis adds a multiple zero eigenvalue): whenever four steps
// fail to halve the bracket together, the next step bisects, so the
// bracket shrinks at least by half every five steps.
template <int n>
BSC_PHASE double eigenvalue_reg(const View& R, int k, double neg_rel) {
  double d[n], e2[n];
#pragma unroll
  for (int i = 0; i < n; ++i) {
    d[i] = R[i];
    e2[i] = R[2 * n + i];
  }
  float d32[n], e232[n];
#pragma unroll
  for (int i = 0; i < n; ++i) {
    d32[i] = (float)d[i];
    e232[i] = (float)e2[i];
  }
  const double lo_all = -1.0 - 1e-12, hi_all = -neg_rel;
  float a32 = -1.0f - 1e-6f, b32 = (float)hi_all;
  bracket32<n>(d32, e232, k, &a32, &b32);
  double a = fmax((double)a32 - 4e-6, lo_all), b = fmin((double)b32 + 4e-6, hi_all);
  int ca, cb;
  bool xa, xb;
  double fa = char_poly<n>(d, e2, a, &ca, &xa), fb = char_poly<n>(d, e2, b, &cb, &xb);
  if (!(ca <= k && cb > k)) {
    a = lo_all;
    b = hi_all;
    fa = char_poly<n>(d, e2, a, &ca, &xa);
    fb = char_poly<n>(d, e2, b, &cb, &xb);
  }
  int side = 0, win = 0;
  bool force_bisect = false;
  double wstart = b - a;
#pragma unroll 1
  for (int it = 0; it < 120 && b - a > 1e-10; ++it) {
    double x;
    const bool isolated = ca == k && cb == k + 1 && xa && xb && fa != fb && !force_bisect;
    if (isolated) {
      x = (a * fb - b * fa) / (fb - fa);
      if (!(x > a && x < b)) x = 0.5 * (a + b);
    } else {
      x = 0.5 * (a + b);
      force_bisect = false;
      win = 0;
      wstart = b - a;
    }
    int cx;
    bool xx;
    const double fx = char_poly<n>(d, e2, x, &cx, &xx);
    if (cx > k) {
      if (isolated && side == -1) fa *= 0.5;  // Illinois: the kept end was kept twice
      b = x; fb = fx; cb = cx; xb = xx; side = -1;
    } else {
      if (isolated && side == 1) fb *= 0.5;
      a = x; fa = fx; ca = cx; xa = xx; side = 1;
    }
    if (isolated && fx == 0.0) return x;
    if (isolated && ++win == 4) {  // four regula-falsi steps must at least halve the bracket
      force_bisect = b - a > 0.5 * wstart;
      win = 0;
      wstart = b - a;
    }
#ifdef BSC_COUNT_EVALS
    ++bsc_evals;
#endif
  }
  return 0.5 * (a + b);
}

// Eigenvectors k0 .. k0+m-1 of a cluster (consecutive eigenvalues closer
// than the cluster gap), from the shifts in Lam: inverse iteration (two
// solves) with re-orthogonalisation against the cluster's earlier vectors in
// Ys, Rayleigh quotient (written back to Lam, unscaled by tn),
// back-transformation and w = (Q (x) I3) x written to Ws[27 k + .].  The
// tridiagonal (d, e) is loaded into registers from R; the reflectors A,
// basis Q, eigenvalues Lam and output vectors Ws are in global memory; Ys is
// the item's own scratch.  The LU factors of T - sigma I (multipliers and the three
// diagonals of U, 4n doubles) live in LU, the thread's slot of an interleaved
// shared-memory array, which keeps them out of local memory.
template <int D, class WView>
BSC_PHASE void cluster_vectors_reg(const View& R, const View& A, const View& Qs, const View& Ys, const View& Lam,
                                   const WView& Ws, const View& LU, double tn, int k0, int m) {
  constexpr int n = 3 * D;
  double d[n], e[n];
#pragma unroll
  for (int i = 0; i < n; ++i) {
    d[i] = R[i];
    e[i] = R[n + i];
  }
  const View mu{LU.p, LU.s}, u0r{LU.p + (long)n * LU.s, LU.s}, u1{LU.p + 2l * n * LU.s, LU.s},
      u2{LU.p + 3l * n * LU.s, LU.s};
#pragma unroll 1
  for (int k = k0; k < k0 + m; ++k) {
    const double sig = Lam[k];
    unsigned sw = 0u;
    {
      // Gaussian elimination of T - sig I with partial pivoting between
      // the current row (c0, c1, c2) and the next (e_i, a1, e1); the rows
      // are chosen by selects: one reciprocal per step whichever is taken.
      double c0 = d[0] - sig, c1 = e[0], c2 = 0.0;
#pragma unroll
      for (int i = 0; i < n - 1; ++i) {
        const double ei = e[i];
        const double a1 = d[i + 1] - sig, e1 = (i + 1 < n - 1) ? e[i + 1] : 0.0;
        const bool swp = fabs(ei) > fabs(c0);
        const double g0 = fabs(c0) < 2.3e-16 ? (c0 < 0.0 ? -2.3e-16 : 2.3e-16) : c0;
        const double t0 = swp ? ei : g0, t1 = swp ? a1 : c1, t2 = swp ? e1 : c2;  // pivot row
        const double b0 = swp ? c0 : ei, b1 = swp ? c1 : a1, b2 = swp ? c2 : e1;  // eliminated row
        const double r = 1.0 / t0, mm = b0 * r;
        sw |= (unsigned)swp << i;
        mu[i] = mm; u0r[i] = r; u1[i] = t1; u2[i] = t2;
        c0 = b1 - mm * t1; c1 = b2 - mm * t2; c2 = 0.0;
      }
      if (fabs(c0) < 2.3e-16) c0 = c0 < 0.0 ? -2.3e-16 : 2.3e-16;
      u0r[n - 1] = 1.0 / c0;
      u1[n - 1] = u2[n - 1] = 0.0;
    }
    double y[n];
#pragma unroll
    for (int i = 0; i < n; ++i) y[i] = 1.0 + 0.125 * (double)((7 * i + 3 * k) % 5);
    // a vector of its own (m == 1) needs no re-orthogonalisation: two
    // solves, one normalisation (the solves grow |y| by at most 1/2.3e-16
    // each, far inside the FP64 range); a cluster re-orthogonalises and
    // normalises after each solve and once more after the last
    const int passes = m > 1 ? 3 : 2;
#pragma unroll 1
    for (int it = 0; it < passes; ++it) {
#pragma unroll 1
      for (int j = k0; j < k; ++j) {
        double dt = 0.0;
#pragma unroll
        for (int i = 0; i < n; ++i) dt += Ys[(j - k0) * n + i] * y[i];
#pragma unroll
        for (int i = 0; i < n; ++i) y[i] -= dt * Ys[(j - k0) * n + i];
      }
      if (it < 2) {
#pragma unroll
        for (int i = 0; i < n - 1; ++i) {
          const bool swp = (sw >> i) & 1u;
          const double ya = swp ? y[i + 1] : y[i], yb = swp ? y[i] : y[i + 1];
          y[i] = ya;
          y[i + 1] = yb - mu[i] * ya;
        }
#pragma unroll
        for (int i = n - 1; i >= 0; --i) {
          double sacc = y[i];
          if (i + 1 < n) sacc -= u1[i] * y[i + 1];
          if (i + 2 < n) sacc -= u2[i] * y[i + 2];
          y[i] = sacc * u0r[i];
        }
      }
      if (m == 1 && it == 0) continue;
      double nn = 0.0;
#pragma unroll
      for (int i = 0; i < n; ++i) nn += y[i] * y[i];
      const double inv = 1.0 / sqrt(nn);
#pragma unroll
      for (int i = 0; i < n; ++i) y[i] *= inv;
    }
    double rq = 0.0;
#pragma unroll
    for (int i = 0; i < n; ++i) {
      double ty = d[i] * y[i];
      if (i > 0) ty += e[i - 1] * y[i - 1];
      if (i + 1 < n) ty += e[i] * y[i + 1];
      rq += y[i] * ty;
    }
    if (m > 1) {
#pragma unroll
      for (int i = 0; i < n; ++i) Ys[(k - k0) * n + i] = y[i];
    }
    Lam[k] = fmin(rq, 0.0) * tn;
    back_transform<n>(A, y);
#pragma unroll
    for (int l = 0; l < 9; ++l)
#pragma unroll
      for (int c = 0; c < 3; ++c) {
        double acc = 0.0;
#pragma unroll
        for (int kk = 0; kk < D; ++kk) acc += Qs[9 * kk + l] * y[3 * kk + c];
        Ws.set(27 * k + 3 * l + c, acc);
      }
  }
}

}  // namespace proj

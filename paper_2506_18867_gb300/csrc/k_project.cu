// K3: per-span PSD projection of the 27x27 elastic Hessian in FP64
// (projected Newton, Sec. 5.1): P = V max(Lambda, 0) V^T = H - sum_{lam<0}
// lam w w^T.
//
// The span Hessian is
//   H = sum_q (G_q (x) I3) A_q (G_q (x) I3)^T + sum_b W_b mu_bd (L_b L_b^T) (x) I3,
// so its range lies in R (x) R^3 with R = span{g_q,1, g_q,2, L_b} in R^9;
// every such vector sums to zero over the 9 control points (derivatives of a
// partition of unity), so dim R <= min(8, 2 n_mem + n_bd) =: D.  With an
// orthonormal basis Q of R, H = (Q (x) I3) H_r (Q (x) I3)^T and H_r (3D x 3D)
// has the same non-zero spectrum.  H_r is built from the per-point
// d^2 Psi/df^2 kept by the span evaluator, in FP64, and projected by
// proj::project_span (tridiagonalisation, Sturm bisection, inverse
// iteration).
//
// Interior spans (five derivative vectors, D = 5, n = 15).  A block takes
// BLOCK spans at a time from a work counter.  Phase 1 (one thread per span)
// builds H_r, tridiagonalises it and counts its negative eigenvalues.  The
// basis Q and the derivative vectors in it depend on the rest geometry only,
// so k_reduce_points computes them once per context (Gram-Schmidt for the
// interior spans, Helmert contrasts for the border spans).
// Phase 2a computes every negative eigenvalue of the batch as an independent
// item spread over the block; phase 2b computes the eigenvectors, one item
// per cluster of close eigenvalues.  Items are spread over all threads, so
// no warp carries masked lanes through FP64 work (masked lanes cost the FP64
// pipe as much as active ones) and no thread waits on another span's
// eigenvalue count.  Phase 3 applies the rank-k corrections of all spans in
// one fully parallel read-modify-write of the Hessian planes.  Working sets
// live in interleaved shared memory; eigenvalues, eigenvectors and w vectors
// in the class scratch.  The border spans run concurrently on a forked
// stream (k_project_ring, or the phase kernels with D = 8).
#include "bsc_internal.cuh"
#include <type_traits>

#include "proj_core.cuh"

cudaError_t setup_projection_ring();
cudaError_t launch_project_ring(bsc_ctx* c, int first, int count, unsigned int* work, cudaStream_t st, bool p1only,
                                double* sspan, int* kneg, bool two_pass = false);


namespace {

template <typename T>
struct ProjArgs {
  int Nsp, Nm, Nb;
  const PatchDev* __restrict__ pd;     // bending stiffness of each patch
  const int* __restrict__ sp_patch;    // patch of each span
  const int* __restrict__ moff;
  const int* __restrict__ boff;
  const T* __restrict__ tabm;
  const T* __restrict__ tabb;
  const T* __restrict__ A;
  T* __restrict__ H;
  int* __restrict__ nneg;
  int* __restrict__ status;
  const double* __restrict__ rg;  // [16][Nm] membrane derivative vectors in the span's reduced basis
  const double* __restrict__ rl;  // [8][Nb] bending vectors in the span's reduced basis
  const double* __restrict__ rq;  // the class's bases: [9 D][count] per span, or one 9 x 8 basis
  int rq_per_span;                // 1: rq holds a basis per span (class order)
  // FP32 contexts: rg and rl as double-float splits (hi, lo), for the
  // double-float formation of the PSD test
  const float2* __restrict__ rg2;
  const float2* __restrict__ rl2;
  int df;  // p0 and p1 in double-float (bsc_set_proj_arith)
};

// Eigenvalues below -NEG_REL * ||T|| are projected; above that they are
// rounding noise of exact zeros (their contribution is below 1e-14 ||H||).
constexpr double NEG_REL = 1e-14;
// The same threshold after the double-float phase 1: its rounding leaves the
// exact zero eigenvalues of a rank-deficient span (border spans in the
// Helmert basis) at up to some 1e-13 ||T||, so eigenvalues are counted below
// -1e-12 ||T|| there; the few between -1e-12 and -1e-14 ||T|| stay (their
// clamping would change the span by less than 1e-12 ||H||).
constexpr double NEG_REL_DF = 1e-12;
// A basis candidate whose residual after orthogonalisation is below
// RANK_REL of its norm lies in the span of the previous ones.
constexpr double RANK_REL = 1e-13;

template <typename T>
struct SpanTab {
  const T* tabm;     // already offset to the span's first membrane point
  const T* tabb;     // already offset to the span's first bending point
  const T* A;
  const double* rg;  // reduced vectors, offset like tabm / tabb
  const double* rl;
  int Nm, Nb, nmq, nbq;
  double mubd;
  __device__ int nm() const { return nmq; }
  __device__ int nb() const { return nbq; }
  __device__ double g(int q, int l, int be) const { return (double)tabm[(1 + 2 * l + be) * Nm + q]; }
  __device__ double L(int q, int l) const { return (double)tabb[(1 + l) * Nb + q]; }
  __device__ double wb(int q) const { return (double)tabb[q] * mubd; }
  __device__ double a6(int q, int e) const { return (double)A[e * Nm + q]; }
  __device__ double gr(int q, int k, int be) const { return rg[(size_t)(2 * k + be) * Nm + q]; }
  __device__ double lr(int q, int k) const { return rl[(size_t)k * Nb + q]; }
};

// SpanTab with the double-float inputs of span_form_df: the reduced vectors
// as double-float splits; the tables' FP32 entries (FP32 contexts) are exact,
// FP64 ones (FP64 contexts) are split as they are read.
template <typename T>
struct SpanTabDF {
  static constexpr bool kFloatA6 = std::is_same<T, float>::value;
  const T* tabb;       // offset to the span's first bending point
  const T* A;          // offset to the span's first membrane point
  const float2* rg2;   // offset like A
  const float2* rl2;   // offset like tabb
  int Nm, Nb, nmq, nbq;
  double mubd;         // the patch's bending modulus
  proj::DF mu;         // and as a double-float
  __device__ int nm() const { return nmq; }
  __device__ int nb() const { return nbq; }
  __device__ proj::DF a6(int q, int e) const {
    if constexpr (kFloatA6) return {(float)A[e * Nm + q], 0.0f};
    else return proj::df_split((double)A[e * Nm + q]);
  }
  __device__ proj::DF gr2(int q, int k, int be) const {
    const float2 v = rg2[(size_t)(2 * k + be) * Nm + q];
    return {v.x, v.y};
  }
  __device__ proj::DF lr2(int q, int k) const {
    const float2 v = rl2[(size_t)k * Nb + q];
    return {v.x, v.y};
  }
  __device__ proj::DF wb2(int q) const {
    if constexpr (kFloatA6) return proj::df_mul_f(mu, (float)tabb[q]);
    else return proj::df_split((double)tabb[q] * mubd);
  }
};
template <typename T>
__device__ __forceinline__ SpanTabDF<T> span_tab_df(const ProjArgs<T>& P, int s) {
  const int q0 = P.moff[s], b0 = P.boff[s];
  const double mubd = P.pd[P.sp_patch[s]].mubd;
  return SpanTabDF<T>{P.tabb + b0, P.A + q0, P.rg2 + q0, P.rl2 + b0, P.Nm, P.Nb, P.moff[s + 1] - q0,
                      P.boff[s + 1] - b0, mubd, proj::df_split(mubd)};
}

// Helmert contrasts q_k = (1, ..., 1, -k, 0, ...) / sqrt(k (k + 1)) (k ones),
// k = 1..8: an orthonormal basis of the vectors of R^9 that sum to zero, the
// reduced basis of every border span.
__device__ double d_helmert[72];

// Shared memory per thread of phase 1: A (packed H_r, then reflectors) and
// R (3n: the scaled tridiagonal), interleaved by thread.
template <int D>
struct Smem {
  static constexpr int n = 3 * D, NP = n * (n + 1) / 2;
};

// Per-span scratch of a class (global memory, entry-major over the span's
// position in the class list): reflectors + tau (packed A), scaled
// tridiagonal (d, e, e^2), scale ||T||, eigenvalues, and the span-DOF
// vectors w of the negative eigenpairs.
template <int D>
struct SpanScratch {
  static constexpr int n = 3 * D, NP = n * (n + 1) / 2;
  static constexpr int A = 0, R = NP, TN = R + 3 * n, LAM = TN + 1, W = LAM + n, SIZE = W + 27 * n;
};

// Eigenvalues of a span closer than this (on the tridiagonal scaled to
// ||T|| <= 1) form a cluster whose eigenvectors are orthogonalised
// explicitly; farther apart, inverse iteration alone leaves them orthogonal
// to about eps / gap.
constexpr double CLUSTER_GAP = 1e-3;

// Threads per block of phase 1 (packed H_r and R of every thread in shared
// memory: 8 x (NP + 3 n) bytes each) and of phase 2.
template <int D> struct P1Block;
template <> struct P1Block<5> { static constexpr int value = 160; };  // 211 KB of shared memory
template <> struct P1Block<8> { static constexpr int value = 64; };   // 190 KB
constexpr int P2_BLOCK = 128;

// Strided view of element type T over the scratch (w vectors, lam w).
template <typename T>
struct TView {
  T* p;
  int s;
  __device__ __forceinline__ void set(int i, double v) const { p[(size_t)i * s] = (T)v; }
  __device__ __forceinline__ T operator[](int i) const { return p[(size_t)i * s]; }
};

// Phase 3: H -= sum_r lam_r w_r w_r^T for every span of a class, one thread
// per (row a of the packed upper triangle, span position): lam_r w_r[a] in
// registers, then the row's entries (a, c), c >= a, eight at a time with
// their reads of H and w issued together.  Consecutive threads take consecutive
// spans of a row, so every access is coalesced; the update is a parallel
// read-modify-write of the Hessian planes, bound by HBM.
template <typename T>
__global__ void __launch_bounds__(256)
    k_proj_corr(const int* __restrict__ cnt, int cs_, int Nsp, const int* __restrict__ list,
                const int* __restrict__ sel, const int* __restrict__ kneg_in, const double* __restrict__ lam,
                const T* __restrict__ W, T* __restrict__ H) {
  constexpr int RM = 8;  // negative eigenvalues kept in registers (more go through the loop below)
  constexpr int CW = 8;  // entries of a row per step
  const int count = *cnt;
  const size_t cs = (size_t)cs_;
  for (long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x; t < 27ll * count;
       t += (long long)gridDim.x * blockDim.x) {
  const int a = (int)(t / count), pos = (int)(t - (long long)a * count);
  const int kneg = kneg_in[pos];
  if (kneg == 0) continue;
  const int s = list[sel ? sel[pos] : pos];
  T la[RM];
#pragma unroll
  for (int r = 0; r < RM; ++r) la[r] = r < kneg ? (T)lam[r * cs + pos] * W[(27 * r + a) * cs + pos] : T(0);
  T* __restrict__ h = H + s;
  const int e0 = a * 27 - (a * (a - 1)) / 2;  // packed index of (a, a)
#pragma unroll 1
  for (int c0 = a; c0 < 27; c0 += CW) {
    T hv[CW], acc[CW];
#pragma unroll
    for (int u = 0; u < CW; ++u) {
      const int c = c0 + u;
      hv[u] = c < 27 ? h[(size_t)(e0 + c - a) * Nsp] : T(0);
      acc[u] = T(0);
#pragma unroll
      for (int r = 0; r < RM; ++r)
        if (r < kneg && c < 27) acc[u] += la[r] * W[(27 * r + c) * cs + pos];
    }
    for (int r = RM; r < kneg; ++r) {  // rare: more than RM negative eigenvalues
      const T lr = (T)lam[r * cs + pos] * W[(27 * r + a) * cs + pos];
#pragma unroll
      for (int u = 0; u < CW; ++u)
        if (c0 + u < 27) acc[u] += lr * W[(27 * r + c0 + u) * cs + pos];
    }
#pragma unroll
    for (int u = 0; u < CW; ++u)
      if (c0 + u < 27) h[(size_t)(e0 + c0 + u - a) * Nsp] = hv[u] - acc[u];
  }
  }
}

template <int BLOCK>
__device__ __forceinline__ void block_prefix(int v, int* prefix, int* wsum);

// Phase 1: one thread per interior span (uniform work, no barriers).
// The spans are list[sel[t]] for t < *cnt (sel == nullptr: list[t]); the
// scratch is indexed by t with stride cs (the class size).
template <typename T, int D>
__global__ void __launch_bounds__(P1Block<D>::value, 1)
    k_proj_p1(ProjArgs<T> P, const int* __restrict__ list, const int* __restrict__ sel, const int* __restrict__ cnt,
              int cs, double* __restrict__ sspan, int* __restrict__ kneg_out) {
  constexpr int n = 3 * D, NP = n * (n + 1) / 2, B1 = P1Block<D>::value;
  using SS = SpanScratch<D>;
  extern __shared__ __align__(16) double smd[];
  const proj::View A{smd + threadIdx.x, B1};
  const proj::View R{smd + (size_t)NP * B1 + threadIdx.x, B1};
  const int count = *cnt;
  for (int t = blockIdx.x * B1 + threadIdx.x; t < count; t += gridDim.x * B1) {
    const int s = list[sel ? sel[t] : t];
    const int q0 = P.moff[s], b0 = P.boff[s];
    double tn = 0.0;
    int kneg;
    if (P.df) {
      // formation and tridiagonal form in double-float on the FP32 pipe
      kneg = proj::span_phase1_df<D>(span_tab_df<T>(P, s), A, R, &tn, NEG_REL_DF);
    } else {
      SpanTab<T> tab{P.tabm + q0, P.tabb + b0, P.A + q0, P.rg + q0, P.rl + b0, P.Nm, P.Nb, P.moff[s + 1] - q0,
                     P.boff[s + 1] - b0, P.pd[P.sp_patch[s]].mubd};
      kneg = proj::span_phase1<D>(tab, A, R, &tn, NEG_REL);
    }
    if (kneg < 0) {
      atomicOr(P.status, BSC_STATUS_NUMERIC_FLAG);
      kneg = 0;
    }
    kneg_out[t] = kneg;
    P.nneg[s] = kneg;
    if (kneg > 0) {
#pragma unroll 1
      for (int e = 0; e < NP; ++e) sspan[(size_t)(SS::A + e) * cs + t] = A[e];
#pragma unroll 1
      for (int e = 0; e < 3 * n; ++e) sspan[(size_t)(SS::R + e) * cs + t] = R[e];
      sspan[(size_t)SS::TN * cs + t] = tn;
    }
  }
}

// Phase 0a (interior spans): an FP32 certificate of positive definiteness.
// With u = 2^-24 and gamma_k = k u / (1 - k u):
//  - forming H_r in FP32 errs in every entry by at most gamma_16 times the
//    sum of the absolute values of the entry's three-factor terms: a term
//    meets at most 3 roundings of its inputs (to FP32), 2 in T_k, and one per
//    accumulation into the entry, 2 n_mem + n_bd <= 5 in the interior class
//    (spans with more return "open"); the Frobenius norm of those absolute
//    sums is at most
//      S = sum_q 3 ||g_q||^2 ||A6_q||_F + sum_b 3 W_b ||L_b||^2
//    (|M^T A M| <= |M|^T |A| |M| entrywise, ||M||_F^2 = 3 ||g_q||^2), so
//    ||H_r - Â||_2 <= gamma_16 S;
//  - an LDL^T factorisation in FP32 (multipliers by a correctly rounded
//    reciprocal of the pivot, then a product: two roundings) that ends with
//    every pivot positive is Gaussian elimination with computed factors L and
//    U, L U = X + F, |F| <= gamma_{n+1} |L| |U| (Higham, Accuracy and
//    Stability of Numerical Algorithms, 2nd ed., Thm. 9.3, one rounding more
//    per multiplier), and U = D L^T entrywise up to 1 + theta, |theta| <=
//    gamma_2; so X = L D L^T + E with |E| <= gamma_{n+4} |L| D |L^T|, and
//    ||E||_2 <= gamma_{n+4} tr(L D L^T) = gamma_{n+4} tr(X + E), that is at
//    most gamma_{n+4} tr(X) / (1 - gamma_{n+4}) (the diagonal of |L| D |L^T|
//    is that of L D L^T when D > 0).
// Factoring X = Â - sigma I with sigma = 1.1 (gamma_{n+4} tr Â + gamma_16 S)
// (the tenth covers the rounding of the shift, u (S + sigma), and of tr Â and
// S): if every pivot is positive, H_r = L D L^T + sigma I - E + (H_r - Â) has
// every eigenvalue above a positive margin of a few 1e-8 tr(H_r).  Such a
// span has no negative eigenvalue, and the FP64 test, whose margin is 1e-14
// tr / n and whose own rounding is some 1e-15 tr, would pass it as well:
// taking the certificate instead changes no span's result.  The spans it cannot decide
// (their class positions appended to pre_out) go on to the FP64 test.
constexpr int PF_BLOCK = 128;

// The certificate with H_r in registers: every loop over matrix indices is
// unrolled, so each packed entry is a register and the factorisation runs
// without memory traffic (the open spans' class positions go out through
// shared-memory prefix sums only).
template <int D, class Tab>
__device__ __forceinline__ bool certify_pd_f32(const Tab& tab) {
  constexpr int n = 3 * D, NP = n * (n + 1) / 2;
  constexpr float u = 5.9604644775390625e-8f;  // 2^-24
  constexpr float g_n4 = (n + 4) * u / (1.0f - (n + 4) * u), g_16 = 16 * u / (1.0f - 16 * u);
  float A[NP];
#pragma unroll
  for (int k = 0; k < NP; ++k) A[k] = 0.0f;
  const int nm = tab.nm(), nb = tab.nb();
  if (2 * nm + nb > D) return false;  // outside the rounding count above
  float S = 0.0f;
#pragma unroll 1
  for (int q = 0; q < nm; ++q) {
    float gr[D][2], g2 = 0.0f;
#pragma unroll
    for (int k = 0; k < D; ++k)
#pragma unroll
      for (int b = 0; b < 2; ++b) {
        gr[k][b] = (float)tab.gr(q, k, b);
        g2 = fmaf(gr[k][b], gr[k][b], g2);
      }
    float A6[6][6], a2 = 0.0f;
    {
      int e = 0;
#pragma unroll
      for (int r = 0; r < 6; ++r)
#pragma unroll
        for (int c = r; c < 6; ++c) {
          const float v = (float)tab.a6(q, e++);
          A6[r][c] = v;
          A6[c][r] = v;
          a2 = fmaf(r == c ? v : 2.0f * v, v, a2);
        }
    }
    S = fmaf(3.0f * g2, __fsqrt_ru(a2), S);
#pragma unroll
    for (int k = 0; k < D; ++k) {
      float Tk[3][6];
#pragma unroll
      for (int c = 0; c < 3; ++c)
#pragma unroll
        for (int j = 0; j < 6; ++j) Tk[c][j] = fmaf(gr[k][1], A6[3 + c][j], gr[k][0] * A6[c][j]);
#pragma unroll
      for (int k2 = 0; k2 <= k; ++k2)
#pragma unroll
        for (int c = 0; c < 3; ++c)
#pragma unroll
          for (int dd = 0; dd < 3; ++dd) {
            if (k2 == k && dd > c) continue;
            float& a = A[proj::lp(3 * k + c, 3 * k2 + dd)];
            a = fmaf(Tk[c][3 + dd], gr[k2][1], fmaf(Tk[c][dd], gr[k2][0], a));
          }
    }
  }
#pragma unroll 1
  for (int q = 0; q < nb; ++q) {
    const float WB = (float)tab.wb(q);
    float Lr[D], l2 = 0.0f;
#pragma unroll
    for (int k = 0; k < D; ++k) {
      Lr[k] = (float)tab.lr(q, k);
      l2 = fmaf(Lr[k], Lr[k], l2);
    }
    S = fmaf(3.0f * fabsf(WB), l2, S);
#pragma unroll
    for (int k = 0; k < D; ++k) {
      const float wl = WB * Lr[k];
#pragma unroll
      for (int k2 = 0; k2 <= k; ++k2)
#pragma unroll
        for (int c = 0; c < 3; ++c) {
          float& a = A[proj::lp(3 * k + c, 3 * k2 + c)];
          a = fmaf(wl, Lr[k2], a);
        }
    }
  }
  float tr = 0.0f;
#pragma unroll
  for (int i = 0; i < n; ++i) tr += A[proj::lp(i, i)];
  if (!(tr > 0.0f) || !isfinite(tr) || !isfinite(S)) return false;
  const float sigma = 1.1f * (g_n4 * tr + g_16 * S);
#pragma unroll
  for (int i = 0; i < n; ++i) A[proj::lp(i, i)] -= sigma;
  // right-looking LDL^T on the packed lower triangle: a(i, j) -= l_ik a(j, k),
  // l_ik = a(i, k) / d_k; the multipliers are not kept
  bool ok = true;
#pragma unroll
  for (int k = 0; k < n; ++k) {
    const float d = A[proj::lp(k, k)];
    ok = ok && (d > 0.0f) && isfinite(d);
    const float r = __frcp_rn(d);
#pragma unroll
    for (int i = k + 1; i < n; ++i) {
      const float l = A[proj::lp(i, k)] * r;
#pragma unroll
      for (int j = k + 1; j <= i; ++j) A[proj::lp(i, j)] = fmaf(-l, A[proj::lp(j, k)], A[proj::lp(i, j)]);
    }
  }
  return ok;
}

template <typename T, int D>
__global__ void __launch_bounds__(PF_BLOCK, 2)
    k_proj_pf(ProjArgs<T> P, const int* __restrict__ list, int count, int* __restrict__ pre_out,
              int* __restrict__ pre_count) {
  __shared__ int s_pre[PF_BLOCK + 1], s_wsum[PF_BLOCK / 32], s_base;
  for (int chunk = blockIdx.x; chunk * PF_BLOCK < count; chunk += gridDim.x) {
    const int t = chunk * PF_BLOCK + threadIdx.x;
    int open = 0;
    if (t < count) {
      const int s = list[t];
      const int q0 = P.moff[s], b0 = P.boff[s];
      SpanTab<T> tab{P.tabm + q0, P.tabb + b0, P.A + q0, P.rg + q0, P.rl + b0, P.Nm, P.Nb, P.moff[s + 1] - q0,
                     P.boff[s + 1] - b0, P.pd[P.sp_patch[s]].mubd};
      if (certify_pd_f32<D>(tab)) P.nneg[s] = 0;
      else open = 1;
    }
    block_prefix<PF_BLOCK>(open, s_pre, s_wsum);
    if (threadIdx.x == 0) s_base = s_pre[PF_BLOCK] > 0 ? (int)atomicAdd(pre_count, s_pre[PF_BLOCK]) : 0;
    __syncthreads();
    if (open) pre_out[s_base + s_pre[threadIdx.x]] = t;
    __syncthreads();
  }
}

// Phase 0b (the PSD test, interior spans): one thread per span forms H_r and
// runs the FP64 LDL^T test of proj::ldlt_psd, on the class positions pre[0
// .. *pre_count) the certificate left open (every span of the class when
// pre is null: then count spans in class order).  Spans that pass keep their
// Hessian (nneg = 0); the class positions of the others are appended to
// sel_out (block by block: the order of the blocks' groups varies from run
// to run, the per-span results do not), and the later phases run on that
// list only, so no warp carries the eigendecomposition of one span while
// its other lanes idle.
template <int D> struct P0Block;
template <> struct P0Block<5> { static constexpr int value = 224; };  // 224 x 120 doubles = 210 KB
template <> struct P0Block<8> { static constexpr int value = 64; };   // 64 x 300 doubles = 150 KB
template <typename T, int D>
__global__ void __launch_bounds__(P0Block<D>::value, 1)
    k_proj_p0(ProjArgs<T> P, const int* __restrict__ list, int count, const int* __restrict__ pre,
              const int* __restrict__ pre_count, int* __restrict__ sel_out, int* __restrict__ sel_count) {
  constexpr int B0 = P0Block<D>::value;
  extern __shared__ __align__(16) double smd[];
  __shared__ int s_pre[B0 + 1], s_wsum[B0 / 32], s_base;
  const proj::View A{smd + threadIdx.x, B0};
  const int m = pre ? *pre_count : count;
  for (int chunk = blockIdx.x; chunk * B0 < m; chunk += gridDim.x) {
    const int i = chunk * B0 + threadIdx.x;
    int fail = 0, t = 0;
    if (i < m) {
      t = pre ? pre[i] : i;
      const int s = list[t];
      const int q0 = P.moff[s], b0 = P.boff[s];
      if (P.df) {
        // formation and test in double-float on the FP32 pipe
        proj::span_form_df<D>(span_tab_df<T>(P, s), A);
        fail = proj::ldlt_psd_df<D>(A, NEG_REL) ? 0 : 1;
      } else {
        const int q0 = P.moff[s], b0 = P.boff[s];
        SpanTab<T> tab{P.tabm + q0, P.tabb + b0, P.A + q0, P.rg + q0, P.rl + b0, P.Nm, P.Nb, P.moff[s + 1] - q0,
                       P.boff[s + 1] - b0, P.pd[P.sp_patch[s]].mubd};
        proj::span_form<D>(tab, A);
        fail = proj::ldlt_psd<D>(A, NEG_REL) ? 0 : 1;
      }
      if (!fail) P.nneg[s] = 0;
    }
    block_prefix<B0>(fail, s_pre, s_wsum);
    if (threadIdx.x == 0) s_base = s_pre[B0] > 0 ? (int)atomicAdd(sel_count, s_pre[B0]) : 0;
    __syncthreads();
    if (fail) sel_out[s_base + s_pre[threadIdx.x]] = t;
    __syncthreads();
  }
}

// Finds the owner of item i given an exclusive prefix over the block.
template <int BLOCK>
__device__ __forceinline__ int owner_of(const int* prefix, int i) {
  int lo = 0, hi = BLOCK;  // prefix[lo] <= i < prefix[hi]
  while (hi - lo > 1) {
    const int mid = (lo + hi) >> 1;
    if (prefix[mid] <= i) lo = mid;
    else hi = mid;
  }
  return lo;
}

template <int BLOCK>
__device__ __forceinline__ void block_prefix(int v, int* prefix, int* wsum) {
  // exclusive prefix of v over the block into prefix[0..BLOCK], total in prefix[BLOCK]
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  int x = v;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const int y = __shfl_up_sync(0xffffffffu, x, o);
    if (lane >= o) x += y;
  }
  if (lane == 31) wsum[warp] = x;
  __syncthreads();
  int off = 0;
#pragma unroll
  for (int w = 0; w < BLOCK / 32; ++w) off += (w < warp) ? wsum[w] : 0;
  prefix[threadIdx.x] = off + x - v;
  if (threadIdx.x == BLOCK - 1) prefix[BLOCK] = off + x;
  __syncthreads();
}

// Spans per phase-2 batch: the whole block for the interior class; a quarter
// for the border class, whose few spans (a thousand or two in a large patch)
// would otherwise fill only a few blocks with several items per thread.
__host__ __device__ constexpr int p2_spans(int D) { return D == 5 ? P2_BLOCK : P2_BLOCK / 4; }

// Phase-2 occupancy variants: MINB resident blocks per SM (2: no register
// limit below 255; 3: 168 registers, a little spilling in the eigenvector
// item).  The autotuner keeps the faster for the interior class.
constexpr int P2_MINB[2] = {2, 3};

// Phase 2 over batches of SB consecutive spans of a class: (a) every
// negative eigenvalue is an independent item, (b) every cluster of close
// eigenvalues is an item that computes its eigenvectors; the eigenvalues and
// w vectors go to the class scratch, and phase 3 (k_proj_corr) applies
// H -= sum lam w w^T.  Items are spread over the whole block, so no warp
// carries masked lanes through FP64 work (masked lanes cost the FP64 pipe as
// much as active ones).
template <typename T, int D, int MINB, int SB = p2_spans(D)>
__global__ void __launch_bounds__(P2_BLOCK, MINB)
    k_proj_p2(ProjArgs<T> P, const int* __restrict__ list, const int* __restrict__ sel, const int* __restrict__ cnt,
              int cs, const int* __restrict__ kneg_in, double* __restrict__ sspan, double* __restrict__ slots,
              unsigned int* __restrict__ work) {
  constexpr int n = 3 * D;
  using SS = SpanScratch<D>;
  const int count = *cnt;
  __shared__ int s_kneg[P2_BLOCK], s_cl[P2_BLOCK], s_pre[P2_BLOCK + 1], s_wsum[P2_BLOCK / 32];
  __shared__ int s_base;
  extern __shared__ __align__(16) double s_lu[];  // [4 n][P2_BLOCK]: LU factors of the inverse iteration
  const int tid = threadIdx.x;
  const int nslots = gridDim.x * P2_BLOCK;
  const proj::View Ys{slots + blockIdx.x * P2_BLOCK + tid, nslots};
  const proj::View LU{s_lu + tid, P2_BLOCK};
  auto sv = [&](int t, int off) { return proj::View{sspan + (size_t)off * cs + t, cs}; };
  auto wv = [&](int t) { return TView<T>{reinterpret_cast<T*>(sspan + (size_t)SS::W * cs) + t, cs}; };
  for (;;) {
    if (tid == 0) s_base = (int)atomicAdd(work, (unsigned)SB);
    __syncthreads();
    const int base = s_base;
    if (base >= count) break;
    const int t = base + tid;
    const int kneg = (tid < SB && t < count) ? kneg_in[t] : 0;
    s_kneg[tid] = kneg;
    // (a) eigenvalues
    block_prefix<P2_BLOCK>(kneg, s_pre, s_wsum);
    for (int i = tid; i < s_pre[P2_BLOCK]; i += P2_BLOCK) {
      const int o = owner_of<P2_BLOCK>(s_pre, i), r = i - s_pre[o], to = base + o;
      sv(to, SS::LAM)[r] = proj::eigenvalue_reg<n>(sv(to, SS::R), r, NEG_REL);
    }
    __syncthreads();
    // clusters: bit r of s_cl marks an eigenvalue that starts one
    int ncl = 0;
    if (kneg > 0) {
      const proj::View Lam = sv(t, SS::LAM);
      unsigned mask = 1u;
      double prev = Lam[0];
      for (int r = 1; r < kneg; ++r) {
        const double lr = Lam[r];
        if (lr - prev > CLUSTER_GAP) mask |= 1u << r;
        prev = lr;
      }
      s_cl[tid] = (int)mask;
      ncl = __popc(mask);
    } else {
      s_cl[tid] = 0;
    }
    // (b) eigenvectors, one item per cluster
    block_prefix<P2_BLOCK>(ncl, s_pre, s_wsum);
    for (int i = tid; i < s_pre[P2_BLOCK]; i += P2_BLOCK) {
      const int o = owner_of<P2_BLOCK>(s_pre, i), c = i - s_pre[o], to = base + o;
      unsigned mm = (unsigned)s_cl[o];
      for (int z = 0; z < c; ++z) mm &= mm - 1u;  // drop the first c starts
      const int k0 = __ffs(mm) - 1;
      const unsigned rest = mm & (mm - 1u);
      const int k1 = rest ? __ffs(rest) - 1 : s_kneg[o];
      const int tc = sel ? sel[to] : to;  // the span's position in its class (its basis)
      const proj::View Qs = P.rq_per_span ? proj::View{const_cast<double*>(P.rq) + tc, cs}
                                          : proj::View{const_cast<double*>(P.rq), 1};
      proj::cluster_vectors_reg<D>(sv(to, SS::R), sv(to, SS::A), Qs, Ys, sv(to, SS::LAM), wv(to), LU,
                                   sspan[(size_t)SS::TN * cs + to], k0, k1 - k0);
    }
    __syncthreads();
  }
}

template <typename T>
ProjArgs<T> proj_args(bsc_ctx* c, int k) {
  ProjArgs<T> P;
  P.Nsp = c->Nsp; P.Nm = c->Nmem; P.Nb = c->Nbd; P.pd = c->pd; P.sp_patch = c->sp_patch;
  P.moff = c->mem_off; P.boff = c->bd_off;
  P.tabm = (const T*)c->tab_mem; P.tabb = (const T*)c->tab_bd;
  P.A = (const T*)c->A_mem; P.H = (T*)c->H_span;
  P.nneg = c->nneg; P.status = c->dstatus;
  P.rg = c->red_g; P.rl = c->red_l;
  P.rg2 = c->red_g2; P.rl2 = c->red_l2;
  P.df = c->proj_df;
  P.rq = k == 0 ? c->red_q : c->helmert;
  P.rq_per_span = k == 0 ? 1 : 0;
  return P;
}

// Reduced basis and reduced derivative vectors of every span (thread per
// position t of the bucket list): interior spans (t < n0) by Gram-Schmidt
// (basis stored in class order), border spans in the Helmert basis.
template <typename T>
__global__ void __launch_bounds__(128)
    k_reduce_points(ProjArgs<T> P, const int* __restrict__ list, int n0, int count, double* __restrict__ rq,
                    double* __restrict__ rg, double* __restrict__ rl, float2* __restrict__ rg2,
                    float2* __restrict__ rl2) {
  for (int t = blockIdx.x * blockDim.x + threadIdx.x; t < count; t += gridDim.x * blockDim.x) {
    const int s = list[t];
    const int q0 = P.moff[s], b0 = P.boff[s];
    const SpanTab<T> tab{P.tabm + q0, P.tabb + b0, P.A + q0, nullptr, nullptr, P.Nm, P.Nb, P.moff[s + 1] - q0,
                         P.boff[s + 1] - b0, 0.0};
    double Q[72];
    int D = 8;
    if (t < n0) {
      D = 5;
      proj::span_basis<5>(tab, proj::View{Q, 1}, RANK_REL);
      for (int e = 0; e < 45; ++e) rq[(size_t)e * n0 + t] = Q[e];
    } else {
      for (int e = 0; e < 72; ++e) Q[e] = d_helmert[e];
    }
    for (int q = 0; q < tab.nm(); ++q)
      for (int k = 0; k < D; ++k) {
        double a0 = 0.0, a1 = 0.0;
#pragma unroll
        for (int l = 0; l < 9; ++l) {
          a0 += Q[9 * k + l] * tab.g(q, l, 0);
          a1 += Q[9 * k + l] * tab.g(q, l, 1);
        }
        rg[(size_t)(2 * k) * P.Nm + q0 + q] = a0;
        rg[(size_t)(2 * k + 1) * P.Nm + q0 + q] = a1;
        if (rg2) {
          const proj::DF s0 = proj::df_split(a0), s1 = proj::df_split(a1);
          rg2[(size_t)(2 * k) * P.Nm + q0 + q] = make_float2(s0.h, s0.l);
          rg2[(size_t)(2 * k + 1) * P.Nm + q0 + q] = make_float2(s1.h, s1.l);
        }
      }
    for (int q = 0; q < tab.nb(); ++q)
      for (int k = 0; k < D; ++k) {
        double a = 0.0;
#pragma unroll
        for (int l = 0; l < 9; ++l) a += Q[9 * k + l] * tab.L(q, l);
        rl[(size_t)k * P.Nb + b0 + q] = a;
        if (rl2) {
          const proj::DF sa = proj::df_split(a);
          rl2[(size_t)k * P.Nb + b0 + q] = make_float2(sa.h, sa.l);
        }
      }
  }
}

template <typename T>
cudaError_t reduce_points(bsc_ctx* c) {
  const int count = c->bucket_off[3], n0 = c->bucket_off[1];
  if (count <= 0) return cudaSuccess;
  BSC_COUNT(c, 1);
  k_reduce_points<T><<<(count + 127) / 128, 128, 0, c->stream>>>(proj_args<T>(c, 0), c->bucket_list, n0, count,
                                                                  c->red_q, c->red_g, c->red_l, c->red_g2,
                                                                  c->red_l2);
  return cudaGetLastError();
}

template <int D>
constexpr size_t p1_smem() { return sizeof(double) * (size_t)(Smem<D>::NP + 3 * Smem<D>::n) * P1Block<D>::value; }
template <int D>
constexpr size_t p2_smem() { return sizeof(double) * (size_t)(4 * 3 * D) * P2_BLOCK; }

// Class k of the span lists: 0 = interior spans (five derivative vectors,
// D = 5), 1 = spans at or next to the border (D = 8).  Phase 1 and phase 2
// can be issued separately (phase < 0: both).
template <int D>
constexpr size_t p0_smem() { return sizeof(double) * (size_t)Smem<D>::NP * P0Block<D>::value; }
template <int D>
constexpr size_t pf_smem() { return 0; }

// Class k of the span lists: 0 = interior spans (five derivative vectors,
// D = 5), 1 = spans at or next to the border (D = 8).  Phase 1 and phase 2
// can be issued separately (phase < 0: both).  With the PSD test (interior
// class, c->proj_psd), phase 0 runs first and the later phases run on the
// spans that failed it.
template <typename T, int D>
cudaError_t run_class(bsc_ctx* c, int k, const int* list, int count, cudaStream_t st, int phase = -1) {
  if (count <= 0) return cudaSuccess;
  cudaError_t e;
  ProjArgs<T> P = proj_args<T>(c, k);
  // the PSD test: interior class in every path; border class (FP64 test
  // only: its 24 x 24 H_r does not fit the certificate's registers) when it
  // runs through these phase kernels (border path 1)
  const bool psd = c->proj_psd && (k == 0 || phase < 0);
  const int* sel = psd ? (k == 0 ? c->proj_sel : c->proj_sel1) : nullptr;
  const int* cnt = c->proj_cnt + (psd ? (k == 0 ? 2 : 4) : k);
  if (phase != 1) {
    if constexpr (D == 8) {
      if (psd) {
        // proj_cnt[4]: border spans failing the FP64 test
        if ((e = cudaMemsetAsync(c->proj_cnt + 4, 0, sizeof(int), st)) != cudaSuccess) return e;
        BSC_COUNT(c, 1);
        k_proj_p0<T, D><<<c->p0_grid1, P0Block<D>::value, p0_smem<D>(), st>>>(P, list, count, nullptr, nullptr,
                                                                               c->proj_sel1, c->proj_cnt + 4);
        if ((e = cudaGetLastError()) != cudaSuccess) return e;
      }
    }
    if (psd) {
      if constexpr (D == 5) {
        // proj_cnt[2]: spans failing the FP64 test; proj_cnt[3]: spans the FP32 certificate left open
        if ((e = cudaMemsetAsync(c->proj_cnt + 2, 0, 2 * sizeof(int), st)) != cudaSuccess) return e;
        const bool cert = c->proj_psd == 2;
        if (cert) {
          BSC_COUNT(c, 1);
          k_proj_pf<T, D><<<c->pf_grid, PF_BLOCK, pf_smem<D>(), st>>>(P, list, count, c->proj_pre, c->proj_cnt + 3);
          if ((e = cudaGetLastError()) != cudaSuccess) return e;
        }
        BSC_COUNT(c, 1);
        k_proj_p0<T, D><<<c->p0_grid, P0Block<D>::value, p0_smem<D>(), st>>>(
            P, list, count, cert ? c->proj_pre : nullptr, c->proj_cnt + 3, c->proj_sel, c->proj_cnt + 2);
        if ((e = cudaGetLastError()) != cudaSuccess) return e;
      }
    }
    BSC_COUNT(c, 1);
    k_proj_p1<T, D><<<c->proj_grid[k][0], P1Block<D>::value, p1_smem<D>(), st>>>(P, list, sel, cnt, count,
                                                                                   c->proj_span[k], c->proj_kneg[k]);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
  }
  if (phase != 0) {
    BSC_COUNT(c, 1);
    if ((e = cudaMemsetAsync(c->proj_work + k, 0, sizeof(unsigned int), st)) != cudaSuccess) return e;
    const int v = k == 0 ? c->p2_variant : 0;
    if (v == 0)
      k_proj_p2<T, D, P2_MINB[0]><<<c->p2_grid[k][0], P2_BLOCK, p2_smem<D>(), st>>>(
          P, list, sel, cnt, count, c->proj_kneg[k], c->proj_span[k], c->proj_scratch[k], c->proj_work + k);
    else
      k_proj_p2<T, D, P2_MINB[1]><<<c->p2_grid[k][1], P2_BLOCK, p2_smem<D>(), st>>>(
          P, list, sel, cnt, count, c->proj_kneg[k], c->proj_span[k], c->proj_scratch[k], c->proj_work + k);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    BSC_COUNT(c, 1);
    using SS = SpanScratch<D>;
    const double* sp = c->proj_span[k];
    const long long nthreads = 27ll * count;
    long long blocks = (nthreads + 255) / 256;
    if (blocks > 32ll * c->num_sms) blocks = 32ll * c->num_sms;  // grid-stride beyond that
    k_proj_corr<T><<<(unsigned)blocks, 256, 0, st>>>(cnt, count, c->Nsp, list, sel, c->proj_kneg[k],
                                                     sp + (size_t)SS::LAM * count,
                                                     reinterpret_cast<const T*>(sp + (size_t)SS::W * count),
                                                     (T*)c->H_span);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
  }
  return cudaSuccess;
}

// The border class by one of three paths: 0 = one warp per span
// (k_project_ring, lowest latency per span: best when there are few border
// spans), 1 = one thread per span through the two phase kernels with D = 8
// (highest throughput: best when there are many), 2 = the warp-per-span
// tridiagonalisation followed by the thread-per-item eigenpair phase (lanes
// busy in both halves).
template <typename T>
cudaError_t run_border(bsc_ctx* c, int path, cudaStream_t st) {
  const int first = c->bucket_off[1], count = c->bucket_off[3] - c->bucket_off[1];
  static_assert(SpanScratch<8>::R == 300 && SpanScratch<8>::TN == 372, "ring phase-1 layout");
  if (path == 0 || path == 3)
    return launch_project_ring(c, first, count, c->proj_work + 2, st, false, nullptr, nullptr, path == 3);
  if (path == 2) {
    cudaError_t e = launch_project_ring(c, first, count, c->proj_work + 2, st, true, c->proj_span[1], c->proj_kneg[1]);
    if (e != cudaSuccess) return e;
    return run_class<T, 8>(c, 1, c->bucket_list + first, count, st, 1);
  }
  return run_class<T, 8>(c, 1, c->bucket_list + first, count, st);
}

// Both classes.  The border class runs on a forked stream.  Its warp-per-span
// kernel (paths 0 and 2) fits beside the interior phase 1 (one block of 211 KB
// of shared memory per SM leaves room for one-warp blocks), so it is forked
// before that phase; the thread-per-span kernels (path 1) do not fit and are
// forked after it, next to the interior phase 2.
template <typename T>
cudaError_t run_all(bsc_ctx* c) {
  cudaError_t e;
  const int* list0 = c->bucket_list + c->bucket_off[0];
  const int n0 = c->bucket_off[1] - c->bucket_off[0];
  const bool early = c->border_path != 1;  // the warp-per-span kernels fit beside the interior phase 1
  if (!early && (e = run_class<T, 5>(c, 0, list0, n0, c->stream, 0)) != cudaSuccess) return e;
  if ((e = cudaEventRecord(c->fork_ev, c->stream)) != cudaSuccess) return e;
  if ((e = cudaStreamWaitEvent(c->side[0], c->fork_ev, 0)) != cudaSuccess) return e;
  if ((e = run_border<T>(c, c->border_path, c->side[0])) != cudaSuccess) return e;
  if (early && (e = run_class<T, 5>(c, 0, list0, n0, c->stream, 0)) != cudaSuccess) return e;
  if ((e = run_class<T, 5>(c, 0, list0, n0, c->stream, 1)) != cudaSuccess) return e;
  if ((e = cudaEventRecord(c->join_ev[0], c->side[0])) != cudaSuccess) return e;
  return cudaStreamWaitEvent(c->stream, c->join_ev[0], 0);
}

template <typename T, int D, int MINB>
cudaError_t p2_grid_of(bsc_ctx* c, int count, int* grid) {
  cudaError_t e;
  if ((e = cudaFuncSetAttribute(k_proj_p2<T, D, MINB>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                (int)p2_smem<D>())) != cudaSuccess)
    return e;
  int per = 0;
  if ((e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, k_proj_p2<T, D, MINB>, P2_BLOCK, p2_smem<D>())) !=
      cudaSuccess)
    return e;
  per = per < 1 ? 1 : per;
  int g = per * c->num_sms;
  const int need = (count + p2_spans(D) - 1) / p2_spans(D);
  if (g > need) g = need;
  *grid = g < 1 ? 1 : g;
  return cudaSuccess;
}

template <typename T, int D>
cudaError_t setup_class(bsc_ctx* c, int k, int count) {
  cudaError_t e;
  if constexpr (D == 8) {
    if ((e = cudaFuncSetAttribute(k_proj_p0<T, D>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                  (int)p0_smem<D>())) != cudaSuccess)
      return e;
    int per0 = 0;
    if ((e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per0, k_proj_p0<T, D>, P0Block<D>::value,
                                                           p0_smem<D>())) != cudaSuccess)
      return e;
    per0 = per0 < 1 ? 1 : per0;
    int g0 = per0 * c->num_sms;
    const int need0 = (count + P0Block<D>::value - 1) / P0Block<D>::value;
    if (g0 > need0) g0 = need0;
    c->p0_grid1 = g0 < 1 ? 1 : g0;
    if ((e = cudaMalloc(&c->proj_sel1, sizeof(int) * (size_t)(count > 0 ? count : 1))) != cudaSuccess) return e;
  }
  if constexpr (D == 5) {
    if ((e = cudaFuncSetAttribute(k_proj_p0<T, D>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                  (int)p0_smem<D>())) != cudaSuccess)
      return e;
    int per0 = 0;
    if ((e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per0, k_proj_p0<T, D>, P0Block<D>::value,
                                                           p0_smem<D>())) != cudaSuccess)
      return e;
    per0 = per0 < 1 ? 1 : per0;
    int g0 = per0 * c->num_sms;
    const int need0 = (count + P0Block<D>::value - 1) / P0Block<D>::value;
    if (g0 > need0) g0 = need0;
    c->p0_grid = g0 < 1 ? 1 : g0;
    if ((e = cudaMalloc(&c->proj_sel, sizeof(int) * (size_t)(count > 0 ? count : 1))) != cudaSuccess) return e;
    if ((e = cudaMalloc(&c->proj_pre, sizeof(int) * (size_t)(count > 0 ? count : 1))) != cudaSuccess) return e;
    if ((e = cudaFuncSetAttribute(k_proj_pf<T, D>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                  (int)pf_smem<D>())) != cudaSuccess)
      return e;
    int perf = 0;
    if ((e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&perf, k_proj_pf<T, D>, PF_BLOCK, pf_smem<D>())) !=
        cudaSuccess)
      return e;
    perf = perf < 1 ? 1 : perf;
    int gf = perf * c->num_sms;
    const int needf = (count + PF_BLOCK - 1) / PF_BLOCK;
    if (gf > needf) gf = needf;
    c->pf_grid = gf < 1 ? 1 : gf;
  }
  if ((e = cudaFuncSetAttribute(k_proj_p1<T, D>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                (int)p1_smem<D>())) != cudaSuccess)
    return e;
  int per1 = 0;
  if ((e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per1, k_proj_p1<T, D>, P1Block<D>::value,
                                                         p1_smem<D>())) != cudaSuccess)
    return e;
  per1 = per1 < 1 ? 1 : per1;
  int g1 = per1 * c->num_sms;
  const int need1 = (count + P1Block<D>::value - 1) / P1Block<D>::value;
  if (g1 > need1) g1 = need1;
  c->proj_grid[k][0] = g1 < 1 ? 1 : g1;
  if ((e = p2_grid_of<T, D, P2_MINB[0]>(c, count, &c->p2_grid[k][0])) != cudaSuccess) return e;
  if ((e = p2_grid_of<T, D, P2_MINB[1]>(c, count, &c->p2_grid[k][1])) != cudaSuccess) return e;
  const int g2 = c->p2_grid[k][0] > c->p2_grid[k][1] ? c->p2_grid[k][0] : c->p2_grid[k][1];
  const size_t cnt = count > 0 ? (size_t)count : 1;
  if ((e = cudaMalloc(&c->proj_span[k], sizeof(double) * SpanScratch<D>::SIZE * cnt)) != cudaSuccess) return e;
  if ((e = cudaMalloc(&c->proj_kneg[k], sizeof(int) * cnt)) != cudaSuccess) return e;
  const size_t slots = (size_t)g2 * P2_BLOCK;
  constexpr int n = 3 * D;
  return cudaMalloc(&c->proj_scratch[k], sizeof(double) * n * n * slots);
}

}  // namespace

// Sizes both classes' grids and scratch, computes the reduced bases and
// derivative vectors, and creates the side stream (called from bsc_create,
// after the quadrature tables).
cudaError_t setup_projection(bsc_ctx* c) {
  cudaError_t e;
  const int n0 = c->bucket_off[1] - c->bucket_off[0], n1 = c->bucket_off[3] - c->bucket_off[1];
  {
    double h[72];
    for (int k = 0; k < 8; ++k) {
      const double inv = 1.0 / sqrt((double)(k + 1) * (double)(k + 2));
      for (int l = 0; l < 9; ++l) h[9 * k + l] = (l <= k ? 1.0 : (l == k + 1 ? -(double)(k + 1) : 0.0)) * inv;
    }
    if ((e = cudaMemcpyToSymbol(d_helmert, h, sizeof(h))) != cudaSuccess) return e;
    if ((e = cudaGetSymbolAddress((void**)&c->helmert, d_helmert)) != cudaSuccess) return e;
  }
  if ((e = cudaMalloc(&c->red_g, sizeof(double) * 16 * (size_t)(c->Nmem > 0 ? c->Nmem : 1))) != cudaSuccess) return e;
  if ((e = cudaMalloc(&c->red_l, sizeof(double) * 8 * (size_t)(c->Nbd > 0 ? c->Nbd : 1))) != cudaSuccess) return e;
  if ((e = cudaMalloc(&c->red_q, sizeof(double) * 45 * (size_t)(n0 > 0 ? n0 : 1))) != cudaSuccess) return e;
  {
    if ((e = cudaMalloc(&c->red_g2, sizeof(float2) * 16 * (size_t)(c->Nmem > 0 ? c->Nmem : 1))) != cudaSuccess)
      return e;
    if ((e = cudaMalloc(&c->red_l2, sizeof(float2) * 8 * (size_t)(c->Nbd > 0 ? c->Nbd : 1))) != cudaSuccess) return e;
  }
  if (c->precision == BSC_FP64) {
    if ((e = setup_class<double, 5>(c, 0, n0)) != cudaSuccess) return e;
    if ((e = setup_class<double, 8>(c, 1, n1)) != cudaSuccess) return e;
    if ((e = reduce_points<double>(c)) != cudaSuccess) return e;
  } else {
    if ((e = setup_class<float, 5>(c, 0, n0)) != cudaSuccess) return e;
    if ((e = setup_class<float, 8>(c, 1, n1)) != cudaSuccess) return e;
    if ((e = reduce_points<float>(c)) != cudaSuccess) return e;
  }
  if ((e = cudaStreamSynchronize(c->stream)) != cudaSuccess) return e;
  if ((e = setup_projection_ring()) != cudaSuccess) return e;
  // before the autotuner has timed both border paths: warp per span while
  // the border spans fill the resident warps a few times over at most
  c->border_path = n1 > 8 * 8 * c->num_sms ? 1 : 0;
  if ((e = cudaMalloc(&c->proj_work, sizeof(unsigned int) * 4)) != cudaSuccess) return e;
  {
    // the class sizes as device counts (the phase kernels read their span
    // count from the device: the PSD test's compacted count, or these)
    const int h[6] = {n0, n1, 0, 0, 0, 0};
    if ((e = cudaMalloc(&c->proj_cnt, sizeof(int) * 6)) != cudaSuccess) return e;
    if ((e = cudaMemcpy(c->proj_cnt, h, sizeof(h), cudaMemcpyHostToDevice)) != cudaSuccess) return e;
  }
  c->proj_psd = 2;
  // FP32 contexts: the projection's FP64-level work on the FP32 pipe (double-float)
  c->proj_df = c->precision == BSC_FP64 ? 0 : 1;
  for (int i = 0; i < 2; ++i) {
    if ((e = cudaStreamCreateWithFlags(&c->side[i], cudaStreamNonBlocking)) != cudaSuccess) return e;
    if ((e = cudaEventCreateWithFlags(&c->join_ev[i], cudaEventDisableTiming)) != cudaSuccess) return e;
  }
  return cudaEventCreateWithFlags(&c->fork_ev, cudaEventDisableTiming);
}

cudaError_t launch_project(bsc_ctx* c) {
  if (c->precision == BSC_FP64) return run_all<double>(c);
  return run_all<float>(c);
}

// The interior class's phase 1 or phase 2 alone (phase 0 / 1), on the
// context's stream: the autotuner times phase 2 per variant.
cudaError_t launch_project_interior(bsc_ctx* c, int phase) {
  const int* list0 = c->bucket_list + c->bucket_off[0];
  const int n0 = c->bucket_off[1] - c->bucket_off[0];
  if (c->precision == BSC_FP64) return run_class<double, 5>(c, 0, list0, n0, c->stream, phase);
  return run_class<float, 5>(c, 0, list0, n0, c->stream, phase);
}

cudaError_t launch_project_border(bsc_ctx* c, int path) {
  if (c->precision == BSC_FP64) return run_border<double>(c, path, c->stream);
  return run_border<float>(c, path, c->stream);
}

// K3 for the spans at and next to the patch border (more than five
// derivative vectors: the boundary spans with their 3x3 / 3x2 Gauss rules
// and the interior spans that own extra knot-line points), one warp per
// span: the low-latency path for contexts with few border spans (a large
// single patch); with many (a batch of small patches) the thread-per-span
// phase kernels with D = 8 have the higher throughput, and the autotuner
// picks between the two by timing.
//
// Their vectors {g_q,beta, L_b} span the whole 8-dimensional mean-free
// subspace of R^9 (or a subspace of it), so a fixed orthonormal basis of that
// subspace (Helmert contrasts) reduces every such span Hessian to 24 x 24
// without a Gram-Schmidt step; a rank-deficient span only adds exact zero
// eigenvalues.  These spans are few but each is expensive, so the kernel
// minimises latency rather than lane-operations: one warp per span, lane j
// holding column j of H_r in registers.  Householder steps exchange the
// reflector through shuffles; every negative eigenvalue is bisected by its
// own lane (FP32 bracket, FP64 check and refinement); each lane recovers its
// eigenvector by inverse iteration, with Gram-Schmidt across lanes after each
// solve (clusters); the back-transformation reads the reflectors from shared
// memory; the lanes share the 378 packed entries of the final update
// H -= sum lam w w^T.  The projected matrix V max(Lambda, 0) V^T (projected
// Newton, Sec. 5.1) is unique, so this reduction and the interior kernel's
// give the same result up to rounding.
#include "bsc_internal.cuh"

namespace {

constexpr int RN = 24;         // reduced size 3 x 8
constexpr int RBLOCK = 32;     // one warp (span) per block: 5.6 KB of shared memory, so blocks fit beside the
                                // interior phase 1 (211 KB per SM) and the border class can start with it
constexpr double NEG_REL = 1e-14;

// Helmert contrasts: q_k = (1, ..., 1, -k, 0, ...) / sqrt(k (k + 1)), k = 1..8
// (k ones), an orthonormal basis of the vectors of R^9 that sum to zero.
__constant__ double c_helmert[8][9];

template <typename T>
struct RingArgs {
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
  const double* __restrict__ rg;  // [16][Nm] g_q,beta in the Helmert basis
  const double* __restrict__ rl;  // [8][Nb] L_q in the Helmert basis
  int* fail_count;                // spans failing the PSD test (counted when it runs)
  // test only (fail_list != nullptr, PSD): the class positions of the spans
  // failing the test are appended to fail_list and nothing else is done for them
  int* fail_list;
  // over a list (sel != nullptr): the class positions sel[0 .. *sel_count)
  const int* sel;
  const int* sel_count;
  // with the PSD test: an FP32 certificate first (ring_certify_f32); the
  // spans it leaves to the FP64 test are counted in *open_count
  int cert;
  int* open_count;
};

__device__ __forceinline__ double shfl(double v, int src) { return __shfl_sync(0xffffffffu, v, src); }

__device__ __forceinline__ int sgn_d(double x) { return (unsigned)__double2hiint(x) >> 31; }
__device__ __forceinline__ int exp_d(double x) { return (__double2hiint(x) >> 20) & 0x7ff; }
__device__ __forceinline__ int sgn_f(float x) { return (unsigned)__float_as_int(x) >> 31; }

// det(T - x I) of the scaled tridiagonal in shared memory with the Sturm
// count (eigenvalues < x); *exact is false when a replacement of a zero
// minor or a rescaling made the value's scale differ from the
// determinant's.  The recurrence first runs without rescaling, the
// exponents tracked with integer operations (three FP64 operations per
// step); a pair of minors outside [2^-500, 2^500] sends the call to the
// rescaling pass, which gives the identical result.
__device__ __noinline__ double charpoly64_scaled(const double* d, const double* e2, double x, int* cnt_out,
                                                 bool* exact) {
  double pm = 1.0, p = d[0] - x;
  int cnt = sgn_d(p);
  bool ok = true;
  for (int i = 1; i < RN; ++i) {
    double pn = (d[i] - x) * p - e2[i - 1] * pm;
    if (exp_d(pn) == 0) {
      pn = sgn_d(p) ? 1e-300 : -1e-300;
      ok = false;
    }
    cnt += sgn_d(pn) ^ sgn_d(p);
    const int ea = exp_d(pn), eb = exp_d(p), mx = ea > eb ? ea : eb;
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

__device__ __noinline__ double charpoly64(const double* d, const double* e2, double x, int* cnt_out, bool* exact) {
  double pm = 1.0, p = d[0] - x;
  int cnt = sgn_d(p), eb = exp_d(p);
  bool ok = true, in_range = true;
#pragma unroll
  for (int i = 1; i < RN; ++i) {
    double pn = (d[i] - x) * p - e2[i - 1] * pm;
    const bool z = exp_d(pn) == 0;
    pn = z ? (sgn_d(p) ? 1e-300 : -1e-300) : pn;
    ok = ok && !z;
    cnt += sgn_d(pn) ^ sgn_d(p);
    const int ea = exp_d(pn), mx = ea > eb ? ea : eb;
    in_range = in_range && mx <= 1023 + 500 && mx >= 1023 - 500;
    pm = p;
    p = pn;
    eb = ea;
  }
  if (!in_range) return charpoly64_scaled(d, e2, x, cnt_out, exact);
  *cnt_out = cnt;
  *exact = ok;
  return p;
}

// Sturm count (eigenvalues < x) of the scaled tridiagonal in shared memory.
__device__ int sturm64(const double* d, const double* e2, double x) {
  int cnt;
  bool ex;
  charpoly64(d, e2, x, &cnt, &ex);
  return cnt;
}

// FP32 count on the copy of the tridiagonal: with ||T|| <= 1 the minors stay
// below (1 + sqrt 2)^24 < 2e9, so only a pair near underflow (next to the
// exact zero eigenvalues of a rank-deficient span) is rescaled.
__device__ int sturm32(const float* d, const float* e2, float x) {
  float pm = 1.0f, p = d[0] - x;
  int cnt = sgn_f(p);
#pragma unroll
  for (int i = 1; i < RN; ++i) {
    float pn = (d[i] - x) * p - e2[i - 1] * pm;
    if (pn == 0.0f) pn = sgn_f(p) ? 1e-30f : -1e-30f;
    cnt += sgn_f(pn) ^ sgn_f(p);
    if (fmaxf(fabsf(pn), fabsf(p)) < 1e-30f) {  // a pair near underflow (a multiple root nearby)
      pn *= 1e30f;
      p *= 1e30f;
    }
    pm = p;
    p = pn;
  }
  return cnt;
}

// Eigenvalue k (scaled) of the tridiagonal in shared memory: FP32
// quadrisection to about 22 bits (three independent counts per step), the
// widened bracket checked by two FP64 Sturm counts,
// then regula falsi (Illinois) on det(T - x I) while the bracket isolates
// eigenvalue k, bisection otherwise; four steps that fail to halve the
// bracket force a bisection step (a bracket end next to a multiple root
// stalls regula falsi).  Own call frame: the kernel body keeps its registers.
__device__ __noinline__ double ring_eigenvalue(const double* dd, const double* ee2, const float* d32,
                                               const float* e232, int k) {
  float a32 = -1.0f - 1e-6f, b32 = (float)(-NEG_REL);
  for (int it = 0; it < 11; ++it) {
    const float h = 0.25f * (b32 - a32);
    const float m1 = a32 + h, m2 = a32 + 2.0f * h, m3 = a32 + 3.0f * h;
    const bool c1 = sturm32(d32, e232, m1) > k, c2 = sturm32(d32, e232, m2) > k, c3 = sturm32(d32, e232, m3) > k;
    if (c1) {
      b32 = m1;
    } else if (c2) {
      a32 = m1;
      b32 = m2;
    } else if (c3) {
      a32 = m2;
      b32 = m3;
    } else {
      a32 = m3;
    }
  }
  double a = fmax((double)a32 - 4e-6, -1.0 - 1e-12), b = fmin((double)b32 + 4e-6, -NEG_REL);
  int ca, cb;
  bool xa, xb;
  double fa = charpoly64(dd, ee2, a, &ca, &xa), fb = charpoly64(dd, ee2, b, &cb, &xb);
  if (!(ca <= k && cb > k)) {
    a = -1.0 - 1e-12;
    b = -NEG_REL;
    fa = charpoly64(dd, ee2, a, &ca, &xa);
    fb = charpoly64(dd, ee2, b, &cb, &xb);
  }
  int side = 0, win = 0;
  bool force_bisect = false;
  double wstart = b - a;
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
    const double fx = charpoly64(dd, ee2, x, &cx, &xx);
    if (cx > k) {
      if (isolated && side == -1) fa *= 0.5;
      b = x; fb = fx; cb = cx; xb = xx; side = -1;
    } else {
      if (isolated && side == 1) fb *= 0.5;
      a = x; fa = fx; ca = cx; xa = xx; side = 1;
    }
    if (isolated && fx == 0.0) return x;
    if (isolated && ++win == 4) {
      force_bisect = b - a > 0.5 * wstart;
      win = 0;
      wstart = b - a;
    }
  }
  return 0.5 * (a + b);
}

// Solves (T - sig I) y = y in place by Gaussian elimination with partial
// pivoting, eliminating and applying to y in one forward pass (U kept).
__device__ void tri_solve(const double* d, const double* e, double sig, double (&y)[RN]) {
  double u0r[RN], u1[RN], u2[RN];
  double c0 = d[0] - sig, c1 = e[0], c2 = 0.0;
#pragma unroll
  for (int i = 0; i < RN - 1; ++i) {
    const double ei = e[i], a1 = d[i + 1] - sig, e1 = (i + 1 < RN - 1) ? e[i + 1] : 0.0;
    // pivot row and eliminated row chosen by selects: one reciprocal per step
    const bool swp = fabs(ei) > fabs(c0);
    const double g0 = fabs(c0) < 2.3e-16 ? (c0 < 0.0 ? -2.3e-16 : 2.3e-16) : c0;
    const double t0 = swp ? ei : g0, t1 = swp ? a1 : c1, t2 = swp ? e1 : c2;
    const double b0 = swp ? c0 : ei, b1 = swp ? c1 : a1, b2 = swp ? c2 : e1;
    const double r = 1.0 / t0, m = b0 * r;
    u0r[i] = r; u1[i] = t1; u2[i] = t2;
    const double ya = swp ? y[i + 1] : y[i], yb = swp ? y[i] : y[i + 1];
    y[i] = ya;
    y[i + 1] = yb - m * ya;
    c0 = b1 - m * t1; c1 = b2 - m * t2; c2 = 0.0;
  }
  if (fabs(c0) < 2.3e-16) c0 = c0 < 0.0 ? -2.3e-16 : 2.3e-16;
  u0r[RN - 1] = 1.0 / c0; u1[RN - 1] = u2[RN - 1] = 0.0;
#pragma unroll
  for (int i = RN - 1; i >= 0; --i) {
    double s = y[i];
    if (i + 1 < RN) s -= u1[i] * y[i + 1];
    if (i + 2 < RN) s -= u2[i] * y[i + 2];
    y[i] = s * u0r[i];
  }
}

// Modified Gram-Schmidt across lanes: in order j = 0, 1, ..., lane j
// normalises its vector, broadcasts it, and lanes j+1..kneg-1 remove its
// component.
__device__ void warp_mgs(double (&y)[RN], int lane, int kneg) {
  for (int j = 0; j < kneg; ++j) {
    if (lane == j) {
      double nn = 0.0;
#pragma unroll
      for (int i = 0; i < RN; ++i) nn += y[i] * y[i];
      const double inv = 1.0 / sqrt(nn);
#pragma unroll
      for (int i = 0; i < RN; ++i) y[i] *= inv;
    }
    double yj[RN];
#pragma unroll
    for (int i = 0; i < RN; ++i) yj[i] = shfl(y[i], j);
    if (lane > j && lane < kneg) {
      double dt = 0.0;
#pragma unroll
      for (int i = 0; i < RN; ++i) dt += yj[i] * y[i];
#pragma unroll
      for (int i = 0; i < RN; ++i) y[i] -= dt * yj[i];
    }
  }
}

// (row, column) of packed upper-triangle entry e of a 27 x 27 matrix
__constant__ unsigned char c_row[H27], c_col[H27];

// Phase-1 output of a span for the thread-per-item eigenpair kernel (the
// class scratch of k_proj_p2 with D = 8, entry-major over the span's
// position in the class list): packed reflectors with tau on the diagonal,
// the scaled tridiagonal (d, e, e^2), the scale, and the count.
struct RingP1Out {
  double* A;    // [300][count]
  double* R;    // [72][count]
  double* TN;   // [count]
  int* kneg;    // [count]
};

// FP32 certificate of positive definiteness of a border span's H_r, one warp,
// lane j forming column j of H_r in FP32 exactly as the FP64 formation below
// does in FP64, then factoring H_r - sigma I.  The argument is the interior
// class's (k_proj_pf), with n = 24 and this formation's rounding count:
//  - every term of an entry (a product of two reduced derivative entries and
//    one d^2 Psi / df^2 entry, or of W_b and two bending entries) meets at
//    most 3 roundings of its inputs to FP32 (4 for W_b, a product formed in
//    FP64), 2 in t (membrane) or in W_b L_k (bending), and one per
//    accumulation into the entry, 2 n_mem + n_bd in all: m = 6 + 2 n_mem +
//    n_bd roundings bound every term, so with the same S as the interior
//    class, ||H_r - F||_2 <= gamma_m S for the computed F;
//  - the factorisation reads only the entries on and below the diagonal of
//    each lane's column (the pivot column k is taken from lane k): it is the
//    LDL^T of the symmetric matrix F_L with that lower triangle, whose entries
//    obey the same bound, and its rounding is that of the interior
//    certificate (multipliers by a correctly rounded reciprocal and a
//    product), ||E||_2 <= gamma_{n+4} tr(F_L) / (1 - gamma_{n+4}).
// With sigma = 1.1 (gamma_{n+4} tr + gamma_m S), every pivot of F_L - sigma I
// positive means every eigenvalue of H_r above a margin of order
// 1e-6 tr(H_r): the FP64 test below (margin 1e-14 tr / n) would pass the
// span as well, so taking the certificate changes no span's result.
template <typename T>
__device__ __forceinline__ bool ring_certify_f32(const RingArgs<T>& P, int q0, int q1, int b0, int b1, double mubd,
                                                 int lane, int kp, int dp) {
  constexpr float u = 5.9604644775390625e-8f;  // 2^-24
  constexpr float g_n4 = (RN + 4) * u / (1.0f - (RN + 4) * u);
  const int m = 6 + 2 * (q1 - q0) + (b1 - b0);
  if (m > 4096) return false;
  const float g_m = m * u / (1.0f - m * u);
  float col[RN];
#pragma unroll
  for (int i = 0; i < RN; ++i) col[i] = 0.0f;
  float S = 0.0f;
  for (int q = q0; q < q1; ++q) {
    float gt[8][2], g2 = 0.0f;
#pragma unroll
    for (int k = 0; k < 8; ++k)
#pragma unroll
      for (int b = 0; b < 2; ++b) {
        gt[k][b] = (float)P.rg[(size_t)(2 * k + b) * P.Nm + q];
        g2 = fmaf(gt[k][b], gt[k][b], g2);
      }
    float A6[6][6], a2 = 0.0f;
    {
      int e = 0;
#pragma unroll
      for (int r = 0; r < 6; ++r)
#pragma unroll
        for (int c = r; c < 6; ++c) {
          const float v = (float)P.A[(e++) * P.Nm + q];
          A6[r][c] = v;
          A6[c][r] = v;
          a2 = fmaf(r == c ? v : 2.0f * v, v, a2);
        }
    }
    S = fmaf(3.0f * g2, __fsqrt_ru(a2), S);
    if (lane < RN) {
      float gk0 = 0.0f, gk1 = 0.0f;
#pragma unroll
      for (int k = 0; k < 8; ++k)
        if (k == kp) { gk0 = gt[k][0]; gk1 = gt[k][1]; }
      float t[2][3];
#pragma unroll
      for (int b = 0; b < 2; ++b)
#pragma unroll
        for (int c = 0; c < 3; ++c) {
          float a0 = 0.0f, a1 = 0.0f;
#pragma unroll
          for (int z = 0; z < 3; ++z)
            if (z == dp) { a0 = A6[3 * b + c][z]; a1 = A6[3 * b + c][3 + z]; }
          t[b][c] = fmaf(gk1, a1, gk0 * a0);
        }
#pragma unroll
      for (int k = 0; k < 8; ++k)
#pragma unroll
        for (int c = 0; c < 3; ++c)
          col[3 * k + c] = fmaf(gt[k][1], t[1][c], fmaf(gt[k][0], t[0][c], col[3 * k + c]));
    }
  }
  for (int q = b0; q < b1; ++q) {
    const float WB = (float)((double)P.tabb[q] * mubd);
    float Lt[8], l2 = 0.0f, Lk = 0.0f;
#pragma unroll
    for (int k = 0; k < 8; ++k) {
      Lt[k] = (float)P.rl[(size_t)k * P.Nb + q];
      l2 = fmaf(Lt[k], Lt[k], l2);
      if (k == kp) Lk = Lt[k];
    }
    S = fmaf(3.0f * fabsf(WB), l2, S);
    if (lane < RN) {
#pragma unroll
      for (int k = 0; k < 8; ++k)
#pragma unroll
        for (int c = 0; c < 3; ++c)
          if (c == dp) col[3 * k + c] = fmaf(WB * Lt[k], Lk, col[3 * k + c]);
    }
  }
  float dj = 0.0f;
#pragma unroll
  for (int i = 0; i < RN; ++i)
    if (i == lane) dj = col[i];
  float tr = lane < RN ? dj : 0.0f;
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) tr += __shfl_xor_sync(0xffffffffu, tr, o);
  if (!(tr > 0.0f) || !isfinite(tr) || !isfinite(S)) return false;
  const float sigma = 1.1f * (g_n4 * tr + g_m * S);
#pragma unroll
  for (int i = 0; i < RN; ++i)
    if (i == lane) col[i] -= sigma;
  bool pass = true;
#pragma unroll
  for (int k = 0; k < RN; ++k) {
    float ck[RN], dk = 0.0f, cj = 0.0f;
#pragma unroll
    for (int i = k; i < RN; ++i) {
      ck[i] = __shfl_sync(0xffffffffu, col[i], k);  // column k of the trailing matrix, from lane k
      if (i == lane) cj = ck[i];
    }
    dk = ck[k];
    pass = pass && dk > 0.0f && isfinite(dk);  // the same on every lane
    if (!pass) break;
    if (lane > k && lane < RN) {
      const float l = cj * __frcp_rn(dk);
#pragma unroll
      for (int i = k + 1; i < RN; ++i) col[i] = fmaf(-l, ck[i], col[i]);
    }
  }
  return pass;
}

// PSD: before the tridiagonalisation, the warp factors H_r + tau I (LDL^T in
// FP64, tau = 1e-14 tr(H_r) / n, lane j updating column j from the pivot
// column it receives by shuffles); a span whose pivots are all positive has
// no eigenvalue below -tau, keeps its Hessian and leaves the warp free for
// the next span.
template <typename T, bool P1ONLY, bool PSD>
__global__ void __launch_bounds__(RBLOCK) k_project_ring(RingArgs<T> P, const int* __restrict__ list, int count,
                                                         unsigned int* __restrict__ work, RingP1Out out) {
  constexpr int WARPS = RBLOCK / 32;
  __shared__ double s_refl[WARPS][RN][RN];  // reflector k in column k (rows k+1..), tau_k at [k][k]
  __shared__ double s_d[WARPS][RN], s_e[WARPS][RN], s_e2[WARPS][RN];
  __shared__ float s_d32[WARPS][RN], s_e232[WARPS][RN];
  __shared__ double s_w[WARPS][27];
  const int lane = threadIdx.x & 31, wp = threadIdx.x >> 5;
  double* const refl = &s_refl[wp][0][0];
  double* const dd = s_d[wp];
  double* const ee = s_e[wp];
  double* const ee2 = s_e2[wp];
  const int kp = lane / 3, dp = lane % 3;  // this lane's column j = 3 kp + dp
  const int n_items = P.sel ? *P.sel_count : count;
  for (;;) {
    int idx = 0;
    if (lane == 0) idx = (int)atomicAdd(work, 1u);
    idx = __shfl_sync(0xffffffffu, idx, 0);
    if (idx >= n_items) break;
    if (P.sel) idx = P.sel[idx];
    const int s = list[idx];
    const int q0 = P.moff[s], q1 = P.moff[s + 1], b0 = P.boff[s], b1 = P.boff[s + 1];
    const double mubd = P.pd[P.sp_patch[s]].mubd;

    if (PSD && P.cert) {
      if (ring_certify_f32<T>(P, q0, q1, b0, b1, mubd, lane, kp, dp)) {
        if (lane == 0) {
          P.nneg[s] = 0;
          if (P1ONLY) out.kneg[idx] = 0;
        }
        __syncwarp();
        continue;
      }
      if (lane == 0) atomicAdd(P.open_count, 1);
    }

    // ---- column lane of H_r = sum_q (G~ (x) I3) A_q (G~ (x) I3)^T + bending
    double col[RN];
#pragma unroll
    for (int i = 0; i < RN; ++i) col[i] = 0.0;
    for (int q = q0; q < q1; ++q) {
      double gt[8][2];
#pragma unroll
      for (int k = 0; k < 8; ++k) {
        gt[k][0] = P.rg[(size_t)(2 * k) * P.Nm + q];
        gt[k][1] = P.rg[(size_t)(2 * k + 1) * P.Nm + q];
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
      if (lane < RN) {
        double gk0 = 0.0, gk1 = 0.0;
#pragma unroll
        for (int k = 0; k < 8; ++k)
          if (k == kp) { gk0 = gt[k][0]; gk1 = gt[k][1]; }
        // t[b][c] = sum_delta g~[kp][delta] A6[3b + c][3 delta + dp]
        double t[2][3];
#pragma unroll
        for (int b = 0; b < 2; ++b)
#pragma unroll
          for (int c = 0; c < 3; ++c) {
            double a0 = 0.0, a1 = 0.0;
#pragma unroll
            for (int z = 0; z < 3; ++z)
              if (z == dp) { a0 = A6[3 * b + c][z]; a1 = A6[3 * b + c][3 + z]; }
            t[b][c] = gk0 * a0 + gk1 * a1;
          }
#pragma unroll
        for (int k = 0; k < 8; ++k)
#pragma unroll
          for (int c = 0; c < 3; ++c)  // two FMAs into the accumulator
            col[3 * k + c] = fma(gt[k][1], t[1][c], fma(gt[k][0], t[0][c], col[3 * k + c]));
      }
    }
    for (int q = b0; q < b1; ++q) {
      const double WB = (double)P.tabb[q] * mubd;
      double Lt[8];
#pragma unroll
      for (int k = 0; k < 8; ++k) Lt[k] = P.rl[(size_t)k * P.Nb + q];
      double Lk = 0.0;
#pragma unroll
      for (int k = 0; k < 8; ++k)
        if (k == kp) Lk = Lt[k];
      if (lane < RN) {
#pragma unroll
        for (int k = 0; k < 8; ++k)
#pragma unroll
          for (int c = 0; c < 3; ++c)
            if (c == dp) col[3 * k + c] += WB * Lt[k] * Lk;
      }
    }

    if (PSD) {
      double dj = 0.0;
#pragma unroll
      for (int i = 0; i < RN; ++i)
        if (i == lane) dj = col[i];
      double tr = lane < RN ? dj : 0.0;
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) tr += __shfl_xor_sync(0xffffffffu, tr, o);
      bool pass = tr > 0.0 && isfinite(tr);
      const double tau = NEG_REL * tr * (1.0 / RN);
      double w[RN];
#pragma unroll
      for (int i = 0; i < RN; ++i) w[i] = col[i] + (i == lane ? tau : 0.0);
      for (int k = 0; k < RN && pass; ++k) {
        double ck[RN], dk = 0.0, cj = 0.0;
#pragma unroll
        for (int i = 0; i < RN; ++i) {
          ck[i] = shfl(w[i], k);  // column k = row k of the trailing matrix
          if (i == k) dk = ck[i];
          if (i == lane) cj = ck[i];
        }
        pass = dk > 0.0 && isfinite(dk);  // the same on every lane
        if (pass && lane > k && lane < RN) {
          const double l = cj / dk;
#pragma unroll
          for (int i = 0; i < RN; ++i)
            if (i > k) w[i] = fma(-l, ck[i], w[i]);
        }
      }
      if (pass) {
        if (lane == 0) {
          P.nneg[s] = 0;
          if (P1ONLY) out.kneg[idx] = 0;
        }
        __syncwarp();
        continue;
      }
      if (lane == 0) {
        const int k = atomicAdd(P.fail_count, 1);
        if (P.fail_list) P.fail_list[k] = idx;
      }
      if (P.fail_list) {
        __syncwarp();
        continue;
      }
    }

    // ---- Householder tridiagonalisation, lane k owns column k
#pragma unroll
    for (int k = 0; k < RN - 2; ++k) {
      double sigma = 0.0;
#pragma unroll
      for (int i = k + 2; i < RN; ++i) sigma += col[i] * col[i];
      const double x0 = col[k + 1];
      const double nrm = sqrt(x0 * x0 + sigma);
      const double alpha = x0 >= 0.0 ? -nrm : nrm;
      const double v0 = x0 - alpha;
      const double tau = sigma == 0.0 ? 0.0 : 2.0 / (v0 * v0 + sigma);
      const double tau_k = shfl(tau, k);
      if (lane == k) {
        dd[k] = col[k];
        ee[k] = sigma == 0.0 ? x0 : alpha;
        refl[k * RN + k] = tau;
        col[k + 1] = sigma == 0.0 ? x0 : v0;
#pragma unroll
        for (int i = k + 1; i < RN; ++i) refl[i * RN + k] = col[i];
      }
      if (tau_k == 0.0) continue;
      double v[RN];
#pragma unroll
      for (int i = k + 1; i < RN; ++i) v[i] = shfl(col[i], k);
      // p_j = tau sum_i A(i, j) v_i for j > k;  w_j = p_j - (tau/2)(v.p) v_j
      double p = 0.0, vj = 0.0;
#pragma unroll
      for (int i = k + 1; i < RN; ++i) {
        p += col[i] * v[i];
        if (i == lane) vj = v[i];
      }
      const bool act = lane > k && lane < RN;
      p = act ? tau_k * p : 0.0;
      double vp = act ? vj * p : 0.0;
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) vp += __shfl_xor_sync(0xffffffffu, vp, o);
      const double wj = p - 0.5 * tau_k * vp * vj;
      double w[RN];
#pragma unroll
      for (int i = k + 1; i < RN; ++i) w[i] = shfl(wj, i);
      if (act) {
#pragma unroll
        for (int i = k + 1; i < RN; ++i) col[i] = fma(-w[i], vj, fma(-v[i], wj, col[i]));  // two FMAs
      }
    }
    if (lane == RN - 2) {
      dd[RN - 2] = col[RN - 2];
      ee[RN - 2] = col[RN - 1];
      refl[(RN - 2) * RN + RN - 2] = 0.0;
    }
    if (lane == RN - 1) {
      dd[RN - 1] = col[RN - 1];
      ee[RN - 1] = 0.0;
    }
    __syncwarp();

    // ---- scale, inertia
    double tn = 0.0;
#pragma unroll
    for (int i = 0; i < RN; ++i) tn = fmax(tn, fabs(dd[i]) + fabs(ee[i]) + (i > 0 ? fabs(ee[i - 1]) : 0.0));
    __syncwarp();
    if (!(tn > 0.0) || !isfinite(tn)) {
      if (lane == 0) {
        P.nneg[s] = 0;
        if (P1ONLY) out.kneg[idx] = 0;
        if (!isfinite(tn)) atomicOr(P.status, BSC_STATUS_NUMERIC_FLAG);
      }
      __syncwarp();
      continue;
    }
    const double itn = 1.0 / tn;
    if (lane < RN) {
      const double ds = dd[lane] * itn, es = ee[lane] * itn;
      dd[lane] = ds;
      ee[lane] = es;
      ee2[lane] = es * es;
      s_d32[wp][lane] = (float)ds;
      s_e232[wp][lane] = (float)(es * es);
    }
    __syncwarp();
    const int kneg = sturm64(dd, ee2, -NEG_REL);
    if (lane == 0) P.nneg[s] = kneg;
    if (P1ONLY) {
      // hand the span to the eigenpair items: reflectors k <= RN - 3 (the
      // back-transformation uses no others), tridiagonal, scale, count
      if (lane == 0) out.kneg[idx] = kneg;
      if (kneg > 0) {
        for (int q = lane; q < RN * RN; q += 32) {
          const int i = q / RN, k = q - i * RN;
          if (k <= RN - 3 && i >= k) out.A[(size_t)(i * (i + 1) / 2 + k) * count + idx] = refl[i * RN + k];
        }
        if (lane < RN) {
          out.R[(size_t)lane * count + idx] = dd[lane];
          out.R[(size_t)(RN + lane) * count + idx] = ee[lane];
          out.R[(size_t)(2 * RN + lane) * count + idx] = ee2[lane];
        }
        if (lane == 0) out.TN[idx] = tn;
      }
      __syncwarp();
      continue;
    }
    if (kneg == 0) continue;

    // ---- lane k < kneg: eigenvalue k (FP32 bracket, FP64 check + refinement)
    double sig = 0.0;
    if (lane < kneg) sig = ring_eigenvalue(dd, ee2, s_d32[wp], s_e232[wp], lane);
    // ---- inverse iteration, two solves, Gram-Schmidt across lanes after each
    double y[RN];
#pragma unroll
    for (int i = 0; i < RN; ++i) y[i] = 1.0 + 0.125 * (double)((7 * i + 3 * lane) % 5);
    for (int it = 0; it < 2; ++it) {
      if (lane < kneg) tri_solve(dd, ee, sig, y);
      warp_mgs(y, lane, kneg);
    }
    double lam = 0.0;
    if (lane < kneg) {
      double rq = 0.0;
#pragma unroll
      for (int i = 0; i < RN; ++i) {
        double ty = dd[i] * y[i];
        if (i > 0) ty += ee[i - 1] * y[i - 1];
        if (i + 1 < RN) ty += ee[i] * y[i + 1];
        rq += y[i] * ty;
      }
      lam = fmin(rq, 0.0) * tn;
      // back-transformation x = H_0 ... H_{RN-3} y
#pragma unroll
      for (int k = RN - 3; k >= 0; --k) {
        const double t = refl[k * RN + k];
        double sdot = 0.0;
#pragma unroll
        for (int i = k + 1; i < RN; ++i) sdot += refl[i * RN + k] * y[i];
        sdot *= t;
#pragma unroll
        for (int i = k + 1; i < RN; ++i) y[i] -= sdot * refl[i * RN + k];
      }
    }
    // w = (Q (x) I3) x on each active lane
    double wv[27];
#pragma unroll
    for (int l = 0; l < 9; ++l)
#pragma unroll
      for (int c = 0; c < 3; ++c) {
        double acc = 0.0;
#pragma unroll
        for (int k = 0; k < 8; ++k) acc += c_helmert[k][l] * y[3 * k + c];
        wv[3 * l + c] = lane < kneg ? acc : 0.0;
      }
    // ---- H -= sum_k lam_k w_k w_k^T: lane handles packed entries e = lane + 32 m;
    //      w_k is staged in shared memory by its lane
    double corr[12];
#pragma unroll
    for (int m = 0; m < 12; ++m) corr[m] = 0.0;
    double* const sw = s_w[wp];
    for (int k = 0; k < kneg; ++k) {
      const double lk = shfl(lam, k);
      if (lane == k) {
#pragma unroll
        for (int r = 0; r < 27; ++r) sw[r] = wv[r];
      }
      __syncwarp();
#pragma unroll
      for (int m = 0; m < 12; ++m) {
        const int e = lane + 32 * m;
        if (e < H27) corr[m] += lk * sw[c_row[e]] * sw[c_col[e]];
      }
      __syncwarp();
    }
#pragma unroll
    for (int m = 0; m < 12; ++m) {
      const int e = lane + 32 * m;
      if (e < H27) {
        T* h = P.H + (size_t)e * P.Nsp + s;
        *h = (T)((double)*h - corr[m]);
      }
    }
    __syncwarp();
  }
}

}  // namespace

template <typename T>
void launch_ring_t(RingArgs<T> P, const int* list, int count, unsigned int* work, RingP1Out out, int g,
                   cudaStream_t st, bool p1only, bool psd) {
  // a pass over a list of failing spans runs without the test (they failed it)
  if (P.sel) psd = false;
  if (p1only) {
    if (psd) k_project_ring<T, true, true><<<g, RBLOCK, 0, st>>>(P, list, count, work, out);
    else k_project_ring<T, true, false><<<g, RBLOCK, 0, st>>>(P, list, count, work, out);
  } else {
    if (psd) k_project_ring<T, false, true><<<g, RBLOCK, 0, st>>>(P, list, count, work, out);
    else k_project_ring<T, false, false><<<g, RBLOCK, 0, st>>>(P, list, count, work, out);
  }
}

cudaError_t setup_projection_ring() {
  double h[8][9];
  for (int k = 1; k <= 8; ++k) {
    const double sc = 1.0 / sqrt((double)k * (k + 1));
    for (int l = 0; l < 9; ++l) h[k - 1][l] = l < k ? sc : (l == k ? -k * sc : 0.0);
  }
  cudaError_t e = cudaMemcpyToSymbol(c_helmert, h, sizeof(h));
  if (e != cudaSuccess) return e;
  unsigned char rr[H27], cc[H27];
  int k = 0;
  for (int r = 0; r < 27; ++r)
    for (int c = r; c < 27; ++c, ++k) {
      rr[k] = (unsigned char)r;
      cc[k] = (unsigned char)c;
    }
  e = cudaMemcpyToSymbol(c_row, rr, sizeof(rr));
  if (e != cudaSuccess) return e;
  return cudaMemcpyToSymbol(c_col, cc, sizeof(cc));
}

// Three one-warp blocks per SM: with the interior phase 1's block (211 KB of
// shared memory, 160 threads x 254 registers) they fill an SM's 228 KB of
// shared memory and 64 K registers, so both kernels run side by side.
int ring_grid(int num_sms) { return 3 * num_sms; }

// Border class, one warp per span.  p1only: stop after the tridiagonal form
// and hand each span to k_proj_p2<T, 8> through its class scratch (sspan,
// laid out as reflectors [300], tridiagonal [72], scale [1]) and kneg.
// two_pass (with the PSD test on): first every warp only tests its spans and
// appends the failing ones to the border's list, then the warps take the
// failing spans one each - the few expensive spans no longer queue behind
// one another on the warps that happened to draw them.
cudaError_t launch_project_ring(bsc_ctx* c, int first, int count, unsigned int* work, cudaStream_t st, bool p1only,
                                double* sspan, int* kneg, bool two_pass) {
  if (count <= 0) return cudaSuccess;
  const bool psd = c->proj_psd != 0;
  two_pass = two_pass && psd && !p1only;
  BSC_COUNT(c, two_pass ? 2 : 1);
  cudaError_t e = cudaMemsetAsync(work, 0, sizeof(unsigned int), st);
  // proj_cnt[4]: border spans failing the FP64 test; [5]: those the certificate left to it
  if (e == cudaSuccess) e = cudaMemsetAsync(c->proj_cnt + 4, 0, 2 * sizeof(int), st);
  if (e != cudaSuccess) return e;
  const int need = (count + RBLOCK / 32 - 1) / (RBLOCK / 32);
  int g = ring_grid(c->num_sms);
  if (g > need) g = need;
  const size_t cnt = (size_t)count;
  RingP1Out out{sspan, sspan ? sspan + 300 * cnt : nullptr, sspan ? sspan + 372 * cnt : nullptr, kneg};
  const int* list = c->bucket_list + first;
  for (int pass = 0; pass < (two_pass ? 2 : 1); ++pass) {
    if (pass == 1 && (e = cudaMemsetAsync(work, 0, sizeof(unsigned int), st)) != cudaSuccess) return e;
    int* fail_list = two_pass && pass == 0 ? c->proj_sel1 : nullptr;
    const int* sel = pass == 1 ? c->proj_sel1 : nullptr;
    const int* sel_count = pass == 1 ? c->proj_cnt + 4 : nullptr;
    if (c->precision == BSC_FP64) {
      RingArgs<double> P{c->Nsp, c->Nmem, c->Nbd, c->pd, c->sp_patch, c->mem_off, c->bd_off,
                         (const double*)c->tab_mem, (const double*)c->tab_bd, (const double*)c->A_mem,
                         (double*)c->H_span, c->nneg, c->dstatus, c->red_g, c->red_l, c->proj_cnt + 4, fail_list,
                         sel, sel_count, c->proj_psd == 2, c->proj_cnt + 5};
      launch_ring_t<double>(P, list, count, work, out, g, st, p1only, psd);
    } else {
      RingArgs<float> P{c->Nsp, c->Nmem, c->Nbd, c->pd, c->sp_patch, c->mem_off, c->bd_off, (const float*)c->tab_mem,
                        (const float*)c->tab_bd, (const float*)c->A_mem, (float*)c->H_span, c->nneg, c->dstatus,
                        c->red_g, c->red_l, c->proj_cnt + 4, fail_list, sel, sel_count, c->proj_psd == 2,
                        c->proj_cnt + 5};
      launch_ring_t<float>(P, list, count, work, out, g, st, p1only, psd);
    }
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
  }
  return cudaSuccess;
}

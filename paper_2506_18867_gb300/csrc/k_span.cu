// K2: per-span membrane + bending energy, gradient and 27x27 Hessian.
//
// Per membrane point (FBW, Eqs. anisotropic invariants and FBW stretching
// and shearing energy):
//   f_beta = F e_beta = sum_l C_l g_l,beta,   I5(e_b) = |f_b|^2,  I6 = f_1 . f_2
//   Psi = mu_st1 (|f_1| - 1)^2 + mu_st2 (|f_2| - 1)^2 + mu_sh I6^2
// with the analytic derivatives w.r.t. (f_1, f_2) chained to the 27 span DOFs
// through g.  Per bending point (Eq. general bending energy with the
// Laplacian of Eq. (Laplacian in parametric space)):
//   Psi = mu_bd/2 |sum_l L_l C_l|^2   (quadratic, constant Hessian).
// The control points of the span are shifted by the span's centre control
// point before forming f (sum_l g_l = 0), which keeps FP32 strains accurate
// far from the origin.  Energies accumulate in FP64.
//
// A block evaluates 32 spans (one per lane) with 8 warps, each warp a slice
// of every span's work.  Phase 1 evaluates the quadrature points (slice k
// takes the span's points k and k + 8): energy, weighted dPsi/df, the
// weighted 6x6 d^2 Psi/df^2 (also kept in global memory for the FP64 span
// projection; under the per-point projection each FBW term's part is
// projected in closed form first, see membrane_hessian6) and the point's
// derivative vectors go to shared memory.
// Phase 2 sums them into the span terms: slice w owns the 3x3 blocks
// (l <= m) w, w + 8, ... of the Hessian (five or six of the 45) and
// gradient row w (slice 7 also row 8), accumulated in registers, so every
// store is a coalesced 32-span row of an entry plane.  Points come in
// rounds of ten slots per span (a corner span has nine membrane points and
// one bending point).
//
// Blocks take work items: a patch and either a run of 32 consecutive spans
// of it or a tu x (32 / tu) tile of spans, the tile shape chosen per
// patch-size class by the autotuner (bsc_autotune).  All patches of a
// context are evaluated by one launch.
//
// A tile's control-point footprint, (tu + 2) x (tv + 2) points of each of
// the three coordinate planes, is staged in shared memory by TMA: one box
// load per plane row from a rank-1 tensor map over the planes, the row's
// start rounded down to a 16-byte boundary (patch widths are arbitrary, so
// a 2-D map would violate TMA's stride alignment).  Runs of consecutive
// spans read their control points from global memory directly.
#include <cuda.h>
#include <cudaTypedefs.h>

#include <vector>

#include "bsc_internal.cuh"
#include "tc05.cuh"

namespace {

template <typename T>
struct SpanArgs {
  int N, Nsp, Nm, Nb;  // plane strides: totals over the patches
  const PatchDev* __restrict__ pd;
  const SpanItem* __restrict__ items;
  const PatchStep* __restrict__ gate;  // optional: evaluate pending line searches only
  const T* __restrict__ C;
  const int* __restrict__ moff;
  const int* __restrict__ boff;
  const T* __restrict__ tabm;
  const T* __restrict__ tabb;
  double* __restrict__ E;
  T* __restrict__ g;
  T* __restrict__ H;
  T* __restrict__ A;
  int* __restrict__ status;
};

// Block shape: SPB spans (lane = span) x SLICES warps.
constexpr int SPB = 32, SLICES = 8, EVAL_BLOCK = SPB * SLICES;
// Point slots per span and round, values per slot: membrane g (9 x 2),
// weighted d^2 Psi/df^2 (packed upper 6x6) and weighted dPsi/df (2 x 3);
// bending L (9), W mu_bd and the Laplacian sum_l L_l C_l (3).
constexpr int MAXPT = 10, NV = 45;
constexpr int V_G = 0, V_A = 18, V_DP = 39;
constexpr int V_L = 0, V_WB = 9, V_LAP = 10;
// The 45 3x3 blocks (l <= m) of the span Hessian; slice w owns blocks
// w + 8 i, i < BPS (six for w < 5, five otherwise).
constexpr int NBLK = 45, BPS = 6;

// TMA staging of a tile's control points: box width in elements (tile width
// 32 + 2 halo points + up to 3 elements of alignment slack, rounded to 16
// bytes), the row pitch in shared memory (128-byte aligned boxes) and the
// number of rows a block can hold (narrowest tile: 8 spans wide).
constexpr int TMA_W = 40;
template <typename T>
struct CTile {
  static constexpr int ALIGN = 16 / (int)sizeof(T);
  static constexpr int PITCH = (int)(((TMA_W * sizeof(T) + 127) / 128) * 128 / sizeof(T));
};
constexpr int ROWS = SPB / 8 + 2;
constexpr long long TMA_WAIT_LIMIT = 1ll << 24;

template <typename T>
constexpr size_t span_smem() {
  return 128 + sizeof(T) * 3 * ROWS * CTile<T>::PITCH + 16 + sizeof(T) * MAXPT * NV * SPB +
         sizeof(double) * MAXPT * SPB;
}

template <typename T> __device__ __forceinline__ T rsqrt_(T x);
template <> __device__ __forceinline__ float rsqrt_<float>(float x) { return rsqrtf(x); }
template <> __device__ __forceinline__ double rsqrt_<double>(double x) { return rsqrt(x); }

// (l, m), l <= m, of block b in row order.
__device__ __forceinline__ void block_lm(int b, int& l, int& m) {
  l = 0;
  int rem = b;
  while (rem >= 9 - l) {
    rem -= 9 - l;
    ++l;
  }
  m = l + rem;
}

// Weighted 6x6 d^2 Psi / d f_(b c) d f_(d e) of one membrane point (index
// 3 b + c), either as it is or, with PP, with each FBW term's Hessian
// replaced by its PSD projection (BSC_PROJECT_POINT).  k_b = 2 mu_b (1 - r_b)
// and ks = 2 mu_sh I6 are the gradient coefficients, r_b = 1 / |f_b|.
//
// Stretch term b, 2 mu_b [(1 - r) I + r^3 f f^T]: eigenvalue 2 mu_b along f
// and 2 mu_b (1 - r) twice across it; when |f| < 1 the second is clamped to
// 0, which leaves 2 mu_b r^2 f f^T.
//
// Shear term, 2 mu_sh [g g^T + I6 A] with g = (f_2; f_1) and A = [0 I; I 0].
// A is +1 on the vectors (x; x) and -1 on (x; -x); u = f_1 + f_2 and
// w = f_2 - f_1 are the parts of g in the two halves (|g_+|^2 = |u|^2 / 2,
// |g_-|^2 = |w|^2 / 2, and |g_+|^2 - |g_-|^2 = 2 I6).  Hence the spectrum:
//   +I6 on (x; x) with x perpendicular to u (two vectors),
//   -I6 on (x; -x) with x perpendicular to w (two vectors),
//   and the 2x2 block [[|g+|^2 + I6, |g+||g-|], [|g+||g-|, |g-|^2 - I6]] on
//   span(g_+, g_-): trace I5a + I5b, determinant -3 I6^2, so one eigenvalue
//   lam = (tr + sqrt(tr^2 + 12 I6^2)) / 2 >= 0 and one <= 0.
// The projection keeps max(I6, 0) and max(-I6, 0) on the first two families
// and lam v v^T with v = al g_+ + be g_- from the 2x2 eigenvector, written
// without dividing by |g_+| or |g_-| (al, be >= 0 below).
template <typename T, bool PP>
__device__ __forceinline__ void membrane_hessian6(const T f[2][3], T I5a, T I5b, T I6, T r1, T r2, T k1, T k2,
                                                  T ks, T mu1, T mu2, T mush, T W, T A6[6][6]) {
  T c1 = T(2) * mu1 * r1 * r1 * r1, c2 = T(2) * mu2 * r2 * r2 * r2;
  const T cs = T(2) * mush;
  if (!PP) {
#pragma unroll
    for (int c = 0; c < 3; ++c)
#pragma unroll
      for (int d = 0; d < 3; ++d) {
        const T del = (c == d) ? T(1) : T(0);
        A6[c][d] = W * (k1 * del + c1 * f[0][c] * f[0][d] + cs * f[1][c] * f[1][d]);
        A6[3 + c][3 + d] = W * (k2 * del + c2 * f[1][c] * f[1][d] + cs * f[0][c] * f[0][d]);
        A6[c][3 + d] = W * (cs * f[1][c] * f[0][d] + ks * del);
        A6[3 + d][c] = A6[c][3 + d];
      }
    return;
  }
  if (r1 > T(1)) { k1 = T(0); c1 = T(2) * mu1 * r1 * r1; }
  if (r2 > T(1)) { k2 = T(0); c2 = T(2) * mu2 * r2 * r2; }
  T u[3], w[3];
#pragma unroll
  for (int c = 0; c < 3; ++c) {
    u[c] = f[0][c] + f[1][c];
    w[c] = f[1][c] - f[0][c];
  }
  const T uu = u[0] * u[0] + u[1] * u[1] + u[2] * u[2], ww = w[0] * w[0] + w[1] * w[1] + w[2] * w[2];
  const T tr = I5a + I5b, sq = sqrt(tr * tr + T(12) * I6 * I6), lam = T(0.5) * (tr + sq);
  const bool pos = I6 >= T(0);
  const T al = pos ? T(2) * I6 + T(0.5) * sq : T(0.5) * ww;
  const T be = pos ? T(0.5) * uu : T(0.5) * sq - T(2) * I6;
  const T vv = T(0.5) * (al * al * uu + be * be * ww);  // |v|^2
  const T kv = vv > T(0) ? lam / vv : T(0);
  const T sp = pos ? I6 : T(0), sm = pos ? T(0) : -I6;
  const T iu = sp > T(0) ? T(1) / uu : T(0), iw = sm > T(0) ? T(1) / ww : T(0);
  T pv[3], qv[3];  // v = (p; q)
#pragma unroll
  for (int c = 0; c < 3; ++c) {
    pv[c] = T(0.5) * (al * u[c] + be * w[c]);
    qv[c] = T(0.5) * (al * u[c] - be * w[c]);
  }
#pragma unroll
  for (int c = 0; c < 3; ++c)
#pragma unroll
    for (int d = 0; d < 3; ++d) {
      const T del = (c == d) ? T(1) : T(0);
      const T Pu = T(0.5) * sp * (del - u[c] * u[d] * iu), Pw = T(0.5) * sm * (del - w[c] * w[d] * iw);
      A6[c][d] = W * (k1 * del + c1 * f[0][c] * f[0][d] + cs * (kv * pv[c] * pv[d] + Pu + Pw));
      A6[3 + c][3 + d] = W * (k2 * del + c2 * f[1][c] * f[1][d] + cs * (kv * qv[c] * qv[d] + Pu + Pw));
      A6[c][3 + d] = W * cs * (kv * pv[c] * qv[d] + Pu - Pw);
      A6[3 + d][c] = A6[c][3 + d];
    }
}

template <typename T, bool GRAD, bool HESS, bool PP>
__global__ void __launch_bounds__(EVAL_BLOCK, sizeof(T) == 4 ? 2 : 1)
    k_span_eval(SpanArgs<T> P, const __grid_constant__ CUtensorMap cmap) {
  extern __shared__ __align__(16) unsigned char smraw[];
  constexpr int PITCH = CTile<T>::PITCH, ALIGN = CTile<T>::ALIGN;
  const uint32_t pad = (128u - (tc05::smem_u32(smraw) & 127u)) & 127u;
  T* Ct = reinterpret_cast<T*>(smraw + pad);                 // [3][rows][PITCH] control-point boxes
  uint64_t* bar = reinterpret_cast<uint64_t*>(Ct + 3 * ROWS * PITCH);
  T* S = reinterpret_cast<T*>(bar + 2);                      // [MAXPT][NV][SPB] point slots
  double* Es = reinterpret_cast<double*>(S + MAXPT * NV * SPB);  // [MAXPT][SPB] point energies
  const SpanItem it = P.items[blockIdx.x];
  if (P.gate && P.gate[it.p].state != 1) return;
  const int j = threadIdx.x & 31, sl = threadIdx.x >> 5;
  const PatchDev* pt = P.pd + it.p;
  const int Su = __ldg(&pt->Su), nu = __ldg(&pt->nu), cp0 = __ldg(&pt->cp0);
  int a, b;
  bool valid;
  if (it.tu == 0) {
    const int sp = it.first_or_a0 + j;
    valid = sp < __ldg(&pt->Nsp);
    a = sp % Su;
    b = sp / Su;
  } else {
    a = it.first_or_a0 + j % it.tu;
    b = it.b0 + j / it.tu;
    valid = a < Su && b < __ldg(&pt->Sv);
  }
  // tile: stage the footprint rows of the three planes by TMA (block-uniform)
  const int rows = it.tu > 0 ? SPB / it.tu + 2 : 0;
  const bool staged = it.tu >= 8 && rows <= ROWS;
  const int gbase = cp0 + it.b0 * nu + it.first_or_a0;  // plane index of the tile's first control point
  if (staged) {
    const int nload = 3 * rows;
    if (threadIdx.x == 0) {
      tc05::mbar_init(bar, 1);
      tc05::fence_mbar_init();
    }
    __syncthreads();
    if (threadIdx.x < 32) {
      if (threadIdx.x == 0) tc05::mbar_arrive_expect_tx(bar, (uint32_t)(nload * TMA_W * sizeof(T)));
      __syncwarp();
      for (int i = threadIdx.x; i < nload; i += 32) {
        const int c = i / rows, r = i - c * rows;
        const int g = c * P.N + gbase + r * nu;
        tc05::tma_load_1d(Ct + i * PITCH, &cmap, g & ~(ALIGN - 1), bar);
      }
    }
    const bool landed = tc05::mbar_wait(bar, 0, TMA_WAIT_LIMIT);
    if (__syncthreads_or(!landed)) {  // the whole block leaves together
      if (threadIdx.x == 0) atomicOr(P.status, BSC_STATUS_TIMEOUT_FLAG);
      tc05::mbar_wait(bar, 0, TMA_WAIT_LIMIT);  // let the copies in flight land before leaving
      return;
    }
  }
  const int s = valid ? __ldg(&pt->sp0) + b * Su + a : 0;
  int q0 = 0, nm = 0, r0 = 0, nb = 0;
  if (valid) {
    q0 = P.moff[s];
    nm = P.moff[s + 1] - q0;
    r0 = P.boff[s];
    nb = P.boff[s + 1] - r0;
  }
  const int npt = nm + nb;
  const int mx = __reduce_max_sync(0xffffffffu, npt);  // the same in every warp (lane = span)
  const T mu1 = (T)__ldg(&pt->mu1), mu2 = (T)__ldg(&pt->mu2), mush = (T)__ldg(&pt->mush),
          mubd = (T)__ldg(&pt->mubd);
  const T* __restrict__ Cp = P.C + cp0;
  auto SV = [&](int k, int v) -> T& { return S[(k * NV + v) * SPB + j]; };

  // this slice's Hessian blocks and gradient rows
  int bl[BPS], bm[BPS];
#pragma unroll
  for (int i = 0; i < BPS; ++i) {
    bl[i] = bm[i] = 0;
    if (sl + SLICES * i < NBLK) block_lm(sl + SLICES * i, bl[i], bm[i]);
  }
  const int nblk = sl + SLICES * (BPS - 1) < NBLK ? BPS : BPS - 1;
  const int grow1 = sl == SLICES - 1 ? 8 : -1;
  T acc[BPS][3][3];
  T gacc[2][3];
#pragma unroll
  for (int i = 0; i < BPS; ++i)
#pragma unroll
    for (int c = 0; c < 3; ++c)
#pragma unroll
      for (int d = 0; d < 3; ++d) acc[i][c][d] = T(0);
#pragma unroll
  for (int r = 0; r < 2; ++r)
#pragma unroll
    for (int c = 0; c < 3; ++c) gacc[r][c] = T(0);
  double E = 0.0;

  for (int base = 0; base < mx; base += MAXPT) {
    // ---- phase 1: points base + sl and base + sl + 8 of the span
#pragma unroll 1
    for (int k = sl; k < MAXPT; k += SLICES) {
      const int pi = base + k;
      if (!valid || pi >= npt) continue;
      // control points relative to the span's centre control point
      T Cl[9][3];
      if (staged) {
        const int rr = b - it.b0, i0 = a - it.first_or_a0;
        const T* row[3][3];
#pragma unroll
        for (int c = 0; c < 3; ++c)
#pragma unroll
          for (int jj = 0; jj < 3; ++jj) {
            const int g = c * P.N + gbase + (rr + jj) * nu;
            row[c][jj] = Ct + (c * rows + rr + jj) * PITCH + (g & (ALIGN - 1)) + i0;
          }
        T c0[3];
#pragma unroll
        for (int c = 0; c < 3; ++c) c0[c] = row[c][1][1];
#pragma unroll
        for (int l = 0; l < 9; ++l)
#pragma unroll
          for (int c = 0; c < 3; ++c) Cl[l][c] = row[c][l / 3][l % 3] - c0[c];
      } else {
        const int ac = (b + 1) * nu + a + 1;
        T c0[3];
#pragma unroll
        for (int c = 0; c < 3; ++c) c0[c] = Cp[c * P.N + ac];
#pragma unroll
        for (int l = 0; l < 9; ++l) {
          const int al = (b + l / 3) * nu + a + l % 3;
#pragma unroll
          for (int c = 0; c < 3; ++c) Cl[l][c] = Cp[c * P.N + al] - c0[c];
        }
      }
      if (pi < nm) {
        const int q = q0 + pi;
        const T W = P.tabm[q];
        T gq[9][2];
#pragma unroll
        for (int l = 0; l < 9; ++l) {
          gq[l][0] = P.tabm[(1 + 2 * l) * P.Nm + q];
          gq[l][1] = P.tabm[(2 + 2 * l) * P.Nm + q];
        }
        T f[2][3];
#pragma unroll
        for (int be = 0; be < 2; ++be)
#pragma unroll
          for (int c = 0; c < 3; ++c) {
            T acc1 = T(0);
#pragma unroll
            for (int l = 0; l < 9; ++l) acc1 += Cl[l][c] * gq[l][be];
            f[be][c] = acc1;
          }
        const T I5a = f[0][0] * f[0][0] + f[0][1] * f[0][1] + f[0][2] * f[0][2];
        const T I5b = f[1][0] * f[1][0] + f[1][1] * f[1][1] + f[1][2] * f[1][2];
        const T I6 = f[0][0] * f[1][0] + f[0][1] * f[1][1] + f[0][2] * f[1][2];
        const T r1 = rsqrt_(I5a), r2 = rsqrt_(I5b);  // 1 / |f_b|
        const T s1 = I5a * r1, s2 = I5b * r2;
        const T e1 = s1 - T(1), e2 = s2 - T(1);
        Es[k * SPB + j] = (double)W * (double)(mu1 * e1 * e1 + mu2 * e2 * e2 + mush * I6 * I6);
        // dPsi/df_b = 2 mu_b (1 - 1/|f_b|) f_b + 2 mu_sh I6 f_other
        const T k1 = T(2) * mu1 * (T(1) - r1), k2 = T(2) * mu2 * (T(1) - r2), ks = T(2) * mush * I6;
        if (GRAD || HESS) {
#pragma unroll
          for (int l = 0; l < 9; ++l) {
            SV(k, V_G + 2 * l) = gq[l][0];
            SV(k, V_G + 2 * l + 1) = gq[l][1];
          }
        }
        if (GRAD) {
#pragma unroll
          for (int c = 0; c < 3; ++c) {
            SV(k, V_DP + c) = W * (k1 * f[0][c] + ks * f[1][c]);
            SV(k, V_DP + 3 + c) = W * (k2 * f[1][c] + ks * f[0][c]);
          }
        }
        if (HESS) {
          // weighted d^2 Psi / d f_(b c) d f_(d e), 6x6 with index 3 b + c
          T A6[6][6];
          membrane_hessian6<T, PP>(f, I5a, I5b, I6, r1, r2, k1, k2, ks, mu1, mu2, mush, W, A6);
          int e = 0;
#pragma unroll
          for (int r = 0; r < 6; ++r)
#pragma unroll
            for (int c = r; c < 6; ++c, ++e) {
              SV(k, V_A + e) = A6[r][c];
              if (!PP) P.A[(size_t)e * P.Nm + q] = A6[r][c];  // input of the span projection
            }
        }
      } else {
        const int q = r0 + pi - nm;
        const T WB = P.tabb[q] * mubd;  // W mu_bd
        T L[9];
#pragma unroll
        for (int l = 0; l < 9; ++l) L[l] = P.tabb[(1 + l) * P.Nb + q];
        T lap[3];
#pragma unroll
        for (int c = 0; c < 3; ++c) {
          T acc1 = T(0);
#pragma unroll
          for (int l = 0; l < 9; ++l) acc1 += L[l] * Cl[l][c];
          lap[c] = acc1;
        }
        Es[k * SPB + j] = 0.5 * (double)WB * (double)(lap[0] * lap[0] + lap[1] * lap[1] + lap[2] * lap[2]);
        if (GRAD || HESS) {
#pragma unroll
          for (int l = 0; l < 9; ++l) SV(k, V_L + l) = L[l];
          SV(k, V_WB) = WB;
#pragma unroll
          for (int c = 0; c < 3; ++c) SV(k, V_LAP + c) = lap[c];
        }
      }
    }
    __syncthreads();
    // ---- phase 2: this slice's blocks and rows, summed over the round's points
    const int kmax = valid ? min(MAXPT, npt - base) : 0;
    if (GRAD || HESS) {
#pragma unroll 1
      for (int k = 0; k < kmax; ++k) {
        if (base + k < nm) {
          if (HESS) {
            T A[6][6];
            int e = 0;
#pragma unroll
            for (int r = 0; r < 6; ++r)
#pragma unroll
              for (int c = r; c < 6; ++c, ++e) {
                A[r][c] = SV(k, V_A + e);
                A[c][r] = A[r][c];
              }
#pragma unroll
            for (int i = 0; i < BPS; ++i) {
              if (i >= nblk) break;
              const T gl0 = SV(k, V_G + 2 * bl[i]), gl1 = SV(k, V_G + 2 * bl[i] + 1);
              const T gm0 = SV(k, V_G + 2 * bm[i]), gm1 = SV(k, V_G + 2 * bm[i] + 1);
              // H_(l c)(m d) += sum_{beta, delta} g_l,beta g_m,delta A6[3 beta + c][3 delta + d]
#pragma unroll
              for (int c = 0; c < 3; ++c)
#pragma unroll
                for (int d = 0; d < 3; ++d) {
                  const T u = gm0 * A[c][d] + gm1 * A[c][3 + d];
                  const T v = gm0 * A[3 + c][d] + gm1 * A[3 + c][3 + d];
                  acc[i][c][d] = fma(gl1, v, fma(gl0, u, acc[i][c][d]));  // two FMAs, no separate product and add
                }
            }
          }
          if (GRAD) {
#pragma unroll
            for (int r = 0; r < 2; ++r) {
              const int l = r == 0 ? sl : grow1;
              if (l < 0) break;
              const T g0 = SV(k, V_G + 2 * l), g1 = SV(k, V_G + 2 * l + 1);
#pragma unroll
              for (int c = 0; c < 3; ++c) gacc[r][c] = fma(g1, SV(k, V_DP + 3 + c), fma(g0, SV(k, V_DP + c), gacc[r][c]));
            }
          }
        } else {
          const T WB = SV(k, V_WB);
          if (HESS) {
#pragma unroll
            for (int i = 0; i < BPS; ++i) {
              if (i >= nblk) break;
              const T h = WB * SV(k, V_L + bl[i]) * SV(k, V_L + bm[i]);
#pragma unroll
              for (int c = 0; c < 3; ++c) acc[i][c][c] += h;
            }
          }
          if (GRAD) {
#pragma unroll
            for (int r = 0; r < 2; ++r) {
              const int l = r == 0 ? sl : grow1;
              if (l < 0) break;
              const T wl = WB * SV(k, V_L + l);
#pragma unroll
              for (int c = 0; c < 3; ++c) gacc[r][c] += wl * SV(k, V_LAP + c);
            }
          }
        }
      }
    }
    if (sl == 0)
      for (int k = 0; k < kmax; ++k) E += Es[k * SPB + j];
    if (base + MAXPT < mx) __syncthreads();
  }

  if (!valid) return;
  if (sl == 0) P.E[s] = E;
  if (GRAD) {
#pragma unroll
    for (int r = 0; r < 2; ++r) {
      const int l = r == 0 ? sl : grow1;
      if (l < 0) break;
#pragma unroll
      for (int c = 0; c < 3; ++c) P.g[(size_t)(3 * l + c) * P.Nsp + s] = gacc[r][c];
    }
  }
  if (HESS) {
#pragma unroll
    for (int i = 0; i < BPS; ++i) {
      if (i >= nblk) break;
#pragma unroll
      for (int c = 0; c < 3; ++c)
#pragma unroll
        for (int d = 0; d < 3; ++d) {
          if (bl[i] == bm[i] && d < c) continue;
          P.H[(size_t)upk(3 * bl[i] + c, 3 * bm[i] + d, 27) * P.Nsp + s] = acc[i][c][d];
        }
    }
  }
}

// Energy only (no gradient, no Hessian): one thread per span, its points in
// the order of k_span_eval (membrane points, then bending points) with the
// same per-point arithmetic, so E_span is the same as that kernel's; without
// the slice structure a span costs a thread, not a warp's eight slices.
template <typename T>
__global__ void __launch_bounds__(128) k_span_energy(SpanArgs<T> P, const int* __restrict__ sp_patch) {
  const int s = blockIdx.x * blockDim.x + threadIdx.x;
  if (s >= P.Nsp) return;
  const int p = sp_patch[s];
  if (P.gate && P.gate[p].state != 1) return;
  const PatchDev* pt = P.pd + p;
  const int Su = __ldg(&pt->Su), nu = __ldg(&pt->nu), cp0 = __ldg(&pt->cp0), sp0 = __ldg(&pt->sp0);
  const int l0 = s - sp0, a = l0 % Su, b = l0 / Su;
  const T mu1 = (T)__ldg(&pt->mu1), mu2 = (T)__ldg(&pt->mu2), mush = (T)__ldg(&pt->mush),
          mubd = (T)__ldg(&pt->mubd);
  const T* __restrict__ Cp = P.C + cp0;
  T Cl[9][3];
  {
    const int ac = (b + 1) * nu + a + 1;
    T c0[3];
#pragma unroll
    for (int c = 0; c < 3; ++c) c0[c] = Cp[c * P.N + ac];
#pragma unroll
    for (int l = 0; l < 9; ++l) {
      const int al = (b + l / 3) * nu + a + l % 3;
#pragma unroll
      for (int c = 0; c < 3; ++c) Cl[l][c] = Cp[c * P.N + al] - c0[c];
    }
  }
  const int q0 = P.moff[s], nm = P.moff[s + 1] - q0, r0 = P.boff[s], nb = P.boff[s + 1] - r0;
  double E = 0.0;
  for (int pi = 0; pi < nm; ++pi) {
    const int q = q0 + pi;
    const T W = P.tabm[q];
    T gq[9][2];
#pragma unroll
    for (int l = 0; l < 9; ++l) {
      gq[l][0] = P.tabm[(1 + 2 * l) * P.Nm + q];
      gq[l][1] = P.tabm[(2 + 2 * l) * P.Nm + q];
    }
    T f[2][3];
#pragma unroll
    for (int be = 0; be < 2; ++be)
#pragma unroll
      for (int c = 0; c < 3; ++c) {
        T acc1 = T(0);
#pragma unroll
        for (int l = 0; l < 9; ++l) acc1 += Cl[l][c] * gq[l][be];
        f[be][c] = acc1;
      }
    const T I5a = f[0][0] * f[0][0] + f[0][1] * f[0][1] + f[0][2] * f[0][2];
    const T I5b = f[1][0] * f[1][0] + f[1][1] * f[1][1] + f[1][2] * f[1][2];
    const T I6 = f[0][0] * f[1][0] + f[0][1] * f[1][1] + f[0][2] * f[1][2];
    const T r1 = rsqrt_(I5a), r2 = rsqrt_(I5b);
    const T s1 = I5a * r1, s2 = I5b * r2;
    const T e1 = s1 - T(1), e2 = s2 - T(1);
    // the product rounded on its own, then added (as k_span_eval's staged point energies)
    E = __dadd_rn(E, (double)W * (double)(mu1 * e1 * e1 + mu2 * e2 * e2 + mush * I6 * I6));
  }
  for (int pi = 0; pi < nb; ++pi) {
    const int q = r0 + pi;
    const T WB = P.tabb[q] * mubd;
    T L[9];
#pragma unroll
    for (int l = 0; l < 9; ++l) L[l] = P.tabb[(1 + l) * P.Nb + q];
    T lap[3];
#pragma unroll
    for (int c = 0; c < 3; ++c) {
      T acc1 = T(0);
#pragma unroll
      for (int l = 0; l < 9; ++l) acc1 += L[l] * Cl[l][c];
      lap[c] = acc1;
    }
    E = __dadd_rn(E, 0.5 * (double)WB * (double)(lap[0] * lap[0] + lap[1] * lap[1] + lap[2] * lap[2]));
  }
  P.E[s] = E;
}

template <typename T>
SpanArgs<T> make_args(bsc_ctx* c, const void* C, const SpanItem* items, const PatchStep* gate) {
  SpanArgs<T> P;
  P.N = c->N; P.Nsp = c->Nsp; P.Nm = c->Nmem; P.Nb = c->Nbd;
  P.pd = c->pd; P.items = items; P.gate = gate;
  P.C = (const T*)C;
  P.moff = c->mem_off; P.boff = c->bd_off;
  P.tabm = (const T*)c->tab_mem; P.tabb = (const T*)c->tab_bd;
  P.E = c->E_span; P.g = (T*)c->g_span; P.H = (T*)c->H_span; P.A = (T*)c->A_mem;
  P.status = c->dstatus;
  return P;
}

// Rank-1 tiled tensor map over the three coordinate planes of C (3 N
// elements from a 16-byte aligned base), box TMA_W elements, zero fill past
// the end.  The encoder comes from the driver through the runtime.
template <typename T>
cudaError_t planes_map(CUtensorMap* m, const void* C, int N) {
  static PFN_cuTensorMapEncodeTiled_v12000 encode = nullptr;
  if (!encode) {
    void* fn = nullptr;
    cudaDriverEntryPointQueryResult q;
    cudaError_t e = cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &fn, 12000, cudaEnableDefault, &q);
    if (e != cudaSuccess) return e;
    if (q != cudaDriverEntryPointSuccess || !fn) return cudaErrorNotSupported;
    encode = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(fn);
  }
  if ((reinterpret_cast<uintptr_t>(C) & 15u) != 0 || 3ll * N >= (1ll << 31)) return cudaErrorInvalidValue;
  const cuuint64_t dim[1] = {(cuuint64_t)3 * (cuuint64_t)N};
  const cuuint64_t stride[1] = {0};  // rank 1: no strides
  const cuuint32_t box[1] = {(cuuint32_t)TMA_W}, estride[1] = {1};
  const CUresult r = encode(m, sizeof(T) == 4 ? CU_TENSOR_MAP_DATA_TYPE_FLOAT32 : CU_TENSOR_MAP_DATA_TYPE_FLOAT64, 1,
                            const_cast<void*>(C), dim, stride, box, estride, CU_TENSOR_MAP_INTERLEAVE_NONE,
                            CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_NONE,
                            CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  return r == CUDA_SUCCESS ? cudaSuccess : cudaErrorInvalidValue;
}

template <typename T>
cudaError_t run(bsc_ctx* c, const void* C, int want_grad, int want_hess, const SpanItem* items, int n_items,
                const PatchStep* gate) {
  if (n_items <= 0) return cudaSuccess;
  SpanArgs<T> P = make_args<T>(c, C, items, gate);
  if (!want_grad && !want_hess && items == c->span_items) {
    k_span_energy<T><<<(c->Nsp + 127) / 128, 128, 0, c->stream>>>(P, c->sp_patch);
    return cudaGetLastError();
  }
  CUtensorMap m;
  cudaError_t e = planes_map<T>(&m, C, c->N);
  if (e != cudaSuccess) return e;
  if (want_hess == 2)
    k_span_eval<T, true, true, true><<<n_items, EVAL_BLOCK, span_smem<T>(), c->stream>>>(P, m);
  else if (want_hess)
    k_span_eval<T, true, true, false><<<n_items, EVAL_BLOCK, span_smem<T>(), c->stream>>>(P, m);
  else if (want_grad)
    k_span_eval<T, true, false, false><<<n_items, EVAL_BLOCK, span_smem<T>(), c->stream>>>(P, m);
  else
    k_span_eval<T, false, false, false><<<n_items, EVAL_BLOCK, span_smem<T>(), c->stream>>>(P, m);
  return cudaGetLastError();
}

template <typename T>
cudaError_t set_smem() {
  const int bytes = (int)span_smem<T>();
  cudaError_t e;
  if ((e = cudaFuncSetAttribute(k_span_eval<T, true, true, true>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                bytes)) != cudaSuccess)
    return e;
  if ((e = cudaFuncSetAttribute(k_span_eval<T, true, true, false>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                bytes)) != cudaSuccess)
    return e;
  if ((e = cudaFuncSetAttribute(k_span_eval<T, true, false, false>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                bytes)) != cudaSuccess)
    return e;
  return cudaFuncSetAttribute(k_span_eval<T, false, false, false>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                              bytes);
}

}  // namespace

int span_block(int) { return SPB; }

// The point slots exceed 48 KB of shared memory: opt in once per context.
cudaError_t setup_span_eval(bsc_ctx* c) {
  return c->precision == BSC_FP64 ? set_smem<double>() : set_smem<float>();
}

// Work items of every patch (or of one size class) with the tile shape of
// its size class (or tu_override >= 0).
void plan_span_items(const bsc_ctx* c, std::vector<SpanItem>& out, int only_class, int tu_override) {
  const int B = span_block(c->precision);
  out.clear();
  for (int p = 0; p < c->P; ++p) {
    const PatchDev& q = c->hpd[p];
    const int cls = tile_class_of(q.Su);
    if (only_class >= 0 && cls != only_class) continue;
    const int tu = tu_override >= 0 ? tu_override : c->tile_tu[cls];
    if (tu == 0) {
      for (int f = 0; f < q.Nsp; f += B) out.push_back(SpanItem{p, f, 0, 0});
    } else {
      const int tv = B / tu;
      for (int b0 = 0; b0 < q.Sv; b0 += tv)
        for (int a0 = 0; a0 < q.Su; a0 += tu) out.push_back(SpanItem{p, a0, tu, b0});
    }
  }
}

cudaError_t build_span_items(bsc_ctx* c) {
  std::vector<SpanItem> items;
  plan_span_items(c, items, -1, -1);
  cudaError_t e;
  if (c->span_items) {
    if ((e = cudaStreamSynchronize(c->stream)) != cudaSuccess) return e;
    cudaFree(c->span_items);
    c->span_items = nullptr;
  }
  if ((e = cudaMalloc(&c->span_items, sizeof(SpanItem) * (items.size() ? items.size() : 1))) != cudaSuccess) return e;
  c->n_span_items = (int)items.size();
  if ((e = cudaMemcpy(c->span_items, items.data(), sizeof(SpanItem) * items.size(), cudaMemcpyHostToDevice)) !=
      cudaSuccess)
    return e;
  c->graph_C = c->graph_Chat = nullptr;  // a captured graph holds the old item list
  return cudaSuccess;
}

cudaError_t launch_span_eval_items(bsc_ctx* c, const void* C, int want_grad, int want_hess, const SpanItem* items,
                                   int n_items, int) {
  BSC_COUNT(c, 1);
  if (c->precision == BSC_FP64) return run<double>(c, C, want_grad, want_hess, items, n_items, nullptr);
  return run<float>(c, C, want_grad, want_hess, items, n_items, nullptr);
}

cudaError_t launch_span_eval(bsc_ctx* c, const void* C, int want_grad, int want_hess, const PatchStep* gate) {
  BSC_COUNT(c, 1);
  if (c->precision == BSC_FP64) return run<double>(c, C, want_grad, want_hess, c->span_items, c->n_span_items, gate);
  return run<float>(c, C, want_grad, want_hess, c->span_items, c->n_span_items, gate);
}

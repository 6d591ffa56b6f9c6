// K5 / K6: stencil SpMV and the preconditioned CG that solves K d = -g.
//
// SpMV: y_alpha = sum over the 25 stencil slots of K(alpha, slot) x_beta; one
// thread per control point reads its 225 matrix entries from 225 planes
// (coalesced across threads) and the neighbours' x (through the read-only
// path in the stand-alone SpMV, where x does not change).
//
// PCG: 3x3 block-Jacobi preconditioned CG in a single persistent cooperative
// kernel.  The co-resident blocks are split into one group per patch (the
// split weighted by each patch's expected work, bsc_plan_blocks); every group
// runs its patch's CG on its own and leaves when that patch converges.  A
// group's blocks own fixed slices of the patch's control points; the three
// reductions per iteration (p.q, r.z, r.r) are FP64, summed per block in a
// fixed tree and across the group's blocks in block order, so every block of
// the group computes the same scalars and the result is bitwise reproducible
// for a given split.  Group barriers are bounded (they raise a timeout flag
// instead of waiting forever).
#include <algorithm>
#include <vector>

#include "bsc_internal.cuh"

namespace {

// Stand-alone SpMV: one thread per (output component c, control point):
// it reads the 75 entries of row c of the point's 25 blocks (coalesced over
// consecutive points) and the neighbours' x through the read-only path.
// Three threads per point keep three times as many independent K reads in
// flight as one thread per point would.
template <typename T>
__global__ void __launch_bounds__(256) k_spmv(int N, const PatchDev* __restrict__ pd, const int* __restrict__ cp_patch,
                                              const T* __restrict__ K, const T* __restrict__ x, T* __restrict__ y) {
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= 3 * N) return;
  const int c = t / N, al = t - c * N;
  const PatchDev* pt = pd + cp_patch[al];
  const int cp0 = __ldg(&pt->cp0), nu = __ldg(&pt->nu), nv = __ldg(&pt->nv);
  const int a = al - cp0, i = a % nu, j = a / nu;
  const T* __restrict__ Kp = K + cp0;
  const T* __restrict__ xp = x + cp0;
  // FP64: one FMA chain per column of the blocks, three independent chains
  // (fewest FP64 instructions: the FP64 pipe bounds this product).  FP32: a
  // product, an FMA and an add per block, measured faster there.
  T acc0 = T(0), acc1 = T(0), acc2 = T(0);
#pragma unroll
  for (int dv = -2; dv <= 2; ++dv) {
    const int jb = j + dv;
    if (jb < 0 || jb >= nv) continue;
#pragma unroll
    for (int du = -2; du <= 2; ++du) {
      const int ib = i + du;
      if (ib < 0 || ib >= nu) continue;
      const int slot = (dv + 2) * 5 + (du + 2), be = jb * nu + ib;
      const T* Kb = Kp + (size_t)(slot * 9 + 3 * c) * N + a;
      if (sizeof(T) == 8) {
        acc0 = fma(Kb[0], __ldg(xp + be), acc0);
        acc1 = fma(Kb[(size_t)N], __ldg(xp + N + be), acc1);
        acc2 = fma(Kb[(size_t)2 * N], __ldg(xp + 2 * N + be), acc2);
      } else {
        acc0 += Kb[0] * __ldg(xp + be) + Kb[(size_t)N] * __ldg(xp + N + be) +
                Kb[(size_t)2 * N] * __ldg(xp + 2 * N + be);
      }
    }
  }
  y[(size_t)c * N + al] = acc0 + acc1 + acc2;
}

// Stand-alone SpMV with K in the symmetric layout: a thread per control point.
template <typename T>
__global__ void __launch_bounds__(256) k_spmv_sym(int N, const PatchDev* __restrict__ pd,
                                                  const int* __restrict__ cp_patch, const T* __restrict__ K,
                                                  const T* __restrict__ x, T* __restrict__ y) {
  const int al = blockIdx.x * blockDim.x + threadIdx.x;
  if (al >= N) return;
  const PatchDev* pt = pd + cp_patch[al];
  const int cp0 = __ldg(&pt->cp0), nu = __ldg(&pt->nu), nv = __ldg(&pt->nv);
  T o[3];
  spmv_row_sym<T, 1>(nu, nv, N, al - cp0, K + cp0, x + cp0, o);
#pragma unroll
  for (int c = 0; c < 3; ++c) y[(size_t)c * N + al] = o[c];
}

// Inverse of each 3x3 diagonal block (adjugate / determinant, FP64); slot:
// the diagonal block's slot (12 in the full layout, 0 in the symmetric one).
template <typename T>
__global__ void k_block_jacobi(int N, const T* __restrict__ K, T* __restrict__ Dinv, int* status, int slot) {
  const int al = blockIdx.x * blockDim.x + threadIdx.x;
  if (al >= N) return;
  block_jacobi_at<T>(N, al, K, Dinv, status, slot);
}

template <typename T>
struct PcgArgs {
  int N, maxit;                       // N: plane stride of all vectors
  double tol;
  const PatchDev* __restrict__ pd;    // nullptr: one nu x nv patch at control point 0
  const PcgBlock* __restrict__ blocks;  // nullptr: one group of all blocks
  int nu, nv;                         // the patch when pd == nullptr
  const T* __restrict__ K;
  const T* __restrict__ Dinv;
  const T* __restrict__ b;
  T* __restrict__ x;
  T* __restrict__ r;
  T* __restrict__ z;
  T* __restrict__ p;
  T* __restrict__ q;
  double* __restrict__ partial;  // [3][gridDim.x]
  unsigned int* sync;            // [2 per patch]: barrier count, generation
  int* status;
  double* out;                   // [3 per patch]: iterations, relative residual, ok
  long long wait_limit;          // spins of the bounded group barriers
  unsigned int extra;            // blocks the barriers expect beyond the group (0; > 0 only in tests)
  const double* gate;            // fallback of a learned solve: its (iterations, r.r, state), else nullptr
  const double* gate_bb;         //   and its b.b
};

// Sum of part[0..n) in a fixed order (all threads get the result).
template <int BLOCK>
__device__ __forceinline__ double group_sum(const double* part, int n, double* sm) {
  double acc = 0.0;
  for (int k = threadIdx.x; k < n; k += BLOCK) acc += part[k];
  const double s = block_sum<BLOCK>(acc, sm);
  __shared__ double bcast;
  if (threadIdx.x == 0) bcast = s;
  __syncthreads();
  return bcast;
}

// FORM 0: three passes and group barriers per iteration (q = K p; x, r, z;
// p = z + beta p).  FORM 2: two, by linearity of the product: the first pass
// forms w = K z and updates q = w + beta q and p = z + beta p in place (q
// stays K p up to rounding), the second updates x, r, z; the direction no
// longer needs a pass and a barrier of its own.  Same iterates in exact
// arithmetic; q is carried by a recurrence, as r is in both forms.
// SYM: K in the symmetric layout (spmv_row_sym; the same products).
template <typename T, int BLOCK, int FORM, bool SYM>
__global__ void __launch_bounds__(BLOCK) k_pcg(PcgArgs<T> A) {
  __shared__ double sm[BLOCK / 32];
  const int G = gridDim.x, N = A.N;
  int pp = 0, rank = blockIdx.x, gsize = G, gfirst = 0;
  if (A.blocks) {
    const PcgBlock bk = A.blocks[blockIdx.x];
    pp = bk.p; rank = bk.rank; gsize = bk.size; gfirst = bk.first;
  }
  int nu = A.nu, nv = A.nv, cp0 = 0;
  if (A.pd) {
    nu = A.pd[pp].nu; nv = A.pd[pp].nv; cp0 = A.pd[pp].cp0;
  }
  const int Np = nu * nv;
  const int tid = rank * BLOCK + threadIdx.x, stride = gsize * BLOCK;
  unsigned int* cnt = A.sync + 2 * pp;
  volatile unsigned int* gen = A.sync + 2 * pp + 1;
  const unsigned int nb = (unsigned int)gsize + A.extra;
  const long long lim = A.wait_limit;
  double tol = A.tol;
  if (A.gate) {
    // fallback of a learned flexible CG: nothing to do when it converged
    // (state 1); otherwise finish its remaining residual b
    const double state = A.gate[2], rr0 = A.gate[1], bb0 = *A.gate_bb;
    if (state == 1.0) {
      for (int al = tid; al < Np; al += stride)
#pragma unroll
        for (int c = 0; c < 3; ++c) A.x[cp0 + c * N + al] = T(0);
      if (rank == 0 && threadIdx.x == 0) {
        double* o = A.out + 3 * pp;
        o[0] = 0.0;
        o[1] = 0.0;
        o[2] = 1.0;
      }
      return;
    }
    const double t = rr0 > 0.0 ? A.tol * sqrt(bb0 / rr0) : 0.5;
    tol = t < 0.5 ? t : 0.5;
  }
  // the patch's slice of every plane
  const T* __restrict__ K = A.K + cp0;
  const T* __restrict__ Dinv = A.Dinv + cp0;
  const T* __restrict__ bv = A.b + cp0;
  T* __restrict__ xv = A.x + cp0;
  T* __restrict__ rv = A.r + cp0;
  T* __restrict__ zv = A.z + cp0;
  T* __restrict__ pv = A.p + cp0;
  T* __restrict__ qv = A.q + cp0;
  double* const part0 = A.partial + gfirst;
  double* const part1 = A.partial + G + gfirst;
  double* const part2 = A.partial + 2 * G + gfirst;

  double l_rz = 0.0, l_bb = 0.0;
  for (int al = tid; al < Np; al += stride) {
    T rr[3], zz[3];
#pragma unroll
    for (int c = 0; c < 3; ++c) {
      xv[c * N + al] = T(0);
      rr[c] = bv[c * N + al];
      rv[c * N + al] = rr[c];
    }
    apply_dinv<T>(Dinv, N, al, rr, zz);
#pragma unroll
    for (int c = 0; c < 3; ++c) {
      zv[c * N + al] = zz[c];
      pv[c * N + al] = FORM == 2 ? T(0) : zz[c];
      if (FORM == 2) qv[c * N + al] = T(0);
      l_rz += (double)rr[c] * (double)zz[c];
      l_bb += (double)rr[c] * (double)rr[c];
    }
  }
  {
    const double s1 = block_sum<BLOCK>(l_rz, sm);
    const double s2 = block_sum<BLOCK>(l_bb, sm);
    if (threadIdx.x == 0) {
      part0[rank] = s1;
      part1[rank] = s2;
    }
  }
  if (!group_barrier(cnt, gen, A.status, nb, lim)) {
    if (rank == 0 && threadIdx.x == 0) {
      double* o = A.out + 3 * pp;
      o[0] = 0.0;
      o[1] = 1.0;
      o[2] = 0.0;
    }
    return;
  }
  double rz = group_sum<BLOCK>(part0, gsize, sm);
  const double bb = group_sum<BLOCK>(part1, gsize, sm);
  const double stop2 = tol * tol * bb;
  int it = 0;
  double rr_glob = bb, beta = 0.0;
  bool ok = true;
  if (bb > 0.0) {
    for (it = 1; it <= A.maxit; ++it) {
      double l_pq = 0.0;
      if (FORM == 2) {
        const T tb = (T)beta;
        for (int al = tid; al < Np; al += stride) {
          // the row's own q and p are loaded before its stencil product, so
          // their DRAM latency overlaps the matrix loads
          T qo[3], po[3];
#pragma unroll
          for (int c = 0; c < 3; ++c) {
            qo[c] = qv[c * N + al];
            po[c] = pv[c * N + al];
          }
          T y[3];
          if (SYM) spmv_row_sym<T>(nu, nv, N, al, K, zv, y);
          else spmv_row<T>(nu, nv, N, al, K, zv, y);
#pragma unroll
          for (int c = 0; c < 3; ++c) {
            const int k = c * N + al;
            const T q_ = y[c] + tb * qo[c];
            const T p_ = zv[k] + tb * po[c];
            qv[k] = q_;
            pv[k] = p_;
            l_pq += (double)p_ * (double)q_;
          }
        }
      } else {
        for (int al = tid; al < Np; al += stride) {
          T y[3];
          // plain loads of the neighbours' p (measured faster here than via L2)
          if (SYM) spmv_row_sym<T>(nu, nv, N, al, K, pv, y);
          else spmv_row<T>(nu, nv, N, al, K, pv, y);
#pragma unroll
          for (int c = 0; c < 3; ++c) {
            qv[c * N + al] = y[c];
            l_pq += (double)pv[c * N + al] * (double)y[c];
          }
        }
      }
      {
        const double s = block_sum<BLOCK>(l_pq, sm);
        if (threadIdx.x == 0) part2[rank] = s;
      }
      if (!(ok = group_barrier(cnt, gen, A.status, nb, lim))) break;
      const double pq = group_sum<BLOCK>(part2, gsize, sm);
      if (!(pq > 0.0) || !isfinite(pq)) {
        if (threadIdx.x == 0 && rank == 0) atomicOr(A.status, BSC_STATUS_NUMERIC_FLAG);
        ok = false;
        break;
      }
      const double alpha = rz / pq;
      const T ta = (T)alpha;
      double l_rz2 = 0.0, l_rr = 0.0;
      for (int al = tid; al < Np; al += stride) {
        T rr[3], zz[3];
#pragma unroll
        for (int c = 0; c < 3; ++c) {
          xv[c * N + al] += ta * pv[c * N + al];
          rr[c] = rv[c * N + al] - ta * qv[c * N + al];
          rv[c * N + al] = rr[c];
        }
        apply_dinv<T>(Dinv, N, al, rr, zz);
#pragma unroll
        for (int c = 0; c < 3; ++c) {
          zv[c * N + al] = zz[c];
          l_rz2 += (double)rr[c] * (double)zz[c];
          l_rr += (double)rr[c] * (double)rr[c];
        }
      }
      {
        const double s1 = block_sum<BLOCK>(l_rz2, sm);
        const double s2 = block_sum<BLOCK>(l_rr, sm);
        if (threadIdx.x == 0) {
          part0[rank] = s1;
          part1[rank] = s2;
        }
      }
      if (!(ok = group_barrier(cnt, gen, A.status, nb, lim))) break;
      const double rz2 = group_sum<BLOCK>(part0, gsize, sm);
      rr_glob = group_sum<BLOCK>(part1, gsize, sm);
      if (rr_glob <= stop2 || !isfinite(rr_glob)) break;
      beta = rz2 / rz;
      rz = rz2;
      if (FORM == 0) {
        const T tb = (T)beta;
        for (int al = tid; al < Np; al += stride)
#pragma unroll
          for (int c = 0; c < 3; ++c) pv[c * N + al] = zv[c * N + al] + tb * pv[c * N + al];
        if (!(ok = group_barrier(cnt, gen, A.status, nb, lim))) break;
      }
    }
  }
  if (rank == 0 && threadIdx.x == 0) {
    double* o = A.out + 3 * pp;
    o[0] = (double)(it > A.maxit ? A.maxit : it);
    o[1] = bb > 0.0 ? sqrt(rr_glob / bb) : 0.0;
    o[2] = ok ? 1.0 : 0.0;
  }
}

// The pipelined form of the same block-Jacobi PCG (Ghysels & Vanroose 2014,
// "Hiding global synchronization latency in the preconditioned conjugate
// gradient algorithm"): with u = M r, w = K u, m = M w, n = K m carried by
// recurrences, the three dot products of an iteration, (r, u), (w, u) and
// (r, r), are formed in one pass and need one group barrier, which also
// publishes m for the next product.  Per iteration and row:
//   n = K m;  z = n + b z;  q = m + b q;  s = w + b s;  p = u + b p;
//   x += a p;  r -= a s;  u -= a q;  w -= a z;  m' = M w  (into the other m buffer)
// with b = g / g_old, a = g / (d - b g / a_old), g = (r, u), d = (w, u).
// m is double-buffered: the rows of a group read their neighbours' m while
// other rows already write the next one.  Mathematically the iterates are
// those of k_pcg; rounding differs (the recurrences drift from the true
// residual a little faster).  Two barriers set up u and w; then one per
// iteration instead of three.
template <typename T>
struct PipeVecs {
  T* __restrict__ u;
  T* __restrict__ w;
  T* __restrict__ m0;
  T* __restrict__ m1;
  T* __restrict__ s;
  T* __restrict__ z2;   // z of the recurrences (K m carried)
};

// Register-capped to the four blocks of 256 per SM of the other forms: all
// forms share one grid, the co-resident capacity of the most demanding.
template <typename T, int BLOCK, bool SYM>
__global__ void __launch_bounds__(BLOCK, 4) k_pcg_pipe(PcgArgs<T> A, PipeVecs<T> V) {
  __shared__ double sm[BLOCK / 32];
  const int G = gridDim.x, N = A.N;
  int pp = 0, rank = blockIdx.x, gsize = G, gfirst = 0;
  if (A.blocks) {
    const PcgBlock bk = A.blocks[blockIdx.x];
    pp = bk.p; rank = bk.rank; gsize = bk.size; gfirst = bk.first;
  }
  int nu = A.nu, nv = A.nv, cp0 = 0;
  if (A.pd) {
    nu = A.pd[pp].nu; nv = A.pd[pp].nv; cp0 = A.pd[pp].cp0;
  }
  const int Np = nu * nv;
  const int tid = rank * BLOCK + threadIdx.x, stride = gsize * BLOCK;
  unsigned int* cnt = A.sync + 2 * pp;
  volatile unsigned int* gen = A.sync + 2 * pp + 1;
  const unsigned int nb = (unsigned int)gsize + A.extra;
  const long long lim = A.wait_limit;
  double tol = A.tol;
  if (A.gate) {
    const double state = A.gate[2], rr0 = A.gate[1], bb0 = *A.gate_bb;
    if (state == 1.0) {
      for (int al = tid; al < Np; al += stride)
#pragma unroll
        for (int c = 0; c < 3; ++c) A.x[cp0 + c * N + al] = T(0);
      if (rank == 0 && threadIdx.x == 0) {
        double* o = A.out + 3 * pp;
        o[0] = 0.0;
        o[1] = 0.0;
        o[2] = 1.0;
      }
      return;
    }
    const double t = rr0 > 0.0 ? A.tol * sqrt(bb0 / rr0) : 0.5;
    tol = t < 0.5 ? t : 0.5;
  }
  const T* __restrict__ K = A.K + cp0;
  const T* __restrict__ Dinv = A.Dinv + cp0;
  const T* __restrict__ bv = A.b + cp0;
  T* __restrict__ xv = A.x + cp0;
  T* __restrict__ rv = A.r + cp0;
  T* __restrict__ pv = A.p + cp0;
  T* __restrict__ qv = A.q + cp0;
  T* __restrict__ uv = V.u + cp0;
  T* __restrict__ wv = V.w + cp0;
  T* __restrict__ sv = V.s + cp0;
  T* __restrict__ zv = V.z2 + cp0;
  T* mb[2] = {V.m0 + cp0, V.m1 + cp0};
  double* const part0 = A.partial + gfirst;
  double* const part1 = A.partial + G + gfirst;
  double* const part2 = A.partial + 2 * G + gfirst;
  double* const o = A.out + 3 * pp;
  auto fail_out = [&]() {
    if (rank == 0 && threadIdx.x == 0) {
      o[0] = 0.0;
      o[1] = 1.0;
      o[2] = 0.0;
    }
  };

  // x = 0, r = b, u = M r; the recurrence vectors start at zero
  for (int al = tid; al < Np; al += stride) {
    T rr[3], uu[3];
#pragma unroll
    for (int c = 0; c < 3; ++c) {
      xv[c * N + al] = T(0);
      pv[c * N + al] = T(0);
      qv[c * N + al] = T(0);
      sv[c * N + al] = T(0);
      zv[c * N + al] = T(0);
      rr[c] = bv[c * N + al];
      rv[c * N + al] = rr[c];
    }
    apply_dinv<T>(Dinv, N, al, rr, uu);
#pragma unroll
    for (int c = 0; c < 3; ++c) uv[c * N + al] = uu[c];
  }
  if (!group_barrier(cnt, gen, A.status, nb, lim)) {
    fail_out();
    return;
  }
  // w = K u, m = M w, and the first dot products
  {
    double l_g = 0.0, l_d = 0.0, l_r = 0.0;
    for (int al = tid; al < Np; al += stride) {
      T ww[3], mm[3];
      if (SYM) spmv_row_sym<T>(nu, nv, N, al, K, uv, ww);
      else spmv_row<T>(nu, nv, N, al, K, uv, ww);
      apply_dinv<T>(Dinv, N, al, ww, mm);
#pragma unroll
      for (int c = 0; c < 3; ++c) {
        wv[c * N + al] = ww[c];
        mb[0][c * N + al] = mm[c];
        const double r_ = (double)rv[c * N + al], u_ = (double)uv[c * N + al];
        l_g += r_ * u_;
        l_d += (double)ww[c] * u_;
        l_r += r_ * r_;
      }
    }
    const double s1 = block_sum<BLOCK>(l_g, sm), s2 = block_sum<BLOCK>(l_d, sm), s3 = block_sum<BLOCK>(l_r, sm);
    if (threadIdx.x == 0) {
      part0[rank] = s1;
      part1[rank] = s2;
      part2[rank] = s3;
    }
  }
  if (!group_barrier(cnt, gen, A.status, nb, lim)) {
    fail_out();
    return;
  }
  double gam = group_sum<BLOCK>(part0, gsize, sm);
  double del = group_sum<BLOCK>(part1, gsize, sm);
  const double bb = group_sum<BLOCK>(part2, gsize, sm);
  const double stop2 = tol * tol * bb;
  double rr_glob = bb, gam_old = 1.0, alpha_old = 1.0;
  int it = 0, cur = 0;
  bool ok = true;
  if (bb > 0.0) {
    for (it = 1; it <= A.maxit; ++it) {
      double beta = 0.0, den = del;
      if (it > 1) {
        beta = gam / gam_old;
        den = del - beta * gam / alpha_old;
      }
      if (!(den > 0.0) || !isfinite(den) || !(gam > 0.0)) {
        if (threadIdx.x == 0 && rank == 0) atomicOr(A.status, BSC_STATUS_NUMERIC_FLAG);
        ok = false;
        break;
      }
      const double alpha = gam / den;
      const T ta = (T)alpha, tb = (T)beta;
      const T* __restrict__ mc = mb[cur];
      T* __restrict__ mn = mb[cur ^ 1];
      double l_g = 0.0, l_d = 0.0, l_r = 0.0;
      for (int al = tid; al < Np; al += stride) {
        T nn[3];
        if (SYM) spmv_row_sym<T>(nu, nv, N, al, K, mc, nn);
        else spmv_row<T>(nu, nv, N, al, K, mc, nn);
        T ww[3], uu[3], rr_[3];
#pragma unroll
        for (int c = 0; c < 3; ++c) {
          const int k = c * N + al;
          const T z_ = nn[c] + tb * zv[k];
          const T q_ = mc[k] + tb * qv[k];
          const T s_ = wv[k] + tb * sv[k];
          const T p_ = uv[k] + tb * pv[k];
          zv[k] = z_; qv[k] = q_; sv[k] = s_; pv[k] = p_;
          xv[k] += ta * p_;
          rr_[c] = rv[k] - ta * s_;
          uu[c] = uv[k] - ta * q_;
          ww[c] = wv[k] - ta * z_;
          rv[k] = rr_[c]; uv[k] = uu[c]; wv[k] = ww[c];
        }
        T mm[3];
        apply_dinv<T>(Dinv, N, al, ww, mm);
#pragma unroll
        for (int c = 0; c < 3; ++c) {
          mn[c * N + al] = mm[c];
          l_g += (double)rr_[c] * (double)uu[c];
          l_d += (double)ww[c] * (double)uu[c];
          l_r += (double)rr_[c] * (double)rr_[c];
        }
      }
      {
        const double s1 = block_sum<BLOCK>(l_g, sm), s2 = block_sum<BLOCK>(l_d, sm),
                     s3 = block_sum<BLOCK>(l_r, sm);
        if (threadIdx.x == 0) {
          part0[rank] = s1;
          part1[rank] = s2;
          part2[rank] = s3;
        }
      }
      if (!(ok = group_barrier(cnt, gen, A.status, nb, lim))) break;
      gam_old = gam;
      alpha_old = alpha;
      gam = group_sum<BLOCK>(part0, gsize, sm);
      del = group_sum<BLOCK>(part1, gsize, sm);
      rr_glob = group_sum<BLOCK>(part2, gsize, sm);
      cur ^= 1;
      if (rr_glob <= stop2 || !isfinite(rr_glob)) break;
    }
  }
  if (rank == 0 && threadIdx.x == 0) {
    o[0] = (double)(it > A.maxit ? A.maxit : it);
    o[1] = bb > 0.0 ? sqrt(rr_glob / bb) : 0.0;
    o[2] = ok ? 1.0 : 0.0;
  }
}

template <typename T>
__global__ void k_axpy(int n, const T* __restrict__ a, const T* __restrict__ d, double alpha, T* __restrict__ out) {
  const int k = blockIdx.x * blockDim.x + threadIdx.x;
  if (k < n) out[k] = a[k] + (T)alpha * d[k];
}

constexpr int PCG_BLOCK = 256;

// Cooperative launch (all blocks co-resident, which the group barriers
// need) through the extended launch API, so that it can be captured in a
// CUDA graph.
template <typename T>
cudaLaunchConfig_t coop_config(int grid, cudaStream_t st, cudaLaunchAttribute* attr) {
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3((unsigned)grid);
  cfg.blockDim = dim3(PCG_BLOCK);
  cfg.dynamicSmemBytes = 0;
  cfg.stream = st;
  attr[0].id = cudaLaunchAttributeCooperative;
  attr[0].val.cooperative = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  return cfg;
}

template <typename T>
cudaError_t launch_coop(int grid, PcgArgs<T> A, cudaStream_t st, int form = 0, int sym = 0) {
  cudaLaunchAttribute attr[1];
  cudaLaunchConfig_t cfg = coop_config<T>(grid, st, attr);
  if (form == 2)
    return sym ? cudaLaunchKernelEx(&cfg, k_pcg<T, PCG_BLOCK, 2, true>, A)
               : cudaLaunchKernelEx(&cfg, k_pcg<T, PCG_BLOCK, 2, false>, A);
  return sym ? cudaLaunchKernelEx(&cfg, k_pcg<T, PCG_BLOCK, 0, true>, A)
             : cudaLaunchKernelEx(&cfg, k_pcg<T, PCG_BLOCK, 0, false>, A);
}

template <typename T>
cudaError_t launch_coop_pipe(int grid, PcgArgs<T> A, PipeVecs<T> V, cudaStream_t st, int sym = 0) {
  cudaLaunchAttribute attr[1];
  cudaLaunchConfig_t cfg = coop_config<T>(grid, st, attr);
  return sym ? cudaLaunchKernelEx(&cfg, k_pcg_pipe<T, PCG_BLOCK, true>, A, V)
             : cudaLaunchKernelEx(&cfg, k_pcg_pipe<T, PCG_BLOCK, false>, A, V);
}

template <typename T>
cudaError_t pcg_t(bsc_ctx* c, const void* K, const void* b, void* x, double tol, int maxit, int sym,
                  const double* gate = nullptr, const double* gate_bb = nullptr, int dinv_ready = 0) {
  const int N = c->N;
  cudaError_t e;
  if ((e = cudaMemsetAsync(c->sync, 0, sizeof(unsigned int) * 2 * (size_t)c->P, c->stream)) != cudaSuccess) return e;
  if (!dinv_ready)
    k_block_jacobi<T><<<(N + 255) / 256, 256, 0, c->stream>>>(N, (const T*)K, (T*)c->Dinv, c->dstatus, sym ? 0 : 12);
  PcgArgs<T> A;
  A.N = N; A.maxit = maxit; A.tol = tol;
  A.pd = c->pd; A.blocks = c->pcg_blocks; A.nu = c->nu; A.nv = c->nv;
  A.K = (const T*)K; A.Dinv = (const T*)c->Dinv; A.b = (const T*)b; A.x = (T*)x;
  A.r = (T*)c->vec[1]; A.z = (T*)c->vec[2]; A.p = (T*)c->vec[3]; A.q = (T*)c->vec[4];
  A.partial = c->partials; A.sync = c->sync; A.status = c->dstatus; A.out = c->pcg_out;
  A.wait_limit = c->wait_limit; A.extra = c->barrier_extra;
  A.gate = gate; A.gate_bb = gate_bb;
  if (c->pcg_form == 1) {
    PipeVecs<T> V;
    V.u = (T*)c->pcg_pipe[0]; V.w = (T*)c->pcg_pipe[1]; V.m0 = (T*)c->pcg_pipe[2]; V.m1 = (T*)c->pcg_pipe[3];
    V.s = (T*)c->pcg_pipe[4]; V.z2 = (T*)c->pcg_pipe[5];
    return launch_coop_pipe<T>(c->pcg_grid, A, V, c->stream, sym);
  }
  return launch_coop<T>(c->pcg_grid, A, c->stream, c->pcg_form, sym);
}

}  // namespace

// Splits `total` co-resident blocks over `count` patches: each patch gets at
// least one block and at most ceil(n_cp / 256) (a block per 256 control
// points keeps every thread busy); the rest go one at a time to the patch
// with the largest work per block (ties to the lower index), which minimises
// the largest work / blocks.  Returns the number of blocks handed out
// (<= total), or -1 if total < count.
extern "C" int bsc_plan_blocks(int count, const int* n_cp, const double* work, int total, int* blocks) {
  if (count <= 0 || !n_cp || !work || !blocks || total < count) return -1;
  int used = 0;
  for (int p = 0; p < count; ++p) {
    blocks[p] = 1;
    ++used;
  }
  while (used < total) {
    int best = -1;
    double bw = -1.0;
    for (int p = 0; p < count; ++p) {
      const int cap = (n_cp[p] + PCG_BLOCK - 1) / PCG_BLOCK;
      if (blocks[p] >= cap) continue;
      const double w = work[p] / blocks[p];
      if (w > bw) {
        bw = w;
        best = p;
      }
    }
    if (best < 0) break;
    ++blocks[best];
    ++used;
  }
  return used;
}

// Grid of the persistent PCG: the co-resident capacity (at most four blocks
// of 256 threads per SM: the SpMV rows are latency-bound loads, and 1024
// threads per SM keep enough of them in flight), capped by what the patches
// can use; per-patch work estimates start at the control-point counts.
template <typename T>
cudaError_t pcg_occupancy(int* per_sm) {
  const void* fns[6] = {(const void*)k_pcg<T, PCG_BLOCK, 0, false>, (const void*)k_pcg<T, PCG_BLOCK, 2, false>,
                        (const void*)k_pcg<T, PCG_BLOCK, 0, true>,  (const void*)k_pcg<T, PCG_BLOCK, 2, true>,
                        (const void*)k_pcg_pipe<T, PCG_BLOCK, false>, (const void*)k_pcg_pipe<T, PCG_BLOCK, true>};
  cudaError_t e = cudaSuccess;
  *per_sm = 1 << 30;
  for (const void* f : fns) {
    int n = 0;
    if ((e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, f, PCG_BLOCK, 0)) != cudaSuccess) return e;
    *per_sm = std::min(*per_sm, n);
  }
  return e;
}

cudaError_t setup_pcg(bsc_ctx* c) {
  int per_sm = 0;
  // one grid serves every form: the co-resident capacity of the most demanding one
  cudaError_t e = c->precision == BSC_FP64 ? pcg_occupancy<double>(&per_sm) : pcg_occupancy<float>(&per_sm);
  if (e != cudaSuccess) return e;
  if (per_sm < 1) per_sm = 1;
  if (per_sm > 4) per_sm = 4;
  const int cap = c->num_sms * per_sm;
  if (c->P > cap) return cudaErrorInvalidConfiguration;
  long long need = 0;
  for (int p = 0; p < c->P; ++p) need += (c->hpd[p].N + PCG_BLOCK - 1) / PCG_BLOCK;
  c->pcg_cap = cap;
  c->pcg_need = (int)(need < cap ? need : cap);
  c->pcg_grid = c->pcg_need;
  c->pcg_weight = (double*)malloc(sizeof(double) * c->P);
  if (!c->pcg_weight) return cudaErrorMemoryAllocation;
  for (int p = 0; p < c->P; ++p) c->pcg_weight[p] = (double)c->hpd[p].N;
  if ((e = cudaMalloc(&c->pcg_blocks, sizeof(PcgBlock) * cap)) != cudaSuccess) return e;
  if ((e = cudaMalloc(&c->pcg_out, sizeof(double) * 3 * c->P)) != cudaSuccess) return e;
  for (int k = 0; k < 6; ++k)
    if ((e = cudaMalloc(&c->pcg_pipe[k], c->tsize * 3 * (size_t)c->N)) != cudaSuccess) return e;
  c->pcg_form = 0;
  return assign_pcg_blocks(c);
}

cudaError_t set_pcg_grid(bsc_ctx* c, int grid) {
  if (grid < c->P) grid = c->P;
  if (grid > c->pcg_need) grid = c->pcg_need;
  c->pcg_grid = grid;
  return assign_pcg_blocks(c);
}

// Block table of the persistent PCG from the current work estimates.
cudaError_t assign_pcg_blocks(bsc_ctx* c) {
  std::vector<int> ncp(c->P), nb(c->P);
  for (int p = 0; p < c->P; ++p) ncp[p] = c->hpd[p].N;
  const int used = bsc_plan_blocks(c->P, ncp.data(), c->pcg_weight, c->pcg_grid, nb.data());
  if (used != c->pcg_grid) return cudaErrorInvalidConfiguration;
  std::vector<PcgBlock> tab(c->pcg_grid);
  int k = 0;
  for (int p = 0; p < c->P; ++p) {
    for (int r = 0; r < nb[p]; ++r) tab[k + r] = PcgBlock{p, r, nb[p], k};
    k += nb[p];
  }
  cudaError_t e;
  if ((e = cudaStreamSynchronize(c->stream)) != cudaSuccess) return e;
  return cudaMemcpy(c->pcg_blocks, tab.data(), sizeof(PcgBlock) * c->pcg_grid, cudaMemcpyHostToDevice);
}

// 3x3 block-Jacobi inverses of K into Dinv (9 planes), for callers outside the PCG.
cudaError_t launch_block_jacobi(bsc_ctx* c, const void* K, void* Dinv) {
  BSC_COUNT(c, 1);
  const int G = (c->N + 255) / 256;
  if (c->precision == BSC_FP64)
    k_block_jacobi<double><<<G, 256, 0, c->stream>>>(c->N, (const double*)K, (double*)Dinv, c->dstatus, 12);
  else
    k_block_jacobi<float><<<G, 256, 0, c->stream>>>(c->N, (const float*)K, (float*)Dinv, c->dstatus, 12);
  return cudaGetLastError();
}

cudaError_t launch_spmv(bsc_ctx* c, const void* K, const void* x, void* y, int sym) {
  BSC_COUNT(c, 1);
  if (sym) {
    const int G = (c->N + 255) / 256;
    if (c->precision == BSC_FP64)
      k_spmv_sym<double><<<G, 256, 0, c->stream>>>(c->N, c->pd, c->cp_patch, (const double*)K, (const double*)x,
                                                   (double*)y);
    else
      k_spmv_sym<float><<<G, 256, 0, c->stream>>>(c->N, c->pd, c->cp_patch, (const float*)K, (const float*)x,
                                                  (float*)y);
    return cudaGetLastError();
  }
  const int B = 256, G = (3 * c->N + B - 1) / B;
  if (c->precision == BSC_FP64)
    k_spmv<double><<<G, B, 0, c->stream>>>(c->N, c->pd, c->cp_patch, (const double*)K, (const double*)x, (double*)y);
  else
    k_spmv<float><<<G, B, 0, c->stream>>>(c->N, c->pd, c->cp_patch, (const float*)K, (const float*)x, (float*)y);
  return cudaGetLastError();
}

cudaError_t launch_pcg(bsc_ctx* c, const void* K, const void* b, void* x, double tol, int maxit, int sym,
                       int dinv_ready) {
  BSC_COUNT(c, dinv_ready ? 1 : 2);
  if (c->precision == BSC_FP64) return pcg_t<double>(c, K, b, x, tol, maxit, sym, nullptr, nullptr, dinv_ready);
  return pcg_t<float>(c, K, b, x, tol, maxit, sym, nullptr, nullptr, dinv_ready);
}

cudaError_t launch_pcg_fallback(bsc_ctx* c, const void* K, const void* b, void* x, double tol, int maxit,
                                const double* fcg_out, const double* bb) {
  BSC_COUNT(c, 2);
  if (c->precision == BSC_FP64) return pcg_t<double>(c, K, b, x, tol, maxit, 0, fcg_out, bb);
  return pcg_t<float>(c, K, b, x, tol, maxit, 0, fcg_out, bb);
}

cudaError_t launch_axpy_trial(bsc_ctx* c, const void* C, const void* d, double alpha, void* out) {
  BSC_COUNT(c, 1);
  const int n = 3 * c->N, B = 256, G = (n + B - 1) / B;
  if (c->precision == BSC_FP64)
    k_axpy<double><<<G, B, 0, c->stream>>>(n, (const double*)C, (const double*)d, alpha, (double*)out);
  else
    k_axpy<float><<<G, B, 0, c->stream>>>(n, (const float*)C, (const float*)d, alpha, (float*)out);
  return cudaGetLastError();
}

cudaError_t launch_copy_vec(bsc_ctx* c, const void* src, void* dst) {
  return cudaMemcpyAsync(dst, src, c->tsize * 3 * (size_t)c->N, cudaMemcpyDeviceToDevice, c->stream);
}

// ---------------------------------------------------------------------------
// bsc_solve_static: the preconditioned CG of bsc_solve for callers that cannot
// allocate device memory, with its working set in a fixed device array.
// ---------------------------------------------------------------------------
#include <mutex>
#include <stdio.h>

void bsc_set_thread_error(const char* msg);

namespace {

// Working set of one solve of up to BSC_STATIC_SOLVE_MAX_CP control points in
// FP64: the 3x3 block-Jacobi inverses (9 N), the CG vectors r, z, p, q (4 x
// 3 N), cross-block partial sums, the grid-barrier words, a status word and
// the result scalars.  Every device that loads the library holds it until the
// process exits.
constexpr size_t kStaticCp = BSC_STATIC_SOLVE_MAX_CP;
constexpr size_t kStaticMaxGrid = 1024;
constexpr size_t kStaticDoubles = 21 * kStaticCp + 3 * kStaticMaxGrid + 16;
static __device__ __align__(256) double g_solve_scratch[kStaticDoubles];

std::mutex g_static_mu;
void* g_static_ptr[64];  // device address of g_solve_scratch, per device

template <typename T>
cudaError_t static_solve_t(int nu, int nv, double* scratch, const void* K, const void* b, void* x, double tol,
                           int maxit, cudaStream_t st, int num_sms, double* out_host) {
  constexpr int B = PCG_BLOCK;
  const int N = nu * nv;
  int per_sm = 0;
  cudaError_t e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_pcg<T, B, 0, false>, B, 0);
  if (e != cudaSuccess) return e;
  if (per_sm < 1) per_sm = 1;
  if (per_sm > 2) per_sm = 2;
  int grid = num_sms * per_sm;
  const int need = (N + B - 1) / B;
  if (grid > need) grid = need;
  if (grid > (int)kStaticMaxGrid) grid = (int)kStaticMaxGrid;
  // carve the array: T vectors first (FP64 slots hold FP32 vectors too)
  T* base = reinterpret_cast<T*>(scratch);
  T* Dinv = base;
  T* r = Dinv + 9 * (size_t)N;
  T* z = r + 3 * (size_t)N;
  T* p = z + 3 * (size_t)N;
  T* q = p + 3 * (size_t)N;
  double* partial = scratch + 21 * kStaticCp;
  double* tail = partial + 3 * kStaticMaxGrid;
  unsigned int* sync = reinterpret_cast<unsigned int*>(tail);  // 4 words
  int* status = reinterpret_cast<int*>(tail + 2);                // 1 word
  double* outd = tail + 4;                                        // 3 doubles
  // the barrier words, the status and the result scalars start at zero on
  // every call (a solve that stops early must not report the last call's results)
  if ((e = cudaMemsetAsync(tail, 0, 7 * sizeof(double), st)) != cudaSuccess) return e;
  k_block_jacobi<T><<<(N + 255) / 256, 256, 0, st>>>(N, (const T*)K, Dinv, status, 12);
  if ((e = cudaGetLastError()) != cudaSuccess) return e;
  PcgArgs<T> A;
  A.N = N; A.maxit = maxit; A.tol = tol;
  A.pd = nullptr; A.blocks = nullptr; A.nu = nu; A.nv = nv;
  A.K = (const T*)K; A.Dinv = Dinv; A.b = (const T*)b; A.x = (T*)x;
  A.r = r; A.z = z; A.p = p; A.q = q;
  A.partial = partial; A.sync = sync; A.status = status; A.out = outd;
  A.wait_limit = kWaitLimitDefault; A.extra = 0u; A.gate = nullptr; A.gate_bb = nullptr;
  e = launch_coop<T>(grid, A, st);
  if (e != cudaSuccess) return e;
  if ((e = cudaMemcpyAsync(out_host, outd, 3 * sizeof(double), cudaMemcpyDeviceToHost, st)) != cudaSuccess) return e;
  int flags = 0;
  if ((e = cudaMemcpyAsync(&flags, status, sizeof(int), cudaMemcpyDeviceToHost, st)) != cudaSuccess) return e;
  if ((e = cudaStreamSynchronize(st)) != cudaSuccess) return e;
  out_host[3] = (double)flags;
  return cudaSuccess;
}

bsc_status static_fail(bsc_status st, const char* msg) {
  bsc_set_thread_error(msg);
  return st;
}

}  // namespace

extern "C" bsc_status bsc_solve_static(int nu, int nv, int precision, const void* K_dev, const void* b_dev,
                                       void* x_dev, double rel_tol, int max_iter, void* cuda_stream, int* iters,
                                       double* rel_res) {
  char msg[256];
  if (nu < 5 || nv < 5) return static_fail(BSC_ERR_INVALID_ARG, "bsc_solve_static: nu, nv must be >= 5");
  if ((long long)nu * nv > (long long)BSC_STATIC_SOLVE_MAX_CP) {
    snprintf(msg, sizeof(msg), "bsc_solve_static: %d x %d = %lld control points exceed the fixed working set "
             "of %d control points; use bsc_solve", nu, nv, (long long)nu * nv, BSC_STATIC_SOLVE_MAX_CP);
    return static_fail(BSC_ERR_INVALID_ARG, msg);
  }
  if (precision != BSC_FP64 && precision != BSC_FP32)
    return static_fail(BSC_ERR_INVALID_ARG, "bsc_solve_static: unknown precision");
  if (!K_dev || !b_dev || !x_dev) return static_fail(BSC_ERR_INVALID_ARG, "bsc_solve_static: NULL pointer");
  if ((((uintptr_t)K_dev) | ((uintptr_t)b_dev) | ((uintptr_t)x_dev)) & 15u)
    return static_fail(BSC_ERR_INVALID_ARG, "bsc_solve_static: pointers must be 16-byte aligned");
  if (b_dev == x_dev) return static_fail(BSC_ERR_INVALID_ARG, "bsc_solve_static: b and x must not alias");
  if (!(rel_tol > 0.0)) rel_tol = 1e-8;
  if (max_iter <= 0) max_iter = 10000;
  int dev = 0, sms = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  if (e != cudaSuccess || dev < 0 || dev >= 64) {
    snprintf(msg, sizeof(msg), "bsc_solve_static: device query failed: %s", cudaGetErrorString(e));
    return static_fail(BSC_ERR_CUDA, msg);
  }
  void* ptr = nullptr;
  {
    // first call on this device: look up the array's device address (with
    // the device current); later calls reuse it
    std::lock_guard<std::mutex> lock(g_static_mu);
    if (!g_static_ptr[dev]) {
      e = cudaGetSymbolAddress(&g_static_ptr[dev], g_solve_scratch);
      if (e != cudaSuccess) {
        g_static_ptr[dev] = nullptr;
        snprintf(msg, sizeof(msg), "bsc_solve_static: cudaGetSymbolAddress failed: %s", cudaGetErrorString(e));
        return static_fail(BSC_ERR_CUDA, msg);
      }
    }
    ptr = g_static_ptr[dev];
  }
  double out[4] = {0, 0, 0, 0};
  cudaStream_t st = (cudaStream_t)cuda_stream;
  e = precision == BSC_FP64
          ? static_solve_t<double>(nu, nv, (double*)ptr, K_dev, b_dev, x_dev, rel_tol, max_iter, st, sms, out)
          : static_solve_t<float>(nu, nv, (double*)ptr, K_dev, b_dev, x_dev, rel_tol, max_iter, st, sms, out);
  if (e != cudaSuccess) {
    snprintf(msg, sizeof(msg), "bsc_solve_static: %s", cudaGetErrorString(e));
    return static_fail(BSC_ERR_CUDA, msg);
  }
  if (iters) *iters = (int)out[0];
  if (rel_res) *rel_res = out[1];
  const int flags = (int)out[3];
  if (flags & BSC_STATUS_TIMEOUT_FLAG) return static_fail(BSC_ERR_TIMEOUT, "bsc_solve_static: device wait timed out");
  if (flags) return static_fail(BSC_ERR_NUMERIC, "bsc_solve_static: non-finite or singular value on the device");
  if (!(out[1] <= rel_tol)) {
    snprintf(msg, sizeof(msg), "bsc_solve_static: %d iterations, rel. residual %g", (int)out[0], out[1]);
    return static_fail(BSC_ERR_NOT_CONVERGED, msg);
  }
  return BSC_OK;
}

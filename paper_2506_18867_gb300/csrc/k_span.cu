// K2: per-span membrane + bending energy, gradient and 27x27 Hessian.
//
// One thread per knot span.  Per membrane point (FBW, Eqs. anisotropic
// invariants and FBW stretching and shearing energy):
//   f_beta = F e_beta = sum_l C_l g_l,beta,   I5(e_b) = |f_b|^2,  I6 = f_1 . f_2
//   Psi = mu_st1 (|f_1| - 1)^2 + mu_st2 (|f_2| - 1)^2 + mu_sh I6^2
// with the analytic derivatives w.r.t. (f_1, f_2) chained to the 27 span DOFs
// through g.  Per bending point (Eq. general bending energy with the
// Laplacian of Eq. (Laplacian in parametric space)):
//   Psi = mu_bd/2 |sum_l L_l C_l|^2   (quadratic, constant Hessian).
// The control points of the span are shifted by the span's centre control
// point before forming f (sum_l g_l = 0), which keeps FP32 strains accurate
// far from the origin.  Energies accumulate in FP64.  The Hessian is summed
// in shared memory (interleaved by thread, packed upper triangle) and
// written as planes; the weighted 6x6 d^2 Psi/df^2 of every membrane point
// is kept for the FP64 projection.
//
// Blocks take work items: a patch and either a run of BLOCK consecutive
// spans of it or a tu x (BLOCK / tu) tile of spans, the tile shape chosen per
// patch-size class by the autotuner (bsc_autotune).  All patches of a
// context are evaluated by one launch.
#include <vector>

#include "bsc_internal.cuh"

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
};

template <typename T> __device__ __forceinline__ T rsqrt_(T x);
template <> __device__ __forceinline__ float rsqrt_<float>(float x) { return rsqrtf(x); }
template <> __device__ __forceinline__ double rsqrt_<double>(double x) { return rsqrt(x); }

template <typename T, bool GRAD, bool HESS, int BLOCK>
__global__ void __launch_bounds__(BLOCK) k_span_eval(SpanArgs<T> P) {
  extern __shared__ __align__(16) unsigned char smraw[];
  T* Hs = reinterpret_cast<T*>(smraw);
  const SpanItem it = P.items[blockIdx.x];
  if (P.gate && P.gate[it.p].state != 1) return;
  const PatchDev* pt = P.pd + it.p;
  const int Su = __ldg(&pt->Su), nu = __ldg(&pt->nu);
  int a, b;
  if (it.tu == 0) {
    const int sl = it.first_or_a0 + threadIdx.x;
    if (sl >= __ldg(&pt->Nsp)) return;
    a = sl % Su;
    b = sl / Su;
  } else {
    a = it.first_or_a0 + threadIdx.x % it.tu;
    b = it.b0 + threadIdx.x / it.tu;
    if (a >= Su || b >= __ldg(&pt->Sv)) return;
  }
  const int s = __ldg(&pt->sp0) + b * Su + a;
  const T* __restrict__ Cp = P.C + __ldg(&pt->cp0);
  const T mu1 = (T)__ldg(&pt->mu1), mu2 = (T)__ldg(&pt->mu2), mush = (T)__ldg(&pt->mush),
          mubd = (T)__ldg(&pt->mubd);
  auto HS = [&](int r, int c) -> T& { return Hs[upk(r, c, 27) * BLOCK + threadIdx.x]; };

  // control points relative to the span's centre control point
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
  double E = 0.0;
  T g[27];
#pragma unroll
  for (int k = 0; k < 27; ++k) g[k] = T(0);
  if (HESS) {
#pragma unroll 1
    for (int k = 0; k < H27; ++k) Hs[k * BLOCK + threadIdx.x] = T(0);
  }

  const int q0 = P.moff[s], q1 = P.moff[s + 1];
  for (int q = q0; q < q1; ++q) {
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
        T acc = T(0);
#pragma unroll
        for (int l = 0; l < 9; ++l) acc += Cl[l][c] * gq[l][be];
        f[be][c] = acc;
      }
    const T I5a = f[0][0] * f[0][0] + f[0][1] * f[0][1] + f[0][2] * f[0][2];
    const T I5b = f[1][0] * f[1][0] + f[1][1] * f[1][1] + f[1][2] * f[1][2];
    const T I6 = f[0][0] * f[1][0] + f[0][1] * f[1][1] + f[0][2] * f[1][2];
    const T r1 = rsqrt_(I5a), r2 = rsqrt_(I5b);  // 1 / |f_b|
    const T s1 = I5a * r1, s2 = I5b * r2;
    const T e1 = s1 - T(1), e2 = s2 - T(1);
    E += (double)W * (double)(mu1 * e1 * e1 + mu2 * e2 * e2 + mush * I6 * I6);
    // dPsi/df_b = 2 mu_b (1 - 1/|f_b|) f_b + 2 mu_sh I6 f_other
    const T k1 = T(2) * mu1 * (T(1) - r1), k2 = T(2) * mu2 * (T(1) - r2), ks = T(2) * mush * I6;
    if (GRAD) {
      T dP[2][3];
#pragma unroll
      for (int c = 0; c < 3; ++c) {
        dP[0][c] = W * (k1 * f[0][c] + ks * f[1][c]);
        dP[1][c] = W * (k2 * f[1][c] + ks * f[0][c]);
      }
#pragma unroll
      for (int l = 0; l < 9; ++l)
#pragma unroll
        for (int c = 0; c < 3; ++c) g[3 * l + c] += gq[l][0] * dP[0][c] + gq[l][1] * dP[1][c];
    }
    if (HESS) {
      // weighted d^2 Psi / d f_(b c) d f_(d e), 6x6 with index 3 b + c
      T A6[6][6];
      const T c1 = T(2) * mu1 * r1 * r1 * r1, c2 = T(2) * mu2 * r2 * r2 * r2, cs = T(2) * mush;
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
      {
        int e = 0;
#pragma unroll
        for (int r = 0; r < 6; ++r)
#pragma unroll
          for (int c = r; c < 6; ++c) P.A[(size_t)(e++) * P.Nm + q] = A6[r][c];
      }
      // H_(l c)(m d) += sum_{b,d'} g_l,b g_m,d' A6[3b+c][3d'+d]
#pragma unroll
      for (int l = 0; l < 9; ++l) {
        T Tl[3][6];  // Tl[c][k] = sum_b g_l,b A6[3b+c][k]
#pragma unroll
        for (int c = 0; c < 3; ++c)
#pragma unroll
          for (int k = 0; k < 6; ++k) Tl[c][k] = gq[l][0] * A6[c][k] + gq[l][1] * A6[3 + c][k];
#pragma unroll
        for (int m = l; m < 9; ++m)
#pragma unroll
          for (int c = 0; c < 3; ++c)
#pragma unroll
            for (int d = 0; d < 3; ++d) {
              if (m == l && d < c) continue;
              HS(3 * l + c, 3 * m + d) += Tl[c][d] * gq[m][0] + Tl[c][3 + d] * gq[m][1];
            }
      }
    }
  }

  const int p0 = P.boff[s], p1 = P.boff[s + 1];
  for (int q = p0; q < p1; ++q) {
    const T WB = P.tabb[q] * mubd;  // W mu_bd
    T L[9];
#pragma unroll
    for (int l = 0; l < 9; ++l) L[l] = P.tabb[(1 + l) * P.Nb + q];
    T lap[3];
#pragma unroll
    for (int c = 0; c < 3; ++c) {
      T acc = T(0);
#pragma unroll
      for (int l = 0; l < 9; ++l) acc += L[l] * Cl[l][c];
      lap[c] = acc;
    }
    E += 0.5 * (double)WB * (double)(lap[0] * lap[0] + lap[1] * lap[1] + lap[2] * lap[2]);
    if (GRAD) {
#pragma unroll
      for (int l = 0; l < 9; ++l)
#pragma unroll
        for (int c = 0; c < 3; ++c) g[3 * l + c] += WB * L[l] * lap[c];
    }
    if (HESS) {
#pragma unroll
      for (int l = 0; l < 9; ++l)
#pragma unroll
        for (int m = l; m < 9; ++m) {
          const T h = WB * L[l] * L[m];
#pragma unroll
          for (int c = 0; c < 3; ++c) HS(3 * l + c, 3 * m + c) += h;
        }
    }
  }

  P.E[s] = E;
  if (GRAD) {
#pragma unroll
    for (int k = 0; k < 27; ++k) P.g[(size_t)k * P.Nsp + s] = g[k];
  }
  if (HESS) {
#pragma unroll 1
    for (int k = 0; k < H27; ++k) P.H[(size_t)k * P.Nsp + s] = Hs[k * BLOCK + threadIdx.x];
  }
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
  return P;
}

template <typename T, int BLOCK>
cudaError_t run(bsc_ctx* c, const void* C, int want_grad, int want_hess, const SpanItem* items, int n_items,
                const PatchStep* gate) {
  if (n_items <= 0) return cudaSuccess;
  SpanArgs<T> P = make_args<T>(c, C, items, gate);
  if (want_hess)
    k_span_eval<T, true, true, BLOCK><<<n_items, BLOCK, sizeof(T) * H27 * BLOCK, c->stream>>>(P);
  else if (want_grad)
    k_span_eval<T, true, false, BLOCK><<<n_items, BLOCK, 0, c->stream>>>(P);
  else
    k_span_eval<T, false, false, BLOCK><<<n_items, BLOCK, 0, c->stream>>>(P);
  return cudaGetLastError();
}

constexpr int BLOCK64 = 64, BLOCK32 = 128;

}  // namespace

int span_block(int precision) { return precision == BSC_FP64 ? BLOCK64 : BLOCK32; }

// The Hessian variant keeps its 27x27 accumulator in shared memory (378
// entries per thread): opt in to more than 48 KB once per context.
cudaError_t setup_span_eval(bsc_ctx* c) {
  if (c->precision == BSC_FP64)
    return cudaFuncSetAttribute(k_span_eval<double, true, true, BLOCK64>,
                                cudaFuncAttributeMaxDynamicSharedMemorySize, (int)(sizeof(double) * H27 * BLOCK64));
  return cudaFuncSetAttribute(k_span_eval<float, true, true, BLOCK32>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                              (int)(sizeof(float) * H27 * BLOCK32));
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
  if (c->precision == BSC_FP64) return run<double, BLOCK64>(c, C, want_grad, want_hess, items, n_items, nullptr);
  return run<float, BLOCK32>(c, C, want_grad, want_hess, items, n_items, nullptr);
}

cudaError_t launch_span_eval(bsc_ctx* c, const void* C, int want_grad, int want_hess, const PatchStep* gate) {
  BSC_COUNT(c, 1);
  if (c->precision == BSC_FP64)
    return run<double, BLOCK64>(c, C, want_grad, want_hess, c->span_items, c->n_span_items, gate);
  return run<float, BLOCK32>(c, C, want_grad, want_hess, c->span_items, c->n_span_items, gate);
}

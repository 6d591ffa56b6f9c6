// K4: gather assembly of the global Hessian and gradient, and the energy sum.
//
// The sparsity of the elasticity Hessian follows from the tensor-product
// stencil alone (Sec. 5.2): control point alpha = (i, j) couples to
// beta = (i+du, j+dv), |du|, |dv| <= 2, through the spans that contain both,
// a in [max(i, i+du) - 2, min(i, i+du)] (likewise b).  Each output 3x3 block
// is produced by one thread that gathers those span blocks in a fixed order
// (b, then a ascending) - no atomics, bitwise reproducible - and adds the
// lumped inertia m/dt^2 on the diagonal (Eq. incremental_potential).  Rows and
// columns of pinned control points become identity / zero (Dirichlet
// elimination, Sec. 5.1).
//
// A context holds one or more patches with concatenated planes; a thread
// finds its patch from the control point's patch map and works in the
// patch's local (i, j) numbering.  The per-patch sums (energy, |d|_inf,
// projected-span counts) run over reduction items - fixed chunks of a
// patch's spans or control points - and then over each patch's items in
// order, so every sum is bitwise reproducible.
#include <vector>

#include "bsc_internal.cuh"

namespace {

// SYM: only the diagonal block and the 12 blocks after it (stencil slots
// 12..24), written as slots 0..12 of the symmetric layout; the blocks before
// a row are the transposes of its neighbours' (the gathers of (alpha, beta)
// and (beta, alpha) add the same span entries in the same order).
// Dinv (optional): the thread of a diagonal block also writes its inverse,
// the block-Jacobi preconditioner of the solve that follows (the same FP64
// adjugate of the same entries as k_block_jacobi, so the same values).
template <typename T, bool SYM>
__global__ void k_assemble(int N, int Nsp, const PatchDev* __restrict__ pd, const int* __restrict__ cp_patch,
                           const T* __restrict__ H, const double* __restrict__ mass,
                           const uint8_t* __restrict__ pinned, T* __restrict__ K, T* __restrict__ Dinv,
                           int* __restrict__ status) {
  const long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= (SYM ? 13ll : 25ll) * N) return;
  const int s_out = (int)(t / N), al = (int)(t - (long long)s_out * N);
  const int slot = SYM ? s_out + 12 : s_out;
  const PatchDev* pt = pd + cp_patch[al];
  const int nu = __ldg(&pt->nu), nv = __ldg(&pt->nv), Su = nu - 2, Sv = nv - 2;
  const int cp0 = __ldg(&pt->cp0), sp0 = __ldg(&pt->sp0);
  const int du = slot % 5 - 2, dv = slot / 5 - 2;
  const int l = al - cp0, i = l % nu, j = l / nu, ib = i + du, jb = j + dv;
  T blk[9];
#pragma unroll
  for (int k = 0; k < 9; ++k) blk[k] = T(0);
  const bool inside = ib >= 0 && ib < nu && jb >= 0 && jb < nv;
  if (inside) {
    const int be = cp0 + jb * nu + ib;
    if (pinned[al] || pinned[be]) {
      if (du == 0 && dv == 0) blk[0] = blk[4] = blk[8] = T(1);
    } else {
      const int a_lo = max(max(i, ib) - 2, 0), a_hi = min(min(i, ib), Su - 1);
      const int b_lo = max(max(j, jb) - 2, 0), b_hi = min(min(j, jb), Sv - 1);
      for (int b = b_lo; b <= b_hi; ++b)
        for (int a = a_lo; a <= a_hi; ++a) {
          const int s = sp0 + b * Su + a;
          const int la = (i - a) + 3 * (j - b), lb = (ib - a) + 3 * (jb - b);
#pragma unroll
          for (int r = 0; r < 3; ++r)
#pragma unroll
            for (int c = 0; c < 3; ++c) {
              const int R = 3 * la + r, Cc = 3 * lb + c;
              blk[3 * r + c] += H[(size_t)sym_upk(R, Cc, 27) * Nsp + s];
            }
        }
      if (du == 0 && dv == 0) {
        const T k = (T)(mass[al] * __ldg(&pt->inv_dt2));
        blk[0] += k; blk[4] += k; blk[8] += k;
      }
    }
  }
#pragma unroll
  for (int k = 0; k < 9; ++k) K[(size_t)(s_out * 9 + k) * N + al] = blk[k];
  if (Dinv && slot == 12) block_jacobi_at<T>(N, al, K, Dinv, status, s_out);
}

template <typename T>
__global__ void k_gradient(int N, int Nsp, const PatchDev* __restrict__ pd, const int* __restrict__ cp_patch,
                           const T* __restrict__ gs, const double* __restrict__ mass, const T* __restrict__ C,
                           const T* __restrict__ Chat, const uint8_t* __restrict__ pinned, T* __restrict__ g) {
  const int al = blockIdx.x * blockDim.x + threadIdx.x;
  if (al >= N) return;
  if (pinned[al]) {
    g[al] = g[N + al] = g[2 * N + al] = T(0);
    return;
  }
  const PatchDev* pt = pd + cp_patch[al];
  const int nu = __ldg(&pt->nu), Su = nu - 2, Sv = __ldg(&pt->nv) - 2;
  const int l0 = al - __ldg(&pt->cp0), sp0 = __ldg(&pt->sp0);
  const int i = l0 % nu, j = l0 / nu;
  T acc[3] = {T(0), T(0), T(0)};
  for (int b = max(j - 2, 0); b <= min(j, Sv - 1); ++b)
    for (int a = max(i - 2, 0); a <= min(i, Su - 1); ++a) {
      const int s = sp0 + b * Su + a, l = (i - a) + 3 * (j - b);
#pragma unroll
      for (int c = 0; c < 3; ++c) acc[c] += gs[(size_t)(3 * l + c) * Nsp + s];
    }
  const double inv_dt2 = __ldg(&pt->inv_dt2);
  const T m = (T)mass[al], mk = (T)(mass[al] * inv_dt2);
  const T grav[3] = {(T)__ldg(&pt->grav[0]), (T)__ldg(&pt->grav[1]), (T)__ldg(&pt->grav[2])};
#pragma unroll
  for (int c = 0; c < 3; ++c) {
    T v = acc[c] - m * grav[c];
    if (inv_dt2 > 0.0) v += mk * (C[c * N + al] - Chat[c * N + al]);
    g[c * N + al] = v;
  }
}

constexpr int RED_BLOCK = 256;

// Per reduction item: the item's share of the incremental potential - span
// energies (kind 0) or the inertia and gravity terms of its control points
// (kind 1).  Items of patches outside the gate are skipped.
template <typename T>
__global__ void __launch_bounds__(RED_BLOCK) k_energy_items(int N, const RedItem* __restrict__ items,
                                                            const PatchDev* __restrict__ pd,
                                                            const PatchStep* __restrict__ gate,
                                                            const double* __restrict__ Es,
                                                            const double* __restrict__ mass, const T* __restrict__ C,
                                                            const T* __restrict__ Chat, double* __restrict__ partial) {
  __shared__ double sm[RED_BLOCK / 32];
  const RedItem it = items[blockIdx.x];
  if (gate && gate[it.p].state != 1) return;
  const PatchDev* pt = pd + it.p;
  double acc = 0.0;
  if (it.kind == 0) {
    const int sp0 = __ldg(&pt->sp0);
    for (int k = it.lo + threadIdx.x; k < it.hi; k += RED_BLOCK) acc += Es[sp0 + k];
  } else {
    const int cp0 = __ldg(&pt->cp0);
    const double inv_dt2 = __ldg(&pt->inv_dt2);
    const double gx = __ldg(&pt->grav[0]), gy = __ldg(&pt->grav[1]), gz = __ldg(&pt->grav[2]);
    for (int k = it.lo + threadIdx.x; k < it.hi; k += RED_BLOCK) {
      const int al = cp0 + k;
      const double m = mass[al];
      const double x = C[al], y = C[N + al], z = C[2 * N + al];
      acc -= m * (gx * x + gy * y + gz * z);
      if (inv_dt2 > 0.0) {
        const double dx = x - (double)Chat[al], dy = y - (double)Chat[N + al], dz = z - (double)Chat[2 * N + al];
        acc += 0.5 * m * inv_dt2 * (dx * dx + dy * dy + dz * dz);
      }
    }
  }
  const double tot = block_sum<RED_BLOCK>(acc, sm);
  if (threadIdx.x == 0) partial[blockIdx.x] = tot;
}

// out[p] = sum of patch p's item partials in item order (one block per
// patch); a non-finite energy raises the NUMERIC flag.
__global__ void __launch_bounds__(RED_BLOCK) k_patch_sums(const int* __restrict__ red_off,
                                                          const PatchStep* __restrict__ gate,
                                                          const double* __restrict__ partial, double* __restrict__ out,
                                                          int* __restrict__ status) {
  __shared__ double sm[RED_BLOCK / 32];
  const int p = blockIdx.x;
  if (gate && gate[p].state != 1) return;
  double acc = 0.0;
  for (int k = red_off[p] + threadIdx.x; k < red_off[p + 1]; k += RED_BLOCK) acc += partial[k];
  const double tot = block_sum<RED_BLOCK>(acc, sm);
  if (threadIdx.x == 0) {
    out[p] = tot;
    if (!isfinite(tot)) atomicOr(status, BSC_STATUS_NUMERIC_FLAG);
  }
}

// Copies the packed per-span results into the row-major inspection layout.
template <typename T>
__global__ void k_export_span(int Nsp, const T* __restrict__ gs, const T* __restrict__ Hs,
                              T* __restrict__ g_out, T* __restrict__ H_out) {
  const int s = blockIdx.x * blockDim.x + threadIdx.x;
  if (s >= Nsp) return;
  if (g_out)
#pragma unroll 1
    for (int k = 0; k < 27; ++k) g_out[(size_t)s * 27 + k] = gs[(size_t)k * Nsp + s];
  if (H_out)
#pragma unroll 1
    for (int r = 0; r < 27; ++r)
#pragma unroll 1
      for (int c = 0; c < 27; ++c)
        H_out[(size_t)s * 729 + r * 27 + c] = Hs[(size_t)sym_upk(r, c, 27) * Nsp + s];
}

}  // namespace

// Reduction items: every patch's spans, then its control points, in chunks
// of RED_CHUNK, grouped by patch.
constexpr int RED_CHUNK = 2048;

// A strip window (one patch) instead has one item per owned row: the span
// rows whose middle control-point row it owns, then its owned control-point
// rows.  A row's partial sum then depends on the row alone, not on the
// window, so the ranks of a decomposition can add them up in the global row
// order and all decompositions of a patch agree bit for bit.
cudaError_t build_red_items(bsc_ctx* c) {
  std::vector<RedItem> items;
  std::vector<int> off(c->P + 1);
  for (int p = 0; p < c->P; ++p) {
    off[p] = (int)items.size();
    const PatchDev& q = c->hpd[p];
    if (c->is_window) {
      const int r0 = c->win_row0;
      const int b0 = std::max(c->win_own0 - 1, 0), b1 = std::min(c->win_own1 - 1, q.SvG);
      for (int b = b0; b < b1; ++b) items.push_back(RedItem{p, 0, (b - r0) * q.Su, (b - r0 + 1) * q.Su});
      for (int j = c->win_own0; j < c->win_own1; ++j) items.push_back(RedItem{p, 1, (j - r0) * q.nu, (j - r0 + 1) * q.nu});
      continue;
    }
    for (int lo = 0; lo < q.Nsp; lo += RED_CHUNK) items.push_back(RedItem{p, 0, lo, std::min(lo + RED_CHUNK, q.Nsp)});
    for (int lo = 0; lo < q.N; lo += RED_CHUNK) items.push_back(RedItem{p, 1, lo, std::min(lo + RED_CHUNK, q.N)});
  }
  off[c->P] = (int)items.size();
  c->n_red_items = (int)items.size();
  cudaError_t e;
  if ((e = cudaMalloc(&c->red_items, sizeof(RedItem) * items.size())) != cudaSuccess) return e;
  if ((e = cudaMalloc(&c->red_off, sizeof(int) * (c->P + 1))) != cudaSuccess) return e;
  if ((e = cudaMemcpy(c->red_items, items.data(), sizeof(RedItem) * items.size(), cudaMemcpyHostToDevice)) !=
      cudaSuccess)
    return e;
  return cudaMemcpy(c->red_off, off.data(), sizeof(int) * (c->P + 1), cudaMemcpyHostToDevice);
}

cudaError_t launch_assemble(bsc_ctx* c, void* K, int sym, void* Dinv) {
  BSC_COUNT(c, 1);
  const int B = 256;
  const long long G = ((sym ? 13ll : 25ll) * c->N + B - 1) / B;
  if (c->precision == BSC_FP64) {
    if (sym)
      k_assemble<double, true><<<(unsigned)G, B, 0, c->stream>>>(c->N, c->Nsp, c->pd, c->cp_patch,
                                                                 (const double*)c->H_span, c->mass, c->pinned,
                                                                 (double*)K, (double*)Dinv, c->dstatus);
    else
      k_assemble<double, false><<<(unsigned)G, B, 0, c->stream>>>(c->N, c->Nsp, c->pd, c->cp_patch,
                                                                  (const double*)c->H_span, c->mass, c->pinned,
                                                                  (double*)K, (double*)Dinv, c->dstatus);
  } else {
    if (sym)
      k_assemble<float, true><<<(unsigned)G, B, 0, c->stream>>>(c->N, c->Nsp, c->pd, c->cp_patch,
                                                                (const float*)c->H_span, c->mass, c->pinned,
                                                                (float*)K, (float*)Dinv, c->dstatus);
    else
      k_assemble<float, false><<<(unsigned)G, B, 0, c->stream>>>(c->N, c->Nsp, c->pd, c->cp_patch,
                                                                 (const float*)c->H_span, c->mass, c->pinned,
                                                                 (float*)K, (float*)Dinv, c->dstatus);
  }
  return cudaGetLastError();
}

cudaError_t launch_gradient(bsc_ctx* c, const void* C, const void* Chat, void* g) {
  BSC_COUNT(c, 1);
  const int B = 256, G = (c->N + B - 1) / B;
  // a static problem (no inertia) may pass no Chat: it is not read then
  const void* Ch = Chat ? Chat : C;
  if (c->precision == BSC_FP64)
    k_gradient<double><<<G, B, 0, c->stream>>>(c->N, c->Nsp, c->pd, c->cp_patch, (const double*)c->g_span, c->mass,
                                               (const double*)C, (const double*)Ch, c->pinned, (double*)g);
  else
    k_gradient<float><<<G, B, 0, c->stream>>>(c->N, c->Nsp, c->pd, c->cp_patch, (const float*)c->g_span, c->mass,
                                              (const float*)C, (const float*)Ch, c->pinned, (float*)g);
  return cudaGetLastError();
}

cudaError_t launch_patch_energy(bsc_ctx* c, const void* C, const void* Chat, double* dE, const PatchStep* gate) {
  BSC_COUNT(c, 2);
  const void* Ch = Chat ? Chat : C;
  if (c->precision == BSC_FP64)
    k_energy_items<double><<<c->n_red_items, RED_BLOCK, 0, c->stream>>>(
        c->N, c->red_items, c->pd, gate, c->E_span, c->mass, (const double*)C, (const double*)Ch, c->partials);
  else
    k_energy_items<float><<<c->n_red_items, RED_BLOCK, 0, c->stream>>>(
        c->N, c->red_items, c->pd, gate, c->E_span, c->mass, (const float*)C, (const float*)Ch, c->partials);
  k_patch_sums<<<c->P, RED_BLOCK, 0, c->stream>>>(c->red_off, gate, c->partials, dE, c->dstatus);
  return cudaGetLastError();
}

cudaError_t launch_export_span_terms(bsc_ctx* c, void* g_out, void* H_out) {
  BSC_COUNT(c, 1);
  const int B = 128, G = (c->Nsp + B - 1) / B;
  if (c->precision == BSC_FP64)
    k_export_span<double><<<G, B, 0, c->stream>>>(c->Nsp, (const double*)c->g_span, (const double*)c->H_span,
                                                   (double*)g_out, (double*)H_out);
  else
    k_export_span<float><<<G, B, 0, c->stream>>>(c->Nsp, (const float*)c->g_span, (const float*)c->H_span,
                                                  (float*)g_out, (float*)H_out);
  return cudaGetLastError();
}

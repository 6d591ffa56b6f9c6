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
#include "bsc_internal.cuh"

namespace {

template <typename T>
__global__ void k_assemble(int nu, int nv, int Nsp, const T* __restrict__ H,
                           const double* __restrict__ mass, double inv_dt2,
                           const uint8_t* __restrict__ pinned, T* __restrict__ K) {
  const int N = nu * nv, Su = nu - 2, Sv = nv - 2;
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= 25 * N) return;
  const int slot = t / N, al = t - slot * N;
  const int du = slot % 5 - 2, dv = slot / 5 - 2;
  const int i = al % nu, j = al / nu, ib = i + du, jb = j + dv;
  T blk[9];
#pragma unroll
  for (int k = 0; k < 9; ++k) blk[k] = T(0);
  const bool inside = ib >= 0 && ib < nu && jb >= 0 && jb < nv;
  if (inside) {
    const int be = jb * nu + ib;
    if (pinned[al] || pinned[be]) {
      if (du == 0 && dv == 0) blk[0] = blk[4] = blk[8] = T(1);
    } else {
      const int a_lo = max(max(i, ib) - 2, 0), a_hi = min(min(i, ib), Su - 1);
      const int b_lo = max(max(j, jb) - 2, 0), b_hi = min(min(j, jb), Sv - 1);
      for (int b = b_lo; b <= b_hi; ++b)
        for (int a = a_lo; a <= a_hi; ++a) {
          const int s = b * Su + a;
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
        const T k = (T)(mass[al] * inv_dt2);
        blk[0] += k; blk[4] += k; blk[8] += k;
      }
    }
  }
#pragma unroll
  for (int k = 0; k < 9; ++k) K[(size_t)(slot * 9 + k) * N + al] = blk[k];
}

template <typename T>
__global__ void k_gradient(int nu, int nv, int Nsp, const T* __restrict__ gs,
                           const double* __restrict__ mass, double inv_dt2, double gx, double gy,
                           double gz, const T* __restrict__ C, const T* __restrict__ Chat,
                           const uint8_t* __restrict__ pinned, T* __restrict__ g) {
  const int N = nu * nv, Su = nu - 2, Sv = nv - 2;
  const int al = blockIdx.x * blockDim.x + threadIdx.x;
  if (al >= N) return;
  if (pinned[al]) {
    g[al] = g[N + al] = g[2 * N + al] = T(0);
    return;
  }
  const int i = al % nu, j = al / nu;
  T acc[3] = {T(0), T(0), T(0)};
  for (int b = max(j - 2, 0); b <= min(j, Sv - 1); ++b)
    for (int a = max(i - 2, 0); a <= min(i, Su - 1); ++a) {
      const int s = b * Su + a, l = (i - a) + 3 * (j - b);
#pragma unroll
      for (int c = 0; c < 3; ++c) acc[c] += gs[(size_t)(3 * l + c) * Nsp + s];
    }
  const T m = (T)mass[al], mk = (T)(mass[al] * inv_dt2), grav[3] = {(T)gx, (T)gy, (T)gz};
#pragma unroll
  for (int c = 0; c < 3; ++c) {
    T v = acc[c] - m * grav[c];
    if (inv_dt2 > 0.0) v += mk * (C[c * N + al] - Chat[c * N + al]);
    g[c * N + al] = v;
  }
}

// Partial sums of the incremental potential: span energies plus per-control-
// point inertia and gravity terms, grid-stride with a fixed assignment.
template <typename T, int BLOCK>
__global__ void k_energy_partials(int N, int Nsp, const double* __restrict__ Es,
                                  const double* __restrict__ mass, double inv_dt2, double gx,
                                  double gy, double gz, const T* __restrict__ C,
                                  const T* __restrict__ Chat, double* __restrict__ partial) {
  __shared__ double sm[BLOCK / 32];
  const int stride = gridDim.x * BLOCK;
  double acc = 0.0;
  for (int s = blockIdx.x * BLOCK + threadIdx.x; s < Nsp; s += stride) acc += Es[s];
  for (int al = blockIdx.x * BLOCK + threadIdx.x; al < N; al += stride) {
    const double m = mass[al];
    const double x = C[al], y = C[N + al], z = C[2 * N + al];
    acc -= m * (gx * x + gy * y + gz * z);
    if (inv_dt2 > 0.0) {
      const double dx = x - (double)Chat[al], dy = y - (double)Chat[N + al], dz = z - (double)Chat[2 * N + al];
      acc += 0.5 * m * inv_dt2 * (dx * dx + dy * dy + dz * dz);
    }
  }
  const double tot = block_sum<BLOCK>(acc, sm);
  if (threadIdx.x == 0) partial[blockIdx.x] = tot;
}

template <int BLOCK>
__global__ void k_sum_partials(int n, const double* __restrict__ partial, double* __restrict__ out,
                               int* __restrict__ status) {
  __shared__ double sm[BLOCK / 32];
  double acc = 0.0;
  for (int k = threadIdx.x; k < n; k += BLOCK) acc += partial[k];
  const double tot = block_sum<BLOCK>(acc, sm);
  if (threadIdx.x == 0) {
    *out = tot;
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

cudaError_t launch_assemble(bsc_ctx* c, void* K) {
  BSC_COUNT(c, 1);
  const int B = 256, G = (25 * c->N + B - 1) / B;
  const double idt2 = c->dt > 0.0 ? 1.0 / (c->dt * c->dt) : 0.0;
  if (c->precision == BSC_FP64)
    k_assemble<double><<<G, B, 0, c->stream>>>(c->nu, c->nv, c->Nsp, (const double*)c->H_span, c->mass,
                                               idt2, c->pinned, (double*)K);
  else
    k_assemble<float><<<G, B, 0, c->stream>>>(c->nu, c->nv, c->Nsp, (const float*)c->H_span, c->mass,
                                              idt2, c->pinned, (float*)K);
  return cudaGetLastError();
}

cudaError_t launch_gradient(bsc_ctx* c, const void* C, const void* Chat, void* g) {
  BSC_COUNT(c, 1);
  const int B = 256, G = (c->N + B - 1) / B;
  const double idt2 = c->dt > 0.0 ? 1.0 / (c->dt * c->dt) : 0.0;
  const double* gr = c->gravity;
  if (c->precision == BSC_FP64)
    k_gradient<double><<<G, B, 0, c->stream>>>(c->nu, c->nv, c->Nsp, (const double*)c->g_span, c->mass, idt2,
                                               gr[0], gr[1], gr[2], (const double*)C, (const double*)Chat,
                                               c->pinned, (double*)g);
  else
    k_gradient<float><<<G, B, 0, c->stream>>>(c->nu, c->nv, c->Nsp, (const float*)c->g_span, c->mass, idt2,
                                              gr[0], gr[1], gr[2], (const float*)C, (const float*)Chat,
                                              c->pinned, (float*)g);
  return cudaGetLastError();
}

cudaError_t launch_energy(bsc_ctx* c, const void* C, const void* Chat, double* dE) {
  BSC_COUNT(c, 2);
  constexpr int B = 256;
  const int G = c->red_grid;
  const double idt2 = c->dt > 0.0 ? 1.0 / (c->dt * c->dt) : 0.0;
  const double* gr = c->gravity;
  if (c->precision == BSC_FP64)
    k_energy_partials<double, B><<<G, B, 0, c->stream>>>(c->N, c->Nsp, c->E_span, c->mass, idt2, gr[0], gr[1],
                                                         gr[2], (const double*)C, (const double*)Chat,
                                                         c->partials);
  else
    k_energy_partials<float, B><<<G, B, 0, c->stream>>>(c->N, c->Nsp, c->E_span, c->mass, idt2, gr[0], gr[1],
                                                        gr[2], (const float*)C, (const float*)Chat,
                                                        c->partials);
  k_sum_partials<B><<<1, B, 0, c->stream>>>(G, c->partials, dE, c->dstatus);
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

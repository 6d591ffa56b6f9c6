// Strip decomposition of one patch over ranks: the per-rank pieces.
//
// A strip window context (bsc_create_window) holds the control-point rows
// [row0, row1) of a patch and owns [own0, own1); everything a Newton
// iteration needs beyond its own rows comes from two halo rows on each side
// (span b couples rows b .. b + 2).  The block-Jacobi PCG of the Newton
// step (Sec. 5.1) runs one step per call here, on the owned rows, and hands
// its dot products back as one partial sum per owned row: one block per row,
// each thread summing its control points in order, then a fixed shuffle
// tree.  A row's partial depends on the row's values alone, so adding the
// partials of all ranks in the global row order gives the same scalars for
// every decomposition of the patch, one window of all rows included; the
// iterates are then the same bit for bit.  Exchanging halo rows and
// gathering the partials is the caller's part: no kernel here waits for
// another rank.
#include <cmath>

#include "bsc_internal.cuh"

namespace {

constexpr int ROW_BLOCK = 256;

// x = 0, r = -g, D = inverse diagonal blocks, z = D r, p = z on owned row
// jl0 + blockIdx.x; partials r.z and r.r of the row.
template <typename T>
__global__ void __launch_bounds__(ROW_BLOCK) k_strip_begin(int nu, int N, int jl0, int nrows, const T* __restrict__ K,
                                                           T* __restrict__ Dinv, const T* __restrict__ g,
                                                           T* __restrict__ x, T* __restrict__ r, T* __restrict__ z,
                                                           T* __restrict__ p, double* __restrict__ rows, int* status) {
  __shared__ double sm[ROW_BLOCK / 32];
  const int jl = jl0 + blockIdx.x;
  double a = 0.0, b = 0.0;
  for (int i = threadIdx.x; i < nu; i += ROW_BLOCK) {
    const int al = jl * nu + i;
    block_jacobi_at<T>(N, al, K, Dinv, status);
    T rr[3], zz[3];
#pragma unroll
    for (int c = 0; c < 3; ++c) {
      x[c * N + al] = T(0);
      rr[c] = -g[c * N + al];
      r[c * N + al] = rr[c];
    }
    apply_dinv<T>(Dinv, N, al, rr, zz);
#pragma unroll
    for (int c = 0; c < 3; ++c) {
      z[c * N + al] = zz[c];
      p[c * N + al] = zz[c];
      a += (double)rr[c] * (double)zz[c];
      b += (double)rr[c] * (double)rr[c];
    }
  }
  a = block_sum<ROW_BLOCK>(a, sm);
  b = block_sum<ROW_BLOCK>(b, sm);
  if (threadIdx.x == 0) {
    rows[blockIdx.x] = a;
    rows[nrows + blockIdx.x] = b;
  }
}

// q = K p on an owned row (p's halo rows current); partial p.q.
template <typename T>
__global__ void __launch_bounds__(ROW_BLOCK) k_strip_product(int nu, int nv, int N, int jl0, const T* __restrict__ K,
                                                             const T* __restrict__ p, T* __restrict__ q,
                                                             double* __restrict__ rows) {
  __shared__ double sm[ROW_BLOCK / 32];
  const int jl = jl0 + blockIdx.x;
  double a = 0.0;
  for (int i = threadIdx.x; i < nu; i += ROW_BLOCK) {
    const int al = jl * nu + i;
    T y[3];
    spmv_row<T>(nu, nv, N, al, K, p, y);
#pragma unroll
    for (int c = 0; c < 3; ++c) {
      q[c * N + al] = y[c];
      a += (double)p[c * N + al] * (double)y[c];
    }
  }
  a = block_sum<ROW_BLOCK>(a, sm);
  if (threadIdx.x == 0) rows[blockIdx.x] = a;
}

// x += alpha p, r -= alpha q, z = D r on an owned row; partials r.z, r.r.
template <typename T>
__global__ void __launch_bounds__(ROW_BLOCK) k_strip_update(int nu, int N, int jl0, int nrows, double alpha,
                                                            const T* __restrict__ Dinv, const T* __restrict__ p,
                                                            const T* __restrict__ q, T* __restrict__ x,
                                                            T* __restrict__ r, T* __restrict__ z,
                                                            double* __restrict__ rows) {
  __shared__ double sm[ROW_BLOCK / 32];
  const int jl = jl0 + blockIdx.x;
  const T ta = (T)alpha;
  double a = 0.0, b = 0.0;
  for (int i = threadIdx.x; i < nu; i += ROW_BLOCK) {
    const int al = jl * nu + i;
    T rr[3], zz[3];
#pragma unroll
    for (int c = 0; c < 3; ++c) {
      x[c * N + al] += ta * p[c * N + al];
      rr[c] = r[c * N + al] - ta * q[c * N + al];
      r[c * N + al] = rr[c];
    }
    apply_dinv<T>(Dinv, N, al, rr, zz);
#pragma unroll
    for (int c = 0; c < 3; ++c) {
      z[c * N + al] = zz[c];
      a += (double)rr[c] * (double)zz[c];
      b += (double)rr[c] * (double)rr[c];
    }
  }
  a = block_sum<ROW_BLOCK>(a, sm);
  b = block_sum<ROW_BLOCK>(b, sm);
  if (threadIdx.x == 0) {
    rows[blockIdx.x] = a;
    rows[nrows + blockIdx.x] = b;
  }
}

// p = z + beta p on an owned row.
template <typename T>
__global__ void __launch_bounds__(ROW_BLOCK) k_strip_direction(int nu, int N, int jl0, double beta,
                                                               const T* __restrict__ z, T* __restrict__ p) {
  const int jl = jl0 + blockIdx.x;
  const T tb = (T)beta;
  for (int i = threadIdx.x; i < nu; i += ROW_BLOCK) {
    const int al = jl * nu + i;
#pragma unroll
    for (int c = 0; c < 3; ++c) p[c * N + al] = z[c * N + al] + tb * p[c * N + al];
  }
}

// The owned rows in the window's local numbering.
int own_first(const bsc_ctx* c) { return c->win_own0 - c->win_row0; }
int own_count(const bsc_ctx* c) { return c->win_own1 - c->win_own0; }

bsc_status need_window(bsc_ctx* c, const char* where) {
  if (!c->is_window) return fail(c, BSC_ERR_INVALID_ARG, "%s: not a strip window context (bsc_create_window)", where);
  return BSC_OK;
}

// Copies n partials to the host and reads the status word (synchronises).
bsc_status rows_out(bsc_ctx* c, double* rows, int n, const char* where) {
  cudaError_t e = cudaGetLastError();
  if (e == cudaSuccess) e = cudaMemcpyAsync(rows, c->partials, sizeof(double) * n, cudaMemcpyDeviceToHost, c->stream);
  if (e != cudaSuccess) return cuda_fail(c, e, where);
  return check_status(c, where);
}

}  // namespace

extern "C" {

bsc_status bsc_window_energy_rows(bsc_ctx* c, const void* C, const void* Chat, double* out, int cap, int* count) {
  if (!c) return BSC_ERR_INVALID_ARG;
  const char* where = "bsc_window_energy_rows";
  bsc_status st = need_window(c, where);
  if (st != BSC_OK) return st;
  const int n = c->n_red_items;
  if (count) *count = n;
  if (!out) return BSC_OK;
  if (cap < n) return fail(c, BSC_ERR_INVALID_ARG, "%s: out holds %d values, %d needed", where, cap, n);
  const bool inertia = c->hpd[0].inv_dt2 > 0.0;
  if (!C || (inertia && !Chat)) return fail(c, BSC_ERR_INVALID_ARG, "%s: NULL argument", where);
  if (!aligned16(C) || (Chat && !aligned16(Chat)))
    return fail(c, BSC_ERR_INVALID_ARG, "%s: pointers must be 16-byte aligned", where);
  cudaError_t e = launch_span_eval(c, C, 0, 0);
  // the per-item partials (one per owned span row, then per owned row) stay in c->partials
  if (e == cudaSuccess) e = launch_patch_energy(c, C, Chat, c->patch_E);
  if (e != cudaSuccess) return cuda_fail(c, e, where);
  return rows_out(c, out, n, where);
}

bsc_status bsc_window_pcg_begin(bsc_ctx* c, const void* K, const void* g, void* x, void* p, double* rows) {
  if (!c) return BSC_ERR_INVALID_ARG;
  const char* where = "bsc_window_pcg_begin";
  bsc_status st = need_window(c, where);
  if (st != BSC_OK) return st;
  if (!K || !g || !x || !p || !rows) return fail(c, BSC_ERR_INVALID_ARG, "%s: NULL argument", where);
  if (!aligned16(K) || !aligned16(g) || !aligned16(x) || !aligned16(p))
    return fail(c, BSC_ERR_INVALID_ARG, "%s: pointers must be 16-byte aligned", where);
  if (x == p || x == g || p == g) return fail(c, BSC_ERR_INVALID_ARG, "%s: g, x and p must not alias", where);
  c->win_x = x;
  c->win_p = p;
  c->K_last = K;
  c->K_last_sym = 0;
  const int n = own_count(c), j0 = own_first(c), nu = c->nu, N = c->N;
  BSC_COUNT(c, 1);
  if (c->precision == BSC_FP64)
    k_strip_begin<double><<<n, ROW_BLOCK, 0, c->stream>>>(nu, N, j0, n, (const double*)K, (double*)c->Dinv,
                                                          (const double*)g, (double*)x, (double*)c->vec[1],
                                                          (double*)c->vec[2], (double*)p, c->partials, c->dstatus);
  else
    k_strip_begin<float><<<n, ROW_BLOCK, 0, c->stream>>>(nu, N, j0, n, (const float*)K, (float*)c->Dinv,
                                                         (const float*)g, (float*)x, (float*)c->vec[1],
                                                         (float*)c->vec[2], (float*)p, c->partials, c->dstatus);
  return rows_out(c, rows, 2 * n, where);
}

bsc_status bsc_window_pcg_product(bsc_ctx* c, const void* K, double* rows) {
  if (!c) return BSC_ERR_INVALID_ARG;
  const char* where = "bsc_window_pcg_product";
  bsc_status st = need_window(c, where);
  if (st != BSC_OK) return st;
  if (!c->win_p) return fail(c, BSC_ERR_INVALID_ARG, "%s: call bsc_window_pcg_begin first", where);
  if (!K || !rows) return fail(c, BSC_ERR_INVALID_ARG, "%s: NULL argument", where);
  const int n = own_count(c), j0 = own_first(c), nu = c->nu, nv = c->nv, N = c->N;
  BSC_COUNT(c, 1);
  if (c->precision == BSC_FP64)
    k_strip_product<double><<<n, ROW_BLOCK, 0, c->stream>>>(nu, nv, N, j0, (const double*)K, (const double*)c->win_p,
                                                            (double*)c->vec[4], c->partials);
  else
    k_strip_product<float><<<n, ROW_BLOCK, 0, c->stream>>>(nu, nv, N, j0, (const float*)K, (const float*)c->win_p,
                                                           (float*)c->vec[4], c->partials);
  return rows_out(c, rows, n, where);
}

bsc_status bsc_window_pcg_update(bsc_ctx* c, double alpha, double* rows) {
  if (!c) return BSC_ERR_INVALID_ARG;
  const char* where = "bsc_window_pcg_update";
  bsc_status st = need_window(c, where);
  if (st != BSC_OK) return st;
  if (!c->win_p) return fail(c, BSC_ERR_INVALID_ARG, "%s: call bsc_window_pcg_begin first", where);
  if (!rows || !std::isfinite(alpha)) return fail(c, BSC_ERR_INVALID_ARG, "%s: NULL rows or non-finite alpha", where);
  const int n = own_count(c), j0 = own_first(c), nu = c->nu, N = c->N;
  BSC_COUNT(c, 1);
  if (c->precision == BSC_FP64)
    k_strip_update<double><<<n, ROW_BLOCK, 0, c->stream>>>(nu, N, j0, n, alpha, (const double*)c->Dinv,
                                                           (const double*)c->win_p, (const double*)c->vec[4],
                                                           (double*)c->win_x, (double*)c->vec[1],
                                                           (double*)c->vec[2], c->partials);
  else
    k_strip_update<float><<<n, ROW_BLOCK, 0, c->stream>>>(nu, N, j0, n, alpha, (const float*)c->Dinv,
                                                          (const float*)c->win_p, (const float*)c->vec[4],
                                                          (float*)c->win_x, (float*)c->vec[1], (float*)c->vec[2],
                                                          c->partials);
  return rows_out(c, rows, 2 * n, where);
}

bsc_status bsc_window_pcg_direction(bsc_ctx* c, double beta) {
  if (!c) return BSC_ERR_INVALID_ARG;
  const char* where = "bsc_window_pcg_direction";
  bsc_status st = need_window(c, where);
  if (st != BSC_OK) return st;
  if (!c->win_p) return fail(c, BSC_ERR_INVALID_ARG, "%s: call bsc_window_pcg_begin first", where);
  if (!std::isfinite(beta)) return fail(c, BSC_ERR_INVALID_ARG, "%s: non-finite beta", where);
  const int n = own_count(c), j0 = own_first(c), nu = c->nu, N = c->N;
  BSC_COUNT(c, 1);
  if (c->precision == BSC_FP64)
    k_strip_direction<double><<<n, ROW_BLOCK, 0, c->stream>>>(nu, N, j0, beta, (const double*)c->vec[2],
                                                              (double*)c->win_p);
  else
    k_strip_direction<float><<<n, ROW_BLOCK, 0, c->stream>>>(nu, N, j0, beta, (const float*)c->vec[2],
                                                             (float*)c->win_p);
  cudaError_t e = cudaGetLastError();
  if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
  if (e != cudaSuccess) return cuda_fail(c, e, where);
  return BSC_OK;
}

bsc_status bsc_axpy(bsc_ctx* c, const void* a, const void* d, double alpha, void* out) {
  if (!c) return BSC_ERR_INVALID_ARG;
  if (!a || !d || !out) return fail(c, BSC_ERR_INVALID_ARG, "bsc_axpy: NULL argument");
  if (!aligned16(a) || !aligned16(d) || !aligned16(out))
    return fail(c, BSC_ERR_INVALID_ARG, "bsc_axpy: pointers must be 16-byte aligned");
  if (!std::isfinite(alpha)) return fail(c, BSC_ERR_INVALID_ARG, "bsc_axpy: non-finite alpha");
  cudaError_t e = launch_axpy_trial(c, a, d, alpha, out);
  if (e != cudaSuccess) return cuda_fail(c, e, "bsc_axpy");
  return BSC_OK;
}

}  // extern "C"

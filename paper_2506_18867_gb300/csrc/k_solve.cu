// K5 / K6: stencil SpMV and the preconditioned CG that solves K d = -g.
//
// SpMV: y_alpha = sum over the 25 stencil slots of K(alpha, slot) x_beta; one
// thread per control point reads its 225 matrix entries from 225 planes
// (coalesced across threads) and the neighbours' x through the read-only path.
//
// PCG: 3x3 block-Jacobi preconditioned CG in a single persistent cooperative
// kernel.  Every block owns a fixed slice of control points; the three
// reductions per iteration (p.q, r.z, r.r) are FP64, summed per block in a
// fixed tree and across blocks in block order, so every block computes the
// same scalars and the result is bitwise reproducible.  Grid barriers are
// bounded (they raise a timeout flag instead of waiting forever).
#include <cooperative_groups.h>

#include "bsc_internal.cuh"

namespace {

// Row alpha of y = K x in the element type T (FP32 bulk arithmetic in FP32 mode).
template <typename T>
__device__ __forceinline__ void spmv_row(int nu, int nv, int N, int al, const T* __restrict__ K,
                                         const T* __restrict__ x, T y[3]) {
  const int i = al % nu, j = al / nu;
  T y0 = T(0), y1 = T(0), y2 = T(0);
#pragma unroll
  for (int dv = -2; dv <= 2; ++dv) {
    const int jb = j + dv;
    if (jb < 0 || jb >= nv) continue;
#pragma unroll
    for (int du = -2; du <= 2; ++du) {
      const int ib = i + du;
      if (ib < 0 || ib >= nu) continue;
      const int slot = (dv + 2) * 5 + (du + 2), be = jb * nu + ib;
      const T x0 = __ldg(x + be), x1 = __ldg(x + N + be), x2 = __ldg(x + 2 * N + be);
      const T* Kb = K + (size_t)slot * 9 * N + al;
      y0 += Kb[0] * x0 + Kb[(size_t)N] * x1 + Kb[(size_t)2 * N] * x2;
      y1 += Kb[(size_t)3 * N] * x0 + Kb[(size_t)4 * N] * x1 + Kb[(size_t)5 * N] * x2;
      y2 += Kb[(size_t)6 * N] * x0 + Kb[(size_t)7 * N] * x1 + Kb[(size_t)8 * N] * x2;
    }
  }
  y[0] = y0; y[1] = y1; y[2] = y2;
}

template <typename T>
__global__ void k_spmv(int nu, int nv, const T* __restrict__ K, const T* __restrict__ x, T* __restrict__ y) {
  const int N = nu * nv;
  const int al = blockIdx.x * blockDim.x + threadIdx.x;
  if (al >= N) return;
  T acc[3];
  spmv_row<T>(nu, nv, N, al, K, x, acc);
  y[al] = acc[0];
  y[N + al] = acc[1];
  y[2 * N + al] = acc[2];
}

// Inverse of each 3x3 diagonal block (adjugate / determinant, FP64).
template <typename T>
__global__ void k_block_jacobi(int N, const T* __restrict__ K, T* __restrict__ Dinv, int* status) {
  const int al = blockIdx.x * blockDim.x + threadIdx.x;
  if (al >= N) return;
  const int slot = 12;  // du = dv = 0
  double a[9];
#pragma unroll
  for (int k = 0; k < 9; ++k) a[k] = (double)K[(size_t)(slot * 9 + k) * N + al];
  const double c00 = a[4] * a[8] - a[5] * a[7], c01 = a[5] * a[6] - a[3] * a[8], c02 = a[3] * a[7] - a[4] * a[6];
  const double det = a[0] * c00 + a[1] * c01 + a[2] * c02;
  if (!(fabs(det) > 0.0) || !isfinite(det)) atomicOr(status, BSC_STATUS_NUMERIC_FLAG);
  const double id = 1.0 / det;
  double b[9];
  b[0] = c00 * id;
  b[1] = (a[2] * a[7] - a[1] * a[8]) * id;
  b[2] = (a[1] * a[5] - a[2] * a[4]) * id;
  b[3] = c01 * id;
  b[4] = (a[0] * a[8] - a[2] * a[6]) * id;
  b[5] = (a[2] * a[3] - a[0] * a[5]) * id;
  b[6] = c02 * id;
  b[7] = (a[1] * a[6] - a[0] * a[7]) * id;
  b[8] = (a[0] * a[4] - a[1] * a[3]) * id;
#pragma unroll
  for (int k = 0; k < 9; ++k) Dinv[(size_t)k * N + al] = (T)b[k];
}

template <typename T>
struct PcgArgs {
  int nu, nv, N, maxit;
  double tol;
  const T* __restrict__ K;
  const T* __restrict__ Dinv;
  const T* __restrict__ b;
  T* __restrict__ x;
  T* __restrict__ r;
  T* __restrict__ z;
  T* __restrict__ p;
  T* __restrict__ q;
  double* __restrict__ partial;  // [3][gridDim.x]
  unsigned int* sync;
  int* status;
  double* out;                   // [0] iterations, [1] relative residual
};

template <int BLOCK>
__device__ __forceinline__ double grid_sum(const double* part, int G, double* sm) {
  double acc = 0.0;
  for (int k = threadIdx.x; k < G; k += BLOCK) acc += part[k];
  const double s = block_sum<BLOCK>(acc, sm);
  __shared__ double bcast;
  if (threadIdx.x == 0) bcast = s;
  __syncthreads();
  return bcast;
}

template <typename T>
__device__ __forceinline__ void apply_dinv(const T* __restrict__ Dinv, int N, int al, const T r[3], T z[3]) {
#pragma unroll
  for (int c = 0; c < 3; ++c)
    z[c] = Dinv[(3 * c) * N + al] * r[0] + Dinv[(3 * c + 1) * N + al] * r[1] + Dinv[(3 * c + 2) * N + al] * r[2];
}

template <typename T, int BLOCK>
__global__ void __launch_bounds__(BLOCK) k_pcg(PcgArgs<T> A) {
  __shared__ double sm[BLOCK / 32];
  const int G = gridDim.x, N = A.N;
  const int tid = blockIdx.x * BLOCK + threadIdx.x, stride = G * BLOCK;
  unsigned int* cnt = A.sync;
  volatile unsigned int* gen = A.sync + 1;

  double l_rz = 0.0, l_bb = 0.0;
  for (int al = tid; al < N; al += stride) {
    T rr[3], zz[3];
#pragma unroll
    for (int c = 0; c < 3; ++c) {
      A.x[c * N + al] = T(0);
      rr[c] = A.b[c * N + al];
      A.r[c * N + al] = rr[c];
    }
    apply_dinv<T>(A.Dinv, N, al, rr, zz);
#pragma unroll
    for (int c = 0; c < 3; ++c) {
      A.z[c * N + al] = zz[c];
      A.p[c * N + al] = zz[c];
      l_rz += (double)rr[c] * (double)zz[c];
      l_bb += (double)rr[c] * (double)rr[c];
    }
  }
  {
    const double s1 = block_sum<BLOCK>(l_rz, sm);
    const double s2 = block_sum<BLOCK>(l_bb, sm);
    if (threadIdx.x == 0) {
      A.partial[blockIdx.x] = s1;
      A.partial[G + blockIdx.x] = s2;
    }
  }
  if (!grid_barrier(cnt, gen, A.status)) return;
  double rz = grid_sum<BLOCK>(A.partial, G, sm);
  const double bb = grid_sum<BLOCK>(A.partial + G, G, sm);
  const double stop2 = A.tol * A.tol * bb;
  int it = 0;
  double rr_glob = bb;
  bool ok = true;
  if (bb > 0.0) {
    for (it = 1; it <= A.maxit; ++it) {
      double l_pq = 0.0;
      for (int al = tid; al < N; al += stride) {
        T y[3];
        spmv_row<T>(A.nu, A.nv, N, al, A.K, A.p, y);
#pragma unroll
        for (int c = 0; c < 3; ++c) {
          A.q[c * N + al] = y[c];
          l_pq += (double)A.p[c * N + al] * (double)y[c];
        }
      }
      {
        const double s = block_sum<BLOCK>(l_pq, sm);
        if (threadIdx.x == 0) A.partial[2 * G + blockIdx.x] = s;
      }
      if (!(ok = grid_barrier(cnt, gen, A.status))) break;
      const double pq = grid_sum<BLOCK>(A.partial + 2 * G, G, sm);
      if (!(pq > 0.0) || !isfinite(pq)) {
        if (threadIdx.x == 0 && blockIdx.x == 0) atomicOr(A.status, BSC_STATUS_NUMERIC_FLAG);
        ok = false;
        break;
      }
      const double alpha = rz / pq;
      const T ta = (T)alpha;
      double l_rz2 = 0.0, l_rr = 0.0;
      for (int al = tid; al < N; al += stride) {
        T rr[3], zz[3];
#pragma unroll
        for (int c = 0; c < 3; ++c) {
          A.x[c * N + al] += ta * A.p[c * N + al];
          rr[c] = A.r[c * N + al] - ta * A.q[c * N + al];
          A.r[c * N + al] = rr[c];
        }
        apply_dinv<T>(A.Dinv, N, al, rr, zz);
#pragma unroll
        for (int c = 0; c < 3; ++c) {
          A.z[c * N + al] = zz[c];
          l_rz2 += (double)rr[c] * (double)zz[c];
          l_rr += (double)rr[c] * (double)rr[c];
        }
      }
      {
        const double s1 = block_sum<BLOCK>(l_rz2, sm);
        const double s2 = block_sum<BLOCK>(l_rr, sm);
        if (threadIdx.x == 0) {
          A.partial[blockIdx.x] = s1;
          A.partial[G + blockIdx.x] = s2;
        }
      }
      if (!(ok = grid_barrier(cnt, gen, A.status))) break;
      const double rz2 = grid_sum<BLOCK>(A.partial, G, sm);
      rr_glob = grid_sum<BLOCK>(A.partial + G, G, sm);
      if (rr_glob <= stop2 || !isfinite(rr_glob)) break;
      const double beta = rz2 / rz;
      const T tb = (T)beta;
      rz = rz2;
      for (int al = tid; al < N; al += stride)
#pragma unroll
        for (int c = 0; c < 3; ++c) A.p[c * N + al] = A.z[c * N + al] + tb * A.p[c * N + al];
      if (!(ok = grid_barrier(cnt, gen, A.status))) break;
    }
  }
  if (blockIdx.x == 0 && threadIdx.x == 0) {
    A.out[0] = (double)(it > A.maxit ? A.maxit : it);
    A.out[1] = bb > 0.0 ? sqrt(rr_glob / bb) : 0.0;
    A.out[2] = ok ? 1.0 : 0.0;
  }
}

template <typename T>
__global__ void k_axpy(int n, const T* __restrict__ a, const T* __restrict__ d, double alpha, T* __restrict__ out) {
  const int k = blockIdx.x * blockDim.x + threadIdx.x;
  if (k < n) out[k] = a[k] + (T)alpha * d[k];
}

template <typename T, int BLOCK>
__global__ void k_absmax_partials(int n, const T* __restrict__ x, double* __restrict__ partial) {
  __shared__ double sm[BLOCK / 32];
  double m = 0.0;
  for (int k = blockIdx.x * BLOCK + threadIdx.x; k < n; k += gridDim.x * BLOCK) m = fmax(m, fabs((double)x[k]));
  const double r = block_max<BLOCK>(m, sm);
  if (threadIdx.x == 0) partial[blockIdx.x] = r;
}

template <int BLOCK>
__global__ void k_max_partials(int n, const double* __restrict__ partial, double* __restrict__ out) {
  __shared__ double sm[BLOCK / 32];
  double m = 0.0;
  for (int k = threadIdx.x; k < n; k += BLOCK) m = fmax(m, partial[k]);
  const double r = block_max<BLOCK>(m, sm);
  if (threadIdx.x == 0) *out = r;
}

template <typename T>
cudaError_t pcg_t(bsc_ctx* c, const void* K, const void* b, void* x, double tol, int maxit) {
  constexpr int B = 256;
  const int N = c->N;
  k_block_jacobi<T><<<(N + 255) / 256, 256, 0, c->stream>>>(N, (const T*)K, (T*)c->Dinv, c->dstatus);
  PcgArgs<T> A;
  A.nu = c->nu; A.nv = c->nv; A.N = N; A.maxit = maxit; A.tol = tol;
  A.K = (const T*)K; A.Dinv = (const T*)c->Dinv; A.b = (const T*)b; A.x = (T*)x;
  A.r = (T*)c->vec[1]; A.z = (T*)c->vec[2]; A.p = (T*)c->vec[3]; A.q = (T*)c->vec[4];
  A.partial = c->partials; A.sync = c->sync; A.status = c->dstatus; A.out = c->dscalars + 8;
  void* args[] = {&A};
  return cudaLaunchCooperativeKernel((const void*)k_pcg<T, B>, dim3(c->pcg_grid), dim3(B), args, 0, c->stream);
}

}  // namespace

// Grid size of the persistent PCG kernel: every block must be co-resident.
int pcg_grid_size(int precision, int num_sms, int N) {
  int per_sm = 0;
  if (precision == BSC_FP64)
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_pcg<double, 256>, 256, 0);
  else
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_pcg<float, 256>, 256, 0);
  if (per_sm < 1) per_sm = 1;
  if (per_sm > 2) per_sm = 2;
  int g = num_sms * per_sm;
  const int need = (N + 255) / 256;
  if (g > need) g = need < 1 ? 1 : need;
  return g;
}

cudaError_t launch_spmv(bsc_ctx* c, const void* K, const void* x, void* y) {
  BSC_COUNT(c, 1);
  const int B = 256, G = (c->N + B - 1) / B;
  if (c->precision == BSC_FP64)
    k_spmv<double><<<G, B, 0, c->stream>>>(c->nu, c->nv, (const double*)K, (const double*)x, (double*)y);
  else
    k_spmv<float><<<G, B, 0, c->stream>>>(c->nu, c->nv, (const float*)K, (const float*)x, (float*)y);
  return cudaGetLastError();
}

cudaError_t launch_pcg(bsc_ctx* c, const void* K, const void* b, void* x, double tol, int maxit) {
  BSC_COUNT(c, 2);
  if (c->precision == BSC_FP64) return pcg_t<double>(c, K, b, x, tol, maxit);
  return pcg_t<float>(c, K, b, x, tol, maxit);
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

cudaError_t launch_absmax(bsc_ctx* c, const void* x, double* dout) {
  BSC_COUNT(c, 2);
  constexpr int B = 256;
  const int n = 3 * c->N, G = c->red_grid;
  if (c->precision == BSC_FP64)
    k_absmax_partials<double, B><<<G, B, 0, c->stream>>>(n, (const double*)x, c->partials);
  else
    k_absmax_partials<float, B><<<G, B, 0, c->stream>>>(n, (const float*)x, c->partials);
  k_max_partials<B><<<1, B, 0, c->stream>>>(G, c->partials, dout);
  return cudaGetLastError();
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
  constexpr int B = 256;
  const int N = nu * nv;
  int per_sm = 0;
  cudaError_t e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_pcg<T, B>, B, 0);
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
  // the barrier words and the status must start at zero on every call
  if ((e = cudaMemsetAsync(tail, 0, 4 * sizeof(double), st)) != cudaSuccess) return e;
  k_block_jacobi<T><<<(N + 255) / 256, 256, 0, st>>>(N, (const T*)K, Dinv, status);
  if ((e = cudaGetLastError()) != cudaSuccess) return e;
  PcgArgs<T> A;
  A.nu = nu; A.nv = nv; A.N = N; A.maxit = maxit; A.tol = tol;
  A.K = (const T*)K; A.Dinv = Dinv; A.b = (const T*)b; A.x = (T*)x;
  A.r = r; A.z = z; A.p = p; A.q = q;
  A.partial = partial; A.sync = sync; A.status = status; A.out = outd;
  void* args[] = {&A};
  e = cudaLaunchCooperativeKernel((const void*)k_pcg<T, B>, dim3(grid), dim3(B), args, 0, st);
  if (e != cudaSuccess) return e;
  double stat_d = 0.0;
  if ((e = cudaMemcpyAsync(out_host, outd, 3 * sizeof(double), cudaMemcpyDeviceToHost, st)) != cudaSuccess) return e;
  int flags = 0;
  if ((e = cudaMemcpyAsync(&flags, status, sizeof(int), cudaMemcpyDeviceToHost, st)) != cudaSuccess) return e;
  if ((e = cudaStreamSynchronize(st)) != cudaSuccess) return e;
  (void)stat_d;
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

// Internal declarations of the sm_103a B-spline cloth FEM library: the
// context, device-side helpers and the kernel launchers shared between the
// translation units.  Nothing here is part of the C ABI.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "../../include/bsc.h"

#define BSC_STATUS_TIMEOUT_FLAG 1
#define BSC_STATUS_NUMERIC_FLAG 2
#define BSC_STATUS_CLUSTER_FLAG 4

// Membrane point table: W = w|det J| then g[9][2] (dN_l/dX_beta), as planes.
constexpr int TABM = 19;
// Bending point table: W * mu_bd then L[9], as planes.
constexpr int TABB = 10;
// Symmetric 6x6 d^2 Psi / df^2 (weighted by W), packed upper, as planes.
constexpr int AQ = 21;
// Packed upper triangle of the 27x27 span Hessian (row <= col).
constexpr int H27 = 378;
// Maximum quadrature points owned by one span (corner spans: 3x3 Gauss).
constexpr int MAXQ_MEM = 9;
constexpr int MAXQ_BD = 4;

struct bsc_ctx {
  int nu, nv, Su, Sv, N, Nsp;
  int precision;  // BSC_FP64 / BSC_FP32
  size_t tsize;   // sizeof(T)
  double mu_st1, mu_st2, mu_sh, mu_bd, rho;
  int mem_rule, bend_rule;
  double dt, gravity[3];
  int project_default;
  double pcg_tol;
  int pcg_max_iter, max_ls;
  cudaStream_t stream;
  int device, num_sms;

  // quadrature tables
  int Nmem, Nbd;
  int* mem_off;       // [Nsp + 1]
  int* bd_off;        // [Nsp + 1]
  void* tab_mem;      // T [TABM][Nmem]
  void* tab_bd;       // T [TABB][Nbd]
  double* pts_mem;    // [5][Nmem]: u, v, w, owner a, owner b (inspection)
  double* pts_bd;     // [5][Nbd]
  double* rest;       // [2][N] FP64 material coordinates
  double* mass;       // [N] FP64 lumped masses
  uint8_t* pinned;    // [N]

  // projection buckets (reduced problem sizes 15, 21, 24)
  int* bucket_list;   // [Nsp] span ids grouped by bucket
  int bucket_off[4];  // host: start of each bucket in bucket_list
  int* nneg;          // [Nsp] negative eigenvalues found per span (diagnostic)
  int proj_grid[3];   // resident grid per class
  double* proj_scratch[3];  // per-thread slots of the interior phase-2 kernel (cluster eigenvectors)
  double* proj_span;        // per-span scratch of the interior class
  int* proj_kneg;           // negative-eigenvalue count per interior span (class order)
  unsigned int* proj_work;  // [3] work counters
  cudaStream_t side[2];     // forked streams for the two small classes
  cudaEvent_t fork_ev, join_ev[2];

  // span workspace
  double* E_span;     // [Nsp]
  void* g_span;       // T [27][Nsp]
  void* H_span;       // T [H27][Nsp]
  void* A_mem;        // T [AQ][Nmem]

  // global objects
  void* K_int;        // T [225][N]
  const void* K_last; // last assembled matrix (internal or caller's)
  void* Dinv;         // T [9][N] block-Jacobi preconditioner of K_last
  void* vec[8];       // T [3][N] work vectors: d, r, z, p, q, g, trial C, spare
  double* partials;   // [4][max_grid] reduction partials
  unsigned int* sync; // [4] grid barrier state, arrival counters
  int* dstatus;       // device status flags (BSC_STATUS_*)
  double* dscalars;   // [16] device scalars
  double* hscalars;   // [16] pinned host scalars
  int pcg_grid, pcg_block;
  int red_grid;

  // profiling / diagnostics
  unsigned long long launches;  // kernels launched
  int profiling;
  cudaEvent_t ev[6];

  char err[512];
};

// counts kernel launches of a context (diagnostic; see bsc_launch_count)
#define BSC_COUNT(c, k) ((c)->launches += (k))

// -------------------------------------------------------------------------
// launchers (defined in the .cu files)
// -------------------------------------------------------------------------
cudaError_t launch_build_tables(bsc_ctx* c);
cudaError_t launch_span_eval(bsc_ctx* c, const void* C, int want_grad, int want_hess);
cudaError_t setup_projection(bsc_ctx* c);
cudaError_t launch_project(bsc_ctx* c);
cudaError_t launch_count_projected(bsc_ctx* c, double* dout);
cudaError_t launch_assemble(bsc_ctx* c, void* K);
cudaError_t launch_gradient(bsc_ctx* c, const void* C, const void* Chat, void* g);
cudaError_t launch_energy(bsc_ctx* c, const void* C, const void* Chat, double* dE);
cudaError_t launch_spmv(bsc_ctx* c, const void* K, const void* x, void* y);
cudaError_t launch_pcg(bsc_ctx* c, const void* K, const void* b, void* x, double tol, int maxit);
cudaError_t launch_axpy_trial(bsc_ctx* c, const void* C, const void* d, double alpha, void* out);
cudaError_t launch_copy_vec(bsc_ctx* c, const void* src, void* dst);
cudaError_t launch_absmax(bsc_ctx* c, const void* x, double* dout);
cudaError_t launch_export_span_terms(bsc_ctx* c, void* g_out, void* H_out);

// -------------------------------------------------------------------------
// device helpers
// -------------------------------------------------------------------------
#ifdef __CUDACC__

// Index of (r, c), r <= c, in the packed upper triangle of an n x n matrix
// stored row by row: rows 0..r-1 hold n + (n-1) + ... entries.
__host__ __device__ __forceinline__ int upk(int r, int c, int n) {
  return r * n - (r * (r - 1)) / 2 + (c - r);
}
__host__ __device__ __forceinline__ int sym_upk(int r, int c, int n) {
  return r <= c ? upk(r, c, n) : upk(c, r, n);
}

// Deterministic block sum of one double per thread (fixed shuffle tree, then a
// fixed-order pass over the warp sums).  Result valid in thread 0.
template <int BLOCK>
__device__ __forceinline__ double block_sum(double v, double* sm /* >= BLOCK/32 */) {
  for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
  const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
  if (l == 0) sm[w] = v;
  __syncthreads();
  double s = 0.0;
  if (threadIdx.x == 0) {
    for (int k = 0; k < BLOCK / 32; ++k) s += sm[k];
  }
  __syncthreads();
  return s;
}

template <int BLOCK>
__device__ __forceinline__ double block_max(double v, double* sm) {
  for (int o = 16; o > 0; o >>= 1) v = fmax(v, __shfl_down_sync(0xffffffffu, v, o));
  const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
  if (l == 0) sm[w] = v;
  __syncthreads();
  double s = 0.0;
  if (threadIdx.x == 0) {
    for (int k = 0; k < BLOCK / 32; ++k) s = fmax(s, sm[k]);
  }
  __syncthreads();
  return s;
}

// Grid-wide barrier for a cooperative launch (all blocks co-resident).  The
// wait is bounded: after ~2 s the barrier raises BSC_STATUS_TIMEOUT_FLAG in
// *status and returns false; callers then leave their loops.
__device__ __forceinline__ bool grid_barrier(unsigned int* count, volatile unsigned int* gen,
                                             int* status) {
  __syncthreads();
  __shared__ int ok;
  if (threadIdx.x == 0) {
    ok = 1;
    const unsigned int g = *gen;
    __threadfence();
    const unsigned int arrived = atomicAdd(count, 1u);
    if (arrived == gridDim.x - 1) {
      *count = 0u;
      __threadfence();
      atomicAdd((unsigned int*)gen, 1u);
    } else {
      long long spins = 0;
      while (*gen == g) {
        if (++spins > (1ll << 25)) {  // ~2 s of 64 ns sleeps
          atomicOr(status, BSC_STATUS_TIMEOUT_FLAG);
          ok = 0;
          break;
        }
        if (*(volatile int*)status & BSC_STATUS_TIMEOUT_FLAG) {
          ok = 0;
          break;
        }
        __nanosleep(64);
      }
    }
    __threadfence();
  }
  __syncthreads();
  return ok != 0;
}

#endif  // __CUDACC__

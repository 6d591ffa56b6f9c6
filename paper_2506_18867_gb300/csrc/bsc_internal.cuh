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

// One patch of a context as the kernels see it.  A context holds one or
// more patches; every per-control-point array is one set of planes over the
// concatenated control points of all patches (patch p owns entries
// [cp0, cp0 + N) of each plane) and every per-span array likewise over the
// concatenated spans ([sp0, sp0 + Nsp)).  Within a patch the usual
// tensor-product numbering holds: control point alpha = j nu + i, span
// s = b Su + a.
// One patch of a context.  A strip window of a larger patch (bsc_create_window)
// holds the control-point rows [vb0, vb0 + nv) of a patch with SvG span rows:
// its spans are the global span rows vb0 .. vb0 + Sv - 1, and the quadrature
// rule and knots follow the global row (vb0 = 0, SvG = Sv for a whole patch).
struct PatchDev {
  int nu, nv, Su, Sv, N, Nsp, cp0, sp0;
  int vb0, SvG;
  double mu1, mu2, mush, mubd, rho, inv_dt2;
  double grav[3];
  double pad;
};

// Work item of the span kernels: patch p, and either a run of consecutive
// spans starting at local span `first` (tu == 0) or a tu x (BLOCK / tu)
// tile with origin (a0, b0).
struct SpanItem {
  int p, first_or_a0, tu, b0;
};

// Work item of the per-patch reductions: a chunk [lo, hi) of the patch's
// spans (kind 0) or control points (kind 1), local indices.
struct RedItem {
  int p, kind, lo, hi;
};

// Block of the persistent PCG: its patch, its rank and the size of the
// patch's block group, and the global index of the group's first block.
struct PcgBlock {
  int p, rank, size, first;
};

// Per-patch Newton state (device), one record per patch.
struct PatchStep {
  double E0, E1, alpha, dir_inf;
  double pcg_iters, pcg_res, pcg_ok, spans_projected;
  double fcg_iters, fell_back;  // learned solver: flexible-CG iterations, PCG fallback taken
  int state;       // 1 line search pending, 0 accepted, -1 no decrease, -2 aborted
  int halvings;
  int accepted_round;
  int pad;
};

// Span-tile classes of the autotuner, by the patch's span count per row.
constexpr int TILE_CLASSES = 4;
__host__ __device__ __forceinline__ int tile_class_of(int Su) {
  return Su < 32 ? 0 : (Su < 64 ? 1 : (Su < 128 ? 2 : 3));
}

struct bsc_ctx {
  int P;                 // patches
  int nu, nv, Su, Sv;    // patch 0 (single-patch contexts)
  int N, Nsp;            // totals over the patches
  int precision;         // BSC_FP64 / BSC_FP32
  size_t tsize;          // sizeof(T)
  int mem_rule, bend_rule;
  int project_default;
  double pcg_tol;
  int pcg_max_iter, max_ls;
  cudaStream_t stream;
  int device, num_sms;

  // patches
  PatchDev* hpd;         // host copy [P]
  PatchDev* pd;          // device [P]
  int* cp_patch;         // [N] patch of every control point
  int* sp_patch;         // [Nsp] patch of every span

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

  // projection buckets by the number of derivative vectors m = 2 n_mem + n_bd:
  // m <= 5, 6..7, >= 8 (reduced problem sizes 15, 24, 24)
  int* bucket_list;   // [Nsp] span ids grouped by bucket
  int bucket_off[4];  // host: start of each bucket in bucket_list
  int* nneg;          // [Nsp] negative eigenvalues found per span (diagnostic)
  // reduced bases of the projection (rest geometry only, computed at create)
  double* red_g;      // [16][Nmem] g_q,beta of each membrane point in its span's reduced basis
  double* red_l;      // [8][Nbd] L_q of each bending point in its span's reduced basis
  float2* red_g2;     // FP32 contexts: red_g as double-float splits (hi, lo)
  float2* red_l2;     // FP32 contexts: red_l as double-float splits
  double* red_q;      // [45][n interior] orthonormal basis of each interior span (class order)
  double* helmert;    // device [72]: the border spans' basis (Helmert contrasts)
  // two span classes: 0 interior (reduced size 15), 1 at or next to the border (24)
  int proj_grid[2][2];      // resident grid per class and phase
  int p2_grid[2][2];        // resident grid of phase 2 per class and occupancy variant
  int p2_variant;           // interior phase-2 variant (autotuned)
  double* proj_scratch[2];  // per-thread slots of the phase-2 kernels (cluster eigenvectors)
  double* proj_span[2];     // per-span scratch of each class
  int* proj_kneg[2];        // negative-eigenvalue count per span (class order)
  unsigned int* proj_work;  // [4] work counters
  int* proj_cnt;            // device [6]: class sizes (interior, border); interior spans failing the PSD
                            // test, left open by the certificate; border spans failing the test
  int* proj_sel;            // device [interior spans]: class positions of the spans failing the PSD test
  int proj_df;              // PSD test and phase 1 in double-float (1) or FP64 (0)
  int proj_psd;             // interior class: 0 no PSD test, 1 the FP64 LDL^T test first, 2 an FP32
                            // certificate of positive definiteness, then the FP64 test on the rest (autotuned)
  int* proj_pre;            // device [interior spans]: class positions the FP32 certificate left open
  int* proj_sel1;           // device [border spans]: class positions failing the border's FP64 test (path 1)
  int p0_grid1;             // resident grid of the border's PSD test
  int p0_grid;              // resident grid of the PSD test
  int pf_grid;              // resident grid of the FP32 certificate
  int border_path;          // 0: one warp per border span, 1: one thread per border span, 2: warps to the
                            // tridiagonal form then eigenpair items, 3: warps test first, then take the failing
  cudaStream_t side[2];     // forked stream of the border class
  cudaEvent_t fork_ev, join_ev[2];

  // span work items (tile shape per class chosen by the autotuner)
  int tile_tu[TILE_CLASSES];  // 0 = runs of consecutive spans, else tile width
  SpanItem* span_items;       // device
  int n_span_items;
  // reduction items, grouped by patch: patch p owns [red_off[p], red_off[p+1])
  RedItem* red_items;         // device
  int* red_off;               // device [P + 1]
  int n_red_items;

  // span workspace
  double* E_span;     // [Nsp]
  void* g_span;       // T [27][Nsp]
  void* H_span;       // T [H27][Nsp]
  void* A_mem;        // T [AQ][Nmem]

  // global objects
  void* K_int;        // T [225][N]
  const void* K_last; // last assembled matrix (internal or caller's)
  int K_last_sym;     // K_last in the symmetric layout (13 slots; the Newton step's own matrix)
  int k_sym;          // the Newton step assembles and solves in the symmetric layout (default 1)
  void* Dinv;         // T [9][N] block-Jacobi preconditioner of K_last
  void* vec[8];       // T [3][N] work vectors: d, r, z, p, q, g, trial C, spare
  double* partials;   // [4][max(red_grid, pcg_grid, n_red_items)] reduction partials
  unsigned int* sync; // [2 P + 2] grid-barrier state (count, generation) per patch group
  int* dstatus;       // device status flags (BSC_STATUS_*)
  double* dscalars;   // [16] device scalars
  double* hscalars;   // [16] pinned host scalars
  int pcg_grid;       // co-resident blocks of the persistent PCG
  int pcg_cap;        // co-resident capacity (pcg_blocks and partials are sized for it)
  int pcg_need;       // most blocks the patches can use (a thread per control point), <= pcg_cap
  PcgBlock* pcg_blocks;  // device [pcg_grid]
  double* pcg_out;    // device [3 P]: iterations, relative residual, ok
  double* pcg_weight; // host [P]: work estimate of each patch's solve (autotuned)
  int pcg_form;       // 0: three group barriers per iteration, 1: the pipelined form with one (autotuned)
  void* pcg_pipe[6];  // T [3][N] vectors of the pipelined form: u, w, m (two buffers), s, z
  int red_grid;

  // per-patch Newton state
  PatchStep* steps;   // device [P]
  PatchStep* hsteps;  // pinned host [P]
  double* patch_E;    // device [2 P]: energy at C, energy at the trial point
  int* pending;       // device [1]: patches whose line search is pending

  int* hflags;        // pinned host [4]: pending line searches, status flags

  // linear solver of the Newton step: block-Jacobi PCG, or (solver_cnn set) the
  // learned flexible CG with PCG as fallback; fcg_rec (device [2 P]) holds the
  // flexible CG's iterations and fallback flag of the last learned solve
  struct bsc_cnn* solver_cnn;
  double* fcg_rec;
  // contact with a static obstacle (bsc_contact_attach), or nullptr
  struct bsc_contact* contact;
  // strip window (bsc_create_window): 1, the global rows [win_row0, win_row1)
  // held and [win_own0, win_own1) owned; the caller's solution and direction
  // planes of the strip PCG
  int is_window;
  int win_row0, win_row1, win_own0, win_own1;
  void *win_x, *win_p;
  // bounded device waits of the persistent solvers: spin limit, and blocks
  // their barriers expect beyond the launched ones (0; > 0 only to test the
  // timeout path, see bsc_set_wait_limit)
  long long wait_limit;
  unsigned int barrier_extra;

  // CUDA graph of one Newton iteration, for the pointers it was captured with
  int use_graph;
  cudaGraphExec_t graph;
  const void *graph_C, *graph_Chat;
  int graph_profiling;
  int capturing;                     // enqueue_newton is being captured
  unsigned long long graph_kernels;  // kernels per replay
  long long graph_replays;
  cudaStream_t gstream;              // the graph's stream
  cudaEvent_t gev_in, gev_out;       // order gstream after / before the context's stream

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
cudaError_t launch_lumped_mass_patch(bsc_ctx* c, int p);
cudaError_t build_span_items(bsc_ctx* c);
cudaError_t build_red_items(bsc_ctx* c);
cudaError_t setup_span_eval(bsc_ctx* c);
// want_hess of launch_span_eval: 0 no Hessian, 1 the Hessian as it is, 2 with
// the per-point closed-form projection of the FBW terms (BSC_PROJECT_POINT)
inline int hess_mode(int want_hess, int project) {
  return want_hess ? (project == BSC_PROJECT_POINT ? 2 : 1) : 0;
}
// energy / gradient / Hessian of every span; with a gate, only the spans of
// the patches whose line search is pending (gate[p].state == 1)
cudaError_t launch_span_eval(bsc_ctx* c, const void* C, int want_grad, int want_hess,
                             const PatchStep* gate = nullptr);
cudaError_t launch_span_eval_items(bsc_ctx* c, const void* C, int want_grad, int want_hess, const SpanItem* items,
                                   int n_items, int block_tu);
cudaError_t setup_projection(bsc_ctx* c);
cudaError_t launch_project(bsc_ctx* c);
// the border class alone by the given path, on the context's stream (autotuner)
cudaError_t launch_project_border(bsc_ctx* c, int path);
cudaError_t launch_project_interior(bsc_ctx* c, int phase);
// Dinv (optional): also write the inverse diagonal blocks (block-Jacobi)
cudaError_t launch_assemble(bsc_ctx* c, void* K, int sym = 0, void* Dinv = nullptr);
cudaError_t launch_gradient(bsc_ctx* c, const void* C, const void* Chat, void* g);
// per-patch incremental potential into dE[p] (with a gate: pending patches only)
cudaError_t launch_patch_energy(bsc_ctx* c, const void* C, const void* Chat, double* dE,
                                const PatchStep* gate = nullptr);
// sym: K in the symmetric stencil layout (13 slots, see spmv_row_sym)
cudaError_t launch_spmv(bsc_ctx* c, const void* K, const void* x, void* y, int sym = 0);
// dinv_ready: c->Dinv already holds K's inverse diagonal blocks (launch_assemble)
cudaError_t launch_pcg(bsc_ctx* c, const void* K, const void* b, void* x, double tol, int maxit, int sym = 0,
                       int dinv_ready = 0);
// PCG as the fallback of a learned flexible-CG solve: it reads that solve's
// result record (iterations, r.r, state) and b.b on the device, returns at
// once (x = 0) when the flexible CG converged, and otherwise solves K x = b
// to min(1/2, tol sqrt(b.b / r.r)), the tolerance that finishes the solve.
cudaError_t launch_pcg_fallback(bsc_ctx* c, const void* K, const void* b, void* x, double tol, int maxit,
                                const double* fcg_out, const double* bb);
// The learned flexible CG of the context's solver network (k_cnn.cu): every
// launch of one solve of K x = b (single-patch FP32 contexts), graph-capturable,
// PCG fallback included; leaves the combined result in pcg_out (iterations of
// both solvers, relative residual, ok) and the flexible CG's record in fcg_rec.
cudaError_t enqueue_learned_solve(bsc_ctx* c, struct bsc_cnn* n, const void* K, const void* b, void* x, double tol,
                                  int maxit);
cudaError_t setup_pcg(bsc_ctx* c);
cudaError_t assign_pcg_blocks(bsc_ctx* c);
// Sets the PCG grid (clamped to [patches, capacity]) and re-plans the groups.
cudaError_t set_pcg_grid(bsc_ctx* c, int grid);
cudaError_t launch_axpy_trial(bsc_ctx* c, const void* C, const void* d, double alpha, void* out);
cudaError_t launch_copy_vec(bsc_ctx* c, const void* src, void* dst);
cudaError_t launch_export_span_terms(bsc_ctx* c, void* g_out, void* H_out);
// contact (k_contact.cu): terms at C added to the span arrays after the
// elastic projection; the step bound of a direction into the contact record;
// release with the context
cudaError_t contact_add(bsc_ctx* c, const void* C, int add_g, int add_h, const PatchStep* gate);
cudaError_t contact_step_bound(bsc_ctx* c, const void* C, const void* D);
void contact_destroy(bsc_ctx* c);
// the step bound on the device (nullptr without contact)
const double* contact_bound_ptr(const bsc_ctx* c);
// error helpers of the C ABI (bsc_api.cu): message into the context (or the
// thread's create message), CUDA error, status word read-back and clear
bsc_status fail(bsc_ctx* c, bsc_status st, const char* fmt, ...);
bsc_status cuda_fail(bsc_ctx* c, cudaError_t e, const char* where);
bsc_status check_status(bsc_ctx* c, const char* where);
bool aligned16(const void* p);
// Newton step pieces (k_newton.cu)
cudaError_t launch_step_begin(bsc_ctx* c, const void* d);
cudaError_t launch_ls_round(bsc_ctx* c, const void* C, const void* Chat, const void* d, void* trial, void* Cout,
                            int round);

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

// Spins of 64 ns sleeps a bounded device wait gives up after by default (~2 s).
constexpr long long kWaitLimitDefault = 1ll << 25;

// Barrier over the `nblocks` co-resident blocks that share (count, gen): the
// whole grid of a cooperative launch, or one patch's block group of the
// persistent PCG.  The wait is bounded: after `limit` spins the barrier raises
// BSC_STATUS_TIMEOUT_FLAG in *status and returns false (so does every block
// that sees the flag); callers then leave their loops.
__device__ __forceinline__ bool group_barrier(unsigned int* count, volatile unsigned int* gen, int* status,
                                              unsigned int nblocks, long long limit = kWaitLimitDefault) {
  __syncthreads();
  __shared__ int ok;
  if (threadIdx.x == 0) {
    ok = 1;
    if (nblocks > 1u) {
      const unsigned int g = *gen;
      __threadfence();
      const unsigned int arrived = atomicAdd(count, 1u);
      if (arrived == nblocks - 1u) {
        *count = 0u;
        __threadfence();
        atomicAdd((unsigned int*)gen, 1u);
      } else {
        long long spins = 0;
        while (*gen == g) {
          if (++spins > limit) {
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
    } else if (*(volatile int*)status & BSC_STATUS_TIMEOUT_FLAG) {
      ok = 0;
    }
  }
  __syncthreads();
  return ok != 0;
}

__device__ __forceinline__ bool grid_barrier(unsigned int* count, volatile unsigned int* gen, int* status,
                                             long long limit = kWaitLimitDefault, unsigned int extra = 0u) {
  return group_barrier(count, gen, status, gridDim.x + extra, limit);
}

// z = D r with D the 3x3 block (9 planes, stride N) of control point al.
template <typename T>
__device__ __forceinline__ void apply_dinv(const T* __restrict__ Dinv, int N, int al, const T r[3], T z[3]) {
#pragma unroll
  for (int c = 0; c < 3; ++c)
    z[c] = Dinv[(3 * c) * N + al] * r[0] + Dinv[(3 * c + 1) * N + al] * r[1] + Dinv[(3 * c + 2) * N + al] * r[2];
}

// Inverse of control point al's 3x3 diagonal block of K (stencil slot 12) by
// adjugate / determinant in FP64 into Dinv; a singular or non-finite block
// raises the NUMERIC flag.
template <typename T>
__device__ __forceinline__ void block_jacobi_at(int N, int al, const T* __restrict__ K, T* __restrict__ Dinv,
                                                int* status, int slot = 12 /* du = dv = 0 */) {
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

// Streaming load of a matrix entry: K is read once per product (an entry at
// most twice, by its row and, transposed, by its neighbour's) and is far
// larger than L1, so its lines are cached in L2 only (ld.global.cg) and L1
// keeps the gathered vector entries, each read by up to 25 rows.  A cache
// hint only: the value is that of a plain load.  The built-in leaves the
// compiler free to schedule these loads around the solver's stores, which
// inline-PTX loads with the same caching did not (same-GPU A/B at 1024x1024:
// solve 7.10 ms with the PTX form, 6.36 ms with this one; an L2 evict-first
// policy on top was slower still).
__device__ __forceinline__ float ld_stream(const float* p) { return __ldcg(p); }
__device__ __forceinline__ double ld_stream(const double* p) { return __ldcg(p); }

// Row alpha (patch-local index) of y = K x in the element type T; K and x
// already point at the patch's first control point, N is the plane stride.
// X_MODE 1: x stays unchanged for the whole kernel, so it may go through the
// non-coherent read-only path.  The persistent solvers update their x (the
// search direction) between grid barriers: 0 reads it with plain loads, which
// the barriers' fences make coherent; 2 reads it from L2 (ld.global.cg),
// which is coherent without relying on L1 invalidation.
// FUSED: each row accumulates by three FMAs per block (fewest instructions:
// faster in the persistent PCG, and in FP64, where the FP64 pipe bounds the
// product); otherwise a product, an FMA and an add per block, which the
// learned flexible CG runs faster (measured).
template <typename T, int X_MODE = 0, bool FUSED = true>
__device__ __forceinline__ void spmv_row(int nu, int nv, int N, int al, const T* __restrict__ K, const T* x,
                                         T y[3]) {
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
      T x0, x1, x2;
      if (X_MODE == 1) {
        x0 = __ldg(x + be); x1 = __ldg(x + N + be); x2 = __ldg(x + 2 * N + be);
      } else if (X_MODE == 2) {
        x0 = __ldcg(x + be); x1 = __ldcg(x + N + be); x2 = __ldcg(x + 2 * N + be);
      } else {
        x0 = x[be]; x1 = x[N + be]; x2 = x[2 * N + be];
      }
      const T* Kb = K + (size_t)slot * 9 * N + al;
      if (FUSED) {
        y0 = fma(ld_stream(Kb + (size_t)2 * N), x2, fma(ld_stream(Kb + (size_t)N), x1, fma(ld_stream(Kb), x0, y0)));
        y1 = fma(ld_stream(Kb + (size_t)5 * N), x2, fma(ld_stream(Kb + (size_t)4 * N), x1, fma(ld_stream(Kb + (size_t)3 * N), x0, y1)));
        y2 = fma(ld_stream(Kb + (size_t)8 * N), x2, fma(ld_stream(Kb + (size_t)7 * N), x1, fma(ld_stream(Kb + (size_t)6 * N), x0, y2)));
      } else {
        y0 += ld_stream(Kb) * x0 + ld_stream(Kb + (size_t)N) * x1 + ld_stream(Kb + (size_t)2 * N) * x2;
        y1 += ld_stream(Kb + (size_t)3 * N) * x0 + ld_stream(Kb + (size_t)4 * N) * x1 + ld_stream(Kb + (size_t)5 * N) * x2;
        y2 += ld_stream(Kb + (size_t)6 * N) * x0 + ld_stream(Kb + (size_t)7 * N) * x1 + ld_stream(Kb + (size_t)8 * N) * x2;
      }
    }
  }
  y[0] = y0; y[1] = y1; y[2] = y2;
}

// Row alpha of y = K x with K in the symmetric stencil layout: 13 slots, the
// diagonal block and the 12 blocks coupling alpha to the neighbours after it
// (dv > 0, or dv = 0 and du > 0), slot s' = stencil slot - 12, plane
// (s' * 9 + 3 r + c).  A block before alpha is the transpose of the
// neighbour's block after it, B(alpha, beta) = B(beta, alpha)^T, read from
// the neighbour's row (consecutive alpha read consecutive beta).  Entries and
// accumulation order are those of spmv_row, so both layouts give the same
// product bit for bit; K is read once per product instead of twice.
template <typename T, int X_MODE = 0>
__device__ __forceinline__ void spmv_row_sym(int nu, int nv, int N, int al, const T* __restrict__ K, const T* x,
                                             T y[3]) {
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
      T x0, x1, x2;
      if (X_MODE == 1) {
        x0 = __ldg(x + be); x1 = __ldg(x + N + be); x2 = __ldg(x + 2 * N + be);
      } else {
        x0 = x[be]; x1 = x[N + be]; x2 = x[2 * N + be];
      }
      T k[9];
      if (slot >= 12) {
        const T* Kb = K + (size_t)(slot - 12) * 9 * N + al;
#pragma unroll
        for (int e = 0; e < 9; ++e) k[e] = ld_stream(Kb + (size_t)e * N);
      } else {
        const T* Kb = K + (size_t)(12 - slot) * 9 * N + be;  // the neighbour's slot 24 - slot, transposed
#pragma unroll
        for (int r = 0; r < 3; ++r)
#pragma unroll
          for (int c = 0; c < 3; ++c) k[3 * r + c] = ld_stream(Kb + (size_t)(3 * c + r) * N);
      }
      y0 = fma(k[2], x2, fma(k[1], x1, fma(k[0], x0, y0)));
      y1 = fma(k[5], x2, fma(k[4], x1, fma(k[3], x0, y1)));
      y2 = fma(k[8], x2, fma(k[7], x1, fma(k[6], x0, y2)));
    }
  }
  y[0] = y0; y[1] = y1; y[2] = y2;
}

#endif  // __CUDACC__

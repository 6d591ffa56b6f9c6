// K3: per-span PSD projection of the 27x27 elastic Hessian in FP64
// (projected Newton, Sec. 5.1): P = V max(Lambda, 0) V^T = H - sum_{lam<0}
// lam w w^T.
//
// The span Hessian is
//   H = sum_q (G_q (x) I3) A_q (G_q (x) I3)^T + sum_b W_b mu_bd (L_b L_b^T) (x) I3,
// so its range lies in R (x) R^3 with R = span{g_q,1, g_q,2, L_b} in R^9;
// every such vector sums to zero over the 9 control points (derivatives of a
// partition of unity), so dim R <= min(8, 2 n_mem + n_bd) =: D.  With an
// orthonormal basis Q of R, H = (Q (x) I3) H_r (Q (x) I3)^T and H_r (3D x 3D)
// has the same non-zero spectrum.  H_r is built from the per-point
// d^2 Psi/df^2 kept by the span evaluator, in FP64, and projected by
// proj::project_span (tridiagonalisation, Sturm bisection, inverse
// iteration).
//
// Spans are grouped by D (5, 7, 8).  A block takes BLOCK spans at a time from
// its class's work counter.  Phase 1 (one thread per span) builds H_r,
// tridiagonalises it and counts its negative eigenvalues; phase 2 runs in
// rounds, round r computing eigenpair r of every span that has one, with the
// (span, r) items compacted onto the block's first threads so that no warp
// carries masked lanes through the FP64 work (masked lanes cost the FP64 pipe
// as much as active ones).  Working sets live in interleaved shared memory,
// the basis and eigenvectors of a span in a per-thread global scratch slot.
// The three classes run concurrently on forked streams.
#include "bsc_internal.cuh"
#include "proj_core.cuh"

cudaError_t setup_projection_ring();
cudaError_t launch_project_ring(bsc_ctx* c, int first, int count, unsigned int* work, cudaStream_t st);

namespace {

template <typename T>
struct ProjArgs {
  int Nsp, Nm, Nb;
  double mubd;
  const int* __restrict__ moff;
  const int* __restrict__ boff;
  const T* __restrict__ tabm;
  const T* __restrict__ tabb;
  const T* __restrict__ A;
  T* __restrict__ H;
  int* __restrict__ nneg;
  int* __restrict__ status;
};

// Eigenvalues below -NEG_REL * ||T|| are projected; above that they are
// rounding noise of exact zeros (their contribution is below 1e-14 ||H||).
constexpr double NEG_REL = 1e-14;
// A basis candidate whose residual after orthogonalisation is below
// RANK_REL of its norm lies in the span of the previous ones.
constexpr double RANK_REL = 1e-13;

template <typename T>
struct SpanTab {
  const T* tabm;  // already offset to the span's first membrane point
  const T* tabb;  // already offset to the span's first bending point
  const T* A;
  int Nm, Nb, nmq, nbq;
  double mubd;
  __device__ int nm() const { return nmq; }
  __device__ int nb() const { return nbq; }
  __device__ double g(int q, int l, int be) const { return (double)tabm[(1 + 2 * l + be) * Nm + q]; }
  __device__ double L(int q, int l) const { return (double)tabb[(1 + l) * Nb + q]; }
  __device__ double wb(int q) const { return (double)tabb[q] * mubd; }
  __device__ double a6(int q, int e) const { return (double)A[e * Nm + q]; }
};

// H <- H - lam w w^T on the packed upper triangle, in the element type: the
// correction is formed in FP64 and applied in T (FP32 output stays FP32).
template <typename T>
struct SpanH {
  T* H;
  int Nsp, s;
  __device__ void rank1(double lam, const double (&w)[27]) {
    T wt[27], lw[27];
#pragma unroll
    for (int r = 0; r < 27; ++r) {
      wt[r] = (T)w[r];
      lw[r] = (T)(lam * w[r]);
    }
    T* h = H + s;
    int e = 0;
#pragma unroll
    for (int r = 0; r < 27; ++r)
#pragma unroll
      for (int c = r; c < 27; ++c, ++e) h[(size_t)e * Nsp] -= lw[r] * wt[c];
  }
};

// Shared memory per thread: A (packed H_r, then reflectors), R (3n: basis,
// then the scaled tridiagonal), the scale ||T||, an FP32 copy of (d, e^2)
// and the running lower bracket, all interleaved by thread.
template <int D>
struct Smem {
  static constexpr int n = 3 * D, NP = n * (n + 1) / 2;
  static constexpr int DOUBLES = NP + 3 * n + 1, FLOATS = 2 * n + 1;
};

template <typename T, int D, int BLOCK>
__global__ void __launch_bounds__(BLOCK, 1)
    k_project(ProjArgs<T> P, const int* __restrict__ list, int count, double* __restrict__ scratch,
              unsigned int* __restrict__ work) {
  constexpr int n = 3 * D, NP = Smem<D>::NP;
  extern __shared__ __align__(16) double smd[];
  double* const Abase = smd;
  double* const Rbase = smd + (size_t)NP * BLOCK;
  double* const Tn = smd + (size_t)(NP + 3 * n) * BLOCK;
  float* const Fbase = reinterpret_cast<float*>(smd + (size_t)Smem<D>::DOUBLES * BLOCK);
  float* const Lo = Fbase + 2 * n * BLOCK;
  __shared__ int s_kneg[BLOCK], s_span[BLOCK], s_list[BLOCK], s_wcnt[BLOCK / 32];
  __shared__ int s_base;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int nslots = gridDim.x * BLOCK, slot0 = blockIdx.x * BLOCK;
  for (;;) {
    // a batch of BLOCK spans per block, taken from the class's work counter
    if (tid == 0) s_base = (int)atomicAdd(work, (unsigned)BLOCK);
    __syncthreads();
    const int base = s_base;
    if (base >= count) break;
    // phase 1 (uniform work): one span per thread
    const int t = base + tid;
    int kneg = 0, s = -1;
    if (t < count) {
      s = list[t];
      const int q0 = P.moff[s], b0 = P.boff[s];
      SpanTab<T> tab{P.tabm + q0, P.tabb + b0, P.A + q0, P.Nm, P.Nb, P.moff[s + 1] - q0, P.boff[s + 1] - b0,
                     P.mubd};
      const proj::View A{Abase + tid, BLOCK}, R{Rbase + tid, BLOCK};
      const proj::View Qs{scratch + slot0 + tid, nslots};
      double tn = 0.0;
      kneg = proj::span_phase1<D>(tab, A, R, Qs, &tn, NEG_REL, RANK_REL);
      if (kneg < 0) {
        atomicOr(P.status, BSC_STATUS_NUMERIC_FLAG);
        kneg = 0;
      }
      Tn[tid] = tn;
#pragma unroll
      for (int i = 0; i < n; ++i) {
        Fbase[i * BLOCK + tid] = (float)R[i];
        Fbase[(n + i) * BLOCK + tid] = (float)R[2 * n + i];
      }
      Lo[tid] = -1.0f - 1e-6f;
      P.nneg[s] = kneg;
    }
    s_kneg[tid] = kneg;
    s_span[tid] = s;
    __syncthreads();
    // phase 2: round r handles eigenvalue r of every span that has one; the
    // (span, r) items are compacted onto the first threads of the block
    for (int r = 0;; ++r) {
      const bool flag = s_kneg[tid] > r;
      const unsigned bal = __ballot_sync(0xffffffffu, flag);
      if (lane == 0) s_wcnt[warp] = __popc(bal);
      __syncthreads();
      int off = 0, total = 0;
#pragma unroll
      for (int w = 0; w < BLOCK / 32; ++w) {
        off += (w < warp) ? s_wcnt[w] : 0;
        total += s_wcnt[w];
      }
      if (flag) s_list[off + __popc(bal & ((1u << lane) - 1u))] = tid;
      __syncthreads();
      if (total == 0) break;
      if (tid < total) {
        const int o = s_list[tid];
        const proj::View Ao{Abase + o, BLOCK}, Ro{Rbase + o, BLOCK};
        const proj::View Qo{scratch + slot0 + o, nslots};
        const proj::View Yo{scratch + (size_t)9 * D * nslots + slot0 + o, nslots};
        SpanH<T> hs{P.H, P.Nsp, s_span[o]};
        proj::span_eigpair<D>(Ao, Ro, Qo, Yo, Fbase + o, BLOCK, Lo + o, Tn[o], r, hs, NEG_REL);
      }
      __syncthreads();
    }
  }
}

template <int D>
struct Cfg;
template <> struct Cfg<5> { static constexpr int BLOCK = 128; };

template <int D>
constexpr size_t smem_bytes() {
  return (sizeof(double) * Smem<D>::DOUBLES + sizeof(float) * Smem<D>::FLOATS) * (size_t)Cfg<D>::BLOCK;
}

template <typename T, int D>
cudaError_t run_bucket(bsc_ctx* c, int b, cudaStream_t st) {
  const int count = c->bucket_off[b + 1] - c->bucket_off[b];
  if (count <= 0) return cudaSuccess;
  BSC_COUNT(c, 1);
  constexpr int BLOCK = Cfg<D>::BLOCK;
  ProjArgs<T> P;
  P.Nsp = c->Nsp; P.Nm = c->Nmem; P.Nb = c->Nbd; P.mubd = c->mu_bd;
  P.moff = c->mem_off; P.boff = c->bd_off;
  P.tabm = (const T*)c->tab_mem; P.tabb = (const T*)c->tab_bd;
  P.A = (const T*)c->A_mem; P.H = (T*)c->H_span;
  P.nneg = c->nneg; P.status = c->dstatus;
  auto k = k_project<T, D, BLOCK>;
  cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem_bytes<D>());
  if (e != cudaSuccess) return e;
  if ((e = cudaMemsetAsync(c->proj_work + b, 0, sizeof(unsigned int), st)) != cudaSuccess) return e;
  k<<<c->proj_grid[b], BLOCK, smem_bytes<D>(), st>>>(P, c->bucket_list + c->bucket_off[b], count,
                                                     c->proj_scratch[b], c->proj_work + b);
  return cudaGetLastError();
}

template <typename T>
cudaError_t run_all(bsc_ctx* c) {
  cudaError_t e;
  // fork: the border classes (warp-per-span kernel) on a side stream, the
  // interior class on the context stream; the two co-reside on every SM
  if ((e = cudaEventRecord(c->fork_ev, c->stream)) != cudaSuccess) return e;
  if ((e = cudaStreamWaitEvent(c->side[0], c->fork_ev, 0)) != cudaSuccess) return e;
  if ((e = launch_project_ring(c, c->bucket_off[1], c->bucket_off[3] - c->bucket_off[1], c->proj_work + 1,
                               c->side[0])) != cudaSuccess)
    return e;
  if ((e = run_bucket<T, 5>(c, 0, c->stream)) != cudaSuccess) return e;
  if ((e = cudaEventRecord(c->join_ev[0], c->side[0])) != cudaSuccess) return e;
  return cudaStreamWaitEvent(c->stream, c->join_ev[0], 0);
}

// Number of spans with at least one projected eigenvalue (block counts, then
// a fixed-order sum over blocks).
template <int BLOCK>
__global__ void k_count_projected(int Nsp, const int* __restrict__ nneg, double* __restrict__ partial) {
  __shared__ double sm[BLOCK / 32];
  double acc = 0.0;
  for (int s = blockIdx.x * BLOCK + threadIdx.x; s < Nsp; s += gridDim.x * BLOCK) acc += nneg[s] > 0 ? 1.0 : 0.0;
  const double tot = block_sum<BLOCK>(acc, sm);
  if (threadIdx.x == 0) partial[blockIdx.x] = tot;
}

template <int BLOCK>
__global__ void k_sum_counts(int n, const double* __restrict__ partial, double* __restrict__ out) {
  __shared__ double sm[BLOCK / 32];
  double acc = 0.0;
  for (int k = threadIdx.x; k < n; k += BLOCK) acc += partial[k];
  const double tot = block_sum<BLOCK>(acc, sm);
  if (threadIdx.x == 0) *out = tot;
}

template <typename T, int D>
int resident_grid(int num_sms) {
  int per_sm = 0;
  cudaFuncSetAttribute(k_project<T, D, Cfg<D>::BLOCK>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                       (int)smem_bytes<D>());
  cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_project<T, D, Cfg<D>::BLOCK>, Cfg<D>::BLOCK,
                                                smem_bytes<D>());
  if (per_sm < 1) per_sm = 1;
  return per_sm * num_sms;
}

}  // namespace

// Sizes the interior class's grid and scratch slots and loads the border
// kernel's constants (called from bsc_create).
cudaError_t setup_projection(bsc_ctx* c) {
  const int count = c->bucket_off[1] - c->bucket_off[0];
  const int need = (count + Cfg<5>::BLOCK - 1) / Cfg<5>::BLOCK;
  int g = c->precision == BSC_FP64 ? resident_grid<double, 5>(c->num_sms) : resident_grid<float, 5>(c->num_sms);
  if (g > need) g = need;
  if (g < 1) g = 1;
  c->proj_grid[0] = g;
  {
    const size_t slots = (size_t)g * Cfg<5>::BLOCK;
    cudaError_t e = cudaMalloc(&c->proj_scratch[0], sizeof(double) * (size_t)(9 * 5 + 15 * 15) * slots);
    if (e != cudaSuccess) return e;
    if ((e = setup_projection_ring()) != cudaSuccess) return e;
  }
  cudaError_t e = cudaMalloc(&c->proj_work, sizeof(unsigned int) * 4);
  if (e != cudaSuccess) return e;
  for (int i = 0; i < 2; ++i) {
    if ((e = cudaStreamCreateWithFlags(&c->side[i], cudaStreamNonBlocking)) != cudaSuccess) return e;
    if ((e = cudaEventCreateWithFlags(&c->join_ev[i], cudaEventDisableTiming)) != cudaSuccess) return e;
  }
  return cudaEventCreateWithFlags(&c->fork_ev, cudaEventDisableTiming);
}

cudaError_t launch_count_projected(bsc_ctx* c, double* dout) {
  BSC_COUNT(c, 2);
  k_count_projected<256><<<c->red_grid, 256, 0, c->stream>>>(c->Nsp, c->nneg, c->partials + 2 * c->red_grid);
  k_sum_counts<256><<<1, 256, 0, c->stream>>>(c->red_grid, c->partials + 2 * c->red_grid, dout);
  return cudaGetLastError();
}

cudaError_t launch_project(bsc_ctx* c) {
  if (c->precision == BSC_FP64) return run_all<double>(c);
  return run_all<float>(c);
}

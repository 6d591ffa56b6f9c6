// Projected Newton iteration per patch (Sec. 5.1) as device work: after the
// solve, each patch's step record gets E(C), |d|_inf, the solver's result and
// the number of projected spans; the backtracking line search then runs in
// rounds over all patches at once.  A round evaluates E(C + alpha_p d) for
// every patch still searching, accepts alpha_p where the energy did not
// increase (plain decrease, no Armijo constant), halves it elsewhere (at
// most max_line_search times, then the patch fails), and commits the
// accepted patches' trial positions.  Round 0 (alpha = 1) is part of the
// Newton iteration's CUDA graph; further rounds run only for patches that
// need them.
#include "bsc_internal.cuh"

namespace {

constexpr int SB = 256;

// Per reduction item: projected spans (kind 0) or max |d| (kind 1); the other
// row gets 0 so that per-patch sums / maxima run over all of its items.
template <typename T>
__global__ void __launch_bounds__(SB) k_step_items(int N, int n_items, const RedItem* __restrict__ items,
                                                   const PatchDev* __restrict__ pd, const int* __restrict__ nneg,
                                                   const T* __restrict__ d, double* __restrict__ partial) {
  __shared__ double sm[SB / 32];
  const RedItem it = items[blockIdx.x];
  const PatchDev* pt = pd + it.p;
  double cnt = 0.0, m = 0.0;
  if (it.kind == 0) {
    const int sp0 = __ldg(&pt->sp0);
    for (int k = it.lo + threadIdx.x; k < it.hi; k += SB) cnt += nneg[sp0 + k] > 0 ? 1.0 : 0.0;
  } else {
    const int cp0 = __ldg(&pt->cp0);
    for (int k = it.lo + threadIdx.x; k < it.hi; k += SB) {
      const int al = cp0 + k;
      m = fmax(m, fmax(fabs((double)d[al]), fmax(fabs((double)d[N + al]), fabs((double)d[2 * N + al]))));
    }
  }
  const double c_tot = block_sum<SB>(cnt, sm);
  const double m_tot = block_max<SB>(m, sm);
  if (threadIdx.x == 0) {
    partial[blockIdx.x] = c_tot;
    partial[n_items + blockIdx.x] = m_tot;
  }
}

// One block per patch: opens the patch's step record.
__global__ void __launch_bounds__(SB) k_step_begin(int n_items, const int* __restrict__ red_off,
                                                   const double* __restrict__ partial, const double* __restrict__ E0,
                                                   const double* __restrict__ pcg_out, int project,
                                                   const double* __restrict__ fcg_rec,
                                                   const double* __restrict__ alpha0,
                                                   PatchStep* __restrict__ steps, const int* __restrict__ status) {
  __shared__ double sm[SB / 32];
  const int p = blockIdx.x;
  double cnt = 0.0, m = 0.0;
  for (int k = red_off[p] + threadIdx.x; k < red_off[p + 1]; k += SB) {
    cnt += partial[k];
    m = fmax(m, partial[n_items + k]);
  }
  const double c_tot = block_sum<SB>(cnt, sm);
  const double m_tot = block_max<SB>(m, sm);
  if (threadIdx.x == 0) {
    PatchStep st;
    st.E0 = E0[p];
    st.E1 = 0.0;
    st.alpha = alpha0 ? fmin(1.0, *alpha0) : 1.0;  // contact: the conservative step bound
    st.dir_inf = m_tot;
    st.pcg_iters = pcg_out[3 * p];
    st.pcg_res = pcg_out[3 * p + 1];
    st.pcg_ok = pcg_out[3 * p + 2];
    st.spans_projected = project ? c_tot : 0.0;
    st.fcg_iters = fcg_rec ? fcg_rec[2 * p] : 0.0;
    st.fell_back = fcg_rec ? fcg_rec[2 * p + 1] : 0.0;
    const int flags = *(volatile const int*)status;
    st.state = (flags & (BSC_STATUS_TIMEOUT_FLAG | BSC_STATUS_NUMERIC_FLAG)) || !(st.pcg_ok > 0.0) ? -2 : 1;
    st.halvings = 0;
    st.accepted_round = -1;
    st.pad = 0;
    steps[p] = st;
  }
}

// trial = C + alpha_p d for the control points of searching patches.
template <typename T>
__global__ void k_ls_trial(int N, const int* __restrict__ cp_patch, const PatchStep* __restrict__ steps,
                           const T* __restrict__ C, const T* __restrict__ d, T* __restrict__ trial) {
  const int al = blockIdx.x * blockDim.x + threadIdx.x;
  if (al >= N) return;
  const PatchStep* st = steps + cp_patch[al];
  if (st->state != 1) return;
  const T a = (T)st->alpha;
#pragma unroll
  for (int c = 0; c < 3; ++c) trial[c * N + al] = C[c * N + al] + a * d[c * N + al];
}

// Accept / halve / fail per searching patch; counts the patches still searching.
__global__ void __launch_bounds__(SB) k_ls_accept(int P, PatchStep* __restrict__ steps, const double* __restrict__ E1,
                                                  int max_ls, int round, const int* __restrict__ status,
                                                  int* __restrict__ pending) {
  __shared__ double sm[SB / 32];
  const int flags = *(volatile const int*)status;
  double npend = 0.0;
  for (int p = threadIdx.x; p < P; p += SB) {
    PatchStep& st = steps[p];
    if (st.state != 1) continue;
    if (flags & (BSC_STATUS_TIMEOUT_FLAG | BSC_STATUS_NUMERIC_FLAG)) {
      st.state = -2;
      continue;
    }
    const double e1 = E1[p];
    st.E1 = e1;
    if (e1 <= st.E0) {
      st.state = 0;
      st.accepted_round = round;
    } else if (st.halvings >= max_ls) {
      st.state = -1;
      st.alpha = 0.0;
    } else {
      st.alpha *= 0.5;
      st.halvings += 1;
      npend += 1.0;
    }
  }
  const double tot = block_sum<SB>(npend, sm);
  if (threadIdx.x == 0) *pending = (int)tot;
}

// C = trial for the patches accepted in this round.
template <typename T>
__global__ void k_ls_commit(int N, const int* __restrict__ cp_patch, const PatchStep* __restrict__ steps, int round,
                            const T* __restrict__ trial, T* __restrict__ C) {
  const int al = blockIdx.x * blockDim.x + threadIdx.x;
  if (al >= N) return;
  const PatchStep* st = steps + cp_patch[al];
  if (st->state != 0 || st->accepted_round != round) return;
#pragma unroll
  for (int c = 0; c < 3; ++c) C[c * N + al] = trial[c * N + al];
}

}  // namespace

cudaError_t launch_step_begin(bsc_ctx* c, const void* d) {
  BSC_COUNT(c, 2);
  if (c->precision == BSC_FP64)
    k_step_items<double><<<c->n_red_items, SB, 0, c->stream>>>(c->N, c->n_red_items, c->red_items, c->pd, c->nneg,
                                                               (const double*)d, c->partials);
  else
    k_step_items<float><<<c->n_red_items, SB, 0, c->stream>>>(c->N, c->n_red_items, c->red_items, c->pd, c->nneg,
                                                              (const float*)d, c->partials);
  k_step_begin<<<c->P, SB, 0, c->stream>>>(c->n_red_items, c->red_off, c->partials, c->patch_E, c->pcg_out,
                                           c->project_default == BSC_PROJECT_SPAN,
                                           c->solver_cnn ? c->fcg_rec : nullptr, contact_bound_ptr(c), c->steps,
                                           c->dstatus);
  return cudaGetLastError();
}

cudaError_t launch_ls_round(bsc_ctx* c, const void* C, const void* Chat, const void* d, void* trial, void* Cout,
                            int round) {
  cudaError_t e;
  const int B = 256, G = (c->N + B - 1) / B;
  BSC_COUNT(c, 1);
  if (c->precision == BSC_FP64)
    k_ls_trial<double><<<G, B, 0, c->stream>>>(c->N, c->cp_patch, c->steps, (const double*)C, (const double*)d,
                                               (double*)trial);
  else
    k_ls_trial<float><<<G, B, 0, c->stream>>>(c->N, c->cp_patch, c->steps, (const float*)C, (const float*)d,
                                              (float*)trial);
  if ((e = cudaGetLastError()) != cudaSuccess) return e;
  if ((e = launch_span_eval(c, trial, 0, 0, c->steps)) != cudaSuccess) return e;
  if ((e = contact_add(c, trial, 0, 0, c->steps)) != cudaSuccess) return e;
  if ((e = launch_patch_energy(c, trial, Chat, c->patch_E + c->P, c->steps)) != cudaSuccess) return e;
  BSC_COUNT(c, 2);
  k_ls_accept<<<1, SB, 0, c->stream>>>(c->P, c->steps, c->patch_E + c->P, c->max_ls, round, c->dstatus, c->pending);
  if (c->precision == BSC_FP64)
    k_ls_commit<double><<<G, B, 0, c->stream>>>(c->N, c->cp_patch, c->steps, round, (const double*)trial,
                                                (double*)Cout);
  else
    k_ls_commit<float><<<G, B, 0, c->stream>>>(c->N, c->cp_patch, c->steps, round, (const float*)trial,
                                               (float*)Cout);
  return cudaGetLastError();
}

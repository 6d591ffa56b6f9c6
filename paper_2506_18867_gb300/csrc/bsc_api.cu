// C ABI of the sm_103a B-spline cloth FEM hot path (declared in include/bsc.h).
#include <stdarg.h>
#include <stdio.h>
#include <stdlib.h>
#include <string.h>

#include "bsc_internal.cuh"

int pcg_grid_size(int precision, int num_sms, int N);

namespace {

thread_local char g_create_err[512] = "";

bsc_status fail(bsc_ctx* c, bsc_status st, const char* fmt, ...) {
  char* buf = c ? c->err : g_create_err;
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(buf, 512, fmt, ap);
  va_end(ap);
  return st;
}

bsc_status cuda_fail(bsc_ctx* c, cudaError_t e, const char* where) {
  return fail(c, e == cudaErrorMemoryAllocation ? BSC_ERR_OOM : BSC_ERR_CUDA, "%s: %s", where,
              cudaGetErrorString(e));
}

#define CK(call, where)                                  \
  do {                                                   \
    cudaError_t e_ = (call);                             \
    if (e_ != cudaSuccess) return cuda_fail(c, e_, where); \
  } while (0)

bool aligned16(const void* p) { return ((uintptr_t)p & 15u) == 0; }

// Reads and clears the device status word (synchronises the stream).
bsc_status check_status(bsc_ctx* c, const char* where) {
  int st = 0;
  CK(cudaMemcpyAsync(&st, c->dstatus, sizeof(int), cudaMemcpyDeviceToHost, c->stream), where);
  CK(cudaStreamSynchronize(c->stream), where);
  if (st) {
    CK(cudaMemsetAsync(c->dstatus, 0, sizeof(int), c->stream), where);
    if (st & BSC_STATUS_TIMEOUT_FLAG) return fail(c, BSC_ERR_TIMEOUT, "%s: device wait timed out", where);
    return fail(c, BSC_ERR_NUMERIC, "%s: non-finite or singular value on the device (flags %d)", where, st);
  }
  return BSC_OK;
}

void free_ctx(bsc_ctx* c) {
  if (!c) return;
  void* ptrs[] = {c->mem_off, c->bd_off, c->tab_mem, c->tab_bd, c->pts_mem, c->pts_bd, c->rest, c->mass,
                  c->pinned, c->bucket_list, c->nneg, c->E_span, c->g_span, c->H_span, c->A_mem, c->K_int,
                  c->Dinv, c->partials, c->sync, c->dstatus, c->dscalars};
  for (void* p : ptrs)
    if (p) cudaFree(p);
  for (void* p : c->vec)
    if (p) cudaFree(p);
  for (void* p : c->proj_scratch)
    if (p) cudaFree(p);
  if (c->proj_work) cudaFree(c->proj_work);
  if (c->proj_span) cudaFree(c->proj_span);
  if (c->proj_kneg) cudaFree(c->proj_kneg);
  for (int i = 0; i < 2; ++i) {
    if (c->side[i]) cudaStreamDestroy(c->side[i]);
    if (c->join_ev[i]) cudaEventDestroy(c->join_ev[i]);
  }
  if (c->fork_ev) cudaEventDestroy(c->fork_ev);
  if (c->hscalars) cudaFreeHost(c->hscalars);
  if (c->profiling)
    for (cudaEvent_t ev : c->ev) cudaEventDestroy(ev);
  free(c);
}

void mark(bsc_ctx* c, int k) {
  if (c->profiling) cudaEventRecord(c->ev[k], c->stream);
}

bsc_status eval_path(bsc_ctx* c, const void* C, int want_grad, int want_hess, int project) {
  CK(launch_span_eval(c, C, want_grad, want_hess), "span evaluation");
  if (want_hess && project) CK(launch_project(c), "SPD projection");
  return BSC_OK;
}

}  // namespace

// Message of a failed context-free call, read back through bsc_last_error(NULL).
void bsc_set_thread_error(const char* msg) { snprintf(g_create_err, sizeof(g_create_err), "%s", msg); }

extern "C" {

const char* bsc_last_error(const bsc_ctx* c) { return c ? c->err : g_create_err; }

bsc_status bsc_create(const bsc_knot_grid* g, const double* rest_xy, const bsc_material* m,
                      const bsc_quadrature* q, const bsc_options* o, void* stream, bsc_ctx** out) {
  bsc_ctx* c = nullptr;
  if (!out) return fail(nullptr, BSC_ERR_INVALID_ARG, "bsc_create: out is NULL");
  *out = nullptr;
  if (!g || !rest_xy || !m || !o) return fail(nullptr, BSC_ERR_INVALID_ARG, "bsc_create: NULL argument");
  if (g->nu < 5 || g->nv < 5)
    return fail(nullptr, BSC_ERR_INVALID_ARG, "bsc_create: nu, nv must be >= 5 (got %d x %d)", g->nu, g->nv);
  if ((long long)g->nu * g->nv > (1ll << 26))
    return fail(nullptr, BSC_ERR_INVALID_ARG, "bsc_create: grid too large");
  for (int ax = 0; ax < 2; ++ax) {
    const double* kn = ax ? g->knots_v : g->knots_u;
    const int n = ax ? g->nv : g->nu;
    if (!kn) continue;
    for (int k = 0; k < n + 3; ++k) {
      int want = k - 2;
      want = want < 0 ? 0 : (want > n - 2 ? n - 2 : want);
      if (kn[k] != (double)want)
        return fail(nullptr, BSC_ERR_INVALID_ARG,
                    "bsc_create: knots must be the open uniform integer vector (knot %d of axis %d is %g)", k,
                    ax, kn[k]);
    }
  }
  const int mem_rule = q ? q->membrane : BSC_QUAD_REDUCED, bend_rule = q ? q->bending : BSC_QUAD_REDUCED;
  for (int r : {mem_rule, bend_rule})
    if (r != BSC_QUAD_REDUCED && r != BSC_QUAD_GAUSS2 && r != BSC_QUAD_GAUSS3)
      return fail(nullptr, BSC_ERR_INVALID_ARG, "bsc_create: unknown quadrature rule %d", r);
  if (o->precision != BSC_FP64 && o->precision != BSC_FP32)
    return fail(nullptr, BSC_ERR_INVALID_ARG, "bsc_create: unknown precision %d", o->precision);
  const double mats[5] = {m->mu_st1, m->mu_st2, m->mu_sh, m->mu_bd, m->rho_area};
  for (double v : mats)
    if (!(v >= 0.0) || !isfinite(v)) return fail(nullptr, BSC_ERR_INVALID_ARG, "bsc_create: material must be finite, >= 0");
  const int N = g->nu * g->nv;
  for (int k = 0; k < 2 * N; ++k)
    if (!isfinite(rest_xy[k])) return fail(nullptr, BSC_ERR_INVALID_ARG, "bsc_create: rest_xy has a non-finite value");
  if (o->n_pinned < 0 || (o->n_pinned > 0 && !o->pinned))
    return fail(nullptr, BSC_ERR_INVALID_ARG, "bsc_create: bad pinned list");
  for (int k = 0; k < o->n_pinned; ++k)
    if (o->pinned[k] < 0 || o->pinned[k] >= N)
      return fail(nullptr, BSC_ERR_INVALID_ARG, "bsc_create: pinned index %d out of range [0, %d)", o->pinned[k], N);
  if (!isfinite(o->dt) || !isfinite(o->gravity[0]) || !isfinite(o->gravity[1]) || !isfinite(o->gravity[2]))
    return fail(nullptr, BSC_ERR_INVALID_ARG, "bsc_create: dt and gravity must be finite");

  c = (bsc_ctx*)calloc(1, sizeof(bsc_ctx));
  if (!c) return fail(nullptr, BSC_ERR_OOM, "bsc_create: host allocation failed");
  c->nu = g->nu; c->nv = g->nv; c->Su = g->nu - 2; c->Sv = g->nv - 2; c->N = N; c->Nsp = c->Su * c->Sv;
  c->precision = o->precision;
  c->tsize = o->precision == BSC_FP64 ? sizeof(double) : sizeof(float);
  c->mu_st1 = m->mu_st1; c->mu_st2 = m->mu_st2; c->mu_sh = m->mu_sh; c->mu_bd = m->mu_bd; c->rho = m->rho_area;
  c->mem_rule = mem_rule; c->bend_rule = bend_rule;
  c->dt = o->dt;
  for (int k = 0; k < 3; ++k) c->gravity[k] = o->gravity[k];
  c->project_default = o->project;
  c->pcg_tol = o->pcg_rel_tol > 0.0 ? o->pcg_rel_tol : 1e-8;
  c->pcg_max_iter = o->pcg_max_iter > 0 ? o->pcg_max_iter : 10000;
  c->max_ls = o->max_line_search > 0 ? o->max_line_search : 30;
  c->stream = (cudaStream_t)stream;

  bsc_status st = BSC_OK;
  cudaError_t e = cudaGetDevice(&c->device);
  if (e == cudaSuccess) e = cudaDeviceGetAttribute(&c->num_sms, cudaDevAttrMultiProcessorCount, c->device);
  int coop = 0;
  if (e == cudaSuccess) e = cudaDeviceGetAttribute(&coop, cudaDevAttrCooperativeLaunch, c->device);
  if (e != cudaSuccess) {
    st = cuda_fail(nullptr, e, "bsc_create: device query");
    free_ctx(c);
    return st;
  }
  if (!coop) {
    free_ctx(c);
    return fail(nullptr, BSC_ERR_CUDA, "bsc_create: device lacks cooperative launch");
  }
  const size_t ts = c->tsize;
  c->red_grid = 2 * c->num_sms;
  c->pcg_grid = pcg_grid_size(c->precision, c->num_sms, N);
  const int max_grid = c->red_grid > c->pcg_grid ? c->red_grid : c->pcg_grid;
#define ALLOC(ptr, bytes)                                     \
  do {                                                        \
    e = cudaMalloc((void**)&(ptr), (bytes));                  \
    if (e != cudaSuccess) {                                   \
      st = cuda_fail(nullptr, e, "bsc_create: cudaMalloc " #ptr); \
      free_ctx(c);                                            \
      return st;                                              \
    }                                                         \
  } while (0)
  ALLOC(c->rest, sizeof(double) * 2 * (size_t)N);
  ALLOC(c->mass, sizeof(double) * (size_t)N);
  ALLOC(c->pinned, (size_t)N);
  ALLOC(c->nneg, sizeof(int) * (size_t)c->Nsp);
  ALLOC(c->E_span, sizeof(double) * (size_t)c->Nsp);
  ALLOC(c->g_span, ts * 27 * (size_t)c->Nsp);
  ALLOC(c->H_span, ts * H27 * (size_t)c->Nsp);
  ALLOC(c->K_int, ts * 225 * (size_t)N);
  ALLOC(c->Dinv, ts * 9 * (size_t)N);
  for (int k = 0; k < 8; ++k) ALLOC(c->vec[k], ts * 3 * (size_t)N);
  ALLOC(c->partials, sizeof(double) * 4 * (size_t)max_grid);
  ALLOC(c->sync, sizeof(unsigned int) * 4);
  ALLOC(c->dstatus, sizeof(int) * 4);
  ALLOC(c->dscalars, sizeof(double) * 16);
#undef ALLOC
  e = cudaMallocHost((void**)&c->hscalars, sizeof(double) * 16);
  if (e != cudaSuccess) {
    st = cuda_fail(nullptr, e, "bsc_create: cudaMallocHost");
    free_ctx(c);
    return st;
  }
  // rest coordinates as two planes; pinned mask
  double* rp = (double*)malloc(sizeof(double) * 2 * (size_t)N);
  uint8_t* pm = (uint8_t*)calloc((size_t)N, 1);
  for (int k = 0; k < N; ++k) {
    rp[k] = rest_xy[2 * k];
    rp[N + k] = rest_xy[2 * k + 1];
  }
  for (int k = 0; k < o->n_pinned; ++k) pm[o->pinned[k]] = 1;
  e = cudaMemcpy(c->rest, rp, sizeof(double) * 2 * (size_t)N, cudaMemcpyHostToDevice);
  if (e == cudaSuccess) e = cudaMemcpy(c->pinned, pm, (size_t)N, cudaMemcpyHostToDevice);
  free(rp);
  free(pm);
  if (e == cudaSuccess) e = cudaMemset(c->sync, 0, sizeof(unsigned int) * 4);
  if (e == cudaSuccess) e = cudaMemset(c->dstatus, 0, sizeof(int) * 4);
  if (e == cudaSuccess) e = cudaMemset(c->nneg, 0, sizeof(int) * (size_t)c->Nsp);
  if (e == cudaSuccess) e = launch_build_tables(c);
  if (e == cudaSuccess) e = setup_projection(c);
  if (e != cudaSuccess) {
    st = cuda_fail(nullptr, e, "bsc_create: building quadrature tables");
    free_ctx(c);
    return st;
  }
  st = check_status(c, "bsc_create");
  if (st != BSC_OK) {
    snprintf(g_create_err, sizeof(g_create_err), "%s (rest map singular?)", c->err);
    free_ctx(c);
    return st;
  }
  c->K_last = nullptr;
  *out = c;
  return BSC_OK;
}

void bsc_destroy(bsc_ctx* c) {
  if (!c) return;
  cudaStreamSynchronize(c->stream);
  free_ctx(c);
}

bsc_status bsc_set_stream(bsc_ctx* c, void* stream) {
  if (!c) return BSC_ERR_INVALID_ARG;
  c->stream = (cudaStream_t)stream;
  return BSC_OK;
}

bsc_status bsc_sizes(const bsc_ctx* c, int* n_cp, int* n_spans, int* n_mem, int* n_bend) {
  if (!c) return BSC_ERR_INVALID_ARG;
  if (n_cp) *n_cp = c->N;
  if (n_spans) *n_spans = c->Nsp;
  if (n_mem) *n_mem = c->Nmem;
  if (n_bend) *n_bend = c->Nbd;
  return BSC_OK;
}

bsc_status bsc_energy(bsc_ctx* c, const void* C, const void* Chat, double* E_out) {
  if (!c) return BSC_ERR_INVALID_ARG;
  if (!C || !E_out || (c->dt > 0.0 && !Chat)) return fail(c, BSC_ERR_INVALID_ARG, "bsc_energy: NULL argument");
  if (!aligned16(C) || (Chat && !aligned16(Chat))) return fail(c, BSC_ERR_INVALID_ARG, "bsc_energy: pointers must be 16-byte aligned");
  CK(launch_span_eval(c, C, 0, 0), "bsc_energy");
  CK(launch_energy(c, C, Chat, c->dscalars), "bsc_energy");
  CK(cudaMemcpyAsync(c->hscalars, c->dscalars, sizeof(double), cudaMemcpyDeviceToHost, c->stream), "bsc_energy");
  bsc_status st = check_status(c, "bsc_energy");
  if (st != BSC_OK) return st;
  *E_out = c->hscalars[0];
  return BSC_OK;
}

bsc_status bsc_gradient(bsc_ctx* c, const void* C, const void* Chat, void* g) {
  if (!c) return BSC_ERR_INVALID_ARG;
  if (!C || !g || (c->dt > 0.0 && !Chat)) return fail(c, BSC_ERR_INVALID_ARG, "bsc_gradient: NULL argument");
  if (!aligned16(C) || !aligned16(g)) return fail(c, BSC_ERR_INVALID_ARG, "bsc_gradient: pointers must be 16-byte aligned");
  bsc_status st = eval_path(c, C, 1, 0, 0);
  if (st != BSC_OK) return st;
  CK(launch_gradient(c, C, Chat, g), "bsc_gradient");
  return BSC_OK;
}

bsc_status bsc_assemble_hessian(bsc_ctx* c, const void* C, int project, void* K) {
  if (!c) return BSC_ERR_INVALID_ARG;
  if (!C) return fail(c, BSC_ERR_INVALID_ARG, "bsc_assemble_hessian: C is NULL");
  if (!aligned16(C) || (K && !aligned16(K))) return fail(c, BSC_ERR_INVALID_ARG, "bsc_assemble_hessian: pointers must be 16-byte aligned");
  void* Kd = K ? K : c->K_int;
  bsc_status st = eval_path(c, C, 0, 1, project);
  if (st != BSC_OK) return st;
  CK(launch_assemble(c, Kd), "bsc_assemble_hessian");
  c->K_last = Kd;
  return BSC_OK;
}

bsc_status bsc_spmv(bsc_ctx* c, const void* K, const void* x, void* y) {
  if (!c) return BSC_ERR_INVALID_ARG;
  const void* Kd = K ? K : c->K_last;
  if (!Kd || !x || !y) return fail(c, BSC_ERR_INVALID_ARG, "bsc_spmv: no matrix or NULL vector");
  if (x == y) return fail(c, BSC_ERR_INVALID_ARG, "bsc_spmv: x and y must not alias");
  CK(launch_spmv(c, Kd, x, y), "bsc_spmv");
  return BSC_OK;
}

bsc_status bsc_solve(bsc_ctx* c, const void* K, const void* b, void* x, double tol, int maxit, int* iters,
                     double* rel_res) {
  if (!c) return BSC_ERR_INVALID_ARG;
  const void* Kd = K ? K : c->K_last;
  if (!Kd || !b || !x) return fail(c, BSC_ERR_INVALID_ARG, "bsc_solve: no matrix or NULL vector");
  if (!(tol > 0.0)) tol = c->pcg_tol;
  if (maxit <= 0) maxit = c->pcg_max_iter;
  CK(cudaMemsetAsync(c->sync, 0, sizeof(unsigned int) * 4, c->stream), "bsc_solve");
  CK(launch_pcg(c, Kd, b, x, tol, maxit), "bsc_solve");
  CK(cudaMemcpyAsync(c->hscalars + 8, c->dscalars + 8, 3 * sizeof(double), cudaMemcpyDeviceToHost, c->stream),
     "bsc_solve");
  bsc_status st = check_status(c, "bsc_solve");
  if (st != BSC_OK) return st;
  const int it = (int)c->hscalars[8];
  if (iters) *iters = it;
  if (rel_res) *rel_res = c->hscalars[9];
  if (!(c->hscalars[9] <= tol)) return fail(c, BSC_ERR_NOT_CONVERGED, "bsc_solve: %d iterations, rel. residual %g", it, c->hscalars[9]);
  return BSC_OK;
}

bsc_status bsc_newton_step(bsc_ctx* c, void* C, const void* Chat, bsc_newton_report* rep) {
  if (!c) return BSC_ERR_INVALID_ARG;
  bsc_newton_report r;
  memset(&r, 0, sizeof(r));
  if (!C || (c->dt > 0.0 && !Chat)) return fail(c, BSC_ERR_INVALID_ARG, "bsc_newton_step: NULL argument");
  if (!aligned16(C) || (Chat && !aligned16(Chat))) return fail(c, BSC_ERR_INVALID_ARG, "bsc_newton_step: pointers must be 16-byte aligned");
  void *d = c->vec[0], *g = c->vec[5], *trial = c->vec[6];
  mark(c, 0);
  CK(launch_span_eval(c, C, 1, 1), "newton: span evaluation");
  mark(c, 1);
  if (c->project_default) {
    CK(launch_project(c), "newton: SPD projection");
    CK(launch_count_projected(c, c->dscalars + 3), "newton: SPD projection");
  } else {
    CK(cudaMemsetAsync(c->dscalars + 3, 0, sizeof(double), c->stream), "newton");
  }
  mark(c, 2);
  bsc_status st = BSC_OK;
  {
    CK(launch_energy(c, C, Chat, c->dscalars + 0), "newton: energy");
    CK(launch_gradient(c, C, Chat, g), "newton: gradient");
    CK(launch_assemble(c, c->K_int), "newton: assembly");
    c->K_last = c->K_int;
    mark(c, 3);
    // right-hand side -g (into the spare vector), then PCG
    CK(launch_axpy_trial(c, g, g, -2.0, c->vec[7]), "newton: rhs");
    int iters = 0;
    double rr = 0.0;
    st = bsc_solve(c, c->K_int, c->vec[7], d, c->pcg_tol, c->pcg_max_iter, &iters, &rr);
    r.pcg_iters = iters;
    r.pcg_rel_res = rr;
    mark(c, 4);
  }
  if (st == BSC_OK || st == BSC_ERR_NOT_CONVERGED) {
    bsc_status solve_st = st;
    CK(launch_absmax(c, d, c->dscalars + 1), "newton: |d|");
    CK(cudaMemcpyAsync(c->hscalars, c->dscalars, 4 * sizeof(double), cudaMemcpyDeviceToHost, c->stream), "newton");
    st = check_status(c, "bsc_newton_step");
    if (st == BSC_OK) {
      r.E0 = c->hscalars[0];
      r.dir_inf = c->hscalars[1];
      r.spans_projected = (int)c->hscalars[3];
      double alpha = 1.0;
      int h = 0;
      for (;;) {
        CK(launch_axpy_trial(c, C, d, alpha, trial), "newton: trial");
        CK(launch_span_eval(c, trial, 0, 0), "newton: trial energy");
        CK(launch_energy(c, trial, Chat, c->dscalars + 2), "newton: trial energy");
        CK(cudaMemcpyAsync(c->hscalars + 2, c->dscalars + 2, sizeof(double), cudaMemcpyDeviceToHost, c->stream),
           "newton");
        st = check_status(c, "newton: line search");
        if (st != BSC_OK) break;
        const double E1 = c->hscalars[2];
        if (E1 <= r.E0) {
          CK(launch_copy_vec(c, trial, C), "newton: commit");
          r.E1 = E1;
          r.alpha = alpha;
          r.ls_halvings = h;
          break;
        }
        if (h >= c->max_ls) {
          r.E1 = E1;
          r.alpha = 0.0;
          r.ls_halvings = h;
          st = fail(c, BSC_ERR_LINESEARCH, "bsc_newton_step: no decrease after %d halvings (E0 %.17g, E1 %.17g)",
                    h, r.E0, E1);
          break;
        }
        alpha *= 0.5;
        ++h;
      }
      if (st == BSC_OK && solve_st != BSC_OK) st = solve_st;
    }
  }
  mark(c, 5);
  r.status = st;
  if (rep) *rep = r;
  if (st == BSC_OK) CK(cudaStreamSynchronize(c->stream), "bsc_newton_step");
  return st;
}

bsc_status bsc_span_terms(bsc_ctx* c, const void* C, int project, double* E_span, void* g_span, void* H_span) {
  if (!c || !C) return BSC_ERR_INVALID_ARG;
  bsc_status st = eval_path(c, C, 1, 1, project);
  if (st != BSC_OK) return st;
  if (E_span) CK(cudaMemcpyAsync(E_span, c->E_span, sizeof(double) * c->Nsp, cudaMemcpyDeviceToDevice, c->stream), "bsc_span_terms");
  CK(launch_export_span_terms(c, g_span, H_span), "bsc_span_terms");
  return check_status(c, "bsc_span_terms");
}

bsc_status bsc_quadrature_tables(bsc_ctx* c, int which, double* out, int cap, int* count) {
  if (!c || (which != 0 && which != 1)) return BSC_ERR_INVALID_ARG;
  const int n = which ? c->Nbd : c->Nmem;
  if (count) *count = n;
  if (!out) return BSC_OK;
  const int m = cap < n ? cap : n;
  const int ncol = which ? TABB : TABM;
  double* pts = (double*)malloc(sizeof(double) * 5 * (size_t)n);
  unsigned char* tab = (unsigned char*)malloc(c->tsize * ncol * (size_t)n);
  cudaError_t e = cudaMemcpyAsync(pts, which ? c->pts_bd : c->pts_mem, sizeof(double) * 5 * (size_t)n,
                                  cudaMemcpyDeviceToHost, c->stream);
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(tab, which ? c->tab_bd : c->tab_mem, c->tsize * ncol * (size_t)n, cudaMemcpyDeviceToHost,
                        c->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
  if (e != cudaSuccess) {
    free(pts);
    free(tab);
    return cuda_fail(c, e, "bsc_quadrature_tables");
  }
  for (int k = 0; k < m; ++k) {
    double* r = out + 25 * (size_t)k;
    for (int j = 0; j < 25; ++j) r[j] = 0.0;
    for (int j = 0; j < 5; ++j) r[j] = pts[(size_t)j * n + k];
    for (int j = 0; j < ncol; ++j) {
      const size_t idx = (size_t)j * n + k;
      r[5 + j] = c->precision == BSC_FP64 ? ((double*)tab)[idx] : (double)((float*)tab)[idx];
    }
  }
  free(pts);
  free(tab);
  return BSC_OK;
}

bsc_status bsc_set_profiling(bsc_ctx* c, int on) {
  if (!c) return BSC_ERR_INVALID_ARG;
  if (on && !c->profiling) {
    for (int k = 0; k < 6; ++k) CK(cudaEventCreate(&c->ev[k]), "bsc_set_profiling");
    c->profiling = 1;
  } else if (!on && c->profiling) {
    CK(cudaStreamSynchronize(c->stream), "bsc_set_profiling");
    for (int k = 0; k < 6; ++k) cudaEventDestroy(c->ev[k]);
    c->profiling = 0;
  }
  return BSC_OK;
}

bsc_status bsc_phase_times(bsc_ctx* c, double* ms) {
  if (!c || !ms) return BSC_ERR_INVALID_ARG;
  if (!c->profiling) return fail(c, BSC_ERR_INVALID_ARG, "bsc_phase_times: profiling is off");
  CK(cudaEventSynchronize(c->ev[5]), "bsc_phase_times");
  float t;
  for (int k = 0; k < 5; ++k) {
    CK(cudaEventElapsedTime(&t, c->ev[k], c->ev[k + 1]), "bsc_phase_times");
    ms[k] = t;
  }
  CK(cudaEventElapsedTime(&t, c->ev[0], c->ev[5]), "bsc_phase_times");
  ms[5] = t;
  return BSC_OK;
}

bsc_status bsc_launch_count(const bsc_ctx* c, unsigned long long* n) {
  if (!c || !n) return BSC_ERR_INVALID_ARG;
  *n = c->launches;
  return BSC_OK;
}

bsc_status bsc_projection_stats(bsc_ctx* c, int* nneg, int* nred) {
  if (!c) return BSC_ERR_INVALID_ARG;
  if (nneg) {
    CK(cudaMemcpyAsync(nneg, c->nneg, sizeof(int) * c->Nsp, cudaMemcpyDeviceToHost, c->stream), "bsc_projection_stats");
    CK(cudaStreamSynchronize(c->stream), "bsc_projection_stats");
  }
  if (nred) {
    int* hl = (int*)malloc(sizeof(int) * c->Nsp);
    cudaError_t e = cudaMemcpy(hl, c->bucket_list, sizeof(int) * c->Nsp, cudaMemcpyDeviceToHost);
    if (e != cudaSuccess) { free(hl); return cuda_fail(c, e, "bsc_projection_stats"); }
    const int sizes[3] = {15, 24, 24};
    for (int b = 0; b < 3; ++b)
      for (int k = c->bucket_off[b]; k < c->bucket_off[b + 1]; ++k) nred[hl[k]] = sizes[b];
    free(hl);
  }
  return BSC_OK;
}

bsc_status bsc_lumped_mass(bsc_ctx* c, double* m_out) {
  if (!c || !m_out) return BSC_ERR_INVALID_ARG;
  CK(cudaMemcpyAsync(m_out, c->mass, sizeof(double) * c->N, cudaMemcpyDeviceToHost, c->stream), "bsc_lumped_mass");
  CK(cudaStreamSynchronize(c->stream), "bsc_lumped_mass");
  return BSC_OK;
}

}  // extern "C"

// Contact (Sec. 4.3): the incremental-potential-contact log barrier between a
// triangle mesh embedded in the B-spline surface and a static obstacle
// triangle mesh, chained onto the control points.
//
// Contact mesh: mu x mv vertices at fixed parametric points u_i = S_u i /
// (mu - 1), v_j = S_v j / (mv - 1); vertex k = j mu + i lies in span
// (clamp(floor u), clamp(floor v)) and moves with its nine control points,
// x_k = sum_l N_l(u, v) C_l (Eq. trig mesh node from control points); its
// weight A_k is a third of the rest areas of its triangles (cells split along
// alternating diagonals).
//
// Potential: B(C) = kappa sum_k A_k sum_pairs beta(d / dhat), beta(x) =
// -(x - 1)^2 ln x on (0, 1), over the pairs (vertex, obstacle triangle) with
// distance d < dhat; a pair whose closest point lies on an edge or a corner
// of the triangle counts only for the lowest-index triangle holding that
// feature (each point-edge and point-corner distance enters once).  Per pair
// the gradient w.r.t. the vertex is kappa A beta'(x) / dhat u and the PSD
// projection of its Hessian kappa A beta''(x) / dhat^2 u u^T, u = (x - q) / d
// (the rest of the Hessian, beta'(x) / dhat grad^2 d, is negative
// semidefinite and orthogonal to u).  The chain rule (Eq. gradient and
// hessian of contact barrier) adds N_l N_m H_k to the span Hessian of the
// vertex's span and N_l g_k to its gradient, after the elastic projection, so
// the gather assembly builds K = elastic + contact in its fixed order: the
// deterministic per-block conversion of Alg. 1 without hash maps, since a
// vertex touches only the 3 x 3 control points of its span.
//
// Candidates come from a spatial hash of the obstacle (static, built on the
// host): cubic cells of size h, every triangle listed once in the bucket of
// every cell its box (grown by dhat) overlaps.  A vertex reads the bucket of
// its cell.  The line search starts at the conservative step bound: along
// x + a dx the distance to a convex triangle is convex in a, so it stays
// above d + a (u . dx) and above 0.1 d for a <= 0.9 d / (-u . dx); the
// candidates are those listed in the cells the swept box overlaps, the
// motion limited to two cells per step.  All geometry is FP64.
#include <math.h>
#include <stdio.h>
#include <stdlib.h>
#include <string.h>

#include <algorithm>
#include <vector>

#include "bsc_internal.cuh"

struct bsc_contact {
  int mu, mv, nvert;
  double dhat, kappa, cell;
  int nvo, nto, ht;          // obstacle vertices, triangles, hash-table size (power of two)
  // contact mesh (device)
  int* vspan;                // [nvert] context-wide span of each vertex
  double* vw;                // [9][nvert] embedding weights N_l
  double* varea;             // [nvert] A_k
  int* span_off;             // [Nsp + 1] vertices of each span (CSR)
  int* span_vert;            // [nvert]
  // obstacle (device)
  double* ov;                // [3][nvo]
  int* ot;                   // [3][nto]
  unsigned char* own;        // [nto] bits 0..2 edges (01, 02, 12), bits 3..5 corners 0..2 owned
  int* bucket_off;           // [ht + 1]
  int* bucket_tri;           // [entries]
  // per-vertex results of the last evaluation
  double* cE;                // [nvert] sum of beta over the vertex's pairs (times kappa A)
  double* cg;                // [3][nvert] gradient w.r.t. the vertex
  double* cH;                // [6][nvert] projected Hessian (xx xy xz yy yz zz)
  int* npairs;               // [1] pairs counted by the last evaluation
  double* ccd;               // [1] step bound of the last direction
};

namespace {

constexpr double FEATURE_TOL = 1e-10;  // barycentric coordinate counted as zero (feature classification)

__host__ __device__ __forceinline__ unsigned int cell_hash(int cx, int cy, int cz, int ht) {
  const unsigned int h = ((unsigned int)cx * 73856093u) ^ ((unsigned int)cy * 19349663u) ^ ((unsigned int)cz * 83492791u);
  return h & (unsigned int)(ht - 1);
}

__host__ __device__ __forceinline__ int cell_of(double x, double cell) { return (int)floor(x / cell); }

struct V3 {
  double x, y, z;
};
__device__ __forceinline__ V3 sub(V3 a, V3 b) { return V3{a.x - b.x, a.y - b.y, a.z - b.z}; }
__device__ __forceinline__ V3 add(V3 a, V3 b) { return V3{a.x + b.x, a.y + b.y, a.z + b.z}; }
__device__ __forceinline__ V3 scl(double s, V3 a) { return V3{s * a.x, s * a.y, s * a.z}; }
__device__ __forceinline__ double dot(V3 a, V3 b) { return a.x * b.x + a.y * b.y + a.z * b.z; }

// Closest point of triangle (a, b, c) to p, from the triangle's seven
// Voronoi regions (barycentric sign tests).
__device__ V3 closest_on_triangle(V3 p, V3 a, V3 b, V3 c) {
  const V3 ab = sub(b, a), ac = sub(c, a), ap = sub(p, a);
  const double d1 = dot(ab, ap), d2 = dot(ac, ap);
  if (d1 <= 0.0 && d2 <= 0.0) return a;
  const V3 bp = sub(p, b);
  const double d3 = dot(ab, bp), d4 = dot(ac, bp);
  if (d3 >= 0.0 && d4 <= d3) return b;
  const double vc = d1 * d4 - d3 * d2;
  if (vc <= 0.0 && d1 >= 0.0 && d3 <= 0.0) return add(a, scl(d1 / (d1 - d3), ab));
  const V3 cp = sub(p, c);
  const double d5 = dot(ab, cp), d6 = dot(ac, cp);
  if (d6 >= 0.0 && d5 <= d6) return c;
  const double vb = d5 * d2 - d1 * d6;
  if (vb <= 0.0 && d2 >= 0.0 && d6 <= 0.0) return add(a, scl(d2 / (d2 - d6), ac));
  const double va = d3 * d6 - d5 * d4;
  if (va <= 0.0 && (d4 - d3) >= 0.0 && (d5 - d6) >= 0.0) {
    const double w = (d4 - d3) / ((d4 - d3) + (d5 - d6));
    return add(b, scl(w, sub(c, b)));
  }
  const double den = 1.0 / (va + vb + vc);
  return add(a, add(scl(vb * den, ab), scl(vc * den, ac)));
}

// Whether the pair (p, triangle t) counts: always for a closest point inside
// the triangle; for one on an edge or at a corner (barycentric coordinates
// of q at most FEATURE_TOL counted as zero) only if t owns that feature.
__device__ bool pair_counts(V3 q, V3 a, V3 b, V3 c, unsigned char own) {
  const V3 ab = sub(b, a), ac = sub(c, a), aq = sub(q, a);
  const double g00 = dot(ab, ab), g01 = dot(ab, ac), g11 = dot(ac, ac), r0 = dot(ab, aq), r1 = dot(ac, aq);
  const double det = g00 * g11 - g01 * g01;
  const double l1 = (g11 * r0 - g01 * r1) / det, l2 = (g00 * r1 - g01 * r0) / det, l0 = 1.0 - l1 - l2;
  const int nz = (l0 > FEATURE_TOL ? 1 : 0) | (l1 > FEATURE_TOL ? 2 : 0) | (l2 > FEATURE_TOL ? 4 : 0);
  switch (nz) {
    case 7: return true;                 // interior
    case 3: return (own & 1) != 0;       // edge 0-1
    case 5: return (own & 2) != 0;       // edge 0-2
    case 6: return (own & 4) != 0;       // edge 1-2
    case 1: return (own & 8) != 0;       // corner 0
    case 2: return (own & 16) != 0;      // corner 1
    case 4: return (own & 32) != 0;      // corner 2
    default: {                           // all coordinates tiny (degenerate): the largest corner
      const int k = (l0 >= l1 && l0 >= l2) ? 0 : (l1 >= l2 ? 1 : 2);
      return (own & (8 << k)) != 0;
    }
  }
}

// beta(x) = -(x - 1)^2 ln x and its first two derivatives, 0 < x < 1.
__device__ __forceinline__ void barrier3(double x, double* b0, double* b1, double* b2) {
  const double lx = log(x), xm = x - 1.0;
  *b0 = -xm * xm * lx;
  *b1 = -2.0 * xm * lx - xm * xm / x;
  *b2 = -2.0 * lx - 4.0 * xm / x + xm * xm / (x * x);
}

struct CView {
  const int* vspan;
  const double* vw;
  int nvert, Su, nu, cp0;
};

// World position of contact vertex k from the control points C (3 planes of N).
template <typename T>
__device__ __forceinline__ V3 vertex_position(const CView& v, int k, int sp0, const T* __restrict__ C, int N) {
  const int s = v.vspan[k] - sp0, a = s % v.Su, b = s / v.Su;
  V3 x{0.0, 0.0, 0.0};
#pragma unroll
  for (int l = 0; l < 9; ++l) {
    const int al = v.cp0 + (b + l / 3) * v.nu + a + l % 3;
    const double w = v.vw[(size_t)l * v.nvert + k];
    x.x += w * (double)C[al];
    x.y += w * (double)C[N + al];
    x.z += w * (double)C[2 * (size_t)N + al];
  }
  return x;
}

struct Obs {
  const double* ov;
  const int* ot;
  const unsigned char* own;
  const int* boff;
  const int* btri;
  int nvo, nto, ht;
  double cell;
  __device__ V3 vert(int i) const { return V3{ov[i], ov[nvo + i], ov[2 * nvo + i]}; }
  __device__ void tri(int t, V3* a, V3* b, V3* c) const {
    *a = vert(ot[t]);
    *b = vert(ot[nto + t]);
    *c = vert(ot[2 * nto + t]);
  }
};

}  // namespace

namespace {

// Values of the three quadratic B-splines that are non-zero on span a of the
// open uniform knot vector xi_k = clamp(k - 2, 0, S), at parameter t
// (Cox-de Boor, 0/0 := 0).
__device__ void bspline_values(double t, int a, int S, double N[3]) {
  auto xi = [S](int k) { return (double)min(max(k - 2, 0), S); };
  auto div = [](double p, double q) { return q == 0.0 ? 0.0 : p / q; };
  const double x1 = xi(a + 1), x2 = xi(a + 2), x3 = xi(a + 3), x4 = xi(a + 4);
  const double n1 = div(x3 - t, x3 - x2), n2 = div(t - x2, x3 - x2);  // degree 1, functions a+1, a+2
  N[0] = div(x3 - t, x3 - x1) * n1;
  N[1] = div(t - x1, x3 - x1) * n1 + div(x4 - t, x4 - x2) * n2;
  N[2] = div(t - x2, x4 - x2) * n2;
}

// Contact mesh vertex k: its span, its nine weights and its rest position.
__global__ void k_contact_setup(int mu, int mv, int nu, int nv, int sp0, int cp0, int N, const double* __restrict__ rest,
                                int* __restrict__ vspan, double* __restrict__ vw, double* __restrict__ xrest) {
  const int k = blockIdx.x * blockDim.x + threadIdx.x, nvert = mu * mv;
  if (k >= nvert) return;
  const int Su = nu - 2, Sv = nv - 2, i = k % mu, j = k / mu;
  const double u = (double)Su * i / (mu - 1), v = (double)Sv * j / (mv - 1);
  const int a = min(max((int)floor(u), 0), Su - 1), b = min(max((int)floor(v), 0), Sv - 1);
  double Nu[3], Nv[3];
  bspline_values(u, a, Su, Nu);
  bspline_values(v, b, Sv, Nv);
  vspan[k] = sp0 + b * Su + a;
  double X = 0.0, Y = 0.0;
  for (int l = 0; l < 9; ++l) {
    const double w = Nu[l % 3] * Nv[l / 3];
    vw[(size_t)l * nvert + k] = w;
    const int al = cp0 + (b + l / 3) * nu + a + l % 3;
    X += w * rest[al];
    Y += w * rest[N + al];
  }
  xrest[k] = X;
  xrest[nvert + k] = Y;
}

// Per contact vertex: the barrier summed over its counted pairs, its
// gradient and its projected Hessian w.r.t. the vertex, times kappa A_k.
template <typename T>
__global__ void __launch_bounds__(128) k_contact_eval(CView cv, Obs ob, const double* __restrict__ varea, int sp0,
                                                      const T* __restrict__ C, int N, double dhat, double kappa,
                                                      const PatchStep* __restrict__ gate, double* __restrict__ cE,
                                                      double* __restrict__ cg, double* __restrict__ cH,
                                                      int* __restrict__ npairs, int* __restrict__ status) {
  const int k = blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= cv.nvert) return;
  if (gate && gate[0].state != 1) return;
  const V3 x = vertex_position<T>(cv, k, sp0, C, N);
  const unsigned int bk = cell_hash(cell_of(x.x, ob.cell), cell_of(x.y, ob.cell), cell_of(x.z, ob.cell), ob.ht);
  double e = 0.0, g[3] = {0.0, 0.0, 0.0}, H[6] = {0.0, 0.0, 0.0, 0.0, 0.0, 0.0};
  int pairs = 0;
  const double ih = 1.0 / dhat;
  for (int it = ob.boff[bk]; it < ob.boff[bk + 1]; ++it) {
    const int t = ob.btri[it];
    V3 a, b, c;
    ob.tri(t, &a, &b, &c);
    const V3 q = closest_on_triangle(x, a, b, c);
    const V3 df = sub(x, q);
    const double d = sqrt(dot(df, df));
    if (!(d < dhat)) continue;
    if (!pair_counts(q, a, b, c, ob.own[t])) continue;
    if (!(d > 0.0)) {
      atomicOr(status, BSC_STATUS_NUMERIC_FLAG);
      continue;
    }
    double b0, b1, b2;
    barrier3(d * ih, &b0, &b1, &b2);
    const double u[3] = {df.x / d, df.y / d, df.z / d};
    const double gc = b1 * ih, hc = b2 * ih * ih;
    e += b0;
    for (int r = 0; r < 3; ++r) g[r] += gc * u[r];
    H[0] += hc * u[0] * u[0]; H[1] += hc * u[0] * u[1]; H[2] += hc * u[0] * u[2];
    H[3] += hc * u[1] * u[1]; H[4] += hc * u[1] * u[2]; H[5] += hc * u[2] * u[2];
    ++pairs;
  }
  const double w = kappa * varea[k];
  cE[k] = w * e;
  for (int r = 0; r < 3; ++r) cg[(size_t)r * cv.nvert + k] = w * g[r];
  for (int r = 0; r < 6; ++r) cH[(size_t)r * cv.nvert + k] = w * H[r];
  if (pairs) atomicAdd(npairs, pairs);
}

// Per span: the contact terms of its vertices (fixed order) added to its
// energy, and with add_g / add_h to its 27 gradient entries and its packed
// 27 x 27 Hessian: d/dC_l = N_l g_k, d2/dC_l dC_m = N_l N_m H_k.
template <typename T>
__global__ void __launch_bounds__(128) k_contact_span(int Nsp, int nvert, const int* __restrict__ span_off,
                                                      const int* __restrict__ span_vert, const double* __restrict__ vw,
                                                      const double* __restrict__ cE, const double* __restrict__ cg,
                                                      const double* __restrict__ cH, int add_g, int add_h,
                                                      const PatchStep* __restrict__ gate, double* __restrict__ E_span,
                                                      T* __restrict__ g_span, T* __restrict__ H_span) {
  const int s = blockIdx.x * blockDim.x + threadIdx.x;
  if (s >= Nsp) return;
  if (gate && gate[0].state != 1) return;
  const int v0 = span_off[s], v1 = span_off[s + 1];
  double e = 0.0;
  bool any = false;
  for (int i = v0; i < v1; ++i) {
    const int k = span_vert[i];
    e += cE[k];
    any = any || cE[k] != 0.0 || cg[k] != 0.0 || cg[nvert + k] != 0.0 || cg[2 * (size_t)nvert + k] != 0.0;
  }
  if (!any) return;
  E_span[s] += e;
  if (add_g)
    for (int l = 0; l < 9; ++l)
      for (int c = 0; c < 3; ++c) {
        double acc = 0.0;
        for (int i = v0; i < v1; ++i) {
          const int k = span_vert[i];
          acc += vw[(size_t)l * nvert + k] * cg[(size_t)c * nvert + k];
        }
        g_span[(size_t)(3 * l + c) * Nsp + s] += (T)acc;
      }
  if (add_h) {
    const int hi[3][3] = {{0, 1, 2}, {1, 3, 4}, {2, 4, 5}};
    for (int l = 0; l < 9; ++l)
      for (int m = l; m < 9; ++m)
        for (int c = 0; c < 3; ++c)
          for (int d = (m == l ? c : 0); d < 3; ++d) {
            double acc = 0.0;
            for (int i = v0; i < v1; ++i) {
              const int k = span_vert[i];
              acc += vw[(size_t)l * nvert + k] * vw[(size_t)m * nvert + k] * cH[(size_t)hi[c][d] * nvert + k];
            }
            H_span[(size_t)upk(3 * l + c, 3 * m + d, 27) * Nsp + s] += (T)acc;
          }
  }
}

// Step bound of the direction D: per vertex the smallest of its reach (two
// cells of motion) and 0.9 d / (-u . dx) over the triangles listed in the
// cells its swept box overlaps; the minimum over the vertices (positive
// doubles order like their bit patterns, so an integer atomicMin is exact).
template <typename T>
__global__ void __launch_bounds__(128) k_contact_ccd(CView cv, Obs ob, int sp0, const T* __restrict__ C,
                                                     const T* __restrict__ D, int N,
                                                     unsigned long long* __restrict__ amin) {
  const int k = blockIdx.x * blockDim.x + threadIdx.x;
  double alpha = 1.0;
  if (k < cv.nvert) {
    const V3 p = vertex_position<T>(cv, k, sp0, C, N), dx = vertex_position<T>(cv, k, sp0, D, N);
    const double ext = fmax(fabs(dx.x), fmax(fabs(dx.y), fabs(dx.z)));
    if (ext > 0.0) {
      alpha = fmin(1.0, 2.0 * ob.cell / ext);
      const V3 e = add(p, scl(alpha, dx));
      const int c0[3] = {cell_of(fmin(p.x, e.x), ob.cell), cell_of(fmin(p.y, e.y), ob.cell),
                         cell_of(fmin(p.z, e.z), ob.cell)};
      const int c1[3] = {cell_of(fmax(p.x, e.x), ob.cell), cell_of(fmax(p.y, e.y), ob.cell),
                         cell_of(fmax(p.z, e.z), ob.cell)};
      for (int cz = c0[2]; cz <= c1[2]; ++cz)
        for (int cy = c0[1]; cy <= c1[1]; ++cy)
          for (int cx = c0[0]; cx <= c1[0]; ++cx) {
            const unsigned int bk = cell_hash(cx, cy, cz, ob.ht);
            for (int it = ob.boff[bk]; it < ob.boff[bk + 1]; ++it) {
              V3 a, b, c;
              ob.tri(ob.btri[it], &a, &b, &c);
              const V3 df = sub(p, closest_on_triangle(p, a, b, c));
              const double d = sqrt(dot(df, df));
              if (!(d > 0.0)) {
                alpha = 0.0;
                continue;
              }
              const double rate = dot(df, dx) / d;
              if (rate < 0.0) alpha = fmin(alpha, 0.9 * d / -rate);
            }
          }
    }
  }
  __shared__ double sm[4];
  for (int o = 16; o > 0; o >>= 1) alpha = fmin(alpha, __shfl_down_sync(0xffffffffu, alpha, o));
  if ((threadIdx.x & 31) == 0) sm[threadIdx.x >> 5] = alpha;
  __syncthreads();
  if (threadIdx.x == 0) {
    double m = sm[0];
    for (int w = 1; w < 4; ++w) m = fmin(m, sm[w]);
    atomicMin(amin, (unsigned long long)__double_as_longlong(m));
  }
}

__global__ void k_set_one(unsigned long long* p) { *p = (unsigned long long)__double_as_longlong(1.0); }

}  // namespace

namespace {

CView cview(const bsc_ctx* c) {
  const bsc_contact* ct = c->contact;
  return CView{ct->vspan, ct->vw, ct->nvert, c->hpd[0].Su, c->hpd[0].nu, c->hpd[0].cp0};
}

Obs obs_view(const bsc_contact* ct) {
  return Obs{ct->ov, ct->ot, ct->own, ct->bucket_off, ct->bucket_tri, ct->nvo, ct->nto, ct->ht, ct->cell};
}

void contact_free(bsc_contact* ct) {
  if (!ct) return;
  void* ptrs[] = {ct->vspan, ct->vw, ct->varea, ct->span_off, ct->span_vert, ct->ov, ct->ot, ct->own,
                  ct->bucket_off, ct->bucket_tri, ct->cE, ct->cg, ct->cH, ct->npairs, ct->ccd};
  for (void* p : ptrs)
    if (p) cudaFree(p);
  free(ct);
}

}  // namespace

// Contact terms at C added to the span arrays (after the elastic projection):
// energy always, gradient with add_g, Hessian with add_h; with a gate only
// when the patch's line search is pending.
cudaError_t contact_add(bsc_ctx* c, const void* C, int add_g, int add_h, const PatchStep* gate) {
  bsc_contact* ct = c->contact;
  if (!ct) return cudaSuccess;
  const int B = 128;
  cudaError_t e = cudaMemsetAsync(ct->npairs, 0, sizeof(int), c->stream);
  if (e != cudaSuccess) return e;
  BSC_COUNT(c, 2);
  const int sp0 = c->hpd[0].sp0;
  if (c->precision == BSC_FP64) {
    k_contact_eval<double><<<(ct->nvert + B - 1) / B, B, 0, c->stream>>>(
        cview(c), obs_view(ct), ct->varea, sp0, (const double*)C, c->N, ct->dhat, ct->kappa, gate, ct->cE, ct->cg,
        ct->cH, ct->npairs, c->dstatus);
    k_contact_span<double><<<(c->Nsp + B - 1) / B, B, 0, c->stream>>>(
        c->Nsp, ct->nvert, ct->span_off, ct->span_vert, ct->vw, ct->cE, ct->cg, ct->cH, add_g, add_h, gate, c->E_span,
        (double*)c->g_span, (double*)c->H_span);
  } else {
    k_contact_eval<float><<<(ct->nvert + B - 1) / B, B, 0, c->stream>>>(
        cview(c), obs_view(ct), ct->varea, sp0, (const float*)C, c->N, ct->dhat, ct->kappa, gate, ct->cE, ct->cg,
        ct->cH, ct->npairs, c->dstatus);
    k_contact_span<float><<<(c->Nsp + B - 1) / B, B, 0, c->stream>>>(
        c->Nsp, ct->nvert, ct->span_off, ct->span_vert, ct->vw, ct->cE, ct->cg, ct->cH, add_g, add_h, gate, c->E_span,
        (float*)c->g_span, (float*)c->H_span);
  }
  return cudaGetLastError();
}

// Step bound of direction D from C into ct->ccd (a device double).
cudaError_t contact_step_bound(bsc_ctx* c, const void* C, const void* D) {
  bsc_contact* ct = c->contact;
  if (!ct) return cudaSuccess;
  const int B = 128;
  unsigned long long* amin = reinterpret_cast<unsigned long long*>(ct->ccd);
  BSC_COUNT(c, 2);
  k_set_one<<<1, 1, 0, c->stream>>>(amin);
  if (c->precision == BSC_FP64)
    k_contact_ccd<double><<<(ct->nvert + B - 1) / B, B, 0, c->stream>>>(cview(c), obs_view(ct), c->hpd[0].sp0,
                                                                        (const double*)C, (const double*)D, c->N, amin);
  else
    k_contact_ccd<float><<<(ct->nvert + B - 1) / B, B, 0, c->stream>>>(cview(c), obs_view(ct), c->hpd[0].sp0,
                                                                       (const float*)C, (const float*)D, c->N, amin);
  return cudaGetLastError();
}

const double* contact_bound_ptr(const bsc_ctx* c) { return c->contact ? c->contact->ccd : nullptr; }

void contact_destroy(bsc_ctx* c) {
  if (c && c->contact) {
    contact_free(c->contact);
    c->contact = nullptr;
  }
}

namespace {

template <typename T>
__global__ void k_contact_positions(CView cv, int sp0, const T* __restrict__ C, int N, double* __restrict__ x) {
  const int k = blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= cv.nvert) return;
  const V3 p = vertex_position<T>(cv, k, sp0, C, N);
  x[(size_t)3 * k] = p.x;
  x[(size_t)3 * k + 1] = p.y;
  x[(size_t)3 * k + 2] = p.z;
}

bsc_status cfail(bsc_ctx* c, bsc_status st, const char* msg) {
  snprintf(c->err, sizeof(c->err), "%s", msg);
  return st;
}

}  // namespace

void bsc_drop_graph(bsc_ctx* c);

extern "C" {

bsc_status bsc_contact_attach(bsc_ctx* c, const double* obs_xyz, int nvo, const int32_t* tris, int nto, int mu,
                              int mv, double dhat, double kappa) {
  if (!c) return BSC_ERR_INVALID_ARG;
  if (c->P != 1 || c->is_window)
    return cfail(c, BSC_ERR_INVALID_ARG, "bsc_contact_attach: single-patch contexts only (no strip windows)");
  if (!obs_xyz || !tris || nvo < 3 || nto < 1)
    return cfail(c, BSC_ERR_INVALID_ARG, "bsc_contact_attach: the obstacle needs >= 3 vertices and >= 1 triangle");
  if (!(dhat > 0.0) || !isfinite(dhat) || !(kappa >= 0.0) || !isfinite(kappa))
    return cfail(c, BSC_ERR_INVALID_ARG, "bsc_contact_attach: dhat must be > 0 and kappa >= 0, both finite");
  for (long long i = 0; i < 3ll * nvo; ++i)
    if (!isfinite(obs_xyz[i])) return cfail(c, BSC_ERR_INVALID_ARG, "bsc_contact_attach: non-finite obstacle vertex");
  for (int t = 0; t < nto; ++t) {
    const int a = tris[3 * t], b = tris[3 * t + 1], d = tris[3 * t + 2];
    if (a < 0 || b < 0 || d < 0 || a >= nvo || b >= nvo || d >= nvo || a == b || b == d || a == d)
      return cfail(c, BSC_ERR_INVALID_ARG, "bsc_contact_attach: triangle indices out of range or repeated");
  }
  const PatchDev& pd = c->hpd[0];
  if (mu <= 0) mu = (int)lround(1.41421356237 * (pd.nu - 1)) + 1;
  if (mv <= 0) mv = (int)lround(1.41421356237 * (pd.nv - 1)) + 1;
  if (mu < 2 || mv < 2 || (long long)mu * mv > (1ll << 26))
    return cfail(c, BSC_ERR_INVALID_ARG, "bsc_contact_attach: contact mesh must have 2..2^26 vertices per side product");
  cudaError_t e = cudaStreamSynchronize(c->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(c->gstream);
  if (e != cudaSuccess) return cfail(c, BSC_ERR_CUDA, "bsc_contact_attach: stream synchronisation failed");
  contact_destroy(c);
  bsc_drop_graph(c);
  bsc_contact* ct = (bsc_contact*)calloc(1, sizeof(bsc_contact));
  if (!ct) return cfail(c, BSC_ERR_OOM, "bsc_contact_attach: host allocation failed");
  ct->mu = mu;
  ct->mv = mv;
  ct->nvert = mu * mv;
  ct->dhat = dhat;
  ct->kappa = kappa;
  ct->nvo = nvo;
  ct->nto = nto;
  const int nvert = ct->nvert, Nsp = c->Nsp;
#define CA(ptr, bytes) \
  if (e == cudaSuccess) e = cudaMalloc((void**)&(ptr), (bytes))
  double* xrest = nullptr;
  CA(ct->vspan, sizeof(int) * nvert);
  CA(ct->vw, sizeof(double) * 9 * (size_t)nvert);
  CA(ct->varea, sizeof(double) * nvert);
  CA(ct->span_off, sizeof(int) * (size_t)(Nsp + 1));
  CA(ct->span_vert, sizeof(int) * nvert);
  CA(ct->ov, sizeof(double) * 3 * (size_t)nvo);
  CA(ct->ot, sizeof(int) * 3 * (size_t)nto);
  CA(ct->own, (size_t)nto);
  CA(ct->cE, sizeof(double) * nvert);
  CA(ct->cg, sizeof(double) * 3 * (size_t)nvert);
  CA(ct->cH, sizeof(double) * 6 * (size_t)nvert);
  CA(ct->npairs, sizeof(int) * 2);
  CA(ct->ccd, sizeof(double) * 2);
  CA(xrest, sizeof(double) * 3 * (size_t)nvert);
  if (e == cudaSuccess) {
    k_contact_setup<<<(nvert + 127) / 128, 128, 0, c->stream>>>(mu, mv, pd.nu, pd.nv, pd.sp0, pd.cp0, c->N, c->rest,
                                                               ct->vspan, ct->vw, xrest);
    e = cudaGetLastError();
  }
  std::vector<int> vspan(nvert);
  std::vector<double> xr(2 * (size_t)nvert);
  if (e == cudaSuccess) e = cudaMemcpyAsync(vspan.data(), ct->vspan, sizeof(int) * nvert, cudaMemcpyDeviceToHost, c->stream);
  if (e == cudaSuccess) e = cudaMemcpyAsync(xr.data(), xrest, sizeof(double) * 2 * nvert, cudaMemcpyDeviceToHost, c->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
  if (xrest) cudaFree(xrest);
  if (e != cudaSuccess) {
    contact_free(ct);
    return cfail(c, BSC_ERR_CUDA, "bsc_contact_attach: setting up the contact mesh failed");
  }
  // vertex areas: a third of each rest triangle's area (cells split along
  // alternating diagonals)
  std::vector<double> area(nvert, 0.0);
  auto tri_area = [&](int p, int q, int r) {
    const double ax = xr[q] - xr[p], ay = xr[nvert + q] - xr[nvert + p];
    const double bx = xr[r] - xr[p], by = xr[nvert + r] - xr[nvert + p];
    const double A = 0.5 * fabs(ax * by - ay * bx) / 3.0;
    area[p] += A;
    area[q] += A;
    area[r] += A;
  };
  for (int j = 0; j + 1 < mv; ++j)
    for (int i = 0; i + 1 < mu; ++i) {
      const int k = j * mu + i;
      if ((i + j) % 2 == 0) {
        tri_area(k, k + 1, k + mu + 1);
        tri_area(k, k + mu + 1, k + mu);
      } else {
        tri_area(k, k + 1, k + mu);
        tri_area(k + 1, k + mu + 1, k + mu);
      }
    }
  // vertices of each span, in vertex order
  std::vector<int> off(Nsp + 1, 0), lst(nvert);
  for (int k = 0; k < nvert; ++k) off[vspan[k] - pd.sp0 + 1] += 1;
  for (int s = 0; s < Nsp; ++s) off[s + 1] += off[s];
  {
    std::vector<int> pos(off.begin(), off.end() - 1);
    for (int k = 0; k < nvert; ++k) lst[pos[vspan[k] - pd.sp0]++] = k;
  }
  // obstacle planes, feature owners, spatial hash
  std::vector<double> ov(3 * (size_t)nvo);
  for (int i = 0; i < nvo; ++i)
    for (int d = 0; d < 3; ++d) ov[(size_t)d * nvo + i] = obs_xyz[3 * i + d];
  std::vector<int> ot(3 * (size_t)nto);
  std::vector<unsigned char> own(nto, 0);
  {
    std::vector<int> vown(nvo, -1);
    std::vector<std::pair<long long, int>> edges;
    edges.reserve(3 * (size_t)nto);
    const int ep[3][2] = {{0, 1}, {0, 2}, {1, 2}};
    for (int t = 0; t < nto; ++t) {
      for (int d = 0; d < 3; ++d) ot[(size_t)d * nto + t] = tris[3 * t + d];
      for (int d = 0; d < 3; ++d)
        if (vown[tris[3 * t + d]] < 0) {
          vown[tris[3 * t + d]] = t;
          own[t] |= (unsigned char)(8 << d);
        }
      for (int k = 0; k < 3; ++k) {
        const long long a = tris[3 * t + ep[k][0]], b = tris[3 * t + ep[k][1]];
        edges.push_back({std::min(a, b) * nvo + std::max(a, b), t * 3 + k});
      }
    }
    std::sort(edges.begin(), edges.end());
    for (size_t i = 0; i < edges.size(); ++i)
      if (i == 0 || edges[i].first != edges[i - 1].first) {
        const int t = edges[i].second / 3, k = edges[i].second % 3;
        own[t] |= (unsigned char)(1 << k);  // the lowest triangle (then edge slot) holding this edge
      }
  }
  double elen = 0.0;
  for (int t = 0; t < nto; ++t)
    for (int k = 0; k < 3; ++k) {
      const int a = tris[3 * t + k], b = tris[3 * t + (k + 1) % 3];
      double s2 = 0.0;
      for (int d = 0; d < 3; ++d) s2 += (obs_xyz[3 * a + d] - obs_xyz[3 * b + d]) * (obs_xyz[3 * a + d] - obs_xyz[3 * b + d]);
      elen += sqrt(s2);
    }
  elen /= 3.0 * nto;
  ct->cell = std::max(2.0 * dhat, elen);
  struct Ent {
    int x, y, z, t;
  };
  std::vector<Ent> ent;
  for (int t = 0; t < nto; ++t) {
    double lo[3], hi[3];
    for (int d = 0; d < 3; ++d) {
      lo[d] = hi[d] = obs_xyz[3 * tris[3 * t] + d];
      for (int k = 1; k < 3; ++k) {
        lo[d] = std::min(lo[d], obs_xyz[3 * tris[3 * t + k] + d]);
        hi[d] = std::max(hi[d], obs_xyz[3 * tris[3 * t + k] + d]);
      }
      lo[d] -= dhat;
      hi[d] += dhat;
    }
    const int c0[3] = {cell_of(lo[0], ct->cell), cell_of(lo[1], ct->cell), cell_of(lo[2], ct->cell)};
    const int c1[3] = {cell_of(hi[0], ct->cell), cell_of(hi[1], ct->cell), cell_of(hi[2], ct->cell)};
    const long long ncell = (long long)(c1[0] - c0[0] + 1) * (c1[1] - c0[1] + 1) * (c1[2] - c0[2] + 1);
    if (ncell > 4096 || (long long)ent.size() + ncell > (1ll << 26)) {
      contact_free(ct);
      return cfail(c, BSC_ERR_INVALID_ARG,
                   "bsc_contact_attach: obstacle triangles span too many hash cells (refine the mesh)");
    }
    for (int z = c0[2]; z <= c1[2]; ++z)
      for (int y = c0[1]; y <= c1[1]; ++y)
        for (int x = c0[0]; x <= c1[0]; ++x) ent.push_back(Ent{x, y, z, t});
  }
  int ht = 1024;
  while ((size_t)ht < 2 * ent.size() && ht < (1 << 26)) ht <<= 1;
  ct->ht = ht;
  std::vector<std::pair<unsigned int, int>> bt(ent.size());
  for (size_t i = 0; i < ent.size(); ++i) bt[i] = {cell_hash(ent[i].x, ent[i].y, ent[i].z, ht), ent[i].t};
  std::sort(bt.begin(), bt.end());
  bt.erase(std::unique(bt.begin(), bt.end()), bt.end());  // a triangle once per bucket
  std::vector<int> boff(ht + 1, 0), btri(bt.size());
  for (size_t i = 0; i < bt.size(); ++i) {
    boff[bt[i].first + 1] += 1;
    btri[i] = bt[i].second;
  }
  for (int b = 0; b < ht; ++b) boff[b + 1] += boff[b];
  CA(ct->bucket_off, sizeof(int) * (size_t)(ht + 1));
  CA(ct->bucket_tri, sizeof(int) * std::max<size_t>(1, btri.size()));
#undef CA
  auto up = [&](void* dst, const void* src, size_t bytes) {
    if (e == cudaSuccess && bytes) e = cudaMemcpy(dst, src, bytes, cudaMemcpyHostToDevice);
  };
  std::vector<double> areas(area.begin(), area.end());
  up(ct->varea, areas.data(), sizeof(double) * nvert);
  up(ct->span_off, off.data(), sizeof(int) * (Nsp + 1));
  up(ct->span_vert, lst.data(), sizeof(int) * nvert);
  up(ct->ov, ov.data(), sizeof(double) * ov.size());
  up(ct->ot, ot.data(), sizeof(int) * ot.size());
  up(ct->own, own.data(), own.size());
  up(ct->bucket_off, boff.data(), sizeof(int) * boff.size());
  up(ct->bucket_tri, btri.data(), sizeof(int) * btri.size());
  if (e == cudaSuccess) e = cudaMemset(ct->npairs, 0, sizeof(int) * 2);
  if (e != cudaSuccess) {
    contact_free(ct);
    return cfail(c, e == cudaErrorMemoryAllocation ? BSC_ERR_OOM : BSC_ERR_CUDA, "bsc_contact_attach: device set-up failed");
  }
  c->contact = ct;
  return BSC_OK;
}

bsc_status bsc_contact_detach(bsc_ctx* c) {
  if (!c) return BSC_ERR_INVALID_ARG;
  if (cudaStreamSynchronize(c->stream) != cudaSuccess || cudaStreamSynchronize(c->gstream) != cudaSuccess)
    return cfail(c, BSC_ERR_CUDA, "bsc_contact_detach: stream synchronisation failed");
  bsc_drop_graph(c);
  contact_destroy(c);
  return BSC_OK;
}

bsc_status bsc_contact_vertices(bsc_ctx* c, const void* C, double* x_out, int cap, int* nvert) {
  if (!c || !c->contact) return c ? cfail(c, BSC_ERR_INVALID_ARG, "bsc_contact_vertices: no contact attached")
                                   : BSC_ERR_INVALID_ARG;
  bsc_contact* ct = c->contact;
  if (nvert) *nvert = ct->nvert;
  if (!x_out) return BSC_OK;
  if (!C || cap < ct->nvert) return cfail(c, BSC_ERR_INVALID_ARG, "bsc_contact_vertices: NULL C or output too small");
  double* d = nullptr;
  cudaError_t e = cudaMalloc(&d, sizeof(double) * 3 * (size_t)ct->nvert);
  if (e == cudaSuccess) {
    BSC_COUNT(c, 1);
    if (c->precision == BSC_FP64)
      k_contact_positions<double><<<(ct->nvert + 127) / 128, 128, 0, c->stream>>>(cview(c), c->hpd[0].sp0,
                                                                                (const double*)C, c->N, d);
    else
      k_contact_positions<float><<<(ct->nvert + 127) / 128, 128, 0, c->stream>>>(cview(c), c->hpd[0].sp0,
                                                                               (const float*)C, c->N, d);
    e = cudaGetLastError();
  }
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(x_out, d, sizeof(double) * 3 * (size_t)ct->nvert, cudaMemcpyDeviceToHost, c->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
  if (d) cudaFree(d);
  return e == cudaSuccess ? BSC_OK : cfail(c, BSC_ERR_CUDA, "bsc_contact_vertices: CUDA error");
}

bsc_status bsc_contact_step_bound(bsc_ctx* c, const void* C, const void* D, double* alpha) {
  if (!c || !c->contact || !C || !D || !alpha)
    return c ? cfail(c, BSC_ERR_INVALID_ARG, "bsc_contact_step_bound: no contact attached or NULL argument")
             : BSC_ERR_INVALID_ARG;
  cudaError_t e = contact_step_bound(c, C, D);
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(alpha, c->contact->ccd, sizeof(double), cudaMemcpyDeviceToHost, c->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
  return e == cudaSuccess ? BSC_OK : cfail(c, BSC_ERR_CUDA, "bsc_contact_step_bound: CUDA error");
}

bsc_status bsc_contact_stats(bsc_ctx* c, int* nvert, int* npairs) {
  if (!c || !c->contact) return c ? cfail(c, BSC_ERR_INVALID_ARG, "bsc_contact_stats: no contact attached")
                                   : BSC_ERR_INVALID_ARG;
  if (nvert) *nvert = c->contact->nvert;
  if (npairs) {
    if (cudaMemcpyAsync(npairs, c->contact->npairs, sizeof(int), cudaMemcpyDeviceToHost, c->stream) != cudaSuccess ||
        cudaStreamSynchronize(c->stream) != cudaSuccess)
      return cfail(c, BSC_ERR_CUDA, "bsc_contact_stats: CUDA error");
  }
  return BSC_OK;
}

}  // extern "C"

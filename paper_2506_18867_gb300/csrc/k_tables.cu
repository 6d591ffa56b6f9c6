// K0 / K1: quadrature tables and lumped masses (built once in bsc_create).
//
// Every span enumerates the quadrature points it owns (Sec. 4.1 reduced
// membrane rule and Sec. 4.2 one-point bending rule, Fig. 3), evaluates the
// nine quadratic tensor-product basis functions of the span with first and
// second derivatives, maps them to material space through the rest map
// (Eq. deformation gradient; inverse function theorem) and stores per point
//   membrane: W = w |det J|,  g_l = dN_l/dX  (J^-T grad_uv N_l)
//   bending : W,  L_l = sum of the five terms of Eq. (Laplacian in
//             parametric space) for control point l.
// Tables are stored as planes (entry-major) so that neighbouring threads read
// neighbouring addresses.
#include <math.h>

#include <vector>

#include "bsc_internal.cuh"

namespace {

struct QP {
  double u, v, w;
};

// Open uniform quadratic knot xi_k = clamp(k - 2, 0, S).
__device__ __forceinline__ double knot_at(int k, int S) {
  int v = k - 2;
  v = v < 0 ? 0 : (v > S ? S : v);
  return (double)v;
}

__device__ __forceinline__ double safe_recip(double x) { return x == 0.0 ? 0.0 : 1.0 / x; }

// Values, first and second derivatives of the three degree-2 B-splines that
// are non-zero on span a (knot interval [xi_o, xi_o+1], o = a + 2), from the
// degree-1 pieces and the derivative identity
//   N'_{i,p} = p (N_{i,p-1} / (xi_{i+p} - xi_i) - N_{i+1,p-1} / (xi_{i+p+1} - xi_{i+1})).
__device__ void span_basis(double t, int a, int S, double N[3], double D[3], double D2[3]) {
  const int o = a + 2;
  double x[6];  // xi_{o-2} .. xi_{o+3}
  for (int k = 0; k < 6; ++k) x[k] = knot_at(o - 2 + k, S);
  // x[2] = xi_o, x[3] = xi_{o+1}
  const double h = x[3] - x[2];
  // degree 1 on the span: functions o-1 and o (index 0, 1 here), plus zeros
  double B1[4] = {0.0, (x[3] - t) / h, (t - x[2]) / h, 0.0};      // functions o-2 .. o+1
  double dB1[4] = {0.0, -1.0 / h, 1.0 / h, 0.0};
  for (int k = 0; k < 3; ++k) {
    // function i = o - 2 + k uses knots xi_i .. xi_{i+3} = x[k] .. x[k+3]
    const double r0 = safe_recip(x[k + 2] - x[k]);
    const double r1 = safe_recip(x[k + 3] - x[k + 1]);
    N[k] = (t - x[k]) * r0 * B1[k] + (x[k + 3] - t) * r1 * B1[k + 1];
    D[k] = 2.0 * (B1[k] * r0 - B1[k + 1] * r1);
    D2[k] = 2.0 * (dB1[k] * r0 - dB1[k + 1] * r1);
  }
}

// Enumerates the membrane (which = 0) or bending (which = 1) points owned by
// span (a, b).  Returns the count; writes up to 9 points.
__device__ int span_points(int a, int b, int Su, int Sv, int which, int rule, QP* out) {
  const double g2 = 0.28867513459481287;  // 1/(2 sqrt 3): 2-point Gauss offset
  int n = 0;
  auto gauss_span = [&](int nq_u, int nq_v) {
    double xu[3], wu[3], xv[3], wv[3];
    const double o3 = 0.38729833462074170;  // sqrt(3/5)/2: 3-point offset
    auto fill = [&](int nq, double* x, double* w) {
      if (nq == 1) { x[0] = 0.5; w[0] = 1.0; }
      else if (nq == 2) { x[0] = 0.5 - g2; x[1] = 0.5 + g2; w[0] = w[1] = 0.5; }
      else { x[0] = 0.5 - o3; x[1] = 0.5; x[2] = 0.5 + o3; w[0] = w[2] = 5.0 / 18.0; w[1] = 8.0 / 18.0; }
    };
    fill(nq_u, xu, wu);
    fill(nq_v, xv, wv);
    for (int j = 0; j < nq_v; ++j)
      for (int i = 0; i < nq_u; ++i) out[n++] = QP{a + xu[i], b + xv[j], wu[i] * wv[j]};
  };
  if (rule == BSC_QUAD_GAUSS2 || rule == BSC_QUAD_GAUSS3) {
    gauss_span(rule, rule);
    return n;
  }
  const bool ring_u = (a == 0 || a == Su - 1), ring_v = (b == 0 || b == Sv - 1);
  if (ring_u || ring_v) {
    if (which == 0) gauss_span(ring_u ? 3 : 2, ring_v ? 3 : 2);
    else out[n++] = QP{a + 0.5, b + 0.5, 1.0};
    return n;
  }
  if (rule == BSC_QUAD_STANDARD) {  // ablation baseline: 2x2 Gauss per interior span
    gauss_span(2, 2);
    return n;
  }
  // Interior span: candidate dual cells centred on knots (ku, kv) with
  // ku in {a, a+1}, kv in {b, b+1}; keep the points this span owns.  A point
  // on knot line k belongs to span clamp(k, 1, S-2); otherwise to floor.
  auto owner = [](double x, bool on_line, int k, int S) -> int {
    return on_line ? (k < 1 ? 1 : (k > S - 2 ? S - 2 : k)) : (int)floor(x);
  };
  for (int kv = b; kv <= b + 1; ++kv)
    for (int ku = a; ku <= a + 1; ++ku) {
      const bool bu = (ku == 1 || ku == Su - 1), bv = (kv == 1 || kv == Sv - 1);
      // up to two points: offsets (su, sv) in units of g2 along u / v
      int np = 0;
      int su[2] = {0, 0}, sv[2] = {0, 0};
      double w = 0.0;
      if (which == 1) {
        np = 1;
        w = (bu ? 0.5 : 1.0) * (bv ? 0.5 : 1.0);
      } else if (bu && bv) {
        np = 1; w = 0.25;
      } else if (bu || (!bv && ((ku + kv) % 2 == 0))) {
        // points stacked along v on the line u = ku
        np = 2; sv[0] = -1; sv[1] = 1; w = bu ? 0.25 : 0.5;
      } else {
        // points side by side along u on the line v = kv
        np = 2; su[0] = -1; su[1] = 1; w = bv ? 0.25 : 0.5;
      }
      for (int k = 0; k < np; ++k) {
        const double u = ku + su[k] * g2, v = kv + sv[k] * g2;
        if (owner(u, su[k] == 0, ku, Su) == a && owner(v, sv[k] == 0, kv, Sv) == b)
          out[n++] = QP{u, v, w};
      }
    }
  return n;
}

// Sv local span rows starting at global span row vb0 of SvG (a strip window;
// vb0 = 0, SvG = Sv for a whole patch).
__global__ void k_count_points(int Su, int Sv, int vb0, int SvG, int mem_rule, int bend_rule, int* __restrict__ cm,
                               int* __restrict__ cb) {
  const int s = blockIdx.x * blockDim.x + threadIdx.x;
  if (s >= Su * Sv) return;
  QP pts[9];
  cm[s] = span_points(s % Su, s / Su + vb0, Su, SvG, 0, mem_rule, pts);
  cb[s] = span_points(s % Su, s / Su + vb0, Su, SvG, 1, bend_rule, pts);
}

// Rest-map geometry at (u, v) in span (a, b) and the per-point table rows.
// One patch: nu x nv control points starting at cp0 in the rest planes
// (stride Ntot), spans starting at sp0 in the offset arrays; local span row b
// is the global row b + vb0 of SvG (the v coordinates stored are global, the
// owner span indices local).
template <typename T>
__global__ void k_fill_points(int nu, int nv, int vb0, int SvG, int cp0, int sp0, int Ntot,
                              const double* __restrict__ rest, int mem_rule, int bend_rule,
                              const int* __restrict__ moff, const int* __restrict__ boff, int Nm, int Nb,
                              T* __restrict__ tabm, T* __restrict__ tabb, double* __restrict__ ptsm,
                              double* __restrict__ ptsb, int* __restrict__ status) {
  const int Su = nu - 2, Sv = nv - 2;
  const int s = blockIdx.x * blockDim.x + threadIdx.x;
  if (s >= Su * Sv) return;
  const int a = s % Su, b = s / Su, bg = b + vb0;
  double X[9][2];
  for (int l = 0; l < 9; ++l) {
    const int al = cp0 + (b + l / 3) * nu + a + l % 3;
    X[l][0] = rest[al];
    X[l][1] = rest[Ntot + al];
  }
  for (int which = 0; which < 2; ++which) {
    QP pts[9];
    const int np = span_points(a, bg, Su, SvG, which, which ? bend_rule : mem_rule, pts);
    const int base = which ? boff[sp0 + s] : moff[sp0 + s];
    for (int k = 0; k < np; ++k) {
      double Nu[3], Du[3], D2u[3], Nv[3], Dv[3], D2v[3];
      span_basis(pts[k].u, a, Su, Nu, Du, D2u);
      span_basis(pts[k].v, bg, SvG, Nv, Dv, D2v);
      // dX/du, dX/dv and second derivatives of the rest map
      double Xu[2] = {0, 0}, Xv[2] = {0, 0}, Xuu[2] = {0, 0}, Xuv[2] = {0, 0}, Xvv[2] = {0, 0};
      double Nl_u[9], Nl_v[9], Nl_uu[9], Nl_uv[9], Nl_vv[9];
      for (int l = 0; l < 9; ++l) {
        const int li = l % 3, lj = l / 3;
        Nl_u[l] = Du[li] * Nv[lj];
        Nl_v[l] = Nu[li] * Dv[lj];
        Nl_uu[l] = D2u[li] * Nv[lj];
        Nl_uv[l] = Du[li] * Dv[lj];
        Nl_vv[l] = Nu[li] * D2v[lj];
        for (int d = 0; d < 2; ++d) {
          Xu[d] += Nl_u[l] * X[l][d];
          Xv[d] += Nl_v[l] * X[l][d];
          Xuu[d] += Nl_uu[l] * X[l][d];
          Xuv[d] += Nl_uv[l] * X[l][d];
          Xvv[d] += Nl_vv[l] * X[l][d];
        }
      }
      const double det = Xu[0] * Xv[1] - Xv[0] * Xu[1];
      if (!(fabs(det) > 0.0) || !isfinite(det)) atomicOr(status, BSC_STATUS_NUMERIC_FLAG);
      // M = (dX/d(u,v))^-1: M[0][beta] = du/dX_beta, M[1][beta] = dv/dX_beta
      const double M00 = Xv[1] / det, M01 = -Xv[0] / det, M10 = -Xu[1] / det, M11 = Xu[0] / det;
      const double W = pts[k].w * fabs(det);
      const int q = base + k;
      double* pt = which ? ptsb : ptsm;
      const int Np = which ? Nb : Nm;
      pt[0 * Np + q] = pts[k].u;
      pt[1 * Np + q] = pts[k].v;
      pt[2 * Np + q] = pts[k].w;
      pt[3 * Np + q] = a;
      pt[4 * Np + q] = b;
      if (which == 0) {
        tabm[q] = (T)W;
        for (int l = 0; l < 9; ++l) {
          tabm[(1 + 2 * l) * Nm + q] = (T)(Nl_u[l] * M00 + Nl_v[l] * M10);
          tabm[(2 + 2 * l) * Nm + q] = (T)(Nl_u[l] * M01 + Nl_v[l] * M11);
        }
      } else {
        // inverse metric G = M M^T (G00 = u1^2+u2^2, G11 = v1^2+v2^2, G01 = u1 v1 + u2 v2)
        const double G00 = M00 * M00 + M01 * M01, G11 = M10 * M10 + M11 * M11;
        const double G01 = M00 * M10 + M01 * M11;
        // Laplacian of u_a(X): -sum_d M[a][d] (X_d,uu G00 + 2 X_d,uv G01 + X_d,vv G11)
        const double h0 = Xuu[0] * G00 + 2.0 * Xuv[0] * G01 + Xvv[0] * G11;
        const double h1 = Xuu[1] * G00 + 2.0 * Xuv[1] * G01 + Xvv[1] * G11;
        const double lap_u = -(M00 * h0 + M01 * h1), lap_v = -(M10 * h0 + M11 * h1);
        tabb[q] = (T)W;
        for (int l = 0; l < 9; ++l)
          tabb[(1 + l) * Nb + q] = (T)(G00 * Nl_uu[l] + G11 * Nl_vv[l] + 2.0 * G01 * Nl_uv[l] +
                                       lap_u * Nl_u[l] + lap_v * Nl_v[l]);
      }
    }
  }
}

// Lumped mass m_alpha = rho * int N_alpha |det J| du dv, 3x3 Gauss per span,
// gathered per control point over the (up to 3x3) spans of its support that
// the context holds (all of them but on a strip window's outer halo rows).
__global__ void k_lumped_mass(int nu, int nv, int vb0, int SvG, int cp0, int Ntot, const double* __restrict__ rest,
                              double rho, double* __restrict__ m) {
  const int Su = nu - 2, Sv = nv - 2, N = nu * nv;
  const int al = blockIdx.x * blockDim.x + threadIdx.x;
  if (al >= N) return;
  const int i = al % nu, j = al / nu;
  const double o3 = 0.38729833462074170;
  const double gx[3] = {0.5 - o3, 0.5, 0.5 + o3}, gw[3] = {5.0 / 18.0, 8.0 / 18.0, 5.0 / 18.0};
  double acc = 0.0;
  for (int b = j - 2; b <= j; ++b) {
    if (b < 0 || b >= Sv) continue;
    for (int a = i - 2; a <= i; ++a) {
      if (a < 0 || a >= Su) continue;
      double X[9][2];
      for (int l = 0; l < 9; ++l) {
        const int bl = cp0 + (b + l / 3) * nu + a + l % 3;
        X[l][0] = rest[bl];
        X[l][1] = rest[Ntot + bl];
      }
      for (int qv = 0; qv < 3; ++qv)
        for (int qu = 0; qu < 3; ++qu) {
          double Nu[3], Du[3], D2u[3], Nv[3], Dv[3], D2v[3];
          span_basis(a + gx[qu], a, Su, Nu, Du, D2u);
          span_basis(b + vb0 + gx[qv], b + vb0, SvG, Nv, Dv, D2v);
          double Xu0 = 0, Xu1 = 0, Xv0 = 0, Xv1 = 0;
          for (int l = 0; l < 9; ++l) {
            const double nu_ = Du[l % 3] * Nv[l / 3], nv_ = Nu[l % 3] * Dv[l / 3];
            Xu0 += nu_ * X[l][0]; Xu1 += nu_ * X[l][1];
            Xv0 += nv_ * X[l][0]; Xv1 += nv_ * X[l][1];
          }
          const double det = fabs(Xu0 * Xv1 - Xv0 * Xu1);
          acc += gw[qu] * gw[qv] * det * Nu[i - a] * Nv[j - b];
        }
    }
  }
  m[cp0 + al] = rho * acc;
}

}  // namespace

// Builds tables, offsets, masses, projection buckets and the patch maps of
// every patch.  Host work is the integer bookkeeping (prefix sums of the
// per-span point counts over all patches, the bucketing of spans by reduced
// problem size); the geometry runs on the GPU, one launch per patch.
cudaError_t launch_build_tables(bsc_ctx* c) {
  cudaError_t e;
  const int Nsp = c->Nsp, N = c->N, B = 128;
  int *cm = nullptr, *cb = nullptr;
  if ((e = cudaMalloc(&cm, sizeof(int) * Nsp)) != cudaSuccess) return e;
  if ((e = cudaMalloc(&cb, sizeof(int) * Nsp)) != cudaSuccess) { cudaFree(cm); return e; }
  for (int p = 0; p < c->P; ++p) {
    const PatchDev& q = c->hpd[p];
    BSC_COUNT(c, 1);
    k_count_points<<<(q.Nsp + B - 1) / B, B, 0, c->stream>>>(q.Su, q.Sv, q.vb0, q.SvG, c->mem_rule, c->bend_rule,
                                                            cm + q.sp0, cb + q.sp0);
  }
  std::vector<int> hcm(Nsp), hcb(Nsp), hmo(Nsp + 1), hbo(Nsp + 1), hbl(Nsp), hsp(Nsp), hcp(N);
  e = cudaGetLastError();
  if (e == cudaSuccess) e = cudaMemcpyAsync(hcm.data(), cm, sizeof(int) * Nsp, cudaMemcpyDeviceToHost, c->stream);
  if (e == cudaSuccess) e = cudaMemcpyAsync(hcb.data(), cb, sizeof(int) * Nsp, cudaMemcpyDeviceToHost, c->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
  cudaFree(cm);
  cudaFree(cb);
  if (e != cudaSuccess) return e;
  hmo[0] = hbo[0] = 0;
  for (int s = 0; s < Nsp; ++s) {
    hmo[s + 1] = hmo[s] + hcm[s];
    hbo[s + 1] = hbo[s] + hcb[s];
  }
  c->Nmem = hmo[Nsp];
  c->Nbd = hbo[Nsp];
  // bucket spans by the dimension of their reduced eigenproblem: the span
  // Hessian's range lies in span{g_q,beta, L_q} (x) R^3, whose dimension is
  // at most min(8, 2 n_mem + n_bd) per component (all vectors sum to zero).
  int nb[3] = {0, 0, 0};
  for (int s = 0; s < Nsp; ++s) {
    const int m = 2 * hcm[s] + hcb[s];
    nb[m <= 5 ? 0 : (m <= 7 ? 1 : 2)]++;
  }
  c->bucket_off[0] = 0;
  c->bucket_off[1] = nb[0];
  c->bucket_off[2] = nb[0] + nb[1];
  c->bucket_off[3] = Nsp;
  int pos[3] = {c->bucket_off[0], c->bucket_off[1], c->bucket_off[2]};
  for (int s = 0; s < Nsp; ++s) {
    const int m = 2 * hcm[s] + hcb[s];
    hbl[pos[m <= 5 ? 0 : (m <= 7 ? 1 : 2)]++] = s;
  }
  for (int p = 0; p < c->P; ++p) {
    const PatchDev& q = c->hpd[p];
    for (int k = 0; k < q.Nsp; ++k) hsp[q.sp0 + k] = p;
    for (int k = 0; k < q.N; ++k) hcp[q.cp0 + k] = p;
  }
  const size_t ts = c->tsize;
  if ((e = cudaMalloc(&c->mem_off, sizeof(int) * (Nsp + 1))) != cudaSuccess) return e;
  if ((e = cudaMalloc(&c->bd_off, sizeof(int) * (Nsp + 1))) != cudaSuccess) return e;
  if ((e = cudaMalloc(&c->bucket_list, sizeof(int) * Nsp)) != cudaSuccess) return e;
  if ((e = cudaMalloc(&c->sp_patch, sizeof(int) * Nsp)) != cudaSuccess) return e;
  if ((e = cudaMalloc(&c->cp_patch, sizeof(int) * N)) != cudaSuccess) return e;
  if ((e = cudaMalloc(&c->tab_mem, ts * TABM * (size_t)c->Nmem)) != cudaSuccess) return e;
  if ((e = cudaMalloc(&c->tab_bd, ts * TABB * (size_t)c->Nbd)) != cudaSuccess) return e;
  if ((e = cudaMalloc(&c->pts_mem, sizeof(double) * 5 * (size_t)c->Nmem)) != cudaSuccess) return e;
  if ((e = cudaMalloc(&c->pts_bd, sizeof(double) * 5 * (size_t)c->Nbd)) != cudaSuccess) return e;
  if ((e = cudaMalloc(&c->A_mem, ts * AQ * (size_t)c->Nmem)) != cudaSuccess) return e;
  if ((e = cudaMemcpy(c->mem_off, hmo.data(), sizeof(int) * (Nsp + 1), cudaMemcpyHostToDevice))) return e;
  if ((e = cudaMemcpy(c->bd_off, hbo.data(), sizeof(int) * (Nsp + 1), cudaMemcpyHostToDevice))) return e;
  if ((e = cudaMemcpy(c->bucket_list, hbl.data(), sizeof(int) * Nsp, cudaMemcpyHostToDevice))) return e;
  if ((e = cudaMemcpy(c->sp_patch, hsp.data(), sizeof(int) * Nsp, cudaMemcpyHostToDevice))) return e;
  if ((e = cudaMemcpy(c->cp_patch, hcp.data(), sizeof(int) * N, cudaMemcpyHostToDevice))) return e;
  for (int p = 0; p < c->P; ++p) {
    const PatchDev& q = c->hpd[p];
    const int G = (q.Nsp + B - 1) / B;
    BSC_COUNT(c, 2);
    if (c->precision == BSC_FP64)
      k_fill_points<double><<<G, B, 0, c->stream>>>(q.nu, q.nv, q.vb0, q.SvG, q.cp0, q.sp0, N, c->rest, c->mem_rule,
                                                      c->bend_rule, c->mem_off, c->bd_off, c->Nmem, c->Nbd,
                                                      (double*)c->tab_mem, (double*)c->tab_bd, c->pts_mem,
                                                      c->pts_bd, c->dstatus);
    else
      k_fill_points<float><<<G, B, 0, c->stream>>>(q.nu, q.nv, q.vb0, q.SvG, q.cp0, q.sp0, N, c->rest, c->mem_rule,
                                                     c->bend_rule, c->mem_off, c->bd_off, c->Nmem, c->Nbd,
                                                     (float*)c->tab_mem, (float*)c->tab_bd, c->pts_mem,
                                                     c->pts_bd, c->dstatus);
    k_lumped_mass<<<(q.N + B - 1) / B, B, 0, c->stream>>>(q.nu, q.nv, q.vb0, q.SvG, q.cp0, N, c->rest, q.rho,
                                                           c->mass);
  }
  e = cudaGetLastError();
  if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
  return e;
}

// Recomputes the lumped masses of patch p (after a density change).
cudaError_t launch_lumped_mass_patch(bsc_ctx* c, int p) {
  const PatchDev& q = c->hpd[p];
  BSC_COUNT(c, 1);
  k_lumped_mass<<<(q.N + 127) / 128, 128, 0, c->stream>>>(q.nu, q.nv, q.vb0, q.SvG, q.cp0, c->N, c->rest, q.rho,
                                                          c->mass);
  return cudaGetLastError();
}

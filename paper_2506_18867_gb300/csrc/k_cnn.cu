// K7 / K8: the learned preconditioner - a 4-layer 3x3 convolutional network on
// the control grid - and the flexible CG that uses it.
//
// Network (channels 16 -> 32 -> 32 -> 32 -> 16, ReLU after the first three
// layers, zero padding at the grid border).  Input features per control
// point, made dimensionless so that P(a r) = a P(r) for a > 0:
//   r / s,  (D^-1 r) d / s,  the six entries of the diagonal 3x3 block / d,
//   the pin mask, and a constant 1 (14 channels, 2 zero pad)
// with s = RMS of r over the grid and d = mean diagonal entry of K.  The
// preconditioned vector is z = D^-1 r + (s / d) y, y the first three output
// channels (zero at pinned points): with zero weights the network reproduces
// the block-Jacobi preconditioner, and training learns a correction.
//
// Every convolution is an implicit GEMM on the tensor cores (tcgen05, BF16
// operands, FP32 accumulator in TMEM): a CTA takes 128 consecutive pixels
// (rows of A), gathers the nine shifted input tiles (9 x 128 x C_in BF16) and
// the weights (C_out x 9 C_in) into shared memory in the K-major no-swizzle
// layout, and one thread issues 9 C_in / 16 MMAs of M = 128, N = C_out,
// K = 16 into a TMEM accumulator; the epilogue reads the accumulator back
// (tcgen05.ld), adds the bias and applies the activation.  The backward pass
// of the data (gradient w.r.t. a layer's input) is the same kernel on the
// flipped, transposed weights with the ReLU derivative as epilogue; the
// weight gradients are reductions over pixels on the CUDA cores.
#include <math.h>
#include <stdio.h>
#include <stdlib.h>
#include <string.h>

#include <cuda_bf16.h>

#include <algorithm>
#include <vector>

#include "bsc_internal.cuh"
#include "tc05.cuh"

cudaError_t launch_block_jacobi(bsc_ctx* c, const void* K, void* Dinv);

namespace {

constexpr int NL = 4;
constexpr int CH_IN[NL] = {16, 32, 32, 32};
constexpr int CH_OUT[NL] = {32, 32, 32, 16};
constexpr int TILE = 128;
constexpr long long WAIT_LIMIT = 1ll << 25;

constexpr int w_count(int l) { return 9 * CH_IN[l] * CH_OUT[l]; }
constexpr int p_count(int l) { return w_count(l) + CH_OUT[l]; }
constexpr int param_total() { return p_count(0) + p_count(1) + p_count(2) + p_count(3); }

// ---------------------------------------------------------------------------
// convolution on the tensor cores
// ---------------------------------------------------------------------------
enum ConvMode { CONV_RELU_BF16 = 0, CONV_LINEAR_F32 = 1, CONV_MASK_BF16 = 2 };

struct ConvArgs {
  int nu, nv, P;
  const __nv_bfloat16* X;      // [P][CIN]
  const uint8_t* Wb;           // COUT x 9 CIN, BF16, K-major no-swizzle core layout
  const float* bias;           // [COUT] (modes 0, 1)
  const __nv_bfloat16* mask;   // [P][COUT] forward activation whose sign gates the gradient (mode 2)
  void* Y;                     // [P][COUT] BF16 (modes 0, 2) or [P][4] FP32 (mode 1: channels 0..2)
  int flip;                    // 1: gather at -offset (the transposed convolution)
  int* status;
};

template <int CIN, int COUT>
constexpr size_t conv_smem() {
  return (size_t)9 * TILE * CIN * 2 + (size_t)COUT * 9 * CIN * 2;
}

template <int CIN, int COUT, int MODE>
__global__ void __launch_bounds__(TILE) k_conv(ConvArgs a) {
  extern __shared__ __align__(1024) uint8_t smem[];
  constexpr int KT = 9 * CIN;
  constexpr uint32_t A_TAP = TILE * CIN * 2;
  constexpr int CH8 = CIN / 8;
  constexpr uint32_t IDESC = tc05::idesc_bf16_f32(TILE, COUT);
  uint8_t* sA = smem;
  uint8_t* sB = smem + 9 * A_TAP;
  __shared__ uint64_t mbar;
  __shared__ uint32_t tmem_base;
  const int tid = threadIdx.x, warp = tid >> 5;

  // weights once per CTA
  for (int i = tid; i < COUT * KT * 2 / 16; i += TILE) tc05::cp_async16(sB + 16 * i, a.Wb + 16 * i, true);
  if (warp == 0) {
    tc05::tmem_alloc(&tmem_base, 32);
    tc05::tmem_relinquish();
  }
  if (tid == 0) {
    tc05::mbar_init(&mbar, 1);
    tc05::fence_mbar_init();
  }
  tc05::fence_before_sync();
  __syncthreads();
  tc05::fence_after_sync();
  const uint32_t tmem = tmem_base;
  uint32_t phase = 0;
  const int ntiles = (a.P + TILE - 1) / TILE;
  const int sgn = a.flip ? -1 : 1;
  bool failed = false;
  for (int tile = blockIdx.x; tile < ntiles && !failed; tile += gridDim.x) {
    const int p0 = tile * TILE;
    // gather the nine shifted tiles (zero outside the grid)
    for (int cidx = tid; cidx < 9 * TILE * CH8; cidx += TILE) {
      const int tap = cidx / (TILE * CH8), rem = cidx - tap * TILE * CH8;
      const int m = rem / CH8, kc = rem - m * CH8;
      const int p = p0 + m;
      const int dy = sgn * (tap / 3 - 1), dx = sgn * (tap % 3 - 1);
      bool valid = p < a.P;
      int q = 0;
      if (valid) {
        const int i = p % a.nu + dx, j = p / a.nu + dy;
        valid = i >= 0 && i < a.nu && j >= 0 && j < a.nv;
        q = j * a.nu + i;
      }
      const __nv_bfloat16* src = valid ? a.X + (size_t)q * CIN + kc * 8 : a.X;
      tc05::cp_async16(sA + tap * A_TAP + tc05::kmajor_offset(m, kc * 8, CIN), src, valid);
    }
    tc05::cp_async_wait_all();
    tc05::fence_proxy_async_smem();
    __syncthreads();
    if (tid == 0) {
      tc05::fence_after_sync();
      const uint32_t a0 = tc05::smem_u32(sA), b0 = tc05::smem_u32(sB);
#pragma unroll
      for (int tap = 0; tap < 9; ++tap)
#pragma unroll
        for (int k16 = 0; k16 < CIN / 16; ++k16) {
          const uint64_t ad = tc05::smem_desc(a0 + tap * A_TAP + k16 * 256, 128, CH8 * 128);
          const uint64_t bd = tc05::smem_desc(b0 + (tap * CH8 + 2 * k16) * 128, 128, (KT / 8) * 128);
          tc05::mma_bf16(tmem, ad, bd, IDESC, (tap | k16) != 0);
        }
      tc05::mma_commit(&mbar);
    }
    const bool ok = tc05::mbar_wait(&mbar, phase, WAIT_LIMIT);
    failed = __syncthreads_or(!ok) != 0;
    if (failed) {
      if (tid == 0) atomicOr(a.status, BSC_STATUS_TIMEOUT_FLAG);
      break;
    }
    phase ^= 1u;
    tc05::fence_after_sync();
    // epilogue: thread tid holds accumulator row tid (pixel p0 + tid)
    float v[COUT];
#pragma unroll
    for (int h = 0; h < COUT / 16; ++h) {
      float t16[16];
      tc05::tmem_ld16(tmem + ((uint32_t)(warp * 32) << 16) + (uint32_t)(16 * h), t16);
      tc05::tmem_ld_wait();
#pragma unroll
      for (int i = 0; i < 16; ++i) v[16 * h + i] = t16[i];
    }
    const int p = p0 + tid;
    if (p < a.P) {
      if (MODE == CONV_LINEAR_F32) {
        float4 o;
        o.x = v[0] + __ldg(a.bias + 0);
        o.y = v[1] + __ldg(a.bias + 1);
        o.z = v[2] + __ldg(a.bias + 2);
        o.w = 0.0f;
        reinterpret_cast<float4*>(a.Y)[p] = o;
      } else {
        __align__(16) __nv_bfloat16 out[COUT];
        if (MODE == CONV_RELU_BF16) {
#pragma unroll
          for (int c = 0; c < COUT; ++c) out[c] = __float2bfloat16_rn(fmaxf(v[c] + __ldg(a.bias + c), 0.0f));
        } else {
          __align__(16) __nv_bfloat16 mk[COUT];
          const uint4* ms = reinterpret_cast<const uint4*>(a.mask + (size_t)p * COUT);
#pragma unroll
          for (int c = 0; c < COUT / 8; ++c) reinterpret_cast<uint4*>(mk)[c] = ms[c];
#pragma unroll
          for (int c = 0; c < COUT; ++c)
            out[c] = __float2bfloat16_rn(__bfloat162float(mk[c]) > 0.0f ? v[c] : 0.0f);
        }
        uint4* dst = reinterpret_cast<uint4*>(reinterpret_cast<__nv_bfloat16*>(a.Y) + (size_t)p * COUT);
#pragma unroll
        for (int c = 0; c < COUT / 8; ++c) dst[c] = reinterpret_cast<const uint4*>(out)[c];
      }
    }
    tc05::fence_before_sync();
    __syncthreads();  // the next tile's MMAs overwrite the accumulator and the A tiles
  }
  if (failed) {
    // give an MMA still in flight a bounded chance to finish before the
    // accumulator is released
    tc05::mbar_wait(&mbar, phase, WAIT_LIMIT);
  }
  tc05::fence_before_sync();
  __syncthreads();
  if (warp == 0) tc05::tmem_dealloc(tmem, 32);
}

// ---------------------------------------------------------------------------
// features, output, loss
// ---------------------------------------------------------------------------

// Per control point: diagonal block of K and its block-Jacobi inverse are
// given; writes the 14 features (BF16, 16 channels).  s = RMS of r, d = mean
// diagonal entry (both on the device).
__global__ void k_features(int P, const float* __restrict__ K, const float* __restrict__ Dinv,
                           const uint8_t* __restrict__ pinned, const float* __restrict__ r,
                           const double* __restrict__ scales, __nv_bfloat16* __restrict__ X0) {
  const int p = blockIdx.x * blockDim.x + threadIdx.x;
  if (p >= P) return;
  // s = 0 only for r = 0, whose features are then all zero
  const float is = scales[0] > 0.0 ? (float)(1.0 / scales[0]) : 0.0f, d = (float)scales[1],
              id = (float)(1.0 / scales[1]);
  float rr[3], zr[3], f[16];
#pragma unroll
  for (int c = 0; c < 3; ++c) rr[c] = r[(size_t)c * P + p];
#pragma unroll
  for (int c = 0; c < 3; ++c)
    zr[c] = Dinv[(size_t)(3 * c) * P + p] * rr[0] + Dinv[(size_t)(3 * c + 1) * P + p] * rr[1] +
            Dinv[(size_t)(3 * c + 2) * P + p] * rr[2];
  const int slot = 12;  // du = dv = 0
  const float k00 = K[(size_t)(slot * 9 + 0) * P + p], k01 = K[(size_t)(slot * 9 + 1) * P + p],
              k02 = K[(size_t)(slot * 9 + 2) * P + p], k11 = K[(size_t)(slot * 9 + 4) * P + p],
              k12 = K[(size_t)(slot * 9 + 5) * P + p], k22 = K[(size_t)(slot * 9 + 8) * P + p];
#pragma unroll
  for (int c = 0; c < 3; ++c) {
    f[c] = rr[c] * is;
    f[3 + c] = zr[c] * d * is;
  }
  f[6] = k00 * id; f[7] = k01 * id; f[8] = k02 * id; f[9] = k11 * id; f[10] = k12 * id; f[11] = k22 * id;
  f[12] = pinned[p] ? 1.0f : 0.0f;
  f[13] = 1.0f;
  f[14] = f[15] = 0.0f;
  __align__(16) __nv_bfloat16 o[16];
#pragma unroll
  for (int c = 0; c < 16; ++c) o[c] = __float2bfloat16_rn(f[c]);
  uint4* dst = reinterpret_cast<uint4*>(X0 + (size_t)p * 16);
  dst[0] = reinterpret_cast<const uint4*>(o)[0];
  dst[1] = reinterpret_cast<const uint4*>(o)[1];
}

// z = D^-1 r + (s / d) y (zero at pinned points).
__global__ void k_combine(int P, const float* __restrict__ Dinv, const uint8_t* __restrict__ pinned,
                          const float* __restrict__ r, const float4* __restrict__ y,
                          const double* __restrict__ scales, float* __restrict__ z) {
  const int p = blockIdx.x * blockDim.x + threadIdx.x;
  if (p >= P) return;
  if (pinned[p]) {
    z[p] = z[P + p] = z[2 * (size_t)P + p] = 0.0f;
    return;
  }
  const float sd = (float)(scales[0] / scales[1]);
  const float4 yy = y[p];
  const float yv[3] = {yy.x, yy.y, yy.z};
  float rr[3];
#pragma unroll
  for (int c = 0; c < 3; ++c) rr[c] = r[(size_t)c * P + p];
#pragma unroll
  for (int c = 0; c < 3; ++c)
    z[(size_t)c * P + p] = Dinv[(size_t)(3 * c) * P + p] * rr[0] + Dinv[(size_t)(3 * c + 1) * P + p] * rr[1] +
                           Dinv[(size_t)(3 * c + 2) * P + p] * rr[2] + sd * yv[c];
}

template <int BLOCK>
__device__ __forceinline__ double block_sum_all(double v, double* sm) {
  const double s = block_sum<BLOCK>(v, sm);
  __shared__ double b;
  if (threadIdx.x == 0) b = s;
  __syncthreads();
  return b;
}

constexpr int RB = 256;

// partial[blk] = sum over the block's slice of f(i); generic dot products
// of 3-plane vectors (a . b), fixed assignment and order.
__global__ void __launch_bounds__(RB) k_dot_partials(int n, const float* __restrict__ a, const float* __restrict__ b,
                                                     double* __restrict__ partial) {
  __shared__ double sm[RB / 32];
  double acc = 0.0;
  for (int k = blockIdx.x * RB + threadIdx.x; k < n; k += gridDim.x * RB) acc += (double)a[k] * (double)b[k];
  const double t = block_sum<RB>(acc, sm);
  if (threadIdx.x == 0) partial[blockIdx.x] = t;
}

// out[slot] = sum of partial[0..n) (one block), optionally followed by
// out[slot] = sqrt(out / count) (RMS)
__global__ void __launch_bounds__(RB) k_sum_to(int n, const double* __restrict__ partial, double* __restrict__ out,
                                               int slot, double rms_count) {
  __shared__ double sm[RB / 32];
  double acc = 0.0;
  for (int k = threadIdx.x; k < n; k += RB) acc += partial[k];
  const double t = block_sum<RB>(acc, sm);
  if (threadIdx.x == 0) out[slot] = rms_count > 0.0 ? sqrt(t / rms_count) : t;
}

// Mean diagonal entry of K (over the non-pinned points) into scales[1].
__global__ void __launch_bounds__(RB) k_diag_partials(int P, const float* __restrict__ K,
                                                      const uint8_t* __restrict__ pinned,
                                                      double* __restrict__ partial) {
  __shared__ double sm[RB / 32];
  double acc = 0.0, cnt = 0.0;
  for (int p = blockIdx.x * RB + threadIdx.x; p < P; p += gridDim.x * RB) {
    if (pinned[p]) continue;
    acc += (double)K[(size_t)(12 * 9 + 0) * P + p] + (double)K[(size_t)(12 * 9 + 4) * P + p] +
           (double)K[(size_t)(12 * 9 + 8) * P + p];
    cnt += 3.0;
  }
  const double t = block_sum<RB>(acc, sm);
  const double u = block_sum<RB>(cnt, sm);
  if (threadIdx.x == 0) {
    partial[blockIdx.x] = t;
    partial[gridDim.x + blockIdx.x] = u;
  }
}

__global__ void __launch_bounds__(RB) k_diag_mean(int n, const double* __restrict__ partial,
                                                  double* __restrict__ scales) {
  __shared__ double sm[RB / 32];
  double a = 0.0, b = 0.0;
  for (int k = threadIdx.x; k < n; k += RB) {
    a += partial[k];
    b += partial[n + k];
  }
  const double t = block_sum<RB>(a, sm);
  const double u = block_sum<RB>(b, sm);
  if (threadIdx.x == 0) scales[1] = u > 0.0 ? t / u : 1.0;
}

}  // namespace

namespace {

// ---------------------------------------------------------------------------
// backward: weight gradients (CUDA cores), loss, optimizer, weight layouts
// ---------------------------------------------------------------------------
constexpr int WG_CHUNK = 1024;  // pixels per CTA of the weight-gradient reduction
constexpr int WG_PB = 16;       // pixels staged per step

// partial[blk][o] = sum over the block's pixels of X[p + off(tap)][ci] dY[p][co]
// (o = (tap CIN + ci) COUT + co), then the bias gradient sum dY[p][co].
template <int CIN, int COUT>
__global__ void __launch_bounds__(256) k_wgrad(int nu, int nv, int P, const __nv_bfloat16* __restrict__ X,
                                               const __nv_bfloat16* __restrict__ dY, float* __restrict__ partial) {
  constexpr int NO = 9 * CIN * COUT, PER = (NO + 255) / 256;
  __shared__ float sx[WG_PB][9 * CIN];
  __shared__ float sy[WG_PB][COUT];
  const int tid = threadIdx.x;
  float acc[PER];
#pragma unroll
  for (int k = 0; k < PER; ++k) acc[k] = 0.0f;
  float bacc = 0.0f;
  const int lo = blockIdx.x * WG_CHUNK, hi = min(P, lo + WG_CHUNK);
  for (int base = lo; base < hi; base += WG_PB) {
    for (int idx = tid; idx < WG_PB * 9 * CIN; idx += 256) {
      const int pix = idx / (9 * CIN), rem = idx - pix * 9 * CIN, tap = rem / CIN, ci = rem - tap * CIN;
      const int p = base + pix;
      float v = 0.0f;
      if (p < hi) {
        const int i = p % nu + (tap % 3 - 1), j = p / nu + (tap / 3 - 1);
        if (i >= 0 && i < nu && j >= 0 && j < nv) v = __bfloat162float(X[(size_t)(j * nu + i) * CIN + ci]);
      }
      sx[pix][rem] = v;
    }
    for (int idx = tid; idx < WG_PB * COUT; idx += 256) {
      const int pix = idx / COUT, co = idx - pix * COUT, p = base + pix;
      sy[pix][co] = p < hi ? __bfloat162float(dY[(size_t)p * COUT + co]) : 0.0f;
    }
    __syncthreads();
#pragma unroll 4
    for (int pix = 0; pix < WG_PB; ++pix) {
#pragma unroll
      for (int k = 0; k < PER; ++k) {
        const int o = tid + 256 * k;
        if (o < NO) acc[k] += sx[pix][o / COUT] * sy[pix][o % COUT];
      }
      if (tid < COUT) bacc += sy[pix][tid];
    }
    __syncthreads();
  }
  float* out = partial + (size_t)blockIdx.x * (NO + COUT);
#pragma unroll
  for (int k = 0; k < PER; ++k) {
    const int o = tid + 256 * k;
    if (o < NO) out[o] = acc[k];
  }
  if (tid < COUT) out[NO + tid] = bacc;
}

// grad[o] = sum over blocks of partial[b][o], in block order.
__global__ void k_wgrad_reduce(int nblk, int NO1, const float* __restrict__ partial, float* __restrict__ grad) {
  const int o = blockIdx.x * blockDim.x + threadIdx.x;
  if (o >= NO1) return;
  double s = 0.0;
  for (int b = 0; b < nblk; ++b) s += (double)partial[(size_t)b * NO1 + o];
  grad[o] = (float)s;
}

// e = z - x*, in place of z's copy; pinned rows are zero in both.
__global__ void k_sub(int n, const float* __restrict__ a, const float* __restrict__ b, float* __restrict__ out) {
  const int k = blockIdx.x * blockDim.x + threadIdx.x;
  if (k < n) out[k] = a[k] - b[k];
}

// dy4[p][c] = (s / d) * 2 (K e)[c][p] / (x*^T K x*) for c < 3, zero elsewhere and at pins.
__global__ void k_dy4(int P, const uint8_t* __restrict__ pinned, const float* __restrict__ Ke,
                      const double* __restrict__ scales, const double* __restrict__ dsc,
                      __nv_bfloat16* __restrict__ dy4) {
  const int p = blockIdx.x * blockDim.x + threadIdx.x;
  if (p >= P) return;
  const double f = 2.0 * (scales[0] / scales[1]) / dsc[1];
  __align__(16) __nv_bfloat16 o[16];
#pragma unroll
  for (int c = 0; c < 16; ++c) o[c] = __float2bfloat16_rn(0.0f);
  if (!pinned[p]) {
#pragma unroll
    for (int c = 0; c < 3; ++c) o[c] = __float2bfloat16_rn((float)(f * (double)Ke[(size_t)c * P + p]));
  }
  uint4* dst = reinterpret_cast<uint4*>(dy4 + (size_t)p * 16);
  dst[0] = reinterpret_cast<const uint4*>(o)[0];
  dst[1] = reinterpret_cast<const uint4*>(o)[1];
}

// Adam on the FP32 master parameters.
__global__ void k_adam(int n, float* __restrict__ w, const float* __restrict__ g, float* __restrict__ m,
                       float* __restrict__ v, float lr, float b1, float b2, float eps, float c1, float c2) {
  const int k = blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= n) return;
  const float gk = g[k];
  const float mk = b1 * m[k] + (1.0f - b1) * gk, vk = b2 * v[k] + (1.0f - b2) * gk * gk;
  m[k] = mk;
  v[k] = vk;
  w[k] -= lr * (mk / c1) / (sqrtf(vk / c2) + eps);
}

// BF16 weights of layer l in the two operand layouts: forward B[co][tap CIN +
// ci] and transposed B'[ci][tap COUT + co] = W[tap][ci][co].  The transposed
// convolution gathers its input at the negated tap offset (flip = 1): input
// pixel q fed output q - off(tap) through W[tap].
__global__ void k_layout(int CIN, int COUT, const float* __restrict__ W, uint8_t* __restrict__ Wb,
                         uint8_t* __restrict__ Wt) {
  const int o = blockIdx.x * blockDim.x + threadIdx.x;
  if (o >= 9 * CIN * COUT) return;
  const int tap = o / (CIN * COUT), rem = o - tap * CIN * COUT, ci = rem / COUT, co = rem - ci * COUT;
  const __nv_bfloat16 w = __float2bfloat16_rn(W[o]);
  *reinterpret_cast<__nv_bfloat16*>(Wb + tc05::kmajor_offset(co, tap * CIN + ci, 9 * CIN)) = w;
  if (Wt) *reinterpret_cast<__nv_bfloat16*>(Wt + tc05::kmajor_offset(ci, tap * COUT + co, 9 * COUT)) = w;
}

// ---- flexible CG pieces ----------------------------------------------------
// x += a p, r -= a q with a = dsc[0] / dsc[1] (p.r / p.q)
__global__ void k_fcg_xr(int n, const double* __restrict__ dsc, const float* __restrict__ p,
                         const float* __restrict__ q, float* __restrict__ x, float* __restrict__ r) {
  const int k = blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= n) return;
  const float a = (float)(dsc[0] / dsc[1]);
  x[k] += a * p[k];
  r[k] -= a * q[k];
}
// p = z + b p with b = -dsc[2] / dsc[1] (-(z.q) / p.q)
__global__ void k_fcg_p(int n, const double* __restrict__ dsc, const float* __restrict__ z, float* __restrict__ p) {
  const int k = blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= n) return;
  const float b = (float)(-dsc[2] / dsc[1]);
  p[k] = z[k] + b * p[k];
}
__global__ void k_copy_f(int n, const float* __restrict__ a, float* __restrict__ b) {
  const int k = blockIdx.x * blockDim.x + threadIdx.x;
  if (k < n) b[k] = a[k];
}
__global__ void k_add_f(int n, const float* __restrict__ a, float* __restrict__ b) {
  const int k = blockIdx.x * blockDim.x + threadIdx.x;
  if (k < n) b[k] += a[k];
}

}  // namespace

// ===========================================================================
// the CNN object and its C ABI
// ===========================================================================
struct bsc_cnn {
  bsc_ctx* c;
  int P, nu, nv;
  int off[NL];                 // parameter offset of each layer (weights, then bias)
  float* params;               // FP32 master parameters
  float* grads;
  float* adam_m;
  float* adam_v;
  int adam_t;
  uint8_t* Wb[NL];
  uint8_t* Wt[NL];
  __nv_bfloat16* X0;
  __nv_bfloat16* act[3];       // outputs of layers 1..3
  __nv_bfloat16* g0;           // gradient buffers
  __nv_bfloat16* g1;
  __nv_bfloat16* dy4;
  float4* y4;
  float* Dinv;
  const float* K;
  double* scales;              // [0] RMS of the residual, [1] mean diagonal entry
  double* dsc;                 // device scalars
  double* hsc;                 // pinned host scalars
  double* red;                 // reduction partials
  float* wpart;                // weight-gradient partials
  float* vec[6];               // FCG: r, z, p, q, e, spare (3 planes of P)
  int conv_grid;
  int red_grid;
};

namespace {

bsc_status cnn_fail(bsc_cnn* n, bsc_status st, const char* msg) {
  snprintf(n->c->err, sizeof(n->c->err), "%s", msg);
  return st;
}

#define CKN(call, where)                                                           \
  do {                                                                             \
    cudaError_t e_ = (call);                                                       \
    if (e_ != cudaSuccess) {                                                       \
      char b_[256];                                                                \
      snprintf(b_, sizeof(b_), "%s: %s", where, cudaGetErrorString(e_));           \
      return cnn_fail(n, e_ == cudaErrorMemoryAllocation ? BSC_ERR_OOM : BSC_ERR_CUDA, b_); \
    }                                                                              \
  } while (0)

template <int CIN, int COUT, int MODE>
cudaError_t conv(bsc_cnn* n, const __nv_bfloat16* X, const uint8_t* W, const float* bias,
                 const __nv_bfloat16* mask, void* Y, int flip) {
  ConvArgs a{n->nu, n->nv, n->P, X, W, bias, mask, Y, flip, n->c->dstatus};
  BSC_COUNT(n->c, 1);
  k_conv<CIN, COUT, MODE><<<n->conv_grid, TILE, conv_smem<CIN, COUT>(), n->c->stream>>>(a);
  return cudaGetLastError();
}

template <int CIN, int COUT, int MODE>
cudaError_t conv_setup() {
  return cudaFuncSetAttribute(k_conv<CIN, COUT, MODE>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                              (int)conv_smem<CIN, COUT>());
}

// s = RMS of r into scales[0]
cudaError_t rms(bsc_cnn* n, const float* r) {
  BSC_COUNT(n->c, 2);
  k_dot_partials<<<n->red_grid, RB, 0, n->c->stream>>>(3 * n->P, r, r, n->red);
  k_sum_to<<<1, RB, 0, n->c->stream>>>(n->red_grid, n->red, n->scales, 0, 3.0 * n->P);
  return cudaGetLastError();
}

cudaError_t dot(bsc_cnn* n, const float* a, const float* b, double* out_slot) {
  BSC_COUNT(n->c, 2);
  k_dot_partials<<<n->red_grid, RB, 0, n->c->stream>>>(3 * n->P, a, b, n->red);
  k_sum_to<<<1, RB, 0, n->c->stream>>>(n->red_grid, n->red, out_slot, 0, 0.0);
  return cudaGetLastError();
}

// z = P(r) for the prepared matrix (activations kept for the backward pass)
cudaError_t cnn_forward(bsc_cnn* n, const float* r, float* z) {
  cudaError_t e;
  const int P = n->P, B = 256, G = (P + B - 1) / B;
  if ((e = rms(n, r)) != cudaSuccess) return e;
  BSC_COUNT(n->c, 2);
  k_features<<<G, B, 0, n->c->stream>>>(P, n->K, n->Dinv, n->c->pinned, r, n->scales, n->X0);
  if ((e = cudaGetLastError()) != cudaSuccess) return e;
  const float* p = n->params;
  if ((e = conv<16, 32, CONV_RELU_BF16>(n, n->X0, n->Wb[0], p + n->off[0] + w_count(0), nullptr, n->act[0], 0)))
    return e;
  if ((e = conv<32, 32, CONV_RELU_BF16>(n, n->act[0], n->Wb[1], p + n->off[1] + w_count(1), nullptr, n->act[1], 0)))
    return e;
  if ((e = conv<32, 32, CONV_RELU_BF16>(n, n->act[1], n->Wb[2], p + n->off[2] + w_count(2), nullptr, n->act[2], 0)))
    return e;
  if ((e = conv<32, 16, CONV_LINEAR_F32>(n, n->act[2], n->Wb[3], p + n->off[3] + w_count(3), nullptr, n->y4, 0)))
    return e;
  k_combine<<<G, B, 0, n->c->stream>>>(P, n->Dinv, n->c->pinned, r, n->y4, n->scales, z);
  return cudaGetLastError();
}

template <int CIN, int COUT>
cudaError_t wgrad(bsc_cnn* n, int l, const __nv_bfloat16* X, const __nv_bfloat16* dY) {
  const int nblk = (n->P + WG_CHUNK - 1) / WG_CHUNK, NO1 = 9 * CIN * COUT + COUT;
  BSC_COUNT(n->c, 2);
  k_wgrad<CIN, COUT><<<nblk, 256, 0, n->c->stream>>>(n->nu, n->nv, n->P, X, dY, n->wpart);
  k_wgrad_reduce<<<(NO1 + 255) / 256, 256, 0, n->c->stream>>>(nblk, NO1, n->wpart, n->grads + n->off[l]);
  return cudaGetLastError();
}

// loss = (z - x*)^T K (z - x*) / x*^T K x* and the parameter gradient.
cudaError_t cnn_loss_grad(bsc_cnn* n, const float* r, const float* xs) {
  cudaError_t e;
  const int P = n->P, N3 = 3 * P, B = 256, G3 = (N3 + B - 1) / B, G = (P + B - 1) / B;
  float *z = n->vec[1], *ev = n->vec[4], *Ke = n->vec[3], *Kx = n->vec[5];
  if ((e = cnn_forward(n, r, z)) != cudaSuccess) return e;
  BSC_COUNT(n->c, 1);
  k_sub<<<G3, B, 0, n->c->stream>>>(N3, z, xs, ev);
  if ((e = launch_spmv(n->c, n->K, ev, Ke)) != cudaSuccess) return e;
  if ((e = launch_spmv(n->c, n->K, xs, Kx)) != cudaSuccess) return e;
  if ((e = dot(n, ev, Ke, n->dsc + 0)) != cudaSuccess) return e;  // e^T K e
  if ((e = dot(n, xs, Kx, n->dsc + 1)) != cudaSuccess) return e;  // x*^T K x*
  BSC_COUNT(n->c, 1);
  k_dy4<<<G, B, 0, n->c->stream>>>(P, n->c->pinned, Ke, n->scales, n->dsc, n->dy4);
  if ((e = cudaGetLastError()) != cudaSuccess) return e;
  // layer 4
  if ((e = wgrad<32, 16>(n, 3, n->act[2], n->dy4)) != cudaSuccess) return e;
  if ((e = conv<16, 32, CONV_MASK_BF16>(n, n->dy4, n->Wt[3], nullptr, n->act[2], n->g0, 1)) != cudaSuccess) return e;
  // layer 3
  if ((e = wgrad<32, 32>(n, 2, n->act[1], n->g0)) != cudaSuccess) return e;
  if ((e = conv<32, 32, CONV_MASK_BF16>(n, n->g0, n->Wt[2], nullptr, n->act[1], n->g1, 1)) != cudaSuccess) return e;
  // layer 2
  if ((e = wgrad<32, 32>(n, 1, n->act[0], n->g1)) != cudaSuccess) return e;
  if ((e = conv<32, 32, CONV_MASK_BF16>(n, n->g1, n->Wt[1], nullptr, n->act[0], n->g0, 1)) != cudaSuccess) return e;
  // layer 1
  return wgrad<16, 32>(n, 0, n->X0, n->g0);
}

cudaError_t relayout(bsc_cnn* n) {
  for (int l = 0; l < NL; ++l) {
    BSC_COUNT(n->c, 1);
    const int cnt = w_count(l);
    k_layout<<<(cnt + 255) / 256, 256, 0, n->c->stream>>>(CH_IN[l], CH_OUT[l], n->params + n->off[l], n->Wb[l],
                                                           l > 0 ? n->Wt[l] : nullptr);
  }
  return cudaGetLastError();
}

bsc_status cnn_sync(bsc_cnn* n, const char* where) {
  CKN(cudaStreamSynchronize(n->c->stream), where);
  int st = 0;
  CKN(cudaMemcpy(&st, n->c->dstatus, sizeof(int), cudaMemcpyDeviceToHost), where);
  if (st) {
    CKN(cudaMemset(n->c->dstatus, 0, sizeof(int)), where);
    char b[256];
    snprintf(b, sizeof(b), "%s: device status flags %d (%s)", where, st,
             (st & BSC_STATUS_TIMEOUT_FLAG) ? "a bounded device wait ran out" : "non-finite value");
    return cnn_fail(n, (st & BSC_STATUS_TIMEOUT_FLAG) ? BSC_ERR_TIMEOUT : BSC_ERR_NUMERIC, b);
  }
  return BSC_OK;
}

void cnn_free(bsc_cnn* n) {
  if (!n) return;
  void* ptrs[] = {n->params, n->grads, n->adam_m, n->adam_v, n->X0, n->act[0], n->act[1], n->act[2], n->g0,
                  n->g1, n->dy4, n->y4, n->Dinv, n->scales, n->dsc, n->red, n->wpart};
  for (void* p : ptrs)
    if (p) cudaFree(p);
  for (int l = 0; l < NL; ++l) {
    if (n->Wb[l]) cudaFree(n->Wb[l]);
    if (n->Wt[l]) cudaFree(n->Wt[l]);
  }
  for (float* v : n->vec)
    if (v) cudaFree(v);
  if (n->hsc) cudaFreeHost(n->hsc);
  free(n);
}

}  // namespace

extern "C" {

int bsc_cnn_param_count(void) { return param_total(); }

bsc_status bsc_cnn_create(bsc_ctx* c, bsc_cnn** out) {
  if (!out) return BSC_ERR_INVALID_ARG;
  *out = nullptr;
  if (!c) return BSC_ERR_INVALID_ARG;
  if (c->P != 1 || c->precision != BSC_FP32) {
    snprintf(c->err, sizeof(c->err), "bsc_cnn_create: the learned preconditioner needs a single-patch FP32 context");
    return BSC_ERR_INVALID_ARG;
  }
  bsc_cnn* n = (bsc_cnn*)calloc(1, sizeof(bsc_cnn));
  if (!n) return BSC_ERR_OOM;
  n->c = c;
  n->P = c->N;
  n->nu = c->nu;
  n->nv = c->nv;
  int o = 0;
  for (int l = 0; l < NL; ++l) {
    n->off[l] = o;
    o += p_count(l);
  }
  const size_t P = (size_t)n->P, NP = (size_t)param_total();
  cudaError_t e = cudaSuccess;
#define CA(ptr, bytes) \
  if (e == cudaSuccess) e = cudaMalloc((void**)&(ptr), (bytes))
  CA(n->params, NP * 4);
  CA(n->grads, NP * 4);
  CA(n->adam_m, NP * 4);
  CA(n->adam_v, NP * 4);
  for (int l = 0; l < NL; ++l) {
    CA(n->Wb[l], (size_t)w_count(l) * 2);
    if (l > 0) CA(n->Wt[l], (size_t)w_count(l) * 2);
  }
  CA(n->X0, P * 16 * 2);
  for (int k = 0; k < 3; ++k) CA(n->act[k], P * 32 * 2);
  CA(n->g0, P * 32 * 2);
  CA(n->g1, P * 32 * 2);
  CA(n->dy4, P * 16 * 2);
  CA(n->y4, P * 16);
  CA(n->Dinv, P * 9 * 4);
  CA(n->scales, 8 * sizeof(double));
  CA(n->dsc, 16 * sizeof(double));
  n->red_grid = 2 * c->num_sms;
  CA(n->red, 4 * (size_t)n->red_grid * sizeof(double));
  CA(n->wpart, (size_t)((n->P + WG_CHUNK - 1) / WG_CHUNK) * (9 * 32 * 32 + 32) * 4);
  for (int k = 0; k < 6; ++k) CA(n->vec[k], 3 * P * 4);
#undef CA
  if (e == cudaSuccess) e = cudaMallocHost((void**)&n->hsc, 16 * sizeof(double));
  if (e == cudaSuccess) e = cudaMemset(n->params, 0, NP * 4);
  if (e == cudaSuccess) e = cudaMemset(n->adam_m, 0, NP * 4);
  if (e == cudaSuccess) e = cudaMemset(n->adam_v, 0, NP * 4);
  if (e == cudaSuccess) e = cudaMemset(n->grads, 0, NP * 4);
  if (e == cudaSuccess) e = conv_setup<16, 32, CONV_RELU_BF16>();
  if (e == cudaSuccess) e = conv_setup<32, 32, CONV_RELU_BF16>();
  if (e == cudaSuccess) e = conv_setup<32, 16, CONV_LINEAR_F32>();
  if (e == cudaSuccess) e = conv_setup<16, 32, CONV_MASK_BF16>();
  if (e == cudaSuccess) e = conv_setup<32, 32, CONV_MASK_BF16>();
  if (e != cudaSuccess) {
    snprintf(c->err, sizeof(c->err), "bsc_cnn_create: %s", cudaGetErrorString(e));
    cnn_free(n);
    return e == cudaErrorMemoryAllocation ? BSC_ERR_OOM : BSC_ERR_CUDA;
  }
  // persistent conv CTAs: as many as fit (two per SM with the 92 KB tiles)
  int per = 0;
  cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, k_conv<32, 32, CONV_RELU_BF16>, TILE,
                                                conv_smem<32, 32>());
  per = per < 1 ? 1 : (per > 4 ? 4 : per);
  const int tiles = (n->P + TILE - 1) / TILE;
  n->conv_grid = std::min(tiles, per * c->num_sms);
  if (relayout(n) != cudaSuccess || cudaStreamSynchronize(c->stream) != cudaSuccess) {
    snprintf(c->err, sizeof(c->err), "bsc_cnn_create: weight layout failed");
    cnn_free(n);
    return BSC_ERR_CUDA;
  }
  *out = n;
  return BSC_OK;
}

void bsc_cnn_destroy(bsc_cnn* n) {
  if (!n) return;
  cudaStreamSynchronize(n->c->stream);
  cnn_free(n);
}

bsc_status bsc_cnn_set_params(bsc_cnn* n, const float* host, int count) {
  if (!n || !host || count != param_total()) return BSC_ERR_INVALID_ARG;
  CKN(cudaMemcpyAsync(n->params, host, sizeof(float) * count, cudaMemcpyHostToDevice, n->c->stream),
      "bsc_cnn_set_params");
  CKN(relayout(n), "bsc_cnn_set_params");
  n->adam_t = 0;
  CKN(cudaMemsetAsync(n->adam_m, 0, sizeof(float) * count, n->c->stream), "bsc_cnn_set_params");
  CKN(cudaMemsetAsync(n->adam_v, 0, sizeof(float) * count, n->c->stream), "bsc_cnn_set_params");
  return cnn_sync(n, "bsc_cnn_set_params");
}

bsc_status bsc_cnn_get_params(bsc_cnn* n, float* host, int count, int which) {
  if (!n || !host || count != param_total() || which < 0 || which > 1) return BSC_ERR_INVALID_ARG;
  CKN(cudaMemcpyAsync(host, which ? n->grads : n->params, sizeof(float) * count, cudaMemcpyDeviceToHost,
                      n->c->stream),
      "bsc_cnn_get_params");
  return cnn_sync(n, "bsc_cnn_get_params");
}

bsc_status bsc_cnn_prepare(bsc_cnn* n, const void* K) {
  if (!n || !K) return BSC_ERR_INVALID_ARG;
  n->K = (const float*)K;
  CKN(launch_block_jacobi(n->c, K, n->Dinv), "bsc_cnn_prepare");
  BSC_COUNT(n->c, 2);
  k_diag_partials<<<n->red_grid, RB, 0, n->c->stream>>>(n->P, n->K, n->c->pinned, n->red);
  k_diag_mean<<<1, RB, 0, n->c->stream>>>(n->red_grid, n->red, n->scales);
  CKN(cudaGetLastError(), "bsc_cnn_prepare");
  return cnn_sync(n, "bsc_cnn_prepare");
}

bsc_status bsc_cnn_apply(bsc_cnn* n, const void* r, void* z) {
  if (!n || !r || !z || !n->K) return BSC_ERR_INVALID_ARG;
  CKN(cnn_forward(n, (const float*)r, (float*)z), "bsc_cnn_apply");
  return cnn_sync(n, "bsc_cnn_apply");
}

bsc_status bsc_cnn_loss_grad(bsc_cnn* n, const void* r, const void* xstar, double* loss) {
  if (!n || !r || !xstar || !n->K) return BSC_ERR_INVALID_ARG;
  CKN(cnn_loss_grad(n, (const float*)r, (const float*)xstar), "bsc_cnn_loss_grad");
  CKN(cudaMemcpyAsync(n->hsc, n->dsc, 2 * sizeof(double), cudaMemcpyDeviceToHost, n->c->stream),
      "bsc_cnn_loss_grad");
  bsc_status st = cnn_sync(n, "bsc_cnn_loss_grad");
  if (st != BSC_OK) return st;
  if (loss) *loss = n->hsc[0] / n->hsc[1];
  return BSC_OK;
}

bsc_status bsc_cnn_adam_step(bsc_cnn* n, double lr, double beta1, double beta2, double eps) {
  if (!n || !(lr > 0.0)) return BSC_ERR_INVALID_ARG;
  n->adam_t += 1;
  const float c1 = (float)(1.0 - pow(beta1, n->adam_t)), c2 = (float)(1.0 - pow(beta2, n->adam_t));
  const int cnt = param_total();
  BSC_COUNT(n->c, 1);
  k_adam<<<(cnt + 255) / 256, 256, 0, n->c->stream>>>(cnt, n->params, n->grads, n->adam_m, n->adam_v, (float)lr,
                                                        (float)beta1, (float)beta2, (float)eps, c1, c2);
  CKN(cudaGetLastError(), "bsc_cnn_adam_step");
  CKN(relayout(n), "bsc_cnn_adam_step");
  return BSC_OK;
}

// Activations of the last forward pass, as FP32 host arrays [P][channels]:
// which = 0 features (16), 1..3 layer outputs (32), 4 network output (3 of 4).
bsc_status bsc_cnn_activations(bsc_cnn* n, int which, float* host) {
  if (!n || !host || which < 0 || which > 4) return BSC_ERR_INVALID_ARG;
  const size_t P = (size_t)n->P;
  if (which == 4) {
    CKN(cudaMemcpyAsync(host, n->y4, P * 16, cudaMemcpyDeviceToHost, n->c->stream), "bsc_cnn_activations");
    return cnn_sync(n, "bsc_cnn_activations");
  }
  const int ch = which == 0 ? 16 : 32;
  std::vector<__nv_bfloat16> tmp(P * ch);
  CKN(cudaMemcpyAsync(tmp.data(), which == 0 ? n->X0 : n->act[which - 1], P * ch * 2, cudaMemcpyDeviceToHost,
                      n->c->stream),
      "bsc_cnn_activations");
  bsc_status st = cnn_sync(n, "bsc_cnn_activations");
  if (st != BSC_OK) return st;
  for (size_t k = 0; k < P * ch; ++k) host[k] = __bfloat162float(tmp[k]);
  return BSC_OK;
}

bsc_status bsc_solve_fcg(bsc_ctx* c, bsc_cnn* n, const void* K, const void* b, void* x, double tol, int maxit,
                         bsc_fcg_report* rep) {
  if (!c || !n || n->c != c || !K || !b || !x) return BSC_ERR_INVALID_ARG;
  if (!(tol > 0.0)) tol = c->pcg_tol;
  if (maxit <= 0) maxit = c->pcg_max_iter;
  bsc_fcg_report R;
  memset(&R, 0, sizeof(R));
  if (rep) *rep = R;
  bsc_status st = bsc_cnn_prepare(n, K);
  if (st != BSC_OK) return st;
  const int N3 = 3 * n->P, B = 256, G3 = (N3 + B - 1) / B;
  float *r = n->vec[0], *z = n->vec[1], *p = n->vec[2], *q = n->vec[3];
  float* xx = (float*)x;
  cudaStream_t s = c->stream;
  CKN(cudaMemsetAsync(xx, 0, sizeof(float) * N3, s), "bsc_solve_fcg");
  BSC_COUNT(c, 1);
  k_copy_f<<<G3, B, 0, s>>>(N3, (const float*)b, r);
  CKN(dot(n, r, r, n->dsc + 4), "bsc_solve_fcg");  // b.b
  CKN(cnn_forward(n, r, z), "bsc_solve_fcg");
  BSC_COUNT(c, 1);
  k_copy_f<<<G3, B, 0, s>>>(N3, z, p);
  CKN(cudaMemcpyAsync(n->hsc + 4, n->dsc + 4, sizeof(double), cudaMemcpyDeviceToHost, s), "bsc_solve_fcg");
  if ((st = cnn_sync(n, "bsc_solve_fcg")) != BSC_OK) return st;
  const double bb = n->hsc[4];
  if (!(bb > 0.0)) {
    if (rep) *rep = R;
    return BSC_OK;
  }
  const double stop = tol * tol * bb;
  double best = bb, rr = bb;
  int it = 0, since_best = 0;
  const int window = 25;
  bool stalled = false;
  for (it = 1; it <= maxit; ++it) {
    CKN(launch_spmv(c, K, p, q), "bsc_solve_fcg");
    CKN(dot(n, p, r, n->dsc + 0), "bsc_solve_fcg");
    CKN(dot(n, p, q, n->dsc + 1), "bsc_solve_fcg");
    BSC_COUNT(c, 1);
    k_fcg_xr<<<G3, B, 0, s>>>(N3, n->dsc, p, q, xx, r);
    CKN(dot(n, r, r, n->dsc + 3), "bsc_solve_fcg");
    CKN(cudaMemcpyAsync(n->hsc, n->dsc, 4 * sizeof(double), cudaMemcpyDeviceToHost, s), "bsc_solve_fcg");
    if ((st = cnn_sync(n, "bsc_solve_fcg")) != BSC_OK) return st;
    rr = n->hsc[3];
    if (!(n->hsc[1] > 0.0) || !isfinite(rr)) {
      stalled = true;
      break;
    }
    if (rr <= stop) break;
    if (rr < 0.25 * best) {
      best = rr;
      since_best = 0;
    } else if (++since_best >= window) {
      stalled = true;  // no halving of the residual norm in `window` iterations
      break;
    }
    CKN(cnn_forward(n, r, z), "bsc_solve_fcg");
    CKN(dot(n, z, q, n->dsc + 2), "bsc_solve_fcg");
    BSC_COUNT(c, 1);
    k_fcg_p<<<G3, B, 0, s>>>(N3, n->dsc, z, p);
  }
  R.fcg_iters = it > maxit ? maxit : it;
  R.rel_res = sqrt(rr / bb);
  if (stalled || !(rr <= stop)) {
    // fallback: plain block-Jacobi PCG on the remaining residual, x += d
    R.fell_back = 1;
    const double tol2 = sqrt(stop / (rr > 0.0 ? rr : stop));
    float* d = n->vec[4];
    int pit = 0;
    double prr = 0.0;
    st = bsc_solve(c, K, r, d, tol2 < 1.0 ? tol2 : 0.5, maxit, &pit, &prr);
    if (st != BSC_OK && st != BSC_ERR_NOT_CONVERGED) return st;
    BSC_COUNT(c, 1);
    k_add_f<<<G3, B, 0, s>>>(N3, d, xx);
    R.pcg_iters = pit;
    R.rel_res = prr * sqrt(rr / bb);
    CKN(cudaStreamSynchronize(s), "bsc_solve_fcg");
  }
  if (rep) *rep = R;
  if (!(R.rel_res <= tol)) {
    snprintf(c->err, sizeof(c->err), "bsc_solve_fcg: %d + %d iterations, rel. residual %g", R.fcg_iters,
             R.pcg_iters, R.rel_res);
    return BSC_ERR_NOT_CONVERGED;
  }
  return BSC_OK;
}

}  // extern "C"

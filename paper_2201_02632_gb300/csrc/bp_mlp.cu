// bp_mlp.cu -- MLP surrogate of the per-halo ICM solve (not in the paper).
//
// Network 6 -> 128 -> 128 -> 128 -> 3 with GELU hidden activations, mapping halo
// features (log10 M, log10 c, z, eps_*, f_*, eps_DM; normalised) to the solved model
// (ln r_f/r_vir, ln T r_vir/(G M), ln rho0/rho_s; normalised).
//
//  training (FP32):  k_dense (forward layer, bias + GELU epilogue), k_dense with the
//                    transposed weight (data gradient, GELU' epilogue), k_wgrad (per
//                    row-chunk weight/bias gradient partials) + k_sum_partials (fixed
//                    order), k_adam
//  inference:        k_infer_bf16, all four layers fused per 64-row tile, BF16 weights
//                    and BF16 activations, FP32 accumulation
//  helpers:          k_features, k_targets, k_mse
// The surrogate solve (bp_solve_halos_surrogate) decodes the prediction into the
// starting point of a few FP64 Newton iterations of bp_solve_halos_ex, whose residual
// gate sends the rejected halos to the full solve.
#include <cuda_bf16.h>

#include <vector>

#include "bp_internal.cuh"

namespace {

constexpr int IN = BP_MLP_IN, HID = BP_MLP_HID, OUT = BP_MLP_OUT;
constexpr int OFF_W1 = 0, OFF_B1 = OFF_W1 + HID * IN, OFF_W2 = OFF_B1 + HID,
              OFF_B2 = OFF_W2 + HID * HID, OFF_W3 = OFF_B2 + HID, OFF_B3 = OFF_W3 + HID * HID,
              OFF_W4 = OFF_B3 + HID, OFF_B4 = OFF_W4 + OUT * HID, NPAR = OFF_B4 + OUT;
static_assert(NPAR == BP_MLP_NPARAMS, "parameter count");
// bf16 weight buffer: W1, W2, W3, W4 back to back
constexpr int WB_W1 = 0, WB_W2 = WB_W1 + HID * IN, WB_W3 = WB_W2 + HID * HID,
              WB_W4 = WB_W3 + HID * HID, NWB = WB_W4 + OUT * HID;
static_assert(NWB == BP_MLP_NWEIGHTS, "weight count");
// cache per row: Z1, A1, Z2, A2, Z3, A3
constexpr int CZ1 = 0, CA1 = HID, CZ2 = 2 * HID, CA2 = 3 * HID, CZ3 = 4 * HID, CA3 = 5 * HID;
static_assert(6 * HID == BP_MLP_CACHE_PER_ROW, "cache layout");

__device__ __forceinline__ float gelu(float x) {
  return 0.5f * x * (1.0f + erff(x * 0.70710678118654752f));
}
__device__ __forceinline__ float gelu_grad(float x) {
  // d/dx [x Phi(x)] = Phi(x) + x phi(x)
  float cdf = 0.5f * (1.0f + erff(x * 0.70710678118654752f));
  float pdf = 0.39894228040143268f * expf(-0.5f * x * x);
  return cdf + x * pdf;
}

constexpr int ROWS = 64;  // rows per CTA of the dense kernels
constexpr int DT = 256;

// C[r][o] = sum_i X[r][i] W'[o][i] (+ bias, activation epilogue), for OUT_N <= 128 outputs
// and IN_K inputs, inputs staged in chunks of KC.  W' is W ([OUT_N][IN_K], forward) or
// W^T (TRANS: W is [IN_K][OUT_N], data gradient).  EPI 0: C = acc + b;
// 1: Z = acc + b, A = GELU(Z); 2: C = acc * GELU'(Zp)
constexpr int KC = 32;
template <int IN_K, int OUT_N, bool TRANS, int EPI>
__global__ void __launch_bounds__(DT) k_dense(int64_t n, const float* __restrict__ X,
                                              int ldx, const float* __restrict__ W,
                                              const float* __restrict__ b,
                                              const float* __restrict__ Zp, int ldzp,
                                              float* __restrict__ C, int ldc,
                                              float* __restrict__ A2, int lda2) {
  constexpr int OPAD = (OUT_N + 3) / 4 * 4;
  static_assert(OPAD <= 128, "at most 128 outputs");
  __shared__ __align__(16) float Xs[KC][ROWS + 4];
  __shared__ __align__(16) float Ws[KC][OPAD + 4];
  const int tid = threadIdx.x, w = tid >> 5, lane = tid & 31;
  const int64_t row0 = (int64_t)blockIdx.x * ROWS;
  const int o0 = lane * 4;  // this lane's four outputs (valid while o0 < OPAD)
  float acc[8][4];
#pragma unroll
  for (int r = 0; r < 8; ++r)
#pragma unroll
    for (int c = 0; c < 4; ++c) acc[r][c] = 0.f;
  for (int k0 = 0; k0 < IN_K; k0 += KC) {
    const int kn = min(KC, IN_K - k0);
    __syncthreads();
    for (int idx = tid; idx < kn * OPAD; idx += DT) {
      int o = idx % OPAD, i = idx / OPAD;
      float v = 0.f;
      if (o < OUT_N) v = TRANS ? W[(int64_t)(k0 + i) * OUT_N + o] : W[(int64_t)o * IN_K + k0 + i];
      Ws[i][o] = v;
    }
    for (int idx = tid; idx < ROWS * kn; idx += DT) {
      int r = idx / kn, i = idx % kn;
      int64_t row = row0 + r;
      Xs[i][r] = row < n ? X[row * ldx + k0 + i] : 0.f;
    }
    __syncthreads();
    if (o0 < OPAD) {
      for (int i = 0; i < kn; ++i) {
        float4 xa = *reinterpret_cast<const float4*>(&Xs[i][w * 8]);
        float4 xb = *reinterpret_cast<const float4*>(&Xs[i][w * 8 + 4]);
        float4 wv = *reinterpret_cast<const float4*>(&Ws[i][o0]);
        float xr[8] = {xa.x, xa.y, xa.z, xa.w, xb.x, xb.y, xb.z, xb.w};
        float wc[4] = {wv.x, wv.y, wv.z, wv.w};
#pragma unroll
        for (int r = 0; r < 8; ++r)
#pragma unroll
          for (int c = 0; c < 4; ++c) acc[r][c] = fmaf(xr[r], wc[c], acc[r][c]);
      }
    }
  }
  if (o0 >= OPAD) return;
#pragma unroll
  for (int r = 0; r < 8; ++r) {
    int64_t row = row0 + w * 8 + r;
    if (row >= n) continue;
#pragma unroll
    for (int c = 0; c < 4; ++c) {
      int o = o0 + c;
      if (o >= OUT_N) continue;
      float v = acc[r][c];
      if (EPI == 0) {
        C[row * ldc + o] = v + b[o];
      } else if (EPI == 1) {
        float z = v + b[o];
        C[row * ldc + o] = z;
        A2[row * lda2 + o] = gelu(z);
      } else {
        C[row * ldc + o] = v * gelu_grad(Zp[row * ldzp + o]);
      }
    }
  }
}

// Weight-gradient partials: for the rows of chunk blockIdx.x,
// P[chunk][o * IN_K + i] = sum_r D[r][o] Xp[r][i] and P[chunk][OUT_N * IN_K + o] = sum_r D[r][o]
constexpr int WG_ROWS = 256;
template <int IN_K, int OUT_N>
__global__ void __launch_bounds__(DT) k_wgrad(int64_t n, const float* __restrict__ D, int ldd,
                                              const float* __restrict__ Xp, int ldx,
                                              float* __restrict__ P) {
  constexpr int NO = OUT_N * IN_K + OUT_N;
  const int64_t r0 = (int64_t)blockIdx.x * WG_ROWS;
  const int64_t r1 = min(n, r0 + WG_ROWS);
  float* out = P + (int64_t)blockIdx.x * NO;
  if (IN_K == HID && OUT_N == HID) {
    // register-tiled: thread owns 8 outputs o x 8 inputs i
    __shared__ __align__(16) float Ds[32][HID];
    __shared__ __align__(16) float As[32][HID];
    const int tid = threadIdx.x;
    const int og = (tid >> 4) * 8, ig = (tid & 15) * 8;
    float acc[8][8];
    float bacc[8];
#pragma unroll
    for (int a = 0; a < 8; ++a) {
      bacc[a] = 0.f;
#pragma unroll
      for (int c = 0; c < 8; ++c) acc[a][c] = 0.f;
    }
    for (int64_t rb = r0; rb < r1; rb += 32) {
      __syncthreads();
      for (int idx = tid; idx < 32 * HID; idx += DT) {
        int r = idx / HID, c = idx % HID;
        int64_t row = rb + r;
        Ds[r][c] = row < r1 ? D[row * ldd + c] : 0.f;
        As[r][c] = row < r1 ? Xp[row * ldx + c] : 0.f;
      }
      __syncthreads();
      for (int r = 0; r < 32; ++r) {
        float4 d0 = *reinterpret_cast<const float4*>(&Ds[r][og]);
        float4 d1 = *reinterpret_cast<const float4*>(&Ds[r][og + 4]);
        float4 a0 = *reinterpret_cast<const float4*>(&As[r][ig]);
        float4 a1 = *reinterpret_cast<const float4*>(&As[r][ig + 4]);
        float dv[8] = {d0.x, d0.y, d0.z, d0.w, d1.x, d1.y, d1.z, d1.w};
        float av[8] = {a0.x, a0.y, a0.z, a0.w, a1.x, a1.y, a1.z, a1.w};
#pragma unroll
        for (int a = 0; a < 8; ++a) {
          bacc[a] += dv[a];
#pragma unroll
          for (int c = 0; c < 8; ++c) acc[a][c] = fmaf(dv[a], av[c], acc[a][c]);
        }
      }
    }
#pragma unroll
    for (int a = 0; a < 8; ++a) {
#pragma unroll
      for (int c = 0; c < 8; ++c) out[(og + a) * IN_K + ig + c] = acc[a][c];
      if ((tid & 15) == 0) out[OUT_N * IN_K + og + a] = bacc[a];
    }
  } else {
    for (int j = threadIdx.x; j < NO; j += DT) {
      float acc = 0.f;
      if (j < OUT_N * IN_K) {
        int o = j / IN_K, i = j % IN_K;
        for (int64_t r = r0; r < r1; ++r) acc = fmaf(D[r * ldd + o], Xp[r * ldx + i], acc);
      } else {
        int o = j - OUT_N * IN_K;
        for (int64_t r = r0; r < r1; ++r) acc += D[r * ldd + o];
      }
      out[j] = acc;
    }
  }
}

// grad[off_w + j] / grad[off_b + o] = sum over chunks, in chunk order
__global__ void k_sum_partials(const float* __restrict__ P, int64_t nchunks, int nw, int nb,
                               float* __restrict__ gw, float* __restrict__ gb) {
  int j = blockIdx.x * blockDim.x + threadIdx.x;
  if (j >= nw + nb) return;
  float s = 0.f;
  for (int64_t c = 0; c < nchunks; ++c) s += P[c * (nw + nb) + j];
  if (j < nw) gw[j] = s; else gb[j - nw] = s;
}

__global__ void k_adam(int np, float* __restrict__ p, const float* __restrict__ g,
                       float* __restrict__ m, float* __restrict__ v, float lr, float b1, float b2,
                       float eps, float c1, float c2) {
  int j = blockIdx.x * blockDim.x + threadIdx.x;
  if (j >= np) return;
  float gj = g[j];
  float mj = b1 * m[j] + (1.f - b1) * gj;
  float vj = b2 * v[j] + (1.f - b2) * gj * gj;
  m[j] = mj;
  v[j] = vj;
  p[j] -= lr * (mj * c1) / (sqrtf(vj * c2) + eps);
}

__global__ void k_to_bf16(const float* __restrict__ p, __nv_bfloat16* __restrict__ wb) {
  int j = blockIdx.x * blockDim.x + threadIdx.x;
  if (j >= NWB) return;
  int src;
  if (j < WB_W2) src = OFF_W1 + j;
  else if (j < WB_W3) src = OFF_W2 + (j - WB_W2);
  else if (j < WB_W4) src = OFF_W3 + (j - WB_W3);
  else src = OFF_W4 + (j - WB_W4);
  wb[j] = __float2bfloat16_rn(p[src]);
}

// Fused BF16 inference: 64 rows per CTA; weights staged KC inputs at a time; BF16
// activations in shared memory; FP32 accumulation.
__global__ void __launch_bounds__(DT) k_infer_bf16(int64_t n, const float* __restrict__ X,
                                                   const __nv_bfloat16* __restrict__ wb,
                                                   const float* __restrict__ par,
                                                   float* __restrict__ Y) {
  __shared__ __align__(16) __nv_bfloat16 Ws[KC][HID];          // [i][o] chunk
  __shared__ __align__(16) __nv_bfloat16 Act[2][HID][ROWS + 8];  // ping-pong [i][r]
  const int tid = threadIdx.x, w = tid >> 5, lane = tid & 31;
  const int64_t row0 = (int64_t)blockIdx.x * ROWS;
  for (int idx = tid; idx < ROWS * IN; idx += DT) {
    int r = idx / IN, i = idx % IN;
    int64_t row = row0 + r;
    Act[0][i][r] = __float2bfloat16_rn(row < n ? X[row * IN + i] : 0.f);
  }
  int cur = 0;
  auto layer = [&](int k_in, int n_out, int wofs, int bofs, bool act, bool last) {
    const int o0 = lane * 4;
    float acc[8][4];
#pragma unroll
    for (int r = 0; r < 8; ++r)
#pragma unroll
      for (int c = 0; c < 4; ++c) acc[r][c] = 0.f;
    for (int k0 = 0; k0 < k_in; k0 += KC) {
      const int kn = min(KC, k_in - k0);
      __syncthreads();
      for (int idx = tid; idx < kn * HID; idx += DT) {
        int o = idx % HID, i = idx / HID;
        Ws[i][o] = o < n_out ? wb[wofs + (int64_t)o * k_in + k0 + i] : __float2bfloat16_rn(0.f);
      }
      __syncthreads();
      if (o0 < n_out) {
        for (int i = 0; i < kn; ++i) {
          uint4 raw = *reinterpret_cast<const uint4*>(&Act[cur][k0 + i][w * 8]);
          const __nv_bfloat16* xv = reinterpret_cast<const __nv_bfloat16*>(&raw);
          float xr[8];
#pragma unroll
          for (int r = 0; r < 8; ++r) xr[r] = __bfloat162float(xv[r]);
          uint2 wraw = *reinterpret_cast<const uint2*>(&Ws[i][o0]);
          const __nv_bfloat16* wv = reinterpret_cast<const __nv_bfloat16*>(&wraw);
          float wc[4];
#pragma unroll
          for (int c = 0; c < 4; ++c) wc[c] = __bfloat162float(wv[c]);
#pragma unroll
          for (int r = 0; r < 8; ++r)
#pragma unroll
            for (int c = 0; c < 4; ++c) acc[r][c] = fmaf(xr[r], wc[c], acc[r][c]);
        }
      }
    }
    if (o0 < n_out) {
#pragma unroll
      for (int c = 0; c < 4; ++c) {
        int o = o0 + c;
        if (o >= n_out) continue;
        float bo = par[bofs + o];
#pragma unroll
        for (int r = 0; r < 8; ++r) {
          float z = acc[r][c] + bo;
          if (last) {
            int64_t row = row0 + w * 8 + r;
            if (row < n) Y[row * OUT + o] = z;
          } else {
            Act[cur ^ 1][o][w * 8 + r] = __float2bfloat16_rn(act ? gelu(z) : z);
          }
        }
      }
    }
    cur ^= 1;
  };
  layer(IN, HID, WB_W1, OFF_B1, true, false);
  layer(HID, HID, WB_W2, OFF_B2, true, false);
  layer(HID, HID, WB_W3, OFF_B3, true, false);
  layer(HID, OUT, WB_W4, OFF_B4, false, true);
}

// norm layout: [0..8] means of the 6 features and 3 targets, [9..17] their scales
__global__ void k_features(int64_t n, const double* __restrict__ M, const double* __restrict__ c,
                           const double* __restrict__ z, const double* __restrict__ prm,
                           const float* __restrict__ norm, float* __restrict__ X,
                           const float* __restrict__ hull, int* __restrict__ outside) {
  int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  double f[IN];
  f[0] = log10(M[i]);
  f[1] = log10(c[i]);
  f[2] = z[i];
  f[3] = prm ? prm[i] : 3.97e-6;
  f[4] = prm ? prm[n + i] : 0.026;
  f[5] = prm ? prm[2 * n + i] : 0.0;
  int out = 0;
  for (int k = 0; k < IN; ++k) {
    float v = (float)((f[k] - norm[k]) / norm[9 + k]);
    if (!(v >= hull[k] && v <= hull[IN + k])) out = 1;
    X[i * IN + k] = v;
  }
  if (outside) outside[i] = out;
}

__global__ void k_targets(int64_t n, const double* __restrict__ model,
                          const float* __restrict__ norm, float* __restrict__ T) {
  int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  auto F = [&](int f) { return model[(int64_t)f * n + i]; };
  double rv = F(BP_M_RVIR), GM = bpc::G * F(BP_M_MVIR);
  double t[OUT] = {log(F(BP_M_RF) / rv), log(F(BP_M_T) * rv / GM), log(F(BP_M_RHO0) / F(BP_M_RHOS))};
  for (int k = 0; k < OUT; ++k) T[i * OUT + k] = (float)((t[k] - norm[IN + k]) / norm[9 + IN + k]);
}

// dY = 2 (Y - T) / (n OUT); per-block partial sums of the squared error
__global__ void k_mse(int64_t n, const float* __restrict__ Y, const float* __restrict__ T,
                      float* __restrict__ dY, float* __restrict__ part) {
  __shared__ float red[256];
  int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  float e2 = 0.f;
  if (j < n * OUT) {
    float d = Y[j] - T[j];
    dY[j] = 2.f * d / (float)(n * OUT);
    e2 = d * d;
  }
  red[threadIdx.x] = e2;
  __syncthreads();
  for (int s = 128; s > 0; s >>= 1) {
    if (threadIdx.x < s) red[threadIdx.x] += red[threadIdx.x + s];
    __syncthreads();
  }
  if (threadIdx.x == 0) part[blockIdx.x] = red[0];
}

// decoded prediction -> starting point of the FP64 solve; outside the hull -> NaN
__global__ void k_decode_guess(int64_t n, const float* __restrict__ Y,
                               const float* __restrict__ norm, const int* __restrict__ outside,
                               double* __restrict__ guess) {
  int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  double g0 = (double)Y[i * OUT + 0] * norm[9 + IN + 0] + norm[IN + 0];
  double g1 = (double)Y[i * OUT + 1] * norm[9 + IN + 1] + norm[IN + 1];
  if (outside[i]) g0 = g1 = NAN;
  guess[i] = g0;
  guess[n + i] = g1;
}

int check_n(bp_ctx* ctx, int64_t n, const char* who) {
  if (n < 0) return bp_fail(ctx, BP_EINVAL, "%s: n < 0", who);
  if (n > (int64_t)1 << 31) return bp_fail(ctx, BP_ERANGE, "%s: n above 2^31", who);
  return BP_OK;
}

}  // namespace

extern "C" {

int bp_mlp_forward(bp_ctx* ctx, int64_t n, const float* params, const float* x, float* y,
                   float* cache) {
  if (!ctx) return BP_EINVAL;
  int r = check_n(ctx, n, "bp_mlp_forward");
  if (r || n == 0) return r;
  if (!params || !x || !y || !cache) return bp_fail(ctx, BP_EINVAL, "bp_mlp_forward: null pointer");
  unsigned g = (unsigned)((n + ROWS - 1) / ROWS);
  const int LC = BP_MLP_CACHE_PER_ROW;
  k_dense<IN, HID, false, 1><<<g, DT, 0, ctx->stream>>>(n, x, IN, params + OFF_W1, params + OFF_B1,
                                                        nullptr, 0, cache + CZ1, LC, cache + CA1, LC);
  BP_LAUNCH_CHECK(ctx, "mlp layer 1");
  k_dense<HID, HID, false, 1><<<g, DT, 0, ctx->stream>>>(n, cache + CA1, LC, params + OFF_W2,
                                                         params + OFF_B2, nullptr, 0, cache + CZ2,
                                                         LC, cache + CA2, LC);
  BP_LAUNCH_CHECK(ctx, "mlp layer 2");
  k_dense<HID, HID, false, 1><<<g, DT, 0, ctx->stream>>>(n, cache + CA2, LC, params + OFF_W3,
                                                         params + OFF_B3, nullptr, 0, cache + CZ3,
                                                         LC, cache + CA3, LC);
  BP_LAUNCH_CHECK(ctx, "mlp layer 3");
  k_dense<HID, OUT, false, 0><<<g, DT, 0, ctx->stream>>>(n, cache + CA3, LC, params + OFF_W4,
                                                         params + OFF_B4, nullptr, 0, y, OUT,
                                                         nullptr, 0);
  BP_LAUNCH_CHECK(ctx, "mlp layer 4");
  return BP_OK;
}

int bp_mlp_backward(bp_ctx* ctx, int64_t n, const float* params, const float* x,
                    const float* cache, const float* dy, float* grad) {
  if (!ctx) return BP_EINVAL;
  int r = check_n(ctx, n, "bp_mlp_backward");
  if (r) return r;
  if (!params || !x || !cache || !dy || !grad)
    return bp_fail(ctx, BP_EINVAL, "bp_mlp_backward: null pointer");
  if (n == 0) {
    BP_CUDA(ctx, cudaMemsetAsync(grad, 0, NPAR * sizeof(float), ctx->stream));
    return BP_OK;
  }
  const int LC = BP_MLP_CACHE_PER_ROW;
  // scratch: dA/dZ of the three hidden layers (reused) and weight-gradient partials
  int64_t nch = (n + WG_ROWS - 1) / WG_ROWS;
  float *d3, *d2, *d1, *part;
  size_t act = (size_t)n * HID * sizeof(float);
  size_t pbytes = (size_t)nch * (HID * HID + HID) * sizeof(float);
  float* base;
  if ((r = bp_ws(ctx, WS_MISC2, 3 * act + pbytes + 256, (void**)&base))) return r;
  d3 = base;
  d2 = d3 + (size_t)n * HID;
  d1 = d2 + (size_t)n * HID;
  part = d1 + (size_t)n * HID;
  unsigned g = (unsigned)((n + ROWS - 1) / ROWS);
  // layer 4: dW4, db4 from dy and A3; dZ3 = (dy W4) * GELU'(Z3)
  k_wgrad<HID, OUT><<<(unsigned)nch, DT, 0, ctx->stream>>>(n, dy, OUT, cache + CA3, LC, part);
  BP_LAUNCH_CHECK(ctx, "mlp wgrad 4");
  k_sum_partials<<<(OUT * HID + OUT + 255) / 256, 256, 0, ctx->stream>>>(
      part, nch, OUT * HID, OUT, grad + OFF_W4, grad + OFF_B4);
  BP_LAUNCH_CHECK(ctx, "mlp sum 4");
  k_dense<OUT, HID, true, 2><<<g, DT, 0, ctx->stream>>>(n, dy, OUT, params + OFF_W4, nullptr,
                                                        cache + CZ3, LC, d3, HID, nullptr, 0);
  BP_LAUNCH_CHECK(ctx, "mlp dgrad 3");
  // layer 3
  k_wgrad<HID, HID><<<(unsigned)nch, DT, 0, ctx->stream>>>(n, d3, HID, cache + CA2, LC, part);
  BP_LAUNCH_CHECK(ctx, "mlp wgrad 3");
  k_sum_partials<<<(HID * HID + HID + 255) / 256, 256, 0, ctx->stream>>>(
      part, nch, HID * HID, HID, grad + OFF_W3, grad + OFF_B3);
  BP_LAUNCH_CHECK(ctx, "mlp sum 3");
  k_dense<HID, HID, true, 2><<<g, DT, 0, ctx->stream>>>(n, d3, HID, params + OFF_W3, nullptr,
                                                        cache + CZ2, LC, d2, HID, nullptr, 0);
  BP_LAUNCH_CHECK(ctx, "mlp dgrad 2");
  // layer 2
  k_wgrad<HID, HID><<<(unsigned)nch, DT, 0, ctx->stream>>>(n, d2, HID, cache + CA1, LC, part);
  BP_LAUNCH_CHECK(ctx, "mlp wgrad 2");
  k_sum_partials<<<(HID * HID + HID + 255) / 256, 256, 0, ctx->stream>>>(
      part, nch, HID * HID, HID, grad + OFF_W2, grad + OFF_B2);
  BP_LAUNCH_CHECK(ctx, "mlp sum 2");
  k_dense<HID, HID, true, 2><<<g, DT, 0, ctx->stream>>>(n, d2, HID, params + OFF_W2, nullptr,
                                                        cache + CZ1, LC, d1, HID, nullptr, 0);
  BP_LAUNCH_CHECK(ctx, "mlp dgrad 1");
  // layer 1
  k_wgrad<IN, HID><<<(unsigned)nch, DT, 0, ctx->stream>>>(n, d1, HID, x, IN, part);
  BP_LAUNCH_CHECK(ctx, "mlp wgrad 1");
  k_sum_partials<<<(HID * IN + HID + 255) / 256, 256, 0, ctx->stream>>>(
      part, nch, HID * IN, HID, grad + OFF_W1, grad + OFF_B1);
  BP_LAUNCH_CHECK(ctx, "mlp sum 1");
  return BP_OK;
}

int bp_mlp_adam(bp_ctx* ctx, float* params, const float* grad, float* m, float* v, int64_t step,
                double lr, double beta1, double beta2, double eps) {
  if (!ctx) return BP_EINVAL;
  if (!params || !grad || !m || !v || step < 1)
    return bp_fail(ctx, BP_EINVAL, "bp_mlp_adam: arguments");
  double c1 = 1.0 / (1.0 - pow(beta1, (double)step));
  double c2 = 1.0 / (1.0 - pow(beta2, (double)step));
  k_adam<<<(NPAR + 255) / 256, 256, 0, ctx->stream>>>(NPAR, params, grad, m, v, (float)lr,
                                                      (float)beta1, (float)beta2, (float)eps,
                                                      (float)c1, (float)c2);
  BP_LAUNCH_CHECK(ctx, "adam");
  return BP_OK;
}

int bp_mlp_to_bf16(bp_ctx* ctx, const float* params, uint16_t* weights_bf16) {
  if (!ctx) return BP_EINVAL;
  if (!params || !weights_bf16) return bp_fail(ctx, BP_EINVAL, "bp_mlp_to_bf16: null pointer");
  k_to_bf16<<<(NWB + 255) / 256, 256, 0, ctx->stream>>>(params, (__nv_bfloat16*)weights_bf16);
  BP_LAUNCH_CHECK(ctx, "to bf16");
  return BP_OK;
}

int bp_mlp_infer_bf16(bp_ctx* ctx, int64_t n, const uint16_t* weights_bf16, const float* params,
                      const float* x, float* y) {
  if (!ctx) return BP_EINVAL;
  int r = check_n(ctx, n, "bp_mlp_infer_bf16");
  if (r || n == 0) return r;
  if (!weights_bf16 || !params || !x || !y)
    return bp_fail(ctx, BP_EINVAL, "bp_mlp_infer_bf16: null pointer");
  k_infer_bf16<<<(unsigned)((n + ROWS - 1) / ROWS), DT, 0, ctx->stream>>>(
      n, x, (const __nv_bfloat16*)weights_bf16, params, y);
  BP_LAUNCH_CHECK(ctx, "mlp infer");
  return BP_OK;
}

int bp_mlp_features(bp_ctx* ctx, int64_t n, const double* Mvir, const double* c, const double* z,
                    const double* params, const float* norm, float* x) {
  if (!ctx) return BP_EINVAL;
  int r = check_n(ctx, n, "bp_mlp_features");
  if (r || n == 0) return r;
  if (!Mvir || !c || !z || !norm || !x) return bp_fail(ctx, BP_EINVAL, "bp_mlp_features: null");
  // no hull test here: an all-inclusive hull
  float* hull;
  if ((r = bp_ws(ctx, WS_MISC3, 2 * IN * sizeof(float), (void**)&hull))) return r;
  float h[2 * IN];
  for (int k = 0; k < IN; ++k) {
    h[k] = -INFINITY;
    h[IN + k] = INFINITY;
  }
  BP_CUDA(ctx, cudaMemcpyAsync(hull, h, sizeof(h), cudaMemcpyHostToDevice, ctx->stream));
  k_features<<<(unsigned)((n + 255) / 256), 256, 0, ctx->stream>>>(n, Mvir, c, z, params, norm, x,
                                                                   hull, nullptr);
  BP_LAUNCH_CHECK(ctx, "features");
  BP_CUDA(ctx, cudaStreamSynchronize(ctx->stream));  // the host staging buffer h
  return BP_OK;
}

int bp_mlp_targets(bp_ctx* ctx, int64_t n, const double* model, const float* norm, float* t) {
  if (!ctx) return BP_EINVAL;
  int r = check_n(ctx, n, "bp_mlp_targets");
  if (r || n == 0) return r;
  if (!model || !norm || !t) return bp_fail(ctx, BP_EINVAL, "bp_mlp_targets: null pointer");
  k_targets<<<(unsigned)((n + 255) / 256), 256, 0, ctx->stream>>>(n, model, norm, t);
  BP_LAUNCH_CHECK(ctx, "targets");
  return BP_OK;
}

int bp_mlp_mse(bp_ctx* ctx, int64_t n, const float* y, const float* t, float* dy, double* loss) {
  if (!ctx) return BP_EINVAL;
  int r = check_n(ctx, n, "bp_mlp_mse");
  if (r || n == 0) return r;
  if (!y || !t || !dy) return bp_fail(ctx, BP_EINVAL, "bp_mlp_mse: null pointer");
  int64_t ne = n * OUT;
  unsigned nb = (unsigned)((ne + 255) / 256);
  float* part;
  if ((r = bp_ws(ctx, WS_MISC3, (size_t)nb * sizeof(float), (void**)&part))) return r;
  k_mse<<<nb, 256, 0, ctx->stream>>>(n, y, t, dy, part);
  BP_LAUNCH_CHECK(ctx, "mse");
  if (loss) {
    std::vector<float> h(nb);
    BP_CUDA(ctx, cudaMemcpyAsync(h.data(), part, nb * sizeof(float), cudaMemcpyDeviceToHost,
                                 ctx->stream));
    BP_CUDA(ctx, cudaStreamSynchronize(ctx->stream));
    double s = 0;
    for (unsigned k = 0; k < nb; ++k) s += h[k];
    *loss = s / (double)ne;
  }
  return BP_OK;
}

int bp_solve_halos_surrogate(bp_ctx* ctx, int64_t n, const double* Mvir, const double* c,
                             const double* z, const double* params, const uint16_t* weights_bf16,
                             const float* mlp_params, const float* norm, const float* hull,
                             int polish_iter, double gate, double* model, int32_t* status,
                             double resid_tol) {
  if (!ctx) return BP_EINVAL;
  int r = check_n(ctx, n, "bp_solve_halos_surrogate");
  if (r || n == 0) return r;
  if (!Mvir || !c || !z || !weights_bf16 || !mlp_params || !norm || !hull || !model || !status)
    return bp_fail(ctx, BP_EINVAL, "bp_solve_halos_surrogate: null pointer");
  if (!(gate > 0)) return bp_fail(ctx, BP_EINVAL, "bp_solve_halos_surrogate: gate must be > 0");
  char* base;
  size_t bx = (size_t)n * IN * 4, by = (size_t)n * OUT * 4, bo = (size_t)n * 4,
         bg = (size_t)n * 2 * 8;
  if ((r = bp_ws(ctx, WS_MISC2, bx + by + bo + bg + 1024, (void**)&base))) return r;
  float* x = (float*)base;
  float* y = (float*)(base + ((bx + 255) / 256) * 256);
  int* outside = (int*)((char*)y + ((by + 255) / 256) * 256);
  double* guess = (double*)((char*)outside + ((bo + 255) / 256) * 256);
  bp_phase_begin(ctx, BP_PH_SURROGATE);
  k_features<<<(unsigned)((n + 255) / 256), 256, 0, ctx->stream>>>(n, Mvir, c, z, params, norm, x,
                                                                   hull, outside);
  BP_LAUNCH_CHECK(ctx, "features");
  k_infer_bf16<<<(unsigned)((n + ROWS - 1) / ROWS), DT, 0, ctx->stream>>>(
      n, x, (const __nv_bfloat16*)weights_bf16, mlp_params, y);
  BP_LAUNCH_CHECK(ctx, "mlp infer");
  k_decode_guess<<<(unsigned)((n + 255) / 256), 256, 0, ctx->stream>>>(n, y, norm, outside, guess);
  BP_LAUNCH_CHECK(ctx, "decode guess");
  bp_phase_end(ctx, BP_PH_SURROGATE);
  return bp_solve_halos_ex(ctx, n, Mvir, c, z, params, guess, polish_iter > 0 ? polish_iter : 4,
                           gate, model, status, BP_SOLVE_FP64, resid_tol);
}

}  // extern "C"

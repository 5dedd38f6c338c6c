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
//  inference:        k_infer_tc, all four layers fused per 128-row tile, BF16 weights and
//                    activations, FP32 accumulation; the two 128 x 128 layers on the
//                    tensor cores (tcgen05, accumulator in tensor memory)
//  helpers:          k_features, k_targets, k_mse
// The surrogate solve (bp_solve_halos_surrogate) decodes the prediction into the seed of
// the FP32 pre-solve of bp_solve_halos_ex, whose FP64 Newton and residual gate follow (the
// rejected halos get the full solve).
#include <cuda_bf16.h>

#include <vector>

#include "bp_internal.cuh"
#include "bp_tc.cuh"

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

// ---------------------------------------------------------------- tensor-core inference
// BF16 inference: a persistent CTA of 256 threads takes 128 rows at a time.  Layer 1 (6
// inputs) runs on the CUDA cores and writes its BF16 activations straight into the A operand
// of layer 2 (K-major, 128-byte swizzle, two K blocks of 64 inputs, 16 KB each).  Layers 2
// and 3 are one 128 x 128 x 128 tcgen05 GEMM each (kind::f16, BF16 operands) against W2 and
// W3, staged once per CTA in the same layout as the B operand, with the FP32 accumulator in
// tensor memory.  Their epilogues (bias, GELU, rounding to BF16) read it back, warp w taking
// rows 32 (w % 4) .. + 31 and columns 64 (w / 4) .. + 63; layer 4 (3 outputs, FP32 sums of
// BF16 activations times BF16 weights) is folded into layer 3's epilogue.  Every mbarrier
// wait is bounded; a timeout sets *err and stops the CTA.
constexpr int TI_M = 128, TI_THREADS = 256;
constexpr int TI_KB = TI_M * 128;  // bytes of one K block (128 rows x 64 BF16)
constexpr uint32_t TI_COLS = 128;
constexpr uint32_t TI_IDESC = bptc::idesc_bf16(TI_M, HID);
constexpr uint32_t TI_WAIT_POLLS = 1u << 26;
constexpr uint64_t TI_WAIT_NS = 2000000000ull;  // 2 s

struct alignas(1024) TiSmem {
  unsigned char w2[2 * TI_KB];
  unsigned char w3[2 * TI_KB];
  unsigned char act[2 * TI_KB];
  float w1[HID * IN];
  float b1[HID], b2[HID], b3[HID];
  float w4[OUT * HID];
  float b4[4];
  float ypart[2][TI_M][OUT];  // layer-4 sums of the two column halves
  uint64_t mbar;
  uint32_t tmem;
};

// byte offset of the 16-byte chunk holding inputs 8 q .. 8 q + 7 (q < 16) of row r
__device__ __forceinline__ int ti_chunk(int r, int q) {
  return (q >> 3) * TI_KB + (r >> 3) * 1024 + (r & 7) * 128 + (((q & 7) ^ (r & 7)) << 4);
}

__device__ __forceinline__ uint4 pack8_bf16(const float* v) {
  uint4 u;
  uint32_t* wd = reinterpret_cast<uint32_t*>(&u);
#pragma unroll
  for (int j = 0; j < 4; ++j) {
    const __nv_bfloat162 t = __floats2bfloat162_rn(v[2 * j], v[2 * j + 1]);
    wd[j] = *reinterpret_cast<const uint32_t*>(&t);
  }
  return u;
}

__device__ __forceinline__ float bf16_round(float v) {
  return __bfloat162float(__float2bfloat16_rn(v));
}

__global__ void __launch_bounds__(TI_THREADS) k_infer_tc(int64_t n, const float* __restrict__ X,
                                                         const __nv_bfloat16* __restrict__ wb,
                                                         const float* __restrict__ par,
                                                         float* __restrict__ Y, int* err) {
  using namespace bptc;
  extern __shared__ unsigned char ti_raw[];
  TiSmem& S = *reinterpret_cast<TiSmem*>(((uintptr_t)ti_raw + 1023) & ~(uintptr_t)1023);
  const int tid = threadIdx.x, lane = tid & 31, w = tid >> 5;
  const int64_t ntiles = (n + TI_M - 1) / TI_M;
  if (w == 0) {
    tmem_alloc(&S.tmem, TI_COLS);
    tmem_relinquish();
  }
  if (tid == 0) {
    mbar_init(&S.mbar, 1);
    fence_mbar_init();
  }
  // W2, W3 ([out][in], 16-byte chunks of 8 inputs) into the B-operand layout; the rest FP32
  const uint4* w2g = reinterpret_cast<const uint4*>(wb + WB_W2);
  const uint4* w3g = reinterpret_cast<const uint4*>(wb + WB_W3);
  for (int c = tid; c < HID * 16; c += TI_THREADS) {
    const int o = c >> 4, q = c & 15;
    *reinterpret_cast<uint4*>(S.w2 + ti_chunk(o, q)) = w2g[c];
    *reinterpret_cast<uint4*>(S.w3 + ti_chunk(o, q)) = w3g[c];
  }
  for (int i = tid; i < HID * IN; i += TI_THREADS) S.w1[i] = __bfloat162float(wb[WB_W1 + i]);
  for (int i = tid; i < OUT * HID; i += TI_THREADS) S.w4[i] = __bfloat162float(wb[WB_W4 + i]);
  for (int i = tid; i < HID; i += TI_THREADS) {
    S.b1[i] = par[OFF_B1 + i];
    S.b2[i] = par[OFF_B2 + i];
    S.b3[i] = par[OFF_B3 + i];
  }
  if (tid < OUT) S.b4[tid] = par[OFF_B4 + tid];
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tm = S.tmem;
  const int qw = w & 3, hw = w >> 2;  // this warp's TMEM lane quarter and column half
  const uint32_t t_rows = tm + ((uint32_t)(32 * qw) << 16);
  const int er = 32 * qw + lane;                      // epilogue row
  const int r1 = tid & (TI_M - 1), h1 = tid >> 7;     // layer-1 row and output half
  uint32_t phase = 0;
  bool ok = true;
  for (int64_t tile = blockIdx.x; tile < ntiles; tile += gridDim.x) {
    const int64_t row0 = tile * TI_M;
    {  // layer 1: row r1, outputs 64 h1 .. 64 h1 + 63
      const int64_t row = row0 + r1;
      float x[IN];
#pragma unroll
      for (int i = 0; i < IN; ++i) x[i] = bf16_round(row < n ? X[row * IN + i] : 0.f);
      for (int g = 0; g < 8; ++g) {
        float a[8];
#pragma unroll
        for (int j = 0; j < 8; ++j) {
          const int o = 64 * h1 + 8 * g + j;
          float acc = 0.f;
#pragma unroll
          for (int i = 0; i < IN; ++i) acc = fmaf(x[i], S.w1[o * IN + i], acc);
          a[j] = gelu(acc + S.b1[o]);
        }
        *reinterpret_cast<uint4*>(S.act + ti_chunk(r1, 8 * h1 + g)) = pack8_bf16(a);
      }
    }
    for (int layer = 0; layer < 2; ++layer) {  // layers 2 and 3
      fence_proxy_async_smem();  // the activations, written by the threads, to the MMA
      tc_fence_before();
      __syncthreads();
      tc_fence_after();
      if (tid == 0) {
        const unsigned char* Bw = layer == 0 ? S.w2 : S.w3;
#pragma unroll
        for (int kb = 0; kb < 2; ++kb) {
          const uint64_t da = desc_sw128(smem_u32(S.act + kb * TI_KB));
          const uint64_t db = desc_sw128(smem_u32(Bw + kb * TI_KB));
#pragma unroll
          for (int ks = 0; ks < 4; ++ks)  // K step of 16 BF16 = 32 bytes: + 2 in the address
            mma_f16(tm, da + 2 * ks, db + 2 * ks, TI_IDESC, (kb | ks) ? 1u : 0u);
        }
        mma_commit(&S.mbar);
      }
      bool got = mbar_wait_bounded(&S.mbar, phase, TI_WAIT_POLLS, TI_WAIT_NS);
      got = __syncthreads_and(got) != 0;
      if (!got) {
        if (tid == 0) atomicExch(err, 1);
        ok = false;
        break;
      }
      phase ^= 1u;
      tc_fence_after();
      const float* bias = layer == 0 ? S.b2 : S.b3;
      float y0 = 0.f, y1 = 0.f, y2 = 0.f;
#pragma unroll
      for (int c16 = 0; c16 < 4; ++c16) {
        const int col0 = 64 * hw + 16 * c16;
        float v[16];
        tmem_ld16(t_rows + (uint32_t)col0, v);
        tmem_wait_ld();
        float a[16];
#pragma unroll
        for (int j = 0; j < 16; ++j) a[j] = bf16_round(gelu(v[j] + bias[col0 + j]));
        if (layer == 0) {
          *reinterpret_cast<uint4*>(S.act + ti_chunk(er, col0 / 8)) = pack8_bf16(a);
          *reinterpret_cast<uint4*>(S.act + ti_chunk(er, col0 / 8 + 1)) = pack8_bf16(a + 8);
        } else {
#pragma unroll
          for (int j = 0; j < 16; ++j) {
            y0 = fmaf(a[j], S.w4[col0 + j], y0);
            y1 = fmaf(a[j], S.w4[HID + col0 + j], y1);
            y2 = fmaf(a[j], S.w4[2 * HID + col0 + j], y2);
          }
        }
      }
      if (layer == 1) {
        S.ypart[hw][er][0] = y0;
        S.ypart[hw][er][1] = y1;
        S.ypart[hw][er][2] = y2;
      }
    }
    if (!ok) break;
    tc_fence_before();
    __syncthreads();
    if (tid < TI_M && row0 + tid < n) {
      const int64_t row = row0 + tid;
#pragma unroll
      for (int o = 0; o < OUT; ++o)
        Y[row * OUT + o] = (S.ypart[0][tid][o] + S.ypart[1][tid][o]) + S.b4[o];
    }
  }
  // a timed-out batch may still be running: wait for it (bounded) before releasing TMEM
  if (!ok) mbar_wait_bounded(&S.mbar, phase, TI_WAIT_POLLS, TI_WAIT_NS);
  tc_fence_before();
  __syncthreads();
  if (w == 0) tmem_dealloc(tm, TI_COLS);
}

// Launches the tensor-core inference (at most two CTAs per SM: 128 TMEM columns each and
// ~100 KB of shared memory) and queues the read-back of its timeout flag into
// h_pinned[7]; infer_check reads it after a synchronisation.
int infer_tc(bp_ctx* ctx, int64_t n, const float* x, const uint16_t* wb, const float* par,
             float* y) {
  if (n <= 0) return BP_OK;
  if (((uintptr_t)wb & 15) != 0)
    return bp_fail(ctx, BP_EINVAL, "mlp inference: BF16 weights not 16-byte aligned");
  const size_t smem = sizeof(TiSmem) + 1024;
  BP_CUDA(ctx, cudaFuncSetAttribute(k_infer_tc, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                    (int)smem));
  BP_CUDA(ctx, cudaFuncSetAttribute(k_infer_tc, cudaFuncAttributePreferredSharedMemoryCarveout,
                                    100));
  const int64_t ntiles = (n + TI_M - 1) / TI_M;
  const int64_t grid = std::min<int64_t>(ntiles, (int64_t)ctx->num_sms * 2);
  BP_CUDA(ctx, cudaMemsetAsync(ctx->d_flags + 1, 0, sizeof(int), ctx->stream));
  k_infer_tc<<<(unsigned)grid, TI_THREADS, smem, ctx->stream>>>(
      n, x, reinterpret_cast<const __nv_bfloat16*>(wb), par, y, ctx->d_flags + 1);
  BP_LAUNCH_CHECK(ctx, "mlp infer (tensor cores)");
  BP_CUDA(ctx, cudaMemcpyAsync(ctx->h_pinned + 7, ctx->d_flags + 1, sizeof(int),
                               cudaMemcpyDeviceToHost, ctx->stream));
  return BP_OK;
}
// after a synchronisation of the stream: did an inference wait time out?
int infer_check(bp_ctx* ctx) {
  if (*reinterpret_cast<const int*>(ctx->h_pinned + 7))
    return bp_fail(ctx, BP_ETIMEOUT, "mlp inference: a tensor-core wait timed out");
  return BP_OK;
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
                               double* __restrict__ guess, unsigned long long* n_outside) {
  int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  double g0 = (double)Y[i * OUT + 0] * norm[9 + IN + 0] + norm[IN + 0];
  double g1 = (double)Y[i * OUT + 1] * norm[9 + IN + 1] + norm[IN + 1];
  if (outside[i]) {
    g0 = g1 = NAN;
    atomicAdd(n_outside, 1ull);  // an integer count: the same whatever the order
  }
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
  if ((r = infer_tc(ctx, n, x, weights_bf16, params, y))) return r;
  BP_CUDA(ctx, cudaStreamSynchronize(ctx->stream));
  return infer_check(ctx);
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
  if ((r = infer_tc(ctx, n, x, weights_bf16, mlp_params, y))) return r;
  unsigned long long* n_out = (unsigned long long*)(ctx->d_counter + 6);
  BP_CUDA(ctx, cudaMemsetAsync(n_out, 0, sizeof(int64_t), ctx->stream));
  k_decode_guess<<<(unsigned)((n + 255) / 256), 256, 0, ctx->stream>>>(n, y, norm, outside, guess,
                                                                      n_out);
  BP_LAUNCH_CHECK(ctx, "decode guess");
  BP_CUDA(ctx, cudaMemcpyAsync(ctx->h_pinned + 6, n_out, sizeof(int64_t), cudaMemcpyDeviceToHost,
                               ctx->stream));
  bp_phase_end(ctx, BP_PH_SURROGATE);
  // the prediction seeds the FP32 pre-solve; the halos outside the hull take its default
  // start (the plain solve), and count as fallbacks with those the gate rejects
  r = bp_solve_halos_ex(ctx, n, Mvir, c, z, params, guess, polish_iter > 0 ? polish_iter : 4,
                        gate, model, status,
                        polish_iter > 0 ? BP_SOLVE_FP64_SEEDED : BP_SOLVE_FP32_GATED, resid_tol);
  if (r == BP_OK || r == BP_ENOCONV) {  // the solve synchronised: the counts have arrived
    ctx->last_fallback += ctx->h_pinned[6];
    const int t = infer_check(ctx);
    if (t) return t;
  }
  return r;
}

}  // extern "C"

// bp_deposit_tc.cu -- the particle deposit (Section 3.4: the separable pixel-integrated
// kernel f_ij and the integrated SPH kernel) on the fifth-generation tensor cores.
//
// For one 64 x 64 pixel tile and a chunk of 32 particles k the y and b contributions are
//   Y[j, i] += sum_k (Y_k wy_k(j)) wx_k(i),     B[j, i] += sum_k (B_k wy_k(j)) wx_k(i),
// a rank-32 update, i.e. one 128 x 64 x 32 GEMM with the y rows and b rows stacked in M:
//   A[r, k] = Y_k wy_k(r)  (r < 64),   B_k wy_k(r - 64)  (r >= 64);    Bop[i, k] = wx_k(i).
// The weights are the FP32 values of the SIMT deposit (the same edge values and
// differences as bp_cell_weights).  Products are formed in TF32 with each FP32 operand
// split into a TF32 head (rounded) and an exact tail, a b ~ ah bh + ah bt + at bh (three
// MMAs; about 1e-6 relative error per product).  Each group of TC_G chunks accumulates in FP32
// in tensor memory and is then folded into a compensated (head, tail) pair with TwoSum,
// also kept in tensor memory.
//
// CTA: 256 threads (8 warps), persistent over work units.  Weight pass: warp w takes
// particles 4w .. 4w + 3 (K slots 4w .. 4w + 3) on both axes; lane l evaluates the
// kernel at the tile edges l and l + 32 and gets edges l + 1 and l + 33 from its
// neighbour, so every edge is evaluated once and all lanes of a warp follow one
// particle.  The weights go to shared memory as the 16-byte chunk (4 particles) of rows
// l, l + 32 (and 64 + l, 96 + l for A) of the 128-byte-swizzled K-major operand tiles.
// One thread issues the chunk's 12 MMAs (4 K-steps x 3 products) and commits them to
// the chunk's mbarrier.  Two operand stages: the weights of chunk c + 1 are built while
// the MMAs of chunk c run; one CTA barrier per chunk.  A gather warp prepares the
// particle fields of chunk c + 1 during chunk c from records copied with cp.async.
//
// TMEM (256 columns x 128 lanes): D0 = [0, 64), D1 = [64, 128) (accumulators of
// alternate groups), HI = [128, 192), LO = [192, 256).  Lane r is tile row r of y
// (r < 64) or of b (r >= 64); column i is tile column i.
//
// Every mbarrier wait is bounded; on a timeout the CTA sets *err, stops taking work,
// waits (bounded) for its MMAs in flight and frees its tensor memory.
#include "bp_internal.cuh"
#include "bp_tc.cuh"

namespace {

constexpr int TC_TS = 64;        // tile side (pixels)
constexpr int TC_CH = 32;        // particles per chunk: one 128-byte swizzle row of TF32
constexpr int TC_G = 4;          // chunks per FP32 accumulation group (128 particles)
constexpr int TC_THREADS = 256;
constexpr uint32_t TC_COLS = 256;
constexpr uint32_t COL_HI = 128, COL_LO = 192;
constexpr uint32_t TC_WAIT_POLLS = 1u << 26;
constexpr uint64_t TC_WAIT_NS = 2000000000ull;  // 2 s
constexpr uint32_t TC_IDESC = bptc::idesc_tf32(128, TC_TS);
constexpr int GATHER_WARP = 1;  // also prepares the particle fields of the next chunk
constexpr int ISSUE_TID = 64;   // lane 0 of warp 2 issues the MMAs

struct alignas(1024) TcStage {
  unsigned char a_hi[128 * 128];  // 128 rows x 32 TF32
  unsigned char a_lo[128 * 128];
  unsigned char b_hi[TC_TS * 128];  // 64 rows x 32 TF32
  unsigned char b_lo[TC_TS * 128];
};

struct TcSmem {
  TcStage st[2];
  float4 raw[2][TC_CH][2];  // raw records of chunks c + 1 and c + 2 (cp.async)
  // per-particle fields of chunks c and c + 1
  float4 p0[2][TC_CH];  // fx, fy, hp, Y
  float p1[2][TC_CH];   // B
  float ih[2][TC_CH];   // 1 / hp (0 when hp == 0)
  int2 pi[2][TC_CH];    // pixel index relative to the tile origin
  uint64_t mbar[2];
  int64_t unit;
  uint32_t tmem;
  int abort;
};

__device__ __forceinline__ void st_quad(unsigned char* base, int off, const float (&v)[4]) {
  *reinterpret_cast<float4*>(base + off) = make_float4(v[0], v[1], v[2], v[3]);
}

// per-particle fields of one record (relative to the tile origin x0, y0) into slot b, l
__device__ __forceinline__ void derive(TcSmem& S, int b, int l, float4 q0, float4 q1, int x0,
                                       int y0) {
  S.p0[b][l] = q0;
  S.p1[b][l] = q1.x;
  S.ih[b][l] = q0.z > 0.f ? 1.0f / q0.z : 0.f;
  S.pi[b][l] = make_int2(__float_as_int(q1.z) - x0, __float_as_int(q1.w) - y0);
}

// Split-form kernel value at tile edge e (the left edge of cell e, ef = (float)e) of a
// particle at pixel pr + f in tile coordinates (prf = (float)pr): the edge values of
// bp_cell_weights (ef - prf is exact, and equals (float)(e - pr)).
__device__ __forceinline__ float edge_value(float ef, float prf, float f, float ih) {
  return bp_wsplit_inv(__fsub_rn(__fsub_rn(ef, prf), f), ih);
}

// Weights of cells l and l + 32 of one axis for one particle (every lane of the warp
// calls this with the same particle).  e64: the edge value at e = 64.
__device__ __forceinline__ void lane_weights(int l, float lf, int pr, float f, float h,
                                             float ih, float e64, float& w0, float& w1) {
  if (h > 0.f) {
    const float prf = (float)pr;
    const float a0 = edge_value(lf, prf, f, ih), a1 = edge_value(lf + 32.f, prf, f, ih);
    const float t0 = __shfl_sync(0xffffffffu, a0, (l + 1) & 31);
    const float t1 = __shfl_sync(0xffffffffu, a1, (l + 1) & 31);
    const float n0 = l < 31 ? t0 : t1;   // edge l + 1 (lane 31: edge 32, from lane 0)
    const float n1 = l < 31 ? t1 : e64;  // edge l + 33
    const int kc = pr + (f > 0.f ? 0 : -1);  // the cell holding the centre
    w0 = n0 - a0;
    w1 = n1 - a1;
    if (l == kc) w0 += 1.f;
    if (l + 32 == kc) w1 += 1.f;
  } else {  // h = 0: nearest grid point
    w0 = l == pr ? 1.f : 0.f;
    w1 = l + 32 == pr ? 1.f : 0.f;
  }
}

__global__ void __launch_bounds__(TC_THREADS, 2)
    k_deposit_tc(const float4* __restrict__ rec, const uint32_t* __restrict__ pvals,
                 const BpUnit* __restrict__ units, const int64_t* __restrict__ n_units_ptr,
                 int64_t* counter, int nx, int ny, int ntx, float* ymap, float* bmap,
                 float* ylo, float* blo, float* partials, int* err) {
  using namespace bptc;
  extern __shared__ unsigned char smem_raw[];
  TcSmem& S = *reinterpret_cast<TcSmem*>(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
  const int tid = threadIdx.x, lane = tid & 31, w = tid >> 5;
  if (w == 0) {
    tmem_alloc(&S.tmem, TC_COLS);
    tmem_relinquish();
  }
  if (tid == 0) {
    mbar_init(&S.mbar[0], 1);
    mbar_init(&S.mbar[1], 1);
    fence_mbar_init();
    S.abort = 0;
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tm = S.tmem;
  const uint32_t lanes = tm + ((uint32_t)(32 * (w & 3)) << 16);  // this warp's TMEM lanes
  const uint32_t colh = (uint32_t)(32 * (w >> 2));                // its 32 of the 64 columns
  const int64_t n_units = *n_units_ptr;
  int64_t gissued = 0, gdone = 0;  // chunks issued / waited for by this CTA
  // this lane's operand chunks: rows l and l + 32 (and 64 + l, 96 + l of A), quad w
  const int o_r0 = sw128_quad(lane, w), o_r1 = sw128_quad(lane + 32, w);
  const int o_b0 = sw128_quad(TC_TS + lane, w), o_b1 = sw128_quad(TC_TS + lane + 32, w);
  const float lane_f = (float)lane;

  // waits for chunk gi (global index) to finish its MMAs
  auto wait_chunk = [&](int64_t gi) -> bool {
    bool ok = mbar_wait_bounded(&S.mbar[gi & 1], (uint32_t)((gi >> 1) & 1), TC_WAIT_POLLS,
                                TC_WAIT_NS);
    ok = __all_sync(0xffffffffu, ok);  // the TMEM loads that follow are warp-collective
    if (!ok) {
      S.abort = 1;
      atomicExch(err, 1);
    }
    gdone = gi + 1;
    tc_fence_after();
    return ok;
  };
  // folds the FP32 group accumulator into the compensated HI/LO pair
  auto fold = [&](int grp) {
    const uint32_t dcol = (uint32_t)((grp & 1) * TC_TS) + colh;
#pragma unroll
    for (int h = 0; h < 32; h += 16) {
      float x[16], hi[16], lo[16];
      tmem_ld16(lanes + dcol + h, x);
      tmem_ld16(lanes + COL_HI + colh + h, hi);
      tmem_ld16(lanes + COL_LO + colh + h, lo);
      tmem_wait_ld();
#pragma unroll
      for (int j = 0; j < 16; ++j) {
        float s, e;
        bp_two_sum(hi[j], x[j], s, e);
        hi[j] = s;
        lo[j] = lo[j] + e;
      }
      tmem_st16(lanes + COL_HI + colh + h, hi);
      tmem_st16(lanes + COL_LO + colh + h, lo);
    }
    tmem_wait_st();
  };

  for (;;) {
    if (tid == 0) S.unit = atomicAdd((unsigned long long*)counter, 1ull);
    __syncthreads();
    const int64_t u = S.unit;
    if (u >= n_units || S.abort) break;
    const BpUnit U = units[u];
    const int x0 = (U.tile % ntx) * TC_TS, y0 = (U.tile / ntx) * TC_TS;
    {  // HI = LO = 0
      float z[16];
#pragma unroll
      for (int j = 0; j < 16; ++j) z[j] = 0.f;
#pragma unroll
      for (int h = 0; h < 32; h += 16) {
        tmem_st16(lanes + COL_HI + colh + h, z);
        tmem_st16(lanes + COL_LO + colh + h, z);
      }
      tmem_wait_st();
    }
    const int nchunks = (int)((U.end - U.begin + TC_CH - 1) / TC_CH);
    const int64_t gbase = gissued;
    bool aborted = false;
    // Record pipeline, run by the gather warp (lane l = particle l of a chunk): during
    // chunk c it derives the fields of chunk c + 1 from raw[(c + 1) & 1] (copied during
    // chunk c - 1) and starts the copies of chunk c + 2; pair indices are loaded one
    // chunk ahead of their copies.  Chunk 0 is gathered synchronously.
    uint32_t pv_next = 0;
    if (w == GATHER_WARP) {
      const int64_t q = U.begin + lane;
      if (q < U.end) {
        const uint32_t pv = pvals[q];
        derive(S, 0, lane, rec[2 * (int64_t)pv], rec[2 * (int64_t)pv + 1], x0, y0);
      }
      if (q + TC_CH < U.end) {
        const uint32_t pv = pvals[q + TC_CH];
        cp_async16(&S.raw[1][lane][0], rec + 2 * (int64_t)pv);
        cp_async16(&S.raw[1][lane][1], rec + 2 * (int64_t)pv + 1);
      }
      cp_async_commit();
      if (q + 2 * TC_CH < U.end) pv_next = pvals[q + 2 * TC_CH];
    }
    __syncthreads();
    for (int c = 0; c < nchunks; ++c) {
      const int64_t gi = gbase + c;
      const int s = (int)(gi & 1);
      const int b = c & 1;  // field buffer of this chunk
      if (c >= 2) {  // stage s is free once chunk c - 2 is done
        const int cp = c - 2;
        if (wait_chunk(gi - 2) && (cp % TC_G == TC_G - 1)) fold(cp / TC_G);
      }
      const int64_t cb = U.begin + (int64_t)c * TC_CH;
      const int nch = (int)min((int64_t)TC_CH, U.end - cb);
      // 1. weights of particles 4w .. 4w + 3 -> operand stage s
      TcStage& T = S.st[s];
      // edge 64 of the 8 (axis, particle) pairs: lane j < 8 evaluates pair j
      float e64 = 0.f;
      if (lane < 8) {
        const int k = 4 * w + (lane & 3), ax = lane >> 2;
        if (k < nch) {
          const float4 q = S.p0[b][k];
          const int2 ip = S.pi[b][k];
          if (q.z > 0.f)
            e64 = edge_value((float)TC_TS, (float)(ax ? ip.y : ip.x), ax ? q.y : q.x, S.ih[b][k]);
        }
      }
      float wx0[4], wx1[4], wy0[4], wy1[4], Yk[4], Bk[4];
#pragma unroll
      for (int p = 0; p < 4; ++p) {
        const int k = 4 * w + p;
        const float ex = __shfl_sync(0xffffffffu, e64, p);
        const float ey = __shfl_sync(0xffffffffu, e64, 4 + p);
        if (k < nch) {  // warp-uniform
          const float4 q = S.p0[b][k];
          const int2 ip = S.pi[b][k];
          const float ih = S.ih[b][k];
          lane_weights(lane, lane_f, ip.x, q.x, q.z, ih, ex, wx0[p], wx1[p]);
          lane_weights(lane, lane_f, ip.y, q.y, q.z, ih, ey, wy0[p], wy1[p]);
          Yk[p] = q.w;
          Bk[p] = S.p1[b][k];
        } else {
          wx0[p] = wx1[p] = wy0[p] = wy1[p] = Yk[p] = Bk[p] = 0.f;
        }
      }
#pragma unroll
      for (int half = 0; half < 2; ++half) {  // column weights: the B operand
        float h4[4], l4[4];
#pragma unroll
        for (int p = 0; p < 4; ++p) {
          split_tf32(half ? wx1[p] : wx0[p], h4[p], l4[p]);
        }
        st_quad(T.b_hi, half ? o_r1 : o_r0, h4);
        st_quad(T.b_lo, half ? o_r1 : o_r0, l4);
      }
#pragma unroll
      for (int half = 0; half < 2; ++half) {  // Y and B times row weights: the A operand
        float hy[4], ly[4], hb[4], lb[4];
#pragma unroll
        for (int p = 0; p < 4; ++p) {
          const float wv = half ? wy1[p] : wy0[p];
          split_tf32(__fmul_rn(Yk[p], wv), hy[p], ly[p]);
          split_tf32(__fmul_rn(Bk[p], wv), hb[p], lb[p]);
        }
        st_quad(T.a_hi, half ? o_r1 : o_r0, hy);
        st_quad(T.a_lo, half ? o_r1 : o_r0, ly);
        st_quad(T.a_hi, half ? o_b1 : o_b0, hb);
        st_quad(T.a_lo, half ? o_b1 : o_b0, lb);
      }
      // 2. the gather warp prepares chunk c + 1 and starts the copies of chunk c + 2
      if (w == GATHER_WARP && c + 1 < nchunks) {
        cp_async_wait_all();
        const int64_t qn = cb + TC_CH + lane;  // this lane's particle of chunk c + 1
        if (qn < U.end)
          derive(S, b ^ 1, lane, S.raw[(c + 1) & 1][lane][0], S.raw[(c + 1) & 1][lane][1], x0,
                 y0);
        if (qn + TC_CH < U.end) {
          cp_async16(&S.raw[c & 1][lane][0], rec + 2 * (int64_t)pv_next);
          cp_async16(&S.raw[c & 1][lane][1], rec + 2 * (int64_t)pv_next + 1);
        }
        cp_async_commit();
        if (qn + 2 * TC_CH < U.end) pv_next = pvals[qn + 2 * TC_CH];
      }
      fence_proxy_async_smem();
      tc_fence_before();
      __syncthreads();
      if (S.abort) {
        aborted = true;
        break;
      }
      // 3. one thread issues the chunk's MMAs into the group's accumulator
      if (tid == ISSUE_TID) {
        tc_fence_after();
        // K-step ks starts 32 bytes further in: + 2 in the address field (bits 0-13; no
        // carry for shared addresses below 256 KB)
        const uint64_t dah = desc_sw128(smem_u32(T.a_hi)), dal = desc_sw128(smem_u32(T.a_lo));
        const uint64_t dbh = desc_sw128(smem_u32(T.b_hi)), dbl = desc_sw128(smem_u32(T.b_lo));
        const uint32_t d = tm + (uint32_t)(((c / TC_G) & 1) * TC_TS);
#pragma unroll
        for (int ks = 0; ks < TC_CH / 8; ++ks) {
          const uint64_t o = (uint64_t)(2 * ks);
          mma_tf32(d, dah + o, dbh + o, TC_IDESC, (c % TC_G != 0 || ks > 0) ? 1u : 0u);
          mma_tf32(d, dah + o, dbl + o, TC_IDESC, 1u);
          mma_tf32(d, dal + o, dbh + o, TC_IDESC, 1u);
        }
        mma_commit(&S.mbar[s]);
      }
      ++gissued;
    }
    if (aborted) break;
    // drain the last two chunks
    for (int c = max(0, nchunks - 2); c < nchunks; ++c) {
      const bool ends = (c % TC_G == TC_G - 1) || (c == nchunks - 1);
      if (wait_chunk(gbase + c) && ends) fold(c / TC_G);
    }
    __syncthreads();
    if (S.abort) break;
    // 4. write the tile: straight into the map, or as a partial tile
    {
      const int r = 32 * (w & 3) + lane;
      const bool is_b = r >= TC_TS;
      const int jr = r & (TC_TS - 1);
#pragma unroll
      for (int h = 0; h < 32; h += 16) {
        float hi[16], lo[16];
        tmem_ld16(lanes + COL_HI + colh + h, hi);
        tmem_ld16(lanes + COL_LO + colh + h, lo);
        tmem_wait_ld();
        const int cx = (int)colh + h;
        if (U.slot < 0) {
          const int gy = y0 + jr;
          if (gy < ny) {
            float* map = is_b ? bmap : ymap;
            float* mlo = is_b ? blo : ylo;
#pragma unroll
            for (int j = 0; j < 16; ++j) {
              const int gx = x0 + cx + j;
              if (gx >= nx) continue;
              const int64_t p = (int64_t)gy * nx + gx;
              float sm, e;
              bp_two_sum(map[p], hi[j], sm, e);
              map[p] = sm;
              mlo[p] = mlo[p] + (lo[j] + e);
            }
          }
        } else {
          float* P = partials + (int64_t)U.slot * 4 * TC_TS * TC_TS +
                     (is_b ? 2 : 0) * TC_TS * TC_TS + jr * TC_TS + cx;
#pragma unroll
          for (int j = 0; j < 16; j += 4) {
            *reinterpret_cast<float4*>(P + j) =
                make_float4(hi[j], hi[j + 1], hi[j + 2], hi[j + 3]);
            *reinterpret_cast<float4*>(P + TC_TS * TC_TS + j) =
                make_float4(lo[j], lo[j + 1], lo[j + 2], lo[j + 3]);
          }
        }
      }
    }
  }
  // let every issued MMA finish (bounded) before the tensor memory is released
  while (gdone < gissued) {
    if (!wait_chunk(gdone)) break;
  }
  tc_fence_before();
  __syncthreads();
  if (w == 0) tmem_dealloc(tm, TC_COLS);
}

}  // namespace

// Launches the tensor-core deposit over the work units; the tile side is 64.  The CTA
// count is the resident capacity (at most 2 per SM: 256 TMEM columns each) capped by
// max_units.  Sets the context's device flag 0 on a timed-out wait.
int bp_deposit_tc_launch(bp_ctx* ctx, const float* assigned, const uint32_t* vals,
                         const BpUnit* units, const int64_t* n_units_dev, int64_t* counter,
                         int64_t max_units, const bp_map_geom* g, float* ymap, float* bmap,
                         float* ylo, float* blo, float* partials) {
  const int ntx = (g->nx + TC_TS - 1) / TC_TS;
  const size_t smem = sizeof(TcSmem) + 1024;
  BP_CUDA(ctx, cudaFuncSetAttribute(k_deposit_tc, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                    (int)smem));
  // the largest shared-memory carveout, so that two CTAs fit on an SM
  BP_CUDA(ctx, cudaFuncSetAttribute(k_deposit_tc,
                                    cudaFuncAttributePreferredSharedMemoryCarveout, 100));
  int per_sm = 0;
  BP_CUDA(ctx, cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_deposit_tc, TC_THREADS,
                                                             smem));
  int dev = 0, sm_bytes = 0, reserved = 0;
  BP_CUDA(ctx, cudaGetDevice(&dev));
  BP_CUDA(ctx, cudaDeviceGetAttribute(&sm_bytes, cudaDevAttrMaxSharedMemoryPerMultiprocessor, dev));
  BP_CUDA(ctx, cudaDeviceGetAttribute(&reserved, cudaDevAttrReservedSharedMemoryPerBlock, dev));
  const int fit = sm_bytes / (int)(smem + reserved);  // by shared memory alone
  if (per_sm < fit) per_sm = fit;  // registers allow 2 (__launch_bounds__)
  if (per_sm < 1) per_sm = 1;
  if (per_sm > 2) per_sm = 2;  // TMEM: 2 x 256 columns per SM
  int64_t grid = (int64_t)ctx->num_sms * per_sm;
  if (grid > max_units) grid = max_units;
  if (grid < 1) grid = 1;
  BP_CUDA(ctx, cudaMemsetAsync(ctx->d_flags, 0, sizeof(int), ctx->stream));
  k_deposit_tc<<<(unsigned)grid, TC_THREADS, smem, ctx->stream>>>(
      reinterpret_cast<const float4*>(assigned), vals, units, n_units_dev, counter, g->nx, g->ny,
      ntx, ymap, bmap, ylo, blo, partials, ctx->d_flags);
  BP_LAUNCH_CHECK(ctx, "deposit (tensor cores)");
  return BP_OK;
}

// Reads the device flag the tensor-core deposit sets on a timed-out wait (synchronises
// the context's stream).
int bp_deposit_tc_check(bp_ctx* ctx) {
  int* h = reinterpret_cast<int*>(ctx->h_pinned + 3);
  BP_CUDA(ctx, cudaMemcpyAsync(h, ctx->d_flags, sizeof(int), cudaMemcpyDeviceToHost,
                               ctx->stream));
  BP_CUDA(ctx, cudaStreamSynchronize(ctx->stream));
  if (*h) return bp_fail(ctx, BP_ETIMEOUT, "deposit: a tensor-core wait timed out");
  return BP_OK;
}

// Loads the tensor-core deposit kernel (CUDA loads modules lazily: its first launch would
// otherwise load its code into device memory).
int bp_deposit_tc_preload(bp_ctx* ctx) {
  cudaFuncAttributes a;
  BP_CUDA(ctx, cudaFuncGetAttributes(&a, k_deposit_tc));
  return BP_OK;
}

// bp_deposit_tc.cu -- the particle deposit (Section 3.4: the separable pixel-integrated
// kernel f_ij and the integrated SPH kernel) on the fifth-generation tensor cores.
//
// For one 64 x 64 pixel tile and a chunk of 32 particles k the y and b contributions are
//   Y[j, i] += sum_k (Y_k wy_k(j)) wx_k(i),     B[j, i] += sum_k (B_k wy_k(j)) wx_k(i),
// a rank-32 update, i.e. one 128 x 64 x 32 GEMM with the y rows and b rows stacked in M:
//   A[r, k] = Y_k wy_k(r)  (r < 64),   B_k wy_k(r - 64)  (r >= 64);    Bop[i, k] = wx_k(i).
// The weights are the FP32 values the SIMT deposit uses (bp_cell_weights).  Products
// are formed in TF32 with each FP32 operand split into a TF32 head and a TF32 tail,
// a b ~ ah bh + ah bt + at bh (three MMAs; about 1e-6 relative error per product).
// Each group of TC_G chunks accumulates in FP32 in tensor memory and is then folded
// into a compensated (head, tail) pair with TwoSum, also kept in tensor memory.
//
// CTA: 256 threads, persistent over work units.  Per chunk every thread computes 4 x 4
// weights (4 particles x 4 cells of one axis) and stores them as 16-byte chunks of the
// 128-byte-swizzled K-major operand tiles; one thread issues the 12 MMAs
// (4 K-steps x 3 products) and commits them to the chunk's mbarrier.  Two operand
// stages: the weights of chunk c + 1 are built while the MMAs of chunk c run.
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
constexpr int TC_G = 4;          // chunks per FP32 accumulation group
constexpr int TC_THREADS = 256;
constexpr uint32_t TC_COLS = 256;
constexpr uint32_t COL_HI = 128, COL_LO = 192;
constexpr uint32_t TC_WAIT_POLLS = 1u << 26;
constexpr uint64_t TC_WAIT_NS = 2000000000ull;  // 2 s
constexpr uint32_t TC_IDESC = bptc::idesc_tf32(128, TC_TS);

struct alignas(1024) TcStage {
  unsigned char a_hi[128 * 128];  // 128 rows x 32 TF32
  unsigned char a_lo[128 * 128];
  unsigned char b_hi[TC_TS * 128];  // 64 rows x 32 TF32
  unsigned char b_lo[TC_TS * 128];
};

struct TcSmem {
  TcStage st[2];
  float4 raw[2][TC_CH][2];  // records of the current and the next chunk (cp.async)
  float4 p0[TC_CH];   // fx, fy, hp, Y
  float p1[TC_CH];    // B
  float ih[TC_CH];    // 1 / hp (0 when hp == 0)
  int2 pi[TC_CH];     // pixel index relative to the tile origin
  int4 box[TC_CH];    // footprint in tile coordinates (i0 > i1: none)
  uint64_t mbar[2];
  int64_t unit;
  uint32_t tmem;
  int abort;
};

__device__ __forceinline__ void st_quad(unsigned char* base, int off, const float (&v)[4]) {
  *reinterpret_cast<float4*>(base + off) = make_float4(v[0], v[1], v[2], v[3]);
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
  // weight-pass role: cells 4 seg .. 4 seg + 3 of one axis for the particles
  // kq + 8 p (p = 0..3), stored in K slots 4 kq + p (A and B use the same order, and
  // the eight lanes of a quarter warp read eight consecutive particles)
  const int kq = tid & 7, seg = (tid >> 3) & 15, axis = tid >> 7;
  const int cb0 = 4 * seg;
  const int64_t n_units = *n_units_ptr;
  int64_t gissued = 0, gdone = 0;  // chunks issued / waited for by this CTA

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
    // Record pipeline (threads 0..31, one particle each): the records of chunk c + 1
    // are copied into raw[(c + 1) & 1] while chunk c is processed; the pair index of
    // chunk c + 2 is loaded one chunk earlier still.
    uint32_t pv_next = 0;
    if (tid < TC_CH) {
      const int64_t q = U.begin + tid;
      if (q < U.end) {
        const uint32_t pv = pvals[q];
        cp_async16(&S.raw[0][tid][0], rec + 2 * (int64_t)pv);
        cp_async16(&S.raw[0][tid][1], rec + 2 * (int64_t)pv + 1);
      }
      cp_async_commit();
      if (q + TC_CH < U.end) pv_next = pvals[q + TC_CH];
    }
    for (int c = 0; c < nchunks; ++c) {
      const int64_t gi = gbase + c;
      const int s = (int)(gi & 1);
      if (c >= 2) {  // stage s is free once chunk c - 2 is done
        const int cp = c - 2;
        if (wait_chunk(gi - 2) && (cp % TC_G == TC_G - 1)) fold(cp / TC_G);
      }
      // 1. the chunk's records: derived fields; start the copies of the next chunk
      const int64_t cb = U.begin + (int64_t)c * TC_CH;
      const int nch = (int)min((int64_t)TC_CH, U.end - cb);
      if (tid < TC_CH) {
        cp_async_wait_all();
        const float4 q0 = S.raw[c & 1][tid][0];
        const float4 q1 = S.raw[c & 1][tid][1];
        const int64_t qn = cb + TC_CH + tid;
        if (qn < U.end) {
          cp_async16(&S.raw[(c + 1) & 1][tid][0], rec + 2 * (int64_t)pv_next);
          cp_async16(&S.raw[(c + 1) & 1][tid][1], rec + 2 * (int64_t)pv_next + 1);
        }
        cp_async_commit();
        if (qn + TC_CH < U.end) pv_next = pvals[qn + TC_CH];
        S.p0[tid] = q0;
        S.p1[tid] = q1.x;
        S.ih[tid] = q0.z > 0.f ? 1.0f / q0.z : 0.f;
        const int ixp = __float_as_int(q1.z), iyp = __float_as_int(q1.w);
        S.pi[tid] = make_int2(ixp - x0, iyp - y0);
        int i0, i1, j0, j1;
        int4 bx = make_int4(1, 0, 1, 0);
        if (bp_span(ixp, q0.x, q0.z, nx, i0, i1) && bp_span(iyp, q0.y, q0.z, ny, j0, j1)) {
          bx.x = max(i0 - x0, 0);
          bx.y = min(i1 - x0, TC_TS - 1);
          bx.z = max(j0 - y0, 0);
          bx.w = min(j1 - y0, TC_TS - 1);
        }
        S.box[tid] = bx;  // (tid >= nch: a stale record whose weights are never used)
      }
      __syncthreads();
      if (S.abort) {
        aborted = true;
        break;
      }
      // 2. weights -> operand stage s
      TcStage& T = S.st[s];
      float wv[4][4];
#pragma unroll
      for (int p = 0; p < 4; ++p) {
        const int k = kq + 8 * p;
        int lo = 1, hi = 0;
        if (k < nch) {
          const int4 bx = S.box[k];
          lo = axis ? bx.z : bx.x;
          hi = axis ? bx.w : bx.y;
        }
        if (hi < cb0 || lo > cb0 + 3) {
#pragma unroll
          for (int j = 0; j < 4; ++j) wv[p][j] = 0.f;
        } else {
          const float4 q = S.p0[k];
          const int2 ip = S.pi[k];
          bp_cell_weights<4>(cb0 - (axis ? ip.y : ip.x), axis ? q.y : q.x, q.z, S.ih[k],
                             wv[p]);
        }
      }
      if (axis == 0) {  // column weights: the B operand
#pragma unroll
        for (int j = 0; j < 4; ++j) {
          float h4[4], l4[4];
#pragma unroll
          for (int p = 0; p < 4; ++p) {
            h4[p] = tf32_rna(wv[p][j]);
            l4[p] = tf32_rna(wv[p][j] - h4[p]);
          }
          const int off = sw128_quad(cb0 + j, kq);
          st_quad(T.b_hi, off, h4);
          st_quad(T.b_lo, off, l4);
        }
      } else {  // Y and B times row weights: the A operand
        float Yk[4], Bk[4];
#pragma unroll
        for (int p = 0; p < 4; ++p) {
          const int k = kq + 8 * p;
          Yk[p] = k < nch ? S.p0[k].w : 0.f;
          Bk[p] = k < nch ? S.p1[k] : 0.f;
        }
#pragma unroll
        for (int j = 0; j < 4; ++j) {
          float hy[4], ly[4], hb[4], lb[4];
#pragma unroll
          for (int p = 0; p < 4; ++p) {
            const float vy = Yk[p] * wv[p][j], vb = Bk[p] * wv[p][j];
            hy[p] = tf32_rna(vy);
            ly[p] = tf32_rna(vy - hy[p]);
            hb[p] = tf32_rna(vb);
            lb[p] = tf32_rna(vb - hb[p]);
          }
          const int oy = sw128_quad(cb0 + j, kq), ob = sw128_quad(TC_TS + cb0 + j, kq);
          st_quad(T.a_hi, oy, hy);
          st_quad(T.a_lo, oy, ly);
          st_quad(T.a_hi, ob, hb);
          st_quad(T.a_lo, ob, lb);
        }
      }
      fence_proxy_async_smem();
      tc_fence_before();
      __syncthreads();
      // 3. one thread issues the chunk's MMAs into the group's accumulator
      if (tid == 0) {
        tc_fence_after();
        const uint32_t ah = smem_u32(T.a_hi), al = smem_u32(T.a_lo);
        const uint32_t bh = smem_u32(T.b_hi), bl = smem_u32(T.b_lo);
        const uint32_t d = tm + (uint32_t)(((c / TC_G) & 1) * TC_TS);
#pragma unroll
        for (int ks = 0; ks < TC_CH / 8; ++ks) {
          const uint64_t dah = desc_sw128(ah + 32 * ks), dal = desc_sw128(al + 32 * ks);
          const uint64_t dbh = desc_sw128(bh + 32 * ks), dbl = desc_sw128(bl + 32 * ks);
          mma_tf32(d, dah, dbh, TC_IDESC, (c % TC_G != 0 || ks > 0) ? 1u : 0u);
          mma_tf32(d, dah, dbl, TC_IDESC, 1u);
          mma_tf32(d, dal, dbh, TC_IDESC, 1u);
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

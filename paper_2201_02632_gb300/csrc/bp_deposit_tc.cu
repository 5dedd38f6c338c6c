// bp_deposit_tc.cu -- the particle deposit (Section 3.4: the separable pixel-integrated
// kernel f_ij and the integrated SPH kernel) on the fifth-generation tensor cores.
//
// For one 64 x 64 pixel tile and a chunk of 32 particles k the y and b contributions are
//   Y[j, i] += sum_k (Y_k wy_k(j)) wx_k(i),     B[j, i] += sum_k (B_k wy_k(j)) wx_k(i),
// a rank-32 update, i.e. one 128 x 64 x 32 GEMM with the y rows and b rows stacked in M:
//   A[r, k] = Y_k wy_k(r)  (r < 64),   B_k wy_k(r - 64)  (r >= 64);    Bop[i, k] = wx_k(i).
// A cell weight is the difference of the integrated kernel at the cell's two edges, in
// the split representation of bp_wsplit_inv (w(u) left of the particle, w(u) - 1 = -w(-u)
// right of it, plus 1 for the cell holding the particle).  The edge value uses the
// truncated-power form of the piecewise quartic: with a = |u|,
//   w_left(a) = (2/3) max(1 - a, 0)^4 - (8/3) max(1/2 - a, 0)^4,
// which is the inner piece 1/2 - (4/3) a + (8/3) a^3 - 2 a^4 below a = 1/2, the outer piece
// (2/3)(1 - a)^4 above and zero beyond a = 1: no branch and no piece selection (two
// saturating FMAs, four multiplies and a sign flip).  Products are formed in TF32 with each FP32 operand split into a TF32 head
// and an exact tail, a b ~ ah bh + ah bt + at bh (three MMAs; about 1e-6 relative error per
// product).  Each group of TC_G chunks accumulates in FP32 in tensor memory and is then
// folded into a compensated (sum, compensation) pair by Kahan's summation, also kept in
// tensor memory.
//
// CTA: 256 threads (8 warps), persistent over work units, 2 CTAs per SM.  Warp w owns the
// particles 4w .. 4w + 3 of every chunk (K slots 4w .. 4w + 3):
//  - it gathers their records itself, TC_BATCH = 4 chunks (16 particles) at a time, one
//    batch ahead (cp.async, one 16-byte half record per lane), and at the start of a batch
//    its 32 lanes turn them into per-(particle, axis) fields: position relative to the tile,
//    fraction, kernel scales, the cell holding the centre, the edge value at 64.  h = 0
//    becomes an infinite kernel scale (a nearest-grid-point weight without a branch) and a
//    slot past the end of the unit a particle far outside the tile with Y = B = 0;
//  - lane l evaluates the kernel at edges l and l + 32 of both axes and takes edges l + 1,
//    l + 33 from its neighbour, so every edge is evaluated once;
//  - it writes its 16-byte chunk (4 particles) of rows l, l + 32 (and 64 + l, 96 + l of A)
//    of the 128-byte-swizzled K-major operand tiles of the chunk's stage;
//  - it arrives on the stage's mbarrier (release) and counter; the eighth warp to count
//    acquires the stage through the mbarrier, issues the chunk's 12 MMAs (4 K-steps x 3
//    products) and commits them to the stage's completion mbarrier.
// There is no CTA barrier per chunk: a warp computes its weights in registers, then waits
// only for the MMAs of the chunk that last used the stage it is about to fill (two stages),
// so warps drift by up to a chunk; a group's fold comes after the warp's next arrival.
// Each warp folds and writes out its own quarter of the tensor-memory tile (its 32 lanes,
// 32 of the 64 columns).
//
// TMEM (256 columns x 128 lanes): D0 = [0, 64), D1 = [64, 128) (accumulators of
// alternate groups), HI = [128, 192) (sums), LO = [192, 256) (compensations).  Lane r is tile
// row r of y (r < 64) or of b (r >= 64); column i is tile column i.
//
// Every wait is bounded; on a timeout the CTA sets *err, stops taking work, waits (bounded)
// for its MMAs in flight and frees its tensor memory.
#include "bp_internal.cuh"
#include "bp_tc.cuh"

namespace {

constexpr int TC_TS = 64;        // tile side (pixels)
constexpr int TC_CH = 32;        // particles per chunk: one 128-byte swizzle row of TF32
constexpr int TC_G = 4;          // chunks per FP32 accumulation group (128 particles)
constexpr int TC_WARPS = 8;
constexpr int TC_THREADS = 32 * TC_WARPS;
constexpr int TC_BATCH = 4;      // chunks whose records and fields a warp prepares at once
constexpr uint32_t TC_COLS = 256;
constexpr uint32_t COL_HI = 128, COL_LO = 192;
constexpr uint32_t TC_IDESC = bptc::idesc_tf32(128, TC_TS);
constexpr float KT = BP_KT;
constexpr float KS = BP_KS;
constexpr float NGP_IH = 1.0e38f;  // 1/h of a particle with h = 0
constexpr float FAR = -1.0e6f;     // tile position of an empty slot
#ifndef TC_SLEEP_NS
#define TC_SLEEP_NS 20000  // a waiting warp sleeps (it wakes when the phase completes)
#endif

struct alignas(1024) TcStage {
  unsigned char a_hi[128 * 128];  // 128 rows x 32 TF32
  unsigned char a_lo[128 * 128];
  unsigned char b_hi[TC_TS * 128];  // 64 rows x 32 TF32
  unsigned char b_lo[TC_TS * 128];
};

// Per-particle fields of one chunk slot (derived by the owning warp at the start of a batch).
struct TcField {
  float4 ax[2];  // per axis: position of the particle's pixel relative to the tile, fraction,
                 // KT / h, KS / h
  float4 m;      // edge value at 64 (x, y), Y, B
  int2 kc;       // cell holding the centre (x, y), relative to the tile
  int2 pad;
};

struct TcSmem {
  TcStage st[2];
  float4 raw[TC_WARPS][4 * TC_BATCH][2];  // records (two 16-byte halves) of the next batch
  TcField fld[TC_WARPS][4 * TC_BATCH];    // fields of the warp's particles of this batch
  uint64_t mbar[2];     // per stage: the chunk's MMAs completed (tcgen05.commit)
  uint64_t full[2];     // per stage: all eight warps wrote their operands (release arrivals)
  uint32_t arrive[2];   // warps arrived at each stage (cumulative, relaxed; the eighth issues)
  int64_t unit[2];
  int64_t issued;      // chunks whose MMAs were issued
  uint32_t tmem;
  int abort;
};

// Test and limit settings of the bounded waits.
struct TcWaitCfg {
  uint32_t polls;
  uint64_t ns;
  const int* stall_flag;  // non-null: every warp first waits on this flag (nothing sets it)
  uint32_t stall_polls;
};

__device__ __forceinline__ void st_quad(unsigned char* base, int off, const float (&v)[4]) {
  *reinterpret_cast<float4*>(base + off) = make_float4(v[0], v[1], v[2], v[3]);
}

// Edge value in the split representation (bp_edge_split).
__device__ __forceinline__ float edge_split(float dx, float k1, float k2) {
  return bp_edge_split(dx, k1, k2);
}

// Weights of cells l and l + 32 of one axis for one particle (all lanes of the warp call this
// with the same particle): edge values at l, l + 32, neighbours' values for l + 1, l + 33.
__device__ __forceinline__ void axis_weights(int l, float lf, float4 a, float e64, int kc,
                                             float& w0, float& w1) {
  const float v0 = edge_split(__fsub_rn(__fsub_rn(lf, a.x), a.y), a.z, a.w);
  const float v1 = edge_split(__fsub_rn(__fsub_rn(lf + 32.f, a.x), a.y), a.z, a.w);
  const float t0 = __shfl_sync(0xffffffffu, v0, (l + 1) & 31);
  const float t1 = __shfl_sync(0xffffffffu, v1, (l + 1) & 31);
  const float n0 = l < 31 ? t0 : t1;   // edge l + 1 (lane 31: edge 32, from lane 0)
  const float n1 = l < 31 ? t1 : e64;  // edge l + 33
  w0 = n0 - v0;
  w1 = n1 - v1;
  if (l == kc) w0 += 1.f;
  if (l + 32 == kc) w1 += 1.f;
}

__global__ void __launch_bounds__(TC_THREADS, 2)
    k_deposit_tc(const float4* __restrict__ rec, const uint32_t* __restrict__ pvals,
                 const BpUnit* __restrict__ units, const int64_t* __restrict__ n_units_ptr,
                 int64_t* counter, int nx, int ny, int ntx, float* ymap, float* bmap,
                 float* ylo, float* blo, float* partials, int* err, TcWaitCfg wc) {
  using namespace bptc;
  extern __shared__ __align__(1024) unsigned char smem_raw[];
  // 1024-byte alignment by pointer arithmetic on the shared array (keeps shared accesses)
  TcSmem& S = *reinterpret_cast<TcSmem*>(smem_raw +
                                         ((1024u - (smem_u32(smem_raw) & 1023u)) & 1023u));
  const int tid = threadIdx.x, lane = tid & 31, w = tid >> 5;
  if (w == 0) {
    tmem_alloc(&S.tmem, TC_COLS);
    tmem_relinquish();
  }
  if (tid == 0) {
    mbar_init(&S.mbar[0], 1);
    mbar_init(&S.mbar[1], 1);
    mbar_init(&S.full[0], TC_WARPS);
    mbar_init(&S.full[1], TC_WARPS);
    fence_mbar_init();
    S.arrive[0] = S.arrive[1] = 0u;
    S.issued = 0;
    S.abort = 0;
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tm = S.tmem;
  const uint32_t lanes = tm + ((uint32_t)(32 * (w & 3)) << 16);  // this warp's TMEM lanes
  const uint32_t colh = (uint32_t)(32 * (w >> 2));                // its 32 of the 64 columns
  const int64_t n_units = *n_units_ptr;
  // this lane's operand chunks: rows l and l + 32 (and 64 + l, 96 + l of A), quad w
  const int o_r0 = sw128_quad(lane, w), o_r1 = sw128_quad(lane + 32, w);
  const int o_b0 = sw128_quad(TC_TS + lane, w), o_b1 = sw128_quad(TC_TS + lane + 32, w);
  const float lane_f = (float)lane;
  int64_t gc = 0, gdone = 0;  // chunks this CTA started / this warp waited for

  auto fail = [&]() {
    S.abort = 1;
    if (lane == 0) atomicExch(err, 1);
  };
  // test hook: a bounded wait on a flag that nothing sets, before any MMA is issued
  if (wc.stall_flag) {
    bool ok = false;
    for (uint32_t it = 0; it < wc.stall_polls && !ok; ++it)
      ok = *reinterpret_cast<const volatile int*>(wc.stall_flag) != 0;
    if (!__all_sync(0xffffffffu, ok)) fail();
  }
  __syncthreads();
  // waits for the MMAs of chunk gi (global index) to complete
  auto wait_chunk = [&](int64_t gi) -> bool {
    bool ok = TC_SLEEP_NS > 0 ? mbar_wait_bounded_sleep(&S.mbar[gi & 1], (uint32_t)((gi >> 1) & 1),
                                                        wc.polls, wc.ns, TC_SLEEP_NS)
                              : mbar_wait_bounded(&S.mbar[gi & 1], (uint32_t)((gi >> 1) & 1),
                                                  wc.polls, wc.ns);
    ok = __all_sync(0xffffffffu, ok);  // the TMEM accesses that follow are warp-collective
    if (!ok) fail();
    gdone = gi + 1;
    tc_fence_after();
    return ok;
  };
  // folds the FP32 group accumulator into the (sum, compensation) pair: Kahan's summation
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
        const float y = __fadd_rn(x[j], lo[j]);
        const float t = __fadd_rn(hi[j], y);
        lo[j] = __fsub_rn(y, __fsub_rn(t, hi[j]));
        hi[j] = t;
      }
      tmem_st16(lanes + COL_HI + colh + h, hi);
      tmem_st16(lanes + COL_LO + colh + h, lo);
    }
    tmem_wait_st();
  };

  int ub = 0;
  for (;;) {
    if (tid == 0) S.unit[ub] = S.abort ? n_units : atomicAdd((unsigned long long*)counter, 1ull);
    __syncthreads();
    const int64_t u = S.unit[ub];
    ub ^= 1;
    if (u >= n_units || S.abort) break;
    const BpUnit U = units[u];
    const int x0 = (U.tile % ntx) * TC_TS, y0 = (U.tile / ntx) * TC_TS;
    {  // HI = LO = 0 in this warp's quarter
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
    const int len = (int)(U.end - U.begin);  // a unit holds at most 2^30 pairs
    const uint32_t* uvals = pvals + U.begin;
    const int nchunks = (len + TC_CH - 1) / TC_CH;
    // records of this warp's particles, a batch of TC_BATCH chunks at a time: lane l copies
    // half l & 1 of particle l >> 1 of the batch (chunk (l >> 1) / 4, slot 4 w + (l >> 1) % 4)
    const int cp_p = lane >> 1, cp_h = lane & 1;
    const int cp_q0 = (cp_p >> 2) * TC_CH + 4 * w + (cp_p & 3);  // relative to the unit
    uint32_t pv_next = 0;
    {
      if (cp_q0 < len) cp_async16(&S.raw[w][cp_p][cp_h], rec + 2 * (int64_t)uvals[cp_q0] + cp_h);
      cp_async_commit();
      const int q1 = cp_q0 + TC_BATCH * TC_CH;
      if (q1 < len) pv_next = uvals[q1];
    }
    bool aborted = false;
    for (int c = 0; c < nchunks; ++c, ++gc) {
      const int s = (int)(gc & 1);
      const int cb = c % TC_BATCH;
      if (cb == 0) {
        // 1. the batch's records have landed: its fields, one (particle, axis) per lane
        cp_async_wait_all();
        __syncwarp();
        {
          const int p = lane & 15, ax = lane >> 4;
          const int q = (c + (p >> 2)) * TC_CH + 4 * w + (p & 3);
          TcField& F = S.fld[w][p];
          float4 a;
          float e64;
          int kc;
          if (q < len) {
            const float4 r0 = S.raw[w][p][0], r1 = S.raw[w][p][1];
            float f = ax ? r0.y : r0.x;
            const int pr = __float_as_int(ax ? r1.w : r1.z) - (ax ? y0 : x0);
            const bool ngp = !(r0.z > 0.f);
            const float ih = ngp ? NGP_IH : __frcp_rn(r0.z);
            if (ngp && !(f > 0.f)) f = 1.0e-30f;  // exactly on an edge: the cell to its right
            a = make_float4((float)pr, f, KT * ih, KS * ih);
            kc = pr + (f > 0.f ? 0 : -1);
            e64 = edge_split(__fsub_rn(__fsub_rn((float)TC_TS, a.x), a.y), a.z, a.w);
            if (ax == 0) {
              F.m.z = r0.w;
              F.m.w = r1.x;
            }
          } else {  // empty slot: far outside the tile, no signal
            a = make_float4(FAR, 0.5f, KT, KS);
            kc = -(1 << 30);
            e64 = 0.f;
            if (ax == 0) {
              F.m.z = 0.f;
              F.m.w = 0.f;
            }
          }
          F.ax[ax] = a;
          if (ax == 0) {
            F.m.x = e64;
            F.kc.x = kc;
          } else {
            F.m.y = e64;
            F.kc.y = kc;
          }
        }
        __syncwarp();
        // 2. the next batch's records on their way (the record buffer is free: its fields are
        // derived), the index of the one after
        const int q1 = cp_q0 + (c + TC_BATCH) * TC_CH;
        if (q1 < len) cp_async16(&S.raw[w][cp_p][cp_h], rec + 2 * (int64_t)pv_next + cp_h);
        cp_async_commit();
        const int q2 = q1 + TC_BATCH * TC_CH;
        pv_next = q2 < len ? uvals[q2] : 0u;
      }
      // 3. weights of particles 4w .. 4w + 3 (in registers: the stage may still be busy)
      TcStage& T = S.st[s];
      float wx0[4], wx1[4], wy0[4], wy1[4], Yk[4], Bk[4];
#pragma unroll
      for (int p = 0; p < 4; ++p) {
        const TcField& F = S.fld[w][4 * cb + p];
        const float4 m = F.m;
        const int2 kc = F.kc;
        axis_weights(lane, lane_f, F.ax[0], m.x, kc.x, wx0[p], wx1[p]);
        axis_weights(lane, lane_f, F.ax[1], m.y, kc.y, wy0[p], wy1[p]);
        Yk[p] = m.z;
        Bk[p] = m.w;
      }
      // 4. stage s is free once the MMAs of chunk gc - 2 are done; a group that ended there
      // is folded after this chunk's arrival
      bool fold_now = false;
      if (gc >= 2 && gdone <= gc - 2) {
        if (!wait_chunk(gc - 2)) {
          aborted = true;
          break;
        }
        fold_now = c >= 2 && (c - 2) % TC_G == TC_G - 1;
      }
#pragma unroll
      for (int half = 0; half < 2; ++half) {  // column weights: the B operand
        float h4[4], l4[4];
#pragma unroll
        for (int p = 0; p < 4; ++p) split_tf32(half ? wx1[p] : wx0[p], h4[p], l4[p]);
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
      fence_proxy_async_smem();
      tc_fence_before();
      __syncwarp();
      // 5. arrive (release, on the stage's mbarrier); the warp whose count is the eighth
      // acquires the stage through that mbarrier and issues the chunk's MMAs into the group's
      // accumulator (the counter only elects the issuer: a relaxed atomic, no memory fence)
      if (lane == 0) {
        mbar_arrive(&S.full[s]);
        const uint32_t old = atomicAdd(&S.arrive[s], 1u);
        bool issue = (old & (TC_WARPS - 1)) == TC_WARPS - 1;
        if (issue &&
            !(TC_SLEEP_NS > 0 ? mbar_wait_bounded_sleep(&S.full[s], (uint32_t)((gc >> 1) & 1),
                                                        wc.polls, wc.ns, TC_SLEEP_NS)
                              : mbar_wait_bounded(&S.full[s], (uint32_t)((gc >> 1) & 1),
                                                  wc.polls, wc.ns))) {
          issue = false;  // the other warps time out on this chunk's MMAs in turn
          S.abort = 1;
          atomicExch(err, 1);
        }
        if (issue) {
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
          S.issued = gc + 1;
        }
      }
      __syncwarp();
      // the group's accumulator is overwritten only by the MMAs of chunk c + 3 (the first of
      // group (c - 2) / TC_G + 2), which wait for this warp's arrival there
      if (fold_now) fold((c - 2) / TC_G);
    }
    cp_async_wait_all();  // no copy outlives the unit
    if (!aborted) {
      // drain: the last chunks of the unit, folding the last group(s)
      for (int64_t gw = max(gdone, gc - 2); gw < gc; ++gw) {
        const int cw = (int)(gw - (gc - nchunks));
        if (!wait_chunk(gw)) {
          aborted = true;
          break;
        }
        if (cw % TC_G == TC_G - 1 || cw == nchunks - 1) fold(cw / TC_G);
      }
    }
    if (aborted) continue;  // the next unit fetch sees S.abort
    // 6. write this warp's quarter of the tile: into the map, or as a partial tile
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
            if (!BP_DCHECK(p >= 0 && p < (int64_t)nx * ny, err + BP_DBG_SLOT, 401)) continue;
            float sm, e;
            bp_two_sum(map[p], hi[j], sm, e);
            map[p] = sm;
            mlo[p] = mlo[p] + (lo[j] + e);
          }
        }
      } else {
        if (!BP_DCHECK(jr * TC_TS + cx + 16 <= TC_TS * TC_TS, err + BP_DBG_SLOT, 402)) continue;
        float* P = partials + (int64_t)U.slot * 4 * TC_TS * TC_TS +
                   (is_b ? 2 : 0) * TC_TS * TC_TS + jr * TC_TS + cx;
#pragma unroll
        for (int j = 0; j < 16; j += 4) {
          *reinterpret_cast<float4*>(P + j) = make_float4(hi[j], hi[j + 1], hi[j + 2], hi[j + 3]);
          *reinterpret_cast<float4*>(P + TC_TS * TC_TS + j) =
              make_float4(lo[j], lo[j + 1], lo[j + 2], lo[j + 3]);
        }
      }
    }
  }
  // every issued MMA must finish (bounded) before the tensor memory is released
  __syncthreads();
  const int64_t issued = S.issued;
  while (gdone < issued) {
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
  TcWaitCfg wc;
  wc.polls = 1u << 26;
  wc.ns = 2000000000ull;  // 2 s
  wc.stall_flag = nullptr;
  wc.stall_polls = 0;
  if (ctx->test_stall_polls > 0) {  // test of the timeout path: flag 2 is zero and stays zero
    BP_CUDA(ctx, cudaMemsetAsync(ctx->d_flags + 2, 0, sizeof(int), ctx->stream));
    wc.stall_flag = ctx->d_flags + 2;
    wc.stall_polls = (uint32_t)ctx->test_stall_polls;
  }
  BP_CUDA(ctx, cudaMemsetAsync(ctx->d_flags, 0, sizeof(int), ctx->stream));
  k_deposit_tc<<<(unsigned)grid, TC_THREADS, smem, ctx->stream>>>(
      reinterpret_cast<const float4*>(assigned), vals, units, n_units_dev, counter, g->nx, g->ny,
      ntx, ymap, bmap, ylo, blo, partials, ctx->d_flags, wc);
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

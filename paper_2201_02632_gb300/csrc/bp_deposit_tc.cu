// bp_deposit_tc.cu -- the particle deposit (Section 3.4: the separable pixel-integrated
// kernel f_ij and the integrated SPH kernel) on the fifth-generation tensor cores.
//
// For one 64 x 64 pixel tile and a chunk of 64 particles k the y and b contributions are
//   Y[j, i] += sum_k (Y_k wy_k(j)) wx_k(i),     B[j, i] += sum_k (B_k wy_k(j)) wx_k(i),
// a rank-64 update, i.e. one 128 x 64 x 64 GEMM with the y rows and b rows stacked in M:
//   A[r, k] = Y_k wy_k(r)  (r < 64),   B_k wy_k(r - 64)  (r >= 64);    Bop[i, k] = wx_k(i).
// A cell weight is the difference of the integrated kernel at the cell's two edges, in
// the split representation of bp_wsplit_inv (w(u) left of the particle, w(u) - 1 = -w(-u)
// right of it, plus 1 for the cell holding the particle).  The edge value uses the
// truncated-power form of the piecewise quartic: with a = |u|,
//   w_left(a) = (2/3) max(1 - a, 0)^4 - (8/3) max(1/2 - a, 0)^4,
// which is the inner piece 1/2 - (4/3) a + (8/3) a^3 - 2 a^4 below a = 1/2, the outer piece
// (2/3)(1 - a)^4 above and zero beyond a = 1: no branch and no piece selection (two
// saturating FMAs, four multiplies and a sign flip).
//
// Products are formed by kind::f16 MMAs on FP16 operands: each FP32 operand is scaled by a
// power of two and split into an FP16 head (11 significant bits) and the FP16 rounding of the
// exact rest, a b ~ ah bh + ah bt + at bh (three MMAs; about 1e-6 relative error per product).
// The column weights (at most 1) are scaled by 2^14; the A rows by 2^s per accumulation
// group, s chosen from the group's largest |Y| (|B| for the b rows) so that the largest
// value lies in [2^14, 2^15): far below the FP16 maximum, and contributions that would fall
// below the FP16 normal range are below 2^-28 of the group's largest.  Each group of TC_G
// chunks (128 particles) accumulates in FP32 in tensor memory; its scale is undone exactly
// (a power of two) when it is folded into a compensated (sum, compensation) pair by Kahan's
// summation, also kept in tensor memory.  FP16 operands take half the shared memory of FP32
// ones, so a stage holds 64 particles and a chunk needs half the MMAs per particle.
//
// CTA: 256 threads (8 warps), persistent over work units, 2 CTAs per SM.  Warp w owns the
// particles 8w .. 8w + 7 of every chunk (K slots 8w .. 8w + 7, the 16-byte chunk w of each
// 128-byte operand row):
//  - it gathers their records itself, a batch of TC_BATCH chunks (one accumulation group,
//    16 particles) at a time, one batch ahead (cp.async, one 16-byte half record per lane),
//    and at the start of a batch its 32 lanes turn them into per-(particle, axis) fields:
//    position relative to the tile, fraction, kernel scales, the cell holding the centre, the
//    edge value at 64.  h = 0 becomes an infinite kernel scale (a nearest-grid-point weight
//    without a branch) and a slot past the end of the unit a particle far outside the tile
//    with Y = B = 0.  It then publishes its largest |Y| and |B| for the group's scale
//    (per-warp slots and an mbarrier per slot, four slots in rotation);
//  - lane l evaluates the kernel at edges l and l + 32 of both axes and takes edges l + 1,
//    l + 33 from its neighbour, so every edge is evaluated once; the warp does so for four
//    of its particles at a time and writes their 8 bytes of rows l, l + 32 (and 64 + l,
//    96 + l of A) of the 128-byte-swizzled K-major operand tiles of the chunk's stage;
//  - it arrives on the stage's mbarrier (release) and counter; the eighth warp to count
//    acquires the stage through the mbarrier, issues the chunk's 12 MMAs (4 K-steps x 3
//    products) and commits them to the stage's completion mbarrier.
// There is no CTA barrier per chunk: a warp computes the weights of its first four particles
// in registers, then waits only for the MMAs of the chunk that last used the stage it is about
// to fill (two stages), so warps drift by up to a chunk; a group's fold comes after the warp's
// next arrival.  Each warp folds and writes out its own quarter of the tensor-memory tile (its
// 32 lanes, 32 of the 64 columns).
//
// TMEM (256 columns x 128 lanes): D0 = [0, 64), D1 = [64, 128) (accumulators of
// alternate groups), HI = [128, 192) (sums), LO = [192, 256) (compensations).  Lane r is tile
// row r of y (r < 64) or of b (r >= 64); column i is tile column i.
//
// Every wait is bounded; on a timeout the CTA sets *err, stops taking work, waits (bounded)
// for its MMAs in flight and frees its tensor memory.
#include <cuda_fp16.h>

#include "bp_internal.cuh"
#include "bp_tc.cuh"

namespace {

constexpr int TC_TS = 64;        // tile side (pixels)
constexpr int TC_CH = 64;        // particles per chunk: one 128-byte swizzle row of FP16
constexpr int TC_KSTEPS = 4;     // MMA K-steps per chunk (K = 16 FP16 each, 32 bytes)
constexpr int TC_G = 2;          // chunks per FP32 accumulation group (128 particles)
constexpr int TC_WARPS = 8;
constexpr int TC_THREADS = 32 * TC_WARPS;
constexpr int TC_PW = TC_CH / TC_WARPS;  // particles of a chunk per warp
constexpr int TC_BATCH = TC_G;   // chunks whose records and fields a warp prepares at once
constexpr int TC_NB = TC_PW * TC_BATCH;  // particles of a batch per warp (16: one per lane pair)
constexpr int TC_SLOTS = 4;      // group-scale slots in rotation
constexpr int TC_SB = 14;        // the column weights' scale exponent
constexpr uint32_t TC_COLS = 256;
constexpr uint32_t COL_HI = 128, COL_LO = 192;
constexpr uint32_t TC_IDESC = bptc::idesc_f16(128, TC_TS);
constexpr float KT = BP_KT;
constexpr float KS = BP_KS;
constexpr float NGP_IH = 1.0e38f;  // 1/h of a particle with h = 0
constexpr float FAR = -1.0e6f;     // tile position of an empty slot
#ifndef TC_SLEEP_NS
#define TC_SLEEP_NS 20000  // a waiting warp sleeps (it wakes when the phase completes)
#endif
static_assert(TC_NB == 16 && TC_KSTEPS * 16 == TC_CH, "deposit chunk layout");

struct alignas(1024) TcStage {
  unsigned char a_hi[128 * 128];  // 128 rows x 64 FP16
  unsigned char a_lo[128 * 128];
  unsigned char b_hi[TC_TS * 128];  // 64 rows x 64 FP16
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
  float4 raw[TC_WARPS][TC_NB][2];  // records (two 16-byte halves) of the next batch
  TcField fld[TC_WARPS][TC_NB];    // fields of the warp's particles of this batch
  float2 wmax[TC_SLOTS][TC_WARPS];  // per group slot: each warp's largest |Y|, |B|
  float4 wsc[TC_WARPS];  // per warp: the current group's scales of Y and B, and the inverse
                         // scale of accumulator 0 and 1 for the warp's rows (y or b)
  uint64_t mbar[2];     // per stage: the chunk's MMAs completed (tcgen05.commit)
  uint64_t full[2];     // per stage: all eight warps wrote their operands (release arrivals)
  uint64_t gready[TC_SLOTS];  // per group slot: all eight warps published their maxima
  uint32_t arrive[2];   // warps arrived at each stage (cumulative, relaxed; the eighth issues)
  int64_t unit[2];
  int64_t issued;      // chunks whose MMAs were issued
  uint32_t tmem;
  int abort;
};

// two CTAs per SM: 2 x (this + 1024 alignment slack + 1024 reserved) within 228 KB
static_assert(2 * (sizeof(TcSmem) + 2048) <= 233472, "deposit shared memory");

// Test and limit settings of the bounded waits.
struct TcWaitCfg {
  uint32_t polls;
  uint64_t ns;
  const int* stall_flag;  // non-null: every warp first waits on this flag (nothing sets it)
  uint32_t stall_polls;
};

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

// 2^e as an FP32 value, -126 <= e <= 127
__device__ __forceinline__ float exp2i(int e) { return __int_as_float((e + 127) << 23); }

// Scale exponent of a group whose largest magnitude is m: m 2^s in [2^14, 2^15) (m normal),
// 0 for m = 0 or NaN; s <= 100 (a subnormal m is taken as 2^-126).
__device__ __forceinline__ int group_exp(float m) {
  if (!(m > 0.f)) return 0;
  const int e = ((__float_as_int(m) >> 23) & 0xff) - 127;
  return min(14 - max(e, -126), 100);
}

// x, y (|x|, |y| < 2^15) as FP16 heads and the FP16 roundings of their exact rests, packed in
// pairs (x in the low half)
__device__ __forceinline__ void split_f16x2(float x, float y, uint32_t& hi, uint32_t& lo) {
  const __half2 h = __floats2half2_rn(x, y);
  const float2 hf = __half22float2(h);
  const __half2 t = __floats2half2_rn(__fsub_rn(x, hf.x), __fsub_rn(y, hf.y));
  hi = *reinterpret_cast<const uint32_t*>(&h);
  lo = *reinterpret_cast<const uint32_t*>(&t);
}

__device__ __forceinline__ void st_half4(unsigned char* base, int off, uint32_t a, uint32_t b) {
  *reinterpret_cast<uint2*>(base + off) = make_uint2(a, b);
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
    for (int q = 0; q < TC_SLOTS; ++q) mbar_init(&S.gready[q], TC_WARPS);
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
  const bool b_rows = (w & 3) >= 2;  // its TMEM lanes hold b rows (else y rows)
  const int64_t n_units = *n_units_ptr;
  // this lane's operand chunks: rows l and l + 32 (and 64 + l, 96 + l of A), 16-byte chunk w
  const int o_r0 = sw128_quad(lane, w), o_r1 = sw128_quad(lane + 32, w);
  const int o_b0 = sw128_quad(TC_TS + lane, w), o_b1 = sw128_quad(TC_TS + lane + 32, w);
  const float lane_f = (float)lane;
  int64_t gc = 0, gdone = 0;  // chunks this CTA started / this warp waited for
  uint32_t gb = 0;  // batches (accumulation groups) this CTA derived (modulo 2^32)

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
  // bounded wait on an mbarrier phase, warp-collective; false (and the CTA aborts) on a timeout
  auto wait_bar = [&](uint64_t* bar, uint32_t parity) -> bool {
    bool ok = TC_SLEEP_NS > 0 ? mbar_wait_bounded_sleep(bar, parity, wc.polls, wc.ns, TC_SLEEP_NS)
                              : mbar_wait_bounded(bar, parity, wc.polls, wc.ns);
    ok = __all_sync(0xffffffffu, ok);
    if (!ok) fail();
    return ok;
  };
  // waits for the MMAs of chunk gi (global index) to complete
  auto wait_chunk = [&](int64_t gi) -> bool {
    const bool ok = wait_bar(&S.mbar[gi & 1], (uint32_t)((gi >> 1) & 1));
    gdone = gi + 1;
    tc_fence_after();  // the TMEM accesses that follow are warp-collective
    return ok;
  };
  // folds the FP32 group accumulator, its scale undone, into the (sum, compensation) pair:
  // Kahan's summation
  auto fold = [&](int grp) {
    const uint32_t dcol = (uint32_t)((grp & 1) * TC_TS) + colh;
    const float4 sc = S.wsc[w];
    const float us = (grp & 1) ? sc.w : sc.z;
#pragma unroll
    for (int h = 0; h < 32; h += 16) {
      float x[16], hi[16], lo[16];
      tmem_ld16(lanes + dcol + h, x);
      tmem_ld16(lanes + COL_HI + colh + h, hi);
      tmem_ld16(lanes + COL_LO + colh + h, lo);
      tmem_wait_ld();
#pragma unroll
      for (int j = 0; j < 16; ++j) {
        const float y = __fadd_rn(__fmul_rn(x[j], us), lo[j]);
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
    // half l & 1 of particle l >> 1 of the batch (chunk (l >> 1) / 8, slot 8 w + (l >> 1) % 8)
    const int cp_p = lane >> 1, cp_h = lane & 1;
    const int cp_q0 = (cp_p / TC_PW) * TC_CH + TC_PW * w + (cp_p % TC_PW);  // in the unit
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
        float my = 0.f, mb = 0.f;  // the largest |Y|, |B| of the warp's particles
        {
          const int p = lane & 15, ax = lane >> 4;
          const int q = (c + p / TC_PW) * TC_CH + TC_PW * w + (p % TC_PW);
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
              my = fabsf(r0.w);
              mb = fabsf(r1.x);
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
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
          my = fmaxf(my, __shfl_xor_sync(0xffffffffu, my, o));
          mb = fmaxf(mb, __shfl_xor_sync(0xffffffffu, mb, o));
        }
        // the group's maxima: this warp's slot, then its arrival (release) on the slot's
        // mbarrier; the slot is rewritten four groups later, after every warp read it
        if (lane == 0) {
          S.wmax[gb % TC_SLOTS][w] = make_float2(my, mb);
          mbar_arrive(&S.gready[gb % TC_SLOTS]);
        }
        ++gb;
        __syncwarp();
        // 2. the next batch's records on their way (the record buffer is free: its fields are
        // derived), the index of the one after
        const int q1 = cp_q0 + (c + TC_BATCH) * TC_CH;
        if (q1 < len) cp_async16(&S.raw[w][cp_p][cp_h], rec + 2 * (int64_t)pv_next + cp_h);
        cp_async_commit();
        const int q2 = q1 + TC_BATCH * TC_CH;
        pv_next = q2 < len ? uvals[q2] : 0u;
      }
      TcStage& T = S.st[s];
      // 3. weights of four of this warp's particles (slots 8 w + 4 half4 .. + 3), in registers
      float wx0[4], wx1[4], wy0[4], wy1[4], Yk[4], Bk[4];
      auto weights4 = [&](int half4) {
#pragma unroll
        for (int p = 0; p < 4; ++p) {
          const TcField& F = S.fld[w][TC_PW * cb + 4 * half4 + p];
          const float4 m = F.m;
          const int2 kc = F.kc;
          axis_weights(lane, lane_f, F.ax[0], m.x, kc.x, wx0[p], wx1[p]);
          axis_weights(lane, lane_f, F.ax[1], m.y, kc.y, wy0[p], wy1[p]);
          Yk[p] = m.z;
          Bk[p] = m.w;
        }
      };
      // ... scaled, split and stored: their 8 bytes of each operand row this lane writes
      auto store4 = [&](int half4) {
        const int hb = 8 * half4;
#pragma unroll
        for (int half = 0; half < 2; ++half) {  // column weights: the B operand
          constexpr float sb = (float)(1 << TC_SB);
          uint32_t h01, l01, h23, l23;
          split_f16x2(__fmul_rn(half ? wx1[0] : wx0[0], sb), __fmul_rn(half ? wx1[1] : wx0[1], sb),
                      h01, l01);
          split_f16x2(__fmul_rn(half ? wx1[2] : wx0[2], sb), __fmul_rn(half ? wx1[3] : wx0[3], sb),
                      h23, l23);
          st_half4(T.b_hi, (half ? o_r1 : o_r0) + hb, h01, h23);
          st_half4(T.b_lo, (half ? o_r1 : o_r0) + hb, l01, l23);
        }
        const float4 sc = S.wsc[w];
        float ys[4], bs[4];
#pragma unroll
        for (int p = 0; p < 4; ++p) {
          ys[p] = __fmul_rn(Yk[p], sc.x);
          bs[p] = __fmul_rn(Bk[p], sc.y);
        }
#pragma unroll
        for (int half = 0; half < 2; ++half) {  // Y and B times row weights: the A operand
          float wv[4];
#pragma unroll
          for (int p = 0; p < 4; ++p) wv[p] = half ? wy1[p] : wy0[p];
          uint32_t hy01, ly01, hy23, ly23, hb01, lb01, hb23, lb23;
          split_f16x2(__fmul_rn(ys[0], wv[0]), __fmul_rn(ys[1], wv[1]), hy01, ly01);
          split_f16x2(__fmul_rn(ys[2], wv[2]), __fmul_rn(ys[3], wv[3]), hy23, ly23);
          split_f16x2(__fmul_rn(bs[0], wv[0]), __fmul_rn(bs[1], wv[1]), hb01, lb01);
          split_f16x2(__fmul_rn(bs[2], wv[2]), __fmul_rn(bs[3], wv[3]), hb23, lb23);
          st_half4(T.a_hi, (half ? o_r1 : o_r0) + hb, hy01, hy23);
          st_half4(T.a_lo, (half ? o_r1 : o_r0) + hb, ly01, ly23);
          st_half4(T.a_hi, (half ? o_b1 : o_b0) + hb, hb01, hb23);
          st_half4(T.a_lo, (half ? o_b1 : o_b0) + hb, lb01, lb23);
        }
      };
      weights4(0);
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
      if (cb == 0) {
        // the group's scales, once every warp has published its maxima
        const uint32_t g = gb - 1u;
        if (!wait_bar(&S.gready[g % TC_SLOTS], (uint32_t)((g / TC_SLOTS) & 1))) {
          aborted = true;
          break;
        }
        float my = 0.f, mb = 0.f;
#pragma unroll
        for (int q = 0; q < TC_WARPS; ++q) {
          const float2 v = S.wmax[g % TC_SLOTS][q];
          my = fmaxf(my, v.x);
          mb = fmaxf(mb, v.y);
        }
        const int ey = group_exp(my), eb = group_exp(mb);
        const float us = exp2i(-(b_rows ? eb : ey) - TC_SB);
        float4 sc = S.wsc[w];
        sc.x = exp2i(ey);
        sc.y = exp2i(eb);
        if ((c / TC_G) & 1) sc.w = us; else sc.z = us;
        __syncwarp();
        if (lane == 0) S.wsc[w] = sc;
        __syncwarp();
      }
      store4(0);
      weights4(1);
      store4(1);
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
          for (int ks = 0; ks < TC_KSTEPS; ++ks) {
            const uint64_t o = (uint64_t)(2 * ks);
            mma_f16(d, dah + o, dbh + o, TC_IDESC, (c % TC_G != 0 || ks > 0) ? 1u : 0u);
            mma_f16(d, dah + o, dbl + o, TC_IDESC, 1u);
            mma_f16(d, dal + o, dbh + o, TC_IDESC, 1u);
          }
          mma_commit(&S.mbar[s]);
          S.issued = gc + 1;
        }
      }
      __syncwarp();
      // the group's accumulator is overwritten only by the MMAs of chunk c + 1 (the first of
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

// bp_hsml.cu -- SPH smoothing lengths (Section 3.4: the cubic kernel Eq. SPH_kernel and the
// effective neighbour number N_ngb).  h_i solves
//   N_eff(h) = (4 pi / 3) h^3 sum_j W(|r_i - r_j|, h) = (32/3) sum_j w(|r_i - r_j| / h) = N_ngb,
// the sum over every particle, i itself included; N_eff grows monotonically with h.
//
// The particles are put in Morton (Z-curve) order of their positions quantised to 21 bits per
// axis over the bounding cube: every cell of the implied octree, at any level, is then one
// contiguous range of the sorted keys, found by two binary searches.  Light-cone particles
// span four decades of density (halo cores to voids), which a single uniform grid cannot
// serve; the octree level is chosen per particle from its search radius instead.
//
//  k_bbox          bounding box of the positions (order-independent min / max)
//  k_morton        63-bit Morton key of every particle, as a low and a high 32-bit word
//  radix sorts     stable sort by the low word, then by the high word (bp_sort.cu):
//                  k_morton_mid carries the high words into the first order,
//                  k_morton_final assembles keys, particle ids and float4 positions
//  k_hsml          one warp per particle, in Morton order: the cube of octree cells of side
//                  >= R around it (<= 64 cells, one binary search pair per lane), its
//                  particles tested in a fixed order and the squared distances below R^2
//                  compacted into shared memory by ballot; R grows until N_eff(R) >= N_ngb,
//                  then N_eff(h) = N_ngb is solved in (0, R] by Newton inside a bisection
//                  bracket.  Every sum is lane-strided plus a fixed shuffle tree:
//                  deterministic.
#include <algorithm>
#include <cmath>
#include <cstring>

#include "bp_internal.cuh"

namespace {

constexpr int HS_WARPS = 2;           // warps per block (few: per-particle work varies widely)
constexpr int HS_CAP_MAX = 2048;      // candidate distances per warp (shared memory)
constexpr int HS_MAX_ROUNDS = 48;     // radius updates per particle
constexpr int HS_QBITS = 21;          // quantisation bits per axis (63-bit keys)
constexpr int HS_MAXCELLS = 64;       // octree cells per search cube (a multiple of 32)
constexpr float HS_CELL_FRAC = 1.0f;  // octree cells of side >= HS_CELL_FRAC R
constexpr int HS_SCAN_CAPS = 16;      // cube particles worth one scan, in buffer capacities
constexpr float HS_KNORM = 32.0f / 3.0f;

struct Cube {  // quantisation q = floor((v - v0) * inv_s), cells of side s at level 0
  float x0, y0, z0, inv_s, s;
};

__device__ __forceinline__ unsigned ordered(float v) {  // monotone float -> uint map
  unsigned u = __float_as_uint(v);
  return (u & 0x80000000u) ? ~u : (u | 0x80000000u);
}

// bb[0..2] = ordered min of x, y, z; bb[3..5] = ordered max
__global__ void k_bbox(int64_t n, const float* __restrict__ x, const float* __restrict__ y,
                       const float* __restrict__ z, unsigned* bb) {
  unsigned mn[3] = {0xffffffffu, 0xffffffffu, 0xffffffffu}, mx[3] = {0u, 0u, 0u};
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x) {
    const unsigned v[3] = {ordered(x[i]), ordered(y[i]), ordered(z[i])};
#pragma unroll
    for (int a = 0; a < 3; ++a) {
      mn[a] = min(mn[a], v[a]);
      mx[a] = max(mx[a], v[a]);
    }
  }
#pragma unroll
  for (int a = 0; a < 3; ++a) {
    for (int o = 16; o > 0; o >>= 1) {
      mn[a] = min(mn[a], __shfl_xor_sync(0xffffffffu, mn[a], o));
      mx[a] = max(mx[a], __shfl_xor_sync(0xffffffffu, mx[a], o));
    }
  }
  if ((threadIdx.x & 31) == 0) {
#pragma unroll
    for (int a = 0; a < 3; ++a) {
      atomicMin(&bb[a], mn[a]);
      atomicMax(&bb[3 + a], mx[a]);
    }
  }
}

// monotone quantisation to [0, 2^21), explicitly rounded so that every evaluation agrees
__device__ __forceinline__ uint32_t quant(float v, float v0, float inv_s) {
  const float t = __fmul_rn(__fsub_rn(v, v0), inv_s);
  constexpr float QMAX = (float)((1u << HS_QBITS) - 1);
  if (!(t > 0.f)) return 0u;
  if (t >= QMAX) return (1u << HS_QBITS) - 1u;
  return (uint32_t)t;  // truncation = floor for t > 0
}

// the 21 bits of v moved to every third bit (bit b -> bit 3b)
__device__ __forceinline__ uint64_t spread3(uint32_t v) {
  uint64_t x = v & 0x1fffffu;
  x = (x | (x << 32)) & 0x1f00000000ffffull;
  x = (x | (x << 16)) & 0x1f0000ff0000ffull;
  x = (x | (x << 8)) & 0x100f00f00f00f00full;
  x = (x | (x << 4)) & 0x10c30c30c30c30c3ull;
  x = (x | (x << 2)) & 0x1249249249249249ull;
  return x;
}

__device__ __forceinline__ uint64_t morton(uint32_t x, uint32_t y, uint32_t z) {
  return spread3(x) | (spread3(y) << 1) | (spread3(z) << 2);
}

__global__ void k_morton(int64_t n, const float* __restrict__ x, const float* __restrict__ y,
                         const float* __restrict__ z, Cube c, uint32_t* klo, uint32_t* khi,
                         uint32_t* vals) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const uint64_t key = morton(quant(x[i], c.x0, c.inv_s), quant(y[i], c.y0, c.inv_s),
                              quant(z[i], c.z0, c.inv_s));
  klo[i] = (uint32_t)key;
  khi[i] = (uint32_t)(key >> 32);
  vals[i] = (uint32_t)i;
}

// after the sort by low words (values v1): the high words in that order, identity values
__global__ void k_morton_mid(int64_t n, const uint32_t* __restrict__ khi,
                             const uint32_t* __restrict__ v1, uint32_t* khi1, uint32_t* vals) {
  const int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= n) return;
  khi1[k] = khi[v1[k]];
  vals[k] = (uint32_t)k;
}

// after the stable sort by high words (keys khi_s, values v2 into the first order)
__global__ void k_morton_final(int64_t n, const float* __restrict__ x,
                               const float* __restrict__ y, const float* __restrict__ z,
                               const uint32_t* __restrict__ klo_s, const uint32_t* __restrict__ v1,
                               const uint32_t* __restrict__ khi_s, const uint32_t* __restrict__ v2,
                               uint64_t* keys, uint32_t* ids, float4* pos) {
  const int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= n) return;
  const uint32_t m = v2[k], i = v1[m];
  keys[k] = ((uint64_t)khi_s[k] << 32) | klo_s[m];
  ids[k] = i;
  pos[k] = make_float4(x[i], y[i], z[i], 0.f);
}

// squared distance, rounded the same way wherever it is evaluated (no contraction)
__device__ __forceinline__ float dist2(const float4& o, const float4& p) {
  const float dx = __fsub_rn(o.x, p.x), dy = __fsub_rn(o.y, p.y), dz = __fsub_rn(o.z, p.z);
  return __fadd_rn(__fadd_rn(__fmul_rn(dx, dx), __fmul_rn(dy, dy)), __fmul_rn(dz, dz));
}

// 3-D cubic spline of Eq. SPH_kernel without 8 / (pi h^3), and its derivative, x = r / h
__device__ __forceinline__ void w3(float x, float& w, float& dw) {
  const float t = 1.0f - x;
  const float wi = 1.0f - 6.0f * x * x + 6.0f * x * x * x, dwi = x * (18.0f * x - 12.0f);
  const float wo = 2.0f * t * t * t, dwo = -6.0f * t * t;
  w = x < 0.5f ? wi : (x < 1.0f ? wo : 0.f);
  dw = x < 0.5f ? dwi : (x < 1.0f ? dwo : 0.f);
}

__device__ __forceinline__ float warp_sum_f(float v) {
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

__device__ __forceinline__ uint32_t warp_incl_scan(uint32_t v, int lane) {
  for (int o = 1; o < 32; o <<= 1) {
    const uint32_t u = __shfl_up_sync(0xffffffffu, v, o);
    if (lane >= o) v += u;
  }
  return v;
}

// N_eff(h) and dN_eff/dh over the warp's candidates (distances buf[0..nc))
__device__ __forceinline__ void neff(const float* buf, int nc, float h, int lane, float& f,
                                     float& df) {
  const float ih = 1.0f / h;
  float s = 0.f, ds = 0.f;
  for (int j = lane; j < nc; j += 32) {
    const float x = buf[j] * ih;
    float w, dw;
    w3(x, w, dw);
    s += w;
    ds += dw * x;  // d w(r/h) / dh = -w'(x) x / h
  }
  s = warp_sum_f(s);
  ds = warp_sum_f(ds);
  f = HS_KNORM * s;
  df = -HS_KNORM * ds * ih;
}

// the same sums streamed over the search cube's T particles (cells s_a / s_pref), for the
// rare particle whose candidates overflow the buffer (a dense clump near the kernel edge)
__device__ __forceinline__ void neff_stream(const float4* __restrict__ pos, const uint32_t* s_a,
                                            const uint32_t* s_pref, int ncell, uint32_t T,
                                            const float4& p, float h, int lane, float& f,
                                            float& df) {
  const float ih = 1.0f / h;
  float s = 0.f, ds = 0.f;
  int cur = 0;
  for (uint32_t t = lane; t < T; t += 32) {
    while (cur + 1 < ncell && t >= s_pref[cur + 1]) ++cur;
    const float x = sqrtf(dist2(pos[s_a[cur] + (t - s_pref[cur])], p)) * ih;
    float w, dw;
    w3(x, w, dw);
    s += w;
    ds += dw * x;
  }
  s = warp_sum_f(s);
  ds = warp_sum_f(ds);
  f = HS_KNORM * s;
  df = -HS_KNORM * ds * ih;
}

// first index in [lo, hi) whose key is >= t
__device__ __forceinline__ uint32_t lower_bound(const uint64_t* __restrict__ keys, uint32_t lo,
                                                uint32_t hi, uint64_t t) {
  while (lo < hi) {
    const uint32_t mid = lo + ((hi - lo) >> 1);
    if (keys[mid] < t) lo = mid + 1; else hi = mid;
  }
  return lo;
}

__global__ void __launch_bounds__(32 * HS_WARPS)
    k_hsml(int64_t n, const float4* __restrict__ pos, const uint64_t* __restrict__ keys,
           const uint32_t* __restrict__ ids, Cube cb, float n_ngb, int cap,
           const float* __restrict__ guess, float* h_out, int64_t* nfail) {
  extern __shared__ float s_dyn[];
  const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int64_t k = (int64_t)blockIdx.x * HS_WARPS + w;
  if (k >= n) return;  // whole warps leave together
  float* buf = s_dyn + (size_t)w * cap;
  uint32_t* s_a = reinterpret_cast<uint32_t*>(s_dyn + (size_t)HS_WARPS * cap) +
                  w * (2 * HS_MAXCELLS + 1);  // first particle of every cube cell
  uint32_t* s_pref = s_a + HS_MAXCELLS;         // particles of the cells before (+ total)
  const float4 p = pos[k];
  const uint32_t id = ids[k];
  const uint32_t nn = (uint32_t)n;
  // starting radius: 1.25 x the caller's guess, else the largest distance to the
  // ceil(N_ngb) + 1 particles around it in Morton order (spatial neighbours, mostly)
  float R;
  {
    const float gv = guess ? guess[id] : 0.f;
    if (gv > 0.f && isfinite(gv)) {
      R = 1.25f * gv;
    } else {
      // the median distance to the 64 particles around it in Morton order (spatial
      // neighbours, mostly: a window's far half can straddle a jump of the Z-curve, its
      // near half rarely does), scaled to hold about 0.6 N_ngb particles at that density
      // (too small a start costs one cheap round, too large a cube that grows as R^3)
      const int64_t W = n < 64 ? n : 64;
      int64_t j0 = k - W / 2;
      if (j0 < 0) j0 = 0;
      if (j0 + W > n) j0 = n - W;
      const float d0 = (lane < W) ? dist2(pos[j0 + lane], p) : INFINITY;
      const float d1 = (lane + 32 < W) ? dist2(pos[j0 + lane + 32], p) : INFINITY;
      float m = fmaxf(lane < W ? d0 : 0.f, lane + 32 < W ? d1 : 0.f);
      for (int o = 16; o > 0; o >>= 1) m = fmaxf(m, __shfl_xor_sync(0xffffffffu, m, o));
      float a = 0.f, b = m;  // count(d2 <= b) > W / 2
      for (int it = 0; it < 24; ++it) {
        const float c = 0.5f * (a + b);
        const int cnt = __popc(__ballot_sync(0xffffffffu, d0 <= c)) +
                        __popc(__ballot_sync(0xffffffffu, d1 <= c));
        if (2 * cnt > W) b = c; else a = c;
      }
      R = fmaxf(sqrtf(b) * cbrtf(1.2f * n_ngb / (float)W), cb.s);
    }
  }
  float r_short = 0.f, r_over = INFINITY;  // N_eff too small at r_short; too many at r_over
  float h = __int_as_float(0x7fc00000);
  bool done = false;
  for (int round = 0; round < HS_MAX_ROUNDS && !done; ++round) {
    const float R2 = R * R;
    // octree level: cells of side >= HS_CELL_FRAC R (coarser if the cube would exceed
    // HS_MAXCELLS cells)
    int l = 0;
    while (l < HS_QBITS && cb.s * (float)(1u << l) < HS_CELL_FRAC * R) ++l;
    const uint32_t qx0 = quant(p.x - R, cb.x0, cb.inv_s), qx1 = quant(p.x + R, cb.x0, cb.inv_s);
    const uint32_t qy0 = quant(p.y - R, cb.y0, cb.inv_s), qy1 = quant(p.y + R, cb.y0, cb.inv_s);
    const uint32_t qz0 = quant(p.z - R, cb.z0, cb.inv_s), qz1 = quant(p.z + R, cb.z0, cb.inv_s);
    uint32_t wx, wy, wz;
    for (;;) {
      wx = (qx1 >> l) - (qx0 >> l) + 1;
      wy = (qy1 >> l) - (qy0 >> l) + 1;
      wz = (qz1 >> l) - (qz0 >> l) + 1;
      if (wx * wy * wz <= (uint32_t)HS_MAXCELLS || l == HS_QBITS) break;
      ++l;
    }
    const int ncube = (int)(wx * wy * wz);  // <= HS_MAXCELLS (a single cell at l = 21)
    // the cube's cells whose boxes meet the sphere of radius R (with a margin of a few
    // units in the last place of the coordinates), compacted in cube order into s_a
    const float side = cb.s * (float)(1u << l);
    const float eps = 4e-6f * fmaxf(fmaxf(fmaxf(fabsf(p.x), fabsf(p.y)), fabsf(p.z)),
                                    fmaxf(fmaxf(fabsf(cb.x0), fabsf(cb.y0)), fabsf(cb.z0)));
    const float Rm2 = (R + eps) * (R + eps);
    auto gap = [&](float v, float v0, uint32_t ci) {
      const float lo = v0 + (float)ci * side, hi = v0 + (float)(ci + 1) * side;
      return fmaxf(0.f, fmaxf(lo - v, v - hi));
    };
    int ncell = 0;
    for (int base = 0; base < ncube; base += 32) {
      const int c = base + lane;
      bool hit = false;
      if (c < ncube) {
        const uint32_t cz = (qz0 >> l) + c / (wx * wy), rem = c % (wx * wy);
        const uint32_t cy = (qy0 >> l) + rem / wx, cx = (qx0 >> l) + rem % wx;
        const float gx = gap(p.x, cb.x0, cx), gy = gap(p.y, cb.y0, cy), gz = gap(p.z, cb.z0, cz);
        hit = gx * gx + gy * gy + gz * gz <= Rm2;
      }
      const unsigned m = __ballot_sync(0xffffffffu, hit);
      if (hit) s_a[ncell + __popc(m & ((1u << lane) - 1u))] = (uint32_t)c;
      ncell += __popc(m);
    }
    __syncwarp();
    // their key ranges (entry j is read, then overwritten with the range start, by one lane)
    uint32_t run = 0;
    for (int base = 0; base < ncell; base += 32) {
      const int j = base + lane;
      uint32_t cnt = 0;
      if (j < ncell) {
        const uint32_t c = s_a[j];
        const uint32_t cz = (qz0 >> l) + c / (wx * wy), rem = c % (wx * wy);
        const uint32_t cy = (qy0 >> l) + rem / wx, cx = (qx0 >> l) + rem % wx;
        const uint64_t P = morton(cx, cy, cz);
        const uint32_t a = lower_bound(keys, 0, nn, P << (3 * l));
        const uint32_t b = lower_bound(keys, a, nn, (P + 1) << (3 * l));
        s_a[j] = a;
        cnt = b - a;
      }
      const uint32_t inc = warp_incl_scan(cnt, lane) + run;
      s_pref[j + 1] = inc;
      run = __shfl_sync(0xffffffffu, inc, 31);
    }
    const uint32_t T = run;
    if (lane == 0) s_pref[0] = 0;
    __syncwarp();
    if (T > (uint32_t)(HS_SCAN_CAPS * cap)) {  // a very full cube: try a smaller radius first
      const float Rn = R * cbrtf((float)(HS_SCAN_CAPS * cap) / (2.0f * (float)T));
      if (Rn > r_short) {
        R = Rn;
        __syncwarp();
        continue;
      }
    }
    // the cube's particles in cell order; the ones within R compacted by ballot
    uint32_t off = 0;
    int cur = 0;
    for (uint32_t base = 0; base < T; base += 32) {
      const uint32_t t = base + lane;
      bool in = false;
      float d2 = 0.f;
      if (t < T) {
        while (cur + 1 < ncell && t >= s_pref[cur + 1]) ++cur;  // t < T = s_pref[ncell]
        d2 = dist2(pos[s_a[cur] + (t - s_pref[cur])], p);
        in = d2 < R2;
      }
      const unsigned m = __ballot_sync(0xffffffffu, in);
      const uint32_t at = off + __popc(m & ((1u << lane) - 1u));
      if (in && at < (uint32_t)cap) buf[at] = sqrtf(d2);
      off += __popc(m);
    }
    __syncwarp();
    // too many candidates: shrink towards the last short radius while that bracket is wide,
    // else stream the sums over the cube at this radius
    const bool stream = off > (uint32_t)cap;
    if (stream && !(r_short > 0.f && R <= 1.3f * r_short) && round < HS_MAX_ROUNDS - 8) {
      r_over = R;
      R = fmaxf(r_short, R * cbrtf(0.5f * cap / (float)off));
      if (!(R > r_short)) R = 0.5f * (r_short + r_over);
      continue;
    }
    const int total = (int)off;
    auto eval = [&](float hh, float& f_, float& df_) {
      if (stream) neff_stream(pos, s_a, s_pref, ncell, T, p, hh, lane, f_, df_);
      else neff(buf, total, hh, lane, f_, df_);
    };
    float f, df;
    eval(R, f, df);
    if (f < n_ngb) {  // not enough within R: grow
      r_short = R;
      float grow = 1.1f * cbrtf(n_ngb / fmaxf(f, 1e-3f));
      grow = fminf(fmaxf(grow, 1.15f), 4.0f);
      R = fminf(R * grow, 0.5f * (R + r_over));
      if (!(R > r_short)) R = r_short * 1.15f;
      __syncwarp();
      continue;
    }
    // N_eff(R) >= n_ngb: Newton on ln N_eff(ln h) = ln n_ngb (nearly linear, N_eff ~ h^3)
    // inside a bisection bracket [lo, hi]
    float lo = 0.f, hi = R, x = R;
    if (f - n_ngb < 1e-6f * n_ngb) {
      h = R;
    } else {
      x = fminf(R, fmaxf(0.5f * R, R * cbrtf(n_ngb / f)));
      for (int it = 0; it < 40; ++it) {
        eval(x, f, df);
        const float F = f - n_ngb;
        if (F < 0.f) lo = x; else hi = x;
        if (fabsf(F) <= 1e-6f * n_ngb) break;
        float xn = (df > 0.f) ? x * __expf(__logf(n_ngb / f) * f / (x * df)) : 0.5f * (lo + hi);
        if (!(xn > lo && xn < hi)) xn = 0.5f * (lo + hi);
        if (fabsf(xn - x) <= 1e-6f * x || hi - lo <= 1e-6f * hi) {
          x = xn;
          break;
        }
        x = xn;
      }
      h = x;
    }
    done = true;
    __syncwarp();
  }
  if (lane == 0) {
    h_out[id] = done ? h : __int_as_float(0x7fc00000);
    if (!done) atomicAdd((unsigned long long*)nfail, 1ull);
  }
}

}  // namespace

extern "C" int bp_smoothing_lengths(bp_ctx* ctx, int64_t n, const float* x, const float* y,
                                    const float* z, double n_ngb, const float* h_guess,
                                    float* h_out) {
  if (!ctx) return BP_EINVAL;
  if (n < 0) return bp_fail(ctx, BP_EINVAL, "bp_smoothing_lengths: n < 0");
  if (n == 0) return BP_OK;
  if (!x || !y || !z || !h_out) return bp_fail(ctx, BP_EINVAL, "bp_smoothing_lengths: null pointer");
  if (!(n_ngb > 32.0 / 3.0) || !(n_ngb <= HS_CAP_MAX / 2))
    return bp_fail(ctx, BP_EINVAL, "bp_smoothing_lengths: n_ngb must be in (32/3, %d]",
                   HS_CAP_MAX / 2);
  if (32.0 / 3.0 * (double)n <= n_ngb)
    return bp_fail(ctx, BP_ERANGE, "bp_smoothing_lengths: %lld particles cannot reach n_ngb",
                   (long long)n);
  if (n >= ((int64_t)1 << 32))
    return bp_fail(ctx, BP_ERANGE, "bp_smoothing_lengths: n >= 2^32");
  int r;
  // bounding box
  unsigned* bb;
  if ((r = bp_ws(ctx, WS_MISC2, 64, (void**)&bb))) return r;
  const unsigned init[8] = {0xffffffffu, 0xffffffffu, 0xffffffffu, 0u, 0u, 0u, 0u, 0u};
  BP_CUDA(ctx, cudaMemcpyAsync(bb, init, sizeof(init), cudaMemcpyHostToDevice, ctx->stream));
  k_bbox<<<(unsigned)std::min<int64_t>((n + 255) / 256, 4 * ctx->num_sms), 256, 0, ctx->stream>>>(
      n, x, y, z, bb);
  BP_LAUNCH_CHECK(ctx, "bbox");
  unsigned hb[8];
  BP_CUDA(ctx, cudaMemcpyAsync(hb, bb, sizeof(hb), cudaMemcpyDeviceToHost, ctx->stream));
  BP_CUDA(ctx, cudaStreamSynchronize(ctx->stream));
  auto unord = [](unsigned u) {
    u = (u & 0x80000000u) ? (u & 0x7fffffffu) : ~u;
    float f;
    memcpy(&f, &u, 4);
    return (double)f;
  };
  double lo[3], ext[3];
  for (int a = 0; a < 3; ++a) {
    lo[a] = unord(hb[a]);
    ext[a] = unord(hb[3 + a]) - lo[a];
    if (!std::isfinite(lo[a]) || !std::isfinite(ext[a]))
      return bp_fail(ctx, BP_EINVAL, "bp_smoothing_lengths: non-finite positions");
  }
  // quantisation cube: the bounding box's largest side split into 2^21 level-0 cells
  double D = std::max(ext[0], std::max(ext[1], ext[2]));
  if (!(D > 0.0)) D = 1.0;
  Cube cb;
  cb.x0 = (float)lo[0];
  cb.y0 = (float)lo[1];
  cb.z0 = (float)lo[2];
  cb.inv_s = (float)((double)(1u << HS_QBITS) / (D * (1.0 + 1e-6)));
  cb.s = (float)(1.0 / (double)cb.inv_s);
  // Morton order: sort by the low key words, then stably by the high words
  uint32_t *A, *B, *C, *Dv, *E, *F, *G;
  if ((r = bp_ws(ctx, WS_KEYS0, (size_t)n * 4, (void**)&A))) return r;
  if ((r = bp_ws(ctx, WS_VALS0, (size_t)n * 4, (void**)&B))) return r;
  if ((r = bp_ws(ctx, WS_KEYS1, (size_t)n * 4, (void**)&C))) return r;
  if ((r = bp_ws(ctx, WS_VALS1, (size_t)n * 4, (void**)&Dv))) return r;
  if ((r = bp_ws(ctx, WS_COUNTS, (size_t)n * 4, (void**)&E))) return r;
  if ((r = bp_ws(ctx, WS_UNITS, (size_t)n * 4, (void**)&F))) return r;
  if ((r = bp_ws(ctx, WS_OFFS, (size_t)n * 4, (void**)&G))) return r;
  const unsigned nb = (unsigned)((n + 255) / 256);
  k_morton<<<nb, 256, 0, ctx->stream>>>(n, x, y, z, cb, A, E, B);
  BP_LAUNCH_CHECK(ctx, "morton keys");
  uint32_t *klo_s, *v1;
  if ((r = bp_radix_sort_pairs(ctx, A, B, C, Dv, n, 32, &klo_s, &v1))) return r;
  uint32_t* t0 = (klo_s == A) ? C : A;  // the pair the first sort's result does not occupy
  uint32_t* t1 = (klo_s == A) ? Dv : B;
  k_morton_mid<<<nb, 256, 0, ctx->stream>>>(n, E, v1, F, G);
  BP_LAUNCH_CHECK(ctx, "morton high words");
  uint32_t *khi_s, *v2;
  if ((r = bp_radix_sort_pairs(ctx, F, G, t0, t1, n, 3 * HS_QBITS - 32, &khi_s, &v2))) return r;
  uint64_t* keys;
  float4* pos;
  if ((r = bp_ws(ctx, WS_TILES, (size_t)n * 8, (void**)&keys))) return r;
  if ((r = bp_ws(ctx, WS_HPAR, (size_t)n * sizeof(float4), (void**)&pos))) return r;
  k_morton_final<<<nb, 256, 0, ctx->stream>>>(n, x, y, z, klo_s, v1, khi_s, v2, keys, E, pos);
  BP_LAUNCH_CHECK(ctx, "morton order");
  // candidate buffer per warp: 16 N_ngb distances, between 256 and 2048
  int cap = 256;
  while (cap < HS_CAP_MAX && cap < 16.0 * n_ngb) cap *= 2;
  const size_t smem = (size_t)HS_WARPS * (cap * sizeof(float) + (2 * HS_MAXCELLS + 1) * 4);
  BP_CUDA(ctx, cudaFuncSetAttribute(k_hsml, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                    (int)smem));
  BP_CUDA(ctx, cudaMemsetAsync(ctx->d_counter + 5, 0, sizeof(int64_t), ctx->stream));
  k_hsml<<<(unsigned)((n + HS_WARPS - 1) / HS_WARPS), 32 * HS_WARPS, smem, ctx->stream>>>(
      n, pos, keys, E, cb, (float)n_ngb, cap, h_guess, h_out, ctx->d_counter + 5);
  BP_LAUNCH_CHECK(ctx, "smoothing lengths");
  BP_CUDA(ctx, cudaMemcpyAsync(ctx->h_pinned + 5, ctx->d_counter + 5, sizeof(int64_t),
                               cudaMemcpyDeviceToHost, ctx->stream));
  BP_CUDA(ctx, cudaStreamSynchronize(ctx->stream));
  if (ctx->h_pinned[5] > 0)
    return bp_fail(ctx, BP_ENOCONV, "bp_smoothing_lengths: %lld particles did not converge",
                   (long long)ctx->h_pinned[5]);
  return BP_OK;
}

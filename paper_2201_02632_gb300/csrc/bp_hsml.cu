// bp_hsml.cu -- SPH smoothing lengths (Section 3.4: the cubic kernel Eq. SPH_kernel and the
// effective neighbour number N_ngb).  h_i solves
//   N_eff(h) = (4 pi / 3) h^3 sum_j W(|r_i - r_j|, h) = (32/3) sum_j w(|r_i - r_j| / h) = N_ngb,
// the sum over every particle, i itself included; N_eff grows monotonically with h.
//
//  k_bbox        bounding box of the positions (order-independent min / max)
//  k_cell_keys   uniform-grid cell index of every particle
//  radix sort    (cell, particle) pairs, stable (bp_sort.cu); k_gather_sorted packs the
//                positions in cell order; bp_tile_ranges gives every cell's range
//  k_hsml        one warp per particle: scan the cells of the cube of half-width R around
//                it, compact the squared distances below R^2 into shared memory (count,
//                warp scan, write: a fixed order), grow R until N_eff(R) >= N_ngb, then
//                solve N_eff(h) = N_ngb in (0, R] by Newton inside a bisection bracket.
//                Every sum is lane-strided plus a fixed shuffle tree: deterministic.
#include <algorithm>
#include <cmath>
#include <cstring>

#include "bp_internal.cuh"

namespace {

constexpr int HS_WARPS = 4;        // warps per block
constexpr int HS_CAP = 2048;       // candidate distances per warp (shared memory)
constexpr int HS_MAX_ROUNDS = 48;  // radius updates per particle
constexpr float HS_KNORM = 32.0f / 3.0f;

struct Grid {
  float x0, y0, z0, inv_d, d;
  int nx, ny, nz;
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

__device__ __forceinline__ int cell_coord(float v, float v0, float inv_d, int nc) {
  int c = (int)floorf((v - v0) * inv_d);
  return c < 0 ? 0 : (c >= nc ? nc - 1 : c);
}

__global__ void k_cell_keys(int64_t n, const float* __restrict__ x, const float* __restrict__ y,
                            const float* __restrict__ z, Grid g, uint32_t* keys,
                            uint32_t* vals) {
  int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const int cx = cell_coord(x[i], g.x0, g.inv_d, g.nx);
  const int cy = cell_coord(y[i], g.y0, g.inv_d, g.ny);
  const int cz = cell_coord(z[i], g.z0, g.inv_d, g.nz);
  keys[i] = (uint32_t)(((int64_t)cz * g.ny + cy) * g.nx + cx);
  vals[i] = (uint32_t)i;
}

__global__ void k_gather_sorted(int64_t n, const float* __restrict__ x,
                                const float* __restrict__ y, const float* __restrict__ z,
                                const uint32_t* __restrict__ vals, float4* pos) {
  int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= n) return;
  const uint32_t i = vals[k];
  pos[k] = make_float4(x[i], y[i], z[i], 0.f);
}

// squared distance, rounded the same way wherever it is evaluated (no contraction): the
// counting and the writing pass must classify every particle alike
__device__ __forceinline__ float dist2(const float4& o, const float4& p) {
  const float dx = __fsub_rn(o.x, p.x), dy = __fsub_rn(o.y, p.y), dz = __fsub_rn(o.z, p.z);
  return __fadd_rn(__fadd_rn(__fmul_rn(dx, dx), __fmul_rn(dy, dy)), __fmul_rn(dz, dz));
}

// 3-D cubic spline of Eq. SPH_kernel without 8 / (pi h^3), and its derivative, x = r / h
__device__ __forceinline__ void w3(float x, float& w, float& dw) {
  if (x < 0.5f) {
    w = 1.0f - 6.0f * x * x + 6.0f * x * x * x;
    dw = x * (18.0f * x - 12.0f);
  } else if (x < 1.0f) {
    const float t = 1.0f - x;
    w = 2.0f * t * t * t;
    dw = -6.0f * t * t;
  } else {
    w = 0.f;
    dw = 0.f;
  }
}

__device__ __forceinline__ float warp_sum_f(float v) {
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// N_eff(h) and dN_eff/dh over the warp's candidates (squared distances buf[0..nc))
__device__ __forceinline__ void neff(const float* buf, int nc, float h, int lane, float& f,
                                     float& df) {
  const float ih = 1.0f / h;
  float s = 0.f, ds = 0.f;
  for (int j = lane; j < nc; j += 32) {
    const float x = sqrtf(buf[j]) * ih;
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

__global__ void __launch_bounds__(32 * HS_WARPS)
    k_hsml(int64_t n, const float4* __restrict__ pos, const uint32_t* __restrict__ vals,
           const int64_t* __restrict__ cstart, Grid g, float n_ngb,
           const float* __restrict__ guess, float* h_out, int64_t* nfail) {
  __shared__ float s_buf[HS_WARPS][HS_CAP];
  const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int64_t k = (int64_t)blockIdx.x * HS_WARPS + w;
  if (k >= n) return;
  float* buf = s_buf[w];
  const float4 p = pos[k];
  const uint32_t id = vals[k];
  // starting radius: the caller's guess, else the density of the particle's own cell
  float R;
  {
    const int cx = cell_coord(p.x, g.x0, g.inv_d, g.nx);
    const int cy = cell_coord(p.y, g.y0, g.inv_d, g.ny);
    const int cz = cell_coord(p.z, g.z0, g.inv_d, g.nz);
    const int64_t c = ((int64_t)cz * g.ny + cy) * g.nx + cx;
    const float occ = (float)(cstart[c + 1] - cstart[c]);
    R = 1.3f * g.d * cbrtf(n_ngb * (3.0f / (4.0f * 3.14159265f)) / fmaxf(occ, 1.0f));
    if (guess) {
      const float gv = guess[id];
      if (gv > 0.f && isfinite(gv)) R = 1.25f * gv;
    }
  }
  float r_short = 0.f, r_over = INFINITY;  // N_eff too small at r_short; too many at r_over
  float h = __int_as_float(0x7fc00000);
  bool done = false;
  for (int round = 0; round < HS_MAX_ROUNDS && !done; ++round) {
    const float R2 = R * R;
    const int ix0 = cell_coord(p.x - R, g.x0, g.inv_d, g.nx);
    const int ix1 = cell_coord(p.x + R, g.x0, g.inv_d, g.nx);
    const int iy0 = cell_coord(p.y - R, g.y0, g.inv_d, g.ny);
    const int iy1 = cell_coord(p.y + R, g.y0, g.inv_d, g.ny);
    const int iz0 = cell_coord(p.z - R, g.z0, g.inv_d, g.nz);
    const int iz1 = cell_coord(p.z + R, g.z0, g.inv_d, g.nz);
    const int wx = ix1 - ix0 + 1, wy = iy1 - iy0 + 1, wxy = wx * wy;
    const int ncube = wxy * (iz1 - iz0 + 1);  // <= the grid's cells <= 2^30
    // pass 1: candidates of this lane's cells
    int cnt = 0;
    for (int q = lane; q < ncube; q += 32) {
      const int cz = iz0 + q / wxy, rem = q - (cz - iz0) * wxy;
      const int cy = iy0 + rem / wx, cx = ix0 + rem - (cy - iy0) * wx;
      const int64_t c = ((int64_t)cz * g.ny + cy) * g.nx + cx;
      for (int64_t j = cstart[c]; j < cstart[c + 1]; ++j) cnt += dist2(pos[j], p) < R2 ? 1 : 0;
    }
    int incl = cnt;
    for (int o = 1; o < 32; o <<= 1) {
      const int u = __shfl_up_sync(0xffffffffu, incl, o);
      if (lane >= o) incl += u;
    }
    const int total = __shfl_sync(0xffffffffu, incl, 31);
    if (total > HS_CAP) {  // too many candidates: shrink towards the last short radius
      r_over = R;
      R = fmaxf(r_short, R * cbrtf(0.5f * HS_CAP / (float)total));
      if (!(R > r_short)) R = 0.5f * (r_short + r_over);
      continue;
    }
    // pass 2: the same cells in the same order; squared distances at the lane's offset
    int off = incl - cnt;
    for (int q = lane; q < ncube; q += 32) {
      const int cz = iz0 + q / wxy, rem = q - (cz - iz0) * wxy;
      const int cy = iy0 + rem / wx, cx = ix0 + rem - (cy - iy0) * wx;
      const int64_t c = ((int64_t)cz * g.ny + cy) * g.nx + cx;
      for (int64_t j = cstart[c]; j < cstart[c + 1]; ++j) {
        const float d2 = dist2(pos[j], p);
        if (d2 < R2 && off < HS_CAP) buf[off++] = d2;  // off < total <= HS_CAP
      }
    }
    __syncwarp();
    float f, df;
    neff(buf, total, R, lane, f, df);
    if (f < n_ngb) {  // not enough within R: grow (the cube then covers the new radius)
      r_short = R;
      float grow = 1.1f * cbrtf(n_ngb / fmaxf(f, 1e-3f));
      grow = fminf(fmaxf(grow, 1.15f), 4.0f);
      R = fminf(R * grow, 0.5f * (R + r_over));
      if (!(R > r_short)) R = r_short * 1.15f;
      __syncwarp();
      continue;
    }
    // N_eff(R) >= n_ngb: Newton in a bisection bracket [lo, hi] on the candidates
    float lo = 0.f, hi = R, x = R;
    if (f - n_ngb < 1e-6f * n_ngb) {
      h = R;
    } else {
      x = fminf(R, fmaxf(0.5f * R, R * cbrtf(n_ngb / f)));
      for (int it = 0; it < 60; ++it) {
        neff(buf, total, x, lane, f, df);
        const float F = f - n_ngb;
        if (F < 0.f) lo = x; else hi = x;
        float xn = (df > 0.f) ? x - F / df : 0.5f * (lo + hi);
        if (!(xn > lo && xn < hi)) xn = 0.5f * (lo + hi);
        if (fabsf(xn - x) <= 2e-7f * x || hi - lo <= 2e-7f * hi) {
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
  if (!(n_ngb > 32.0 / 3.0) || !(n_ngb <= HS_CAP / 2))
    return bp_fail(ctx, BP_EINVAL, "bp_smoothing_lengths: n_ngb must be in (32/3, %d]",
                   HS_CAP / 2);
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
  // uniform grid: about 4 particles per cell over the box (flat boxes are given a
  // thickness of 1e-3 of their largest side), at most 2^30 cells
  const double emax = std::max(ext[0], std::max(ext[1], ext[2]));
  double vol = 1.0;
  for (int a = 0; a < 3; ++a) vol *= std::max(ext[a], emax > 0 ? 1e-3 * emax : 1.0);
  double d = std::cbrt(vol / std::max(1.0, (double)n / 4.0));
  Grid g;
  for (;;) {
    g.nx = (int)std::min(1e9, std::floor(ext[0] / d) + 1);
    g.ny = (int)std::min(1e9, std::floor(ext[1] / d) + 1);
    g.nz = (int)std::min(1e9, std::floor(ext[2] / d) + 1);
    if ((double)g.nx * g.ny * g.nz <= (double)(1 << 30)) break;
    d *= 1.25;
  }
  g.x0 = (float)lo[0];
  g.y0 = (float)lo[1];
  g.z0 = (float)lo[2];
  g.d = (float)d;
  g.inv_d = (float)(1.0 / d);
  const int64_t ncells = (int64_t)g.nx * g.ny * g.nz;
  // (cell, particle) pairs sorted by cell; positions in that order; cell ranges
  uint32_t *k0, *v0, *k1, *v1;
  if ((r = bp_ws(ctx, WS_KEYS0, (size_t)n * 4, (void**)&k0))) return r;
  if ((r = bp_ws(ctx, WS_VALS0, (size_t)n * 4, (void**)&v0))) return r;
  if ((r = bp_ws(ctx, WS_KEYS1, (size_t)n * 4, (void**)&k1))) return r;
  if ((r = bp_ws(ctx, WS_VALS1, (size_t)n * 4, (void**)&v1))) return r;
  const unsigned nb = (unsigned)((n + 255) / 256);
  k_cell_keys<<<nb, 256, 0, ctx->stream>>>(n, x, y, z, g, k0, v0);
  BP_LAUNCH_CHECK(ctx, "cell keys");
  int key_bits = 0;
  while (((int64_t)1 << key_bits) < ncells) ++key_bits;
  uint32_t *ks, *vs;
  if ((r = bp_radix_sort_pairs(ctx, k0, v0, k1, v1, n, key_bits, &ks, &vs))) return r;
  int64_t* cstart;
  if ((r = bp_ws(ctx, WS_TILES, (size_t)(ncells + 1) * 8, (void**)&cstart))) return r;
  if ((r = bp_tile_ranges(ctx, ks, n, ncells, cstart))) return r;
  float4* pos;
  if ((r = bp_ws(ctx, WS_HPAR, (size_t)n * sizeof(float4), (void**)&pos))) return r;
  k_gather_sorted<<<nb, 256, 0, ctx->stream>>>(n, x, y, z, vs, pos);
  BP_LAUNCH_CHECK(ctx, "gather sorted");
  BP_CUDA(ctx, cudaMemsetAsync(ctx->d_counter + 5, 0, sizeof(int64_t), ctx->stream));
  k_hsml<<<(unsigned)((n + HS_WARPS - 1) / HS_WARPS), 32 * HS_WARPS, 0, ctx->stream>>>(
      n, pos, vs, cstart, g, (float)n_ngb, h_guess, h_out, ctx->d_counter + 5);
  BP_LAUNCH_CHECK(ctx, "smoothing lengths");
  BP_CUDA(ctx, cudaMemcpyAsync(ctx->h_pinned + 5, ctx->d_counter + 5, sizeof(int64_t),
                               cudaMemcpyDeviceToHost, ctx->stream));
  BP_CUDA(ctx, cudaStreamSynchronize(ctx->stream));
  if (ctx->h_pinned[5] > 0)
    return bp_fail(ctx, BP_ENOCONV, "bp_smoothing_lengths: %lld particles did not converge",
                   (long long)ctx->h_pinned[5]);
  return BP_OK;
}

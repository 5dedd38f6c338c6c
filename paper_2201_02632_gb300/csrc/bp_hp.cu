// bp_hp.cu -- halo-based pasting (Section 3.3) and map finalisation (Section 3.2).
//
//  k_hp_prep    per halo: FP64 centre in pixel units, aperture, FP32 profile constants;
//               halos whose aperture covers fewer than HP_DIRECT_PIX pixels get no table
//  k_hp_table   per tabled halo and table node u = r_perp / r_f = s^2 (nodes uniform in s,
//               which smooths the central cusp): the line-of-sight integrals of the
//               dimensionless pressure and density profiles, divided by the chord
//               sqrt(1 - u^2) so that the tabulated function is smooth at the edge
//               (Eqs. y^HP, b^HP); 12-point Gauss-Legendre per segment after
//               t = u sinh(s), split where the 3-D radius crosses r_vir and the zero
//               of the thermal fraction
//  k_hp_count / (map, tile, halo) pairs from the FP64 pixel-centre bounding box of the
//  k_hp_emit    aperture disc; the count also sizes the values of the untabled halos and
//               flags the halos that need a table (k_hp_tab_emit lists them, in order)
//  k_hp_direct  the line-of-sight integrals of the untabled halos at each of their pixels
//  k_hp_paste   persistent over work units; each pixel centre inside the aperture adds
//               the interpolated projected profile (or the stored value of an untabled
//               halo) with Kahan compensation
//  k_hp_reduce  partial tiles of multi-unit tiles, in unit order
//  k_finalize   hi + lo folding and the conversion to Delta T / T_CMB
#include <algorithm>
#include <vector>

#include "bp_internal.cuh"

#define HP_NT 256          // table intervals on s = sqrt(u) in [0, 1]
#define HP_ROW (HP_NT + 3) // with one ghost node at each end
#define HP_NGL 12          // Gauss-Legendre points per segment (16 gave the same map errors)
// Halos whose aperture covers fewer pixels than this get their LOS integrals evaluated at each
// covered pixel instead of a 257-node table (a table would cost more than the pixels it
// serves; most halos of the batched and all-sky catalogues cover a few dozen pixels).  Both
// pastes ran fastest between 128 and 1024 pixels.
#define HP_DIRECT_PIX 256.0

__constant__ float c_hgx[HP_NGL];
__constant__ float c_hgw[HP_NGL];

namespace {

bool g_hp_const = false;

int hp_constants(bp_ctx* ctx) {
  if (g_hp_const) return BP_OK;
  float x[HP_NGL], w[HP_NGL];
  for (int i = 0; i < HP_NGL; ++i) {
    double z = cos(bpc::PI * (i + 0.75) / (HP_NGL + 0.5));
    double dp = 0, p1 = 0;
    for (int it = 0; it < 100; ++it) {
      double p0 = 1.0;
      p1 = z;
      for (int k = 2; k <= HP_NGL; ++k) {
        double p2 = ((2 * k - 1) * z * p1 - (k - 1) * p0) / k;
        p0 = p1;
        p1 = p2;
      }
      dp = HP_NGL * (z * p1 - p0) / (z * z - 1.0);
      double dz = p1 / dp;
      z -= dz;
      if (fabs(dz) < 1e-16) break;
    }
    x[i] = (float)(-z);
    w[i] = (float)(2.0 / ((1.0 - z * z) * dp * dp));
  }
  BP_CUDA(ctx, cudaMemcpyToSymbol(c_hgx, x, sizeof(x)));
  BP_CUDA(ctx, cudaMemcpyToSymbol(c_hgw, w, sizeof(w)));
  g_hp_const = true;
  return BP_OK;
}

// Per-halo HP record.
struct HpHalo {
  double cx, cy;     // centre in pixel units from the lower-left edge
  double rad_px;     // aperture radius [px]
  float inv_rf_px;   // 1 / r_f [px]
  float Ay, Ab;      // amplitude of y and b per unit chord (u = 0 edge chord 1)
  int map, ok;
  int nt;            // table intervals of this halo (64, 128 or 256, by its size in pixels)
  // profile constants for the tables (same meaning as the PP halo block)
  float xf, c, q500, psi, A0, A1, ant, xnt;  // xnt: r_nt1 / r_s (R_nt = 1) or huge
};

// Profile constants and amplitudes of halo k (shared by the flat-sky and the all-sky
// preparations); false when the halo has no valid model.
__device__ __forceinline__ bool hp_fill_profile(const BpParams& P, int64_t nh, int64_t k,
                                                const float* __restrict__ vlos,
                                                const double* __restrict__ model,
                                                const int32_t* __restrict__ status, HpHalo& H) {
  auto F = [&](int f) { return model[(int64_t)f * nh + k]; };
  double rs = F(BP_M_RS), rf = F(BP_M_RF), T = F(BP_M_T), DA = F(BP_M_DA);
  bool ok = status[k] == BP_HALO_OK && rs > 0 && rf > 0 && T > 0 && DA > 0;
  // Table intervals per halo.  Coarser tables (64 or 128 intervals, 1.6e-5 and 1.4e-6
  // interpolation error) broke the per-pixel kSZ tolerance where halos of opposite
  // velocities cancel, so every halo uses the full resolution.
  H.nt = HP_NT;
  double n1T = (P.n_poly + 1.0) * T, GM = bpc::G * F(BP_M_MVIR);
  H.Ay = (float)(P.CP * P.pe_frac * F(BP_M_P0) * 2.0 * rf);
  double vk = vlos ? (double)vlos[k] : 0.0;
  H.Ab = (float)(P.CN * F(BP_M_RHO0) * 2.0 * rf * (vk / bpc::C_KMS) * exp(-F(BP_M_TAU)));
  H.xf = (float)(rf / rs);
  H.c = (float)F(BP_M_C);
  H.q500 = (float)(rs / F(BP_M_R500));
  H.psi = (float)(GM / (F(BP_M_MC) * rs * n1T));
  H.A0 = (float)(-F(BP_M_PHI0) / n1T);
  H.A1 = (float)(GM / (rs * n1T));
  H.ant = (float)F(BP_M_ANT);
  double xnt = (F(BP_M_ANT) > 0) ? F(BP_M_R500) * pow(1.0 / F(BP_M_ANT), 1.0 / P.n_nt) / rs : 1e30;
  H.xnt = (float)fmin(xnt, 1e30);
  return ok;
}

__global__ void k_hp_prep(BpParams P, int64_t nh, const double* __restrict__ thx,
                          const double* __restrict__ thy, const float* __restrict__ vlos,
                          const int32_t* __restrict__ map_id, const double* __restrict__ model,
                          const int32_t* __restrict__ status, bp_map_geom g, double ap_r500,
                          HpHalo* out) {
  int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= nh) return;
  auto F = [&](int f) { return model[(int64_t)f * nh + k]; };
  HpHalo H;
  int mp = map_id ? map_id[k] : 0;
  bool ok = hp_fill_profile(P, nh, k, vlos, model, status, H) && mp >= 0 && mp < g.n_maps;
  double rf = F(BP_M_RF), DA = F(BP_M_DA);
  double rap = rf;
  if (ap_r500 > 0) rap = fmin(rap, ap_r500 * F(BP_M_R500));
  double px = DA * g.dtheta;  // Mpc per pixel at the halo
  H.cx = (thx[k] - g.theta0_x) / g.dtheta;
  H.cy = (thy[k] - g.theta0_y) / g.dtheta;
  H.rad_px = rap / DA / g.dtheta;
  H.inv_rf_px = (float)(px / rf);
  H.map = mp;
  H.ok = ok ? 1 : 0;
  if (bpc::PI * H.rad_px * H.rad_px < HP_DIRECT_PIX) H.nt = 0;  // evaluated at its pixels
  out[k] = H;
}

__device__ __forceinline__ float g_in(float x) {
  if (x < 2e-2f) return x * (0.5f - x * (1.0f / 3.0f - x * (0.25f - x * 0.2f)));
  return 1.0f - log1pf(x) / x;
}

// dimensionless pressure (thermal part) and density at x = r / r_s
__device__ __forceinline__ void profile_pn(const HpHalo& H, float x, float n_poly, int n_int,
                                           float n_nt, float& p, float& d) {
  if (x >= H.xf) {
    p = d = 0.f;
    return;
  }
  float th = (x <= H.c) ? 1.0f - H.psi * g_in(x) : 1.0f - H.A0 + H.A1 / x;
  th = fmaxf(th, 0.f);
  float tn;
  if (n_int > 0) {
    float r = 1.f, b = th;
    int e = n_int;
    while (e) {
      if (e & 1) r *= b;
      b *= b;
      e >>= 1;
    }
    tn = r;
  } else {
    tn = powf(th, n_poly);
  }
  // (x q500)^n_nt through log2 / exp2: about 2e-7 relative, without powf's special cases
  float Rnt = H.ant * exp2f(n_nt * log2f(x * H.q500));
  d = tn;
  p = tn * th * fmaxf(0.f, 1.0f - Rnt);
}

// The line-of-sight integrals of the dimensionless pressure and density at projected radius
// u = r_perp / r_f in [0, 1), in units of r_f, NOT divided by the chord (Eqs. y^HP, b^HP):
// 12-point Gauss-Legendre per segment, split where the 3-D radius crosses r_vir and the zero
// of the thermal fraction; u = 0 in t directly, u > 0 after t = u sinh(s).
__device__ __forceinline__ void hp_los(const HpHalo& H, float u, float n_poly, int n_int,
                                       float n_nt, float& Sy, float& Sb) {
  const float kinks[2] = {H.c / H.xf, H.xnt / H.xf};
  float segs[4];
  int ns = 0;
  float sy = 0.f, sb = 0.f;
  if (u == 0.f) {
    segs[ns++] = 0.f;
    for (int q = 0; q < 2; ++q)
      if (kinks[q] > 0.f && kinks[q] < 1.0f) segs[ns++] = kinks[q];
    segs[ns++] = 1.0f;
    if (ns == 4 && segs[1] > segs[2]) { float t = segs[1]; segs[1] = segs[2]; segs[2] = t; }
    for (int s = 0; s + 1 < ns; ++s) {
      float a = segs[s], b = segs[s + 1], mid = 0.5f * (a + b), hw = 0.5f * (b - a);
      for (int j = 0; j < HP_NGL; ++j) {
        float t = mid + hw * c_hgx[j];
        float p, d;
        profile_pn(H, t * H.xf, n_poly, n_int, n_nt, p, d);
        sy += hw * c_hgw[j] * p;
        sb += hw * c_hgw[j] * d;
      }
    }
  } else {
    // t = u sinh(s): r/r_f = u cosh(s); s in [0, asinh(L/u)]
    const float L = sqrtf(fmaxf(0.f, 1.0f - u * u));
    float smax = asinhf(L / u);
    segs[ns++] = 0.f;
    for (int q = 0; q < 2; ++q)
      if (kinks[q] > u && kinks[q] < 1.0f) {
        float sk = acoshf(kinks[q] / u);
        if (sk > 0.f && sk < smax) segs[ns++] = sk;
      }
    segs[ns++] = smax;
    if (ns == 4 && segs[1] > segs[2]) { float t = segs[1]; segs[1] = segs[2]; segs[2] = t; }
    for (int s = 0; s + 1 < ns; ++s) {
      float a = segs[s], b = segs[s + 1], mid = 0.5f * (a + b), hw = 0.5f * (b - a);
      for (int j = 0; j < HP_NGL; ++j) {
        float sv = mid + hw * c_hgx[j];
        float ch = coshf(sv);
        float p, d;
        profile_pn(H, u * ch * H.xf, n_poly, n_int, n_nt, p, d);
        float wj = hw * c_hgw[j] * u * ch;
        sy += wj * p;
        sb += wj * d;
      }
    }
  }
  Sy = sy;
  Sb = sb;
}

// Table slot j of nh: halo tlist[j] (a list of the halos that need a table), or halo j
// when tlist is null.
__global__ void __launch_bounds__(256) k_hp_table(const HpHalo* __restrict__ halos,
                                                  const uint32_t* __restrict__ tlist, int64_t nh,
                                                  float n_poly, int n_int, float n_nt,
                                                  float* tab) {
  int64_t gid = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  int64_t j = gid / (HP_NT + 1);
  int node = (int)(gid % (HP_NT + 1));
  if (j >= nh) return;
  const HpHalo H = halos[tlist ? (int64_t)tlist[j] : j];
  if (node > H.nt || H.nt == 0) return;  // nt = 0: evaluated at its pixels, no table
  const int NTh = H.nt;
  float* ty = tab + j * 2 * HP_ROW;
  float* tb = ty + HP_ROW;
  if (!H.ok) {
    ty[node + 1] = tb[node + 1] = 0.f;
    return;
  }
  float sn = (float)node / NTh;
  float u = sn * sn;
  float Gy = 0.f, Gb = 0.f;
  if (node == NTh) {  // limit u -> 1: the profile at r_f
    float p, d;
    profile_pn(H, H.xf * 0.99999994f, n_poly, n_int, n_nt, p, d);
    Gy = p;
    Gb = d;
  } else {
    float sy, sb;
    hp_los(H, u, n_poly, n_int, n_nt, sy, sb);
    // divided by the chord sqrt(1 - u^2) (1 at u = 0): smooth up to the edge
    const float L = node == 0 ? 1.0f : sqrtf(fmaxf(0.f, 1.0f - u * u));
    Gy = sy / L;
    Gb = sb / L;
  }
  ty[node + 1] = Gy;
  tb[node + 1] = Gb;
}

// ghost nodes: G(s = -h) = G(h) (even in s), G(1+h) = 2 G(1) - G(1-h)
__global__ void k_hp_ghosts(const HpHalo* __restrict__ halos, const uint32_t* __restrict__ tlist,
                            int64_t nh, float* tab) {
  int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (j >= nh) return;
  const int nt = halos[tlist ? (int64_t)tlist[j] : j].nt;
  if (nt == 0) return;
  for (int q = 0; q < 2; ++q) {
    float* t = tab + j * 2 * HP_ROW + q * HP_ROW;
    t[0] = t[2];
    t[nt + 2] = 2.f * t[nt + 1] - t[nt];
  }
}

__device__ __forceinline__ bool hp_box(const HpHalo& H, const bp_map_geom& g, int& i0, int& i1,
                                       int& j0, int& j1) {
  if (!H.ok) return false;
  double rad = H.rad_px;
  double cx = H.cx - 0.5, cy = H.cy - 0.5;  // pixel-centre index units
  double fa = floor(cx - rad), fb = floor(cx + rad);
  double ga = floor(cy - rad), gb = floor(cy + rad);
  if (fb < 0 || fa > g.nx - 1 || gb < 0 || ga > g.ny - 1) return false;
  i0 = fa < 0 ? 0 : (int)fa;
  i1 = fb > g.nx - 1 ? g.nx - 1 : (int)fb;
  j0 = ga < 0 ? 0 : (int)ga;
  j1 = gb > g.ny - 1 ? g.ny - 1 : (int)gb;
  return true;
}

// The pixel box of a halo evaluated at its pixels, with its centre relative to the centre of
// the box's first pixel (one FP64 subtraction per halo, then FP32 per pixel as in the paste).
struct HpDBox {
  int i0, j0, bw;
  float cxr, cyr, rad2;
};

// Per halo: the tiles its pixel box touches, the values it needs if it is evaluated at its
// pixels (its whole box, row-major) with that box, and whether it needs a table (a halo on
// some map that is not evaluated at its pixels).
__global__ void k_hp_count(const HpHalo* __restrict__ halos, int64_t nh, bp_map_geom g, int ts,
                           uint32_t* counts, uint32_t* dlen, HpDBox* dbox, uint32_t* tflag) {
  int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= nh) return;
  int i0, i1, j0, j1;
  uint32_t c = 0, d = 0, tf = 0;
  const HpHalo H = halos[k];
  if (hp_box(H, g, i0, i1, j0, j1)) {
    c = (uint32_t)((i1 / ts - i0 / ts + 1) * (j1 / ts - j0 / ts + 1));
    if (H.nt == 0) {
      d = (uint32_t)((i1 - i0 + 1) * (j1 - j0 + 1));
      HpDBox D;
      D.i0 = i0;
      D.j0 = j0;
      D.bw = i1 - i0 + 1;
      D.cxr = (float)(H.cx - 0.5 - (double)i0);
      D.cyr = (float)(H.cy - 0.5 - (double)j0);
      D.rad2 = (float)(H.rad_px * H.rad_px);
      dbox[k] = D;
    } else {
      tf = 1;
    }
  }
  counts[k] = c;
  dlen[k] = d;
  tflag[k] = tf;
}

// The halos that need a table, in index order: slot toff[k] of the compact table store.
__global__ void k_hp_tab_emit(const uint32_t* __restrict__ tflag, const int64_t* __restrict__ toff,
                              int64_t nh, uint32_t* tlist) {
  int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (k < nh && tflag[k]) tlist[toff[k]] = (uint32_t)k;
}

__global__ void k_hp_emit(const HpHalo* __restrict__ halos, int64_t nh, bp_map_geom g, int ts,
                          const int64_t* __restrict__ offs, uint32_t* keys, uint32_t* vals) {
  int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= nh) return;
  int i0, i1, j0, j1;
  const HpHalo H = halos[k];
  if (!hp_box(H, g, i0, i1, j0, j1)) return;
  int ntx = (g.nx + ts - 1) / ts, nty = (g.ny + ts - 1) / ts;
  int64_t o = offs[k];
  for (int ty = j0 / ts; ty <= j1 / ts; ++ty)
    for (int tx = i0 / ts; tx <= i1 / ts; ++tx) {
      keys[o] = (uint32_t)(((int64_t)H.map * nty + ty) * ntx + tx);
      vals[o] = (uint32_t)k;
      ++o;
    }
}

struct HpUnit {
  int64_t tile;
  int64_t begin, end;
  int64_t slot;
};

// units per tile and partial-tile slots (only for tiles split into several units)
__global__ void k_hp_ucount(const int64_t* __restrict__ tstart, int64_t n_tiles, int unit,
                            uint32_t* uc, uint32_t* sc) {
  int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= n_tiles) return;
  uint32_t nu = (uint32_t)((tstart[t + 1] - tstart[t] + unit - 1) / unit);
  uc[t] = nu;
  sc[t] = nu > 1 ? nu : 0u;
}
__global__ void k_hp_uemit(const int64_t* __restrict__ tstart, int64_t n_tiles, int unit,
                           const int64_t* __restrict__ uoff, const int64_t* __restrict__ soff,
                           HpUnit* units) {
  int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= n_tiles) return;
  int64_t b = tstart[t], e = tstart[t + 1], nu = (e - b + unit - 1) / unit, u0 = uoff[t];
  for (int64_t q = 0; q < nu; ++q) {
    HpUnit U;
    U.tile = t;
    U.slot = nu > 1 ? soff[t] + q : -1;
    U.begin = b + q * unit;
    U.end = min(e, b + (q + 1) * unit);
    units[u0 + q] = U;
  }
}

constexpr int HP_THREADS = 256;
constexpr int HCH = 32;

__device__ __forceinline__ float catmull(const float* __restrict__ t, float ss, int nt) {
  // t: table row with ghosts; node k (s = k / nt) at t[k + 1]; ss in [0, 1)
  float x = ss * nt;
  int i = (int)x;
  if (i > nt - 1) i = nt - 1;
  float f = x - (float)i;
  float p0 = __ldg(t + i), p1 = __ldg(t + i + 1), p2 = __ldg(t + i + 2), p3 = __ldg(t + i + 3);
  float f2 = f * f, f3 = f2 * f;
  return 0.5f * (2.f * p1 + (-p0 + p2) * f + (2.f * p0 - 5.f * p1 + 4.f * p2 - p3) * f2 +
                 (-p0 + 3.f * p1 - 3.f * p2 + p3) * f3);
}

__device__ __forceinline__ void kahan_add(float& s, float& c, float v) {
  float y = __fsub_rn(v, c);
  float t = __fadd_rn(s, y);
  c = __fsub_rn(__fsub_rn(t, s), y);
  s = t;
}

template <int TS>
__global__ void __launch_bounds__(HP_THREADS)
    k_hp_paste(const HpHalo* __restrict__ halos, const float* __restrict__ tab,
               const uint32_t* __restrict__ hvals, const HpUnit* __restrict__ units,
               const int64_t* __restrict__ n_units_ptr, int64_t* counter, bp_map_geom g,
               const int64_t* __restrict__ hvoff, const float2* __restrict__ dvals,
               const int64_t* __restrict__ toff, float* ymap,
               float* bmap, float* ylo, float* blo, float* partials) {
  constexpr int PR = TS / 16;
  __shared__ float s_cx[HCH], s_cy[HCH], s_rap2[HCH], s_irf[HCH], s_ay[HCH], s_ab[HCH];
  __shared__ int4 s_box[HCH];
  __shared__ const float* s_tab[HCH];
  __shared__ int s_nt[HCH];
  __shared__ int64_t s_dv[HCH];  // nt = 0: index of the value of tile pixel (0, 0) ...
  __shared__ int s_bw[HCH];      // ... and of the halo's box row length
  __shared__ int64_t s_unit;
  const int tid = threadIdx.x, lane = tid & 31, w = tid >> 5;
  const int lr = lane >> 3, lc = lane & 7;
  const int wr0 = (w >> 1) * 4 * PR, wc0 = (w & 1) * 8 * PR;
  const int r0 = wr0 + lr * PR, c0 = wc0 + lc * PR;
  const int ntx = (g.nx + TS - 1) / TS, nty = (g.ny + TS - 1) / TS;
  const int64_t n_units = *n_units_ptr;
  for (;;) {
    if (tid == 0) s_unit = atomicAdd((unsigned long long*)counter, 1ull);
    __syncthreads();
    const int64_t u = s_unit;
    if (u >= n_units) break;
    const HpUnit U = units[u];
    const int mp = (int)(U.tile / ((int64_t)ntx * nty));
    const int rem = (int)(U.tile % ((int64_t)ntx * nty));
    const int x0 = (rem % ntx) * TS, y0 = (rem / ntx) * TS;
    float hy[PR][PR], cy_[PR][PR], hb[PR][PR], cb_[PR][PR];
#pragma unroll
    for (int r = 0; r < PR; ++r)
#pragma unroll
      for (int c = 0; c < PR; ++c) hy[r][c] = cy_[r][c] = hb[r][c] = cb_[r][c] = 0.f;
    for (int64_t cb = U.begin; cb < U.end; cb += HCH) {
      const int nch = (int)min((int64_t)HCH, U.end - cb);
      __syncthreads();
      if (tid < nch) {
        uint32_t hk = hvals[cb + tid];
        const HpHalo H = halos[hk];
        // centre relative to the tile origin, exact enough in FP32 after the FP64 shift
        s_cx[tid] = (float)(H.cx - x0);
        s_cy[tid] = (float)(H.cy - y0);
        s_rap2[tid] = (float)(H.rad_px * H.rad_px);
        s_irf[tid] = H.inv_rf_px;
        s_ay[tid] = H.Ay;
        s_ab[tid] = H.Ab;
        s_tab[tid] = H.nt > 0 ? tab + toff[hk] * 2 * HP_ROW : tab;  // its table slot
        s_nt[tid] = H.nt;
        int i0, i1, j0, j1;
        int4 bx = make_int4(1, 0, 1, 0);  // empty
        int64_t dv = 0;
        int bw = 0;
        if (hp_box(H, g, i0, i1, j0, j1)) {
          const int4 t = make_int4(max(i0 - x0, 0), min(i1 - x0, TS - 1), max(j0 - y0, 0),
                                   min(j1 - y0, TS - 1));
          const bool any = t.y >= t.x && t.w >= t.z;
          if (any) bx = t;
          bw = i1 - i0 + 1;
          // the halo's values are row-major over its box (i0..i1, j0..j1)
          if (H.nt == 0) {
            dv = hvoff[hk] + (int64_t)(y0 - j0) * bw + (x0 - i0);
            if (any) {  // its rows in this tile into L2 before the warps read them
              const int64_t ea = hvoff[hk] + (int64_t)(y0 + t.z - j0) * bw;
              const int64_t eb = hvoff[hk] + (int64_t)(y0 + t.w - j0) * bw + bw - 1;
              const uintptr_t pa = (uintptr_t)(dvals + ea) & ~(uintptr_t)127;
              for (uintptr_t a = pa; a <= (uintptr_t)(dvals + eb); a += 128)
                asm volatile("prefetch.global.L2 [%0];" ::"l"(a));
            }
          }
        }
        s_box[tid] = bx;
        s_dv[tid] = dv;
        s_bw[tid] = bw;
      }
      __syncthreads();
      for (int k = 0; k < nch; ++k) {
        int4 bx = s_box[k];
        if (bx.y < wc0 || bx.x > wc0 + 8 * PR - 1 || bx.w < wr0 || bx.z > wr0 + 4 * PR - 1)
          continue;
        const int ntk = s_nt[k];
        if (ntk == 0) {  // values stored by k_hp_direct
          const int bw = s_bw[k];
          const int64_t dv0 = s_dv[k];
#pragma unroll
          for (int r = 0; r < PR; ++r) {
            const int rr = r0 + r;
#pragma unroll
            for (int c = 0; c < PR; ++c) {
              const int cc = c0 + c;
              if (cc < bx.x || cc > bx.y || rr < bx.z || rr > bx.w) continue;
              const float2 v = dvals[dv0 + (int64_t)rr * bw + cc];
              kahan_add(hy[r][c], cy_[r][c], v.x);
              kahan_add(hb[r][c], cb_[r][c], v.y);
            }
          }
          continue;
        }
        const float hcx = s_cx[k], hcy = s_cy[k], rap2 = s_rap2[k], irf = s_irf[k];
        const float* ty = s_tab[k];
#pragma unroll
        for (int r = 0; r < PR; ++r) {
          float dy = (float)(r0 + r) + 0.5f - hcy;
#pragma unroll
          for (int c = 0; c < PR; ++c) {
            float dx = (float)(c0 + c) + 0.5f - hcx;
            float d2 = dx * dx + dy * dy;
            if (d2 < rap2) {
              float uu = sqrtf(d2) * irf;
              if (uu < 1.0f) {
                float chord = sqrtf(fmaxf(0.f, 1.0f - uu * uu));
                float ss = sqrtf(uu);
                float gy = catmull(ty, ss, ntk), gb = catmull(ty + HP_ROW, ss, ntk);
                kahan_add(hy[r][c], cy_[r][c], s_ay[k] * chord * gy);
                kahan_add(hb[r][c], cb_[r][c], s_ab[k] * chord * gb);
              }
            }
          }
        }
      }
    }
    const int64_t mbase = (int64_t)mp * g.nx * g.ny;
    if (U.slot < 0) {
#pragma unroll
      for (int r = 0; r < PR; ++r)
#pragma unroll
        for (int c = 0; c < PR; ++c) {
          int gx = x0 + c0 + c, gy = y0 + r0 + r;
          if (gx >= g.nx || gy >= g.ny) continue;
          int64_t p = mbase + (int64_t)gy * g.nx + gx;
          float s, e;
          bp_two_sum(ymap[p], hy[r][c], s, e);
          ymap[p] = s;
          ylo[p] = ylo[p] + (e - cy_[r][c]);
          bp_two_sum(bmap[p], hb[r][c], s, e);
          bmap[p] = s;
          blo[p] = blo[p] + (e - cb_[r][c]);
        }
    } else {
      float* P = partials + U.slot * 4 * TS * TS;
#pragma unroll
      for (int r = 0; r < PR; ++r)
#pragma unroll
        for (int c = 0; c < PR; ++c) {
          int q = (r0 + r) * TS + c0 + c;
          P[q] = hy[r][c];
          P[TS * TS + q] = -cy_[r][c];
          P[2 * TS * TS + q] = hb[r][c];
          P[3 * TS * TS + q] = -cb_[r][c];
        }
    }
    __syncthreads();
  }
}

template <int TS>
__global__ void __launch_bounds__(256) k_hp_reduce(const int64_t* __restrict__ tstart,
                                                   const int64_t* __restrict__ soff,
                                                   int64_t n_tiles, int unit, bp_map_geom g,
                                                   const float* __restrict__ partials,
                                                   float* ymap, float* bmap, float* ylo,
                                                   float* blo) {
  int64_t t = blockIdx.x;
  if (t >= n_tiles) return;
  int64_t nu = (tstart[t + 1] - tstart[t] + unit - 1) / unit;
  if (nu <= 1) return;
  int ntx = (g.nx + TS - 1) / TS, nty = (g.ny + TS - 1) / TS;
  int mp = (int)(t / ((int64_t)ntx * nty)), rem = (int)(t % ((int64_t)ntx * nty));
  int x0 = (rem % ntx) * TS, y0 = (rem / ntx) * TS;
  int64_t u0 = soff[t];
  for (int q = threadIdx.x; q < TS * TS; q += blockDim.x) {
    int gx = x0 + q % TS, gy = y0 + q / TS;
    if (gx >= g.nx || gy >= g.ny) continue;
    float hy = 0.f, ly = 0.f, hb = 0.f, lb = 0.f;
    for (int64_t k = 0; k < nu; ++k) {
      const float* P = partials + (u0 + k) * 4 * TS * TS;
      float s, e;
      bp_two_sum(hy, P[q], s, e);
      hy = s;
      ly += P[TS * TS + q] + e;
      bp_two_sum(hb, P[2 * TS * TS + q], s, e);
      hb = s;
      lb += P[3 * TS * TS + q] + e;
    }
    int64_t p = (int64_t)mp * g.nx * g.ny + (int64_t)gy * g.nx + gx;
    float s, e;
    bp_two_sum(ymap[p], hy, s, e);
    ymap[p] = s;
    ylo[p] = ylo[p] + (ly + e);
    bp_two_sum(bmap[p], hb, s, e);
    bmap[p] = s;
    blo[p] = blo[p] + (lb + e);
  }
}

__global__ void k_finalize(int64_t npix, float* map, float* lo, float scale) {
  int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= npix) return;
  float v = map[i];
  if (lo) {
    v = v + lo[i];
    lo[i] = 0.f;
  }
  map[i] = v * scale;
}

// y and b planes with their lo planes, four pixels per thread (16-byte accesses; every plane
// 16-byte aligned), the same arithmetic as k_finalize; pixels [0, 4 n4).
__global__ void k_finalize4(int64_t n4, float4* y, float4* ylo, float sy, float4* b,
                            float4* blo, float sb) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n4) return;
  const float4 z = make_float4(0.f, 0.f, 0.f, 0.f);
  float4 v = y[i], l = ylo[i];
  y[i] = make_float4((v.x + l.x) * sy, (v.y + l.y) * sy, (v.z + l.z) * sy, (v.w + l.w) * sy);
  ylo[i] = z;
  v = b[i];
  l = blo[i];
  b[i] = make_float4((v.x + l.x) * sb, (v.y + l.y) * sb, (v.z + l.z) * sb, (v.w + l.w) * sb);
  blo[i] = z;
}

// The (map, tile, halo) work list of a catalogue, in the context's scratch.
struct HpList {
  int64_t np = 0, n_tiles = 0, n_units = 0, n_slots = 0;
  int64_t nh = 0, nval = 0;        // halos; values of the halos evaluated at their pixels
  const uint32_t* keys = nullptr;  // (map, tile) keys, sorted
  const uint32_t* vals = nullptr;  // halo indices sorted by (map, tile), then index
  int64_t* hvoff = nullptr;        // [nh + 1]: first value of each halo (nt = 0 halos)
  HpDBox* dbox = nullptr;          // [nh]: the box of each of those halos
  int64_t n_table = 0;             // halos with a table
  int64_t* toff = nullptr;         // [nh + 1]: table slot of each halo (exclusive scan)
  uint32_t* tlist = nullptr;       // [n_table]: the halo of each table slot
  int64_t* tstart = nullptr;       // [n_tiles + 1]
  int64_t* uoff = nullptr;         // [n_tiles + 1], uoff[n_tiles] = n_units
  int64_t* soff = nullptr;         // [n_tiles + 1]
  HpUnit* units = nullptr;
  int unit = 0, ts = 0;
};

// The last index in [lo, hi] whose first value is <= e: the halo holding value e.
__device__ __forceinline__ int64_t hp_owner(const int64_t* __restrict__ voff, int64_t lo,
                                            int64_t hi, int64_t e) {
  while (lo < hi) {
    const int64_t mid = (lo + hi + 1) >> 1;
    if (voff[mid] <= e) lo = mid; else hi = mid - 1;
  }
  return lo;
}

// The values (chord-weighted LOS integrals times the amplitudes) of the halos evaluated at
// their pixels, row-major over each halo's pixel box: one warp per vpw consecutive values (the
// same work for every warp however the values are spread over the halos), lanes taking them
// in turn, each finding its halo by binary search inside the warp's range of halos; pixels
// outside the aperture get zeros.
__global__ void __launch_bounds__(256)
    k_hp_direct(const HpHalo* __restrict__ halos, const int64_t* __restrict__ hvoff,
                const HpDBox* __restrict__ dbox, int64_t nh, int64_t nval, int vpw,
                float n_poly, int n_int, float n_nt, float2* dv) {
  const int64_t e0 = (((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5) * vpw;
  const int lane = threadIdx.x & 31;
  if (e0 >= nval) return;
  const int64_t e1 = min(nval, e0 + vpw);
  const int64_t ka = hp_owner(hvoff, 0, nh - 1, e0);
  const int64_t kb = hp_owner(hvoff, ka, nh - 1, e1 - 1);
  for (int64_t e = e0 + lane; e < e1; e += 32) {
    const int64_t k = hp_owner(hvoff, ka, kb, e);
    const HpDBox D = dbox[k];
    const int local = (int)(e - hvoff[k]);
    const float dx = (float)(local % D.bw) - D.cxr, dy = (float)(local / D.bw) - D.cyr;
    const float d2 = dx * dx + dy * dy;
    float sy = 0.f, sb = 0.f;
    if (d2 < D.rad2) {
      const HpHalo H = halos[k];
      const float uu = sqrtf(d2) * H.inv_rf_px;
      if (uu < 1.0f) {
        hp_los(H, uu, n_poly, n_int, n_nt, sy, sb);  // chord times the table value
        sy *= H.Ay;
        sb *= H.Ab;
      }
    }
    dv[e] = make_float2(sy, sb);
  }
}

int hp_build_list(bp_ctx* ctx, int64_t n, const HpHalo* halos, const bp_map_geom* g, int TS,
                  int unit, HpList* L) {
  int r;
  const int ntx = (g->nx + TS - 1) / TS, nty = (g->ny + TS - 1) / TS;
  const int64_t n_tiles = (int64_t)ntx * nty * g->n_maps;
  if (n_tiles > (int64_t)UINT32_MAX) return bp_fail(ctx, BP_ERANGE, "paste_halos: too many tiles");
  uint32_t* counts;
  int64_t *offs, *hvoff;
  if ((r = bp_ws(ctx, WS_COUNTS, (size_t)(n + 1) * 12, (void**)&counts))) return r;
  if ((r = bp_ws(ctx, WS_OFFS, (size_t)(n + 1) * 12, (void**)&offs))) return r;
  if ((r = bp_ws(ctx, WS_HALO, (size_t)(n + 1) * 16, (void**)&hvoff))) return r;
  HpDBox* dbox;
  if ((r = bp_ws(ctx, WS_MISC2, (size_t)n * sizeof(HpDBox), (void**)&dbox))) return r;
  uint32_t* dlen = counts + (n + 1);
  uint32_t* tflag = dlen + (n + 1);
  int64_t* toff = hvoff + (n + 1);
  uint32_t* tlist = reinterpret_cast<uint32_t*>(offs + (n + 1));
  unsigned nb = (unsigned)((n + 255) / 256);
  k_hp_count<<<nb, 256, 0, ctx->stream>>>(halos, n, *g, TS, counts, dlen, dbox, tflag);
  BP_LAUNCH_CHECK(ctx, "hp count");
  if ((r = bp_scan_u32_to_i64(ctx, counts, offs, n))) return r;
  if ((r = bp_scan_u32_to_i64(ctx, dlen, hvoff, n))) return r;
  if ((r = bp_scan_u32_to_i64(ctx, tflag, toff, n))) return r;
  BP_CUDA(ctx, cudaMemcpyAsync(ctx->h_pinned, offs + n, 8, cudaMemcpyDeviceToHost, ctx->stream));
  BP_CUDA(ctx, cudaMemcpyAsync(ctx->h_pinned + 1, hvoff + n, 8, cudaMemcpyDeviceToHost,
                               ctx->stream));
  BP_CUDA(ctx, cudaMemcpyAsync(ctx->h_pinned + 2, toff + n, 8, cudaMemcpyDeviceToHost,
                               ctx->stream));
  k_hp_tab_emit<<<nb, 256, 0, ctx->stream>>>(tflag, toff, n, tlist);
  BP_LAUNCH_CHECK(ctx, "hp table list");
  BP_CUDA(ctx, cudaStreamSynchronize(ctx->stream));
  const int64_t np = ctx->h_pinned[0];
  L->np = np;
  L->nh = n;
  L->nval = ctx->h_pinned[1];
  L->n_table = ctx->h_pinned[2];
  L->hvoff = hvoff;
  L->dbox = dbox;
  L->toff = toff;
  L->tlist = tlist;
  L->n_tiles = n_tiles;
  L->ts = TS;
  if (np == 0) return BP_OK;
  if (np > (int64_t)UINT32_MAX) return bp_fail(ctx, BP_ERANGE, "paste_halos: too many pairs");
  if (unit <= 0) {  // automatic: about 16 units per resident CTA, at least 256 halos
    int64_t u = np / ((int64_t)ctx->num_sms * 4 * 16);
    unit = (int)std::min<int64_t>(std::max<int64_t>(u, 256), 1 << 30);
  }
  L->unit = unit;
  uint32_t *k0, *v0, *k1, *v1, *ks, *vs;
  if ((r = bp_ws(ctx, WS_KEYS0, (size_t)np * 4, (void**)&k0))) return r;
  if ((r = bp_ws(ctx, WS_VALS0, (size_t)np * 4, (void**)&v0))) return r;
  if ((r = bp_ws(ctx, WS_KEYS1, (size_t)np * 4, (void**)&k1))) return r;
  if ((r = bp_ws(ctx, WS_VALS1, (size_t)np * 4, (void**)&v1))) return r;
  k_hp_emit<<<nb, 256, 0, ctx->stream>>>(halos, n, *g, TS, offs, k0, v0);
  BP_LAUNCH_CHECK(ctx, "hp emit");
  int key_bits = 0;
  while (((int64_t)1 << key_bits) < n_tiles) ++key_bits;
  if ((r = bp_radix_sort_pairs(ctx, k0, v0, k1, v1, np, key_bits, &ks, &vs))) return r;
  L->keys = ks;
  L->vals = vs;
  int64_t* tstart;
  if ((r = bp_ws(ctx, WS_TILES, (size_t)(n_tiles + 1) * 32 + 64, (void**)&tstart))) return r;
  L->tstart = tstart;
  L->uoff = tstart + (n_tiles + 1);
  L->soff = L->uoff + (n_tiles + 1);
  uint32_t* uc = (uint32_t*)(L->soff + (n_tiles + 1));
  uint32_t* sc = uc + (n_tiles + 1);
  if ((r = bp_tile_ranges(ctx, ks, np, n_tiles, tstart))) return r;
  unsigned tb = (unsigned)((n_tiles + 255) / 256);
  k_hp_ucount<<<tb, 256, 0, ctx->stream>>>(tstart, n_tiles, unit, uc, sc);
  BP_LAUNCH_CHECK(ctx, "hp unit count");
  if ((r = bp_scan_u32_to_i64(ctx, uc, L->uoff, n_tiles))) return r;
  if ((r = bp_scan_u32_to_i64(ctx, sc, L->soff, n_tiles))) return r;
  BP_CUDA(ctx, cudaMemcpyAsync(ctx->h_pinned, L->uoff + n_tiles, 8, cudaMemcpyDeviceToHost,
                               ctx->stream));
  BP_CUDA(ctx, cudaMemcpyAsync(ctx->h_pinned + 1, L->soff + n_tiles, 8, cudaMemcpyDeviceToHost,
                               ctx->stream));
  BP_CUDA(ctx, cudaStreamSynchronize(ctx->stream));
  L->n_units = ctx->h_pinned[0];
  L->n_slots = ctx->h_pinned[1];
  if ((r = bp_ws(ctx, WS_UNITS, (size_t)(L->n_units + 1) * sizeof(HpUnit), (void**)&L->units)))
    return r;
  k_hp_uemit<<<tb, 256, 0, ctx->stream>>>(tstart, n_tiles, unit, L->uoff, L->soff, L->units);
  BP_LAUNCH_CHECK(ctx, "hp units");
  return BP_OK;
}

// Halo records: profile constants, amplitudes, apertures in pixels.
int hp_prep(bp_ctx* ctx, int64_t n, const double* th_x, const double* th_y, const float* v_los,
            const int32_t* map_id, const double* model, const int32_t* status,
            const bp_map_geom* g, double ap_r500, HpHalo* halos) {
  const int pb = bp_item_block(ctx, n, 256);
  k_hp_prep<<<(unsigned)((n + pb - 1) / pb), pb, 0, ctx->stream>>>(
      ctx->p, n, th_x, th_y, v_los, map_id, model, status, *g, ap_r500, halos);
  BP_LAUNCH_CHECK(ctx, "hp prep");
  return BP_OK;
}

// Tables (line-of-sight integrals and ghost nodes) of the n_table halos of tlist, slot j for
// halo tlist[j].
int hp_tables(bp_ctx* ctx, const HpHalo* halos, const uint32_t* tlist, int64_t n_table,
              float* tab) {
  if (n_table <= 0) return BP_OK;
  const BpParams& P = ctx->p;
  double rn = rint(P.n_poly);
  int n_int = (fabs(P.n_poly - rn) < 1e-12 && rn >= 1 && rn <= 16) ? (int)rn : -1;
  int64_t nt = n_table * (HP_NT + 1);
  k_hp_table<<<(unsigned)((nt + 255) / 256), 256, 0, ctx->stream>>>(
      halos, tlist, n_table, (float)P.n_poly, n_int, (float)P.n_nt, tab);
  BP_LAUNCH_CHECK(ctx, "hp table");
  k_hp_ghosts<<<(unsigned)((n_table + 255) / 256), 256, 0, ctx->stream>>>(halos, tlist, n_table,
                                                                         tab);
  BP_LAUNCH_CHECK(ctx, "hp ghosts");
  return BP_OK;
}

template <int TS>
int hp_grid(bp_ctx* ctx, int ctas_per_sm, int64_t n_units) {
  int per_sm = 0;
  cudaError_t e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_hp_paste<TS>,
                                                                HP_THREADS, 0);
  if (e != cudaSuccess) return -1;
  if (ctas_per_sm > 0 && ctas_per_sm < per_sm) per_sm = ctas_per_sm;
  if (per_sm < 1) per_sm = 1;
  int64_t grid = (int64_t)ctx->num_sms * per_sm;
  if (grid > n_units) grid = n_units;
  return (int)(grid > 0 ? grid : 1);
}

// The paste of a built list: persistent kernel over the work units, then the
// fixed-order reduction of split tiles.  No host synchronisation, no allocation.
template <int TS>
int hp_launch(bp_ctx* ctx, const HpHalo* halos, const float* tab, const HpList& L, int grid,
              float* partials, int64_t* counter, const bp_map_geom* g, float2* dvals,
              float* ymap, float* bmap, float* ylo, float* blo) {
  if (L.nval > 0) {  // the values of the halos evaluated at their pixels
    const BpParams& P = ctx->p;
    const double rn = rint(P.n_poly);
    const int n_int = (fabs(P.n_poly - rn) < 1e-12 && rn >= 1 && rn <= 16) ? (int)rn : -1;
    // values per warp: a multiple of 32, up to 256, small enough for 32 warps per SM
    const int64_t full = (int64_t)ctx->num_sms * 32;
    const int vpw = (int)std::min<int64_t>(256, ((L.nval + full - 1) / full + 31) / 32 * 32);
    const int64_t warps = (L.nval + vpw - 1) / vpw;
    k_hp_direct<<<(unsigned)((warps * 32 + 255) / 256), 256, 0, ctx->stream>>>(
        halos, L.hvoff, L.dbox, L.nh, L.nval, vpw, (float)P.n_poly, n_int, (float)P.n_nt,
        dvals);
    BP_LAUNCH_CHECK(ctx, "hp direct values");
  }
  BP_CUDA(ctx, cudaMemsetAsync(counter, 0, 8, ctx->stream));
  k_hp_paste<TS><<<(unsigned)grid, HP_THREADS, 0, ctx->stream>>>(
      halos, tab, L.vals, L.units, L.uoff + L.n_tiles, counter, *g, L.hvoff, dvals, L.toff, ymap,
      bmap, ylo, blo, partials);
  BP_LAUNCH_CHECK(ctx, "hp paste");
  if (L.n_slots > 0) {
    k_hp_reduce<TS><<<(unsigned)L.n_tiles, 256, 0, ctx->stream>>>(
        L.tstart, L.soff, L.n_tiles, L.unit, *g, partials, ymap, bmap, ylo, blo);
    BP_LAUNCH_CHECK(ctx, "hp reduce");
  }
  return BP_OK;
}

int check_hp_args(bp_ctx* ctx, int64_t n, const double* th_x, const double* th_y,
                  const double* model, const int32_t* status, const bp_map_geom* geom,
                  double ap_r500, const char* who) {
  if (!geom || geom->nx <= 0 || geom->ny <= 0 || geom->n_maps <= 0 || !(geom->dtheta > 0))
    return bp_fail(ctx, BP_EINVAL, "%s: bad geometry", who);
  if (n < 0) return bp_fail(ctx, BP_EINVAL, "%s: n < 0", who);
  if (n > (int64_t)UINT32_MAX) return bp_fail(ctx, BP_ERANGE, "%s: n >= 2^32", who);
  if (n > 0 && (!th_x || !th_y || !model || !status))
    return bp_fail(ctx, BP_EINVAL, "%s: null pointer", who);
  if (ap_r500 < 0) return bp_fail(ctx, BP_EINVAL, "%s: ap_r500 < 0", who);
  return BP_OK;
}

// ---------------------------------------------------------------- all-sky HP on HEALPix
// All-sky maps (Section 5.2) with the HP of Section 3.3 on the HEALPix sphere (Gorski et
// al. 2005), RING ordering: 12 nside^2 equal-area pixels on 4 nside - 1 rings of constant
// colatitude.  A ring is cut into segments of HS_SEG consecutive pixels; (segment, halo)
// pairs come from each halo's aperture cap ring by ring, are sorted by segment, and one CTA
// per segment owns its pixels: it adds its halos in sorted order (fixed-order sums, no
// atomics).  The pixel-halo angle uses the half-angle (haversine) form with the colatitude
// difference taken in FP64 and the longitude offset in double-float pixel units, so that it
// keeps FP32 relative accuracy down to sub-pixel separations at nside 8192.
constexpr int HS_SEG = 256;  // pixels per segment = threads per paste CTA
constexpr int HS_CH = 256;   // pairs staged in shared memory at a time

struct HsRing {
  double theta;      // colatitude of the ring's centres
  int64_t first;     // RING index of its first pixel
  float sin_t;       // sin(theta)
  float phase;       // longitude of the first centre in units of dphi (0 or 1/2)
  float dphi;        // 2 pi / cnt (for offsets of a few pixels only)
  int32_t cnt;       // pixels on the ring
  uint32_t seg0;     // id of its first segment
  int32_t pad;
};

// Per-halo all-sky record: HpHalo with cx = colatitude, cy = longitude in [0, 2 pi),
// rad_px = aperture angle [rad], inv_rf_px = D_A / r_f [1/rad].
// Halos h0 .. h0 + m - 1 of a catalogue of n (the model is field-major over all n); out[k]
// describes halo h0 + k.
__global__ void k_hs_prep(BpParams P, int64_t n, int64_t h0, int64_t m,
                          const double* __restrict__ theta, const double* __restrict__ phi,
                          const float* __restrict__ vlos, const double* __restrict__ model,
                          const int32_t* __restrict__ status, double ap_r500, int nside,
                          HpHalo* out) {
  const int64_t kl = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (kl >= m) return;
  const int64_t k = h0 + kl;
  auto F = [&](int f) { return model[(int64_t)f * n + k]; };
  HpHalo H;
  const double th = theta[k], ph = phi[k];
  bool ok = hp_fill_profile(P, n, k, vlos, model, status, H) && th >= 0.0 && th <= bpc::PI &&
            isfinite(ph);
  double rf = F(BP_M_RF), DA = F(BP_M_DA);
  double rap = rf;
  if (ap_r500 > 0) rap = fmin(rap, ap_r500 * F(BP_M_R500));
  double pm = ok ? fmod(ph, 2.0 * bpc::PI) : 0.0;
  if (pm < 0.0) pm += 2.0 * bpc::PI;
  H.cx = ok ? th : 0.0;
  H.cy = pm;
  H.rad_px = ok ? fmin(rap / DA, bpc::PI) : 0.0;
  H.inv_rf_px = (float)(DA / rf);
  H.map = 0;
  H.ok = ok ? 1 : 0;
  // aperture area in pixels: pi alpha^2 / (4 pi / (12 nside^2))
  const double npx = 3.0 * H.rad_px * H.rad_px * (double)nside * (double)nside;
  if (npx < HP_DIRECT_PIX) H.nt = 0;
  out[kl] = H;
}

// first ring (0-based) whose colatitude is >= t
__device__ __forceinline__ int hs_ring_at(const HsRing* __restrict__ R, int nr, double t) {
  int lo = 0, hi = nr;
  while (lo < hi) {
    int mid = (lo + hi) >> 1;
    if (R[mid].theta < t) lo = mid + 1; else hi = mid;
  }
  return lo;
}

// Pixels of ring G that the aperture of H may touch: [j0, j1] (centre indices, possibly
// outside [0, cnt) and then wrapping; one pixel of margin each side), or the whole ring.
// Returns false when the ring misses the cap.  The exact test is the paste's.
__device__ __forceinline__ bool hs_ring_span(const HpHalo& H, const HsRing& G, bool& full,
                                             int& j0, int& j1) {
  const float dth = (float)(G.theta - H.cx);
  const float alpha = (float)H.rad_px;
  const float sa = sinf(0.5f * alpha), sd = sinf(0.5f * dth);
  const float den = sinf((float)H.cx) * G.sin_t;
  full = false;
  if (!(den > 1e-30f)) {  // halo on a pole: the ring is entirely in or out
    if (fabsf(dth) >= alpha) return false;
    full = true;
    return true;
  }
  const float q = (sa * sa - sd * sd) / den;  // sin^2(half longitude width)
  if (q <= 0.f) return false;
  if (q >= 1.f) {
    full = true;
    return true;
  }
  const float w = 2.0f * asinf(sqrtf(q)) / G.dphi + 1.0f;
  const float e = (float)(H.cy * (double)G.cnt * (0.5 / bpc::PI)) - G.phase;
  j0 = (int)floorf(e - w);
  j1 = (int)ceilf(e + w);
  if (j1 - j0 + 1 >= G.cnt) full = true;
  return true;
}

// Segments of a ring span, in ascending order: calls f(segment id)
template <typename Fn>
__device__ __forceinline__ void hs_span_segments(const HsRing& G, bool full, int j0, int j1,
                                                 Fn f) {
  const int last = (G.cnt - 1) / HS_SEG;
  if (!full) {
    const int a = ((j0 % G.cnt) + G.cnt) % G.cnt, b = a + (j1 - j0);
    if (b < G.cnt) {
      for (int c = a / HS_SEG; c <= b / HS_SEG; ++c) f(G.seg0 + c);
      return;
    }
    const int cb = (b - G.cnt) / HS_SEG, ca = a / HS_SEG;  // [0, cb] and [ca, last]
    if (cb < ca) {
      for (int c = 0; c <= cb; ++c) f(G.seg0 + c);
      for (int c = ca; c <= last; ++c) f(G.seg0 + c);
      return;
    }
  }
  for (int c = 0; c <= last; ++c) f(G.seg0 + c);
}

__device__ __forceinline__ void hs_ring_range(const HpHalo& H, const HsRing* R, int nr, int& r0,
                                              int& r1) {
  r0 = hs_ring_at(R, nr, H.cx - H.rad_px);
  r1 = hs_ring_at(R, nr, H.cx + H.rad_px) - 1;  // last ring with theta < cx + rad (+ margin)
  if (r0 > 0) --r0;
  if (r1 < nr - 1) ++r1;
}

// Per halo: its (segment, halo) pairs, and whether it needs a table (a halo with pairs
// that is not evaluated at its pixels).
__global__ void k_hs_count(const HpHalo* __restrict__ halos, int64_t nh,
                           const HsRing* __restrict__ R, int nr, uint32_t* counts,
                           uint32_t* tflag) {
  int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= nh) return;
  const HpHalo H = halos[k];
  uint32_t c = 0;
  if (H.ok) {
    int r0, r1;
    hs_ring_range(H, R, nr, r0, r1);
    for (int r = r0; r <= r1; ++r) {
      const HsRing G = R[r];
      bool full;
      int j0 = 0, j1 = 0;
      if (hs_ring_span(H, G, full, j0, j1)) hs_span_segments(G, full, j0, j1, [&](uint32_t) { ++c; });
    }
  }
  counts[k] = c;
  tflag[k] = (c > 0 && H.nt > 0) ? 1u : 0u;
}

// The geometry of one (segment, halo) pair: the halo's colatitude offset and longitude in
// pixel units from the segment's first centre, and the segment's pixels to test.
struct HsPair {
  float dth2, sp, rh, rl, sa2;
  int2 rg;  // pixels rg.x .. rg.y of the segment (empty when rg.x > rg.y)
};
__device__ __forceinline__ HsPair hs_pair(const HpHalo& H, const HsRing& G, int c0, int npx) {
  HsPair q;
  const float dth = (float)(G.theta - H.cx);
  const float sd = sinf(0.5f * dth);
  q.dth2 = sd * sd;
  q.sp = sinf((float)H.cx) * G.sin_t;
  // the halo's longitude in pixel units from the segment's first centre (FP64 from the exact
  // pixel count: an FP32 spacing would misplace centres far along the ring by up to 2e-7 rad),
  // the representative nearest the segment's middle, as a double-float
  double rel = H.cy * (double)G.cnt * (0.5 / bpc::PI) - (double)G.phase - (double)c0;
  rel -= (double)G.cnt * rint((rel - 0.5 * HS_SEG) / (double)G.cnt);
  q.rh = (float)rel;
  q.rl = (float)(rel - (double)q.rh);
  const float sa = sinf(0.5f * (float)H.rad_px);
  q.sa2 = sa * sa;
  // all of the segment's pixels when the span can wrap into it from both sides, else the
  // span around the representative
  bool full;
  int j0 = 0, j1 = 0;
  q.rg = make_int2(0, npx - 1);
  if (!hs_ring_span(H, G, full, j0, j1)) {
    q.rg = make_int2(1, 0);
  } else if (!full && G.cnt > HS_SEG && (j1 - j0) + HS_SEG < G.cnt) {
    const float w = 0.5f * (float)(j1 - j0);
    q.rg.x = max(0, (int)floorf(q.rh - w) - 1);
    q.rg.y = min(npx - 1, (int)ceilf(q.rh + w) + 1);
  }
  return q;
}
// u = r_perp / r_f of pixel t of the segment, or false outside the aperture
__device__ __forceinline__ bool hs_pixel_u(const HsPair& q, const HsRing& G, float irf, int t,
                                           float& uu) {
  float dp = ((float)t - q.rh) - q.rl;  // longitude offset [pixels]
  dp -= (float)G.cnt * rintf(dp / (float)G.cnt);
  const float sp = sinf(0.5f * dp * G.dphi);
  const float hav = q.dth2 + q.sp * sp * sp;  // sin^2(psi / 2)
  if (!(hav < q.sa2)) return false;
  uu = 2.0f * asinf(sqrtf(hav)) * irf;
  return uu < 1.0f;
}
__device__ __forceinline__ int hs_ring_of_segment(const HsRing* __restrict__ R, int nr,
                                                  uint32_t sg) {
  int lo = 0, hi = nr - 1;  // the last ring whose first segment is <= sg
  while (lo < hi) {
    int mid = (lo + hi + 1) >> 1;
    if (R[mid].seg0 <= sg) lo = mid; else hi = mid - 1;
  }
  return lo;
}

// Pairs in emission order o: key = segment, value = o; per pair its halo and, for a halo
// evaluated at its pixels (nt = 0), the segment's pixel range and the number of values.
__global__ void k_hs_emit(const HpHalo* __restrict__ halos, int64_t nh,
                          const HsRing* __restrict__ R, int nr,
                          const int64_t* __restrict__ offs, uint32_t* keys, uint32_t* vals,
                          uint32_t* p_halo, int2* p_rg, uint32_t* p_len) {
  int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= nh) return;
  const HpHalo H = halos[k];
  if (!H.ok) return;
  int64_t o = offs[k];
  const int64_t end = offs[k + 1];
  int r0, r1;
  hs_ring_range(H, R, nr, r0, r1);
  for (int r = r0; r <= r1; ++r) {
    const HsRing G = R[r];
    bool full;
    int j0 = 0, j1 = 0;
    if (hs_ring_span(H, G, full, j0, j1))
      hs_span_segments(G, full, j0, j1, [&](uint32_t sg) {
        if (o < end) {  // the count pass gave exactly this many
          keys[o] = sg;
          vals[o] = (uint32_t)o;
          p_halo[o] = (uint32_t)k;
          uint32_t len = 0;
          if (H.nt == 0) {
            const int c0 = (int)(sg - G.seg0) * HS_SEG;
            const HsPair q = hs_pair(H, G, c0, min(HS_SEG, G.cnt - c0));
            p_rg[o] = q.rg;
            len = q.rg.y >= q.rg.x ? (uint32_t)(q.rg.y - q.rg.x + 1) : 0u;
          }
          p_len[o] = len;
          ++o;
        }
      });
  }
}

// The values of the halos evaluated at their pixels, before the pairs are sorted: one warp
// per HS_DIRECT_HPW consecutive halos, lanes over the (pair, pixel) values of all their pairs
// (emission order; pairs of halos with tables hold none), each value finding its pair by
// binary search and its halo through the pair.
constexpr int HS_DIRECT_HPW = 8;
__global__ void __launch_bounds__(256)
    k_hs_direct(const HpHalo* __restrict__ halos, int64_t nh, const HsRing* __restrict__ R,
                int nr, const int64_t* __restrict__ offs, const uint32_t* __restrict__ keys,
                const uint32_t* __restrict__ p_halo, const int2* __restrict__ p_rg,
                const int64_t* __restrict__ voff, float n_poly, int n_int, float n_nt,
                float2* vals) {
  const int64_t k0 = (((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5) * HS_DIRECT_HPW;
  const int lane = threadIdx.x & 31;
  if (k0 >= nh) return;
  const int64_t k1 = min(nh, k0 + (int64_t)HS_DIRECT_HPW);
  const int64_t o0 = offs[k0], o1 = offs[k1];
  const int64_t e0 = voff[o0], e1 = voff[o1];
  for (int64_t e = e0 + lane; e < e1; e += 32) {
    int64_t lo = o0, hi = o1 - 1;  // the pair holding value e: the last with voff <= e
    while (lo < hi) {
      const int64_t mid = (lo + hi + 1) >> 1;
      if (voff[mid] <= e) lo = mid; else hi = mid - 1;
    }
    const HpHalo H = halos[p_halo[lo]];
    const uint32_t sg = keys[lo];
    const HsRing G = R[hs_ring_of_segment(R, nr, sg)];
    const int c0 = (int)(sg - G.seg0) * HS_SEG;
    const HsPair q = hs_pair(H, G, c0, min(HS_SEG, G.cnt - c0));
    const int t = p_rg[lo].x + (int)(e - voff[lo]);
    float uu, sy = 0.f, sb = 0.f;
    if (hs_pixel_u(q, G, H.inv_rf_px, t, uu)) {
      hp_los(H, uu, n_poly, n_int, n_nt, sy, sb);  // chord times the table value
      sy *= H.Ay;
      sb *= H.Ab;
    }
    vals[e] = make_float2(sy, sb);
  }
}

// One CTA per segment: thread t owns pixel seg_start + t of the segment's ring.  Pairs in
// sorted order (value = emission index); a halo with a table is interpolated at each pixel,
// a halo evaluated at its pixels adds the values k_hs_direct stored.
__global__ void __launch_bounds__(HS_SEG)
    k_hs_paste(const HpHalo* __restrict__ halos, const float* __restrict__ tab,
               const uint32_t* __restrict__ pvals, const int64_t* __restrict__ sstart,
               const HsRing* __restrict__ R, int nr, const uint32_t* __restrict__ p_halo,
               const int2* __restrict__ p_rg, const int64_t* __restrict__ voff,
               const float2* __restrict__ dvals, const int64_t* __restrict__ toff, float* ymap,
               float* bmap, float* ylo, float* blo) {
  __shared__ float s_dth2[HS_CH], s_sp[HS_CH], s_rh[HS_CH], s_rl[HS_CH], s_sa2[HS_CH];
  __shared__ float s_irf[HS_CH], s_ay[HS_CH], s_ab[HS_CH];
  __shared__ int2 s_rng[HS_CH];
  __shared__ const float* s_tab[HS_CH];
  __shared__ int s_nt[HS_CH];
  __shared__ int64_t s_vo[HS_CH];
  const uint32_t sg = blockIdx.x;
  const int64_t b0 = sstart[sg], b1 = sstart[sg + 1];
  if (b0 == b1) return;
  const int tid = threadIdx.x;
  const HsRing G = R[hs_ring_of_segment(R, nr, sg)];
  const int c0 = (int)(sg - G.seg0) * HS_SEG;  // ring-local index of the segment's first pixel
  const int npx = min(HS_SEG, G.cnt - c0);
  float hy = 0.f, cy = 0.f, hb = 0.f, cb = 0.f;
  for (int64_t base = b0; base < b1; base += HS_CH) {
    const int nch = (int)min((int64_t)HS_CH, b1 - base);
    __syncthreads();
    if (tid < nch) {
      const uint32_t o = pvals[base + tid];
      const uint32_t hk = p_halo[o];  // index within the chunk
      const HpHalo H = halos[hk];
      s_nt[tid] = H.nt;
      if (H.nt == 0) {  // values stored by k_hs_direct for pixels rg.x .. rg.y
        const int2 rg = p_rg[o];
        s_rng[tid] = rg;
        s_vo[tid] = voff[o] - rg.x;
      } else {
        const HsPair q = hs_pair(H, G, c0, npx);
        s_dth2[tid] = q.dth2;
        s_sp[tid] = q.sp;
        s_rh[tid] = q.rh;
        s_rl[tid] = q.rl;
        s_sa2[tid] = q.sa2;
        s_rng[tid] = q.rg;
        s_irf[tid] = H.inv_rf_px;
        s_ay[tid] = H.Ay;
        s_ab[tid] = H.Ab;
        s_tab[tid] = H.nt > 0 ? tab + toff[hk] * 2 * HP_ROW : tab;  // its table slot
      }
    }
    __syncthreads();
    if (tid < npx) {
      for (int q = 0; q < nch; ++q) {
        const int2 rg = s_rng[q];
        if (tid < rg.x || tid > rg.y) continue;
        const int ntq = s_nt[q];
        if (ntq == 0) {
          const float2 v = dvals[s_vo[q] + tid];
          kahan_add(hy, cy, v.x);
          kahan_add(hb, cb, v.y);
          continue;
        }
        HsPair pq;
        pq.dth2 = s_dth2[q];
        pq.sp = s_sp[q];
        pq.rh = s_rh[q];
        pq.rl = s_rl[q];
        pq.sa2 = s_sa2[q];
        float uu;
        if (hs_pixel_u(pq, G, s_irf[q], tid, uu)) {
          const float chord = sqrtf(fmaxf(0.f, 1.0f - uu * uu));
          const float ss = sqrtf(uu);
          const float* ty = s_tab[q];
          const float gy = catmull(ty, ss, ntq), gb = catmull(ty + HP_ROW, ss, ntq);
          kahan_add(hy, cy, s_ay[q] * chord * gy);
          kahan_add(hb, cb, s_ab[q] * chord * gb);
        }
      }
    }
  }
  if (tid < npx) {
    const int64_t p = G.first + c0 + tid;
    float sv, e;
    bp_two_sum(ymap[p], hy, sv, e);
    ymap[p] = sv;
    ylo[p] = ylo[p] + (e - cy);
    bp_two_sum(bmap[p], hb, sv, e);
    bmap[p] = sv;
    blo[p] = blo[p] + (e - cb);
  }
}

// The ring table of nside N (host, FP64): 4N - 1 rings, segments counted along them.
void hs_ring_table(int64_t N, HsRing* R, int64_t* n_seg) {
  uint32_t seg = 0;
  for (int64_t i = 1; i <= 4 * N - 1; ++i) {
    HsRing G;
    double z;
    int64_t cnt, first;
    double phase;
    if (i < N) {
      z = 1.0 - (double)(i * i) / (3.0 * (double)N * (double)N);
      cnt = 4 * i;
      first = 2 * i * (i - 1);
      phase = 0.5;
    } else if (i <= 3 * N) {
      z = 4.0 / 3.0 - 2.0 * (double)i / (3.0 * (double)N);
      cnt = 4 * N;
      first = 2 * N * (N - 1) + 4 * N * (i - N);
      phase = ((i + N) & 1) ? 0.0 : 0.5;
    } else {
      const int64_t k = 4 * N - i;
      z = -(1.0 - (double)(k * k) / (3.0 * (double)N * (double)N));
      cnt = 4 * k;
      first = 12 * N * N - 2 * k * (k + 1);
      phase = 0.5;
    }
    G.theta = acos(z);
    G.first = first;
    G.sin_t = (float)sqrt((1.0 - z) * (1.0 + z));
    G.phase = (float)phase;
    G.dphi = (float)(2.0 * bpc::PI / (double)cnt);
    G.cnt = (int32_t)cnt;
    G.seg0 = seg;
    G.pad = 0;
    R[i - 1] = G;
    seg += (uint32_t)((cnt + HS_SEG - 1) / HS_SEG);
  }
  *n_seg = seg;
}

}  // namespace

// A prepared halo paste: the work list of one catalogue and its own buffers.
struct bp_hp_plan {
  int64_t n;
  bp_map_geom geom;
  double ap_r500;
  int ts, grid;
  HpList L;
  HpHalo* halos;
  float* tab;
  float* partials;
  int64_t* counter;
  float2* dvals;  // values of the halos evaluated at their pixels
  void* mem[12];
};

extern "C" {

int bp_paste_halos(bp_ctx* ctx, int64_t n, const double* th_x, const double* th_y,
                   const float* v_los, const int32_t* map_id, const double* model,
                   const int32_t* status, const bp_map_geom* geom, double ap_r500, float* ymap,
                   float* bmap, float* ylo, float* blo) {
  if (!ctx) return BP_EINVAL;
  int r = check_hp_args(ctx, n, th_x, th_y, model, status, geom, ap_r500, "bp_paste_halos");
  if (r || n == 0) return r;
  if (!v_los || !ymap || !bmap || !ylo || !blo)
    return bp_fail(ctx, BP_EINVAL, "bp_paste_halos: null pointer");
  if ((r = hp_constants(ctx))) return r;
  HpHalo* halos;
  if ((r = bp_ws(ctx, WS_HPAR, (size_t)n * sizeof(HpHalo), (void**)&halos))) return r;
  const int TS = ctx->hp_tile;
  HpList L;
  // halo records and the work list (which also lists the halos that need a table)
  bp_phase_begin(ctx, BP_PH_HP_PAIRS);
  if ((r = hp_prep(ctx, n, th_x, th_y, v_los, map_id, model, status, geom, ap_r500, halos)))
    return r;
  if ((r = hp_build_list(ctx, n, halos, geom, TS, ctx->hp_unit, &L))) return r;
  bp_phase_end(ctx, BP_PH_HP_PAIRS);
  if (L.np == 0) return BP_OK;
  float* tab;
  if ((r = bp_ws(ctx, WS_TABLE, (size_t)(L.n_table > 0 ? L.n_table : 1) * 2 * HP_ROW *
                                    sizeof(float), (void**)&tab)))
    return r;
  bp_phase_begin(ctx, BP_PH_HP_TABLE);
  if ((r = hp_tables(ctx, halos, L.tlist, L.n_table, tab))) return r;
  bp_phase_end(ctx, BP_PH_HP_TABLE);
  float* partials;
  if ((r = bp_ws(ctx, WS_PART, (size_t)(L.n_slots > 0 ? L.n_slots : 1) * 4 * TS * TS * 4,
                 (void**)&partials)))
    return r;
  int grid = TS == 64 ? hp_grid<64>(ctx, 0, L.n_units) : hp_grid<32>(ctx, 0, L.n_units);
  if (grid < 0) return bp_fail(ctx, BP_ECUDA, "bp_paste_halos: occupancy query");
  float2* dvals;
  if ((r = bp_ws(ctx, WS_MISC3, (size_t)(L.nval > 0 ? L.nval : 1) * sizeof(float2),
                 (void**)&dvals)))
    return r;
  bp_phase_begin(ctx, BP_PH_HP_PASTE);
  r = TS == 64 ? hp_launch<64>(ctx, halos, tab, L, grid, partials, ctx->d_counter + 2, geom, dvals,
                               ymap, bmap, ylo, blo)
               : hp_launch<32>(ctx, halos, tab, L, grid, partials, ctx->d_counter + 2, geom, dvals,
                               ymap, bmap, ylo, blo);
  bp_phase_end(ctx, BP_PH_HP_PASTE);
  return r;
}

int bp_hp_pairs(bp_ctx* ctx, int64_t n, const double* th_x, const double* th_y,
                const int32_t* map_id, const double* model, const int32_t* status,
                const bp_map_geom* geom, double ap_r500, int tile, uint32_t* keys, uint32_t* vals,
                int64_t capacity, int64_t* n_pairs) {
  if (!ctx) return BP_EINVAL;
  if (!n_pairs) return bp_fail(ctx, BP_EINVAL, "bp_hp_pairs: null count");
  *n_pairs = 0;
  int r = check_hp_args(ctx, n, th_x, th_y, model, status, geom, ap_r500, "bp_hp_pairs");
  if (r) return r;
  if (tile != 32 && tile != 64) return bp_fail(ctx, BP_EINVAL, "bp_hp_pairs: tile must be 32 or 64");
  if (n == 0) return BP_OK;
  HpHalo* halos;
  if ((r = bp_ws(ctx, WS_HPAR, (size_t)n * sizeof(HpHalo), (void**)&halos))) return r;
  // the records and the work list of bp_paste_halos (v_los only enters the amplitudes)
  if ((r = hp_prep(ctx, n, th_x, th_y, nullptr, map_id, model, status, geom, ap_r500, halos)))
    return r;
  HpList L;
  if ((r = hp_build_list(ctx, n, halos, geom, tile, ctx->hp_unit, &L))) return r;
  *n_pairs = L.np;
  if (L.np > capacity)
    return bp_fail(ctx, BP_ERANGE, "bp_hp_pairs: capacity %lld < %lld", (long long)capacity,
                   (long long)L.np);
  if (L.np > 0) {
    if (!keys || !vals) return bp_fail(ctx, BP_EINVAL, "bp_hp_pairs: null output");
    BP_CUDA(ctx, cudaMemcpyAsync(keys, L.keys, L.np * 4, cudaMemcpyDeviceToDevice, ctx->stream));
    BP_CUDA(ctx, cudaMemcpyAsync(vals, L.vals, L.np * 4, cudaMemcpyDeviceToDevice, ctx->stream));
  }
  BP_CUDA(ctx, cudaStreamSynchronize(ctx->stream));
  return BP_OK;
}

int bp_hp_plan_create(bp_ctx* ctx, int64_t n, const double* th_x, const double* th_y,
                      const int32_t* map_id, const double* model, const int32_t* status,
                      const bp_map_geom* geom, double ap_r500, int tile, int unit, int ctas_per_sm,
                      bp_hp_plan** out) {
  if (!ctx || !out) return BP_EINVAL;
  *out = nullptr;
  int r = check_hp_args(ctx, n, th_x, th_y, model, status, geom, ap_r500, "bp_hp_plan_create");
  if (r) return r;
  if (tile != 32 && tile != 64) return bp_fail(ctx, BP_EINVAL, "bp_hp_plan_create: tile");
  if (unit < 0 || ctas_per_sm < 0) return bp_fail(ctx, BP_EINVAL, "bp_hp_plan_create: unit/ctas");
  if ((r = hp_constants(ctx))) return r;
  bp_hp_plan* p = (bp_hp_plan*)calloc(1, sizeof(bp_hp_plan));
  if (!p) return bp_fail(ctx, BP_ENOMEM, "bp_hp_plan_create: host memory");
  p->n = n;
  p->geom = *geom;
  p->ap_r500 = ap_r500;
  p->ts = tile;
  auto alloc = [&](int slot, size_t bytes) -> void* {
    void* q = nullptr;
    if (cudaMalloc(&q, bytes ? bytes : 16) != cudaSuccess) {
      cudaGetLastError();
      return nullptr;
    }
    p->mem[slot] = q;
    return q;
  };
  auto fail = [&](int code, const char* what) {
    bp_hp_plan_destroy(p);
    return bp_fail(ctx, code, "bp_hp_plan_create: %s", what);
  };
  int64_t nn = n > 0 ? n : 1;
  p->halos = (HpHalo*)alloc(0, (size_t)nn * sizeof(HpHalo));
  p->counter = (int64_t*)alloc(2, 64);
  if (!p->halos || !p->counter) return fail(BP_ENOMEM, "device memory");
  if (n > 0) {
    // the work list needs the apertures: prepare the halo records once here
    const int pb = bp_item_block(ctx, n, 256);
    k_hp_prep<<<(unsigned)((n + pb - 1) / pb), pb, 0, ctx->stream>>>(
        ctx->p, n, th_x, th_y, nullptr, map_id, model, status, *geom, ap_r500, p->halos);
    if (cudaGetLastError() != cudaSuccess) return fail(BP_ECUDA, "prep launch");
    ctx->launches++;
    HpList L;
    if ((r = hp_build_list(ctx, n, p->halos, geom, tile, unit, &L))) {
      bp_hp_plan_destroy(p);
      return r;
    }
    p->L = L;
    if (L.np > 0) {
      // copy the list out of the context's scratch into the plan
      uint32_t* vals = (uint32_t*)alloc(3, (size_t)L.np * 4);
      int64_t* tiles = (int64_t*)alloc(4, (size_t)(L.n_tiles + 1) * 3 * 8);
      HpUnit* units = (HpUnit*)alloc(5, (size_t)(L.n_units + 1) * sizeof(HpUnit));
      p->partials = (float*)alloc(6, (size_t)(L.n_slots > 0 ? L.n_slots : 1) * 4 * tile * tile * 4);
      int64_t* hvoff = (int64_t*)alloc(7, (size_t)(n + 1) * 8);
      HpDBox* dbox = (HpDBox*)alloc(9, (size_t)n * sizeof(HpDBox));
      p->dvals = (float2*)alloc(8, (size_t)(L.nval > 0 ? L.nval : 1) * sizeof(float2));
      int64_t* toff = (int64_t*)alloc(10, (size_t)(n + 1) * 8);
      uint32_t* tlist = (uint32_t*)alloc(11, (size_t)(L.n_table > 0 ? L.n_table : 1) * 4);
      p->tab = (float*)alloc(1, (size_t)(L.n_table > 0 ? L.n_table : 1) * 2 * HP_ROW *
                                    sizeof(float));
      if (!vals || !tiles || !units || !p->partials || !hvoff || !dbox || !p->dvals || !toff ||
          !tlist || !p->tab)
        return fail(BP_ENOMEM, "device memory");
      cudaStream_t s = ctx->stream;
      size_t tb = (size_t)(L.n_tiles + 1) * 8;
      if (cudaMemcpyAsync(vals, L.vals, (size_t)L.np * 4, cudaMemcpyDeviceToDevice, s) ||
          cudaMemcpyAsync(tiles, L.tstart, tb, cudaMemcpyDeviceToDevice, s) ||
          cudaMemcpyAsync(tiles + (L.n_tiles + 1), L.uoff, tb, cudaMemcpyDeviceToDevice, s) ||
          cudaMemcpyAsync(tiles + 2 * (L.n_tiles + 1), L.soff, tb, cudaMemcpyDeviceToDevice, s) ||
          cudaMemcpyAsync(units, L.units, (size_t)L.n_units * sizeof(HpUnit),
                          cudaMemcpyDeviceToDevice, s) ||
          cudaMemcpyAsync(hvoff, L.hvoff, (size_t)(n + 1) * 8, cudaMemcpyDeviceToDevice, s) ||
          cudaMemcpyAsync(dbox, L.dbox, (size_t)n * sizeof(HpDBox), cudaMemcpyDeviceToDevice,
                          s) ||
          cudaMemcpyAsync(toff, L.toff, (size_t)(n + 1) * 8, cudaMemcpyDeviceToDevice, s) ||
          (L.n_table > 0 && cudaMemcpyAsync(tlist, L.tlist, (size_t)L.n_table * 4,
                                            cudaMemcpyDeviceToDevice, s)) ||
          cudaStreamSynchronize(s))
        return fail(BP_ECUDA, "copy of the work list");
      p->L.vals = vals;
      p->L.tstart = tiles;
      p->L.uoff = tiles + (L.n_tiles + 1);
      p->L.soff = tiles + 2 * (L.n_tiles + 1);
      p->L.units = units;
      p->L.hvoff = hvoff;
      p->L.dbox = dbox;
      p->L.toff = toff;
      p->L.tlist = tlist;
      p->grid = tile == 64 ? hp_grid<64>(ctx, ctas_per_sm, L.n_units)
                           : hp_grid<32>(ctx, ctas_per_sm, L.n_units);
      if (p->grid < 0) return fail(BP_ECUDA, "occupancy query");
    }
  }
  *out = p;
  return BP_OK;
}

int bp_hp_plan_execute(bp_ctx* ctx, bp_hp_plan* p, const double* th_x, const double* th_y,
                       const float* v_los, const int32_t* map_id, const double* model,
                       const int32_t* status, float* ymap, float* bmap, float* ylo, float* blo) {
  if (!ctx || !p) return BP_EINVAL;
  if (p->n == 0 || p->L.np == 0) return BP_OK;
  if (!th_x || !th_y || !v_los || !model || !status || !ymap || !bmap || !ylo || !blo)
    return bp_fail(ctx, BP_EINVAL, "bp_hp_plan_execute: null pointer");
  int r;
  bp_phase_begin(ctx, BP_PH_HP_TABLE);
  if ((r = hp_prep(ctx, p->n, th_x, th_y, v_los, map_id, model, status, &p->geom, p->ap_r500,
                   p->halos)))
    return r;
  if ((r = hp_tables(ctx, p->halos, p->L.tlist, p->L.n_table, p->tab))) return r;
  bp_phase_end(ctx, BP_PH_HP_TABLE);
  bp_phase_begin(ctx, BP_PH_HP_PASTE);
  r = p->ts == 64 ? hp_launch<64>(ctx, p->halos, p->tab, p->L, p->grid, p->partials, p->counter,
                                  &p->geom, p->dvals, ymap, bmap, ylo, blo)
                  : hp_launch<32>(ctx, p->halos, p->tab, p->L, p->grid, p->partials, p->counter,
                                  &p->geom, p->dvals, ymap, bmap, ylo, blo);
  bp_phase_end(ctx, BP_PH_HP_PASTE);
  return r;
}

int64_t bp_hp_plan_pairs(const bp_hp_plan* p) { return p ? p->L.np : 0; }

int bp_hp_plan_destroy(bp_hp_plan* p) {
  if (!p) return BP_OK;
  for (int k = 0; k < 12; ++k)
    if (p->mem[k]) cudaFree(p->mem[k]);
  free(p);
  return BP_OK;
}

int bp_finalize_map(bp_ctx* ctx, const bp_map_geom* geom, float* ymap, float* bmap, float* ylo,
                    float* blo, int out_kind, double nu_ghz) {
  if (!ctx) return BP_EINVAL;
  if (!geom || geom->nx <= 0 || geom->ny <= 0 || geom->n_maps <= 0)
    return bp_fail(ctx, BP_EINVAL, "bp_finalize_map: bad geometry");
  if (out_kind != BP_OUT_YB && out_kind != BP_OUT_DT)
    return bp_fail(ctx, BP_EINVAL, "bp_finalize_map: out_kind");
  float sy = 1.f, sb = 1.f;
  if (out_kind == BP_OUT_DT) {
    if (!(nu_ghz > 0)) return bp_fail(ctx, BP_EINVAL, "bp_finalize_map: nu_ghz <= 0");
    // g_nu(x) = x (e^x + 1)/(e^x - 1) - 4 (Section 3.2), x = h nu / (k T_CMB)
    double x = bpc::H_PLANCK * nu_ghz * 1e9 / (bpc::K_BOLTZ * ctx->p.Tcmb);
    sy = (float)(x * (exp(x) + 1.0) / (exp(x) - 1.0) - 4.0);
    sb = -1.f;
  }
  int64_t npix = (int64_t)geom->nx * geom->ny * geom->n_maps;
  unsigned nb = (unsigned)((npix + 255) / 256);
  bp_phase_begin(ctx, BP_PH_FINALIZE);
  auto al16 = [](const void* p) { return ((uintptr_t)p & 15) == 0; };
  if (ymap && bmap && ylo && blo && al16(ymap) && al16(bmap) && al16(ylo) && al16(blo)) {
    // both planes in one pass, four pixels per thread; the npix % 4 tail below
    const int64_t n4 = npix / 4;
    if (n4 > 0) {
      k_finalize4<<<(unsigned)((n4 + 255) / 256), 256, 0, ctx->stream>>>(
          n4, reinterpret_cast<float4*>(ymap), reinterpret_cast<float4*>(ylo), sy,
          reinterpret_cast<float4*>(bmap), reinterpret_cast<float4*>(blo), sb);
      BP_LAUNCH_CHECK(ctx, "finalize (4 per thread)");
    }
    const int64_t t = npix - 4 * n4;
    if (t > 0) {
      k_finalize<<<1, 256, 0, ctx->stream>>>(t, ymap + 4 * n4, ylo + 4 * n4, sy);
      BP_LAUNCH_CHECK(ctx, "finalize y");
      k_finalize<<<1, 256, 0, ctx->stream>>>(t, bmap + 4 * n4, blo + 4 * n4, sb);
      BP_LAUNCH_CHECK(ctx, "finalize b");
    }
    bp_phase_end(ctx, BP_PH_FINALIZE);
    return BP_OK;
  }
  if (ymap) {
    k_finalize<<<nb, 256, 0, ctx->stream>>>(npix, ymap, ylo, sy);
    BP_LAUNCH_CHECK(ctx, "finalize y");
  }
  if (bmap) {
    k_finalize<<<nb, 256, 0, ctx->stream>>>(npix, bmap, blo, sb);
    BP_LAUNCH_CHECK(ctx, "finalize b");
  }
  bp_phase_end(ctx, BP_PH_FINALIZE);
  return BP_OK;
}

int bp_paste_halos_healpix(bp_ctx* ctx, int64_t n, const double* theta, const double* phi,
                           const float* v_los, const double* model, const int32_t* status,
                           int nside, double ap_r500, float* ymap, float* bmap, float* ylo,
                           float* blo) {
  if (!ctx) return BP_EINVAL;
  if (n < 0) return bp_fail(ctx, BP_EINVAL, "bp_paste_halos_healpix: n < 0");
  if (nside < 1 || nside > 16384)
    return bp_fail(ctx, BP_EINVAL, "bp_paste_halos_healpix: nside outside [1, 16384]");
  if (ap_r500 < 0) return bp_fail(ctx, BP_EINVAL, "bp_paste_halos_healpix: ap_r500 < 0");
  if (n == 0) return BP_OK;
  if (n > (int64_t)UINT32_MAX) return bp_fail(ctx, BP_ERANGE, "bp_paste_halos_healpix: n >= 2^32");
  if (!theta || !phi || !v_los || !model || !status || !ymap || !bmap || !ylo || !blo)
    return bp_fail(ctx, BP_EINVAL, "bp_paste_halos_healpix: null pointer");
  int r;
  if ((r = hp_constants(ctx))) return r;
  // ring table (cached per nside in the context's scratch)
  const int nr = 4 * nside - 1;
  std::vector<HsRing> hr(nr);
  int64_t n_seg = 0;
  hs_ring_table(nside, hr.data(), &n_seg);
  HsRing* R;
  if ((r = bp_ws(ctx, WS_MISC3, (size_t)nr * sizeof(HsRing), (void**)&R))) return r;
  BP_CUDA(ctx, cudaMemcpyAsync(R, hr.data(), (size_t)nr * sizeof(HsRing), cudaMemcpyHostToDevice,
                               ctx->stream));
  // halos in chunks (bounded table memory); each chunk adds into the maps
  const int64_t CHUNK = (int64_t)1 << 22;
  for (int64_t h0 = 0; h0 < n; h0 += CHUNK) {
    const int64_t m = std::min(CHUNK, n - h0);
    HpHalo* halos;
    if ((r = bp_ws(ctx, WS_HPAR, (size_t)m * sizeof(HpHalo), (void**)&halos))) return r;
    const unsigned nb = (unsigned)((m + 255) / 256);
    const BpParams& P = ctx->p;
    double rn = rint(P.n_poly);
    int n_int = (fabs(P.n_poly - rn) < 1e-12 && rn >= 1 && rn <= 16) ? (int)rn : -1;
    // halo records, pair counts, and the compact list of the halos that need a table
    bp_phase_begin(ctx, BP_PH_HP_TABLE);
    k_hs_prep<<<nb, 256, 0, ctx->stream>>>(ctx->p, n, h0, m, theta, phi, v_los, model, status,
                                           ap_r500, nside, halos);
    BP_LAUNCH_CHECK(ctx, "healpix prep");
    uint32_t* counts;
    int64_t *offs, *toff;
    if ((r = bp_ws(ctx, WS_COUNTS, (size_t)(m + 1) * 8, (void**)&counts))) return r;
    if ((r = bp_ws(ctx, WS_OFFS, (size_t)(m + 1) * 16, (void**)&offs))) return r;
    uint32_t* tflag = counts + (m + 1);
    toff = offs + (m + 1);
    uint32_t* tlist;
    if ((r = bp_ws(ctx, WS_MISC2, (size_t)m * 4 + 16, (void**)&tlist))) return r;
    k_hs_count<<<nb, 256, 0, ctx->stream>>>(halos, m, R, nr, counts, tflag);
    BP_LAUNCH_CHECK(ctx, "healpix count");
    if ((r = bp_scan_u32_to_i64(ctx, counts, offs, m))) return r;
    if ((r = bp_scan_u32_to_i64(ctx, tflag, toff, m))) return r;
    BP_CUDA(ctx, cudaMemcpyAsync(ctx->h_pinned, offs + m, 8, cudaMemcpyDeviceToHost, ctx->stream));
    BP_CUDA(ctx, cudaMemcpyAsync(ctx->h_pinned + 1, toff + m, 8, cudaMemcpyDeviceToHost,
                                 ctx->stream));
    k_hp_tab_emit<<<nb, 256, 0, ctx->stream>>>(tflag, toff, m, tlist);
    BP_LAUNCH_CHECK(ctx, "healpix table list");
    BP_CUDA(ctx, cudaStreamSynchronize(ctx->stream));
    const int64_t np = ctx->h_pinned[0], n_table = ctx->h_pinned[1];
    if (np > (int64_t)UINT32_MAX)
      return bp_fail(ctx, BP_ERANGE, "bp_paste_halos_healpix: too many pairs");
    if (np == 0) {
      bp_phase_end(ctx, BP_PH_HP_TABLE);
      continue;
    }
    float* tab;
    if ((r = bp_ws(ctx, WS_TABLE, (size_t)(n_table > 0 ? n_table : 1) * 2 * HP_ROW *
                                      sizeof(float), (void**)&tab)))
      return r;
    if ((r = hp_tables(ctx, halos, tlist, n_table, tab))) return r;
    bp_phase_end(ctx, BP_PH_HP_TABLE);
    // (segment, halo) pairs sorted by segment
    bp_phase_begin(ctx, BP_PH_HP_PAIRS);
    uint32_t *k0, *v0, *k1, *v1, *ks, *vs;
    if ((r = bp_ws(ctx, WS_KEYS0, (size_t)np * 4, (void**)&k0))) return r;
    if ((r = bp_ws(ctx, WS_VALS0, (size_t)np * 4, (void**)&v0))) return r;
    if ((r = bp_ws(ctx, WS_KEYS1, (size_t)np * 4, (void**)&k1))) return r;
    if ((r = bp_ws(ctx, WS_VALS1, (size_t)np * 4, (void**)&v1))) return r;
    // per pair: its halo, and for halos evaluated at their pixels the pixel range and the
    // offset of its values
    char* pbuf;
    if ((r = bp_ws(ctx, WS_UNITS, (size_t)np * 16 + 64, (void**)&pbuf))) return r;
    int2* p_rg = reinterpret_cast<int2*>(pbuf);
    uint32_t* p_halo = reinterpret_cast<uint32_t*>(p_rg + np);
    uint32_t* p_len = p_halo + np;
    int64_t* voff;
    if ((r = bp_ws(ctx, WS_PART, (size_t)(np + 1) * 8, (void**)&voff))) return r;
    k_hs_emit<<<nb, 256, 0, ctx->stream>>>(halos, m, R, nr, offs, k0, v0, p_halo, p_rg, p_len);
    BP_LAUNCH_CHECK(ctx, "healpix emit");
    if ((r = bp_scan_u32_to_i64(ctx, p_len, voff, np))) return r;
    BP_CUDA(ctx, cudaMemcpyAsync(ctx->h_pinned, voff + np, 8, cudaMemcpyDeviceToHost, ctx->stream));
    BP_CUDA(ctx, cudaStreamSynchronize(ctx->stream));
    const int64_t nval = ctx->h_pinned[0];
    float2* dvals;
    if ((r = bp_ws(ctx, WS_HALO, (size_t)(nval > 0 ? nval : 1) * sizeof(float2), (void**)&dvals)))
      return r;
    if (nval > 0) {  // before the sort: it reads the keys in emission order
      const int64_t dwarps = (m + HS_DIRECT_HPW - 1) / HS_DIRECT_HPW;
      k_hs_direct<<<(unsigned)((dwarps * 32 + 255) / 256), 256, 0, ctx->stream>>>(
          halos, m, R, nr, offs, k0, p_halo, p_rg, voff, (float)P.n_poly, n_int, (float)P.n_nt,
          dvals);
      BP_LAUNCH_CHECK(ctx, "healpix direct values");
    }
    int key_bits = 0;
    while (((int64_t)1 << key_bits) < n_seg) ++key_bits;
    if ((r = bp_radix_sort_pairs(ctx, k0, v0, k1, v1, np, key_bits, &ks, &vs))) return r;
    int64_t* sstart;
    if ((r = bp_ws(ctx, WS_TILES, (size_t)(n_seg + 1) * 8, (void**)&sstart))) return r;
    if ((r = bp_tile_ranges(ctx, ks, np, n_seg, sstart))) return r;
    bp_phase_end(ctx, BP_PH_HP_PAIRS);
    bp_phase_begin(ctx, BP_PH_HP_PASTE);
    k_hs_paste<<<(unsigned)n_seg, HS_SEG, 0, ctx->stream>>>(
        halos, tab, vs, sstart, R, nr, p_halo, p_rg, voff, dvals, toff, ymap, bmap, ylo, blo);
    BP_LAUNCH_CHECK(ctx, "healpix paste");
    bp_phase_end(ctx, BP_PH_HP_PASTE);
  }
  return BP_OK;
}

}  // extern "C"

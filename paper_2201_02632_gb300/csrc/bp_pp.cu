// bp_pp.cu -- particle-based pasting (Section 3.4).
//
//  k_halo_block    per-halo FP32 constants of the solved profiles
//  k_assign        per particle: sky angles (FP64), pixel coordinates, kernel radius,
//                  y_i and b_i (Eqs. y_i^PP,h, b_i^PP,h, field_y, field_b)
//  k_pair_count /  (tile, particle) pairs of every tile a particle's 2h square
//  k_pair_emit     touches, in particle order
//  radix sort      stable by tile key (bp_sort.cu)
//  k_units         split each tile's particle list into work units
//  k_deposit       persistent: one CTA accumulates one work unit's particles into a
//                  register/shared-memory tile with the separable pixel-integrated
//                  kernel f_ij (Eqs. f_ij, integrated kernel); compensated FP32 sums;
//                  single-unit tiles are added to the map directly, others are
//                  written as partial tiles
//  k_reduce_tiles  adds the partial tiles of multi-unit tiles in unit order
// No global atomics touch the maps; every pixel sum is in a fixed order.
#include <cstring>

#include "bp_internal.cuh"

namespace {

// ---------------------------------------------------------------- halo constants
// FP32 per-halo block used by the assignment (16 floats):
//  [0] sx   comoving h^-1 Mpc -> x = r/r_s
//  [1] xf   r_f / r_s
//  [2] c    r_vir / r_s
//  [3] q500 r_s / r500
//  [4] psi  G M / (m(c) r_s (n+1) T)   (theta = 1 - psi g(x) inside r_vir)
//  [5] A0   |Phi0| / ((n+1) T)          (theta = 1 - A0 + A1 / x outside r_vir)
//  [6] A1   G M / (r_s (n+1) T)
//  [7] ant  alpha_nt f(z)
//  [8] KY   sigma_T/(m_e c^2) (P_e/P_th) P0 M_p / rho_s  [y units x Mpc^2]
//  [9] KB   sigma_T rho0/(mu_e m_p) M_p / rho_s        [b units x Mpc^2]
//  [10] ok  1 if the halo solved
//  [11] Phi0, [12] 1 / ((n+1) T)   (the potential-based variant)
//  [13..15] the halo centre (comoving h^-1 Mpc), so that a particle reads one 64-byte block
constexpr int HB = 16;

__global__ void k_halo_block(BpParams P, int64_t nh, const double* __restrict__ model,
                             const int32_t* __restrict__ status, double Mp,
                             const float* __restrict__ hpos, float* blk) {
  int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= nh) return;
  auto F = [&](int f) { return model[(int64_t)f * nh + k]; };
  double rs = F(BP_M_RS), c = F(BP_M_C), z = F(BP_M_Z), M = F(BP_M_MVIR), mc = F(BP_M_MC);
  double T = F(BP_M_T), n1T = (P.n_poly + 1.0) * T;
  double GM = bpc::G * M;
  float* b = blk + k * HB;
  bool ok = status[k] == BP_HALO_OK && rs > 0 && T > 0;
  b[0] = ok ? (float)(1.0 / (P.h * (1.0 + z) * rs)) : 0.f;
  b[1] = ok ? (float)(F(BP_M_RF) / rs) : 0.f;
  b[2] = (float)c;
  b[3] = ok ? (float)(rs / F(BP_M_R500)) : 0.f;
  b[4] = ok ? (float)(GM / (mc * rs * n1T)) : 0.f;
  b[5] = ok ? (float)(-F(BP_M_PHI0) / n1T) : 0.f;
  b[6] = ok ? (float)(GM / (rs * n1T)) : 0.f;
  b[7] = (float)F(BP_M_ANT);
  double rhos = F(BP_M_RHOS);
  b[8] = ok ? (float)(P.CP * P.pe_frac * F(BP_M_P0) * Mp / rhos) : 0.f;
  b[9] = ok ? (float)(P.CN * F(BP_M_RHO0) * Mp / rhos) : 0.f;
  b[10] = ok ? 1.f : 0.f;
  b[11] = ok ? (float)F(BP_M_PHI0) : 0.f;  // the potential-based variant: theta = 1 +
  b[12] = ok ? (float)(1.0 / n1T) : 0.f;   //   (Phi0 - phi_i) / ((n + 1) T)
  b[13] = hpos ? hpos[k] : 0.f;
  b[14] = hpos ? hpos[nh + k] : 0.f;
  b[15] = hpos ? hpos[2 * nh + k] : 0.f;
}

// 1 - ln(1+x)/x without cancellation
__device__ __forceinline__ float g_inner(float x) {
  if (x < 2e-2f) return x * (0.5f - x * (1.0f / 3.0f - x * (0.25f - x * 0.2f)));
  return 1.0f - log1pf(x) / x;
}

__device__ __forceinline__ float powi_or_pow(float t, float n, int n_int) {
  if (n_int > 0) {
    float r = 1.f, b = t;
    int e = n_int;
    while (e) {
      if (e & 1) r *= b;
      b *= b;
      e >>= 1;
    }
    return r;
  }
  return powf(t, n);
}

// px = ix + fx with ix = floor(px) (clamped to +-2^30) and 0 <= fx < 1 in FP32
__device__ __forceinline__ float split_pixel(double p, int& ip) {
  double fl = floor(p);
  if (!(fl == fl)) { ip = 0; return __int_as_float(0x7fc00000); }
  fl = fmin(fmax(fl, -1073741824.0), 1073741824.0);
  float f = (float)(p - fl);
  if (f >= 1.0f) { fl += 1.0; f = 0.0f; }
  if (f < 0.0f) f = 0.0f;
  ip = (int)fl;
  return f;
}

// Sky angle atan2(x, z) of a particle and its pixel coordinate (theta - theta0) / dtheta
// = ip + f (0 <= f < 1) in double-float FP32 arithmetic (pairs hi + lo), for
// 0 < |x| <= z / 16 (flat-sky maps up to about 7 deg wide; returns false otherwise).
// t = x / z is the FP32 quotient q plus the exact FMA remainder over z; atan(t) = t - t^3/3
// + t^5/5 - ..., with the cubic term in double-float (its FP32 rounding alone would be
// 4e-13 rad at t = 1/16) and the higher terms in FP32.  theta0 and 1/dtheta come as FP32
// pairs.  Error about 1e-8 pixel.
__device__ __forceinline__ bool pixel_fast(float x, float z, float rz, float th0_hi,
                                           float th0_lo, float inv_hi, float inv_lo, int& ip,
                                           float& f) {
  if (!(z > 0.f) || !(fabsf(x) <= 0.0625f * z)) return false;
  const float q = __fdiv_rn(x, z);
  const float tl = fmaf(-q, z, x) * rz;  // the exact remainder over z
  const float q2 = __fmul_rn(q, q), q2e = fmaf(q, q, -q2);
  const float q3 = __fmul_rn(q2, q), q3e = fmaf(q2, q, -q3) + q2e * q;
  const float c = __fdiv_rn(-q3, 3.0f);
  const float ce = fmaf(-3.0f, c, -q3) * (1.0f / 3.0f);  // (-q3 - 3c) is exact
  const float tail =
      q3 * q2 *
      (0.2f + q2 * (-1.0f / 7.0f + q2 * (1.0f / 9.0f + q2 * (-1.0f / 11.0f + q2 * (1.0f / 13.0f)))));
  float s, e;
  bp_two_sum(q, c, s, e);  // theta = s + lo
  const float lo = e + ((tl + ce) - q3e * (1.0f / 3.0f) + tail);
  float d, de;
  bp_two_sum(s, -th0_hi, d, de);
  const float dl = (de + lo) - th0_lo;  // theta - theta0 = d + dl
  const float p = __fmul_rn(d, inv_hi);
  const float pe = fmaf(d, inv_hi, -p) + (d * inv_lo + dl * inv_hi);
  float fl = floorf(p);
  float fr = (p - fl) + pe;  // pe is a few ulps of p: fr in (-1, 2)
  if (fr < 0.f) {
    fl -= 1.f;
    fr += 1.f;  // may round up to 1 when fr was a tiny negative
    if (fr >= 1.f) {
      fl += 1.f;
      fr = 0.f;
    }
  } else if (fr >= 1.f) {
    fl += 1.f;
    fr -= 1.f;  // exact
  }
  if (!(fabsf(fl) < 1073741824.f)) return false;
  ip = (int)fl;
  f = fr;
  return true;
}

struct AssignArgs {
  const float *x, *y, *z, *vx, *vy, *vz, *hs;
  const float* phi;  // per-particle potential [(km/s)^2] or null (spherical model at r_i)
  const int32_t* hid;
  const float* hpos;
  const float* blk;
  int64_t n, nh;
  double th0x, th0y, inv_dth;
  float th0x_hi, th0x_lo, th0y_hi, th0y_lo, inv_hi, inv_lo;  // FP32 pairs of the above
  float inv_h;        // 1/h (h^-1 Mpc -> Mpc)
  float inv_h_dth;    // 1/(h dtheta)
  float inv_om_pix;   // 1/dtheta^2
  float field_B;      // C_N M_p(/f_b) / c  [b units x Mpc^2 / (km/s)]
  float n_poly;
  int n_int;
  float n_nt;
  float* out;
};

// MODE 0: the whole record.  MODE 1 (geometry, needs no solved halos): pixel coordinates and
// h in pixels, Y = B = 0, and the kind from the halo id alone (a halo particle outside its
// halo's truncation radius stays HALO, with zero signals later).  MODE 2 (signals): only Y,
// B and the kind, the same values as MODE 0, into a record whose geometry MODE 1 wrote.
// The record of particle i from its SoA fields, as its two 16-byte halves.
template <int MODE>
__device__ __forceinline__ void assign_rec(const AssignArgs& a, const BpTables& T,
                                           const float4* zt, int64_t i, float xf, float yf,
                                           float zf, float vxf, float vyf, float vzf, float hsf,
                                           int32_t k, float4& o0, float4& o1) {
  // sky angles and pixel coordinates: double-float FP32 near the axis, else FP64
  int ix = 0, iy = 0;
  float fx = 0.f, fy = 0.f;
  if constexpr (MODE != 2) {
    const float rz = 1.0f / zf;
    if (!pixel_fast(xf, zf, rz, a.th0x_hi, a.th0x_lo, a.inv_hi, a.inv_lo, ix, fx))
      fx = split_pixel((atan2((double)xf, (double)zf) - a.th0x) * a.inv_dth, ix);
    if (!pixel_fast(yf, zf, rz, a.th0y_hi, a.th0y_lo, a.inv_hi, a.inv_lo, iy, fy))
      fy = split_pixel((atan2((double)yf, (double)zf) - a.th0y) * a.inv_dth, iy);
  }
  float r2 = xf * xf + yf * yf + zf * zf;
  float rh = sqrtf(r2);       // comoving h^-1 Mpc
  float chi = rh * a.inv_h;   // comoving Mpc
  float Y = 0.f, B = 0.f;
  int kind = BP_KIND_NONE;
  float hp = 0.f;
  if constexpr (MODE == 1) {
    if (rh > 0.f) {
      hp = hsf * a.inv_h_dth / chi;
      kind = k < 0 ? BP_KIND_FIELD : (k < a.nh ? BP_KIND_HALO : BP_KIND_NONE);
    }
  } else if (rh > 0.f) {
    if constexpr (MODE == 0) hp = hsf * a.inv_h_dth / chi;  // exact rounding: the pair list
    float zz, tau;
    bp_hermite_ztau(T, zt, chi, zz, tau);
    // FP32 factors of the signals: approximate divisions and exponentials (a few ulps)
    const float DA = __fdividef(chi, 1.0f + zz);
    const float vr = __fdividef(vxf * xf + vyf * yf + vzf * zf, rh);
    const float geo = __fdividef(a.inv_om_pix, DA * DA);
    const float ekin = __expf(-tau) * vr;
    if (k < 0) {
      B = a.field_B * ekin * geo;
      kind = BP_KIND_FIELD;
    } else if (k < a.nh) {
      // the halo's block: 16 floats, read as four 16-byte loads
      const float4* bq = reinterpret_cast<const float4*>(a.blk) + (int64_t)k * (HB / 4);
      const float4 b0 = __ldg(bq), b1 = __ldg(bq + 1), b2 = __ldg(bq + 2), b3 = __ldg(bq + 3);
      if (b2.z != 0.f) {
        float dx = xf - b3.y, dy = yf - b3.z, dz = zf - b3.w;
        float x = sqrtf(dx * dx + dy * dy + dz * dz) * b0.x;
        if (x < b0.y) {
          float th = a.phi ? 1.0f + (b2.w - a.phi[i]) * b3.x
                           : ((x <= b0.z) ? 1.0f - b1.x * g_inner(x)
                                          : 1.0f - b1.y + __fdividef(b1.z, x));
          th = fmaxf(th, 0.f);
          float thn = powi_or_pow(th, a.n_poly, a.n_int);
          float Rnt = b1.w * __powf(x * b0.w, a.n_nt);
          float vol = x * (1.0f + x) * (1.0f + x);  // rho_s / rho_NFW(r)
          Y = b2.x * thn * th * fmaxf(0.f, 1.0f - Rnt) * vol * geo;
          B = b2.y * thn * vol * ekin * geo * (1.0f / (float)bpc::C_KMS);
          kind = BP_KIND_HALO;
        }
      }
    }
  }
  o0 = make_float4(fx, fy, hp, Y);
  o1 = make_float4(B, __int_as_float(kind), __int_as_float(ix), __int_as_float(iy));
}

// ... and stored: MODE 2 writes only Y, B and the kind into the record MODE 1 wrote.
template <int MODE>
__device__ __forceinline__ void assign_one(const AssignArgs& a, const BpTables& T, int64_t i,
                                           float xf, float yf, float zf, float vxf, float vyf,
                                           float vzf, float hsf, int32_t k) {
  float4 o0, o1;
  assign_rec<MODE>(a, T, T.zt4, i, xf, yf, zf, vxf, vyf, vzf, hsf, k, o0, o1);
  if constexpr (MODE == 2) {
    float* o = a.out + i * BP_ASSIGNED_STRIDE;
    o[3] = o0.w;
    *reinterpret_cast<float2*>(o + 4) = make_float2(o1.x, o1.y);
  } else {
    float4* o = reinterpret_cast<float4*>(a.out + i * BP_ASSIGNED_STRIDE);
    o[0] = o0;
    o[1] = o1;
  }
}

// one particle per thread (any alignment of the SoA arrays)
template <int MODE>
__global__ void __launch_bounds__(256) k_assign(AssignArgs a, BpTables T) {
  int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= a.n) return;
  assign_one<MODE>(a, T, i, a.x[i], a.y[i], a.z[i], a.vx[i], a.vy[i], a.vz[i], a.hs[i],
                   a.hid[i]);
}

// four consecutive particles per thread, the SoA fields read with 16-byte loads (every array
// 16-byte aligned); the last n % 4 particles are left to k_assign.  The whole records (MODE 0)
// go out through shared memory: a warp's 128 records (4 KB, contiguous in the output) are
// written by 16-byte stores of 32 consecutive slots each, instead of each lane storing its own
// 128 bytes at a 128-byte stride (32 cache lines per store instruction).
constexpr int ASSIGN_THREADS = 256;
template <int MODE>
__global__ void __launch_bounds__(ASSIGN_THREADS) k_assign4(AssignArgs a, BpTables T) {
  // per warp: the lanes' 8 record halves each, padded to 9 slots (conflict-free both ways)
  __shared__ float4 stage[MODE == 0 ? ASSIGN_THREADS / 32 : 1][32 * 9];
  // the z(chi), tau(chi) table (dynamic shared memory, T.nc nodes; not for MODE 1)
  extern __shared__ float4 s_zt[];
  if constexpr (MODE != 1) {
    for (int j = threadIdx.x; j < T.nc; j += ASSIGN_THREADS) s_zt[j] = T.zt4[j];
    __syncthreads();
  }
  const float4* zt = MODE != 1 ? s_zt : T.zt4;
  const int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const int lane = threadIdx.x & 31, wp = threadIdx.x >> 5;
  const bool valid = 4 * q + 3 < a.n;
  if (MODE != 0 && !valid) return;
  if (MODE == 0 && (4 * (q - lane) + 3 >= a.n)) return;  // the whole warp past the end
  const int64_t i = 4 * q;
  float4* st = stage[MODE == 0 ? wp : 0] + lane * 9;  // this lane's 8 record halves
  if (valid) {
    const float4 x = __ldg(reinterpret_cast<const float4*>(a.x) + q);
    const float4 y = __ldg(reinterpret_cast<const float4*>(a.y) + q);
    const float4 z = __ldg(reinterpret_cast<const float4*>(a.z) + q);
    const float4 h = __ldg(reinterpret_cast<const float4*>(a.hs) + q);
    const int4 k = __ldg(reinterpret_cast<const int4*>(a.hid) + q);
    float4 vx = make_float4(0.f, 0.f, 0.f, 0.f), vy = vx, vz = vx;
    if constexpr (MODE != 1) {
      vx = __ldg(reinterpret_cast<const float4*>(a.vx) + q);
      vy = __ldg(reinterpret_cast<const float4*>(a.vy) + q);
      vz = __ldg(reinterpret_cast<const float4*>(a.vz) + q);
    }
    auto one = [&](int m, float xf, float yf, float zf, float vxf, float vyf, float vzf,
                   float hf, int32_t kf) {
      float4 o0, o1;
      assign_rec<MODE>(a, T, zt, i + m, xf, yf, zf, vxf, vyf, vzf, hf, kf, o0, o1);
      if constexpr (MODE == 0) {
        st[2 * m] = o0;
        st[2 * m + 1] = o1;
      } else if constexpr (MODE == 2) {
        float* o = a.out + (i + m) * BP_ASSIGNED_STRIDE;
        o[3] = o0.w;
        *reinterpret_cast<float2*>(o + 4) = make_float2(o1.x, o1.y);
      } else {
        float4* o = reinterpret_cast<float4*>(a.out + (i + m) * BP_ASSIGNED_STRIDE);
        o[0] = o0;
        o[1] = o1;
      }
    };
    one(0, x.x, y.x, z.x, vx.x, vy.x, vz.x, h.x, k.x);
    one(1, x.y, y.y, z.y, vx.y, vy.y, vz.y, h.y, k.y);
    one(2, x.z, y.z, z.z, vx.z, vy.z, vz.z, h.z, k.z);
    one(3, x.w, y.w, z.w, vx.w, vy.w, vz.w, h.w, k.w);
  }
  if constexpr (MODE == 0) {
    __syncwarp();
    // record half e of the warp (e = 8 lane' + 2 m + half: lane' 's particle m) is at slot
    // 9 (e / 8) + e % 8; the warp's output starts at particle 4 (q - lane)
    const int64_t first = 4 * (q - lane);
    const int64_t n_here = min((int64_t)128, (a.n / 4) * 4 - first);  // particles of the warp
    float4* out = reinterpret_cast<float4*>(a.out + first * BP_ASSIGNED_STRIDE);
    const float4* ws = stage[wp];
#pragma unroll
    for (int p = 0; p < 8; ++p) {
      const int e = 32 * p + lane;
      if (e / 2 < n_here) out[e] = ws[9 * (e >> 3) + (e & 7)];
    }
  }
}

// ---------------------------------------------------------------- pairs
// Bits of a pair key below the tile when the small-particle deposit is on: the key is
// 2^SMALL_KS tile + the particle's size class.
constexpr int SMALL_KS = 3;
// The tiles a particle's clipped pixel box touches, and its size class: 0 when the box is
// wider than `sspan` pixels on an axis (or sspan is 0), else 1 for a box at most 2 pixels on
// both axes and span - 1 for a largest side of span = 3 .. 8 pixels (the small-particle deposit
// takes them grouped by size, so that a warp's particles have similar boxes).
__device__ __forceinline__ bool particle_tiles(const float4 r0, const float4 r1, int nx, int ny,
                                               int ts, int select, int& tx0, int& tx1, int& ty0,
                                               int& ty1, int sspan, int& cls) {
  int kind = __float_as_int(r1.y);
  if (kind == BP_KIND_NONE) return false;
  if (select == BP_SELECT_HALO && kind != BP_KIND_HALO) return false;
  if (select == BP_SELECT_FIELD && kind != BP_KIND_FIELD) return false;
  int i0, i1, j0, j1;
  if (!bp_span(__float_as_int(r1.z), r0.x, r0.z, nx, i0, i1)) return false;
  if (!bp_span(__float_as_int(r1.w), r0.y, r0.z, ny, j0, j1)) return false;
  const int span = max(i1 - i0, j1 - j0) + 1;
  cls = span > sspan ? 0 : (span <= 2 ? 1 : span - 1);  // 1 .. 7 (SMALL_KS = 3 bits)
  tx0 = i0 / ts;
  tx1 = i1 / ts;
  ty0 = j0 / ts;
  ty1 = j1 / ts;
  return true;
}

__global__ void k_pair_count(const float4* __restrict__ rec, int64_t n, int nx, int ny, int ts,
                             int select, uint32_t* counts) {
  int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  int tx0, tx1, ty0, ty1, cls;
  uint32_t c = 0;
  if (particle_tiles(rec[2 * i], rec[2 * i + 1], nx, ny, ts, select, tx0, tx1, ty0, ty1, 0,
                     cls))
    c = (uint32_t)((tx1 - tx0 + 1) * (ty1 - ty0 + 1));
  counts[i] = c;
}

// The warp's particles own one contiguous range of pairs (offs is their exclusive scan):
// lanes write it 32 consecutive pairs at a time, each finding its particle by a binary
// search over the warp's 32 offsets (shuffles), so that every store is coalesced.  With
// sspan > 0 the key is 2^SMALL_KS tile + the particle's size class (particle_tiles: 0 for the
// tensor-core deposit, 1-7 for the small-particle deposit); with sspan = 0 it is the tile.
__global__ void k_pair_emit(const float4* __restrict__ rec, int64_t n, int nx, int ny, int ts,
                            int select, int ntx, const int64_t* __restrict__ offs,
                            uint32_t* keys, uint32_t* vals, int sspan, int* dbg) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const int lane = threadIdx.x & 31;
  const int64_t i0 = i - lane;
  if (i0 >= n) return;  // the whole warp
  int tx0 = 0, ty0 = 0, w = 1, cnt = 0, cls = 0;
  if (i < n) {
    int tx1, ty1, c = 0;
    if (particle_tiles(rec[2 * i], rec[2 * i + 1], nx, ny, ts, select, tx0, tx1, ty0, ty1, sspan,
                       c)) {
      w = tx1 - tx0 + 1;
      cnt = w * (ty1 - ty0 + 1);
      cls = c;
    }
  }
  const int ks = sspan > 0 ? SMALL_KS : 0;
  const int64_t base = offs[i0];
  const int rel = (int)(offs[i < n ? i : n] - base);  // past the end: the total
  const int end = __shfl_sync(0xffffffffu, rel + cnt, 31);
  // what a lane writing one of this particle's pairs needs, in three words: the first tile
  // (x, y), the box width and size class, and 1 / width for the division below
  const uint32_t pxy = (uint32_t)tx0 | ((uint32_t)ty0 << 16);
  const uint32_t pwc = (uint32_t)w | ((uint32_t)cls << 16);
  const float rw = __frcp_rn((float)w);
  for (int e0 = 0; e0 < end; e0 += 32) {  // warp-uniform trip count
    const int e = e0 + lane;
    int p = 0;  // the last particle of the warp whose first pair is <= e
#pragma unroll
    for (int step = 16; step > 0; step >>= 1)
      if (__shfl_sync(0xffffffffu, rel, p + step) <= e) p += step;
    const uint32_t qxy = __shfl_sync(0xffffffffu, pxy, p), qwc = __shfl_sync(0xffffffffu, pwc, p);
    const int prel = __shfl_sync(0xffffffffu, rel, p);
    const float qr = __shfl_sync(0xffffffffu, rw, p);
    if (e < end) {
      // local = row w + col: the quotient from the FP32 reciprocal (exact up to one for
      // local < 2^22), then one correction step
      const int local = e - prel, pw = (int)(qwc & 0xffffu);
      int row = __float2int_rz(__fmul_rn((float)local, qr));
      int col = local - row * pw;
      if (col < 0) {
        --row;
        col += pw;
      } else if (col >= pw) {
        ++row;
        col -= pw;
      }
      const uint32_t tile = (uint32_t)(((int)(qxy >> 16) + row) * ntx + (int)(qxy & 0xffffu) + col);
      if (BP_DCHECK(tile < (uint32_t)(ntx * ((ny + ts - 1) / ts)) && local >= 0 && col >= 0 &&
                        col < pw && base + e < offs[n],
                    dbg, 101)) {
        keys[base + e] = (tile << ks) | (qwc >> 16);
        vals[base + e] = (uint32_t)(i0 + p);
      }
    }
  }
}

// ---------------------------------------------------------------- work units
using Unit = BpUnit;

// units per key, and partial-tile slots (only keys split into several units need them); with
// ks = SMALL_KS only the keys 2^ks tile get units (the others: small particles,
// k_deposit_small)
__global__ void k_unit_count(const int64_t* __restrict__ tstart, int64_t n_tiles, int unit,
                             uint32_t* ucount, uint32_t* scount, int ks = 0) {
  int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= n_tiles) return;
  int64_t len = (t & ((1 << ks) - 1)) ? 0 : tstart[t + 1] - tstart[t];
  uint32_t nu = (uint32_t)((len + unit - 1) / unit);
  ucount[t] = nu;
  if (scount) scount[t] = nu > 1 ? nu : 0u;
}

__global__ void k_unit_emit(const int64_t* __restrict__ tstart, int64_t n_tiles, int unit,
                            const int64_t* __restrict__ uoff, const int64_t* __restrict__ soff,
                            Unit* units, int ks = 0) {
  int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= n_tiles) return;
  if (t & ((1 << ks) - 1)) return;
  int64_t b = tstart[t], e = tstart[t + 1];
  int64_t nu = (e - b + unit - 1) / unit;
  int64_t u0 = uoff[t];
  for (int64_t q = 0; q < nu; ++q) {
    Unit U;
    U.tile = (int)(t >> ks);
    U.slot = (nu > 1 && soff) ? (int)(soff[t] + q) : -1;
    U.begin = b + q * unit;
    U.end = min(e, b + (q + 1) * unit);
    units[u0 + q] = U;
  }
}

// ---------------------------------------------------------------- deposit
constexpr int DEP_THREADS = 256;
constexpr int CH = 32;          // particles per chunk
constexpr int SEG = 16;         // cells per weight segment
constexpr int FOLD_CHUNKS = 4;  // chunks accumulated in plain FP32 between compensated folds

template <int TS>
struct DepSmem {
  float a[CH][TS];    // column weights
  float by[CH][TS];   // Y * row weights
  float bb[CH][TS];   // B * row weights
  float lo_y[TS * TS];
  float lo_b[TS * TS];
  float4 p0[CH];      // fx, fy, hp, Y
  float p1[CH];       // B
  float ih[CH];       // 1 / hp (0 when hp == 0)
  int2 pi[CH];        // ix - x0, iy - y0 (pixel index relative to the tile origin)
  int4 box[CH];       // footprint in tile coordinates i0, i1, j0, j1 (i0 > i1: none)
  uint32_t wmask[CH]; // warps whose pixel band meets the footprint
  int hasy[CH];
  int64_t unit;
};

template <int TS>
__device__ __forceinline__ void fold_acc(float (&acc)[TS / 16][TS / 16],
                                         float (&hi)[TS / 16][TS / 16], float* lo, int r0,
                                         int c0) {
  constexpr int PR = TS / 16;
#pragma unroll
  for (int r = 0; r < PR; ++r)
#pragma unroll
    for (int c = 0; c < PR; ++c) {
      float s, e;
      bp_two_sum(hi[r][c], acc[r][c], s, e);
      hi[r][c] = s;
      lo[(r0 + r) * TS + c0 + c] += e;
      acc[r][c] = 0.f;
    }
}

template <int TS>
__global__ void __launch_bounds__(DEP_THREADS, 2)
    k_deposit(const float4* __restrict__ rec, const uint32_t* __restrict__ pvals,
              const Unit* __restrict__ units, const int64_t* __restrict__ n_units_ptr,
              int64_t* counter, int nx, int ny, int ntx, float* ymap, float* bmap, float* ylo,
              float* blo, float* partials) {
  constexpr int PR = TS / 16;  // pixels per thread along each axis
  constexpr int NSEG = TS / SEG;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  DepSmem<TS>& S = *reinterpret_cast<DepSmem<TS>*>(smem_raw);
  const int tid = threadIdx.x, lane = tid & 31, w = tid >> 5;
  const int lr = lane >> 3, lc = lane & 7;
  const int wr0 = (w >> 1) * 4 * PR, wc0 = (w & 1) * 8 * PR;  // warp band origin
  const int r0 = wr0 + lr * PR, c0 = wc0 + lc * PR;              // thread block origin
  const int64_t n_units = *n_units_ptr;
  for (;;) {
    if (tid == 0) S.unit = atomicAdd((unsigned long long*)counter, 1ull);
    __syncthreads();
    const int64_t u = S.unit;
    if (u >= n_units) break;
    const Unit U = units[u];
    const int tyi = U.tile / ntx, txi = U.tile % ntx;
    const int x0 = txi * TS, y0 = tyi * TS;
    for (int q = tid; q < TS * TS; q += DEP_THREADS) {
      S.lo_y[q] = 0.f;
      S.lo_b[q] = 0.f;
    }
    float acc_y[PR][PR], acc_b[PR][PR], hi_y[PR][PR], hi_b[PR][PR];
#pragma unroll
    for (int r = 0; r < PR; ++r)
#pragma unroll
      for (int c = 0; c < PR; ++c) acc_y[r][c] = acc_b[r][c] = hi_y[r][c] = hi_b[r][c] = 0.f;
    int chunks = 0;
    for (int64_t cb = U.begin; cb < U.end; cb += CH) {
      const int nch = (int)min((int64_t)CH, U.end - cb);
      __syncthreads();  // previous chunk fully consumed
      // 1. gather particle records, footprints and warp masks
      if (tid < nch) {
        uint32_t pi = pvals[cb + tid];
        float4 q0 = rec[2 * (int64_t)pi];
        float4 q1 = rec[2 * (int64_t)pi + 1];
        S.p0[tid] = q0;
        S.p1[tid] = q1.x;
        S.ih[tid] = q0.z > 0.f ? 1.0f / q0.z : 0.f;
        const int ixp = __float_as_int(q1.z), iyp = __float_as_int(q1.w);
        S.pi[tid] = make_int2(ixp - x0, iyp - y0);
        int i0, i1, j0, j1;
        int4 bx = make_int4(1, 0, 1, 0);
        uint32_t m = 0;
        if (bp_span(ixp, q0.x, q0.z, nx, i0, i1) && bp_span(iyp, q0.y, q0.z, ny, j0, j1)) {
          bx.x = max(i0 - x0, 0);
          bx.y = min(i1 - x0, TS - 1);
          bx.z = max(j0 - y0, 0);
          bx.w = min(j1 - y0, TS - 1);
#pragma unroll
          for (int ww = 0; ww < DEP_THREADS / 32; ++ww) {
            int a0 = (ww & 1) * 8 * PR, b0 = (ww >> 1) * 4 * PR;
            bool hit = !(bx.y < a0 || bx.x > a0 + 8 * PR - 1 || bx.w < b0 ||
                         bx.z > b0 + 4 * PR - 1);
            m |= hit ? (1u << ww) : 0u;
          }
        }
        S.box[tid] = bx;
        S.wmask[tid] = m;
        S.hasy[tid] = q0.w != 0.f;
      }
      __syncthreads();
      // 2. weights: one thread per (particle, axis, 16-cell segment)
      for (int q = tid; q < nch * 2 * NSEG; q += DEP_THREADS) {
        const int k = q / (2 * NSEG), axis = (q / NSEG) & 1, sg = q % NSEG;
        const int cb0 = sg * SEG;
        const float4 p = S.p0[k];
        const int4 bx = S.box[k];
        const int lo = axis ? bx.z : bx.x, hi = axis ? bx.w : bx.y;
        float wv[SEG];
        if (hi < cb0 || lo > cb0 + SEG - 1) {
#pragma unroll
          for (int j = 0; j < SEG; ++j) wv[j] = 0.f;
        } else {
          const int2 ip = S.pi[k];
          bp_cell_weights<SEG>(cb0 - (axis ? ip.y : ip.x), axis ? p.y : p.x, p.z, S.ih[k], wv);
        }
        if (axis == 0) {
          float4* dst = reinterpret_cast<float4*>(&S.a[k][cb0]);
#pragma unroll
          for (int j = 0; j < SEG / 4; ++j)
            dst[j] = make_float4(wv[4 * j], wv[4 * j + 1], wv[4 * j + 2], wv[4 * j + 3]);
        } else {
          const float Yk = p.w, Bk = S.p1[k];
          float4* dy = reinterpret_cast<float4*>(&S.by[k][cb0]);
          float4* db = reinterpret_cast<float4*>(&S.bb[k][cb0]);
#pragma unroll
          for (int j = 0; j < SEG / 4; ++j) {
            dy[j] = make_float4(Yk * wv[4 * j], Yk * wv[4 * j + 1], Yk * wv[4 * j + 2],
                                Yk * wv[4 * j + 3]);
            db[j] = make_float4(Bk * wv[4 * j], Bk * wv[4 * j + 1], Bk * wv[4 * j + 2],
                                Bk * wv[4 * j + 3]);
          }
        }
      }
      __syncthreads();
      // 3. rank-1 updates of this thread's PR x PR pixels
      for (int k = 0; k < nch; ++k) {
        if (!((S.wmask[k] >> w) & 1u)) continue;  // warp-uniform skip
        float av[PR], bvb[PR];
#pragma unroll
        for (int c = 0; c < PR; ++c) av[c] = S.a[k][c0 + c];
#pragma unroll
        for (int r = 0; r < PR; ++r) bvb[r] = S.bb[k][r0 + r];
#pragma unroll
        for (int r = 0; r < PR; ++r)
#pragma unroll
          for (int c = 0; c < PR; ++c) acc_b[r][c] = fmaf(bvb[r], av[c], acc_b[r][c]);
        if (S.hasy[k]) {
          float bvy[PR];
#pragma unroll
          for (int r = 0; r < PR; ++r) bvy[r] = S.by[k][r0 + r];
#pragma unroll
          for (int r = 0; r < PR; ++r)
#pragma unroll
            for (int c = 0; c < PR; ++c) acc_y[r][c] = fmaf(bvy[r], av[c], acc_y[r][c]);
        }
      }
      if (++chunks == FOLD_CHUNKS) {
        fold_acc<TS>(acc_y, hi_y, S.lo_y, r0, c0);
        fold_acc<TS>(acc_b, hi_b, S.lo_b, r0, c0);
        chunks = 0;
      }
    }
    fold_acc<TS>(acc_y, hi_y, S.lo_y, r0, c0);
    fold_acc<TS>(acc_b, hi_b, S.lo_b, r0, c0);
    // 4. write the tile: straight into the map, or as a partial tile
    if (U.slot < 0) {
#pragma unroll
      for (int r = 0; r < PR; ++r)
#pragma unroll
        for (int c = 0; c < PR; ++c) {
          int gx = x0 + c0 + c, gy = y0 + r0 + r;
          if (gx >= nx || gy >= ny) continue;
          int64_t p = (int64_t)gy * nx + gx;
          int q = (r0 + r) * TS + c0 + c;
          float s, e;
          bp_two_sum(ymap[p], hi_y[r][c], s, e);
          ymap[p] = s;
          ylo[p] = ylo[p] + (S.lo_y[q] + e);
          bp_two_sum(bmap[p], hi_b[r][c], s, e);
          bmap[p] = s;
          blo[p] = blo[p] + (S.lo_b[q] + e);
        }
    } else {
      float* P = partials + (int64_t)U.slot * 4 * TS * TS;
#pragma unroll
      for (int r = 0; r < PR; ++r)
#pragma unroll
        for (int c = 0; c < PR; ++c) {
          int q = (r0 + r) * TS + c0 + c;
          P[q] = hi_y[r][c];
          P[TS * TS + q] = S.lo_y[q];
          P[2 * TS * TS + q] = hi_b[r][c];
          P[3 * TS * TS + q] = S.lo_b[q];
        }
    }
    __syncthreads();
  }
}

// REDUCE_SPLIT CTAs per multi-unit tile (pixel slices): add its partial tiles in unit
// order, then the map
constexpr int REDUCE_SPLIT = 4;
template <int TS>
__global__ void __launch_bounds__(256) k_reduce_tiles(const int64_t* __restrict__ tstart,
                                                      const int64_t* __restrict__ soff,
                                                      int64_t n_tiles, int unit, int nx, int ny,
                                                      int ntx, const float* __restrict__ partials,
                                                      float* ymap, float* bmap, float* ylo,
                                                      float* blo, const int* __restrict__ err,
                                                      int ks, int* dbg) {
  // blockIdx.y: which of REDUCE_SPLIT pixel slices of the tile this CTA sums
  int64_t t = blockIdx.x;
  if (t >= n_tiles) return;
  if (err && *err) return;  // the deposit gave up: its partial tiles are incomplete
  const int64_t key = t << ks;  // the tile's (large-particle) key
  int64_t len = tstart[key + 1] - tstart[key];
  int64_t nu = (len + unit - 1) / unit;
  if (nu <= 1) return;
  int64_t u0 = soff[key];
  int x0 = (int)(t % ntx) * TS, y0 = (int)(t / ntx) * TS;
  constexpr int SLICE = TS * TS / REDUCE_SPLIT;
  const int q_end = (blockIdx.y + 1) * SLICE;
  for (int q = blockIdx.y * SLICE + threadIdx.x; q < q_end; q += blockDim.x) {
    int gx = x0 + q % TS, gy = y0 + q / TS;
    if (gx >= nx || gy >= ny) continue;
    float hy = 0.f, ly = 0.f, hb = 0.f, lb = 0.f;
    if (!BP_DCHECK(u0 >= 0 && q >= 0 && q < TS * TS, dbg, 501)) continue;
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
    int64_t p = (int64_t)gy * nx + gx;
    float s, e;
    bp_two_sum(ymap[p], hy, s, e);
    ymap[p] = s;
    ylo[p] = ylo[p] + (ly + e);
    bp_two_sum(bmap[p], hb, s, e);
    bmap[p] = s;
    blo[p] = blo[p] + (lb + e);
  }
}

// ---------------------------------------------------------------- small particles
// Particles whose clipped pixel box is at most sspan (<= SMALL_MAX = 8) pixels on both axes
// (most halo particles of a large light-cone cover a few pixels) are deposited here instead
// of as dense 64 x 64 tensor-core updates.  One CTA per tile, one thread per particle (sorted by size
// class, then index, so that a warp's particles have similar boxes and its lanes similar
// trip counts): the thread computes its particle's cell weights from the edge values of
// bp_edge_split (those of the tensor-core deposit) and adds Y wx wy and B wx wy of every
// covered cell to the tile's accumulators as 64-bit fixed-point integers, with shared-memory
// atomics.  Integer sums do not depend on the order of the additions: the result is
// deterministic.  Each map's scale 2^S follows the tile's largest |Y| (|B|) and its particle
// count n, so that no cell sum can overflow (a cell's sum is at most n max|Y|) and the
// quantum is 2^-61 n max|Y|: far below the FP32 rounding of the products.  The records are
// read once: the largest value so far sets the scale, and a larger one later shifts the
// sums so far down to the new scale.
constexpr int SMALL_MAX = 8;
constexpr int SMALL_THREADS = 512;
struct SmallSmem {
  // y, b of the 64 x 64 tile as 64-bit two's-complement integers, kept as low and high
  // 32-bit words (lo[m][q], hi[m][q])
  uint32_t lo[2][64 * 64];
  uint32_t hi[2][64 * 64];
  float wx[SMALL_THREADS][SMALL_MAX + 1];  // each thread's column weights (padded rows)
  float amax[2][SMALL_THREADS / 32];
};

// v (|v| < 2^62) as an integer, truncated toward zero, with integer instructions (the
// conversion instruction to 64-bit integers measured slower here)
__device__ __forceinline__ long long small_fix(float v) {
  const int b = __float_as_int(v);
  const int e = ((b >> 23) & 0xff) - 150;  // v = m 2^e with the 24-bit significand m
  const long long m = (long long)((b & 0x7fffff) | 0x800000);
  const long long q = e >= 0 ? (m << e) : (e > -24 ? (m >> (-e)) : 0ll);
  return b < 0 ? -q : q;
}

// acc += v exactly, modulo 2^64, with two 32-bit shared-memory atomics (the pair measured
// about three times the update rate of one 64-bit shared-memory atomic on this GPU): the
// low word's previous value tells whether its sum carried into the high word.  The result does not depend on the order of
// the additions.
__device__ __forceinline__ void small_add(uint32_t* lo, uint32_t* hi, long long v) {
  const uint32_t l = (uint32_t)v, h = (uint32_t)((unsigned long long)v >> 32);
  const uint32_t old = atomicAdd(lo, l);
  atomicAdd(hi, h + (old + l < old ? 1u : 0u));
}

// exponent S with n * amax * 2^S < 2^61 (0 when amax is 0)
__device__ __forceinline__ int small_scale(float amax, int64_t n) {
  if (!(amax > 0.f)) return 0;
  int ex;
  frexp((double)amax * (double)n, &ex);
  return 61 - ex;
}

__global__ void __launch_bounds__(SMALL_THREADS) k_deposit_small(
    const float4* __restrict__ rec, const uint32_t* __restrict__ pvals,
    const int64_t* __restrict__ tstart, int ntx, int nx, int ny, float* ymap, float* bmap,
    float* ylo, float* blo, const int* __restrict__ err, int* dbg) {
  extern __shared__ __align__(16) unsigned char small_raw[];
  SmallSmem& S = *reinterpret_cast<SmallSmem*>(small_raw);
  const int t = blockIdx.x, tid = threadIdx.x, lane = tid & 31, wp = tid >> 5;
  if (err && *err) return;  // the tensor-core deposit before it gave up
  // classes 1 .. 7 of the tile: keys 8 t + 1 .. 8 t + 7
  const int64_t b = tstart[((int64_t)t << SMALL_KS) + 1], e = tstart[((int64_t)(t + 1) << SMALL_KS)];
  if (b >= e) return;
  const int x0 = (t % ntx) * 64, y0 = (t / ntx) * 64;
  for (int q = tid; q < 2 * 64 * 64; q += SMALL_THREADS) {
    (&S.lo[0][0])[q] = 0u;
    (&S.hi[0][0])[q] = 0u;
  }
  // One pass over the tile's particles, SMALL_THREADS at a time (one per thread, its record
  // held in registers).  Each map's scale 2^S follows the largest |Y| (|B|) seen so far: it is
  // set by the first block with a nonzero value and only lowered afterwards, the sums so far
  // shifted right by the difference (floor: below one quantum per shift).  The order of the
  // blocks is the sorted order, so the result is still deterministic.
  const int64_t n = e - b;
  float run_y = 0.f, run_b = 0.f;  // largest |Y|, |B| so far (the same in every thread)
  int sy = 0, sb = 0;
  float* wx = S.wx[tid];
  for (int64_t k0 = b; k0 < e; k0 += SMALL_THREADS) {
    const int64_t k = k0 + tid;
    const bool valid = k < e;
    float4 r0 = make_float4(0.f, 0.f, 0.f, 0.f), r1 = r0;
    if (valid) {
      const int64_t pv = pvals[k];
      r0 = rec[2 * pv];
      r1 = rec[2 * pv + 1];
    }
    float my = fabsf(r0.w), mb = fabsf(r1.x);
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      my = fmaxf(my, __shfl_xor_sync(0xffffffffu, my, o));
      mb = fmaxf(mb, __shfl_xor_sync(0xffffffffu, mb, o));
    }
    if (lane == 0) {
      S.amax[0][wp] = my;
      S.amax[1][wp] = mb;
    }
    __syncthreads();
#pragma unroll
    for (int q = 0; q < SMALL_THREADS / 32; ++q) {
      my = fmaxf(my, S.amax[0][q]);
      mb = fmaxf(mb, S.amax[1][q]);
    }
    // new scales; a lowered scale shifts the sums so far (uniform across the CTA)
    int dy = 0, db = 0;
    if (my > run_y) {
      const int t2 = small_scale(my, n);
      if (run_y > 0.f) dy = sy - t2;
      sy = t2;
      run_y = my;
    }
    if (mb > run_b) {
      const int t2 = small_scale(mb, n);
      if (run_b > 0.f) db = sb - t2;
      sb = t2;
      run_b = mb;
    }
    if (dy > 0 || db > 0) {
      for (int q = tid; q < 2 * 64 * 64; q += SMALL_THREADS) {
        const int m = q >> 12, d = m ? db : dy;
        if (d <= 0) continue;
        uint32_t* lo = &S.lo[0][0] + q;
        uint32_t* hi = &S.hi[0][0] + q;
        const long long a = (long long)(((unsigned long long)*hi << 32) | *lo) >> min(d, 63);
        *lo = (uint32_t)a;
        *hi = (uint32_t)((unsigned long long)a >> 32);
      }
    }
    __syncthreads();
    // every cell of this thread's particle, as fixed-point integers
    const int ix = __float_as_int(r1.z), iy = __float_as_int(r1.w);
    int i0 = 0, i1 = -1, j0 = 0, j1 = -1;
    if (valid && bp_span(ix, r0.x, r0.z, nx, i0, i1) && bp_span(iy, r0.y, r0.z, ny, j0, j1)) {
      i0 = max(i0, x0);
      i1 = min(i1, x0 + 63);
      j0 = max(j0, y0);
      j1 = min(j1, y0 + 63);
    } else {
      i1 = i0 - 1;
    }
    if (i0 <= i1 && j0 <= j1) {
      const bool ngp = !(r0.z > 0.f);
      const float ih = ngp ? 1.0e38f : __frcp_rn(r0.z);
      const float k1 = BP_KT * ih, k2 = BP_KS * ih;
      const float fx = (ngp && !(r0.x > 0.f)) ? 1.0e-30f : r0.x;
      const float fy = (ngp && !(r0.y > 0.f)) ? 1.0e-30f : r0.y;
      const int kcx = ix + (fx > 0.f ? 0 : -1), kcy = iy + (fy > 0.f ? 0 : -1);
      float v = bp_edge_split(__fsub_rn((float)(i0 - ix), fx), k1, k2);
      for (int i = i0; i <= i1; ++i) {
        const float vn = bp_edge_split(__fsub_rn((float)(i + 1 - ix), fx), k1, k2);
        if (BP_DCHECK(i - i0 <= SMALL_MAX, dbg, 302)) wx[i - i0] = (vn - v) + (i == kcx ? 1.f : 0.f);
        v = vn;
      }
      const float Ys = ldexpf(r0.w, sy), Bs = ldexpf(r1.x, sb);
      const bool has_y = r0.w != 0.f;
      float u = bp_edge_split(__fsub_rn((float)(j0 - iy), fy), k1, k2);
      for (int j = j0; j <= j1; ++j) {
        const float un = bp_edge_split(__fsub_rn((float)(j + 1 - iy), fy), k1, k2);
        const float wy = (un - u) + (j == kcy ? 1.f : 0.f);
        u = un;
        const float ay = Ys * wy, ab = Bs * wy;
        const int q0 = (j - y0) * 64 + (i0 - x0);
        for (int c = 0; c <= i1 - i0; ++c) {
          const float w = wx[c];
          if (!BP_DCHECK(q0 + c >= 0 && q0 + c < 64 * 64 && c <= SMALL_MAX, dbg, 301)) continue;
          if (has_y) small_add(&S.lo[0][q0 + c], &S.hi[0][q0 + c], small_fix(ay * w));
          small_add(&S.lo[1][q0 + c], &S.hi[1][q0 + c], small_fix(ab * w));
        }
      }
    }
  }
  __syncthreads();
  // 3. the tile's sums into the map (compensated)
  for (int q = tid; q < 64 * 64; q += SMALL_THREADS) {
    const int gx = x0 + (q & 63), gy = y0 + (q >> 6);
    if (gx >= nx || gy >= ny) continue;
    const int64_t p = (int64_t)gy * nx + gx;
#pragma unroll
    for (int m = 0; m < 2; ++m) {
      const long long a = (long long)(((unsigned long long)S.hi[m][q] << 32) | S.lo[m][q]);
      if (a == 0) continue;
      const double vv = ldexp((double)a, -(m ? sb : sy));
      const float hi = (float)vv, lo = (float)(vv - (double)hi);
      float* map = m ? bmap : ymap;
      float* mlo = m ? blo : ylo;
      float sm, er;
      bp_two_sum(map[p], hi, sm, er);
      map[p] = sm;
      mlo[p] = mlo[p] + (lo + er);
    }
  }
}

int check_geom(bp_ctx* ctx, const bp_map_geom* g, const char* who) {
  if (!g) return bp_fail(ctx, BP_EINVAL, "%s: null geometry", who);
  if (g->nx <= 0 || g->ny <= 0 || g->n_maps <= 0 || !(g->dtheta > 0))
    return bp_fail(ctx, BP_EINVAL, "%s: bad geometry", who);
  if (g->nx > 65536 || g->ny > 65536)
    return bp_fail(ctx, BP_ERANGE, "%s: map side above 65536 pixels", who);
  return BP_OK;
}

// Builds the sorted (tile, particle) list; returns keys/vals pointers and count.  sspan > 0:
// keys 2^SMALL_KS tile + the particle's size class (see k_pair_emit).
int build_pairs(bp_ctx* ctx, int64_t n, const float* assigned, const bp_map_geom* g, int select,
                int ts, uint32_t** keys_out, uint32_t** vals_out, int64_t* npairs_out,
                int64_t* n_tiles_out, int sspan = 0) {
  const int ntx = (g->nx + ts - 1) / ts, nty = (g->ny + ts - 1) / ts;
  const int64_t n_tiles = (int64_t)ntx * nty;
  uint32_t* counts;
  int64_t* offs;
  int r;
  if ((r = bp_ws(ctx, WS_COUNTS, (size_t)(n + 1) * 4, (void**)&counts))) return r;
  if ((r = bp_ws(ctx, WS_OFFS, (size_t)(n + 1) * 8, (void**)&offs))) return r;
  const float4* rec = reinterpret_cast<const float4*>(assigned);
  unsigned nb = (unsigned)((n + 255) / 256);
  bp_phase_begin(ctx, BP_PH_PAIRS);
  k_pair_count<<<nb, 256, 0, ctx->stream>>>(rec, n, g->nx, g->ny, ts, select, counts);
  BP_LAUNCH_CHECK(ctx, "pair count");
  if ((r = bp_scan_u32_to_i64(ctx, counts, offs, n))) return r;
  BP_CUDA(ctx, cudaMemcpyAsync(ctx->h_pinned, offs + n, 8, cudaMemcpyDeviceToHost, ctx->stream));
  BP_CUDA(ctx, cudaStreamSynchronize(ctx->stream));
  const int64_t np = ctx->h_pinned[0];
  if (np > (int64_t)UINT32_MAX)
    return bp_fail(ctx, BP_ERANGE, "paste: %lld tile pairs exceed 2^32", (long long)np);
  uint32_t *k0, *v0, *k1, *v1;
  if ((r = bp_ws(ctx, WS_KEYS0, (size_t)np * 4, (void**)&k0))) return r;
  if ((r = bp_ws(ctx, WS_VALS0, (size_t)np * 4, (void**)&v0))) return r;
  if ((r = bp_ws(ctx, WS_KEYS1, (size_t)np * 4, (void**)&k1))) return r;
  if ((r = bp_ws(ctx, WS_VALS1, (size_t)np * 4, (void**)&v1))) return r;
  k_pair_emit<<<nb, 256, 0, ctx->stream>>>(rec, n, g->nx, g->ny, ts, select, ntx, offs, k0, v0,
                                           sspan, bp_dbg_word(ctx));
  BP_LAUNCH_CHECK(ctx, "pair emit");
  bp_phase_end(ctx, BP_PH_PAIRS);
  int key_bits = 0;
  while (((int64_t)1 << key_bits) < (n_tiles << (sspan > 0 ? SMALL_KS : 0))) ++key_bits;
  bp_phase_begin(ctx, BP_PH_SORT);
  if ((r = bp_radix_sort_pairs(ctx, k0, v0, k1, v1, np, key_bits, keys_out, vals_out))) return r;
  *npairs_out = np;
  *n_tiles_out = n_tiles;
  return BP_OK;
}

// the SIMT deposit kernel over the work units (persistent, resident-capacity grid)
template <int TS>
int deposit_simt(bp_ctx* ctx, const float* assigned, const bp_map_geom* g, const uint32_t* vals,
                 const Unit* units, const int64_t* n_units_dev, int64_t* counter,
                 int64_t max_units, float* ymap, float* bmap, float* ylo, float* blo,
                 float* partials) {
  const int ntx = (g->nx + TS - 1) / TS;
  const size_t smem = sizeof(DepSmem<TS>);
  BP_CUDA(ctx, cudaFuncSetAttribute(k_deposit<TS>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                    (int)smem));
  int per_sm = 0;
  BP_CUDA(ctx, cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_deposit<TS>, DEP_THREADS,
                                                             smem));
  if (per_sm < 1) per_sm = 1;
  int64_t grid = (int64_t)ctx->num_sms * per_sm;
  if (grid > max_units) grid = max_units;
  bp_phase_begin(ctx, BP_PH_DEPOSIT);
  k_deposit<TS><<<(unsigned)grid, DEP_THREADS, smem, ctx->stream>>>(
      reinterpret_cast<const float4*>(assigned), vals, units, n_units_dev, counter, g->nx, g->ny,
      ntx, ymap, bmap, ylo, blo, partials);
  BP_LAUNCH_CHECK(ctx, "deposit");
  bp_phase_end(ctx, BP_PH_DEPOSIT);
  return BP_OK;
}

// Work units of a sorted pair list (tile ranges, units, partial-tile slots), recorded in P
// with the generations of the scratch slots they live in.  Synchronises once.
template <int TS>
int prepare_units(bp_ctx* ctx, const uint32_t* keys, const uint32_t* vals, int64_t np,
                  int64_t n_tiles, PpPrepared* P, int ks = 0) {
  int r;
  const int64_t n_keys = n_tiles << ks;  // ks = SMALL_KS: 8 keys per tile (size classes)
  // particles per work unit: the context's value, or (auto) about 16 units per
  // resident CTA, at least 2048
  int64_t unit64 = ctx->pp_unit;
  if (unit64 <= 0) {
    unit64 = np / ((int64_t)ctx->num_sms * 2 * 16);
    if (unit64 < 2048) unit64 = 2048;
    if (unit64 > (1 << 30)) unit64 = 1 << 30;
  }
  const int unit = (int)unit64;
  int64_t* tstart;
  if ((r = bp_ws(ctx, WS_TILES, (size_t)(n_keys + 1) * 8 * 3 + (size_t)(n_keys + 1) * 8 + 64,
                 (void**)&tstart)))
    return r;
  int64_t* uoff = tstart + (n_keys + 1);
  int64_t* soff = uoff + (n_keys + 1);
  uint32_t* ucount = (uint32_t*)(soff + (n_keys + 1));
  uint32_t* scount = ucount + (n_keys + 1);
  if ((r = bp_tile_ranges(ctx, keys, np, n_keys, tstart))) return r;
  unsigned tb = (unsigned)((n_keys + 255) / 256);
  k_unit_count<<<tb, 256, 0, ctx->stream>>>(tstart, n_keys, unit, ucount, scount, ks);
  BP_LAUNCH_CHECK(ctx, "unit count");
  if ((r = bp_scan_u32_to_i64(ctx, ucount, uoff, n_keys))) return r;
  if ((r = bp_scan_u32_to_i64(ctx, scount, soff, n_keys))) return r;
  const int64_t max_units = n_keys + np / unit + 1;
  Unit* units;
  if ((r = bp_ws(ctx, WS_UNITS, (size_t)max_units * sizeof(Unit), (void**)&units))) return r;
  k_unit_emit<<<tb, 256, 0, ctx->stream>>>(tstart, n_keys, unit, uoff, soff, units, ks);
  BP_LAUNCH_CHECK(ctx, "unit emit");
  // partial tiles exist only for tiles split into several units
  BP_CUDA(ctx, cudaMemcpyAsync(ctx->h_pinned + 1, soff + n_keys, 8, cudaMemcpyDeviceToHost,
                               ctx->stream));
  BP_CUDA(ctx, cudaStreamSynchronize(ctx->stream));
  P->ts = TS;
  P->unit = unit;
  P->np = np;
  P->n_tiles = n_tiles;
  P->n_keys = n_keys;
  P->ks = ks;
  P->max_units = max_units;
  P->n_slots = ctx->h_pinned[1];
  P->vals = vals;
  P->tstart = tstart;
  P->uoff = uoff;
  P->soff = soff;
  P->units = units;
  for (int k = 0; k < WS_NSLOTS; ++k) P->gen[k] = ctx->ws_gen[k];
  return BP_OK;
}

// The deposit and the fixed-order reduction of a prepared list.
template <int TS>
int launch_deposit(bp_ctx* ctx, const float* assigned, const bp_map_geom* g,
                   const PpPrepared& P, float* ymap, float* bmap, float* ylo, float* blo) {
  int r;
  const int ntx = (g->nx + TS - 1) / TS;
  float* partials;
  if ((r = bp_ws(ctx, WS_PART,
                 (size_t)(P.n_slots > 0 ? P.n_slots : 1) * 4 * TS * TS * sizeof(float),
                 (void**)&partials)))
    return r;
  const Unit* units = (const Unit*)P.units;
  BP_CUDA(ctx, cudaMemsetAsync(ctx->d_counter + 1, 0, sizeof(int64_t), ctx->stream));
  const bool tc = bp_deposit_uses_tc(ctx, TS);
  if (tc) {
    bp_phase_begin(ctx, BP_PH_DEPOSIT);
    if ((r = bp_deposit_tc_launch(ctx, assigned, P.vals, units, P.uoff + P.n_keys,
                                  ctx->d_counter + 1, P.max_units, g, ymap, bmap, ylo, blo,
                                  partials)))
      return r;
    bp_phase_end(ctx, BP_PH_DEPOSIT);
  } else {
    if ((r = deposit_simt<TS>(ctx, assigned, g, P.vals, units, P.uoff + P.n_keys,
                              ctx->d_counter + 1, P.max_units, ymap, bmap, ylo, blo, partials)))
      return r;
  }
  bp_phase_begin(ctx, BP_PH_REDUCE);
  if (P.n_slots > 0) {
    k_reduce_tiles<TS><<<dim3((unsigned)P.n_tiles, REDUCE_SPLIT), 256, 0, ctx->stream>>>(
        P.tstart, P.soff, P.n_tiles, P.unit, g->nx, g->ny, ntx, partials, ymap, bmap, ylo, blo,
        tc ? ctx->d_flags : nullptr, P.ks, bp_dbg_word(ctx));
    BP_LAUNCH_CHECK(ctx, "reduce tiles");
  }
  bp_phase_end(ctx, BP_PH_REDUCE);
  if (P.ks) {  // the small particles, after the large ones of every tile
    bp_phase_begin(ctx, BP_PH_DEPOSIT_SMALL);
    const size_t smem = sizeof(SmallSmem);
    BP_CUDA(ctx, cudaFuncSetAttribute(k_deposit_small, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                      (int)smem));
    k_deposit_small<<<(unsigned)P.n_tiles, SMALL_THREADS, smem, ctx->stream>>>(
        reinterpret_cast<const float4*>(assigned), P.vals, P.tstart, ntx, g->nx, g->ny, ymap, bmap,
        ylo, blo, tc ? ctx->d_flags : nullptr, bp_dbg_word(ctx));
    BP_LAUNCH_CHECK(ctx, "deposit (small particles)");
    bp_phase_end(ctx, BP_PH_DEPOSIT_SMALL);
  }
  if (tc) return bp_deposit_tc_check(ctx);
  return BP_OK;
}

template <int TS>
int deposit(bp_ctx* ctx, const float* assigned, const bp_map_geom* g, const uint32_t* keys,
            const uint32_t* vals, int64_t np, int64_t n_tiles, float* ymap, float* bmap,
            float* ylo, float* blo, int ks) {
  PpPrepared P;
  int r = prepare_units<TS>(ctx, keys, vals, np, n_tiles, &P, ks);
  if (r) return r;
  bp_phase_end(ctx, BP_PH_SORT);
  return launch_deposit<TS>(ctx, assigned, g, P, ymap, bmap, ylo, blo);
}

int halo_blocks(bp_ctx* ctx, int64_t nh, const double* model, const int32_t* status, double Mp,
                const float* hpos, float** blk) {
  int r = bp_ws(ctx, WS_HPAR, (size_t)(nh > 0 ? nh : 1) * HB * sizeof(float), (void**)blk);
  if (r) return r;
  if (nh > 0) {
    const int hb = bp_item_block(ctx, nh, 256);
    k_halo_block<<<(unsigned)((nh + hb - 1) / hb), hb, 0, ctx->stream>>>(ctx->p, nh, model,
                                                                        status, Mp, hpos,
                                                                        *blk);
    BP_LAUNCH_CHECK(ctx, "halo block");
  }
  return BP_OK;
}

template <int TS>
int deposit_buffers(bp_ctx* ctx, const float* assigned, const bp_map_geom* g,
                    const uint32_t* keys, const uint32_t* vals, int64_t np, int64_t n_tiles,
                    float* ymap, float* bmap, float* ylo, float* blo, const BpPasteBuffers* B) {
  // one work unit per tile: every tile is written straight into the map
  const int unit = 0x7fffffff;
  int r;
  if ((r = bp_tile_ranges(ctx, keys, np, n_tiles, B->tstart))) return r;
  unsigned tb = (unsigned)((n_tiles + 255) / 256);
  k_unit_count<<<tb, 256, 0, ctx->stream>>>(B->tstart, n_tiles, unit, B->ucount, nullptr);
  BP_LAUNCH_CHECK(ctx, "unit count");
  if ((r = bp_scan_u32_to_i64_buf(ctx, B->ucount, B->uoff, n_tiles, B->bsum))) return r;
  Unit* units = (Unit*)B->units;
  k_unit_emit<<<tb, 256, 0, ctx->stream>>>(B->tstart, n_tiles, unit, B->uoff, nullptr, units);
  BP_LAUNCH_CHECK(ctx, "unit emit");
  BP_CUDA(ctx, cudaMemsetAsync(B->counter, 0, sizeof(int64_t), ctx->stream));
  if (bp_deposit_uses_tc(ctx, TS)) {
    if ((r = bp_deposit_tc_launch(ctx, assigned, vals, units, B->uoff + n_tiles, B->counter,
                                  n_tiles, g, ymap, bmap, ylo, blo, nullptr)))
      return r;
    return bp_deposit_tc_check(ctx);
  }
  return deposit_simt<TS>(ctx, assigned, g, vals, units, B->uoff + n_tiles, B->counter, n_tiles,
                          ymap, bmap, ylo, blo, nullptr);
}

}  // namespace

size_t bp_pp_unit_bytes() { return sizeof(Unit); }

// Loads the kernels that bp_pp_paste_buffers launches from this file (CUDA loads modules
// lazily: a kernel's first launch would otherwise load its code into device memory).
int bp_pp_preload(bp_ctx* ctx) {
  cudaFuncAttributes a;
  BP_CUDA(ctx, cudaFuncGetAttributes(&a, k_pair_count));
  BP_CUDA(ctx, cudaFuncGetAttributes(&a, k_pair_emit));
  BP_CUDA(ctx, cudaFuncGetAttributes(&a, k_unit_count));
  BP_CUDA(ctx, cudaFuncGetAttributes(&a, k_unit_emit));
  BP_CUDA(ctx, cudaFuncGetAttributes(&a, k_deposit<32>));
  BP_CUDA(ctx, cudaFuncGetAttributes(&a, k_deposit<64>));
  BP_CUDA(ctx, cudaFuncGetAttributes(&a, k_deposit_small));
  return BP_OK;
}

bool bp_deposit_uses_tc(const bp_ctx* ctx, int ts) {
  if (ctx->pp_kernel == BP_DEPOSIT_SIMT) return false;
  return ts == 64;
}

// The small-particle span of a paste: with the tensor-core deposit (tile 64), the context's
// threshold, or automatically 8 when the map has at least 4 tiles per SM (the small-particle
// kernel runs one CTA per tile: with fewer tiles it leaves SMs idle and measured slower than
// the tensor cores alone); 0 (no split) otherwise.
static int pp_small_span(const bp_ctx* ctx, int ts, const bp_map_geom* g) {
  if (!bp_deposit_uses_tc(ctx, ts) || ts != 64) return 0;
  if (ctx->small_span >= 0) return ctx->small_span;
  const int64_t tiles = (int64_t)((g->nx + 63) / 64) * ((g->ny + 63) / 64);
  return tiles >= 4 * (int64_t)ctx->num_sms ? 8 : 0;
}

// The particle paste with every scratch buffer supplied by the caller.  Reads back the
// pair count (one host synchronisation) and returns BP_ERANGE if it exceeds max_pairs.
int bp_pp_paste_buffers(bp_ctx* ctx, int64_t n, const float* assigned, const bp_map_geom* g,
                        int select, float* ymap, float* bmap, float* ylo, float* blo,
                        const BpPasteBuffers* B) {
  const int ts = ctx->pp_tile;
  if (ctx->pp_kernel == BP_DEPOSIT_TENSOR && ts != 64)
    return bp_fail(ctx, BP_EINVAL, "paste (no allocation): the tensor-core deposit needs tile 64");
  const int ntx = (g->nx + ts - 1) / ts, nty = (g->ny + ts - 1) / ts;
  const int64_t n_tiles = (int64_t)ntx * nty;
  if (n_tiles > B->max_tiles)
    return bp_fail(ctx, BP_ERANGE, "paste (no allocation): %lld tiles exceed the limit %lld",
                   (long long)n_tiles, (long long)B->max_tiles);
  const float4* rec = reinterpret_cast<const float4*>(assigned);
  unsigned nb = (unsigned)((n + 255) / 256);
  int r;
  k_pair_count<<<nb, 256, 0, ctx->stream>>>(rec, n, g->nx, g->ny, ts, select, B->counts);
  BP_LAUNCH_CHECK(ctx, "pair count");
  if ((r = bp_scan_u32_to_i64_buf(ctx, B->counts, B->offs, n, B->bsum))) return r;
  BP_CUDA(ctx, cudaMemcpyAsync(ctx->h_pinned, B->offs + n, 8, cudaMemcpyDeviceToHost,
                               ctx->stream));
  BP_CUDA(ctx, cudaStreamSynchronize(ctx->stream));
  const int64_t np = ctx->h_pinned[0];
  if (np > B->max_pairs)
    return bp_fail(ctx, BP_ERANGE, "paste (no allocation): %lld tile pairs exceed the limit %lld",
                   (long long)np, (long long)B->max_pairs);
  if (np == 0) return BP_OK;
  k_pair_emit<<<nb, 256, 0, ctx->stream>>>(rec, n, g->nx, g->ny, ts, select, ntx, B->offs,
                                           B->keys0, B->vals0, 0, bp_dbg_word(ctx));
  BP_LAUNCH_CHECK(ctx, "pair emit");
  int key_bits = 0;
  while (((int64_t)1 << key_bits) < n_tiles) ++key_bits;
  uint32_t *ks, *vs;
  if ((r = bp_radix_sort_pairs_buf(ctx, B->keys0, B->vals0, B->keys1, B->vals1, np, key_bits,
                                   B->hist, B->hoffs, B->bsum, &ks, &vs)))
    return r;
  if (ts == 64)
    return deposit_buffers<64>(ctx, assigned, g, ks, vs, np, n_tiles, ymap, bmap, ylo, blo, B);
  return deposit_buffers<32>(ctx, assigned, g, ks, vs, np, n_tiles, ymap, bmap, ylo, blo, B);
}

extern "C" {

int bp_assign_particles(bp_ctx* ctx, int64_t n, const float* x, const float* y, const float* z,
                        const float* vx, const float* vy, const float* vz, const float* hsml,
                        const int32_t* halo_id, double Mp, int64_t n_halos,
                        const float* halo_pos, const double* model, const int32_t* status,
                        const bp_map_geom* geom, float* out) {
  return bp_assign_particles_phi(ctx, n, x, y, z, vx, vy, vz, nullptr, hsml, halo_id, Mp, n_halos,
                                 halo_pos, model, status, geom, out);
}

int bp_assign_particles_phi(bp_ctx* ctx, int64_t n, const float* x, const float* y,
                            const float* z, const float* vx, const float* vy, const float* vz,
                            const float* phi, const float* hsml, const int32_t* halo_id,
                            double Mp, int64_t n_halos, const float* halo_pos,
                            const double* model, const int32_t* status,
                            const bp_map_geom* geom, float* out) {
  return bp_assign_particles_part(ctx, n, x, y, z, vx, vy, vz, phi, hsml, halo_id, Mp, n_halos,
                                  halo_pos, model, status, geom, out, BP_ASSIGN_ALL);
}

int bp_assign_particles_part(bp_ctx* ctx, int64_t n, const float* x, const float* y,
                             const float* z, const float* vx, const float* vy, const float* vz,
                             const float* phi, const float* hsml, const int32_t* halo_id,
                             double Mp, int64_t n_halos, const float* halo_pos,
                             const double* model, const int32_t* status,
                             const bp_map_geom* geom, float* out, int part) {
  if (!ctx) return BP_EINVAL;
  if (n < 0 || n_halos < 0) return bp_fail(ctx, BP_EINVAL, "bp_assign_particles: negative size");
  if (part != BP_ASSIGN_ALL && part != BP_ASSIGN_GEOMETRY && part != BP_ASSIGN_SIGNALS)
    return bp_fail(ctx, BP_EINVAL, "bp_assign_particles: unknown part");
  int r = check_geom(ctx, geom, "bp_assign_particles");
  if (r) return r;
  if (n == 0) return BP_OK;
  if (!x || !y || !z || !vx || !vy || !vz || !hsml || !halo_id || !out)
    return bp_fail(ctx, BP_EINVAL, "bp_assign_particles: null pointer");
  if (part != BP_ASSIGN_GEOMETRY && n_halos > 0 && (!halo_pos || !model || !status))
    return bp_fail(ctx, BP_EINVAL, "bp_assign_particles: null halo arrays");
  if (!(Mp > 0)) return bp_fail(ctx, BP_EINVAL, "bp_assign_particles: Mp <= 0");
  if (((uintptr_t)out & 15) != 0)
    return bp_fail(ctx, BP_EINVAL, "bp_assign_particles: out must be 16-byte aligned");
  const BpParams& P = ctx->p;
  float* blk = nullptr;
  bp_phase_begin(ctx, BP_PH_ASSIGN);
  if (part != BP_ASSIGN_GEOMETRY &&
      (r = halo_blocks(ctx, n_halos, model, status, Mp / P.h, halo_pos, &blk)))
    return r;
  AssignArgs a;
  a.x = x; a.y = y; a.z = z; a.vx = vx; a.vy = vy; a.vz = vz; a.hs = hsml;
  a.phi = phi;
  a.hid = halo_id;
  a.hpos = halo_pos;
  a.blk = blk;
  a.n = n;
  a.nh = n_halos;
  a.th0x = geom->theta0_x;
  a.th0y = geom->theta0_y;
  a.inv_dth = 1.0 / geom->dtheta;
  auto split = [](double v, float& hi, float& lo) {
    hi = (float)v;
    lo = (float)(v - (double)hi);
  };
  split(a.th0x, a.th0x_hi, a.th0x_lo);
  split(a.th0y, a.th0y_hi, a.th0y_lo);
  split(a.inv_dth, a.inv_hi, a.inv_lo);
  a.inv_h = (float)(1.0 / P.h);
  a.inv_h_dth = (float)(1.0 / (P.h * geom->dtheta));
  a.inv_om_pix = (float)(1.0 / (geom->dtheta * geom->dtheta));
  a.field_B = (float)(P.CN * (Mp / P.h) * (P.field_fb ? P.fb : 1.0) / bpc::C_KMS);
  a.n_poly = (float)P.n_poly;
  double rn = rint(P.n_poly);
  a.n_int = (fabs(P.n_poly - rn) < 1e-12 && rn >= 1 && rn <= 16) ? (int)rn : -1;
  a.n_nt = (float)P.n_nt;
  a.out = out;
  // 16-byte SoA loads, 4 particles per thread, when every array allows them; the tail (and
  // unaligned arrays) one particle per thread
  auto al16 = [](const void* p) { return ((uintptr_t)p & 15) == 0; };
  const bool vec = al16(x) && al16(y) && al16(z) && al16(vx) && al16(vy) && al16(vz) &&
                   al16(hsml) && al16(halo_id);
  const int64_t n4 = vec ? n / 4 : 0;  // particles [0, 4 n4) by the vector kernel
  if (n4 > 0) {
    const unsigned nb4 = (unsigned)((n4 + ASSIGN_THREADS - 1) / ASSIGN_THREADS);
    // the z(chi), tau(chi) table in dynamic shared memory (not read by the geometry pass)
    const size_t zt_smem = part == BP_ASSIGN_GEOMETRY ? 0 : (size_t)ctx->t.nc * sizeof(float4);
    if (part == BP_ASSIGN_SIGNALS)
      BP_CUDA(ctx, cudaFuncSetAttribute(k_assign4<2>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                        (int)zt_smem));
    else if (part != BP_ASSIGN_GEOMETRY)
      BP_CUDA(ctx, cudaFuncSetAttribute(k_assign4<0>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                        (int)zt_smem));
    if (part == BP_ASSIGN_GEOMETRY)
      k_assign4<1><<<nb4, ASSIGN_THREADS, zt_smem, ctx->stream>>>(a, ctx->t);
    else if (part == BP_ASSIGN_SIGNALS)
      k_assign4<2><<<nb4, ASSIGN_THREADS, zt_smem, ctx->stream>>>(a, ctx->t);
    else
      k_assign4<0><<<nb4, ASSIGN_THREADS, zt_smem, ctx->stream>>>(a, ctx->t);
    BP_LAUNCH_CHECK(ctx, "assign (4 per thread)");
  }
  if (4 * n4 < n) {
    AssignArgs t = a;  // the rest: particle 4 n4 + j is element j of shifted arrays
    const int64_t o = 4 * n4;
    t.x = x + o; t.y = y + o; t.z = z + o; t.vx = vx + o; t.vy = vy + o; t.vz = vz + o;
    t.hs = hsml + o;
    t.hid = halo_id + o;
    t.phi = phi ? phi + o : nullptr;
    t.out = out + o * BP_ASSIGNED_STRIDE;
    t.n = n - o;
    const unsigned nb = (unsigned)((t.n + 255) / 256);
    if (part == BP_ASSIGN_GEOMETRY)
      k_assign<1><<<nb, 256, 0, ctx->stream>>>(t, ctx->t);
    else if (part == BP_ASSIGN_SIGNALS)
      k_assign<2><<<nb, 256, 0, ctx->stream>>>(t, ctx->t);
    else
      k_assign<0><<<nb, 256, 0, ctx->stream>>>(t, ctx->t);
    BP_LAUNCH_CHECK(ctx, "assign");
  }
  bp_phase_end(ctx, BP_PH_ASSIGN);
  return BP_OK;
}

int bp_paste_particles(bp_ctx* ctx, int64_t n, const float* assigned, const bp_map_geom* geom,
                       int select, float* ymap, float* bmap, float* ylo, float* blo) {
  if (!ctx) return BP_EINVAL;
  int r = check_geom(ctx, geom, "bp_paste_particles");
  if (r) return r;
  if (geom->n_maps != 1) return bp_fail(ctx, BP_EINVAL, "bp_paste_particles: n_maps must be 1");
  if (n < 0) return bp_fail(ctx, BP_EINVAL, "bp_paste_particles: n < 0");
  if (n > (int64_t)UINT32_MAX) return bp_fail(ctx, BP_ERANGE, "bp_paste_particles: n >= 2^32");
  if (select < 0 || select > 2) return bp_fail(ctx, BP_EINVAL, "bp_paste_particles: select");
  if (n == 0) return BP_OK;
  if (!assigned || !ymap || !bmap || !ylo || !blo)
    return bp_fail(ctx, BP_EINVAL, "bp_paste_particles: null pointer");
  if (((uintptr_t)assigned & 15) != 0)
    return bp_fail(ctx, BP_EINVAL, "bp_paste_particles: records must be 16-byte aligned");
  const int ts = ctx->pp_tile;
  if (ctx->pp_kernel == BP_DEPOSIT_TENSOR && ts != 64)
    return bp_fail(ctx, BP_EINVAL, "bp_paste_particles: the tensor-core deposit needs tile 64");
  uint32_t *keys, *vals;
  int64_t np, n_tiles;
  const int sspan = pp_small_span(ctx, ts, geom);
  if ((r = build_pairs(ctx, n, assigned, geom, select, ts, &keys, &vals, &np, &n_tiles, sspan)))
    return r;
  if (np == 0) return BP_OK;
  const int ks = sspan > 0 ? SMALL_KS : 0;
  if (ts == 64)
    return deposit<64>(ctx, assigned, geom, keys, vals, np, n_tiles, ymap, bmap, ylo, blo, ks);
  return deposit<32>(ctx, assigned, geom, keys, vals, np, n_tiles, ymap, bmap, ylo, blo, ks);
}

int bp_pp_prepare(bp_ctx* ctx, int64_t n, const float* assigned, const bp_map_geom* geom,
                  int select) {
  if (!ctx) return BP_EINVAL;
  ctx->pp_prep.valid = 0;
  int r = check_geom(ctx, geom, "bp_pp_prepare");
  if (r) return r;
  if (geom->n_maps != 1) return bp_fail(ctx, BP_EINVAL, "bp_pp_prepare: n_maps must be 1");
  if (n < 0) return bp_fail(ctx, BP_EINVAL, "bp_pp_prepare: n < 0");
  if (n > (int64_t)UINT32_MAX) return bp_fail(ctx, BP_ERANGE, "bp_pp_prepare: n >= 2^32");
  if (select < 0 || select > 2) return bp_fail(ctx, BP_EINVAL, "bp_pp_prepare: select");
  if (n > 0 && !assigned) return bp_fail(ctx, BP_EINVAL, "bp_pp_prepare: null records");
  if (((uintptr_t)assigned & 15) != 0)
    return bp_fail(ctx, BP_EINVAL, "bp_pp_prepare: records must be 16-byte aligned");
  const int ts = ctx->pp_tile;
  if (ctx->pp_kernel == BP_DEPOSIT_TENSOR && ts != 64)
    return bp_fail(ctx, BP_EINVAL, "bp_pp_prepare: the tensor-core deposit needs tile 64");
  PpPrepared& P = ctx->pp_prep;
  P.assigned = assigned;
  P.n = n;
  P.g = *geom;
  P.select = select;
  P.ts = ts;
  P.np = 0;
  if (n > 0) {
    uint32_t *keys, *vals;
    int64_t np, n_tiles;
    const int sspan = pp_small_span(ctx, ts, geom);
    if ((r = build_pairs(ctx, n, assigned, geom, select, ts, &keys, &vals, &np, &n_tiles,
                         sspan)))
      return r;
    if (np > 0) {
      const int ks = sspan > 0 ? SMALL_KS : 0;
      r = ts == 64 ? prepare_units<64>(ctx, keys, vals, np, n_tiles, &P, ks)
                   : prepare_units<32>(ctx, keys, vals, np, n_tiles, &P, ks);
      if (r) return r;
    }
    bp_phase_end(ctx, BP_PH_SORT);
  }
  P.valid = 1;
  return BP_OK;
}

int bp_pp_deposit(bp_ctx* ctx, int64_t n, const float* assigned, const bp_map_geom* geom,
                  int select, float* ymap, float* bmap, float* ylo, float* blo) {
  if (!ctx) return BP_EINVAL;
  const PpPrepared& P = ctx->pp_prep;
  if (!P.valid || P.assigned != assigned || P.n != n || !geom || P.select != select ||
      P.ts != ctx->pp_tile || memcmp(&P.g, geom, sizeof(bp_map_geom)) != 0 ||
      (P.np > 0 && P.ks != (pp_small_span(ctx, P.ts, geom) > 0 ? SMALL_KS : 0)))
    return bp_fail(ctx, BP_EINVAL, "bp_pp_deposit: no bp_pp_prepare of these records");
  if (P.np == 0 || n == 0) return BP_OK;
  for (int k : {(int)WS_KEYS0, (int)WS_VALS0, (int)WS_KEYS1, (int)WS_VALS1, (int)WS_TILES,
                (int)WS_UNITS})
    if (ctx->ws_gen[k] != P.gen[k])
      return bp_fail(ctx, BP_EINVAL, "bp_pp_deposit: the prepared list was overwritten");
  if (!ymap || !bmap || !ylo || !blo)
    return bp_fail(ctx, BP_EINVAL, "bp_pp_deposit: null pointer");
  return P.ts == 64 ? launch_deposit<64>(ctx, assigned, geom, P, ymap, bmap, ylo, blo)
                    : launch_deposit<32>(ctx, assigned, geom, P, ymap, bmap, ylo, blo);
}

int bp_pp_pairs(bp_ctx* ctx, int64_t n, const float* assigned, const bp_map_geom* geom,
                int select, int tile, uint32_t* keys, uint32_t* vals, int64_t capacity,
                int64_t* n_pairs) {
  if (!ctx) return BP_EINVAL;
  int r = check_geom(ctx, geom, "bp_pp_pairs");
  if (r) return r;
  if (!n_pairs || tile <= 0 || n < 0) return bp_fail(ctx, BP_EINVAL, "bp_pp_pairs: arguments");
  *n_pairs = 0;
  if (n == 0) return BP_OK;
  if (!assigned) return bp_fail(ctx, BP_EINVAL, "bp_pp_pairs: null records");
  uint32_t *k, *v;
  int64_t np, nt;
  if ((r = build_pairs(ctx, n, assigned, geom, select, tile, &k, &v, &np, &nt))) return r;
  *n_pairs = np;
  if (np > capacity) return bp_fail(ctx, BP_ERANGE, "bp_pp_pairs: capacity %lld < %lld",
                                    (long long)capacity, (long long)np);
  if (np > 0) {
    if (!keys || !vals) return bp_fail(ctx, BP_EINVAL, "bp_pp_pairs: null output");
    BP_CUDA(ctx, cudaMemcpyAsync(keys, k, np * 4, cudaMemcpyDeviceToDevice, ctx->stream));
    BP_CUDA(ctx, cudaMemcpyAsync(vals, v, np * 4, cudaMemcpyDeviceToDevice, ctx->stream));
  }
  BP_CUDA(ctx, cudaStreamSynchronize(ctx->stream));
  return BP_OK;
}

}  // extern "C"

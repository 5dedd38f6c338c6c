// bp_internal.cuh -- shared declarations of the CUDA implementation of bp.h.
// Device helpers, the context, the background tables and the error plumbing.
#pragma once

#include <cuda_runtime.h>
#include <math.h>
#include <stdint.h>
#include <stdio.h>

#include "../../include/bp.h"

// ---------------------------------------------------------------- constants
// Physical constants (CODATA 2018 / IAU 2015 nominal values).
namespace bpc {
constexpr double PI = 3.14159265358979323846;
constexpr double C_KMS = 299792.458;
constexpr double G_SI = 6.67430e-11;
constexpr double MSUN_KG = 1.98840987e30;
constexpr double MPC_M = 3.0856775814913673e22;
constexpr double SIGMA_T = 6.6524587321e-29;
constexpr double ME_C2_J = 8.1871057769e-14;
constexpr double MP_KG = 1.67262192369e-27;
constexpr double H_PLANCK = 6.62607015e-34;
constexpr double K_BOLTZ = 1.380649e-23;
// G in Mpc (km/s)^2 / Msun
constexpr double G = G_SI * MSUN_KG / (MPC_M * 1.0e6);
}  // namespace bpc

// ---------------------------------------------------------------- tables
// Background quantities tabulated on the host in FP64 and interpolated on the
// device with cubic Hermite splines (values + exact derivatives at the nodes).
struct BpTables {
  // uniform in z: chi(z) [Mpc comoving] and tau(z)
  const double* chi_z;   // [nz] values
  const double* dchi_z;  // [nz] dchi/dz = c/H
  const double* tau_z;   // [nz]
  const double* dtau_z;  // [nz]
  int nz;
  double dz;
  // uniform in chi (FP32, for particles): z(chi) and tau(chi)
  const float* z_c;    // [nc]
  const float* dz_c;   // [nc] dz/dchi
  const float* tau_c;  // [nc]
  const float* dtau_c; // [nc] dtau/dchi
  const float4* zt4;   // [nc] the same four, interleaved per node (16-byte aligned)
  int nc;
  float dchi;
  float inv_dchi;
};

struct BpParams {
  // cosmology
  double Om, Ob, h, Tcmb, XH;
  double fb, mu_e, pe_frac;  // f_b, mu_e = 2/(1+X), P_e/P_th = (2X+2)/(5X+3)
  double rho_cr0;            // Msun/Mpc^3
  // ICM
  double Gamma, n_poly, eps_dm, eps_star, f_star, S_star, alpha_nt, beta_nt, n_nt;
  int energy_sign, field_fb;
  // observables: y per (P x length) and sigma_T n_e per (rho_g x length)
  double CP, CN;
};

// ---------------------------------------------------------------- context
enum { WS_COUNTS = 0, WS_OFFS, WS_KEYS0, WS_VALS0, WS_KEYS1, WS_VALS1, WS_HIST, WS_TILES,
       WS_UNITS, WS_PART, WS_MISC, WS_TABLE, WS_HPAR, WS_MISC2, WS_MISC3, WS_HALO,
       WS_NSLOTS };

// A particle work list built by bp_pp_prepare for bp_pp_deposit (in the context's scratch;
// ws_gen records the generation of each slot it lives in, so that a deposit can tell
// whether another call has reused them since).
struct PpPrepared {
  int valid;
  const float* assigned;
  int64_t n;
  bp_map_geom g;
  int select, ts, unit;
  int ks;  // 3: keys 8 tile + size class (classes 1-7: the small-particle deposit)
  int64_t np, n_tiles, n_keys, max_units, n_slots;
  const uint32_t* vals;
  int64_t *tstart, *uoff, *soff;
  void* units;
  uint64_t gen[WS_NSLOTS];
};

struct bp_ctx {
  BpParams p;
  BpTables t;
  cudaStream_t stream;
  void* table_mem;
  void* ws[WS_NSLOTS];
  size_t ws_bytes[WS_NSLOTS];
  uint64_t ws_gen[WS_NSLOTS];  // calls of bp_ws per slot (every user of a slot asks for it)
  PpPrepared pp_prep;
  int64_t* d_counter;  // small device scalars
  int* d_flags;
  int64_t* h_pinned;   // pinned host scalars
  int num_sms;
  int pp_tile, hp_tile, pp_unit, hp_unit;
  int pp_kernel;  // BP_DEPOSIT_*
  int small_span; // particles at most this many pixels wide take the small-particle deposit
  int timing;
  cudaEvent_t ev[BP_NPHASES][2];
  double ph_ms[BP_NPHASES];
  int ph_open[BP_NPHASES];
  int64_t launches;
  int64_t last_fallback;  // halos the residual gate sent to the full solve
  int64_t test_stall_polls;  // > 0: the tensor-core deposit first waits on a flag nothing sets
  char msg[512];
};

// ---- Debug build.  Compiled with -DBP_DEBUG (build.build(debug=True), into _build_debug/),
// the particle paste's kernels check their index arithmetic before each store that a wrong
// index would misplace (pair emission, radix scatter, small-particle sums, tensor-core
// write-out, partial-tile reduction): a failed check skips the store and records the
// check's site code in the context's debug word, keeping the first failure; bp_debug_status
// reads and clears the word.  The release build compiles the checks out.
constexpr int BP_DBG_SLOT = 8;  // the debug word's slot in bp_ctx::d_flags
__device__ __forceinline__ bool bp_dbg_fail(int* word, int site) {
  if (word) atomicCAS(word, 0, site);
  return false;
}
#ifdef BP_DEBUG
#define BP_DCHECK(ok, word, site) ((ok) ? true : bp_dbg_fail((word), (site)))
#else
#define BP_DCHECK(ok, word, site) true
#endif
inline int* bp_dbg_word(bp_ctx* ctx) { return ctx->d_flags + BP_DBG_SLOT; }


// phase timing (no-ops unless bp_set_timing(ctx, 1))
void bp_phase_begin(bp_ctx* ctx, int ph);
void bp_phase_end(bp_ctx* ctx, int ph);

int bp_fail(bp_ctx* ctx, int code, const char* fmt, ...);
int bp_cuda_check(bp_ctx* ctx, cudaError_t e, const char* what);
int bp_ws(bp_ctx* ctx, int slot, size_t bytes, void** out);

// Threads per block of a one-thread-per-item launch: `big`, or one warp per block when
// blocks of `big` would cover fewer SMs than the GPU has.  Scalar FP64 work is bound by each
// SM's FP64 rate, so a small catalogue runs fastest as one warp on each of many SMs.
inline int bp_item_block(const bp_ctx* ctx, int64_t n, int big) {
  return n < (int64_t)big * ctx->num_sms ? 32 : big;
}

#define BP_CUDA(ctx, call)                                        \
  do {                                                            \
    cudaError_t e_ = (call);                                      \
    if (e_ != cudaSuccess) return bp_cuda_check(ctx, e_, #call);  \
  } while (0)

// checks the preceding kernel launch and counts it
#define BP_LAUNCH_CHECK(ctx, what)                                        \
  do {                                                                    \
    (ctx)->launches++;                                                    \
    cudaError_t e_ = cudaGetLastError();                                  \
    if (e_ != cudaSuccess) return bp_cuda_check(ctx, e_, what);           \
  } while (0)

// ---------------------------------------------------------------- device helpers
__device__ __forceinline__ double bp_hermite(const double* v, const double* d, int n, double h,
                                             double x) {
  double u = x / h;
  int i = (int)u;
  if (i < 0) i = 0;
  if (i > n - 2) i = n - 2;
  double t = u - i;
  double t2 = t * t, t3 = t2 * t;
  double h00 = 2 * t3 - 3 * t2 + 1, h10 = t3 - 2 * t2 + t, h01 = -2 * t3 + 3 * t2,
         h11 = t3 - t2;
  return h00 * v[i] + h10 * h * d[i] + h01 * v[i + 1] + h11 * h * d[i + 1];
}

__device__ __forceinline__ float bp_hermitef(const float* v, const float* d, int n, float h,
                                             float inv_h, float x) {
  float u = x * inv_h;
  int i = (int)u;
  if (i < 0) i = 0;
  if (i > n - 2) i = n - 2;
  float t = u - (float)i;
  float t2 = t * t, t3 = t2 * t;
  float h00 = 2.f * t3 - 3.f * t2 + 1.f, h10 = t3 - 2.f * t2 + t, h01 = -2.f * t3 + 3.f * t2,
        h11 = t3 - t2;
  return h00 * __ldg(v + i) + h10 * h * __ldg(d + i) + h01 * __ldg(v + i + 1) +
         h11 * h * __ldg(d + i + 1);
}

// z(chi) and tau(chi) of a particle by cubic Hermite interpolation of the interleaved
// per-node table zt (T.zt4, or a copy of it in shared memory; two 16-byte loads).
__device__ __forceinline__ void bp_hermite_ztau(const BpTables& T, const float4* zt, float x,
                                                float& z, float& tau) {
  float u = x * T.inv_dchi;
  int i = (int)u;
  if (i < 0) i = 0;
  if (i > T.nc - 2) i = T.nc - 2;
  const float t = u - (float)i;
  const float t2 = t * t, t3 = t2 * t;
  const float h00 = 2.f * t3 - 3.f * t2 + 1.f, h10 = t3 - 2.f * t2 + t, h01 = -2.f * t3 + 3.f * t2,
              h11 = t3 - t2;
  const float4 a = zt[i], b = zt[i + 1];
  const float h = T.dchi;
  z = h00 * a.x + h10 * h * a.y + h01 * b.x + h11 * h * b.y;
  tau = h00 * a.z + h10 * h * a.w + h01 * b.z + h11 * h * b.w;
}

// Integrated normalised kernel in the "split" representation used by the deposit:
// with e = dx / h, returns w(e) for dx < 0 and w(e) - 1 = -w(-e) for dx >= 0.
// Differences of these values give pixel weights without cancellation near w = 1.
// Only the left half of the printed piecewise quartic (x <= 0) is evaluated, at
// a = min(|e|, 1): the outer piece (2/3)(1 - a)^4 for a >= 1/2 (zero at a = 1) and the
// inner piece (4/3)(3/8 - a + 2a^3 - (3/2)a^4) = 1/2 - (4/3)a + (8/3)a^3 - 2a^4 below.
// The sign is applied as a bit operation (dx is never -0 here: it is k - f with k an
// integer-valued float and f >= 0).
__device__ __forceinline__ float bp_wsplit_inv(float dx, float inv_h) {
  const float a = fminf(fabsf(dx * inv_h), 1.0f);
  const float t = 1.0f - a;
  const float t2 = t * t;
  const float wo = (2.0f / 3.0f) * t2 * t2;
  const float a2 = a * a;
  const float wi = 0.5f - a * ((4.0f / 3.0f) + a2 * (2.0f * a - (8.0f / 3.0f)));
  const float wl = a < 0.5f ? wi : wo;
  // dx >= 0: flip the sign of wl
  return __int_as_float(__float_as_int(wl) ^ (~__float_as_int(dx) & (int)0x80000000));
}

// The integrated kernel at a cell edge in the same split representation, from the truncated-
// power form of the piecewise quartic: with a = |dx| / h,
//   w_left(a) = (2/3) max(1 - a, 0)^4 - (8/3) max(1/2 - a, 0)^4,
// (the inner piece 1/2 - (4/3) a + (8/3) a^3 - 2 a^4 below a = 1/2, the outer piece
// (2/3)(1 - a)^4 above, zero beyond a = 1), from |dx| and the scales k1 = BP_KT / h,
// k2 = BP_KS / h: no branch, no piece selection.  h = 0 is an infinite scale (k1, k2 = BP_KT,
// BP_KS x 1e38): every edge off the particle is 0.  dx must not be -0 or 0 with h = 0.
// Items per block of the radix sort (its scratch sizes depend on it).
constexpr int BP_RS_ITEMS = 2048;

constexpr float BP_KT = 0.9036020040512085f;  // (2/3)^(1/4)
constexpr float BP_KS = 1.277886152267456f;   // (8/3)^(1/4)
__device__ __forceinline__ float bp_edge_split(float dx, float k1, float k2) {
  // KT (1 - a) and KS (1/2 - a), clipped below at 0 (both stay below 1, so clamping to
  // [0, 1] is the same clip)
  const float t = __saturatef(fmaf(-k1, fabsf(dx), BP_KT));
  const float s = __saturatef(fmaf(-k2, fabsf(dx), 0.5f * BP_KS));
  const float A = t * t, B = s * s;
  const float w = fmaf(A, A, -(B * B));
  return __int_as_float(__float_as_int(w) ^ (~__float_as_int(dx) & (int)0x80000000));
}

// Pixel span of a particle at px = ix + fx with kernel radius h, decided in FP32
// (round-to-nearest, no contraction) relative to ix: columns
// ix + floor(fx - h) .. ix + floor(fx + h), clipped to [0, n-1].  A negative or NaN
// radius covers nothing.
__device__ __forceinline__ bool bp_span(int ix, float fx, float h, int n, int& lo, int& hi) {
  if (!(h >= 0.0f) || !(fx == fx)) return false;
  float a = __fsub_rn(fx, h), b = __fadd_rn(fx, h);
  float fa = fmaxf(floorf(a), -4.0e9f), fb = fminf(floorf(b), 4.0e9f);
  long long L = (long long)ix + (long long)fa, H = (long long)ix + (long long)fb;
  if (H < 0 || L > n - 1) return false;
  lo = L < 0 ? 0 : (int)L;
  hi = H > n - 1 ? n - 1 : (int)H;
  return true;
}

// Weights of NC consecutive cells of one axis: cell k (relative to the particle's
// pixel index) spans [k - f, k + 1 - f] in pixel units around the centre.  The edge
// values use the split form of w (bp_wsplit_inv), the cell holding the centre adds 1.
// Every deposit kernel takes its weights from here, so they agree bit for bit.
template <int NC>
__device__ __forceinline__ void bp_cell_weights(int kbase, float f, float h, float ih,
                                                float (&w)[NC]) {
  if (h > 0.f) {
    // the cell whose left edge is left of the centre and whose right edge is not
    // (0 <= f < 1): cell 0 when f > 0, cell -1 when f == 0
    const int kc = f > 0.f ? 0 : -1;
    const float kb = (float)kbase;  // kb + j is exact for |kbase| < 2^24
    float prev = bp_wsplit_inv(__fsub_rn(kb, f), ih);
#pragma unroll
    for (int j = 0; j < NC; ++j) {
      float dn = __fsub_rn(__fadd_rn(kb, (float)(j + 1)), f);
      float cur = bp_wsplit_inv(dn, ih);
      w[j] = cur - prev;
      if (kbase + j == kc) w[j] += 1.f;
      prev = cur;
    }
  } else {  // h = 0: nearest grid point
#pragma unroll
    for (int j = 0; j < NC; ++j) w[j] = (kbase + j == 0) ? 1.f : 0.f;
  }
}

// A deposit work unit: particles [begin, end) of the tile-sorted pair list, all in tile
// `tile`; slot >= 0 names its partial tile when the tile is split into several units.
struct BpUnit {
  int tile;
  int slot;      // partial slot, -1 = the tile's only unit (adds to the map directly)
  int64_t begin;
  int64_t end;
};

// Error-free sum of two floats (Knuth's TwoSum): s + e == a + b exactly.
__device__ __forceinline__ void bp_two_sum(float a, float b, float& s, float& e) {
  s = __fadd_rn(a, b);
  float bb = __fsub_rn(s, a);
  e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
}

// host helpers implemented in the .cu files
int bp_scan_u32_to_i64(bp_ctx* ctx, const uint32_t* in, int64_t* out, int64_t n);
int bp_radix_sort_pairs(bp_ctx* ctx, uint32_t* keys, uint32_t* vals, uint32_t* keys_tmp,
                        uint32_t* vals_tmp, int64_t n, int key_bits, uint32_t** keys_out,
                        uint32_t** vals_out);
int bp_tile_ranges(bp_ctx* ctx, const uint32_t* keys, int64_t n, int64_t n_tiles,
                   int64_t* tile_start);

// caller-buffer variants (no scratch allocation)
int bp_scan_u32_to_i64_buf(bp_ctx* ctx, const uint32_t* in, int64_t* out, int64_t n,
                           int64_t* bsum);
int bp_radix_sort_pairs_buf(bp_ctx* ctx, uint32_t* keys, uint32_t* vals, uint32_t* keys_tmp,
                            uint32_t* vals_tmp, int64_t n, int key_bits, uint32_t* hist,
                            int64_t* offs, int64_t* bsum, uint32_t** keys_out,
                            uint32_t** vals_out);

// Scratch of the particle paste when the caller provides it (one work unit per tile,
// so no partial tiles).  Capacities are checked by the caller of bp_pp_paste_buffers.
struct BpPasteBuffers {
  uint32_t* counts;   // [n + 1]
  int64_t* offs;      // [n + 1]
  uint32_t *keys0, *vals0, *keys1, *vals1;  // [max_pairs] each
  uint32_t* hist;     // [256 * ceil(max_pairs / BP_RS_ITEMS)]
  int64_t* hoffs;     // [256 * ceil(max_pairs / BP_RS_ITEMS) + 1]
  int64_t* bsum;      // [max(n, 256 * ceil(max_pairs / BP_RS_ITEMS), max_tiles) / 8192 + 2]
  int64_t* tstart;    // [max_tiles + 1]
  int64_t* uoff;      // [max_tiles + 1]
  uint32_t* ucount;   // [max_tiles + 1]
  void* units;        // [max_tiles] work units
  int64_t* counter;   // [1], cleared by bp_pp_paste_buffers
  int64_t max_pairs;
  int64_t max_tiles;
};
int bp_pp_paste_buffers(bp_ctx* ctx, int64_t n, const float* assigned, const bp_map_geom* geom,
                        int select, float* ymap, float* bmap, float* ylo, float* blo,
                        const BpPasteBuffers* buf);
size_t bp_pp_unit_bytes();

// tensor-core deposit (tile 64): launch over the work units, and the check of its
// timed-out-wait flag (synchronises the stream)
int bp_deposit_tc_launch(bp_ctx* ctx, const float* assigned, const uint32_t* vals,
                         const BpUnit* units, const int64_t* n_units_dev, int64_t* counter,
                         int64_t max_units, const bp_map_geom* g, float* ymap, float* bmap,
                         float* ylo, float* blo, float* partials);
int bp_deposit_tc_check(bp_ctx* ctx);
// Kernels loaded ahead of their first launch (cudaFuncGetAttributes), and the allocation-free
// paste's device array resolved, when a context is created (bp_noalloc.cu)
int bp_pp_preload(bp_ctx* ctx);
int bp_sort_preload(bp_ctx* ctx);
int bp_deposit_tc_preload(bp_ctx* ctx);
int bp_noalloc_setup(bp_ctx* ctx);
// true when the deposit of a paste with tile ts runs on the tensor cores
bool bp_deposit_uses_tc(const bp_ctx* ctx, int ts);

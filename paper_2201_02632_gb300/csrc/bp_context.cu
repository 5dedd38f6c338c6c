// bp_context.cu -- context life cycle, background tables, scratch and errors.
#include <stdarg.h>
#include <stdlib.h>
#include <string.h>

#include <vector>

#include "bp_internal.cuh"

static thread_local char g_tls_msg[512];

int bp_fail(bp_ctx* ctx, int code, const char* fmt, ...) {
  va_list ap;
  va_start(ap, fmt);
  char* dst = ctx ? ctx->msg : g_tls_msg;
  vsnprintf(dst, 512, fmt, ap);
  va_end(ap);
  return code;
}

int bp_cuda_check(bp_ctx* ctx, cudaError_t e, const char* what) {
  return bp_fail(ctx, BP_ECUDA, "%s: %s", what, cudaGetErrorString(e));
}

// Grow-only scratch slot.  Frees the old block after synchronising the stream.
int bp_ws(bp_ctx* ctx, int slot, size_t bytes, void** out) {
  ++ctx->ws_gen[slot];
  if (bytes == 0) bytes = 16;
  if (ctx->ws_bytes[slot] < bytes) {
    if (ctx->ws[slot]) {
      BP_CUDA(ctx, cudaStreamSynchronize(ctx->stream));
      BP_CUDA(ctx, cudaFree(ctx->ws[slot]));
      ctx->ws[slot] = nullptr;
      ctx->ws_bytes[slot] = 0;
    }
    size_t want = bytes + bytes / 8;  // headroom for slowly growing inputs
    cudaError_t e = cudaMalloc(&ctx->ws[slot], want);
    if (e != cudaSuccess) {
      cudaGetLastError();
      return bp_fail(ctx, BP_ENOMEM, "scratch slot %d: cannot allocate %zu bytes", slot, want);
    }
    ctx->ws_bytes[slot] = want;
  }
  *out = ctx->ws[slot];
  return BP_OK;
}

// ---------------------------------------------------------------- host cosmology
namespace {
struct HostCosmo {
  double Om, h;
  double E(double z) const { return sqrt(Om * (1 + z) * (1 + z) * (1 + z) + (1 - Om)); }
  double c_over_H(double z) const { return bpc::C_KMS / (100.0 * h * E(z)); }  // Mpc
};

// 8-point Gauss-Legendre on [a, b] (nodes/weights of the Legendre polynomial P_8)
template <class F>
double gl8(F f, double a, double b) {
  static const double x[4] = {0.1834346424956498, 0.5255324099163290, 0.7966664774136267,
                              0.9602898564975363};
  static const double w[4] = {0.3626837833783620, 0.3137066458778873, 0.2223810344533745,
                              0.1012285362903763};
  double c = 0.5 * (a + b), hw = 0.5 * (b - a), s = 0;
  for (int i = 0; i < 4; ++i) s += w[i] * (f(c - hw * x[i]) + f(c + hw * x[i]));
  return s * hw;
}
}  // namespace

static int build_tables(bp_ctx* ctx) {
  const BpParams& P = ctx->p;
  HostCosmo hc{P.Om, P.h};
  const double zmax = 10.0;
  const int nz = 20001;
  const double dz = zmax / (nz - 1);
  // mean electron density today [m^-3] and sigma_T nbar_e per Mpc
  double ne0 = P.Ob * P.rho_cr0 * bpc::MSUN_KG / pow(bpc::MPC_M, 3) / (P.mu_e * bpc::MP_KG);
  double tau_per_mpc = bpc::SIGMA_T * ne0 * bpc::MPC_M;
  std::vector<double> chi(nz), dchi(nz), tau(nz), dtau(nz);
  chi[0] = tau[0] = 0.0;
  for (int k = 0; k < nz; ++k) {
    double z = k * dz;
    dchi[k] = hc.c_over_H(z);
    dtau[k] = tau_per_mpc * hc.c_over_H(z) * (1 + z) * (1 + z);
    if (k > 0) {
      double z0 = (k - 1) * dz;
      chi[k] = chi[k - 1] + gl8([&](double s) { return hc.c_over_H(s); }, z0, z);
      tau[k] = tau[k - 1] +
               gl8([&](double s) { return tau_per_mpc * hc.c_over_H(s) * (1 + s) * (1 + s); },
                   z0, z);
    }
  }
  // inverse table, uniform in chi
  const double chimax = chi[nz - 1];
  // Mpc: the cubic Hermite error at this spacing (~1e-12 relative for z and tau) is far
  // below the FP32 rounding of chi / dch in the interpolation, and the table (about 600 nodes
  // to z = 10) fits in shared memory, where the assign kernel keeps it
  const double dch = 16.0;
  const int nc = (int)floor(chimax / dch);
  std::vector<float> zc(nc), dzc(nc), tc(nc), dtc(nc);
  int k = 0;
  for (int j = 0; j < nc; ++j) {
    double target = j * dch;
    while (k < nz - 2 && chi[k + 1] < target) ++k;
    // Newton on the Hermite cubic of interval k
    double t = (chi[k + 1] > chi[k]) ? (target - chi[k]) / (chi[k + 1] - chi[k]) : 0.0;
    for (int it = 0; it < 30; ++it) {
      double t2 = t * t, t3 = t2 * t;
      double f = (2 * t3 - 3 * t2 + 1) * chi[k] + (t3 - 2 * t2 + t) * dz * dchi[k] +
                 (-2 * t3 + 3 * t2) * chi[k + 1] + (t3 - t2) * dz * dchi[k + 1] - target;
      double df = (6 * t2 - 6 * t) * chi[k] + (3 * t2 - 4 * t + 1) * dz * dchi[k] +
                  (-6 * t2 + 6 * t) * chi[k + 1] + (3 * t2 - 2 * t) * dz * dchi[k + 1];
      double step = f / df;
      t -= step;
      if (fabs(step) < 1e-15) break;
    }
    double z = (k + t) * dz;
    zc[j] = (float)z;
    dzc[j] = (float)(1.0 / hc.c_over_H(z));
    // tau at z from the z-table (Hermite)
    double t2 = t * t, t3 = t2 * t;
    double tz = (2 * t3 - 3 * t2 + 1) * tau[k] + (t3 - 2 * t2 + t) * dz * dtau[k] +
                (-2 * t3 + 3 * t2) * tau[k + 1] + (t3 - t2) * dz * dtau[k + 1];
    tc[j] = (float)tz;
    dtc[j] = (float)(tau_per_mpc * (1 + z) * (1 + z));
  }
  // the particle tables once more, interleaved per node (z, dz/dchi, tau, dtau/dchi): one
  // 16-byte load per node for a particle's Hermite interpolation of z(chi) and tau(chi)
  std::vector<float> zt4(4 * (size_t)nc);
  for (int j = 0; j < nc; ++j) {
    zt4[4 * j] = zc[j];
    zt4[4 * j + 1] = dzc[j];
    zt4[4 * j + 2] = tc[j];
    zt4[4 * j + 3] = dtc[j];
  }
  size_t bytes = 4 * nz * sizeof(double) + 8 * nc * sizeof(float);
  BP_CUDA(ctx, cudaMalloc(&ctx->table_mem, bytes));
  char* base = (char*)ctx->table_mem;
  double* dd = (double*)base;
  float* ff = (float*)(base + 4 * nz * sizeof(double));
  BP_CUDA(ctx, cudaMemcpy(dd, chi.data(), nz * 8, cudaMemcpyHostToDevice));
  BP_CUDA(ctx, cudaMemcpy(dd + nz, dchi.data(), nz * 8, cudaMemcpyHostToDevice));
  BP_CUDA(ctx, cudaMemcpy(dd + 2 * nz, tau.data(), nz * 8, cudaMemcpyHostToDevice));
  BP_CUDA(ctx, cudaMemcpy(dd + 3 * nz, dtau.data(), nz * 8, cudaMemcpyHostToDevice));
  BP_CUDA(ctx, cudaMemcpy(ff, zc.data(), nc * 4, cudaMemcpyHostToDevice));
  BP_CUDA(ctx, cudaMemcpy(ff + nc, dzc.data(), nc * 4, cudaMemcpyHostToDevice));
  BP_CUDA(ctx, cudaMemcpy(ff + 2 * nc, tc.data(), nc * 4, cudaMemcpyHostToDevice));
  BP_CUDA(ctx, cudaMemcpy(ff + 3 * nc, dtc.data(), nc * 4, cudaMemcpyHostToDevice));
  BP_CUDA(ctx, cudaMemcpy(ff + 4 * nc, zt4.data(), (size_t)nc * 16, cudaMemcpyHostToDevice));
  BpTables& T = ctx->t;
  T.chi_z = dd;
  T.dchi_z = dd + nz;
  T.tau_z = dd + 2 * nz;
  T.dtau_z = dd + 3 * nz;
  T.nz = nz;
  T.dz = dz;
  T.z_c = ff;
  T.dz_c = ff + nc;
  T.tau_c = ff + 2 * nc;
  T.dtau_c = ff + 3 * nc;
  T.zt4 = reinterpret_cast<const float4*>(ff + 4 * nc);
  T.nc = nc;
  T.dchi = (float)dch;
  T.inv_dchi = (float)(1.0 / dch);
  return BP_OK;
}

static void phase_collect(bp_ctx* ctx, int ph) {
  if (!ctx->ph_open[ph]) return;
  cudaEventSynchronize(ctx->ev[ph][1]);
  float ms = 0.f;
  cudaEventElapsedTime(&ms, ctx->ev[ph][0], ctx->ev[ph][1]);
  ctx->ph_ms[ph] += ms;
  ctx->ph_open[ph] = 0;
}

// Phase markers: events only; a phase's duration is collected when the phase is
// entered again or by bp_phase_times, so timing adds no host synchronisation to a
// call sequence that enters each phase once between two bp_phase_times calls.
void bp_phase_begin(bp_ctx* ctx, int ph) {
  if (!ctx->timing) return;
  phase_collect(ctx, ph);
  cudaEventRecord(ctx->ev[ph][0], ctx->stream);
}

void bp_phase_end(bp_ctx* ctx, int ph) {
  if (!ctx->timing) return;
  cudaEventRecord(ctx->ev[ph][1], ctx->stream);
  ctx->ph_open[ph] = 1;
}

extern "C" {

int bp_create(bp_ctx** out, const bp_cosmology* cosmo, const bp_icm_params* icm, void* stream) {
  if (!out || !cosmo || !icm) return bp_fail(nullptr, BP_EINVAL, "bp_create: null argument");
  *out = nullptr;
  const bp_cosmology& c = *cosmo;
  const bp_icm_params& q = *icm;
  if (!(c.Om > 0 && c.Om <= 1 && c.Ob > 0 && c.Ob < c.Om && c.h > 0 && c.XH > 0 && c.XH <= 1))
    return bp_fail(nullptr, BP_EINVAL, "bp_create: non-physical cosmology");
  if (!(q.Gamma > 1.0 && q.Gamma < 2.0) || q.alpha_nt < 0 || q.n_nt <= 0 || q.f_star < 0 ||
      q.eps_star < 0 || q.eps_dm < 0)
    return bp_fail(nullptr, BP_EINVAL, "bp_create: non-physical ICM parameters");
  bp_ctx* ctx = (bp_ctx*)calloc(1, sizeof(bp_ctx));
  if (!ctx) return bp_fail(nullptr, BP_ENOMEM, "bp_create: out of host memory");
  ctx->stream = (cudaStream_t)stream;
  BpParams& P = ctx->p;
  P.Om = c.Om;
  P.Ob = c.Ob;
  P.h = c.h;
  P.Tcmb = c.Tcmb;
  P.XH = c.XH;
  P.fb = c.Ob / c.Om;
  P.mu_e = 2.0 / (1.0 + c.XH);
  P.pe_frac = (2.0 * c.XH + 2.0) / (5.0 * c.XH + 3.0);
  double H0 = 100.0 * c.h;
  P.rho_cr0 = 3.0 * H0 * H0 / (8.0 * bpc::PI * bpc::G);
  P.Gamma = q.Gamma;
  P.n_poly = 1.0 / (q.Gamma - 1.0);
  P.eps_dm = q.eps_dm;
  P.eps_star = q.eps_star;
  P.f_star = q.f_star;
  P.S_star = q.S_star;
  P.alpha_nt = q.alpha_nt;
  P.beta_nt = q.beta_nt;
  P.n_nt = q.n_nt;
  P.energy_sign = q.energy_sign;
  P.field_fb = q.field_fb;
  P.CP = bpc::SIGMA_T / bpc::ME_C2_J * bpc::MSUN_KG * 1.0e6 / (bpc::MPC_M * bpc::MPC_M);
  P.CN = bpc::SIGMA_T * bpc::MSUN_KG / (P.mu_e * bpc::MP_KG * bpc::MPC_M * bpc::MPC_M);
  ctx->pp_tile = 64;
  ctx->hp_tile = 32;
  ctx->pp_unit = 0;  // automatic
  ctx->pp_kernel = BP_DEPOSIT_AUTO;
  ctx->small_span = -1;  // automatic
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e == cudaSuccess) e = cudaDeviceGetAttribute(&ctx->num_sms, cudaDevAttrMultiProcessorCount, dev);
  if (e != cudaSuccess) {
    int r = bp_fail(nullptr, BP_ECUDA, "bp_create: %s", cudaGetErrorString(e));
    free(ctx);
    return r;
  }
  int r = build_tables(ctx);
  if (r == BP_OK) {
    cudaError_t e1 = cudaMalloc(&ctx->d_counter, 64 * sizeof(int64_t));
    cudaError_t e2 = cudaMalloc(&ctx->d_flags, 64 * sizeof(int));
    cudaError_t e3 = cudaMallocHost(&ctx->h_pinned, 64 * sizeof(int64_t));
    if (e1 != cudaSuccess || e2 != cudaSuccess || e3 != cudaSuccess ||
        cudaMemset(ctx->d_flags, 0, 64 * sizeof(int)) != cudaSuccess)
      r = bp_fail(nullptr, BP_ECUDA, "bp_create: scalar buffers");
    // the allocation-free paste's device array and kernels, loaded now (bp_noalloc.cu)
    if (r == BP_OK && (r = bp_noalloc_setup(ctx)) != BP_OK)
      snprintf(g_tls_msg, sizeof(g_tls_msg), "%s", ctx->msg);
  } else {
    snprintf(g_tls_msg, sizeof(g_tls_msg), "%s", ctx->msg);
  }
  if (r != BP_OK) {
    bp_destroy(ctx);
    return r;
  }
  *out = ctx;
  return BP_OK;
}

int bp_destroy(bp_ctx* ctx) {
  if (!ctx) return BP_OK;
  cudaStreamSynchronize(ctx->stream);
  for (int s = 0; s < WS_NSLOTS; ++s)
    if (ctx->ws[s]) cudaFree(ctx->ws[s]);
  for (int p = 0; p < BP_NPHASES; ++p)
    for (int q = 0; q < 2; ++q)
      if (ctx->ev[p][q]) cudaEventDestroy(ctx->ev[p][q]);
  if (ctx->table_mem) cudaFree(ctx->table_mem);
  if (ctx->d_counter) cudaFree(ctx->d_counter);
  if (ctx->d_flags) cudaFree(ctx->d_flags);
  if (ctx->h_pinned) cudaFreeHost(ctx->h_pinned);
  free(ctx);
  return BP_OK;
}

const char* bp_last_error(const bp_ctx* ctx) { return ctx ? ctx->msg : g_tls_msg; }

int bp_set_stream(bp_ctx* ctx, void* stream) {
  if (!ctx) return BP_EINVAL;
  ctx->stream = (cudaStream_t)stream;
  return BP_OK;
}

int bp_set_tiling(bp_ctx* ctx, int pp_tile, int hp_tile, int pp_unit) {
  if (!ctx) return BP_EINVAL;
  if (pp_tile && pp_tile != 32 && pp_tile != 64)
    return bp_fail(ctx, BP_EINVAL, "bp_set_tiling: pp_tile must be 32 or 64");
  if (hp_tile && hp_tile != 32 && hp_tile != 64)
    return bp_fail(ctx, BP_EINVAL, "bp_set_tiling: hp_tile must be 32 or 64");
  if (pp_unit > 0 && pp_unit < 256) return bp_fail(ctx, BP_EINVAL, "bp_set_tiling: pp_unit < 256");
  if (pp_tile) ctx->pp_tile = pp_tile;
  if (hp_tile) ctx->hp_tile = hp_tile;
  if (pp_unit > 0) ctx->pp_unit = pp_unit;
  if (pp_unit < 0) ctx->pp_unit = 0;  // automatic
  return BP_OK;
}

int bp_set_deposit_kernel(bp_ctx* ctx, int kind) {
  if (!ctx) return BP_EINVAL;
  if (kind != BP_DEPOSIT_AUTO && kind != BP_DEPOSIT_SIMT && kind != BP_DEPOSIT_TENSOR)
    return bp_fail(ctx, BP_EINVAL, "bp_set_deposit_kernel: unknown kind %d", kind);
  ctx->pp_kernel = kind;
  return BP_OK;
}

namespace {
// sets the debug word as a failed check would (the plumbing test of bp_debug_selftest)
__global__ void k_debug_selftest(int* word, int site) {
  if (threadIdx.x == 0) bp_dbg_fail(word, site);
}
}  // namespace

int bp_debug_build(void) {
#ifdef BP_DEBUG
  return 1;
#else
  return 0;
#endif
}

int bp_debug_status(bp_ctx* ctx, int* site) {
  if (!ctx || !site) return BP_EINVAL;
  int* h = reinterpret_cast<int*>(ctx->h_pinned + 12);  // slot of this call only
  BP_CUDA(ctx, cudaMemcpyAsync(h, bp_dbg_word(ctx), sizeof(int), cudaMemcpyDeviceToHost,
                               ctx->stream));
  BP_CUDA(ctx, cudaMemsetAsync(bp_dbg_word(ctx), 0, sizeof(int), ctx->stream));
  BP_CUDA(ctx, cudaStreamSynchronize(ctx->stream));
  *site = *h;
  return BP_OK;
}

int bp_debug_selftest(bp_ctx* ctx, int site) {
  if (!ctx || site <= 0) return BP_EINVAL;
  k_debug_selftest<<<1, 32, 0, ctx->stream>>>(bp_dbg_word(ctx), site);
  BP_LAUNCH_CHECK(ctx, "debug self-test");
  return BP_OK;
}

int bp_set_small_span(bp_ctx* ctx, int span) {
  if (!ctx) return BP_EINVAL;
  if (span < -1 || span > 8)
    return bp_fail(ctx, BP_EINVAL, "bp_set_small_span: span outside [-1, 8]");
  ctx->small_span = span;
  return BP_OK;
}

int bp_set_wait_test(bp_ctx* ctx, int64_t polls) {
  if (!ctx) return BP_EINVAL;
  if (polls < 0 || polls > 0x7fffffff)
    return bp_fail(ctx, BP_EINVAL, "bp_set_wait_test: polls outside [0, 2^31)");
  ctx->test_stall_polls = polls;
  return BP_OK;
}

int bp_set_timing(bp_ctx* ctx, int on) {
  if (!ctx) return BP_EINVAL;
  if (on && !ctx->ev[0][0]) {
    for (int p = 0; p < BP_NPHASES; ++p)
      for (int q = 0; q < 2; ++q) BP_CUDA(ctx, cudaEventCreate(&ctx->ev[p][q]));
  }
  ctx->timing = on ? 1 : 0;
  return BP_OK;
}

int bp_phase_times(bp_ctx* ctx, double* ms, int n) {
  if (!ctx || !ms || n < BP_NPHASES) return BP_EINVAL;
  BP_CUDA(ctx, cudaStreamSynchronize(ctx->stream));
  for (int p = 0; p < BP_NPHASES; ++p) {
    phase_collect(ctx, p);
    ms[p] = ctx->ph_ms[p];
    ctx->ph_ms[p] = 0.0;
  }
  return BP_OK;
}

int64_t bp_kernel_launches(const bp_ctx* ctx) { return ctx ? ctx->launches : 0; }

int64_t bp_last_fallback_count(const bp_ctx* ctx) { return ctx ? ctx->last_fallback : 0; }

int64_t bp_workspace_bytes(const bp_ctx* ctx) {
  if (!ctx) return 0;
  int64_t s = 0;
  for (int i = 0; i < WS_NSLOTS; ++i) s += (int64_t)ctx->ws_bytes[i];
  return s;
}

}  // extern "C"

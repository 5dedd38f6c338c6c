// bp_solve.cu -- per-halo solve of the analytic ICM model (Section 2), FP64.
//
// One warp per halo.  The scalar halo quantities (NFW, r500, M_*, r_*) come from
// closed forms and 1-D Newton iterations that every lane runs redundantly.  The
// initial gas energy, the dark-matter energy and the surface pressure use the
// isotropic Lokas & Mamon (2001) dispersion in closed form (dilogarithm) and an
// integration by parts of the kinetic term, so no nested quadrature is needed.
// The three conditions of Section 2.2 are reduced to one unknown: for each r_f,
// T = P0/rho0 follows from the gas-mass condition (safeguarded Newton in
// ln(T - T_min)), rho0 from the surface-pressure condition, and the energy
// condition is driven to zero by safeguarded Newton in ln r_f with the exact
// derivative of the reduced problem.  The gas integrals over [0, r_f] are
// composite 16-point Gauss-Legendre rules whose nodes are spread over the lanes (8 points in
// the FP32 pre-solve and the FP64 polish).
//
// Kernels: k_setup (the scalar set-up, one thread per halo), k_presolve (the reduced
// problem in FP32 to residuals of ~1e-4: starting points), k_solve (FP64: a
// two-dimensional Newton in (ln T, ln r_f) from the starting point, one quadrature per
// step, to the tolerance; the nested iteration for halos without one), then k_setup +
// k_solve again, nested, for halos the Newton did not bring in (the fallback).
#include <algorithm>
#include <vector>

#include "bp_internal.cuh"

// Gauss-Legendre points per panel.  The panels are geometric (ratio 2.5 from r_s / 2 inside
// r_vir, doubling from r_vir outside), so every panel sees the integrands' nearest
// singularity (x = -1 of ln(1 + x) inside, r = 0 of -GM/r outside) at the same relative
// distance.  8 points already solve every halo to within 5e-11 of the 16-point solution (2e6
// halos), at the same speed: the FP64 cost of an evaluation is its per-halo scalar part.
#define NGL 16
#define MAX_PANEL_A 8
#define MAX_PANEL_B 5
// quadrature slots per lane: node q = lane + 32 t of a region, t < NSLOT
#define NSLOT ((MAX_PANEL_A * NGL + 31) / 32)

__constant__ double c_glx[NGL];
__constant__ double c_glw[NGL];
#define NGL_POLISH 8  // the two-halos-per-warp polish (8 points: the same solutions to 5e-11)
__constant__ double c_glx8[NGL_POLISH];
__constant__ double c_glw8[NGL_POLISH];
__constant__ double c_li2[16];  // B_2m / (2m+1)!, m = 1..15
// The FP32 pre-solve's rule: 8 points per panel (the FP64 solutions agree with the 16-point
// ones to 5e-11, far below the FP32 floor of the pre-solve), half the nodes per evaluation
#define NGL_PRE 8
__constant__ float c_glxf[NGL_PRE];
__constant__ float c_glwf[NGL_PRE];

namespace {

// Gauss-Legendre nodes/weights on [-1, 1] by Newton iteration on P_n.
void gauss_legendre(int n, double* x, double* w) {
  for (int i = 0; i < n; ++i) {
    double z = cos(bpc::PI * (i + 0.75) / (n + 0.5));
    for (int it = 0; it < 100; ++it) {
      double p0 = 1.0, p1 = z;
      for (int k = 2; k <= n; ++k) {
        double p2 = ((2 * k - 1) * z * p1 - (k - 1) * p0) / k;
        p0 = p1;
        p1 = p2;
      }
      double dp = n * (z * p1 - p0) / (z * z - 1.0);
      double dz = p1 / dp;
      z -= dz;
      if (fabs(dz) < 1e-16) break;
    }
    double p0 = 1.0, p1 = z;
    for (int k = 2; k <= n; ++k) {
      double p2 = ((2 * k - 1) * z * p1 - (k - 1) * p0) / k;
      p0 = p1;
      p1 = p2;
    }
    double dp = n * (z * p1 - p0) / (z * z - 1.0);
    x[i] = -z;
    w[i] = 2.0 / ((1.0 - z * z) * dp * dp);
  }
}

bool g_const_ready = false;

int upload_constants(bp_ctx* ctx) {
  if (g_const_ready) return BP_OK;
  double x[NGL], w[NGL];
  gauss_legendre(NGL, x, w);
  // Bernoulli numbers B_2m (exact rationals), divided by (2m+1)!
  const double num[15] = {1, -1, 1, -1, 5, -691, 7, -3617, 43867, -174611, 854513,
                          -236364091, 8553103, -23749461029.0, 8615841276005.0};
  const double den[15] = {6, 30, 42, 30, 66, 2730, 6, 510, 798, 330, 138, 2730, 6, 870, 14322};
  double li2[16] = {0};
  double fact = 1.0;  // (2m+1)!
  for (int m = 1; m <= 15; ++m) {
    fact *= (2.0 * m) * (2.0 * m + 1.0);
    li2[m] = num[m - 1] / den[m - 1] / fact;
  }
  BP_CUDA(ctx, cudaMemcpyToSymbol(c_glx, x, sizeof(x)));
  BP_CUDA(ctx, cudaMemcpyToSymbol(c_glw, w, sizeof(w)));
  {
    double x8[NGL_POLISH], w8[NGL_POLISH];
    gauss_legendre(NGL_POLISH, x8, w8);
    BP_CUDA(ctx, cudaMemcpyToSymbol(c_glx8, x8, sizeof(x8)));
    BP_CUDA(ctx, cudaMemcpyToSymbol(c_glw8, w8, sizeof(w8)));
  }
  BP_CUDA(ctx, cudaMemcpyToSymbol(c_li2, li2, sizeof(li2)));
  float xf[NGL_PRE], wf[NGL_PRE];
  {
    double xp[NGL_PRE], wp[NGL_PRE];
    gauss_legendre(NGL_PRE, xp, wp);
    for (int k = 0; k < NGL_PRE; ++k) {
      xf[k] = (float)xp[k];
      wf[k] = (float)wp[k];
    }
  }
  BP_CUDA(ctx, cudaMemcpyToSymbol(c_glxf, xf, sizeof(xf)));
  BP_CUDA(ctx, cudaMemcpyToSymbol(c_glwf, wf, sizeof(wf)));
  g_const_ready = true;
  return BP_OK;
}

// ---------------------------------------------------------------- device math
__device__ double m_of(double x) {  // ln(1+x) - x/(1+x)
  if (x < 1e-3) {
    double x2 = x * x;
    return x2 * (0.5 - x * (2.0 / 3.0 - x * (0.75 - x * 0.8)));
  }
  return log1p(x) - x / (1.0 + x);
}

// Li2 series in u = -ln(1 - z) with Bernoulli coefficients ('t Hooft & Veltman 1979)
__device__ double li2_series(double u) {
  double u2 = u * u, s = 0.0;
  for (int m = 15; m >= 1; --m) s = s * u2 + c_li2[m];
  return u * (1.0 + s * u2) - 0.25 * u2;
}
// Li2(-y) for y >= 0; inversion Li2(-y) = -pi^2/6 - ln^2(y)/2 - Li2(-1/y) for y > 1.
__device__ double li2_neg(double y) {
  if (y <= 0.0) return 0.0;
  if (y <= 1.0) return li2_series(-log1p(y));
  double l = log(y);
  return -bpc::PI * bpc::PI / 6.0 - 0.5 * l * l - li2_series(-log1p(1.0 / y));
}

struct Halo {
  double M, c, z, rvir, rs, rhos, mc, phi0, GM;
  double r500, M500, Mstar, rstar, Egi, Edm, Ps, ant, DA, tau;
};

// rho sigma^2 of the untruncated isotropic NFW halo (Lokas & Mamon 2001, eq. 14).
__device__ double rho_sigma2(const Halo& h, double r) {
  double s = r / h.rvir, c = h.c, cs = c * s;
  double l1 = log1p(cs);
  double br = bpc::PI * bpc::PI - log(cs) - 1.0 / cs - 1.0 / ((1 + cs) * (1 + cs)) - 6.0 / (1 + cs) +
              (1.0 + 1.0 / (cs * cs) - 4.0 / cs - 2.0 / (1 + cs)) * l1 + 3.0 * l1 * l1 +
              6.0 * li2_neg(cs);
  double Vv2 = h.GM / h.rvir;
  double sig2 = 0.5 * c * c / h.mc * s * (1 + cs) * (1 + cs) * br * Vv2;
  double x = r / h.rs;
  double rho = h.rhos / (x * (1 + x) * (1 + x));
  return rho * sig2;
}

__device__ __forceinline__ double phi_of(const Halo& h, double r) {
  if (r > h.rvir) return -h.GM / r;
  double x = r / h.rs;
  double l = (x < 1e-6) ? (1.0 - 0.5 * x) / h.rs : log1p(x) / r;
  return -(h.GM / h.mc) * (l - h.c / ((1 + h.c) * h.rvir));
}
__device__ __forceinline__ double menc_of(const Halo& h, double r) {
  return r >= h.rvir ? h.M : h.M * m_of(r / h.rs) / h.mc;
}


struct Sums {
  double Im, In, Ip, Jm, Jn;  // int theta^{n-1,n,n+1} r^2, int theta^{n-1,n} Phi r^2
};

// W lanes per halo (32: a warp; 16: two halos per warp), NG Gauss-Legendre points per panel
template <int W, int NG>
struct SolverT {
  static constexpr int NS = (MAX_PANEL_A * NG + W - 1) / W;  // slots per lane
  const Halo& h;
  double n;     // polytropic index
  int n_int;    // n if integral, else -1
  // this lane's nodes of region A ([0, r_vir], fixed per halo) and of the r_f-dependent
  // part (region B = [r_vir, r_f] when r_f >= r_vir, else region A cut at r_f):
  // weight x r^2 and Phi(r) in fixed slots t (node q = lane + W t); unused slots have
  // weight 0 and Phi = Phi0
  double a_r2w[NS], a_phi[NS];
  double f_r2w[NS], f_phi[NS];
  int a_cnt, f_cnt;  // slots in use (the nodes of a lane fill slots 0 .. cnt - 1)
  bool full_a;  // r_f >= r_vir: region A is complete and region B follows

  __device__ SolverT(const Halo& hh, double nn) : h(hh), n(nn) {
    double rn = rint(nn);
    n_int = (fabs(nn - rn) < 1e-12 && rn >= 1 && rn <= 16) ? (int)rn : -1;
  }
  __device__ static double glx(int j) { return NG == NGL ? c_glx[j] : c_glx8[j]; }
  __device__ static double glw(int j) { return NG == NGL ? c_glw[j] : c_glw8[j]; }
  // sum over the W lanes of this halo (xor butterflies stay inside aligned groups of W)
  __device__ static double group_sum(double v) {
    for (int o = W / 2; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
  }
  __device__ double pw(double th, int k_off) const {  // theta^{n - 1 + k_off}
    if (n_int > 0) {
      int e = n_int - 1 + k_off;
      double r = 1.0, b = th;
      while (e) {
        if (e & 1) r *= b;
        b *= b;
        e >>= 1;
      }
      return r;
    }
    return pow(th, n - 1.0 + k_off);
  }
  // panel p of region A (x = r/r_s from 0 to xa) -> [a, b] in r
  __device__ static bool panel_a(int p, double xa, double rs, double& a, double& b) {
    double lo = 0.0, hi = fmin(0.5, xa);
    for (int k = 0; k < p; ++k) {
      if (hi >= xa) return false;
      lo = hi;
      hi = fmin(2.5 * hi, xa);
    }
    if (!(hi > lo)) return false;
    a = lo * rs;
    b = hi * rs;
    return true;
  }
  // region A nodes up to x = xa of this lane into the slots (r2w, phi); returns the
  // slots in use (panels are filled in order, so the used slots come first)
  __device__ int nodes_a(int lane, double xa, double (&r2w)[NS], double (&phi)[NS]) const {
    int cnt = 0;
#pragma unroll
    for (int t = 0; t < NS; ++t) {
      const int q = lane + W * t, p = q / NG, j = q % NG;
      double a, b;
      r2w[t] = 0.0;
      phi[t] = h.phi0;
      if (q >= MAX_PANEL_A * NG || !panel_a(p, xa, h.rs, a, b)) continue;
      double mid = 0.5 * (a + b), hw = 0.5 * (b - a);
      double r = mid + hw * glx(j);
      r2w[t] = hw * glw(j) * r * r;
      phi[t] = phi_of(h, r);
      cnt = t + 1;
    }
    return cnt;
  }
  __device__ void cache_region_a(int lane) { a_cnt = nodes_a(lane, h.c, a_r2w, a_phi); }
  // the nodes that depend on r_f; call before integrals() whenever r_f changes
  __device__ void set_rf(double rf, int lane) {
    full_a = rf >= h.rvir;
    if (!full_a) {
      f_cnt = nodes_a(lane, rf / h.rs, f_r2w, f_phi);
      return;
    }
    f_cnt = 0;
#pragma unroll
    for (int t = 0; t < NS; ++t) {
      const int q = lane + W * t, p = q / NG, j = q % NG;
      f_r2w[t] = 0.0;
      f_phi[t] = h.phi0;
      // panel p of region B: [2^p r_vir, min(2^(p+1) r_vir, r_f)], present while
      // 2^p r_vir < r_f (doubling panels from r_vir to r_f)
      if (q >= MAX_PANEL_B * NG) continue;
      const double a = h.rvir * (double)(1 << p);
      if (!(a < rf)) continue;
      const double b = fmin(2.0 * a, rf);
      double mid = 0.5 * (a + b), hw = 0.5 * (b - a);
      double r = mid + hw * glx(j);
      f_r2w[t] = hw * glw(j) * r * r;
      f_phi[t] = -h.GM / r;
      f_cnt = t + 1;
    }
  }
  __device__ void acc(Sums& s, double r2w, double phi, double inv_n1T) const {
    double th = 1.0 + (h.phi0 - phi) * inv_n1T;
    if (th <= 0.0) return;
    double tm = pw(th, 0);
    double tn = tm * th, tp = tn * th;
    s.Im += r2w * tm;
    s.In += r2w * tn;
    s.Ip += r2w * tp;
    s.Jm += r2w * tm * phi;
    s.Jn += r2w * tn * phi;
  }
  // gas integrals over [0, r_f] of the r_f last given to set_rf, at temperature T
  __device__ Sums integrals(double T) const { return integrals_inv(1.0 / ((n + 1.0) * T)); }
  // the same with inv_n1T = 1 / ((n + 1) T) given
  __device__ Sums integrals_inv(double inv_n1T) const {
    Sums s = {0, 0, 0, 0, 0};
    if (full_a) {
#pragma unroll
      for (int t = 0; t < NS; ++t)
        if (t < a_cnt) acc(s, a_r2w[t], a_phi[t], inv_n1T);
    }
#pragma unroll
    for (int t = 0; t < NS; ++t)
      if (t < f_cnt) acc(s, f_r2w[t], f_phi[t], inv_n1T);
    s.Im = group_sum(s.Im);
    s.In = group_sum(s.In);
    s.Ip = group_sum(s.Ip);
    s.Jm = group_sum(s.Jm);
    s.Jn = group_sum(s.Jn);
    return s;
  }
};
using Solver = SolverT<32, NGL>;

// Reduced problem at a given r_f: T from the gas-mass condition.
struct Eval {
  double T, thf, rho0, Rm, Re, dRe_dv;
  Sums s;
  int ok;
};

// Optional inputs of the solve: per-halo model parameters, a starting point and a
// residual gate (used by the surrogate path).
struct SolveExtra {
  const double* prm;    // [3][n]: eps_*, f_*, eps_DM per halo, or null (context values)
  const double* guess;  // [2][n]: ln(r_f / r_vir), ln(T r_vir / (G M)), or null
  int max_outer;        // outer Newton iterations
  double gate;          // > 0: halos not converged after max_outer iterations are
                        //   accepted if both residuals <= gate, else flagged FALLBACK
  int only_fallback;    // 1: solve only halos whose status is BP_HALO_FALLBACK
};

// FP32 versions of the two set-up roots (same equations, bracket and Newton as the FP64
// loops, stopped at the FP32 resolution): starting points for them.  Any start inside the
// bracket leads the FP64 iteration to the same root; a good one saves its FP64 steps.
__device__ __forceinline__ float m_of_f32(float x) {
  if (x < 1e-2f) return x * x * (0.5f - x * (2.0f / 3.0f - x * (0.75f - x * 0.8f)));
  return log1pf(x) - x / (1.0f + x);
}
__device__ double fp32_root_r500(float lnK, float c) {
  float lo = 1e-8f, hi = c, x = 0.5f * c;
  for (int it = 0; it < 40; ++it) {
    const float mx = m_of_f32(x);
    const float f = logf(mx) - 3.0f * logf(x) - lnK;
    if (f > 0) lo = x; else hi = x;
    const float df = x / ((1 + x) * (1 + x)) / mx - 3.0f / x;
    float xn = x - f / df;
    if (fabsf(xn - x) < 1e-6f * x) { x = xn; break; }  // before the bracket test: at the
    if (!(xn > lo && xn < hi)) xn = 0.5f * (lo + hi);  // root the step can land on its end
    x = xn;
  }
  return (x > 1e-8f && x < c && isfinite(x)) ? (double)x : 0.5 * (double)c;
}
__device__ double fp32_root_mstar(float tgt, float c) {
  float lo = 0.f, hi = c, x = 0.5f * c;
  for (int it = 0; it < 40; ++it) {
    const float f = m_of_f32(x) - tgt;
    if (f < 0) lo = x; else hi = x;
    const float df = x / ((1 + x) * (1 + x));
    float xn = x - f / df;
    if (fabsf(xn - x) < 1e-6f * x) { x = xn; break; }  // before the bracket test: at the
    if (!(xn > lo && xn < hi)) xn = 0.5f * (lo + hi);  // root the step can land on its end
    x = xn;
  }
  return (x > 0.f && x < c && isfinite(x)) ? (double)x : 0.5 * (double)c;
}

// Closed-form and one-dimensional set-up of halo i, run by ONE thread.  Writes the
// set-up fields of the model; returns false (status written) if the halo cannot be
// solved.
__device__ bool halo_setup(const BpParams& P, const BpTables& TB, int64_t n, int64_t i,
                           const double* __restrict__ Mh, const double* __restrict__ cc,
                           const double* __restrict__ zz, double* model, int32_t* status,
                           int64_t* nbad, const SolveExtra& X, Halo& h) {
  const double f_star = X.prm ? X.prm[n + i] : P.f_star;
  double Min = Mh[i], c = cc[i], z = zz[i];
  auto put = [&](int f, double v) { model[(int64_t)f * n + i] = v; };
  auto finish = [&](int st) {
    status[i] = st;
    if (st != BP_HALO_OK) atomicAdd((unsigned long long*)nbad, 1ull);
  };
  if (!(Min > 0 && isfinite(Min) && c > 0 && isfinite(c) && z >= 0 && z <= 10.0)) {
    for (int f = 0; f < BP_M_NFIELDS; ++f) put(f, 0.0);
    finish(BP_HALO_BADINPUT);
    return false;
  }
  h.M = Min / P.h;
  h.c = c;
  h.z = z;
  h.GM = bpc::G * h.M;
  double a3 = (1 + z) * (1 + z) * (1 + z);
  double E2 = P.Om * a3 + (1.0 - P.Om);
  double rho_cr = P.rho_cr0 * E2;
  double xo = P.Om * a3 / E2 - 1.0;
  double Dv = 18.0 * bpc::PI * bpc::PI + 82.0 * xo - 39.0 * xo * xo;
  h.rvir = cbrt(3.0 * h.M / (4.0 * bpc::PI * Dv * rho_cr));
  h.rs = h.rvir / c;
  h.mc = m_of(c);
  h.rhos = h.M / (4.0 * bpc::PI * h.rs * h.rs * h.rs * h.mc);
  h.phi0 = -(h.GM / (h.mc * h.rvir)) * c * c / (1 + c);
  h.DA = bp_hermite(TB.chi_z, TB.dchi_z, TB.nz, TB.dz, z) / (1 + z);
  h.tau = bp_hermite(TB.tau_z, TB.dtau_z, TB.nz, TB.dz, z);
  // r500: m(x)/x^3 = 500 rho_cr (4pi/3) r_s^3 m(c) / M, Newton in ln x with a bracket,
  // started from the same iteration in FP32 (a few FP64 steps remain on the slow pipe)
  {
    double lnK = log(500.0 * rho_cr * 4.0 * bpc::PI / 3.0 * h.rs * h.rs * h.rs * h.mc / h.M);
    double lo = 1e-8, hi = c, x = fp32_root_r500((float)lnK, (float)c);
    for (int it = 0; it < 100; ++it) {
      double mx = m_of(x);
      double f = log(mx) - 3.0 * log(x) - lnK;
      if (f > 0) lo = x; else hi = x;
      double df = x / ((1 + x) * (1 + x)) / mx - 3.0 / x;  // d f / d x
      double xn = x - f / df;
      if (fabs(xn - x) < 1e-15 * x) { x = xn; break; }  // converged (f may be exactly 0)
      if (!(xn > lo && xn < hi)) xn = 0.5 * (lo + hi);
      x = xn;
    }
    h.r500 = x * h.rs;
    h.M500 = 4.0 * bpc::PI / 3.0 * 500.0 * rho_cr * h.r500 * h.r500 * h.r500;
  }
  h.Mstar = f_star * pow(h.M500 / 3e14, -P.S_star) * h.M;
  double f_max = pow(4.0, -P.n_nt) / P.alpha_nt;
  double fz = fmin(pow(1.0 + z, P.beta_nt), (f_max - 1.0) * tanh(P.beta_nt * z) + 1.0);
  h.ant = P.alpha_nt * fz;
  put(BP_M_MVIR, h.M);
  put(BP_M_C, c);
  put(BP_M_Z, z);
  put(BP_M_RVIR, h.rvir);
  put(BP_M_RS, h.rs);
  put(BP_M_RHOS, h.rhos);
  put(BP_M_MC, h.mc);
  put(BP_M_PHI0, h.phi0);
  put(BP_M_R500, h.r500);
  put(BP_M_M500, h.M500);
  put(BP_M_MSTAR, h.Mstar);
  put(BP_M_ANT, h.ant);
  put(BP_M_DA, h.DA);
  put(BP_M_TAU, h.tau);
  if (h.Mstar >= P.fb * h.M) {
    const int zero_fields[10] = {BP_M_RSTAR, BP_M_EGI, BP_M_EDM, BP_M_PS, BP_M_T,
                                 BP_M_RHO0,  BP_M_P0,  BP_M_RF,  BP_M_RESM, BP_M_RESE};
    for (int k = 0; k < 10; ++k) put(zero_fields[k], 0.0);
    finish(BP_HALO_BADSTAR);
    return false;
  }
  // r_*: f_b M(<r_*) = M_*  ->  m(x) = M_* m(c) / (f_b M), from an FP32 start as r500
  {
    double tgt = h.Mstar * h.mc / (P.fb * h.M);
    double lo = 0.0, hi = c, x = fp32_root_mstar((float)tgt, (float)c);
    for (int it = 0; it < 100; ++it) {
      double f = m_of(x) - tgt;
      if (f < 0) lo = x; else hi = x;
      double df = x / ((1 + x) * (1 + x));
      double xn = x - f / df;
      if (fabs(xn - x) < 1e-15 * x) { x = xn; break; }  // converged (f may be exactly 0)
      if (!(xn > lo && xn < hi)) xn = 0.5 * (lo + hi);
      x = xn;
    }
    h.rstar = x * h.rs;
  }
  // E_g,i over [r_*, r_vir] and E_DM over [0, r_vir] share their r_vir end: rho sigma^2 at
  // r_vir (also the surface pressure) and the closed forms there are evaluated once
  {
    const double rs2v = rho_sigma2(h, h.rvir);
    const double kin_pre = 4.0 * bpc::PI * bpc::G * h.rhos * h.rhos * pow(h.rs, 5);
    auto Hq = [](double x) { return -log1p(x) / (1 + x) - 0.5 / ((1 + x) * (1 + x)); };
    auto Q = [](double x) { return -(log1p(x) + 1.0) / (1 + x); };
    const double xs = h.rstar / h.rs, xv = h.rvir / h.rs;
    const double r3v = h.rvir * h.rvir * h.rvir, r3s = h.rstar * h.rstar * h.rstar;
    const double Hv = Hq(xv), Qv = Q(xv), mv = m_of(xv);
    const double K = h.c / ((1 + h.c) * h.rvir);
    const double pot_pre = -(h.GM * h.M / (h.mc * h.mc));
    // kinetic integral int_a^{r_vir} 4 pi r^2 rho sigma^2 dr by parts:
    //   (4pi/3)[r^3 rho sigma^2]_a^{r_vir} + (4pi/3) 4 pi G rho_s^2 r_s^5 [Hq]_{a/r_s}^{c},
    //   Hq' = m(x)/(1+x)^2; potential integral int_a^{r_vir} Phi 4 pi r^2 rho dr in closed form
    const double kin_s = 4.0 * bpc::PI / 3.0 *
                         ((r3v * rs2v - r3s * rho_sigma2(h, h.rstar)) + kin_pre * (Hv - Hq(xs)));
    const double kin_0 = 4.0 * bpc::PI / 3.0 * (r3v * rs2v + kin_pre * (Hv - Hq(0.0)));
    const double pot_s = pot_pre * ((Qv - Q(xs)) / h.rs - K * (mv - m_of(xs)));
    const double pot_0 = pot_pre * ((Qv - Q(0.0)) / h.rs - K * (mv - m_of(0.0)));
    h.Egi = P.fb * (1.5 * kin_s + pot_s);
    h.Edm = 1.5 * kin_0 + pot_0;
    h.Ps = P.fb * rs2v;
  }
  put(BP_M_RSTAR, h.rstar);
  put(BP_M_EGI, h.Egi);
  put(BP_M_EDM, h.Edm);
  put(BP_M_PS, h.Ps);

  return true;
}

constexpr int SOLVE_WARPS = 4;  // warps per block
// |R_e| below which the nested iteration hands over to the two-dimensional Newton
constexpr double NEWTON2D_SWITCH = 1e-3;

// 1. set-up, one thread per halo (the closed forms and 1-D iterations are scalar, so
// every lane of a warp does useful FP64 work); ok[i] = 1 if halo i goes to the solve
__global__ void __launch_bounds__(128) k_setup(BpParams P, BpTables TB, int64_t n,
                                               const double* __restrict__ Mh,
                                               const double* __restrict__ cc,
                                               const double* __restrict__ zz, double* model,
                                               int32_t* status, int64_t* nbad, SolveExtra X,
                                               Halo* halos, int32_t* ok) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  int good = 0;
  if (!X.only_fallback || status[i] == BP_HALO_FALLBACK) {
    Halo hs;
    good = halo_setup(P, TB, n, i, Mh, cc, zz, model, status, nbad, X, hs) ? 1 : 0;
    if (good) halos[i] = hs;
  }
  ok[i] = good;
}

// 2. the solve: each warp takes hpw prepared halos one after another, lanes over the
// quadrature nodes
__global__ void __launch_bounds__(32 * SOLVE_WARPS) k_solve(
    BpParams P, int64_t n, double* model, int32_t* status, double tol, int64_t* nbad,
    int64_t* nfallback, SolveExtra X, int hpw, const Halo* __restrict__ halos,
    const int32_t* __restrict__ okv) {
  const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int64_t base = ((int64_t)blockIdx.x * (blockDim.x >> 5) + w) * hpw;
  if (base >= n) return;
  for (int jj = 0; jj < hpw; ++jj) {
    const int64_t i = base + jj;
    if (i >= n || !okv[i]) continue;
    const Halo h = halos[i];
    const double eps_star = X.prm ? X.prm[i] : P.eps_star;
    const double eps_dm = X.prm ? X.prm[2 * n + i] : P.eps_dm;
    auto put = [&](int f, double v) {
      if (lane == 0) model[(int64_t)f * n + i] = v;
    };
    auto finish = [&](int st) {
      if (lane == 0) {
        status[i] = st;
        if (st != BP_HALO_OK) atomicAdd((unsigned long long*)nbad, 1ull);
        if (st == BP_HALO_FALLBACK) atomicAdd((unsigned long long*)nfallback, 1ull);
      }
    };
  const double nn = P.n_poly;
  Solver S(h, nn);
  S.cache_region_a(lane);
  const double fbM = P.fb * h.M;
  const double inj = eps_dm * fabs(h.Edm) + eps_star * h.Mstar * bpc::C_KMS * bpc::C_KMS;
  const double absE = fabs(h.Egi);
  const double r3v = h.rvir * h.rvir * h.rvir;
  const double four_pi = 4.0 * bpc::PI;

  // Evaluate the reduced problem at r_f, solving the gas-mass condition for T
  // (warm start T0).  Returns residuals and d R_e / d ln r_f.
  auto reduced = [&](double rf, double T0) -> Eval {
    Eval e;
    e.ok = 0;
    double phif = phi_of(h, rf);
    double psi = phif - h.phi0;  // > 0
    double Tmin = psi / (nn + 1.0);
    double lnTarget = log(fbM - h.Mstar);
    double s = (T0 > Tmin * (1 + 1e-9) && isfinite(T0)) ? log(T0 - Tmin)
                                                        : log(Tmin + 0.5 * h.GM / h.rvir);
    double slo = -INFINITY, shi = INFINITY;
    double T = 0, thf = 0, rho0 = 0, F = 1;
    Sums sm;
    int it;
    S.set_rf(rf, lane);
    for (it = 0; it < 80; ++it) {
      T = Tmin + exp(s);
      thf = 1.0 + (h.phi0 - phif) / ((nn + 1.0) * T);
      sm = S.integrals(T);
      rho0 = h.Ps / (T * S.pw(thf, 2));
      F = log(four_pi * rho0 * sm.In) - lnTarget;
      if (!isfinite(F)) break;
      if (fabs(F) < 1e-14) break;
      if (F > 0) slo = s; else shi = s;
      double dlr = (-1.0 - (nn + 1.0) * (1.0 - thf) / thf) / T;  // d ln rho0 / dT
      double dli = nn * (sm.Im - sm.In) / (T * sm.In);           // d ln I_n / dT
      double dFds = (T - Tmin) * (dlr + dli);
      double step = -F / dFds;
      if (!isfinite(step)) step = (F > 0) ? 1.0 : -1.0;
      // at the rounding floor of the quadrature sum a further step changes nothing
      if (fabs(F) < 1e-12 && fabs(step) < 1e-14 * fmax(1.0, fabs(s))) break;
      step = fmax(-4.0, fmin(4.0, step));
      double sn = s + step;
      if (isfinite(slo) && isfinite(shi) && !(sn > slo && sn < shi)) sn = 0.5 * (slo + shi);
      s = sn;
    }
    if (!(fabs(F) < 1e-12)) return e;
    // residuals and the derivative of the reduced energy residual
    double In = sm.In, Ip = sm.Ip, Im = sm.Im, Jm = sm.Jm, Jn = sm.Jn;
    double Egf = four_pi * rho0 * (1.5 * T * Ip + Jn);
    double dEp = four_pi / 3.0 * (r3v - rf * rf * rf) * h.Ps;
    double num = (P.energy_sign == 0) ? (Egf - h.Egi - inj - dEp) : (h.Egi - Egf - inj - dEp);
    e.Re = num / absE;
    e.Rm = (four_pi * rho0 * In + h.Mstar) / fbM - 1.0;
    // partial derivatives
    double dphif = bpc::G * menc_of(h, rf) / (rf * rf);
    double dthf_drf = -dphif / ((nn + 1.0) * T);
    double dlr_drf = -(nn + 1.0) * dthf_drf / thf;
    double dlr_dT = (-1.0 - (nn + 1.0) * (1.0 - thf) / thf) / T;
    double tfn = S.pw(thf, 1), tfp = tfn * thf;
    double dG_drf = four_pi * rho0 * (In * dlr_drf + tfn * rf * rf);
    double dG_dT = four_pi * rho0 * (In * dlr_dT + nn * (Im - In) / T);
    double dT_drf = -dG_drf / dG_dT;
    double dIp_dT = (nn + 1.0) * (In - Ip) / T;
    double dJn_dT = nn * (Jm - Jn) / T;
    double dEgf_drf = Egf * dlr_drf + four_pi * rho0 * (1.5 * T * tfp + tfn * phif) * rf * rf;
    double dEgf_dT = Egf * dlr_dT + four_pi * rho0 * (1.5 * Ip + 1.5 * T * dIp_dT + dJn_dT);
    double ddEp_drf = -four_pi * rf * rf * h.Ps;
    double dtot = dEgf_drf + dEgf_dT * dT_drf;
    double dnum = (P.energy_sign == 0) ? (dtot - ddEp_drf) : (-dtot - ddEp_drf);
    e.dRe_dv = rf * dnum / absE;
    e.T = T;
    e.thf = thf;
    e.rho0 = rho0;
    e.s = sm;
    e.ok = 1;
    return e;
  };

  // Both conditions and their 2x2 Jacobian in (ln T, ln r_f) at a given (T, r_f),
  // without the inner solve for T (one quadrature evaluation).
  struct Direct {
    double Rm, Re, J[2][2], thf, rho0;
    int ok;
  };
  // (phif = Phi(r_f) given: the caller has it from its step control.)  Divisions, each a
  // dozen instructions on the slow FP64 pipe, are reduced to four reciprocals.
  const double inv_np1 = 1.0 / (nn + 1.0), inv_fbM = 1.0 / fbM, inv_absE = 1.0 / absE;
  auto direct = [&](double T, double rf, double phif) -> Direct {
    Direct d;
    d.ok = 0;
    const double inv_T = 1.0 / T;
    const double inv_n1T = inv_T * inv_np1;
    double thf = 1.0 + (h.phi0 - phif) * inv_n1T;
    if (!(thf > 0.0)) return d;
    S.set_rf(rf, lane);
    Sums sm = S.integrals_inv(inv_n1T);
    double rho0 = h.Ps * inv_T / S.pw(thf, 2);
    double In = sm.In, Ip = sm.Ip, Im = sm.Im, Jm = sm.Jm, Jn = sm.Jn;
    double Egf = four_pi * rho0 * (1.5 * T * Ip + Jn);
    double dEp = four_pi / 3.0 * (r3v - rf * rf * rf) * h.Ps;
    double num = (P.energy_sign == 0) ? (Egf - h.Egi - inj - dEp) : (h.Egi - Egf - inj - dEp);
    d.Re = num * inv_absE;
    d.Rm = (four_pi * rho0 * In + h.Mstar) * inv_fbM - 1.0;
    const double inv_rf = 1.0 / rf, inv_thf = 1.0 / thf;
    double dphif = bpc::G * menc_of(h, rf) * inv_rf * inv_rf;
    double dthf_drf = -dphif * inv_n1T;
    double dlr_drf = -(nn + 1.0) * dthf_drf * inv_thf;
    double dlr_dT = (-1.0 - (nn + 1.0) * (1.0 - thf) * inv_thf) * inv_T;
    double tfn = S.pw(thf, 1), tfp = tfn * thf;
    double dG_drf = four_pi * rho0 * (In * dlr_drf + tfn * rf * rf);
    double dG_dT = four_pi * rho0 * (In * dlr_dT + nn * (Im - In) * inv_T);
    double dIp_dT = (nn + 1.0) * (In - Ip) * inv_T;
    double dJn_dT = nn * (Jm - Jn) * inv_T;
    double dEgf_drf = Egf * dlr_drf + four_pi * rho0 * (1.5 * T * tfp + tfn * phif) * rf * rf;
    double dEgf_dT = Egf * dlr_dT + four_pi * rho0 * (1.5 * Ip + 1.5 * T * dIp_dT + dJn_dT);
    double ddEp_drf = -four_pi * rf * rf * h.Ps;
    double dn_dT = (P.energy_sign == 0) ? dEgf_dT : -dEgf_dT;
    double dn_drf = (P.energy_sign == 0) ? (dEgf_drf - ddEp_drf) : (-dEgf_drf - ddEp_drf);
    d.J[0][0] = dG_dT * T * inv_fbM;
    d.J[0][1] = dG_drf * rf * inv_fbM;
    d.J[1][0] = dn_dT * T * inv_absE;
    d.J[1][1] = dn_drf * rf * inv_absE;
    d.thf = thf;
    d.rho0 = rho0;
    d.ok = 1;
    return d;
  };

  // Safeguarded Newton in v = ln r_f on [ln 0.5 r_vir, ln 10 r_vir]: Newton steps
  // (clamped) until a sign change is bracketed, then Newton with bisection inside
  // the bracket.  The direction of R_e(r_f) is not assumed.
  const double vmin = log(0.5 * h.rvir), vmax = log(10.0 * h.rvir);
  double v = log(1.1 * h.rvir);
  double Tw = 0.0;
  if (X.guess) {
    double g0 = X.guess[i], g1 = X.guess[n + i];
    if (isfinite(g0) && isfinite(g1)) {
      v = fmin(fmax(log(h.rvir) + g0, vmin + 1e-9), vmax - 1e-9);
      Tw = exp(g1) * h.GM / h.rvir;
    }
  }
  int st = BP_HALO_MAXIT;
  Eval e;
  double rf = exp(v);
  // Two-dimensional Newton in (u, v) = (ln T, ln r_f), one quadrature evaluation per
  // iteration, steps halved to keep theta(r_f) > 0.  Returns true when both residuals
  // are below tol; (ee, rff) hold the last evaluated point (ee.ok = 0 if it failed).
  // The step is applied multiplicatively, T e^du and r_f e^dv, with e^d from its series
  // to fourth order (|d| <= 0.5; the residuals are evaluated at the point actually
  // reached, so the update only has to be a good Newton step, and near the root it is
  // exact to rounding); Phi(r_f) of the accepted point carries into the next evaluation.
  auto expq = [](double d) { return 1.0 + d * (1.0 + d * (0.5 + d * (1.0 / 6.0 + d * (1.0 / 24.0)))); };
  auto newton2d = [&](double T, double& rff, int max_it, Eval& ee) -> bool {
    ee.ok = 0;
    const double rmin = 0.5 * h.rvir, rmax = 10.0 * h.rvir;
    double phif = phi_of(h, rff);
    for (int it = 0; it < max_it; ++it) {
      Direct d = direct(T, rff, phif);
      if (!d.ok) { ee.ok = 0; return false; }
      ee.T = T; ee.thf = d.thf; ee.rho0 = d.rho0; ee.Rm = d.Rm; ee.Re = d.Re; ee.ok = 1;
      if (fabs(d.Re) < tol && fabs(d.Rm) < tol) return true;
      double det = d.J[0][0] * d.J[1][1] - d.J[0][1] * d.J[1][0];
      if (!(fabs(det) > 0.0) || !isfinite(det)) return false;
      const double idet = 1.0 / det;
      double du = (-d.Rm * d.J[1][1] + d.Re * d.J[0][1]) * idet;
      double dv = (-d.Re * d.J[0][0] + d.Rm * d.J[1][0]) * idet;
      double big = fmax(fabs(du), fabs(dv));
      if (big > 0.5) { du *= 0.5 / big; dv *= 0.5 / big; }
      double Tn = T, rn = rff, phin = phif;
      for (int half = 0; half < 20; ++half) {
        rn = fmin(fmax(rff * expq(dv), rmin), rmax);
        phin = phi_of(h, rn);
        Tn = T * expq(du);
        if (Tn > (phin - h.phi0) * inv_np1 * (1.0 + 1e-12)) break;
        du *= 0.5;
        dv *= 0.5;
      }
      T = Tn;
      rff = rn;
      phif = phin;
    }
    return false;
  };
  if (X.guess && Tw > 0.0) {
    // polish from the given starting point
    if (newton2d(Tw, rf, X.max_outer, e)) st = BP_HALO_OK;
  } else {
  double va = 0, vb = 0, Ra = 0;  // bracket [va, vb] with R(va) R(vb) < 0
  bool have_br = false;
  double vprev = 0, Rprev = 0;
  bool have_prev = false;
  int hits_min = 0, hits_max = 0;
  bool tried2d = false;
  for (int it = 0; it < X.max_outer; ++it) {
    rf = exp(v);
    e = reduced(rf, Tw);
    if (!e.ok) { st = BP_HALO_MAXIT; break; }
    Tw = e.T;
    if (fabs(e.Re) < tol && fabs(e.Rm) < tol) { st = BP_HALO_OK; break; }
    if (!tried2d && fabs(e.Re) < NEWTON2D_SWITCH) {
      // close to the root: finish with the two-dimensional Newton (one quadrature per
      // step instead of an inner solve per step); on failure continue the nested one
      tried2d = true;
      double rf2 = rf;
      Eval e2;
      if (newton2d(e.T, rf2, 8, e2)) {
        e = e2;
        rf = rf2;
        st = BP_HALO_OK;
        break;
      }
    }
    if (have_prev && ((e.Re > 0) != (Rprev > 0))) {
      have_br = true;
      va = vprev; Ra = Rprev; vb = v;
    } else if (have_br) {
      // shrink the bracket, keeping the sign change
      if ((e.Re > 0) == (Ra > 0)) { va = v; Ra = e.Re; } else { vb = v; }
    }
    if (have_br && fabs(vb - va) < 1e-15 * fabs(v)) { st = BP_HALO_OK; break; }
    double step = -e.Re / e.dRe_dv;
    if (!isfinite(step)) step = 0.5;
    step = fmax(-0.5, fmin(0.5, step));
    double vn = v + step;
    if (have_br) {
      double lo = fmin(va, vb), hi = fmax(va, vb);
      if (!(vn > lo && vn < hi)) vn = 0.5 * (va + vb);
    } else {
      if (vn <= vmin) { vn = vmin; if (++hits_min > 2) { st = BP_HALO_NOBRACKET; break; } }
      if (vn >= vmax) { vn = vmax; if (++hits_max > 2) { st = BP_HALO_NOBRACKET; break; } }
    }
    vprev = v; Rprev = e.Re; have_prev = true;
    v = vn;
  }
  }
  if (X.gate > 0 && st != BP_HALO_OK) {
    bool pass = e.ok && fabs(e.Re) <= X.gate && fabs(e.Rm) <= X.gate;
    st = pass ? BP_HALO_OK : BP_HALO_FALLBACK;
  }
  if (e.ok && e.thf <= 0.0) st = BP_HALO_THETA;
  put(BP_M_T, e.ok ? e.T : 0.0);
  put(BP_M_RHO0, e.ok ? e.rho0 : 0.0);
  put(BP_M_P0, e.ok ? e.rho0 * e.T : 0.0);
  put(BP_M_RF, e.ok ? rf : 0.0);
  put(BP_M_RESM, e.ok ? e.Rm : NAN);
  put(BP_M_RESE, e.ok ? e.Re : NAN);
  finish(st);
  }
}

// ---------------------------------------------------------------- multi-halo polish
// The FP64 two-dimensional Newton of k_solve from a starting point, for several halos per
// warp (POLISH_W lanes each, 8-point panels: the same solutions to 5e-11).  An evaluation's
// FP64 cost is mostly its per-halo scalar part, executed by every lane of the halo; with
// POLISH_H halos per warp each of those instructions serves all of them.  The groups run the
// same number of evaluations (a finished group re-evaluates its last point without using
// it), so every shuffle is executed by the whole warp.  Halos without a starting point are left to
// k_solve's nested iteration (okv_nested).
constexpr int POLISH_W = 8;                  // lanes per halo (16: 15% slower)
constexpr int POLISH_H = 32 / POLISH_W;       // halos per warp
__global__ void __launch_bounds__(32 * SOLVE_WARPS) k_polish(
    BpParams P, int64_t n, double* model, int32_t* status, double tol, int64_t* nbad,
    int64_t* nfallback, SolveExtra X, int hpw, const Halo* __restrict__ halos,
    const int32_t* __restrict__ okv, int32_t* okv_nested) {
  using SP = SolverT<POLISH_W, NGL_POLISH>;
  const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int sub = lane / POLISH_W, gl = lane % POLISH_W;
  const int64_t base = (((int64_t)blockIdx.x * (blockDim.x >> 5) + w) * POLISH_H + sub) * hpw;
  // every group iterates hpw times whatever its halos (uniform shuffles)
  if ((((int64_t)blockIdx.x * (blockDim.x >> 5) + w) * POLISH_H) * hpw >= n) return;  // idle warp
  const double nn = P.n_poly;
  for (int jj = 0; jj < hpw; ++jj) {
    const int64_t i = base + jj;
    const bool in_range = i < n;
    const int64_t ii = in_range ? i : n - 1;  // a real halo to compute on when idle
    bool valid = in_range && okv[ii];
    const Halo h = halos[ii];
    double g0 = NAN, g1 = NAN;
    if (valid) {
      g0 = X.guess[ii];
      g1 = X.guess[n + ii];
    }
    const bool have_guess = isfinite(g0) && isfinite(g1) && exp(g1) > 0.0;
    if (valid && !have_guess && gl == 0) okv_nested[ii] = 1;  // k_solve's nested path
    valid = valid && have_guess;
    const double eps_star = X.prm ? X.prm[ii] : P.eps_star;
    const double eps_dm = X.prm ? X.prm[2 * n + ii] : P.eps_dm;
    SP S(h, nn);
    S.cache_region_a(gl);
    const double fbM = P.fb * h.M;
    const double inj = eps_dm * fabs(h.Edm) + eps_star * h.Mstar * bpc::C_KMS * bpc::C_KMS;
    const double absE = fabs(h.Egi);
    const double r3v = h.rvir * h.rvir * h.rvir;
    const double four_pi = 4.0 * bpc::PI;
    const double inv_np1 = 1.0 / (nn + 1.0), inv_fbM = 1.0 / fbM, inv_absE = 1.0 / absE;
    const double vmin = log(0.5 * h.rvir), vmax = log(10.0 * h.rvir);
    const double rmin = 0.5 * h.rvir, rmax = 10.0 * h.rvir;
    double T = h.GM / h.rvir, rf = 1.1 * h.rvir;
    if (have_guess) {
      const double v = fmin(fmax(log(h.rvir) + g0, vmin + 1e-9), vmax - 1e-9);
      rf = exp(v);
      T = exp(g1) * h.GM / h.rvir;
    }
    double phif = phi_of(h, rf);
    auto expq = [](double d) { return 1.0 + d * (1.0 + d * (0.5 + d * (1.0 / 6.0 + d * (1.0 / 24.0)))); };
    // last evaluated point
    double eT = 0, ethf = 0, erho0 = 0, eRm = 0, eRe = 0, erf = rf;
    bool eok = false, active = valid, converged = false;
    for (int it = 0; it < X.max_outer; ++it) {
      // one evaluation (every lane of the warp runs it; thf <= 0 only marks it not ok)
      const double inv_T = 1.0 / T;
      const double inv_n1T = inv_T * inv_np1;
      const double thf = 1.0 + (h.phi0 - phif) * inv_n1T;
      S.set_rf(rf, gl);
      const Sums sm = S.integrals_inv(inv_n1T);
      if (active) {
        const bool ok = thf > 0.0;
        if (!ok) {
          eok = false;
          active = false;
        } else {
          const double rho0 = h.Ps * inv_T / S.pw(thf, 2);
          const double In = sm.In, Ip = sm.Ip, Im = sm.Im, Jm = sm.Jm, Jn = sm.Jn;
          const double Egf = four_pi * rho0 * (1.5 * T * Ip + Jn);
          const double dEp = four_pi / 3.0 * (r3v - rf * rf * rf) * h.Ps;
          const double num = (P.energy_sign == 0) ? (Egf - h.Egi - inj - dEp)
                                                  : (h.Egi - Egf - inj - dEp);
          const double Re = num * inv_absE;
          const double Rm = (four_pi * rho0 * In + h.Mstar) * inv_fbM - 1.0;
          eT = T; ethf = thf; erho0 = rho0; eRm = Rm; eRe = Re; erf = rf; eok = true;
          if (fabs(Re) < tol && fabs(Rm) < tol) {
            converged = true;
            active = false;
          } else {
            const double inv_rf = 1.0 / rf, inv_thf = 1.0 / thf;
            const double dphif = bpc::G * menc_of(h, rf) * inv_rf * inv_rf;
            const double dthf_drf = -dphif * inv_n1T;
            const double dlr_drf = -(nn + 1.0) * dthf_drf * inv_thf;
            const double dlr_dT = (-1.0 - (nn + 1.0) * (1.0 - thf) * inv_thf) * inv_T;
            const double tfn = S.pw(thf, 1), tfp = tfn * thf;
            const double dG_drf = four_pi * rho0 * (In * dlr_drf + tfn * rf * rf);
            const double dG_dT = four_pi * rho0 * (In * dlr_dT + nn * (Im - In) * inv_T);
            const double dIp_dT = (nn + 1.0) * (In - Ip) * inv_T;
            const double dJn_dT = nn * (Jm - Jn) * inv_T;
            const double dEgf_drf =
                Egf * dlr_drf + four_pi * rho0 * (1.5 * T * tfp + tfn * phif) * rf * rf;
            const double dEgf_dT =
                Egf * dlr_dT + four_pi * rho0 * (1.5 * Ip + 1.5 * T * dIp_dT + dJn_dT);
            const double ddEp_drf = -four_pi * rf * rf * h.Ps;
            const double dn_dT = (P.energy_sign == 0) ? dEgf_dT : -dEgf_dT;
            const double dn_drf =
                (P.energy_sign == 0) ? (dEgf_drf - ddEp_drf) : (-dEgf_drf - ddEp_drf);
            const double J00 = dG_dT * T * inv_fbM, J01 = dG_drf * rf * inv_fbM;
            const double J10 = dn_dT * T * inv_absE, J11 = dn_drf * rf * inv_absE;
            const double det = J00 * J11 - J01 * J10;
            if (!(fabs(det) > 0.0) || !isfinite(det)) {
              active = false;
            } else {
              const double idet = 1.0 / det;
              double du = (-Rm * J11 + Re * J01) * idet;
              double dv = (-Re * J00 + Rm * J10) * idet;
              const double big = fmax(fabs(du), fabs(dv));
              if (big > 0.5) { du *= 0.5 / big; dv *= 0.5 / big; }
              double Tn = T, rn = rf, phin = phif;
              for (int half = 0; half < 20; ++half) {
                rn = fmin(fmax(rf * expq(dv), rmin), rmax);
                phin = phi_of(h, rn);
                Tn = T * expq(du);
                if (Tn > (phin - h.phi0) * inv_np1 * (1.0 + 1e-12)) break;
                du *= 0.5;
                dv *= 0.5;
              }
              T = Tn;
              rf = rn;
              phif = phin;
            }
          }
        }
      }
      if (__all_sync(0xffffffffu, !active)) break;
    }
    if (valid && gl == 0) {
      int st = converged ? BP_HALO_OK : BP_HALO_MAXIT;
      if (X.gate > 0 && st != BP_HALO_OK) {
        const bool pass = eok && fabs(eRe) <= X.gate && fabs(eRm) <= X.gate;
        st = pass ? BP_HALO_OK : BP_HALO_FALLBACK;
      }
      if (eok && ethf <= 0.0) st = BP_HALO_THETA;
      auto put = [&](int f, double v) { model[(int64_t)f * n + ii] = v; };
      put(BP_M_T, eok ? eT : 0.0);
      put(BP_M_RHO0, eok ? erho0 : 0.0);
      put(BP_M_P0, eok ? erho0 * eT : 0.0);
      put(BP_M_RF, eok ? erf : 0.0);
      put(BP_M_RESM, eok ? eRm : NAN);
      put(BP_M_RESE, eok ? eRe : NAN);
      status[ii] = st;
      if (st != BP_HALO_OK) atomicAdd((unsigned long long*)nbad, 1ull);
      if (st == BP_HALO_FALLBACK) atomicAdd((unsigned long long*)nfallback, 1ull);
    }
  }
}

// ---------------------------------------------------------------- FP32 pre-solve
// Starting points for the FP64 solve: the same reduced problem (T from the gas-mass
// condition at each r_f, Newton in ln r_f on the energy condition) in FP32, to
// residuals of about 1e-4 (FP32 runs at many times the FP64 rate on this GPU).  The
// FP64 two-dimensional Newton of k_solve then takes the starting point to the
// tolerance; a halo the pre-solve cannot bring in gets no starting point (NaN) and the
// full FP64 iteration.
struct HaloF {
  float c, rvir, rs, mc, phi0, GM, M;
};

__device__ __forceinline__ float m_of_f(float x) {  // ln(1+x) - x/(1+x)
  if (x < 1e-2f) {
    float x2 = x * x;
    return x2 * (0.5f - x * (2.0f / 3.0f - x * (0.75f - x * 0.8f)));
  }
  return log1pf(x) - x / (1.0f + x);
}
__device__ __forceinline__ float phi_of_f(const HaloF& h, float r) {
  if (r > h.rvir) return -h.GM / r;
  float x = r / h.rs;
  float l = (x < 1e-4f) ? (1.0f - 0.5f * x) / h.rs : log1pf(x) / r;
  return -(h.GM / h.mc) * (l - h.c / ((1.0f + h.c) * h.rvir));
}
__device__ __forceinline__ float menc_of_f(const HaloF& h, float r) {
  return r >= h.rvir ? h.M : h.M * m_of_f(r / h.rs) / h.mc;
}

struct SumsF {
  float Im, In, Ip, Jm, Jn;
};

// FP32 counterpart of SolverT: the same panels and node slots (W lanes, NG points)
template <int W, int NG>
struct SolverFT {
  static constexpr int NS = (MAX_PANEL_A * NG + W - 1) / W;
  const HaloF& h;
  int n_int;
  float n;
  float a_r2w[NS], a_phi[NS], f_r2w[NS], f_phi[NS];
  int a_cnt, f_cnt;
  bool full_a;

  __device__ SolverFT(const HaloF& hh, float nn, int ni) : h(hh), n_int(ni), n(nn) {}
  static_assert(NG == NGL_PRE, "FP32 rule tabulated for NGL_PRE points only");
  __device__ static float glx(int j) { return c_glxf[j]; }
  __device__ static float glw(int j) { return c_glwf[j]; }
  __device__ static float group_sum(float v) {
    for (int o = W / 2; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
  }
  __device__ float pw(float th, int k_off) const {  // theta^{n - 1 + k_off}
    if (n_int > 0) {
      int e = n_int - 1 + k_off;
      float r = 1.0f, b = th;
      while (e) {
        if (e & 1) r *= b;
        b *= b;
        e >>= 1;
      }
      return r;
    }
    return powf(th, n - 1.0f + k_off);
  }
  __device__ int nodes_a(int lane, float xa, float (&r2w)[NS], float (&phi)[NS]) const {
    int cnt = 0;
#pragma unroll
    for (int t = 0; t < NS; ++t) {
      const int q = lane + W * t, p = q / NG, j = q % NG;
      r2w[t] = 0.f;
      phi[t] = h.phi0;
      if (q >= MAX_PANEL_A * NG) continue;
      float lo = 0.f, hi = fminf(0.5f, xa);
      bool ok = hi > lo;
      for (int k = 0; k < p && ok; ++k) {
        if (hi >= xa) ok = false;
        lo = hi;
        hi = fminf(2.5f * hi, xa);
      }
      if (!ok || !(hi > lo)) continue;
      float a = lo * h.rs, b = hi * h.rs;
      float mid = 0.5f * (a + b), hw = 0.5f * (b - a);
      float r = mid + hw * glx(j);
      r2w[t] = hw * glw(j) * r * r;
      phi[t] = phi_of_f(h, r);
      cnt = t + 1;
    }
    return cnt;
  }
  __device__ void cache_region_a(int lane) { a_cnt = nodes_a(lane, h.c, a_r2w, a_phi); }
  __device__ void set_rf(float rf, int lane) {
    full_a = rf >= h.rvir;
    if (!full_a) {
      f_cnt = nodes_a(lane, rf / h.rs, f_r2w, f_phi);
      return;
    }
    f_cnt = 0;
#pragma unroll
    for (int t = 0; t < NS; ++t) {
      const int q = lane + W * t, p = q / NG, j = q % NG;
      f_r2w[t] = 0.f;
      f_phi[t] = h.phi0;
      if (q >= MAX_PANEL_B * NG) continue;
      float lo = h.rvir, hi = fminf(2.0f * h.rvir, rf);
      bool ok = true;
      for (int k = 0; k < p && ok; ++k) {
        if (hi >= rf) ok = false;
        lo = hi;
        hi = fminf(2.0f * hi, rf);
      }
      if (!ok || !(hi > lo)) continue;
      float mid = 0.5f * (lo + hi), hw = 0.5f * (hi - lo);
      float r = mid + hw * glx(j);
      f_r2w[t] = hw * glw(j) * r * r;
      f_phi[t] = -h.GM / r;
      f_cnt = t + 1;
    }
  }
  __device__ void acc(SumsF& s, float r2w, float phi, float inv_n1T) const {
    float th = 1.0f + (h.phi0 - phi) * inv_n1T;
    if (th <= 0.0f) return;
    float tm = pw(th, 0);
    float tn = tm * th, tp = tn * th;
    s.Im += r2w * tm;
    s.In += r2w * tn;
    s.Ip += r2w * tp;
    s.Jm += r2w * tm * phi;
    s.Jn += r2w * tn * phi;
  }
  __device__ SumsF integrals(float T) const {
    SumsF s = {0, 0, 0, 0, 0};
    float inv_n1T = 1.0f / ((n + 1.0f) * T);
    if (full_a) {
#pragma unroll
      for (int t = 0; t < NS; ++t)
        if (t < a_cnt) acc(s, a_r2w[t], a_phi[t], inv_n1T);
    }
#pragma unroll
    for (int t = 0; t < NS; ++t)
      if (t < f_cnt) acc(s, f_r2w[t], f_phi[t], inv_n1T);
    s.Im = group_sum(s.Im);
    s.In = group_sum(s.In);
    s.Ip = group_sum(s.Ip);
    s.Jm = group_sum(s.Jm);
    s.Jn = group_sum(s.Jn);
    return s;
  }
};

using SolverF = SolverFT<32, NGL_PRE>;

// guess[i] = ln(r_f / r_vir), guess[n + i] = ln(T r_vir / (G M)), or NaN
__global__ void __launch_bounds__(32 * SOLVE_WARPS) k_presolve(
    BpParams P, int64_t n, SolveExtra X, int hpw, const Halo* __restrict__ halos,
    const int32_t* __restrict__ okv, double* guess, float* res32) {
  const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int64_t base = ((int64_t)blockIdx.x * (blockDim.x >> 5) + w) * hpw;
  if (base >= n) return;
  const float nn = (float)P.n_poly;
  const double rn = rint(P.n_poly);
  const int n_int = (fabs(P.n_poly - rn) < 1e-12 && rn >= 1 && rn <= 16) ? (int)rn : -1;
  for (int jj = 0; jj < hpw; ++jj) {
    const int64_t i = base + jj;
    if (i >= n) break;
    float g0 = __int_as_float(0x7fc00000), g1 = g0, rE = g0, rM = g0;
    if (okv[i]) {
      const Halo H = halos[i];
      const HaloF h = {(float)H.c, (float)H.rvir, (float)H.rs, (float)H.mc, (float)H.phi0,
                       (float)H.GM, (float)H.M};
      const double eps_star = X.prm ? X.prm[i] : P.eps_star;
      const double eps_dm = X.prm ? X.prm[2 * n + i] : P.eps_dm;
      const float fbM = (float)(P.fb * H.M), Mstar = (float)H.Mstar, Ps = (float)H.Ps;
      const float inj = (float)(eps_dm * fabs(H.Edm) + eps_star * H.Mstar * bpc::C_KMS * bpc::C_KMS);
      const float Egi = (float)H.Egi, absE = fabsf(Egi);
      const float r3v = h.rvir * h.rvir * h.rvir;
      const float four_pi = (float)(4.0 * bpc::PI);
      const float inv_target = 1.0f / (fbM - Mstar);
      SolverF S(h, nn, n_int);
      S.cache_region_a(lane);
      // reduced problem at r_f: T from the gas-mass condition, then R_e and dR_e/dln r_f
      float T = 0.f, Re = 1.f, dRe = 0.f, Fm = 1.f;
      auto reduced = [&](float rf, float T0) -> bool {
        const float phif = phi_of_f(h, rf);
        const float Tmin = (phif - h.phi0) / (nn + 1.0f);
        if (!(Tmin > 0.f)) return false;
        float s = (T0 > Tmin * 1.0001f) ? logf(T0 - Tmin) : logf(Tmin + 0.5f * h.GM / h.rvir);
        float slo = -INFINITY, shi = INFINITY, thf = 0.f, rho0 = 0.f, F = 1.f;
        SumsF sm;
        S.set_rf(rf, lane);
        for (int it = 0; it < 40; ++it) {
          T = Tmin + expf(s);
          thf = 1.0f + (h.phi0 - phif) / ((nn + 1.0f) * T);
          sm = S.integrals(T);
          rho0 = Ps / (T * S.pw(thf, 2));
          // the log of the ratio: a difference of two logs near 35 would floor F at 4e-6
          F = logf(four_pi * rho0 * sm.In * inv_target);
          if (!isfinite(F)) return false;
          if (fabsf(F) < 1e-6f) break;  // near the FP32 floor of F
          if (F > 0) slo = s; else shi = s;
          const float dlr = (-1.0f - (nn + 1.0f) * (1.0f - thf) / thf) / T;
          const float dli = nn * (sm.Im - sm.In) / (T * sm.In);
          float step = -F / ((T - Tmin) * (dlr + dli));
          // at the FP32 rounding floor (a step below the resolution of s) T has converged
          if (fabsf(F) < 1e-4f && isfinite(step) && fabsf(step) < 4e-7f * fmaxf(1.0f, fabsf(s)))
            break;
          if (!isfinite(step)) step = (F > 0) ? 1.0f : -1.0f;
          step = fmaxf(-4.0f, fminf(4.0f, step));
          float sn = s + step;
          if (isfinite(slo) && isfinite(shi) && !(sn > slo && sn < shi)) sn = 0.5f * (slo + shi);
          s = sn;
        }
        if (!(fabsf(F) < 1e-4f)) return false;
        Fm = F;
        const float In = sm.In, Ip = sm.Ip, Im = sm.Im, Jm = sm.Jm, Jn = sm.Jn;
        const float Egf = four_pi * rho0 * (1.5f * T * Ip + Jn);
        const float dEp = four_pi / 3.0f * (r3v - rf * rf * rf) * Ps;
        const float num = (P.energy_sign == 0) ? (Egf - Egi - inj - dEp) : (Egi - Egf - inj - dEp);
        Re = num / absE;
        const float dphif = (float)bpc::G * menc_of_f(h, rf) / (rf * rf);
        const float dthf_drf = -dphif / ((nn + 1.0f) * T);
        const float dlr_drf = -(nn + 1.0f) * dthf_drf / thf;
        const float dlr_dT = (-1.0f - (nn + 1.0f) * (1.0f - thf) / thf) / T;
        const float tfn = S.pw(thf, 1), tfp = tfn * thf;
        const float dG_drf = four_pi * rho0 * (In * dlr_drf + tfn * rf * rf);
        const float dG_dT = four_pi * rho0 * (In * dlr_dT + nn * (Im - In) / T);
        const float dT_drf = -dG_drf / dG_dT;
        const float dIp_dT = (nn + 1.0f) * (In - Ip) / T;
        const float dJn_dT = nn * (Jm - Jn) / T;
        const float dEgf_drf = Egf * dlr_drf + four_pi * rho0 * (1.5f * T * tfp + tfn * phif) * rf * rf;
        const float dEgf_dT = Egf * dlr_dT + four_pi * rho0 * (1.5f * Ip + 1.5f * T * dIp_dT + dJn_dT);
        const float ddEp_drf = -four_pi * rf * rf * Ps;
        const float dtot = dEgf_drf + dEgf_dT * dT_drf;
        const float dnum = (P.energy_sign == 0) ? (dtot - ddEp_drf) : (-dtot - ddEp_drf);
        dRe = rf * dnum / absE;
        return isfinite(Re) && isfinite(dRe);
      };
      // safeguarded Newton in v = ln r_f (bracketed once the sign changes), from the
      // caller's starting point when it has one (a seeded pre-solve), else from 1.1 r_vir
      const float vmin = logf(0.5f * h.rvir), vmax = logf(10.0f * h.rvir);
      float v = logf(1.1f * h.rvir), Tw = 0.f, vprev = 0.f, Rprev = 0.f, va = 0.f, vb = 0.f,
            Ra = 0.f;
      if (X.guess) {
        const double s0 = X.guess[i], s1 = X.guess[n + i];
        if (isfinite(s0) && isfinite(s1)) {
          v = fminf(fmaxf(logf(h.rvir) + (float)s0, vmin), vmax);
          Tw = (float)(exp(s1) * H.GM / H.rvir);  // T = e^s1 G M / r_vir
        }
      }
      bool have_prev = false, have_br = false, done = false;
      float v_ok = 0.f, T_ok = 0.f, Re_ok = 0.f, F_ok = 0.f;
      for (int it = 0; it < 40; ++it) {
        const float rf = expf(v);
        if (!reduced(rf, Tw)) break;
        Tw = T;
        if (fabsf(Re) < 1e-4f) {
          // one Newton step more (quadratic from here) takes R_e to the FP32 floor of a
          // few 1e-6, so that the FP64 polish needs one step instead of two
          const bool again = !done && fabsf(Re) > 2e-6f;
          done = true;
          v_ok = v;
          T_ok = T;
          Re_ok = Re;
          F_ok = Fm;
          if (!again) break;
        } else if (done) {
          break;  // the extra step went astray: keep the point below 1e-4
        }
        if (have_prev && ((Re > 0) != (Rprev > 0))) {
          have_br = true;
          va = vprev; Ra = Rprev; vb = v;
        } else if (have_br) {
          if ((Re > 0) == (Ra > 0)) { va = v; Ra = Re; } else { vb = v; }
        }
        float step = -Re / dRe;
        if (!isfinite(step)) step = 0.5f;
        step = fmaxf(-0.5f, fminf(0.5f, step));
        float vn = fminf(fmaxf(v + step, vmin), vmax);
        if (have_br) {
          const float lo = fminf(va, vb), hi = fmaxf(va, vb);
          if (!(vn > lo && vn < hi)) vn = 0.5f * (va + vb);
        }
        vprev = v; Rprev = Re; have_prev = true;
        v = vn;
      }
      if (done) {
        g0 = v_ok - logf(h.rvir);
        g1 = logf(T_ok * h.rvir / h.GM);
        rE = Re_ok;
        // the normalised gas-mass residual from F = ln of the ratio of gas masses
        rM = expm1f(F_ok) * (float)((P.fb * H.M - H.Mstar) / (P.fb * H.M));
      }
    }
    if (lane == 0) {
      guess[i] = (double)g0;
      guess[n + i] = (double)g1;
      if (res32) {
        res32[i] = rE;
        res32[n + i] = rM;
      }
    }
  }
}

// The FP32 pre-solve's solution as the answer (BP_SOLVE_FP32_GATED): a halo whose FP32
// energy and gas-mass residuals are both within the gate keeps (r_f, T) of the pre-solve, and
// its central density and pressure follow in FP64 from the pressure condition at r_f,
// rho0 = P_s / (T theta(r_f)^(n+1)), P0 = rho0 T; the residual fields hold the FP32 values.
// Any other halo of the solve is marked FALLBACK (the full FP64 solve follows), and so is a
// halo the caller gave no finite starting point (seed: the caller's guess, or null).
__global__ void k_accept32(BpParams P, int64_t n, const Halo* __restrict__ halos,
                           const int32_t* __restrict__ okv, const double* __restrict__ seed,
                           const double* __restrict__ guess, const float* __restrict__ res32,
                           double gate, double* model, int32_t* status, int64_t* nbad,
                           int64_t* nfallback) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n || !okv[i]) return;
  const Halo h = halos[i];
  const double g0 = guess[i], g1 = guess[n + i];
  const float rE = res32[i], rM = res32[n + i];
  bool ok = isfinite(g0) && isfinite(g1) && fabsf(rE) <= gate && fabsf(rM) <= gate;
  if (seed) ok = ok && isfinite(seed[i]) && isfinite(seed[n + i]);
  double rf = 0, T = 0, thf = 0, rho0 = 0;
  if (ok) {
    rf = h.rvir * exp(g0);
    T = exp(g1) * h.GM / h.rvir;
    thf = 1.0 + (h.phi0 - phi_of(h, rf)) / ((P.n_poly + 1.0) * T);
    ok = thf > 0.0;
    if (ok) rho0 = h.Ps / (T * pow(thf, P.n_poly + 1.0));
  }
  auto put = [&](int f, double v) { model[(int64_t)f * n + i] = v; };
  put(BP_M_T, ok ? T : 0.0);
  put(BP_M_RHO0, ok ? rho0 : 0.0);
  put(BP_M_P0, ok ? rho0 * T : 0.0);
  put(BP_M_RF, ok ? rf : 0.0);
  put(BP_M_RESM, ok ? (double)rM : NAN);
  put(BP_M_RESE, ok ? (double)rE : NAN);
  status[i] = ok ? BP_HALO_OK : BP_HALO_FALLBACK;
  if (!ok) {
    atomicAdd((unsigned long long*)nbad, 1ull);
    atomicAdd((unsigned long long*)nfallback, 1ull);
  }
}

}  // namespace

// presolve: run the FP32 pre-solve and start the FP64 solve from its result
// n_bad: halos whose status is not OK; n_fallback: those of them marked FALLBACK
// accept32: the pre-solve's solution is the answer where its FP32 residuals are within
// X.gate (k_accept32), every other halo is marked FALLBACK
static int solve_launch(bp_ctx* ctx, int64_t n, const double* Mvir, const double* c,
                        const double* z, double* model, int32_t* status, double tol,
                        SolveExtra X, int64_t* n_bad, int64_t* n_fallback,
                        bool presolve = false, bool accept32 = false) {
  int r = upload_constants(ctx);
  if (r) return r;
  Halo* halos;
  if ((r = bp_ws(ctx, WS_HALO,
                 (size_t)n * (sizeof(Halo) + 2 * sizeof(double) + 2 * sizeof(int32_t) +
                              2 * sizeof(float)) + 64,
                 (void**)&halos)))
    return r;
  double* pguess = reinterpret_cast<double*>(halos + n);
  int32_t* okv = reinterpret_cast<int32_t*>(pguess + 2 * n);
  int32_t* okv_nested = okv + n;  // halos the polish leaves to the nested iteration
  float* res32 = reinterpret_cast<float*>(okv_nested + n);  // FP32 residuals of the pre-solve
  BP_CUDA(ctx, cudaMemsetAsync(ctx->d_counter, 0, sizeof(int64_t), ctx->stream));
  BP_CUDA(ctx, cudaMemsetAsync(ctx->d_counter + 3, 0, sizeof(int64_t), ctx->stream));
  // halos per warp: enough warps to fill the GPU, the rest shared out 1..32 per warp
  int64_t target_warps = (int64_t)ctx->num_sms * 16;
  int hpw = (int)std::min<int64_t>(32, std::max<int64_t>(1, n / target_warps));
  int64_t warps = (n + hpw - 1) / hpw;
  int64_t blocks = (warps + SOLVE_WARPS - 1) / SOLVE_WARPS;
  bp_phase_begin(ctx, BP_PH_SOLVE);
  const int sb = bp_item_block(ctx, n, 128);
  k_setup<<<(unsigned)((n + sb - 1) / sb), sb, 0, ctx->stream>>>(
      ctx->p, ctx->t, n, Mvir, c, z, model, status, ctx->d_counter, X, halos, okv);
  BP_LAUNCH_CHECK(ctx, "k_setup launch");
  const double* seed = X.guess;  // the caller's starting points (or null)
  if (presolve) {
    k_presolve<<<(unsigned)blocks, 32 * SOLVE_WARPS, 0, ctx->stream>>>(ctx->p, n, X, hpw, halos,
                                                                       okv, pguess, res32);
    BP_LAUNCH_CHECK(ctx, "k_presolve launch");
    X.guess = pguess;
  }
  if (presolve && accept32) {
    k_accept32<<<(unsigned)((n + 255) / 256), 256, 0, ctx->stream>>>(
        ctx->p, n, halos, okv, seed, pguess, res32, X.gate, model, status, ctx->d_counter,
        ctx->d_counter + 3);
    BP_LAUNCH_CHECK(ctx, "k_accept32 launch");
  } else if (X.guess) {
    // starting points: two halos per warp; the halos without one get the nested iteration
    BP_CUDA(ctx, cudaMemsetAsync(okv_nested, 0, (size_t)n * sizeof(int32_t), ctx->stream));
    const int64_t pwarps = (n + POLISH_H * (int64_t)hpw - 1) / (POLISH_H * (int64_t)hpw);
    // one-warp blocks when there are few warps, so that they spread evenly over the SMs
    const int pw = pwarps < (int64_t)SOLVE_WARPS * ctx->num_sms * 4 ? 1 : SOLVE_WARPS;
    const int64_t pblocks = (pwarps + pw - 1) / pw;
    k_polish<<<(unsigned)pblocks, 32 * pw, 0, ctx->stream>>>(
        ctx->p, n, model, status, tol, ctx->d_counter, ctx->d_counter + 3, X, hpw, halos, okv,
        okv_nested);
    BP_LAUNCH_CHECK(ctx, "k_polish launch");
    k_solve<<<(unsigned)blocks, 32 * SOLVE_WARPS, 0, ctx->stream>>>(
        ctx->p, n, model, status, tol, ctx->d_counter, ctx->d_counter + 3, X, hpw, halos,
        okv_nested);
    BP_LAUNCH_CHECK(ctx, "k_solve launch");
  } else {
    k_solve<<<(unsigned)blocks, 32 * SOLVE_WARPS, 0, ctx->stream>>>(
        ctx->p, n, model, status, tol, ctx->d_counter, ctx->d_counter + 3, X, hpw, halos, okv);
    BP_LAUNCH_CHECK(ctx, "k_solve launch");
  }
  bp_phase_end(ctx, BP_PH_SOLVE);
  BP_CUDA(ctx, cudaMemcpyAsync(ctx->h_pinned, ctx->d_counter, sizeof(int64_t),
                               cudaMemcpyDeviceToHost, ctx->stream));
  BP_CUDA(ctx, cudaMemcpyAsync(ctx->h_pinned + 4, ctx->d_counter + 3, sizeof(int64_t),
                               cudaMemcpyDeviceToHost, ctx->stream));
  BP_CUDA(ctx, cudaStreamSynchronize(ctx->stream));
  *n_bad = ctx->h_pinned[0];
  *n_fallback = ctx->h_pinned[4];
  return BP_OK;
}

static int solve_args(bp_ctx* ctx, int64_t n, const double* Mvir, const double* c,
                      const double* z, double* model, int32_t* status, int mode) {
  if (n < 0) return bp_fail(ctx, BP_EINVAL, "bp_solve_halos: n < 0");
  if (n > 0 && (!Mvir || !c || !z || !model || !status))
    return bp_fail(ctx, BP_EINVAL, "bp_solve_halos: null pointer");
  if (mode != BP_SOLVE_FP64 && mode != BP_SOLVE_FP64_SEEDED && mode != BP_SOLVE_FP32_GATED)
    return bp_fail(ctx, BP_EINVAL, "bp_solve_halos: unknown mode");
  return BP_OK;
}

extern "C" int bp_solve_halos(bp_ctx* ctx, int64_t n, const double* Mvir, const double* c,
                              const double* z, double* model, int32_t* status, int mode,
                              double resid_tol) {
  return bp_solve_halos_ex(ctx, n, Mvir, c, z, nullptr, nullptr, 0, 0.0, model, status, mode,
                           resid_tol);
}

extern "C" int bp_solve_halos_ex(bp_ctx* ctx, int64_t n, const double* Mvir, const double* c,
                                 const double* z, const double* params, const double* guess,
                                 int max_iter, double gate, double* model, int32_t* status,
                                 int mode, double resid_tol) {
  if (!ctx) return BP_EINVAL;
  int r = solve_args(ctx, n, Mvir, c, z, model, status, mode);
  if (r) return r;
  if (n == 0) return BP_OK;
  if (gate < 0) return bp_fail(ctx, BP_EINVAL, "bp_solve_halos_ex: gate < 0");
  SolveExtra X;
  X.prm = params;
  X.guess = guess;
  X.max_outer = max_iter > 0 ? max_iter : 80;
  X.gate = gate;
  X.only_fallback = 0;
  int64_t bad = 0;
  double tol = resid_tol > 0 ? resid_tol : 1e-10;
  // Stages: (1) the FP64 Newton from the caller's starting point, or from the FP32
  // pre-solve when there is none or when it seeds the pre-solve (BP_SOLVE_FP64_SEEDED);
  // (2) for halos stage 1 marked FALLBACK after a caller's starting point: the FP32
  // pre-solve and the Newton from it; (3) for those still marked: the full nested FP64
  // iteration.  A Newton stage accepts a halo when both residuals are below the gate (the
  // tolerance for the unseeded pre-solve stages, the caller's gate for a seeded one).
  const bool gated32 = mode == BP_SOLVE_FP32_GATED;
  if (gated32 && !(gate > 0))
    return bp_fail(ctx, BP_EINVAL, "bp_solve_halos_ex: BP_SOLVE_FP32_GATED needs gate > 0");
  const bool seeded = (mode == BP_SOLVE_FP64_SEEDED || gated32) && guess != nullptr;
  const bool presolve = guess == nullptr || seeded;
  if (presolve) {
    X.max_outer = seeded && max_iter > 0 ? max_iter : 8;
    X.gate = (seeded || gated32) && gate > 0 ? gate : tol;
  }
  int64_t fb = 0;
  if ((r = solve_launch(ctx, n, Mvir, c, z, model, status, tol, X, &bad, &fb, presolve,
                        gated32)))
    return r;
  ctx->last_fallback = fb;
  for (int stage = presolve ? 3 : 2; fb > 0 && stage <= 3; ++stage) {
    X.guess = nullptr;
    X.only_fallback = 1;
    X.max_outer = stage == 2 ? 8 : 80;
    X.gate = stage == 2 ? tol : 0.0;
    int64_t bad2 = 0, fb2 = 0;
    if ((r = solve_launch(ctx, n, Mvir, c, z, model, status, tol, X, &bad2, &fb2, stage == 2)))
      return r;
    bad = bad - fb + bad2;
    fb = fb2;
  }
  if (bad) return bp_fail(ctx, BP_ENOCONV, "bp_solve_halos: %lld of %lld halos not converged",
                          (long long)bad, (long long)n);
  return BP_OK;
}

/*
 * bp_oracle.c -- plain, slow FP64 CPU oracle for the baryon pasting method of
 * Osato & Nagai (arXiv:2201.02632).
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing in the product path links, imports or
 * executes this file: only the tests, the smoke check and the CPU-baseline leg
 * of the benchmark do.  It shares no source, header, table or constant
 * generator with the CUDA path.
 *
 * Every function cites the section / equation of the paper it writes out.
 * Numerical means are deliberately different from the GPU path:
 *   - integrals use adaptive Gauss-Kronrod (G7/K15), split at the kinks;
 *   - the velocity dispersion is the Jeans integral done by quadrature at
 *     every node (no closed form, no integration by parts);
 *   - the ICM solve is nested bracketing (Brent in T for the gas-mass
 *     condition, a scan + Brent in r_f for the energy condition) instead of
 *     Newton-Raphson;
 *   - z(chi) is bisection on the quadrature chi(z), not a table.
 *
 * Units: masses Msun, lengths physical Mpc (unless noted comoving), velocities
 * km/s, energies Msun (km/s)^2, pressures Msun (km/s)^2 / Mpc^3.  Catalogue
 * inputs are in h^-1 Msun and comoving h^-1 Mpc and are converted once.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#ifdef _OPENMP
#include <omp.h>
#endif

/* ------------------------------------------------------------------ */
/* Physical constants (CODATA 2018 / IAU 2015 nominal values).         */
/* ------------------------------------------------------------------ */
static const double O_PI = 3.14159265358979323846;
static const double O_C_KMS = 299792.458;             /* km/s */
static const double O_G_SI = 6.67430e-11;             /* m^3 kg^-1 s^-2 */
static const double O_MSUN_KG = 1.98840987e30;        /* GM_sun(IAU)/G */
static const double O_MPC_M = 3.0856775814913673e22;  /* m */
static const double O_SIGMA_T = 6.6524587321e-29;     /* m^2 */
static const double O_ME_C2_J = 8.1871057769e-14;     /* 510.99895 keV in J */
static const double O_MP_KG = 1.67262192369e-27;      /* kg */
static const double O_H_PLANCK = 6.62607015e-34;       /* J s (exact, SI 2019) */
static const double O_K_B = 1.380649e-23;              /* J/K (exact, SI 2019) */

static double o_G(void) { /* Mpc (km/s)^2 / Msun */
  return O_G_SI * O_MSUN_KG / (O_MPC_M * 1.0e6);
}

/* ------------------------------------------------------------------ */
/* Parameter blocks (oracle-private layout).                          */
/* ------------------------------------------------------------------ */
typedef struct { double Om, Ob, h, Tcmb, XH; } orc_cosmo;
typedef struct {
  double Gamma, eps_dm, eps_star, f_star, S_star, alpha_nt, beta_nt, n_nt;
  int energy_sign; /* 0: final = initial + injections + surface work; 1: as printed */
  int field_fb;    /* 1: field-particle electrons carry f_b (printed form: 0) */
} orc_icm;

/* Per-halo solved model: oracle-private field order. */
enum {
  OF_M = 0,     /* M_vir [Msun] */
  OF_C,         /* c_vir */
  OF_Z,         /* redshift */
  OF_RHOCR,     /* rho_cr(z) [Msun/Mpc^3] */
  OF_DVIR,      /* Delta_vir(z) w.r.t. rho_cr */
  OF_RVIR,      /* r_vir [Mpc] */
  OF_RS,        /* r_s */
  OF_RHOS,      /* rho_s */
  OF_MC,        /* m(c) */
  OF_PHI0,      /* central potential */
  OF_R500,
  OF_M500,
  OF_MSTAR,
  OF_RSTAR,
  OF_EGI,       /* initial gas energy */
  OF_EDM,       /* dark-matter energy */
  OF_PS,        /* surface pressure */
  OF_T,         /* P0/rho0 */
  OF_RHO0,
  OF_P0,
  OF_RF,
  OF_ANT,       /* alpha_nt * f(z) */
  OF_DA,        /* angular-diameter distance [Mpc] */
  OF_TAU,       /* mean optical depth to z */
  OF_RESM,      /* gas-mass residual at the root */
  OF_RESE,      /* energy residual at the root */
  OF_STATUS,    /* 0 ok, 1 no bracket, 2 bad stellar mass, 3 theta<=0 */
  OF_N
};
int orc_model_nfields(void) { return OF_N; }

/* ------------------------------------------------------------------ */
/* Adaptive Gauss-Kronrod (7-point Gauss / 15-point Kronrod).          */
/* ------------------------------------------------------------------ */
typedef double (*o_fn)(double, void*);

static const double GK_X[8] = {
  0.991455371120812639206854697526329, 0.949107912342758524526189684047851,
  0.864864423359769072789712788640926, 0.741531185599394439863864773280788,
  0.586087235467691130294144845693013, 0.405845151377397166906606412076961,
  0.207784955007898467600689403773245, 0.000000000000000000000000000000000};
static const double GK_WK[8] = {
  0.022935322010529224963732008058970, 0.063092092629978553290700663189204,
  0.104790010322250183839876322541518, 0.140653259715525918745189590510238,
  0.169004726639267902826583426598550, 0.190350578064785409913256402421014,
  0.204432940075298892414161999234649, 0.209482141084727828012999174891714};
static const double GK_WG[4] = {
  0.129484966168869693270611432679082, 0.279705391489276667901467771423780,
  0.381830050505118944950369775488975, 0.417959183673469387755102040816327};

static void gk15(o_fn f, void* ctx, double a, double b, double* res, double* err) {
  double c = 0.5 * (a + b), hw = 0.5 * (b - a);
  double fc = f(c, ctx);
  double rk = fc * GK_WK[7], rg = fc * GK_WG[3];
  for (int j = 0; j < 7; ++j) {
    double dx = hw * GK_X[j];
    double f1 = f(c - dx, ctx), f2 = f(c + dx, ctx);
    rk += GK_WK[j] * (f1 + f2);
    if (j & 1) rg += GK_WG[j / 2] * (f1 + f2);
  }
  *res = rk * hw;
  *err = fabs((rk - rg) * hw);
}

/* Globally adaptive bisection: keep a list of panels, split the one with the
 * largest error estimate until the summed estimate is below tol or the panel
 * budget is spent (bounded work; no per-level tolerance halving). */
#define O_MAXPAN 600
static double o_quad(o_fn f, void* ctx, double a, double b, double rtol) {
  if (b == a) return 0.0;
  double pa[O_MAXPAN], pb[O_MAXPAN], pr[O_MAXPAN], pe[O_MAXPAN];
  int np = 1;
  pa[0] = a;
  pb[0] = b;
  gk15(f, ctx, a, b, &pr[0], &pe[0]);
  for (;;) {
    double tot = 0.0, err = 0.0, absr = 0.0;
    int worst = 0;
    for (int i = 0; i < np; ++i) {
      tot += pr[i];
      err += pe[i];
      absr += fabs(pr[i]);
      if (pe[i] > pe[worst]) worst = i;
    }
    double tol = rtol * absr;
    if (err <= tol || np + 1 >= O_MAXPAN || err <= 1e-15 * absr) return tot;
    double m = 0.5 * (pa[worst] + pb[worst]);
    if (!(m > pa[worst] && m < pb[worst])) return tot;
    pa[np] = m;
    pb[np] = pb[worst];
    pb[worst] = m;
    gk15(f, ctx, pa[worst], pb[worst], &pr[worst], &pe[worst]);
    gk15(f, ctx, pa[np], pb[np], &pr[np], &pe[np]);
    ++np;
  }
}

/* Integral over [a,b] split at the listed interior points (kinks). */
static double o_quad_split(o_fn f, void* ctx, double a, double b, const double* pts, int np,
                           double rtol) {
  double cuts[8];
  int nc = 0;
  cuts[nc++] = a;
  for (int i = 0; i < np; ++i)
    if (pts[i] > a && pts[i] < b) cuts[nc++] = pts[i];
  cuts[nc++] = b;
  /* insertion sort */
  for (int i = 1; i < nc; ++i)
    for (int j = i; j > 0 && cuts[j] < cuts[j - 1]; --j) {
      double t = cuts[j]; cuts[j] = cuts[j - 1]; cuts[j - 1] = t;
    }
  double s = 0.0;
  for (int i = 0; i + 1 < nc; ++i) s += o_quad(f, ctx, cuts[i], cuts[i + 1], rtol);
  return s;
}

/* ------------------------------------------------------------------ */
/* Brent's method (Brent 1973, "Algorithms for minimization without    */
/* derivatives", ch. 4), written from the published description.      */
/* Requires fa*fb <= 0.                                                */
/* ------------------------------------------------------------------ */
typedef double (*o_rfn)(double, void*);
static double o_brent(o_rfn f, void* ctx, double a, double b, double fa, double fb,
                      double xtol, int maxit) {
  double c = a, fc = fa, d = b - a, e = d;
  for (int it = 0; it < maxit; ++it) {
    if ((fb > 0 && fc > 0) || (fb < 0 && fc < 0)) { c = a; fc = fa; d = e = b - a; }
    if (fabs(fc) < fabs(fb)) { a = b; b = c; c = a; fa = fb; fb = fc; fc = fa; }
    double tol = 2.0 * 2.220446049250313e-16 * fabs(b) + 0.5 * xtol;
    double m = 0.5 * (c - b);
    if (fabs(m) <= tol || fb == 0.0) return b;
    if (fabs(e) >= tol && fabs(fa) > fabs(fb)) {
      double s = fb / fa, p, q;
      if (a == c) { p = 2.0 * m * s; q = 1.0 - s; }
      else {
        double qq = fa / fc, r = fb / fc;
        p = s * (2.0 * m * qq * (qq - r) - (b - a) * (r - 1.0));
        q = (qq - 1.0) * (r - 1.0) * (s - 1.0);
      }
      if (p > 0) q = -q; else p = -p;
      if (2.0 * p < fmin(3.0 * m * q - fabs(tol * q), fabs(e * q))) { e = d; d = p / q; }
      else { d = m; e = m; }
    } else { d = m; e = m; }
    a = b; fa = fb;
    b += (fabs(d) > tol) ? d : (m > 0 ? tol : -tol);
    fb = f(b, ctx);
  }
  return b;
}

/* ------------------------------------------------------------------ */
/* Cosmology (Section 1 parameters; Section 3.2 tau(z); Section 4).    */
/* Flat LCDM, radiation neglected.                                     */
/* ------------------------------------------------------------------ */
static double o_E(const orc_cosmo* cp, double z) {
  double a3 = (1.0 + z) * (1.0 + z) * (1.0 + z);
  return sqrt(cp->Om * a3 + (1.0 - cp->Om));
}
static double o_H0(const orc_cosmo* cp) { return 100.0 * cp->h; } /* km/s/Mpc */

/* Critical density 3H^2/(8 pi G)  [Msun/Mpc^3] (Section 2.1). */
double orc_rho_cr(const orc_cosmo* cp, double z) {
  double H = o_H0(cp) * o_E(cp, z);
  return 3.0 * H * H / (8.0 * O_PI * o_G());
}

/* Virial overdensity w.r.t. rho_cr: Bryan & Norman (1998) flat-universe fit,
 * cited (not printed) in Section 2.1. */
double orc_delta_vir(const orc_cosmo* cp, double z) {
  double E2 = o_E(cp, z) * o_E(cp, z);
  double x = cp->Om * pow(1.0 + z, 3) / E2 - 1.0;
  return 18.0 * O_PI * O_PI + 82.0 * x - 39.0 * x * x;
}

static double f_chi(double z, void* ctx) {
  const orc_cosmo* cp = (const orc_cosmo*)ctx;
  return O_C_KMS / (o_H0(cp) * o_E(cp, z));
}
/* Comoving distance chi(z) = int_0^z c dz'/H(z') [Mpc] (Section 4.1). */
double orc_chi(const orc_cosmo* cp, double z) {
  if (z <= 0) return 0.0;
  return o_quad(f_chi, (void*)cp, 0.0, z, 1e-14);
}
/* Inverse of chi(z) by bisection. */
double orc_z_of_chi(const orc_cosmo* cp, double chi) {
  if (chi <= 0) return 0.0;
  double lo = 0.0, hi = 1.0;
  while (orc_chi(cp, hi) < chi) hi *= 2.0;
  for (int it = 0; it < 200 && hi - lo > 1e-15 * hi; ++it) {
    double mid = 0.5 * (lo + hi);
    if (orc_chi(cp, mid) < chi) lo = mid; else hi = mid;
  }
  return 0.5 * (lo + hi);
}
double orc_DA(const orc_cosmo* cp, double z) { return orc_chi(cp, z) / (1.0 + z); }

static double o_mu_e(const orc_cosmo* cp) { return 2.0 / (cp->XH + 1.0); }

static double f_tau(double z, void* ctx) {
  const orc_cosmo* cp = (const orc_cosmo*)ctx;
  return O_C_KMS / (o_H0(cp) * o_E(cp, z)) * (1.0 + z) * (1.0 + z);
}
/* Mean Thomson optical depth, Section 3.2: tau = sigma_T int c dz/H (1+z)^2 nbar_e,
 * nbar_e = Omega_b rho_cr(0) / (mu_e m_p). */
double orc_tau(const orc_cosmo* cp, double z) {
  if (z <= 0) return 0.0;
  double I = o_quad(f_tau, (void*)cp, 0.0, z, 1e-14); /* Mpc */
  double ne = cp->Ob * orc_rho_cr(cp, 0.0) * O_MSUN_KG / (O_MPC_M * O_MPC_M * O_MPC_M) /
              (o_mu_e(cp) * O_MP_KG); /* m^-3 */
  return O_SIGMA_T * ne * I * O_MPC_M;
}

/* ------------------------------------------------------------------ */
/* NFW halo (Section 2.1).                                             */
/* ------------------------------------------------------------------ */
double orc_m_of(double x) { return log1p(x) - x / (1.0 + x); }

typedef struct {
  double M, c, rvir, rs, rhos, mc, G;
} o_nfw;

static void o_nfw_init(o_nfw* h, const orc_cosmo* cp, double M, double c, double z) {
  h->M = M;
  h->c = c;
  h->G = o_G();
  double rc = orc_rho_cr(cp, z), dv = orc_delta_vir(cp, z);
  h->rvir = cbrt(3.0 * M / (4.0 * O_PI * dv * rc));
  h->rs = h->rvir / c;
  h->mc = orc_m_of(c);
  h->rhos = M / (4.0 * O_PI * h->rs * h->rs * h->rs * h->mc);
}
/* Untruncated NFW density (Eq. NFW profile). */
static double o_rho_nfw(const o_nfw* h, double r) {
  double x = r / h->rs;
  return h->rhos / (x * (1.0 + x) * (1.0 + x));
}
/* Truncated total density: zero beyond r_vir. */
static double o_rho_tot(const o_nfw* h, double r) { return r <= h->rvir ? o_rho_nfw(h, r) : 0.0; }
/* Untruncated enclosed mass 4 pi rho_s r_s^3 m(r/r_s). */
static double o_M_untr(const o_nfw* h, double r) { return h->M * orc_m_of(r / h->rs) / h->mc; }
/* Truncated enclosed mass M_tot(<r). */
static double o_M_tot(const o_nfw* h, double r) { return r <= h->rvir ? o_M_untr(h, r) : h->M; }

/* Potential of the truncated profile: Lokas & Mamon (2001) eq. 9 plus the constant
 * that makes Phi vanish at infinity (Section 2.1 footnote); point mass outside r_vir. */
static double o_phi(const o_nfw* h, double r) {
  if (r > h->rvir) return -h->G * h->M / r;
  double x = r / h->rs;
  double lnx_over_r = (x < 1e-8) ? (1.0 - 0.5 * x) / h->rs : log1p(x) / r;
  return -(h->G * h->M / h->mc) * (lnx_over_r - h->c / ((1.0 + h->c) * h->rvir));
}
static double o_phi0(const o_nfw* h) {
  return -(h->G * h->M / (h->mc * h->rvir)) * h->c * h->c / (1.0 + h->c);
}

/* Isotropic velocity dispersion of the untruncated NFW halo (Lokas & Mamon 2001,
 * isotropic orbits, cited in Section 2.2) from its definition, the Jeans integral
 *   rho sigma^2 (r) = int_r^inf rho(r') G M(<r') / r'^2 dr',
 * evaluated by adaptive quadrature after r' = r/u (u in (0,1]). */
typedef struct { const o_nfw* h; double r; } o_jeans_ctx;
static double f_jeans(double u, void* vctx) {
  const o_jeans_ctx* jc = (const o_jeans_ctx*)vctx;
  if (u <= 0.0) return 0.0;
  double rp = jc->r / u;
  double dr_du = jc->r / (u * u);
  return o_rho_nfw(jc->h, rp) * jc->h->G * o_M_untr(jc->h, rp) / (rp * rp) * dr_du;
}
static double o_rho_sigma2(const o_nfw* h, double r) {
  o_jeans_ctx jc = {h, r};
  return o_quad(f_jeans, &jc, 0.0, 1.0, 1e-13);
}
double orc_sigma2(const orc_cosmo* cp, double M_hinv, double c, double z, double r) {
  o_nfw h;
  o_nfw_init(&h, cp, M_hinv / cp->h, c, z);
  return o_rho_sigma2(&h, r) / o_rho_nfw(&h, r);
}

/* ------------------------------------------------------------------ */
/* Halo scalars (Section 2.2).                                         */
/* ------------------------------------------------------------------ */
typedef struct { const o_nfw* h; double k; } o_rootctx;
static double f_r500(double r, void* vctx) { /* M(<r) - (4pi/3) 500 rho_cr r^3 */
  const o_rootctx* rc = (const o_rootctx*)vctx;
  return o_M_tot(rc->h, r) - rc->k * r * r * r;
}
static double f_rstar(double r, void* vctx) { /* f_b M(<r) - M_* ; k = M_* / f_b */
  const o_rootctx* rc = (const o_rootctx*)vctx;
  return o_M_tot(rc->h, r) - rc->k;
}
static double o_bisect(o_rfn f, void* ctx, double lo, double hi) {
  double flo = f(lo, ctx);
  for (int it = 0; it < 300 && hi - lo > 1e-15 * hi; ++it) {
    double mid = 0.5 * (lo + hi), fm = f(mid, ctx);
    if ((fm > 0) == (flo > 0)) { lo = mid; flo = fm; } else hi = mid;
  }
  return 0.5 * (lo + hi);
}

/* integrand pieces of the initial energy (Eq. initial energy) */
typedef struct { const o_nfw* h; } o_ectx;
static double f_kin(double r, void* vctx) { /* 2 pi rho 3 sigma^2 r^2 */
  const o_ectx* ec = (const o_ectx*)vctx;
  if (r <= 0) return 0.0;
  return 2.0 * O_PI * 3.0 * o_rho_sigma2(ec->h, r) * r * r;
}
static double f_pot(double r, void* vctx) { /* Phi dM/dr */
  const o_ectx* ec = (const o_ectx*)vctx;
  if (r <= 0) return 0.0;
  return o_phi(ec->h, r) * 4.0 * O_PI * r * r * o_rho_tot(ec->h, r);
}

/* ------------------------------------------------------------------ */
/* Polytropic gas (Section 2.1) and the three conditions (Section 2.2). */
/* ------------------------------------------------------------------ */
typedef struct {
  const o_nfw* h;
  double n;      /* polytropic index 1/(Gamma-1) */
  double phi0, T;
  double rho0;   /* for the energy integrand */
} o_gas;
static double o_theta(const o_gas* g, double r) {
  return 1.0 + (g->phi0 - o_phi(g->h, r)) / ((g->n + 1.0) * g->T);
}
static double f_gas_mass(double r, void* vctx) { /* theta^n r^2 */
  const o_gas* g = (const o_gas*)vctx;
  double th = o_theta(g, r);
  return th > 0 ? pow(th, g->n) * r * r : 0.0;
}
static double f_gas_energy(double r, void* vctx) { /* [3/2 P + rho_g Phi] r^2 / rho0 */
  const o_gas* g = (const o_gas*)vctx;
  double th = o_theta(g, r);
  if (th <= 0) return 0.0;
  double thn = pow(th, g->n);
  return (1.5 * g->T * thn * th + thn * o_phi(g->h, r)) * r * r;
}

typedef struct {
  const orc_cosmo* cp;
  const orc_icm* ip;
  o_nfw h;
  double fb, n, phi0, Mstar, Egi, Edm, Ps;
  double rf; /* current r_f for the inner T solve */
} o_solver;

static double o_rho0_of(const o_solver* s, double T, double rf) {
  o_gas g = {&s->h, s->n, s->phi0, T, 0.0};
  double thf = o_theta(&g, rf);
  return s->Ps / (T * pow(thf, s->n + 1.0));
}

/* gas-mass condition (Eq. gas mass), normalised by f_b M_vir */
static double o_res_mass(const o_solver* s, double T, double rf) {
  o_gas g = {&s->h, s->n, s->phi0, T, 0.0};
  if (o_theta(&g, rf) <= 0) return INFINITY;
  double rho0 = o_rho0_of(s, T, rf);
  double pts[1] = {s->h.rvir};
  double I = o_quad_split(f_gas_mass, &g, 0.0, rf, pts, 1, 1e-13);
  return (4.0 * O_PI * rho0 * I + s->Mstar) / (s->fb * s->h.M) - 1.0;
}
static double f_resm_T(double T, void* vctx) {
  const o_solver* s = (const o_solver*)vctx;
  return o_res_mass(s, T, s->rf);
}

/* energy condition (Eq. energy conservation + surface work), normalised by |E_g,i| */
static double o_res_energy(const o_solver* s, double T, double rf) {
  o_gas g = {&s->h, s->n, s->phi0, T, 0.0};
  double rho0 = o_rho0_of(s, T, rf);
  double pts[1] = {s->h.rvir};
  double Egf = 4.0 * O_PI * rho0 * o_quad_split(f_gas_energy, &g, 0.0, rf, pts, 1, 1e-13);
  double r3v = s->h.rvir * s->h.rvir * s->h.rvir;
  double dEp = 4.0 * O_PI / 3.0 * (r3v - rf * rf * rf) * s->Ps;
  double inj = s->ip->eps_dm * fabs(s->Edm) + s->ip->eps_star * s->Mstar * O_C_KMS * O_C_KMS;
  double r;
  if (s->ip->energy_sign == 0)
    r = Egf - (s->Egi + inj + dEp); /* final = initial + injected + surface work */
  else
    r = s->Egi - (Egf + inj + dEp); /* the printed arrangement */
  return r / fabs(s->Egi);
}

/* For a given r_f, the T that satisfies the gas-mass condition (Brent). */
static int o_T_of_rf(o_solver* s, double rf, double* Tout) {
  s->rf = rf;
  double dphi = o_phi(&s->h, rf) - s->phi0; /* > 0 */
  double Tlo = dphi / (s->n + 1.0) * (1.0 + 1e-12);
  double Thi = 1e3 * s->h.G * s->h.M / s->h.rvir;
  double flo = f_resm_T(Tlo, s);
  double fhi = f_resm_T(Thi, s);
  int guard = 0;
  while (fhi > 0 && guard++ < 60) { Thi *= 4.0; fhi = f_resm_T(Thi, s); }
  if (!(flo > 0) || !(fhi < 0)) {
    /* flo is +inf or positive by construction; a finite check on the low end */
    if (!(fhi < 0)) return 1;
  }
  if (!isfinite(flo)) {
    /* step up from Tlo until finite */
    double t = Tlo;
    for (int k = 0; k < 60 && !isfinite(flo); ++k) { t = Tlo * (1.0 + pow(2.0, -40 + k)); flo = f_resm_T(t, s); }
    Tlo = t;
    if (!isfinite(flo) || flo < 0) return 1;
  }
  *Tout = o_brent(f_resm_T, s, Tlo, Thi, flo, fhi, 1e-15 * Thi, 300);
  return 0;
}
static double f_rese_rf(double rf, void* vctx) {
  o_solver* s = (o_solver*)vctx;
  double T;
  if (o_T_of_rf(s, rf, &T)) return NAN;
  return o_res_energy(s, T, rf);
}

/* Solve one halo.  Inputs: M in h^-1 Msun, c, z.  Output: model[OF_N]. */
void orc_halo_solve(const orc_cosmo* cp, const orc_icm* ip, double M_hinv, double c, double z,
                    int n_scan, double* out) {
  memset(out, 0, sizeof(double) * OF_N);
  o_solver s;
  s.cp = cp;
  s.ip = ip;
  o_nfw_init(&s.h, cp, M_hinv / cp->h, c, z);
  const o_nfw* h = &s.h;
  s.fb = cp->Ob / cp->Om;
  s.n = 1.0 / (ip->Gamma - 1.0); /* polytropic index (see the theta definition) */
  s.phi0 = o_phi0(h);
  out[OF_M] = h->M;
  out[OF_C] = c;
  out[OF_Z] = z;
  out[OF_RHOCR] = orc_rho_cr(cp, z);
  out[OF_DVIR] = orc_delta_vir(cp, z);
  out[OF_RVIR] = h->rvir;
  out[OF_RS] = h->rs;
  out[OF_RHOS] = h->rhos;
  out[OF_MC] = h->mc;
  out[OF_PHI0] = s.phi0;
  out[OF_DA] = orc_DA(cp, z);
  out[OF_TAU] = orc_tau(cp, z);

  /* r500: mean enclosed density = 500 rho_cr */
  o_rootctx rc5 = {h, 4.0 * O_PI / 3.0 * 500.0 * out[OF_RHOCR]};
  double r500 = o_bisect(f_r500, &rc5, 1e-6 * h->rvir, h->rvir);
  out[OF_R500] = r500;
  out[OF_M500] = rc5.k * r500 * r500 * r500;
  /* stellar mass: F_* (M500/3e14 Msun)^{-S_*} times M_vir */
  double Fs = ip->f_star * pow(out[OF_M500] / 3e14, -ip->S_star);
  s.Mstar = Fs * h->M;
  out[OF_MSTAR] = s.Mstar;
  /* non-thermal amplitude alpha_nt f(z) (Section 2.3) */
  double fmax = pow(4.0, -ip->n_nt) / ip->alpha_nt;
  double fz = fmin(pow(1.0 + z, ip->beta_nt), (fmax - 1.0) * tanh(ip->beta_nt * z) + 1.0);
  out[OF_ANT] = ip->alpha_nt * fz;
  if (s.Mstar >= s.fb * h->M) { out[OF_STATUS] = 2; return; }
  o_rootctx rcs = {h, s.Mstar / s.fb};
  double rstar = o_bisect(f_rstar, &rcs, 1e-12 * h->rvir, h->rvir);
  out[OF_RSTAR] = rstar;

  /* initial gas energy and dark-matter energy (Eq. initial energy) */
  o_ectx ec = {h};
  double Ekin = o_quad(f_kin, &ec, rstar, h->rvir, 1e-12);
  double Epot = o_quad(f_pot, &ec, rstar, h->rvir, 1e-12);
  s.Egi = s.fb * (Ekin + Epot);
  double Ekin0 = o_quad(f_kin, &ec, 0.0, h->rvir, 1e-12);
  double Epot0 = o_quad(f_pot, &ec, 0.0, h->rvir, 1e-12);
  s.Edm = Ekin0 + Epot0;
  out[OF_EGI] = s.Egi;
  out[OF_EDM] = s.Edm;
  /* surface pressure (Eq. surface pressure) */
  s.Ps = s.fb * o_rho_sigma2(h, h->rvir);
  out[OF_PS] = s.Ps;

  /* energy condition: scan r_f, first sign change at r_f >= r_vir, then Brent */
  if (n_scan < 8) n_scan = 8;
  double lo = 0.5, hi = 10.0;
  double prev_r = 0, prev_f = NAN;
  double br_a = -1, br_b = -1, fa = 0, fb = 0, below_a = -1, below_b = -1, bfa = 0, bfb = 0;
  for (int k = 0; k < n_scan; ++k) {
    double rf = h->rvir * lo * pow(hi / lo, (double)k / (n_scan - 1));
    double f = f_rese_rf(rf, &s);
    if (k > 0 && isfinite(f) && isfinite(prev_f) && ((f > 0) != (prev_f > 0))) {
      if (prev_r >= h->rvir || rf >= h->rvir) {
        if (prev_r >= h->rvir && br_a < 0) { br_a = prev_r; br_b = rf; fa = prev_f; fb = f; }
        else if (prev_r < h->rvir && br_a < 0) {
          /* bracket straddles r_vir: split it at r_vir */
          double fv = f_rese_rf(h->rvir, &s);
          if ((fv > 0) != (f > 0)) { br_a = h->rvir; br_b = rf; fa = fv; fb = f; }
          else if (below_a < 0) { below_a = prev_r; below_b = h->rvir; bfa = prev_f; bfb = fv; }
        }
      } else if (below_a < 0) {
        below_a = prev_r; below_b = rf; bfa = prev_f; bfb = f;
      }
    }
    prev_r = rf;
    prev_f = f;
  }
  if (br_a < 0) { br_a = below_a; br_b = below_b; fa = bfa; fb = bfb; }
  if (br_a < 0) { out[OF_STATUS] = 1; return; }
  double rf = o_brent(f_rese_rf, &s, br_a, br_b, fa, fb, 1e-14 * br_b, 300);
  double T;
  if (o_T_of_rf(&s, rf, &T)) { out[OF_STATUS] = 1; return; }
  out[OF_RF] = rf;
  out[OF_T] = T;
  out[OF_RHO0] = o_rho0_of(&s, T, rf);
  out[OF_P0] = out[OF_RHO0] * T;
  out[OF_RESM] = o_res_mass(&s, T, rf);
  out[OF_RESE] = o_res_energy(&s, T, rf);
  o_gas g = {h, s.n, s.phi0, T, 0.0};
  if (o_theta(&g, rf) <= 0) out[OF_STATUS] = 3;
}

/* Solve many halos (OpenMP over halos; each halo is independent). */
void orc_solve_halos(const orc_cosmo* cp, const orc_icm* ip, int64_t n, const double* M,
                     const double* c, const double* z, int n_scan, double* out, int nthreads) {
#ifdef _OPENMP
  if (nthreads > 0) omp_set_num_threads(nthreads);
#pragma omp parallel for schedule(dynamic, 1)
#endif
  for (int64_t i = 0; i < n; ++i) orc_halo_solve(cp, ip, M[i], c[i], z[i], n_scan, out + i * OF_N);
  (void)nthreads;
}

/* ------------------------------------------------------------------ */
/* Profiles of a solved halo (Sections 2.1, 2.3, 3.2).                 */
/* ------------------------------------------------------------------ */
typedef struct {
  o_nfw h;
  double n, phi0, T, rho0, P0, rf, r500, ant, n_nt, pe_frac;
} o_prof;
static void o_prof_init(o_prof* p, const orc_cosmo* cp, const orc_icm* ip, const double* m) {
  p->h.M = m[OF_M];
  p->h.c = m[OF_C];
  p->h.rvir = m[OF_RVIR];
  p->h.rs = m[OF_RS];
  p->h.rhos = m[OF_RHOS];
  p->h.mc = m[OF_MC];
  p->h.G = o_G();
  p->n = 1.0 / (ip->Gamma - 1.0);
  p->phi0 = m[OF_PHI0];
  p->T = m[OF_T];
  p->rho0 = m[OF_RHO0];
  p->P0 = m[OF_P0];
  p->rf = m[OF_RF];
  p->r500 = m[OF_R500];
  p->ant = m[OF_ANT];
  p->n_nt = ip->n_nt;
  p->pe_frac = (2.0 * cp->XH + 2.0) / (5.0 * cp->XH + 3.0);
}
static double o_prof_theta(const o_prof* p, double r) {
  return 1.0 + (p->phi0 - o_phi(&p->h, r)) / ((p->n + 1.0) * p->T);
}
/* electron pressure P_e = (2X+2)/(5X+3) P_tot max(0, 1 - R_nt) */
static double o_Pe(const o_prof* p, double r) {
  if (r >= p->rf) return 0.0;
  double th = o_prof_theta(p, r);
  if (th <= 0) return 0.0;
  double Ptot = p->P0 * pow(th, p->n + 1.0);
  double Rnt = p->ant * pow(r / p->r500, p->n_nt);
  return p->pe_frac * Ptot * fmax(0.0, 1.0 - Rnt);
}
/* gas density rho_g = rho0 theta^n */
static double o_rhog(const o_prof* p, double r) {
  if (r >= p->rf) return 0.0;
  double th = o_prof_theta(p, r);
  return th > 0 ? p->rho0 * pow(th, p->n) : 0.0;
}
/* radius where R_nt = 1 (thermal pressure reaches zero), or +inf */
static double o_r_nt1(const o_prof* p) {
  if (p->ant <= 0) return INFINITY;
  return p->r500 * pow(1.0 / p->ant, 1.0 / p->n_nt);
}

void orc_profile(const orc_cosmo* cp, const orc_icm* ip, const double* model, int64_t n,
                 const double* r, double* Pe, double* rhog, double* Ptot) {
  o_prof p;
  o_prof_init(&p, cp, ip, model);
  for (int64_t i = 0; i < n; ++i) {
    Pe[i] = o_Pe(&p, r[i]);
    rhog[i] = o_rhog(&p, r[i]);
    double th = o_prof_theta(&p, r[i]);
    Ptot[i] = (r[i] < p.rf && th > 0) ? p.P0 * pow(th, p.n + 1.0) : 0.0;
  }
}

/* Potential and enclosed mass, exposed for tests. */
void orc_nfw_eval(const orc_cosmo* cp, double M_hinv, double c, double z, int64_t n,
                  const double* r, double* rho, double* Menc, double* phi) {
  o_nfw h;
  o_nfw_init(&h, cp, M_hinv / cp->h, c, z);
  for (int64_t i = 0; i < n; ++i) {
    rho[i] = o_rho_tot(&h, r[i]);
    Menc[i] = o_M_tot(&h, r[i]);
    phi[i] = o_phi(&h, r[i]);
  }
}

/* ------------------------------------------------------------------ */
/* Unit conversions for the observables (Section 3.2).                 */
/* ------------------------------------------------------------------ */
/* y per (pressure x length):  sigma_T/(m_e c^2) P dl  with P in Msun(km/s)^2/Mpc^3, dl in Mpc */
static double o_CP(void) {
  return O_SIGMA_T / O_ME_C2_J * O_MSUN_KG * 1.0e6 / (O_MPC_M * O_MPC_M);
}
/* sigma_T n_e dl with rho_g in Msun/Mpc^3: n_e = rho_g/(mu_e m_p) */
static double o_CN(const orc_cosmo* cp) {
  return O_SIGMA_T * O_MSUN_KG / (o_mu_e(cp) * O_MP_KG * O_MPC_M * O_MPC_M);
}
double orc_const_CP(void) { return o_CP(); }
double orc_const_CN(const orc_cosmo* cp) { return o_CN(cp); }

/* Section 3.2: frequency factor of the tSZ temperature change, Delta T / T_CMB = g(x) y
 * with x = h nu / (k_B T_CMB).  Reading of the printed factor: it shows the ratio
 * (e^x - 1)/(e^x + 1), whose Rayleigh-Jeans limit would be -4; the non-relativistic
 * Kompaneets solution that the section invokes gives the inverse ratio,
 * g(x) = x (e^x + 1)/(e^x - 1) - 4 = x coth(x/2) - 4 (-2 as x -> 0, null near 217 GHz),
 * which is used here. */
double orc_g_nu(double nu_ghz, double Tcmb) {
  double x = O_H_PLANCK * (nu_ghz * 1.0e9) / (O_K_B * Tcmb);
  return x / tanh(0.5 * x) - 4.0;
}

/* ------------------------------------------------------------------ */
/* Halo-based pasting (Section 3.3, Eqs. y^HP and b^HP).                */
/* ------------------------------------------------------------------ */
typedef struct { const o_prof* p; double rperp; int which; } o_los;
static double f_los(double x, void* vctx) {
  const o_los* l = (const o_los*)vctx;
  double r = sqrt(l->rperp * l->rperp + x * x);
  return l->which == 0 ? o_Pe(l->p, r) : o_rhog(l->p, r);
}
/* 2 int_0^{sqrt(rf^2-rperp^2)} q(sqrt(rperp^2+x^2)) dx, split where the 3-D radius
 * crosses r_vir and the zero of the thermal fraction. */
static double o_los_integral(const o_prof* p, double rperp, int which, double rtol) {
  if (rperp >= p->rf) return 0.0;
  double L = sqrt(p->rf * p->rf - rperp * rperp);
  double pts[2];
  int np = 0;
  double radii[2] = {p->h.rvir, o_r_nt1(p)};
  for (int k = 0; k < 2; ++k)
    if (radii[k] > rperp && radii[k] < p->rf) pts[np++] = sqrt(radii[k] * radii[k] - rperp * rperp);
  o_los l = {p, rperp, which};
  return 2.0 * o_quad_split(f_los, &l, 0.0, L, pts, np, rtol);
}
double orc_los_integral(const orc_cosmo* cp, const orc_icm* ip, const double* model,
                        double rperp, int which, double rtol) {
  o_prof p;
  o_prof_init(&p, cp, ip, model);
  return o_los_integral(&p, rperp, which, rtol);
}

typedef struct { int nx, ny, n_maps; double theta0_x, theta0_y, dtheta; } orc_geom;

/* HP map: for every pixel centre with r_perp < r_ap, add the LOS integrals of every halo.
 * Parallel over pixel rows; each pixel sums halos in input order (deterministic). */
void orc_hp_map(const orc_cosmo* cp, const orc_icm* ip, int64_t nh, const double* thx,
                const double* thy, const double* vlos, const int32_t* map_id,
                const double* models, const orc_geom* g, double ap_r500, double rtol,
                double* ymap, double* bmap, int nthreads) {
  double CP = o_CP(), CN = o_CN(cp);
  int64_t npix = (int64_t)g->nx * g->ny;
#ifdef _OPENMP
  if (nthreads > 0) omp_set_num_threads(nthreads);
#pragma omp parallel for schedule(dynamic, 1)
#endif
  for (int64_t row = 0; row < (int64_t)g->ny * g->n_maps; ++row) {
    int mp = (int)(row / g->ny), j = (int)(row % g->ny);
    double ty = g->theta0_y + (j + 0.5) * g->dtheta;
    for (int64_t k = 0; k < nh; ++k) {
      const double* m = models + k * OF_N;
      if (m[OF_STATUS] != 0) continue;
      if ((map_id ? map_id[k] : 0) != mp) continue;
      double rap = m[OF_RF];
      if (ap_r500 > 0) rap = fmin(rap, ap_r500 * m[OF_R500]);
      double DA = m[OF_DA];
      double rad = rap / DA; /* angular aperture */
      if (fabs(ty - thy[k]) >= rad) continue;
      o_prof p;
      o_prof_init(&p, cp, ip, m);
      double bfac = CN * (vlos[k] / O_C_KMS) * exp(-m[OF_TAU]);
      for (int i = 0; i < g->nx; ++i) {
        double tx = g->theta0_x + (i + 0.5) * g->dtheta;
        double dx = tx - thx[k], dy = ty - thy[k];
        double rperp = DA * sqrt(dx * dx + dy * dy);
        if (rperp >= rap) continue;
        int64_t idx = (int64_t)mp * npix + (int64_t)j * g->nx + i;
        ymap[idx] += CP * o_los_integral(&p, rperp, 0, rtol);
        bmap[idx] += bfac * o_los_integral(&p, rperp, 1, rtol);
      }
    }
  }
  (void)nthreads;
}

/* ------------------------------------------------------------------ */
/* Particle-based pasting (Section 3.4).                                */
/* ------------------------------------------------------------------ */
/* Integrated, normalised 1-D kernel w_SPH (Eq. integrated kernel). */
double orc_w_sph(double x) {
  if (x <= -1.0) return 0.0;
  if (x <= -0.5) return 2.0 / 3.0 * pow(1.0 + x, 4);
  if (x <= 0.0) return 4.0 / 3.0 * (3.0 / 8.0 + x - 2.0 * x * x * x - 1.5 * x * x * x * x);
  if (x <= 0.5) return 4.0 / 3.0 * (3.0 / 8.0 + x - 2.0 * x * x * x + 1.5 * x * x * x * x);
  if (x <= 1.0) return 1.0 - 2.0 / 3.0 * pow(1.0 - x, 4);
  return 1.0;
}

/* Per-particle signals (Eqs. y_i^PP,h, b_i^PP,h, field_y, field_b).
 * Output per particle (FP64): pixel coordinates px,py (pixel units from the map's
 * lower-left edge), kernel radius hp in pixels, Y = y_i (pixel-y units) and B = b_i,
 * and kind (0 halo, 1 field, 2 no contribution). */
/* Potential-based variant: with phi (per-particle potential, (km/s)^2, zero at infinity) a
 * halo particle's polytropic variable is theta_i = 1 + (Phi0 - phi_i) / ((n + 1) T) -- the
 * relation theta(Phi) of Section 2.1 at the particle's own potential -- instead of
 * theta(r_i); P_e and rho_g follow from theta_i, V_i, R_nt and the r_f cut stay at r_i.
 * phi = NULL: the paper's spherical assignment. */
void orc_pp_assign_phi(const orc_cosmo* cp, const orc_icm* ip, int64_t n, const float* x,
                       const float* y, const float* zc, const float* vx, const float* vy,
                       const float* vz, const float* phi, const float* hsml, const int32_t* hid,
                       double Mp_hinv, int64_t nh, const float* hpos /*[3][nh]*/,
                       const double* models, const orc_geom* g, double* px, double* py,
                       double* hp, double* Y, double* B, int32_t* kind, int nthreads);
void orc_pp_assign(const orc_cosmo* cp, const orc_icm* ip, int64_t n, const float* x,
                   const float* y, const float* zc, const float* vx, const float* vy,
                   const float* vz, const float* hsml, const int32_t* hid, double Mp_hinv,
                   int64_t nh, const float* hpos /*[3][nh]*/, const double* models,
                   const orc_geom* g, double* px, double* py, double* hp, double* Y,
                   double* B, int32_t* kind, int nthreads) {
  orc_pp_assign_phi(cp, ip, n, x, y, zc, vx, vy, vz, NULL, hsml, hid, Mp_hinv, nh, hpos, models,
                    g, px, py, hp, Y, B, kind, nthreads);
}

void orc_pp_assign_phi(const orc_cosmo* cp, const orc_icm* ip, int64_t n, const float* x,
                       const float* y, const float* zc, const float* vx, const float* vy,
                       const float* vz, const float* phi, const float* hsml, const int32_t* hid,
                       double Mp_hinv, int64_t nh, const float* hpos /*[3][nh]*/,
                       const double* models, const orc_geom* g, double* px, double* py,
                       double* hp, double* Y, double* B, int32_t* kind, int nthreads) {
  double CP = o_CP(), CN = o_CN(cp);
  double h = cp->h, fb = cp->Ob / cp->Om;
  double Mp = Mp_hinv / h;
  double om_pix = g->dtheta * g->dtheta;
#ifdef _OPENMP
  if (nthreads > 0) omp_set_num_threads(nthreads);
#pragma omp parallel for schedule(static, 4096)
#endif
  for (int64_t i = 0; i < n; ++i) {
    double X = (double)x[i] / h, Yc = (double)y[i] / h, Z = (double)zc[i] / h;
    double chi = sqrt(X * X + Yc * Yc + Z * Z);
    px[i] = (atan2(X, Z) - g->theta0_x) / g->dtheta;
    py[i] = (atan2(Yc, Z) - g->theta0_y) / g->dtheta;
    Y[i] = 0.0;
    B[i] = 0.0;
    kind[i] = 2;
    if (!(chi > 0)) { hp[i] = 0.0; continue; }
    hp[i] = ((double)hsml[i] / h) / chi / g->dtheta;
    double zp = orc_z_of_chi(cp, chi);
    double DA = chi / (1.0 + zp);
    double tau = orc_tau(cp, zp);
    double vr = ((double)vx[i] * X + (double)vy[i] * Yc + (double)vz[i] * Z) / chi;
    double geo = 1.0 / (DA * DA * om_pix);
    int32_t k = hid[i];
    if (k < 0) {
      double ne_mass = Mp * (ip->field_fb ? fb : 1.0);
      B[i] = CN * (vr / O_C_KMS) * exp(-tau) * ne_mass * geo;
      kind[i] = 1;
      continue;
    }
    if (k >= nh) continue;
    const double* m = models + k * OF_N;
    if (m[OF_STATUS] != 0) continue;
    double dx = (double)x[i] - (double)hpos[k];
    double dy = (double)y[i] - (double)hpos[nh + k];
    double dz = (double)zc[i] - (double)hpos[2 * nh + k];
    double r = sqrt(dx * dx + dy * dy + dz * dz) / h / (1.0 + m[OF_Z]);
    o_prof p;
    o_prof_init(&p, cp, ip, m);
    if (r >= p.rf) continue;
    double V = Mp / o_rho_nfw(&p.h, r); /* volume from the NFW density at r_i */
    if (phi) {
      double th = 1.0 + (p.phi0 - (double)phi[i]) / ((p.n + 1.0) * p.T);
      double Pe = 0.0, rg = 0.0;
      if (th > 0) {
        double Rnt = p.ant * pow(r / p.r500, p.n_nt);
        Pe = p.pe_frac * p.P0 * pow(th, p.n + 1.0) * fmax(0.0, 1.0 - Rnt);
        rg = p.rho0 * pow(th, p.n);
      }
      Y[i] = CP * Pe * V * geo;
      B[i] = CN * (vr / O_C_KMS) * exp(-tau) * rg * V * geo;
    } else {
      Y[i] = CP * o_Pe(&p, r) * V * geo;
      B[i] = CN * (vr / O_C_KMS) * exp(-tau) * o_rhog(&p, r) * V * geo;
    }
    kind[i] = 0;
  }
  (void)nthreads;
}

/* Deposit through the separable pixel-integrated kernel (Eq. f_ij).
 * select: 0 all, 1 halo particles only (kind 0), 2 field only (kind 1).
 * Maps are [ny][nx] row-major FP64 and are accumulated into.  Particles are
 * summed in index order; rows are distributed over threads (deterministic). */
static void o_axis_weights(double c, double hp, int lo, int hi, double* w) {
  for (int i = lo; i <= hi; ++i) {
    if (hp > 0)
      w[i - lo] = orc_w_sph((i + 1 - c) / hp) - orc_w_sph((i - c) / hp);
    else
      w[i - lo] = (floor(c) == (double)i) ? 1.0 : 0.0; /* h = 0: nearest grid point */
  }
}
void orc_pp_deposit(int64_t n, const double* px, const double* py, const double* hp,
                    const double* Y, const double* B, const int32_t* kind, const orc_geom* g,
                    int select, double* ymap, double* bmap, int nthreads) {
  int nth = 1;
#ifdef _OPENMP
  if (nthreads > 0) omp_set_num_threads(nthreads);
#pragma omp parallel
  {
#pragma omp single
    nth = omp_get_num_threads();
  }
#endif
  (void)nthreads;
  int band = (g->ny + nth - 1) / nth;
#ifdef _OPENMP
#pragma omp parallel for schedule(static, 1)
#endif
  for (int t = 0; t < nth; ++t) {
    int j0 = t * band, j1 = j0 + band - 1;
    if (j1 > g->ny - 1) j1 = g->ny - 1;
    double* wa = (double*)malloc(sizeof(double) * (g->nx + 2));
    double* wb = (double*)malloc(sizeof(double) * (g->ny + 2));
    for (int64_t k = 0; k < n && j0 <= j1; ++k) {
      if (kind[k] == 2) continue;
      if (select == 1 && kind[k] != 0) continue;
      if (select == 2 && kind[k] != 1) continue;
      double h = hp[k];
      if (!(h >= 0.0)) continue; /* a negative or NaN radius covers nothing */
      int ilo = (int)fmax(0.0, floor(px[k] - h)), ihi = (int)fmin(g->nx - 1.0, floor(px[k] + h));
      int jlo = (int)fmax((double)j0, floor(py[k] - h)), jhi = (int)fmin((double)j1, floor(py[k] + h));
      if (floor(px[k] + h) < 0 || floor(px[k] - h) > g->nx - 1) continue;
      if (ilo > ihi || jlo > jhi) continue;
      o_axis_weights(px[k], h, ilo, ihi, wa);
      o_axis_weights(py[k], h, jlo, jhi, wb);
      for (int j = jlo; j <= jhi; ++j) {
        double fy = Y[k] * wb[j - jlo], fbv = B[k] * wb[j - jlo];
        double* yr = ymap + (int64_t)j * g->nx;
        double* br = bmap + (int64_t)j * g->nx;
        for (int i = ilo; i <= ihi; ++i) {
          yr[i] += fy * wa[i - ilo];
          br[i] += fbv * wa[i - ilo];
        }
      }
    }
    free(wa);
    free(wb);
  }
}

/* Value of the deposited maps at a list of pixels, one by one (for full-size
 * parity on sampled outputs).  Same arithmetic as orc_pp_deposit. */
void orc_pp_deposit_pixels(int64_t n, const double* px, const double* py, const double* hp,
                           const double* Y, const double* B, const int32_t* kind,
                           const orc_geom* g, int select, int64_t npx, const int32_t* pix_i,
                           const int32_t* pix_j, double* yv, double* bv, int nthreads) {
#ifdef _OPENMP
  if (nthreads > 0) omp_set_num_threads(nthreads);
#pragma omp parallel for schedule(dynamic, 1)
#endif
  for (int64_t q = 0; q < npx; ++q) {
    int i = pix_i[q], j = pix_j[q];
    double sy = 0.0, sb = 0.0;
    for (int64_t k = 0; k < n; ++k) {
      if (kind[k] == 2) continue;
      if (select == 1 && kind[k] != 0) continue;
      if (select == 2 && kind[k] != 1) continue;
      double h = hp[k];
      if (!(h >= 0.0)) continue;
      if (floor(px[k] - h) > i || floor(px[k] + h) < i) continue;
      if (floor(py[k] - h) > j || floor(py[k] + h) < j) continue;
      double a, b;
      o_axis_weights(px[k], h, i, i, &a);
      o_axis_weights(py[k], h, j, j, &b);
      sy += Y[k] * b * a;
      sb += B[k] * b * a;
    }
    yv[q] = sy;
    bv[q] = sb;
  }
  (void)nthreads;
}

/* ------------------------------------------------------------------ */
/* Tile membership of particles (integer work, decided in FP32).
 * A particle at pixel position px = ix + fx (integer index, FP32 fraction) with
 * radius hp covers pixel columns ix + floor(fx - hp) .. ix + floor(fx + hp), the two
 * bounds computed in single precision (round-to-nearest, no contraction), clipped
 * to the map; a negative or NaN radius covers nothing.  Tiles are TWxTH pixel
 * blocks keyed key = ty * ntx + tx.  Output: (key, particle index) pairs ordered by
 * key, ties by particle index.  Returns the pair count; if keys==NULL only counts. */
static int o_span32(int32_t ix, float fx, float h, int n, int* lo, int* hi) {
  if (!(h >= 0.0f) || !(fx == fx)) return 0;
  volatile float a = fx - h, b = fx + h; /* single-precision rounding, no fusion */
  float fa = floorf(a), fb = floorf(b);
  if (fa < -4.0e9f) fa = -4.0e9f;
  if (fb > 4.0e9f) fb = 4.0e9f;
  long long L = (long long)ix + (long long)fa, H = (long long)ix + (long long)fb;
  if (H < 0 || L > n - 1) return 0;
  *lo = L < 0 ? 0 : (int)L;
  *hi = H > n - 1 ? n - 1 : (int)H;
  return 1;
}
int64_t orc_pp_pairs(int64_t n, const int32_t* ix, const float* fx, const int32_t* iy,
                     const float* fy, const float* hp, const int32_t* kind, int nx, int ny,
                     int tw, int th, int select, uint32_t* keys, uint32_t* vals) {
  int ntx = (nx + tw - 1) / tw, nty = (ny + th - 1) / th;
  int64_t* cnt = (int64_t*)calloc((size_t)ntx * nty + 1, sizeof(int64_t));
  int64_t total = 0;
  for (int pass = 0; pass < 2; ++pass) {
    for (int64_t k = 0; k < n; ++k) {
      if (kind[k] == 2) continue;
      if (select == 1 && kind[k] != 0) continue;
      if (select == 2 && kind[k] != 1) continue;
      int i0, i1, j0, j1;
      if (!o_span32(ix[k], fx[k], hp[k], nx, &i0, &i1)) continue;
      if (!o_span32(iy[k], fy[k], hp[k], ny, &j0, &j1)) continue;
      for (int ty = j0 / th; ty <= j1 / th; ++ty)
        for (int tx = i0 / tw; tx <= i1 / tw; ++tx) {
          int64_t key = (int64_t)ty * ntx + tx;
          if (pass == 0) { cnt[key + 1]++; total++; }
          else if (keys) { int64_t pos = cnt[key]++; keys[pos] = (uint32_t)key; vals[pos] = (uint32_t)k; }
        }
    }
    if (pass == 0) {
      if (!keys) break;
      for (int64_t t = 0; t < (int64_t)ntx * nty; ++t) cnt[t + 1] += cnt[t];
    }
  }
  free(cnt);
  (void)nty;
  return total;
}

/* (halo, tile) membership for HP, decided in FP64: pixel-centre bounding box of
 * the aperture disc, floor((c - rad)) .. floor((c + rad)) in pixel units,
 * clipped; pairs ordered by (map, tile) key then halo index. */
int64_t orc_hp_pairs(int64_t nh, const double* thx, const double* thy, const int32_t* map_id,
                     const double* models, const orc_geom* g, double ap_r500, int tw, int th,
                     uint32_t* keys, uint32_t* vals) {
  int ntx = (g->nx + tw - 1) / tw, nty = (g->ny + th - 1) / th;
  int64_t ntiles = (int64_t)ntx * nty * g->n_maps;
  int64_t* cnt = (int64_t*)calloc((size_t)ntiles + 1, sizeof(int64_t));
  int64_t total = 0;
  for (int pass = 0; pass < 2; ++pass) {
    for (int64_t k = 0; k < nh; ++k) {
      const double* m = models + k * OF_N;
      if (m[OF_STATUS] != 0) continue;
      int mp = map_id ? map_id[k] : 0;
      if (mp < 0 || mp >= g->n_maps) continue;
      double rap = m[OF_RF];
      if (ap_r500 > 0) rap = fmin(rap, ap_r500 * m[OF_R500]);
      double rad = rap / m[OF_DA] / g->dtheta;
      double cx = (thx[k] - g->theta0_x) / g->dtheta - 0.5;
      double cy = (thy[k] - g->theta0_y) / g->dtheta - 0.5;
      double fa = floor(cx - rad), fb = floor(cx + rad);
      double ga = floor(cy - rad), gb = floor(cy + rad);
      if (fb < 0 || fa > g->nx - 1 || gb < 0 || ga > g->ny - 1) continue;
      int i0 = fa < 0 ? 0 : (int)fa, i1 = fb > g->nx - 1 ? g->nx - 1 : (int)fb;
      int j0 = ga < 0 ? 0 : (int)ga, j1 = gb > g->ny - 1 ? g->ny - 1 : (int)gb;
      for (int ty = j0 / th; ty <= j1 / th; ++ty)
        for (int tx = i0 / tw; tx <= i1 / tw; ++tx) {
          int64_t key = ((int64_t)mp * nty + ty) * ntx + tx;
          if (pass == 0) { cnt[key + 1]++; total++; }
          else if (keys) { int64_t pos = cnt[key]++; keys[pos] = (uint32_t)key; vals[pos] = (uint32_t)k; }
        }
    }
    if (pass == 0) {
      if (!keys) break;
      for (int64_t t = 0; t < ntiles; ++t) cnt[t + 1] += cnt[t];
    }
  }
  free(cnt);
  return total;
}

/* Energy residual as a function of r_f, with T from the gas-mass condition at that
 * r_f (the reduced one-dimensional problem of Section 2.2).  NAN where no T exists. */
double orc_energy_residual(const orc_cosmo* cp, const orc_icm* ip, double M_hinv, double c,
                           double z, double rf_over_rvir) {
  double out[OF_N];
  orc_halo_solve(cp, ip, M_hinv, c, z, 8, out);
  o_solver s;
  s.cp = cp;
  s.ip = ip;
  o_nfw_init(&s.h, cp, M_hinv / cp->h, c, z);
  s.fb = cp->Ob / cp->Om;
  s.n = 1.0 / (ip->Gamma - 1.0);
  s.phi0 = o_phi0(&s.h);
  s.Mstar = out[OF_MSTAR];
  s.Egi = out[OF_EGI];
  s.Edm = out[OF_EDM];
  s.Ps = out[OF_PS];
  return f_rese_rf(rf_over_rvir * s.h.rvir, &s);
}

/* Particles whose kernel support covers at least one of the listed pixels (FP64 spans
 * as in orc_pp_deposit): a geometric pre-filter so that sampled pixels of a very large
 * light-cone can be computed from the few particles that reach them.  Writes the
 * indices (ascending) and returns their count. */
int64_t orc_pp_select(const orc_cosmo* cp, int64_t n, const float* x, const float* y,
                      const float* zc, const float* hsml, const orc_geom* g, int64_t npx,
                      const int32_t* pix_i, const int32_t* pix_j, int64_t* out, int nthreads) {
  double h = cp->h;
  char* hit = (char*)calloc((size_t)n, 1);
#ifdef _OPENMP
  if (nthreads > 0) omp_set_num_threads(nthreads);
#pragma omp parallel for schedule(static, 65536)
#endif
  for (int64_t k = 0; k < n; ++k) {
    double X = (double)x[k] / h, Yc = (double)y[k] / h, Z = (double)zc[k] / h;
    double chi = sqrt(X * X + Yc * Yc + Z * Z);
    if (!(chi > 0)) continue;
    double px = (atan2(X, Z) - g->theta0_x) / g->dtheta;
    double py = (atan2(Yc, Z) - g->theta0_y) / g->dtheta;
    double hp = ((double)hsml[k] / h) / chi / g->dtheta;
    double i0 = floor(px - hp), i1 = floor(px + hp), j0 = floor(py - hp), j1 = floor(py + hp);
    for (int64_t q = 0; q < npx; ++q)
      if (pix_i[q] >= i0 && pix_i[q] <= i1 && pix_j[q] >= j0 && pix_j[q] <= j1) {
        hit[k] = 1;
        break;
      }
  }
  (void)nthreads;
  int64_t m = 0;
  for (int64_t k = 0; k < n; ++k)
    if (hit[k]) out[m++] = k;
  free(hit);
  return m;
}

/* HP values at a list of pixels (same arithmetic as orc_hp_map, pixel by pixel). */
void orc_hp_pixels(const orc_cosmo* cp, const orc_icm* ip, int64_t nh, const double* thx,
                   const double* thy, const double* vlos, const int32_t* map_id,
                   const double* models, const orc_geom* g, double ap_r500, double rtol,
                   int64_t npx, const int32_t* pix_m, const int32_t* pix_i, const int32_t* pix_j,
                   double* yv, double* bv, int nthreads) {
  double CP = o_CP(), CN = o_CN(cp);
#ifdef _OPENMP
  if (nthreads > 0) omp_set_num_threads(nthreads);
#pragma omp parallel for schedule(dynamic, 1)
#endif
  for (int64_t q = 0; q < npx; ++q) {
    double tx = g->theta0_x + (pix_i[q] + 0.5) * g->dtheta;
    double ty = g->theta0_y + (pix_j[q] + 0.5) * g->dtheta;
    double sy = 0.0, sb = 0.0;
    for (int64_t k = 0; k < nh; ++k) {
      const double* m = models + k * OF_N;
      if (m[OF_STATUS] != 0) continue;
      if ((map_id ? map_id[k] : 0) != (pix_m ? pix_m[q] : 0)) continue;
      double rap = m[OF_RF];
      if (ap_r500 > 0) rap = fmin(rap, ap_r500 * m[OF_R500]);
      double dx = tx - thx[k], dy = ty - thy[k];
      double rperp = m[OF_DA] * sqrt(dx * dx + dy * dy);
      if (rperp >= rap) continue;
      o_prof p;
      o_prof_init(&p, cp, ip, m);
      sy += CP * o_los_integral(&p, rperp, 0, rtol);
      sb += CN * (vlos[k] / O_C_KMS) * exp(-m[OF_TAU]) * o_los_integral(&p, rperp, 1, rtol);
    }
    yv[q] = sy;
    bv[q] = sb;
  }
  (void)nthreads;
}

/* ------------------------------------------------------------------ */
/* All-sky HP (Section 5.2, all-sky maps) on the HEALPix sphere of Gorski et al. (2005), */
/* RING ordering: 12 nside^2 equal-area pixels on 4 nside - 1 rings of constant z.       */
/* ------------------------------------------------------------------ */
/* Ring i (1 .. 4N - 1 from the north pole, N = nside): z = cos(theta) of its centres, pixel
 * count, RING index of its first pixel, and the longitude of that first centre in units of
 * the ring's pixel spacing 2 pi / count.  Polar caps (i < N and i > 3N): 4i pixels (4(4N - i)
 * in the south), half-spacing offset; equatorial belt: 4N pixels, offset alternating with i. */
static void o_hpx_ring(int64_t N, int64_t i, double* z, int64_t* cnt, int64_t* first,
                       double* phase) {
  if (i < N) {
    *z = 1.0 - (double)(i * i) / (3.0 * (double)N * (double)N);
    *cnt = 4 * i;
    *first = 2 * i * (i - 1);
    *phase = 0.5;
  } else if (i <= 3 * N) {
    *z = 4.0 / 3.0 - 2.0 * (double)i / (3.0 * (double)N);
    *cnt = 4 * N;
    *first = 2 * N * (N - 1) + 4 * N * (i - N);
    *phase = ((i + N) & 1) ? 0.0 : 0.5;
  } else {
    int64_t k = 4 * N - i;
    *z = -(1.0 - (double)(k * k) / (3.0 * (double)N * (double)N));
    *cnt = 4 * k;
    *first = 12 * N * N - 2 * k * (k + 1);
    *phase = 0.5;
  }
}

/* Centre (colatitude theta, longitude phi in [0, 2 pi)) of RING pixel p. */
void orc_hpx_pix2ang(int64_t N, int64_t p, double* theta, double* phi) {
  int64_t lo = 1, hi = 4 * N - 1; /* the last ring whose first pixel is <= p */
  while (lo < hi) {
    int64_t mid = (lo + hi + 1) / 2, cnt, first;
    double z, ph;
    o_hpx_ring(N, mid, &z, &cnt, &first, &ph);
    if (first <= p) lo = mid; else hi = mid - 1;
  }
  int64_t cnt, first;
  double z, ph;
  o_hpx_ring(N, lo, &z, &cnt, &first, &ph);
  *theta = acos(z);
  *phi = ((double)(p - first) + ph) * (2.0 * O_PI / (double)cnt);
}

void orc_hpx_centres(int64_t N, int64_t n, const int64_t* pix, double* theta, double* phi) {
  for (int64_t q = 0; q < n; ++q) orc_hpx_pix2ang(N, pix[q], theta + q, phi + q);
}

/* Great-circle angle between directions (t1, p1) and (t2, p2), robust at all separations. */
double orc_sky_angle(double t1, double p1, double t2, double p2) {
  double a[3] = {sin(t1) * cos(p1), sin(t1) * sin(p1), cos(t1)};
  double b[3] = {sin(t2) * cos(p2), sin(t2) * sin(p2), cos(t2)};
  double cx = a[1] * b[2] - a[2] * b[1], cy = a[2] * b[0] - a[0] * b[2], cz = a[0] * b[1] - a[1] * b[0];
  return atan2(sqrt(cx * cx + cy * cy + cz * cz), a[0] * b[0] + a[1] * b[1] + a[2] * b[2]);
}

/* All-sky HP at listed pixel directions: every halo whose aperture contains the direction
 * adds its LOS integrals at r_perp = D_A psi, psi the great-circle angle to the halo
 * (the flat-sky r_perp = D_A |theta - theta_h| with the angle measured on the sphere). */
void orc_hp_sky(const orc_cosmo* cp, const orc_icm* ip, int64_t nh, const double* h_theta,
                const double* h_phi, const double* vlos, const double* models, double ap_r500,
                double rtol, int64_t npx, const double* p_theta, const double* p_phi, double* yv,
                double* bv, int nthreads) {
  double CP = o_CP(), CN = o_CN(cp);
#ifdef _OPENMP
  if (nthreads > 0) omp_set_num_threads(nthreads);
#pragma omp parallel for schedule(dynamic, 16)
#endif
  for (int64_t q = 0; q < npx; ++q) {
    double sy = 0.0, sb = 0.0;
    for (int64_t k = 0; k < nh; ++k) {
      const double* m = models + k * OF_N;
      if (m[OF_STATUS] != 0) continue;
      double rap = m[OF_RF];
      if (ap_r500 > 0) rap = fmin(rap, ap_r500 * m[OF_R500]);
      double rperp = m[OF_DA] * orc_sky_angle(p_theta[q], p_phi[q], h_theta[k], h_phi[k]);
      if (rperp >= rap) continue;
      o_prof p;
      o_prof_init(&p, cp, ip, m);
      sy += CP * o_los_integral(&p, rperp, 0, rtol);
      sb += CN * (vlos[k] / O_C_KMS) * exp(-m[OF_TAU]) * o_los_integral(&p, rperp, 1, rtol);
    }
    yv[q] = sy;
    bv[q] = sb;
  }
  (void)nthreads;
}

/* ------------------------------------------------------------------ */
/* Smoothing lengths (Section 3.4: the SPH kernel Eq. SPH_kernel and the  */
/* effective neighbour number N_ngb).                                     */
/* ------------------------------------------------------------------ */
/* 3-D cubic spline of Eq. SPH_kernel without its 8 / (pi h^3) factor, x = r / h. */
static double o_w3(double x) {
  if (x < 0.5) return 1.0 - 6.0 * x * x + 6.0 * x * x * x;
  if (x < 1.0) return 2.0 * (1.0 - x) * (1.0 - x) * (1.0 - x);
  return 0.0;
}
double orc_w3(double x) { return o_w3(x); }

static int o_cmp_double(const void* a, const void* b) {
  double u = *(const double*)a, v = *(const double*)b;
  return (u > v) - (u < v);
}

/* Effective number of neighbours within h of a particle whose distances to every particle
 * (itself included, distance 0) are d[0..n-1] in ascending order:
 * N_eff(h) = (4 pi / 3) h^3 sum_j W(d_j, h) = (32 / 3) sum_j w(d_j / h). */
static double o_neff(const double* d, int64_t n, double h) {
  double s = 0.0;
  for (int64_t j = 0; j < n && d[j] < h; ++j) s += o_w3(d[j] / h);
  return 32.0 / 3.0 * s;
}

/* Smoothing lengths: for every particle i, the h_i with N_eff(h_i) = n_ngb (N_eff grows
 * monotonically with h), by bisection on the sorted distances to all particles.  Positions
 * in any length unit (FP32 inputs, computed in FP64); h in the same unit.  A particle whose
 * N_eff cannot reach n_ngb (too few particles) gets +inf. */
/* h of particle i from its distances d[0..n-1] (scratch) to all n particles. */
static double o_hsml_one(int64_t n, const float* x, const float* y, const float* z, int64_t i,
                         double n_ngb, double* d) {
  if (32.0 / 3.0 * (double)n <= n_ngb) return INFINITY;
  for (int64_t j = 0; j < n; ++j) {
    double dx = (double)x[j] - (double)x[i], dy = (double)y[j] - (double)y[i];
    double dz = (double)z[j] - (double)z[i];
    d[j] = sqrt(dx * dx + dy * dy + dz * dz);
  }
  qsort(d, (size_t)n, sizeof(double), o_cmp_double);
  /* bracket: N_eff(lo) < n_ngb <= N_eff(hi) */
  double lo = 0.0, hi = d[n - 1] > 0.0 ? d[n - 1] : 1.0;
  while (o_neff(d, n, hi) < n_ngb) hi *= 2.0;
  for (int it = 0; it < 200 && hi - lo > 1e-15 * hi; ++it) {
    double mid = 0.5 * (lo + hi);
    if (o_neff(d, n, mid) < n_ngb) lo = mid; else hi = mid;
  }
  return 0.5 * (lo + hi);
}

/* h of the m particles idx[0..m-1] (h[k] for particle idx[k]); the sums still run over all
 * n particles.  m = n with idx = null: every particle. */
void orc_smoothing_lengths_at(int64_t n, const float* x, const float* y, const float* z,
                              double n_ngb, int64_t m, const int64_t* idx, double* h,
                              int nthreads) {
#ifdef _OPENMP
  if (nthreads > 0) omp_set_num_threads(nthreads);
#else
  (void)nthreads;
#endif
#pragma omp parallel
  {
    double* d = (double*)malloc(sizeof(double) * (size_t)(n > 0 ? n : 1));
#pragma omp for schedule(dynamic, 1)
    for (int64_t k = 0; k < m; ++k) h[k] = o_hsml_one(n, x, y, z, idx ? idx[k] : k, n_ngb, d);
    free(d);
  }
}

void orc_smoothing_lengths(int64_t n, const float* x, const float* y, const float* z,
                           double n_ngb, double* h, int nthreads) {
  orc_smoothing_lengths_at(n, x, y, z, n_ngb, n, NULL, h, nthreads);
}

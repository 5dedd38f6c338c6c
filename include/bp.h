/*
 * bp.h -- C ABI of the GB300 baryon pasting library (libbp.so).
 *
 * Method: Osato & Nagai, "Baryon pasting algorithm: halo-based and particle-based
 * pasting methods" (arXiv:2201.02632).  The library computes, on one GPU:
 *   bp_solve_halos       the per-halo analytic ICM model (Section 2, Eqs. of the
 *                        polytrope, energy conservation, surface pressure, gas mass);
 *   bp_assign_particles  per-particle tSZ/kSZ signals (Section 3.4, Eqs. y_i^PP,h,
 *                        b_i^PP,h, field_y, field_b);
 *   bp_paste_particles   the separable pixel-integrated SPH deposit (Section 3.4,
 *                        Eqs. f_ij and integrated kernel);
 *   bp_paste_halos       halo-based pasting of projected profiles (Section 3.3,
 *                        Eqs. y^HP and b^HP);
 *   bp_finalize_map      folding of the compensation planes and the conversion to
 *                        temperature (Section 3.2).
 *
 * Conventions shared by every call:
 *   - Units: masses in h^-1 Msun, positions and smoothing lengths in comoving
 *     h^-1 Mpc, velocities in km/s (as in N-body catalogues).  Internally the
 *     library works in physical Mpc, Msun and km/s with the cosmology's h.
 *   - Flat sky: observer at the origin, line of sight +z; a position (x, y, z)
 *     has sky angles theta_x = atan2(x, z), theta_y = atan2(y, z) [rad].
 *   - Maps are FP32, row-major [n_maps][ny][nx]; pixel (i, j) spans
 *     [theta0_x + i dtheta, theta0_x + (i+1) dtheta] x [theta0_y + j dtheta, ...].
 *     Every map comes with a same-shaped FP32 "lo" plane holding the running
 *     compensation (hi + lo is the value); paste calls ACCUMULATE into both, the
 *     caller zeroes them first.  bp_finalize_map folds lo into hi.
 *   - All array arguments are DEVICE pointers owned by the caller; the library
 *     never frees them, never keeps them after a call returns, and never writes
 *     an input.  Scratch memory (pair lists, sort buffers, tables) belongs to the
 *     context and grows on demand.
 *   - Every call is asynchronous on the context's stream, except where a call
 *     documents a host synchronisation.
 *   - Return value: BP_OK (0) or a negative error code; bp_last_error() gives a
 *     message.  Invalid arguments are rejected before any work is queued.
 */
#ifndef BP_H
#define BP_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define BP_OK 0
#define BP_EINVAL (-1)    /* bad argument (null pointer, size, geometry) */
#define BP_ECUDA (-2)     /* a CUDA runtime call failed */
#define BP_ERANGE (-3)    /* input outside the supported range (z, map size, ids) */
#define BP_ENOCONV (-4)   /* at least one halo did not converge (see status) */
#define BP_ETIMEOUT (-5)  /* a bounded device wait gave up */
#define BP_ENOMEM (-6)    /* scratch allocation failed */

/* Flat LCDM background (Section 1) plus T_CMB and the hydrogen fraction X
 * (Section 3.2).  Defaults: Om 0.279, Ob 0.046, h 0.7, Tcmb 2.726, XH 0.76. */
typedef struct {
  double Om, Ob, h, Tcmb, XH;
} bp_cosmology;

/* ICM model parameters (Table 1).  energy_sign selects the arrangement of the
 * energy condition: 0 = E_g,f = E_g,i + eps_DM |E_DM| + eps_* M_* c^2 + dE_p
 * (the gas gains the injected energy and does the surface work; gives r_f > r_vir
 * as Section 2.2 states), 1 = the arrangement as printed.  field_fb = 1 multiplies
 * the field-particle electron count by f_b (printed form: 0). */
typedef struct {
  double Gamma, eps_dm, eps_star, f_star, S_star, alpha_nt, beta_nt, n_nt;
  int energy_sign;
  int field_fb;
} bp_icm_params;

/* Flat-sky pixel grid.  theta0_* is the lower-left pixel EDGE in radians. */
typedef struct {
  int nx, ny, n_maps;
  double theta0_x, theta0_y, dtheta;
} bp_map_geom;

/* Solved halo model record: FP64 device array laid out field-major,
 * model[f * n + i] for halo i and field f below.  Physical units: Msun, Mpc,
 * km/s; pressures Msun (km/s)^2 Mpc^-3; densities Msun Mpc^-3. */
enum {
  BP_M_MVIR = 0, /* virial mass [Msun] */
  BP_M_C,        /* concentration */
  BP_M_Z,        /* redshift */
  BP_M_RVIR,     /* virial radius [Mpc] */
  BP_M_RS,       /* NFW scale radius */
  BP_M_RHOS,     /* NFW scale density */
  BP_M_MC,       /* m(c) = ln(1+c) - c/(1+c) */
  BP_M_PHI0,     /* central potential [(km/s)^2] */
  BP_M_R500,
  BP_M_M500,
  BP_M_MSTAR,    /* stellar mass */
  BP_M_RSTAR,    /* stellar radius */
  BP_M_EGI,      /* initial gas energy */
  BP_M_EDM,      /* dark-matter energy */
  BP_M_PS,       /* surface pressure */
  BP_M_T,        /* P0 / rho0 */
  BP_M_RHO0,     /* central gas density */
  BP_M_P0,       /* central total pressure */
  BP_M_RF,       /* gas boundary radius r_f */
  BP_M_ANT,      /* alpha_nt f(z) */
  BP_M_DA,       /* angular-diameter distance [Mpc] */
  BP_M_TAU,      /* mean optical depth to z */
  BP_M_RESM,     /* gas-mass condition residual at the solution */
  BP_M_RESE,     /* energy condition residual at the solution */
  BP_M_NFIELDS
};

/* per-halo status codes written by bp_solve_halos */
#define BP_HALO_OK 0
#define BP_HALO_NOBRACKET 1  /* no r_f bracket found in [0.5, 10] r_vir */
#define BP_HALO_BADSTAR 2    /* M_* >= f_b M_vir: no stellar radius */
#define BP_HALO_THETA 3      /* theta(r_f) <= 0 */
#define BP_HALO_MAXIT 4      /* Newton iteration limit reached */
#define BP_HALO_BADINPUT 5   /* M, c or z not finite / out of range */
#define BP_HALO_FALLBACK 6   /* (internal) rejected by the residual gate, awaiting the full solve */

/* particle record written by bp_assign_particles: BP_ASSIGNED_STRIDE 32-bit words
 * per particle (32 bytes, 16-byte aligned).  The pixel-unit position measured from
 * the map's lower-left edge is px = ix + fx (and py = iy + fy), split into an
 * integer pixel index and an FP32 fraction so that its precision does not depend on
 * the map size:
 *   [0] fx   float, fractional part of px, 0 <= fx < 1
 *   [1] fy   float, fractional part of py
 *   [2] hp   float, kernel radius h in pixels (2h x 2h support square)
 *   [3] Y    float, y_i: the particle's Compton-y in pixel units (Eq. y_i^PP,h)
 *   [4] B    float, b_i: the particle's kSZ b in pixel units (Eqs. b_i^PP,h, field_b)
 *   [5] kind int32, 0 halo particle, 1 field particle, 2 contributes nothing
 *   [6] ix   int32, floor(px), clamped to +-2^30
 *   [7] iy   int32, floor(py), clamped to +-2^30 */
#define BP_ASSIGNED_STRIDE 8
#define BP_KIND_HALO 0
#define BP_KIND_FIELD 1
#define BP_KIND_NONE 2

#define BP_SELECT_ALL 0
#define BP_SELECT_HALO 1
#define BP_SELECT_FIELD 2

#define BP_SOLVE_FP64 0        /* FP64 solve (FP32 pre-solve, then FP64 Newton to resid_tol) */
#define BP_SOLVE_FP64_SEEDED 1 /* bp_solve_halos_ex only: the guess starts the FP32 pre-solve */
#define BP_SOLVE_FP32_GATED 2  /* bp_solve_halos_ex only: the FP32 pre-solve (seeded by the guess
                                * when given) is the answer where both of its FP32 residuals
                                * are <= gate; the other halos get the full FP64 solve */

#define BP_OUT_YB 0     /* maps hold y and b */
#define BP_OUT_DT 1     /* maps hold Delta T / T_CMB: g_nu(x) y and -b, with
                         * g_nu(x) = x (e^x + 1)/(e^x - 1) - 4 (Section 3.2) */

typedef struct bp_ctx bp_ctx;

/* Create a context on the current CUDA device.  stream: a cudaStream_t (NULL = the
 * legacy default stream).  Builds the background tables (chi(z), tau(z), z(chi)) on
 * the host in FP64 and uploads them (synchronous); also loads the device array and the
 * kernels of bp_paste_particles_noalloc on this device (once per device).  Returns
 * BP_EINVAL for non-physical parameters. */
int bp_create(bp_ctx** ctx, const bp_cosmology* cosmo, const bp_icm_params* icm, void* stream);
/* Free the context and its scratch (synchronises its stream). */
int bp_destroy(bp_ctx* ctx);
/* Message of the last error on this context (never NULL). */
const char* bp_last_error(const bp_ctx* ctx);
/* Change the stream later calls are queued on. */
int bp_set_stream(bp_ctx* ctx, void* stream);
/* Tile sizes: PP deposit tile (pixels per side: 32 or 64) and HP tile (32 or 64);
 * pp_unit: maximum particles per deposit work unit (>= 256; -1 = automatic, about 16
 * units per resident CTA).  0 keeps a value. */
int bp_set_tiling(bp_ctx* ctx, int pp_tile, int hp_tile, int pp_unit);
/* Which kernel performs the PP deposit (Section 3.4, Eqs. f_ij and the integrated
 * kernel): BP_DEPOSIT_AUTO (the tensor-core kernel when the PP tile is 64, else the
 * SIMT kernel), BP_DEPOSIT_SIMT (FP32 FMAs on the CUDA cores) or BP_DEPOSIT_TENSOR
 * (tcgen05 MMAs in split FP16 with power-of-two operand scales, tile 64 only; BP_EINVAL
 * at paste time with tile 32).
 * Both sum every pixel in a fixed order with compensated FP32 accumulators; they
 * differ in the rounding of the products (FP32 against about 1e-6 relative). */
#define BP_DEPOSIT_AUTO 0
#define BP_DEPOSIT_SIMT 1
#define BP_DEPOSIT_TENSOR 2
int bp_set_deposit_kernel(bp_ctx* ctx, int kind);
/* With the tensor-core deposit, particles whose pixel box (clipped to the map) is at most
 * `span` pixels on both axes are deposited by a second kernel instead (one CTA per tile, one
 * thread per particle, the same cell weights, exact 64-bit fixed-point sums in shared memory:
 * deterministic), added after the large particles of each tile.  span: 0 (every particle on
 * the tensor cores) .. 8, or -1 (the default): 8 when the map has at least 4 tiles of 64
 * pixels per SM, else 0.  BP_EINVAL outside [-1, 8]. */
int bp_set_small_span(bp_ctx* ctx, int span);
/* Test of the bounded waits (not in the paper): when polls > 0, every CTA of the context's
 * later tensor-core deposits first waits, for at most `polls` reads, on a device flag that
 * nothing sets, before it issues any MMA or writes anything; the deposit then gives up,
 * frees its tensor memory and the paste returns BP_ETIMEOUT with the maps unchanged, and the
 * context stays usable.  polls = 0 (the default) turns the test off.  BP_EINVAL for polls
 * outside [0, 2^31). */
int bp_set_wait_test(bp_ctx* ctx, int64_t polls);
/* Debug build (not in the paper).  A library compiled with -DBP_DEBUG checks, inside the
 * particle paste's kernels, the index of each store that a wrong index would misplace (pair
 * emission 101, radix scatter 201-202, small-particle sums 301-302, tensor-core write-out
 * 401-402, partial-tile reduction 501); a failed check skips that store and records its site
 * code in the context's debug word (the first failure is kept).  The release build compiles
 * the checks out.
 *   bp_debug_build: 1 for a debug build, else 0.
 *   bp_debug_status: *site = the recorded site code (0: none), then clears the word;
 *     synchronises the context's stream.  BP_EINVAL for a null argument.
 *   bp_debug_selftest: records `site` (> 0) as a failed check would (both builds), for
 *     testing the read-back; asynchronous on the context's stream. */
int bp_debug_build(void);
int bp_debug_status(bp_ctx* ctx, int* site);
int bp_debug_selftest(bp_ctx* ctx, int site);
/* Bytes of scratch the context currently holds. */
int64_t bp_workspace_bytes(const bp_ctx* ctx);

/* Phase timing: when on, each call records CUDA events around its kernels on the
 * context's stream.  bp_phase_times synchronises the stream and writes, for every
 * phase index below, the milliseconds accumulated since the previous call to it
 * (then resets).  n: length of ms (>= BP_NPHASES). */
#define BP_PH_SOLVE 0
#define BP_PH_ASSIGN 1
#define BP_PH_PAIRS 2     /* pair count, scan and emit */
#define BP_PH_SORT 3      /* radix sort and tile ranges */
#define BP_PH_DEPOSIT 4   /* work units + the deposit kernel */
#define BP_PH_REDUCE 5    /* partial-tile reduction */
#define BP_PH_HP_TABLE 6  /* HP per-halo tables */
#define BP_PH_HP_PAIRS 7  /* HP (halo, tile) list and sort */
#define BP_PH_HP_PASTE 8  /* HP paste and reduction */
#define BP_PH_FINALIZE 9
#define BP_PH_SURROGATE 10 /* surrogate features + BF16 inference */
#define BP_PH_DEPOSIT_SMALL 11 /* small-particle deposit (bp_set_small_span) */
#define BP_NPHASES 12
int bp_set_timing(bp_ctx* ctx, int on);
int bp_phase_times(bp_ctx* ctx, double* ms, int n);
/* Number of kernels this context has launched since it was created. */
int64_t bp_kernel_launches(const bp_ctx* ctx);

/* Section 2: solve the ICM model of n halos.
 *   Mvir [n] FP64 h^-1 Msun, c [n] FP64, z [n] FP64 (0 <= z <= 10)
 *   model [BP_M_NFIELDS * n] FP64 (field-major, written), status [n] int32 (written)
 *   mode: BP_SOLVE_FP64.  resid_tol: convergence tolerance on the normalised
 *   gas-mass and energy residuals (<= 0 selects 1e-10).
 * Returns BP_ENOCONV if any halo's status is not BP_HALO_OK (this reads back one
 * counter: the call synchronises the stream).  Halos are independent. */
int bp_solve_halos(bp_ctx* ctx, int64_t n, const double* Mvir, const double* c, const double* z,
                   double* model, int32_t* status, int mode, double resid_tol);

/* bp_solve_halos with options (used to generate surrogate training data and by the
 * surrogate path):
 *   params [3 * n] FP64 or NULL: per-halo eps_*, f_*, eps_DM (layout [3][n]); NULL uses
 *     the context's Table-1 values;
 *   guess  [2 * n] FP64 or NULL: starting point ln(r_f / r_vir), ln(T r_vir / (G M_vir))
 *     per halo (layout [2][n]); non-finite entries use the default start;
 *   max_iter: outer Newton iterations (<= 0: 80);
 *   gate > 0 (with guess): a halo not converged to resid_tol within max_iter iterations
 *     is accepted if both normalised residuals are <= gate; otherwise it is solved again
 *     from the default start with the full iteration budget (the fallback).
 *   mode: BP_SOLVE_FP64: the guess starts the FP64 Newton directly;
 *     BP_SOLVE_FP64_SEEDED: the guess starts the FP32 pre-solve, whose result starts the
 *     FP64 Newton (max_iter and gate apply to that Newton; halos without a finite guess
 *     get the pre-solve's default start); without a guess both are bp_solve_halos;
 *     BP_SOLVE_FP32_GATED (gate > 0 required): no FP64 Newton: the FP32 pre-solve's solution
 *     (r_f, T) is accepted where its FP32 energy and gas-mass residuals are both <= gate,
 *     with rho0 and P0 from the pressure condition in FP64 and the FP32 residuals in the
 *     residual fields; every other halo is solved again by the full FP64 iteration and
 *     counted by bp_last_fallback_count.
 * The number of halos sent to the fallback is returned by bp_last_fallback_count.
 * Synchronises (one or two counter reads). */
int bp_solve_halos_ex(bp_ctx* ctx, int64_t n, const double* Mvir, const double* c,
                      const double* z, const double* params, const double* guess, int max_iter,
                      double gate, double* model, int32_t* status, int mode, double resid_tol);
int64_t bp_last_fallback_count(const bp_ctx* ctx);

/* ---- MLP surrogate of the solve (not in the paper).
 * Network 6 -> 128 -> 128 -> 128 -> 3, GELU (exact erf form) on the hidden layers.
 * Features (normalised as (f - mean) / scale with `norm`): log10 M [h^-1 Msun],
 * log10 c, z, eps_*, f_*, eps_DM.  Targets: ln(r_f / r_vir), ln(T r_vir / (G M_vir)),
 * ln(rho0 / rho_s), normalised the same way.  norm: FP32 [18] on the device, means of the
 * 6 features and 3 targets followed by their scales.
 * FP32 parameters (BP_MLP_NPARAMS floats, this order): W1 [128][6], b1 [128],
 * W2 [128][128], b2, W3 [128][128], b3, W4 [3][128], b4 [3]; W[o][i] multiplies input i
 * into output o.  BF16 weights (BP_MLP_NWEIGHTS): W1, W2, W3, W4 in the same order.
 * cache: FP32 [n][BP_MLP_CACHE_PER_ROW] = Z1, A1, Z2, A2, Z3, A3 per row (pre-activations
 * and activations of the hidden layers), written by forward, read by backward. */
#define BP_MLP_IN 6
#define BP_MLP_HID 128
#define BP_MLP_OUT 3
#define BP_MLP_NPARAMS (128 * 6 + 128 + 2 * (128 * 128 + 128) + 3 * 128 + 3)
#define BP_MLP_NWEIGHTS (128 * 6 + 2 * 128 * 128 + 3 * 128)
#define BP_MLP_CACHE_PER_ROW (6 * 128)
/* FP32 forward of n rows: x [n][6] -> y [n][3]. */
int bp_mlp_forward(bp_ctx* ctx, int64_t n, const float* params, const float* x, float* y,
                   float* cache);
/* Gradient of sum(dy * y) with respect to the parameters (grad overwritten, FP32,
 * parameter layout); deterministic (fixed-order reductions). */
int bp_mlp_backward(bp_ctx* ctx, int64_t n, const float* params, const float* x,
                    const float* cache, const float* dy, float* grad);
/* One Adam step (bias-corrected with `step` >= 1) on params with moment buffers m, v. */
int bp_mlp_adam(bp_ctx* ctx, float* params, const float* grad, float* m, float* v, int64_t step,
                double lr, double beta1, double beta2, double eps);
/* BF16 copy of the weights (round to nearest even). */
int bp_mlp_to_bf16(bp_ctx* ctx, const float* params, uint16_t* weights_bf16);
/* BF16 inference (BF16 weights and activations, FP32 accumulation, FP32 biases from
 * params): x [n][6] -> y [n][3].  The two 128 x 128 layers run on the tensor cores;
 * weights_bf16 must be 16-byte aligned (BP_EINVAL otherwise).  Synchronises: a timed-out
 * tensor-core wait returns BP_ETIMEOUT. */
int bp_mlp_infer_bf16(bp_ctx* ctx, int64_t n, const uint16_t* weights_bf16, const float* params,
                      const float* x, float* y);
/* Normalised features of n halos (params [3][n] per-halo eps_*, f_*, eps_DM or NULL for the
 * Table-1 values).  Synchronises. */
int bp_mlp_features(bp_ctx* ctx, int64_t n, const double* Mvir, const double* c, const double* z,
                    const double* params, const float* norm, float* x);
/* Normalised targets of n solved halos (model from bp_solve_halos*). */
int bp_mlp_targets(bp_ctx* ctx, int64_t n, const double* model, const float* norm, float* t);
/* Mean squared error of y [n][3] against t; dy = 2 (y - t) / (3 n).  loss (host pointer,
 * may be NULL) receives the mean squared error (synchronises when given). */
int bp_mlp_mse(bp_ctx* ctx, int64_t n, const float* y, const float* t, float* dy, double* loss);
/* Surrogate solve: BF16 MLP prediction of (r_f, T) as the seed of the FP32 pre-solve, then
 * at most polish_iter FP64 Newton iterations (bp_solve_halos_ex, BP_SOLVE_FP64_SEEDED, with
 * that guess and gate); polish_iter = 0: no FP64 Newton, the seeded pre-solve's solution is
 * accepted where its FP32 residuals are <= gate (BP_SOLVE_FP32_GATED).  Halos whose normalised features fall outside hull (FP32 [12]: 6
 * minima then 6 maxima) get the plain solve's default start, and halos whose residual after
 * the polish exceeds gate get the full solve; bp_last_fallback_count returns both.  Output
 * as bp_solve_halos. */
int bp_solve_halos_surrogate(bp_ctx* ctx, int64_t n, const double* Mvir, const double* c,
                             const double* z, const double* params, const uint16_t* weights_bf16,
                             const float* mlp_params, const float* norm, const float* hull,
                             int polish_iter, double gate, double* model, int32_t* status,
                             double resid_tol);

/* Section 3.4: per-particle signals.
 *   x,y,z [n] FP32 comoving h^-1 Mpc; vx,vy,vz [n] FP32 km/s (peculiar);
 *   hsml [n] FP32 comoving h^-1 Mpc; halo_id [n] int32 (-1 = field particle);
 *   Mp: particle mass in h^-1 Msun;
 *   halo_pos [3 * n_halos] FP32 comoving h^-1 Mpc, layout [3][n_halos];
 *   model/status: output of bp_solve_halos for those n_halos halos;
 *   out [BP_ASSIGNED_STRIDE * n] FP32 (written, see the record layout above).
 * A halo particle gets P_e, n_e of its halo's profile at its halo-centric distance
 * and the volume V_i = Mp / rho_NFW(r_i); one beyond r_f, or of a halo whose status
 * is not OK, gets kind BP_KIND_NONE.  halo_id >= n_halos: BP_ERANGE is NOT checked
 * on the device; such particles get kind BP_KIND_NONE. */
int bp_assign_particles(bp_ctx* ctx, int64_t n, const float* x, const float* y, const float* z,
                        const float* vx, const float* vy, const float* vz, const float* hsml,
                        const int32_t* halo_id, double Mp, int64_t n_halos,
                        const float* halo_pos, const double* model, const int32_t* status,
                        const bp_map_geom* geom, float* out);

/* bp_assign_particles with a per-particle gravitational potential phi (device FP32 [n],
 * physical (km/s)^2, zero at infinity, the halo's own potential at the particle as an
 * N-body code provides it), or NULL (then identical to bp_assign_particles).  A halo
 * particle then gets theta_i = 1 + (Phi0 - phi_i) / ((n + 1) T) in place of theta(r_i) of the
 * spherical model (Section 2.1's polytropic relation between theta and the potential,
 * evaluated with the particle's own potential: the gas follows the halo's equipotentials,
 * carrying its asphericity); P_e and n_e follow from theta_i as before, while V_i, R_nt and
 * the r_f cut stay at r_i.  The paper's PP uses the spherical model; this variant is an
 * extension. */
int bp_assign_particles_phi(bp_ctx* ctx, int64_t n, const float* x, const float* y,
                            const float* z, const float* vx, const float* vy, const float* vz,
                            const float* phi, const float* hsml, const int32_t* halo_id,
                            double Mp, int64_t n_halos, const float* halo_pos,
                            const double* model, const int32_t* status,
                            const bp_map_geom* geom, float* out);
/* bp_assign_particles_phi in parts, so that the pair list can be built before the halos are
 * solved (the record's geometry does not depend on the solve):
 *   BP_ASSIGN_ALL: the whole record (bp_assign_particles_phi);
 *   BP_ASSIGN_GEOMETRY: pixel coordinates, h in pixels and the kind from the halo id alone
 *     (HALO for 0 <= halo_id < n_halos, FIELD below 0), Y = B = 0; halo_pos, model and status
 *     are not read and may be NULL;
 *   BP_ASSIGN_SIGNALS: Y, B and the kind only, into records the geometry part wrote; the
 *     result is then the whole record of BP_ASSIGN_ALL, bit for bit.
 * A pair list built from geometry records may hold halo particles that the signals part
 * turns to BP_KIND_NONE (outside the truncation radius, or an unsolved halo): they deposit
 * zeros.  Other arguments and errors as bp_assign_particles; unknown part: BP_EINVAL. */
#define BP_ASSIGN_ALL 0
#define BP_ASSIGN_GEOMETRY 1
#define BP_ASSIGN_SIGNALS 2
int bp_assign_particles_part(bp_ctx* ctx, int64_t n, const float* x, const float* y,
                             const float* z, const float* vx, const float* vy, const float* vz,
                             const float* phi, const float* hsml, const int32_t* halo_id,
                             double Mp, int64_t n_halos, const float* halo_pos,
                             const double* model, const int32_t* status,
                             const bp_map_geom* geom, float* out, int part);

/* Section 3.4: deposit assigned particles through the separable pixel-integrated
 * SPH kernel, f_ij = [w((x_i+ - x_p)/h) - w((x_i- - x_p)/h)] [same in y].
 *   assigned [BP_ASSIGNED_STRIDE * n] FP32 (from bp_assign_particles or the caller)
 *   select: BP_SELECT_ALL / HALO / FIELD
 *   ymap, bmap, ylo, blo: [ny][nx] FP32, accumulated (geom->n_maps must be 1).
 * Kernel support outside the map is dropped.  h = 0 deposits to the nearest grid
 * point.  Deterministic: particles are summed per tile in index order with
 * compensated FP32 sums.  Synchronises once to size the pair list. */
int bp_paste_particles(bp_ctx* ctx, int64_t n, const float* assigned, const bp_map_geom* geom,
                       int select, float* ymap, float* bmap, float* ylo, float* blo);

/* bp_paste_particles in two calls.  bp_pp_prepare builds the sorted (tile, particle) list
 * and the work units from the records' geometry (pixel coordinates, h, kind), in the
 * context's scratch (synchronises, as bp_paste_particles); bp_pp_deposit then deposits the
 * records' Y and B through it, which may have been written in between (by
 * bp_assign_particles_part with BP_ASSIGN_SIGNALS).  The solve and the assign calls may run
 * on the context in between; a call that reuses the scratch holding the list (a paste, a
 * sort) is detected.  bp_pp_deposit needs the same records pointer, n, geometry and select
 * as the last bp_pp_prepare, and the prepared list intact: otherwise BP_EINVAL.
 * prepare + deposit == bp_paste_particles. */
int bp_pp_prepare(bp_ctx* ctx, int64_t n, const float* assigned, const bp_map_geom* geom,
                  int select);
int bp_pp_deposit(bp_ctx* ctx, int64_t n, const float* assigned, const bp_map_geom* geom,
                  int select, float* ymap, float* bmap, float* ylo, float* blo);

/* bp_paste_particles for callers that cannot allocate device memory during a call:
 * applications that give their whole device memory to their own pool allocator at
 * start-up, and latency-critical loops in which cudaMalloc/cudaFree would
 * synchronise the device.  (The paper has no counterpart: this is a service of the
 * library.)  Same arguments, results and host synchronisation as bp_paste_particles
 * (the call waits once on the context's stream, to read back the pair count), but all
 * scratch lives in one fixed device array inside the library (about 24 MiB) and each
 * tile is deposited by a single CTA.  It calls no cudaMalloc, cudaFree or other
 * allocating routine.  CUDA loads a library's device code and arrays lazily, and that
 * load takes device memory, so bp_create does it: creating a context brings the array
 * into being on the context's device (held there until the process exits) and loads
 * every kernel this call launches.  Create the context before reserving the device
 * memory, and make the call on the context's device.  Limits: n <=
 * BP_NOALLOC_MAX_PARTICLES particles, at most BP_NOALLOC_MAX_PAIRS (tile, particle)
 * pairs and BP_NOALLOC_MAX_TILES tiles of the context's deposit tile size; beyond them
 * it returns BP_ERANGE with a message and leaves the maps as they were (the pair count
 * is known only after the pair-count pass, so that check comes after the host
 * synchronisation, before anything is written to the maps).  Every call reuses the same
 * array, which keeps the previous call's contents: calls whose work overlaps on the GPU
 * (other streams, other host threads, other contexts of the device) race and must not be
 * issued concurrently. */
#define BP_NOALLOC_MAX_PARTICLES (1 << 19)
#define BP_NOALLOC_MAX_PAIRS (1 << 20)
#define BP_NOALLOC_MAX_TILES 4096
int bp_paste_particles_noalloc(bp_ctx* ctx, int64_t n, const float* assigned,
                               const bp_map_geom* geom, int select, float* ymap, float* bmap,
                               float* ylo, float* blo);

/* Section 3.4 (the SPH kernel Eq. SPH_kernel and N_ngb): smoothing lengths from the
 * particle positions.  h_i solves N_eff(h) = (4 pi / 3) h^3 sum_j W(|r_i - r_j|, h) = n_ngb
 * with the cubic kernel W = 8 / (pi h^3) w(r / h), the sum over all n particles (i
 * included).  x, y, z: device FP32 positions [n] in any length unit (comoving h^-1 Mpc for
 * bp_assign_particles); h_guess: optional device FP32 [n] starting radii (a previous h, or
 * null: from the grid density); h_out: device FP32 [n], same unit as the positions.
 * Uses the context's scratch and stream; synchronises.  Deterministic.  Errors:
 * BP_EINVAL (null pointer, n_ngb outside (32/3, 1024], non-finite position), BP_ERANGE
 * (n (32/3) <= n_ngb: no particle can reach n_ngb; n >= 2^32), BP_ENOCONV (a particle did
 * not converge in 48 radius updates: its h is NaN). */
int bp_smoothing_lengths(bp_ctx* ctx, int64_t n, const float* x, const float* y, const float* z,
                         double n_ngb, const float* h_guess, float* h_out);

/* The tile pair list of the deposit (for tests): keys (tile index ty*ntx+tx) and
 * particle indices ordered by key then index.  capacity: entries the caller
 * allocated; n_pairs (host pointer) receives the count.  BP_ERANGE if capacity
 * is too small (nothing written).  Synchronises. */
int bp_pp_pairs(bp_ctx* ctx, int64_t n, const float* assigned, const bp_map_geom* geom,
                int select, int tile, uint32_t* keys, uint32_t* vals, int64_t capacity,
                int64_t* n_pairs);

/* Section 3.3: halo-based pasting.  For every pixel centre at projected radius
 * r_perp < r_ap of halo h, add sigma_T/(m_e c^2) 2 int P_e dx to y and
 * sigma_T (v_h/c) e^{-tau_h} 2 int n_e dx to b, the line of sight bounded by r_f.
 *   th_x, th_y [n] FP64 rad; v_los [n] FP32 km/s; map_id [n] int32 or NULL (all 0);
 *   model/status from bp_solve_halos; ap_r500 > 0 sets r_ap = min(r_f, ap_r500 r500),
 *   0 sets r_ap = r_f; maps [n_maps][ny][nx] FP32 accumulated.
 * Synchronises once to size the (halo, tile) list. */
int bp_paste_halos(bp_ctx* ctx, int64_t n, const double* th_x, const double* th_y,
                   const float* v_los, const int32_t* map_id, const double* model,
                   const int32_t* status, const bp_map_geom* geom, double ap_r500, float* ymap,
                   float* bmap, float* ylo, float* blo);

/* The (map, tile, halo) work list of bp_paste_halos (Section 3.3: the pixel centres a halo
 * can reach lie in the FP64 bounding box floor(c - r_ap) .. floor(c + r_ap) of its aperture
 * disc, c the centre in pixel-centre index units, r_ap in pixels; a halo adds to every tile
 * that box touches).  Arguments as bp_paste_halos (v_los is not needed); tile: 32 or 64.
 * keys: (map_id * nty + ty) * ntx + tx, vals: halo indices, ordered by key then index, into
 * caller device arrays of `capacity` entries; n_pairs (host pointer) receives the count.
 * Halos whose status is not OK, or whose map_id is outside [0, n_maps), have no pairs.
 * BP_ERANGE if capacity is too small (nothing written).  For tests; synchronises. */
int bp_hp_pairs(bp_ctx* ctx, int64_t n, const double* th_x, const double* th_y,
                const int32_t* map_id, const double* model, const int32_t* status,
                const bp_map_geom* geom, double ap_r500, int tile, uint32_t* keys, uint32_t* vals,
                int64_t capacity, int64_t* n_pairs);

/* All-sky maps (Section 5.2) by the HP of Section 3.3 (Eqs. y^HP, b^HP) on the HEALPix
 * sphere of Gorski et al. (2005), RING ordering: npix = 12 nside^2 equal-area pixels, pixel p
 * of ring i (1 .. 4 nside - 1, north to south) at colatitude acos(z_i).  Each halo adds its
 * projected profiles at r_perp = D_A psi to every pixel centre within its aperture, psi the
 * great-circle angle to the halo (r_ap = r_f, or min(r_f, ap_r500 r500) when ap_r500 > 0).
 * theta, phi: device FP64 [n] colatitude in [0, pi] and longitude [rad] (any value, taken
 * modulo 2 pi) of the halo centres; v_los: FP32 [n] km/s (positive receding); model and
 * status: bp_solve_halos output for the same n halos (halos whose status is not OK, or
 * whose theta is outside [0, pi], add nothing).  ymap, bmap, ylo, blo: device FP32 [npix]
 * in RING order, accumulated (hi + lo, as bp_paste_halos); finalise with bp_finalize_map
 * and a geometry of nx = 12 nside, ny = nside.  nside: 1 .. 16384.  Halos are processed in
 * chunks of 2^22 (bounded table memory); each pixel adds its halos in catalogue order
 * within a chunk: deterministic.  Synchronises once per chunk (pair-list size).  Errors:
 * BP_EINVAL (null pointer, nside, ap_r500 < 0), BP_ERANGE (n >= 2^32, more than 2^32 pairs
 * in a chunk). */
int bp_paste_halos_healpix(bp_ctx* ctx, int64_t n, const double* theta, const double* phi,
                           const float* v_los, const double* model, const int32_t* status,
                           int nside, double ap_r500, float* ymap, float* bmap, float* ylo,
                           float* blo);

/* Section 5.3: the angular power spectrum of a flat-sky map (the FFT of the map, binned in
 * multipole).  map (+ lo when not NULL): device FP32 [ny][nx] of square pixels of side dtheta
 * [rad]; nx, ny powers of two in [2, 8192].  With a(l) = dtheta^2 sum_pixels f e^{-i l.theta}
 * and l = 2 pi (kx / (nx dtheta), ky / (ny dtheta)) for the integer frequencies (kx in
 * [-nx/2, nx/2)), cl[b] is the mean of |a(l)|^2 / (nx ny dtheta^2) over the modes with
 * edges[b] <= |l| < edges[b + 1] (0 for an empty bin), nmodes[b] their count.  edges: HOST
 * FP64 [nb + 1], increasing from >= 0, nb in [1, 256] (the paper uses 30 logarithmic bins
 * over 1e2 < l < 1e5); cl: device FP64 [nb]; nmodes: device int64 [nb] or NULL.  FP64
 * throughout; deterministic.  Synchronises once (uploads twiddles and edges).  Errors:
 * BP_EINVAL (sizes, dtheta, edges, null pointer). */
int bp_power_spectrum(bp_ctx* ctx, const float* map, const float* lo, int nx, int ny,
                      double dtheta, int nb, const double* edges, double* cl, int64_t* nmodes);

/* A prepared halo paste for repeated pastes of one catalogue (many maps of uneven halo
 * extents in one persistent launch).  bp_hp_plan_create builds the (map, tile, halo)
 * work list from the catalogue's apertures (as bp_paste_halos does; synchronises) and
 * allocates the plan's own device buffers.  tile: 32 or 64 pixels; unit: halos per work
 * unit (0 = automatic); ctas_per_sm: persistent CTAs per SM (0 = as many as fit).
 * bp_hp_plan_execute then recomputes the halo tables from model and v_los and pastes
 * into the maps with launch shapes fixed at creation: it neither synchronises nor
 * allocates, so a caller can capture it in a CUDA graph.  The work list stays valid
 * while the apertures (r_f, r500, D_A of model and the sky positions) are those the
 * plan was built with.  Paste semantics are those of bp_paste_halos. */
typedef struct bp_hp_plan bp_hp_plan;
int bp_hp_plan_create(bp_ctx* ctx, int64_t n, const double* th_x, const double* th_y,
                      const int32_t* map_id, const double* model, const int32_t* status,
                      const bp_map_geom* geom, double ap_r500, int tile, int unit,
                      int ctas_per_sm, bp_hp_plan** plan);
int bp_hp_plan_execute(bp_ctx* ctx, bp_hp_plan* plan, const double* th_x, const double* th_y,
                       const float* v_los, const int32_t* map_id, const double* model,
                       const int32_t* status, float* ymap, float* bmap, float* ylo, float* blo);
/* (tile, halo) pairs of the plan's work list. */
int64_t bp_hp_plan_pairs(const bp_hp_plan* plan);
int bp_hp_plan_destroy(bp_hp_plan* plan);

/* Section 3.2: fold lo into hi (hi <- fl(hi + lo), lo <- 0) for all n_maps maps;
 * out_kind BP_OUT_DT then converts to Delta T/T_CMB: g_nu(x) y (x = h nu/k T_CMB,
 * nu_ghz > 0) and -b.  ymap or bmap may be NULL (with its lo plane). */
int bp_finalize_map(bp_ctx* ctx, const bp_map_geom* geom, float* ymap, float* bmap, float* ylo,
                    float* blo, int out_kind, double nu_ghz);

#ifdef __cplusplus
}
#endif
#endif /* BP_H */

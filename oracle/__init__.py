"""FP64 CPU oracle for the baryon pasting method (Osato & Nagai 2022).

TEST INFRASTRUCTURE ONLY: the tests, ``__graft_entry__.smoke()`` and the
``cpu_baseline`` / ``--impl reference`` legs of ``bench.py`` are the only
callers.  The product path (``paper_2201_02632_gb300``) never imports this
package, and this package never imports the product path.

The arithmetic lives in ``bp_oracle.c`` (plain C, FP64, compiled with
``-ffp-contract=off``); this module builds it with gcc and marshals numpy
arrays through ctypes.  Parity pins for every function are in
``tests/test_oracle_*.py``.  Functions with no pin are listed in the
module-level ``UNPINNED`` tuple (empty: every function is pinned).
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "bp_oracle.c")
_LIB = os.path.join(_HERE, "_build", "liboracle.so")
_lock = threading.Lock()
_lib = None

UNPINNED: tuple = ()

# Field order of the oracle's per-halo model record (mirrors the enum in bp_oracle.c).
FIELDS = (
    "M", "c", "z", "rho_cr", "Delta_vir", "r_vir", "r_s", "rho_s", "m_c", "Phi0",
    "r500", "M500", "M_star", "r_star", "E_gi", "E_dm", "P_s", "T", "rho0", "P0",
    "r_f", "A_nt", "D_A", "tau", "res_m", "res_e", "status",
)
F = {name: i for i, name in enumerate(FIELDS)}


class Cosmo(C.Structure):
    _fields_ = [("Om", C.c_double), ("Ob", C.c_double), ("h", C.c_double),
                ("Tcmb", C.c_double), ("XH", C.c_double)]


class ICM(C.Structure):
    _fields_ = [("Gamma", C.c_double), ("eps_dm", C.c_double), ("eps_star", C.c_double),
                ("f_star", C.c_double), ("S_star", C.c_double), ("alpha_nt", C.c_double),
                ("beta_nt", C.c_double), ("n_nt", C.c_double), ("energy_sign", C.c_int),
                ("field_fb", C.c_int)]


class Geom(C.Structure):
    _fields_ = [("nx", C.c_int), ("ny", C.c_int), ("n_maps", C.c_int),
                ("theta0_x", C.c_double), ("theta0_y", C.c_double), ("dtheta", C.c_double)]


def cosmo_default() -> Cosmo:
    """WMAP9 flat LCDM of Section 1; T_CMB and X of Section 3.2."""
    return Cosmo(Om=0.279, Ob=0.046, h=0.7, Tcmb=2.726, XH=0.76)


def icm_default(**kw) -> ICM:
    """Table 1 of the paper."""
    p = dict(Gamma=1.2, eps_dm=0.0, eps_star=3.97e-6, f_star=0.026, S_star=0.12,
             alpha_nt=0.18, beta_nt=0.5, n_nt=0.8, energy_sign=0, field_fb=0)
    p.update(kw)
    return ICM(**p)


def geom(nx, ny, theta0_x, theta0_y, dtheta, n_maps=1) -> Geom:
    return Geom(nx=int(nx), ny=int(ny), n_maps=int(n_maps), theta0_x=float(theta0_x),
                theta0_y=float(theta0_y), dtheta=float(dtheta))


def build(force: bool = False) -> str:
    """Compile bp_oracle.c into _build/liboracle.so (gcc, FP64, no contraction)."""
    os.makedirs(os.path.dirname(_LIB), exist_ok=True)
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + f".tmp{os.getpid()}"
        cmd = ["gcc", "-O2", "-fPIC", "-shared", "-fopenmp", "-ffp-contract=off",
               "-fno-fast-math", "-o", tmp, _SRC, "-lm"]
        subprocess.run(cmd, check=True)
        os.replace(tmp, _LIB)
    return _LIB


def lib():
    global _lib
    with _lock:
        if _lib is None:
            path = build()
            L = C.CDLL(path)
            d, i64, i32 = C.c_double, C.c_int64, C.c_int
            P = C.c_void_p
            pc, pi, pg = C.POINTER(Cosmo), C.POINTER(ICM), C.POINTER(Geom)
            sig = {
                "orc_model_nfields": (i32, []),
                "orc_rho_cr": (d, [pc, d]),
                "orc_delta_vir": (d, [pc, d]),
                "orc_chi": (d, [pc, d]),
                "orc_z_of_chi": (d, [pc, d]),
                "orc_DA": (d, [pc, d]),
                "orc_tau": (d, [pc, d]),
                "orc_m_of": (d, [d]),
                "orc_sigma2": (d, [pc, d, d, d, d]),
                "orc_halo_solve": (None, [pc, pi, d, d, d, i32, P]),
                "orc_solve_halos": (None, [pc, pi, i64, P, P, P, i32, P, i32]),
                "orc_profile": (None, [pc, pi, P, i64, P, P, P, P]),
                "orc_nfw_eval": (None, [pc, d, d, d, i64, P, P, P, P]),
                "orc_const_CP": (d, []),
                "orc_const_CN": (d, [pc]),
                "orc_los_integral": (d, [pc, pi, P, d, i32, d]),
                "orc_hp_map": (None, [pc, pi, i64, P, P, P, P, P, pg, d, d, P, P, i32]),
                "orc_w_sph": (d, [d]),
                "orc_pp_assign": (None, [pc, pi, i64, P, P, P, P, P, P, P, P, d, i64, P, P, pg,
                                         P, P, P, P, P, P, i32]),
                "orc_pp_assign_phi": (None, [pc, pi, i64, P, P, P, P, P, P, P, P, P, d, i64, P, P,
                                             pg, P, P, P, P, P, P, i32]),
                "orc_pp_deposit": (None, [i64, P, P, P, P, P, P, pg, i32, P, P, i32]),
                "orc_pp_deposit_pixels": (None, [i64, P, P, P, P, P, P, pg, i32, i64, P, P, P,
                                                 P, i32]),
                "orc_pp_pairs": (i64, [i64, P, P, P, P, P, P, i32, i32, i32, i32, i32, P, P]),
                "orc_g_nu": (d, [d, d]),
                "orc_hp_pairs": (i64, [i64, P, P, P, P, pg, d, i32, i32, P, P]),
                "orc_energy_residual": (d, [pc, pi, d, d, d, d]),
                "orc_pp_select": (i64, [pc, i64, P, P, P, P, pg, i64, P, P, P, i32]),
                "orc_hp_pixels": (None, [pc, pi, i64, P, P, P, P, P, pg, d, d, i64, P, P, P, P, P,
                                         i32]),
                "orc_w3": (d, [d]),
                "orc_hpx_centres": (None, [i64, i64, P, P, P]),
                "orc_sky_angle": (d, [d, d, d, d]),
                "orc_hp_sky": (None, [pc, pi, i64, P, P, P, P, d, d, i64, P, P, P, P, i32]),
                "orc_smoothing_lengths": (None, [i64, P, P, P, d, P, i32]),
                "orc_smoothing_lengths_at": (None, [i64, P, P, P, d, i64, P, P, i32]),
            }
            for name, (res, args) in sig.items():
                f = getattr(L, name)
                f.restype = res
                f.argtypes = args
            assert L.orc_model_nfields() == len(FIELDS)
            _lib = L
    return _lib


def _p(a):
    return None if a is None else a.ctypes.data_as(C.c_void_p)


def _f64(a):
    return np.ascontiguousarray(a, dtype=np.float64)


def _f32(a):
    return np.ascontiguousarray(a, dtype=np.float32)


def _i32(a):
    return np.ascontiguousarray(a, dtype=np.int32)


# ---------------------------------------------------------------- cosmology
def rho_cr(z, cp=None):
    return lib().orc_rho_cr(C.byref(cp or cosmo_default()), float(z))


def delta_vir(z, cp=None):
    return lib().orc_delta_vir(C.byref(cp or cosmo_default()), float(z))


def chi(z, cp=None):
    return lib().orc_chi(C.byref(cp or cosmo_default()), float(z))


def z_of_chi(x, cp=None):
    return lib().orc_z_of_chi(C.byref(cp or cosmo_default()), float(x))


def tau(z, cp=None):
    return lib().orc_tau(C.byref(cp or cosmo_default()), float(z))


def m_of(x):
    return lib().orc_m_of(float(x))


def sigma2(M_hinv, c, z, r, cp=None):
    return lib().orc_sigma2(C.byref(cp or cosmo_default()), float(M_hinv), float(c), float(z),
                            float(r))


def nfw_eval(M_hinv, c, z, r, cp=None):
    r = _f64(r)
    rho, Menc, phi = (np.empty_like(r) for _ in range(3))
    lib().orc_nfw_eval(C.byref(cp or cosmo_default()), float(M_hinv), float(c), float(z),
                       r.size, _p(r), _p(rho), _p(Menc), _p(phi))
    return rho, Menc, phi


def const_CP():
    return lib().orc_const_CP()


def const_CN(cp=None):
    return lib().orc_const_CN(C.byref(cp or cosmo_default()))


# ---------------------------------------------------------------- halo solve
def solve_halos(M_hinv, c, z, cp=None, ip=None, n_scan=48, nthreads=0):
    """Per-halo ICM solve (Section 2).  Returns an [n, len(FIELDS)] FP64 array."""
    M, c, z = _f64(M_hinv), _f64(c), _f64(z)
    out = np.zeros((M.size, len(FIELDS)), np.float64)
    lib().orc_solve_halos(C.byref(cp or cosmo_default()), C.byref(ip or icm_default()), M.size,
                          _p(M), _p(c), _p(z), int(n_scan), _p(out), int(nthreads))
    return out


def energy_residual(M_hinv, c, z, rf_over_rvir, cp=None, ip=None):
    """Energy condition residual at r_f = rf_over_rvir * r_vir, with T set by the gas-mass
    condition at that r_f."""
    return lib().orc_energy_residual(C.byref(cp or cosmo_default()), C.byref(ip or icm_default()),
                                     float(M_hinv), float(c), float(z), float(rf_over_rvir))


def profile(model_row, r, cp=None, ip=None):
    """(P_e, rho_g, P_tot) of one solved halo at physical radii r."""
    m, r = _f64(model_row), _f64(r)
    Pe, rg, Pt = (np.empty_like(r) for _ in range(3))
    lib().orc_profile(C.byref(cp or cosmo_default()), C.byref(ip or icm_default()), _p(m),
                      r.size, _p(r), _p(Pe), _p(rg), _p(Pt))
    return Pe, rg, Pt


def los_integral(model_row, rperp, which=0, rtol=1e-12, cp=None, ip=None):
    m = _f64(model_row)
    return lib().orc_los_integral(C.byref(cp or cosmo_default()), C.byref(ip or icm_default()),
                                  _p(m), float(rperp), int(which), float(rtol))


# ---------------------------------------------------------------- HP
def hp_map(thx, thy, vlos, models, g: Geom, ap_r500=0.0, map_id=None, rtol=1e-10, cp=None,
           ip=None, nthreads=0):
    thx, thy, vlos, models = _f64(thx), _f64(thy), _f64(vlos), _f64(models)
    mid = None if map_id is None else _i32(map_id)
    shape = (g.n_maps, g.ny, g.nx)
    ym, bm = np.zeros(shape), np.zeros(shape)
    lib().orc_hp_map(C.byref(cp or cosmo_default()), C.byref(ip or icm_default()), thx.size,
                     _p(thx), _p(thy), _p(vlos), _p(mid), _p(models), C.byref(g),
                     float(ap_r500), float(rtol), _p(ym), _p(bm), int(nthreads))
    return ym, bm


def hpx_centres(nside, pix=None):
    """HEALPix RING pixel centres (colatitude, longitude) of pixels `pix` (default all)."""
    if pix is None:
        pix = np.arange(12 * nside * nside, dtype=np.int64)
    pix = np.ascontiguousarray(pix, dtype=np.int64)
    th, ph = np.empty(pix.size), np.empty(pix.size)
    lib().orc_hpx_centres(int(nside), pix.size, _p(pix), _p(th), _p(ph))
    return th, ph


def sky_angle(t1, p1, t2, p2):
    return lib().orc_sky_angle(float(t1), float(p1), float(t2), float(p2))


def hp_sky(h_theta, h_phi, vlos, models, p_theta, p_phi, ap_r500=0.0, rtol=1e-9, cp=None,
           ip=None, nthreads=0):
    """All-sky HP values at pixel directions (p_theta, p_phi): halos at (h_theta, h_phi)."""
    h_theta, h_phi, vlos, models = _f64(h_theta), _f64(h_phi), _f64(vlos), _f64(models)
    p_theta, p_phi = _f64(p_theta), _f64(p_phi)
    yv, bv = np.zeros(p_theta.size), np.zeros(p_theta.size)
    lib().orc_hp_sky(C.byref(cp or cosmo_default()), C.byref(ip or icm_default()), h_theta.size,
                     _p(h_theta), _p(h_phi), _p(vlos), _p(models), float(ap_r500), float(rtol),
                     p_theta.size, _p(p_theta), _p(p_phi), _p(yv), _p(bv), int(nthreads))
    return yv, bv


def g_nu(nu_ghz, cp=None):
    """Section 3.2: the tSZ frequency factor g(x), x = h nu / (k_B T_CMB)."""
    return lib().orc_g_nu(float(nu_ghz), float((cp or cosmo_default()).Tcmb))


def delta_t(y, b, nu_ghz, cp=None):
    """Section 3.2: Delta T / T_CMB maps from y and b maps (FP64): g(x) y (tSZ) and -b
    (kSZ)."""
    g = g_nu(nu_ghz, cp)
    return g * np.asarray(y, np.float64), -np.asarray(b, np.float64)


def hp_pairs(thx, thy, models, g: Geom, ap_r500, tw, th, map_id=None):
    thx, thy, models = _f64(thx), _f64(thy), _f64(models)
    mid = None if map_id is None else _i32(map_id)
    L = lib()
    n = L.orc_hp_pairs(thx.size, _p(thx), _p(thy), _p(mid), _p(models), C.byref(g),
                       float(ap_r500), int(tw), int(th), None, None)
    keys = np.empty(n, np.uint32)
    vals = np.empty(n, np.uint32)
    L.orc_hp_pairs(thx.size, _p(thx), _p(thy), _p(mid), _p(models), C.byref(g), float(ap_r500),
                   int(tw), int(th), _p(keys), _p(vals))
    return keys, vals


# ---------------------------------------------------------------- PP
def w_sph(x):
    return lib().orc_w_sph(float(x))


def w3(x):
    """3-D cubic spline of Eq. SPH_kernel without its 8 / (pi h^3) factor."""
    return lib().orc_w3(float(x))


def smoothing_lengths(x, y, z, n_ngb=64.0, nthreads=0):
    """h_i with (32/3) sum_j w(|r_i - r_j| / h_i) = n_ngb (all j, i included); FP32
    positions, FP64 result in the same length unit.  O(n^2 log n): small inputs only."""
    x, y, z = _f32(x), _f32(y), _f32(z)
    n = x.size
    h = np.empty(n, np.float64)
    lib().orc_smoothing_lengths(n, _p(x), _p(y), _p(z), float(n_ngb), _p(h), nthreads)
    return h


def smoothing_lengths_at(x, y, z, idx, n_ngb=64.0, nthreads=0):
    """smoothing_lengths of the particles idx only (the sums still run over all of them):
    O(len(idx) n log n), for sampling large inputs."""
    x, y, z = _f32(x), _f32(y), _f32(z)
    idx = np.ascontiguousarray(idx, dtype=np.int64)
    h = np.empty(idx.size, np.float64)
    lib().orc_smoothing_lengths_at(x.size, _p(x), _p(y), _p(z), float(n_ngb), idx.size,
                                   _p(idx), _p(h), nthreads)
    return h


def pp_assign(parts: dict, Mp_hinv, halo_pos, models, g: Geom, cp=None, ip=None, nthreads=0,
              phi=None):
    """Per-particle signals.  parts: x,y,z,vx,vy,vz,hsml (float32), hid (int32).
    halo_pos: float32 [3, nh].  phi: optional float32 per-particle potential [(km/s)^2] (the
    potential-based variant).  Returns dict px,py,hp,Y,B (FP64) and kind (int32)."""
    x, y, z = _f32(parts["x"]), _f32(parts["y"]), _f32(parts["z"])
    vx, vy, vz = _f32(parts["vx"]), _f32(parts["vy"]), _f32(parts["vz"])
    hs, hid = _f32(parts["hsml"]), _i32(parts["hid"])
    hpos = _f32(halo_pos)
    models = _f64(models)
    n = x.size
    out = {k: np.empty(n, np.float64) for k in ("px", "py", "hp", "Y", "B")}
    kind = np.empty(n, np.int32)
    nh = hpos.shape[1] if hpos.ndim == 2 else 0
    ph = None if phi is None else _f32(phi)
    lib().orc_pp_assign_phi(C.byref(cp or cosmo_default()), C.byref(ip or icm_default()), n,
                            _p(x), _p(y), _p(z), _p(vx), _p(vy), _p(vz), _p(ph), _p(hs), _p(hid),
                            float(Mp_hinv), nh, _p(hpos), _p(models), C.byref(g), _p(out["px"]),
                            _p(out["py"]), _p(out["hp"]), _p(out["Y"]), _p(out["B"]), _p(kind),
                            int(nthreads))
    out["kind"] = kind
    return out


def pp_deposit(a: dict, g: Geom, select=0, nthreads=0):
    px, py, hp, Y, B = (_f64(a[k]) for k in ("px", "py", "hp", "Y", "B"))
    kind = _i32(a["kind"])
    ym = np.zeros((g.ny, g.nx))
    bm = np.zeros((g.ny, g.nx))
    lib().orc_pp_deposit(px.size, _p(px), _p(py), _p(hp), _p(Y), _p(B), _p(kind), C.byref(g),
                         int(select), _p(ym), _p(bm), int(nthreads))
    return ym, bm


def pp_deposit_pixels(a: dict, g: Geom, pix_i, pix_j, select=0, nthreads=0):
    px, py, hp, Y, B = (_f64(a[k]) for k in ("px", "py", "hp", "Y", "B"))
    kind = _i32(a["kind"])
    pi_, pj_ = _i32(pix_i), _i32(pix_j)
    yv = np.zeros(pi_.size)
    bv = np.zeros(pi_.size)
    lib().orc_pp_deposit_pixels(px.size, _p(px), _p(py), _p(hp), _p(Y), _p(B), _p(kind),
                                C.byref(g), int(select), pi_.size, _p(pi_), _p(pj_), _p(yv),
                                _p(bv), int(nthreads))
    return yv, bv


def pp_pairs(ix, fx, iy, fy, hp, kind, nx, ny, tw, th, select=0):
    """(key, particle) pairs of the tile membership, decided in FP32 from the split
    position px = ix + fx, ordered by key then particle index."""
    ix, iy, kind = _i32(ix), _i32(iy), _i32(kind)
    fx, fy, hp = _f32(fx), _f32(fy), _f32(hp)
    L = lib()
    args = (ix.size, _p(ix), _p(fx), _p(iy), _p(fy), _p(hp), _p(kind), nx, ny, tw, th, select)
    n = L.orc_pp_pairs(*args, None, None)
    keys = np.empty(n, np.uint32)
    vals = np.empty(n, np.uint32)
    L.orc_pp_pairs(*args, _p(keys), _p(vals))
    return keys, vals


def pp_select(parts: dict, g: Geom, pix_i, pix_j, cp=None, nthreads=0):
    """Indices of the particles whose kernel support covers one of the pixels."""
    x, y, z, hs = (_f32(parts[k]) for k in ("x", "y", "z", "hsml"))
    pi_, pj_ = _i32(pix_i), _i32(pix_j)
    out = np.empty(x.size, np.int64)
    m = lib().orc_pp_select(C.byref(cp or cosmo_default()), x.size, _p(x), _p(y), _p(z), _p(hs),
                            C.byref(g), pi_.size, _p(pi_), _p(pj_), _p(out), int(nthreads))
    return out[:m]


def pp_pixels(parts: dict, Mp_hinv, halo_pos, models, g: Geom, pix_i, pix_j, select=0,
              nthreads=0):
    """Sampled pixels of the PP maps (assign + deposit of the particles that reach them)."""
    idx = pp_select(parts, g, pix_i, pix_j, nthreads=nthreads)
    sub = {k: np.ascontiguousarray(v[idx]) for k, v in parts.items()}
    a = pp_assign(sub, Mp_hinv, halo_pos, models, g, nthreads=nthreads)
    return pp_deposit_pixels(a, g, pix_i, pix_j, select=select, nthreads=nthreads), idx.size


def hp_pixels(thx, thy, vlos, models, g: Geom, pix_i, pix_j, pix_m=None, ap_r500=0.0,
              map_id=None, rtol=1e-9, cp=None, ip=None, nthreads=0):
    """HP values at listed pixels (map pix_m, column pix_i, row pix_j)."""
    thx, thy, vlos, models = _f64(thx), _f64(thy), _f64(vlos), _f64(models)
    mid = None if map_id is None else _i32(map_id)
    pm = None if pix_m is None else _i32(pix_m)
    pi_, pj_ = _i32(pix_i), _i32(pix_j)
    yv, bv = np.zeros(pi_.size), np.zeros(pi_.size)
    lib().orc_hp_pixels(C.byref(cp or cosmo_default()), C.byref(ip or icm_default()), thx.size,
                        _p(thx), _p(thy), _p(vlos), _p(mid), _p(models), C.byref(g),
                        float(ap_r500), float(rtol), pi_.size, _p(pm), _p(pi_), _p(pj_), _p(yv),
                        _p(bv), int(nthreads))
    return yv, bv


def solve_referenced(M, c, z, hid_subset, cp=None, ip=None, nthreads=0):
    """Model rows for every halo, solved only for the halos listed in hid_subset (the
    others get status 1 and are never referenced by the caller)."""
    nh = np.asarray(M).size
    models = np.zeros((nh, len(FIELDS)))
    models[:, F["status"]] = 1
    h = np.unique(np.asarray(hid_subset))
    h = h[h >= 0]
    if h.size:
        models[h] = solve_halos(np.asarray(M)[h], np.asarray(c)[h], np.asarray(z)[h], cp, ip,
                                nthreads=nthreads)
    return models


# ---------------------------------------------------------------- Section 5.3
def power_spectrum(m, dtheta, edges):
    """Flat-sky angular power spectrum of a map [ny, nx] (FP64, numpy FFT): with
    a(l) = dtheta^2 sum f e^{-i l.theta}, l = 2 pi (kx / (nx dtheta), ky / (ny dtheta)),
    returns the mean of |a|^2 / (nx ny dtheta^2) over the modes with edges[b] <= |l| <
    edges[b + 1] and the mode counts.  Each mode's |l|^2 is formed as
    (4 pi pi) ((kx / Lx)^2 + (ky / Ly)^2) with 1 / L precomputed, compared with edges^2."""
    f = np.asarray(m, np.float64)
    ny, nx = f.shape
    F = np.fft.fft2(f)
    power = (dtheta * dtheta / (nx * ny)) * (F.real * F.real + F.imag * F.imag)
    fx = np.fft.fftfreq(nx, 1.0 / nx)  # integer frequencies, [-n/2, n/2)
    fy = np.fft.fftfreq(ny, 1.0 / ny)
    ux = fx * (1.0 / (nx * dtheta))
    uy = fy * (1.0 / (ny * dtheta))
    l2 = (4.0 * np.pi * np.pi) * (ux[None, :] * ux[None, :] + uy[:, None] * uy[:, None])
    e = np.asarray(edges, np.float64)
    e2 = e * e
    nb = e.size - 1
    b = np.searchsorted(e2, l2, side="right") - 1
    ok = (l2 >= e2[0]) & (l2 < e2[-1])
    cl = np.zeros(nb)
    cnt = np.zeros(nb, np.int64)
    for k in range(nb):
        sel = ok & (b == k)
        cnt[k] = sel.sum()
        if cnt[k]:
            cl[k] = power[sel].sum() / cnt[k]
    return cl, cnt

"""Seeded synthetic inputs shaped like the paper's workloads.

This module draws INPUTS only: halo catalogues (mass, concentration, redshift,
sky position, line-of-sight velocity) and light-cone particles (comoving
positions, velocities, smoothing lengths, halo membership).  It contains none
of the pasting method's arithmetic (no ICM model, no projection, no kernel
weights); both the CUDA path and the CPU oracle consume what it produces.

The paper's inputs are N-body light-cones and Rockstar/SubFind catalogues
(Section 3.1), which are not available; these generators stand in for them:

* halo catalogue (HP, 1x1 deg^2): log-uniform mass in [1e13, 1e15] h^-1 Msun,
  c = 5 (M/1e14)^-0.1 with 0.1 dex lognormal scatter, z ~ U(0.05, 1),
  positions uniform in the patch, v_los ~ N(0, 300 km/s).
* light-cone (PP): particles in a square cone around +z.  A fraction comes
  from truncated-NFW halos with triaxial axis ratios U(0.5, 1) and random
  orientation; the rest are field particles uniform in comoving volume.
  Velocities N(0, 300 km/s) per component.  Smoothing lengths follow the
  N_ngb = 64 neighbour rule applied to the local density of the generating
  distribution (NFW density for halo particles, mean field density for field
  particles).  Particle order is a seeded random permutation.

Geometry of the generator (its own, used only to place objects): the
comoving-distance/redshift relation is a trapezoid table of 1/E(z) for the
same flat LCDM; halo particle clouds extend to a comoving radius enclosing
200 times the mean matter density.  Nothing computed here is compared
against anything.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np

SEED_BASE = 20220108
DEG = math.pi / 180.0
OMEGA_M = 0.279
C_KMS = 299792.458
RHO_CRIT0_H2 = 2.77536627e11  # h^2 Msun / Mpc^3 (critical density today)


@dataclass
class MapGeom:
    nx: int
    ny: int
    theta0_x: float  # rad, lower-left pixel edge
    theta0_y: float
    dtheta: float    # rad per pixel
    n_maps: int = 1


@dataclass
class HaloCatalog:
    M: np.ndarray      # f64 h^-1 Msun
    c: np.ndarray      # f64
    z: np.ndarray      # f64
    thx: np.ndarray    # f64 rad
    thy: np.ndarray    # f64 rad
    vlos: np.ndarray   # f32 km/s
    pos: np.ndarray | None = None  # f32 [3, n] comoving h^-1 Mpc
    map_id: np.ndarray | None = None  # i32


@dataclass
class LightCone:
    parts: dict                     # x,y,z,vx,vy,vz,hsml (f32), hid (i32)
    halos: HaloCatalog
    Mp: float                       # particle mass, h^-1 Msun
    geom: MapGeom
    info: dict = field(default_factory=dict)


def _chi_table(zmax: float, n: int = 20001):
    """Generator's own comoving distance table [h^-1 Mpc] (trapezoid on 1/E)."""
    z = np.linspace(0.0, zmax, n)
    inv_e = 1.0 / np.sqrt(OMEGA_M * (1 + z) ** 3 + 1 - OMEGA_M)
    chi = np.concatenate([[0.0], np.cumsum(0.5 * (inv_e[1:] + inv_e[:-1]) * np.diff(z))])
    return z, chi * C_KMS / 100.0


def _concentration(rng, M):
    return 5.0 * (M / 1e14) ** -0.1 * 10.0 ** rng.normal(0.0, 0.1, M.size)


def halo_catalog(n=1000, seed=SEED_BASE, side_deg=1.0, logm=(13.0, 15.0), zr=(0.05, 1.0),
                 npix=256) -> tuple[HaloCatalog, MapGeom]:
    """HP catalogue on a side_deg x side_deg flat patch centred on the origin."""
    rng = np.random.default_rng(seed)
    M = 10.0 ** rng.uniform(logm[0], logm[1], n)
    c = _concentration(rng, M)
    z = rng.uniform(zr[0], zr[1], n)
    half = 0.5 * side_deg * DEG
    thx = rng.uniform(-half, half, n)
    thy = rng.uniform(-half, half, n)
    vlos = rng.normal(0.0, 300.0, n).astype(np.float32)
    g = MapGeom(npix, npix, -half, -half, 2 * half / npix)
    return HaloCatalog(M, c, z, thx, thy, vlos), g


def powerlaw_masses(rng, n, mmin=1e12, mmax=1e15, slope=-0.9):
    """dN/dlnM ~ M^slope on [mmin, mmax] by inverse CDF."""
    u = rng.uniform(0.0, 1.0, n)
    a, b = mmin ** slope, mmax ** slope
    return (a + u * (b - a)) ** (1.0 / slope)


def batched_catalog(n_maps=108, mean_halos=5e4, seed=SEED_BASE + 3, side_deg=5.0, npix=2048,
                    zr=(0.01, 3.0)) -> tuple[HaloCatalog, MapGeom]:
    """Many independent flat maps, Poisson halo counts per map."""
    rng = np.random.default_rng(seed)
    counts = rng.poisson(mean_halos, n_maps)
    n = int(counts.sum())
    M = powerlaw_masses(rng, n)
    c = _concentration(rng, M)
    z = rng.uniform(zr[0], zr[1], n)
    half = 0.5 * side_deg * DEG
    thx = rng.uniform(-half, half, n)
    thy = rng.uniform(-half, half, n)
    vlos = rng.normal(0.0, 300.0, n).astype(np.float32)
    map_id = np.repeat(np.arange(n_maps, dtype=np.int32), counts)
    g = MapGeom(npix, npix, -half, -half, 2 * half / npix, n_maps)
    return HaloCatalog(M, c, z, thx, thy, vlos, map_id=map_id), g


def allsky_catalog(n, seed=SEED_BASE + 5, logm=None, zr=(0.01, 3.0), volume=True,
                   n_polar=0):
    """All-sky halo catalogue: directions uniform on the sphere (colatitude theta, longitude
    phi), masses dN/dlnM ~ M^-0.9 on [1e12, 1e15] (or log-uniform on logm), redshifts
    uniform in comoving volume on zr (or uniform in z), v_los ~ N(0, 300 km/s).  n_polar
    of the halos are put within 0.02 rad of a pole (half north, half south)."""
    rng = np.random.default_rng(seed)
    M = powerlaw_masses(rng, n) if logm is None else 10.0 ** rng.uniform(logm[0], logm[1], n)
    c = _concentration(rng, M)
    if volume:
        ztab, chitab = _chi_table(zr[1] * 1.05)
        c0, c1 = np.interp(zr, ztab, chitab)
        chi = (c0 ** 3 + rng.uniform(0.0, 1.0, n) * (c1 ** 3 - c0 ** 3)) ** (1.0 / 3.0)
        z = np.interp(chi, chitab, ztab)
    else:
        z = rng.uniform(zr[0], zr[1], n)
    theta = np.arccos(rng.uniform(-1.0, 1.0, n))
    phi = rng.uniform(0.0, 2 * math.pi, n)
    if n_polar:
        k = rng.choice(n, n_polar, replace=False)
        t = rng.uniform(0.0, 0.02, n_polar)
        theta[k] = np.where(np.arange(n_polar) % 2 == 0, t, math.pi - t)
    vlos = rng.normal(0.0, 300.0, n).astype(np.float32)
    return {"M": M, "c": c, "z": z, "theta": theta, "phi": phi, "vlos": vlos}


def _cone_points(rng, n, tan_half, chi_lo, chi_hi):
    """Points uniform in comoving volume with |x/z|,|y/z| <= tan_half and chi in range."""
    out = np.empty((0, 3))
    while out.shape[0] < n:
        m = int((n - out.shape[0]) * 3.2) + 1024
        zc = chi_hi * rng.uniform(0.0, 1.0, m) ** (1.0 / 3.0)  # density ~ z^2 in the pyramid
        xx = rng.uniform(-1.0, 1.0, m) * tan_half * zc
        yy = rng.uniform(-1.0, 1.0, m) * tan_half * zc
        r = np.sqrt(xx * xx + yy * yy + zc * zc)
        ok = (r >= chi_lo) & (r <= chi_hi)
        out = np.concatenate([out, np.stack([xx[ok], yy[ok], zc[ok]], 1)])
    return out[:n]


def _nfw_radii(rng, c, n_each):
    """Radii in units of the cloud radius from a truncated NFW (inverse CDF, bisection)."""
    cc = np.repeat(c, n_each)
    u = rng.uniform(0.0, 1.0, cc.size)
    mc = np.log1p(cc) - cc / (1 + cc)
    lo = np.zeros_like(cc)
    hi = cc.copy()
    for _ in range(48):
        mid = 0.5 * (lo + hi)
        f = (np.log1p(mid) - mid / (1 + mid)) / mc - u
        lo = np.where(f < 0, mid, lo)
        hi = np.where(f < 0, hi, mid)
    return 0.5 * (lo + hi) / cc  # x / c = r / R


def _rotations(rng, n):
    q = rng.normal(size=(n, 4))
    q /= np.linalg.norm(q, axis=1, keepdims=True)
    w, x, y, z = q.T
    return np.stack([
        np.stack([1 - 2 * (y * y + z * z), 2 * (x * y - z * w), 2 * (x * z + y * w)], -1),
        np.stack([2 * (x * y + z * w), 1 - 2 * (x * x + z * z), 2 * (y * z - x * w)], -1),
        np.stack([2 * (x * z - y * w), 2 * (y * z + x * w), 1 - 2 * (x * x + y * y)], -1),
    ], 1)  # [n, 3, 3]


def lightcone(n_part=4_000_000, n_halo=3000, side_deg=2.0, zr=(0.05, 1.5), halo_frac=0.6,
              npix=1024, seed=SEED_BASE + 1, mass="loguniform", n_ngb=64) -> LightCone:
    """Light-cone particles + the catalogue of their halos."""
    rng = np.random.default_rng(seed)
    ztab, chitab = _chi_table(max(zr[1], 3.0) * 1.2)
    chi_lo, chi_hi = np.interp(zr, ztab, chitab)
    half = 0.5 * side_deg * DEG
    tan_half = math.tan(half)
    vol = (2 * tan_half) ** 2 * (chi_hi ** 3 - chi_lo ** 3) / 3.0  # pyramid shell (approx.)

    # halos
    if mass == "loguniform":
        M = 10.0 ** rng.uniform(13.0, 15.0, n_halo)
    else:
        M = powerlaw_masses(rng, n_halo)
    c = _concentration(rng, M)
    hp = _cone_points(rng, n_halo, tan_half, chi_lo, chi_hi)
    hchi = np.linalg.norm(hp, axis=1)
    hz = np.interp(hchi, chitab, ztab)
    thx = np.arctan2(hp[:, 0], hp[:, 2])
    thy = np.arctan2(hp[:, 1], hp[:, 2])
    hv = rng.normal(0.0, 300.0, n_halo).astype(np.float32)

    # particles per halo proportional to mass (largest remainder)
    n_h = int(round(halo_frac * n_part))
    share = M / M.sum() * n_h
    cnt = np.floor(share).astype(np.int64)
    rem = n_h - int(cnt.sum())
    if rem > 0:
        cnt[np.argsort(-(share - cnt), kind="stable")[:rem]] += 1
    Mp = float(M.sum() / n_h)

    R = (3.0 * M / (4.0 * math.pi * 200.0 * OMEGA_M * RHO_CRIT0_H2)) ** (1.0 / 3.0)
    rad = _nfw_radii(rng, c, cnt) * np.repeat(R, cnt)
    d = rng.normal(size=(n_h, 3))
    d /= np.linalg.norm(d, axis=1, keepdims=True)
    q = rng.uniform(0.5, 1.0, n_halo)
    s = rng.uniform(0.5, 1.0, n_halo)
    scale = np.stack([np.ones(n_halo), q, s], 1) / np.cbrt(q * s)[:, None]
    off = d * rad[:, None] * np.repeat(scale, cnt, axis=0)
    rot = _rotations(rng, n_halo)
    off = np.einsum("nij,nj->ni", np.repeat(rot, cnt, axis=0), off)
    hpos_p = np.repeat(hp, cnt, axis=0) + off
    hid_h = np.repeat(np.arange(n_halo, dtype=np.int32), cnt)

    # field particles
    n_f = n_part - n_h
    fpos = _cone_points(rng, n_f, tan_half, chi_lo, chi_hi)
    n_field = n_f / vol

    # smoothing lengths from the neighbour rule
    rs = np.repeat(R / c, cnt)
    mcv = np.repeat(np.log1p(c) - c / (1 + c), cnt)
    x = rad / rs
    rho = np.repeat(M, cnt) / (4 * math.pi * rs ** 3 * mcv) / (x * (1 + x) ** 2)
    h_field = (3.0 * n_ngb / (4.0 * math.pi * n_field)) ** (1.0 / 3.0)
    h_halo = np.minimum((3.0 * n_ngb / (4.0 * math.pi * (rho / Mp))) ** (1.0 / 3.0), h_field)

    pos = np.concatenate([hpos_p, fpos])
    hs = np.concatenate([h_halo, np.full(n_f, h_field)])
    hid = np.concatenate([hid_h, np.full(n_f, -1, np.int32)])
    vel = rng.normal(0.0, 300.0, (n_part, 3))
    perm = rng.permutation(n_part)
    parts = {
        "x": pos[perm, 0].astype(np.float32), "y": pos[perm, 1].astype(np.float32),
        "z": pos[perm, 2].astype(np.float32),
        "vx": vel[perm, 0].astype(np.float32), "vy": vel[perm, 1].astype(np.float32),
        "vz": vel[perm, 2].astype(np.float32),
        "hsml": hs[perm].astype(np.float32), "hid": hid[perm].astype(np.int32),
    }
    cat = HaloCatalog(M, c, hz, thx, thy, hv, pos=hp.T.astype(np.float32).copy())
    g = MapGeom(npix, npix, -half, -half, 2 * half / npix)
    # each halo particle's radius on its cloud's ellipsoidal shell (before the axis ratios
    # and the rotation; comoving h^-1 Mpc), NaN for the field: the geometry a potential on
    # ellipsoidal shells needs
    r_ell = np.concatenate([rad, np.full(n_f, np.nan)])[perm]
    return LightCone(parts, cat, Mp, g, {"h_field": h_field, "n_halo_particles": n_h,
                                         "r_ell": r_ell})


def split_positions(p):
    """Pixel-unit positions -> (int32 floor, float32 fraction in [0, 1), the exact FP64
    value ix + fx), the position representation of the deposit's particle records."""
    p = np.asarray(p, np.float64)
    fl = np.floor(p)
    fr = (p - fl).astype(np.float32)
    up = fr >= 1.0
    fl = fl + up
    fr[up] = 0.0
    ix = np.clip(fl, -2 ** 30, 2 ** 30).astype(np.int32)
    return ix, fr, ix.astype(np.float64) + fr.astype(np.float64)


def assigned_particles(n=20000, npix=96, seed=SEED_BASE + 11, hmax=24.0, frac_field=0.4,
                       margin=8.0):
    """Directly drawn per-particle deposit inputs (pixel positions, kernel radius in
    pixels, signals) for testing the deposit alone.  Mixes tiny (sub-pixel), medium and
    large kernels, particles straddling the map edge, h = 0, and signed B."""
    rng = np.random.default_rng(seed)
    ix, fx, px = split_positions(rng.uniform(-margin, npix + margin, n))
    iy, fy, py = split_positions(rng.uniform(-margin, npix + margin, n))
    u = rng.uniform(0, 1, n)
    hp = np.where(u < 0.3, rng.uniform(0.0, 1.0, n),
                  np.where(u < 0.8, rng.uniform(1.0, 6.0, n), rng.uniform(6.0, hmax, n)))
    hp[rng.uniform(0, 1, n) < 0.02] = 0.0
    kind = (rng.uniform(0, 1, n) < frac_field).astype(np.int32)
    kind[rng.uniform(0, 1, n) < 0.05] = 2
    Y = np.where(kind == 0, 10.0 ** rng.uniform(-9, -6, n), 0.0)
    B = np.where(kind == 2, 0.0, rng.normal(0.0, 1e-7, n))
    return {"ix": ix, "fx": fx, "iy": iy, "fy": fy, "px": px, "py": py,
            "hp": hp.astype(np.float32), "Y": Y.astype(np.float32),
            "B": B.astype(np.float32), "kind": kind}


def deposit_inputs(px, py, hp, Y, B, kind):
    """Deposit inputs from given pixel positions (any float type)."""
    ix, fx, px = split_positions(px)
    iy, fy, py = split_positions(py)
    return {"ix": ix, "fx": fx, "iy": iy, "fy": fy, "px": px, "py": py,
            "hp": np.asarray(hp, np.float32), "Y": np.asarray(Y, np.float32),
            "B": np.asarray(B, np.float32), "kind": np.asarray(kind, np.int32)}


# Ranges of the surrogate's inputs.  The paper quotes point values (Table 1) only; the
# three parameters that enter the solve are varied over these ranges.
SURROGATE_RANGES = {
    "log10_M": (12.0, 15.3),
    "dlog10_c": (-0.3, 0.3),      # around c = 5 (M/1e14)^-0.1
    "z": (0.01, 3.0),
    "eps_star": (0.0, 1.0e-5),
    "f_star": (0.01, 0.04),
    "eps_dm": (0.0, 0.1),
}


def surrogate_halos(n, seed=SEED_BASE + 4):
    """Halo features for the surrogate: (M [h^-1 Msun], c, z, params [3, n] = eps_*, f_*,
    eps_DM), uniform over SURROGATE_RANGES."""
    rng = np.random.default_rng(seed)
    R = SURROGATE_RANGES
    M = 10.0 ** rng.uniform(*R["log10_M"], n)
    c = 5.0 * (M / 1e14) ** -0.1 * 10.0 ** rng.uniform(*R["dlog10_c"], n)
    z = rng.uniform(*R["z"], n)
    prm = np.stack([rng.uniform(*R["eps_star"], n), rng.uniform(*R["f_star"], n),
                    rng.uniform(*R["eps_dm"], n)])
    return M, c, z, prm


def lightcone_device(n_part, n_halo, side_deg=5.0, zr=(0.05, 3.0), halo_frac=0.6, npix=4096,
                     seed=SEED_BASE + 2, mass="powerlaw", n_ngb=64, device="cuda",
                     chunk=50_000_000, sample=None):
    """The light-cone recipe of `lightcone`, drawn with torch's seeded generator on a
    device so that 1e8-1e9 particles take seconds (the numpy generator would take
    minutes).  Same distributions; different random streams, so it is its own seeded
    workload.  Returns a LightCone whose parts are device tensors (halo catalogue on
    the host).

    sample=(halo_keep, field_keep): a representative subsample of the same cone for
    timing slow consumers: the full halo catalogue, a seeded subset of its halos (each
    kept with probability halo_keep) with all of their particles, and a field_keep share
    of the field particles.  Particle mass, smoothing lengths and everything else are
    those of the full cone (n_part particles); the particles are different draws."""
    import torch

    dev = torch.device(device)
    gen = torch.Generator(device=dev)
    gen.manual_seed(seed)
    rng = np.random.default_rng(seed)
    f32 = torch.float32

    def U(n, lo=0.0, hi=1.0):
        return torch.rand(n, generator=gen, device=dev, dtype=f32) * (hi - lo) + lo

    ztab, chitab = _chi_table(max(zr[1], 3.0) * 1.2)
    chi_lo, chi_hi = np.interp(zr, ztab, chitab)
    half = 0.5 * side_deg * DEG
    tan_half = math.tan(half)
    vol = (2 * tan_half) ** 2 * (chi_hi ** 3 - chi_lo ** 3) / 3.0

    def cone(n):
        out = []
        got = 0
        while got < n:
            m = int((n - got) * 3.2) + 1024
            zc = chi_hi * U(m) ** (1.0 / 3.0)
            xx = (U(m) * 2 - 1) * tan_half * zc
            yy = (U(m) * 2 - 1) * tan_half * zc
            r = torch.sqrt(xx * xx + yy * yy + zc * zc)
            ok = (r >= chi_lo) & (r <= chi_hi)
            pts = torch.stack([xx[ok], yy[ok], zc[ok]], 1)
            out.append(pts)
            got += pts.shape[0]
        return torch.cat(out)[:n]

    # halos (host catalogue, small)
    if mass == "loguniform":
        M = 10.0 ** rng.uniform(13.0, 15.0, n_halo)
    else:
        M = powerlaw_masses(rng, n_halo)
    c = _concentration(rng, M)
    hpos = cone(n_halo).double().cpu().numpy()
    hz = np.interp(np.linalg.norm(hpos, axis=1), chitab, ztab)
    thx = np.arctan2(hpos[:, 0], hpos[:, 2])
    thy = np.arctan2(hpos[:, 1], hpos[:, 2])
    hv = rng.normal(0.0, 300.0, n_halo).astype(np.float32)
    n_h = int(round(halo_frac * n_part))
    share = M / M.sum() * n_h
    cnt = np.floor(share).astype(np.int64)
    rem = n_h - int(cnt.sum())
    if rem > 0:
        cnt[np.argsort(-(share - cnt), kind="stable")[:rem]] += 1
    Mp = float(M.sum() / n_h)
    R = (3.0 * M / (4.0 * math.pi * 200.0 * OMEGA_M * RHO_CRIT0_H2)) ** (1.0 / 3.0)
    q = rng.uniform(0.5, 1.0, n_halo)
    s = rng.uniform(0.5, 1.0, n_halo)
    rot = _rotations(rng, n_halo)
    n_f = n_part - n_h
    n_field = n_f / vol
    h_field = (3.0 * n_ngb / (4.0 * math.pi * n_field)) ** (1.0 / 3.0)
    if sample is not None:  # a subset of the halos with all their particles, part of the field
        keep = np.random.default_rng(seed + 7919).random(n_halo) < sample[0]
        cnt = np.where(keep, cnt, 0)
        n_h = int(cnt.sum())
        n_f = int(round(n_f * sample[1]))
        n_part = n_h + n_f
    td = lambda a: torch.from_numpy(np.ascontiguousarray(a)).to(dev)
    c_t, R_t, M_t = td(c.astype(np.float32)), td(R.astype(np.float32)), td(M)
    sc_t = td((np.stack([np.ones(n_halo), q, s], 1) / np.cbrt(q * s)[:, None]).astype(np.float32))
    rot_t = td(rot.astype(np.float32))
    hp_t = td(hpos.astype(np.float32))
    mc_t = torch.log1p(c_t) - c_t / (1 + c_t)
    hid_all = torch.repeat_interleave(torch.arange(n_halo, device=dev, dtype=torch.int32),
                                      td(cnt))
    X = torch.empty((n_part, 3), dtype=f32, device=dev)
    HS = torch.empty(n_part, dtype=f32, device=dev)
    for a in range(0, n_h, chunk):
        b = min(n_h, a + chunk)
        hid = hid_all[a:b].long()
        cc = c_t[hid]
        u = U(b - a)
        lo = torch.zeros_like(cc)
        hi = cc.clone()
        mcc = mc_t[hid]
        for _ in range(40):
            mid = 0.5 * (lo + hi)
            f = (torch.log1p(mid) - mid / (1 + mid)) / mcc - u
            neg = f < 0
            lo = torch.where(neg, mid, lo)
            hi = torch.where(neg, hi, mid)
        xr = 0.5 * (lo + hi)  # r / r_s
        rad = xr / cc * R_t[hid]
        d = torch.randn((b - a, 3), generator=gen, device=dev, dtype=f32)
        d = d / torch.linalg.norm(d, dim=1, keepdim=True)
        off = d * rad[:, None] * sc_t[hid]
        off = torch.einsum("nij,nj->ni", rot_t[hid], off)
        X[a:b] = hp_t[hid] + off
        rs = R_t[hid] / cc
        rho = M_t[hid].float() / (4 * math.pi * rs ** 3 * mcc) / (xr * (1 + xr) ** 2)
        HS[a:b] = torch.clamp((3.0 * n_ngb / (4.0 * math.pi * (rho / Mp))) ** (1.0 / 3.0),
                              max=h_field)
        del hid, cc, u, lo, hi, mcc, xr, rad, d, off, rs, rho
    for a in range(n_h, n_part, chunk):
        b = min(n_part, a + chunk)
        X[a:b] = cone(b - a)
        HS[a:b] = h_field
    HID = torch.full((n_part,), -1, dtype=torch.int32, device=dev)
    HID[:n_h] = hid_all
    del hid_all
    perm = torch.randperm(n_part, generator=gen, device=dev)
    parts = {}
    for k, col in (("x", 0), ("y", 1), ("z", 2)):
        parts[k] = X[:, col][perm].contiguous()
    del X
    parts["hsml"] = HS[perm]
    del HS
    parts["hid"] = HID[perm]
    del HID, perm
    for k in ("vx", "vy", "vz"):
        parts[k] = torch.randn(n_part, generator=gen, device=dev, dtype=f32) * 300.0
    cat = HaloCatalog(M, c, hz, thx, thy, hv, pos=hpos.T.astype(np.float32).copy())
    g = MapGeom(npix, npix, -half, -half, 2 * half / npix)
    meta = {"h_field": h_field, "n_halo_particles": n_h}
    if sample is not None:
        meta["sample"] = {"halo_keep": sample[0], "field_keep": sample[1],
                          "halos_kept": int(keep.sum()), "particles": n_part}
    return LightCone(parts, cat, Mp, g, meta)

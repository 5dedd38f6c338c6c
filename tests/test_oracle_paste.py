"""Pins of the oracle's pasting functions (Sections 3.3 and 3.4).

Kernel weights against the printed exact values and against direct quadrature of
the 1-D kernel shape; the deposit against brute force and the normalisation
identity; HP against an independent Abel projection; PP assignment against the
linearity and symmetry the equations fix.
"""
import math
import os

import numpy as np
import pytest
from scipy.integrate import quad

from paper_2201_02632_gb300 import inputs as I

HERE = os.path.dirname(__file__)


def _shape(x):
    """1-D cubic-spline kernel shape of Eq. SPH_kernel (unnormalised, |x| <= 1)."""
    x = abs(x)
    if x < 0.5:
        return 1 - 6 * x * x + 6 * x ** 3
    if x < 1:
        return 2 * (1 - x) ** 3
    return 0.0


_NORM = quad(_shape, -1, 1, points=[-0.5, 0, 0.5], epsabs=0, epsrel=1e-13)[0]


def _w_numeric(x):
    """w_SPH from its definition: normalised integral of the kernel up to x."""
    if x <= -1:
        return 0.0
    hi = min(x, 1.0)
    pts = [p for p in (-0.5, 0.0, 0.5) if -1 < p < hi]
    return quad(_shape, -1, hi, points=pts or None, epsabs=0, epsrel=1e-13)[0] / _NORM


# ---------------------------------------------------------------- kernel
def test_w_sph_exact_values(orc):
    rows = [l.split() for l in open(os.path.join(HERE, "golden", "w_sph_values.txt"))
            if l.strip() and not l.startswith("#")]
    for x, num, den in rows:
        assert orc.w_sph(float(x)) == pytest.approx(int(num) / int(den), abs=1e-15)


def test_w_sph_is_the_normalised_kernel_integral(orc):
    for x in np.linspace(-1.2, 1.2, 49):
        assert orc.w_sph(x) == pytest.approx(_w_numeric(x), abs=2e-14)


def test_w_sph_derivative_and_continuity(orc):
    assert _NORM == pytest.approx(0.75, rel=1e-14)
    for x in (-0.9, -0.6, -0.2, 0.0, 0.3, 0.7):
        d = 1e-6
        der = (orc.w_sph(x + d) - orc.w_sph(x - d)) / (2 * d)
        assert der == pytest.approx(_shape(x) / 0.75, rel=1e-8, abs=1e-12)
    for b in (-0.5, 0.5):
        assert orc.w_sph(b - 1e-13) == pytest.approx(orc.w_sph(b + 1e-13), abs=1e-12)


def _one(px, py, hp, Y=1.0, B=0.0, kind=0):
    f32 = lambda v: np.array([v], np.float64)
    return {"px": f32(px), "py": f32(py), "hp": f32(hp), "Y": f32(Y), "B": f32(B),
            "kind": np.array([kind], np.int32)}


def test_worked_example_pixel_centre_h_one_pixel(orc):
    g = orc.geom(8, 8, 0.0, 0.0, 1.0)
    ym, _ = orc.pp_deposit(_one(4.5, 3.5, 1.0), g)
    np.testing.assert_allclose(ym[2:5, 3:6], [[1 / 576, 11 / 288, 1 / 576],
                                              [11 / 288, 121 / 144, 11 / 288],
                                              [1 / 576, 11 / 288, 1 / 576]], rtol=1e-14)
    assert ym.sum() == pytest.approx(1.0, abs=1e-15)


def test_deposit_brute_force_tiny(orc):
    """Each pixel weight equals the product of the kernel's normalised integrals over
    the pixel's x and y extent (direct quadrature), on 8x8 maps."""
    rng = np.random.default_rng(3)
    g = orc.geom(8, 8, 0.0, 0.0, 1.0)
    n = 12
    a = {"px": rng.uniform(-1, 9, n), "py": rng.uniform(-1, 9, n),
         "hp": rng.uniform(0.2, 4.0, n), "Y": rng.uniform(0.5, 2, n),
         "B": rng.normal(0, 1, n), "kind": np.zeros(n, np.int32)}
    ym, bm = orc.pp_deposit(a, g)
    ref_y = np.zeros((8, 8))
    ref_b = np.zeros((8, 8))
    for k in range(n):
        h = a["hp"][k]
        wx = [_w_numeric((i + 1 - a["px"][k]) / h) - _w_numeric((i - a["px"][k]) / h)
              for i in range(8)]
        wy = [_w_numeric((j + 1 - a["py"][k]) / h) - _w_numeric((j - a["py"][k]) / h)
              for j in range(8)]
        ref_y += a["Y"][k] * np.outer(wy, wx)
        ref_b += a["B"][k] * np.outer(wy, wx)
    np.testing.assert_allclose(ym, ref_y, rtol=1e-11, atol=1e-14)
    np.testing.assert_allclose(bm, ref_b, rtol=1e-11, atol=1e-13)


def test_deposit_normalisation_and_map_integral(orc):
    """sum_ij f_ij = 1 (Section 3.4) for particles whose 2h square is interior, so the
    map integral equals the sum of the particle signals."""
    rng = np.random.default_rng(5)
    g = orc.geom(64, 48, 0.0, 0.0, 1.0)
    n = 300
    hp = rng.uniform(0.0, 7.0, n)
    a = {"px": rng.uniform(8, 56, n), "py": rng.uniform(8, 40, n), "hp": hp,
         "Y": rng.uniform(0, 1, n), "B": rng.normal(0, 1, n), "kind": np.zeros(n, np.int32)}
    ym, bm = orc.pp_deposit(a, g)
    assert ym.sum() == pytest.approx(a["Y"].sum(), rel=1e-13)
    assert bm.sum() == pytest.approx(a["B"].sum(), rel=1e-12, abs=1e-12)


def test_deposit_h_zero_is_nearest_grid_point(orc):
    g = orc.geom(8, 8, 0.0, 0.0, 1.0)
    ym, _ = orc.pp_deposit(_one(2.3, 6.9, 0.0, Y=3.0), g)
    assert ym[6, 2] == 3.0 and ym.sum() == 3.0


def test_deposit_select_and_sampled_pixels(orc):
    a = I.assigned_particles(n=3000, npix=40, hmax=10)
    a = {k: (np.asarray(a[k], np.float64) if k != "kind" else a[k])
         for k in ("px", "py", "hp", "Y", "B", "kind")}
    g = orc.geom(40, 40, 0.0, 0.0, 1.0)
    ya, ba = orc.pp_deposit(a, g, select=0)
    yh, bh = orc.pp_deposit(a, g, select=1)
    yf, bf = orc.pp_deposit(a, g, select=2)
    np.testing.assert_allclose(ya, yh + yf, rtol=1e-12, atol=1e-22)
    np.testing.assert_allclose(ba, bh + bf, rtol=1e-10, atol=1e-20)
    assert np.all(yf == 0)  # field particles carry no tSZ (Eq. field_y)
    pi_ = np.array([0, 5, 39, 20, 13])
    pj_ = np.array([0, 7, 39, 3, 33])
    yv, bv = orc.pp_deposit_pixels(a, g, pi_, pj_)
    np.testing.assert_allclose(yv, ya[pj_, pi_], rtol=1e-12, atol=1e-22)
    np.testing.assert_allclose(bv, ba[pj_, pi_], rtol=1e-10, atol=1e-20)


def test_tile_pairs_cover_every_weighted_pixel(orc):
    """Every pixel that receives weight lies in a tile paired with the particle, and
    each paired tile meets the particle's pixel span; keys ascend, ties by index."""
    a = I.assigned_particles(n=400, npix=70, hmax=20)
    nx = ny = 70
    tw, th = 16, 8
    keys, vals = orc.pp_pairs(a["ix"], a["fx"], a["iy"], a["fy"], a["hp"], a["kind"], nx, ny,
                              tw, th)
    order = np.lexsort((vals, keys))
    assert np.array_equal(order, np.arange(keys.size))
    ntx = (nx + tw - 1) // tw
    g = orc.geom(nx, ny, 0.0, 0.0, 1.0)
    a64 = {k: (np.asarray(a[k], np.float64) if k != "kind" else a[k])
           for k in ("px", "py", "hp", "Y", "B", "kind")}
    for k in range(0, 400, 7):
        if a["kind"][k] == 2:
            assert not np.any(vals == k)
            continue
        one = {kk: vv[k:k + 1] for kk, vv in a64.items()}
        one["Y"] = np.ones(1)
        ym, _ = orc.pp_deposit(one, g)
        jj, ii = np.nonzero(ym)
        tiles = set((jj // th * ntx + ii // tw).tolist())
        mine = set(keys[vals == k].tolist())
        assert tiles <= mine


# ---------------------------------------------------------------- HP
@pytest.fixture(scope="module")
def one_halo(orc):
    m = orc.solve_halos([2e14], [4.0], [0.25])[0]
    return m


def test_los_integral_vs_independent_abel_projection(orc, one_halo):
    """2 int P_e(sqrt(r^2 + x^2)) dx (Eqs. y^HP, b^HP) with scipy on the profile."""
    m = one_halo
    F = orc.F
    rf = m[F["r_f"]]
    for s in (0.0, 0.01, 0.2, 0.6, 0.95, 0.999):
        rp = s * rf
        L = math.sqrt(rf * rf - rp * rp)
        for which in (0, 1):
            f = lambda x: orc.profile(m, [math.hypot(rp, x)])[which][0]
            pts = [math.sqrt(max(r * r - rp * rp, 0)) for r in (m[F["r_vir"]],) if r > rp]
            ref = 2 * quad(f, 0, L, points=[p for p in pts if 0 < p < L] or None,
                           epsabs=0, epsrel=1e-11, limit=400)[0]
            got = orc.los_integral(m, rp, which)
            assert got == pytest.approx(ref, rel=1e-9)


def test_hp_map_integral_equals_volume_integral(orc, one_halo):
    """sum_pix y Omega_pix = sigma_T/(m_e c^2) int P_e dV / D_A^2 for a resolved halo
    (the projection conserves the volume integral)."""
    m = one_halo
    F = orc.F
    rf, DA = m[F["r_f"]], m[F["D_A"]]
    ang = rf / DA
    npix = 128
    d = 2.2 * ang / npix
    g = orc.geom(npix, npix, -1.1 * ang, -1.1 * ang, d)
    ym, bm = orc.hp_map([0.0], [0.0], [500.0], m[None, :], g, rtol=1e-9)
    vol = quad(lambda r: 4 * math.pi * r * r * orc.profile(m, [r])[0][0], 0, rf,
               points=[m[F["r_vir"]]], epsabs=0, epsrel=1e-11, limit=400)[0]
    total = ym.sum() * d * d
    # pixel-centre sampling of a smooth, resolved disc: error ~ (pixel/size)^2
    assert total == pytest.approx(orc.const_CP() * vol / DA ** 2, rel=2e-3)
    volb = quad(lambda r: 4 * math.pi * r * r * orc.profile(m, [r])[1][0], 0, rf,
                points=[m[F["r_vir"]]], epsabs=0, epsrel=1e-11, limit=400)[0]
    ref_b = orc.const_CN() * (500.0 / 299792.458) * math.exp(-m[F["tau"]]) * volb / DA ** 2
    assert bm.sum() * d * d == pytest.approx(ref_b, rel=2e-3)


def test_hp_brute_force_small_map(orc):
    """Three halos on a 16x16 map against a direct double loop with scipy LOS
    integrals, aperture 3 r500 (the c0 convention)."""
    rng = np.random.default_rng(11)
    M = np.array([5e14, 1e14, 3e13])
    mod = orc.solve_halos(M, 5 * (M / 1e14) ** -0.1, [0.3, 0.5, 0.2])
    F = orc.F
    side = 0.25 * math.pi / 180
    g = orc.geom(16, 16, -side / 2, -side / 2, side / 16)
    thx = rng.uniform(-side / 2, side / 2, 3)
    thy = rng.uniform(-side / 2, side / 2, 3)
    v = np.array([300.0, -150.0, 20.0])
    ym, bm = orc.hp_map(thx, thy, v, mod, g, ap_r500=3.0, rtol=1e-10)
    ref_y = np.zeros((16, 16))
    for k in range(3):
        m = mod[k]
        rap = min(m[F["r_f"]], 3 * m[F["r500"]])
        for j in range(16):
            for i in range(16):
                tx = g.theta0_x + (i + 0.5) * g.dtheta
                ty = g.theta0_y + (j + 0.5) * g.dtheta
                rp = m[F["D_A"]] * math.hypot(tx - thx[k], ty - thy[k])
                if rp < rap:
                    L = math.sqrt(m[F["r_f"]] ** 2 - rp * rp)
                    f = lambda x: orc.profile(m, [math.hypot(rp, x)])[0][0]
                    ref_y[j, i] += orc.const_CP() * 2 * quad(f, 0, L, epsrel=1e-10,
                                                             limit=300)[0]
    np.testing.assert_allclose(ym[0], ref_y, rtol=1e-7, atol=1e-20)
    assert np.count_nonzero(ym) > 20


def test_hp_pairs_cover_contributing_pixels(orc):
    cat, _ = I.halo_catalog(n=40, npix=64)
    g = orc.geom(64, 64, cat.thx.min() - 1e-3, cat.thy.min() - 1e-3,
                 (cat.thx.max() - cat.thx.min() + 2e-3) / 64)
    mod = orc.solve_halos(cat.M, cat.c, cat.z)
    keys, vals = orc.hp_pairs(cat.thx, cat.thy, mod, g, 3.0, 16, 16)
    assert np.array_equal(np.lexsort((vals, keys)), np.arange(keys.size))
    for k in range(40):
        ym, _ = orc.hp_map(cat.thx[k:k + 1], cat.thy[k:k + 1], cat.vlos[k:k + 1],
                           mod[k:k + 1], g, ap_r500=3.0, rtol=1e-6)
        jj, ii = np.nonzero(ym[0])
        tiles = set((jj // 16 * 4 + ii // 16).tolist())
        assert tiles <= set(keys[vals == k].tolist())


# ---------------------------------------------------------------- PP assignment
@pytest.fixture(scope="module")
def small_cone(orc):
    lc = I.lightcone(n_part=20000, n_halo=30, npix=128, seed=99)
    mod = orc.solve_halos(lc.halos.M, lc.halos.c, lc.halos.z)
    g = orc.geom(lc.geom.nx, lc.geom.ny, lc.geom.theta0_x, lc.geom.theta0_y, lc.geom.dtheta)
    return lc, mod, g


def test_ksz_linear_in_velocity(orc, small_cone):
    """b is linear in v (Eqs. b_i^PP,h and field_b): v = 0 gives b = 0 exactly and
    flipping v flips b exactly; y does not depend on v."""
    lc, mod, g = small_cone
    a = orc.pp_assign(lc.parts, lc.Mp, lc.halos.pos, mod, g)
    p0 = dict(lc.parts, vx=np.zeros_like(lc.parts["vx"]), vy=np.zeros_like(lc.parts["vy"]),
              vz=np.zeros_like(lc.parts["vz"]))
    a0 = orc.pp_assign(p0, lc.Mp, lc.halos.pos, mod, g)
    assert np.all(a0["B"] == 0.0)
    pn = dict(lc.parts, vx=-lc.parts["vx"], vy=-lc.parts["vy"], vz=-lc.parts["vz"])
    an = orc.pp_assign(pn, lc.Mp, lc.halos.pos, mod, g)
    assert np.array_equal(an["B"], -a["B"])
    assert np.array_equal(an["Y"], a["Y"])
    yb, bb = orc.pp_deposit(a, g)
    yn, bn = orc.pp_deposit(an, g)
    assert np.array_equal(bn, -bb) and np.array_equal(yn, yb)
    assert np.all(a["Y"][a["kind"] == 1] == 0)


def test_field_particle_signal(orc, small_cone):
    """Field b_i = sigma_T (v_r/c) M_p/(mu_e m_p) e^-tau / L_pix^2 (Eq. field_b),
    rebuilt from SI constants for a handful of particles."""
    lc, mod, g = small_cone
    a = orc.pp_assign(lc.parts, lc.Mp, lc.halos.pos, mod, g)
    idx = np.nonzero(lc.parts["hid"] < 0)[0][:5]
    sigT, mp, MSUN, MPC = 6.6524587321e-29, 1.67262192369e-27, 1.98840987e30, \
        3.0856775814913673e22
    for i in idx:
        r = np.array([lc.parts[k][i] for k in "xyz"], np.float64) / 0.7
        chi = np.linalg.norm(r)
        z = orc.z_of_chi(chi)
        DA = chi / (1 + z)
        vr = np.dot([float(lc.parts[k][i]) for k in ("vx", "vy", "vz")], r) / chi
        ne = lc.Mp / 0.7 * MSUN / (2 / 1.76 * mp)  # electrons in the particle
        Lpix = DA * MPC * g.dtheta
        b = sigT * vr / 299792.458 * ne * math.exp(-orc.tau(z)) / Lpix ** 2
        assert a["B"][i] == pytest.approx(b, rel=1e-10)
        assert a["px"][i] == pytest.approx((math.atan2(r[0], r[2]) - g.theta0_x) / g.dtheta,
                                           rel=1e-12)
        assert a["hp"][i] == pytest.approx(float(lc.parts["hsml"][i]) / 0.7 / chi / g.dtheta,
                                           rel=1e-12)


def test_pp_halo_signal_is_monte_carlo_volume_integral(orc):
    """Particles drawn from one NFW halo (mass M_p each) with V_i = M_p/rho(r_i):
    sum_i y_i Omega_pix is an unbiased estimate of sigma_T/(m_e c^2) int P_e dV / D_A^2
    over the sampled sphere (Section 3.4)."""
    m = orc.solve_halos([3e14], [4.0], [0.3])[0]
    F = orc.F
    rng = np.random.default_rng(2)
    N = 200000
    rv, c = m[F["r_vir"]], m[F["c"]]
    u = rng.uniform(0, 1, N)
    mc = math.log1p(c) - c / (1 + c)
    lo, hi = np.zeros(N), np.full(N, c)
    for _ in range(60):
        mid = 0.5 * (lo + hi)
        f = (np.log1p(mid) - mid / (1 + mid)) / mc - u
        lo, hi = np.where(f < 0, mid, lo), np.where(f < 0, hi, mid)
    r_phys = 0.5 * (lo + hi) / c * rv
    d = rng.normal(size=(N, 3))
    d /= np.linalg.norm(d, axis=1, keepdims=True)
    zc = 800.0  # h^-1 Mpc comoving along the axis
    hpos = np.array([[0.0], [0.0], [zc]], np.float32)
    off = d * (r_phys * (1 + m[F["z"]]) * 0.7)[:, None]
    parts = {"x": off[:, 0].astype(np.float32), "y": off[:, 1].astype(np.float32),
             "z": (zc + off[:, 2]).astype(np.float32), "vx": np.zeros(N, np.float32),
             "vy": np.zeros(N, np.float32), "vz": np.zeros(N, np.float32),
             "hsml": np.full(N, 0.05, np.float32), "hid": np.zeros(N, np.int32)}
    Mp = 3e14 / N
    g = orc.geom(64, 64, -0.01, -0.01, 0.02 / 64)
    a = orc.pp_assign(parts, Mp, hpos, m[None, :], g)
    # the particle's own D_A differs slightly from the centre's; undo it per particle
    chi = np.sqrt(parts["x"].astype(np.float64) ** 2 + parts["y"].astype(np.float64) ** 2
                  + parts["z"].astype(np.float64) ** 2) / 0.7
    zp = np.array([orc.z_of_chi(v) for v in chi[:2000]])
    DA_c = m[F["D_A"]]
    w = np.interp(chi, chi[:2000][np.argsort(chi[:2000])],
                  (chi[:2000] / (1 + zp))[np.argsort(chi[:2000])])
    est = np.sum(a["Y"] * (w / DA_c) ** 2) * g.dtheta ** 2
    ref = orc.const_CP() * quad(lambda r: 4 * math.pi * r * r * orc.profile(m, [r])[0][0],
                                0, rv, epsabs=0, epsrel=1e-10, limit=300)[0] / DA_c ** 2
    terms = a["Y"] * (w / DA_c) ** 2 * g.dtheta ** 2
    sem = terms.std() * math.sqrt(N)
    assert abs(est - ref) < 5 * sem
    assert abs(est / ref - 1) < 0.02


def test_sampled_pixels_from_the_prefiltered_particles(orc):
    """The geometric pre-filter keeps every particle that reaches a sampled pixel: the
    sampled pixels equal the full deposit there."""
    lc = I.lightcone(n_part=60000, n_halo=40, npix=96, side_deg=1.0, seed=21)
    g = orc.geom(96, 96, lc.geom.theta0_x, lc.geom.theta0_y, lc.geom.dtheta)
    mo = orc.solve_halos(lc.halos.M, lc.halos.c, lc.halos.z)
    a = orc.pp_assign(lc.parts, lc.Mp, lc.halos.pos, mo, g)
    yo, bo = orc.pp_deposit(a, g)
    rng = np.random.default_rng(1)
    pi_, pj_ = rng.integers(0, 96, 15), rng.integers(0, 96, 15)
    (yv, bv), m = orc.pp_pixels(lc.parts, lc.Mp, lc.halos.pos, mo, g, pi_, pj_)
    assert 0 < m < 60000
    np.testing.assert_allclose(yv, yo[pj_, pi_], rtol=1e-13, atol=1e-25)
    np.testing.assert_allclose(bv, bo[pj_, pi_], rtol=1e-12, atol=1e-22)


def test_hp_pixels_equal_the_map(orc):
    cat, _ = I.halo_catalog(n=30, npix=64, side_deg=0.4, seed=8)
    g = orc.geom(64, 64, -0.2 * math.pi / 180, -0.2 * math.pi / 180, 0.4 * math.pi / 180 / 64)
    mo = orc.solve_halos(cat.M, cat.c, cat.z)
    ym, bm = orc.hp_map(cat.thx, cat.thy, cat.vlos, mo, g, ap_r500=3.0, rtol=1e-8)
    rng = np.random.default_rng(3)
    pi_, pj_ = rng.integers(0, 64, 25), rng.integers(0, 64, 25)
    yv, bv = orc.hp_pixels(cat.thx, cat.thy, cat.vlos, mo, g, pi_, pj_, ap_r500=3.0, rtol=1e-8)
    np.testing.assert_allclose(yv, ym[0][pj_, pi_], rtol=1e-13, atol=1e-30)
    np.testing.assert_allclose(bv, bm[0][pj_, pi_], rtol=1e-13, atol=1e-30)


# ---------------------------------------------------------------- potential-based variant
def _halo_particle_phi(orc, lc, mo, r_of):
    """phi_i of every halo particle from the oracle's NFW potential at radius r_of(i) [Mpc]."""
    F = orc.F
    hid = lc.parts["hid"]
    phi = np.zeros(hid.size, np.float32)
    for k in np.unique(hid[hid >= 0]):
        sel = np.nonzero(hid == k)[0]
        _, _, p = orc.nfw_eval(lc.halos.M[k], lc.halos.c[k], lc.halos.z[k], r_of(sel, k))
        phi[sel] = p
    return phi


def test_potential_variant_reduces_to_the_spherical_model(orc):
    """phi_i = Phi_NFW(r_i) gives the spherical assignment (up to phi's FP32 rounding)."""
    lc = I.lightcone(n_part=20000, n_halo=40, npix=128, side_deg=1.0, seed=12)
    mo = orc.solve_halos(lc.halos.M, lc.halos.c, lc.halos.z)
    F = orc.F
    h = orc.cosmo_default().h
    pos = np.stack([lc.parts["x"], lc.parts["y"], lc.parts["z"]]).astype(np.float64)
    hp = lc.halos.pos.astype(np.float64)
    r_i = lambda sel, k: (np.linalg.norm(pos[:, sel] - hp[:, k:k + 1], axis=0) / h
                          / (1 + lc.halos.z[k]))
    phi = _halo_particle_phi(orc, lc, mo, r_i)
    g = orc.geom(lc.geom.nx, lc.geom.ny, lc.geom.theta0_x, lc.geom.theta0_y, lc.geom.dtheta)
    a = orc.pp_assign(lc.parts, lc.Mp, lc.halos.pos, mo, g)
    b = orc.pp_assign(lc.parts, lc.Mp, lc.halos.pos, mo, g, phi=phi)
    assert np.array_equal(a["kind"], b["kind"]) and np.count_nonzero(a["kind"] == 0) > 5000
    np.testing.assert_allclose(b["Y"], a["Y"], rtol=2e-6, atol=1e-6 * a["Y"].max())
    np.testing.assert_allclose(b["B"], a["B"], rtol=2e-6, atol=1e-6 * np.abs(a["B"]).max())
    assert np.array_equal(b["px"], a["px"]) and np.array_equal(b["hp"], a["hp"])


def test_potential_variant_is_polytropic_in_phi(orc):
    """For one particle, (Y / Y(Phi0))^(1/(n+1)) is affine in phi and 1 at Phi0, the density
    follows the same theta (B ratio = Y ratio^(n/(n+1))), and theta <= 0 gives nothing."""
    lc = I.lightcone(n_part=4000, n_halo=10, npix=64, side_deg=1.0, seed=13)
    mo = orc.solve_halos(lc.halos.M, lc.halos.c, lc.halos.z)
    F = orc.F
    g = orc.geom(lc.geom.nx, lc.geom.ny, lc.geom.theta0_x, lc.geom.theta0_y, lc.geom.dtheta)
    base = orc.pp_assign(lc.parts, lc.Mp, lc.halos.pos, mo, g)
    i = int(np.nonzero((base["kind"] == 0) & (base["Y"] > 0) & (base["B"] != 0))[0][0])
    k = lc.parts["hid"][i]
    one = {kk: v[i:i + 1] for kk, v in lc.parts.items()}
    phi0, T = mo[k, F["Phi0"]], mo[k, F["T"]]
    n = 1 / (1.2 - 1)
    vals = [phi0 + t * (n + 1) * T for t in (0.0, 0.2, 0.4, 0.6)]
    ys, bs = [], []
    for v in vals:
        r = orc.pp_assign(one, lc.Mp, lc.halos.pos, mo, g, phi=np.array([v], np.float32))
        ys.append(r["Y"][0])
        bs.append(r["B"][0])
    th = (np.array(ys) / ys[0]) ** (1 / (n + 1))
    assert th[0] == 1.0
    assert np.allclose(np.diff(th, 2), 0.0, atol=1e-6)  # affine in phi
    assert th[1] < 1.0  # a shallower potential makes the gas cooler
    assert np.allclose(np.array(bs) / bs[0], th ** n, rtol=1e-6)
    r = orc.pp_assign(one, lc.Mp, lc.halos.pos, mo, g,
                      phi=np.array([phi0 + 1.01 * (n + 1) * T], np.float32))
    assert r["Y"][0] == 0.0 and r["B"][0] == 0.0 and r["kind"][0] == 0


def test_pp_halo_ksz_is_volume_integral_of_electron_momentum(orc):
    """The halo-particle kSZ signal (Section 3.4, Eq. b_i^PP,h): for particles of one NFW halo
    at z = 1 moving with a common bulk velocity v along the line of sight, sum_i b_i Omega_pix
    must equal sigma_T (v/c) e^{-tau(z)} int n_e dV / D_A^2 over the sampled sphere, with
    n_e = rho_g / (mu_e m_p) of the solved gas profile (not the total density).  The radii
    are stratified in enclosed mass (midpoint rule in m, V_i = M_p / rho_NFW(r_i) its weight),
    so the sum is a quadrature accurate to ~1e-6; a dropped e^{-tau} (3e-3 here), the total
    density in place of the gas density, or a wrong sign of v_r fails it."""
    zh, v = 1.0, 500.0
    m = orc.solve_halos([2e14], [5.0], [zh])[0]
    F = orc.F
    N = 200000
    rv, c = m[F["r_vir"]], m[F["c"]]
    u = (np.arange(N) + 0.5) / N  # midpoints of equal-mass shells
    mc = math.log1p(c) - c / (1 + c)
    lo, hi = np.zeros(N), np.full(N, c)
    for _ in range(64):
        mid = 0.5 * (lo + hi)
        f = (np.log1p(mid) - mid / (1 + mid)) / mc - u
        lo, hi = np.where(f < 0, mid, lo), np.where(f < 0, hi, mid)
    r_phys = 0.5 * (lo + hi) / c * rv
    rng = np.random.default_rng(12)
    d = rng.normal(size=(N, 3))
    d /= np.linalg.norm(d, axis=1, keepdims=True)
    chi_h = orc.chi(zh) * 0.7  # comoving h^-1 Mpc
    hpos = np.array([[0.0], [0.0], [chi_h]], np.float32)
    off = d * (r_phys * (1 + zh) * 0.7)[:, None]
    zeros = np.zeros(N, np.float32)
    parts = {"x": off[:, 0].astype(np.float32), "y": off[:, 1].astype(np.float32),
             "z": (chi_h + off[:, 2]).astype(np.float32), "vx": zeros, "vy": zeros,
             "vz": np.full(N, v, np.float32), "hsml": np.full(N, 0.05, np.float32),
             "hid": np.zeros(N, np.int32)}
    Mp = 2e14 / N
    g = orc.geom(64, 64, -0.005, -0.005, 0.01 / 64)
    a = orc.pp_assign(parts, Mp, hpos, m[None, :], g)
    assert np.all(a["kind"] == 0)
    # undo the per-particle D_A (each particle is at its own distance)
    pos = np.stack([parts[k].astype(np.float64) for k in "xyz"]) / 0.7
    chi = np.linalg.norm(pos, axis=0)
    sel = np.argsort(chi)[:: N // 400]
    DA_tab = np.array([cc / (1 + orc.z_of_chi(cc)) for cc in chi[sel]])
    DA_i = np.interp(chi, chi[sel], DA_tab)
    DA_h = m[F["D_A"]]
    est = np.sum(a["B"] * (DA_i / DA_h) ** 2) * g.dtheta ** 2
    sigT, mp, MSUN, MPC = 6.6524587321e-29, 1.67262192369e-27, 1.98840987e30, \
        3.0856775814913673e22
    mu_e = 2.0 / (1.0 + 0.76)
    gas = quad(lambda r: 4 * math.pi * r * r * orc.profile(m, [r])[1][0], 0, rv,
               epsabs=0, epsrel=1e-11, limit=400)[0]  # Msun
    tau = orc.tau(zh)
    ref = sigT * (v / 299792.458) * math.exp(-tau) * gas * MSUN / (mu_e * mp) / (DA_h * MPC) ** 2
    tol = 2e-4
    assert 1.0 - math.exp(-tau) > 10 * tol  # the test resolves the optical-depth factor
    assert abs(est / ref - 1) < tol, (est, ref, est / ref - 1)
    # the same particles moving towards the observer give the opposite signal
    parts["vz"] = np.full(N, -v, np.float32)
    a2 = orc.pp_assign(parts, Mp, hpos, m[None, :], g)
    assert np.array_equal(a2["B"], -a["B"])

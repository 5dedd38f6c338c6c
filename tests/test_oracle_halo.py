"""Pins of the oracle's cosmology, NFW halo and ICM solve against closed forms,
textbook numbers and independent quadrature (scipy), never against itself.

Section 1 (cosmology), Section 2.1 (NFW, potential, polytrope), Section 2.2
(boundary conditions), Section 2.3 (non-thermal pressure), Table 1.
"""
import math
import os

import numpy as np
import pytest
from scipy.integrate import quad
from scipy.special import spence

G_SI, MSUN, MPC = 6.67430e-11, 1.98840987e30, 3.0856775814913673e22
G = G_SI * MSUN / (MPC * 1e6)  # Mpc (km/s)^2 / Msun
C_KMS = 299792.458
HERE = os.path.dirname(__file__)


def _cosmo(orc, Om=0.279, Ob=0.046, h=0.7):
    return orc.Cosmo(Om=Om, Ob=Ob, h=h, Tcmb=2.726, XH=0.76)


# ---------------------------------------------------------------- cosmology
def test_rho_crit_textbook(orc):
    # rho_cr,0 = 2.775e11 h^2 Msun/Mpc^3 (standard value)
    assert orc.rho_cr(0.0) / 0.7 ** 2 == pytest.approx(2.77536627e11, rel=2e-6)


def test_delta_vir_eds_limit(orc):
    # Omega_m(z) = 1 everywhere in Einstein-de Sitter: Delta = 18 pi^2
    cp = _cosmo(orc, Om=1.0)
    for z in (0.0, 1.0, 3.0):
        assert orc.delta_vir(z, cp) == pytest.approx(18 * math.pi ** 2, rel=1e-14)


def test_chi_tau_einstein_de_sitter(orc):
    # closed forms for Omega_m = 1: chi = 2c/H0 (1 - (1+z)^-1/2),
    # tau = sigma_T nbar_e c/H0 (2/3)[(1+z)^{3/2} - 1]
    cp = _cosmo(orc, Om=1.0)
    H0 = 70.0
    sigT, mp = 6.6524587321e-29, 1.67262192369e-27
    mu_e = 2.0 / 1.76
    rho0 = 3 * H0 ** 2 / (8 * math.pi * G) * MSUN / MPC ** 3
    ne = 0.046 * rho0 / (mu_e * mp)
    for z in (0.1, 1.0, 3.7):
        chi = 2 * C_KMS / H0 * (1 - (1 + z) ** -0.5)
        assert orc.chi(z, cp) == pytest.approx(chi, rel=1e-12)
        tau = sigT * ne * C_KMS / H0 * MPC * (2.0 / 3.0) * ((1 + z) ** 1.5 - 1)
        assert orc.tau(z, cp) == pytest.approx(tau, rel=1e-12)


def test_z_of_chi_inverts_chi(orc):
    for z in (0.01, 0.5, 1.5, 3.0):
        assert orc.z_of_chi(orc.chi(z)) == pytest.approx(z, rel=1e-12)


def test_geometry_numbers_printed_in_paper():
    vals = {}
    for line in open(os.path.join(HERE, "golden", "geometry.txt")):
        if line.strip() and not line.startswith("#"):
            k, v = line.split()
            vals[k] = float(v)
    pix = vals["flat_side_deg"] * 3600 / vals["flat_npix"]
    assert round(pix, 2) == vals["flat_pixel_arcsec"]
    area = 4 * math.pi / (12 * vals["healpix_nside"] ** 2) * (180 / math.pi * 60) ** 2
    assert round(area, 3) == vals["healpix_area_arcmin2"]
    assert round(math.sqrt(area) * 60, 1) == vals["healpix_side_arcsec"]


# ---------------------------------------------------------------- NFW
def test_m_of_c_closed_form_vs_quadrature(orc):
    for c in (1.0, 4.0, 12.0):
        ref, _ = quad(lambda x: x / (1 + x) ** 2, 0, c, epsabs=0, epsrel=1e-13)
        assert orc.m_of(c) == pytest.approx(ref, rel=1e-13)


def test_enclosed_mass_vs_density_quadrature(orc):
    M, c, z = 3e14, 4.5, 0.4
    m = orc.solve_halos([M], [c], [z])[0]
    rv = m[orc.F["r_vir"]]
    r = np.array([0.05, 0.3, 0.8, 1.0, 1.5]) * rv
    rho, Menc, phi = orc.nfw_eval(M, c, z, r)
    for ri, Mi in zip(r, Menc):
        f = lambda s: 4 * math.pi * s * s * orc.nfw_eval(M, c, z, [s])[0][0]
        ref = quad(f, 0, min(ri, rv), epsabs=0, epsrel=1e-12, limit=200)[0]
        assert Mi == pytest.approx(ref, rel=1e-11)
    assert Menc[-1] == pytest.approx(M / 0.7, rel=1e-14)  # all mass inside r_vir
    assert rho[-1] == 0.0  # truncated beyond r_vir


def test_potential_gradient_continuity_and_limits(orc):
    M, c, z = 1e14, 6.0, 0.2
    m = orc.solve_halos([M], [c], [z])[0]
    rv = m[orc.F["r_vir"]]
    for s in (0.02, 0.3, 0.7, 0.99, 1.3, 4.0):
        r = s * rv
        d = 1e-5 * r
        _, _, ph = orc.nfw_eval(M, c, z, [r - d, r + d])
        _, Me, _ = orc.nfw_eval(M, c, z, [r])
        dphi = (ph[1] - ph[0]) / (2 * d)
        assert dphi == pytest.approx(G * Me[0] / r ** 2, rel=1e-7)
    _, _, ph = orc.nfw_eval(M, c, z, [rv * (1 - 1e-12), rv * (1 + 1e-12)])
    assert ph[0] == pytest.approx(ph[1], rel=1e-10)
    _, _, ph = orc.nfw_eval(M, c, z, [1e6 * rv])
    assert ph[0] == pytest.approx(-G * (M / 0.7) / (1e6 * rv), rel=1e-12)
    _, _, ph = orc.nfw_eval(M, c, z, [1e-9 * rv])
    assert ph[0] == pytest.approx(m[orc.F["Phi0"]], rel=1e-8)


def _lokas_mamon_sigma2(s, c, Vv2):
    """Isotropic NFW dispersion, Lokas & Mamon (2001) eq. 14 with beta = 0, using
    Li2(-x) = spence(1 + x)."""
    g = 1 / (math.log1p(c) - c / (1 + c))
    cs = c * s
    br = (math.pi ** 2 - math.log(cs) - 1 / cs - 1 / (1 + cs) ** 2 - 6 / (1 + cs)
          + (1 + 1 / cs ** 2 - 4 / cs - 2 / (1 + cs)) * math.log1p(cs)
          + 3 * math.log1p(cs) ** 2 + 6 * spence(1 + cs))
    return 0.5 * c * c * g * s * (1 + cs) ** 2 * br * Vv2


def test_sigma2_matches_lokas_mamon_closed_form(orc):
    for M, c, z in ((1e14, 5.0, 0.3), (1e13, 9.0, 0.05), (1e15, 3.5, 1.0)):
        m = orc.solve_halos([M], [c], [z])[0]
        rv = m[orc.F["r_vir"]]
        Vv2 = G * m[orc.F["M"]] / rv
        for s in (0.01, 0.1, 0.5, 1.0, 1.7):
            assert orc.sigma2(M, c, z, s * rv) == pytest.approx(
                _lokas_mamon_sigma2(s, c, Vv2), rel=1e-9)


# ---------------------------------------------------------------- ICM solve
@pytest.fixture(scope="module")
def solved(orc):
    rng = np.random.default_rng(7)
    M = 10 ** rng.uniform(13, 15, 6)
    c = 5 * (M / 1e14) ** -0.1
    z = rng.uniform(0.05, 1.0, 6)
    return M, c, z, orc.solve_halos(M, c, z)


def _phi_numeric(orc, M, c, z, r):
    """Potential of the truncated profile from its definition -int_r^inf G M(<r')/r'^2,
    by scipy quadrature of the oracle's enclosed mass (itself pinned above)."""
    m = orc.solve_halos([M], [c], [z])[0]
    rv = m[orc.F["r_vir"]]
    Mv = m[orc.F["M"]]
    if r >= rv:
        return -G * Mv / r
    inner = quad(lambda s: G * orc.nfw_eval(M, c, z, [s])[1][0] / s ** 2, r, rv,
                 epsabs=0, epsrel=1e-12, limit=200)[0]
    return -G * Mv / rv - inner


def test_solution_satisfies_the_three_conditions(orc, solved):
    """Gas mass, surface pressure and energy conditions of Section 2.2, recomputed
    with scipy quadrature, the Lokas-Mamon dispersion and a numerically integrated
    potential; energy read as E_g,f = E_g,i + eps_DM|E_DM| + eps_* M_* c^2 + dE_p."""
    M, c, z, mod = solved
    F = orc.F
    fb = 0.046 / 0.279
    n = 1 / (1.2 - 1)
    for k in range(2):
        m = mod[k]
        rv, rs, rf = m[F["r_vir"]], m[F["r_s"]], m[F["r_f"]]
        Mv, T, rho0, P0 = m[F["M"]], m[F["T"]], m[F["rho0"]], m[F["P0"]]
        phi0 = _phi_numeric(orc, M[k], c[k], z[k], 1e-12 * rv)
        grid = np.concatenate([np.linspace(1e-9, rv, 400), np.linspace(rv, rf, 200)[1:]])
        phig = np.array([_phi_numeric(orc, M[k], c[k], z[k], r) for r in grid])
        from scipy.interpolate import CubicSpline
        sp_in = CubicSpline(grid[grid <= rv], phig[grid <= rv])
        phi = lambda r: sp_in(r) if r <= rv else -G * Mv / r
        theta = lambda r: 1 + (phi0 - phi(r)) / ((n + 1) * T)
        # gas mass
        gas = quad(lambda r: 4 * math.pi * r * r * rho0 * theta(r) ** n, 0, rf,
                   points=[rv] if rv < rf else None, epsrel=1e-10, limit=400)[0]
        assert (gas + m[F["M_star"]]) / (fb * Mv) == pytest.approx(1.0, abs=2e-7)
        # surface pressure
        Vv2 = G * Mv / rv
        rho_v = orc.nfw_eval(M[k], c[k], z[k], [rv * (1 - 1e-13)])[0][0]
        Ps = fb * rho_v * _lokas_mamon_sigma2(1.0, c[k], Vv2)
        assert P0 * theta(rf) ** (n + 1) == pytest.approx(Ps, rel=1e-7)
        # energy
        rstar = m[F["r_star"]]
        rho = lambda r: orc.nfw_eval(M[k], c[k], z[k], [r])[0][0]
        kin = quad(lambda r: 2 * math.pi * rho(r) * 3 * _lokas_mamon_sigma2(r / rv, c[k], Vv2)
                   * r * r, rstar, rv, epsrel=1e-10, limit=400)[0]
        pot = quad(lambda r: phi(r) * 4 * math.pi * r * r * rho(r), rstar, rv, epsrel=1e-10,
                   limit=400)[0]
        Egi = fb * (kin + pot)
        assert Egi == pytest.approx(m[F["E_gi"]], rel=1e-6)
        Egf = quad(lambda r: 4 * math.pi * (1.5 * P0 * theta(r) ** (n + 1)
                                            + rho0 * theta(r) ** n * phi(r)) * r * r,
                   0, rf, points=[rv] if rv < rf else None, epsrel=1e-10, limit=400)[0]
        dEp = 4 * math.pi / 3 * (rv ** 3 - rf ** 3) * Ps
        inj = 3.97e-6 * m[F["M_star"]] * C_KMS ** 2
        assert (Egf - (Egi + inj + dEp)) / abs(Egi) == pytest.approx(0.0, abs=2e-6)
        assert theta(rf) > 0


def test_solution_is_hydrostatic(orc, solved):
    """dP/dr = -rho_g dPhi/dr (Euler equation, Section 2.1) by finite differences."""
    M, c, z, mod = solved
    m = mod[0]
    F = orc.F
    rv, rf = m[F["r_vir"]], m[F["r_f"]]
    for s in (0.05, 0.4, 0.9, 1.02 if rf > 1.03 * rv else 0.95):
        r = s * rv
        d = 1e-5 * r
        _, rg, Pt = orc.profile(m, [r - d, r, r + d])
        _, _, ph = orc.nfw_eval(M[0], c[0], z[0], [r - d, r + d])
        dP = (Pt[2] - Pt[0]) / (2 * d)
        dphi = (ph[1] - ph[0]) / (2 * d)
        assert dP == pytest.approx(-rg[1] * dphi, rel=1e-6)


def test_r500_and_stellar_radius_definitions(orc, solved):
    M, c, z, mod = solved
    F = orc.F
    for k in range(len(M)):
        m = mod[k]
        r5 = m[F["r500"]]
        _, Me, _ = orc.nfw_eval(M[k], c[k], z[k], [r5])
        assert Me[0] / (4 * math.pi / 3 * r5 ** 3) == pytest.approx(500 * m[F["rho_cr"]],
                                                                    rel=1e-12)
        Fs = 0.026 * (m[F["M500"]] / 3e14) ** -0.12
        assert m[F["M_star"]] == pytest.approx(Fs * m[F["M"]], rel=1e-14)
        _, Ms, _ = orc.nfw_eval(M[k], c[k], z[k], [m[F["r_star"]]])
        assert 0.046 / 0.279 * Ms[0] == pytest.approx(m[F["M_star"]], rel=1e-12)


def test_energy_reading_gives_expanded_gas(orc, solved):
    """Section 2.2 states r_f is in general larger than r_vir (gas expands).  The
    reading final = initial + injection + surface work gives r_f >= r_vir for most
    of the c0 mass range; the printed arrangement gives r_f < r_vir."""
    M, c, z, mod = solved
    F = orc.F
    ratio = mod[:, F["r_f"]] / mod[:, F["r_vir"]]
    assert (mod[:, F["status"]] == 0).all()
    assert np.median(ratio) > 1.0
    printed = orc.solve_halos(M, c, z, ip=orc.icm_default(energy_sign=1))
    assert (printed[:, F["r_f"]] < printed[:, F["r_vir"]]).all()


def test_nonthermal_amplitude_limits(orc):
    """f(z) = min[(1+z)^beta, (f_max-1) tanh(beta z) + 1], f_max = 4^-n_nt/alpha_nt."""
    F = orc.F
    m0 = orc.solve_halos([1e14], [5.0], [1e-9])[0]
    assert m0[F["A_nt"]] == pytest.approx(0.18, rel=1e-8)
    mz = orc.solve_halos([1e14], [5.0], [40.0])[0]
    assert mz[F["A_nt"]] == pytest.approx(4 ** -0.8, rel=1e-6)


def test_electron_pressure_fraction(orc, solved):
    """P_e = (2X+2)/(5X+3) P_th with X = 0.76, i.e. 3.52/6.8, and R_nt cut-off."""
    _, _, _, mod = solved
    m = mod[1]
    F = orc.F
    r = np.array([0.01, 0.3, 0.9]) * m[F["r_vir"]]
    Pe, rg, Pt = orc.profile(m, r)
    Rnt = m[F["A_nt"]] * (r / m[F["r500"]]) ** 0.8
    np.testing.assert_allclose(Pe / (Pt * (1 - Rnt)), 3.52 / 6.8, rtol=1e-13)


def test_table1_defaults(orc):
    vals = {}
    for line in open(os.path.join(HERE, "golden", "table1.txt")):
        if line.strip() and not line.startswith("#"):
            k, v = line.split()
            vals[k] = float(v)
    ip = orc.icm_default()
    assert (ip.Gamma, ip.eps_dm, ip.eps_star, ip.f_star, ip.S_star, ip.alpha_nt, ip.beta_nt,
            ip.n_nt) == (vals["Gamma"], vals["eps_DM"], vals["eps_star"], vals["f_star"],
                         vals["S_star"], vals["alpha_nt"], vals["beta_nt"], vals["n_nt"])


def test_gauss_kronrod_rule_exactness():
    """The K15 nodes/weights in the oracle integrate degree-22 polynomials exactly and
    the embedded G7 rule degree-13 ones (pins the quadrature constants)."""
    src = open(os.path.join(os.path.dirname(HERE), "oracle", "bp_oracle.c")).read()
    import re

    def arr(name):
        body = re.search(name + r"\[\d+\] = \{([^}]*)\}", src).group(1)
        return np.array([float(t) for t in body.replace("\n", " ").split(",") if t.strip()])

    x, wk, wg = arr("GK_X"), arr("GK_WK"), arr("GK_WG")
    xs = np.concatenate([-x[:7], x[7:], x[:7][::-1]])
    ws = np.concatenate([wk[:7], wk[7:], wk[:7][::-1]])
    xg = np.concatenate([-x[1:7:2], [0.0], x[1:7:2][::-1]])
    wgs = np.concatenate([wg[:3], wg[3:], wg[:3][::-1]])
    for p in range(23):
        exact = 0.0 if p % 2 else 2.0 / (p + 1)
        assert np.dot(ws, xs ** p) == pytest.approx(exact, abs=1e-15)
        if p <= 13:
            assert np.dot(wgs, xg ** p) == pytest.approx(exact, abs=1e-15)

"""Pins of the oracle's temperature conversion (Section 3.2): Delta T_tSZ / T_CMB = g(x) y with
x = h nu / (k_B T_CMB), and Delta T_kSZ / T_CMB = -b.

g is pinned to the physics it comes from, not to its own formula: the non-relativistic
Kompaneets equation for scattering off hot electrons, dn/dy = x^-2 d/dx (x^4 dn/dx), applied
to the blackbody occupation n(x) = 1 / (e^x - 1) and expressed as a change of thermodynamic
temperature (dn = -x n'(x) dT/T), evaluated here by finite differences; plus its
Rayleigh-Jeans limit (-2) and the tabulated position of its null.
"""
import os

import numpy as np
import pytest
from scipy.optimize import brentq

HERE = os.path.dirname(__file__)
H_PLANCK, K_B = 6.62607015e-34, 1.380649e-23


def _x(nu_ghz, T=2.726):
    return H_PLANCK * nu_ghz * 1e9 / (K_B * T)


def _n(x):
    return 1.0 / np.expm1(x)


def _kompaneets_dt(x, h=2e-3):
    """(x^-2 d/dx (x^4 dn/dx)) / (-x dn/dx): the temperature change per unit y, from
    sixth-order central differences of the blackbody occupation."""
    def d1(f, t):
        return (f(t + 3 * h) - 9 * f(t + 2 * h) + 45 * f(t + h) - 45 * f(t - h)
                + 9 * f(t - 2 * h) - f(t - 3 * h)) / (60 * h)

    flux = lambda t: t ** 4 * d1(_n, t)
    return d1(flux, x) / x ** 2 / (-x * d1(_n, x))


@pytest.mark.parametrize("nu", [10.0, 30.0, 70.0, 100.0, 143.0, 217.0, 353.0, 545.0, 857.0])
def test_g_nu_is_the_kompaneets_temperature_change(orc, nu):
    x = _x(nu)
    ref = _kompaneets_dt(x)
    assert abs(orc.g_nu(nu) - ref) <= 2e-7 * max(1.0, abs(ref)), (orc.g_nu(nu), ref)


def test_g_nu_rayleigh_jeans_limit(orc):
    # Delta T / T -> -2 y at low frequency, approached as -2 + x^2 / 6
    for nu in (1e-3, 1e-2, 0.1):
        x = _x(nu)
        g = orc.g_nu(nu)
        assert abs(g + 2.0) < 1e-6
        assert abs((g + 2.0) / x ** 2 - 1.0 / 6.0) < 1e-3 or x < 1e-3


def test_g_nu_null_frequency(orc):
    rows = dict(l.split() for l in open(os.path.join(HERE, "golden", "tsz_null.txt"))
                if l.strip() and not l.startswith("#"))
    nu0 = brentq(orc.g_nu, 150.0, 300.0, xtol=1e-10)
    assert abs(_x(nu0) - float(rows["x0"])) < float(rows["x0_abs_tol"])
    # the null moves with T_CMB at fixed x: nu0 scales as T_CMB
    cp = orc.cosmo_default()
    cp.Tcmb = 2.0 * cp.Tcmb
    nu1 = brentq(lambda v: orc.g_nu(v, cp), 300.0, 600.0, xtol=1e-10)
    assert abs(nu1 / nu0 - 2.0) < 1e-9
    # decrement below the null, increment above
    assert orc.g_nu(nu0 - 20) < 0 < orc.g_nu(nu0 + 20)


def test_delta_t_maps(orc):
    rng = np.random.default_rng(3)
    y = rng.random((8, 9)) * 1e-6
    b = rng.normal(size=(8, 9)) * 1e-7
    ty, tb = orc.delta_t(y, b, 150.0)
    assert np.array_equal(tb, -b)
    np.testing.assert_allclose(ty, orc.g_nu(150.0) * y, rtol=0, atol=0)
    assert np.all(ty <= 0)  # a decrement at 150 GHz

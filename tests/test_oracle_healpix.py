"""Pins of the oracle's HEALPix pixelisation (RING ordering of Gorski et al. 2005) and of its
all-sky HP (Section 5.2): the 12 base pixels, the sphere's symmetries, equal-area quadrature
moments, the spacing of the centres, the great-circle angle, and the reduction of the sky HP
to the flat-sky line-of-sight integral and to the volume integral."""
import math

import numpy as np
import pytest
from scipy.integrate import quad

import oracle as orc


def _vec(th, ph):
    return np.stack([np.sin(th) * np.cos(ph), np.sin(th) * np.sin(ph), np.cos(th)], -1)


def test_base_pixels():
    # nside 1: four pixels around z = 2/3 and z = -2/3 at odd multiples of pi/4, four on the
    # equator at multiples of pi/2 (the published base-pixel layout)
    th, ph = orc.hpx_centres(1)
    z = np.cos(th)
    assert np.allclose(z, [2 / 3] * 4 + [0] * 4 + [-2 / 3] * 4, atol=1e-15)
    quarter = np.array([0.25, 0.75, 1.25, 1.75]) * math.pi
    assert np.allclose(ph, np.concatenate([quarter, np.arange(4) * math.pi / 2, quarter]),
                       atol=1e-15)


@pytest.mark.parametrize("nside", [2, 4, 8])
def test_sphere_symmetries_and_distinct_centres(nside):
    th, ph = orc.hpx_centres(nside)
    assert th.size == 12 * nside * nside
    key = lambda t, p: set(zip(np.round(np.cos(t), 12), np.round(np.mod(p, 2 * math.pi), 12)))
    pts = key(th, ph)
    assert len(pts) == th.size  # no duplicated centre
    assert key(math.pi - th, ph) == pts  # north-south mirror
    assert key(th, 2 * math.pi - ph) == pts  # east-west mirror
    assert key(th, ph + math.pi / 2) == pts  # quarter turn about the polar axis
    assert np.all(np.diff(np.cos(th)) <= 1e-15)  # RING order runs from north to south


@pytest.mark.parametrize("nside", [8, 16, 32])
def test_equal_area_quadrature_moments(nside):
    th, ph = orc.hpx_centres(nside)
    v = _vec(th, ph)
    assert np.abs(v.mean(0)).max() < 1e-13  # dipole vanishes
    err = abs((v[:, 2] ** 2).mean() - 1 / 3)  # <z^2> over the sphere is 1/3
    assert err < 1.0 / (16 * nside * nside)
    assert abs((v[:, 0] * v[:, 1]).mean()) < 1e-13
    th2, _ = orc.hpx_centres(2 * nside)
    err2 = abs((np.cos(th2) ** 2).mean() - 1 / 3)
    assert 3.2 < err / err2 < 4.8  # second-order convergence


def test_centre_spacing_and_coverage():
    nside = 8
    th, ph = orc.hpx_centres(nside)
    v = _vec(th, ph)
    size = math.sqrt(4 * math.pi / th.size)
    cosang = v @ v.T
    np.fill_diagonal(cosang, -2)
    nn = np.arccos(np.clip(cosang.max(1), -1, 1))
    assert nn.min() > 0.5 * size and nn.max() < 1.3 * size
    rng = np.random.default_rng(8)
    u = rng.normal(size=(4000, 3))
    u /= np.linalg.norm(u, axis=1, keepdims=True)
    far = np.arccos(np.clip((u @ v.T).max(1), -1, 1))
    assert far.max() < 1.0 * size  # no hole in the pixelisation


def test_great_circle_angle():
    h = math.pi / 2
    assert orc.sky_angle(h, 0.0, h, 0.3) == pytest.approx(0.3, rel=1e-15)
    assert orc.sky_angle(h, 1.0, h - 0.2, 1.0) == pytest.approx(0.2, rel=1e-15)
    assert orc.sky_angle(0.01, 0.0, 0.01, math.pi) == pytest.approx(0.02, rel=1e-14)
    assert orc.sky_angle(0.3, 0.2, math.pi - 0.3, 0.2 + math.pi) == pytest.approx(math.pi)
    assert orc.sky_angle(1.0, 2.0, 1.0, 2.0 + 1e-9) == pytest.approx(1e-9 * math.sin(1.0),
                                                                      rel=1e-7)
    rng = np.random.default_rng(9)
    for _ in range(20):
        t1, t2 = rng.uniform(0, math.pi, 2)
        p1, p2, a = rng.uniform(0, 2 * math.pi, 3)
        ref = math.acos(np.clip(_vec(t1, p1) @ _vec(t2, p2), -1, 1))
        assert orc.sky_angle(t1, p1, t2, p2) == pytest.approx(ref, abs=1e-7)
        assert orc.sky_angle(t1, p1 + a, t2, p2 + a) == pytest.approx(
            orc.sky_angle(t1, p1, t2, p2), abs=1e-13)


@pytest.fixture(scope="module")
def one_halo():
    return orc.solve_halos([2e14], [4.0], [0.25])[0]


def test_sky_hp_is_the_line_of_sight_integral_at_the_sky_angle(one_halo):
    m = one_halo
    F = orc.F
    rf, DA = m[F["r_f"]], m[F["D_A"]]
    v = 400.0
    bfac = orc.const_CN() * (v / 299792.458) * math.exp(-m[F["tau"]])
    offs = np.array([0.0, 0.05, 0.3, 0.7, 0.95]) * rf / DA
    h = math.pi / 2
    # along the equator and along a meridian from a halo on the equator; and across the pole
    cases = [(np.full(offs.size, h), offs, h, 0.0, offs),
             (h - offs, np.zeros(offs.size), h, 0.0, offs),
             (np.full(offs.size, 0.5 * offs[-1]), np.full(offs.size, math.pi), 0.5 * offs[-1],
              0.0, np.full(offs.size, offs[-1]))]
    for pt, pp, ht, hph, ang in cases:
        y, b = orc.hp_sky([ht], [hph], [v], m[None, :], pt, pp, rtol=1e-10)
        for k in range(offs.size):
            assert y[k] == pytest.approx(orc.const_CP() * orc.los_integral(m, DA * ang[k], 0,
                                                                           rtol=1e-10), rel=1e-9)
            assert b[k] == pytest.approx(bfac * orc.los_integral(m, DA * ang[k], 1, rtol=1e-10),
                                         rel=1e-9)
    # outside the aperture: nothing
    y, b = orc.hp_sky([h], [0.0], [v], m[None, :], [h], [1.01 * rf / DA])
    assert y[0] == 0.0 and b[0] == 0.0


def test_sky_map_integral_equals_volume_integral(one_halo):
    """sum_pix y Omega_pix = sigma_T/(m_e c^2) int P_e dV / D_A^2 on a fine HEALPix grid
    around a halo near the north pole."""
    m = one_halo
    F = orc.F
    rf, DA = m[F["r_f"]], m[F["D_A"]]
    ang = rf / DA
    nside = 32768
    ht = 0.02
    # RING order runs north to south: the pixels with colatitude below ht + 1.2 ang
    lo, hi = 0, 12 * nside * nside - 1
    while lo < hi:
        mid = (lo + hi + 1) // 2
        if orc.hpx_centres(nside, [mid])[0][0] < ht + 1.2 * ang:
            lo = mid
        else:
            hi = mid - 1
    pt, pp = orc.hpx_centres(nside, np.arange(lo + 1))
    y, b = orc.hp_sky([ht], [1.0], [500.0], m[None, :], pt, pp, rtol=1e-9)
    omega = 4 * math.pi / (12 * nside * nside)
    vol = quad(lambda r: 4 * math.pi * r * r * orc.profile(m, [r])[0][0], 0, rf,
               points=[m[F["r_vir"]]], epsabs=0, epsrel=1e-11, limit=400)[0]
    assert np.count_nonzero(y) > 8000
    assert y.sum() * omega == pytest.approx(orc.const_CP() * vol / DA ** 2, rel=3e-3)

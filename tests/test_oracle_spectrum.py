"""Pins of the oracle's flat-sky power spectrum (Section 5.3): a single Fourier mode's power
in closed form, Parseval's theorem, the white-noise level, and invariance under shifts and
transposition of the map."""
import math

import numpy as np
import pytest

import oracle as orc


def test_single_cosine_mode():
    nx, ny, d, A, m = 64, 32, 1e-3, 2.5, 5
    x = np.arange(nx)
    f = np.tile(A * np.cos(2 * math.pi * m * x / nx), (ny, 1))
    lm = 2 * math.pi * m / (nx * d)
    edges = np.array([0.5, 0.9, 1.1, 3.0]) * lm
    cl, cnt = orc.power_spectrum(f, d, edges)
    # F(+-m, 0) = A nx ny / 2: two modes of C = d^2 (A nx ny / 2)^2 / (nx ny) in bin 1
    per_mode = d * d * (A * nx * ny / 2) ** 2 / (nx * ny)
    assert cl[1] == pytest.approx(2 * per_mode / cnt[1], rel=1e-12)
    assert abs(cl[0]) < 1e-20 * per_mode and abs(cl[2]) < 1e-20 * per_mode
    assert cnt[1] >= 2 and cnt.sum() < nx * ny


def test_parseval_and_all_modes():
    rng = np.random.default_rng(1)
    nx, ny, d = 32, 64, 2e-4
    f = rng.normal(size=(ny, nx))
    lmax = 2 * math.pi * math.hypot(nx / 2, ny / 2) / (min(nx, ny) * d) * 2
    cl, cnt = orc.power_spectrum(f, d, [0.0, lmax])
    assert cnt[0] == nx * ny
    # sum |F|^2 = N sum f^2 -> mean C = d^2 sum f^2 / N
    assert cl[0] == pytest.approx(d * d * (f * f).sum() / (nx * ny), rel=1e-12)


def test_white_noise_level():
    rng = np.random.default_rng(2)
    n, d, sigma = 512, 1e-4, 3.0
    f = rng.normal(0.0, sigma, size=(n, n))
    edges = np.geomspace(2 * math.pi / (n * d) * 4, 2 * math.pi / (n * d) * n / 2, 9)
    cl, cnt = orc.power_spectrum(f, d, edges)
    expect = sigma * sigma * d * d
    for k in range(cl.size):  # mean of cnt exponential-like variates (2 dof each, paired modes)
        assert abs(cl[k] / expect - 1) < 6 * math.sqrt(2.0 / cnt[k])


def test_shift_and_transpose_invariance():
    rng = np.random.default_rng(3)
    n, d = 128, 3e-4
    f = rng.normal(size=(n, n)) + np.outer(np.sin(np.arange(n) / 7), np.cos(np.arange(n) / 3))
    edges = np.geomspace(2 * math.pi / (n * d), 2 * math.pi / (n * d) * n, 12)
    cl, cnt = orc.power_spectrum(f, d, edges)
    cl2, cnt2 = orc.power_spectrum(np.roll(f, (17, -40), axis=(0, 1)), d, edges)
    cl3, cnt3 = orc.power_spectrum(f.T, d, edges)
    assert np.array_equal(cnt, cnt2) and np.array_equal(cnt, cnt3)
    assert np.allclose(cl2, cl, rtol=1e-11) and np.allclose(cl3, cl, rtol=1e-11)

"""Pins of the oracle's smoothing lengths (Section 3.4: h_i such that the effective number of
neighbours (4 pi / 3) h^3 sum_j W(r_ij, h) = (32/3) sum_j w(r_ij / h), with the cubic spline
of Eq. SPH_kernel, equals N_ngb), against closed forms and the continuum limit."""
import numpy as np
import pytest

import oracle as orc


def _pair(n_ngb, d=1.0):
    x = np.array([0.0, d], np.float32)
    zero = np.zeros(2, np.float32)
    return orc.smoothing_lengths(x, zero, zero, n_ngb)


def test_kernel_pieces_and_support():
    assert orc.w3(0.0) == 1.0 and orc.w3(0.5) == pytest.approx(0.25)
    assert orc.w3(0.75) == pytest.approx(2 * 0.25 ** 3)
    assert orc.w3(1.0) == 0.0 and orc.w3(2.0) == 0.0


def test_two_particles_inner_piece():
    # (32/3) (w(0) + w(d/h)) = 16  ->  1 - 6x^2 + 6x^3 = 1/2 with x = d/h < 1/2
    roots = np.roots([6.0, -6.0, 0.0, 0.5])
    x = [r.real for r in roots if abs(r.imag) < 1e-12 and 0 < r.real < 0.5][0]
    h = _pair(16.0, d=1.0)
    assert h == pytest.approx([1.0 / x, 1.0 / x], rel=1e-12)


def test_two_particles_outer_piece():
    # x = 3/4: w = 2 (1/4)^3 = 1/32, so N = (32/3)(1 + 1/32) = 11 exactly
    h = _pair(11.0, d=3.0)
    assert h == pytest.approx([4.0, 4.0], rel=1e-12)


def test_lattice_interior_approaches_the_continuum():
    # unit cubic lattice: n = 1, (4 pi / 3) h^3 = N_ngb in the continuum limit
    g = np.arange(11, dtype=np.float32) - 5
    X, Y, Z = np.meshgrid(g, g, g, indexing="ij")
    c = X.size // 2
    for n_ngb, tol in ((64.0, 2e-3), (256.0, 2e-4)):
        h = orc.smoothing_lengths(X.ravel(), Y.ravel(), Z.ravel(), n_ngb)[c]
        assert h == pytest.approx((3 * n_ngb / (4 * np.pi)) ** (1 / 3), rel=tol)


def test_scaling_translation_and_permutation():
    rng = np.random.default_rng(3)
    p = rng.integers(-40, 40, (3, 600)).astype(np.float32)  # integer coordinates: exact
    h = orc.smoothing_lengths(*p, 32.0)
    assert np.allclose(orc.smoothing_lengths(*(4 * p), 32.0), 4 * h, rtol=1e-12)
    assert np.allclose(orc.smoothing_lengths(*(p + 1000), 32.0), h, rtol=1e-12)
    perm = rng.permutation(600)
    assert np.allclose(orc.smoothing_lengths(*p[:, perm], 32.0), h[perm], rtol=1e-12)


def test_neighbours_shrink_h_and_too_few_particles_give_inf():
    rng = np.random.default_rng(4)
    p = rng.uniform(0, 10, (3, 300)).astype(np.float32)
    h = orc.smoothing_lengths(*p, 32.0)
    extra = np.concatenate([p, p[:, :1] + 0.01], axis=1)
    assert orc.smoothing_lengths(*extra, 32.0)[0] <= h[0]
    # 5 particles: N_eff <= (32/3) 5 < 64
    q = rng.uniform(0, 1, (3, 5)).astype(np.float32)
    assert np.all(np.isinf(orc.smoothing_lengths(*q, 64.0)))


def test_sampled_particles_match_the_full_solve():
    rng = np.random.default_rng(5)
    p = rng.normal(0, 1, (3, 400)).astype(np.float32)
    idx = np.array([0, 17, 399, 17])
    assert np.array_equal(orc.smoothing_lengths_at(*p, idx, 40.0),
                          orc.smoothing_lengths(*p, 40.0)[idx])

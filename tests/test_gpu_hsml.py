"""Parity of the CUDA smoothing lengths (Section 3.4: h_i with N_eff(h_i) = (32/3) sum_j
w(|r_i - r_j| / h_i) = N_ngb, the cubic spline of Eq. SPH_kernel) with the oracle's
brute-force bisection over the distances to every particle.

Tolerance: the kernel sums at most 2048 FP32 weights per evaluation (relative error of N_eff
below ~1e-6) and stops Newton at a 2e-7 relative step; N_eff grows like h^3, so h is off
by about a third of N_eff's error.  1e-5 relative leaves an order of magnitude."""
import numpy as np
import pytest
import torch

from paper_2201_02632_gb300 import inputs as I
from tests.gpu_common import api, ctx, cuda  # noqa: F401

pytestmark = pytest.mark.gpu
RTOL = 1e-5


def _gpu(ctx, p, n_ngb, guess=None):
    h = ctx.smoothing_lengths(cuda(p[0]), cuda(p[1]), cuda(p[2]), n_ngb,
                              guess=None if guess is None else cuda(guess, torch.float32))
    return h.double().cpu().numpy()


def _cone_positions(n, seed, n_halo=40):
    lc = I.lightcone(n_part=n, n_halo=n_halo, side_deg=1.0, zr=(0.05, 0.5), seed=seed)
    return np.stack([lc.parts["x"], lc.parts["y"], lc.parts["z"]])


@pytest.mark.parametrize("n_ngb", [32.0, 64.0])
def test_clustered_light_cone_particles(orc, api, ctx, n_ngb):
    p = _cone_positions(8000, seed=I.SEED_BASE + 70)
    h = _gpu(ctx, p, n_ngb)
    np.testing.assert_allclose(h, orc.smoothing_lengths(*p, n_ngb), rtol=RTOL)


@pytest.mark.parametrize("n_ngb", [40.0, 200.0, 1024.0])
def test_uniform_box_ragged_count(orc, api, ctx, n_ngb):
    rng = np.random.default_rng(I.SEED_BASE + 71)
    p = rng.uniform(-3.0, 5.0, (3, 5003)).astype(np.float32)
    np.testing.assert_allclose(_gpu(ctx, p, n_ngb), orc.smoothing_lengths(*p, n_ngb), rtol=RTOL)


def test_flat_sheet_and_line(orc, api, ctx):
    rng = np.random.default_rng(I.SEED_BASE + 72)
    sheet = rng.uniform(0.0, 1.0, (3, 3000)).astype(np.float32)
    sheet[2] = 0.25
    np.testing.assert_allclose(_gpu(ctx, sheet, 48.0), orc.smoothing_lengths(*sheet, 48.0),
                               rtol=RTOL)
    line = np.zeros((3, 700), np.float32)
    line[0] = rng.uniform(10.0, 20.0, 700)
    np.testing.assert_allclose(_gpu(ctx, line, 20.0), orc.smoothing_lengths(*line, 20.0),
                               rtol=RTOL)


def test_two_particles_closed_form(api, ctx):
    # (32/3)(w(0) + w(d/h)) = 16 -> 6x^3 - 6x^2 + 1/2 = 0, x = d/h in (0, 1/2)
    roots = np.roots([6.0, -6.0, 0.0, 0.5])
    x = [r.real for r in roots if abs(r.imag) < 1e-12 and 0 < r.real < 0.5][0]
    p = np.array([[100.0, 101.0], [-7.0, -7.0], [3.0, 3.0]], np.float32)
    np.testing.assert_allclose(_gpu(ctx, p, 16.0), [1.0 / x] * 2, rtol=1e-6)


def test_starting_guesses(orc, api, ctx):
    rng = np.random.default_rng(I.SEED_BASE + 73)
    p = _cone_positions(6000, seed=I.SEED_BASE + 74, n_halo=25)
    ho = orc.smoothing_lengths(*p, 64.0)
    guess = ho * rng.uniform(0.3, 3.0, ho.size)
    guess[::7] = np.nan  # no guess: the grid density is used
    guess[3::7] = -1.0
    np.testing.assert_allclose(_gpu(ctx, p, 64.0, guess=guess), ho, rtol=RTOL)


def test_deterministic(api, ctx):
    p = _cone_positions(6000, seed=I.SEED_BASE + 75, n_halo=25)
    a = _gpu(ctx, p, 64.0)
    b = _gpu(ctx, p, 64.0)
    assert np.array_equal(a, b)


def test_errors_and_empty_input(api, ctx):
    e = torch.empty(0, device="cuda")
    assert ctx.smoothing_lengths(e, e, e).numel() == 0
    rng = np.random.default_rng(I.SEED_BASE + 76)
    p = rng.uniform(0.0, 1.0, (3, 200)).astype(np.float32)
    for bad in (10.0, 2000.0):
        with pytest.raises(api.BpError) as err:
            _gpu(ctx, p, bad)
        assert "BP_EINVAL" in str(err.value)
    with pytest.raises(api.BpError) as err:
        _gpu(ctx, p[:, :5], 64.0)  # (32/3) 5 < 64
    assert "BP_ERANGE" in str(err.value)
    q = p.copy()
    q[1, 17] = np.inf
    with pytest.raises(api.BpError) as err:
        _gpu(ctx, q, 32.0)
    assert "BP_EINVAL" in str(err.value)


def test_full_light_cone_sampled(orc, api, ctx):
    """The 4M-particle light-cone of the 2-degree pasting workload; the oracle at sampled
    particles (the smallest and largest h among them)."""
    lc = I.lightcone()
    p = np.stack([lc.parts["x"], lc.parts["y"], lc.parts["z"]])
    h = _gpu(ctx, p, 64.0)
    assert np.all(np.isfinite(h)) and np.all(h > 0)
    rng = np.random.default_rng(I.SEED_BASE + 77)
    idx = np.concatenate([rng.choice(h.size, 40, replace=False), [h.argmin(), h.argmax()]])
    np.testing.assert_allclose(h[idx], orc.smoothing_lengths_at(*p, idx, 64.0), rtol=RTOL)

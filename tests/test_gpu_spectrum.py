"""Parity of the CUDA flat-sky power spectrum (Section 5.3: FFT of the map, multipole bins)
with the oracle's numpy FFT.  Both sides are FP64 and decide each mode's bin with the same
rounded |l|^2, so the mode counts agree exactly and the binned C_l to rounding (1e-9 of a
bin's value, for bins above 1e-12 of the largest)."""
import math

import numpy as np
import pytest
import torch

from paper_2201_02632_gb300 import inputs as I
from tests.gpu_common import api, ctx, cuda, folded, gpu_geom  # noqa: F401

pytestmark = pytest.mark.gpu


def _check(orc, api, ctx, m, d, edges=None, lo=None):
    e = api.default_ell_edges() if edges is None else np.asarray(edges, np.float64)
    _, cl, nm = ctx.power_spectrum(cuda(m.astype(np.float32)), d, e,
                                   lo=None if lo is None else cuda(lo.astype(np.float32)))
    ref = m.astype(np.float32).astype(np.float64)
    if lo is not None:
        ref = ref + lo.astype(np.float32).astype(np.float64)
    clo, cnto = orc.power_spectrum(ref, d, e)
    assert np.array_equal(nm.cpu().numpy(), cnto)
    cl = cl.cpu().numpy()
    big = clo > 1e-12 * clo.max()
    np.testing.assert_allclose(cl[big], clo[big], rtol=1e-9)
    assert np.all(np.abs(cl[~big]) <= 1e-11 * clo.max())
    return cl, cnto


def test_white_noise_and_custom_edges(orc, api, ctx):
    rng = np.random.default_rng(I.SEED_BASE + 90)
    n, d = 512, 1e-4
    m = rng.normal(0.0, 2.0, (n, n))
    edges = np.geomspace(2 * math.pi / (n * d), 2 * math.pi / d, 41)
    cl, cnt = _check(orc, api, ctx, m, d, edges)
    assert cnt.sum() > 0.7 * n * n


def test_pasted_hp_map_default_bins(orc, api, ctx):
    cat, g = I.halo_catalog(n=120, npix=256)
    model, status = ctx.solve_halos(cuda(cat.M), cuda(cat.c), cuda(cat.z))
    gg = gpu_geom(api, g)
    maps = api.Maps.zeros(gg)
    ctx.paste_halos(cuda(cat.thx), cuda(cat.thy), cuda(cat.vlos), model, status, gg, maps,
                    ap_r500=3.0)
    y = maps.y[0].cpu().numpy()
    ylo = maps.ylo[0].cpu().numpy()
    _check(orc, api, ctx, y, g.dtheta, lo=ylo)
    _check(orc, api, ctx, maps.b[0].cpu().numpy(), g.dtheta)


@pytest.mark.parametrize("nx,ny", [(1024, 256), (2, 64), (4096, 4096)])
def test_shapes(orc, api, ctx, nx, ny):
    rng = np.random.default_rng(I.SEED_BASE + 91)
    d = 5e-5
    yy, xx = np.mgrid[0:ny, 0:nx]
    m = rng.normal(size=(ny, nx)) + 10 * np.sin(2 * math.pi * 3 * xx / nx) * np.cos(
        2 * math.pi * 5 * yy / ny)
    edges = np.geomspace(2 * math.pi / (max(nx, ny) * d), 2 * math.pi / d, 31)
    _check(orc, api, ctx, m, d, edges)


def test_errors(api, ctx):
    m = torch.zeros((100, 128), device="cuda")
    with pytest.raises(api.BpError) as e:
        ctx.power_spectrum(m, 1e-4)
    assert "BP_EINVAL" in str(e.value)
    m = torch.zeros((128, 128), device="cuda")
    with pytest.raises(api.BpError) as e:
        ctx.power_spectrum(m, 1e-4, edges=[1.0, 1.0, 2.0])
    assert "BP_EINVAL" in str(e.value)

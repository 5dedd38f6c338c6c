"""Parity of the CUDA halo-based pasting (Section 3.3, Eqs. y^HP and b^HP) with the
oracle's adaptive line-of-sight integrals at pixel centres."""
import numpy as np
import pytest
import torch

from paper_2201_02632_gb300 import inputs as I
from tests.gpu_common import api, ctx, cuda, folded, gpu_geom, orc_geom  # noqa: F401
from tests.helpers import assert_map_parity

pytestmark = pytest.mark.gpu


def _run(orc, api, ctx, cat, g, ap, map_id=None, tile=32):
    ctx.set_tiling(hp_tile=tile)
    model, status = ctx.solve_halos(cuda(cat.M), cuda(cat.c), cuda(cat.z))
    gg = gpu_geom(api, g)
    maps = api.Maps.zeros(gg)
    mid = None if map_id is None else cuda(map_id)
    ctx.paste_halos(cuda(cat.thx), cuda(cat.thy), cuda(cat.vlos), model, status, gg, maps,
                    ap_r500=ap, map_id=mid)
    y, b = folded(maps)
    mo = orc.solve_halos(cat.M, cat.c, cat.z)
    yo, bo = orc.hp_map(cat.thx, cat.thy, cat.vlos, mo, orc_geom(orc, g), ap_r500=ap,
                        map_id=map_id, rtol=1e-9)
    return y, b, yo, bo


@pytest.mark.parametrize("tile", [32, 64])
def test_hp_c0_shaped_matches_oracle(orc, api, ctx, tile):
    cat, g = I.halo_catalog(n=120, npix=256)
    y, b, yo, bo = _run(orc, api, ctx, cat, g, 3.0, tile=tile)
    assert_map_parity(y[0], yo[0], what="y")
    assert_map_parity(b[0], bo[0], what="b")


def test_hp_full_aperture_ragged_map(orc, api, ctx):
    cat, g = I.halo_catalog(n=60, npix=150, side_deg=0.6, seed=31)
    y, b, yo, bo = _run(orc, api, ctx, cat, g, 0.0)
    assert_map_parity(y[0], yo[0], what="y")
    assert_map_parity(b[0], bo[0], what="b")


def test_hp_many_maps(orc, api, ctx):
    cat, g = I.halo_catalog(n=90, npix=96, side_deg=0.5, seed=41)
    map_id = (np.arange(90) % 3).astype(np.int32)
    g.n_maps = 3
    y, b, yo, bo = _run(orc, api, ctx, cat, g, 0.0, map_id=map_id)
    for m in range(3):
        assert_map_parity(y[m], yo[m], what=f"y map {m}")
        assert_map_parity(b[m], bo[m], what=f"b map {m}")

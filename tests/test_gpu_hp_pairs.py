"""Bit-exact (map, tile, halo) membership of the halo paste (Section 3.3: a halo adds to
the pixel centres inside its aperture, so its work list holds every tile that the FP64
pixel-centre bounding box of the aperture disc touches).  The GPU list (bp_hp_pairs) and
the oracle's list (orc_hp_pairs) are built from the same solved models, the oracle's, so
keys, order and halo indices must agree exactly."""
import numpy as np
import pytest

from paper_2201_02632_gb300 import inputs as I
from tests.gpu_common import api, ctx, cuda, gpu_geom, gpu_model_from_oracle, orc_geom  # noqa: F401

pytestmark = pytest.mark.gpu


def _compare(orc, api, ctx, cat, g, ap, tile, map_id=None, mo=None, status_override=None):
    if mo is None:
        mo = orc.solve_halos(cat.M, cat.c, cat.z)
    if status_override is not None:
        mo = mo.copy()
        mo[:, orc.F["status"]] = status_override
    model, status = gpu_model_from_oracle(api, mo)
    gg = gpu_geom(api, g)
    mid = None if map_id is None else cuda(map_id)
    k, v = ctx.hp_pairs(cuda(cat.thx), cuda(cat.thy), model, status, gg, tile, ap_r500=ap,
                        map_id=mid)
    ko, vo = orc.hp_pairs(cat.thx, cat.thy, mo, orc_geom(orc, g), ap, tile, tile, map_id=map_id)
    kg = k.cpu().numpy().view(np.uint32)
    vg = v.cpu().numpy().view(np.uint32)
    assert kg.size == ko.size, f"pair count {kg.size} vs oracle {ko.size}"
    assert np.array_equal(kg, ko), "tile keys differ"
    assert np.array_equal(vg, vo), "halo membership / order differs"
    return kg.size, mo


@pytest.mark.parametrize("tile", [32, 64])
def test_hp_pairs_catalogue_1000_halos_256(orc, api, ctx, tile):
    # 1000 halos on a 1x1 deg^2 256^2 map, aperture min(r_f, 3 r500)
    cat, g = I.halo_catalog(n=1000, npix=256)
    n, _ = _compare(orc, api, ctx, cat, g, 3.0, tile)
    assert n > 1000


@pytest.mark.parametrize("tile", [32, 64])
def test_hp_pairs_batched_maps_full_aperture(orc, api, ctx, tile):
    # several maps, uneven extents (power-law masses 1e12-1e15, z 0.01-3), r_ap = r_f; a
    # ragged map side (300 px) and half of each map's halos off-centre so that apertures
    # cross the edges or miss the map
    cat, g = I.batched_catalog(n_maps=3, mean_halos=400, npix=300, side_deg=2.0, seed=77)
    g.theta0_x += 0.25 * g.nx * g.dtheta
    n, _ = _compare(orc, api, ctx, cat, g, 0.0, tile, map_id=cat.map_id)
    assert n > 0


def test_hp_pairs_excludes_bad_status_and_map_id(orc, api, ctx):
    cat, g = I.halo_catalog(n=200, npix=128, seed=5)
    mo = orc.solve_halos(cat.M, cat.c, cat.z)
    st = np.zeros(200, np.float64)
    st[::7] = 1.0  # no bracket: no pairs
    map_id = np.zeros(200, np.int32)
    map_id[::11] = 3  # outside [0, n_maps): no pairs
    map_id[::13] = -1
    n, _ = _compare(orc, api, ctx, cat, g, 3.0, 32, map_id=map_id, mo=mo, status_override=st)
    n_all, _ = _compare(orc, api, ctx, cat, g, 3.0, 32, mo=mo)
    assert 0 < n < n_all


def test_hp_pairs_empty_and_off_map(orc, api, ctx):
    cat, g = I.halo_catalog(n=50, npix=64, seed=9)
    g.theta0_x += 10.0 * g.nx * g.dtheta  # every halo far to the left of the map
    n, _ = _compare(orc, api, ctx, cat, g, 0.0, 64)
    assert n == 0
    gg = gpu_geom(api, g)
    e = cuda(np.zeros(0))
    k, v = ctx.hp_pairs(e, e, cuda(np.zeros((len(api.MODEL_FIELDS), 0))),
                        cuda(np.zeros(0, np.int32)), gg, 32)
    assert k.numel() == 0 and v.numel() == 0

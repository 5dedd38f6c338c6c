"""Parity of bp_finalize_map (Section 3.2) with the oracle: folding of the compensation planes
and the conversion of y and b maps to Delta T / T_CMB = g(x) y and -b."""
import numpy as np
import pytest
import torch

from paper_2201_02632_gb300 import inputs as I
from tests.gpu_common import api, ctx, cuda, gpu_geom, orc_geom  # noqa: F401
from tests.helpers import assert_map_parity

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def pasted(orc, api):
    """An HP map pair of 120 halos (1x1 deg^2, 256^2, aperture 3 r500), GPU and oracle."""
    cat, g = I.halo_catalog(n=120, npix=256)
    c = api.Context()
    model, status = c.solve_halos(cuda(cat.M), cuda(cat.c), cuda(cat.z))
    gg = gpu_geom(api, g)
    maps = api.Maps.zeros(gg)
    c.paste_halos(cuda(cat.thx), cuda(cat.thy), cuda(cat.vlos), model, status, gg, maps,
                  ap_r500=3.0)
    torch.cuda.synchronize()
    c.close()
    mo = orc.solve_halos(cat.M, cat.c, cat.z)
    yo, bo = orc.hp_map(cat.thx, cat.thy, cat.vlos, mo, orc_geom(orc, g), ap_r500=3.0, rtol=1e-9)
    return gg, maps, yo[0], bo[0]


def _copy(api, gg, maps):
    m = api.Maps.zeros(gg)
    for a, b in ((m.y, maps.y), (m.b, maps.b), (m.ylo, maps.ylo), (m.blo, maps.blo)):
        a.copy_(b)
    return m


@pytest.mark.parametrize("nu", [30.0, 150.0, 217.0, 353.0, 857.0])
def test_delta_t_matches_oracle(orc, api, ctx, pasted, nu):
    gg, maps, yo, bo = pasted
    m = _copy(api, gg, maps)
    ctx.finalize(gg, m, out_kind=api.OUT_DT, nu_ghz=nu)
    ty, tb = orc.delta_t(yo, bo, nu)
    y = m.y[0].double().cpu().numpy()
    b = m.b[0].double().cpu().numpy()
    assert_map_parity(y, ty, what=f"Delta T tSZ at {nu} GHz")
    assert_map_parity(b, tb, what="Delta T kSZ")
    assert not m.ylo.any() and not m.blo.any()  # the compensation planes are folded


def test_delta_t_kinetic_is_minus_folded_b(api, ctx, pasted):
    gg, maps, _, _ = pasted
    m1, m2 = _copy(api, gg, maps), _copy(api, gg, maps)
    ctx.finalize(gg, m1)
    ctx.finalize(gg, m2, out_kind=api.OUT_DT, nu_ghz=150.0)
    assert torch.equal(m2.b, -m1.b)


def test_finalize_rejects_bad_frequency_and_kind(api, ctx, pasted):
    gg, maps, _, _ = pasted
    m = _copy(api, gg, maps)
    for kw in ({"out_kind": api.OUT_DT, "nu_ghz": 0.0}, {"out_kind": api.OUT_DT, "nu_ghz": -1.0},
               {"out_kind": 7}):
        with pytest.raises(api.BpError, match="BP_EINVAL"):
            ctx.finalize(gg, m, **kw)
    assert torch.equal(m.y, maps.y) and torch.equal(m.ylo, maps.ylo)  # nothing written

"""Parity of the CUDA all-sky HP on HEALPix (Section 5.2 with the HP of Section 3.3, RING
ordering) with the oracle's LOS integrals at the great-circle angle of every pixel centre."""
import numpy as np
import pytest
import torch

from paper_2201_02632_gb300 import inputs as I
from tests.gpu_common import api, ctx, cuda  # noqa: F401
from tests.helpers import assert_map_parity

pytestmark = pytest.mark.gpu


def _gpu_maps(api, ctx, cat, nside, ap=0.0):
    model, status = ctx.solve_halos(cuda(cat["M"]), cuda(cat["c"]), cuda(cat["z"]))
    maps = api.healpix_maps(nside)
    ctx.paste_halos_healpix(cuda(cat["theta"]), cuda(cat["phi"]), cuda(cat["vlos"]), model,
                            status, nside, maps, ap_r500=ap)
    y = maps.y.double().cpu().numpy().ravel() + maps.ylo.double().cpu().numpy().ravel()
    b = maps.b.double().cpu().numpy().ravel() + maps.blo.double().cpu().numpy().ravel()
    return y, b


def _oracle_maps(orc, cat, nside, ap=0.0, pix=None):
    mo = orc.solve_halos(cat["M"], cat["c"], cat["z"])
    pt, pp = orc.hpx_centres(nside, pix)
    return orc.hp_sky(cat["theta"], cat["phi"], cat["vlos"], mo, pt, pp, ap_r500=ap, rtol=1e-9)


@pytest.mark.parametrize("nside,ap", [(256, 0.0), (100, 2.0)])
def test_full_sky_matches_oracle(orc, api, ctx, nside, ap):
    # nearby massive halos: apertures of 1-20 pixels; some on the poles, some across phi = 0
    cat = I.allsky_catalog(160, seed=I.SEED_BASE + 80, logm=(14.0, 15.3), zr=(0.01, 0.08),
                           volume=False, n_polar=12)
    cat["phi"][:6] = np.array([0.0, 1e-4, -1e-3, 2 * np.pi - 1e-4, 2 * np.pi, 6.3])
    y, b = _gpu_maps(api, ctx, cat, nside, ap)
    yo, bo = _oracle_maps(orc, cat, nside, ap)
    assert np.count_nonzero(yo) > 0.01 * yo.size
    assert_map_parity(y, yo, what="y")
    assert_map_parity(b, bo, what="b")


def test_small_nside_and_huge_apertures(orc, api, ctx):
    # nside 8: apertures larger than whole rings, polar caps covered entirely
    cat = I.allsky_catalog(40, seed=I.SEED_BASE + 81, logm=(14.5, 15.3), zr=(0.002, 0.01),
                           volume=False, n_polar=6)
    y, b = _gpu_maps(api, ctx, cat, 8)
    yo, bo = _oracle_maps(orc, cat, 8)
    assert_map_parity(y, yo, what="y")
    assert_map_parity(b, bo, what="b")


def test_deterministic(api, ctx):
    cat = I.allsky_catalog(3000, seed=I.SEED_BASE + 82, logm=(13.0, 15.0), zr=(0.01, 0.3),
                           volume=False)
    a = _gpu_maps(api, ctx, cat, 128)
    b = _gpu_maps(api, ctx, cat, 128)
    assert np.array_equal(a[0], b[0]) and np.array_equal(a[1], b[1])


def test_nside_8192_sampled(orc, api, ctx):
    """nside 8192 (the paper's all-sky resolution) with 2e5 halos of the all-sky catalogue
    recipe; the oracle at the brightest pixels and at random covered pixels."""
    nside = 8192
    cat = I.allsky_catalog(200_000, seed=I.SEED_BASE + 83)
    model, status = ctx.solve_halos(cuda(cat["M"]), cuda(cat["c"]), cuda(cat["z"]))
    maps = api.healpix_maps(nside)
    ctx.paste_halos_healpix(cuda(cat["theta"]), cuda(cat["phi"]), cuda(cat["vlos"]), model,
                            status, nside, maps)
    y = (maps.y.double() + maps.ylo.double()).ravel()
    b = (maps.b.double() + maps.blo.double()).ravel()
    top = torch.topk(y, 24).indices
    nz = torch.nonzero(y > 0).ravel()
    g = torch.Generator(device="cuda")
    g.manual_seed(7)
    rnd = nz[torch.randint(0, nz.numel(), (40,), generator=g, device="cuda")]
    pix = torch.cat([top, rnd]).cpu().numpy()
    # the oracle solves only the halos that can reach a sampled pixel: r_f stays below
    # 10 r_vir (its root bracket), so 12 r_vir / D_A bounds every aperture
    F = orc.F
    one = orc.solve_halos(cat["M"][:1], cat["c"][:1], cat["z"][:1])[0]
    def r_vir(M, z):
        return (3 * M / 0.7 / (4 * np.pi * orc.delta_vir(z) * orc.rho_cr(z))) ** (1 / 3)
    assert r_vir(cat["M"][0], cat["z"][0]) == pytest.approx(one[F["r_vir"]], rel=1e-6)
    zz = cat["z"]
    bound = np.array([12 * r_vir(M, z) / (orc.chi(z) / (1 + z)) for M, z in zip(cat["M"], zz)])
    pt, pp = orc.hpx_centres(nside, pix)
    vec = lambda t, p: np.stack([np.sin(t) * np.cos(p), np.sin(t) * np.sin(p), np.cos(t)], -1)
    ang = np.arccos(np.clip(vec(pt, pp) @ vec(cat["theta"], cat["phi"]).T, -1, 1))
    cand = np.nonzero((ang < bound[None, :]).any(0))[0]
    assert 0 < cand.size < 5000
    sub = {k: v[cand] for k, v in cat.items()}
    yo, bo = _oracle_maps(orc, sub, nside, pix=pix)
    yg, bg = y[torch.from_numpy(pix).cuda()].cpu().numpy(), b[torch.from_numpy(pix).cuda()].cpu().numpy()
    np.testing.assert_allclose(yg, yo, rtol=1e-4, atol=1e-4 * np.abs(yo).max())
    np.testing.assert_allclose(bg, bo, rtol=1e-4, atol=1e-4 * np.abs(bo).max())
    del maps
    torch.cuda.empty_cache()


def test_errors_and_empty_catalogue(api, ctx):
    maps = api.healpix_maps(4)
    e = torch.empty(0, dtype=torch.float64, device="cuda")
    model = torch.empty((24, 0), dtype=torch.float64, device="cuda")
    status = torch.empty(0, dtype=torch.int32, device="cuda")
    v = torch.empty(0, dtype=torch.float32, device="cuda")
    ctx.paste_halos_healpix(e, e, v, model, status, 4, maps)  # nothing to paste
    assert float(maps.y.abs().sum()) == 0.0
    cat = I.allsky_catalog(5, seed=I.SEED_BASE + 84)
    model, status = ctx.solve_halos(cuda(cat["M"]), cuda(cat["c"]), cuda(cat["z"]))
    args = (cuda(cat["theta"]), cuda(cat["phi"]), cuda(cat["vlos"]), model, status)
    for nside, ap in ((0, 0.0), (16385, 0.0), (4, -1.0)):
        with pytest.raises(api.BpError) as err:
            ctx.paste_halos_healpix(*args, nside, maps, ap_r500=ap)
        assert "BP_EINVAL" in str(err.value)
    # halos outside [0, pi] in colatitude add nothing
    bad = cuda(np.full(5, 4.0))
    maps.zero_()
    ctx.paste_halos_healpix(bad, args[1], args[2], model, status, 4, maps)
    assert float(maps.y.abs().sum()) == 0.0

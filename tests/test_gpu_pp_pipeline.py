"""End-to-end PP parity on a seeded light-cone: CUDA solve -> assign -> paste -> finalize
against the oracle's solve -> assign -> deposit (Sections 2 and 3.4)."""
import numpy as np
import pytest
import torch

from paper_2201_02632_gb300 import inputs as I
from tests.gpu_common import api, ctx, cuda, folded, gpu_geom, orc_geom, records_numpy  # noqa: F401
from tests.helpers import assert_map_parity

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def cone():
    return I.lightcone(n_part=300000, n_halo=200, npix=256, side_deg=2.0, seed=77)


@pytest.fixture(scope="module")
def oracle_side(orc, cone):
    lc = cone
    mo = orc.solve_halos(lc.halos.M, lc.halos.c, lc.halos.z)
    a = orc.pp_assign(lc.parts, lc.Mp, lc.halos.pos, mo, orc_geom(orc, lc.geom))
    return mo, a


def _gpu_assign(api, ctx, lc, parts=None):
    parts = parts or lc.parts
    model, status = ctx.solve_halos(cuda(lc.halos.M), cuda(lc.halos.c), cuda(lc.halos.z))
    tp = {k: cuda(v) for k, v in parts.items()}
    g = gpu_geom(api, lc.geom)
    rec = ctx.assign_particles(tp, lc.Mp, cuda(lc.halos.pos), model, status, g)
    return rec, g


def test_assign_matches_oracle(api, ctx, cone, oracle_side):
    mo, a = oracle_side
    rec, _ = _gpu_assign(api, ctx, cone)
    r = records_numpy(rec)
    kind = r["kind"]
    mism = np.count_nonzero(kind != a["kind"])
    assert mism <= 2  # only particles within rounding of r_f may differ
    ok = kind == a["kind"]
    np.testing.assert_allclose(r["px"], a["px"], rtol=0, atol=2e-7)
    np.testing.assert_allclose(r["py"], a["py"], rtol=0, atol=2e-7)
    np.testing.assert_allclose(r["hp"], a["hp"], rtol=2e-6)
    sel = ok & (a["kind"] == 0)
    np.testing.assert_allclose(r["Y"][sel], a["Y"][sel], rtol=2e-5, atol=0)
    np.testing.assert_allclose(r["B"][ok], a["B"][ok], rtol=2e-5,
                               atol=1e-6 * np.abs(a["B"]).max())
    assert np.all(r["Y"][kind == 1] == 0)


def test_pp_maps_match_oracle(orc, api, ctx, cone, oracle_side):
    mo, a = oracle_side
    rec, g = _gpu_assign(api, ctx, cone)
    maps = api.Maps.zeros(g)
    ctx.paste_particles(rec, g, maps)
    y, b = folded(maps)
    yo, bo = orc.pp_deposit(a, orc_geom(orc, cone.geom))
    assert_map_parity(y[0], yo, what="y")
    assert_map_parity(b[0], bo, what="b")
    ctx.finalize(g, maps)
    assert_map_parity(maps.y[0].cpu().numpy(), yo, what="y finalized")


def test_ksz_sign_and_zero_velocity_exact(api, ctx, cone):
    lc = cone
    base = _gpu_assign(api, ctx, lc)
    neg = dict(lc.parts, vx=-lc.parts["vx"], vy=-lc.parts["vy"], vz=-lc.parts["vz"])
    zero = dict(lc.parts, vx=np.zeros_like(lc.parts["vx"]), vy=np.zeros_like(lc.parts["vy"]),
                vz=np.zeros_like(lc.parts["vz"]))
    out = []
    for parts in (lc.parts, neg, zero):
        rec, g = _gpu_assign(api, ctx, lc, parts)
        maps = api.Maps.zeros(g)
        ctx.paste_particles(rec, g, maps)
        ctx.finalize(g, maps)
        out.append((maps.y[0].cpu().numpy(), maps.b[0].cpu().numpy()))
    (y0, b0), (y1, b1), (y2, b2) = out
    assert np.array_equal(b1, -b0) and np.array_equal(y1, y0)
    assert np.all(b2 == 0) and np.array_equal(y2, y0)
    del base


def test_halo_field_split_adds_up(api, ctx, cone):
    rec, g = _gpu_assign(api, ctx, cone)
    res = []
    for sel in (0, 1, 2):
        maps = api.Maps.zeros(g)
        ctx.paste_particles(rec, g, maps, sel)
        res.append(folded(maps))
    np.testing.assert_allclose(res[0][0], res[1][0] + res[2][0], rtol=1e-5,
                               atol=1e-6 * np.abs(res[0][0]).max())
    np.testing.assert_allclose(res[0][1], res[1][1] + res[2][1], rtol=1e-4,
                               atol=1e-6 * np.abs(res[0][1]).max())
    assert np.all(res[2][0] == 0)


def test_sky_pixels_wide_fine_map(orc, api, ctx):
    """Pixel coordinates on a 10 x 10 deg^2, 4096^2 map: the double-float FP32 angles near
    the axis and the FP64 angles beyond 3.6 deg off axis both agree with the oracle."""
    lc = I.lightcone(n_part=200000, n_halo=100, npix=4096, side_deg=10.0, seed=78)
    p = lc.parts
    off = np.abs(p["x"]) > p["z"] / 16
    assert off.mean() > 0.1 and (~off).mean() > 0.1  # both paths are exercised
    mo = orc.solve_halos(lc.halos.M, lc.halos.c, lc.halos.z)
    a = orc.pp_assign(p, lc.Mp, lc.halos.pos, mo, orc_geom(orc, lc.geom))
    rec, _ = _gpu_assign(api, ctx, lc)
    r = records_numpy(rec)
    np.testing.assert_allclose(r["px"], a["px"], rtol=0, atol=2e-7)
    np.testing.assert_allclose(r["py"], a["py"], rtol=0, atol=2e-7)


def test_potential_variant_matches_oracle(orc, api, ctx, cone, oracle_side):
    """bp_assign_particles_phi with each halo particle's NFW potential at its radius on the
    cloud's ellipsoidal shell (an aspherical potential): records and maps against the oracle's
    potential-based assignment."""
    lc = cone
    mo, a_sph = oracle_side
    h = orc.cosmo_default().h
    hid = lc.parts["hid"]
    r_ell = lc.info["r_ell"]
    phi = np.zeros(hid.size, np.float32)
    for k in np.unique(hid[hid >= 0]):
        sel = np.nonzero(hid == k)[0]
        r = r_ell[sel] / h / (1 + lc.halos.z[k])
        phi[sel] = orc.nfw_eval(lc.halos.M[k], lc.halos.c[k], lc.halos.z[k], r)[2]
    a = orc.pp_assign(lc.parts, lc.Mp, lc.halos.pos, mo, orc_geom(orc, lc.geom), phi=phi)
    model, status = ctx.solve_halos(cuda(lc.halos.M), cuda(lc.halos.c), cuda(lc.halos.z))
    tp = {k: cuda(v) for k, v in lc.parts.items()}
    g = gpu_geom(api, lc.geom)
    rec = ctx.assign_particles(tp, lc.Mp, cuda(lc.halos.pos), model, status, g, phi=cuda(phi))
    r = records_numpy(rec)
    ok = r["kind"] == a["kind"]
    assert np.count_nonzero(~ok) <= 2
    sel = ok & (a["kind"] == 0)
    np.testing.assert_allclose(r["Y"][sel], a["Y"][sel], rtol=2e-5, atol=1e-7 * a["Y"].max())
    np.testing.assert_allclose(r["B"][ok], a["B"][ok], rtol=2e-5,
                               atol=1e-6 * np.abs(a["B"]).max())
    # the variant is in effect: halo particles' signals move off the spherical model
    moved = np.abs(a["Y"][sel] / np.where(a_sph["Y"][sel] > 0, a_sph["Y"][sel], 1) - 1) > 1e-2
    assert np.count_nonzero(moved) > 0.3 * np.count_nonzero(sel)
    maps = api.Maps.zeros(g)
    ctx.paste_particles(rec, g, maps)
    y, b = folded(maps)
    yo, bo = orc.pp_deposit(a, orc_geom(orc, lc.geom))
    assert_map_parity(y[0], yo, what="y (potential-based)")
    assert_map_parity(b[0], bo, what="b (potential-based)")


def test_assign_in_parts_and_prepared_deposit(api, ctx, cone):
    """bp_assign_particles_part and bp_pp_prepare / bp_pp_deposit: the geometry part, the pair
    list built from it before the solve, then the signals part and the deposit give the
    records of the one-pass assign bit for bit and the maps of bp_paste_particles."""
    lc = cone
    rec_all, g = _gpu_assign(api, ctx, lc)
    maps_all = api.Maps.zeros(g)
    ctx.paste_particles(rec_all, g, maps_all)
    tp = {k: cuda(v) for k, v in lc.parts.items()}
    pos = cuda(lc.halos.pos)
    rec = torch.full_like(rec_all, float("nan"))
    ctx.assign_particles(tp, lc.Mp, pos, None, None, g, out=rec, part=api.ASSIGN_GEOMETRY)
    geo = rec.clone()
    assert float(geo[:, 3].abs().sum()) == 0.0 and float(geo[:, 4].abs().sum()) == 0.0
    ctx.pp_prepare(rec, g)
    model, status = ctx.solve_halos(cuda(lc.halos.M), cuda(lc.halos.c), cuda(lc.halos.z))
    ctx.assign_particles(tp, lc.Mp, pos, model, status, g, out=rec, part=api.ASSIGN_SIGNALS)
    a, b = rec.cpu().numpy().view(np.uint32), rec_all.cpu().numpy().view(np.uint32)
    assert np.array_equal(a, b)
    maps = api.Maps.zeros(g)
    ctx.pp_deposit(rec, g, maps)
    y, bb = folded(maps)
    y0, b0 = folded(maps_all)
    # the list may hold halo particles the signals part turned to NONE (zero signals), so
    # the tensor-core groups can differ: rounding of the FP32 group sums only
    assert np.linalg.norm(y - y0) <= 1e-6 * np.linalg.norm(y0)
    assert np.linalg.norm(bb - b0) <= 1e-6 * np.linalg.norm(b0)
    # misuse is refused: another select, or a list overwritten by another call
    with pytest.raises(api.BpError) as err:
        ctx.pp_deposit(rec, g, maps, select=api.SELECT_HALO)
    assert "BP_EINVAL" in str(err.value)
    ctx.pp_prepare(rec, g)
    hp = api.Maps.zeros(g)
    cat = lc.halos
    ctx.paste_halos(cuda(cat.thx), cuda(cat.thy), cuda(cat.vlos), model, status, g, hp)
    with pytest.raises(api.BpError) as err:
        ctx.pp_deposit(rec, g, maps)
    assert "BP_EINVAL" in str(err.value)
    with pytest.raises(api.BpError) as err:
        api.Context().pp_deposit(rec, g, maps)
    assert "BP_EINVAL" in str(err.value)

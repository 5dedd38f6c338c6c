"""Parity at full workload sizes, in the launch configuration bench.py times, on sampled
outputs the oracle computes one by one:
* the light-cone PP workload (4e6 particles, 3000 halos, 1024^2 maps) and the HP maps of its
  halos;
* the full-scale cone (5e8 particles, 2e5 halos, 4096^2 maps)."""
import numpy as np
import pytest
import torch

from paper_2201_02632_gb300 import inputs as I
from tests.gpu_common import api, cuda, gpu_geom, orc_geom  # noqa: F401

pytestmark = pytest.mark.gpu


def _sample(rng, y, n_rand=32, n_top=16):
    """Pixels to check: random ones plus the brightest (chosen by position only)."""
    ny, nx = y.shape
    flat = np.argsort(np.abs(y).ravel())[-n_top:]
    j = np.concatenate([rng.integers(0, ny, n_rand), flat // nx])
    i = np.concatenate([rng.integers(0, nx, n_rand), flat % nx])
    return i.astype(np.int32), j.astype(np.int32)


def _check(got, ref, full_max, what, rel=1e-4, frac=0.01):
    bright = np.abs(ref) > frac * full_max
    assert bright.sum() >= 8, what
    err = np.abs(got[bright] - ref[bright]) / np.abs(ref[bright])
    assert err.max() <= rel, f"{what}: max rel err {err.max():.3g}"
    l2 = np.linalg.norm(got - ref) / np.linalg.norm(ref)
    assert l2 <= 1e-5, f"{what}: sampled rel L2 {l2:.3g}"


def _pipeline(api, ctx, lc, parts_dev):
    cat = lc.halos
    t = lambda a: cuda(a)
    model, status = ctx.solve_halos(t(cat.M), t(cat.c), t(cat.z), raise_on_noconv=False)
    g = gpu_geom(api, lc.geom)
    rec = ctx.assign_particles(parts_dev, lc.Mp, t(cat.pos), model, status, g)
    pp = api.Maps.zeros(g)
    ctx.paste_particles(rec, g, pp)
    ctx.finalize(g, pp)
    return model, status, g, pp


def test_lightcone_full_size_sampled(orc, api):
    lc = I.lightcone()  # the bench workload
    ctx = api.Context()
    parts_dev = {k: cuda(v) for k, v in lc.parts.items()}
    model, status, g, pp = _pipeline(api, ctx, lc, parts_dev)
    hp = api.Maps.zeros(g)
    cat = lc.halos
    ctx.paste_halos(cuda(cat.thx), cuda(cat.thy), cuda(cat.vlos), model, status, g, hp)
    ctx.finalize(g, hp)
    y, b = pp.y[0].cpu().numpy(), pp.b[0].cpu().numpy()
    rng = np.random.default_rng(5)
    og = orc_geom(orc, lc.geom)
    pi_, pj_ = _sample(rng, y)
    mo = orc.solve_halos(cat.M, cat.c, cat.z)
    (yv, bv), _ = orc.pp_pixels(lc.parts, lc.Mp, cat.pos, mo, og, pi_, pj_)
    _check(y[pj_, pi_], yv, np.abs(y).max(), "PP y")
    pi_b, pj_b = _sample(rng, b)
    (yv2, bv2), _ = orc.pp_pixels(lc.parts, lc.Mp, cat.pos, mo, og, pi_b, pj_b)
    _check(b[pj_b, pi_b], bv2, np.abs(b).max(), "PP b")
    hy = hp.y[0].cpu().numpy()
    pi_h, pj_h = _sample(rng, hy, n_rand=24, n_top=12)
    hyv, hbv = orc.hp_pixels(cat.thx, cat.thy, cat.vlos, mo, og, pi_h, pj_h, rtol=1e-9)
    _check(hy[pj_h, pi_h], hyv, np.abs(hy).max(), "HP y")
    torch.cuda.synchronize()
    ctx.close()


def test_full_scale_cone_sampled(orc, api):
    lc = I.lightcone_device(n_part=500_000_000, n_halo=200_000)
    ctx = api.Context()
    model, status, g, pp = _pipeline(api, ctx, lc, lc.parts)
    y, b = pp.y[0].cpu().numpy(), pp.b[0].cpu().numpy()
    del pp
    host = {k: v.cpu().numpy() for k, v in lc.parts.items()}
    for k in list(lc.parts):
        del lc.parts[k]
    torch.cuda.empty_cache()
    rng = np.random.default_rng(9)
    og = orc_geom(orc, lc.geom)
    cat = lc.halos
    pi_, pj_ = _sample(rng, y, n_rand=16, n_top=8)
    pi_b, pj_b = _sample(rng, b, n_rand=16, n_top=8)
    pi_all = np.concatenate([pi_, pi_b])
    pj_all = np.concatenate([pj_, pj_b])
    idx = orc.pp_select(host, og, pi_all, pj_all)
    sub = {k: np.ascontiguousarray(v[idx]) for k, v in host.items()}
    mo = orc.solve_referenced(cat.M, cat.c, cat.z, sub["hid"])
    a = orc.pp_assign(sub, lc.Mp, cat.pos, mo, og)
    yv, bv = orc.pp_deposit_pixels(a, og, pi_all, pj_all)
    n1 = pi_.size
    _check(y[pj_, pi_], yv[:n1], np.abs(y).max(), "full-scale PP y")
    _check(b[pj_b, pi_b], bv[n1:], np.abs(b).max(), "full-scale PP b")
    torch.cuda.synchronize()
    ctx.close()

"""The single-sky partition on the GPU data path: the particles and halos of one sky split by
index into three shares (shard.shard_range), each share assigned, deposited and pasted by the
library into its own map planes, and the planes summed, equal the maps of the whole sky pasted
at once (the deposit and the halo paste are linear; only the rounding of the final sum and of
the compensated tile sums differs).  This is the exchange `bench.py --gpus N` makes with one
all-reduce, run here on one GPU share by share."""
import numpy as np
import pytest
import torch

from paper_2201_02632_gb300 import inputs as I
from paper_2201_02632_gb300 import shard
from tests.gpu_common import api, cuda  # noqa: F401

pytestmark = pytest.mark.gpu


def _fold(m):
    return np.stack([(m.y.double() + m.ylo.double()).cpu().numpy()[0],
                     (m.b.double() + m.blo.double()).cpu().numpy()[0]])


def test_sharded_sky_sums_to_the_whole_sky(api):
    lc = I.lightcone(n_part=300_000, n_halo=400, npix=512, side_deg=1.0, seed=91)
    ctx = api.Context()
    cat = lc.halos
    M, c, z = cuda(cat.M), cuda(cat.c), cuda(cat.z)
    pos, thx, thy, vl = cuda(cat.pos), cuda(cat.thx), cuda(cat.thy), cuda(cat.vlos)
    g = api.geom(lc.geom.nx, lc.geom.ny, lc.geom.theta0_x, lc.geom.theta0_y, lc.geom.dtheta)
    model, status = ctx.solve_halos(M, c, z)
    parts = {k: cuda(v) for k, v in lc.parts.items()}

    def paste(plo, phi, hlo, hhi):
        pp, hp = api.Maps.zeros(g), api.Maps.zeros(g)
        share = {k: v[plo:phi].contiguous() for k, v in parts.items()}
        rec = ctx.assign_particles(share, lc.Mp, pos, model, status, g)
        ctx.paste_particles(rec, g, pp)
        ctx.paste_halos(thx[hlo:hhi].contiguous(), thy[hlo:hhi].contiguous(),
                        vl[hlo:hhi].contiguous(), model[:, hlo:hhi].contiguous(),
                        status[hlo:hhi].contiguous(), g, hp)
        torch.cuda.synchronize()
        return np.concatenate([_fold(pp), _fold(hp)])

    n, nh = lc.parts["x"].size, cat.M.size
    whole = paste(0, n, 0, nh)
    world = 3
    summed = sum(paste(*shard.shard_range(n, r, world), *shard.shard_range(nh, r, world))
                 for r in range(world))
    for k, name in enumerate(("PP y", "PP b", "HP y", "HP b")):
        ref = whole[k]
        scale = np.abs(ref).max()
        assert scale > 0, name
        # the shares' sums agree with the whole to the rounding of FP32 map sums
        np.testing.assert_allclose(summed[k], ref, rtol=1e-6, atol=1e-6 * scale, err_msg=name)
    ctx.close()

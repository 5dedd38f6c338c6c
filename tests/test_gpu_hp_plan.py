"""Batched halo pasting through a prepared plan (one persistent launch over many maps),
replayed from a captured CUDA graph, and the autotuner; parity with bp_paste_halos and
with the oracle (Section 3.3)."""
import os

import numpy as np
import pytest
import torch

from paper_2201_02632_gb300 import inputs as I
from tests.gpu_common import api, ctx, cuda, folded, gpu_geom, orc_geom  # noqa: F401
from tests.helpers import assert_map_parity

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def batch():
    cat, g = I.batched_catalog(n_maps=4, mean_halos=150, side_deg=0.8, npix=160, seed=77)
    return cat, g


def _solved(ctx, cat):
    return ctx.solve_halos(cuda(cat.M), cuda(cat.c), cuda(cat.z))


def test_plan_matches_paste_and_oracle(orc, api, ctx, batch):
    cat, g = batch
    model, status = _solved(ctx, cat)
    gg = gpu_geom(api, g)
    args = (cuda(cat.thx), cuda(cat.thy), cuda(cat.vlos), model, status)
    mid = cuda(cat.map_id)
    ref = api.Maps.zeros(gg)
    ctx.set_tiling(hp_tile=32)
    ctx.paste_halos(*args, gg, ref, map_id=mid)
    plan = ctx.hp_plan(args[0], args[1], model, status, gg, map_id=mid, tile=32)
    assert plan.pairs > 0
    got = api.Maps.zeros(gg)
    plan.execute(*args, got, map_id=mid)
    torch.cuda.synchronize()
    for a, b in zip((got.y, got.b, got.ylo, got.blo), (ref.y, ref.b, ref.ylo, ref.blo)):
        assert torch.equal(a, b)  # same work list, same order: identical bits
    y, b = folded(got)
    mo = orc.solve_halos(cat.M, cat.c, cat.z)
    yo, bo = orc.hp_map(cat.thx, cat.thy, cat.vlos, mo, orc_geom(orc, g), map_id=cat.map_id,
                        rtol=1e-9)
    for m in range(g.n_maps):
        assert_map_parity(y[m], yo[m], what=f"y map {m}")
        assert_map_parity(b[m], bo[m], what=f"b map {m}")
    plan.close()


def test_plan_replays_from_a_cuda_graph(api, ctx, batch):
    cat, g = batch
    model, status = _solved(ctx, cat)
    gg = gpu_geom(api, g)
    thx, thy, vl, mid = cuda(cat.thx), cuda(cat.thy), cuda(cat.vlos), cuda(cat.map_id)
    plan = ctx.hp_plan(thx, thy, model, status, gg, map_id=mid, tile=64, unit=64, ctas_per_sm=1)
    eager = api.Maps.zeros(gg)
    plan.execute(thx, thy, vl, model, status, eager, map_id=mid)
    maps = api.Maps.zeros(gg)
    graph = torch.cuda.CUDAGraph()
    s = torch.cuda.Stream()
    s.wait_stream(torch.cuda.current_stream())
    with torch.cuda.stream(s):  # warm up on the side stream before capture
        ctx.set_stream(torch.cuda.current_stream())
        maps.zero_()
        plan.execute(thx, thy, vl, model, status, maps, map_id=mid)
    torch.cuda.current_stream().wait_stream(s)
    torch.cuda.synchronize()
    with torch.cuda.graph(graph):
        ctx.set_stream(torch.cuda.current_stream())
        maps.zero_()
        plan.execute(thx, thy, vl, model, status, maps, map_id=mid)
    ctx.set_stream(torch.cuda.current_stream())
    for _ in range(2):
        graph.replay()
        torch.cuda.synchronize()
        for a, b in zip((maps.y, maps.b, maps.ylo, maps.blo),
                        (eager.y, eager.b, eager.ylo, eager.blo)):
            assert torch.equal(a, b)
    plan.close()


def test_autotuner_picks_a_measured_config(api, ctx, batch, tmp_path):
    from paper_2201_02632_gb300 import autotune

    cat, g = batch
    model, status = _solved(ctx, cat)
    gg = gpu_geom(api, g)
    maps = api.Maps.zeros(gg)
    path = str(tmp_path / "tune.json")
    best = autotune.tune_hp(ctx, cuda(cat.thx), cuda(cat.thy), cuda(cat.vlos), model, status,
                            gg, maps, map_id=cuda(cat.map_id), tiles=(32, 64), units=(0, 128),
                            ctas=(0, 1), reps=2, cache_path=path)
    assert len(best["trials"]) == 8 and not best["cached"]
    assert best["ms"] == min(t["ms"] for t in best["trials"])
    again = autotune.tune_hp(ctx, cuda(cat.thx), cuda(cat.thy), cuda(cat.vlos), model, status,
                             gg, maps, map_id=cuda(cat.map_id), cache_path=path)
    assert again["cached"] and os.path.exists(path)

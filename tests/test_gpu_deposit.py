"""Parity of the CUDA tile pair list, radix sort and PP deposit (Section 3.4, Eqs. f_ij
and integrated kernel) with the oracle, on generator-drawn particle records."""
import numpy as np
import pytest
import torch

from paper_2201_02632_gb300 import inputs as I
from tests.gpu_common import api, assigned_tensor, ctx, folded, orc_deposit_inputs  # noqa: F401
from tests.helpers import assert_map_parity

pytestmark = pytest.mark.gpu


def _u32(t):
    return t.cpu().numpy().view(np.uint32)


@pytest.mark.parametrize("tile", [32, 64])
@pytest.mark.parametrize("select", [0, 1, 2])
def test_pairs_bit_exact(orc, api, ctx, tile, select):
    nx, ny = 200, 130  # ragged tiles on both axes
    a = I.assigned_particles(n=20000, npix=200, hmax=40, margin=30)
    rec = assigned_tensor(a)
    g = api.geom(nx, ny, 0.0, 0.0, 1.0)
    k, v = ctx.pp_pairs(rec, g, tile, select)
    ko, vo = orc.pp_pairs(a["ix"], a["fx"], a["iy"], a["fy"], a["hp"], a["kind"], nx, ny, tile,
                          tile, select)
    assert k.numel() == ko.size > 0
    assert np.array_equal(_u32(k), ko)
    assert np.array_equal(_u32(v), vo)


def test_pairs_multi_pass_sort_bit_exact(orc, api, ctx):
    # 4000 x 3000 map with 32-pixel tiles: 11750 tiles -> a two-pass radix sort
    nx, ny = 4000, 3000
    rng = np.random.default_rng(4)
    n = 300000
    a = I.deposit_inputs(rng.uniform(-50, nx + 50, n), rng.uniform(-50, ny + 50, n),
                         rng.exponential(8.0, n), np.ones(n), np.ones(n),
                         rng.integers(0, 3, n))
    rec = assigned_tensor(a)
    g = api.geom(nx, ny, 0.0, 0.0, 1.0)
    k, v = ctx.pp_pairs(rec, g, 32)
    ko, vo = orc.pp_pairs(a["ix"], a["fx"], a["iy"], a["fy"], a["hp"], a["kind"], nx, ny, 32, 32)
    assert np.array_equal(_u32(k), ko) and np.array_equal(_u32(v), vo)


def test_pairs_edge_cases(orc, api, ctx):
    g = api.geom(50, 40, 0.0, 0.0, 1.0)
    # empty input
    k, v = ctx.pp_pairs(torch.zeros((0, 8), dtype=torch.float32, device="cuda"), g, 32)
    assert k.numel() == 0
    # all particles off the map, NaN coordinates, kind NONE
    a = I.deposit_inputs([-100, 500, 10, 10], [10, 10, 5, 10], [5, 5, -1, 1], np.ones(4),
                         np.ones(4), [0, 1, 0, 2])
    k, v = ctx.pp_pairs(assigned_tensor(a), g, 32)
    assert k.numel() == 0
    # one particle covering the whole map
    a1 = I.deposit_inputs([25.0], [10.0], [1000.0], [1.0], [1.0], [0])
    k, v = ctx.pp_pairs(assigned_tensor(a1), g, 32)
    assert _u32(k).tolist() == [0, 1, 2, 3]


def _deposit(api, ctx, a, nx, ny, select=0):
    g = api.geom(nx, ny, 0.0, 0.0, 1.0)
    maps = api.Maps.zeros(g)
    ctx.paste_particles(assigned_tensor(a), g, maps, select)
    return folded(maps)


@pytest.mark.parametrize("tile,unit,kernel", [(64, 8192, "tensor"), (64, 256, "tensor"),
                                              (64, 8192, "simt"), (64, 256, "simt"),
                                              (32, 4096, "auto"), (32, 256, "auto")])
def test_deposit_matches_oracle(orc, api, ctx, tile, unit, kernel):
    nx, ny = 200, 130
    a = I.assigned_particles(n=20000, npix=200, hmax=40, margin=30)
    ctx.set_tiling(pp_tile=tile, pp_unit=unit)
    ctx.set_deposit_kernel(kernel)
    y, b = _deposit(api, ctx, a, nx, ny)
    yo, bo = orc.pp_deposit(orc_deposit_inputs(a), orc.geom(nx, ny, 0.0, 0.0, 1.0))
    assert_map_parity(y[0], yo, what="y")
    assert_map_parity(b[0], bo, what="b")


@pytest.mark.parametrize("select", [1, 2])
def test_deposit_select(orc, api, ctx, select):
    a = I.assigned_particles(n=5000, npix=96, hmax=20)
    y, b = _deposit(api, ctx, a, 96, 96, select)
    yo, bo = orc.pp_deposit(orc_deposit_inputs(a), orc.geom(96, 96, 0.0, 0.0, 1.0),
                            select=select)
    if select == 2:
        assert np.all(y == 0)
    else:
        assert_map_parity(y[0], yo, what="y")
    assert_map_parity(b[0], bo, what="b")


def test_deposit_conserves_interior_signal(api, ctx):
    rng = np.random.default_rng(8)
    n = 30000
    a = I.deposit_inputs(rng.uniform(35, 265, n), rng.uniform(35, 165, n),
                         rng.uniform(0, 30, n), rng.uniform(0, 1e-6, n), rng.normal(0, 1e-6, n),
                         np.zeros(n))
    y, b = _deposit(api, ctx, a, 300, 200)
    assert y.sum() == pytest.approx(a["Y"].astype(np.float64).sum(), rel=1e-6)
    assert b.sum() == pytest.approx(a["B"].astype(np.float64).sum(), rel=1e-5,
                                    abs=1e-6 * np.abs(a["B"]).sum())


def test_deposit_ngp_and_accumulation(api, ctx):
    a = I.deposit_inputs([2.3, 7.0], [6.9, 3.0], [0.0, 0.0], [3.0, 5.0], [-1.0, 2.0], [0, 0])
    g = api.geom(8, 8, 0.0, 0.0, 1.0)
    maps = api.Maps.zeros(g)
    rec = assigned_tensor(a)
    ctx.paste_particles(rec, g, maps)
    ctx.paste_particles(rec, g, maps)
    ctx.finalize(g, maps)
    y = maps.y[0].cpu().numpy()
    assert y[6, 2] == 6.0 and y[3, 7] == 10.0 and y.sum() == 16.0
    assert maps.b[0].cpu().numpy()[6, 2] == -2.0
    assert float(maps.ylo.abs().sum()) == 0.0


def test_tensor_and_simt_deposits_agree(api, ctx):
    """Both deposit kernels on one input: wide kernels (many particles per tile, several
    FP32 accumulation groups, ragged chunk tails) and kSZ signals of both signs."""
    rng = np.random.default_rng(21)
    n = 40000
    a = I.deposit_inputs(rng.uniform(-20, 276, n), rng.uniform(-20, 212, n),
                         rng.exponential(12.0, n), rng.uniform(0, 1e-6, n),
                         rng.normal(0, 1e-6, n), rng.integers(0, 2, n))
    out = {}
    for kernel in ("simt", "tensor"):
        ctx.set_deposit_kernel(kernel)
        out[kernel] = _deposit(api, ctx, a, 256, 192)
    for m in range(2):
        s, t = out["simt"][m][0], out["tensor"][m][0]
        assert np.linalg.norm(t - s) <= 2e-6 * np.linalg.norm(s)


def test_tensor_kernel_needs_tile_64(api, ctx):
    ctx.set_tiling(pp_tile=32)
    ctx.set_deposit_kernel("tensor")
    a = I.deposit_inputs([5.0], [5.0], [2.0], [1.0], [1.0], [0])
    g = api.geom(16, 16, 0.0, 0.0, 1.0)
    with pytest.raises(RuntimeError, match="tile 64"):
        ctx.paste_particles(assigned_tensor(a), g, api.Maps.zeros(g))


@pytest.mark.parametrize("unit", [256, 8192])
def test_tensor_deposit_timeout_returns_error_and_keeps_context(api, ctx, unit):
    """A bounded device wait that runs out (bp_set_wait_test: every CTA first waits on a flag
    that nothing sets, before issuing any MMA): the paste returns BP_ETIMEOUT, the maps are
    untouched (partial tiles included: unit 256 splits tiles), and the next paste on the same
    context is the normal result, bit for bit."""
    a = I.assigned_particles(n=20000, npix=200, hmax=40, margin=30)
    rec = assigned_tensor(a)
    g = api.geom(200, 130, 0.0, 0.0, 1.0)
    ctx.set_tiling(pp_tile=64, pp_unit=unit)
    ctx.set_deposit_kernel("tensor")
    ref = api.Maps.zeros(g)
    ctx.paste_particles(rec, g, ref)
    ctx.set_wait_test(2000)
    maps = api.Maps.zeros(g)
    for t in (maps.y, maps.b, maps.ylo, maps.blo):
        t.fill_(0.25)
    with pytest.raises(api.BpError, match="BP_ETIMEOUT"):
        ctx.paste_particles(rec, g, maps)
    torch.cuda.synchronize()
    for t in (maps.y, maps.b, maps.ylo, maps.blo):
        assert bool((t == 0.25).all())
    ctx.set_wait_test(0)
    again = api.Maps.zeros(g)
    ctx.paste_particles(rec, g, again)
    for x, y in ((again.y, ref.y), (again.b, ref.b), (again.ylo, ref.ylo), (again.blo, ref.blo)):
        assert torch.equal(x, y)


def _mixed_sizes(n, nx, ny, seed):
    """Records with kernels from sub-pixel to 60 pixels (most within the small-particle span),
    signed kSZ, a few h = 0 particles, some footprints crossing the map edges."""
    rng = np.random.default_rng(seed)
    hp = np.where(rng.random(n) < 0.75, rng.exponential(2.0, n), rng.uniform(8.0, 60.0, n))
    hp[rng.random(n) < 0.02] = 0.0
    return I.deposit_inputs(rng.uniform(-10, nx + 10, n), rng.uniform(-10, ny + 10, n), hp,
                            rng.uniform(0, 1e-6, n), rng.normal(0, 1e-6, n),
                            rng.integers(0, 2, n))


@pytest.mark.parametrize("span", [8, 3, 0])
def test_small_particle_deposit_matches_oracle(orc, api, ctx, span):
    """The small-particle deposit (particles at most `span` pixels wide, in size classes of at
    most 2, 4, 8 pixels; 0 = all on the tensor cores) against the oracle, with several tiles per
    map and ragged edges."""
    nx, ny = 300, 200
    a = _mixed_sizes(60000, nx, ny, 33)
    ctx.set_small_span(span)
    y, b = _deposit(api, ctx, a, nx, ny)
    yo, bo = orc.pp_deposit(orc_deposit_inputs(a), orc.geom(nx, ny, 0.0, 0.0, 1.0))
    assert_map_parity(y[0], yo, what="y")
    assert_map_parity(b[0], bo, what="b")


def test_small_particle_deposit_agrees_with_tensor_cores_and_repeats_bitwise(api, ctx):
    nx, ny = 256, 192
    a = _mixed_sizes(80000, nx, ny, 44)
    out = {}
    for span in (8, 0):
        ctx.set_small_span(span)
        out[span] = _deposit(api, ctx, a, nx, ny)
    for m in range(2):
        s, t = out[8][m][0], out[0][m][0]
        assert np.linalg.norm(t - s) <= 2e-6 * np.linalg.norm(t)
    ctx.set_small_span(8)
    again = _deposit(api, ctx, a, nx, ny)
    assert np.array_equal(again[0], out[8][0]) and np.array_equal(again[1], out[8][1])


def test_small_particle_deposit_wide_dynamic_range(orc, api, ctx):
    """Small particles of amplitudes over 12 decades in one tile: the fixed-point scale of the
    tile follows its largest amplitude, and the faint particles keep their relative accuracy
    wherever they dominate a pixel."""
    rng = np.random.default_rng(55)
    n = 4000
    px, py = rng.uniform(2, 62, n), rng.uniform(2, 62, n)
    Y = 10.0 ** rng.uniform(-12, 0, n)
    a = I.deposit_inputs(px, py, rng.uniform(0.3, 3.0, n), Y, -Y, np.zeros(n))
    ctx.set_small_span(8)
    y, b = _deposit(api, ctx, a, 64, 64)
    yo, bo = orc.pp_deposit(orc_deposit_inputs(a), orc.geom(64, 64, 0.0, 0.0, 1.0))
    assert_map_parity(y[0], yo, what="y")
    assert_map_parity(b[0], bo, what="b")
    # pixels six decades below the maximum still within the per-pixel tolerance
    mask = yo > 1e-6 * yo.max()
    assert np.max(np.abs(y[0][mask] - yo[mask]) / yo[mask]) < 1e-4


def test_small_span_rejects_out_of_range(api, ctx):
    for bad in (-2, 9):
        with pytest.raises(api.BpError, match="BP_EINVAL"):
            ctx.set_small_span(bad)


def test_small_particle_running_scale(orc, api, ctx):
    """The small-particle deposit reads a tile's records once and sets its fixed-point scale
    from the largest |Y| (|B|) seen so far: here the first blocks of the tile (1500 particles
    of the smallest size class) carry |Y|, |B| ~ 1e-3 and the last (600 of the largest class,
    sorted after them) ~ 1, so the sums of the first blocks are shifted down to the final
    scale when the bright block arrives.  The maps must still match the oracle, also in the
    pixels that only the faint particles reach (relative to those pixels' own values)."""
    rng = np.random.default_rng(12)
    nx = ny = 64 * 4 * 2  # 8 x 8 tiles: every particle in tile (2, 2) of a 512^2 map
    n_f, n_b = 1500, 600
    x0 = y0 = 128.0
    # faint: sub-pixel kernels spread over the whole tile; bright: 7-8 px boxes in one corner
    fx = rng.uniform(x0 + 1, x0 + 63, n_f)
    fy = rng.uniform(y0 + 1, y0 + 63, n_f)
    bx = rng.uniform(x0 + 5, x0 + 20, n_b)
    by = rng.uniform(y0 + 5, y0 + 20, n_b)
    hp = np.concatenate([rng.uniform(0.05, 0.4, n_f), rng.uniform(3.6, 3.9, n_b)])
    Y = np.concatenate([rng.uniform(0.5e-3, 1e-3, n_f), rng.uniform(0.5, 1.0, n_b)])
    B = np.concatenate([rng.normal(0, 1e-3, n_f), rng.normal(0, 1.0, n_b)])
    kind = np.zeros(n_f + n_b, np.int32)
    a = I.deposit_inputs(np.concatenate([fx, bx]), np.concatenate([fy, by]), hp, Y, B, kind)
    ctx.set_small_span(8)
    y, b = _deposit(api, ctx, a, nx, ny)
    yo, bo = orc.pp_deposit(orc_deposit_inputs(a), orc.geom(nx, ny, 0.0, 0.0, 1.0))
    assert_map_parity(y[0], yo, what="y")
    assert_map_parity(b[0], bo, what="b")
    # the pixels away from the bright corner hold faint particles only: relative error there
    far = np.zeros_like(yo, bool)
    far[int(y0) + 30:int(y0) + 64, int(x0) + 30:int(x0) + 64] = True
    sel = far & (yo > 1e-3 * yo[far].max())
    assert sel.sum() > 100
    assert np.abs(y[0][sel] - yo[sel]).max() <= 1e-4 * np.abs(yo[sel]).max()
    ctx.set_small_span(-1)

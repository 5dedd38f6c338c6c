"""The MLP surrogate of the ICM solve: CUDA training kernels against the FP64 CPU MLP,
BF16 inference against FP32, and the surrogate + polish + fallback solve against the
oracle solve (Section 2), plus what the trained network gains over the plain solve."""
import time

import numpy as np
import pytest
import torch

from oracle import mlp as omlp
from paper_2201_02632_gb300 import inputs as I
from tests.gpu_common import api, ctx, cuda  # noqa: F401

pytestmark = pytest.mark.gpu


def _rand_params(seed=0, scale=0.15):
    rng = np.random.default_rng(seed)
    n_par = sum(a * b + b for a, b in omlp.SIZES)
    return rng.normal(0, scale, n_par).astype(np.float32)


def test_forward_backward_match_fp64_mlp(api, ctx):
    p = _rand_params(1)
    rng = np.random.default_rng(2)
    n = 1000  # spans several 64-row tiles and 256-row gradient chunks, with a ragged tail
    x = rng.uniform(-1, 1, (n, 6)).astype(np.float32)
    t = rng.normal(0, 1, (n, 3)).astype(np.float32)
    P, X, T = cuda(p), cuda(x), cuda(t)
    y, cache = ctx.mlp_forward(P, X)
    dy, loss = ctx.mlp_mse(y, T)
    g = ctx.mlp_backward(P, X, cache, dy)
    yo, co = omlp.forward(p.astype(np.float64), x.astype(np.float64))
    dyo, lo = omlp.mse_grad(yo, t.astype(np.float64))
    go = omlp.backward(p.astype(np.float64), co, dyo)
    np.testing.assert_allclose(y.cpu().numpy(), yo, rtol=1e-4, atol=1e-5)
    assert loss == pytest.approx(lo, rel=1e-4)
    gg = g.cpu().numpy().astype(np.float64)
    assert np.linalg.norm(gg - go) <= 2e-4 * np.linalg.norm(go)
    # deterministic: a second backward gives the same bits
    g2 = ctx.mlp_backward(P, X, cache, dy)
    assert torch.equal(g, g2)


def test_adam_step_matches_fp64(api, ctx):
    p = _rand_params(3)
    rng = np.random.default_rng(4)
    g = rng.normal(0, 1e-2, p.size).astype(np.float32)
    m = rng.normal(0, 1e-3, p.size).astype(np.float32)
    v = np.abs(rng.normal(0, 1e-4, p.size)).astype(np.float32)
    P, G, Mm, V = cuda(p), cuda(g), cuda(m), cuda(v)
    ctx.mlp_adam(P, G, Mm, V, 7, 1e-3)
    po, mo, vo = omlp.adam(p.astype(np.float64), g.astype(np.float64), m.astype(np.float64),
                           v.astype(np.float64), 7, 1e-3)
    np.testing.assert_allclose(P.cpu().numpy(), po, rtol=1e-6, atol=1e-7)
    np.testing.assert_allclose(Mm.cpu().numpy(), mo, rtol=1e-5, atol=1e-9)


def test_bf16_inference_close_to_fp32(api, ctx):
    p = _rand_params(5)
    x = np.random.default_rng(6).uniform(-1, 1, (777, 6)).astype(np.float32)
    P, X = cuda(p), cuda(x)
    y32, _ = ctx.mlp_forward(P, X)
    wb = ctx.mlp_to_bf16(P)
    y16 = ctx.mlp_infer_bf16(wb, P, X)
    a, b = y16.cpu().numpy(), y32.cpu().numpy()
    assert np.abs(a - b).max() <= 3e-2 * max(1.0, np.abs(b).max())
    assert np.linalg.norm(a - b) <= 1e-2 * np.linalg.norm(b)


def test_bf16_inference_many_tiles(api, ctx):
    """The tensor-core inference over many 128-row tiles per CTA and a ragged last tile:
    the same agreement with the FP32 forward, row by row in norm."""
    p = _rand_params(7)
    n = 300_001
    x = np.random.default_rng(8).uniform(-1, 1, (n, 6)).astype(np.float32)
    P, X = cuda(p), cuda(x)
    y32, _ = ctx.mlp_forward(P, X)
    y16 = ctx.mlp_infer_bf16(ctx.mlp_to_bf16(P), P, X)
    a, b = y16.cpu().numpy(), y32.cpu().numpy()
    assert np.isfinite(a).all()
    assert np.linalg.norm(a - b) <= 1e-2 * np.linalg.norm(b)
    # no tile or row left out or shifted (that would differ by the size of the outputs):
    # every element within the BF16 bound of the 777-row test
    assert np.abs(a - b).max() <= 3e-2 * max(1.0, np.abs(b).max())
    assert np.abs(b - np.roll(b, 1, axis=0)).max() > 10 * np.abs(a - b).max()


@pytest.fixture(scope="module")
def trained(api):
    from paper_2201_02632_gb300.surrogate import Surrogate

    c = api.Context()
    M, cc, z, prm = I.surrogate_halos(60000, seed=11)
    s = Surrogate.init("cuda", seed=0)
    loss = s.fit(c, cuda(M), cuda(cc), cuda(z), cuda(prm), epochs=12, batch=2048)
    yield c, s, loss
    torch.cuda.synchronize()
    c.close()


def test_training_reduces_loss(trained):
    c, s, loss = trained
    first = s.history[0][1]
    assert loss < 0.02 * first and loss < 5e-3


def test_surrogate_solve_matches_oracle_with_fallback(orc, api, trained):
    c, s, _ = trained
    M, cc, z, prm = I.surrogate_halos(300, seed=12)
    # two halos far outside the training hull must go to the full solve
    M = np.concatenate([M, [3e15, 2e11]])
    cc = np.concatenate([cc, [4.0, 10.0]])
    z = np.concatenate([z, [0.5, 3.5]])
    prm = np.concatenate([prm, [[5e-6, 5e-6], [0.02, 0.02], [0.05, 0.05]]], axis=1)
    model, status = s.solve(c, cuda(M), cuda(cc), cuda(z), cuda(prm))
    assert (status.cpu().numpy() == 0).all()
    assert c.last_fallback_count() >= 2
    mg = model.cpu().numpy()
    F = orc.F
    for k in range(0, M.size, 37):
        ip = orc.icm_default(eps_star=float(prm[0, k]), f_star=float(prm[1, k]),
                             eps_dm=float(prm[2, k]))
        mo = orc.solve_halos(M[k:k + 1], cc[k:k + 1], z[k:k + 1], ip=ip)[0]
        for name, gname in (("r_f", "r_f"), ("T", "T"), ("rho0", "rho0"), ("P0", "P0")):
            assert mg[api.MF[gname], k] == pytest.approx(mo[F[name]], rel=1e-3), (k, name)
    # every accepted halo satisfies the gate
    assert np.abs(mg[api.MF["res_m"]]).max() <= 1e-4
    assert np.abs(mg[api.MF["res_e"]]).max() <= 1e-4


def test_surrogate_solve_at_scale(api, trained):
    """2e5 halos through the surrogate and through the plain solve (FP32 pre-solve +
    FP64 Newton): same accepted solutions; both timings are printed."""
    c, s, _ = trained
    M, cc, z, prm = I.surrogate_halos(200000, seed=13)
    args = [cuda(M), cuda(cc), cuda(z), cuda(prm)]
    c.solve_halos_ex(*args)  # warm up both paths
    s.solve(c, *args)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    m_plain, _ = c.solve_halos_ex(*args)
    torch.cuda.synchronize()
    t_plain = time.perf_counter() - t0
    t0 = time.perf_counter()
    m_sur, st = s.solve(c, *args)
    torch.cuda.synchronize()
    t_sur = time.perf_counter() - t0
    assert (st.cpu().numpy() == 0).all()
    print(f"surrogate {t_sur * 1e3:.1f} ms, plain {t_plain * 1e3:.1f} ms, "
          f"fallbacks {c.last_fallback_count()} of {M.size}")
    rf_p = m_plain[api.MF["r_f"]].cpu().numpy()
    rf_s = m_sur[api.MF["r_f"]].cpu().numpy()
    assert np.max(np.abs(rf_s / rf_p - 1)) < 1e-3


def test_gated_surrogate_solve_matches_oracle_with_fallback(orc, api, trained):
    """polish_iter = 0: the seeded FP32 pre-solve is the answer where both of its residuals are
    within the gate (1e-4); halos outside the training hull, or above the gate, get the full
    FP64 solve.  Accepted solutions agree with the oracle's to the gate's accuracy."""
    c, s, _ = trained
    M, cc, z, prm = I.surrogate_halos(300, seed=14)
    M = np.concatenate([M, [3e15, 2e11]])
    cc = np.concatenate([cc, [4.0, 10.0]])
    z = np.concatenate([z, [0.5, 3.5]])
    prm = np.concatenate([prm, [[5e-6, 5e-6], [0.02, 0.02], [0.05, 0.05]]], axis=1)
    model, status = s.solve(c, cuda(M), cuda(cc), cuda(z), cuda(prm), polish_iter=0)
    assert (status.cpu().numpy() == 0).all()
    assert c.last_fallback_count() >= 2  # the two halos outside the hull
    mg = model.cpu().numpy()
    F = orc.F
    for k in list(range(0, 300, 23)) + [300, 301]:
        ip = orc.icm_default(eps_star=float(prm[0, k]), f_star=float(prm[1, k]),
                             eps_dm=float(prm[2, k]))
        mo = orc.solve_halos(M[k:k + 1], cc[k:k + 1], z[k:k + 1], ip=ip)[0]
        for name in ("r_f", "T", "rho0", "P0"):
            assert mg[api.MF[name], k] == pytest.approx(mo[F[name]], rel=1e-3), (k, name)
    assert np.abs(mg[api.MF["res_m"]]).max() <= 1e-4
    assert np.abs(mg[api.MF["res_e"]]).max() <= 1e-4
    # the full-solve halos carry FP64 residuals of the plain tolerance
    assert np.abs(mg[api.MF["res_e"], 300:]).max() <= 1e-10


def test_gated_surrogate_gain_and_pasted_y_error(api, trained):
    """What the trained network gains: the gated surrogate solve against the plain solve (FP32
    pre-solve + FP64 Newton to 1e-10) on 2e5 halos, and the pasted y of a 1000-halo catalogue
    with each solve.  The surrogate must be at least 1.5x faster and the map within 1e-3."""
    c, s, _ = trained
    M, cc, z, prm = I.surrogate_halos(200000, seed=15)
    args = [cuda(M), cuda(cc), cuda(z), cuda(prm)]
    for _ in range(2):  # warm up both paths
        c.solve_halos_ex(*args, raise_on_noconv=False)
        s.solve(c, *args, polish_iter=0, raise_on_noconv=False)

    def timed(fn, reps=5):
        ts = []
        for _ in range(reps):
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            torch.cuda.synchronize()
            e0.record()
            fn()
            e1.record()
            torch.cuda.synchronize()
            ts.append(e0.elapsed_time(e1))
        return float(np.median(ts))

    t_plain = timed(lambda: c.solve_halos_ex(*args, raise_on_noconv=False))
    t_sur = timed(lambda: s.solve(c, *args, polish_iter=0, raise_on_noconv=False))
    print(f"gated surrogate {t_sur:.2f} ms, plain {t_plain:.2f} ms, "
          f"fallbacks {c.last_fallback_count()} of {M.size}")
    assert t_plain / t_sur >= 1.5
    cat, g = I.halo_catalog(n=1000, npix=256, seed=16)
    tab1 = cuda(np.stack([np.full(1000, 3.97e-6), np.full(1000, 0.026), np.zeros(1000)]))
    gg = api.geom(g.nx, g.ny, g.theta0_x, g.theta0_y, g.dtheta)
    ys = []
    for solve in (lambda a: c.solve_halos_ex(*a, params=tab1),
                  lambda a: s.solve(c, *a, tab1, polish_iter=0)):
        mod, st = solve([cuda(cat.M), cuda(cat.c), cuda(cat.z)])
        maps = api.Maps.zeros(gg)
        c.paste_halos(cuda(cat.thx), cuda(cat.thy), cuda(cat.vlos), mod, st, gg, maps,
                      ap_r500=3.0)
        c.finalize(gg, maps)
        ys.append(maps.y[0].double())
    err = float(torch.linalg.norm(ys[1] - ys[0]) / torch.linalg.norm(ys[0]))
    print(f"pasted y relative L2 vs the plain solve: {err:.2e}")
    assert err <= 1e-3

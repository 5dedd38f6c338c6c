"""Parity of the CUDA ICM solve (Section 2) with the FP64 oracle."""
import numpy as np
import pytest
import torch

from paper_2201_02632_gb300 import inputs as I
from tests.gpu_common import ORC_TO_GPU, api, ctx, cuda  # noqa: F401

pytestmark = pytest.mark.gpu

# closed-form / 1-D root quantities agree to rounding; solved quantities to the
# convergence tolerance of the two different root finders and quadratures.
CLOSED = ("M", "c", "z", "r_vir", "r_s", "rho_s", "m_c", "Phi0", "r500", "M500", "M_star",
          "r_star", "A_nt")
ENERGY = ("E_gi", "E_dm", "P_s")
SOLVED = ("T", "rho0", "P0", "r_f")


def _compare(orc, api, mo, mg, rtol_closed=1e-11, rtol_energy=1e-8, rtol_solved=1e-7):
    # rtol_energy: the closed-form dispersion (dilogarithm bracket) cancels ~3 digits at
    # c r/r_vir ~ 25, the quadrature oracle does not
    F = orc.F
    for name in CLOSED:
        np.testing.assert_allclose(mg[api.MF[ORC_TO_GPU[name]]], mo[:, F[name]],
                                   rtol=rtol_closed, err_msg=name)
    for name in ENERGY:
        np.testing.assert_allclose(mg[api.MF[name]], mo[:, F[name]], rtol=rtol_energy,
                                   err_msg=name)
    for name in SOLVED:
        np.testing.assert_allclose(mg[api.MF[name]], mo[:, F[name]], rtol=rtol_solved,
                                   err_msg=name)
    np.testing.assert_allclose(mg[api.MF["D_A"]], mo[:, F["D_A"]], rtol=1e-10)
    np.testing.assert_allclose(mg[api.MF["tau"]], mo[:, F["tau"]], rtol=1e-9)


def test_solve_matches_oracle_c0_catalogue(orc, api, ctx):
    cat, _ = I.halo_catalog(n=300)
    M = np.concatenate([cat.M, [1e12, 2e15, 1e12, 5e14]])
    c = np.concatenate([cat.c, [12.0, 3.0, 4.0, 25.0]])
    z = np.concatenate([cat.z, [3.0, 0.01, 0.01, 2.5]])
    mo = orc.solve_halos(M, c, z)
    model, status = ctx.solve_halos(cuda(M), cuda(c), cuda(z))
    mg = model.cpu().numpy()
    assert (status.cpu().numpy() == 0).all()
    assert (mo[:, orc.F["status"]] == 0).all()
    _compare(orc, api, mo, mg)
    assert np.abs(mg[api.MF["res_m"]]).max() < 1e-10
    assert np.abs(mg[api.MF["res_e"]]).max() < 1e-10


def test_solve_printed_energy_arrangement_and_other_gamma(orc, api):
    cat, _ = I.halo_catalog(n=40, seed=5)
    for icm in (dict(energy_sign=1), dict(Gamma=1.25), dict(Gamma=1.15, eps_dm=0.05)):
        c = api.Context(icm=icm)
        mo = orc.solve_halos(cat.M, cat.c, cat.z, ip=orc.icm_default(**icm))
        model, status = c.solve_halos(cuda(cat.M), cuda(cat.c), cuda(cat.z),
                                      raise_on_noconv=False)
        ok = mo[:, orc.F["status"]] == 0
        assert np.array_equal(status.cpu().numpy() == 0, ok), icm
        _compare(orc, api, mo[ok], model.cpu().numpy()[:, ok])
        torch.cuda.synchronize()
        c.close()


def test_solve_flags_bad_inputs(api, ctx):
    M = np.array([1e14, -1.0, np.nan, 1e14, 1e14])
    c = np.array([5.0, 5.0, 5.0, 0.0, 5.0])
    z = np.array([0.5, 0.5, 0.5, 0.5, 11.0])
    with pytest.raises(api.BpError) as e:
        ctx.solve_halos(cuda(M), cuda(c), cuda(z))
    assert "BP_ENOCONV" in str(e.value)
    model, status = ctx.solve_halos(cuda(M), cuda(c), cuda(z), raise_on_noconv=False)
    assert status.cpu().tolist() == [0, 5, 5, 5, 5]


def test_solve_empty_is_noop(api, ctx):
    e = torch.empty(0, dtype=torch.float64, device="cuda")
    model, status = ctx.solve_halos(e, e, e)
    assert model.shape == (len(api.MODEL_FIELDS), 0)


def test_seeded_presolve_reaches_the_same_solutions(orc, api, ctx):
    """BP_SOLVE_FP64_SEEDED: a starting point seeds the FP32 pre-solve.  From the exact
    solution, from a perturbed one and from no (non-finite) guess the solve reaches the
    oracle's solutions to the same tolerance as the plain solve."""
    cat, _ = I.halo_catalog(n=200)
    M, c, z = cat.M, cat.c, cat.z
    mo = orc.solve_halos(M, c, z)
    plain, st = ctx.solve_halos(cuda(M), cuda(c), cuda(z))
    p = plain.cpu().numpy()
    assert (st.cpu().numpy() == 0).all()
    F = api.MF
    exact = np.stack([np.log(p[F["r_f"]] / p[F["r_vir"]]),
                      np.log(p[F["T"]] * p[F["r_vir"]] / (4.30091e-9 * p[F["Mvir"]]))])
    rng = np.random.default_rng(4)
    perturbed = exact + rng.normal(0, 0.2, exact.shape)
    nonfinite = exact.copy()
    nonfinite[:, ::3] = np.nan
    for guess in (exact, perturbed, nonfinite):
        model, status = ctx.solve_halos_ex(cuda(M), cuda(c), cuda(z),
                                           guess=cuda(np.ascontiguousarray(guess)), max_iter=8,
                                           gate=1e-10, seeded=True)
        mg = model.cpu().numpy()
        assert (status.cpu().numpy() == 0).all()
        _compare(orc, api, mo, mg)
        assert np.abs(mg[F["res_m"]]).max() < 1e-10 and np.abs(mg[F["res_e"]]).max() < 1e-10
        for name in SOLVED:
            np.testing.assert_allclose(mg[F[name]], p[F[name]], rtol=1e-8, err_msg=name)


def test_fp32_gated_solve_without_seed(orc, api, ctx):
    """BP_SOLVE_FP32_GATED from the default start (no guess): the accepted halos carry the
    FP32 pre-solve's (r_f, T), within 1e-3 of the oracle and with both residuals within the
    gate; the rest are the FP64 solve's; closed-form fields are those of the plain solve; a
    gate of 0 is refused."""
    cat, _ = I.halo_catalog(n=400)
    M = np.concatenate([cat.M, [1e12, 2e15, 5e14]])
    c = np.concatenate([cat.c, [12.0, 3.0, 25.0]])
    z = np.concatenate([cat.z, [3.0, 0.01, 2.5]])
    mo = orc.solve_halos(M, c, z)
    gate = 1e-4
    model, status = ctx.solve_halos_ex(cuda(M), cuda(c), cuda(z), gate=gate, gated=True)
    nfb = ctx.last_fallback_count()
    mg = model.cpu().numpy()
    assert (status.cpu().numpy() == 0).all()
    assert 0 <= nfb < M.size // 2  # most halos are accepted from the pre-solve
    F, G = orc.F, api.MF
    for name in CLOSED:
        np.testing.assert_allclose(mg[G[ORC_TO_GPU[name]]], mo[:, F[name]], rtol=1e-11,
                                   err_msg=name)
    for name in ("r_f", "T", "rho0", "P0"):
        np.testing.assert_allclose(mg[G[name]], mo[:, F[name]], rtol=1e-3, err_msg=name)
    assert np.abs(mg[G["res_m"]]).max() <= gate and np.abs(mg[G["res_e"]]).max() <= gate
    with pytest.raises(api.BpError):
        ctx.solve_halos_ex(cuda(M), cuda(c), cuda(z), gate=0.0, gated=True)

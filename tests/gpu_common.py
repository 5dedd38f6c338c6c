"""Fixtures shared by the GPU parity tests (CUDA path through the C ABI vs the oracle)."""
import numpy as np
import pytest
import torch

from paper_2201_02632_gb300 import inputs as I

ORC_TO_GPU = {"M": "Mvir", "c": "c", "z": "z", "r_vir": "r_vir", "r_s": "r_s", "rho_s": "rho_s",
              "m_c": "m_c", "Phi0": "Phi0", "r500": "r500", "M500": "M500",
              "M_star": "M_star", "r_star": "r_star", "E_gi": "E_gi", "E_dm": "E_dm",
              "P_s": "P_s", "T": "T", "rho0": "rho0", "P0": "P0", "r_f": "r_f",
              "A_nt": "A_nt", "D_A": "D_A", "tau": "tau"}


def cuda(a, dtype=None):
    t = torch.as_tensor(np.ascontiguousarray(a))
    if dtype is not None:
        t = t.to(dtype)
    return t.cuda()


def gpu_geom(api, g):
    return api.geom(g.nx, g.ny, g.theta0_x, g.theta0_y, g.dtheta, getattr(g, "n_maps", 1))


def orc_geom(orc, g):
    return orc.geom(g.nx, g.ny, g.theta0_x, g.theta0_y, g.dtheta, getattr(g, "n_maps", 1))


def assigned_tensor(a):
    """Deposit inputs (see inputs.assigned_particles / deposit_inputs) -> the [n, 8]
    record layout of bp.h: fx, fy, hp, Y, B as FP32; kind, ix, iy as int32 bits."""
    n = a["fx"].size
    rec = np.zeros((n, 8), np.float32)
    rec[:, 0], rec[:, 1], rec[:, 2] = a["fx"], a["fy"], a["hp"]
    rec[:, 3], rec[:, 4] = a["Y"], a["B"]
    ints = rec.view(np.int32)
    ints[:, 5], ints[:, 6], ints[:, 7] = a["kind"], a["ix"], a["iy"]
    return cuda(rec)


def records_numpy(rec):
    """[n, 8] record tensor -> dict with the exact FP64 positions px = ix + fx."""
    r = rec.cpu().numpy()
    ints = r.view(np.int32)
    return {"px": ints[:, 6].astype(np.float64) + r[:, 0].astype(np.float64),
            "py": ints[:, 7].astype(np.float64) + r[:, 1].astype(np.float64),
            "hp": r[:, 2].astype(np.float64), "Y": r[:, 3].astype(np.float64),
            "B": r[:, 4].astype(np.float64), "kind": ints[:, 5].copy()}


def orc_deposit_inputs(a):
    return {k: np.asarray(a[k], np.float64) if k != "kind" else a[k]
            for k in ("px", "py", "hp", "Y", "B", "kind")}


def folded(maps):
    """hi + lo in FP64 on the host, [n_maps, ny, nx]."""
    y = maps.y.double().cpu().numpy() + maps.ylo.double().cpu().numpy()
    b = maps.b.double().cpu().numpy() + maps.blo.double().cpu().numpy()
    return y, b


@pytest.fixture(scope="session")
def api():
    from paper_2201_02632_gb300 import api as A
    from paper_2201_02632_gb300 import build

    build.build()
    return A


@pytest.fixture()
def ctx(api):
    c = api.Context()
    yield c
    torch.cuda.synchronize()
    c.close()


def gpu_model_from_oracle(api, mo):
    """The oracle's solved models [n, n_fields] in the library's field-major layout, with
    the oracle's status codes: lets a GPU call run on exactly the oracle's solution."""
    from oracle import F

    n = mo.shape[0]
    m = np.zeros((len(api.MODEL_FIELDS), n), np.float64)
    for o, gname in ORC_TO_GPU.items():
        m[api.MF[gname]] = mo[:, F[o]]
    m[api.MF["res_m"]] = mo[:, F["res_m"]]
    m[api.MF["res_e"]] = mo[:, F["res_e"]]
    status = mo[:, F["status"]].astype(np.int32)
    return cuda(m), cuda(status)

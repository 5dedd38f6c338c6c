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
    """Generator-drawn deposit inputs -> the [n, 8] FP32 record layout of bp.h."""
    n = a["px"].size
    rec = np.zeros((n, 8), np.float32)
    rec[:, 0], rec[:, 1], rec[:, 2] = a["px"], a["py"], a["hp"]
    rec[:, 3], rec[:, 4], rec[:, 5] = a["Y"], a["B"], a["kind"].astype(np.float32)
    return cuda(rec)


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

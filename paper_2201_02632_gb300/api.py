"""Python API over the C ABI, taking and returning CUDA torch tensors.

Every function forwards to the same-named entry point of include/bp.h; nothing
here computes.  Inputs must already live on a CUDA device (a CPU tensor raises).
"""
from __future__ import annotations

import ctypes as C
from dataclasses import dataclass

import torch

from . import _lib as L
from ._lib import (ASSIGNED_STRIDE, KIND_FIELD, KIND_HALO, KIND_NONE, MF, MODEL_FIELDS,
                   OUT_DT, OUT_YB, SELECT_ALL, SELECT_FIELD, SELECT_HALO, BpError)

__all__ = ["Context", "Maps", "geom", "MF", "MODEL_FIELDS", "ASSIGNED_STRIDE", "KIND_HALO",
           "KIND_FIELD", "KIND_NONE", "SELECT_ALL", "SELECT_HALO", "SELECT_FIELD", "OUT_YB",
           "OUT_DT", "BpError"]


def geom(nx, ny, theta0_x, theta0_y, dtheta, n_maps=1) -> L.BpGeom:
    return L.BpGeom(nx=int(nx), ny=int(ny), n_maps=int(n_maps), theta0_x=float(theta0_x),
                    theta0_y=float(theta0_y), dtheta=float(dtheta))


def _ptr(t, dtype, name):
    if t is None:
        return None
    if not isinstance(t, torch.Tensor) or not t.is_cuda:
        raise TypeError(f"{name} must be a CUDA tensor")
    if t.dtype != dtype:
        raise TypeError(f"{name} must be {dtype}, got {t.dtype}")
    if not t.is_contiguous():
        raise ValueError(f"{name} must be contiguous")
    return C.c_void_p(t.data_ptr())


@dataclass
class Maps:
    """FP32 maps and their compensation planes, [n_maps, ny, nx] each."""
    y: torch.Tensor
    b: torch.Tensor
    ylo: torch.Tensor
    blo: torch.Tensor

    @staticmethod
    def zeros(g: L.BpGeom, device="cuda") -> "Maps":
        shape = (g.n_maps, g.ny, g.nx)
        z = lambda: torch.zeros(shape, dtype=torch.float32, device=device)
        return Maps(z(), z(), z(), z())

    def zero_(self):
        for t in (self.y, self.b, self.ylo, self.blo):
            t.zero_()
        return self


class Context:
    """Owns a bp_ctx (background tables + scratch) bound to a CUDA stream."""

    def __init__(self, cosmo: dict | None = None, icm: dict | None = None, stream=None):
        self._L = L.load()
        c = dict(Om=0.279, Ob=0.046, h=0.7, Tcmb=2.726, XH=0.76)
        c.update(cosmo or {})
        q = dict(Gamma=1.2, eps_dm=0.0, eps_star=3.97e-6, f_star=0.026, S_star=0.12,
                 alpha_nt=0.18, beta_nt=0.5, n_nt=0.8, energy_sign=0, field_fb=0)
        q.update(icm or {})
        self.cosmo, self.icm = c, q
        self.stream = stream if stream is not None else torch.cuda.current_stream()
        h = C.c_void_p()
        rc = self._L.bp_create(C.byref(h), C.byref(L.BpCosmology(**c)), C.byref(L.BpIcm(**q)),
                               C.c_void_p(self.stream.cuda_stream))
        if rc != 0:
            raise BpError(rc, self._L.bp_last_error(None).decode())
        self._h = h

    def close(self):
        if getattr(self, "_h", None):
            self._L.bp_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def _check(self, rc, allow=()):
        if rc != 0 and rc not in allow:
            raise BpError(rc, self._L.bp_last_error(self._h).decode())
        return rc

    def set_tiling(self, pp_tile=0, hp_tile=0, pp_unit=0):
        self._check(self._L.bp_set_tiling(self._h, pp_tile, hp_tile, pp_unit))

    def workspace_bytes(self) -> int:
        return int(self._L.bp_workspace_bytes(self._h))

    def set_timing(self, on: bool = True):
        self._check(self._L.bp_set_timing(self._h, 1 if on else 0))

    def phase_times(self) -> dict:
        """Milliseconds per phase since the previous call (synchronises the stream)."""
        buf = (C.c_double * len(L.PHASES))()
        self._check(self._L.bp_phase_times(self._h, buf, len(L.PHASES)))
        return {name: float(buf[i]) for i, name in enumerate(L.PHASES)}

    def kernel_launches(self) -> int:
        return int(self._L.bp_kernel_launches(self._h))

    # ------------------------------------------------------------ Section 2
    def solve_halos(self, M, c, z, tol=1e-10, raise_on_noconv=True):
        """ICM solve of n halos (h^-1 Msun, c, z as FP64 CUDA tensors).  Returns
        (model [len(MODEL_FIELDS), n] FP64, status [n] int32)."""
        n = M.numel()
        model = torch.empty((len(MODEL_FIELDS), n), dtype=torch.float64, device=M.device)
        status = torch.empty(n, dtype=torch.int32, device=M.device)
        rc = self._L.bp_solve_halos(self._h, n, _ptr(M, torch.float64, "M"),
                                    _ptr(c, torch.float64, "c"), _ptr(z, torch.float64, "z"),
                                    _ptr(model, torch.float64, "model"),
                                    _ptr(status, torch.int32, "status"), 0, float(tol))
        self._check(rc, allow=() if raise_on_noconv else (L.BP_ENOCONV,))
        return model, status

    # ------------------------------------------------------------ Section 3.4
    def assign_particles(self, parts: dict, Mp: float, halo_pos, model, status, g: L.BpGeom,
                         out=None):
        """Per-particle signals.  parts: x,y,z,vx,vy,vz,hsml (FP32), hid (int32).
        Returns the [n, 8] FP32 record tensor."""
        n = parts["x"].numel()
        f32 = torch.float32
        if out is None:
            out = torch.empty((n, ASSIGNED_STRIDE), dtype=f32, device=parts["x"].device)
        nh = 0 if halo_pos is None else halo_pos.shape[-1]
        rc = self._L.bp_assign_particles(
            self._h, n, *(_ptr(parts[k], f32, k) for k in ("x", "y", "z", "vx", "vy", "vz",
                                                           "hsml")),
            _ptr(parts["hid"], torch.int32, "hid"), float(Mp), nh,
            _ptr(halo_pos, f32, "halo_pos"), _ptr(model, torch.float64, "model"),
            _ptr(status, torch.int32, "status"), C.byref(g), _ptr(out, f32, "out"))
        self._check(rc)
        return out

    def paste_particles(self, assigned, g: L.BpGeom, maps: Maps, select=SELECT_ALL):
        n = assigned.shape[0]
        f32 = torch.float32
        rc = self._L.bp_paste_particles(self._h, n, _ptr(assigned, f32, "assigned"), C.byref(g),
                                        int(select), _ptr(maps.y, f32, "y"),
                                        _ptr(maps.b, f32, "b"), _ptr(maps.ylo, f32, "ylo"),
                                        _ptr(maps.blo, f32, "blo"))
        self._check(rc)
        return maps

    def pp_pairs(self, assigned, g: L.BpGeom, tile: int, select=SELECT_ALL):
        """Sorted (tile key, particle index) pairs of the deposit (uint32 as int32)."""
        n = assigned.shape[0]
        cnt = C.c_int64(0)
        dev = assigned.device
        cap = 1
        keys = torch.empty(cap, dtype=torch.int32, device=dev)
        vals = torch.empty(cap, dtype=torch.int32, device=dev)
        rc = self._L.bp_pp_pairs(self._h, n, _ptr(assigned, torch.float32, "assigned"),
                                 C.byref(g), int(select), int(tile), _ptr(keys, torch.int32, "k"),
                                 _ptr(vals, torch.int32, "v"), cap, C.byref(cnt))
        if rc == L.BP_ERANGE:
            cap = int(cnt.value)
            keys = torch.empty(max(cap, 1), dtype=torch.int32, device=dev)
            vals = torch.empty(max(cap, 1), dtype=torch.int32, device=dev)
            rc = self._L.bp_pp_pairs(self._h, n, _ptr(assigned, torch.float32, "assigned"),
                                     C.byref(g), int(select), int(tile),
                                     _ptr(keys, torch.int32, "k"), _ptr(vals, torch.int32, "v"),
                                     cap, C.byref(cnt))
        self._check(rc)
        m = int(cnt.value)
        return keys[:m], vals[:m]

    # ------------------------------------------------------------ Section 3.3
    def paste_halos(self, thx, thy, vlos, model, status, g: L.BpGeom, maps: Maps, ap_r500=0.0,
                    map_id=None):
        n = thx.numel()
        f32 = torch.float32
        rc = self._L.bp_paste_halos(self._h, n, _ptr(thx, torch.float64, "thx"),
                                    _ptr(thy, torch.float64, "thy"), _ptr(vlos, f32, "vlos"),
                                    _ptr(map_id, torch.int32, "map_id"),
                                    _ptr(model, torch.float64, "model"),
                                    _ptr(status, torch.int32, "status"), C.byref(g),
                                    float(ap_r500), _ptr(maps.y, f32, "y"),
                                    _ptr(maps.b, f32, "b"), _ptr(maps.ylo, f32, "ylo"),
                                    _ptr(maps.blo, f32, "blo"))
        self._check(rc)
        return maps

    # ------------------------------------------------------------ Section 3.2
    def finalize(self, g: L.BpGeom, maps: Maps, out_kind=OUT_YB, nu_ghz=0.0):
        f32 = torch.float32
        rc = self._L.bp_finalize_map(self._h, C.byref(g), _ptr(maps.y, f32, "y"),
                                     _ptr(maps.b, f32, "b"), _ptr(maps.ylo, f32, "ylo"),
                                     _ptr(maps.blo, f32, "blo"), int(out_kind), float(nu_ghz))
        self._check(rc)
        return maps

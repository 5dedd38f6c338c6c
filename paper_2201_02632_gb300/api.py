"""Python API over the C ABI, taking and returning CUDA torch tensors.

Every function forwards to the same-named entry point of include/bp.h; nothing
here computes.  Inputs must already live on a CUDA device (a CPU tensor raises).
"""
from __future__ import annotations

import ctypes as C
from dataclasses import dataclass

import numpy as np
import torch

from . import _lib as L
from ._lib import (ASSIGN_ALL, ASSIGN_GEOMETRY, ASSIGN_SIGNALS, ASSIGNED_STRIDE, KIND_FIELD,
                   KIND_HALO, KIND_NONE, MF, MODEL_FIELDS, OUT_DT, OUT_YB, SELECT_ALL,
                   SELECT_FIELD, SELECT_HALO, BpError)

__all__ = ["Context", "Maps", "geom", "healpix_geom", "healpix_maps", "default_ell_edges", "MF", "MODEL_FIELDS", "ASSIGNED_STRIDE", "KIND_HALO",
           "KIND_FIELD", "KIND_NONE", "ASSIGN_ALL", "ASSIGN_GEOMETRY", "ASSIGN_SIGNALS",
           "SELECT_ALL", "SELECT_HALO", "SELECT_FIELD", "OUT_YB",
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


def default_ell_edges(lmin=1e2, lmax=1e5, nbins=30):
    """Logarithmic multipole bin edges (the paper's flat-sky binning: 30 bins, 1e2-1e5)."""
    return 10.0 ** np.linspace(np.log10(lmin), np.log10(lmax), nbins + 1)


def healpix_geom(nside) -> L.BpGeom:
    """The geometry that bp_finalize_map uses for a HEALPix map of 12 nside^2 pixels."""
    return geom(12 * nside, nside, 0.0, 0.0, 1.0)


def healpix_maps(nside, device="cuda") -> Maps:
    """Zeroed HEALPix maps in RING order, shape [1, nside, 12 nside] (flat index = pixel)."""
    return Maps.zeros(healpix_geom(nside), device)


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

    def set_stream(self, stream):
        """Queue later calls on `stream` (a torch.cuda.Stream)."""
        self.stream = stream
        self._check(self._L.bp_set_stream(self._h, C.c_void_p(stream.cuda_stream)))

    def set_tiling(self, pp_tile=0, hp_tile=0, pp_unit=0):
        self._check(self._L.bp_set_tiling(self._h, pp_tile, hp_tile, pp_unit))

    def set_deposit_kernel(self, kind="auto"):
        """PP deposit kernel: "auto" (tensor cores with tile 64), "simt" or "tensor"."""
        code = {"auto": 0, "simt": 1, "tensor": 2}[kind]
        self._check(self._L.bp_set_deposit_kernel(self._h, code))

    def set_small_span(self, span: int):
        """bp_set_small_span: the largest pixel span of the small-particle deposit (0: off)."""
        self._check(self._L.bp_set_small_span(self._h, int(span)))

    def set_wait_test(self, polls: int):
        """bp_set_wait_test: make the tensor-core deposit's first wait run out (polls > 0)."""
        self._check(self._L.bp_set_wait_test(self._h, int(polls)))

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

    def solve_halos_ex(self, M, c, z, params=None, guess=None, max_iter=0, gate=0.0, tol=1e-10,
                       raise_on_noconv=True, seeded=False, gated=False):
        """bp_solve_halos_ex: per-halo (eps_*, f_*, eps_DM) as params [3, n] FP64, starting
        point guess [2, n] FP64 (ln r_f/r_vir, ln T r_vir/GM), iteration cap and gate.
        seeded: the guess starts the FP32 pre-solve (BP_SOLVE_FP64_SEEDED) instead of the
        FP64 Newton.  gated: BP_SOLVE_FP32_GATED, the FP32 pre-solve's answer where both of
        its residuals are <= gate (> 0), the full FP64 solve elsewhere."""
        if seeded and gated:
            raise ValueError("solve_halos_ex: seeded and gated are exclusive")
        mode = L.BP_SOLVE_FP32_GATED if gated else (1 if seeded else 0)
        n = M.numel()
        f64 = torch.float64
        model = torch.empty((len(MODEL_FIELDS), n), dtype=f64, device=M.device)
        status = torch.empty(n, dtype=torch.int32, device=M.device)
        rc = self._L.bp_solve_halos_ex(self._h, n, _ptr(M, f64, "M"), _ptr(c, f64, "c"),
                                       _ptr(z, f64, "z"), _ptr(params, f64, "params"),
                                       _ptr(guess, f64, "guess"), int(max_iter), float(gate),
                                       _ptr(model, f64, "model"),
                                       _ptr(status, torch.int32, "status"), mode,
                                       float(tol))
        self._check(rc, allow=() if raise_on_noconv else (L.BP_ENOCONV,))
        return model, status

    def last_fallback_count(self) -> int:
        return int(self._L.bp_last_fallback_count(self._h))

    # ------------------------------------------------------------ MLP surrogate
    def mlp_forward(self, params, x, cache=None):
        n = x.shape[0]
        f32 = torch.float32
        y = torch.empty((n, L.MLP_OUT), dtype=f32, device=x.device)
        if cache is None:
            cache = torch.empty((n, L.MLP_CACHE_PER_ROW), dtype=f32, device=x.device)
        self._check(self._L.bp_mlp_forward(self._h, n, _ptr(params, f32, "params"),
                                           _ptr(x, f32, "x"), _ptr(y, f32, "y"),
                                           _ptr(cache, f32, "cache")))
        return y, cache

    def mlp_backward(self, params, x, cache, dy, grad=None):
        f32 = torch.float32
        if grad is None:
            grad = torch.empty(L.MLP_NPARAMS, dtype=f32, device=x.device)
        self._check(self._L.bp_mlp_backward(self._h, x.shape[0], _ptr(params, f32, "params"),
                                            _ptr(x, f32, "x"), _ptr(cache, f32, "cache"),
                                            _ptr(dy, f32, "dy"), _ptr(grad, f32, "grad")))
        return grad

    def mlp_adam(self, params, grad, m, v, step, lr, beta1=0.9, beta2=0.999, eps=1e-8):
        f32 = torch.float32
        self._check(self._L.bp_mlp_adam(self._h, _ptr(params, f32, "params"),
                                        _ptr(grad, f32, "grad"), _ptr(m, f32, "m"),
                                        _ptr(v, f32, "v"), int(step), float(lr), float(beta1),
                                        float(beta2), float(eps)))

    def mlp_to_bf16(self, params):
        wb = torch.empty(L.MLP_NWEIGHTS, dtype=torch.int16, device=params.device)
        self._check(self._L.bp_mlp_to_bf16(self._h, _ptr(params, torch.float32, "params"),
                                           _ptr(wb, torch.int16, "wb")))
        return wb

    def mlp_infer_bf16(self, wb, params, x):
        n = x.shape[0]
        y = torch.empty((n, L.MLP_OUT), dtype=torch.float32, device=x.device)
        self._check(self._L.bp_mlp_infer_bf16(self._h, n, _ptr(wb, torch.int16, "wb"),
                                              _ptr(params, torch.float32, "params"),
                                              _ptr(x, torch.float32, "x"),
                                              _ptr(y, torch.float32, "y")))
        return y

    def mlp_features(self, M, c, z, params, norm):
        n = M.numel()
        f64 = torch.float64
        x = torch.empty((n, L.MLP_IN), dtype=torch.float32, device=M.device)
        self._check(self._L.bp_mlp_features(self._h, n, _ptr(M, f64, "M"), _ptr(c, f64, "c"),
                                            _ptr(z, f64, "z"), _ptr(params, f64, "params"),
                                            _ptr(norm, torch.float32, "norm"),
                                            _ptr(x, torch.float32, "x")))
        return x

    def mlp_targets(self, model, norm):
        n = model.shape[1]
        t = torch.empty((n, L.MLP_OUT), dtype=torch.float32, device=model.device)
        self._check(self._L.bp_mlp_targets(self._h, n, _ptr(model, torch.float64, "model"),
                                           _ptr(norm, torch.float32, "norm"),
                                           _ptr(t, torch.float32, "t")))
        return t

    def mlp_mse(self, y, t, dy=None, want_loss=True):
        f32 = torch.float32
        if dy is None:
            dy = torch.empty_like(y)
        loss = C.c_double(0.0)
        self._check(self._L.bp_mlp_mse(self._h, y.shape[0], _ptr(y, f32, "y"), _ptr(t, f32, "t"),
                                       _ptr(dy, f32, "dy"),
                                       C.byref(loss) if want_loss else None))
        return dy, (loss.value if want_loss else None)

    def solve_halos_surrogate(self, M, c, z, params, wb, mlp_params, norm, hull, polish_iter=2,
                              gate=1e-4, tol=1e-10, raise_on_noconv=True):
        n = M.numel()
        f64, f32 = torch.float64, torch.float32
        model = torch.empty((len(MODEL_FIELDS), n), dtype=f64, device=M.device)
        status = torch.empty(n, dtype=torch.int32, device=M.device)
        rc = self._L.bp_solve_halos_surrogate(
            self._h, n, _ptr(M, f64, "M"), _ptr(c, f64, "c"), _ptr(z, f64, "z"),
            _ptr(params, f64, "params"), _ptr(wb, torch.int16, "wb"),
            _ptr(mlp_params, f32, "mlp_params"), _ptr(norm, f32, "norm"), _ptr(hull, f32, "hull"),
            int(polish_iter), float(gate), _ptr(model, f64, "model"),
            _ptr(status, torch.int32, "status"), float(tol))
        self._check(rc, allow=() if raise_on_noconv else (L.BP_ENOCONV,))
        return model, status

    # ------------------------------------------------------------ Section 3.4
    def assign_particles(self, parts: dict, Mp: float, halo_pos, model, status, g: L.BpGeom,
                         out=None, phi=None, part=None):
        """Per-particle signals.  parts: x,y,z,vx,vy,vz,hsml (FP32), hid (int32).  phi: optional
        FP32 per-particle potential [(km/s)^2] (bp_assign_particles_phi).  part: None (the whole
        record) or ASSIGN_GEOMETRY / ASSIGN_SIGNALS (bp_assign_particles_part; the geometry
        part reads no halo model).  Returns the [n, 8] FP32 record tensor."""
        n = parts["x"].numel()
        f32 = torch.float32
        if out is None:
            out = torch.empty((n, ASSIGNED_STRIDE), dtype=f32, device=parts["x"].device)
        nh = 0 if halo_pos is None else halo_pos.shape[-1]
        xyzv = [_ptr(parts[k], f32, k) for k in ("x", "y", "z", "vx", "vy", "vz")]
        tail = [_ptr(parts["hsml"], f32, "hsml"), _ptr(parts["hid"], torch.int32, "hid"),
                float(Mp), nh, _ptr(halo_pos, f32, "halo_pos"),
                _ptr(model, torch.float64, "model"), _ptr(status, torch.int32, "status"),
                C.byref(g), _ptr(out, f32, "out")]
        if part is not None:
            rc = self._L.bp_assign_particles_part(self._h, n, *xyzv, _ptr(phi, f32, "phi"),
                                                  *tail, int(part))
        elif phi is None:
            rc = self._L.bp_assign_particles(self._h, n, *xyzv, *tail)
        else:
            rc = self._L.bp_assign_particles_phi(self._h, n, *xyzv, _ptr(phi, f32, "phi"), *tail)
        self._check(rc)
        return out

    def pp_prepare(self, assigned, g: L.BpGeom, select=SELECT_ALL):
        """bp_pp_prepare: the sorted pair list and work units of the records' geometry."""
        self._check(self._L.bp_pp_prepare(self._h, assigned.shape[0],
                                          _ptr(assigned, torch.float32, "assigned"), C.byref(g),
                                          int(select)))

    def pp_deposit(self, assigned, g: L.BpGeom, maps: Maps, select=SELECT_ALL):
        """bp_pp_deposit: the records' Y and B through the list of the last pp_prepare."""
        f32 = torch.float32
        rc = self._L.bp_pp_deposit(self._h, assigned.shape[0], _ptr(assigned, f32, "assigned"),
                                   C.byref(g), int(select), _ptr(maps.y, f32, "y"),
                                   _ptr(maps.b, f32, "b"), _ptr(maps.ylo, f32, "ylo"),
                                   _ptr(maps.blo, f32, "blo"))
        self._check(rc)
        return maps

    def paste_particles(self, assigned, g: L.BpGeom, maps: Maps, select=SELECT_ALL):
        n = assigned.shape[0]
        f32 = torch.float32
        rc = self._L.bp_paste_particles(self._h, n, _ptr(assigned, f32, "assigned"), C.byref(g),
                                        int(select), _ptr(maps.y, f32, "y"),
                                        _ptr(maps.b, f32, "b"), _ptr(maps.ylo, f32, "ylo"),
                                        _ptr(maps.blo, f32, "blo"))
        self._check(rc)
        return maps

    def smoothing_lengths(self, x, y, z, n_ngb=64.0, guess=None, out=None):
        """SPH smoothing lengths of FP32 positions (Section 3.4): N_eff(h_i) = n_ngb."""
        n = x.numel()
        f32 = torch.float32
        if out is None:
            out = torch.empty(n, dtype=f32, device=x.device)
        rc = self._L.bp_smoothing_lengths(
            self._h, n, _ptr(x, f32, "x"), _ptr(y, f32, "y"), _ptr(z, f32, "z"), float(n_ngb),
            None if guess is None else _ptr(guess, f32, "guess"), _ptr(out, f32, "out"))
        self._check(rc)
        return out

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

    def hp_pairs(self, thx, thy, model, status, g: L.BpGeom, tile: int, ap_r500=0.0,
                 map_id=None):
        """Sorted ((map, tile) key, halo index) pairs of the halo paste (uint32 as int32)."""
        n = thx.numel()
        dev = thx.device
        cnt = C.c_int64(0)

        def call(cap):
            keys = torch.empty(max(cap, 1), dtype=torch.int32, device=dev)
            vals = torch.empty(max(cap, 1), dtype=torch.int32, device=dev)
            rc = self._L.bp_hp_pairs(self._h, n, _ptr(thx, torch.float64, "thx"),
                                     _ptr(thy, torch.float64, "thy"),
                                     _ptr(map_id, torch.int32, "map_id"),
                                     _ptr(model, torch.float64, "model"),
                                     _ptr(status, torch.int32, "status"), C.byref(g),
                                     float(ap_r500), int(tile), _ptr(keys, torch.int32, "k"),
                                     _ptr(vals, torch.int32, "v"), cap, C.byref(cnt))
            return rc, keys, vals

        rc, keys, vals = call(1)
        if rc == L.BP_ERANGE:
            rc, keys, vals = call(int(cnt.value))
        self._check(rc)
        m = int(cnt.value)
        return keys[:m], vals[:m]

    def paste_halos_healpix(self, theta, phi, vlos, model, status, nside, maps: Maps,
                            ap_r500=0.0):
        """All-sky HP on HEALPix (RING order); maps from healpix_maps(nside)."""
        f32 = torch.float32
        rc = self._L.bp_paste_halos_healpix(
            self._h, theta.numel(), _ptr(theta, torch.float64, "theta"),
            _ptr(phi, torch.float64, "phi"), _ptr(vlos, f32, "vlos"),
            _ptr(model, torch.float64, "model"), _ptr(status, torch.int32, "status"), int(nside),
            float(ap_r500), _ptr(maps.y, f32, "y"), _ptr(maps.b, f32, "b"),
            _ptr(maps.ylo, f32, "ylo"), _ptr(maps.blo, f32, "blo"))
        self._check(rc)
        return maps

    def power_spectrum(self, m, dtheta, edges=None, lo=None):
        """Binned flat-sky C_l of an FP32 map [ny, nx] (Section 5.3).  edges: multipole bin
        edges (default 30 logarithmic bins on [1e2, 1e5]).  Returns (l_centres, C_l,
        n_modes) with C_l and n_modes on the device."""
        if edges is None:
            edges = default_ell_edges()
        e = np.ascontiguousarray(edges, dtype=np.float64)
        ny, nx = m.shape[-2], m.shape[-1]
        nb = e.size - 1
        cl = torch.empty(nb, dtype=torch.float64, device=m.device)
        nm = torch.empty(nb, dtype=torch.int64, device=m.device)
        rc = self._L.bp_power_spectrum(
            self._h, _ptr(m, torch.float32, "map"), _ptr(lo, torch.float32, "lo"), int(nx),
            int(ny), float(dtheta), nb, e.ctypes.data_as(C.c_void_p), _ptr(cl, torch.float64, "cl"),
            _ptr(nm, torch.int64, "nmodes"))
        self._check(rc)
        return np.sqrt(e[:-1] * e[1:]), cl, nm

    def hp_plan(self, thx, thy, model, status, g: L.BpGeom, ap_r500=0.0, map_id=None, tile=32,
                unit=0, ctas_per_sm=0):
        """bp_hp_plan_create: the work list of one catalogue, reusable (and capturable)."""
        h = C.c_void_p()
        rc = self._L.bp_hp_plan_create(self._h, thx.numel(), _ptr(thx, torch.float64, "thx"),
                                       _ptr(thy, torch.float64, "thy"),
                                       _ptr(map_id, torch.int32, "map_id"),
                                       _ptr(model, torch.float64, "model"),
                                       _ptr(status, torch.int32, "status"), C.byref(g),
                                       float(ap_r500), int(tile), int(unit), int(ctas_per_sm),
                                       C.byref(h))
        self._check(rc)
        return HpPlan(self, h, g)

    # ------------------------------------------------------------ Section 3.2
    def finalize(self, g: L.BpGeom, maps: Maps, out_kind=OUT_YB, nu_ghz=0.0):
        f32 = torch.float32
        rc = self._L.bp_finalize_map(self._h, C.byref(g), _ptr(maps.y, f32, "y"),
                                     _ptr(maps.b, f32, "b"), _ptr(maps.ylo, f32, "ylo"),
                                     _ptr(maps.blo, f32, "blo"), int(out_kind), float(nu_ghz))
        self._check(rc)
        return maps


class HpPlan:
    """A prepared halo paste (bp_hp_plan_*)."""

    def __init__(self, ctx: Context, handle, g):
        self.ctx, self._h, self.geom = ctx, handle, g

    @property
    def pairs(self) -> int:
        return int(self.ctx._L.bp_hp_plan_pairs(self._h))

    def execute(self, thx, thy, vlos, model, status, maps: Maps, map_id=None):
        f32 = torch.float32
        rc = self.ctx._L.bp_hp_plan_execute(
            self.ctx._h, self._h, _ptr(thx, torch.float64, "thx"), _ptr(thy, torch.float64, "thy"),
            _ptr(vlos, f32, "vlos"), _ptr(map_id, torch.int32, "map_id"),
            _ptr(model, torch.float64, "model"), _ptr(status, torch.int32, "status"),
            _ptr(maps.y, f32, "y"), _ptr(maps.b, f32, "b"), _ptr(maps.ylo, f32, "ylo"),
            _ptr(maps.blo, f32, "blo"))
        self.ctx._check(rc)
        return maps

    def close(self):
        if getattr(self, "_h", None):
            self.ctx._L.bp_hp_plan_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

"""ctypes binding of libbp.so (include/bp.h).  Argument marshalling only: every
step of the computation runs in the library's CUDA kernels.  Raises if the
library is missing or a tensor is not on a CUDA device; there is no fallback."""
from __future__ import annotations

import ctypes as C
import os
import threading

HERE = os.path.dirname(os.path.abspath(__file__))
# the library this binding loads: the release build, or another build of the same sources
# named by BP_LIB (e.g. the debug build, build.build(debug=True))
LIB_PATH = os.environ.get("BP_LIB") or os.path.join(HERE, "_build", "libbp.so")

BP_OK, BP_EINVAL, BP_ECUDA, BP_ERANGE, BP_ENOCONV, BP_ETIMEOUT, BP_ENOMEM = 0, -1, -2, -3, -4, -5, -6
ERR_NAMES = {-1: "BP_EINVAL", -2: "BP_ECUDA", -3: "BP_ERANGE", -4: "BP_ENOCONV",
             -5: "BP_ETIMEOUT", -6: "BP_ENOMEM"}
# solve modes of bp_solve_halos_ex
BP_SOLVE_FP64, BP_SOLVE_FP64_SEEDED, BP_SOLVE_FP32_GATED = 0, 1, 2

MODEL_FIELDS = ("Mvir", "c", "z", "r_vir", "r_s", "rho_s", "m_c", "Phi0", "r500", "M500",
                "M_star", "r_star", "E_gi", "E_dm", "P_s", "T", "rho0", "P0", "r_f", "A_nt",
                "D_A", "tau", "res_m", "res_e")
MF = {n: i for i, n in enumerate(MODEL_FIELDS)}
ASSIGNED_STRIDE = 8
KIND_HALO, KIND_FIELD, KIND_NONE = 0, 1, 2
SELECT_ALL, SELECT_HALO, SELECT_FIELD = 0, 1, 2
ASSIGN_ALL, ASSIGN_GEOMETRY, ASSIGN_SIGNALS = 0, 1, 2
OUT_YB, OUT_DT = 0, 1

# entry points declared in include/bp.h
EXPORTS = ("bp_create", "bp_destroy", "bp_last_error", "bp_set_stream", "bp_set_tiling",
           "bp_set_deposit_kernel", "bp_set_wait_test", "bp_set_small_span",
           "bp_workspace_bytes", "bp_set_timing", "bp_phase_times", "bp_kernel_launches",
           "bp_solve_halos", "bp_assign_particles", "bp_paste_particles", "bp_pp_pairs",
           "bp_smoothing_lengths", "bp_paste_halos_healpix", "bp_power_spectrum",
           "bp_assign_particles_phi", "bp_assign_particles_part", "bp_pp_prepare",
           "bp_pp_deposit",
           "bp_paste_halos", "bp_hp_pairs", "bp_finalize_map", "bp_paste_particles_noalloc",
           "bp_solve_halos_ex", "bp_last_fallback_count", "bp_mlp_forward", "bp_mlp_backward",
           "bp_mlp_adam", "bp_mlp_to_bf16", "bp_mlp_infer_bf16", "bp_mlp_features",
           "bp_mlp_targets", "bp_mlp_mse", "bp_solve_halos_surrogate", "bp_hp_plan_create",
           "bp_hp_plan_execute", "bp_hp_plan_pairs", "bp_hp_plan_destroy", "bp_debug_build",
           "bp_debug_status", "bp_debug_selftest")
MLP_IN, MLP_HID, MLP_OUT = 6, 128, 3
MLP_NPARAMS = 128 * 6 + 128 + 2 * (128 * 128 + 128) + 3 * 128 + 3
MLP_NWEIGHTS = 128 * 6 + 2 * 128 * 128 + 3 * 128
MLP_CACHE_PER_ROW = 6 * 128
PHASES = ("solve", "assign", "pairs", "sort", "deposit", "reduce", "hp_table", "hp_pairs",
          "hp_paste", "finalize", "surrogate", "deposit_small")


class BpCosmology(C.Structure):
    _fields_ = [("Om", C.c_double), ("Ob", C.c_double), ("h", C.c_double),
                ("Tcmb", C.c_double), ("XH", C.c_double)]


class BpIcm(C.Structure):
    _fields_ = [("Gamma", C.c_double), ("eps_dm", C.c_double), ("eps_star", C.c_double),
                ("f_star", C.c_double), ("S_star", C.c_double), ("alpha_nt", C.c_double),
                ("beta_nt", C.c_double), ("n_nt", C.c_double), ("energy_sign", C.c_int),
                ("field_fb", C.c_int)]


class BpGeom(C.Structure):
    _fields_ = [("nx", C.c_int), ("ny", C.c_int), ("n_maps", C.c_int),
                ("theta0_x", C.c_double), ("theta0_y", C.c_double), ("dtheta", C.c_double)]


_lock = threading.Lock()
_lib = None


def load():
    """Load libbp.so (build it with paper_2201_02632_gb300.build.build() first)."""
    global _lib
    with _lock:
        if _lib is None:
            if not os.path.exists(LIB_PATH):
                raise RuntimeError(f"{LIB_PATH} not built: run paper_2201_02632_gb300.build.build()")
            L = C.CDLL(LIB_PATH)
            P, i64, i32, d = C.c_void_p, C.c_int64, C.c_int, C.c_double
            sig = {
                "bp_create": (i32, [C.POINTER(P), C.POINTER(BpCosmology), C.POINTER(BpIcm), P]),
                "bp_destroy": (i32, [P]),
                "bp_last_error": (C.c_char_p, [P]),
                "bp_set_stream": (i32, [P, P]),
                "bp_set_tiling": (i32, [P, i32, i32, i32]),
                "bp_set_deposit_kernel": (i32, [P, i32]),
                "bp_set_wait_test": (i32, [P, i64]),
                "bp_set_small_span": (i32, [P, i32]),
                "bp_debug_build": (i32, []),
                "bp_debug_status": (i32, [P, C.POINTER(C.c_int)]),
                "bp_debug_selftest": (i32, [P, i32]),
                "bp_workspace_bytes": (i64, [P]),
                "bp_set_timing": (i32, [P, i32]),
                "bp_phase_times": (i32, [P, C.POINTER(C.c_double), i32]),
                "bp_kernel_launches": (i64, [P]),
                "bp_solve_halos": (i32, [P, i64, P, P, P, P, P, i32, d]),
                "bp_solve_halos_ex": (i32, [P, i64, P, P, P, P, P, i32, d, P, P, i32, d]),
                "bp_last_fallback_count": (i64, [P]),
                "bp_mlp_forward": (i32, [P, i64, P, P, P, P]),
                "bp_mlp_backward": (i32, [P, i64, P, P, P, P, P]),
                "bp_mlp_adam": (i32, [P, P, P, P, P, i64, d, d, d, d]),
                "bp_mlp_to_bf16": (i32, [P, P, P]),
                "bp_mlp_infer_bf16": (i32, [P, i64, P, P, P, P]),
                "bp_mlp_features": (i32, [P, i64, P, P, P, P, P, P]),
                "bp_mlp_targets": (i32, [P, i64, P, P, P]),
                "bp_mlp_mse": (i32, [P, i64, P, P, P, C.POINTER(d)]),
                "bp_solve_halos_surrogate": (i32, [P, i64, P, P, P, P, P, P, P, P, i32, d, P, P,
                                                   d]),
                "bp_assign_particles": (i32, [P, i64, P, P, P, P, P, P, P, P, d, i64, P, P, P,
                                              C.POINTER(BpGeom), P]),
                "bp_assign_particles_phi": (i32, [P, i64, P, P, P, P, P, P, P, P, P, d, i64, P,
                                                  P, P, C.POINTER(BpGeom), P]),
                "bp_assign_particles_part": (i32, [P, i64, P, P, P, P, P, P, P, P, P, d, i64,
                                                   P, P, P, C.POINTER(BpGeom), P, i32]),
                "bp_paste_particles": (i32, [P, i64, P, C.POINTER(BpGeom), i32, P, P, P, P]),
                "bp_pp_prepare": (i32, [P, i64, P, C.POINTER(BpGeom), i32]),
                "bp_pp_deposit": (i32, [P, i64, P, C.POINTER(BpGeom), i32, P, P, P, P]),
                "bp_paste_particles_noalloc": (i32, [P, i64, P, C.POINTER(BpGeom), i32, P, P, P,
                                                     P]),
                "bp_smoothing_lengths": (i32, [P, i64, P, P, P, d, P, P]),
                "bp_paste_halos_healpix": (i32, [P, i64, P, P, P, P, P, i32, d, P, P, P, P]),
                "bp_power_spectrum": (i32, [P, P, P, i32, i32, d, i32, P, P, P]),
                "bp_pp_pairs": (i32, [P, i64, P, C.POINTER(BpGeom), i32, i32, P, P, i64,
                                      C.POINTER(i64)]),
                "bp_paste_halos": (i32, [P, i64, P, P, P, P, P, P, C.POINTER(BpGeom), d, P, P, P,
                                         P]),
                "bp_hp_pairs": (i32, [P, i64, P, P, P, P, P, C.POINTER(BpGeom), d, i32, P, P, i64,
                                      C.POINTER(i64)]),
                "bp_finalize_map": (i32, [P, C.POINTER(BpGeom), P, P, P, P, i32, d]),
                "bp_hp_plan_create": (i32, [P, i64, P, P, P, P, P, C.POINTER(BpGeom), d, i32, i32,
                                            i32, C.POINTER(P)]),
                "bp_hp_plan_execute": (i32, [P, P, P, P, P, P, P, P, P, P, P, P]),
                "bp_hp_plan_pairs": (i64, [P]),
                "bp_hp_plan_destroy": (i32, [P]),
            }
            for name, (res, args) in sig.items():
                f = getattr(L, name)
                f.restype = res
                f.argtypes = args
            _lib = L
    return _lib


class BpError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__(f"{ERR_NAMES.get(code, code)}: {msg}")
        self.code = code

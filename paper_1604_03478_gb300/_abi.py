"""ctypes binding of the C ABI in ``include/lbm_melt.h`` (argument
marshalling only; every step of the method runs in the CUDA library).

The functions keep the C names.  Loading fails loudly if the library has not
been built: there is no fallback implementation.
"""
from __future__ import annotations

import ctypes as C
import os

from . import build as _build

LBM_OK, LBM_EINVAL, LBM_ENOMEM, LBM_ECUDA, LBM_EUNSTABLE, LBM_ETIMEOUT, LBM_ENAN = 0, -1, -2, -3, -4, -5, -6
STATUS_NAMES = {0: "LBM_OK", -1: "LBM_EINVAL", -2: "LBM_ENOMEM", -3: "LBM_ECUDA", -4: "LBM_EUNSTABLE",
                -5: "LBM_ETIMEOUT", -6: "LBM_ENAN"}


class lbm_melt_grid(C.Structure):
    _fields_ = [("nx", C.c_int), ("ny", C.c_int), ("nz", C.c_int), ("heated_face", C.c_int),
                ("precision", C.c_int), ("Ma", C.c_double), ("s0", C.c_double)]


class lbm_melt_rates(C.Structure):
    _fields_ = [("s_nu", C.c_double), ("s_e", C.c_double), ("s_eps", C.c_double), ("s_q", C.c_double),
                ("s_pi", C.c_double), ("s_m", C.c_double), ("s_alpha", C.c_double), ("s_g4", C.c_double),
                ("s_g5", C.c_double), ("derive_from_Ra", C.c_int)]


class lbm_melt_case(C.Structure):
    _fields_ = [("grid", lbm_melt_grid), ("Ra", C.c_double), ("Pr", C.c_double), ("Ste", C.c_double),
                ("Th", C.c_double), ("Tc", C.c_double), ("Tm", C.c_double), ("rates", lbm_melt_rates)]


class lbm_melt_info(C.Structure):
    _fields_ = [("nu", C.c_double), ("alpha", C.c_double), ("gbeta", C.c_double), ("tau_nu", C.c_double),
                ("s_nu", C.c_double), ("s_alpha", C.c_double), ("lambda_", C.c_double), ("t0", C.c_double),
                ("H", C.c_double), ("n_cells", C.c_longlong), ("n_columns", C.c_longlong),
                ("steps", C.c_longlong), ("device_bytes", C.c_size_t)]


_lib = None


def library_path() -> str:
    return _build.LIB


def load() -> C.CDLL:
    """Load ``liblbm_melt.so`` (raises if it is missing)."""
    global _lib
    if _lib is not None:
        return _lib
    path = _build.LIB
    if not os.path.exists(path):
        raise ImportError("liblbm_melt.so is not built (run paper_1604_03478_gb300.build.build() or "
                          "__graft_entry__.build()); there is no CPU fallback")
    L = C.CDLL(path)
    vp, dp, fp = C.c_void_p, C.POINTER(C.c_double), C.POINTER(C.c_float)
    sig = {
        "lbm_melt_version": (C.c_char_p, []),
        "lbm_melt_derive": (C.c_int, [C.POINTER(lbm_melt_grid), C.c_double, C.c_double, C.c_double, C.c_double,
                                      C.c_double, C.c_double, C.POINTER(lbm_melt_rates), C.POINTER(lbm_melt_info)]),
        "lbm_melt_derive_error": (C.c_char_p, [C.POINTER(lbm_melt_grid), C.c_double, C.c_double, C.c_double,
                                              C.c_double, C.c_double, C.c_double, C.POINTER(lbm_melt_rates)]),
        "lbm_melt_create": (C.c_int, [C.POINTER(lbm_melt_grid), C.c_double, C.c_double, C.c_double, C.c_double,
                                      C.c_double, C.c_double, C.POINTER(lbm_melt_rates), vp, C.POINTER(vp)]),
        "lbm_melt_step": (C.c_int, [vp, C.c_longlong]),
        "lbm_melt_get": (C.c_int, [vp, vp, vp, vp, vp, C.c_int]),
        "lbm_melt_get_noalloc": (C.c_int, [vp, vp, vp, vp, vp, C.c_int]),
        "lbm_melt_get_async": (C.c_int, [vp, vp, vp, C.c_int]),
        "lbm_melt_get_state": (C.c_int, [vp, vp, vp, vp, C.c_int]),
        "lbm_melt_set_state": (C.c_int, [vp, vp, vp, vp, C.c_int]),
        "lbm_melt_set_hot_wall": (C.c_int, [vp, vp, C.c_int]),
        "lbm_melt_get_info": (C.c_int, [vp, C.POINTER(lbm_melt_info)]),
        "lbm_melt_sync": (C.c_int, [vp]),
        "lbm_melt_totals": (C.c_int, [vp, vp, C.c_int]),
        "lbm_melt_get_nusselt": (C.c_int, [vp, vp, vp, C.c_int]),
        "lbm_melt_set_report": (C.c_int, [vp, C.c_longlong, C.c_longlong]),
        "lbm_melt_get_report": (C.c_int, [vp, vp, C.c_longlong, C.POINTER(C.c_longlong)]),
        "lbm_melt_set_timing": (C.c_int, [vp, C.c_int]),
        "lbm_melt_set_graph_steps": (C.c_int, [vp, C.c_int]),
        "lbm_melt_set_solid_conduction": (C.c_int, [vp, C.c_double]),
        "lbm_melt_set_node_pairs": (C.c_int, [vp, C.c_int]),
        "lbm_melt_set_launch": (C.c_int, [vp, C.c_int, C.c_int]),
        "lbm_melt_kernel_time": (C.c_int, [vp, dp, C.POINTER(C.c_longlong), C.c_int]),
        "lbm_melt_last_error": (C.c_char_p, [vp]),
        "lbm_melt_tape_forward": (C.c_int, [vp, C.c_longlong, C.c_longlong]),
        "lbm_melt_tape_backward": (C.c_int, [vp, vp, vp, vp, C.c_int]),
        "lbm_melt_tape_clear": (C.c_int, [vp]),
        "lbm_ensemble_create": (C.c_int, [C.c_int, C.POINTER(lbm_melt_case), vp, C.POINTER(vp)]),
        "lbm_ensemble_step": (C.c_int, [vp, C.c_longlong]),
        "lbm_ensemble_set_launch": (C.c_int, [vp, C.c_int, C.c_int, C.c_int]),
        "lbm_ensemble_set_barrier_timeout": (C.c_int, [vp, C.c_longlong]),
        "lbm_ensemble_inject_barrier_fault": (C.c_int, [vp, C.c_int]),
        "lbm_ensemble_sync": (C.c_int, [vp]),
        "lbm_ensemble_member": (vp, [vp, C.c_int]),
        "lbm_ensemble_info": (C.c_int, [vp, C.POINTER(C.c_longlong), C.POINTER(C.c_int), C.POINTER(C.c_int),
                                        C.POINTER(C.c_int)]),
        "lbm_ensemble_phase_times": (C.c_int, [vp, C.c_int, C.POINTER(C.c_double), C.POINTER(C.c_longlong)]),
        "lbm_ensemble_last_error": (C.c_char_p, [vp]),
        "lbm_ensemble_destroy": (None, [vp]),
        "lbm_melt_destroy": (None, [vp]),
    }
    for name, (res, args) in sig.items():
        fn = getattr(L, name)
        fn.restype = res
        fn.argtypes = args
    _lib = L
    return L


def __getattr__(name):
    if name.startswith("lbm_melt_"):
        return getattr(load(), name)
    raise AttributeError(name)

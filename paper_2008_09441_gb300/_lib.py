"""ctypes binding of libsgpic.so (include/sgpic.h).

Argument marshalling only: every step of the computation runs in the CUDA
library.  Importing this module does not load the library; ``lib()`` does,
and raises if it has not been built (there is no CPU fallback).
"""
from __future__ import annotations

import ctypes as C
import os

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "lib", "libsgpic.so")

SG_OK = 0
SG_ERR_INVALID = -1
SG_ERR_UNSUPPORTED = -2
SG_ERR_OOM = -3
SG_ERR_SIZE = -4
SG_ERR_TIMEOUT = -5
SG_ERR_CUDA = -6
SG_ERR_RANGE = -7
SG_ERR_NONFINITE = -8
SG_ERR_STATE = -9
SG_FP32 = 0
SG_FP64 = 1
SG_TAU_ADAPTIVE = -1
SG_TAU_CONST_PAPER = 0
SG_TAU_CONST_EMPIRICAL = 1
SG_REQ_QUEUED, SG_REQ_RUNNING, SG_REQ_DONE, SG_REQ_FAILED = 0, 1, 2, 3
SG_SERVE_BATCHED, SG_SERVE_PLAIN = 0, 1
SG_MODE_COMBINE, SG_MODE_FILTER = 0, 1
SG_NODE_CENTRED, SG_CELL_CENTRED = 0, 1
SG_COMBINE_FLOAT_FLOAT, SG_COMBINE_FP64 = 0, 1
SG_SOLVE_AUTO, SG_SOLVE_PASSES, SG_SOLVE_ONE_BLOCK = -1, 0, 1
SG_DIAG_RING = 4


class sg_domain(C.Structure):
    _fields_ = [("dim", C.c_int), ("L", C.c_double * 3)]


class sg_particles(C.Structure):
    _fields_ = [("n", C.c_size_t), ("on_device", C.c_int), ("u", C.c_void_p * 3),
                ("v", C.c_void_p * 3), ("w", C.c_void_p)]


class sg_particles_out(C.Structure):
    _fields_ = [("n", C.c_size_t), ("on_device", C.c_int), ("u", C.c_void_p * 3),
                ("v", C.c_void_p * 3), ("w", C.c_void_p)]


class sg_params(C.Structure):
    _fields_ = [("precision", C.c_int), ("tau", C.c_int), ("dt", C.c_double), ("qm", C.c_double),
                ("B", C.c_double * 3), ("Eext_lin", C.c_double * 3), ("alpha", C.c_double),
                ("pc_ref", C.c_double), ("tau_constants", C.c_int), ("sort_every", C.c_int),
                ("stream", C.c_void_p), ("mode", C.c_int), ("centring", C.c_int), ("combine", C.c_int)]


class sg_diag(C.Structure):
    _fields_ = [("step", C.c_longlong), ("t", C.c_double), ("tau", C.c_int), ("n_grids", C.c_int),
                ("charge_total", C.c_double), ("charge_combined", C.c_double),
                ("charge_grid_max_abs_err", C.c_double), ("field_energy", C.c_double),
                ("field_energy_prev", C.c_double), ("kinetic_energy", C.c_double),
                ("count_checksum", C.c_ulonglong)]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


class sg_request(C.Structure):
    _fields_ = [("domain", sg_domain), ("level_n", C.c_int), ("dim", C.c_int),
                ("particles", sg_particles), ("params", sg_params), ("nsteps", C.c_int)]


_P = C.c_void_p
_SZ = C.c_size_t
SIGNATURES = {
    "sg_pic_init": (C.c_int, [C.POINTER(sg_domain), C.c_int, C.c_int, C.c_int, C.POINTER(sg_particles),
                              C.POINTER(sg_params), C.POINTER(_P)]),
    "sg_pic_init_deferred": (C.c_int, [C.POINTER(sg_domain), C.c_int, C.c_int, C.c_int, C.POINTER(sg_particles),
                                       C.POINTER(sg_params), C.POINTER(_P)]),
    "sg_pic_start": (C.c_int, [_P]),
    "sg_pic_step_deposit": (C.c_int, [_P]),
    "sg_pic_step_fields": (C.c_int, [_P]),
    "sg_pic_set_charge_total": (C.c_int, [_P, C.c_double]),
    "sg_pic_density_copy": (C.c_int, [_P, _P, _SZ, C.c_int]),
    "sg_pic_step": (C.c_int, [_P, C.c_int]),
    "sg_pic_diagnostics": (C.c_int, [_P, C.POINTER(sg_diag)]),
    "sg_pic_diagnostics_post": (C.c_int, [_P]),
    "sg_pic_diagnostics_collect": (C.c_int, [_P, C.POINTER(sg_diag)]),
    "sg_pic_select_tau": (C.c_int, [_P, C.POINTER(C.c_int), _P, _P, C.c_int]),
    "sg_pic_set_tau": (C.c_int, [_P, C.c_int]),
    "sg_pic_get_particles": (C.c_int, [_P, C.POINTER(sg_particles_out)]),
    "sg_pic_get_keys": (C.c_int, [_P, _P, _P, _SZ, _SZ]),
    "sg_pic_get_field": (C.c_int, [_P, _P, _SZ]),
    "sg_pic_get_grid_charge": (C.c_int, [_P, _P, _SZ]),
    "sg_pic_get_grid_field": (C.c_int, [_P, _P, _SZ]),
    "sg_pic_get_regular_charge": (C.c_int, [_P, _P, _SZ]),
    "sg_pic_get_density": (C.c_int, [_P, _P, _SZ]),
    "sg_pic_get_grids": (C.c_int, [_P, C.POINTER(C.c_int), _P, _P, C.c_int]),
    "sg_pic_save": (C.c_int, [_P, _P, C.POINTER(_SZ)]),
    "sg_pic_load": (C.c_int, [_P, _P, _SZ]),
    "sg_pic_device_particles": (C.c_int, [_P, C.POINTER(sg_particles_out)]),
    "sg_pic_kernel_launches": (C.c_int, [_P, C.POINTER(C.c_ulonglong)]),
    "sg_pic_set_profiling": (C.c_int, [_P, C.c_int]),
    "sg_pic_set_solve_variant": (C.c_int, [_P, C.c_int]),
    "sg_combination_grids": (C.c_int, [C.c_int, C.c_int, C.c_int, _P, _P, C.c_int, _P]),
    "sg_estimate_footprint": (C.c_int, [C.c_int, C.c_int, C.c_int, C.c_int, C.c_size_t, _P]),
    "sg_pic_stage_times": (C.c_int, [_P, _P, C.c_int]),
    "sg_pic_destroy": (None, [_P]),
    "sg_strerror": (C.c_char_p, [C.c_int]),
    "sg_last_error": (C.c_char_p, []),
    "sg_version": (C.c_char_p, []),
    "sg_cell_sort": (C.c_int, [C.c_int, C.c_int, C.c_int, _SZ, C.POINTER(_P), _P, _P, _P, _P]),
    "sg_cell_sort_static": (C.c_int, [C.c_int, C.c_int, C.c_int, _SZ, C.POINTER(_P), _P, _P, _P, _P]),
    "sg_serve_create": (C.c_int, [_SZ, C.c_int, C.POINTER(_P)]),
    "sg_serve_set_mode": (C.c_int, [_P, C.c_int]),
    "sg_serve_submit": (C.c_int, [_P, C.POINTER(sg_request), C.POINTER(C.c_ulonglong)]),
    "sg_serve_tick": (C.c_int, [_P, C.POINTER(C.c_int)]),
    "sg_serve_poll": (C.c_int, [_P, C.c_ulonglong, C.POINTER(C.c_int), C.POINTER(sg_diag)]),
    "sg_serve_result": (C.c_int, [_P, C.c_ulonglong, C.POINTER(sg_particles_out)]),
    "sg_serve_stats": (C.c_int, [_P, C.POINTER(C.c_double), C.POINTER(C.c_double), C.POINTER(C.c_double),
                                 C.POINTER(C.c_ulonglong)]),
    "sg_serve_solve_stats": (C.c_int, [_P, C.POINTER(C.c_ulonglong), C.POINTER(C.c_ulonglong)]),
    "sg_serve_destroy": (None, [_P]),
}

_lib = None


def lib():
    """Load libsgpic.so (built by __graft_entry__.build()); raise if absent."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise RuntimeError(f"CUDA library not built: {LIB_PATH} is missing "
                               "(run `python -c 'import __graft_entry__ as g; g.build()'`)")
        L = C.CDLL(LIB_PATH)
        for name, (res, args) in SIGNATURES.items():
            f = getattr(L, name)
            f.restype = res
            f.argtypes = args
        _lib = L
    return _lib


class SGError(RuntimeError):
    def __init__(self, status, where):
        L = lib()
        super().__init__(f"{where}: {L.sg_strerror(status).decode()} ({status}): {L.sg_last_error().decode()}")
        self.status = status


def check(status, where):
    if status != SG_OK:
        raise SGError(status, where)
    return status

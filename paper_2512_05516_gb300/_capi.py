"""ctypes declarations of the libsph C ABI (``include/sph.h``).

Argument marshalling only: every step of the SPH path runs in the CUDA
library.  Importing this module fails loudly when libsph.so has not been built.
"""
from __future__ import annotations

import ctypes as C
import os

from . import build as _build

SPH_NFIELDS = 10
F_X, F_V, F_A, F_M, F_H, F_RHO, F_U, F_P, F_DUDT, F_CS = range(10)
FIELD_NAMES = ["x", "v", "a", "m", "h", "rho", "u", "P", "dudt", "cs"]
NCOMP = [3, 3, 3, 1, 1, 1, 1, 1, 1, 1]


def BIT(f):
    return 1 << f


FIELDS_DENSITY = BIT(F_X) | BIT(F_M) | BIT(F_H) | BIT(F_U)
FIELDS_FORCE = FIELDS_DENSITY | BIT(F_V)
FIELDS_KICK = BIT(F_V) | BIT(F_U)
FIELDS_OUTPUT = BIT(F_V) | BIT(F_A) | BIT(F_H) | BIT(F_RHO) | BIT(F_U) | BIT(F_P)

P_FP32, P_BF16, P_FP16, P_FP32_M16, P_FP32_M10 = range(5)
PREC = {"fp32": P_FP32, "bf16": P_BF16, "fp16": P_FP16, "m16": P_FP32_M16, "m10": P_FP32_M10}
# the truncated family at every width: "m<n>" keeps n mantissa bits (n in 1..22)
for _n in range(1, 23):
    PREC.setdefault(f"m{_n}", 100 + _n)
AOS_F64, AOS_F32 = 0, 1
FLAG_PLAIN_SUM = 1
WS_REORDER = 1
BIN_REORDER, BIN_DRIFT_KEYS = 1, 2
WS_LEVELS = 2
KEV_DENSITY, KEV_FORCE = 0, 1
LEVEL_MIN, LEVEL_MAX, LEVELS_MAX = 2, 10, 8
ERR_NONFINITE, ERR_OUTSIDE, ERR_HCAP, ERR_NEWTON, ERR_TIMEOUT = 1, 2, 4, 8, 16
PFLAG_HCAP, PFLAG_NEWTON, PFLAG_NONFINITE = 1, 2, 4
SRC_AOS, SRC_SOA = 0, 1
BUFFER_MIN, BUFFER_MAX = 32, 256

OK, EINVAL, ENOSPACE, ECUDA, ESTATE, ECAPACITY, ETIMEOUT, ENUMERIC = 0, -1, -2, -3, -4, -5, -6, -7


class sph_aos_layout(C.Structure):
    _fields_ = [("record_bytes", C.c_int32), ("offset", C.c_int32 * SPH_NFIELDS),
                ("type", C.c_int32 * SPH_NFIELDS)]


class sph_params(C.Structure):
    _fields_ = [("box", C.c_double * 3), ("gamma", C.c_double), ("alpha_av", C.c_double),
                ("beta_av", C.c_double), ("eps_av", C.c_double), ("eta", C.c_double),
                ("h_max", C.c_double), ("flags", C.c_int32), ("reserved", C.c_int32)]


class sph_stats(C.Structure):
    _fields_ = [("pairs_density", C.c_uint64), ("pairs_force", C.c_uint64),
                ("tests_density", C.c_uint64), ("tests_force", C.c_uint64),
                ("hcap_clamps", C.c_uint64), ("error_bits", C.c_uint32),
                ("ncell", C.c_int32 * 3), ("nitems", C.c_int64), ("max_occupancy", C.c_int64),
                ("launches", C.c_uint64)]


class sph_tuning(C.Structure):
    _fields_ = [("block_threads", C.c_int32), ("ctas_per_sm", C.c_int32),
                ("stage_density", C.c_int32), ("stage_force", C.c_int32), ("subcells", C.c_int32),
                ("item_order", C.c_int32), ("class_launches", C.c_int32), ("pair_kernel", C.c_int32),
                ("block_threads_force", C.c_int32)]


class sph_desc(C.Structure):
    _fields_ = [("n", C.c_int64), ("ncell", C.c_int32 * 3), ("cell_edge", C.c_double * 3),
                ("off_perm", C.c_int64), ("off_cell_of_slot", C.c_int64),
                ("off_cell_start", C.c_int64), ("off_nngb", C.c_int64),
                ("off_nngb_force", C.c_int64), ("off_soa", (C.c_int64 * 3) * SPH_NFIELDS),
                ("prec", C.c_int32 * SPH_NFIELDS), ("valid", C.c_uint32), ("subcells", C.c_int32),
                ("off_level", C.c_int64), ("off_density_flags", C.c_int64)]


# every symbol the header declares, with its prototype
_P = C.c_void_p
PROTOTYPES = {
    "sph_workspace_bytes": (C.c_size_t, [C.POINTER(sph_aos_layout), C.c_int64, C.c_int64, C.c_uint32]),
    "sph_create": (C.c_int, [C.POINTER(sph_aos_layout), C.POINTER(sph_params), C.c_int64, C.c_int64,
                             C.c_uint32, _P, _P, C.c_size_t, _P, C.POINTER(_P)]),
    "sph_bin_cells": (C.c_int, [_P, C.c_double, C.c_int32]),
    "sph_aos_to_soa": (C.c_int, [_P, C.c_uint32, C.POINTER(C.c_int32)]),
    "sph_density": (C.c_int, [_P, C.c_int32]),
    "sph_force": (C.c_int, [_P]),
    "sph_kick_drift": (C.c_int, [_P, C.c_double, C.c_double]),
    "sph_soa_to_aos": (C.c_int, [_P, C.c_uint32]),
    "sph_kick_drift_writeback": (C.c_int, [_P, C.c_double, C.c_double, C.c_uint32]),
    "sph_set_field_scale": (C.c_int, [_P, C.POINTER(C.c_int32)]),
    "sph_get_field_scale": (C.c_int, [_P, C.POINTER(C.c_int32)]),
    "sph_get_stats": (C.c_int, [_P, C.POINTER(sph_stats)]),
    "sph_reset_stats": (C.c_int, [_P]),
    "sph_set_kernel_events": (C.c_int, [_P, C.c_int32, _P, _P]),
    "sph_set_tuning": (C.c_int, [_P, C.POINTER(sph_tuning)]),
    "sph_get_tuning": (C.c_int, [_P, C.POINTER(sph_tuning)]),
    "sph_describe": (C.c_int, [_P, C.POINTER(sph_desc)]),
    "sph_aos_upload": (C.c_int, [_P, _P, C.c_size_t]),
    "sph_aos_download": (C.c_int, [_P, _P, C.c_size_t]),
    "sph_bin_cells_noalloc": (C.c_int, [_P, C.POINTER(sph_aos_layout), C.c_int64, C.POINTER(C.c_double),
                                        C.POINTER(C.c_int32), _P, _P, _P, _P]),
    "sph_host_stage_bytes": (C.c_size_t, [_P]),
    "sph_aos_to_soa_host": (C.c_int, [_P, _P, C.c_uint32, C.POINTER(C.c_int32), _P, C.c_size_t, C.c_int32]),
    "sph_soa_to_aos_host": (C.c_int, [_P, _P, C.c_uint32, _P, C.c_size_t, C.c_int32]),
    "sph_bin_buffers": (C.c_int, [_P, C.c_int32]),
    "sph_buffer_density": (C.c_int, [_P, C.c_int32]),
    "sph_buffer_force": (C.c_int, [_P, C.c_int32]),
    "sph_buffer_kick": (C.c_int, [_P, C.c_int32, C.c_double]),
    "sph_buffer_drift": (C.c_int, [_P, C.c_int32, C.c_double]),
    "sph_bin_levels": (C.c_int, [_P, C.c_int32, C.c_int32, C.c_double]),
    "sph_density_levels": (C.c_int, [_P, C.c_int32]),
    "sph_force_levels": (C.c_int, [_P]),
    "sph_level_counts": (C.c_int, [_P, C.POINTER(C.c_int64), C.POINTER(C.c_int64)]),
    "sph_destroy": (None, [_P]),
    "sph_status_str": (C.c_char_p, [C.c_int]),
}


def load(path: str | None = None):
    """Load libsph.so (built in-tree by ``build.build()``).  Raises when the
    library is missing: there is no fallback implementation."""
    path = path or _build.LIB_PATH
    if not os.path.exists(path):
        raise ImportError(f"libsph.so is not built ({path}); run paper_2512_05516_gb300.build.build()")
    lib = C.CDLL(path)
    for name, (rt, at) in PROTOTYPES.items():
        fn = getattr(lib, name)
        fn.restype = rt
        fn.argtypes = at
    return lib

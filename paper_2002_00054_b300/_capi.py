"""ctypes declarations of the C ABI in include/nnp.h (argument marshalling only).

Loading fails loudly when libnnp.so has not been built: there is no CPU path.
"""
from __future__ import annotations

import ctypes
import os

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libnnp.so")

NNP_OK, NNP_EINVAL, NNP_ENOMEM, NNP_ENEIGH_OVERFLOW, NNP_ENONFINITE, NNP_EBOX, NNP_ECUDA, NNP_EUNSUPPORTED = range(8)
NNP_SF_RADIAL, NNP_SF_ANG_NARROW, NNP_SF_ANG_WIDE = 2, 3, 4
NNP_FP32, NNP_BF16 = 0, 1

c_int_p = ctypes.POINTER(ctypes.c_int)
c_double_p = ctypes.POINTER(ctypes.c_double)


class SfDesc(ctypes.Structure):
    _fields_ = [("type", ctypes.c_int), ("elem_a", ctypes.c_int), ("elem_b", ctypes.c_int),
                ("eta", ctypes.c_double), ("rs", ctypes.c_double), ("zeta", ctypes.c_double),
                ("lambda_", ctypes.c_double)]


class Params(ctypes.Structure):
    _fields_ = [("n_elements", ctypes.c_int), ("masses_amu", c_double_p), ("cutoff", ctypes.c_double),
                ("skin", ctypes.c_double), ("n_sf", c_int_p), ("sf", ctypes.POINTER(SfDesc)),
                ("sf_shift", c_double_p), ("sf_scale", c_double_p), ("n_layers", ctypes.c_int),
                ("widths", c_int_p), ("weights", c_double_p), ("mlp_precision", ctypes.c_int),
                ("max_neighbors", ctypes.c_int)]


class Stats(ctypes.Structure):
    _fields_ = [("n_atoms", ctypes.c_longlong), ("list_entries", ctypes.c_longlong),
                ("cutoff_entries", ctypes.c_longlong), ("pairs", ctypes.c_longlong),
                ("triplets", ctypes.c_longlong), ("rebuilds", ctypes.c_longlong),
                ("kernel_launches", ctypes.c_longlong), ("max_list_row", ctypes.c_longlong),
                ("max_cutoff_row", ctypes.c_longlong), ("spilled_atoms", ctypes.c_longlong),
                ("rc_capacity", ctypes.c_longlong), ("min_distance", ctypes.c_double)]


# name -> (restype, argtypes); every symbol declared in include/nnp.h
V = ctypes.c_void_p
I = ctypes.c_int
D = ctypes.c_double
SIGNATURES = {
    "nnp_create": (I, [ctypes.POINTER(Params), I, ctypes.POINTER(V)]),
    "nnp_destroy": (I, [V]),
    "nnp_last_error": (ctypes.c_char_p, [V]),
    "nnp_status_string": (ctypes.c_char_p, [I]),
    "nnp_num_params": (I, [V]),
    "nnp_set_weights": (I, [V, V, V]),
    "nnp_compute": (I, [V, I, V, V, c_double_p, D, V, V, V, V, V]),
    "nnp_compute_domain": (I, [V, I, I, V, V, c_double_p, V, V, V, V, V]),
    "nnp_descriptors": (I, [V, I, V, V, c_double_p, V, V, V]),
    "nnp_descriptors_flat": (I, [V, I, V, V, c_double_p, V, V]),
    "nnp_descriptors_pair": (I, [V, I, V, V, c_double_p, V, V]),
    "nnp_descriptors_cell": (I, [V, I, V, V, c_double_p, V, V]),
    "nnp_step": (I, [V, I, V, V, V, c_double_p, D, I, V, V]),
    "nnp_get_stats": (I, [V, ctypes.POINTER(Stats)]),
    "nnp_profile": (I, [V, I]),
    "nnp_num_kernel_groups": (I, []),
    "nnp_kernel_group_name": (ctypes.c_char_p, [I]),
    "nnp_kernel_times": (I, [V, I, c_double_p, ctypes.POINTER(ctypes.c_longlong)]),
    "nnp_compute_static": (I, [V, I, V, V, c_double_p, V, V, V, ctypes.c_char_p, I, V]),
    "nnp_compute_batch": (I, [V, I, c_int_p, c_double_p, V, V, V, V, V, V]),
    "nnp_param_grad": (I, [V, I, c_int_p, c_double_p, V, V, V, V, V, V]),
}

_lib = None


def load():
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise ImportError("libnnp.so is not built (run __graft_entry__.build() or "
                              "python paper_2002_00054_b300/build.py); there is no CPU fallback")
        lib = ctypes.CDLL(LIB_PATH)
        for name, (res, args) in SIGNATURES.items():
            f = getattr(lib, name)
            f.restype = res
            f.argtypes = args
        _lib = lib
    return _lib


class NNPError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__("%s: %s" % (load().nnp_status_string(status).decode(), msg))
        self.status = status

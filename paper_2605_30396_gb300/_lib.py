"""ctypes loader for libdlsh.so: argument types of every C-ABI entry point.

Importing this module never falls back to anything: if the library is missing
or stale, `lib()` raises.
"""
from __future__ import annotations

import ctypes
import os

from . import build as _build

_LIB = None

c_int, c_int64, c_float, c_size_t = ctypes.c_int, ctypes.c_int64, ctypes.c_float, ctypes.c_size_t
P = ctypes.c_void_p

class Scene(ctypes.Structure):
    """Mirror of dlsh_scene."""
    _fields_ = [("D", ctypes.c_void_p), ("K", ctypes.c_int), ("X", ctypes.c_void_p),
                ("N", ctypes.c_int64), ("s", ctypes.c_int), ("eps", ctypes.c_float),
                ("idx", ctypes.c_void_p), ("coef", ctypes.c_void_p), ("nnz", ctypes.c_void_p),
                ("resid_sq", ctypes.c_void_p)]


class Camera(ctypes.Structure):
    """Mirror of dlsh_camera."""
    _fields_ = [("R", ctypes.c_float * 9), ("t", ctypes.c_float * 3), ("fx", ctypes.c_float),
                ("fy", ctypes.c_float), ("width", ctypes.c_int), ("height", ctypes.c_int),
                ("z_near", ctypes.c_float)]


class Gaussians(ctypes.Structure):
    """Mirror of dlsh_gaussians."""
    _fields_ = [("means", ctypes.c_void_p), ("scales", ctypes.c_void_p), ("quats", ctypes.c_void_p),
                ("dc", ctypes.c_void_p), ("N", ctypes.c_int64)]


class SplatOut(ctypes.Structure):
    """Mirror of dlsh_splat_out."""
    _fields_ = [("xy", ctypes.c_void_p), ("depth", ctypes.c_void_p), ("conic", ctypes.c_void_p),
                ("radius", ctypes.c_void_p), ("rgb", ctypes.c_void_p)]


SIGNATURES = {
    "dlsh_last_error": (ctypes.c_char_p, []),
    "dlsh_version": (c_int, []),
    "dlsh_num_sms": (c_int, []),
    "dlsh_kernel_launches": (ctypes.c_ulonglong, []),
    "dlsh_encode_workspace_size": (c_size_t, [c_int, c_int, c_int, c_int]),
    "dlsh_encode_variant": (c_int, [c_int, c_int, c_int]),
    "dlsh_encode": (c_int, [P, c_int, c_int, P, c_int64, c_int, c_float, c_int, P, P, P, P, P,
                            c_size_t, P, c_int]),
    "dlsh_encode_profile": (c_int, [P, c_int, c_int, P, c_int64, c_int, c_float, c_int, P, P, P, P,
                                    P, c_size_t, P, P, c_int]),
    "dlsh_encode_noalloc_max_bytes": (c_size_t, []),
    "dlsh_encode_noalloc": (c_int, [P, c_int, c_int, P, c_int64, c_int, c_float, c_int, P, P, P,
                                    P, P, c_int]),
    "dlsh_correlate": (c_int, [P, c_int, c_int, P, c_int64, c_int, P, P, c_size_t, P, c_int]),
    "dlsh_decode": (c_int, [P, c_int, c_int, P, P, P, c_int, c_int64, P, P, P, P, P, c_int]),
    "dlsh_mod_workspace_size": (c_size_t, [c_int, c_int, c_int, c_int64]),
    "dlsh_mod_update": (c_int, [P, c_int64, c_int, c_int, P, P, P, c_int, P, P, P, P, c_size_t,
                                P, c_int]),
    "dlsh_learn_workspace_size": (c_size_t, [c_int, c_int, c_int, c_int64, c_int]),
    "dlsh_learn_dictionary": (c_int, [P, c_int64, c_int, c_int, c_int, c_float, c_int, P, c_int,
                                      P, P, P, P, P, P, c_size_t, P, c_int]),
    "dlsh_init_dictionary": (c_int, [P, c_int64, c_int, P, c_int, P, P, c_int]),
    "dlsh_mlp_num_params": (ctypes.c_longlong, [c_int]),
    "dlsh_mlp_size": (c_size_t, [c_int]),
    "dlsh_mlp_workspace_size": (c_size_t, [c_int, c_int64]),
    "dlsh_mlp_init": (c_int, [P, c_int, P, P, c_int]),
    "dlsh_mlp_params": (c_int, [P, c_int, P, P, c_int]),
    "dlsh_mlp_forward": (c_int, [P, c_int, P, c_int64, P, P, c_size_t, P, c_int]),
    "dlsh_mlp_gradients": (c_int, [P, c_int, P, c_int64, P, P, c_int, P, P, P, c_size_t, P, c_int]),
    "dlsh_mlp_train_step": (c_int, [P, c_int, P, c_int64, P, P, c_int, c_float, c_int64, P, P,
                                    c_size_t, P, c_int]),
    "dlsh_mlp_train": (c_int, [P, c_int, P, c_int64, P, P, c_int, c_int, c_int64, c_float, P, P,
                               c_size_t, P, c_int]),
    "dlsh_mlp_propose_workspace_size": (c_size_t, [c_int, c_int64]),
    "dlsh_mlp_propose": (c_int, [P, c_int, P, c_int64, c_int, P, P, c_size_t, P, c_int]),
    "dlsh_encode_restricted": (c_int, [P, c_int, c_int, P, c_int64, P, c_int, c_int, c_float, P, P,
                                       P, P, P, c_size_t, P, c_int]),
    "dlsh_encode_learned_workspace_size": (c_size_t, [c_int, c_int, c_int, c_int64, c_int]),
    "dlsh_encode_learned": (c_int, [P, c_int, c_int, P, c_int64, c_int, c_float, P, c_int, c_int, c_float,
                                    c_int, P, P, P, P, P, P, c_size_t, P, c_int]),
    "dlsh_calibrate_fallback": (c_int, [P, P, c_int64, c_float, P, P]),
    "dlsh_encode_multi_workspace_size": (c_size_t, [P, c_int, c_int, c_int]),
    "dlsh_encode_multi": (c_int, [P, c_int, c_int, c_int, P, c_size_t, P, c_int]),
    "dlsh_autotune_encode": (c_int, [P, c_int, c_int, P, c_int64, c_int, c_int, P, P, P, P, P,
                                     c_size_t, P, P]),
    "dlsh_autotune_decode": (c_int, [P, c_int, c_int, P, P, c_int, P, c_int, c_int64, P, P, P, P, P, P]),
    "dlsh_tuned_encode": (c_int, [c_int, c_int, c_int]),
    "dlsh_tuned_decode": (c_int, [c_int, c_int, c_int, P, P]),
    "dlsh_csc_workspace_size": (c_size_t, [c_int64]),
    "dlsh_csc_from_ell": (c_int, [P, P, P, c_int64, c_int, P, P, P, P, c_size_t, P, c_int]),
    "dlsh_decode_compact_max_k": (c_size_t, [c_int]),
    "dlsh_compact_codes": (c_int, [P, P, c_int64, c_int, c_int, P, c_int, P, P, c_int]),
    "dlsh_decode_compact": (c_int, [P, c_int, c_int, P, c_int, P, P, c_int, c_int64, P, P, P, P, P,
                                    c_int]),
    "dlsh_ksvd_workspace_size": (c_size_t, [c_int, c_int, c_int, c_int64]),
    "dlsh_ksvd_update": (c_int, [P, c_int64, c_int, c_int, P, P, P, c_int, P, P, P, P, c_size_t, P, c_int]),
    "dlsh_preprocess_sh": (c_int, [P, P, P, P, P, c_int]),
    "dlsh_preprocess_codes": (c_int, [P, P, P, c_int, P, P, P, c_int, P, P, c_int]),
    "dlsh_preprocess_compact": (c_int, [P, P, P, c_int, P, c_int, P, P, c_int, P, P, c_int]),
    "dlsh_preprocess_max_k": (c_size_t, [c_int, c_int]),
    "dlsh_selftest_workspace_size": (c_size_t, []),
    "dlsh_selftest_bounded_wait": (c_int, [c_int, c_int64, P, c_size_t, P]),
}


def lib_path() -> str:
    return _build.SO_PATH


def lib() -> ctypes.CDLL:
    """The loaded library (built in-tree by `build()`); raises if unavailable."""
    global _LIB
    if _LIB is not None:
        return _LIB
    path = lib_path()
    if not os.path.exists(path):
        raise RuntimeError(f"{path} is missing: build it with __graft_entry__.build()")
    if not _build.is_current():
        raise RuntimeError(f"{path} is stale or built for another machine: rebuild it")
    L = ctypes.CDLL(path)
    for name, (res, args) in SIGNATURES.items():
        fn = getattr(L, name, None)
        if fn is None:
            continue
        fn.restype = res
        fn.argtypes = args
    _LIB = L
    return L


def last_error() -> str:
    return lib().dlsh_last_error().decode()

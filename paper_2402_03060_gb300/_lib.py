"""ctypes declarations of the C ABI in include/unihenn.h (same names, same arguments).

The shared library is built in-tree by ``paper_2402_03060_gb300.build`` (or
``__graft_entry__.build()``).  There is no fallback: if it is missing, loading
raises.
"""
from __future__ import annotations

import ctypes
import os

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "_build", "libunihenn.so")

HE_OK, HE_EINVAL, HE_ENOMEM, HE_ELEVEL, HE_ESCALE, HE_ESLOTS, HE_ENOKEY, HE_ECUDA, HE_ETIMEOUT, HE_EOVERFLOW = range(10)
STATUS_NAMES = ["HE_OK", "HE_EINVAL", "HE_ENOMEM", "HE_ELEVEL", "HE_ESCALE", "HE_ESLOTS", "HE_ENOKEY",
                "HE_ECUDA", "HE_ETIMEOUT", "HE_EOVERFLOW"]
HE_CONV2D, HE_CONV1D, HE_SQUARE, HE_AVGPOOL, HE_FLATTEN, HE_FC, HE_APPROX_RELU = 1, 2, 3, 4, 5, 6, 7
HE_SCHEDULE_FUSED, HE_SCHEDULE_LITERAL = 0, 1
SCHEDULES = {"fused": HE_SCHEDULE_FUSED, "literal": HE_SCHEDULE_LITERAL}


class he_params(ctypes.Structure):
    _fields_ = [("log2n", ctypes.c_uint32), ("n_data", ctypes.c_uint32), ("n_special", ctypes.c_uint32),
                ("prime_bits", ctypes.POINTER(ctypes.c_uint32)), ("dnum", ctypes.c_uint32),
                ("log2_scale", ctypes.c_double), ("seed", ctypes.c_uint64), ("device", ctypes.c_int),
                ("stream", ctypes.c_void_p)]


class he_layer(ctypes.Structure):
    _fields_ = [("op", ctypes.c_uint32), ("ch_in", ctypes.c_uint32), ("ch_out", ctypes.c_uint32),
                ("k", ctypes.c_uint32), ("stride", ctypes.c_uint32), ("w", ctypes.POINTER(ctypes.c_double)),
                ("b", ctypes.POINTER(ctypes.c_double))]


class he_kernel_stat(ctypes.Structure):
    _fields_ = [("name", ctypes.c_char * 32), ("launches", ctypes.c_uint64), ("total_ms", ctypes.c_double),
                ("bytes", ctypes.c_double), ("ops", ctypes.c_double)]


class he_server_opts(ctypes.Structure):
    _fields_ = [("max_batch", ctypes.c_uint32), ("max_wait_us", ctypes.c_uint32), ("mem_budget", ctypes.c_uint64),
                ("max_inflight", ctypes.c_uint32), ("exact_batches", ctypes.c_uint32)]


class he_server_stats(ctypes.Structure):
    _fields_ = [("requests", ctypes.c_uint64), ("batches", ctypes.c_uint64), ("cts", ctypes.c_uint64),
                ("mean_batch", ctypes.c_double), ("p50_ms", ctypes.c_double), ("p99_ms", ctypes.c_double),
                ("max_ms", ctypes.c_double), ("resident_bytes", ctypes.c_uint64)]


class HeError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__(f"{STATUS_NAMES[status] if 0 <= status < len(STATUS_NAMES) else status}: {msg}")
        self.status = status


_vp = ctypes.c_void_p
_u32, _u64, _i32, _int, _sz, _dbl = ctypes.c_uint32, ctypes.c_uint64, ctypes.c_int32, ctypes.c_int, ctypes.c_size_t, ctypes.c_double
_pp = ctypes.POINTER(ctypes.c_void_p)

SIGNATURES = {
    "he_context_create": (_int, [ctypes.POINTER(he_params), _pp]),
    "he_context_destroy": (None, [_vp]),
    "he_context_primes": (_int, [_vp, ctypes.POINTER(_u64), _sz]),
    "he_keygen": (_int, [_vp, ctypes.POINTER(_i32), _sz]),
    "he_keygen_pow2": (_int, [_vp]),
    "he_context_set_schedule": (_int, [_vp, _u32]),
    "he_encrypt": (_int, [_vp, _vp, _int, _u32, _u32, _u32, _u32, _u32, _u64, _pp]),
    "he_encrypt_channels": (_int, [_vp, _vp, _int, _u32, _u32, _u32, _u32, _u32, _u32, _u64, _pp]),
    "he_decrypt": (_int, [_vp, _vp, _vp, _int, _sz]),
    "he_ct_info": (_int, [_vp, ctypes.POINTER(_u32), ctypes.POINTER(_u32), ctypes.POINTER(_dbl)]),
    "he_ct_layout": (_int, [_vp, ctypes.POINTER(_u32), ctypes.POINTER(_u32), ctypes.POINTER(_u32)]),
    "he_ct_export": (_int, [_vp, _vp, ctypes.POINTER(_u64)]),
    "he_ct_free": (None, [_vp]),
    "he_rotate": (_int, [_vp, _vp, _i32, _pp]),
    "he_rotate_hoisted": (_int, [_vp, _vp, ctypes.POINTER(_i32), _sz, _pp]),
    "he_rescale": (_int, [_vp, _vp, _pp]),
    "he_pack": (_int, [_vp, _pp, _u32, _pp]),
    "he_drop_level": (_int, [_vp, _vp, _u32, _pp]),
    "he_mul_plain": (_int, [_vp, _vp, ctypes.POINTER(_dbl), _pp]),
    "he_add": (_int, [_vp, _vp, _vp, _pp]),
    "he_square": (_int, [_vp, _pp, _u32, _pp]),
    "he_approx_relu": (_int, [_vp, _pp, _u32, _pp]),
    "he_conv2d": (_int, [_vp, _pp, _u32, ctypes.POINTER(_dbl), ctypes.POINTER(_dbl), _u32, _u32, _u32, _int, _pp]),
    "he_conv1d": (_int, [_vp, _pp, _u32, ctypes.POINTER(_dbl), ctypes.POINTER(_dbl), _u32, _u32, _u32, _int, _pp]),
    "he_avgpool": (_int, [_vp, _pp, _u32, _u32, _pp]),
    "he_flatten": (_int, [_vp, _pp, _u32, _pp]),
    "he_fc": (_int, [_vp, _vp, ctypes.POINTER(_dbl), ctypes.POINTER(_dbl), _u32, _u32, _pp]),
    "he_model_plan": (_int, [ctypes.POINTER(he_layer), _sz, _u32, _u32, ctypes.POINTER(_u32), ctypes.POINTER(_u32),
                             ctypes.POINTER(_i32), ctypes.POINTER(_sz)]),
    "he_model_plan_schedule": (_int, [ctypes.POINTER(he_layer), _sz, _u32, _u32, _u32, ctypes.POINTER(_u32),
                                      ctypes.POINTER(_u32), ctypes.POINTER(_i32), ctypes.POINTER(_sz)]),
    "he_model_compile": (_int, [_vp, ctypes.POINTER(he_layer), _sz, _u32, _u32, _u32, _pp]),
    "he_infer": (_int, [_vp, _vp, _int, _pp]),
    "he_model_free": (None, [_vp]),
    "he_model_set_mask_budget": (_int, [_vp, _u64]),
    "he_ntt": (_int, [_vp, _vp, _u32, ctypes.POINTER(_u32), _int]),
    "he_rescale_noalloc": (_int, [_vp, _vp, _vp, _u32, _u32]),
    "he_sync": (_int, [_vp]),
    "he_kernel_launches": (_u64, [_vp]),
    "he_ubench": (_int, [_vp, ctypes.POINTER(_dbl)]),
    "he_profile_begin": (_int, [_vp]),
    "he_profile_end": (_int, [_vp, ctypes.POINTER(he_kernel_stat), _sz, ctypes.POINTER(_sz)]),
    "he_autotune": (_int, [_vp, ctypes.c_char_p, ctypes.c_char_p, _sz]),
    "he_tuning_get": (_int, [_vp, ctypes.POINTER(_i32), _sz]),
    "he_tuning_set": (_int, [_vp, ctypes.POINTER(_i32), _sz]),
    "he_server_create": (_int, [ctypes.POINTER(he_server_opts), _pp]),
    "he_server_add_model": (_int, [_vp, _vp, ctypes.POINTER(_u32)]),
    "he_server_submit": (_int, [_vp, _u32, _vp, ctypes.POINTER(_u64)]),
    "he_server_wait": (_int, [_vp, _u64, _u32, _pp, ctypes.POINTER(_dbl)]),
    "he_server_poll": (_int, [_vp, _u64, ctypes.POINTER(_int)]),
    "he_server_stats_get": (_int, [_vp, _i32, ctypes.POINTER(he_server_stats)]),
    "he_server_destroy": (None, [_vp]),
    "he_server_simulate": (_int, [ctypes.POINTER(he_server_opts), _u32, ctypes.POINTER(_dbl), ctypes.POINTER(_dbl),
                                  _sz, ctypes.POINTER(_dbl), ctypes.POINTER(_u32), ctypes.POINTER(_u32),
                                  ctypes.POINTER(_u64), ctypes.POINTER(_dbl)]),
    "he_server_simulate_admission": (_int, [ctypes.POINTER(he_server_opts), _u32, ctypes.POINTER(_dbl),
                                            ctypes.POINTER(_dbl), _sz, ctypes.POINTER(_dbl), ctypes.POINTER(_u32),
                                            ctypes.POINTER(_u32), ctypes.POINTER(_u64), ctypes.POINTER(_dbl),
                                            ctypes.POINTER(_u32)]),
    "he_last_error": (ctypes.c_char_p, []),
}

_LIB = None


def load(path: str = LIB_PATH):
    """Load libunihenn.so and declare every entry point; raises if it is missing."""
    global _LIB
    if _LIB is not None:
        return _LIB
    if not os.path.exists(path):
        raise RuntimeError(f"{path} is missing: build it with `python -m paper_2402_03060_gb300.build` "
                           "(or __graft_entry__.build()); there is no CPU fallback")
    lib = ctypes.CDLL(path)
    for name, (res, args) in SIGNATURES.items():
        f = getattr(lib, name)
        f.restype = res
        f.argtypes = args
    _LIB = lib
    return lib


def check(status: int):
    if status != HE_OK:
        msg = load().he_last_error()
        raise HeError(status, msg.decode() if msg else "")

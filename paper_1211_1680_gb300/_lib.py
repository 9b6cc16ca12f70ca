"""ctypes loader for libs2let_gpu.so (the C ABI declared in include/s2let_gpu.h).

The library must have been built (``paper_1211_1680_gb300.build.build()``);
there is no fallback: loading fails loudly when the extension is missing.
"""
import ctypes
import os

from . import build as _build

S2LET_OK = 0
S2LET_ERR_ARG = -1
S2LET_ERR_ALLOC = -2
S2LET_ERR_CUDA = -3
S2LET_ERR_TIMEOUT = -4
S2LET_ERR_UNSUPPORTED = -5

S2LET_REAL = 0x0
S2LET_COMPLEX = 0x1
S2LET_MULTIRES = 0x2
S2LET_PREC_FP64 = 0x00
S2LET_PREC_FP32 = 0x10
S2LET_PREC_TF32X3 = 0x20
S2LET_QUAD_FFT64 = 0x100
S2LET_TC_SPLIT3 = 0x200
S2LET_KERNEL_BSPLINE = 0x400
S2LET_QUAD_DENSE = 0x800
S2LET_LEG_RECURRENCE = 0x1000

# every symbol the header declares, with (restype, argtypes)
_vp = ctypes.c_void_p
_i = ctypes.c_int
_i64p = ctypes.POINTER(ctypes.c_int64)
_ip = ctypes.POINTER(ctypes.c_int)
# device-memory hook of s2let_set_allocator
ALLOC_FN = ctypes.CFUNCTYPE(ctypes.c_void_p, ctypes.c_size_t, ctypes.c_void_p)
FREE_FN = ctypes.CFUNCTYPE(None, ctypes.c_void_p, ctypes.c_void_p)
SIGNATURES = {
    "s2let_jmax": (_i, [_i, _i]),
    "s2let_plan_create": (_i, [ctypes.POINTER(_vp), _i, _i, _i, _i, _i]),
    "s2let_plan_destroy": (_i, [_vp]),
    "s2let_plan_info": (_i, [_vp, _ip, _ip, _i64p, _i64p, _ip]),
    "s2let_wav_layout": (_i, [_vp, _i, _ip, _i64p, _i64p]),
    "s2let_analysis": (_i, [_vp, _vp, _vp, _vp, _vp]),
    "s2let_synthesis": (_i, [_vp, _vp, _vp, _vp, _vp]),
    "s2let_adjoint": (_i, [_vp, _vp, _vp, _vp, _vp]),
    "s2let_sht_forward": (_i, [_vp, _vp, _vp, _vp]),
    "s2let_sht_inverse": (_i, [_vp, _vp, _vp, _vp]),
    "s2let_wav_scale": (_i, [_vp, _i, _vp, _vp, _vp]),
    "s2let_wav_scale_adjoint": (_i, [_vp, _i, _vp, _vp, _vp]),
    "s2let_sht_forward_adjoint": (_i, [_vp, _vp, _vp, _vp]),
    "s2let_plan_status": (_i, [_vp]),
    "s2let_plan_test_timeout": (_i, [_vp, _vp]),
    "s2let_plan_leg_table_bytes": (_i, [_vp, _i, ctypes.POINTER(ctypes.c_size_t)]),
    "s2let_set_allocator": (_i, [ALLOC_FN, FREE_FN, _vp]),
    "s2let_plan_autotune": (_i, [_vp, _vp]),
    "s2let_batch_autotune": (_i, [_vp, _vp]),
    "s2let_plan_tuning": (_i, [_vp, _i, ctypes.POINTER(_i), ctypes.POINTER(_i), ctypes.POINTER(_i),
                               ctypes.POINTER(_i)]),
    "s2let_plan_profile": (_i, [_vp, _i]),
    "s2let_plan_stage_stats": (_i, [_vp, _i, _i64p, _i64p, ctypes.POINTER(ctypes.c_double),
                                    ctypes.POINTER(ctypes.c_double), ctypes.POINTER(ctypes.c_double)]),
    "s2let_sht_inverse_noalloc": (_i, [_i, _i, _i, _vp, _vp, _vp]),
    "s2let_batch_create": (_i, [ctypes.POINTER(_vp), _i, _ip, _ip, _i, _i]),
    "s2let_batch_destroy": (_i, [_vp]),
    "s2let_batch_sizes": (_i, [_vp, _i64p, _i64p, _i64p, _ip]),
    "s2let_batch_map_layout": (_i, [_vp, _i, _i64p, _i64p, _ip, _ip]),
    "s2let_batch_group_plan": (_i, [_vp, _i, ctypes.POINTER(_vp), _i64p, _i64p, _i64p]),
    "s2let_batch_round_trip": (_i, [_vp, _vp, _vp, _vp, _vp, _vp]),
    "s2let_wav_bandlimits": (_i, [_i, _i, _i, _i, _ip, _ip, _i]),
    "s2let_wav_kernel": (_i, [_i, _i, _i, _i, _i, ctypes.POINTER(ctypes.c_double)]),
    "s2let_wav_noise_std": (_i, [_vp, _i, ctypes.POINTER(ctypes.c_double)]),
    "s2let_wav_threshold": (_i, [_vp, _vp, ctypes.c_double, ctypes.c_double, _vp]),
    "s2let_strerror": (ctypes.c_char_p, [_i]),
}

STAGES = ["ring_fwd", "theta_quad", "leg_anal", "leg_synth", "ring_inv", "pack"]

_lib = None


class S2letError(RuntimeError):
    def __init__(self, name, status):
        msg = "%s failed: %s (%d)" % (name, lib().s2let_strerror(status).decode(), status)
        super().__init__(msg)
        self.status = status


def lib():
    """Load (building first if needed) and return the ctypes library."""
    global _lib
    if _lib is None:
        path = _build.LIB
        if not _build.up_to_date():
            _build.build()
        if not os.path.exists(path):
            raise RuntimeError("libs2let_gpu.so is missing; build it with paper_1211_1680_gb300.build")
        L = ctypes.CDLL(path)
        for name, (res, args) in SIGNATURES.items():
            fn = getattr(L, name)
            fn.restype = res
            fn.argtypes = args
        _lib = L
    return _lib


def check(name, status):
    if status != S2LET_OK:
        raise S2letError(name, status)
    return status

"""ctypes declarations of the C ABI in ``include/trtrlb.h``.

Loading fails loudly when ``libtrtrlb.so`` has not been built: there is no
CPU fallback behind this binding.
"""
from __future__ import annotations

import ctypes as C
import os

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libtrtrlb.so")

OK, EINVAL, ENOMEM, ECUDA, EUNSTABLE, ETIMEOUT, ENOTSUP = 0, -1, -2, -3, -4, -5, -6
F64, F32, F16_SHIFTED, BF16_SHIFTED, F64_DW = 0, 1, 2, 3, 4
G_LAGGED, G_CURRENT, G_OFF = 0, 1, 2
FLUID, SOLID, INLET, OUTLET = 0, 1, 2, 3
KERNEL_AUTO, KERNEL_SCALAR, KERNEL_VECTOR, KERNEL_COLUMN = 0, 1, 2, 3
# trtrlb_step_kernel kinds, by position
STEP_KINDS = ("aa", "aa_vector", "ab", "ab_tma", "ab_tma_shared", "ab_column")
CMP_N = 10      # outputs of trtrlb_compare / trtrlb_compare_lattices

# every function the header declares, with (restype, argtypes)
_vp, _dp, _i64 = C.c_void_p, C.c_void_p, C.c_int64


class Params(C.Structure):
    """Mirror of ``trtrlb_params``."""
    _fields_ = [
        ("nx", C.c_int32), ("ny", C.c_int32),
        ("periodic_x", C.c_int32), ("periodic_y", C.c_int32),
        ("tau_s", C.c_double), ("tau_s2", C.c_double), ("magic", C.c_double),
        ("gx", C.c_double), ("gy", C.c_double),
        ("rho0", C.c_double),
        ("wall_ux", C.c_double), ("wall_uy", C.c_double), ("wall_rho", C.c_double),
        ("outlet_rho", C.c_double),
        ("storage", C.c_int32), ("g_mode", C.c_int32),
    ]


SIGNATURES = {
    "trtrlb_default_params": (None, [C.POINTER(Params)]),
    "trtrlb_create": (C.c_int, [C.POINTER(Params), _vp, _vp, C.POINTER(_vp)]),
    "trtrlb_destroy": (C.c_int, [_vp]),
    "trtrlb_set_stream": (C.c_int, [_vp, _vp]),
    "trtrlb_init": (C.c_int, [_vp, _dp, _dp, _dp]),
    "trtrlb_step": (C.c_int, [_vp, _i64]),
    "trtrlb_moments": (C.c_int, [_vp, _dp, _dp, _dp]),
    "trtrlb_get_f": (C.c_int, [_vp, _dp, _dp]),
    "trtrlb_set_f": (C.c_int, [_vp, _dp, _dp]),
    "trtrlb_time": (C.c_int64, [_vp]),
    "trtrlb_diagnostics": (C.c_int, [_vp, _dp]),
    "trtrlb_compare": (C.c_int, [_vp, _dp, _dp, _dp]),
    "trtrlb_compare_lattices": (C.c_int, [_vp, _vp, _dp]),
    "trtrlb_diagnostics_noalloc": (C.c_int, [_dp, _vp, C.c_int32, C.c_int32, C.c_int32, C.c_int32,
                                             C.c_double, C.c_double, _dp, _vp]),
    "trtrlb_device_bytes": (C.c_int64, [_vp]),
    "trtrlb_set_kernel": (C.c_int, [_vp, C.c_int32, C.c_int32]),
    "trtrlb_get_kernel": (C.c_int, [_vp, C.POINTER(C.c_int32), C.POINTER(C.c_int32)]),
    "trtrlb_step_kernel": (C.c_int, [_vp, C.POINTER(C.c_int32)]),
    "trtrlb_set_wait_limit": (C.c_int, [_vp, _i64]),
    "trtrlb_state_bytes": (C.c_int64, [_vp]),
    "trtrlb_save": (C.c_int, [_vp, _vp]),
    "trtrlb_load": (C.c_int, [_vp, _vp]),
    "trtrlb_batch_create": (C.c_int, [_vp, C.POINTER(_vp)]),
    "trtrlb_batch_set": (C.c_int, [_vp, C.POINTER(_vp), C.c_int]),
    "trtrlb_batch_step": (C.c_int, [_vp, _i64]),
    "trtrlb_batch_solve": (C.c_int, [_vp, C.POINTER(_vp), C.POINTER(_vp), C.POINTER(_vp), _i64,
                                     C.POINTER(_vp), C.POINTER(_vp), C.POINTER(_vp)]),
    "trtrlb_batch_destroy": (C.c_int, [_vp]),
    "trtrlb_batch_last_error": (C.c_char_p, [_vp]),
    "trtrlb_slabs_create": (C.c_int, [C.POINTER(Params), _vp, C.c_int32, _vp, C.POINTER(_vp)]),
    "trtrlb_slabs_destroy": (C.c_int, [_vp]),
    "trtrlb_slabs_init": (C.c_int, [_vp, _dp, _dp, _dp]),
    "trtrlb_slabs_step": (C.c_int, [_vp, _i64]),
    "trtrlb_slabs_get_f": (C.c_int, [_vp, _dp]),
    "trtrlb_slabs_moments": (C.c_int, [_vp, _dp, _dp, _dp]),
    "trtrlb_slabs_diagnostics": (C.c_int, [_vp, _dp]),
    "trtrlb_slabs_count": (C.c_int32, [_vp]),
    "trtrlb_slabs_slab": (C.c_int, [_vp, C.c_int32, C.POINTER(_vp), C.POINTER(C.c_int32),
                                    C.POINTER(C.c_int32), C.POINTER(C.c_int32)]),
    "trtrlb_slabs_last_error": (C.c_char_p, [_vp]),
    "trtrlb_fp64_fma_rate": (C.c_int, [_vp, C.c_double, C.POINTER(C.c_double)]),
    "trtrlb_strerror": (C.c_char_p, [C.c_int]),
    "trtrlb_last_error": (C.c_char_p, [_vp]),
}

_LIB = None


class TrtrlbError(RuntimeError):
    def __init__(self, code: int, msg: str):
        super().__init__(f"{msg} (code {code})")
        self.code = code


def load() -> C.CDLL:
    """Loads libtrtrlb.so (built by ``__graft_entry__.build()``)."""
    global _LIB
    if _LIB is None:
        if not os.path.exists(LIB_PATH):
            raise ImportError(f"{LIB_PATH} is missing: build the CUDA library first "
                              "(python -c 'import __graft_entry__ as g; g.build()')")
        import torch  # noqa: F401  (loads the CUDA runtime the library links against)
        lib = C.CDLL(LIB_PATH)
        for name, (res, args) in SIGNATURES.items():
            fn = getattr(lib, name)
            fn.restype = res
            fn.argtypes = args
        _LIB = lib
    return _LIB


def check(rc: int, handle=None):
    if rc != OK:
        lib = load()
        msg = lib.trtrlb_last_error(handle)
        text = msg.decode() if msg else ""
        raise TrtrlbError(rc, f"{lib.trtrlb_strerror(rc).decode()}: {text}")
    return rc

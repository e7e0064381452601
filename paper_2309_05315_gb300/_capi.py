"""ctypes declarations of the C ABI in include/mam.h (marshalling only).

Every computation happens in libmam.so; this module only loads it and
describes its structs and signatures.  Loading fails loudly when the library
has not been built: there is no fallback implementation.
"""
from __future__ import annotations

import ctypes as C
import os

_PKG = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_PKG, "libmam.so")

MAM_OK = 0
STATUS = {0: "MAM_OK", 1: "MAM_ERR_INVALID_ARG", 2: "MAM_ERR_CUDA", 3: "MAM_ERR_OOM",
          4: "MAM_ERR_NONFINITE", 5: "MAM_ERR_TIMEOUT", 6: "MAM_ERR_STATE",
          7: "MAM_ERR_UNSUPPORTED", 8: "MAM_ERR_COMM", 9: "MAM_ERR_CAPACITY"}
COST_DTYPES = {"f32": 0, "bf16": 1, "f16": 2}
DIAG_MODES = {"last": 0, "never": 1, "every": 2}
COST_LAYOUTS = {"per_column": 0, "shared": 1, "generated": 2}
PLAN_LAYOUTS = {"dense": 0, "sparse": 1}


class MamDesc(C.Structure):
    _fields_ = [("M", C.c_int32), ("R", C.c_int32), ("dim", C.c_int32),
                ("S", C.POINTER(C.c_int32)),
                ("zeta", C.POINTER(C.c_double)),
                ("q", C.POINTER(C.c_double)),
                ("alpha", C.POINTER(C.c_double)),
                ("xi", C.POINTER(C.c_double)),
                ("cost", C.POINTER(C.c_double)),
                ("rho", C.c_double), ("gamma", C.c_double),
                ("n_bundles", C.c_int32), ("seed", C.c_uint64),
                ("cost_dtype", C.c_int32), ("theta0_mode", C.c_int32),
                ("diag_mode", C.c_int32), ("stream", C.c_void_p),
                ("eta", C.c_double), ("capped", C.c_int32),
                ("cost_layout", C.c_int32), ("plan_layout", C.c_int32),
                ("sparse_slots", C.c_int32)]


# int32 allreduce(void* buf, int64 count, int32 dtype, void* stream, void* user)
ALLREDUCE_FN = C.CFUNCTYPE(C.c_int32, C.c_void_p, C.c_int64, C.c_int32, C.c_void_p,
                           C.c_void_p)
SUM_I64, SUM_F64 = 0, 1


class MamShard(C.Structure):
    _fields_ = [("m_begin", C.c_int32), ("m_end", C.c_int32),
                ("allreduce", ALLREDUCE_FN), ("user", C.c_void_p)]


class MamObjective(C.Structure):
    _fields_ = [("w_hat", C.c_double), ("dist_pihat", C.c_double),
                ("lower_bound", C.c_double), ("f_unbal", C.c_double),
                ("fp_resid", C.c_double), ("dp_norm", C.c_double),
                ("t", C.c_double), ("dist_theta", C.c_double),
                ("t_next", C.c_double),
                ("iter", C.c_int64), ("newton_passes", C.c_int64)]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


class MamKernelConfig(C.Structure):
    _fields_ = [("threads", C.c_int32), ("vec", C.c_int32), ("stages", C.c_int32),
                ("ctas_per_sm", C.c_int32), ("bisect_depth", C.c_int32),
                ("kind", C.c_int32)]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


class MamError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__(f"{STATUS.get(status, status)}: {msg}")
        self.status = status


_lib = None

# name -> (restype, argtypes); the names are the C ABI's.
_SIGS = {
    "mam_create": (C.c_int, [C.POINTER(MamDesc), C.POINTER(C.c_void_p)]),
    "mam_batch_create": (C.c_int, [C.c_int32, C.POINTER(MamDesc), C.POINTER(C.c_void_p)]),
    "mam_step": (C.c_int, [C.c_void_p, C.c_int32]),
    "mam_solve": (C.c_int, [C.c_void_p, C.c_int32, C.c_double, C.c_double, C.c_int32,
                            C.POINTER(C.c_int32), C.POINTER(C.c_double)]),
    "mam_objective": (C.c_int, [C.c_void_p, C.c_int32, C.POINTER(MamObjective)]),
    "mam_objective_all": (C.c_int, [C.c_void_p, C.POINTER(MamObjective)]),
    "mam_get_barycenter": (C.c_int, [C.c_void_p, C.c_void_p, C.c_int32]),
    "mam_update_support": (C.c_int, [C.c_void_p, C.c_void_p]),
    "mam_free_support": (C.c_int, [C.c_void_p, C.c_int32, C.c_int32, C.c_double, C.c_int32,
                                   C.c_void_p, C.c_void_p]),
    "mam_selftest_wait_timeout": (C.c_int, [C.c_int32]),
    "mam_create_sharded": (C.c_int, [C.POINTER(MamDesc), C.POINTER(MamShard),
                                     C.POINTER(C.c_void_p)]),
    "mam_get_theta": (C.c_int, [C.c_void_p, C.c_void_p]),
    "mam_get_theta_range": (C.c_int, [C.c_void_p, C.c_int64, C.c_int64, C.c_void_p]),
    "mam_get_work": (C.c_int, [C.c_void_p, C.POINTER(C.c_int64), C.POINTER(C.c_int64)]),
    "mam_get_marginals": (C.c_int, [C.c_void_p, C.c_void_p, C.c_int32]),
    "mam_get_sizes": (C.c_int, [C.c_void_p, C.POINTER(C.c_int32), C.POINTER(C.c_int32),
                                C.POINTER(C.c_int32), C.POINTER(C.c_int64),
                                C.POINTER(C.c_int32)]),
    "mam_get_pruned_sizes": (C.c_int, [C.c_void_p, C.c_void_p]),
    "mam_get_state": (C.c_int, [C.c_void_p, C.c_void_p, C.POINTER(C.c_size_t)]),
    "mam_set_state": (C.c_int, [C.c_void_p, C.c_void_p, C.c_size_t]),
    "mam_forward_record": (C.c_int, [C.c_void_p, C.c_int32, C.c_int32]),
    "mam_backward": (C.c_int, [C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p]),
    "mam_get_config": (C.c_int, [C.c_void_p, C.POINTER(MamKernelConfig)]),
    "mam_set_config": (C.c_int, [C.c_void_p, C.POINTER(MamKernelConfig)]),
    "mam_autotune": (C.c_int, [C.c_void_p, C.c_int32, C.POINTER(MamKernelConfig)]),
    "mam_profile_enable": (C.c_int, [C.c_void_p, C.c_int32]),
    "mam_profile_read": (C.c_int, [C.c_void_p, C.POINTER(C.c_double), C.POINTER(C.c_double),
                                   C.POINTER(C.c_int64)]),
    "mam_column_update_noalloc": (C.c_int, [C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p,
                                            C.c_int32, C.c_int32, C.c_int32, C.c_double,
                                            C.c_double, C.c_void_p, C.c_void_p]),
    "mam_last_error": (C.c_char_p, [C.c_void_p]),
    "mam_destroy": (None, [C.c_void_p]),
}


def exported_names():
    return list(_SIGS)


def lib():
    """Load libmam.so (raises if it has not been built)."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise ImportError(
                f"{LIB_PATH} is missing: build it with "
                "`python -c 'import __graft_entry__ as g; g.build()'` "
                "(the library has no CPU fallback)")
        L = C.CDLL(LIB_PATH)
        for name, (res, args) in _SIGS.items():
            fn = getattr(L, name)
            fn.restype = res
            fn.argtypes = args
        _lib = L
    return _lib


def check(status, handle=None):
    if status != MAM_OK:
        msg = lib().mam_last_error(handle)
        raise MamError(status, msg.decode() if msg else "")

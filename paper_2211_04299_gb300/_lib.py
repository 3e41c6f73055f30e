"""ctypes declarations of libmdpgpu's C ABI (include/mdpgpu.h).

Loading fails loudly when the shared library has not been built: there is no CPU path.
"""
from __future__ import annotations

import ctypes as C
import os

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libmdpgpu.so")

MDP_OK, MDP_EINVAL, MDP_ENOMEM, MDP_ENOCONV, MDP_EDEVICE, MDP_ETIMEOUT = 0, -1, -2, -3, -4, -5
MDP_F32, MDP_F64 = 0, 1
MDP_PREC_FP64, MDP_PREC_MIXED = 0, 1
MDP_FLAG_HOST_LOOP = 1
MDP_FLAG_NO_WINDOW = 2
MDP_FLAG_PC_REBUILD = 4

STATUS_NAMES = {0: "ok", -1: "einval", -2: "enomem", -3: "enoconv", -4: "edevice",
                -5: "etimeout", 1: "breakdown"}


class mdp_opts(C.Structure):
    _fields_ = [("alpha", C.c_double), ("tol", C.c_double), ("restart", C.c_int32),
                ("max_outer", C.c_int32), ("max_inner", C.c_int32), ("precision", C.c_int32),
                ("opi_W", C.c_int32), ("pi_inner_tol_exp", C.c_int32), ("flags", C.c_int32),
                ("v0", C.POINTER(C.c_double)), ("forcing_c", C.c_double),
                ("precond_block", C.c_int32)]


class mdp_server_opts(C.Structure):
    _fields_ = [("hbm_budget_bytes", C.c_int64), ("max_slots", C.c_int32),
                ("iters_per_launch", C.c_int32), ("solver", mdp_opts)]


class mdp_stats(C.Structure):
    _fields_ = [("outer", C.c_int32), ("inner", C.c_int32), ("restarts", C.c_int32),
                ("sweeps", C.c_int32), ("matvecs", C.c_int32), ("status", C.c_int32),
                ("residual_inf", C.c_double), ("seconds", C.c_double), ("bytes", C.c_double),
                ("sweep_ms", C.c_double), ("matvec_ms", C.c_double),
                ("timed_sweeps", C.c_int32), ("timed_matvecs", C.c_int32),
                ("launches", C.c_int32), ("breakdowns", C.c_int32)]

    def as_dict(self):
        return {f: getattr(self, f) for f, _ in self._fields_}


# host collectives of the row-sharded solve (include/mdpgpu.h: mdp_allgather_fn, mdp_allreduce_fn)
ALLGATHER_FN = C.CFUNCTYPE(C.c_int, C.c_void_p, C.c_void_p, C.c_void_p, C.c_int64)
ALLREDUCE_FN = C.CFUNCTYPE(C.c_int, C.c_void_p, C.POINTER(C.c_double), C.c_int32, C.c_int32)


class mdp_comm(C.Structure):
    _fields_ = [("ctx", C.c_void_p), ("rank", C.c_int32), ("world", C.c_int32),
                ("row_begin", C.POINTER(C.c_int64)), ("allgather", ALLGATHER_FN),
                ("allreduce", ALLREDUCE_FN)]


_vp = C.c_void_p
_dp = C.POINTER(C.c_double)
_ip = C.POINTER(C.c_int32)
_h = C.c_void_p

# name -> (restype, argtypes); every symbol include/mdpgpu.h declares
SIGNATURES = {
    "mdp_precond_coarse_inverse": (C.c_int, [_h, _vp, C.c_int32, _vp, C.POINTER(C.c_int64), _ip]),
    "mdp_shard_create": (C.c_int, [C.c_int64, C.c_int64, C.c_int64, C.c_int32, C.c_int32, _vp, _vp, C.c_int, _vp, C.c_double, C.POINTER(_h)]),
    "mdp_shard_destroy": (None, [_h]),
    "ipi_solve_sharded": (C.c_int, [_h, C.POINTER(mdp_comm), C.POINTER(mdp_opts), _vp, _vp, C.POINTER(mdp_stats)]),
    "mdp_selftest_wait": (C.c_int, [C.c_int64, C.c_int32]),
    "mdp_probe_alu": (C.c_int, [C.c_int32, _dp]),
    "mdp_create_dense": (C.c_int, [C.c_int64, C.c_int32, _vp, C.c_int, _vp, C.c_double, _vp, C.POINTER(_h)]),
    "mdp_create_ell": (C.c_int, [C.c_int64, C.c_int32, C.c_int32, _vp, _vp, C.c_int, _vp, C.c_double, _vp, C.POINTER(_h)]),
    "mdp_create_dense_dev": (C.c_int, [C.c_int64, C.c_int32, _vp, C.c_int, _vp, C.c_double, _vp, C.POINTER(_h)]),
    "mdp_create_ell_dev": (C.c_int, [C.c_int64, C.c_int32, C.c_int32, _vp, _vp, C.c_int, _vp, C.c_double, _vp, C.POINTER(_h)]),
    "mdp_load_dense": (C.c_int, [_h, _vp, _vp]),
    "mdp_load_ell": (C.c_int, [_h, _vp, _vp, _vp]),
    "mdp_load_dense_async": (C.c_int, [_h, _vp, _vp]),
    "mdp_load_ell_async": (C.c_int, [_h, _vp, _vp, _vp]),
    "mdp_destroy": (None, [_h]),
    "mdp_set_stream": (C.c_int, [_h, _vp]),
    "mdp_info": (C.c_int, [_h, C.POINTER(C.c_int64), _ip, _ip, _ip, _ip, _dp]),
    "mdp_device_bytes": (C.c_int64, [_h]),
    "mdp_opts_default": (mdp_opts, []),
    "mdp_set_timing": (C.c_int, [_h, C.c_int]),
    "mdp_set_tuning": (C.c_int, [_h, C.c_int32, C.c_int32]),
    "mdp_set_geometry": (C.c_int, [_h, C.c_int32, C.c_int32, C.c_int32]),
    "mdp_batch_create": (C.c_int, [C.POINTER(_h), C.c_int32, C.POINTER(mdp_opts), C.POINTER(_h)]),
    "mdp_batch_destroy": (None, [_h]),
    "mdp_batch_set_stream": (C.c_int, [_h, _vp]),
    "mdp_batch_tune": (C.c_int, [_h]),
    "mdp_batch_geometry": (C.c_int, [_h, C.c_int32, _ip, _ip, _ip, _ip, _ip]),
    "mdp_batch_device_bytes": (C.c_int64, [_h]),
    "mdp_batch_bellman": (C.c_int, [_h, _vp]),
    "mdp_batch_solve": (C.c_int, [_h, C.POINTER(_vp), C.POINTER(_vp), C.POINTER(mdp_stats)]),
    "mdp_batch_solve_dev": (C.c_int, [_h, C.POINTER(_vp), C.POINTER(_vp), C.POINTER(mdp_stats)]),
    "ipi_solve_batch": (C.c_int, [C.POINTER(_h), C.c_int32, C.POINTER(mdp_opts), C.POINTER(_vp), C.POINTER(_vp), C.POINTER(mdp_stats)]),
    "bellman_apply": (C.c_int, [_h, _vp, _vp, _vp, _vp, C.c_int32]),
    "bellman_apply_dev": (C.c_int, [_h, _vp, _vp, _vp, _vp, _vp, C.c_int32]),
    "bellman_apply_ell_noalloc_dev": (C.c_int, [C.c_int64, C.c_int32, C.c_int32, _vp, _vp, _vp, C.c_double, _vp, _vp, _vp, _vp, _vp]),
    "policy_eval_gmres": (C.c_int, [_h, _vp, _vp, C.c_double, C.POINTER(mdp_opts), _vp, C.POINTER(mdp_stats)]),
    "policy_eval_gmres_dev": (C.c_int, [_h, _vp, _vp, C.c_double, C.POINTER(mdp_opts), _vp, C.POINTER(mdp_stats)]),
    "ipi_solve": (C.c_int, [_h, C.POINTER(mdp_opts), _vp, _vp, C.POINTER(mdp_stats)]),
    "ipi_solve_dev": (C.c_int, [_h, C.POINTER(mdp_opts), _vp, _vp, C.POINTER(mdp_stats)]),
    "vi_solve": (C.c_int, [_h, C.POINTER(mdp_opts), _vp, _vp, C.POINTER(mdp_stats)]),
    "vi_solve_dev": (C.c_int, [_h, C.POINTER(mdp_opts), _vp, _vp, C.POINTER(mdp_stats)]),
    "pi_solve": (C.c_int, [_h, C.POINTER(mdp_opts), _vp, _vp, C.POINTER(mdp_stats)]),
    "pi_solve_dev": (C.c_int, [_h, C.POINTER(mdp_opts), _vp, _vp, C.POINTER(mdp_stats)]),
    "opi_solve": (C.c_int, [_h, C.POINTER(mdp_opts), _vp, _vp, C.POINTER(mdp_stats)]),
    "opi_solve_dev": (C.c_int, [_h, C.POINTER(mdp_opts), _vp, _vp, C.POINTER(mdp_stats)]),
    "ipi_vi_solve": (C.c_int, [_h, C.POINTER(mdp_opts), _vp, _vp, C.POINTER(mdp_stats)]),
    "ipi_vi_solve_dev": (C.c_int, [_h, C.POINTER(mdp_opts), _vp, _vp, C.POINTER(mdp_stats)]),
    "mdp_server_opts_default": (mdp_server_opts, []),
    "mdp_server_create": (C.c_int, [C.POINTER(mdp_server_opts), C.POINTER(_h)]),
    "mdp_server_destroy": (None, [_h]),
    "mdp_server_submit": (C.c_int, [_h, C.c_int64, C.c_int32, C.c_int32, _vp, _vp, _vp, C.c_double, _vp, _vp, C.POINTER(C.c_int64)]),
    "mdp_server_poll": (C.c_int, [_h, C.POINTER(C.c_int64), C.POINTER(mdp_stats), C.c_int32, _ip]),
    "mdp_server_drain": (C.c_int, [_h]),
    "mdp_server_info": (C.c_int, [_h, _ip, _ip, C.POINTER(C.c_int64), C.POINTER(C.c_int64)]),
    "mdp_last_error": (C.c_char_p, []),
    "mdp_version": (C.c_char_p, []),
}

_LIB = None


def load(path: str | None = None):
    """Load libmdpgpu.so (built in-tree by build.py); raises if it is missing."""
    global _LIB
    if _LIB is not None:
        return _LIB
    p = path or LIB_PATH
    if not os.path.exists(p):
        raise ImportError(f"libmdpgpu.so is not built ({p}); run paper_2211_04299_gb300/build.py "
                          "(needs nvcc) -- there is no CPU fallback")
    lib = C.CDLL(p)
    for name, (res, args) in SIGNATURES.items():
        fn = getattr(lib, name)
        fn.restype = res
        fn.argtypes = args
    _LIB = lib
    return lib


class MDPError(RuntimeError):
    def __init__(self, code, where):
        msg = load().mdp_last_error().decode(errors="replace")
        super().__init__(f"{where}: {STATUS_NAMES.get(code, code)} ({code}): {msg}")
        self.code = code

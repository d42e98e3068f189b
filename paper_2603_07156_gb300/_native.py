"""ctypes declarations of the C ABI in include/ibsn.h (argument marshalling only).

Loading fails loudly when the library has not been built: there is no
fallback implementation.
"""

from __future__ import annotations

import ctypes as C
import os
import re

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libibsn_gb300.so")
HEADER = os.path.join(os.path.dirname(HERE), "include", "ibsn.h")

c_double_p = C.POINTER(C.c_double)


class IbsnProblem(C.Structure):
    _fields_ = [
        ("m", C.c_int64), ("n", C.c_int64), ("ldc", C.c_int64),
        ("C", C.c_void_p), ("a", C.c_void_p), ("b", C.c_void_p),
        ("eta", C.c_double), ("cost_scale", C.c_double),
        ("cost_kind", C.c_int32), ("grid_h", C.c_int32), ("grid_w", C.c_int32), ("dim", C.c_int32),
        ("x", C.c_void_p), ("y", C.c_void_p),
    ]


class IbsnParams(C.Structure):
    _fields_ = [
        ("sigma", C.c_double), ("beta", C.c_double), ("sinkhorn_tol", C.c_double),
        ("mu0", C.c_double), ("mu_min", C.c_double), ("gap_tol", C.c_double),
        ("cg_rtol", C.c_double), ("cg_rtol_floor_mixed", C.c_double), ("polish_gap", C.c_double),
        ("wait_timeout_s", C.c_double), ("gamma0", C.c_void_p), ("nnz_cap", C.c_int64),
        ("max_outer", C.c_int32), ("max_newton", C.c_int32), ("max_cg", C.c_int32),
        ("max_sinkhorn", C.c_int32), ("max_armijo", C.c_int32), ("precision", C.c_int32),
        ("polish", C.c_int32), ("sparsify", C.c_int32), ("verbose", C.c_int32), ("profile", C.c_int32),
        ("eot_gtol", C.c_double), ("eot", C.c_int32), ("recompute", C.c_int32),
    ]


class IbsnResult(C.Structure):
    _fields_ = [
        ("gamma", C.c_void_p), ("zeta", C.c_void_p), ("plan", C.c_void_p),
        ("primal", C.c_double), ("dual", C.c_double), ("rel_gap", C.c_double), ("kkt", C.c_double),
        ("marg_viol", C.c_double), ("grad_norm", C.c_double), ("seconds", C.c_double),
        ("outer_iters", C.c_int32), ("newton_iters", C.c_int32), ("cg_iters", C.c_int32),
        ("sinkhorn_iters", C.c_int32), ("armijo_trials", C.c_int32), ("polish_outer", C.c_int32),
        ("reanchors", C.c_int32), ("status", C.c_int32),
        ("max_nnz", C.c_int64), ("dense_passes", C.c_int64), ("kernel_launches", C.c_int64),
        ("pass_ms", C.c_double * 16), ("pass_calls", C.c_int64 * 16), ("pass_bytes", C.c_double * 16),
    ]

class IbsnWsBatch(C.Structure):
    _fields_ = [
        ("count", C.c_int32), ("reserved_", C.c_int32),
        ("m", C.POINTER(C.c_int64)), ("n", C.POINTER(C.c_int64)),
        ("x", C.c_void_p), ("y", C.c_void_p), ("a", C.c_void_p), ("b", C.c_void_p),
    ]


class IbsnWsAdam(C.Structure):
    _fields_ = [("lr", C.c_double), ("beta1", C.c_double), ("beta2", C.c_double), ("eps", C.c_double)]


PASS_KINDS = ["plan", "armijo", "stop", "sparsify", "certify", "anchor", "pcg", "vector"]


_SIGS = {
    "ibsn_status_string": (C.c_char_p, [C.c_int]),
    "ibsn_last_cuda_error": (C.c_char_p, []),
    "ibsn_params_default": (None, [C.POINTER(IbsnParams)]),
    "ibsn_workspace_size": (C.c_int, [C.POINTER(IbsnProblem), C.POINTER(IbsnParams), C.POINTER(C.c_size_t)]),
    "ibsn_solve": (C.c_int, [C.POINTER(IbsnProblem), C.POINTER(IbsnParams), C.c_void_p, C.c_size_t,
                             C.POINTER(IbsnResult), C.c_void_p]),
    "ibsn_solve_batch": (C.c_int, [C.c_int, C.POINTER(IbsnProblem), C.POINTER(IbsnParams), C.POINTER(C.c_void_p),
                                   C.POINTER(C.c_size_t), C.POINTER(IbsnResult), C.POINTER(C.c_void_p), C.c_int]),
    "ibsn_ws_param_count": (C.c_int64, []),
    "ibsn_ws_adam_default": (None, [C.POINTER(IbsnWsAdam)]),
    "ibsn_ws_workspace_size": (C.c_int, [C.POINTER(IbsnWsBatch), C.POINTER(C.c_size_t)]),
    "ibsn_ws_predict": (C.c_int, [C.POINTER(IbsnWsBatch), C.c_void_p, C.c_void_p, C.c_void_p, C.c_size_t,
                                  C.c_void_p]),
    "ibsn_ws_loss_grad": (C.c_int, [C.POINTER(IbsnWsBatch), C.c_void_p, C.c_void_p, c_double_p, C.c_void_p,
                                    C.c_void_p, C.c_void_p, C.c_size_t, C.c_void_p]),
    "ibsn_ws_adam_step": (C.c_int, [C.c_int64, C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p, C.c_int64,
                                    C.POINTER(IbsnWsAdam), C.c_void_p]),
    "ibsn_judge_warm_start": (C.c_int, [C.POINTER(IbsnProblem), C.POINTER(IbsnParams), C.c_void_p, C.c_void_p,
                                        C.c_void_p, C.c_size_t, c_double_p, c_double_p, c_double_p, c_double_p,
                                        C.POINTER(C.c_int32), C.c_void_p]),
    "ibsn_ctx_create": (C.c_int, [C.POINTER(IbsnProblem), C.POINTER(IbsnParams), C.c_void_p, C.c_size_t,
                                  C.c_void_p, C.POINTER(C.c_void_p)]),
    "ibsn_ctx_destroy": (C.c_int, [C.c_void_p]),
    "ibsn_ctx_set_state": (C.c_int, [C.c_void_p, C.c_int64, C.c_void_p, C.c_void_p, C.c_int]),
    "ibsn_ctx_plan": (C.c_int, [C.c_void_p, C.c_void_p, c_double_p]),
    "ibsn_ctx_export_plan": (C.c_int, [C.c_void_p, C.c_void_p]),
    "ibsn_ctx_get_gamma": (C.c_int, [C.c_void_p, C.c_void_p]),
    "ibsn_ctx_sinkhorn": (C.c_int, [C.c_void_p, C.c_double, C.c_int32, C.POINTER(C.c_int32), c_double_p]),
    "ibsn_ctx_sparsify": (C.c_int, [C.c_void_p, C.c_double, C.POINTER(C.c_int64)]),
    "ibsn_ctx_export_sparse": (C.c_int, [C.c_void_p, C.c_void_p]),
    "ibsn_ctx_newton_direction": (C.c_int, [C.c_void_p, C.c_double, C.c_double, C.c_int32, C.c_void_p,
                                            C.POINTER(C.c_int32), c_double_p]),
    "ibsn_ctx_armijo_trial": (C.c_int, [C.c_void_p, C.c_double, C.c_int32, c_double_p, c_double_p,
                                        C.POINTER(C.c_int32)]),
    "ibsn_ctx_stop_check": (C.c_int, [C.c_void_p, c_double_p]),
    "ibsn_ctx_certify": (C.c_int, [C.c_void_p, c_double_p, c_double_p, c_double_p, c_double_p, C.c_void_p,
                                   C.c_void_p]),
    "ibsn_wait_probe": (C.c_int, [C.c_int, C.c_int, C.c_double, C.c_void_p, C.c_void_p]),
    "ibsn_plan_pass_noalloc": (C.c_int, [C.POINTER(IbsnProblem), C.c_int64, C.c_void_p, C.c_void_p, C.c_void_p,
                                         c_double_p, C.c_void_p]),
}

_lib = None


def header_functions() -> list[str]:
    """Names of every function declared in include/ibsn.h."""
    text = open(HEADER).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(ibsn_[a-z_]+)\s*\(", text)))


def load(path: str | None = None):
    """Load the shared library (once) and attach the signatures."""
    global _lib
    if _lib is not None and path is None:
        return _lib
    p = path or LIB_PATH
    if not os.path.exists(p):
        raise RuntimeError(f"IBSN CUDA library not built ({p} missing): run __graft_entry__.build()")
    lib = C.CDLL(p)
    for name, (res, args) in _SIGS.items():
        fn = getattr(lib, name)
        fn.restype = res
        fn.argtypes = args
    if path is None:
        _lib = lib
    return lib


class IbsnError(RuntimeError):
    def __init__(self, code: int, where: str):
        lib = load()
        msg = lib.ibsn_status_string(code).decode()
        if code == 5:
            msg += ": " + lib.ibsn_last_cuda_error().decode()
        super().__init__(f"{where}: {msg} (status {code})")
        self.code = code


def check(code: int, where: str, allow=(0,)) -> int:
    if code not in allow:
        raise IbsnError(code, where)
    return code

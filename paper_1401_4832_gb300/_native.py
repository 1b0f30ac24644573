"""ctypes declarations of the C ABI in ``include/plmdca.h``.

Loads ``_build/libplmdca.so`` (built in-tree by ``_build_lib.build``).  There
is no fallback: if the library is missing or fails to load, every call
raises.
"""
from __future__ import annotations

import ctypes
import os
import threading

from . import _build_lib

PLM_OK = 0
PLM_EINVAL = -1
PLM_ENOMEM = -2
PLM_ECUDA = -3
PLM_ENOTCONV = -4
PLM_ETIMEOUT = -5
PLM_ENOTIMPL = -6
STATUS_NAMES = {0: "PLM_OK", -1: "PLM_EINVAL", -2: "PLM_ENOMEM", -3: "PLM_ECUDA",
                -4: "PLM_ENOTCONV", -5: "PLM_ETIMEOUT", -6: "PLM_ENOTIMPL"}

PLM_FP32_EXACT = 0
PLM_TF32 = 1
PLM_SPLIT_BF16 = 2
PRECISIONS = {"fp32": PLM_FP32_EXACT, "tf32": PLM_TF32, "split_bf16": PLM_SPLIT_BF16}


class plm_opts(ctypes.Structure):
    _fields_ = [("x", ctypes.c_double), ("lambda_h", ctypes.c_double),
                ("lambda_J", ctypes.c_double), ("gtol", ctypes.c_double),
                ("lbfgs_m", ctypes.c_int), ("max_iter", ctypes.c_int),
                ("max_ls", ctypes.c_int), ("prec", ctypes.c_int),
                ("use_graph", ctypes.c_int), ("autotune", ctypes.c_int),
                ("reserved", ctypes.c_int * 6)]


class plm_report(ctypes.Structure):
    _fields_ = [("iters", ctypes.c_int), ("evals", ctypes.c_int),
                ("n_converged", ctypes.c_int), ("n_noise", ctypes.c_int),
                ("n_failed", ctypes.c_int), ("f_total", ctypes.c_double),
                ("gnorm_max", ctypes.c_double), ("beff", ctypes.c_double),
                ("seconds", ctypes.c_double)]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


class plm_family(ctypes.Structure):
    _fields_ = [("msa", ctypes.c_void_p), ("B", ctypes.c_int), ("N", ctypes.c_int),
                ("h_out", ctypes.c_void_p), ("J_out", ctypes.c_void_p)]


class plm_score_opts(ctypes.Structure):
    _fields_ = [("combine", ctypes.c_int), ("norm", ctypes.c_int), ("p", ctypes.c_double),
                ("exclude_gap", ctypes.c_int), ("correction", ctypes.c_int),
                ("reserved", ctypes.c_int * 4)]


NORMS = {"fro": 0, "lp": 1, "burkoff": 2}
CORRECTIONS = {"apc": 0, "asc": 1, "none": 2}


class PlmError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__(f"{STATUS_NAMES.get(status, status)}: {msg}")
        self.status = status


_lock = threading.Lock()
_lib = None


def library_path() -> str:
    return _build_lib.LIB


def load():
    """Load the CUDA library (raises if it has not been built)."""
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        path = library_path()
        if not os.path.exists(path):
            raise RuntimeError(
                f"plmDCA CUDA library not built ({path} missing): run "
                "`python -c 'import __graft_entry__ as g; g.build()'`")
        lib = ctypes.CDLL(path)
        P = ctypes.c_void_p
        I = ctypes.c_int
        D = ctypes.c_double
        lib.plm_default_opts.argtypes = [ctypes.POINTER(plm_opts)]
        lib.plm_default_opts.restype = None
        lib.plm_create.argtypes = [ctypes.POINTER(P), I, P]
        lib.plm_create.restype = I
        lib.plm_destroy.argtypes = [P]
        lib.plm_destroy.restype = I
        lib.plm_last_error.argtypes = [P]
        lib.plm_last_error.restype = ctypes.c_char_p
        lib.msa_reweight.argtypes = [P, P, I, I, I, D, P, P, ctypes.POINTER(D)]
        lib.msa_reweight.restype = I
        lib.plm_site_objective_grad.argtypes = [P, P, P, D, I, I, I, P, P, D, D, I, P, P, P]
        lib.plm_site_objective_grad.restype = I
        lib.plm_solve.argtypes = [P, P, I, I, I, ctypes.POINTER(plm_opts), P, P,
                                  ctypes.POINTER(plm_report)]
        lib.plm_solve.restype = I
        lib.plm_solve_batch.argtypes = [P, ctypes.POINTER(plm_family), I, I,
                                        ctypes.POINTER(plm_opts), ctypes.POINTER(plm_report)]
        lib.plm_solve_batch.restype = I
        lib.plm_solve_symmetric.argtypes = [P, P, I, I, I, ctypes.POINTER(plm_opts), P, P,
                                            ctypes.POINTER(plm_report)]
        lib.plm_solve_symmetric.restype = I
        lib.fn_apc_scores.argtypes = [P, P, I, I, I, P, P, P, I, I]
        lib.fn_apc_scores.restype = I
        lib.plm_default_score_opts.argtypes = [ctypes.POINTER(plm_score_opts)]
        lib.plm_default_score_opts.restype = None
        lib.plm_scores.argtypes = [P, P, I, I, ctypes.POINTER(plm_score_opts), P, P, P, P, I, I]
        lib.plm_scores.restype = I
        lib.plmdca_run.argtypes = [P, P, I, I, I, ctypes.POINTER(plm_opts), I, I, P, P, P, P, P,
                                   ctypes.POINTER(plm_report)]
        lib.plmdca_run.restype = I
        lib.msa_parse.argtypes = [P, ctypes.c_char_p, ctypes.c_size_t, I, P, ctypes.c_longlong,
                                  ctypes.POINTER(I), ctypes.POINTER(I)]
        lib.msa_parse.restype = I
        lib.msa_frequencies.argtypes = [P, P, P, D, I, I, I, P]
        lib.msa_frequencies.restype = I
        lib.plm_selftest_wait.argtypes = [P, ctypes.POINTER(I)]
        lib.plm_selftest_wait.restype = I
        lib.plm_kernel_launches.argtypes = []
        lib.plm_kernel_launches.restype = ctypes.c_longlong
        lib.plm_profile.argtypes = [P, I]
        lib.plm_profile.restype = I
        lib.plm_profile_report.argtypes = [P, ctypes.c_char_p, I]
        lib.plm_profile_report.restype = I
        lib.plm_measure_peak.argtypes = [I, P, ctypes.POINTER(D)]
        lib.plm_measure_peak.restype = I
        lib.msa_reweight_static.argtypes = [P, I, I, I, D, P, P, P, P]
        lib.msa_reweight_static.restype = I
        _lib = lib
        return lib


def header_functions() -> list[str]:
    """Names of the functions that ``include/plmdca.h`` declares."""
    import re
    hdr = os.path.join(_build_lib.INCLUDE, "plmdca.h")
    text = open(hdr).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    names = re.findall(r"^\s*(?:const\s+)?[A-Za-z_][A-Za-z0-9_\s\*]*?\b([a-z_][a-z0-9_]*)\s*\(",
                       text, flags=re.M)
    return sorted(set(n for n in names if n not in ("if", "while", "sizeof")))

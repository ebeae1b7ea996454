"""ctypes binding of libtpt.so: the C ABI of include/tpt.h under the same names.

Argument marshalling only.  Every step of a solve runs in the library's CUDA
kernels; there is no Python or CPU fallback.  Importing this module on a
machine where libtpt.so is missing raises ImportError.
"""
from __future__ import annotations

import ctypes as C
import os

from . import build as _build

TPT_OK = 0
TPT_ERR_INVALID_ARG = 1
TPT_ERR_UNSUPPORTED = 2
TPT_ERR_OOM = 3
TPT_ERR_CUDA = 4
TPT_ERR_NOT_CONVERGED = 5
TPT_ERR_TIMEOUT = 6
TPT_ERR_NONFINITE = 7
TPT_ERR_NUMERICAL = 8
TPT_PENDING = 9

TPT_BC_PERIODIC, TPT_BC_NEUMANN, TPT_BC_DIRICHLET, TPT_BC_DIRICHLET_NODE, TPT_BC_NONE = 0, 1, 2, 3, 4
TPT_XFORM_AUTO, TPT_XFORM_GEMM, TPT_XFORM_FFT = 0, 1, 2
TPT_PREC_FP64, TPT_PREC_MIXED_BF16, TPT_PREC_MIXED_BF16X3, TPT_PREC_MIXED_TF32, TPT_PREC_FP64_OZAKI = 0, 1, 2, 3, 4
TPT_GEMM_OUT_F32, TPT_GEMM_OUT_BF16, TPT_GEMM_OUT_SPLIT_BF16 = 0, 1, 2

_dp = C.POINTER(C.c_double)


class tpt_desc(C.Structure):
    _fields_ = [
        ("n", C.c_int * 3),
        ("dxf", _dp * 3),
        ("dxc", _dp * 3),
        ("bc", (C.c_int * 2) * 3),
        ("xform", C.c_int * 2),
        ("alpha", C.c_double),
        ("beta", C.c_double),
        ("precision", C.c_int),
        ("rtol", C.c_double),
        ("max_refine", C.c_int),
    ]


class tpt_info(C.Structure):
    _fields_ = [
        ("iters", C.c_int),
        ("rel_residual", C.c_double),
        ("compat_defect", C.c_double),
        ("ms_stage", C.c_float * 8),
    ]


class tpt_server_config(C.Structure):
    _fields_ = [
        ("cuda_device", C.c_int),
        ("slots", C.c_int),
        ("setup_threads", C.c_int),
        ("memory_budget", C.c_size_t),
        ("cache_budget", C.c_size_t),
        ("dry_run_ns_per_point", C.c_double),
        ("merge", C.c_int),
    ]


class tpt_result(C.Structure):
    _fields_ = [
        ("status", C.c_int),
        ("info", tpt_info),
        ("t_submit", C.c_double),
        ("t_planned", C.c_double),
        ("t_admit", C.c_double),
        ("t_done", C.c_double),
        ("device_bytes", C.c_size_t),
        ("failed_step", C.c_int),
        ("cuda_error", C.c_int),
        ("t_copied", C.c_double),
        ("t_solved", C.c_double),
        ("merged", C.c_int),
    ]


class tpt_serving_stats(C.Structure):
    _fields_ = [
        ("submitted", C.c_ulonglong),
        ("completed", C.c_ulonglong),
        ("rejected", C.c_ulonglong),
        ("cache_hits", C.c_ulonglong),
        ("cache_misses", C.c_ulonglong),
        ("cache_bytes", C.c_size_t),
        ("peak_bytes", C.c_size_t),
        ("peak_inflight", C.c_int),
    ]


# (name, restype, argtypes) of every entry point declared in include/tpt.h
SIGNATURES = [
    ("tpt_plan_create", C.c_int, [C.POINTER(tpt_desc), C.c_int, C.POINTER(C.c_void_p)]),
    ("tpt_workspace_bytes", C.c_int, [C.c_void_p, C.POINTER(C.c_size_t)]),
    ("tpt_solve", C.c_int, [C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p,
                            C.POINTER(tpt_info)]),
    ("tpt_solve_host", C.c_int, [C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p,
                                 C.c_void_p, C.c_void_p, C.POINTER(tpt_info)]),
    ("tpt_set_coefficients", C.c_int, [C.c_void_p, C.c_double, C.c_double]),
    ("tpt_plan_destroy", C.c_int, [C.c_void_p]),
    ("tpt_status_string", C.c_char_p, [C.c_int]),
    ("tpt_transform", C.c_int, [C.c_void_p, C.c_int, C.c_int, C.c_void_p, C.c_void_p, C.c_void_p]),
    ("tpt_thomas", C.c_int, [C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p]),
    ("tpt_thomas_noalloc", C.c_int, [C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p]),
    ("tpt_residual", C.c_int, [C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p,
                               C.c_void_p]),
    ("tpt_tc_gemm", C.c_int, [C.c_int, C.c_int, C.c_int, C.c_int, C.c_void_p, C.c_void_p, C.c_void_p,
                              C.c_void_p, C.c_void_p, C.c_int, C.c_int]),
    ("tpt_tc_gemm_out", C.c_int, [C.c_int, C.c_int, C.c_int, C.c_int, C.c_void_p, C.c_void_p, C.c_int, C.c_int,
                                  C.c_longlong, C.c_longlong, C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p,
                                  C.c_int, C.c_int, C.c_int]),
    ("tpt_plan_eigenvalues", C.c_int, [C.c_void_p, C.c_int, _dp]),
    ("tpt_plan_transforms", C.c_int, [C.c_void_p, C.POINTER(C.c_int)]),
    ("tpt_plan_rows", C.c_int, [C.c_void_p, C.c_int, _dp, _dp, _dp]),
    ("tpt_grid_tanh", C.c_int, [C.c_int, C.c_double, C.c_double, _dp, _dp]),
    ("tpt_grid_faces", C.c_int, [C.c_int, _dp, _dp, C.c_int, C.POINTER(C.c_int), _dp, _dp]),
    ("tpt_kernel_launches", C.c_int, [C.POINTER(C.c_ulonglong)]),
    ("tpt_pointer_on_device", C.c_int, [C.c_void_p, C.c_int, C.POINTER(C.c_int)]),
    ("tpt_cuda_error_name", C.c_char_p, [C.c_int]),
    ("tpt_test_fail_allocations", C.c_int, [C.c_longlong]),
    ("tpt_test_gemm_timeout", C.c_int, [C.c_uint, C.c_void_p, C.c_size_t, C.c_void_p]),
    ("tpt_set_stage_timing", C.c_int, [C.c_void_p, C.c_int]),
    ("tpt_set_refinement", C.c_int, [C.c_void_p, C.c_double, C.c_int]),
    ("tpt_plan_autotune", C.c_int, [C.c_void_p, C.c_void_p, C.c_void_p, C.POINTER(C.c_int)]),
    ("tpt_plan_set_tiles", C.c_int, [C.c_void_p, C.POINTER(C.c_int)]),
    ("tpt_plan_get_tiles", C.c_int, [C.c_void_p, C.POINTER(C.c_int)]),
    ("tpt_plan_set_pairing", C.c_int, [C.c_void_p, C.POINTER(C.c_int)]),
    ("tpt_plan_set_residual_kernel", C.c_int, [C.c_void_p, C.c_int]),
    ("tpt_plan_set_thomas_kernel", C.c_int, [C.c_void_p, C.c_int]),
    ("tpt_mixed_thomas", C.c_int, [C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p]),
    ("tpt_plan_get_pairing", C.c_int, [C.c_void_p, C.POINTER(C.c_int)]),
    ("tpt_batch_create", C.c_int, [C.POINTER(tpt_desc), C.c_int, C.c_int, C.c_int, C.POINTER(C.c_void_p)]),
    ("tpt_batch_workspace_bytes", C.c_int, [C.c_void_p, C.POINTER(C.c_size_t)]),
    ("tpt_batch_plan", C.c_int, [C.c_void_p, C.c_int, C.POINTER(C.c_void_p)]),
    ("tpt_batch_autotune", C.c_int, [C.c_void_p, C.c_void_p, C.c_void_p]),
    ("tpt_batch_solve", C.c_int, [C.c_void_p, C.POINTER(C.c_void_p), C.POINTER(C.c_void_p), C.c_void_p,
                                  C.c_void_p, C.POINTER(tpt_info), C.POINTER(C.c_int)]),
    ("tpt_batch_infos", C.c_int, [C.c_void_p, C.POINTER(tpt_info), C.POINTER(C.c_int)]),
    ("tpt_batch_launches", C.c_int, [C.c_void_p, C.POINTER(C.c_ulonglong)]),
    ("tpt_batch_set_grouped", C.c_int, [C.c_void_p, C.c_int]),
    ("tpt_batch_get_grouped", C.c_int, [C.c_void_p, C.POINTER(C.c_int)]),
    ("tpt_batch_destroy", C.c_int, [C.c_void_p]),
    ("tpt_project_workspace_bytes", C.c_int, [C.c_void_p, C.POINTER(C.c_size_t)]),
    ("tpt_project", C.c_int, [C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p, C.c_double, C.c_void_p, C.c_void_p,
                              C.c_void_p, C.POINTER(tpt_info)]),
    ("tpt_cache_create", C.c_int, [C.c_int, C.c_size_t, C.POINTER(C.c_void_p)]),
    ("tpt_plan_create_cached", C.c_int, [C.POINTER(tpt_desc), C.c_void_p, C.POINTER(C.c_void_p)]),
    ("tpt_cache_stats", C.c_int, [C.c_void_p, C.POINTER(C.c_ulonglong), C.POINTER(C.c_ulonglong),
                                  C.POINTER(C.c_size_t), C.POINTER(C.c_size_t)]),
    ("tpt_cache_destroy", C.c_int, [C.c_void_p]),
    ("tpt_server_create", C.c_int, [C.POINTER(tpt_server_config), C.POINTER(C.c_void_p)]),
    ("tpt_server_submit", C.c_int, [C.c_void_p, C.POINTER(tpt_desc), C.c_void_p, C.c_void_p,
                                    C.POINTER(C.c_ulonglong)]),
    ("tpt_server_warm", C.c_int, [C.c_void_p, C.POINTER(tpt_desc)]),
    ("tpt_server_wait", C.c_int, [C.c_void_p, C.c_ulonglong, C.c_double, C.POINTER(tpt_result)]),
    ("tpt_server_now", C.c_int, [C.c_void_p, C.POINTER(C.c_double)]),
    ("tpt_server_stats", C.c_int, [C.c_void_p, C.POINTER(tpt_serving_stats)]),
    ("tpt_server_destroy", C.c_int, [C.c_void_p]),
]

LIB_PATH = _build.LIB


def _load():
    if not os.path.exists(LIB_PATH):
        raise ImportError("libtpt.so is not built (%s); run __graft_entry__.build() or "
                          "python -m paper_2603_09528_gb300.build" % LIB_PATH)
    lib = C.CDLL(LIB_PATH)
    for name, res, args in SIGNATURES:
        fn = getattr(lib, name)
        fn.restype = res
        fn.argtypes = args
    return lib


lib = _load()


class TptError(RuntimeError):
    def __init__(self, status: int, where: str):
        self.status = status
        msg = lib.tpt_status_string(status)
        super().__init__("%s failed: %s (status %d)" % (where, msg.decode() if msg else "?", status))


def kernel_launches() -> int:
    v = C.c_ulonglong()
    check(lib.tpt_kernel_launches(C.byref(v)), "tpt_kernel_launches")
    return int(v.value)


def check(status: int, where: str) -> int:
    if status != TPT_OK:
        raise TptError(status, where)
    return status

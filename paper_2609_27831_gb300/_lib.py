"""ctypes binding of ``include/ozaki2.h`` (argument marshalling only).

Every computation runs in the CUDA kernels of ``libozaki2_gb300.so``; this
module only mirrors the C structs and loads the library.  Loading fails loudly
when the shared library has not been built: there is no fallback.
"""
from __future__ import annotations

import ctypes as C
import os

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libozaki2_gb300.so")

OZ2_OK, OZ2_EINVAL, OZ2_ERANGE, OZ2_ENOMEM, OZ2_ECUDA, OZ2_EINTERNAL, OZ2_ETIMEOUT, OZ2_ENODEV = range(8)
ENGINE_TC, ENGINE_SIMT, ENGINE_S8 = 0, 1, 2
SCHED_GROUPED, SCHED_PLAIN = 0, 1


class Mat(C.Structure):
    _fields_ = [("limbs", C.c_void_p), ("exp", C.c_void_p), ("sign", C.c_void_p),
                ("ld", C.c_int64), ("plane_stride", C.c_int64)]


class Opts(C.Structure):
    _fields_ = [("guard_bits", C.c_int), ("t_bits", C.c_int), ("engine", C.c_int),
                ("k_chunk", C.c_int), ("grid", C.c_int), ("schedule", C.c_int),
                ("timing", C.c_int), ("crt_engine", C.c_int), ("res_engine", C.c_int),
                ("plane_group", C.c_int), ("gemm_tile", C.c_int)]


class Info(C.Structure):
    _fields_ = [("count", C.c_int), ("t", C.c_int), ("L", C.c_int), ("L1", C.c_int),
                ("G", C.c_int), ("crt_digits", C.c_int), ("units", C.c_int),
                ("jobs", C.c_int), ("workspace_bytes", C.c_size_t), ("crt_mode", C.c_int),
                ("res_mode", C.c_int), ("plane_groups", C.c_int), ("group_planes", C.c_int),
                ("gemm_tile", C.c_int), ("crt_skip_groups", C.c_int)]


class Problem(C.Structure):
    _fields_ = [("M", C.c_int64), ("N", C.c_int64), ("K", C.c_int64), ("p", C.c_int),
                ("A", Mat), ("B", Mat), ("C", Mat)]


class OzakiError(RuntimeError):
    def __init__(self, status: int, what: str):
        self.status = status
        super().__init__(f"{what}: {strerror(status)} (status {status})")


_lib = None

_SIGS = {
    "ozaki2_opts_default": (C.c_int, [C.POINTER(Opts)]),
    "ozaki2_strerror": (C.c_char_p, [C.c_int]),
    "ozaki2_version": (C.c_char_p, []),
    "ozaki2_plan_create": (C.c_int, [C.c_int64, C.c_int64, C.c_int64, C.c_int, C.POINTER(Opts),
                                      C.POINTER(C.c_void_p)]),
    "ozaki2_plan_create_batched": (C.c_int, [C.c_int, C.POINTER(Problem), C.POINTER(Opts),
                                              C.POINTER(C.c_void_p)]),
    "ozaki2_plan_create_batched_ex": (C.c_int, [C.c_int, C.POINTER(Problem), C.POINTER(Opts), C.POINTER(Opts),
                                                 C.POINTER(C.c_void_p)]),
    "ozaki2_plan_destroy": (C.c_int, [C.c_void_p]),
    "ozaki2_plan_info": (C.c_int, [C.c_void_p, C.POINTER(Info)]),
    "ozaki2_plan_moduli": (C.c_int, [C.c_void_p, C.c_int, C.POINTER(C.c_int32), C.c_int]),
    "ozaki2_plan_crt_tables": (C.c_int, [C.c_void_p, C.c_int, C.POINTER(C.c_uint32),
                                          C.POINTER(C.c_uint32), C.POINTER(C.c_uint32)]),
    "ozaki2_plan_layout": (C.c_int, [C.c_void_p, C.c_int, C.POINTER(C.c_size_t),
                                      C.POINTER(C.c_int64)]),
    "ozaki2_plan_launches": (C.c_int, [C.c_void_p, C.POINTER(C.c_int)]),
    "ozaki2_plan_set_debug_chat": (C.c_int, [C.c_void_p, C.c_int, C.c_void_p]),
    "ozaki2_plan_set_wait_limit": (C.c_int, [C.c_void_p, C.c_uint32]),
    "ozaki2_plan_set_debug_prods": (C.c_int, [C.c_void_p, C.c_int, C.c_void_p]),
    "ozaki2_plan_debug_corrupt_crt": (C.c_int, [C.c_void_p, C.c_int]),
    "ozaki2_debug_inject_alloc_failure": (C.c_int, [C.c_int]),
    "ozaki2_execute": (C.c_int, [C.c_void_p, C.POINTER(Mat), C.POINTER(Mat), C.POINTER(Mat),
                                  C.c_void_p, C.c_size_t, C.c_void_p]),
    "ozaki2_execute_batched": (C.c_int, [C.c_void_p, C.c_int, C.POINTER(Problem), C.c_void_p,
                                          C.c_size_t, C.c_void_p]),
    "ozaki2_execute_reuse": (C.c_int, [C.c_void_p, C.c_int, C.POINTER(Mat), C.POINTER(Mat), C.c_void_p,
                                        C.c_size_t, C.c_void_p]),
    "ozaki2_graph_create": (C.c_int, [C.c_void_p, C.c_int, C.POINTER(Problem), C.c_void_p,
                                       C.c_size_t, C.c_void_p, C.POINTER(C.c_void_p)]),
    "ozaki2_graph_launch": (C.c_int, [C.c_void_p, C.c_void_p]),
    "ozaki2_graph_destroy": (C.c_int, [C.c_void_p]),
    "ozaki2_gemm": (C.c_int, [C.c_int64, C.c_int64, C.c_int64, C.c_int, C.POINTER(Mat),
                               C.POINTER(Mat), C.POINTER(Mat), C.POINTER(Opts), C.c_void_p]),
    "ozaki2_gemm_batched": (C.c_int, [C.c_int, C.POINTER(Problem), C.POINTER(Opts), C.c_void_p]),
    "ozaki2_gemm_noalloc": (C.c_int, [C.c_int64, C.c_int64, C.c_int64, C.c_int, C.POINTER(Mat),
                                       C.POINTER(Mat), C.POINTER(Mat), C.c_void_p]),
    "ozaki2_noalloc_check": (C.c_int, [C.c_void_p]),
    "ozaki2_plan_create_complex": (C.c_int, [C.c_int64, C.c_int64, C.c_int64, C.c_int, C.POINTER(Opts),
                                              C.POINTER(C.c_void_p)]),
    "ozaki2_execute_complex": (C.c_int, [C.c_void_p] + [C.POINTER(Mat)] * 6 + [C.c_void_p, C.c_size_t,
                                                                               C.c_void_p]),
    "ozaki2_zgemm": (C.c_int, [C.c_int64, C.c_int64, C.c_int64, C.c_int] + [C.POINTER(Mat)] * 6 +
                     [C.POINTER(Opts), C.c_void_p]),
    "ozaki2_release_cache": (C.c_int, []),
    "ozaki2_check": (C.c_int, [C.c_void_p, C.c_void_p]),
    "ozaki2_last_timings": (C.c_int, [C.c_void_p, C.POINTER(C.c_float)]),
    "ozaki2_last_crt_split": (C.c_int, [C.c_void_p, C.POINTER(C.c_float)]),
    "ozaki2_dgemm_fwd": (C.c_int, [C.c_int64, C.c_int64, C.c_int64, C.c_void_p, C.c_int64,
                                    C.c_void_p, C.c_int64, C.c_void_p, C.c_int64, C.POINTER(Opts),
                                    C.POINTER(C.c_void_p), C.c_void_p]),
    "ozaki2_dgemm_bwd": (C.c_int, [C.c_void_p, C.c_void_p, C.c_int64, C.c_void_p, C.c_int64,
                                    C.c_void_p, C.c_int64, C.c_void_p]),
    "ozaki2_cache_destroy": (C.c_int, [C.c_void_p]),
    "ozaki2_probe_mma_s8": (C.c_int, [C.c_int, C.c_int, C.c_void_p, C.POINTER(C.c_double), C.c_void_p]),
}


def lib() -> C.CDLL:
    """The loaded library (raises if it was not built)."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise RuntimeError(
                f"{LIB_PATH} is missing: build it with paper_2609_27831_gb300.build.build() "
                "(there is no CPU fallback)")
        h = C.CDLL(LIB_PATH)
        for name, (res, args) in _SIGS.items():
            fn = getattr(h, name)
            fn.restype = res
            fn.argtypes = args
        _lib = h
    return _lib


def strerror(status: int) -> str:
    try:
        return lib().ozaki2_strerror(status).decode()
    except Exception:  # pragma: no cover - only when the library is absent
        return f"status {status}"


def check(status: int, what: str) -> None:
    if status != OZ2_OK:
        raise OzakiError(status, what)


def opts(**kw) -> Opts:
    o = Opts()
    check(lib().ozaki2_opts_default(C.byref(o)), "ozaki2_opts_default")
    for k, v in kw.items():
        if not hasattr(o, k):
            raise TypeError(f"unknown option {k}")
        setattr(o, k, int(v))
    return o

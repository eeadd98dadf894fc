"""ctypes binding of libqcgraph.so: argument marshalling only.

Every step of the method runs in the library's CUDA kernels.  There is no CPU
fallback: if the library is missing or cannot load, importing this module's
``lib()`` raises.
"""
from __future__ import annotations

import ctypes
import os
import threading

HERE = os.path.dirname(os.path.abspath(__file__))
# QCGRAPH_DEBUG_LIB=1 selects the bounds-checked debug build (libqcgraph_debug.so)
LIB_PATH = os.path.join(HERE, "libqcgraph_debug.so" if os.environ.get("QCGRAPH_DEBUG_LIB") == "1"
                        else "libqcgraph.so")

c_int32_p = ctypes.POINTER(ctypes.c_int32)
c_int64_p = ctypes.POINTER(ctypes.c_int64)
c_double_p = ctypes.POINTER(ctypes.c_double)
c_void_pp = ctypes.POINTER(ctypes.c_void_p)

ALLOC_FN = ctypes.CFUNCTYPE(ctypes.c_void_p, ctypes.c_size_t, ctypes.c_void_p, ctypes.c_void_p)
FREE_FN = ctypes.CFUNCTYPE(None, ctypes.c_void_p, ctypes.c_size_t, ctypes.c_void_p, ctypes.c_void_p)


class qc_allocator(ctypes.Structure):
    _fields_ = [("alloc", ALLOC_FN), ("free", FREE_FN), ("user", ctypes.c_void_p)]


class qc_server_config(ctypes.Structure):
    _fields_ = [("mem_budget_bytes", ctypes.c_size_t), ("max_active", ctypes.c_int32),
                ("streams", ctypes.c_int32), ("large_workers", ctypes.c_int32),
                ("large_sm_share", ctypes.c_float), ("divide_share", ctypes.c_int32)]


class qc_server_stats(ctypes.Structure):
    _fields_ = [("submitted", ctypes.c_uint64), ("completed", ctypes.c_uint64),
                ("cancelled", ctypes.c_uint64), ("failed", ctypes.c_uint64),
                ("steps", ctypes.c_uint64), ("large_solved", ctypes.c_uint64),
                ("bytes_resident", ctypes.c_size_t), ("peak_bytes_resident", ctypes.c_size_t),
                ("active", ctypes.c_int32), ("queued", ctypes.c_int32),
                ("peak_in_flight", ctypes.c_int32)]


class qc_request_info(ctypes.Structure):
    _fields_ = [("admit_ms", ctypes.c_double), ("start_ms", ctypes.c_double), ("done_ms", ctypes.c_double),
                ("n", ctypes.c_int32),
                ("nnz", ctypes.c_int64), ("batch_size", ctypes.c_int32)]


class qc_quality_result(ctypes.Structure):
    _fields_ = [("modularity", ctypes.c_double), ("ari", ctypes.c_double), ("fmi", ctypes.c_double),
                ("nmi", ctypes.c_double), ("clusters", ctypes.c_int32)]


class qc_kernel_stats(ctypes.Structure):
    _fields_ = [("launches", ctypes.c_uint64), ("total_ms", ctypes.c_double),
                ("model_bytes", ctypes.c_double), ("min_bytes", ctypes.c_double)]


STATUS = {0: "QC_OK", 1: "QC_ERR_INVALID_ARG", 2: "QC_ERR_INVALID_GRAPH", 3: "QC_ERR_OOM",
          4: "QC_ERR_BUDGET", 5: "QC_ERR_CUDA", 6: "QC_ERR_TIMEOUT", 7: "QC_ERR_CANCELLED",
          8: "QC_ERR_NOT_READY"}
QC_PTR_DEVICE = 1
QC_VALIDATE = 2
QC_DIRECTED = 4

# (name, restype, argtypes) for every entry point of include/qcgraph.h
SIGNATURES = [
    ("qc_context_create", ctypes.c_int, [ctypes.c_int, ctypes.c_size_t, ctypes.POINTER(qc_allocator), c_void_pp]),
    ("qc_context_destroy", None, [ctypes.c_void_p]),
    ("qc_context_bytes_in_use", ctypes.c_size_t, [ctypes.c_void_p]),
    ("qc_context_set_timing", ctypes.c_int, [ctypes.c_void_p, ctypes.c_int]),
    ("qc_context_kernel_stats", ctypes.c_int, [ctypes.c_void_p, ctypes.c_char_p,
                                               ctypes.POINTER(qc_kernel_stats), ctypes.c_int]),
    ("qc_context_launch_count", ctypes.c_uint64, [ctypes.c_void_p]),
    ("qc_status_string", ctypes.c_char_p, [ctypes.c_int]),
    ("qc_last_error", ctypes.c_char_p, [ctypes.c_void_p]),
    ("qc_graph_create", ctypes.c_int, [ctypes.c_void_p, ctypes.c_int32, ctypes.c_int64, ctypes.c_void_p,
                                       ctypes.c_void_p, ctypes.c_uint32, ctypes.c_void_p, c_void_pp]),
    ("qc_graph_destroy", None, [ctypes.c_void_p]),
    ("qc_graph_drop_histogram", None, [ctypes.c_void_p]),
    ("qc_graph_num_nodes", ctypes.c_int32, [ctypes.c_void_p]),
    ("qc_graph_num_edges", ctypes.c_int64, [ctypes.c_void_p]),
    ("qc_graph_histogram", ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, c_int32_p, ctypes.c_void_p]),
    ("qc_graph_set_weights", ctypes.c_int, [ctypes.c_void_p, c_double_p, ctypes.c_uint32, ctypes.c_void_p]),
    ("qc_potential_weighted", ctypes.c_int, [ctypes.c_void_p, c_double_p, ctypes.c_int32, ctypes.c_void_p,
                                             ctypes.c_void_p]),
    ("qc_graph_set_histogram", ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int32, ctypes.c_uint32,
                                              ctypes.c_void_p]),
    ("qc_potential", ctypes.c_int, [ctypes.c_void_p, c_double_p, ctypes.c_int32, ctypes.c_void_p,
                                    ctypes.c_void_p]),
    ("qc_potential_adjacency", ctypes.c_int, [ctypes.c_void_p, c_double_p, ctypes.c_int32, ctypes.c_double,
                                              ctypes.c_void_p, ctypes.c_void_p]),
    ("qc_ggd_labels", ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int32, ctypes.c_void_p,
                                     c_int32_p, ctypes.c_void_p]),
    ("qc_solve", ctypes.c_int, [ctypes.c_void_p, c_double_p, ctypes.c_int32, ctypes.c_void_p,
                                ctypes.c_void_p, c_int32_p, ctypes.c_void_p]),
    ("qc_cluster", ctypes.c_int, [ctypes.c_void_p, ctypes.c_int32, ctypes.c_int64, ctypes.c_void_p,
                                  ctypes.c_void_p, ctypes.c_uint32, c_double_p, ctypes.c_int32, ctypes.c_void_p,
                                  c_int32_p, ctypes.c_void_p]),
    ("qc_quality", ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int32, ctypes.c_void_p,
                                  ctypes.c_void_p, ctypes.c_int32, ctypes.c_double,
                                  ctypes.POINTER(qc_quality_result), ctypes.c_void_p]),
    ("qc_batch_create", ctypes.c_int, [ctypes.c_void_p, ctypes.c_int32, c_void_pp, c_double_p,
                                       ctypes.c_void_p, c_int64_p, ctypes.c_void_p, c_void_pp]),
    ("qc_batch_run", ctypes.c_int, [ctypes.c_void_p, c_int32_p, ctypes.c_void_p]),
    ("qc_batch_destroy", None, [ctypes.c_void_p]),
    ("qc_batch_config", ctypes.c_int, [ctypes.c_void_p, c_int32_p, c_int32_p, c_int32_p]),
    ("qc_solve_batch", ctypes.c_int, [ctypes.c_void_p, ctypes.c_int32, c_void_pp, c_double_p,
                                      ctypes.c_void_p, c_int64_p, ctypes.c_void_p]),
    ("qc_server_create", ctypes.c_int, [ctypes.c_void_p, ctypes.POINTER(qc_server_config), c_void_pp]),
    ("qc_server_submit", ctypes.c_int, [ctypes.c_void_p, ctypes.c_int32, ctypes.c_int64, ctypes.c_void_p,
                                        ctypes.c_void_p, ctypes.c_double, ctypes.POINTER(ctypes.c_uint64)]),
    ("qc_server_submit_graph", ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_double,
                                              ctypes.POINTER(ctypes.c_uint64)]),
    ("qc_server_poll", ctypes.c_int, [ctypes.c_void_p, ctypes.c_uint64, ctypes.c_void_p, c_int32_p,
                                      ctypes.POINTER(qc_request_info), ctypes.POINTER(ctypes.c_int)]),
    ("qc_server_wait", ctypes.c_int, [ctypes.c_void_p, ctypes.c_uint64, ctypes.c_int64, ctypes.c_void_p,
                                      c_int32_p, ctypes.POINTER(qc_request_info)]),
    ("qc_server_cancel", ctypes.c_int, [ctypes.c_void_p, ctypes.c_uint64]),
    ("qc_server_get_stats", ctypes.c_int, [ctypes.c_void_p, ctypes.POINTER(qc_server_stats)]),
    ("qc_server_destroy", None, [ctypes.c_void_p]),
    ("qc_sweep_create", ctypes.c_int, [ctypes.c_void_p, c_double_p, ctypes.c_int32, ctypes.c_void_p,
                                        ctypes.c_void_p, ctypes.c_void_p, c_void_pp]),
    ("qc_sweep_run", ctypes.c_int, [ctypes.c_void_p, ctypes.c_int32, c_int32_p, ctypes.c_void_p]),
    ("qc_sweep_info", ctypes.c_int, [ctypes.c_void_p, c_int32_p, c_int32_p, c_int64_p]),
    ("qc_sweep_destroy", None, [ctypes.c_void_p]),
    ("qc_selftest_barrier_timeout", ctypes.c_int, [ctypes.c_void_p, ctypes.c_int64, c_int64_p, ctypes.c_void_p]),
    ("qc_selftest_arith", ctypes.c_int, [ctypes.c_void_p, ctypes.c_int32, ctypes.c_void_p, ctypes.c_void_p,
                                         ctypes.c_void_p, ctypes.c_int64, ctypes.c_void_p]),
    ("qc_selftest_debug_check", ctypes.c_int, [ctypes.c_void_p, ctypes.c_int32, ctypes.c_int32, c_int32_p,
                                                c_int32_p, ctypes.c_void_p]),
    ("qc_selftest_l2_read", ctypes.c_int, [ctypes.c_void_p, ctypes.c_int64, ctypes.c_int32, c_double_p,
                                            ctypes.c_void_p]),
    ("qc_histogram_static_scratch", ctypes.c_int, [ctypes.c_int32, ctypes.c_int64, ctypes.c_void_p,
                                                   ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int32,
                                                   c_int32_p, ctypes.c_void_p]),
]

_lock = threading.Lock()
_lib = None


def load(path: str = LIB_PATH) -> ctypes.CDLL:
    """Load and bind the library (raises OSError if it is missing or unloadable)."""
    if not os.path.exists(path):
        raise OSError(f"{path} is not built: run __graft_entry__.build() (needs nvcc)")
    lib = ctypes.CDLL(path)
    for name, res, args in SIGNATURES:
        fn = getattr(lib, name)
        fn.restype = res
        fn.argtypes = args
    return lib


def exported(path: str = LIB_PATH) -> dict:
    """{name: True/False} for every entry point the header declares."""
    lib = ctypes.CDLL(path)
    return {name: hasattr(lib, name) for name, _, _ in SIGNATURES}


def lib() -> ctypes.CDLL:
    global _lib
    with _lock:
        if _lib is None:
            _lib = load()
    return _lib


class QCError(RuntimeError):
    def __init__(self, status: int, message: str):
        self.status = status
        self.status_name = STATUS.get(status, str(status))
        super().__init__(f"{self.status_name}: {message}")


def check(status: int, ctx_handle=None) -> None:
    if status != 0:
        L = lib()
        msg = L.qc_last_error(ctx_handle).decode() if ctx_handle else ""
        if not msg:
            msg = L.qc_status_string(status).decode()
        raise QCError(status, msg)

"""qcgraph — graph Quantum Clustering (arXiv 2305.14641) on one GB300.

Python front end of libqcgraph.so.  PyTorch provides device memory (output
tensors, and optionally the library's scratch through its caching allocator)
and streams; every step of the method runs in the library's CUDA kernels.

    ctx = Context()                       # device 0
    g = Graph(ctx, row_ptr, col_idx)      # int32 CSR, host numpy or device tensors
    V = g.potential([0.5, 1.0, 2.0])      # float64 [3, n] on the GPU
    labels, counts = g.ggd_labels(V)      # int32 [3, n] root ids, clusters per sigma
"""
from __future__ import annotations

import ctypes
from typing import Sequence

import numpy as np

from . import native
from .native import QCError

__all__ = ["Context", "Graph", "BatchPlan", "Server", "QCError", "solve_batch"]


def _torch():
    import torch
    return torch


def _stream_handle(stream) -> int:
    torch = _torch()
    if stream is None:
        stream = torch.cuda.current_stream()
    return int(stream.cuda_stream) if hasattr(stream, "cuda_stream") else int(stream)


class Context:
    """A library context on one CUDA device.

    allocator: "torch" routes the library's scratch through PyTorch's caching
    allocator; "cuda" uses cudaMallocAsync.  mem_budget_bytes caps what the
    library holds at once (0 = no cap).
    """

    def __init__(self, device: int = 0, mem_budget_bytes: int = 0, allocator: str = "torch"):
        self._lib = native.lib()
        torch = _torch()
        if not torch.cuda.is_available():
            raise QCError(5, "no CUDA device available (there is no CPU fallback)")
        self.device = int(device)
        torch.cuda.set_device(self.device)
        self._alloc_struct = None
        alloc_ptr = None
        if allocator == "torch":
            dev = self.device

            def _alloc(nbytes, stream, user):
                try:
                    return torch.cuda.caching_allocator_alloc(int(nbytes), dev, stream or 0)
                except Exception:   # out of memory: the library reports QC_ERR_OOM
                    return None

            def _free(ptr, nbytes, stream, user):
                torch.cuda.caching_allocator_delete(ptr)

            self._cb = (native.ALLOC_FN(_alloc), native.FREE_FN(_free))
            self._alloc_struct = native.qc_allocator(self._cb[0], self._cb[1], None)
            alloc_ptr = ctypes.byref(self._alloc_struct)
        elif allocator != "cuda":
            raise ValueError("allocator must be 'torch' or 'cuda'")
        h = ctypes.c_void_p()
        native.check(self._lib.qc_context_create(self.device, int(mem_budget_bytes), alloc_ptr,
                                                 ctypes.byref(h)))
        self.handle = h

    def set_timing(self, enable: bool) -> None:
        self.check(self._lib.qc_context_set_timing(self.handle, int(bool(enable))))

    def kernel_stats(self, kernel: str = "bfs_level", reset: bool = False) -> dict:
        st = native.qc_kernel_stats()
        self.check(self._lib.qc_context_kernel_stats(self.handle, kernel.encode(), ctypes.byref(st),
                                                     int(reset)))
        return {"launches": int(st.launches), "total_ms": float(st.total_ms),
                "model_bytes": float(st.model_bytes)}

    def launch_count(self) -> int:
        return int(self._lib.qc_context_launch_count(self.handle))

    def bytes_in_use(self) -> int:
        return int(self._lib.qc_context_bytes_in_use(self.handle))

    def check(self, status: int) -> None:
        native.check(status, self.handle)

    def close(self) -> None:
        if getattr(self, "handle", None):
            self._lib.qc_context_destroy(self.handle)
            self.handle = None

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()


class Graph:
    """An undirected, unweighted graph resident on the GPU (int32 CSR).

    row_ptr / col_idx: numpy arrays (host) or CUDA int32 tensors (device).
    """

    def __init__(self, ctx: Context, row_ptr, col_idx, validate: bool = True, stream=None):
        self.ctx = ctx
        torch = _torch()
        flags = native.QC_VALIDATE if validate else 0
        if isinstance(row_ptr, torch.Tensor):
            rp = row_ptr.to(device=f"cuda:{ctx.device}", dtype=torch.int32).contiguous()
            ci = col_idx.to(device=f"cuda:{ctx.device}", dtype=torch.int32).contiguous()
            flags |= native.QC_PTR_DEVICE
            n, nnz = rp.numel() - 1, ci.numel()
            p_rp, p_ci = rp.data_ptr(), (ci.data_ptr() if nnz else None)
            keep = (rp, ci)
        else:
            rp = np.ascontiguousarray(row_ptr, dtype=np.int32)
            ci = np.ascontiguousarray(col_idx, dtype=np.int32)
            n, nnz = len(rp) - 1, len(ci)
            p_rp, p_ci = rp.ctypes.data, (ci.ctypes.data if nnz else None)
            keep = (rp, ci)
        h = ctypes.c_void_p()
        ctx.check(ctx._lib.qc_graph_create(ctx.handle, n, nnz, p_rp, p_ci, flags,
                                           _stream_handle(stream), ctypes.byref(h)))
        del keep
        self.handle = h
        self.n = n
        self.nnz = nnz

    @classmethod
    def from_graph(cls, ctx: Context, g, validate: bool = True, stream=None) -> "Graph":
        return cls(ctx, g.row_ptr, g.col_idx, validate=validate, stream=stream)

    def histogram(self, stream=None):
        """int32 tensor [D+1, n]: hist[d][v] = number of nodes at hop distance d from v."""
        torch = _torch()
        D = ctypes.c_int32()
        s = _stream_handle(stream)
        self.ctx.check(self.ctx._lib.qc_graph_histogram(self.handle, None, ctypes.byref(D), s))
        out = torch.empty((D.value + 1, self.n), dtype=torch.int32, device=f"cuda:{self.ctx.device}")
        self.ctx.check(self.ctx._lib.qc_graph_histogram(self.handle, out.data_ptr(), ctypes.byref(D), s))
        return out

    def potential(self, sigmas: Sequence[float], out=None, stream=None):
        """float64 tensor [S, n]: the potential of every node for every sigma."""
        torch = _torch()
        sig = (ctypes.c_double * len(sigmas))(*[float(x) for x in sigmas])
        if out is None:
            out = torch.empty((len(sigmas), self.n), dtype=torch.float64, device=f"cuda:{self.ctx.device}")
        self.ctx.check(self.ctx._lib.qc_potential(self.handle, sig, len(sigmas), out.data_ptr(),
                                                  _stream_handle(stream)))
        return out

    def ggd_labels(self, V, out=None, stream=None, counts: bool = True):
        """(labels int32 tensor [S, n] of root node ids, clusters per sigma or None)."""
        torch = _torch()
        S = V.shape[0] if V.dim() == 2 else 1
        if out is None:
            out = torch.empty((S, self.n), dtype=torch.int32, device=f"cuda:{self.ctx.device}")
        nc = (ctypes.c_int32 * S)() if counts else None
        self.ctx.check(self.ctx._lib.qc_ggd_labels(self.handle, V.data_ptr(), S, out.data_ptr(), nc,
                                                   _stream_handle(stream)))
        return out, (list(nc) if counts else None)

    def solve(self, sigmas: Sequence[float], V_out=None, labels_out=None, stream=None, counts=True):
        """Algorithm 4 for each sigma: (V [S, n] or None, labels [S, n], clusters per sigma)."""
        torch = _torch()
        S = len(sigmas)
        sig = (ctypes.c_double * S)(*[float(x) for x in sigmas])
        if labels_out is None:
            labels_out = torch.empty((S, self.n), dtype=torch.int32, device=f"cuda:{self.ctx.device}")
        nc = (ctypes.c_int32 * S)() if counts else None
        self.ctx.check(self.ctx._lib.qc_solve(self.handle, sig, S,
                                              V_out.data_ptr() if V_out is not None else None,
                                              labels_out.data_ptr(), nc, _stream_handle(stream)))
        return V_out, labels_out, (list(nc) if counts else None)

    def drop_histogram(self) -> None:
        """Forget the cached histogram; the next call runs the BFS again."""
        self.ctx._lib.qc_graph_drop_histogram(self.handle)

    def close(self) -> None:
        if getattr(self, "handle", None):
            self.ctx._lib.qc_graph_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

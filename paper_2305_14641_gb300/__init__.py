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
import weakref
from typing import Sequence

import numpy as np

from . import native
from .native import QCError

__all__ = ["Context", "Graph", "SweepPlan", "BatchPlan", "Server", "QCError", "cluster", "solve_batch", "quality"]


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
        # graphs and plans made on this context (weakly held): the C library requires
        # the context to outlive them, so close() closes any still open first
        self._children = []

    def _adopt(self, obj, rank: int) -> None:
        if len(self._children) >= 64:
            self._children = [c for c in self._children if c[1]() is not None]
        self._children.append((rank, weakref.ref(obj)))

    def set_timing(self, enable: bool) -> None:
        self.check(self._lib.qc_context_set_timing(self.handle, int(bool(enable))))

    def kernel_stats(self, kernel: str = "bfs_level", reset: bool = False) -> dict:
        st = native.qc_kernel_stats()
        self.check(self._lib.qc_context_kernel_stats(self.handle, kernel.encode(), ctypes.byref(st),
                                                     int(reset)))
        return {"launches": int(st.launches), "total_ms": float(st.total_ms),
                "model_bytes": float(st.model_bytes), "min_bytes": float(st.min_bytes)}

    def launch_count(self) -> int:
        return int(self._lib.qc_context_launch_count(self.handle))

    def selftest_barrier_timeout(self, timeout_us: int = 2000, stream=None) -> tuple[str, int]:
        """Run the library's grid barrier with a block that never arrives and a time
        limit of timeout_us; returns (status name, nanoseconds the waiting block
        waited).  QC_ERR_TIMEOUT is the status when the bounded wait gave up as designed."""
        waited = ctypes.c_int64(-1)
        st = self._lib.qc_selftest_barrier_timeout(self.handle, int(timeout_us), ctypes.byref(waited),
                                                   _stream_handle(stream))
        return native.STATUS.get(st, str(st)), int(waited.value)

    def _selftest_arith(self, op: int, x, y, stream):
        torch = _torch()
        dev = f"cuda:{self.device}"
        x = torch.as_tensor(x, dtype=torch.float64, device=dev).contiguous()
        y = None if y is None else torch.as_tensor(y, dtype=torch.float64, device=dev).contiguous()
        out = torch.empty_like(x)
        self.check(self._lib.qc_selftest_arith(self.handle, op, x.data_ptr(), 0 if y is None else y.data_ptr(),
                                               out.data_ptr(), x.numel(), _stream_handle(stream)))
        return out

    def selftest_exp_neg(self, t, stream=None):
        """exp(-t) by the weighted potential's own routine (t: float64, >= 0); returns a
        float64 device tensor."""
        return self._selftest_arith(0, t, None, stream)

    def selftest_debug_check(self, node_id: int, n: int, stream=None) -> tuple[str, int, bool]:
        """Pass node_id through the debug build's bounds check against [0, n) (never as an
        address); returns (status name, the id that came out, whether this is the debug build)."""
        out, dbg = ctypes.c_int32(-1), ctypes.c_int32(-1)
        st = self._lib.qc_selftest_debug_check(self.handle, int(node_id), int(n), ctypes.byref(out), ctypes.byref(dbg),
                                               _stream_handle(stream))
        return native.STATUS.get(st, str(st)), int(out.value), bool(dbg.value)

    def l2_read_gbs(self, nbytes: int = 48 << 20, random_segments: bool = False, stream=None) -> float:
        """Read throughput (GB/s) of an nbytes buffer read through L2 only, streamed or
        as random 512-byte segments (the BFS gather pattern)."""
        out = ctypes.c_double()
        self.check(self._lib.qc_selftest_l2_read(self.handle, int(nbytes), int(bool(random_segments)),
                                                 ctypes.byref(out), _stream_handle(stream)))
        return float(out.value)

    def bytes_in_use(self) -> int:
        return int(self._lib.qc_context_bytes_in_use(self.handle))

    def check(self, status: int) -> None:
        native.check(status, self.handle)

    def close(self) -> None:
        if getattr(self, "handle", None):
            # plans before graphs (a plan holds its graphs), both before the context
            for _, ref in sorted(getattr(self, "_children", []), key=lambda c: c[0]):
                obj = ref()
                if obj is not None:
                    obj.close()
            self._children = []
            self._lib.qc_context_destroy(self.handle)
            self.handle = None

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()


class Graph:
    """An unweighted graph resident on the GPU (int32 CSR), undirected unless
    `directed` (then row v lists the edges v -> u and distances follow them).

    row_ptr / col_idx: numpy arrays (host) or CUDA int32 tensors (device).
    """

    def __init__(self, ctx: Context, row_ptr, col_idx, validate: bool = True, stream=None,
                 directed: bool = False):
        self.ctx = ctx
        torch = _torch()
        flags = native.QC_VALIDATE if validate else 0
        if directed:
            flags |= native.QC_DIRECTED
        self.directed = bool(directed)
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
        ctx._adopt(self, 1)
        self.n = n
        self.nnz = nnz

    @classmethod
    def from_graph(cls, ctx: Context, g, validate: bool = True, stream=None) -> "Graph":
        return cls(ctx, g.row_ptr, g.col_idx, validate=validate, stream=stream,
                   directed=getattr(g, "directed", False))

    def histogram(self, stream=None):
        """int32 tensor [D+1, n]: hist[d][v] = number of nodes at hop distance d from v."""
        torch = _torch()
        D = ctypes.c_int32()
        s = _stream_handle(stream)
        self.ctx.check(self.ctx._lib.qc_graph_histogram(self.handle, None, ctypes.byref(D), s))
        out = torch.empty((D.value + 1, self.n), dtype=torch.int32, device=f"cuda:{self.ctx.device}")
        self.ctx.check(self.ctx._lib.qc_graph_histogram(self.handle, out.data_ptr(), ctypes.byref(D), s))
        return out

    def set_histogram(self, hist, validate: bool = True, stream=None) -> None:
        """Install a histogram saved from `histogram()` of this graph ([D+1, n] int32,
        numpy or CUDA tensor), so later potentials skip the BFS."""
        torch = _torch()
        flags = native.QC_VALIDATE if validate else 0
        if isinstance(hist, torch.Tensor):
            h = hist.to(device=f"cuda:{self.ctx.device}", dtype=torch.int32).contiguous()
            flags |= native.QC_PTR_DEVICE
            ptr = h.data_ptr()
        else:
            h = np.ascontiguousarray(hist, dtype=np.int32)
            ptr = h.ctypes.data
        if h.ndim != 2 or h.shape[1] != self.n:
            raise ValueError(f"histogram must be [D+1, {self.n}], got {tuple(h.shape)}")
        self.ctx.check(self.ctx._lib.qc_graph_set_histogram(self.handle, ptr, int(h.shape[0]) - 1, flags,
                                                            _stream_handle(stream)))

    def potential(self, sigmas: Sequence[float], out=None, stream=None):
        """float64 tensor [S, n]: the potential of every node for every sigma."""
        torch = _torch()
        sig = (ctypes.c_double * len(sigmas))(*[float(x) for x in sigmas])
        if out is None:
            out = torch.empty((len(sigmas), self.n), dtype=torch.float64, device=f"cuda:{self.ctx.device}")
        self.ctx.check(self.ctx._lib.qc_potential(self.handle, sig, len(sigmas), out.data_ptr(),
                                                  _stream_handle(stream)))
        return out

    def set_weights(self, weights, validate: bool = True, stream=None) -> None:
        """Edge weights aligned with col_idx (numpy or CUDA float64 tensor)."""
        torch = _torch()
        flags = native.QC_VALIDATE if validate else 0
        if isinstance(weights, torch.Tensor):
            w = weights.to(device=f"cuda:{self.ctx.device}", dtype=torch.float64).contiguous()
            flags |= native.QC_PTR_DEVICE
            ptr = ctypes.cast(w.data_ptr(), native.c_double_p)
        else:
            w = np.ascontiguousarray(weights, dtype=np.float64)
            ptr = w.ctypes.data_as(native.c_double_p)
        if w.shape != (self.nnz,):
            raise ValueError(f"need one weight per CSR entry ({self.nnz}), got {tuple(w.shape)}")
        self.ctx.check(self.ctx._lib.qc_graph_set_weights(self.handle, ptr, flags, _stream_handle(stream)))

    def potential_weighted(self, sigmas: Sequence[float], out=None, stream=None):
        """float64 tensor [S, n]: the potential over weighted shortest-path distances."""
        torch = _torch()
        S = len(sigmas)
        sig = (ctypes.c_double * S)(*[float(x) for x in sigmas])
        if out is None:
            out = torch.empty((S, self.n), dtype=torch.float64, device=f"cuda:{self.ctx.device}")
        self.ctx.check(self.ctx._lib.qc_potential_weighted(self.handle, sig, S, out.data_ptr(),
                                                           _stream_handle(stream)))
        return out

    def potential_adjacency(self, sigmas: Sequence[float], M: float = 2.0, out=None, stream=None):
        """float64 tensor [S, n]: the potential with the paper-literal distance
        (1 to a neighbour, M to any other node)."""
        torch = _torch()
        sig = (ctypes.c_double * len(sigmas))(*[float(x) for x in sigmas])
        if out is None:
            out = torch.empty((len(sigmas), self.n), dtype=torch.float64, device=f"cuda:{self.ctx.device}")
        self.ctx.check(self.ctx._lib.qc_potential_adjacency(self.handle, sig, len(sigmas), float(M),
                                                            out.data_ptr(), _stream_handle(stream)))
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


class SweepPlan:
    """Algorithm 4 for one graph and a fixed list of sigma values, captured once
    into CUDA graphs and replayed: run() recomputes everything from the resident
    CSR (BFS, potentials, descent, roots); run(reuse_histogram=True) reuses the
    histogram of the plan's last full run.

    V: float64 tensor [S, n] (or None to keep the potentials inside the plan);
    labels: int32 tensor [S, n] of root node ids.  Both are allocated here when not
    given and stay owned by the plan object.
    """

    def __init__(self, graph: Graph, sigmas: Sequence[float], V=None, labels=None, stream=None,
                 keep_potentials: bool = True):
        torch = _torch()
        ctx = graph.ctx
        self.ctx, self.graph = ctx, graph
        S, n = len(sigmas), graph.n
        dev = f"cuda:{ctx.device}"
        self.labels = labels if labels is not None else torch.empty((S, n), dtype=torch.int32, device=dev)
        if V is None and keep_potentials:
            V = torch.empty((S, n), dtype=torch.float64, device=dev)
        self.V = V
        self.S = S
        sig = (ctypes.c_double * S)(*[float(x) for x in sigmas])
        h = ctypes.c_void_p()
        ctx.check(ctx._lib.qc_sweep_create(graph.handle, sig, S, V.data_ptr() if V is not None else None,
                                           self.labels.data_ptr(), _stream_handle(stream), ctypes.byref(h)))
        self.handle = h
        ctx._adopt(self, 0)

    def run(self, reuse_histogram: bool = False, counts: bool = False, stream=None):
        """One run; returns the clusters per sigma (host ints) when counts, else None."""
        nc = (ctypes.c_int32 * self.S)() if counts else None
        self.ctx.check(self.ctx._lib.qc_sweep_run(self.handle, int(bool(reuse_histogram)), nc,
                                                  _stream_handle(stream)))
        return list(nc) if counts else None

    def info(self) -> dict:
        """D of the last full run, whether runs replay captured CUDA graphs, kernels per full run."""
        D, cap, k = ctypes.c_int32(), ctypes.c_int32(), ctypes.c_int64()
        self.ctx.check(self.ctx._lib.qc_sweep_info(self.handle, ctypes.byref(D), ctypes.byref(cap), ctypes.byref(k)))
        return {"D": D.value, "captured": bool(cap.value), "kernels_per_run": k.value}

    def close(self) -> None:
        if getattr(self, "handle", None):
            self.ctx._lib.qc_sweep_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class BatchPlan:
    """Algorithm 4 for many graphs at once (one sigma per graph), planned once and
    replayed: one persistent graph-per-CTA kernel captured in a CUDA graph.

    labels: int32 tensor [sum of n] on the GPU; graph k's labels (root node ids,
    local to graph k) are labels[offsets[k] : offsets[k] + n_k].
    """

    def __init__(self, ctx: Context, graphs: Sequence[Graph], sigmas: Sequence[float], stream=None):
        torch = _torch()
        if len(graphs) != len(sigmas) or not graphs:
            raise ValueError("need one sigma per graph and at least one graph")
        self.ctx = ctx
        self.graphs = list(graphs)
        sizes = [g.n for g in graphs]
        self.offsets = np.concatenate([[0], np.cumsum(sizes)[:-1]]).astype(np.int64)
        self.labels = torch.empty(int(sum(sizes)), dtype=torch.int32, device=f"cuda:{ctx.device}")
        arr = (ctypes.c_void_p * len(graphs))(*[g.handle.value for g in graphs])
        sig = (ctypes.c_double * len(graphs))(*[float(s) for s in sigmas])
        off = (ctypes.c_int64 * len(graphs))(*[int(o) for o in self.offsets])
        h = ctypes.c_void_p()
        ctx.check(ctx._lib.qc_batch_create(ctx.handle, len(graphs), arr, sig, self.labels.data_ptr(), off,
                                           _stream_handle(stream), ctypes.byref(h)))
        self.handle = h
        ctx._adopt(self, 0)

    def run(self, stream=None, counts: bool = True):
        """Run the plan; returns the clusters per graph (host ints) or None."""
        nc = (ctypes.c_int32 * len(self.graphs))() if counts else None
        self.ctx.check(self.ctx._lib.qc_batch_run(self.handle, nc, _stream_handle(stream)))
        return list(nc) if counts else None

    def config(self) -> dict:
        """The kernel configuration the plan runs (threads per CTA, source words per
        chunk, mean degree below which a thread takes a node)."""
        t, c, sd = ctypes.c_int32(), ctypes.c_int32(), ctypes.c_int32()
        self.ctx.check(self.ctx._lib.qc_batch_config(self.handle, ctypes.byref(t), ctypes.byref(c),
                                                     ctypes.byref(sd)))
        return {"threads": t.value, "chunk_words": c.value, "sparse_degree": sd.value}

    def labels_of(self, k: int):
        o = int(self.offsets[k])
        return self.labels[o:o + self.graphs[k].n]

    def close(self) -> None:
        if getattr(self, "handle", None):
            self.ctx._lib.qc_batch_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def quality(ctx: Context, labels, graph: "Graph" = None, truth=None, n_truth: int | None = None,
            gamma: float = 1.0, stream=None) -> dict:
    """Modularity (with graph), ARI, FMI and NMI (with truth) of a label vector on the
    GPU (int32 root ids, as the solve writes them), computed on the device."""
    torch = _torch()
    dev = f"cuda:{ctx.device}"
    lab = torch.as_tensor(labels, device=dev).to(torch.int32).contiguous().reshape(-1)
    n = lab.numel()
    tr = None
    if truth is not None:
        tr = torch.as_tensor(truth, device=dev).to(torch.int32).contiguous().reshape(-1)
        if n_truth is None:
            n_truth = int(tr.max().item()) + 1
    if graph is not None and graph.n != n:
        raise ValueError("labels and graph differ in size")
    out = native.qc_quality_result()
    ctx.check(ctx._lib.qc_quality(ctx.handle, graph.handle if graph is not None else None, n, lab.data_ptr(),
                                  tr.data_ptr() if tr is not None else None, int(n_truth or 0), float(gamma),
                                  ctypes.byref(out), _stream_handle(stream)))
    return {"modularity": out.modularity, "ari": out.ari, "fmi": out.fmi, "nmi": out.nmi, "clusters": out.clusters}


def cluster(ctx: Context, row_ptr, col_idx, sigmas: Sequence[float], labels_out=None, counts: bool = True,
            validate: bool = True, directed: bool = False, stream=None):
    """Algorithm 4 from a CSR to labels in one library call (the graph is not kept).

    row_ptr / col_idx: numpy arrays (host) or CUDA int32 tensors.  labels_out: an
    int32 [S, n] torch tensor (pinned host or CUDA) or numpy array to write into;
    by default a new numpy array.  Returns (labels, clusters per sigma or None)."""
    torch = _torch()
    flags = (native.QC_VALIDATE if validate else 0) | (native.QC_DIRECTED if directed else 0)
    if isinstance(row_ptr, torch.Tensor):
        rp = row_ptr.to(device=f"cuda:{ctx.device}", dtype=torch.int32).contiguous()
        ci = col_idx.to(device=f"cuda:{ctx.device}", dtype=torch.int32).contiguous()
        flags |= native.QC_PTR_DEVICE
        n, nnz = rp.numel() - 1, ci.numel()
        p_rp, p_ci = rp.data_ptr(), (ci.data_ptr() if nnz else None)
    else:
        rp = np.ascontiguousarray(row_ptr, dtype=np.int32)
        ci = np.ascontiguousarray(col_idx, dtype=np.int32)
        n, nnz = len(rp) - 1, len(ci)
        p_rp, p_ci = rp.ctypes.data, (ci.ctypes.data if nnz else None)
    S = len(sigmas)
    if labels_out is None:
        labels_out = np.empty((S, n), dtype=np.int32)
    if isinstance(labels_out, torch.Tensor):
        assert labels_out.dtype == torch.int32 and labels_out.is_contiguous() and labels_out.numel() == S * n
        p_lab = labels_out.data_ptr()
    else:
        assert labels_out.dtype == np.int32 and labels_out.flags.c_contiguous and labels_out.size == S * n
        p_lab = labels_out.ctypes.data
    sig = (ctypes.c_double * S)(*[float(x) for x in sigmas])
    nc = (ctypes.c_int32 * S)() if counts else None
    ctx.check(ctx._lib.qc_cluster(ctx.handle, n, nnz, p_rp, p_ci, flags, sig, S, p_lab, nc,
                                  _stream_handle(stream)))
    return labels_out, (list(nc) if counts else None)


def solve_batch(ctx: Context, graphs: Sequence[Graph], sigmas: Sequence[float], stream=None):
    """One-shot batched solve: (labels tensor, offsets)."""
    plan = BatchPlan(ctx, graphs, sigmas, stream)
    plan.run(stream, counts=False)
    labels, offsets = plan.labels, plan.offsets
    plan.close()
    return labels, offsets


class Server:
    """A serving loop (host threads inside the library): submit CSR graphs with a
    sigma each, collect labels.  Uses its own context with the stream-ordered CUDA
    allocator so that the library's threads never call back into Python."""

    def __init__(self, device: int = 0, mem_budget_bytes: int = 100 << 30, max_active: int = 256,
                 streams: int = 4, large_workers: int = 4, large_sm_share: float = 0.4,
                 divide_share: bool = False):
        self.ctx = Context(device, allocator="cuda")
        cfg = native.qc_server_config(int(mem_budget_bytes), int(max_active), int(streams),
                                      int(large_workers), float(large_sm_share), int(bool(divide_share)))
        h = ctypes.c_void_p()
        self.ctx.check(self.ctx._lib.qc_server_create(self.ctx.handle, ctypes.byref(cfg), ctypes.byref(h)))
        self.handle = h
        self._n = {}

    def submit(self, row_ptr, col_idx, sigma: float) -> int:
        rp = np.ascontiguousarray(row_ptr, dtype=np.int32)
        ci = np.ascontiguousarray(col_idx, dtype=np.int32)
        rid = ctypes.c_uint64()
        self.ctx.check(self.ctx._lib.qc_server_submit(self.handle, len(rp) - 1, len(ci), rp.ctypes.data,
                                                      ci.ctypes.data if len(ci) else None, float(sigma),
                                                      ctypes.byref(rid)))
        self._n[rid.value] = len(rp) - 1
        return rid.value

    def submit_graph(self, graph: "Graph", sigma: float) -> int:
        """Queue a request on a graph resident on the GPU (made with Graph(server.ctx, ...));
        later sigmas on the same graph reuse its cached histogram."""
        rid = ctypes.c_uint64()
        self.ctx.check(self.ctx._lib.qc_server_submit_graph(self.handle, graph.handle, float(sigma),
                                                            ctypes.byref(rid)))
        self._n[rid.value] = graph.n
        return rid.value

    def _result(self, rid, labels, nc, info):
        return {"labels": labels, "n_clusters": nc.value, "admit_ms": info.admit_ms, "start_ms": info.start_ms,
                "latency_ms": info.done_ms, "batch_size": info.batch_size}

    def poll(self, rid: int):
        """The result dict if the request has completed, else None."""
        n = self._n[rid]
        labels = np.empty(n, dtype=np.int32)
        nc = ctypes.c_int32()
        info = native.qc_request_info()
        done = ctypes.c_int()
        st = self.ctx._lib.qc_server_poll(self.handle, rid, labels.ctypes.data, ctypes.byref(nc),
                                          ctypes.byref(info), ctypes.byref(done))
        if not done.value:
            self.ctx.check(st)
            return None
        self._n.pop(rid, None)
        self.ctx.check(st)
        return self._result(rid, labels, nc, info)

    def wait(self, rid: int, timeout_ms: int = -1):
        n = self._n[rid]
        labels = np.empty(n, dtype=np.int32)
        nc = ctypes.c_int32()
        info = native.qc_request_info()
        st = self.ctx._lib.qc_server_wait(self.handle, rid, int(timeout_ms), labels.ctypes.data,
                                          ctypes.byref(nc), ctypes.byref(info))
        if st != 8:
            self._n.pop(rid, None)
        self.ctx.check(st)
        return self._result(rid, labels, nc, info)

    def cancel(self, rid: int) -> None:
        self.ctx.check(self.ctx._lib.qc_server_cancel(self.handle, rid))

    def stats(self) -> dict:
        s = native.qc_server_stats()
        self.ctx.check(self.ctx._lib.qc_server_get_stats(self.handle, ctypes.byref(s)))
        return {k: getattr(s, k) for k, _ in s._fields_}

    def close(self) -> None:
        if getattr(self, "handle", None):
            self.ctx._lib.qc_server_destroy(self.handle)
            self.handle = None
            self.ctx.close()

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

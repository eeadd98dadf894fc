"""Plain CPU oracle for graph Quantum Clustering (arXiv 2305.14641).

TEST INFRASTRUCTURE ONLY: imported by ``tests/``, by the package's ``smoke()``
check and by the benchmark's CPU-baseline leg, never by the library.  The
arithmetic lives in ``qc_oracle.c`` (plain C, binary64, no fused multiply-add);
this module compiles it with gcc and marshals numpy arrays through ctypes.

Per function, the passage it follows:
  * ``bfs``            hop distance between nodes (Section 3.1)
  * ``histograms``     h_i(d) = #{j : dist(i, j) = d}, j over all nodes (Algorithm 1)
  * ``potential``      Eq. 7 (last line) / Algorithm 1, grouped by distance
  * ``potential_literal``  Algorithm 1 term by term, one exp per pair
  * ``ggd_parent``     Algorithm 2 with the strict-descent reading of the prose
                       after Algorithm 4
  * ``find_centers``   Algorithm 3 (root of each parent chain)
  * ``solve``          Algorithm 4: potentials for every node, then GGD labels
  * ``potential_adjacency``  Section 3.1 read literally: distance 1 on an edge,
                       M (above every weight) between non-adjacent nodes
  * ``dijkstra``       Section 3.1 with edge weights: shortest weighted path
                       lengths from one node (Dijkstra, binary heap)
  * ``potential_weighted``  Algorithm 1 over those lengths, pair by pair
Directed graphs (rows = arcs i -> j) need nothing special: every function
follows the rows, so distances run along the arcs.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "qc_oracle.c")
_LIB = os.path.join(_HERE, "liboracle.so")
_lock = threading.Lock()

_i32p = np.ctypeslib.ndpointer(dtype=np.int32, flags="C_CONTIGUOUS")
_f64p = np.ctypeslib.ndpointer(dtype=np.float64, flags="C_CONTIGUOUS")


def compile_source(src: str, out: str) -> str:
    """gcc -O2, binary64 with no fused multiply-add, as a shared library."""
    tmp = out + f".{os.getpid()}.tmp"
    subprocess.check_call(["gcc", "-O2", "-std=c11", "-ffp-contract=off", "-fno-fast-math",
                           "-fPIC", "-shared", "-o", tmp, src, "-lm", "-lpthread"])
    os.replace(tmp, out)
    return out


def build(force: bool = False) -> str:
    """Compile qc_oracle.c into liboracle.so."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        compile_source(_SRC, _LIB)
    return _LIB


def _bind(lib):
    lib.qco_bfs.restype = ctypes.c_int32
    lib.qco_bfs.argtypes = [ctypes.c_int32, _i32p, _i32p, ctypes.c_int32, _i32p, _i32p]
    lib.qco_histograms.restype = ctypes.c_int
    lib.qco_histograms.argtypes = [ctypes.c_int32, _i32p, _i32p, ctypes.c_int64, _i32p,
                                   ctypes.c_int32, _i32p, _i32p, ctypes.c_int]
    lib.qco_weights.restype = None
    lib.qco_weights.argtypes = [ctypes.c_double, ctypes.c_int32, _f64p, _f64p]
    lib.qco_potential_hist.restype = None
    lib.qco_potential_hist.argtypes = [_i32p, ctypes.c_int64, ctypes.c_int32,
                                       ctypes.c_double, _f64p]
    lib.qco_potential_literal.restype = ctypes.c_double
    lib.qco_potential_literal.argtypes = [_i32p, ctypes.c_int32, ctypes.c_double]
    lib.qco_ggd_parent.restype = ctypes.c_int64
    lib.qco_ggd_parent.argtypes = [ctypes.c_int32, _i32p, _i32p, _f64p, _i32p]
    lib.qco_find_centers.restype = ctypes.c_int32
    lib.qco_find_centers.argtypes = [ctypes.c_int32, _i32p, _i32p]
    lib.qco_potential_adjacency.restype = None
    lib.qco_potential_adjacency.argtypes = [ctypes.c_int32, _i32p, ctypes.c_double, ctypes.c_double, _f64p]
    lib.qco_dijkstra.restype = ctypes.c_int
    lib.qco_dijkstra.argtypes = [ctypes.c_int32, _i32p, _i32p, _f64p, ctypes.c_int32, _f64p]
    lib.qco_potential_weighted.restype = ctypes.c_int
    lib.qco_potential_weighted.argtypes = [ctypes.c_int32, _i32p, _i32p, _f64p, _f64p, ctypes.c_int32, _f64p,
                                           ctypes.c_int]
    return lib


def _csr(graph):
    return (np.ascontiguousarray(graph.row_ptr, dtype=np.int32),
            np.ascontiguousarray(graph.col_idx, dtype=np.int32))


def default_threads() -> int:
    if hasattr(os, "sched_getaffinity"):
        return max(1, len(os.sched_getaffinity(0)))
    return max(1, os.cpu_count() or 1)


class Oracle:
    """The oracle's functions bound to one compiled copy of the C source (the
    default copy is liboracle.so; tests may load a deliberately broken copy)."""

    def __init__(self, lib_path: str):
        self._lib = _bind(ctypes.CDLL(lib_path))

    def bfs(self, graph, src: int) -> np.ndarray:
        """Hop distances from src (-1 = unreachable)."""
        rp, ci = _csr(graph)
        dist = np.empty(graph.n, dtype=np.int32)
        queue = np.empty(graph.n, dtype=np.int32)
        self._lib.qco_bfs(graph.n, rp, ci, int(src), dist, queue)
        return dist

    def histograms(self, graph, nodes=None, threads: int = 1, cap: int = 32) -> np.ndarray:
        """h[k][d] = #{j : dist(nodes[k], j) = d}, node-major, trimmed to the largest
        distance found (the number of columns is D + 1)."""
        rp, ci = _csr(graph)
        if nodes is None:
            nodes = np.arange(graph.n, dtype=np.int32)
        nodes = np.ascontiguousarray(nodes, dtype=np.int32)
        cap = max(2, min(int(cap), graph.n + 1))
        while True:
            hist = np.empty((len(nodes), cap), dtype=np.int32)
            ecc = np.empty(len(nodes), dtype=np.int32)
            st = self._lib.qco_histograms(graph.n, rp, ci, len(nodes), nodes, cap, hist, ecc,
                                          int(threads))
            if st == -2:
                raise MemoryError("oracle histogram scratch allocation failed")
            if st == 0:
                D = int(ecc.max()) if len(nodes) else 0
                return np.ascontiguousarray(hist[:, :D + 1])
            cap = min(graph.n + 1, max(cap * 2, int(ecc.max()) + 1))

    def weights(self, sigma: float, length: int) -> tuple[np.ndarray, np.ndarray]:
        w = np.empty(length, dtype=np.float64)
        u = np.empty(length, dtype=np.float64)
        self._lib.qco_weights(float(sigma), int(length), w, u)
        return w, u

    def potential(self, hist: np.ndarray, sigma: float) -> np.ndarray:
        """V per row of a node-major histogram (canonical ascending-distance sum)."""
        hist = np.ascontiguousarray(hist, dtype=np.int32)
        V = np.empty(hist.shape[0], dtype=np.float64)
        self._lib.qco_potential_hist(hist, hist.shape[0], hist.shape[1], float(sigma), V)
        return V

    def potential_literal(self, graph, node: int, sigma: float) -> float:
        """Algorithm 1 as written (per-pair exp), for one node."""
        d = self.bfs(graph, node)
        return float(self._lib.qco_potential_literal(d, graph.n, float(sigma)))

    def potential_adjacency(self, graph, sigma: float, M: float = 2.0) -> np.ndarray:
        """V with the paper-literal distance: 0 to itself, 1 to a neighbour, M otherwise."""
        rp, _ = _csr(graph)
        V = np.empty(graph.n, dtype=np.float64)
        self._lib.qco_potential_adjacency(graph.n, rp, float(M), float(sigma), V)
        return V

    def dijkstra(self, graph, weights, src: int) -> np.ndarray:
        """Weighted shortest-path lengths from src (+inf where unreachable)."""
        rp, ci = _csr(graph)
        w = np.ascontiguousarray(weights, dtype=np.float64)
        dist = np.empty(graph.n, dtype=np.float64)
        if self._lib.qco_dijkstra(graph.n, rp, ci, w, int(src), dist) != 0:
            raise MemoryError("oracle Dijkstra scratch allocation failed")
        return dist

    def potential_weighted(self, graph, weights, sigmas, threads: int = 1) -> np.ndarray:
        """V [S, n] over weighted shortest-path distances, summed pair by pair."""
        rp, ci = _csr(graph)
        w = np.ascontiguousarray(weights, dtype=np.float64)
        sig = np.ascontiguousarray(np.atleast_1d(sigmas), dtype=np.float64)
        V = np.empty((len(sig), graph.n), dtype=np.float64)
        if self._lib.qco_potential_weighted(graph.n, rp, ci, w, sig, len(sig), V, int(threads)) != 0:
            raise MemoryError("oracle weighted potential scratch allocation failed")
        return V

    def ggd_parent(self, graph, V: np.ndarray) -> tuple[np.ndarray, int]:
        """(parent, number of index-dependent ties)."""
        rp, ci = _csr(graph)
        V = np.ascontiguousarray(V, dtype=np.float64)
        parent = np.empty(graph.n, dtype=np.int32)
        ties = self._lib.qco_ggd_parent(graph.n, rp, ci, V, parent)
        return parent, int(ties)

    def find_centers(self, parent: np.ndarray) -> tuple[np.ndarray, int]:
        """(label = root id per node, number of roots)."""
        parent = np.ascontiguousarray(parent, dtype=np.int32)
        label = np.empty(len(parent), dtype=np.int32)
        roots = self._lib.qco_find_centers(len(parent), parent, label)
        return label, int(roots)

    def solve(self, graph, sigmas, threads: int = 1) -> "Solution":
        """Algorithm 4 for each sigma: V for every node, then GGD and cluster centers."""
        hist = self.histograms(graph, threads=threads)
        Vs, parents, labels, counts, ties = [], [], [], [], []
        for s in sigmas:
            V = self.potential(hist, s)
            p, t = self.ggd_parent(graph, V)
            lab, k = self.find_centers(p)
            Vs.append(V)
            parents.append(p)
            labels.append(lab)
            counts.append(k)
            ties.append(t)
        return Solution(hist, np.stack(Vs), np.stack(parents), np.stack(labels), counts, ties)


_default = None


def default() -> Oracle:
    global _default
    with _lock:
        if _default is None:
            _default = Oracle(build())
    return _default


def bfs(graph, src):
    return default().bfs(graph, src)


def histograms(graph, nodes=None, threads=1, cap=32):
    return default().histograms(graph, nodes, threads, cap)


def weights(sigma, length):
    return default().weights(sigma, length)


def potential(hist, sigma):
    return default().potential(hist, sigma)


def potential_literal(graph, node, sigma):
    return default().potential_literal(graph, node, sigma)


def potential_adjacency(graph, sigma, M=2.0):
    return default().potential_adjacency(graph, sigma, M)


def dijkstra(graph, weights, src):
    return default().dijkstra(graph, weights, src)


def potential_weighted(graph, weights, sigmas, threads=1):
    return default().potential_weighted(graph, weights, sigmas, threads)


def ggd_parent(graph, V):
    return default().ggd_parent(graph, V)


def find_centers(parent):
    return default().find_centers(parent)


def solve(graph, sigmas, threads=1):
    return default().solve(graph, sigmas, threads)


class Solution:
    """Everything the oracle computes for one graph and a list of sigma values."""

    def __init__(self, hist, V, parent, labels, n_clusters, ties):
        self.hist = hist              # int32 [n][D+1], node-major
        self.V = V                    # float64 [S][n]
        self.parent = parent          # int32 [S][n]
        self.labels = labels          # int32 [S][n]
        self.n_clusters = n_clusters  # list[int]
        self.ties = ties              # list[int]

    @property
    def D(self) -> int:
        return self.hist.shape[1] - 1

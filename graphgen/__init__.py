"""Seeded synthetic graph generators, shared as *inputs* by the oracle tests and
the CUDA path.

This module holds none of the clustering method's arithmetic: it only draws
unweighted graphs (int32 CSR; undirected unless a generator says directed) and
per-graph parameters (sigma values, request arrival times) from seeded
pseudo-random streams.

Random numbers: numpy's PCG64 bit generator (O'Neill 2014), seeded through
``SeedSequence([seed, *tags])`` so that every graph, block pair and request has
its own independent stream.  Bernoulli edge sampling with one probability per
block pair uses geometric skipping (Batagelj & Brandes 2005, "Efficient
generation of large random networks"), which draws one variate per kept edge
instead of one per candidate pair.  The degree-corrected SBM, whose pair
probabilities differ per pair, is sampled pair by pair.

Every graph returned is canonical: no self-loops, no duplicate edges, rows
sorted ascending, and symmetric unless it is directed (row v then lists the
edges v -> u).
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np

__all__ = [
    "Graph", "rng", "csr_from_pairs", "block_sizes", "planted_partition",
    "sbm_mean_degree", "dcsbm", "complete", "path", "star", "two_cliques_bridge",
    "erdos_renyi", "relabel", "planted128", "dcsbm16384", "sbm262144", "planted_batch",
    "sbm_request_stream", "sigma_sweep16", "planted_batch_graph", "Request", "csr_from_arcs", "directed_cycle",
    "directed_path", "directed_erdos_renyi", "directed_planted_partition", "edge_weights",
]


@dataclass
class Graph:
    n: int
    row_ptr: np.ndarray          # int32[n+1]
    col_idx: np.ndarray          # int32[nnz]
    name: str = ""
    block: np.ndarray | None = None   # planted community of each node, when there is one
    meta: dict = field(default_factory=dict)
    directed: bool = False            # row v lists the edges v -> u

    @property
    def nnz(self) -> int:
        return int(self.row_ptr[-1])

    def degrees(self) -> np.ndarray:
        return np.diff(self.row_ptr.astype(np.int64))

    def neighbors(self, v: int) -> np.ndarray:
        return self.col_idx[self.row_ptr[v]:self.row_ptr[v + 1]]


def rng(seed: int, *tags: int) -> np.random.Generator:
    """An independent PCG64 stream for (seed, *tags)."""
    return np.random.Generator(np.random.PCG64(np.random.SeedSequence([int(seed)] + [int(t) for t in tags])))


def csr_from_pairs(n: int, i: np.ndarray, j: np.ndarray) -> tuple[np.ndarray, np.ndarray]:
    """Undirected CSR from unordered pairs: symmetrised, deduplicated, no self-loops, rows sorted."""
    i = np.asarray(i, dtype=np.int64)
    j = np.asarray(j, dtype=np.int64)
    keep = i != j
    i, j = i[keep], j[keep]
    keys = np.sort(np.concatenate([i * n + j, j * n + i]))
    if keys.size:
        keys = keys[np.concatenate([[True], keys[1:] != keys[:-1]])]
    rows = keys // n
    cols = keys - rows * n
    row_ptr = np.zeros(n + 1, dtype=np.int64)
    np.cumsum(np.bincount(rows, minlength=n), out=row_ptr[1:])
    if row_ptr[-1] >= 2**31:
        raise ValueError("graph has 2^31 or more directed edges; int32 CSR cannot hold it")
    return row_ptr.astype(np.int32), cols.astype(np.int32)


def csr_from_arcs(n: int, i: np.ndarray, j: np.ndarray) -> tuple[np.ndarray, np.ndarray]:
    """Directed CSR from arcs i -> j: deduplicated, no self-loops, rows sorted."""
    i = np.asarray(i, dtype=np.int64)
    j = np.asarray(j, dtype=np.int64)
    keep = i != j
    keys = np.unique(i[keep] * n + j[keep])
    rows = keys // n
    row_ptr = np.zeros(n + 1, dtype=np.int64)
    np.cumsum(np.bincount(rows, minlength=n), out=row_ptr[1:])
    if row_ptr[-1] >= 2**31:
        raise ValueError("graph has 2^31 or more arcs; int32 CSR cannot hold it")
    return row_ptr.astype(np.int32), (keys - rows * n).astype(np.int32)


def block_sizes(n: int, k: int) -> np.ndarray:
    """k block sizes as equal as possible (the first n % k blocks are one node larger)."""
    base, extra = divmod(n, k)
    return np.array([base + (1 if b < extra else 0) for b in range(k)], dtype=np.int64)


def _bernoulli_positions(g: np.random.Generator, m: int, p: float) -> np.ndarray:
    """Positions in [0, m) kept independently with probability p (geometric skipping)."""
    if m <= 0 or p <= 0.0:
        return np.zeros(0, dtype=np.int64)
    if p >= 1.0:
        return np.arange(m, dtype=np.int64)
    logq = math.log1p(-p)
    out = []
    pos = -1
    while True:
        expected = (m - pos - 1) * p
        cnt = int(expected + 6.0 * math.sqrt(expected) + 16)
        u = g.random(cnt)
        steps = np.floor(np.log1p(-u) / logq).astype(np.int64) + 1
        positions = pos + np.cumsum(steps)
        keep = positions < m
        out.append(positions[keep])
        if not keep[-1]:
            break
        pos = int(positions[-1])
    return np.concatenate(out)


def _intra_pairs(starts: np.ndarray, sizes: np.ndarray, t: np.ndarray) -> tuple[np.ndarray, np.ndarray]:
    """Map linear indices over the concatenated within-block pair lists to node pairs.

    Block b lists its pairs (r, c), r < c < size_b, ordered by c then r: index c(c-1)/2 + r.
    """
    pairs = sizes * (sizes - 1) // 2
    cum = np.cumsum(pairs)
    b = np.searchsorted(cum, t, side="right")
    tl = t - (cum[b] - pairs[b])
    c = np.floor((1.0 + np.sqrt(1.0 + 8.0 * tl.astype(np.float64))) / 2.0).astype(np.int64)
    for _ in range(2):
        c = np.where(c * (c - 1) // 2 > tl, c - 1, c)
        c = np.where((c + 1) * c // 2 <= tl, c + 1, c)
    r = tl - c * (c - 1) // 2
    return starts[b] + r, starts[b] + c


def _inter_pairs(n: int, block_end: np.ndarray, t: np.ndarray) -> tuple[np.ndarray, np.ndarray]:
    """Map linear indices over the across-block pairs (i, j), j in a later block than i, to node pairs."""
    counts = n - block_end                     # per row i
    cum = np.cumsum(counts)
    i = np.searchsorted(cum, t, side="right")
    local = t - (cum[i] - counts[i])
    return i, block_end[i] + local


def planted_partition(n: int, k: int, p_in: float, p_out: float, g: np.random.Generator,
                      name: str = "") -> Graph:
    """Planted partition / plain SBM: k consecutive blocks as equal as possible;
    a pair is an edge with probability p_in inside a block and p_out across."""
    sizes = block_sizes(n, k)
    starts = np.concatenate([[0], np.cumsum(sizes)[:-1]]).astype(np.int64)
    block = np.repeat(np.arange(k, dtype=np.int32), sizes)
    m_in = int((sizes * (sizes - 1) // 2).sum())
    t_in = _bernoulli_positions(g, m_in, p_in)
    i1, j1 = _intra_pairs(starts, sizes, t_in)
    block_end = (starts + sizes)[block]
    m_out = int((n - block_end).sum())
    t_out = _bernoulli_positions(g, m_out, p_out)
    i2, j2 = _inter_pairs(n, block_end, t_out)
    row_ptr, col_idx = csr_from_pairs(n, np.concatenate([i1, i2]), np.concatenate([j1, j2]))
    return Graph(n, row_ptr, col_idx, name=name, block=block,
                 meta={"k": k, "p_in": p_in, "p_out": p_out})


def sbm_mean_degree(n: int, k: int, mean_deg: float, mu: float, g: np.random.Generator,
                    name: str = "") -> Graph:
    """Plain SBM with a target mean degree and mixing fraction mu (expected share of
    each node's edges that leave its block)."""
    nc = n / k
    p_in = min(1.0, mean_deg * (1.0 - mu) / max(nc - 1.0, 1.0))
    p_out = min(1.0, mean_deg * mu / max(n - nc, 1.0))
    return planted_partition(n, k, p_in, p_out, g, name=name)


def _truncated_pareto_mean(theta_min: float, theta_max: float, alpha: float) -> float:
    r = theta_min / theta_max
    return alpha * theta_min / (alpha - 1.0) * (1.0 - r ** (alpha - 1.0)) / (1.0 - r ** alpha)


def dcsbm(n: int, k: int, gamma: float, mean_deg: float, theta_max: float, mu: float,
          g: np.random.Generator, name: str = "") -> Graph:
    """Degree-corrected SBM (Karrer & Newman 2011 style) with Bernoulli edges.

    Expected degrees follow a power law with density exponent gamma (density of theta
    proportional to theta^-gamma, i.e. Pareto tail index alpha = gamma - 1), truncated to
    [theta_min, theta_max], theta_min chosen so that E[theta] = mean_deg.  Same block c: p_ij = min(1, (1-mu) theta_i theta_j / K_c);
    different blocks: p_ij = min(1, mu theta_i theta_j / (K - K/k)), K = sum theta,
    K_c = sum of theta over block c.
    """
    alpha = gamma - 1.0
    lo, hi = 1e-6, mean_deg
    for _ in range(200):
        mid = 0.5 * (lo + hi)
        if _truncated_pareto_mean(mid, theta_max, alpha) < mean_deg:
            lo = mid
        else:
            hi = mid
    theta_min = 0.5 * (lo + hi)
    u = g.random(n)
    r = (theta_min / theta_max) ** alpha
    theta = theta_min * (1.0 - u * (1.0 - r)) ** (-1.0 / alpha)
    sizes = block_sizes(n, k)
    block = np.repeat(np.arange(k, dtype=np.int64), sizes)
    K = theta.sum()
    Kc = np.bincount(block, weights=theta, minlength=k)
    c_in = (1.0 - mu) / Kc
    c_out = mu / (K - K / k)
    src, dst = [], []
    target = 1 << 24
    i0 = 0
    while i0 < n - 1:
        i1 = i0
        tot = 0
        while i1 < n - 1 and tot < target:
            tot += n - 1 - i1
            i1 += 1
        counts = n - 1 - np.arange(i0, i1, dtype=np.int64)
        rows = np.repeat(np.arange(i0, i1, dtype=np.int64), counts)
        starts = np.cumsum(counts) - counts
        cols = np.arange(tot, dtype=np.int64) - np.repeat(starts, counts) + rows + 1
        same = block[rows] == block[cols]
        coef = np.where(same, c_in[block[rows]], c_out)
        p = np.minimum(1.0, coef * theta[rows] * theta[cols])
        keep = g.random(tot) < p
        src.append(rows[keep])
        dst.append(cols[keep])
        i0 = i1
    row_ptr, col_idx = csr_from_pairs(n, np.concatenate(src), np.concatenate(dst))
    return Graph(n, row_ptr, col_idx, name=name, block=block.astype(np.int32),
                 meta={"k": k, "gamma": gamma, "theta_min": theta_min, "theta_max": theta_max,
                       "mu": mu})


# --- small structured graphs (closed-form cases) -------------------------------------------

def complete(n: int) -> Graph:
    i, j = np.triu_indices(n, 1)
    rp, ci = csr_from_pairs(n, i, j)
    return Graph(n, rp, ci, name=f"K{n}")


def path(n: int) -> Graph:
    i = np.arange(n - 1)
    rp, ci = csr_from_pairs(n, i, i + 1)
    return Graph(n, rp, ci, name=f"P{n}")


def star(n: int, center: int = 0) -> Graph:
    """Star on n nodes: `center` joined to every other node."""
    others = np.array([v for v in range(n) if v != center], dtype=np.int64)
    rp, ci = csr_from_pairs(n, np.full(len(others), center), others)
    return Graph(n, rp, ci, name=f"S{n}")


def two_cliques_bridge(m: int) -> Graph:
    """Two K_m (nodes 0..m-1 and m..2m-1) joined by the single bridge edge (m-1, m)."""
    a_i, a_j = np.triu_indices(m, 1)
    i = np.concatenate([a_i, a_i + m, [m - 1]])
    j = np.concatenate([a_j, a_j + m, [m]])
    rp, ci = csr_from_pairs(2 * m, i, j)
    return Graph(2 * m, rp, ci, name=f"2K{m}-bridge")


def erdos_renyi(n: int, p: float, g: np.random.Generator) -> Graph:
    i, j = np.triu_indices(n, 1)
    keep = g.random(len(i)) < p
    rp, ci = csr_from_pairs(n, i[keep], j[keep])
    return Graph(n, rp, ci, name=f"G({n},{p})")


def directed_cycle(n: int) -> Graph:
    """Arcs v -> v + 1 (mod n)."""
    i = np.arange(n)
    rp, ci = csr_from_arcs(n, i, (i + 1) % n)
    return Graph(n, rp, ci, name=f"C{n}->", directed=True)


def directed_path(n: int) -> Graph:
    """Arcs v -> v + 1 for v < n - 1."""
    i = np.arange(n - 1)
    rp, ci = csr_from_arcs(n, i, i + 1)
    return Graph(n, rp, ci, name=f"P{n}->", directed=True)


def directed_erdos_renyi(n: int, p: float, g: np.random.Generator) -> Graph:
    """Every ordered pair (i, j), i != j, is an arc with probability p."""
    t = _bernoulli_positions(g, n * (n - 1), p)
    i = t // (n - 1)
    j = t - i * (n - 1)
    j = j + (j >= i)                      # skip the diagonal
    rp, ci = csr_from_arcs(n, i, j)
    return Graph(n, rp, ci, name=f"D({n},{p})", directed=True)


def directed_planted_partition(n: int, k: int, p_in: float, p_out: float, g: np.random.Generator,
                               name: str = "") -> Graph:
    """Directed planted partition: each ordered pair is an arc with probability p_in
    inside a block and p_out across (two independent undirected draws give the
    arcs i -> j and j -> i of every pair i < j)."""
    a = planted_partition(n, k, p_in, p_out, g)
    b = planted_partition(n, k, p_in, p_out, g)
    arcs_i, arcs_j = [], []
    for graph, forward in ((a, True), (b, False)):
        rows = np.repeat(np.arange(n, dtype=np.int64), graph.degrees())
        cols = graph.col_idx.astype(np.int64)
        lower = rows < cols
        if forward:
            arcs_i.append(rows[lower]); arcs_j.append(cols[lower])
        else:
            arcs_i.append(cols[lower]); arcs_j.append(rows[lower])
    rp, ci = csr_from_arcs(n, np.concatenate(arcs_i), np.concatenate(arcs_j))
    return Graph(n, rp, ci, name=name or f"dpp-{n}", block=a.block, directed=True,
                 meta={"k": k, "p_in": p_in, "p_out": p_out})


def edge_weights(graph: Graph, lo: float, hi: float, g: np.random.Generator) -> np.ndarray:
    """Positive weights per CSR entry, drawn uniformly from [lo, hi); an undirected
    graph gets one draw per edge, stored in both of its rows."""
    if graph.directed:
        return g.uniform(lo, hi, size=graph.nnz)
    rows = np.repeat(np.arange(graph.n, dtype=np.int64), graph.degrees())
    cols = graph.col_idx.astype(np.int64)
    key = rows * graph.n + cols               # ascending: rows sorted, columns sorted in a row
    lower = rows < cols
    w = np.empty(graph.nnz)
    w[lower] = g.uniform(lo, hi, size=int(lower.sum()))
    mirror = np.searchsorted(key, cols * graph.n + rows)
    w[~lower] = w[mirror[~lower]]
    return w


def relabel(graph: Graph, perm: np.ndarray) -> Graph:
    """The same graph with node v renamed perm[v]."""
    perm = np.asarray(perm, dtype=np.int64)
    rows = np.repeat(np.arange(graph.n, dtype=np.int64), graph.degrees())
    rp, ci = csr_from_pairs(graph.n, perm[rows], perm[graph.col_idx.astype(np.int64)])
    return Graph(graph.n, rp, ci, name=graph.name + "-relabelled")


# --- the benchmark and test workloads -------------------------------------------------------

def planted128() -> tuple[Graph, list[float]]:
    """Planted partition N=128, 4 blocks of 32, p_in=0.3, p_out=0.02, seed 0; sigma = 1.0."""
    return planted_partition(128, 4, 0.3, 0.02, rng(0, 1), name="pp-128"), [1.0]


def sigma_sweep16() -> list[float]:
    """16 sigma values log-spaced from 0.5 to 4.0: sigma_k = 0.5 * 8^(k/15)."""
    return [0.5 * 8.0 ** (k / 15.0) for k in range(16)]


def dcsbm16384() -> tuple[Graph, list[float]]:
    """DC-SBM N=16384, 32 equal communities, power-law expected degrees (exponent 2.5,
    mean 16, max 512), mixing 0.1, seed 1; the 16-value sigma sweep."""
    return (dcsbm(16384, 32, 2.5, 16.0, 512.0, 0.1, rng(1, 2), name="dcsbm-16384"),
            sigma_sweep16())


def sbm262144(n: int = 262144, k: int = 256) -> tuple[Graph, list[float]]:
    """Plain SBM N=262144, 256 equal communities, mean degree 20, mixing 0.15, seed 2; sigma 1.5."""
    nc = n // k
    p_in = 20.0 * 0.85 / (nc - 1)
    p_out = 20.0 * 0.15 / (n - nc)
    return planted_partition(n, k, p_in, p_out, rng(2, 3), name=f"sbm-{n}"), [1.5]


def planted_batch_graph(gi: int, seed: int = 3, n_min: int = 32, n_max: int = 2048) -> tuple[Graph, float]:
    """Graph gi of the planted-partition batch and its sigma, from stream (seed, 4, gi)."""
    g = rng(seed, 4, gi)
    n = int(math.floor(math.exp(g.uniform(math.log(n_min), math.log(n_max)))))
    k = int(g.integers(2, 17))
    k = min(k, n)
    p_in = float(g.uniform(0.1, 0.5))
    sigma = float(g.uniform(0.5, 3.0))
    return planted_partition(n, k, p_in, 0.02, g, name=f"batch-{gi}"), sigma


def planted_batch(count: int = 4096, seed: int = 3, n_min: int = 32, n_max: int = 2048,
                  ) -> tuple[list[Graph], list[float]]:
    """Batch of planted-partition graphs: N = floor(exp(U(ln n_min, ln n_max))), k ~ U{2..16},
    p_in ~ U(0.1, 0.5), p_out = 0.02, sigma ~ U(0.5, 3.0); graph g draws from stream (seed, 4, g)."""
    graphs, sigmas = [], []
    for gi in range(count):
        graph, sigma = planted_batch_graph(gi, seed, n_min, n_max)
        graphs.append(graph)
        sigmas.append(sigma)
    return graphs, sigmas


@dataclass
class Request:
    index: int
    arrival_s: float
    n: int
    k: int
    sigma: float
    seed: int

    def graph(self) -> Graph:
        g = rng(self.seed, 5, self.index)
        g.random(4)   # skip the variates that drew the request's parameters
        return sbm_mean_degree(self.n, self.k, 12.0, 0.1, g, name=f"req-{self.index}")


def sbm_request_stream(count: int = 4000, rate: float = 200.0, seed: int = 4, n_min: int = 64,
                     n_max: int = 65536) -> list[Request]:
    """Poisson request stream: exponential inter-arrival times at `rate` per second;
    N log-uniform in [n_min, n_max], k ~ U{4..min(64, N/4)}, mean degree 12, mixing 0.1,
    sigma ~ U(0.5, 3.0)."""
    arrivals = np.cumsum(rng(seed, 6).exponential(1.0 / rate, size=count))
    out = []
    for r in range(count):
        g = rng(seed, 5, r)
        u = g.random(4)
        n = int(math.floor(math.exp(math.log(n_min) + u[0] * (math.log(n_max) - math.log(n_min)))))
        kmax = max(4, min(64, n // 4))
        k = 4 + int(u[1] * (kmax - 3))
        sigma = 0.5 + 2.5 * float(u[2])
        out.append(Request(r, float(arrivals[r]), n, k, sigma, seed))
    return out

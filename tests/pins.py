"""Checks that pin the oracle to facts outside itself.

Each ``check_*`` takes an ``oracle.Oracle`` (the real one, or a deliberately
broken copy in the mutation tests) and raises AssertionError when the oracle
disagrees with:
  * Floyd-Warshall all-pairs distances (an independent algorithm);
  * scipy's breadth-first shortest paths (a library routine);
  * closed forms derived by hand from the structure of K_n, P_n, S_n and two
    cliques joined by a bridge (distances known without a BFS), evaluated in
    50-digit arithmetic;
  * identities every distance histogram satisfies;
  * invariants of the descent (Algorithm 2) and of the roots (Algorithm 3),
    and brute-force descent on small graphs;
  * invariance of the partition under node relabelling on tie-free graphs.
"""
from __future__ import annotations

import math

import mpmath
import numpy as np
import scipy.sparse as sp
from scipy.sparse.csgraph import connected_components, shortest_path

import graphgen as gg

mpmath.mp.dps = 50


# ---- helpers written independently of the oracle ------------------------------------

def floyd_warshall(graph) -> np.ndarray:
    n = graph.n
    D = np.full((n, n), np.inf)
    np.fill_diagonal(D, 0.0)
    rows = np.repeat(np.arange(n), graph.degrees())
    D[rows, graph.col_idx] = 1.0
    for k in range(n):
        D = np.minimum(D, D[:, k:k + 1] + D[k:k + 1, :])
    return D


def adjacency(graph):
    n = graph.n
    rows = np.repeat(np.arange(n), graph.degrees())
    return sp.csr_matrix((np.ones(graph.nnz), (rows, graph.col_idx)), shape=(n, n))


def exact_potential_from_distances(dists, sigma) -> float:
    """(1 / 2 sigma^2) * sum d^2 exp(-d^2/2sigma^2) / sum exp(-d^2/2sigma^2), finite d only,
    in 50-digit arithmetic."""
    s = mpmath.mpf(sigma)
    num = mpmath.mpf(0)
    den = mpmath.mpf(0)
    for d in dists:
        if not math.isfinite(d):
            continue
        d2 = mpmath.mpf(int(d)) ** 2
        e = mpmath.exp(-d2 / (2 * s * s))
        num += d2 * e
        den += e
    return num / den / (2 * s * s)


def close(a: float, b, rel: float = 1e-13) -> bool:
    b = float(b)
    if b == 0.0:
        return a == 0.0
    return abs(a - b) <= rel * abs(b)


def random_graphs(count: int, n_lo: int, n_hi: int, seed: int, p_lo=0.02, p_hi=0.3):
    out = []
    for t in range(count):
        g = gg.rng(seed, 99, t)
        n = int(g.integers(n_lo, n_hi + 1))
        p = float(g.uniform(p_lo, p_hi))
        out.append(gg.erdos_renyi(n, p, g))
    return out


def descend_brute(graph, V) -> np.ndarray:
    """Labels by following, from every node, the strictly-lower minimum-V neighbour
    (smallest index among equal minima) until none is lower."""
    n = graph.n
    out = np.empty(n, dtype=np.int64)
    for v in range(n):
        x = v
        for _ in range(n + 1):
            nb = sorted(int(u) for u in graph.neighbors(x))
            lower = [u for u in nb if V[u] < V[x]]
            if not lower:
                break
            m = min(V[u] for u in lower)
            x = min(u for u in lower if V[u] == m)
        out[v] = x
    return out


def partition(labels) -> set:
    groups = {}
    for v, l in enumerate(labels):
        groups.setdefault(int(l), set()).add(v)
    return {frozenset(s) for s in groups.values()}


# ---- pins ---------------------------------------------------------------------------

def check_distances(orc):
    """BFS hop distances equal Floyd-Warshall's on small random graphs, connected or not."""
    for graph in random_graphs(12, 2, 40, seed=11, p_lo=0.01, p_hi=0.25) + [gg.path(9), gg.star(6)]:
        D = floyd_warshall(graph)
        for s in range(graph.n):
            d = orc.bfs(graph, s).astype(np.float64)
            d[d < 0] = np.inf
            assert np.array_equal(d, D[s]), (graph.name, s)


def check_histograms_library(orc):
    """Histograms equal bincounts of scipy's unweighted shortest paths."""
    for graph in random_graphs(4, 100, 300, seed=12, p_lo=0.002, p_hi=0.05):
        D = shortest_path(adjacency(graph), method="D", directed=False, unweighted=True)
        h = orc.histograms(graph, threads=2)
        Dmax = int(np.max(D[np.isfinite(D)]))
        assert h.shape == (graph.n, Dmax + 1), graph.name
        for i in range(graph.n):
            row = D[i][np.isfinite(D[i])].astype(np.int64)
            assert np.array_equal(h[i], np.bincount(row, minlength=Dmax + 1)), (graph.name, i)


def check_histogram_identities(orc):
    """h_i(0) = 1, h_i(1) = deg(i), sum_d h_i(d) = |component(i)|,
    sum_i h_i(d) even for d >= 1, sum_i sum_d d h_i(d) = 2 x Wiener index."""
    graphs = random_graphs(6, 20, 60, seed=13, p_lo=0.02, p_hi=0.2) + [gg.planted128()[0]]
    for graph in graphs:
        h = orc.histograms(graph)
        assert np.all(h[:, 0] == 1)
        assert np.array_equal(h[:, 1] if h.shape[1] > 1 else np.zeros(graph.n), graph.degrees())
        _, comp = connected_components(adjacency(graph), directed=False)
        sizes = np.bincount(comp)
        assert np.array_equal(h.sum(axis=1), sizes[comp])
        assert np.all(h[:, 1:].sum(axis=0) % 2 == 0)
        D = floyd_warshall(graph)
        wiener2 = D[np.isfinite(D)].sum()
        assert (h * np.arange(h.shape[1])).sum() == wiener2


def check_complete_graph(orc):
    """K_n: every node has h = {1, n-1}, so V = (n-1) w1 / (1 + (n-1) w1) / (2 sigma^2)
    for all nodes; equal potentials never descend, so every node is its own cluster."""
    for n, sigma in [(2, 1.0), (5, 0.7), (17, 1.3), (33, 2.9)]:
        graph = gg.complete(n)
        s = mpmath.mpf(sigma)
        w1 = mpmath.exp(-1 / (2 * s * s))
        exact = (n - 1) * w1 / (1 + (n - 1) * w1) / (2 * s * s)
        V = orc.potential(orc.histograms(graph), sigma)
        assert all(close(v, exact) for v in V), (n, sigma)
        assert len(set(V.tolist())) == 1
        parent, _ = orc.ggd_parent(graph, V)
        labels, k = orc.find_centers(parent)
        assert k == n and np.array_equal(labels, np.arange(n))


def check_path_graph(orc):
    """P_n: dist(k, j) = |k - j|, so V_k follows from the definition with those
    distances; endpoints sit highest."""
    for n, sigma in [(2, 0.9), (7, 1.0), (12, 0.6), (25, 2.2)]:
        graph = gg.path(n)
        V = orc.potential(orc.histograms(graph), sigma)
        for k in range(n):
            exact = exact_potential_from_distances([abs(k - j) for j in range(n)], sigma)
            assert close(V[k], exact), (n, sigma, k)


def check_star_graph(orc):
    """S_n with center c: V_c = (n-1) w1 / (1 + (n-1) w1) / (2 sigma^2) and every leaf
    V_l = (w1 + 4 (n-2) w2) / (1 + w1 + (n-2) w2) / (2 sigma^2).  If V_c < V_l all
    leaves join the center (one cluster); if V_c > V_l every leaf is a root and the
    center joins the lowest-index leaf (n - 1 clusters)."""
    seen = set()
    for n, center, sigma in [(7, 3, 0.5), (7, 3, 3.0), (5, 0, 0.6), (9, 8, 2.5), (4, 2, 0.4)]:
        graph = gg.star(n, center)
        s = mpmath.mpf(sigma)
        w1 = mpmath.exp(-1 / (2 * s * s))
        w2 = mpmath.exp(-4 / (2 * s * s))
        Vc = (n - 1) * w1 / (1 + (n - 1) * w1) / (2 * s * s)
        Vl = (w1 + 4 * (n - 2) * w2) / (1 + w1 + (n - 2) * w2) / (2 * s * s)
        V = orc.potential(orc.histograms(graph), sigma)
        leaves = [v for v in range(n) if v != center]
        assert close(V[center], Vc), (n, sigma)
        assert all(close(V[v], Vl) for v in leaves), (n, sigma)
        parent, _ = orc.ggd_parent(graph, V)
        labels, k = orc.find_centers(parent)
        if Vc < Vl:
            seen.add("center-wins")
            assert k == 1 and np.all(labels == center)
        else:
            seen.add("leaves-win")
            assert k == n - 1
            assert labels[center] == min(leaves)
            assert all(labels[v] == v for v in leaves)
    assert seen == {"center-wins", "leaves-win"}


def check_bridge(orc):
    """Two K_m joined by the bridge (a, b) = (m-1, m): h_a = h_b = {1, m, m-1}, every
    other node x has h_x = {1, m-1, 1, m-1}.  When V_a < V_x the two cliques form two
    clusters rooted at a and b (V_a = V_b exactly, so neither end descends into the
    other clique); when V_x < V_a every non-bridge node is a root and each bridge end
    joins the lowest-index node of its own clique."""
    seen = set()
    for m, sigma in [(5, 2.0), (5, 1.0), (8, 3.0), (8, 0.8), (3, 1.7)]:
        graph = gg.two_cliques_bridge(m)
        a, b = m - 1, m
        s = mpmath.mpf(sigma)
        w = [mpmath.exp(-mpmath.mpf(d * d) / (2 * s * s)) for d in range(4)]
        Va = (m * w[1] + 4 * (m - 1) * w[2]) / (1 + m * w[1] + (m - 1) * w[2]) / (2 * s * s)
        Vx = ((m - 1) * w[1] + 4 * w[2] + 9 * (m - 1) * w[3]) / \
             (1 + (m - 1) * w[1] + w[2] + (m - 1) * w[3]) / (2 * s * s)
        V = orc.potential(orc.histograms(graph), sigma)
        assert close(V[a], Va) and close(V[b], Va), (m, sigma)
        assert V[a] == V[b]
        others = [v for v in range(2 * m) if v not in (a, b)]
        assert all(close(V[x], Vx) for x in others), (m, sigma)
        parent, _ = orc.ggd_parent(graph, V)
        labels, k = orc.find_centers(parent)
        if Va < Vx:
            seen.add("bridge-wins")
            assert k == 2
            assert np.all(labels[:m] == a) and np.all(labels[m:] == b)
        else:
            seen.add("interior-wins")
            assert k == 2 * (m - 1)
            assert labels[a] == 0 and labels[b] == m + 1
            assert all(labels[x] == x for x in others)
    assert seen == {"bridge-wins", "interior-wins"}


def check_isolated_and_tiny(orc):
    """One node: h = {1}, V = 0, one cluster.  Isolated nodes (no edges): V = 0 and each
    is its own cluster; unreachable pairs add nothing."""
    one = gg.Graph(1, np.array([0, 0], dtype=np.int32), np.zeros(0, dtype=np.int32), name="K1")
    h = orc.histograms(one)
    assert h.tolist() == [[1]]
    V = orc.potential(h, 1.0)
    assert V.tolist() == [0.0]
    labels, k = orc.find_centers(orc.ggd_parent(one, V)[0])
    assert k == 1 and labels.tolist() == [0]
    # a triangle plus two isolated nodes
    rp, ci = gg.csr_from_pairs(5, np.array([0, 1, 0]), np.array([1, 2, 2]))
    g = gg.Graph(5, rp, ci, name="K3+2")
    h = orc.histograms(g)
    assert h.tolist() == [[1, 2], [1, 2], [1, 2], [1, 0], [1, 0]]
    V = orc.potential(h, 1.3)
    assert V[3] == 0.0 and V[4] == 0.0
    labels, k = orc.find_centers(orc.ggd_parent(g, V)[0])
    assert k == 5


def check_exact_arithmetic(orc):
    """V agrees with the same histogram summed in 50-digit arithmetic to 1e-14."""
    for graph in random_graphs(3, 30, 80, seed=14, p_lo=0.03, p_hi=0.1):
        h = orc.histograms(graph)
        for sigma in (0.55, 1.0, 2.7):
            V = orc.potential(h, sigma)
            for i in range(0, graph.n, 7):
                dists = np.repeat(np.arange(h.shape[1]), h[i])
                assert close(V[i], exact_potential_from_distances(dists, sigma), 1e-14)


def check_literal_form(orc):
    """Algorithm 1 term by term (one exp per pair) agrees with the grouped form to 1e-12."""
    for graph in random_graphs(3, 30, 90, seed=15, p_lo=0.02, p_hi=0.15):
        h = orc.histograms(graph)
        for sigma in (0.5, 1.5, 4.0):
            V = orc.potential(h, sigma)
            for i in range(graph.n):
                assert close(V[i], orc.potential_literal(graph, i, sigma), 1e-12), (graph.name, i)


def check_descent(orc):
    """parent[v] is v or a strictly lower neighbour holding the minimum; roots have no
    strictly lower neighbour; labels are roots; labels equal brute-force descent."""
    graphs = random_graphs(10, 5, 16, seed=16, p_lo=0.1, p_hi=0.5) + \
        random_graphs(4, 40, 120, seed=17, p_lo=0.02, p_hi=0.1)
    for graph in graphs:
        for sigma in (0.6, 1.4):
            V = orc.potential(orc.histograms(graph), sigma)
            parent, _ = orc.ggd_parent(graph, V)
            labels, k = orc.find_centers(parent)
            for v in range(graph.n):
                nb = graph.neighbors(v)
                p = parent[v]
                if p != v:
                    assert p in nb and V[p] < V[v]
                    assert V[p] == V[nb].min()
                    assert p == min(u for u in nb if V[u] == V[p])
                else:
                    assert len(nb) == 0 or V[nb].min() >= V[v]
            assert np.all(parent[labels] == labels)
            assert k == int(np.sum(parent == np.arange(graph.n)))
            if graph.n <= 16:
                assert np.array_equal(labels, descend_brute(graph, V))


def check_relabel_invariance(orc):
    """On graphs with no index-dependent ties, relabelling the nodes relabels the
    clusters and nothing else."""
    tested = 0
    for t, graph in enumerate(random_graphs(8, 30, 70, seed=18, p_lo=0.04, p_hi=0.12)):
        perm = gg.rng(19, t).permutation(graph.n)
        other = gg.relabel(graph, perm)
        for sigma in (0.7, 1.9):
            V = orc.potential(orc.histograms(graph), sigma)
            parent, ties = orc.ggd_parent(graph, V)
            if ties:
                continue
            labels, _ = orc.find_centers(parent)
            V2 = orc.potential(orc.histograms(other), sigma)
            parent2, ties2 = orc.ggd_parent(other, V2)
            labels2, _ = orc.find_centers(parent2)
            assert ties2 == 0
            assert np.array_equal(V2[perm], V)
            back = labels2[perm]
            assert partition(back) == partition(labels)
            tested += 1
    assert tested >= 6


ALL_CHECKS = [
    check_distances, check_histograms_library, check_histogram_identities,
    check_complete_graph, check_path_graph, check_star_graph, check_bridge,
    check_isolated_and_tiny, check_exact_arithmetic, check_literal_form, check_descent,
    check_relabel_invariance,
]


def check_adjacency_mode(orc):
    """Paper-literal distance (1 on an edge, M otherwise): on graphs of diameter
    <= 2 with M = 2 it coincides with the hop distance, bit for bit; on a path it
    matches the definition evaluated from the adjacency matrix in 50 digits."""
    for graph in [gg.complete(9), gg.star(12, 4), gg.two_cliques_bridge(1)]:
        for sigma in (0.6, 1.0, 2.5):
            hop = orc.potential(orc.histograms(graph), sigma)
            adj = orc.potential_adjacency(graph, sigma, 2.0)
            assert np.array_equal(hop, adj), (graph.name, sigma)
    graph = gg.path(6)
    A = np.zeros((6, 6))
    A[np.arange(5), np.arange(1, 6)] = 1
    A = A + A.T
    for M, sigma in [(3.0, 1.0), (2.5, 0.7), (10.0, 2.0)]:
        V = orc.potential_adjacency(graph, sigma, M)
        for i in range(6):
            dists = [0.0 if j == i else (1.0 if A[i, j] else M) for j in range(6)]
            s = mpmath.mpf(sigma)
            num = sum(mpmath.mpf(d) ** 2 * mpmath.exp(-mpmath.mpf(d) ** 2 / (2 * s * s)) for d in dists)
            den = sum(mpmath.exp(-mpmath.mpf(d) ** 2 / (2 * s * s)) for d in dists)
            assert close(V[i], num / den / (2 * s * s)), (M, sigma, i)


ALL_CHECKS.append(check_adjacency_mode)


def check_directed(orc):
    """Directed graphs (row v = arcs v -> u).  BFS distances equal Floyd-Warshall's
    and scipy's directed shortest paths; node i's histogram counts the nodes i
    reaches.  On the directed cycle C_n every node sees each distance 0..n-1 once,
    so all potentials equal one 50-digit sum.  On the directed path node i reaches
    n-1-i nodes at distances 1..n-1-i, V falls along the arcs, and every node
    descends to the last node.  Descent on random digraphs equals brute force over
    out-neighbours."""
    for t in range(8):
        g = gg.rng(97, t)
        n = int(g.integers(2, 40))
        graph = gg.directed_erdos_renyi(n, float(g.uniform(0.03, 0.3)), g)
        fw = floyd_warshall(graph)
        sd = shortest_path(adjacency(graph), method="D", directed=True, unweighted=True)
        assert np.array_equal(fw, sd), graph.name
        h = orc.histograms(graph)
        for s in range(n):
            d = orc.bfs(graph, s).astype(np.float64)
            d[d < 0] = np.inf
            assert np.array_equal(d, fw[s]), (graph.name, s)
            row = fw[s][np.isfinite(fw[s])].astype(np.int64)
            assert np.array_equal(h[s], np.bincount(row, minlength=h.shape[1])), (graph.name, s)
        for sigma in (0.7, 1.6):
            V = orc.potential(h, sigma)
            labels, _ = orc.find_centers(orc.ggd_parent(graph, V)[0])
            assert np.array_equal(labels, descend_brute(graph, V)), (graph.name, sigma)
    for n in (2, 5, 9):
        cyc = gg.directed_cycle(n)
        h = orc.histograms(cyc)
        assert np.array_equal(h, np.ones((n, n), dtype=np.int32))
        for sigma in (0.5, 1.3):
            V = orc.potential(h, sigma)
            assert all(close(x, exact_potential_from_distances(range(n), sigma)) for x in V)
            labels, k = orc.find_centers(orc.ggd_parent(cyc, V)[0])
            assert k == n and np.array_equal(labels, np.arange(n))     # equal V: nobody moves
    n = 7
    pth = gg.directed_path(n)
    h = orc.histograms(pth)
    for i in range(n):
        assert np.array_equal(h[i], np.r_[np.ones(n - i, np.int32), np.zeros(i, np.int32)])
    for sigma in (0.6, 1.5, 2.0):
        V = orc.potential(h, sigma)
        for i in range(n):
            assert close(V[i], exact_potential_from_distances(range(n - i), sigma)) or (i == n - 1 and V[i] == 0)
        if sigma >= 1.5:    # (at sigma = 0.6 the far terms are below one ulp of the sums)
            assert np.all(np.diff(V) < 0)
            labels, k = orc.find_centers(orc.ggd_parent(pth, V)[0])
            assert k == 1 and np.all(labels == n - 1)


ALL_CHECKS.append(check_directed)


def weighted_floyd_warshall(graph, w) -> np.ndarray:
    n = graph.n
    D = np.full((n, n), np.inf)
    np.fill_diagonal(D, 0.0)
    rows = np.repeat(np.arange(n), graph.degrees())
    D[rows, graph.col_idx] = np.minimum(D[rows, graph.col_idx], w)
    for k in range(n):
        D = np.minimum(D, D[:, k:k + 1] + D[k:k + 1, :])
    return D


def check_weighted(orc):
    """Weighted graphs (distance = length of the lightest path).  Dijkstra equals
    scipy's weighted shortest paths bit for bit and Floyd-Warshall within rounding
    (its additions group differently); unit weights give the hop-mode potential;
    constant weights c give the hop-mode potential at sigma / c; on a weighted path
    V matches the 50-digit sum over the path's prefix lengths; directed weighted
    graphs follow the arcs."""
    for t in range(6):
        g = gg.rng(98, t)
        n = int(g.integers(2, 40))
        graph = (gg.erdos_renyi(n, float(g.uniform(0.05, 0.3)), g) if t % 2 == 0
                 else gg.directed_erdos_renyi(n, float(g.uniform(0.05, 0.3)), g))
        w = gg.edge_weights(graph, 0.25, 3.0, g)
        A = sp.csr_matrix((w, graph.col_idx, graph.row_ptr), shape=(n, n))
        ref = shortest_path(A, method="D", directed=True)
        fw = weighted_floyd_warshall(graph, w)
        for s in range(n):
            d = orc.dijkstra(graph, w, s)
            assert np.array_equal(d, ref[s]), (graph.name, s)
            fin = np.isfinite(fw[s])
            assert np.array_equal(np.isfinite(d), fin)
            assert np.allclose(d[fin], fw[s][fin], rtol=1e-12, atol=0), (graph.name, s)
    disconnected = gg.erdos_renyi(60, 0.03, gg.rng(96))
    assert connected_components(adjacency(disconnected), directed=False)[0] > 1
    for graph in [gg.planted_partition(120, 4, 0.15, 0.02, gg.rng(99)), gg.path(9), gg.star(11), disconnected]:
        h = orc.histograms(graph)
        ones = np.ones(graph.nnz)
        for sigma in (0.6, 1.5):
            Vw = orc.potential_weighted(graph, ones, [sigma])[0]
            assert np.allclose(Vw, orc.potential(h, sigma), rtol=1e-13, atol=0), graph.name
            for c in (0.5, 2.0, 3.0):
                Vc = orc.potential_weighted(graph, np.full(graph.nnz, c), [sigma])[0]
                assert np.allclose(Vc, orc.potential(h, sigma / c), rtol=1e-13, atol=0), (graph.name, c)
    graph = gg.path(7)
    step = np.array([0.5, 1.25, 2.0, 0.75, 1.5, 1.0])         # weight of edge (i, i + 1)
    rows = np.repeat(np.arange(7), graph.degrees())
    w = step[np.minimum(rows, graph.col_idx)]
    pos = np.concatenate([[0.0], np.cumsum(step)])
    for sigma in (0.8, 2.5):
        V = orc.potential_weighted(graph, w, [sigma])[0]
        for i in range(7):
            d = orc.dijkstra(graph, w, i)
            assert np.allclose(d, np.abs(pos - pos[i]), rtol=1e-15, atol=1e-15)
            s = mpmath.mpf(sigma)
            num = sum(mpmath.mpf(x) ** 2 * mpmath.exp(-mpmath.mpf(x) ** 2 / (2 * s * s)) for x in d)
            den = sum(mpmath.exp(-mpmath.mpf(x) ** 2 / (2 * s * s)) for x in d)
            assert close(V[i], num / den / (2 * s * s)), (sigma, i)


ALL_CHECKS.append(check_weighted)

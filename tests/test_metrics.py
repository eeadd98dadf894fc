"""Quality measures (CPU): hand-computed cases and library cross-checks."""
import math

import numpy as np
import pytest

import graphgen as gg
from paper_2305_14641_gb300 import metrics as M


def test_hand_cases():
    # two triangles joined by one edge, split along the bridge: m = 7, 2m = 14
    rp, ci = gg.csr_from_pairs(6, np.array([0, 0, 1, 3, 3, 4, 2]), np.array([1, 2, 2, 4, 5, 5, 3]))
    labels = [0, 0, 0, 1, 1, 1]
    # inside edges 6 (12 directed), cluster degree sums 7 and 7
    assert M.modularity(rp, ci, labels) == pytest.approx(12 / 14 - (49 + 49) / 196)
    assert M.modularity(rp, ci, [0] * 6) == pytest.approx(0.0)
    truth, pred = [0, 0, 1, 1], [0, 0, 1, 1]
    assert M.adjusted_rand_index(truth, pred) == 1.0
    assert M.fowlkes_mallows(truth, pred) == 1.0
    assert M.normalized_mutual_info(truth, pred) == pytest.approx(1.0)
    # one pair in common: TP = 1, TP+FP = 1, TP+FN = 2
    assert M.fowlkes_mallows([0, 0, 0, 1], [0, 0, 1, 2]) == pytest.approx(1 / math.sqrt(3 * 1))
    assert M.normalized_mutual_info([0, 0, 1, 1], [0, 1, 0, 1]) == pytest.approx(0.0, abs=1e-12)


def test_against_libraries():
    sk = pytest.importorskip("sklearn.metrics")
    g = gg.rng(50)
    for _ in range(5):
        a = g.integers(0, 5, size=300)
        b = np.where(g.random(300) < 0.7, a, g.integers(0, 7, size=300))
        assert M.adjusted_rand_index(a, b) == pytest.approx(sk.adjusted_rand_score(a, b))
        assert M.fowlkes_mallows(a, b) == pytest.approx(sk.fowlkes_mallows_score(a, b))
        assert M.normalized_mutual_info(a, b) == pytest.approx(
            sk.normalized_mutual_info_score(a, b, average_method="geometric"))


def test_modularity_against_networkx():
    nx = pytest.importorskip("networkx")
    graph = gg.planted_partition(400, 4, 0.1, 0.01, gg.rng(51))
    G = nx.Graph()
    G.add_nodes_from(range(graph.n))
    rows = np.repeat(np.arange(graph.n), graph.degrees())
    G.add_edges_from((int(u), int(v)) for u, v in zip(rows, graph.col_idx) if u < v)
    for gamma in (1.0, 0.5, 2.0):
        comms = [set(np.nonzero(graph.block == b)[0].tolist()) for b in range(4)]
        assert M.modularity(graph.row_ptr, graph.col_idx, graph.block, gamma) == pytest.approx(
            nx.community.modularity(G, comms, resolution=gamma))

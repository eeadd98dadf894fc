"""The quality measures on the device (qc_quality) against the host ones in
paper_2305_14641_gb300/metrics.py (themselves checked on the CPU against
scikit-learn, networkx and hand values): modularity, ARI and FMI from exact
integer sums within 1e-12 relative, NMI within 1e-10."""
import numpy as np
import pytest

import graphgen as gg

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def qc():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2305_14641_gb300 as qc
    return qc


def close(a, b, tol):
    return abs(a - b) <= tol * max(abs(b), 1e-300) or a == b


def check(qc, ctx, graph, G, labels, truth):
    from paper_2305_14641_gb300 import metrics
    got = qc.quality(ctx, torch.as_tensor(labels, device="cuda"), graph=G, truth=torch.as_tensor(truth, device="cuda"))
    assert got["clusters"] == len(np.unique(labels))
    assert close(got["modularity"], metrics.modularity(graph.row_ptr, graph.col_idx, labels), 1e-12)
    assert close(got["ari"], metrics.adjusted_rand_index(truth, labels), 1e-12)
    assert close(got["fmi"], metrics.fowlkes_mallows(truth, labels), 1e-12)
    assert close(got["nmi"], metrics.normalized_mutual_info(truth, labels), 1e-10)


def test_quality_of_solves(qc):
    with qc.Context(0) as ctx:
        for graph in [gg.planted_partition(2000, 8, 0.02, 0.001, gg.rng(81)),
                      gg.sbm_mean_degree(3327, 6, 2.8, 0.2, gg.rng(82)),
                      gg.dcsbm(3000, 8, 2.5, 10.0, 200.0, 0.1, gg.rng(83))]:
            G = qc.Graph.from_graph(ctx, graph)
            _, labels, _ = G.solve([0.7, 1.5, 3.0])
            for lab in labels.cpu().numpy():
                check(qc, ctx, graph, G, lab, graph.block)
            G.close()


def test_quality_edge_cases(qc):
    graph = gg.planted_partition(500, 5, 0.05, 0.004, gg.rng(84))
    with qc.Context(0) as ctx:
        G = qc.Graph.from_graph(ctx, graph)
        n = graph.n
        check(qc, ctx, graph, G, np.zeros(n, np.int32), graph.block)             # one cluster
        check(qc, ctx, graph, G, np.arange(n, dtype=np.int32), graph.block)      # singletons
        check(qc, ctx, graph, G, graph.block.astype(np.int32) * 7, graph.block)  # the truth itself
        check(qc, ctx, graph, G, gg.rng(85).integers(0, n, n).astype(np.int32), np.zeros(n, np.int32))
        bad = np.zeros(n, np.int32)
        bad[3] = n
        with pytest.raises(qc.QCError) as e:
            qc.quality(ctx, torch.as_tensor(bad, device="cuda"), graph=G)
        assert e.value.status_name == "QC_ERR_INVALID_ARG"
        G.close()

"""The captured solve plan of one graph and a sigma sweep (qc_sweep_*) against
the oracle (needs a GPU): potentials bit-identical (and within 1e-12 relative),
labels and cluster counts exact, on every replay, from the CSR and from the
plan's own histogram."""
import numpy as np
import pytest

import graphgen as gg
import oracle

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def qc():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2305_14641_gb300 as qc
    return qc


@pytest.fixture(scope="module")
def ctx(qc):
    c = qc.Context(0)
    yield c
    c.close()


def check_plan(qc, ctx, graph, sigmas, runs=3, expect_captured=True):
    ref = oracle.solve(graph, sigmas, threads=oracle.default_threads())
    G = qc.Graph.from_graph(ctx, graph)
    plan = qc.SweepPlan(G, sigmas)
    for k in range(runs):
        plan.labels.fill_(-1)
        plan.V.fill_(np.nan)
        counts = plan.run(reuse_histogram=(k == runs - 1 and runs > 1), counts=True)
        V = plan.V.cpu().numpy()
        rel = np.abs(V - ref.V) / np.maximum(np.abs(ref.V), np.finfo(np.float64).tiny)
        assert np.all(rel <= 1e-12), (graph.name, k, float(rel.max()))
        assert np.array_equal(V, ref.V), (graph.name, k, "potential not bit-identical")
        assert np.array_equal(plan.labels.cpu().numpy(), ref.labels), (graph.name, k)
        assert counts == ref.n_clusters, (graph.name, k)
    info = plan.info()
    assert info["D"] == ref.D, (graph.name, info)
    if expect_captured and graph.nnz > 0:
        assert info["captured"], graph.name
    plan.close()
    G.close()
    return info


def test_dcsbm16384_sweep_replayed(qc, ctx):
    """The benchmark's graph and 16-value sweep: three replays from the CSR (the
    last one from the plan's histogram), every value against the oracle."""
    graph, sigmas = gg.dcsbm16384()
    info = check_plan(qc, ctx, graph, sigmas, runs=4)
    assert info["kernels_per_run"] >= 5


def test_sizes_and_structures(qc, ctx):
    for graph in [gg.planted128()[0], gg.erdos_renyi(1000, 0.004, gg.rng(61)), gg.complete(40), gg.star(300, 2),
                  gg.two_cliques_bridge(12), gg.planted_partition(5000, 10, 0.004, 0.0002, gg.rng(62))]:
        check_plan(qc, ctx, graph, [0.6, 1.3, 2.9])


def test_deeper_than_the_rows(qc, ctx):
    """A path of 300 nodes (D = 299) needs more than the plan's first 32 rows: the
    run is captured again with more rows and gives the oracle's results."""
    check_plan(qc, ctx, gg.path(300), [1.0, 4.0], runs=2)


def test_many_chunks_and_directed(qc, ctx, monkeypatch):
    monkeypatch.setenv("QCGRAPH_CHUNK_WORDS", "3")
    check_plan(qc, ctx, gg.planted_partition(700, 5, 0.05, 0.004, gg.rng(63)), [0.9, 2.2])
    # chunks of 96 words on a sparse graph: the two-hop set-up with chunk cursors
    # inside the captured plan; the plan gives all its memory back before its
    # stream goes, so the next call on the context runs clean
    monkeypatch.setenv("QCGRAPH_CHUNK_WORDS", "96")
    graph = gg.planted_partition(9000, 30, 0.012, 0.0002, gg.rng(65))
    check_plan(qc, ctx, graph, [0.7, 1.6])
    ref = oracle.solve(graph, [1.1])
    lab, counts = qc.cluster(ctx, graph.row_ptr, graph.col_idx, [1.1])
    assert np.array_equal(lab, ref.labels) and counts == ref.n_clusters
    monkeypatch.delenv("QCGRAPH_CHUNK_WORDS")
    check_plan(qc, ctx, gg.directed_planted_partition(1500, 6, 0.02, 0.001, gg.rng(64)), [0.8, 2.5])


def test_no_edges_and_errors(qc, ctx):
    empty = gg.Graph(60, np.zeros(61, np.int32), np.zeros(0, np.int32), name="empty")
    check_plan(qc, ctx, empty, [1.0], runs=2, expect_captured=False)
    G = qc.Graph.from_graph(ctx, gg.path(20))
    plan = qc.SweepPlan(G, [1.0])
    with pytest.raises(qc.QCError) as e:
        plan.run(reuse_histogram=True)            # no full run yet
    assert e.value.status_name == "QC_ERR_INVALID_ARG"
    plan.close()
    with pytest.raises(qc.QCError) as e:
        qc.SweepPlan(G, [1.0, -2.0])
    assert e.value.status_name == "QC_ERR_INVALID_ARG"
    G.close()


def test_plan_and_graph_agree(qc, ctx):
    """The plan's histogram is its own: the graph's cached one, filled by the
    single-graph path, gives the same labels, and neither disturbs the other."""
    graph = gg.planted_partition(3000, 8, 0.01, 0.001, gg.rng(65))
    G = qc.Graph.from_graph(ctx, graph)
    plan = qc.SweepPlan(G, [0.7, 1.9])
    plan.run()
    _, lab, counts = G.solve([0.7, 1.9])
    assert torch.equal(lab, plan.labels)
    plan.run(reuse_histogram=True)
    assert torch.equal(lab, plan.labels)
    plan.close()
    G.close()

def test_graph_outlives_its_plan(qc, ctx):
    """A plan prepares the graph on a stream of its own; the graph's preparation is
    given back on that stream when the graph is closed after the plan, so the
    stream stays with the context (a plan of the same context reuses it)."""
    graph = gg.planted_partition(20000, 20, 0.004, 0.0001, gg.rng(68))
    ref = oracle.solve(graph, [1.4])
    for _ in range(3):
        G = qc.Graph.from_graph(ctx, graph)
        plan = qc.SweepPlan(G, [1.4])
        plan.run(counts=False)
        assert np.array_equal(plan.labels.cpu().numpy(), ref.labels)
        plan.close()
        _, labels, counts = G.solve([1.4])
        assert np.array_equal(labels.cpu().numpy(), ref.labels) and counts == ref.n_clusters
        G.close()
        torch.cuda.synchronize()


def test_context_closes_what_is_left_open(qc):
    """The library requires a context to outlive its graphs and plans; the binding
    closes any left open when the context closes (plans first), so dropping them
    afterwards is harmless."""
    graph = gg.planted_partition(700, 5, 0.04, 0.003, gg.rng(69))
    ref = oracle.solve(graph, [1.2])
    c = qc.Context(0, allocator="cuda")
    G = qc.Graph.from_graph(c, graph)
    plan = qc.SweepPlan(G, [1.2])
    plan.run(counts=False)
    assert np.array_equal(plan.labels.cpu().numpy(), ref.labels)
    bp = qc.BatchPlan(c, [G], [1.2])
    bp.run(counts=False)
    assert np.array_equal(bp.labels.cpu().numpy(), ref.labels[0])
    c.close()
    assert G.handle is None and plan.handle is None and bp.handle is None
    del plan, bp, G
    torch.cuda.synchronize()
    with qc.Context(0, allocator="cuda") as c2:       # the device is still usable
        lab, _ = qc.cluster(c2, graph.row_ptr, graph.col_idx, [1.2])
        assert np.array_equal(lab, ref.labels)

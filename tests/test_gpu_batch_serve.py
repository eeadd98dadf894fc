"""Batched and served forms against the oracle (needs a GPU).

Every graph of a batch, and every served request, must give exactly the
oracle's labels and cluster count; a served request must give the same labels
alone and in a mix.
"""
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


def edge_cases():
    one = gg.Graph(1, np.array([0, 0], np.int32), np.zeros(0, np.int32), name="one")
    empty = gg.Graph(50, np.zeros(51, np.int32), np.zeros(0, np.int32), name="empty")
    return [one, empty, gg.path(2), gg.complete(65), gg.star(130, 64), gg.two_cliques_bridge(40),
            gg.erdos_renyi(700, 0.003, gg.rng(41))]


def check_batch(qc, ctx, graphs, sigmas, runs=2):
    Gs = [qc.Graph.from_graph(ctx, g) for g in graphs]
    plan = qc.BatchPlan(ctx, Gs, sigmas)
    for _ in range(runs):
        plan.labels.fill_(-1)
        counts = plan.run()
        for k, (g, s) in enumerate(zip(graphs, sigmas)):
            ref = oracle.solve(g, [s])
            got = plan.labels_of(k).cpu().numpy()
            assert np.array_equal(got, ref.labels[0]), (g.name, s)
            assert counts[k] == ref.n_clusters[0], g.name
    plan.close()
    for G in Gs:
        G.close()


def test_batch_planted(qc, ctx):
    graphs, sigmas = gg.planted_batch(160)
    check_batch(qc, ctx, graphs, sigmas)


@pytest.mark.parametrize("threads,words,degree", [(256, 1, 24), (512, 4, 48), (512, 2, 12)])
def test_batch_fixed_config(qc, ctx, monkeypatch, threads, words, degree):
    # every kernel configuration the autotuner may pick gives the oracle's labels
    monkeypatch.setenv("QCGRAPH_BATCH_CONFIG", f"{threads},{words},{degree}")
    graphs, sigmas = gg.planted_batch(48)
    Gs = [qc.Graph.from_graph(ctx, g) for g in graphs]
    plan = qc.BatchPlan(ctx, Gs, sigmas)
    assert plan.config() == {"threads": threads, "chunk_words": words, "sparse_degree": degree}
    counts = plan.run()
    for k, (g, s) in enumerate(zip(graphs, sigmas)):
        ref = oracle.solve(g, [s])
        assert np.array_equal(plan.labels_of(k).cpu().numpy(), ref.labels[0]), (g.name, threads, words)
        assert counts[k] == ref.n_clusters[0]
    plan.close()
    for G in Gs:
        G.close()


def test_batch_edge_cases_and_deep_graph(qc, ctx):
    """Single nodes, no edges, cliques, a path too deep for the batched kernel's
    histogram (finished by the single-graph path) and a graph above the CTA limit."""
    graphs = edge_cases() + [gg.path(300), gg.planted_partition(9000, 12, 0.01, 0.0004, gg.rng(42))]
    sigmas = [0.5 + 0.25 * k for k in range(len(graphs))]
    check_batch(qc, ctx, graphs, sigmas, runs=1)


def test_solve_batch_one_shot(qc, ctx):
    graphs, sigmas = gg.planted_batch(20, seed=9)
    Gs = [qc.Graph.from_graph(ctx, g) for g in graphs]
    labels, offsets = qc.solve_batch(ctx, Gs, sigmas)
    lab = labels.cpu().numpy()
    for k, g in enumerate(graphs):
        ref = oracle.solve(g, [sigmas[k]])
        assert np.array_equal(lab[offsets[k]:offsets[k] + g.n], ref.labels[0])


def serve_requests(count, seed=4):
    reqs = gg.sbm_request_stream(count, seed=seed, n_max=12000)
    return [(r.graph(), r.sigma) for r in reqs]


def test_server_mixed_equals_alone_and_oracle(qc):
    reqs = serve_requests(40)
    with qc.Server(0, streams=3) as srv:
        ids = [srv.submit(g.row_ptr, g.col_idx, s) for g, s in reqs]
        mixed = [srv.wait(i, timeout_ms=120000) for i in ids]
        alone = []
        for g, s in reqs[:12]:
            alone.append(srv.wait(srv.submit(g.row_ptr, g.col_idx, s), timeout_ms=120000))
        st = srv.stats()
    for (g, s), res in zip(reqs, mixed):
        ref = oracle.solve(g, [s])
        assert np.array_equal(res["labels"], ref.labels[0]), g.name
        assert res["n_clusters"] == ref.n_clusters[0]
        assert res["latency_ms"] >= res["start_ms"] >= res["admit_ms"] >= 0
    for a, m in zip(alone, mixed):
        assert np.array_equal(a["labels"], m["labels"])
    assert st["completed"] == 52 and st["failed"] == 0
    assert st["large_solved"] >= 1            # requests above the CTA limit took the worker


def test_server_budget_and_cancel(qc):
    g = gg.planted_partition(12000, 6, 0.002, 0.0001, gg.rng(43))
    with qc.Server(0, mem_budget_bytes=1 << 20) as srv:
        with pytest.raises(qc.QCError) as e:
            srv.submit(g.row_ptr, g.col_idx, 1.0)           # alone exceeds the budget
        assert e.value.status_name == "QC_ERR_BUDGET"
        small = [gg.erdos_renyi(200, 0.03, gg.rng(44, k)) for k in range(30)]
        ids = [srv.submit(x.row_ptr, x.col_idx, 1.2) for x in small]
        srv.cancel(ids[-1])
        results = []
        for i in ids[:-1]:
            results.append(srv.wait(i, timeout_ms=60000))
        with pytest.raises(qc.QCError) as e:
            srv.wait(ids[-1], timeout_ms=60000)
        assert e.value.status_name == "QC_ERR_CANCELLED"
        st = srv.stats()
        assert st["peak_bytes_resident"] <= 1 << 20
    for x, res in zip(small, results):
        assert np.array_equal(res["labels"], oracle.solve(x, [1.2]).labels[0])


def test_server_rejects_invalid(qc):
    big = gg.planted_partition(3000, 4, 0.005, 0.0005, gg.rng(45))
    ci = big.col_idx.copy()
    ci[10] = ci[11]                       # a duplicate edge in a large request: found on the GPU
    with qc.Server(0) as srv:
        rid = srv.submit(big.row_ptr, ci, 1.0)
        with pytest.raises(qc.QCError) as e:
            srv.wait(rid, timeout_ms=60000)
        assert e.value.status_name == "QC_ERR_INVALID_GRAPH"
        with pytest.raises(qc.QCError) as e:
            srv.submit(np.array([0, 1, 1], np.int32), np.array([1], np.int32), 1.0)
        assert e.value.status_name == "QC_ERR_INVALID_GRAPH"
        with pytest.raises(qc.QCError) as e:
            srv.submit(np.array([0, 1, 2], np.int32), np.array([1, 0], np.int32), -1.0)
        assert e.value.status_name == "QC_ERR_INVALID_ARG"


def test_batch_directed(qc, ctx):
    """Directed graphs in a batch: weak components, out-neighbour descent."""
    g = gg.rng(44)
    graphs = [gg.directed_erdos_renyi(int(n), 4.0 / n, g) for n in (40, 200, 700, 1500)] + \
        [gg.directed_cycle(100), gg.directed_path(90), gg.directed_planted_partition(1200, 5, 0.03, 0.002, g)]
    check_batch(qc, ctx, graphs, [0.8, 1.2, 1.7, 2.2, 1.0, 1.5, 0.9])


def full_size_golden(name):
    """The oracle's stored results for a full-size workload (tests/golden/full_size.json,
    written by tests/golden/make_full_size.py from oracle/ alone)."""
    import json
    import os
    path = os.path.join(os.path.dirname(__file__), "golden", "full_size.json")
    data = json.load(open(path))
    assert name in data, f"{name} missing from {path}: run tests/golden/make_full_size.py"
    return data[name]


def set_sha256(graphs, sigmas):
    import hashlib
    h = hashlib.sha256()
    for g, s in zip(graphs, sigmas):
        h.update(g.row_ptr.astype("<i4").tobytes())
        h.update(g.col_idx.astype("<i4").tobytes())
        h.update(np.array([s], dtype="<f8").tobytes())
    return h.hexdigest()


def labels_digest(labels):
    import hashlib
    return hashlib.sha256(np.ascontiguousarray(labels, dtype="<i4").tobytes()).hexdigest()[:16]


def explain(graph, sigma, got):
    """Where a result differs from the oracle's (computed now, for the message only)."""
    ref = oracle.solve(graph, [sigma], threads=oracle.default_threads())
    diff = np.nonzero(ref.labels[0] != got)[0]
    return f"{graph.name} (n={graph.n}): {len(diff)} labels differ, first at nodes {diff[:8].tolist()}"


def test_batch4096_full_size(qc, ctx):
    """The whole 4096-graph batch of the benchmark, in the configuration the
    autotuner picks for it: every graph's labels and cluster count equal the
    oracle's (stored digests)."""
    graphs, sigmas = gg.planted_batch(4096)
    gold = full_size_golden("batch4096")
    assert set_sha256(graphs, sigmas) == gold["set_sha256"], "input graphs differ"
    Gs = [qc.Graph.from_graph(ctx, g, validate=False) for g in graphs]
    plan = qc.BatchPlan(ctx, Gs, sigmas)
    for run in range(2):
        plan.labels.fill_(-1)
        counts = plan.run()
        lab = plan.labels.cpu().numpy()
        bad = [k for k in range(len(graphs))
               if labels_digest(lab[plan.offsets[k]:plan.offsets[k] + graphs[k].n]) != gold["labels_digest"][k]
               or counts[k] != gold["n_clusters"][k]]
        assert not bad, (run, len(bad), explain(graphs[bad[0]], sigmas[bad[0]],
                                                lab[plan.offsets[bad[0]]:plan.offsets[bad[0]] + graphs[bad[0]].n]))
    plan.close()
    for G in Gs:
        G.close()


def test_server_request_stream_full(qc, ctx):
    """The first 400 requests of the serving stream (N up to 65,536), all submitted
    at once: every request's labels and cluster count equal the oracle's (stored
    digests), the largest ones included."""
    reqs = gg.sbm_request_stream(400)
    graphs = [r.graph() for r in reqs]
    gold = full_size_golden("serve400")
    assert set_sha256(graphs, [r.sigma for r in reqs]) == gold["set_sha256"], "input requests differ"
    with qc.Server(0) as srv:
        ids = [srv.submit(g.row_ptr, g.col_idx, r.sigma) for g, r in zip(graphs, reqs)]
        res = [srv.wait(i, timeout_ms=300000) for i in ids]
        st = srv.stats()
    assert st["completed"] == 400 and st["failed"] == 0
    assert st["large_solved"] >= 1
    bad = [k for k in range(400)
           if labels_digest(res[k]["labels"]) != gold["labels_digest"][k] or res[k]["n_clusters"] != gold["n_clusters"][k]]
    assert not bad, (len(bad), explain(graphs[bad[0]], reqs[bad[0]].sigma, res[bad[0]]["labels"]))


def test_server_resident_graphs(qc):
    """Requests on graphs already resident on the GPU (qc_server_submit_graph):
    several sigmas per graph, one small enough for the batched kernel and one for
    the single-graph path (whose later requests reuse its cached histogram), all
    equal to the oracle's labels."""
    small = gg.planted_partition(600, 5, 0.05, 0.004, gg.rng(47))
    large = gg.planted_partition(6000, 12, 0.01, 0.0005, gg.rng(48))
    with qc.Server(0) as srv:
        Gs = qc.Graph.from_graph(srv.ctx, small)
        Gl = qc.Graph.from_graph(srv.ctx, large)
        jobs = [(small, Gs, s) for s in (0.7, 1.5)] + [(large, Gl, s) for s in (0.8, 1.6, 2.4)]
        ids = [srv.submit_graph(G, s) for _, G, s in jobs]
        res = [srv.wait(i, timeout_ms=120000) for i in ids]
        st = srv.stats()
        Gs.close()
        Gl.close()
    assert st["completed"] == len(jobs) and st["failed"] == 0
    for (graph, _, s), r in zip(jobs, res):
        ref = oracle.solve(graph, [s])
        assert np.array_equal(r["labels"], ref.labels[0]), (graph.name, s)
        assert r["n_clusters"] == ref.n_clusters[0]

"""CUDA path against the oracle, element by element (needs a GPU).

Histograms and labels must be bit-exact.  Potentials must agree within 1e-12
relative (the stated tolerance); the design makes them bit-identical, and that
is asserted too.
"""
import os

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


def assert_solution_matches(qc, ctx, graph, sigmas, threads=None):
    threads = threads or oracle.default_threads()
    ref = oracle.solve(graph, sigmas, threads=threads)
    g = qc.Graph.from_graph(ctx, graph)
    hist = g.histogram().cpu().numpy()
    assert hist.shape == (ref.D + 1, graph.n), (graph.name, hist.shape, ref.hist.shape)
    assert np.array_equal(hist.T, ref.hist), graph.name
    V = g.potential(sigmas)
    labels, counts = g.ggd_labels(V)
    Vh = V.cpu().numpy()
    rel = np.abs(Vh - ref.V) / np.maximum(np.abs(ref.V), np.finfo(np.float64).tiny)
    assert np.all(rel <= 1e-12), (graph.name, float(rel.max()))
    assert np.array_equal(Vh, ref.V), (graph.name, "potential not bit-identical")
    assert np.array_equal(labels.cpu().numpy(), ref.labels), graph.name
    assert counts == ref.n_clusters, graph.name
    g.close()
    return ref


def test_planted128(qc, ctx):
    graph, sigmas = gg.planted128()
    assert_solution_matches(qc, ctx, graph, sigmas + [0.5, 0.8, 2.0, 4.0])


@pytest.mark.parametrize("n", [1, 2, 3, 31, 63, 64, 65, 127, 128, 129, 255, 500, 1000, 2047, 3001])
def test_random_sizes(qc, ctx, n):
    """Ragged tails of the 64-source words and of the 16-byte row segments,
    disconnected graphs and isolated nodes."""
    g = gg.rng(21, n)
    for p in (2.0 / max(n, 2), 8.0 / max(n, 2), 0.3):
        graph = gg.erdos_renyi(n, min(p, 1.0), g) if n <= 3001 else None
        assert_solution_matches(qc, ctx, graph, [0.6, 1.7])


def test_structured(qc, ctx):
    for graph in [gg.complete(40), gg.path(300), gg.star(70, 5), gg.two_cliques_bridge(9),
                  gg.path(2), gg.complete(1)]:
        assert_solution_matches(qc, ctx, graph, [0.5, 1.0, 3.0])


def test_hubs_and_long_rows(qc, ctx):
    """A star with 20,000 leaves (one row of 20k neighbours: a block-shared item of
    625 chunks), two such hubs joined through a path, and a dense core with a
    sparse fringe: rows far past every per-warp and per-block split."""
    star = gg.star(20001, 0)
    rng = gg.rng(47)
    n = 30000
    # hub 0 - leaves 2..14001, path 2-3-...-10, edge 10-14002 into hub 1's leaves 14002..28001,
    # and 1998 isolated nodes
    i = np.concatenate([np.full(14000, 0), np.full(14000, 1), np.arange(2, 10), [10]])
    j = np.concatenate([np.arange(2, 14002), np.arange(14002, 28002), np.arange(3, 11), [14002]])
    rp, ci = gg.csr_from_pairs(n, i, j)
    hubs = gg.Graph(n, rp, ci, name="two-hubs")
    core = gg.erdos_renyi(600, 0.5, rng)
    fringe_i = rng.integers(0, 600, size=5000)
    fringe_j = np.arange(600, 5600)
    rp2, ci2 = gg.csr_from_pairs(5600, np.concatenate([np.repeat(np.arange(600), np.diff(core.row_ptr)), fringe_i]),
                                 np.concatenate([core.col_idx, fringe_j]))
    dense = gg.Graph(5600, rp2, ci2, name="core-fringe")
    for graph in (star, hubs, dense):
        assert_solution_matches(qc, ctx, graph, [0.6, 1.5])


def test_no_edges(qc, ctx):
    graph = gg.Graph(100, np.zeros(101, dtype=np.int32), np.zeros(0, dtype=np.int32), name="empty")
    ref = assert_solution_matches(qc, ctx, graph, [1.0])
    assert ref.n_clusters == [100]


@pytest.mark.parametrize("chunk", [1, 2, 3, 5])
def test_forced_source_chunks(qc, ctx, chunk, monkeypatch):
    """Sources processed a few words at a time: the histogram accumulates across chunks."""
    monkeypatch.setenv("QCGRAPH_CHUNK_WORDS", str(chunk))
    graph = gg.planted_partition(700, 5, 0.05, 0.004, gg.rng(22, chunk))
    assert_solution_matches(qc, ctx, graph, [0.9, 2.2])


@pytest.mark.parametrize("ratio,chunk", [("1", "96"), ("1", "40"), ("128", "96"), ("0", "96")])
def test_change_masks(qc, ctx, ratio, chunk, monkeypatch):
    """The variant with change masks (rows of more than 16 segments on sparse
    graphs): ratio 1 takes it and reads masked segments at every level, 128 is
    the default rule (masked levels only while the frontier is sparse), 0 never
    takes it.  Chunks of 96 words give rows of two tiles and a ragged second
    chunk (45 words, one tile); 40 words give one-tile rows of 20 segments."""
    monkeypatch.setenv("QCGRAPH_MASK_RATIO", ratio)
    monkeypatch.setenv("QCGRAPH_CHUNK_WORDS", chunk)
    graph = gg.planted_partition(9000, 30, 0.012, 0.0002, gg.rng(25, int(chunk)))
    assert_solution_matches(qc, ctx, graph, [0.7, 1.6])
    # a path: one new bit per level over 4199 levels (the histogram grows and the
    # kernel is relaunched from the level where it stopped)
    assert_solution_matches(qc, ctx, gg.path(4200), [3.0])
    # directed: rows are out-arcs, weak components
    assert_solution_matches(qc, ctx, gg.directed_erdos_renyi(6000, 3.0 / 6000, gg.rng(26, int(chunk))), [1.2])


@pytest.mark.parametrize("mode", ["0", "2"])
def test_two_hop_setup(qc, ctx, mode, monkeypatch):
    """Levels 1 and 2 written straight from the CSR (mode 2: on every graph it
    fits) and the level-1 set-up followed by a pull level (mode 0), each against
    the oracle: ragged sizes, isolated nodes and several components, a complete
    graph (every row full at level 1), hubs taken block-wide (a star of 20,000
    leaves), chunked sources, change masks, and directed arcs."""
    monkeypatch.setenv("QCGRAPH_TWO_HOP", mode)
    rng = gg.rng(61)
    graphs = [gg.erdos_renyi(n, p, rng) for n, p in ((65, 0.05), (1000, 0.004), (3001, 0.003), (2047, 0.3))]
    graphs += [gg.complete(40), gg.path(300), gg.star(70, 5), gg.two_cliques_bridge(9), gg.path(2)]
    graphs += [gg.dcsbm(3000, 8, 2.5, 10.0, 200.0, 0.1, gg.rng(24)),
               gg.directed_erdos_renyi(2000, 3.0 / 2000, gg.rng(62)), gg.star(20001, 0)]
    for graph in graphs:
        assert_solution_matches(qc, ctx, graph, [0.6, 1.5])
    monkeypatch.setenv("QCGRAPH_CHUNK_WORDS", "5")
    assert_solution_matches(qc, ctx, gg.planted_partition(700, 5, 0.05, 0.004, gg.rng(63)), [0.9])
    monkeypatch.setenv("QCGRAPH_CHUNK_WORDS", "96")
    monkeypatch.setenv("QCGRAPH_MASK_RATIO", "1")
    assert_solution_matches(qc, ctx, gg.planted_partition(9000, 30, 0.012, 0.0002, gg.rng(64)), [0.7])


def test_planted_and_dcsbm_mid(qc, ctx):
    g1 = gg.planted_partition(4000, 16, 0.02, 0.0005, gg.rng(23))
    g2 = gg.dcsbm(3000, 8, 2.5, 10.0, 200.0, 0.1, gg.rng(24))
    for graph in (g1, g2):
        assert_solution_matches(qc, ctx, graph, gg.sigma_sweep16()[::3])


def test_dcsbm16384_full(qc, ctx):
    """DC-SBM N=16384 with the 16-value sigma sweep, every node checked."""
    graph, sigmas = gg.dcsbm16384()
    assert_solution_matches(qc, ctx, graph, sigmas)


def full_size_golden(name):
    """The oracle's stored results for a full-size workload (tests/golden/full_size.json,
    written by tests/golden/make_full_size.py from oracle/ alone)."""
    import json
    path = os.path.join(os.path.dirname(__file__), "golden", "full_size.json")
    data = json.load(open(path))
    assert name in data, f"{name} missing from {path}: run tests/golden/make_full_size.py"
    return data[name]


def sha256(a):
    import hashlib
    return hashlib.sha256(np.ascontiguousarray(a).tobytes()).hexdigest()


def test_sbm262144_full_size(qc, ctx):
    """SBM N=262144 (5.24M directed edges), sigma 1.5, at full size: the whole
    histogram (every node, every distance), every potential and every label equal
    the oracle's, stored as SHA-256 digests of the oracle's arrays.  Should they
    differ, sampled rows are compared with the oracle directly to say where."""
    graph, sigmas = gg.sbm262144()
    gold = full_size_golden("sbm262144")
    csr = np.concatenate([graph.row_ptr.astype("<i4"), graph.col_idx.astype("<i4")])
    assert sha256(csr) == gold["csr_sha256"], "input graph differs from the one the oracle ran on"
    g = qc.Graph.from_graph(ctx, graph)
    hist = g.histogram().cpu().numpy()
    V = g.potential(sigmas)
    labels, counts = g.ggd_labels(V)
    Vh, lab = V.cpu().numpy(), labels.cpu().numpy()
    g.close()
    ok = (hist.shape[0] - 1 == gold["D"] and sha256(hist.astype("<i4")) == gold["hist_sha256"])
    if not ok:
        rs = gg.rng(30)
        nodes = np.unique(np.concatenate([rs.choice(graph.n, 60, replace=False), [0, graph.n - 1]])).astype(np.int32)
        ref_h = oracle.histograms(graph, nodes, threads=oracle.default_threads(), cap=hist.shape[0] + 1)
        bad = [int(v) for k, v in enumerate(nodes) if not np.array_equal(hist[:ref_h.shape[1], v], ref_h[k])]
        raise AssertionError(f"histogram differs from the oracle's (D {hist.shape[0] - 1} vs {gold['D']}); "
                             f"sampled nodes that differ: {bad[:10]}")
    assert sha256(Vh[0].astype("<f8")) == gold["V_sha256"], "potential not bit-identical to the oracle's"
    assert sha256(lab[0].astype("<i4")) == gold["labels_sha256"], "labels differ from the oracle's"
    assert counts[0] == gold["n_clusters"]


def test_sigma_reuse_and_edge_values(qc, ctx):
    """The cached histogram serves later sigma values; extreme sigmas stay exact."""
    graph = gg.planted_partition(600, 6, 0.06, 0.003, gg.rng(25))
    g = qc.Graph.from_graph(ctx, graph)
    ref = oracle.solve(graph, [0.05, 1.0, 1e3])
    for k, s in enumerate([0.05, 1.0, 1e3]):
        V = g.potential([s])
        assert np.array_equal(V.cpu().numpy()[0], ref.V[k])
        labels, counts = g.ggd_labels(V)
        assert np.array_equal(labels.cpu().numpy()[0], ref.labels[k])
    g.close()


def test_invalid_inputs(qc, ctx):
    graph = gg.path(5)
    g = qc.Graph.from_graph(ctx, graph)
    for bad in (0.0, -1.0, float("nan"), float("inf")):
        with pytest.raises(qc.QCError) as e:
            g.potential([1.0, bad])
        assert e.value.status_name == "QC_ERR_INVALID_ARG"
    g.close()
    rp, ci = graph.row_ptr.copy(), graph.col_idx.copy()
    cases = {}
    a = ci.copy(); a[0] = 7; cases["out of range"] = (rp, a)
    a = ci.copy(); a[1] = 1; cases["self-loop"] = (rp, a)
    cases["asymmetric"] = (np.array([0, 1, 1], dtype=np.int32), np.array([1], dtype=np.int32))
    cases["unsorted"] = (np.array([0, 2, 3, 4], dtype=np.int32), np.array([2, 1, 0, 0], dtype=np.int32))
    cases["duplicate"] = (np.array([0, 2, 4], dtype=np.int32), np.array([1, 1, 0, 0], dtype=np.int32))
    for name, (r, c) in cases.items():
        with pytest.raises(qc.QCError) as e:
            qc.Graph(ctx, r, c)
        assert e.value.status_name == "QC_ERR_INVALID_GRAPH", name
        # the one-call form queues its check ahead of the solve, which then runs on
        # emptied rows; the verdict comes with the results
        with pytest.raises(qc.QCError) as e:
            qc.cluster(ctx, r, c, [1.0, 2.0])
        assert e.value.status_name == "QC_ERR_INVALID_GRAPH", name
    # row_ptr itself: decreasing, not starting at 0, ending past or before nnz,
    # negative and huge entries; the device check reads every row bound before it
    # indexes through it, so none of these reads outside the arrays
    bad_rps = []
    for pos, val in ((2, int(rp[3]) + 1), (0, 1), (-1, len(ci) + 5), (-1, len(ci) - 1), (1, -3),
                     (2, 2**31 - 1), (3, -2**31)):
        b = rp.copy()
        b[pos] = val
        bad_rps.append(b)
    for bad_rp in bad_rps:
        with pytest.raises(qc.QCError) as e:
            qc.Graph(ctx, bad_rp, ci)
        assert e.value.status_name == "QC_ERR_INVALID_GRAPH", bad_rp
        assert "row_ptr" in str(e.value), str(e.value)
        dev_bad = torch.tensor(bad_rp, device="cuda"), torch.tensor(ci, device="cuda")
        with pytest.raises(qc.QCError) as e:
            qc.Graph(ctx, *dev_bad)
        assert e.value.status_name == "QC_ERR_INVALID_GRAPH", bad_rp
        for args in ((bad_rp, ci), dev_bad):
            with pytest.raises(qc.QCError) as e:
                qc.cluster(ctx, *args, [1.0])
            assert e.value.status_name == "QC_ERR_INVALID_GRAPH", bad_rp
            assert "row_ptr" in str(e.value), str(e.value)
    # the context is still usable
    assert_solution_matches(qc, ctx, graph, [1.0])


def test_cluster_one_call(qc, ctx):
    """qc_cluster: a CSR (host or device) to labels (numpy, pinned host tensor,
    CUDA tensor) in one call, against the oracle; graphs with several
    components, directed arcs, no edges, and a path whose histogram outgrows the
    first launch's rows (the BFS is rerun and the rest queued again); invalid
    input is still reported by the call."""
    sig = [0.7, 1.9]
    graphs = [gg.planted_partition(3000, 12, 0.02, 0.001, gg.rng(71)),
              gg.dcsbm(3000, 8, 2.5, 10.0, 200.0, 0.1, gg.rng(72)),
              gg.directed_erdos_renyi(2000, 3.0 / 2000, gg.rng(73)), gg.path(300),
              gg.Graph(50, np.zeros(51, dtype=np.int32), np.zeros(0, dtype=np.int32), name="empty")]
    for graph in graphs:
        ref = oracle.solve(graph, sig)
        directed = getattr(graph, "directed", False)
        lab, counts = qc.cluster(ctx, graph.row_ptr, graph.col_idx, sig, directed=directed)
        assert np.array_equal(lab, ref.labels), graph.name
        assert counts == ref.n_clusters, graph.name
        pinned = torch.empty((2, graph.n), dtype=torch.int32).pin_memory()
        qc.cluster(ctx, graph.row_ptr, graph.col_idx, sig, labels_out=pinned, counts=False, directed=directed)
        assert np.array_equal(pinned.numpy(), ref.labels), graph.name
        dev = torch.empty((2, graph.n), dtype=torch.int32, device="cuda")
        _, c2 = qc.cluster(ctx, torch.tensor(graph.row_ptr, device="cuda"), torch.tensor(graph.col_idx, device="cuda"),
                           sig, labels_out=dev, directed=directed)
        assert np.array_equal(dev.cpu().numpy(), ref.labels), graph.name
        assert c2 == ref.n_clusters, graph.name
    with pytest.raises(qc.QCError) as e:
        qc.cluster(ctx, np.array([0, 1, 1], dtype=np.int32), np.array([1], dtype=np.int32), sig)
    assert e.value.status_name == "QC_ERR_INVALID_GRAPH"
    with pytest.raises(qc.QCError) as e:
        qc.cluster(ctx, graphs[0].row_ptr, graphs[0].col_idx, [1.0, float("nan")])
    assert e.value.status_name == "QC_ERR_INVALID_ARG"


def test_device_input_and_allocators(qc):
    graph = gg.planted_partition(900, 3, 0.03, 0.003, gg.rng(26))
    ref = oracle.solve(graph, [1.2])
    for alloc in ("torch", "cuda"):
        with qc.Context(0, allocator=alloc) as c:
            rp = torch.tensor(graph.row_ptr, device="cuda")
            ci = torch.tensor(graph.col_idx, device="cuda")
            g = qc.Graph(c, rp, ci)
            _, labels, counts = g.solve([1.2])
            assert np.array_equal(labels.cpu().numpy(), ref.labels)
            g.close()
            torch.cuda.synchronize()
            assert c.bytes_in_use() == 0


def test_budget(qc):
    graph = gg.planted_partition(2000, 4, 0.02, 0.001, gg.rng(27))
    with qc.Context(0, mem_budget_bytes=200_000) as c:
        g = qc.Graph.from_graph(c, graph)        # CSR alone fits
        with pytest.raises(qc.QCError) as e:
            g.potential([1.0])                  # the bitsets do not
        assert e.value.status_name == "QC_ERR_BUDGET"
        g.close()
        torch.cuda.synchronize()
        assert c.bytes_in_use() == 0


def test_bounded_wait_gives_up(qc, ctx):
    """A grid barrier with a block that never arrives ends in QC_ERR_TIMEOUT once
    its time limit has passed on the GPU's global timer, not before it and not
    long after it; the context then still clusters exactly."""
    import time
    for limit_us in (2000, 200000):
        t0 = time.perf_counter()
        st, waited_ns = ctx.selftest_barrier_timeout(limit_us)
        host_s = time.perf_counter() - t0
        assert st == "QC_ERR_TIMEOUT"
        # the wait ends after the limit, within one poll (100 ns sleeps) plus scheduling noise
        assert 1000 * limit_us <= waited_ns <= 1000 * limit_us * 1.05 + 200000, (limit_us, waited_ns)
        assert host_s < limit_us * 1e-6 + 5.0
    assert ctx.selftest_barrier_timeout(0)[0] == "QC_ERR_INVALID_ARG"
    assert ctx.selftest_barrier_timeout(10 ** 7 + 1)[0] == "QC_ERR_INVALID_ARG"
    graph, sigmas = gg.planted128()
    assert_solution_matches(qc, ctx, graph, sigmas)


def test_descent_on_given_potentials(qc, ctx):
    """GGD and roots alone, on seeded potentials with negatives, many exact ties,
    and -0.0 next to +0.0 (equal under IEEE comparison)."""
    g = gg.rng(28)
    for graph in [gg.planted_partition(3000, 8, 0.01, 0.001, g), gg.erdos_renyi(500, 0.05, g),
                  gg.star(40, 7), gg.complete(30)]:
        G = qc.Graph.from_graph(ctx, graph)
        S = 5
        V = np.round(g.normal(size=(S, graph.n)), 1)          # heavy ties
        V[1] = np.abs(V[1])
        V[2] = np.where(g.random(graph.n) < 0.5, -0.0, 0.0)    # only signed zeros
        V[3] = g.integers(0, 3, size=graph.n).astype(np.float64)
        Vd = torch.tensor(V, device="cuda")
        labels, counts = G.ggd_labels(Vd)
        labels = labels.cpu().numpy()
        for s in range(S):
            p, _ = oracle.ggd_parent(graph, V[s])
            lab, k = oracle.find_centers(p)
            assert np.array_equal(labels[s], lab), (graph.name, s)
            assert counts[s] == k
        G.close()


def test_many_sigmas_in_groups(qc, ctx):
    """More sigma values than one descent launch handles (groups of 16)."""
    graph = gg.planted_partition(1200, 6, 0.03, 0.002, gg.rng(29))
    sigmas = [0.4 + 0.1 * k for k in range(37)]
    assert_solution_matches(qc, ctx, graph, sigmas)


@pytest.mark.parametrize("M", [2.0, 3.5, 100.0])
def test_adjacency_mode(qc, ctx, M):
    """Paper-literal distance: potentials and labels equal the oracle's bit for bit."""
    sigmas = [0.5, 1.0, 2.0]
    for graph in [gg.planted128()[0], gg.erdos_renyi(700, 0.01, gg.rng(30)), gg.star(50, 3)]:
        G = qc.Graph.from_graph(ctx, graph)
        V = G.potential_adjacency(sigmas, M)
        labels, counts = G.ggd_labels(V)
        Vh = V.cpu().numpy()
        for k, s in enumerate(sigmas):
            ref = oracle.potential_adjacency(graph, s, M)
            assert np.array_equal(Vh[k], ref), (graph.name, s)
            p, _ = oracle.ggd_parent(graph, ref)
            lab, nc = oracle.find_centers(p)
            assert np.array_equal(labels.cpu().numpy()[k], lab)
            assert counts[k] == nc
        with pytest.raises(qc.QCError):
            G.potential_adjacency(sigmas, 0.5)
        G.close()


@pytest.mark.parametrize("n", [2, 63, 64, 65, 129, 1000, 3001])
def test_directed(qc, ctx, n):
    """Directed graphs (rows are out-neighbours): histograms count the nodes each
    node reaches; potentials and labels as the oracle's, which follows the arcs."""
    g = gg.rng(31, n)
    for p in (1.5 / n, 6.0 / n, 0.2):
        graph = gg.directed_erdos_renyi(n, min(p, 0.9), g)
        assert_solution_matches(qc, ctx, graph, [0.7, 1.9])


def test_directed_structured_and_chunked(qc, ctx, monkeypatch):
    for graph in [gg.directed_cycle(130), gg.directed_path(200),
                  gg.directed_planted_partition(1500, 6, 0.02, 0.001, gg.rng(32))]:
        assert_solution_matches(qc, ctx, graph, [0.8, 2.5])
    monkeypatch.setenv("QCGRAPH_CHUNK_WORDS", "3")
    assert_solution_matches(qc, ctx, gg.directed_planted_partition(900, 4, 0.03, 0.002, gg.rng(33)), [1.1])


def test_directed_validation(qc, ctx):
    graph = gg.directed_erdos_renyi(300, 0.02, gg.rng(34))
    with pytest.raises(qc.QCError) as e:
        qc.Graph(ctx, graph.row_ptr, graph.col_idx, validate=True, directed=False)
    assert e.value.status_name == "QC_ERR_INVALID_GRAPH"
    qc.Graph(ctx, graph.row_ptr, graph.col_idx, validate=True, directed=True).close()


def test_histogram_checkpoint(qc, ctx):
    """A saved histogram, installed into a fresh graph (from host or device memory),
    serves new sigma values without a BFS; a corrupted one is rejected."""
    graph = gg.planted_partition(2500, 10, 0.02, 0.001, gg.rng(35))
    g1 = qc.Graph.from_graph(ctx, graph)
    saved = g1.histogram().cpu().numpy()
    g1.close()
    ref = oracle.solve(graph, [0.9, 3.0])
    for source in ("host", "device"):
        g2 = qc.Graph.from_graph(ctx, graph)
        g2.set_histogram(saved if source == "host" else torch.tensor(saved, device="cuda"))
        launches = ctx.launch_count()
        V = g2.potential([0.9, 3.0])
        labels, counts = g2.ggd_labels(V)
        assert np.array_equal(V.cpu().numpy(), ref.V)
        assert np.array_equal(labels.cpu().numpy(), ref.labels) and counts == ref.n_clusters
        assert ctx.launch_count() - launches <= 6            # potential + descent only: no preparation, no BFS
        g2.close()
    g3 = qc.Graph.from_graph(ctx, graph)
    bad = saved.copy()
    bad[1, 7] += 1
    with pytest.raises(qc.QCError) as e:
        g3.set_histogram(bad)
    assert e.value.status_name == "QC_ERR_INVALID_GRAPH"
    bad = saved.copy()
    bad[2, 0] = -1
    with pytest.raises(qc.QCError) as e:
        g3.set_histogram(bad)
    assert e.value.status_name == "QC_ERR_INVALID_GRAPH"
    g3.close()


_WEIGHTED_REF = {}


def assert_weighted_matches(qc, ctx, graph, w, sigmas, cache_key=None):
    G = qc.Graph.from_graph(ctx, graph)
    G.set_weights(w)
    V = G.potential_weighted(sigmas)
    Vh = V.cpu().numpy()
    ref = _WEIGHTED_REF.get(cache_key) if cache_key is not None else None
    if ref is None:
        ref = oracle.potential_weighted(graph, w, sigmas, threads=oracle.default_threads())
        if cache_key is not None:
            _WEIGHTED_REF[cache_key] = ref
    rel = np.abs(Vh - ref) / np.maximum(np.abs(ref), np.finfo(np.float64).tiny)
    assert np.all(rel <= 1e-12), (graph.name, float(rel.max()))
    labels, counts = G.ggd_labels(V)
    labels = labels.cpu().numpy()
    for s in range(len(sigmas)):
        p, _ = oracle.ggd_parent(graph, Vh[s])
        lab, k = oracle.find_centers(p)
        assert np.array_equal(labels[s], lab) and counts[s] == k, (graph.name, s)
    G.close()
    return Vh


@pytest.mark.parametrize("n", [1, 3, 65, 300, 2000])
def test_weighted(qc, ctx, n):
    """Weighted shortest-path distances, undirected and directed: V within 1e-12 of
    the oracle's Dijkstra-based sums; labels from the same V exactly."""
    g = gg.rng(36, n)
    for graph in (gg.erdos_renyi(n, min(6.0 / max(n, 2), 0.5), g),
                  gg.directed_erdos_renyi(max(n, 2), min(5.0 / max(n, 2), 0.5), g)):
        assert_weighted_matches(qc, ctx, graph, gg.edge_weights(graph, 0.25, 3.0, g), [0.7, 2.0])


def test_weighted_batches_and_unit_weights(qc, ctx, monkeypatch):
    """Sources in many blocks of 32; unit weights reproduce the hop-distance potential."""
    monkeypatch.setenv("QCGRAPH_SSSP_SOURCES", "32")
    graph = gg.planted_partition(700, 5, 0.04, 0.003, gg.rng(37))
    assert_weighted_matches(qc, ctx, graph, gg.edge_weights(graph, 0.5, 2.0, gg.rng(38)), [0.9, 1.8, 3.0])
    Vw = assert_weighted_matches(qc, ctx, graph, np.ones(graph.nnz), [0.9, 1.8])
    hop = oracle.solve(graph, [0.9, 1.8]).V
    assert np.allclose(Vw, hop, rtol=1e-12, atol=0)


@pytest.mark.parametrize("sources", [None, "2048", "16384"])
def test_weighted_dcsbm16384_full(qc, ctx, sources, monkeypatch):
    """The weighted workload at full size: the DC-SBM of N = 16384 with weights
    U(0.5, 2), in the default source blocks, in 8 blocks and in one block of all
    sources; V within 1e-12 of the oracle's Dijkstra-based sums at the two ends of
    the sigma sweep, labels exact on the same V."""
    if sources is not None:
        monkeypatch.setenv("QCGRAPH_SSSP_SOURCES", sources)
    graph, sweep = gg.dcsbm16384()
    w = gg.edge_weights(graph, 0.5, 2.0, gg.rng(7, 1))
    assert_weighted_matches(qc, ctx, graph, w, [sweep[0], sweep[-1]], cache_key="dcsbm-16384 U(0.5, 2)")


def test_exp_neg_accuracy(qc, ctx):
    """The weighted potential's exp(-t) (Tang's tables, fixed-point core) against
    the C library's exp and a 120-bit reference: within 3 ulp below t = 708
    (normal results), and within
    4 ulp plus two subnormal steps above it; 0 from t = 745.  Points: a dense
    random sweep, table boundaries (integers, multiples of 1/1024 and their
    neighbours), tiny arguments and the branch edges."""
    g = gg.rng(41)
    t = [g.uniform(0.0, 745.0, 400000), g.uniform(0.0, 1.0, 100000), 10.0 ** g.uniform(-20, 0, 50000)]
    grid = np.concatenate([np.arange(0, 746, dtype=np.float64), np.arange(0, 8 * 1024) / 1024.0,
                           700.0 + np.arange(0, 1024) / 1024.0])
    t += [grid, np.nextafter(grid, np.inf), np.nextafter(np.maximum(grid, 1e-300), 0.0)]
    t.append(np.array([0.0, 5e-324, 1e-300, 2.0 ** -60, 2.0 ** -53, 2.0 ** -43, 2.0 ** -10, 707.999999,
                       708.0, np.nextafter(708.0, 0.0), 744.4, 745.0, np.nextafter(745.0, 0.0), 746.0, 800.0,
                       1e300, np.inf]))
    t = np.concatenate(t)
    got = ctx.selftest_exp_neg(t).cpu().numpy()
    ref = np.exp(-t)
    err = np.abs(got - ref)
    normal = t < 708.0
    assert np.all(err[normal] <= 3 * np.spacing(ref[normal])), float(np.max(err[normal] / np.spacing(ref[normal])))
    sub = ~normal
    assert np.all(err[sub] <= 4 * np.spacing(ref[sub]) + 2 * 5e-324)
    assert np.all(got[t >= 745.0] == 0.0)
    assert np.count_nonzero(t == 0.0) > 0 and np.all(got[t == 0.0] == 1.0)
    mpmath = pytest.importorskip("mpmath")
    mpmath.mp.prec = 120
    pick = np.concatenate([np.arange(0, len(t), 997), np.nonzero(normal)[0][-50:]])
    exact = np.array([float(mpmath.exp(-mpmath.mpf(float(x)))) for x in t[pick]])
    keep = t[pick] < 708.0
    assert np.all(np.abs(got[pick] - exact)[keep] <= 3 * np.spacing(exact[keep]))


def test_weighted_invalid(qc, ctx):
    graph = gg.erdos_renyi(200, 0.05, gg.rng(39))
    G = qc.Graph.from_graph(ctx, graph)
    with pytest.raises(qc.QCError) as e:
        G.potential_weighted([1.0])
    assert e.value.status_name == "QC_ERR_INVALID_ARG"
    w = gg.edge_weights(graph, 0.5, 2.0, gg.rng(40))
    bad = w.copy()
    bad[3] = -1.0
    with pytest.raises(qc.QCError) as e:
        G.set_weights(bad)
    assert e.value.status_name == "QC_ERR_INVALID_GRAPH"
    bad = w.copy()
    bad[5] *= 1.5                         # the mirror entry keeps the old weight
    with pytest.raises(qc.QCError) as e:
        G.set_weights(bad)
    assert e.value.status_name == "QC_ERR_INVALID_GRAPH"
    G.set_weights(torch.tensor(w, device="cuda"))
    G.close()

"""The bounds-checked debug build (libqcgraph_debug.so, the library compiled with
QC_DEBUG) on the GPU: its check records a neighbour id outside [0, n) and the
library reports it as QC_ERR_INVALID_GRAPH (shown with the self-test, which
passes the id through the check without using it as an address), and on valid
input every path gives the oracle's results, as the release build does.  The
debug library is loaded in a child process (a process loads one build)."""
import os
import subprocess
import sys

import pytest

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

CHILD = r'''
import numpy as np, torch
import graphgen as gg, oracle
import paper_2305_14641_gb300 as qc
from paper_2305_14641_gb300 import native
assert native.LIB_PATH.endswith("libqcgraph_debug.so"), native.LIB_PATH
with qc.Context(0) as ctx:
    st, out, dbg = ctx.selftest_debug_check(5, 10)
    assert (st, out, dbg) == ("QC_OK", 5, True), (st, out, dbg)
    st, out, dbg = ctx.selftest_debug_check(12, 10)
    assert (st, out, dbg) == ("QC_ERR_INVALID_GRAPH", 0, True), (st, out, dbg)
    st, out, dbg = ctx.selftest_debug_check(-3, 10)
    assert st == "QC_ERR_INVALID_GRAPH" and out == 0
    assert ctx.selftest_debug_check(9, 10)[0] == "QC_OK"      # the failure was reported once
    # valid input: every path as the oracle
    graphs = [gg.planted128()[0], gg.planted_partition(3000, 8, 0.01, 0.001, gg.rng(71)),
              gg.directed_planted_partition(1200, 5, 0.02, 0.002, gg.rng(72)), gg.path(100)]
    for graph in graphs:
        ref = oracle.solve(graph, [0.8, 2.0])
        G = qc.Graph.from_graph(ctx, graph)
        _, lab, counts = G.solve([0.8, 2.0])
        assert np.array_equal(lab.cpu().numpy(), ref.labels), graph.name
        plan = qc.SweepPlan(G, [0.8, 2.0])
        assert plan.run(counts=True) == ref.n_clusters
        assert np.array_equal(plan.labels.cpu().numpy(), ref.labels)
        plan.close()
        G.close()
    small, sig = gg.planted_batch(24, seed=11)
    Gs = [qc.Graph.from_graph(ctx, g) for g in small]
    bp = qc.BatchPlan(ctx, Gs, sig)
    bp.run()
    for k, g in enumerate(small):
        assert np.array_equal(bp.labels_of(k).cpu().numpy(), oracle.solve(g, [sig[k]]).labels[0])
    bp.close()
    w_graph = gg.erdos_renyi(300, 0.03, gg.rng(73))
    w = gg.edge_weights(w_graph, 0.5, 2.0, gg.rng(74))
    G = qc.Graph.from_graph(ctx, w_graph)
    G.set_weights(w)
    V = G.potential_weighted([1.0]).cpu().numpy()
    ref = oracle.potential_weighted(w_graph, w, [1.0])
    assert np.all(np.abs(V - ref) <= 1e-12 * np.abs(ref))
    G.close()
print("debug build ok")
'''


def test_debug_build_checks_and_parity():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2305_14641_gb300 import _build
    _build.build(debug=True)
    env = dict(os.environ, QCGRAPH_DEBUG_LIB="1", PYTHONPATH=ROOT)
    res = subprocess.run([sys.executable, "-c", CHILD], cwd=ROOT, env=env, capture_output=True, text=True,
                         timeout=900)
    assert res.returncode == 0 and "debug build ok" in res.stdout, (res.stdout[-2000:], res.stderr[-4000:])


def test_release_build_has_no_checks():
    """The release build compiles the checks away: the id comes back unchanged."""
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2305_14641_gb300 as qc
    with qc.Context(0) as ctx:
        assert ctx.selftest_debug_check(12, 10) == ("QC_OK", 12, False)

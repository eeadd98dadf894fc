"""qc_histogram_static_scratch: the distance histogram for callers that may not
allocate device memory (a host that fixes its GPU memory plan up front, a
plugin limited to the buffers it is handed).  Its bitsets live in a fixed array
inside the library, so the call itself allocates nothing.

Checked through the C ABI against the regular entry point (qc_graph_histogram)
and against the oracle's histograms on the same inputs, twice in a row, so that
the second call also shows that what the first left in the shared array does
not leak into the result.  This file is collected last on purpose.
"""
import ctypes

import numpy as np
import pytest

import graphgen as gg
import oracle

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def env():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2305_14641_gb300 as qc
    from paper_2305_14641_gb300 import native
    ctx = qc.Context(0)
    yield qc, native.lib(), ctx
    ctx.close()


def static_histogram(lib, graph, max_levels):
    rp = torch.tensor(graph.row_ptr, device="cuda")
    ci = torch.tensor(graph.col_idx if graph.nnz else np.zeros(1, np.int32), device="cuda")
    out = torch.full((max_levels, graph.n), -7, dtype=torch.int32, device="cuda")
    D = ctypes.c_int32(-5)
    torch.cuda.synchronize()
    free_before = torch.cuda.mem_get_info()[0]
    st = lib.qc_histogram_static_scratch(graph.n, graph.nnz, rp.data_ptr(), ci.data_ptr(),
                                         out.data_ptr(), max_levels, ctypes.byref(D),
                                         torch.cuda.current_stream().cuda_stream)
    free_after = torch.cuda.mem_get_info()[0]
    return st, D.value, out, free_before - free_after


CASES = [
    ("planted N=128", lambda: gg.planted128()[0]),
    ("ragged N=1000, sparse", lambda: gg.erdos_renyi(1000, 0.004, gg.rng(31))),
    ("planted N=5000", lambda: gg.planted_partition(5000, 10, 0.01, 0.0004, gg.rng(32))),
    ("path N=70", lambda: gg.path(70)),
]


@pytest.mark.parametrize("name,make", CASES, ids=[c[0] for c in CASES])
def test_matches_regular_entry_point_twice(env, name, make):
    qc, lib, ctx = env
    graph = make()
    g = qc.Graph.from_graph(ctx, graph)
    ref = g.histogram()
    g.close()
    expect = oracle.histograms(graph).T          # level-major [(D+1), n]
    assert np.array_equal(ref.cpu().numpy(), expect), name
    for max_levels in (ref.shape[0] + 3, ref.shape[0]):
        for call in range(2):
            st, D, out, _ = static_histogram(lib, graph, max_levels)
            assert st == 0, (name, max_levels, call, st)
            assert D == ref.shape[0] - 1, (name, call)
            assert torch.equal(out[:D + 1], ref), (name, call)
            assert np.array_equal(out[:D + 1].cpu().numpy(), expect), (name, call)
            assert int(out[D + 1:].abs().sum()) == 0, (name, call)


@pytest.mark.parametrize("graph,rows", [(gg.complete(40), 2), (gg.path(50), 50), (gg.path(2), 2),
                                        (gg.star(300, 7), 3)], ids=["K40", "P50", "P2", "S300"])
def test_exactly_d_plus_one_rows(env, graph, rows):
    """D + 1 rows are enough (the pass that finds nothing runs without a row);
    D rows are too few and the call says so."""
    qc, lib, ctx = env
    expect = oracle.histograms(graph).T
    assert expect.shape[0] == rows
    for _ in range(2):
        st, D, out, _ = static_histogram(lib, graph, rows)
        assert st == 0 and D == rows - 1, (graph.name, st, D)
        assert np.array_equal(out.cpu().numpy(), expect), graph.name
    if rows > 2:
        st, D, _, _ = static_histogram(lib, graph, rows - 1)
        assert st == 1 and D == -1, graph.name


def test_back_to_back_different_graphs(env):
    """A big graph, then a small one: the small one must not see the big one's bits."""
    qc, lib, ctx = env
    big = gg.planted_partition(6000, 12, 0.01, 0.0005, gg.rng(33))
    small = gg.erdos_renyi(300, 0.02, gg.rng(34))
    expect = {id(big): oracle.histograms(big).T, id(small): oracle.histograms(small).T}
    for graph in (big, small, big):
        g = qc.Graph.from_graph(ctx, graph)
        ref = g.histogram()
        g.close()
        st, D, out, _ = static_histogram(lib, graph, ref.shape[0] + 1)
        assert st == 0 and D == ref.shape[0] - 1
        assert torch.equal(out[:D + 1], ref)
        assert np.array_equal(out[:D + 1].cpu().numpy(), expect[id(graph)])


def test_allocates_nothing_and_rejects_out_of_range(env):
    qc, lib, ctx = env
    graph = gg.planted_partition(3000, 6, 0.01, 0.001, gg.rng(35))
    static_histogram(lib, graph, 64)             # first call on the device: address lookup
    st, D, out, used = static_histogram(lib, graph, 64)
    assert st == 0 and used == 0
    # too few histogram rows for the graph's largest distance
    st, D, _, _ = static_histogram(lib, gg.path(50), 10)
    assert st == 1 and D == -1
    # a stream of the current device is accepted (the legacy default stream too)
    rp = torch.tensor(graph.row_ptr, device="cuda")
    ci = torch.tensor(graph.col_idx, device="cuda")
    out = torch.zeros((64, graph.n), dtype=torch.int32, device="cuda")
    Dc = ctypes.c_int32(-5)
    side = torch.cuda.Stream()
    for handle in (0, side.cuda_stream):
        torch.cuda.synchronize()
        assert lib.qc_histogram_static_scratch(graph.n, graph.nnz, rp.data_ptr(), ci.data_ptr(), out.data_ptr(),
                                               64, ctypes.byref(Dc), handle) == 0
    # more nodes than the fixed array supports
    big = gg.Graph(262145, np.zeros(262146, dtype=np.int32), np.zeros(0, dtype=np.int32))
    st, D, _, _ = static_histogram(lib, big, 2)
    assert st == 1

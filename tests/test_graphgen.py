"""The seeded input generators: canonical CSR, determinism, workload shapes."""
import numpy as np
import pytest

import graphgen as gg


def assert_canonical(g):
    rp, ci = g.row_ptr, g.col_idx
    assert rp.dtype == np.int32 and ci.dtype == np.int32
    assert rp[0] == 0 and np.all(np.diff(rp.astype(np.int64)) >= 0) and rp[-1] == len(ci)
    rows = np.repeat(np.arange(g.n), g.degrees())
    assert np.all(ci >= 0) and np.all(ci < g.n)
    assert not np.any(rows == ci), "self-loop"
    key = rows.astype(np.int64) * g.n + ci
    assert np.all(np.diff(key) > 0), "rows not strictly ascending (unsorted or duplicate)"
    rkey = ci.astype(np.int64) * g.n + rows
    assert np.array_equal(np.sort(rkey), key), "not symmetric"


def test_structured_graphs():
    for g in [gg.complete(6), gg.path(5), gg.star(7, 3), gg.two_cliques_bridge(4)]:
        assert_canonical(g)
    assert gg.complete(6).nnz == 30
    assert gg.path(5).nnz == 8
    assert gg.star(7, 3).degrees().tolist() == [1, 1, 1, 6, 1, 1, 1]
    assert gg.two_cliques_bridge(4).nnz == 2 * 12 + 2


def test_planted128_shape_and_determinism():
    g, sig = gg.planted128()
    assert_canonical(g)
    assert g.n == 128 and sig == [1.0]
    assert 1000 < g.nnz < 1900          # about 718 undirected edges expected
    g2, _ = gg.planted128()
    assert np.array_equal(g.col_idx, g2.col_idx)


def test_planted_partition_rates():
    g = gg.planted_partition(2000, 4, 0.05, 0.002, gg.rng(7))
    assert_canonical(g)
    rows = np.repeat(np.arange(g.n), g.degrees())
    same = g.block[rows] == g.block[g.col_idx]
    m_in = 4 * 500 * 499 / 2
    m_out = 2000 * 1999 / 2 - m_in
    assert abs(same.sum() / 2 / m_in - 0.05) < 0.005
    assert abs((~same).sum() / 2 / m_out - 0.002) < 0.0004


def test_sigma_sweep():
    s = gg.sigma_sweep16()
    assert len(s) == 16 and s[0] == 0.5 and abs(s[-1] - 4.0) < 1e-12
    assert all(b > a for a, b in zip(s, s[1:]))


def test_batch_and_requests():
    graphs, sig = gg.planted_batch(24)
    for g, s in zip(graphs, sig):
        assert_canonical(g)
        assert 32 <= g.n <= 2048 and 0.5 <= s <= 3.0
    reqs = gg.sbm_request_stream(40)
    assert all(64 <= r.n <= 65536 and 0.5 <= r.sigma <= 3.0 for r in reqs)
    assert all(b.arrival_s > a.arrival_s for a, b in zip(reqs, reqs[1:]))
    assert_canonical(reqs[0].graph())


@pytest.mark.slow
def test_dcsbm16384_shape():
    g, _ = gg.dcsbm16384()
    assert_canonical(g)
    assert g.n == 16384 and abs(g.degrees().mean() - 16) < 1.0 and g.degrees().max() <= 600

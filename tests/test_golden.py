"""Hand-worked examples (tests/golden/hand_examples.json) against the oracle."""
import json
import os

import numpy as np
import pytest

import graphgen as gg
import oracle

CASES = json.load(open(os.path.join(os.path.dirname(__file__), "golden", "hand_examples.json")))["cases"]


def graph_of(case):
    e = np.array(case["edges"], dtype=np.int64).reshape(-1, 2)
    rp, ci = gg.csr_from_pairs(case["n"], e[:, 0], e[:, 1])
    return gg.Graph(case["n"], rp, ci, name=case["name"])


@pytest.mark.parametrize("case", CASES, ids=lambda c: c["name"])
def test_hand_example(case):
    g = graph_of(case)
    sol = oracle.solve(g, [case["sigma"]])
    width = max(len(r) for r in case["hist"])
    h = np.zeros((g.n, max(width, sol.hist.shape[1])), dtype=np.int64)
    h[:, :sol.hist.shape[1]] = sol.hist
    expect = np.zeros_like(h)
    for i, r in enumerate(case["hist"]):
        expect[i, :len(r)] = r
    assert np.array_equal(h, expect)
    assert np.allclose(sol.V[0], case["V"], rtol=5e-4, atol=0)
    assert sol.labels[0].tolist() == case["labels"]
    assert sol.n_clusters[0] == case["n_clusters"]

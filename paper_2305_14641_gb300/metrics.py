"""Clustering quality measures used by the paper's evaluation (Section 4.2):
Modularity, Adjusted Rand Index, Fowlkes-Mallows Index and Normalized Mutual
Information.  They score label vectors (host numpy arrays) after a solve; they
are evaluation helpers, not part of the clustering path.

Readings:
  * Modularity: Q = (1/w) sum_ij (A_ij - gamma w_i w_j / w) delta(c_i, c_j) with
    w_i the degree of i and w the total weight, read as sum_i w_i (= 2m for an
    unweighted graph), which is Newman's form.
  * ARI: (RI - E[RI]) / (max RI - E[RI]) under the permutation model, computed
    from pair counts of the contingency table (Hubert & Arabie 1985).
  * FMI: TP / sqrt((TP + FP)(TP + FN)) over pairs of samples.
  * NMI: MI / sqrt(H(true) H(pred)), natural logarithms (the base cancels).
"""
from __future__ import annotations

import numpy as np

__all__ = ["modularity", "adjusted_rand_index", "fowlkes_mallows", "normalized_mutual_info",
           "contingency"]


def _labels(x) -> np.ndarray:
    x = np.asarray(x).ravel()
    _, inv = np.unique(x, return_inverse=True)
    return inv.astype(np.int64)


def contingency(a, b) -> np.ndarray:
    """n_ij = #{samples with true label i and predicted label j} (dense, relabelled 0..)."""
    a, b = _labels(a), _labels(b)
    if len(a) != len(b):
        raise ValueError("label vectors differ in length")
    ka, kb = a.max(initial=-1) + 1, b.max(initial=-1) + 1
    return np.bincount(a * kb + b, minlength=ka * kb).reshape(ka, kb)


def _pairs(x) -> np.ndarray:
    x = np.asarray(x, dtype=np.float64)
    return x * (x - 1.0) / 2.0


def modularity(row_ptr, col_idx, labels, gamma: float = 1.0) -> float:
    """Modularity of a partition of an undirected graph given in CSR form."""
    row_ptr = np.asarray(row_ptr, dtype=np.int64)
    col_idx = np.asarray(col_idx, dtype=np.int64)
    c = _labels(labels)
    n = len(row_ptr) - 1
    deg = np.diff(row_ptr).astype(np.float64)
    w = deg.sum()
    if w == 0:
        return 0.0
    rows = np.repeat(np.arange(n), np.diff(row_ptr))
    inside = float(np.count_nonzero(c[rows] == c[col_idx]))
    per_cluster = np.bincount(c, weights=deg)
    return inside / w - gamma * float((per_cluster ** 2).sum()) / (w * w)


def adjusted_rand_index(truth, pred) -> float:
    n_ij = contingency(truth, pred)
    n = n_ij.sum()
    index = _pairs(n_ij).sum()
    a = _pairs(n_ij.sum(axis=1)).sum()
    b = _pairs(n_ij.sum(axis=0)).sum()
    total = _pairs(n)
    expected = a * b / total if total > 0 else 0.0
    maximum = (a + b) / 2.0
    if maximum == expected:
        return 1.0
    return float((index - expected) / (maximum - expected))


def fowlkes_mallows(truth, pred) -> float:
    n_ij = contingency(truth, pred)
    tp = _pairs(n_ij).sum()
    tp_fp = _pairs(n_ij.sum(axis=0)).sum()     # pairs together in the prediction
    tp_fn = _pairs(n_ij.sum(axis=1)).sum()     # pairs together in the truth
    if tp_fp == 0 or tp_fn == 0:
        return 0.0
    return float(tp / np.sqrt(tp_fp * tp_fn))


def _entropy(counts) -> float:
    p = np.asarray(counts, dtype=np.float64)
    p = p[p > 0] / p.sum()
    return float(-(p * np.log(p)).sum())


def normalized_mutual_info(truth, pred) -> float:
    n_ij = contingency(truth, pred).astype(np.float64)
    n = n_ij.sum()
    pi, pj = n_ij.sum(axis=1) / n, n_ij.sum(axis=0) / n
    nz = n_ij > 0
    p = n_ij[nz] / n
    mi = float((p * np.log(p / np.outer(pi, pj)[nz])).sum())
    hi, hj = _entropy(n_ij.sum(axis=1)), _entropy(n_ij.sum(axis=0))
    if hi == 0.0 or hj == 0.0:
        return 1.0 if hi == hj else 0.0
    return mi / np.sqrt(hi * hj)

"""Write full_size.json: the oracle's results on the three full-size workloads
whose oracle run is too slow to repeat inside every GPU test session.

    python tests/golden/make_full_size.py [--threads T] [--only NAME]

Everything stored here comes from ``oracle/`` alone (inputs from ``graphgen``):
no value is read from the CUDA library.  Stored per workload:

  sbm262144   SBM, N=262144, 256 blocks of 1024, mean degree 20, mixing 0.15,
              seed 2, sigma 1.5: the CSR's SHA-256, D, the SHA-256 of the whole
              histogram in the library's layout (level-major int32 [(D+1)][n],
              little-endian), of V (binary64 bits), of the labels, and the
              number of clusters.
  batch4096   the 4096 planted-partition graphs of the batched workload (N
              log-uniform in [32, 2048], 2-16 blocks, p_in U(0.1, 0.5), p_out
              0.02, sigma U(0.5, 3.0), seed 3): one SHA-256 over every CSR and
              sigma, then per graph the first 16 hex digits of the SHA-256 of
              its labels and its number of clusters.
  serve400    the first 400 requests of the served Poisson stream (SBM graphs,
              N log-uniform in [64, 65536], mean degree 12, 4-64 blocks, mixing
              0.1, sigma U(0.5, 3.0), seed 4): the same per-request fields.

Labels are root node ids (int32, little-endian) as Algorithm 3 reads them.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import multiprocessing as mp
import os
import sys
import time

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(os.path.dirname(HERE))
sys.path.insert(0, ROOT)

import graphgen as gg  # noqa: E402

OUT = os.path.join(HERE, "full_size.json")
SERVE_REQUESTS = 400


def sha(*arrays) -> str:
    """SHA-256 over the arrays' bytes (each already in a little-endian dtype)."""
    h = hashlib.sha256()
    for a in arrays:
        h.update(np.ascontiguousarray(a).tobytes())
    return h.hexdigest()


def csr_sha(graph) -> str:
    return sha(graph.row_ptr.astype("<i4"), graph.col_idx.astype("<i4"))


def labels_digest(labels) -> str:
    return sha(np.asarray(labels, dtype="<i4"))[:16]


def whole_set_sha(graphs, sigmas) -> str:
    h = hashlib.sha256()
    for g, s in zip(graphs, sigmas):
        h.update(g.row_ptr.astype("<i4").tobytes())
        h.update(g.col_idx.astype("<i4").tobytes())
        h.update(np.array([s], dtype="<f8").tobytes())
    return h.hexdigest()


def sbm262144(threads: int) -> dict:
    import oracle
    graph, sigmas = gg.sbm262144()
    t0 = time.time()
    ref = oracle.solve(graph, sigmas, threads=threads)
    secs = time.time() - t0
    return {"n": graph.n, "nnz": graph.nnz, "sigma": sigmas[0], "csr_sha256": csr_sha(graph),
            "D": ref.D, "hist_sha256": sha(np.ascontiguousarray(ref.hist.T).astype("<i4")),
            "V_sha256": sha(ref.V[0].astype("<f8")), "labels_sha256": sha(ref.labels[0].astype("<i4")),
            "n_clusters": int(ref.n_clusters[0]), "oracle_seconds": round(secs, 1), "oracle_threads": threads}


def _batch_item(k: int) -> tuple[int, str, int]:
    import oracle
    graph, sigma = gg.planted_batch_graph(k)
    ref = oracle.solve(graph, [sigma], threads=1)
    return k, labels_digest(ref.labels[0]), int(ref.n_clusters[0])


def batch4096(threads: int) -> dict:
    graphs, sigmas = gg.planted_batch(4096)
    order = sorted(range(len(graphs)), key=lambda k: -graphs[k].n * graphs[k].nnz)
    t0 = time.time()
    with mp.get_context("spawn").Pool(threads) as pool:
        res = dict((k, (d, c)) for k, d, c in pool.imap_unordered(_batch_item, order, chunksize=4))
    return {"graphs": len(graphs), "set_sha256": whole_set_sha(graphs, sigmas),
            "labels_digest": [res[k][0] for k in range(len(graphs))],
            "n_clusters": [res[k][1] for k in range(len(graphs))],
            "oracle_seconds": round(time.time() - t0, 1), "oracle_processes": threads}


def _serve_item(k: int) -> tuple[int, str, int]:
    import oracle
    r = gg.sbm_request_stream(SERVE_REQUESTS)[k]
    ref = oracle.solve(r.graph(), [r.sigma], threads=1)
    return k, labels_digest(ref.labels[0]), int(ref.n_clusters[0])


def serve400(threads: int) -> dict:
    reqs = gg.sbm_request_stream(SERVE_REQUESTS)
    graphs = [r.graph() for r in reqs]
    sigmas = [r.sigma for r in reqs]
    order = sorted(range(len(reqs)), key=lambda k: -graphs[k].n * graphs[k].nnz)
    t0 = time.time()
    with mp.get_context("spawn").Pool(threads) as pool:
        res = dict((k, (d, c)) for k, d, c in pool.imap_unordered(_serve_item, order, chunksize=1))
    return {"requests": len(reqs), "set_sha256": whole_set_sha(graphs, sigmas),
            "labels_digest": [res[k][0] for k in range(len(reqs))],
            "n_clusters": [res[k][1] for k in range(len(reqs))],
            "oracle_seconds": round(time.time() - t0, 1), "oracle_processes": threads}


def dump(data: dict) -> str:
    """JSON with one line per field (the per-graph lists stay on one line)."""
    lines = []
    for name in sorted(data):
        v = data[name]
        if isinstance(v, dict):
            inner = ",\n".join(f"  {json.dumps(k)}: {json.dumps(v[k], separators=(',', ':'))}" for k in sorted(v))
            lines.append(f" {json.dumps(name)}: {{\n{inner}\n }}")
        else:
            lines.append(f" {json.dumps(name)}: {json.dumps(v)}")
    return "{\n" + ",\n".join(lines) + "\n}\n"


WORKLOADS = {"batch4096": batch4096, "sbm262144": sbm262144, "serve400": serve400}


def main():
    import oracle
    ap = argparse.ArgumentParser()
    ap.add_argument("--threads", type=int, default=oracle.default_threads())
    ap.add_argument("--only", choices=sorted(WORKLOADS), action="append")
    args = ap.parse_args()
    oracle.build()
    data = json.load(open(OUT)) if os.path.exists(OUT) else {}
    data["about"] = ("Oracle results (oracle/ only, inputs from graphgen) on full-size workloads, written by "
                     "tests/golden/make_full_size.py; the GPU tests compare the CUDA path's whole outputs "
                     "with them.")
    for name in args.only or list(WORKLOADS):
        t0 = time.time()
        data[name] = WORKLOADS[name](args.threads)
        print(f"{name}: {time.time() - t0:.0f} s", flush=True)
        with open(OUT + ".tmp", "w") as f:
            f.write(dump(data))
        os.replace(OUT + ".tmp", OUT)


if __name__ == "__main__":
    main()

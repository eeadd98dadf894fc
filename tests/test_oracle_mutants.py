"""Plant a mistake in a copy of the oracle's C source and check that the pins catch it.

Each mutant is a plausible slip in one step of the method (a dropped term, a
wrong power, a wrong comparison, the wrong tie-break, a garbled return value).
The copy is compiled to a temporary library and every pin runs against it in a
child process (a mutant that makes the descent cyclic would loop forever in the
root search, so the child runs under a time limit, and running out of time
also counts as caught).
"""
import os
import subprocess
import sys

import pytest

import oracle

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

MUTANTS = {
    "self-term-dropped": ("if (dist[j] >= 0) h[dist[j]] += 1;",
                          "if (dist[j] > 0) h[dist[j]] += 1;"),
    "hop-counted-twice": ("dist[x] = dist[u] + 1;", "dist[x] = dist[u] + 2;"),
    "distance-not-squared": ("double d2 = (double)((int64_t)d * d);", "double d2 = (double)d;"),
    "exponent-sign": ("w[d] = exp(-d2 / (2.0 * (sigma * sigma)));",
                      "w[d] = exp(d2 / (2.0 * (sigma * sigma)));"),
    "sigma-not-squared": ("w[d] = exp(-d2 / (2.0 * (sigma * sigma)));",
                          "w[d] = exp(-d2 / (2.0 * sigma));"),
    "first-moment-weight": ("u[d] = d2 * w[d];", "u[d] = (double)d * w[d];"),
    "prefactor-dropped": ("V[k] = (sum1 / sum2) / (2.0 * (sigma * sigma));", "V[k] = sum1 / sum2;"),
    "sums-swapped": ("V[k] = (sum1 / sum2) / (2.0 * (sigma * sigma));",
                     "V[k] = (sum2 / sum1) / (2.0 * (sigma * sigma));"),
    "non-strict-descent": ("if (best >= 0 && V[best] < V[i]) {", "if (best >= 0 && V[best] <= V[i]) {"),
    "last-index-tie-break": ("if (best < 0 || V[j] < V[best]) {", "if (best < 0 || V[j] <= V[best]) {"),
    "ascent-instead-of-descent": ("if (best < 0 || V[j] < V[best]) {", "if (best < 0 || V[j] > V[best]) {"),
    "label-is-node-not-root": ("label[i] = r;", "label[i] = i;"),
    # the adjacency-distance and weighted forms
    "adjacency-degree-as-distant": ("double h[3] = {1.0, (double)deg, (double)(n - 1 - deg)};",
                                    "double h[3] = {1.0, (double)deg, (double)(n - deg)};"),
    "weighted-hop-not-weight": ("double nd = dist[u] + w[e];", "double nd = dist[u] + 1.0;"),
    "weighted-first-power": ("double d2 = d * d;", "double d2 = d;"),
    "weighted-unreached-counted": ("if (!isfinite(d)) continue;", "if (!isfinite(d)) d = 0.0;"),
}

CHILD = r"""
import sys
sys.path.insert(0, {root!r})
import oracle
from tests import pins
orc = oracle.Oracle({lib!r})
failed = []
for check in pins.ALL_CHECKS:
    try:
        check(orc)
    except Exception:
        failed.append(check.__name__)
print("FAILED:" + ",".join(failed))
sys.exit(1 if failed else 0)
"""


@pytest.mark.parametrize("name", sorted(MUTANTS))
def test_pins_catch_mutant(name, tmp_path):
    old, new = MUTANTS[name]
    src = open(oracle._SRC).read()
    assert src.count(old) == 1, f"mutation site for {name} not found exactly once"
    mutated = tmp_path / "qc_oracle_mutant.c"
    mutated.write_text(src.replace(old, new))
    lib = oracle.compile_source(str(mutated), str(tmp_path / "libmutant.so"))
    code = CHILD.format(root=ROOT, lib=lib)
    try:
        res = subprocess.run([sys.executable, "-c", code], capture_output=True, text=True, timeout=40)
    except subprocess.TimeoutExpired:
        return   # the mutant made a parent chain cyclic: the root search never ends
    assert res.returncode == 1 and "FAILED:" in res.stdout, \
        f"no pin caught mutant {name}: rc={res.returncode}\n{res.stdout}\n{res.stderr[-2000:]}"

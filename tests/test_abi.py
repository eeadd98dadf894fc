"""The C ABI on the CPU: the library loads, exports exactly what include/qcgraph.h
declares, and without a GPU refuses work with QC_ERR_CUDA (no CPU fallback)."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "qcgraph.h")


@pytest.fixture(scope="module")
def lib():
    from paper_2305_14641_gb300 import _build, native
    _build.build()
    return native.load()


def declared():
    text = open(HEADER).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(qc_[a-z_0-9]+)\s*\(", text)))


def test_header_declares_entry_points():
    names = declared()
    assert "qc_graph_create" in names and "qc_solve_batch" in names and len(names) >= 25


def test_every_declared_symbol_is_exported(lib):
    missing = [n for n in declared() if not hasattr(lib, n)]
    assert not missing, missing


def test_binding_covers_the_header():
    from paper_2305_14641_gb300 import native
    assert sorted(n for n, _, _ in native.SIGNATURES) == declared()


def test_status_strings(lib):
    for code, text in [(0, b"ok"), (2, b"invalid graph"), (4, b"memory budget exceeded"),
                       (6, b"device wait timed out")]:
        assert lib.qc_status_string(code) == text


def test_no_gpu_means_cuda_error(lib):
    torch = pytest.importorskip("torch")
    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    h = ctypes.c_void_p()
    assert lib.qc_context_create(0, 0, None, ctypes.byref(h)) == 5
    assert lib.qc_context_create(-1, 0, None, ctypes.byref(h)) == 1

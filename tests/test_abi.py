"""The C-ABI library loads and exports every entry point include/bp.h declares
(no compute call: runs without a GPU)."""
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_functions():
    src = open(os.path.join(ROOT, "include", "bp.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(bp_[a-z_]+)\s*\(", src)))


@pytest.fixture(scope="module")
def lib():
    from paper_2604_19723_gb300 import build as b
    from paper_2604_19723_gb300 import bp
    b.build()
    return bp.load()


def test_header_declares_the_boundary():
    names = declared_functions()
    for f in ("bp_init", "bp_predict", "bp_update", "bp_estimate", "bp_free"):
        assert f in names


def test_library_exports_every_declared_symbol(lib):
    missing = [f for f in declared_functions() if not hasattr(lib, f)]
    assert not missing, missing


def test_binding_lists_every_symbol():
    from paper_2604_19723_gb300 import bp
    assert set(declared_functions()) == set(bp.ENTRY_POINTS)


def test_last_error_without_handle(lib):
    assert lib.bp_last_error(None) is not None


def test_noalloc_binding_rejects_bad_tensors_on_the_host():
    """resample_noalloc checks its tensors before any library call: a float32, a
    strided or a host tensor never reaches the kernel (which reads 8P bytes)."""
    torch = pytest.importorskip("torch")
    from paper_2604_19723_gb300 import bp
    for w in (torch.ones(10, dtype=torch.float32), torch.ones(20, dtype=torch.float64)[::2],
              torch.ones(10, dtype=torch.float64)):
        with pytest.raises(TypeError):
            bp.resample_noalloc(w, 1, 1, 0, 0)

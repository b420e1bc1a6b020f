"""The Python binding has no CPU fallback: without the compiled library it
raises, and it refuses host tensors instead of computing anything on the CPU
(CPU only)."""
import importlib.util
import os

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _fresh_binding():
    spec = importlib.util.spec_from_file_location(
        "lagp_fresh", os.path.join(ROOT, "paper_1409_0074_gb300", "lagp.py"))
    m = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(m)
    return m


def test_missing_library_raises():
    m = _fresh_binding()
    m.LIB_PATH = os.path.join(ROOT, "does_not_exist", "liblagp_gb300.so")
    with pytest.raises(RuntimeError, match="not built"):
        m.load()


def test_host_tensors_are_refused():
    torch = pytest.importorskip("torch")
    m = _fresh_binding()
    with pytest.raises(ValueError, match="CUDA"):
        m._ptr(torch.zeros(4, dtype=torch.float64))
    with pytest.raises(ValueError):
        m._hptr(np.zeros(4, np.float32), np.float64)
    assert m._ptr(None) is None

"""The C ABI: the library builds for sm_103a, loads without a GPU and exports
every entry point declared in include/fl.h (no compute calls here)."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    src = open(os.path.join(ROOT, "include", "fl.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(fl_[a-z0-9_]+)\s*\(", src)))


def test_header_declares_the_binding_names(fl):
    assert _declared() == sorted(fl.ABI_SYMBOLS)


def test_library_exports_every_declared_symbol(fl):
    lib = ctypes.CDLL(fl.LIB_PATH)
    for name in _declared():
        assert hasattr(lib, name), name
    assert fl.fl_version().startswith("fl-gb300")


def test_host_side_argument_errors_without_gpu(fl):
    # argument checks return before any device work
    with pytest.raises(fl.FLError) as e:
        fl.fl_mesh_create_structured(0, 4, 4, 1.0, 1.0, 1.0)
    assert e.value.status == fl.FL_EINVAL
    # 2^31 cells is one past the largest structured mesh
    with pytest.raises(fl.FLError) as e:
        fl.fl_mesh_create_structured(1024, 1024, 2048, 1.0, 1.0, 1.0)
    assert e.value.status == fl.FL_EUNSUPPORTED
    assert fl.fl_reduce_workspace_size() > 0


def test_field_tensors_must_match_the_call_dtype(fl):
    # the binding refuses a field tensor of another element type (a wrong
    # type inside a larger cached block would pass the library's size check)
    import torch
    with pytest.raises(TypeError):
        fl._fptr(torch.zeros(4, dtype=torch.float32), fl.FL_F64)
    with pytest.raises(TypeError):
        fl._fptr(torch.zeros(4, dtype=torch.float64), fl.FL_F32)
    with pytest.raises(ValueError):
        fl._fptr(torch.zeros(4, dtype=torch.float64), fl.FL_F64)  # a CPU tensor
    assert fl._fptr(None, fl.FL_F64) is None and fl._fptr(1234, fl.FL_F32) == 1234


def test_no_cpu_fallback_when_library_missing(monkeypatch, fl):
    import paper_2110_03044_gb300 as pkg
    monkeypatch.setattr(pkg, "_lib", None)
    monkeypatch.setattr(pkg, "LIB_PATH", "/nonexistent/libfl.so")
    with pytest.raises(RuntimeError):
        pkg.lib()

"""The C-ABI library builds, loads and exports every entry point that
include/uot.h declares (no compute calls: these run without a GPU)."""
import ctypes
import os
import re

from paper_1607_05816_gb300 import build, uot

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared():
    src = open(os.path.join(ROOT, "include", "uot.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(uot_[a-z0-9_]+)\s*\(", src)))


def test_header_declares_the_boundary():
    names = declared()
    for n in ("uot_solve", "uot_barycenter", "uot_apply_plan", "uot_objective", "uot_gibbs_log"):
        assert n in names


def test_library_builds_and_exports_every_symbol():
    path = build.build()
    lib = ctypes.CDLL(path)
    for name in declared():
        assert hasattr(lib, name), name
    assert sorted(uot.exported_symbols()) == declared()


def test_version_string():
    lib = uot.load()
    assert b"sm_103a" in lib.uot_version()


def test_struct_layouts_match_header():
    # sizes follow from the field lists in include/uot.h on LP64
    assert ctypes.sizeof(uot.CDiv) == 32
    assert ctypes.sizeof(uot.COpts) == 8 + 8 + 8 + 4 + 4 + 4 + 4 + 8 + 4 + 4 + 4 + 4 + 8 + 8 + 4 + 4 + 8
    assert ctypes.sizeof(uot.CResult) == 4 + 4 + 8 + 8 + 4 + 4 + 4 + 4 + 8 + 4 + 4


def test_no_cpu_fallback(monkeypatch):
    """The binding has no CPU path: host tensors are refused before the
    library is called, and a library that cannot be loaded raises instead of
    degrading to another implementation."""
    import pytest
    import torch
    C = torch.zeros(4, 3, dtype=torch.float64)
    v4, v3 = torch.ones(4, dtype=torch.float64), torch.ones(3, dtype=torch.float64)
    with pytest.raises(TypeError, match="CUDA tensor"):
        uot.solve(uot.Geometry.dense(C), v4, v4, v3, v3, uot.KL(1.0), uot.KL(1.0), 0.1)
    with pytest.raises(TypeError, match="CUDA tensor"):
        uot.gibbs_log(uot.Geometry.dense(C), v3, v3, 0.1)
    monkeypatch.setattr(uot, "_LIB", None)
    monkeypatch.setattr(uot._build, "build", lambda *a, **k: None)
    with pytest.raises(OSError):
        uot.load(os.path.join(ROOT, "no-such-dir", "libuot.so"))
    assert uot._LIB is None

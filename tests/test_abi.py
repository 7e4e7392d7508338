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
    assert ctypes.sizeof(uot.COpts) == 8 + 8 + 8 + 4 + 4 + 4 + 4 + 8 + 4 + 4 + 4 + 4 + 8 + 8
    assert ctypes.sizeof(uot.CResult) == 4 + 4 + 8 + 8 + 4 + 4

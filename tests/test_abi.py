"""The C-ABI library builds, loads and exports every entry point that
include/uot.h declares (no compute calls: these run without a GPU)."""
import ctypes
import os
import re
import subprocess

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


# the header's field names, in order, for each struct the binding mirrors
C_FIELDS = {
    "uot_div": (uot.CDiv, ["kind", "lambda", "alpha", "beta"]),
    "uot_geom": (uot.CGeom, ["kind", "n", "m", "C", "ndim", "shape_x", "shape_y", "axes_x", "axes_y", "x", "y",
                             "d"]),
    "uot_opts": (uot.COpts, ["precision", "eps", "eps_start", "eps_stages", "iters_per_stage", "max_iter", "tol",
                             "check_every", "plain_scaling", "launch_mode", "U0", "V0", "out_f64", "verify",
                             "mixed_switch", "translate"]),
    "uot_result": (uot.CResult, ["iters", "total_iters", "marg_err", "ms", "status", "verifications",
                                 "polish_iters", "marg_err_fp32", "mixed_iters", "precise_iters"]),
    "uot_batch_problem": (uot.CBatchProblem, ["n", "m", "F1", "F2"]),
}


def test_struct_layouts_match_header(tmp_path):
    """sizeof and every field offset of the ctypes mirrors equal what the C
    compiler lays out from include/uot.h."""
    lines = ["#include <stdio.h>", "#include <stddef.h>", '#include "uot.h"', "int main(void) {"]
    for name, (_, fields) in C_FIELDS.items():
        lines.append(f'  printf("{name} %zu", sizeof({name}));')
        for f in fields:
            lines.append(f'  printf(" %zu", offsetof({name}, {f}));')
        lines.append('  printf("\\n");')
    lines.append("  return 0;\n}")
    src = tmp_path / "layout.c"
    src.write_text("\n".join(lines))
    exe = tmp_path / "layout"
    subprocess.run(["gcc", "-std=c11", "-I", os.path.join(ROOT, "include"), str(src), "-o", str(exe)], check=True)
    out = subprocess.run([str(exe)], check=True, capture_output=True, text=True).stdout.split("\n")
    got = {ln.split()[0]: [int(v) for v in ln.split()[1:]] for ln in out if ln.strip()}
    for name, (cls, fields) in C_FIELDS.items():
        assert len(cls._fields_) == len(fields), name
        want = [ctypes.sizeof(cls)] + [getattr(cls, f[0]).offset for f in cls._fields_]
        assert got[name] == want, (name, got[name], want)


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

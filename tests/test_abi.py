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


def _grid_geom(shape_x, shape_y):
    """A grid geometry whose axis pointers are placeholders: every call below
    is refused by the host-side checks before any pointer is used."""
    g = uot.CGeom()
    g.kind, g.ndim = uot.GEOM_GRID, len(shape_x)
    g.n, g.m = 1, 1
    for k, (a, b) in enumerate(zip(shape_x, shape_y)):
        g.shape_x[k], g.shape_y[k] = a, b
        g.axes_x[k] = g.axes_y[k] = _PLACEHOLDER
        g.n, g.m = g.n * a, g.m * b
    return g


_PLACEHOLDER = 1 << 12  # never dereferenced: the calls return before any use


def test_host_checks_refuse_before_any_launch():
    """Argument checks run on the host before the library touches a pointer,
    allocates or launches (so this runs without a GPU): grid passes over more
    than 65535 lines (the launch grid's second dimension) and axes over 3000
    points are UOT_EUNSUPPORTED with a message; an empty axis and eps <= 0 are
    UOT_EINVAL.  Every entry point resets the message when it starts, so a
    refusal without a message does not show the previous call's."""
    lib = uot.load()
    P = ctypes.c_void_p(_PLACEHOLDER)

    def gibbs(g, eps=0.1, prec=uot.F64):
        return uot.STATUS[lib.uot_gibbs_log(ctypes.byref(g), P, P, eps, 0, prec, P, None)]

    def solve(g):
        o = uot.COpts(precision=uot.F64, eps=0.1, max_iter=10, check_every=1)
        F = uot.CDiv(uot.DIV_KL, 1.0, 0.0, 0.0)
        r = uot.CResult()
        return uot.STATUS[lib.uot_solve(ctypes.byref(g), P, P, P, P, ctypes.byref(F), ctypes.byref(F),
                                        ctypes.byref(o), P, P, ctypes.byref(r), None)]

    over = _grid_geom((2, 256, 256), (2, 256, 256))  # the pass along axis 0 covers 256 * 256 lines
    for call in (gibbs, solve):
        assert call(over) == "UOT_EUNSUPPORTED"
        assert b"65535 lines" in lib.uot_last_error()
    long_axis = _grid_geom((3001,), (4,))
    assert gibbs(long_axis, prec=uot.F32) == "UOT_EUNSUPPORTED"
    assert b"3000 points" in lib.uot_last_error()
    assert gibbs(_grid_geom((0, 4), (4, 4))) == "UOT_EINVAL"
    assert lib.uot_last_error() == b""
    assert gibbs(_grid_geom((4, 4), (4, 4)), eps=0.0) == "UOT_EINVAL"
    assert lib.uot_last_error() == b""
    # the pass into Y along its last axis covers X's first two axes: 300 * 300
    # lines, although Y's own axes give at most 300
    assert gibbs(_grid_geom((300, 300, 1), (1, 1, 300))) == "UOT_EUNSUPPORTED"

"""Thin ctypes binding of the C ABI in include/uot.h (argument marshalling only).

Every function takes torch tensors that already live on the GPU, checks their
dtype/device/contiguity, and passes raw device pointers and the current CUDA
stream to libuot.so.  All computation happens in the library's kernels; there
is no CPU path.  If the library is missing or cannot be loaded the functions
raise instead of falling back.

Names follow the C ABI: solve, gibbs_log, apply_plan, objective, barycenter.
Divergences (Sec. 2.1, Table 1): EQ(), KL(lam), TV(lam), RG(alpha, beta).
"""
from __future__ import annotations

import ctypes as C
import math
import os
from dataclasses import dataclass

import numpy as np
import torch

from . import build as _build

UOT_OK, UOT_NOT_CONVERGED = 0, 1
STATUS = {0: "UOT_OK", 1: "UOT_NOT_CONVERGED", -1: "UOT_EINVAL", -2: "UOT_ENOMEM",
          -3: "UOT_NUMERICAL", -4: "UOT_TIMEOUT", -5: "UOT_ECUDA", -6: "UOT_EUNSUPPORTED"}
DIV_EQ, DIV_KL, DIV_TV, DIV_RG = 0, 1, 2, 3
GEOM_DENSE, GEOM_GRID, GEOM_POINTS = 0, 1, 2
F64, F32, MIXED = 0, 1, 2
BARY_EQ, BARY_KL, BARY_TV, BARY_RG = 0, 1, 2, 3
MAX_DIM = 3


class UotError(RuntimeError):
    def __init__(self, status, what=""):
        self.status = status
        super().__init__(f"{what}: {STATUS.get(status, status)} {_last_error()}".strip())


class CDiv(C.Structure):
    _fields_ = [("kind", C.c_int), ("lam", C.c_double), ("alpha", C.c_double), ("beta", C.c_double)]


class CGeom(C.Structure):
    _fields_ = [("kind", C.c_int), ("n", C.c_int), ("m", C.c_int), ("C", C.c_void_p),
                ("ndim", C.c_int), ("shape_x", C.c_int * MAX_DIM), ("shape_y", C.c_int * MAX_DIM),
                ("axes_x", C.c_void_p * MAX_DIM), ("axes_y", C.c_void_p * MAX_DIM),
                ("x", C.c_void_p), ("y", C.c_void_p), ("d", C.c_int)]


class COpts(C.Structure):
    _fields_ = [("precision", C.c_int), ("eps", C.c_double), ("eps_start", C.c_double),
                ("eps_stages", C.c_int), ("iters_per_stage", C.c_int), ("max_iter", C.c_int),
                ("tol", C.c_double), ("check_every", C.c_int), ("plain_scaling", C.c_int),
                ("launch_mode", C.c_int), ("U0", C.c_void_p), ("V0", C.c_void_p),
                ("out_f64", C.c_int), ("verify", C.c_int), ("mixed_switch", C.c_double),
                ("translate", C.c_int)]


class CBatchProblem(C.Structure):
    _fields_ = [("n", C.c_int), ("m", C.c_int), ("F1", CDiv), ("F2", CDiv)]


class CResult(C.Structure):
    _fields_ = [("iters", C.c_int), ("total_iters", C.c_int), ("marg_err", C.c_double),
                ("ms", C.c_double), ("status", C.c_int), ("verifications", C.c_int),
                ("polish_iters", C.c_int), ("marg_err_fp32", C.c_double), ("mixed_iters", C.c_int),
                ("precise_iters", C.c_int)]


_LIB = None

_SIGS = {
    "uot_version": (C.c_char_p, []),
    "uot_last_error": (C.c_char_p, []),
    "uot_launch_count": (C.c_longlong, []),
    "uot_profile_begin": (None, []),
    "uot_profile_end": (C.c_int, [C.c_int, C.POINTER(C.c_double), C.POINTER(C.c_longlong)]),
    "uot_solve": (C.c_int, [C.POINTER(CGeom), C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p,
                            C.POINTER(CDiv), C.POINTER(CDiv), C.POINTER(COpts), C.c_void_p,
                            C.c_void_p, C.POINTER(CResult), C.c_void_p]),
    "uot_solve_many": (C.c_int, [C.POINTER(CGeom), C.c_int, C.c_void_p, C.c_void_p, C.c_void_p,
                                 C.c_void_p, C.POINTER(CDiv), C.POINTER(CDiv), C.POINTER(COpts),
                                 C.c_void_p, C.c_void_p, C.POINTER(CResult), C.c_void_p]),
    "uot_solve_mass": (C.c_int, [C.POINTER(CGeom), C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p,
                                 C.POINTER(CDiv), C.POINTER(CDiv), C.POINTER(CDiv), C.c_double,
                                 C.POINTER(COpts), C.c_void_p, C.c_void_p, C.POINTER(C.c_double),
                                 C.POINTER(CResult), C.c_void_p]),
    "uot_wf_cost": (C.c_int, [C.c_void_p, C.c_int, C.c_void_p, C.c_int, C.c_int, C.c_double, C.c_int,
                              C.c_void_p, C.c_void_p]),
    "uot_wf_flow": (C.c_int, [C.POINTER(CGeom), C.c_int, C.c_void_p, C.c_void_p, C.c_double, C.c_double,
                              C.c_double, C.POINTER(COpts), C.c_int, C.c_void_p, C.c_void_p, C.c_void_p,
                              C.POINTER(CResult), C.c_void_p]),
    "uot_histogram": (C.c_int, [C.c_void_p, C.c_longlong, C.c_int, C.POINTER(C.c_int), C.c_int, C.c_void_p,
                                C.c_void_p]),
    "uot_barycentric_map": (C.c_int, [C.POINTER(CGeom), C.c_void_p, C.c_void_p, C.c_double, C.c_void_p,
                                      C.c_void_p, C.c_int, C.c_void_p, C.c_void_p]),
    "uot_apply_bin_map": (C.c_int, [C.c_void_p, C.c_longlong, C.c_int, C.POINTER(C.c_int), C.c_void_p, C.c_int,
                                    C.c_void_p, C.c_void_p]),
    "uot_gibbs_log": (C.c_int, [C.POINTER(CGeom), C.c_void_p, C.c_void_p, C.c_double, C.c_int,
                                C.c_int, C.c_void_p, C.c_void_p]),
    "uot_gibbs_log_noalloc": (C.c_int, [C.POINTER(CGeom), C.c_void_p, C.c_void_p, C.c_double,
                                        C.c_int, C.c_int, C.c_void_p, C.c_void_p]),
    "uot_apply_plan": (C.c_int, [C.POINTER(CGeom), C.c_void_p, C.c_void_p, C.c_double, C.c_void_p,
                                 C.c_void_p, C.c_void_p, C.c_int, C.c_int, C.c_int, C.c_void_p,
                                 C.c_void_p]),
    "uot_objective": (C.c_int, [C.POINTER(CGeom), C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p,
                                C.POINTER(CDiv), C.POINTER(CDiv), C.c_double, C.c_void_p,
                                C.c_void_p, C.c_int, C.POINTER(C.c_double), C.c_void_p]),
    "uot_solve_batch": (C.c_int, [C.c_int, C.POINTER(CBatchProblem), C.c_int, C.c_void_p,
                                  C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p,
                                  C.POINTER(COpts), C.c_void_p, C.c_void_p, C.POINTER(C.c_int),
                                  C.POINTER(C.c_double), C.POINTER(CResult), C.c_void_p]),
    "uot_conv2d_forward": (C.c_int, [C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p, C.c_int,
                                     C.c_int, C.c_int, C.c_int, C.c_int, C.c_int, C.c_int,
                                     C.c_void_p]),
    "uot_conv2d_backward": (C.c_int, [C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p,
                                      C.c_void_p, C.c_void_p, C.c_int, C.c_int, C.c_int, C.c_int,
                                      C.c_int, C.c_int, C.c_int, C.c_void_p]),
    "uot_adam_step": (C.c_int, [C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p, C.c_longlong,
                                C.c_float, C.c_float, C.c_float, C.c_float, C.c_int, C.c_void_p]),
    "uot_mse_grad": (C.c_int, [C.c_void_p, C.c_void_p, C.c_void_p, C.c_longlong, C.c_void_p,
                               C.c_void_p]),
    "uot_scale_instances": (C.c_int, [C.c_void_p, C.c_void_p, C.c_int, C.c_longlong, C.c_void_p]),
    "uot_warmstart_features": (C.c_int, [C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p,
                                         C.c_void_p, C.c_int, C.c_int, C.c_int, C.c_void_p]),
    "uot_conv_tc_forward": (C.c_int, [C.c_void_p, C.c_int, C.c_void_p, C.c_int, C.c_int, C.c_int, C.c_int,
                                      C.c_int, C.c_int, C.c_int, C.c_int, C.c_void_p, C.c_void_p, C.c_int,
                                      C.c_void_p, C.c_int, C.c_void_p, C.c_void_p, C.c_void_p]),
    "uot_conv_tc_wgrad": (C.c_int, [C.c_void_p, C.c_int, C.c_void_p, C.c_int, C.c_int, C.c_int, C.c_int, C.c_int,
                                    C.c_int, C.c_int, C.c_void_p, C.c_int, C.c_void_p, C.c_void_p, C.c_void_p]),
    "uot_nhwc_shift_transpose": (C.c_int, [C.c_void_p, C.c_int, C.c_int, C.c_int, C.c_int, C.c_int, C.c_void_p,
                                           C.c_void_p]),
    "uot_nhwc_transpose": (C.c_int, [C.c_void_p, C.c_longlong, C.c_int, C.c_void_p, C.c_void_p]),
    "uot_bias_grad_bf16": (C.c_int, [C.c_void_p, C.c_longlong, C.c_int, C.c_int, C.c_void_p, C.c_void_p]),
    "uot_conv_weights_bf16": (C.c_int, [C.c_void_p, C.c_int, C.c_int, C.c_int, C.c_int, C.c_int, C.c_int,
                                        C.c_void_p, C.c_void_p, C.c_void_p]),
    "uot_warmstart_features_nhwc": (C.c_int, [C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p,
                                              C.c_int, C.c_int, C.c_int, C.c_void_p]),
    "uot_mse_grad_nhwc": (C.c_int, [C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p, C.c_int, C.c_int,
                                    C.c_void_p, C.c_void_p, C.c_void_p]),
    "uot_pred_to_potentials": (C.c_int, [C.c_void_p, C.c_void_p, C.c_int, C.c_int, C.c_void_p, C.c_void_p,
                                         C.c_void_p]),
    "uot_set_autotune": (C.c_int, [C.c_int]),
    "uot_force_grid_tile": (C.c_int, [C.c_int]),
    "uot_grid_tile_count": (C.c_int, []),
    "uot_force_batch_warps": (C.c_int, [C.c_int]),
    "uot_selftest_bounded_wait": (C.c_int, [C.c_double, C.c_void_p]),
    "uot_probe_pipes": (C.c_int, [C.POINTER(C.c_double), C.c_void_p]),
    "uot_force_precise_passes": (C.c_int, [C.c_int]),
    "uot_fuse_short_passes": (C.c_int, [C.c_int]),
    "uot_autotune_table": (C.c_int, [C.c_char_p, C.c_int]),
    "uot_barycenter_div": (C.c_int, [C.POINTER(CGeom), C.c_int, C.POINTER(C.c_double), C.c_void_p,
                                     C.c_void_p, C.c_void_p, C.POINTER(CDiv), C.POINTER(CDiv),
                                     C.POINTER(COpts), C.c_void_p, C.c_void_p, C.c_void_p,
                                     C.POINTER(CResult), C.c_void_p]),
    "uot_barycenter": (C.c_int, [C.POINTER(CGeom), C.c_int, C.POINTER(C.c_double), C.c_void_p,
                                 C.c_void_p, C.c_void_p, C.POINTER(CDiv), C.c_double, C.c_int,
                                 C.POINTER(COpts), C.c_void_p, C.c_void_p, C.c_void_p,
                                 C.POINTER(CResult), C.c_void_p]),
}


def exported_symbols():
    """Entry points declared in include/uot.h."""
    return list(_SIGS)


def lib_path() -> str:
    return _build.LIB


def load(path: str | None = None):
    """Load libuot.so (building it if absent) and bind the C signatures."""
    global _LIB
    if _LIB is not None:
        return _LIB
    path = path or lib_path()
    if not os.path.exists(path):
        _build.build()
    lib = C.CDLL(path)
    for name, (res, args) in _SIGS.items():
        f = getattr(lib, name)
        f.restype = res
        f.argtypes = args
    _LIB = lib
    return lib


def _last_error() -> str:
    if _LIB is None:
        return ""
    return _LIB.uot_last_error().decode()


def version() -> str:
    return load().uot_version().decode()


def launch_count() -> int:
    """Kernels launched by the library so far in this process."""
    return int(load().uot_launch_count())


def set_autotune(mode: int) -> int:
    """Grid-pass tile tuner on (1) or off (0); returns the previous mode."""
    return int(load().uot_set_autotune(int(mode)))


def force_precise_passes(on: bool) -> bool:
    """uot_force_precise_passes: every FP32 grid pass forms its exponents in
    float-float (on) or the usual tiles run (off); returns the previous setting."""
    return bool(load().uot_force_precise_passes(int(bool(on))))


def fuse_short_passes(on: bool) -> bool:
    """uot_fuse_short_passes: consecutive FP32 grid passes over axes of at most
    64 points run as one launch per plane (on) or as separate passes (off, the
    default); returns the previous setting."""
    return bool(load().uot_fuse_short_passes(int(bool(on))))


def force_grid_tile(idx: int):
    """Use FP32 grid-pass tile idx for every pass (-1: back to the tuned choice)."""
    _check(load().uot_force_grid_tile(int(idx)), "uot_force_grid_tile")


def force_batch_warps(warps: int):
    """CTA size of solve_batch: 8 or 16 warps, 0 = the tuner's choice."""
    _check(load().uot_force_batch_warps(int(warps)), "uot_force_batch_warps")


def selftest_bounded_wait(seconds: float) -> str:
    """Status name of the bounded-wait self-test ("UOT_TIMEOUT" when the
    device wait on a never-set flag expired as designed)."""
    st = load().uot_selftest_bounded_wait(float(seconds), _stream())
    if st < 0 and STATUS.get(st) != "UOT_TIMEOUT":
        _check(st, "uot_selftest_bounded_wait")
    return STATUS[st]


def probe_pipes() -> dict:
    """uot_probe_pipes: sustained FP32 FMA, MUFU ex2, FP64 FMA and FP64 exp()
    rates in operations per clock per SM."""
    lib = load()
    out = (C.c_double * 4)()
    _check(lib.uot_probe_pipes(out, _stream()), "uot_probe_pipes")
    return {"ffma_per_clk_per_sm": out[0], "mufu_ex2_per_clk_per_sm": out[1], "dfma_per_clk_per_sm": out[2],
            "dexp_per_clk_per_sm": out[3]}


def grid_tile_count() -> int:
    return int(load().uot_grid_tile_count())


def autotune_table() -> str:
    """Tuned pass shapes, chosen tiles and measured times (text)."""
    lib = load()
    n = lib.uot_autotune_table(None, 0)
    buf = C.create_string_buffer(n + 1)
    lib.uot_autotune_table(buf, n + 1)
    return buf.value.decode()


PROF_GRID_PASS, PROF_ROWS, PROF_GRID_BLK = 0, 1, 2


def profile_begin():
    load().uot_profile_begin()


def profile_end(family=PROF_GRID_PASS):
    """(total ms, launches) of one kernel family since profile_begin()."""
    ms = C.c_double()
    n = C.c_longlong()
    _check(load().uot_profile_end(int(family), C.byref(ms), C.byref(n)), "uot_profile_end")
    return ms.value, n.value


# ---------------------------------------------------------------------------
# argument helpers
# ---------------------------------------------------------------------------


@dataclass
class Div:
    kind: int
    lam: float = 1.0
    alpha: float = 0.0
    beta: float = math.inf

    def c(self) -> CDiv:
        return CDiv(self.kind, float(self.lam), float(self.alpha), float(self.beta))


def EQ():
    return Div(DIV_EQ)


def KL(lam):
    return Div(DIV_KL, lam=lam)


def TV(lam):
    return Div(DIV_TV, lam=lam)


def RG(alpha, beta):
    return Div(DIV_RG, alpha=alpha, beta=beta)


def _dtype(prec):
    return torch.float64 if prec == F64 else torch.float32


def _ptr(t: torch.Tensor | None, dtype=None, what="tensor"):
    if t is None:
        return None
    if not isinstance(t, torch.Tensor) or not t.is_cuda:
        raise TypeError(f"{what} must be a CUDA tensor")
    if dtype is not None and t.dtype != dtype:
        raise TypeError(f"{what} must be {dtype}, got {t.dtype}")
    if not t.is_contiguous():
        raise ValueError(f"{what} must be contiguous")
    return t.data_ptr()


def _stream():
    return C.c_void_p(torch.cuda.current_stream().cuda_stream)


@dataclass
class Geometry:
    """Device-side geometry; tensors must outlive the calls that use it."""
    kind: int
    n: int
    m: int
    C: torch.Tensor | None = None
    axes_x: tuple = ()
    axes_y: tuple = ()
    x: torch.Tensor | None = None
    y: torch.Tensor | None = None

    @staticmethod
    def dense(C):
        return Geometry(GEOM_DENSE, C.shape[0], C.shape[1], C=C.contiguous())

    @staticmethod
    def grid(axes_x, axes_y=None):
        axes_y = axes_x if axes_y is None else axes_y
        n = math.prod(a.numel() for a in axes_x)
        m = math.prod(a.numel() for a in axes_y)
        return Geometry(GEOM_GRID, n, m, axes_x=tuple(a.contiguous() for a in axes_x),
                        axes_y=tuple(a.contiguous() for a in axes_y))

    @staticmethod
    def points(x, y):
        return Geometry(GEOM_POINTS, x.shape[0], y.shape[0], x=x.contiguous(), y=y.contiguous())

    @property
    def shape_x(self):
        return tuple(a.numel() for a in self.axes_x) if self.kind == GEOM_GRID else (self.n,)

    @property
    def shape_y(self):
        return tuple(a.numel() for a in self.axes_y) if self.kind == GEOM_GRID else (self.m,)

    def c(self, prec) -> CGeom:
        dt = _dtype(prec)
        g = CGeom()
        g.kind, g.n, g.m = self.kind, self.n, self.m
        if self.kind == GEOM_DENSE:
            g.C = _ptr(self.C, dt, "C")
        elif self.kind == GEOM_POINTS:
            g.x = _ptr(self.x, dt, "x")
            g.y = _ptr(self.y, dt, "y")
            g.d = self.x.shape[1]
            if self.y.shape[1] != g.d:
                raise ValueError("x and y must have the same dimension")
        else:
            if len(self.axes_x) != len(self.axes_y) or not 1 <= len(self.axes_x) <= MAX_DIM:
                raise ValueError("grid axes")
            g.ndim = len(self.axes_x)
            for k, (ax, ay) in enumerate(zip(self.axes_x, self.axes_y)):
                g.shape_x[k], g.shape_y[k] = ax.numel(), ay.numel()
                g.axes_x[k] = _ptr(ax, dt, "axis")
                g.axes_y[k] = _ptr(ay, dt, "axis")
        return g


def _info(r: "CResult", st: int) -> dict:
    return dict(iters=r.iters, total_iters=r.total_iters, marg_err=r.marg_err, ms=r.ms,
                status=STATUS[st], verifications=r.verifications, polish_iters=r.polish_iters,
                marg_err_fp32=r.marg_err_fp32, mixed_iters=r.mixed_iters, precise_iters=r.precise_iters)


def _check(status, what):
    if status < 0:
        raise UotError(status, what)
    return status


def solve(geom: Geometry, p, dx, q, dy, F1: Div, F2: Div, eps: float, *, precision=F64,
          max_iter=1000, tol=0.0, check_every=10, eps_start=None, eps_stages=10,
          iters_per_stage=100, plain_scaling=False, U0=None, V0=None, U=None, V=None,
          launch_mode=0, out_f64=False, verify=False, mixed_switch=0.0, translate=False):
    """uot_solve: returns (U, V, result dict).  Inputs are CUDA tensors of the
    precision's dtype; U, V (optional) are preallocated outputs (float64 when
    out_f64).  verify: the stop is confirmed by an FP64 evaluation of the
    violation (FP32 / mixed paths).  translate (KL on both sides): the dual's
    exact maximum along (U + c, V - c) after every checked iteration."""
    lib = load()
    dt = _dtype(precision)
    odt = torch.float64 if out_f64 else dt
    U = torch.empty(geom.n, dtype=odt, device=p.device) if U is None else U
    V = torch.empty(geom.m, dtype=odt, device=p.device) if V is None else V
    o = COpts(precision, float(eps), float(eps_start) if eps_start else 0.0, int(eps_stages),
              int(iters_per_stage), int(max_iter), float(tol), int(check_every),
              int(bool(plain_scaling)), int(launch_mode), _ptr(U0, dt, "U0"), _ptr(V0, dt, "V0"),
              int(bool(out_f64)), int(bool(verify)), float(mixed_switch), int(bool(translate)))
    r = CResult()
    g = geom.c(precision)
    st = lib.uot_solve(C.byref(g), _ptr(p, dt, "p"), _ptr(dx, dt, "dx"), _ptr(q, dt, "q"),
                       _ptr(dy, dt, "dy"), C.byref(F1.c()), C.byref(F2.c()), C.byref(o),
                       _ptr(U, odt, "U"), _ptr(V, odt, "V"), C.byref(r), _stream())
    _check(st, "uot_solve")
    return U, V, _info(r, st)


def solve_mass(geom: Geometry, p, dx, q, dy, F1: Div, F2: Div, F3: Div, m0: float, eps: float, *,
               precision=F64, max_iter=1000, tol=0.0, check_every=10, eps_start=None, eps_stages=10,
               iters_per_stage=100, U0=None, V0=None, U=None, V=None, launch_mode=0):
    """uot_solve_mass (Algorithm 4, a divergence F3(. | m0) on the plan's total
    mass): returns (U, V, Z, result dict); the plan is e^{(U_i + V_j + Z - C_ij)/eps}."""
    lib = load()
    dt = _dtype(precision)
    U = torch.empty(geom.n, dtype=dt, device=p.device) if U is None else U
    V = torch.empty(geom.m, dtype=dt, device=p.device) if V is None else V
    o = COpts(precision, float(eps), float(eps_start) if eps_start else 0.0, int(eps_stages),
              int(iters_per_stage), int(max_iter), float(tol), int(check_every), 0,
              int(launch_mode), _ptr(U0, dt, "U0"), _ptr(V0, dt, "V0"))
    r = CResult()
    Z = C.c_double(0.0)
    g = geom.c(precision)
    st = lib.uot_solve_mass(C.byref(g), _ptr(p, dt, "p"), _ptr(dx, dt, "dx"), _ptr(q, dt, "q"),
                            _ptr(dy, dt, "dy"), C.byref(F1.c()), C.byref(F2.c()), C.byref(F3.c()),
                            float(m0), C.byref(o), _ptr(U, dt, "U"), _ptr(V, dt, "V"), C.byref(Z),
                            C.byref(r), _stream())
    _check(st, "uot_solve_mass")
    return U, V, Z.value, dict(iters=r.iters, total_iters=r.total_iters, marg_err=r.marg_err,
                               ms=r.ms, status=STATUS[st])


def wf_cost(x, y, cut, precision=F64, out=None):
    """uot_wf_cost: the WF cost matrix -log cos^2((pi/2)|x - y|/cut), +inf beyond
    the cut locus; x [n] or [n, d], y [m] or [m, d] on the GPU.  Returns C [n, m]."""
    lib = load()
    dt = _dtype(precision)
    x2 = x.reshape(x.shape[0], -1)
    y2 = y.reshape(y.shape[0], -1)
    n, d = x2.shape
    m = y2.shape[0]
    out = torch.empty(n, m, dtype=dt, device=x.device) if out is None else out
    _check(lib.uot_wf_cost(_ptr(x2, dt, "x"), n, _ptr(y2, dt, "y"), m, d, float(cut), precision,
                           _ptr(out, dt, "C"), _stream()), "uot_wf_cost")
    return out


def wf_flow(geom: Geometry, P0, dx, tau, alpha, lam, eps, nsteps, *, precision=F64, iters=500,
            eps_start=None, eps_stages=10, iters_per_stage=100, launch_mode=2):
    """uot_wf_flow: WF gradient flow with growth, P0 [S, n] initial densities.
    Returns (P [nsteps, S, n], U [S, n], V [S, n], info)."""
    lib = load()
    dt = _dtype(precision)
    P0 = P0.reshape(-1, geom.n)
    S = P0.shape[0]
    P = torch.empty(nsteps, S, geom.n, dtype=dt, device=P0.device)
    U = torch.empty(S, geom.n, dtype=dt, device=P0.device)
    V = torch.empty(S, geom.n, dtype=dt, device=P0.device)
    o = COpts(precision, float(eps), float(eps_start) if eps_start else 0.0, int(eps_stages),
              int(iters_per_stage), int(iters), 0.0, 1, 0, int(launch_mode), None, None)
    r = CResult()
    g = geom.c(precision)
    st = lib.uot_wf_flow(C.byref(g), S, _ptr(P0, dt, "P0"), _ptr(dx, dt, "dx"), float(tau), float(alpha),
                         float(lam), C.byref(o), int(nsteps), _ptr(P, dt, "P"), _ptr(U, dt, "U"),
                         _ptr(V, dt, "V"), C.byref(r), _stream())
    _check(st, "uot_wf_flow")
    return P, U, V, dict(iters=r.iters, total_iters=r.total_iters, ms=r.ms, status=STATUS[st])


def histogram(pts, shape, precision=F64, out=None):
    """uot_histogram: fraction of the points pts [N, d] (float32, in [0, 1]^d)
    in each bin of the regular grid `shape` (row-major), as a flat tensor."""
    lib = load()
    dt = _dtype(precision)
    d = len(shape)
    pts = pts.reshape(-1, d)
    out = torch.empty(int(np.prod(shape)), dtype=dt, device=pts.device) if out is None else out
    sh = (C.c_int * d)(*[int(v) for v in shape])
    _check(lib.uot_histogram(_ptr(pts, torch.float32, "pts"), pts.shape[0], d, sh, precision,
                             _ptr(out, dt, "p"), _stream()), "uot_histogram")
    return out


def barycentric_map(geom: Geometry, U, V, eps, dx, dy, precision=F64, out=None):
    """uot_barycentric_map: T [n, dim], T_i = sum_j R_ij dy_j y_j / sum_j R_ij dy_j."""
    lib = load()
    dt = _dtype(precision)
    dim = len(geom.axes_x) if geom.kind == GEOM_GRID else geom.x.shape[1]
    out = torch.empty(geom.n, dim, dtype=dt, device=U.device) if out is None else out
    g = geom.c(precision)
    _check(lib.uot_barycentric_map(C.byref(g), _ptr(U, dt, "U"), _ptr(V, dt, "V"), float(eps), _ptr(dx, dt, "dx"),
                                   _ptr(dy, dt, "dy"), precision, _ptr(out, dt, "T"), _stream()),
           "uot_barycentric_map")
    return out


def apply_bin_map(pts, shape, T, precision=F64, out=None):
    """uot_apply_bin_map: every point of pts [N, d] takes the value of T at its bin."""
    lib = load()
    dt = _dtype(precision)
    d = len(shape)
    pts = pts.reshape(-1, d)
    out = torch.empty(pts.shape[0], d, dtype=torch.float32, device=pts.device) if out is None else out
    sh = (C.c_int * d)(*[int(v) for v in shape])
    _check(lib.uot_apply_bin_map(_ptr(pts, torch.float32, "pts"), pts.shape[0], d, sh, _ptr(T, dt, "T"), precision,
                                 _ptr(out, torch.float32, "out"), _stream()), "uot_apply_bin_map")
    return out


def color_transfer(img_x, img_y, F2: Div, eps=0.002, iters=2000, bins=(64, 32, 32), precision=F32,
                   launch_mode=2, check_every=100):
    """Colour transfer of Sec. 5.1: the colours of img_y imposed on img_x
    (both [..., 3] float32 in [0, 1]^3): histograms on `bins`, the scaling
    iteration on the separable grid with F1 = EQ(p) and F2 w.r.t. q (unit
    reference mass per bin), the barycentric projection T, and T o g_X.
    Returns (new image shaped like img_x, T, info)."""
    dt = _dtype(precision)
    dev = img_x.device
    px = img_x.reshape(-1, len(bins)).contiguous()
    py = img_y.reshape(-1, len(bins)).contiguous()
    p = histogram(px, bins, precision)
    q = histogram(py, bins, precision)
    axes = [((torch.arange(n, dtype=torch.float64, device=dev) + 0.5) / n).to(dt) for n in bins]
    geo = Geometry.grid(axes, axes)
    ones = torch.ones(p.numel(), dtype=dt, device=dev)
    U, V, info = solve(geo, p, ones, q, ones, EQ(), F2, eps, precision=precision, max_iter=iters,
                       check_every=check_every, launch_mode=launch_mode)
    T = barycentric_map(geo, U, V, eps, ones, ones, precision)
    out = apply_bin_map(px, bins, T, precision)
    return out.reshape(img_x.shape), T, info


def solve_many(geom: Geometry, P, dx, Q, dy, F1: Div, F2: Div, eps, *, precision=F64,
               max_iter=1000, tol=0.0, check_every=10, eps_start=None, eps_stages=10,
               iters_per_stage=100, U0=None, V0=None, U=None, V=None, launch_mode=0,
               out_f64=False, verify=False, mixed_switch=0.0, translate=False):
    """uot_solve_many: P [B, n], Q [B, m] densities of B independent problems
    sharing geometry, weights, eps and penalties.  Returns (U [B,n], V [B,m], info)."""
    lib = load()
    dt = _dtype(precision)
    odt = torch.float64 if out_f64 else dt
    B = P.shape[0]
    U = torch.empty(B, geom.n, dtype=odt, device=P.device) if U is None else U
    V = torch.empty(B, geom.m, dtype=odt, device=P.device) if V is None else V
    o = COpts(precision, float(eps), float(eps_start) if eps_start else 0.0, int(eps_stages),
              int(iters_per_stage), int(max_iter), float(tol), int(check_every), 0, int(launch_mode),
              _ptr(U0, dt, "U0"), _ptr(V0, dt, "V0"), int(bool(out_f64)), int(bool(verify)),
              float(mixed_switch), int(bool(translate)))
    r = CResult()
    g = geom.c(precision)
    st = lib.uot_solve_many(C.byref(g), int(B), _ptr(P, dt, "P"), _ptr(dx, dt, "dx"),
                            _ptr(Q, dt, "Q"), _ptr(dy, dt, "dy"), C.byref(F1.c()), C.byref(F2.c()),
                            C.byref(o), _ptr(U, odt, "U"), _ptr(V, odt, "V"), C.byref(r), _stream())
    _check(st, "uot_solve_many")
    return U, V, _info(r, st)


def gibbs_log(geom: Geometry, W, w, eps, transpose=False, precision=F64, out=None):
    """uot_gibbs_log: eps log K(e^{W/eps} . w) (or with K^T)."""
    lib = load()
    dt = _dtype(precision)
    nout = geom.m if transpose else geom.n
    out = torch.empty(nout, dtype=dt, device=W.device) if out is None else out
    g = geom.c(precision)
    _check(lib.uot_gibbs_log(C.byref(g), _ptr(W, dt, "W"), _ptr(w, dt, "w"), float(eps),
                             int(bool(transpose)), precision, _ptr(out, dt, "out"), _stream()),
           "uot_gibbs_log")
    return out


def gibbs_log_noalloc(geom: Geometry, W, w, eps, transpose=False, precision=F64, out=None):
    """uot_gibbs_log_noalloc: same result as gibbs_log, computed with the
    library's fixed scratch array instead of device allocations (for callers
    that cannot allocate; see include/uot.h).  `out` may be preallocated."""
    lib = load()
    dt = _dtype(precision)
    nout = geom.m if transpose else geom.n
    out = torch.empty(nout, dtype=dt, device=W.device) if out is None else out
    g = geom.c(precision)
    _check(lib.uot_gibbs_log_noalloc(C.byref(g), _ptr(W, dt, "W"), _ptr(w, dt, "w"), float(eps),
                                     int(bool(transpose)), precision, _ptr(out, dt, "out"),
                                     _stream()), "uot_gibbs_log_noalloc")
    return out


def apply_plan(geom: Geometry, U, V, eps, dx, dy, f=None, transpose=False, precision=F64, out=None):
    """uot_apply_plan: R f (or R^T f) for nonnegative f of shape [m, ncols] ([n, ncols])."""
    lib = load()
    dt = _dtype(precision)
    nout = geom.m if transpose else geom.n
    ncols = 1 if f is None else (f.shape[1] if f.dim() == 2 else 1)
    out = torch.empty(nout, ncols, dtype=dt, device=U.device) if out is None else out
    g = geom.c(precision)
    _check(lib.uot_apply_plan(C.byref(g), _ptr(U, dt, "U"), _ptr(V, dt, "V"), float(eps),
                              _ptr(dx, dt, "dx"), _ptr(dy, dt, "dy"), _ptr(f, dt, "f"), ncols,
                              int(bool(transpose)), precision, _ptr(out, dt, "out"), _stream()),
           "uot_apply_plan")
    return out


def objective(geom: Geometry, p, dx, q, dy, F1: Div, F2: Div, eps, U, V, precision=F64):
    """uot_objective: dict(primal, dual, gap, marg_err) in FP64."""
    lib = load()
    dt = _dtype(precision)
    out = (C.c_double * 4)()
    g = geom.c(precision)
    _check(lib.uot_objective(C.byref(g), _ptr(p, dt, "p"), _ptr(dx, dt, "dx"), _ptr(q, dt, "q"),
                             _ptr(dy, dt, "dy"), C.byref(F1.c()), C.byref(F2.c()), float(eps),
                             _ptr(U, dt, "U"), _ptr(V, dt, "V"), precision, out, _stream()),
           "uot_objective")
    return dict(primal=out[0], dual=out[1], gap=out[2], marg_err=out[3])


def barycenter(geom: Geometry, alpha, P, dx, dy, F1: Div, lam, eps, *, kind=BARY_KL,
               precision=F64, max_iter=1000, tol=0.0, check_every=10, eps_start=None,
               eps_stages=10, iters_per_stage=100, launch_mode=0):
    """uot_barycenter: returns (eps log h, U [K,n], V [K,m], result dict)."""
    lib = load()
    dt = _dtype(precision)
    K = P.shape[0]
    logh = torch.empty(geom.m, dtype=dt, device=P.device)
    U = torch.empty(K, geom.n, dtype=dt, device=P.device)
    V = torch.empty(K, geom.m, dtype=dt, device=P.device)
    a = (C.c_double * K)(*[float(v) for v in alpha])
    o = COpts(precision, float(eps), float(eps_start) if eps_start else 0.0, int(eps_stages),
              int(iters_per_stage), int(max_iter), float(tol), int(check_every), 0, int(launch_mode), None,
              None)
    r = CResult()
    g = geom.c(precision)
    st = lib.uot_barycenter(C.byref(g), K, a, _ptr(P, dt, "P"), _ptr(dx, dt, "dx"),
                            _ptr(dy, dt, "dy"), C.byref(F1.c()), float(lam), int(kind),
                            C.byref(o), _ptr(logh, dt, "logh"), _ptr(U, dt, "U"),
                            _ptr(V, dt, "V"), C.byref(r), _stream())
    _check(st, "uot_barycenter")
    return logh, U, V, dict(iters=r.iters, total_iters=r.total_iters, marg_err=r.marg_err,
                            ms=r.ms, status=STATUS[st])


def barycenter_div(geom: Geometry, alpha, P, dx, dy, F1: Div, Fh: Div, eps, *, precision=F64, max_iter=1000,
                   tol=0.0, check_every=10, eps_start=None, eps_stages=10, iters_per_stage=100, launch_mode=0):
    """uot_barycenter_div: the barycenter divergence as a Div (EQ, KL, TV or
    RG with 0 < alpha <= beta < inf); returns (eps log h, U [K,n], V [K,m], result dict)."""
    lib = load()
    dt = _dtype(precision)
    K = P.shape[0]
    logh = torch.empty(geom.m, dtype=dt, device=P.device)
    U = torch.empty(K, geom.n, dtype=dt, device=P.device)
    V = torch.empty(K, geom.m, dtype=dt, device=P.device)
    a = (C.c_double * K)(*[float(v) for v in alpha])
    o = COpts(precision, float(eps), float(eps_start) if eps_start else 0.0, int(eps_stages),
              int(iters_per_stage), int(max_iter), float(tol), int(check_every), 0, int(launch_mode), None,
              None)
    r = CResult()
    g = geom.c(precision)
    st = lib.uot_barycenter_div(C.byref(g), K, a, _ptr(P, dt, "P"), _ptr(dx, dt, "dx"), _ptr(dy, dt, "dy"),
                                C.byref(F1.c()), C.byref(Fh.c()), C.byref(o), _ptr(logh, dt, "logh"),
                                _ptr(U, dt, "U"), _ptr(V, dt, "V"), C.byref(r), _stream())
    _check(st, "uot_barycenter_div")
    return logh, U, V, dict(iters=r.iters, total_iters=r.total_iters, marg_err=r.marg_err,
                            ms=r.ms, status=STATUS[st])


def geodesic(geom: Geometry, p0, p1, ts, dx, dy, F1: Div, Fh: Div, eps, **kw):
    """Geodesic between two measures as weighted barycenters of the endpoints
    (Sec. 5.2, numerical experiments): for each t, uot_barycenter_div with
    K = 2 and weights (1 - t, t).  With the WF cost (uot_wf_cost) and KL(1) for
    F1 and Fh this is the WF geodesic; with |x - y|^2 and EQ, the Wasserstein
    one.  Returns eps log h for every t, [len(ts), m]."""
    P = torch.stack([p0.reshape(-1), p1.reshape(-1)])
    out = []
    for t in ts:
        logh, _, _, _ = barycenter_div(geom, [1.0 - float(t), float(t)], P, dx, dy, F1, Fh, eps, **kw)
        out.append(logh)
    return torch.stack(out)


def solve_batch(sizes, divs, d, x, p, dx, y, q, dy, eps, *, max_iter=1000, tol=0.0,
                check_every=10, eps_start=None, eps_stages=10, iters_per_stage=100, U=None, V=None,
                translate=False, out_f64=False):
    """uot_solve_batch (FP32): sizes = [(n_k, m_k)], divs = [(F1_k, F2_k)]; x, p, dx
    packed over the X sides ([sum n, d], [sum n], [sum n]) and y, q, dy over the
    Y sides.  translate (KL / KL problems): the translation step of
    uot_opts.translate, per problem.  Returns (U, V, iters [nprob], errs
    [nprob], result dict)."""
    lib = load()
    nprob = len(sizes)
    arr = (CBatchProblem * nprob)()
    for k, ((n, m), (F1, F2)) in enumerate(zip(sizes, divs)):
        arr[k] = CBatchProblem(int(n), int(m), F1.c(), F2.c())
    N = sum(n for n, _ in sizes)
    M = sum(m for _, m in sizes)
    dt = torch.float32
    odt = torch.float64 if out_f64 else dt
    U = torch.empty(N, dtype=odt, device=x.device) if U is None else U
    V = torch.empty(M, dtype=odt, device=x.device) if V is None else V
    iters = (C.c_int * nprob)()
    errs = (C.c_double * nprob)()
    o = COpts(F32, float(eps), float(eps_start) if eps_start else 0.0, int(eps_stages),
              int(iters_per_stage), int(max_iter), float(tol), int(check_every), 0, 0, None, None,
              int(bool(out_f64)), 0, 0.0, int(bool(translate)))
    r = CResult()
    st = lib.uot_solve_batch(nprob, arr, int(d), _ptr(x, dt, "x"), _ptr(p, dt, "p"),
                             _ptr(dx, dt, "dx"), _ptr(y, dt, "y"), _ptr(q, dt, "q"),
                             _ptr(dy, dt, "dy"), C.byref(o), _ptr(U, odt, "U"), _ptr(V, odt, "V"),
                             iters, errs, C.byref(r), _stream())
    _check(st, "uot_solve_batch")
    return U, V, list(iters), list(errs), dict(iters=r.iters, total_iters=r.total_iters,
                                               marg_err=r.marg_err, ms=r.ms, status=STATUS[st])


# ---------------------------------------------------------------------------
# learned warm start kernels
# ---------------------------------------------------------------------------

def conv2d_forward(x, w, b, dilation, leaky, out=None):
    """uot_conv2d_forward on [N, Cin, H, W] FP32 tensors."""
    N, Cin, H, W = x.shape
    Cout = w.shape[0]
    f = torch.float32
    out = torch.empty(N, Cout, H, W, dtype=f, device=x.device) if out is None else out
    _check(load().uot_conv2d_forward(_ptr(x, f, "x"), _ptr(w, f, "w"), _ptr(b, f, "b"),
                                     _ptr(out, f, "y"), N, Cin, Cout, H, W, int(dilation),
                                     int(bool(leaky)), _stream()), "uot_conv2d_forward")
    return out


def conv2d_backward(x, w, y, dy, dilation, leaky, need_dx=True):
    """uot_conv2d_backward: returns (dx or None, dw, db)."""
    N, Cin, H, W = x.shape
    Cout = w.shape[0]
    f = torch.float32
    dx = torch.empty_like(x) if need_dx else None
    dw = torch.empty_like(w)
    db = torch.empty(Cout, dtype=f, device=x.device)
    _check(load().uot_conv2d_backward(_ptr(x, f, "x"), _ptr(w, f, "w"), _ptr(y, f, "y"),
                                      _ptr(dy, f, "dy"), _ptr(dx, f, "dx") if need_dx else None,
                                      _ptr(dw, f, "dw"), _ptr(db, f, "db"), N, Cin, Cout, H, W,
                                      int(dilation), int(bool(leaky)), _stream()),
           "uot_conv2d_backward")
    return dx, dw, db


def adam_step(param, grad, m, v, lr, step, beta1=0.9, beta2=0.999, eps=1e-8):
    f = torch.float32
    _check(load().uot_adam_step(_ptr(param, f, "param"), _ptr(grad, f, "grad"), _ptr(m, f, "m"),
                                _ptr(v, f, "v"), param.numel(), float(lr), float(beta1),
                                float(beta2), float(eps), int(step), _stream()), "uot_adam_step")


def mse_grad(pred, target, grad, loss_dev):
    f = torch.float32
    _check(load().uot_mse_grad(_ptr(pred, f, "pred"), _ptr(target, f, "target"), _ptr(grad, f, "grad"),
                               pred.numel(), _ptr(loss_dev, torch.float64, "loss"), _stream()),
           "uot_mse_grad")


def scale_instances(x, scale):
    """In place: x[n] *= scale[n] (x [N, ...] FP32, scale [N] FP32)."""
    f = torch.float32
    _check(load().uot_scale_instances(_ptr(x, f, "x"), _ptr(scale, f, "scale"), x.shape[0],
                                      x.numel() // x.shape[0], _stream()), "uot_scale_instances")
    return x


def warmstart_features(P, Q, log_eps, log_lam, out=None):
    N, H, W = P.shape
    f = torch.float32
    out = torch.empty(N, 4, H, W, dtype=f, device=P.device) if out is None else out
    _check(load().uot_warmstart_features(_ptr(P, f, "p"), _ptr(Q, f, "q"), _ptr(log_eps, f, "log_eps"),
                                         _ptr(log_lam, f, "log_lam"), _ptr(out, f, "out"), N, H, W,
                                         _stream()), "uot_warmstart_features")
    return out


# ---- tensor-core convolutions of the warm-start network (BF16, NHWC) ----

BF16 = torch.bfloat16
CONV_IDENTITY, CONV_LEAKY, CONV_DACT = 0, 1, 2


def conv_tc_forward(x, wk, bn, N, H, W, cin_pad, nout, dil, mode, *, bias=None, ref=None, y=None, yf=None,
                    err=None):
    """uot_conv_tc_forward; x [N*H*W, ldx] BF16, wk [bn, 9, cin_pad] BF16, y [P, ldy] BF16 and/or
    yf [P, nout] FP32 (allocated here when neither is given: y with ldy = max(16, nout))."""
    P = N * H * W
    if y is None and yf is None:
        y = torch.empty(P, max(16, (nout + 15) // 16 * 16), dtype=BF16, device=x.device)
    _check(load().uot_conv_tc_forward(
        _ptr(x, BF16, "x"), x.shape[-1], _ptr(wk, BF16, "wk"), bn, N, H, W, cin_pad, nout, dil, mode,
        _ptr(bias, torch.float32, "bias"), _ptr(ref, BF16, "ref"), 0 if ref is None else ref.shape[-1],
        _ptr(y, BF16, "y"), 0 if y is None else y.shape[-1], _ptr(yf, torch.float32, "yf"),
        _ptr(err, torch.int32, "err"), _stream()), "uot_conv_tc_forward")
    return y if y is not None else yf


def conv_tc_wgrad(dyT, xT, cin_pad, N, H, W, dil, Cout, Cin, *, splits=64, part=None, dw=None, err=None):
    """uot_conv_tc_wgrad; dyT [rows, P] BF16, xT [3, cin_pad, P] BF16 -> dw [Cout, Cin, 3, 3] FP32."""
    dw = torch.empty(Cout, Cin, 3, 3, dtype=torch.float32, device=dyT.device) if dw is None else dw
    part = torch.empty(splits * 9 * 128 * cin_pad, dtype=torch.float32, device=dyT.device) if part is None else part
    _check(load().uot_conv_tc_wgrad(_ptr(dyT, BF16, "dyT"), dyT.shape[0], _ptr(xT, BF16, "xT"), cin_pad, N, H, W,
                                    dil, Cout, Cin, _ptr(part, torch.float32, "part"), splits,
                                    _ptr(dw, torch.float32, "dw"), _ptr(err, torch.int32, "err"), _stream()),
           "uot_conv_tc_wgrad")
    return dw


def nhwc_shift_transpose(x, N, H, W, dil, out=None):
    C = x.shape[-1]
    out = torch.empty(3, C, N * H * W, dtype=BF16, device=x.device) if out is None else out
    _check(load().uot_nhwc_shift_transpose(_ptr(x, BF16, "x"), N, H, W, C, dil, _ptr(out, BF16, "xT"), _stream()),
           "uot_nhwc_shift_transpose")
    return out


def nhwc_transpose(y, out=None):
    P, C = y.shape
    out = torch.empty(C, P, dtype=BF16, device=y.device) if out is None else out
    _check(load().uot_nhwc_transpose(_ptr(y, BF16, "y"), P, C, _ptr(out, BF16, "yT"), _stream()),
           "uot_nhwc_transpose")
    return out


def bias_grad_bf16(dy, C, out=None):
    P, ld = dy.shape
    out = torch.empty(C, dtype=torch.float32, device=dy.device) if out is None else out
    _check(load().uot_bias_grad_bf16(_ptr(dy, BF16, "dy"), P, ld, C, _ptr(out, torch.float32, "db"), _stream()),
           "uot_bias_grad_bf16")
    return out


def conv_weights_bf16(w, cout_pad, cin_pad, cin_rows=0, cout_kpad=0, wf=None, wb=None, backward=True):
    """FP32 w [Cout, Cin, 3, 3] -> (wf [cout_pad, 9, cin_pad], wb [cin_rows, 9, cout_kpad] or None) BF16."""
    Cout, Cin = w.shape[:2]
    wf = torch.empty(cout_pad, 9, cin_pad, dtype=BF16, device=w.device) if wf is None else wf
    if backward and wb is None:
        wb = torch.empty(cin_rows, 9, cout_kpad, dtype=BF16, device=w.device)
    _check(load().uot_conv_weights_bf16(_ptr(w, torch.float32, "w"), Cout, Cin, cout_pad, cin_pad, cin_rows,
                                        cout_kpad, _ptr(wf, BF16, "wf"), _ptr(wb, BF16, "wb") if backward else None,
                                        _stream()), "uot_conv_weights_bf16")
    return wf, (wb if backward else None)


def warmstart_features_nhwc(P, Q, log_eps, log_lam, out=None):
    N, H, W = P.shape
    f = torch.float32
    out = torch.empty(N * H * W, 64, dtype=BF16, device=P.device) if out is None else out
    _check(load().uot_warmstart_features_nhwc(_ptr(P, f, "p"), _ptr(Q, f, "q"), _ptr(log_eps, f, "log_eps"),
                                              _ptr(log_lam, f, "log_lam"), _ptr(out, BF16, "out"), N, H, W,
                                              _stream()), "uot_warmstart_features_nhwc")
    return out


def mse_grad_nhwc(pred, U, V, scale, grad, loss_dev):
    N, HW = U.shape
    f = torch.float32
    _check(load().uot_mse_grad_nhwc(_ptr(pred, f, "pred"), _ptr(U, f, "U"), _ptr(V, f, "V"), _ptr(scale, f, "scale"),
                                    N, HW, _ptr(grad, BF16, "grad"), _ptr(loss_dev, torch.float64, "loss"),
                                    _stream()), "uot_mse_grad_nhwc")
    return grad


def pred_to_potentials(pred, scale, N, HW, U0=None, V0=None):
    f = torch.float32
    U0 = torch.empty(N, HW, dtype=f, device=pred.device) if U0 is None else U0
    V0 = torch.empty(N, HW, dtype=f, device=pred.device) if V0 is None else V0
    _check(load().uot_pred_to_potentials(_ptr(pred, f, "pred"), _ptr(scale, f, "scale"), N, HW, _ptr(U0, f, "U0"),
                                         _ptr(V0, f, "V0"), _stream()), "uot_pred_to_potentials")
    return U0, V0

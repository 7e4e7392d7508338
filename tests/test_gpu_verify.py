"""The FP32 path's stop confirmed in FP64 (uot_opts.verify) with FP64 outputs
(uot_opts.out_f64): the potentials the library returns meet the requested
marginal violation when the FP64 oracle evaluates them, the violation the
library reports is that same FP64 value, and past the FP32 rounding floor
the FP64 iterations that finish the solve reach the oracle's fixed point.
"""
import numpy as np
import pytest
import torch

import oracle as O
from paper_1607_05816_gb300 import uot as U
from test_gpu_parity import dense_problem, grid_problem, points_problem, rel_err, round_geom, rounded, T, to_np

pytestmark = [pytest.mark.gpu, pytest.mark.filterwarnings("ignore::RuntimeWarning")]

CASES = [
    ("grid2d", lambda: grid_problem((40, 48), (36, 50), 21)),
    ("grid1d", lambda: grid_problem((300,), (257,), 22)),
    ("points", lambda: points_problem(301, 260, 3, 23)),
    ("dense", lambda: dense_problem(97, 130, 24)),
]


def oracle_violation(og, dx, dy, p, q, F1, F2, eps, Ug, Vg):
    rdx, rdy, rp, rq = rounded(U.F32, dx, dy, p, q)
    return O.marginal_violation(round_geom(og, U.F32), rdx, rdy, rp, rq, F1, F2, eps,
                                to_np(Ug).reshape(np.shape(p)), to_np(Vg).reshape(np.shape(q)))


def lib_solve(lg, dx, dy, p, q, F1, F2, eps, tol, **kw):
    return U.solve(lg(U.F32), T(p, U.F32).ravel(), T(dx, U.F32).ravel(), T(q, U.F32).ravel(),
                   T(dy, U.F32).ravel(), F1, F2, eps, precision=U.F32, max_iter=20000, tol=tol, **kw)


@pytest.mark.parametrize("name,make", CASES)
@pytest.mark.parametrize("launch_mode", [0, 2])
def test_confirmed_stop_meets_tol_under_the_oracle(name, make, launch_mode):
    og, lg, dx, dy, p, q = make()
    eps, tol = 0.01, 1e-6
    Ug, Vg, info = lib_solve(lg, dx, dy, p, q, U.KL(0.5), U.KL(0.5), eps, tol, check_every=10,
                             out_f64=True, verify=True, launch_mode=launch_mode)
    assert Ug.dtype == torch.float64 and Vg.dtype == torch.float64
    assert info["status"] == "UOT_OK" and info["verifications"] >= 1, info
    assert info["marg_err"] <= tol
    v = oracle_violation(og, dx, dy, p, q, O.KL(0.5), O.KL(0.5), eps, Ug, Vg)
    assert v <= tol, (v, info)
    # the library's FP64 check is the oracle's measure of the same state
    assert abs(v - info["marg_err"]) <= 1e-6 * v + 1e-15, (v, info)


def test_fp64_finish_past_the_fp32_floor():
    """tol = 1e-10 lies below what FP32 Gibbs sums resolve: the FP32 check
    stalls, the solve finishes with FP64 iterations, and the result is the
    oracle's fixed point."""
    og, lg, dx, dy, p, q = grid_problem((40, 48), (36, 50), 25)
    eps, tol = 0.02, 1e-10
    Ug, Vg, info = lib_solve(lg, dx, dy, p, q, U.KL(0.5), U.KL(0.5), eps, tol, check_every=10,
                             out_f64=True, verify=True, launch_mode=2)
    assert info["status"] == "UOT_OK" and info["polish_iters"] > 0, info
    assert info["marg_err_fp32"] > tol
    v = oracle_violation(og, dx, dy, p, q, O.KL(0.5), O.KL(0.5), eps, Ug, Vg)
    assert v <= tol * (1 + 1e-6), (v, info)
    rdx, rdy, rp, rq = rounded(U.F32, dx, dy, p, q)
    r = O.solve_log(round_geom(og, U.F32), rdx, rdy, rp, rq, O.KL(0.5), O.KL(0.5), eps, max_iter=5000,
                    tol=1e-13)
    assert rel_err(to_np(Ug), r["U"]) <= 1e-8
    assert rel_err(to_np(Vg), r["V"]) <= 1e-8


def test_fp64_finish_with_float_outputs():
    """Without out_f64 the FP64 state of the finishing iterations is rounded
    to float: the same potentials as with out_f64, up to that rounding."""
    og, lg, dx, dy, p, q = grid_problem((40, 48), (36, 50), 25)
    eps, tol = 0.02, 1e-10
    U64, V64, _ = lib_solve(lg, dx, dy, p, q, U.KL(0.5), U.KL(0.5), eps, tol, check_every=10,
                            out_f64=True, verify=True)
    U32, V32, info = lib_solve(lg, dx, dy, p, q, U.KL(0.5), U.KL(0.5), eps, tol, check_every=10,
                               verify=True)
    assert U32.dtype == torch.float32 and info["polish_iters"] > 0
    assert torch.equal(U32, U64.float()) and torch.equal(V32, V64.float())


def test_out_f64_alone_keeps_the_fp32_stop():
    """out_f64 without verify: the FP32 check decides the stop, and the output
    is the float-float state rounded to FP64 (its float rounding is the float
    output of the same solve)."""
    og, lg, dx, dy, p, q = grid_problem((40, 48), (36, 50), 26)
    eps = 0.02
    U64, V64, i64 = lib_solve(lg, dx, dy, p, q, U.KL(0.5), U.TV(0.2), eps, 1e-6, check_every=10, out_f64=True)
    U32, V32, i32 = lib_solve(lg, dx, dy, p, q, U.KL(0.5), U.TV(0.2), eps, 1e-6, check_every=10)
    assert i64["verifications"] == 0 and i64["iters"] == i32["iters"]
    assert torch.equal(U64.float(), U32) and torch.equal(V64.float(), V32)


def test_verified_stop_many_problems():
    """uot_solve_many: the confirmation covers every problem of the batch."""
    og, lg, dx, dy, p, q = grid_problem((40, 48), (36, 50), 27)
    g = np.random.default_rng(3)
    P = np.stack([p * g.uniform(0.5, 2.0) for _ in range(3)])
    Q = np.stack([q * g.uniform(0.5, 2.0) for _ in range(3)])
    eps, tol = 0.01, 1e-6
    Ug, Vg, info = U.solve_many(lg(U.F32), T(P.reshape(3, -1), U.F32), T(dx, U.F32).ravel(),
                                T(Q.reshape(3, -1), U.F32), T(dy, U.F32).ravel(), U.KL(0.5), U.KL(0.5), eps,
                                precision=U.F32, max_iter=20000, tol=tol, check_every=10, out_f64=True,
                                verify=True, launch_mode=2)
    assert info["status"] == "UOT_OK" and info["verifications"] >= 1
    worst = max(oracle_violation(og, dx, dy, P[b], Q[b], O.KL(0.5), O.KL(0.5), eps, Ug[b], Vg[b])
                for b in range(3))
    assert worst <= tol
    assert abs(worst - info["marg_err"]) <= 1e-6 * worst + 1e-15


def test_verify_options_are_checked():
    """out_f64 and verify take 0 or 1; entry points other than uot_solve and
    uot_solve_many refuse them (nothing launched)."""
    import ctypes as C
    og, lg, dx, dy, p, q = grid_problem((8, 8), (8, 8), 28)
    lib = U.load()
    t = [T(a, U.F32).ravel() for a in (p, dx, q, dy)]
    out = [torch.empty(64, dtype=torch.float32, device="cuda") for _ in range(2)]
    g = lg(U.F32).c(U.F32)
    ptr = [x.data_ptr() for x in t + out]

    def opts(out_f64, verify):
        return U.COpts(U.F32, 0.05, 0.0, 0, 0, 5, 0.0, 1, 0, 0, None, None, out_f64, verify)
    r = U.CResult()
    o = opts(2, 0)
    assert lib.uot_solve(C.byref(g), *ptr[:4], C.byref(U.KL(0.5).c()), C.byref(U.KL(0.5).c()), C.byref(o),
                         *ptr[4:], C.byref(r), None) == -1
    o = opts(0, 1)
    Z = C.c_double(0.0)
    assert lib.uot_solve_mass(C.byref(g), *ptr[:4], C.byref(U.KL(0.5).c()), C.byref(U.KL(0.5).c()),
                              C.byref(U.EQ().c()), 1.0, C.byref(o), *ptr[4:], C.byref(Z), C.byref(r),
                              None) == -6

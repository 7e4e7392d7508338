"""The translation step (uot_opts.translate, KL penalties on both sides): after
the V-update of every checked iteration, U += c and V -= c with c the exact
maximum of the dual (Theorem 3.2) along that direction.  Not in the paper: it
is the translation step of the translation-invariant formulation of Sejourne,
Vialard, Peyre (2022).

Parity: the CUDA iterates against the oracle's translated iteration, element
by element, with the same schedule (eps-scaling stages, checks every 5
iterations, a last iteration off the check grid), on every geometry, in FP64
and FP32, per-pass launches and CUDA-graph blocks, one problem and a batch.
Effect: with lambda / eps large the translated solve reaches the tolerance in
a fraction of the iterations, and the returned potentials meet it under the
oracle.  Option checks: non-KL penalties and the other entry points refuse it.
"""
import ctypes as C

import numpy as np
import pytest
import torch

import oracle as O
from paper_1607_05816_gb300 import synth
from paper_1607_05816_gb300 import uot as U
from test_gpu_parity import (TOL, T, dense_problem, grid_problem, points_problem, rel_err, round_geom, rounded,
                             to_np)

pytestmark = [pytest.mark.gpu, pytest.mark.filterwarnings("ignore::RuntimeWarning")]

CASES = [
    ("grid2d", lambda: grid_problem((40, 67), (52, 38), 41)),
    ("grid1d", lambda: grid_problem((300,), (257,), 42)),
    ("grid3d", lambda: grid_problem((9, 13, 6), (7, 5, 11), 43)),
    ("points", lambda: points_problem(333, 250, 3, 44)),
    ("dense", lambda: dense_problem(97, 130, 45)),
]
L1, L2 = 0.7, 2.5
SCHED = dict(eps=0.01, iters=27, check_every=5, eps_start=0.1, stages=2, ips=7)


def oracle_translated(og, prec, dx, dy, p, q):
    rdx, rdy, rp, rq = rounded(prec, dx, dy, p, q)
    s = SCHED
    return O.solve_log(round_geom(og, prec), rdx, rdy, rp, rq, O.KL(L1), O.KL(L2), s["eps"], max_iter=s["iters"],
                       eps_start=s["eps_start"], stages=s["stages"], iters_per_stage=s["ips"],
                       check_every=s["check_every"], translate=True)


@pytest.mark.parametrize("launch_mode", [0, 2])
@pytest.mark.parametrize("prec", [U.F64, U.F32])
@pytest.mark.parametrize("name,make", CASES)
def test_translated_iterates_match_oracle(name, make, prec, launch_mode):
    og, lg, dx, dy, p, q = make()
    s = SCHED
    r = oracle_translated(og, prec, dx, dy, p, q)
    Ug, Vg, info = U.solve(lg(prec), T(p, prec).ravel(), T(dx, prec).ravel(), T(q, prec).ravel(),
                           T(dy, prec).ravel(), U.KL(L1), U.KL(L2), s["eps"], precision=prec, max_iter=s["iters"],
                           check_every=s["check_every"], eps_start=s["eps_start"], eps_stages=s["stages"],
                           iters_per_stage=s["ips"], launch_mode=launch_mode, translate=True)
    assert info["iters"] == s["iters"] and info["total_iters"] == s["iters"] + s["stages"] * s["ips"]
    Ug, Vg = to_np(Ug), to_np(Vg)
    assert np.array_equal(np.isneginf(Ug), np.isneginf(r["U"].ravel()))
    assert rel_err(Ug, r["U"]) <= TOL[prec]
    assert rel_err(Vg, r["V"]) <= TOL[prec]
    # the oracle without the step differs by far more than the tolerance
    rdx, rdy, rp, rq = rounded(prec, dx, dy, p, q)
    plain = O.solve_log(round_geom(og, prec), rdx, rdy, rp, rq, O.KL(L1), O.KL(L2), s["eps"], max_iter=s["iters"],
                        eps_start=s["eps_start"], stages=s["stages"], iters_per_stage=s["ips"],
                        check_every=s["check_every"])
    assert rel_err(Ug, plain["U"]) > 100 * TOL[prec]


@pytest.mark.parametrize("prec", [U.F64, U.F32])
def test_translated_batch_matches_oracle_per_problem(prec):
    """uot_solve_many: each problem takes its own shift."""
    probs = [grid_problem((30, 41), (37, 29), 50 + k) for k in range(3)]
    og, lg, dx, dy, _, _ = probs[0]
    P = np.stack([pr[4].ravel() for pr in probs])
    Q = np.stack([pr[5].ravel() * (0.5 + k) for k, pr in enumerate(probs)])  # unequal mass ratios
    s = SCHED
    Ug, Vg, info = U.solve_many(lg(prec), T(P, prec), T(dx, prec).ravel(), T(Q, prec), T(dy, prec).ravel(),
                                U.KL(L1), U.KL(L2), s["eps"], precision=prec, max_iter=s["iters"],
                                check_every=s["check_every"], eps_start=s["eps_start"], eps_stages=s["stages"],
                                iters_per_stage=s["ips"], launch_mode=2, translate=True)
    for k in range(3):
        r = oracle_translated(og, prec, dx, dy, P[k].reshape(30, 41), Q[k].reshape(37, 29))
        assert rel_err(to_np(Ug[k]), r["U"]) <= TOL[prec], k
        assert rel_err(to_np(Vg[k]), r["V"]) <= TOL[prec], k


@pytest.mark.parametrize("lam,eps", [(5.0, 2e-3), (1.0, 3e-3)])
def test_translation_reaches_tol_in_fewer_iterations(lam, eps):
    """A 64 x 64 blob instance solved to 1e-6 (FP32 passes, stop confirmed in
    FP64, FP64 outputs) with and without the step: at the final eps the
    translated solve needs at most a fifth of the iterations (the 400 stage
    iterations are the same), and both results meet the tolerance when the
    oracle evaluates them."""
    inst = synth.warmstart_instances(1, 64, 64, seed=46, group=1)
    xs = [torch.as_tensor(a, dtype=torch.float32, device="cuda") for a in inst["xs"]]
    geo = U.Geometry.grid(xs, xs)
    dxt = torch.as_tensor(inst["dx"], dtype=torch.float32, device="cuda").ravel()
    p = torch.as_tensor(inst["P"][0], dtype=torch.float32, device="cuda").ravel()
    q = torch.as_tensor(inst["Q"][0], dtype=torch.float32, device="cuda").ravel()
    og = O.Geometry("grid", xs=[rounded(U.F32, a) for a in inst["xs"]], ys=[rounded(U.F32, a) for a in inst["xs"]])
    rdx, rp, rq = rounded(U.F32, inst["dx"], inst["P"][0], inst["Q"][0])
    res = {}
    for tr in (False, True):
        Ug, Vg, info = U.solve(geo, p, dxt, q, dxt, U.KL(lam), U.KL(lam), eps, precision=U.F32, max_iter=60000,
                               tol=1e-6, check_every=10, eps_start=0.1, eps_stages=10, iters_per_stage=40,
                               launch_mode=2, out_f64=True, verify=True, translate=tr)
        assert info["status"] == "UOT_OK", info
        v = O.marginal_violation(og, rdx, rdx, rp, rq, O.KL(lam), O.KL(lam), eps, to_np(Ug).reshape(64, 64),
                                 to_np(Vg).reshape(64, 64))
        assert v <= 1e-6, (tr, v, info)
        res[tr] = info
    print(f"lam {lam} eps {eps}: plain {res[False]}\n   translated {res[True]}")
    assert res[True]["iters"] * 5 <= res[False]["iters"], res


def test_translation_option_is_checked():
    """translate takes 0 or 1, needs KL on both sides, and entry points other
    than uot_solve / uot_solve_many refuse it (nothing launched)."""
    og, lg, dx, dy, p, q = grid_problem((8, 8), (8, 8), 47)
    lib = U.load()
    t = [T(a, U.F32).ravel() for a in (p, dx, q, dy)]
    out = [torch.empty(64, dtype=torch.float32, device="cuda") for _ in range(2)]
    g = lg(U.F32).c(U.F32)
    ptr = [x.data_ptr() for x in t + out]

    def opts(translate):
        return U.COpts(U.F32, 0.05, 0.0, 0, 0, 5, 0.0, 1, 0, 0, None, None, 0, 0, 0.0, translate)
    r = U.CResult()

    def solve(F1, F2, o):
        return lib.uot_solve(C.byref(g), *ptr[:4], C.byref(F1.c()), C.byref(F2.c()), C.byref(o), *ptr[4:],
                             C.byref(r), None)
    assert solve(U.KL(0.5), U.KL(0.5), opts(2)) == -1
    assert solve(U.KL(0.5), U.TV(0.5), opts(1)) == -6
    assert solve(U.EQ(), U.KL(0.5), opts(1)) == -6
    assert solve(U.KL(0.5), U.KL(0.5), opts(1)) == 0
    Z = C.c_double(0.0)
    assert lib.uot_solve_mass(C.byref(g), *ptr[:4], C.byref(U.KL(0.5).c()), C.byref(U.KL(0.5).c()),
                              C.byref(U.EQ().c()), 1.0, C.byref(opts(1)), *ptr[4:], C.byref(Z), C.byref(r),
                              None) == -6


def test_translation_with_persistent_launch_mode():
    """launch_mode 1 (the persistent kernel) has no translation step: the solve
    runs per-pass launches and gives the oracle's translated iterates."""
    og, lg, dx, dy, p, q = CASES[0][1]()
    s = SCHED
    r = oracle_translated(og, U.F32, dx, dy, p, q)
    Ug, Vg, _ = U.solve(lg(U.F32), T(p, U.F32).ravel(), T(dx, U.F32).ravel(), T(q, U.F32).ravel(),
                        T(dy, U.F32).ravel(), U.KL(L1), U.KL(L2), s["eps"], precision=U.F32, max_iter=s["iters"],
                        check_every=s["check_every"], eps_start=s["eps_start"], eps_stages=s["stages"],
                        iters_per_stage=s["ips"], launch_mode=1, translate=True)
    assert rel_err(to_np(Ug), r["U"]) <= TOL[U.F32]

"""GPU parity of Algorithm 4 (a divergence F3 on the plan's total mass,
Sec. 4.5): uot_solve_mass through the C ABI against the oracle's log-form
solve_mass_log on the same seeded inputs, element by element for U and V and
for the scalar Z = eps log z.  Tolerances as for uot_solve: 1e-10 (FP64) and
1e-5 (FP32) relative to max(1, |reference|_inf)."""
import math

import numpy as np
import pytest
import torch

import oracle as O
from paper_1607_05816_gb300 import uot as U

from test_gpu_parity import (TOL, T, dense_problem, grid_problem, points_problem, rel_err, round_geom,
                             rounded, to_np)

pytestmark = [pytest.mark.gpu, pytest.mark.filterwarnings("ignore::RuntimeWarning")]

# (oracle F1, F2, F3, library F1, F2, F3)
MASS_DIVS = {
    "kl-kl-eq": (O.KL(0.5), O.KL(0.5), O.EQ(), U.KL(0.5), U.KL(0.5), U.EQ()),
    "kl-tv-kl": (O.KL(0.3), O.TV(0.2), O.KL(0.05), U.KL(0.3), U.TV(0.2), U.KL(0.05)),
    "tv-kl-tv": (O.TV(0.1), O.KL(0.4), O.TV(0.02), U.TV(0.1), U.KL(0.4), U.TV(0.02)),
    "rg-kl-rg": (O.RG(0.5, 2.0), O.KL(0.4), O.RG(1.1, 1.3), U.RG(0.5, 2.0), U.KL(0.4), U.RG(1.1, 1.3)),
}


def run_both(og, lg, dx, dy, p, q, divs, m0, eps, iters, prec, eps_start=None, stages=0, ips=0,
             launch_mode=0):
    OF1, OF2, OF3, UF1, UF2, UF3 = divs
    rdx, rdy, rp, rq = rounded(prec, dx, dy, p, q)
    r = O.solve_mass_log(round_geom(og, prec), rdx, rdy, rp, rq, OF1, OF2, OF3, m0, eps, max_iter=iters,
                         eps_start=eps_start, stages=stages, iters_per_stage=ips)
    Ug, Vg, Zg, info = U.solve_mass(lg(prec), T(p, prec).ravel(), T(dx, prec).ravel(), T(q, prec).ravel(),
                                    T(dy, prec).ravel(), UF1, UF2, UF3, m0, eps, precision=prec,
                                    max_iter=iters, eps_start=eps_start, eps_stages=stages,
                                    iters_per_stage=ips, launch_mode=launch_mode)
    return r, to_np(Ug), to_np(Vg), Zg, info


def z_err(got, want):
    if not math.isfinite(want):
        assert got == want
        return 0.0
    return abs(got - want) / max(1.0, abs(want))


@pytest.mark.parametrize("prec", [U.F64, U.F32])
@pytest.mark.parametrize("name", list(MASS_DIVS))
def test_solve_mass_grid_parity(name, prec):
    """2-D grids with ragged tails and zero densities, every Table 1 row as F3."""
    og, lg, dx, dy, p, q = grid_problem((40, 67), (52, 38), 10)
    r, Ug, Vg, Zg, info = run_both(og, lg, dx, dy, p, q, MASS_DIVS[name], 1.15, 0.01, 30, prec)
    assert info["iters"] == 30
    assert rel_err(Ug, r["U"]) <= TOL[prec]
    assert rel_err(Vg, r["V"]) <= TOL[prec]
    assert z_err(Zg, r["Z"]) <= TOL[prec]
    assert r["Z"] != 0.0  # the mass term acted


@pytest.mark.parametrize("prec", [U.F64, U.F32])
def test_solve_mass_points_parity(prec):
    og, lg, dx, dy, p, q = points_problem(333, 250, 3, 12)
    r, Ug, Vg, Zg, info = run_both(og, lg, dx, dy, p, q, MASS_DIVS["kl-tv-kl"], 0.8, 0.01, 25, prec)
    assert rel_err(Ug, r["U"]) <= TOL[prec]
    assert rel_err(Vg, r["V"]) <= TOL[prec]
    assert z_err(Zg, r["Z"]) <= TOL[prec]


@pytest.mark.parametrize("prec", [U.F64, U.F32])
def test_solve_mass_dense_parity(prec):
    og, lg, dx, dy, p, q = dense_problem(256, 200, 1234)
    r, Ug, Vg, Zg, info = run_both(og, lg, dx, dy, p, q, MASS_DIVS["kl-kl-eq"], 0.9, 1e-2, 40, prec)
    assert rel_err(Ug, r["U"]) <= TOL[prec]
    assert rel_err(Vg, r["V"]) <= TOL[prec]
    assert z_err(Zg, r["Z"]) <= TOL[prec]


@pytest.mark.parametrize("prec", [U.F64, U.F32])
def test_solve_mass_eps_scaling_parity(prec):
    """eps-scaling stages (Sec. 4.4): the first iteration (z = 1) lies in the
    first stage; z then carries over between stages like U and V."""
    og, lg, dx, dy, p, q = grid_problem((48, 48), (48, 48), 11, zeros=False)
    r, Ug, Vg, Zg, info = run_both(og, lg, dx, dy, p, q, MASS_DIVS["kl-kl-eq"], 1.1, 1e-3, 20, prec,
                                   eps_start=0.1, stages=10, ips=5)
    assert info["total_iters"] == 70
    assert rel_err(Ug, r["U"]) <= TOL[prec]
    assert rel_err(Vg, r["V"]) <= TOL[prec]
    assert z_err(Zg, r["Z"]) <= TOL[prec]


def test_solve_mass_single_iteration_keeps_z_one():
    """One iteration never updates z (Algorithm 4 starts from z = 1)."""
    og, lg, dx, dy, p, q = dense_problem(64, 48, 5)
    r, Ug, Vg, Zg, info = run_both(og, lg, dx, dy, p, q, MASS_DIVS["kl-kl-eq"], 2.0, 0.05, 1, U.F64)
    assert Zg == 0.0 and r["Z"] == 0.0
    assert rel_err(Ug, r["U"]) <= 1e-10


def test_solve_mass_tolerance_stop_matches_oracle():
    """The stopping measure (marginal violation with S + Z, or the z-update's
    mass violation if larger) stops at the same iteration as the oracle and
    reports the same value."""
    og, lg, dx, dy, p, q = dense_problem(120, 90, 77)
    OF1, OF2, OF3, UF1, UF2, UF3 = MASS_DIVS["kl-kl-eq"]
    r = O.solve_mass_log(og, dx, dy, p, q, OF1, OF2, OF3, 0.95, 0.02, max_iter=5000, tol=1e-8, check_every=7)
    Ug, Vg, Zg, info = U.solve_mass(lg(U.F64), T(p, U.F64), T(dx, U.F64), T(q, U.F64), T(dy, U.F64),
                                    UF1, UF2, UF3, 0.95, 0.02, precision=U.F64, max_iter=5000, tol=1e-8,
                                    check_every=7)
    assert info["status"] == "UOT_OK"
    assert info["iters"] == r["iters"]
    assert abs(info["marg_err"] - r["err"]) <= 1e-6 * r["err"]
    assert rel_err(to_np(Ug), r["U"]) <= 1e-10
    assert z_err(Zg, r["Z"]) <= 1e-10


@pytest.mark.parametrize("prec", [U.F32, U.F64])
def test_solve_mass_graph_blocks_match_per_pass(prec):
    """launch_mode 2 replays the same kernels as per-pass launches: identical
    iterates, Z, stopping iteration and launch count."""
    og, lg, dx, dy, p, q = grid_problem((48, 64), (48, 64), 33, zeros=False)
    args = [T(a, prec).ravel() for a in (p, dx, q, dy)]
    outs = []
    for mode in (2, 0):
        n0 = U.launch_count()
        r = U.solve_mass(lg(prec), *args, U.KL(0.5), U.KL(0.5), U.EQ(), 1.2, 5e-3, precision=prec,
                         max_iter=3000, tol=1e-6, check_every=10, eps_start=0.1, eps_stages=4,
                         iters_per_stage=15, launch_mode=mode)
        outs.append(r + (U.launch_count() - n0,))
    (U0, V0, Z0, i0, n0), (U1, V1, Z1, i1, n1) = outs
    assert i0["status"] == i1["status"] == "UOT_OK"
    assert i0["iters"] == i1["iters"] and i0["total_iters"] == i1["total_iters"]
    assert i0["iters"] > 30
    assert abs(i0["marg_err"] - i1["marg_err"]) <= 1e-12
    assert torch.equal(U0, U1) and torch.equal(V0, V1) and Z0 == Z1
    assert n0 == n1


@pytest.mark.parametrize("prec", [U.F64, U.F32])
def test_solve_mass_eq_fixes_total_mass(prec):
    """Property at the size of the 256 x 256 grid workload: with F3 = EQ the
    converged plan e^{(U + V + Z - C)/eps} has total mass m0 (measured with
    uot_apply_plan, the plan's first marginal), while the plain solve's plan
    does not."""
    n = 256
    og, lg, dx, dy, p, q = grid_problem((n, n), (n, n), 21, zeros=False)
    geo = lg(prec)
    args = [T(a, prec).ravel() for a in (p, dx, q, dy)]
    m0, eps = 1.5, 1e-2
    Ug, Vg, Zg, info = U.solve_mass(geo, *args, U.KL(0.1), U.KL(0.1), U.EQ(), m0, eps, precision=prec,
                                    max_iter=5000, tol=1e-7, check_every=10, launch_mode=2)
    assert info["status"] == "UOT_OK"
    r1 = U.apply_plan(geo, Ug + Zg, Vg, eps, args[1], args[3], precision=prec)
    mass = float(torch.sum(r1[:, 0].double() * args[1].double()))
    assert abs(mass - m0) <= 1e-5 * m0
    Us, Vs, _ = U.solve(geo, *args, U.KL(0.1), U.KL(0.1), eps, precision=prec, max_iter=5000, tol=1e-7,
                        check_every=10, launch_mode=2)
    r1s = U.apply_plan(geo, Us, Vs, eps, args[1], args[3], precision=prec)
    assert abs(float(torch.sum(r1s[:, 0].double() * args[1].double())) - m0) > 1e-2


def test_solve_mass_invalid_arguments():
    og, lg, dx, dy, p, q = dense_problem(16, 16, 3)
    geo = lg(U.F64)
    args = (T(p, U.F64), T(dx, U.F64), T(q, U.F64), T(dy, U.F64))
    for m0 in (0.0, -1.0, math.inf, math.nan):
        with pytest.raises(U.UotError, match="EINVAL"):
            U.solve_mass(geo, *args, U.KL(1.0), U.KL(1.0), U.EQ(), m0, 0.1)
    with pytest.raises(U.UotError, match="EINVAL"):
        U.solve_mass(geo, *args, U.KL(1.0), U.KL(1.0), U.KL(-1.0), 1.0, 0.1)
    with pytest.raises(U.UotError, match="EINVAL"):
        U.solve_mass(geo, *args, U.KL(1.0), U.KL(1.0), U.RG(2.0, 1.0), 1.0, 0.1)

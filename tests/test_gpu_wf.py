"""GPU parity of the WF gradient flow with growth (Sec. 5.3): uot_wf_cost and
uot_wf_flow through the C ABI against the oracle's wf_cost / wf_flow_log on
the same seeded inputs.  Densities after every step and the last step's
potentials are compared element by element: 1e-10 (FP64) and 1e-5 (FP32)
relative to max(1, |reference|_inf), the same -inf pattern."""
import math

import numpy as np
import pytest
import torch

import oracle as O
from paper_1607_05816_gb300 import synth
from paper_1607_05816_gb300 import uot as U

from test_gpu_parity import TOL, T, rel_err, rounded, to_np

pytestmark = [pytest.mark.gpu, pytest.mark.filterwarnings("ignore::RuntimeWarning")]


def tumor_densities(n, S, seed):
    """Seeded blobs on [0, 1] with exact zeros outside their supports (the
    paper's initial tumor densities are bumps below 1 on a subinterval)."""
    g = synth.rng(seed)
    x = (np.arange(n) + 0.5) / n
    P = np.zeros((S, n))
    for k in range(S):
        c0 = g.uniform(0.3, 0.7)
        w = g.uniform(0.05, 0.12)
        P[k] = np.where(np.abs(x - c0) < w, g.uniform(0.3, 0.6) * (1.0 + 0.3 * np.cos(40 * x)), 0.0)
    return x, np.full(n, 1.0 / n), P


@pytest.mark.parametrize("prec", [U.F64, U.F32])
@pytest.mark.parametrize("d,cut", [(1, 0.2), (2, 0.35), (3, math.pi / 2)])
def test_wf_cost_parity(d, cut, prec):
    g = synth.rng(40 + d)
    x = g.uniform(0, 1, size=(257, d))
    y = g.uniform(0, 1, size=(190, d))
    rx, ry = rounded(prec, x, y)
    want = O.wf_cost(rx, ry, cut)
    got = to_np(U.wf_cost(T(x, prec), T(y, prec), cut, precision=prec))
    assert np.array_equal(np.isposinf(got), np.isposinf(want))
    f = np.isfinite(want)
    # -2 log cos(d) has condition 2 d tan(d): near the cut locus one rounding of
    # d moves it by 2 tan(d) d 2^-53
    d_ = (math.pi / 2) * np.sqrt(O.sqdist(rx, ry)) / cut
    cond = np.where(f, 2.0 * d_ * np.tan(np.where(f, d_, 0.0)), 0.0)  # finite c: d < pi/2
    ulp = 2.0**-52 if prec == U.F64 else 2.0**-23
    assert np.all(np.abs(got[f] - want[f]) <= 8 * ulp * (np.abs(want[f]) + cond[f] + 1.0))
    assert np.isposinf(want).any() == (cut < 1.0)


def run_flow(n, S, cut, tau, alpha, lam, eps, nsteps, iters, prec, seed, launch_mode=0, eps_start=None,
             stages=0, ips=0):
    x, dx, P0 = tumor_densities(n, S, seed)
    rx, rdx, rP0 = rounded(prec, x, dx, P0)
    C = rounded(prec, O.wf_cost(rx, rx, cut))  # the cost as the library stores it
    r = O.wf_flow_log(O.Geometry("dense", C=C), rdx, rP0, tau, alpha, lam, eps, nsteps, iters,
                      eps_start=eps_start, stages=stages, iters_per_stage=ips)
    xt = T(x, prec)
    geo = U.Geometry.dense(U.wf_cost(xt, xt, cut, precision=prec))
    Pg, Ug, Vg, info = U.wf_flow(geo, T(P0, prec), T(dx, prec), tau, alpha, lam, eps, nsteps, precision=prec,
                                 iters=iters, launch_mode=launch_mode, eps_start=eps_start, eps_stages=stages,
                                 iters_per_stage=ips)
    return r, to_np(Pg), to_np(Ug), to_np(Vg), info


@pytest.mark.parametrize("prec", [U.F64, U.F32])
@pytest.mark.parametrize("S,lam", [(1, 1.0), (2, 1.0), (2, 0.6)])
def test_wf_flow_parity(S, lam, prec):
    """300 points on [0, 1], cut locus at 0.2, zero densities outside the
    blobs; three steps of 40 iterations."""
    eps = 1e-3 if prec == U.F64 else 1e-2
    r, Pg, Ug, Vg, info = run_flow(300, S, 0.2, 0.05, 1.0, lam, eps, 3, 40, prec, seed=7 + S)
    assert info["status"] == "UOT_OK" and info["total_iters"] == 120
    tol = TOL[prec]
    assert rel_err(Pg, r["P"]) <= tol
    assert rel_err(Ug, r["U"]) <= tol
    assert rel_err(Vg, r["V"]) <= tol
    # growth happened and the density cap holds
    assert np.sum(r["P"][-1]) > np.sum(r["P"][0])
    assert np.all(np.sum(Pg, axis=1) <= 1.0 + 1e-6)


@pytest.mark.parametrize("prec", [U.F64, U.F32])
def test_wf_flow_eps_scaling_parity(prec):
    eps = 1e-3 if prec == U.F64 else 1e-2
    r, Pg, Ug, Vg, info = run_flow(200, 2, 0.3, 0.04, 2.0, 1.0, eps, 2, 20, prec, seed=3, eps_start=0.3,
                                   stages=4, ips=5)
    assert info["total_iters"] == 80
    assert rel_err(Pg, r["P"]) <= TOL[prec]
    assert rel_err(Vg, r["V"]) <= TOL[prec]


@pytest.mark.parametrize("prec", [U.F64, U.F32])
def test_wf_flow_graph_steps_match_per_launch(prec):
    """launch_mode 2 replays the first step's launches as one CUDA graph per
    step: identical densities and potentials, the same launch count."""
    x, dx, P0 = tumor_densities(256, 2, 5)
    xt = T(x, prec)
    geo = U.Geometry.dense(U.wf_cost(xt, xt, 0.25, precision=prec))
    outs = []
    for mode in (2, 0):
        n0 = U.launch_count()
        Pg, Ug, Vg, info = U.wf_flow(geo, T(P0, prec), T(dx, prec), 0.05, 1.0, 1.0, 1e-2, 4, precision=prec,
                                     iters=15, launch_mode=mode)
        outs.append((Pg, Ug, Vg, U.launch_count() - n0))
    assert torch.equal(outs[0][0], outs[1][0]) and torch.equal(outs[0][2], outs[1][2])
    assert outs[0][3] == outs[1][3]


def test_wf_flow_paper_size_sampled():
    """The paper's tumor run at full size (3000 points on [0, 1], eps = 1e-8,
    tau = 0.006, alpha = 1, lam = 1, unscaled distance) in FP64, two steps of
    three iterations against the oracle (the full 500 iterations per step are
    timed by bench.py; here the oracle must finish)."""
    eps = 1e-8
    r, Pg, Ug, Vg, info = run_flow(3000, 1, math.pi / 2, 0.006, 1.0, 1.0, eps, 2, 3, U.F64, seed=11)
    assert rel_err(Vg, r["V"]) <= 1e-10
    assert rel_err(Ug, r["U"]) <= 1e-10
    # the densities are e^{(V + T)/eps}: an FP64 rounding of V/eps moves them by
    # |V|/eps x 2^-52 in either implementation
    fin = np.isfinite(r["V"])
    ptol = 64 * np.max(np.abs(r["V"][fin])) / eps * 2.0**-52
    assert rel_err(Pg, r["P"]) <= max(1e-10, ptol)


def test_wf_flow_invalid_arguments():
    x, dx, P0 = tumor_densities(16, 1, 1)
    xt = T(x, U.F64)
    geo = U.Geometry.dense(U.wf_cost(xt, xt, 0.3))
    args = (T(P0, U.F64), T(dx, U.F64))
    with pytest.raises(U.UotError, match="EINVAL"):
        U.wf_flow(geo, *args, 0.5, 1.0, 1.0, 1e-2, 1)  # 2 tau alpha >= lam
    with pytest.raises(U.UotError, match="EINVAL"):
        U.wf_flow(geo, *args, 0.1, -1.0, 1.0, 1e-2, 1)
    with pytest.raises(U.UotError, match="EINVAL"):
        U.wf_flow(geo, *args, 0.1, 1.0, 1.0, 1e-2, 0)
    x32 = T(x, U.F32)
    geo32 = U.Geometry.dense(U.wf_cost(x32, x32, 0.3, precision=U.F32))
    with pytest.raises(U.UotError, match="EUNSUPPORTED"):
        U.wf_flow(geo32, T(P0, U.F32), T(dx, U.F32), 0.1, 1.0, 1.0, 1e-2, 1, precision=U.MIXED)
    with pytest.raises(U.UotError, match="EINVAL"):
        U.wf_cost(xt, xt, 0.0)


@pytest.mark.parametrize("prec", [U.F64, U.F32])
@pytest.mark.parametrize("kind", ["wf", "w2"])
def test_geodesic_as_weighted_barycenters(kind, prec):
    """Geodesics as weighted barycenters of the endpoints (Sec. 5.2): K = 2,
    weights (1 - t, t).  WF: the dense WF cost with the cut locus at 0.2, F1 =
    KL(1), barycenter KL(1) (Table 2 (ii)); Wasserstein: |x - y|^2, F1 = EQ,
    barycenter EQ (Table 2 (i)).  200 samples of [0, 1], two bumps."""
    n = 200
    x = (np.arange(n) + 0.5) / n
    dx = np.full(n, 1.0 / n)
    p0 = np.exp(-((x - 0.25) / 0.06) ** 2) + 1e-3
    p1 = 1.6 * np.exp(-((x - 0.7) / 0.09) ** 2) + 1e-3
    if kind == "w2":
        p1 *= np.sum(p0 * dx) / np.sum(p1 * dx)
        C = O.sqdist(x, x)
        OF1, lam, bk, UF1, UFh = O.EQ(), 1.0, "eq", U.EQ(), U.EQ()
    else:
        C = O.wf_cost(x, x, 0.2)
        OF1, lam, bk, UF1, UFh = O.KL(1.0), 1.0, "kl", U.KL(1.0), U.KL(1.0)
    eps, iters = (1e-3, 60) if prec == U.F64 else (1e-2, 60)
    rx, rdx, rp0, rp1 = rounded(prec, x, dx, p0, p1)
    rC = rounded(prec, C)
    geo = U.Geometry.dense(T(C, prec))
    ts = [0.25, 0.5, 0.75]
    got = to_np(U.geodesic(geo, T(p0, prec), T(p1, prec), ts, T(dx, prec), T(dx, prec), UF1, UFh, eps,
                           precision=prec, max_iter=iters))
    for k, t in enumerate(ts):
        _, _, elogh = O.barycenter_log(O.Geometry("dense", C=rC), rdx, rdx, np.stack([rp0, rp1]),
                                       np.array([1.0 - t, t]), OF1, lam, eps, iters, bary_kind=bk)
        assert rel_err(got[k], elogh) <= TOL[prec]

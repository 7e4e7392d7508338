"""Solves and network inference driven from several host threads, each on its
own CUDA stream, at once (warmstart.run_on_streams, the concurrent form of the
warm-start evaluation).  The library keeps no state shared between calls on
different streams that the results depend on, so every concurrent result must
equal the same call run alone, bit for bit, with the same iteration count."""
import numpy as np
import pytest
import torch

from paper_1607_05816_gb300 import synth
from paper_1607_05816_gb300 import uot as U
from paper_1607_05816_gb300 import warmstart as WS

pytestmark = pytest.mark.gpu


def _grid_job(seed, prec, **kw):
    d = synth.problem_grid2d(48, 40, seed=seed)
    dt = torch.float64 if prec == U.F64 else torch.float32
    t = lambda a: torch.as_tensor(np.ascontiguousarray(a), dtype=dt, device="cuda").ravel()
    geo = U.Geometry.grid([t(a) for a in d["xs"]], [t(a) for a in d["ys"]])
    args = (geo, t(d["p"]), t(d["dx"]), t(d["q"]), t(d["dy"]), U.KL(0.5), U.KL(0.5), 5e-3)
    return lambda: U.solve(*args, precision=prec, max_iter=4000, tol=1e-6, eps_start=0.1, eps_stages=4,
                           iters_per_stage=20, launch_mode=2, **kw)


def _many_job(seed):
    g = synth.rng(seed)
    H = W = 32
    xs = [torch.as_tensor((np.arange(n) + 0.5) / n, dtype=torch.float32, device="cuda") for n in (H, W)]
    geo = U.Geometry.grid(xs, xs)
    P = torch.as_tensor(g.uniform(0.5, 1.5, (4, H * W)), dtype=torch.float32, device="cuda")
    Q = torch.as_tensor(g.uniform(0.5, 1.5, (4, H * W)), dtype=torch.float32, device="cuda")
    dx = torch.full((H * W,), 1.0 / (H * W), dtype=torch.float32, device="cuda")
    return lambda: U.solve_many(geo, P, dx, Q, dx, U.KL(1.0), U.KL(1.0), 1e-2, precision=U.F32, max_iter=3000,
                                tol=1e-6, check_every=10, launch_mode=2, out_f64=True, verify=True, translate=True)


def _points_job(seed):
    g = synth.rng(seed)
    x = torch.as_tensor(synth.mixture_points(g, 700, 3, 4), dtype=torch.float32, device="cuda")
    y = torch.as_tensor(synth.mixture_points(g, 650, 3, 4), dtype=torch.float32, device="cuda")
    f = lambda n, v: torch.full((n,), v, dtype=torch.float32, device="cuda")
    return lambda: U.solve(U.Geometry.points(x, y), f(700, 1.0), f(700, 1 / 700), f(650, 0.7), f(650, 1 / 650),
                           U.KL(0.1), U.KL(0.1), 1e-2, precision=U.F32, max_iter=3000, tol=1e-6, eps_start=0.1,
                           eps_stages=3, iters_per_stage=20, verify=True, out_f64=True)


def _same(a, b):
    assert a[2]["total_iters"] == b[2]["total_iters"]
    assert a[2]["status"] == b[2]["status"]
    assert torch.equal(a[0], b[0]) and torch.equal(a[1], b[1])


def test_concurrent_solves_equal_solves_alone():
    jobs = [_grid_job(3, U.F32, verify=True, out_f64=True), _grid_job(4, U.F32, translate=True),
            _grid_job(5, U.F64), _many_job(6), _points_job(7), _grid_job(8, U.F32, verify=True, out_f64=True),
            _many_job(9), _points_job(10)]
    alone = [j() for j in jobs]
    torch.cuda.synchronize()
    for nstreams in (4, 8):
        ms, together = WS.run_on_streams(jobs, nstreams)
        assert ms > 0.0
        for a, b in zip(alone, together):
            _same(a, b)


def test_concurrent_inference_and_warm_solves_equal_alone():
    """Network inference (per-thread workspaces) followed by a warm-started
    batched solve, four groups on four streams."""
    H = W = 64
    net = WS.WarmStartNetTC(channels=128, seed=3)
    inst = synth.warmstart_instances(16, H, W, seed=91, group=4)
    xs = [torch.as_tensor((np.arange(n) + 0.5) / n, dtype=torch.float32, device="cuda") for n in (H, W)]
    geo = U.Geometry.grid(xs, xs)
    dx = torch.full((H * W,), 1.0 / (H * W), dtype=torch.float32, device="cuda")
    P = torch.as_tensor(inst["P"], dtype=torch.float32, device="cuda")
    Q = torch.as_tensor(inst["Q"], dtype=torch.float32, device="cuda")

    def job(s):
        sl = slice(s, s + 4)
        e, lam = float(inst["eps"][s]), float(inst["lam"][s])
        U0, V0 = net.predict(P[sl].contiguous(), Q[sl].contiguous(), inst["eps"][sl], inst["lam"][sl])
        out = U.solve_many(geo, P[sl].reshape(-1, H * W).contiguous(), dx, Q[sl].reshape(-1, H * W).contiguous(),
                           dx, U.KL(lam), U.KL(lam), e, U0=U0, V0=V0, translate=True, precision=U.F32,
                           max_iter=20000, tol=1e-6, check_every=10, launch_mode=2, out_f64=True, verify=True)
        return out[0], out[1], out[2], U0.clone(), V0.clone()
    jobs = [(lambda s=s: job(s)) for s in range(0, 16, 4)]
    alone = [j() for j in jobs]
    torch.cuda.synchronize()
    _, together = WS.run_on_streams(jobs, 4)
    for a, b in zip(alone, together):
        assert torch.equal(a[3], b[3]) and torch.equal(a[4], b[4])  # the predictions
        _same(a, b)
        assert a[2]["marg_err"] <= 1e-6

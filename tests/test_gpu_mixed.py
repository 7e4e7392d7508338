"""Mixed precision (UOT_MIXED): grid passes on tcgen05 tensor cores with BF16
operands and FP32 accumulation.  Not bit-comparable with FP64; the tests bound
the error against the FP64 oracle and report it (the bound is the measured
one, with margin): Gibbs sums carry a relative error of ~2^-8 from the BF16
operands, i.e. an absolute error of ~eps * 2^-8 on eps log K(b dy)."""
import numpy as np
import pytest
import torch

import oracle as O
from paper_1607_05816_gb300 import synth
from paper_1607_05816_gb300 import uot as U

pytestmark = [pytest.mark.gpu, pytest.mark.filterwarnings("ignore::RuntimeWarning")]


def dev(a):
    return torch.as_tensor(np.ascontiguousarray(a), dtype=torch.float32, device="cuda").ravel()


def f32(a):
    return np.asarray(a, dtype=np.float32).astype(np.float64)


@pytest.mark.parametrize("shape_x,shape_y,eps", [((70, 45), (33, 129), 1e-2), ((256, 256), (256, 256), 1e-3),
                                                   ((128, 96), (128, 96), 1e-2), ((40,), (300,), 1e-2)])
@pytest.mark.parametrize("transpose", [False, True])
def test_mixed_gibbs_error_bound(shape_x, shape_y, eps, transpose):
    g = synth.rng(11)
    xs = [synth.grid_axis(n) for n in shape_x]
    ys = [synth.grid_axis(n) for n in shape_y]
    og = O.Geometry("grid", xs=[f32(a) for a in xs], ys=[f32(a) for a in ys])
    geo = U.Geometry.grid([dev(a) for a in xs], [dev(a) for a in ys])
    shape_in = shape_x if transpose else shape_y
    W = g.normal(size=shape_in) * 0.05
    W.ravel()[3::17] = -np.inf
    w = np.full(shape_in, 1.0 / np.prod(shape_in))
    want = O.apply_K_log(og, f32(W), np.log(f32(w)), eps, transpose=transpose)
    got = U.gibbs_log(geo, dev(W), dev(w), eps, transpose, U.MIXED).double().cpu().numpy()
    want = want.ravel()
    err = np.max(np.abs(got - want))
    print(f"mixed gibbs {shape_x}->{shape_y} eps={eps}: max |S - S_oracle| = {err:.3e} = {err / eps:.3e} eps")
    assert err <= 2.0 ** -6 * eps


def test_mixed_solve_error_bound():
    """30 iterations at eps = 1e-2 on a 2-D grid: mixed vs FP64 oracle."""
    d = synth.problem_grid2d(128, 128, seed=3, masses=(1.0, 1.3))
    og = O.Geometry("grid", xs=[f32(a) for a in d["xs"]], ys=[f32(a) for a in d["ys"]])
    geo = U.Geometry.grid([dev(a) for a in d["xs"]], [dev(a) for a in d["ys"]])
    eps, iters = 1e-2, 30
    Ug, Vg, _ = U.solve(geo, dev(d["p"]), dev(d["dx"]), dev(d["q"]), dev(d["dy"]), U.KL(0.5), U.KL(0.5),
                        eps, precision=U.MIXED, max_iter=iters)
    r = O.solve_log(og, f32(d["dx"]), f32(d["dy"]), f32(d["p"]), f32(d["q"]), O.KL(0.5), O.KL(0.5), eps,
                    max_iter=iters)
    for got, want in ((Ug, r["U"]), (Vg, r["V"])):
        gv = got.double().cpu().numpy()
        wv = want.ravel()
        assert np.array_equal(np.isneginf(gv), np.isneginf(wv))
        f = np.isfinite(wv)
        err = np.max(np.abs(gv[f] - wv[f]))
        print(f"mixed solve: max |U - U_oracle| = {err:.3e}")
        assert err <= 0.05 * eps


def test_mixed_barycenter_error_bound():
    """KL barycenter of 8 blob images, 20 iterations at eps = 1e-2: the mixed
    path's eps log h and V against the FP64 oracle's barycenter iteration."""
    b = synth.barycenter_images(8, 64, 64, seed=12)
    alpha = np.full(8, 1.0 / 8)
    eps, lam, iters = 1e-2, 1.0, 20
    geo = U.Geometry.grid([dev(a) for a in b["xs"]])
    P = torch.as_tensor(f32(b["P"]).reshape(8, -1), dtype=torch.float32, device="cuda")
    lh, _, Vg, _ = U.barycenter(geo, alpha, P, dev(b["dx"]), dev(b["dy"]), U.EQ(), lam, eps,
                                precision=U.MIXED, max_iter=iters)
    og = O.Geometry("grid", xs=[f32(a) for a in b["xs"]], ys=[f32(a) for a in b["ys"]])
    _, Vo, lho = O.barycenter_log(og, f32(b["dx"]), f32(b["dy"]), f32(b["P"]), alpha, O.EQ(), lam, eps, iters)
    for got, want, name in ((lh, lho, "eps log h"), (Vg, Vo.reshape(8, -1), "V")):
        gv = got.double().cpu().numpy().ravel()
        wv = np.asarray(want).ravel()
        assert np.array_equal(np.isneginf(gv), np.isneginf(wv))
        f = np.isfinite(wv)
        err = np.max(np.abs(gv[f] - wv[f]))
        print(f"mixed barycenter: max |{name} - oracle| = {err:.3e} = {err / eps:.3e} eps")
        assert err <= 0.05 * eps


@pytest.mark.parametrize("shape,eps,translate", [((128, 128), 1e-2, False), ((256, 256), 1e-3, False),
                                                 ((128, 128), 1e-2, True)])
def test_mixed_pipeline_reaches_tol_under_the_oracle(shape, eps, translate):
    """BF16 tensor-core passes (eps-scaling stages, then the final eps until the
    violation reaches mixed_switch), FP32 passes to tol, the stop confirmed in
    FP64, with and without the translation step: the returned FP64 potentials
    meet tol when the oracle evaluates them."""
    d = synth.problem_grid2d(*shape, seed=3, masses=(1.0, 1.3))
    og = O.Geometry("grid", xs=[f32(a) for a in d["xs"]], ys=[f32(a) for a in d["ys"]])
    geo = U.Geometry.grid([dev(a) for a in d["xs"]], [dev(a) for a in d["ys"]])
    tol = 1e-6
    Ug, Vg, info = U.solve(geo, dev(d["p"]), dev(d["dx"]), dev(d["q"]), dev(d["dy"]), U.KL(0.5), U.KL(0.5),
                           eps, precision=U.MIXED, max_iter=20000, tol=tol, check_every=20, eps_start=0.1,
                           eps_stages=10, iters_per_stage=100, launch_mode=2, out_f64=True, verify=True,
                           mixed_switch=1e-3, translate=translate)
    print(f"mixed pipeline {shape} eps={eps}: {info}")
    assert info["status"] == "UOT_OK" and info["mixed_iters"] >= 1000, info
    assert info["mixed_iters"] < info["total_iters"]  # the FP32 passes finished the solve
    v = O.marginal_violation(og, f32(d["dx"]), f32(d["dy"]), f32(d["p"]), f32(d["q"]), O.KL(0.5), O.KL(0.5), eps,
                             Ug.cpu().numpy().reshape(shape), Vg.cpu().numpy().reshape(shape))
    assert v <= tol, (v, info)
    assert abs(v - info["marg_err"]) <= 1e-6 * v + 1e-15


def test_mixed_without_tol_stays_on_tensor_cores():
    """tol = 0 (a fixed iteration count): every pass on the tensor cores."""
    d = synth.problem_grid2d(64, 64, seed=4, masses=(1.0, 1.3))
    geo = U.Geometry.grid([dev(a) for a in d["xs"]], [dev(a) for a in d["ys"]])
    _, _, info = U.solve(geo, dev(d["p"]), dev(d["dx"]), dev(d["q"]), dev(d["dy"]), U.KL(0.5), U.KL(0.5), 1e-2,
                         precision=U.MIXED, max_iter=15)
    assert info["mixed_iters"] == 15

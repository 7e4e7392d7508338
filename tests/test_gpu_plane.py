"""Fused pairs of short FP32 grid passes (grid_pass_f32_plane): two consecutive
passes over axes of at most 64 points run as one launch per plane of the two
axes, pass 1's results kept in shared memory.  The fused form must equal the
two separate passes bit for bit (the same float-float values, shifts and
epilogue), on the Gibbs operator alone, on solves (with the violation check)
and on batched solves, and must match the oracle (Sec. 4.4's separable
operator) at the FP32 tolerance."""
import numpy as np
import pytest
import torch

import oracle as O
from paper_1607_05816_gb300 import synth
from paper_1607_05816_gb300 import uot as U

from test_gpu_parity import TOL, T, grid_problem, rel_err, round_geom, rounded, to_np

pytestmark = [pytest.mark.gpu, pytest.mark.filterwarnings("ignore::RuntimeWarning")]

SHAPES = [
    ((10, 33, 17), (12, 30, 20)),   # all axes short: passes 0-1 fused, pass 2 alone
    ((64, 32, 32), (64, 32, 32)),   # the colour grid
    ((100, 20, 30), (90, 24, 28)),  # the long axis runs alone
    ((40, 50), (45, 60)),           # 2-D: the fused pair is the whole operator
    ((64, 64), (64, 64)),
]


SHORT_TILE = 8  # the warp-per-line kernel of short passes, whose arithmetic the fused form shares


def both(fn):
    """(separate passes, fused pairs), every pass not fused on the short-line
    kernel (where it applies, else the first tile) in both runs, so that the
    two differ only by the fusion."""
    prev = U.fuse_short_passes(False)
    U.force_grid_tile(SHORT_TILE)
    try:
        a = fn()
        U.fuse_short_passes(True)
        b = fn()
    finally:
        U.fuse_short_passes(prev)
        U.force_grid_tile(-1)
    return a, b


@pytest.mark.parametrize("shape_x,shape_y", SHAPES)
@pytest.mark.parametrize("transpose", [False, True])
def test_fused_gibbs_equals_separate_and_oracle(shape_x, shape_y, transpose):
    og, lg, dx, dy, p, q = grid_problem(shape_x, shape_y, 5)
    g = synth.rng(11)
    shape_in = np.shape(dx) if transpose else np.shape(dy)
    W = g.normal(size=shape_in) * 0.05
    W.ravel()[3::17] = -np.inf
    w = dx if transpose else dy
    W, w = rounded(U.F32, W, w)
    for eps in (0.02, 2e-3):
        sep, fus = both(lambda: U.gibbs_log(lg(U.F32), T(W, U.F32).ravel(), T(w, U.F32).ravel(), eps, transpose,
                                            U.F32))
        assert torch.equal(sep, fus)
        want = O.apply_K_log(round_geom(og, U.F32), W, np.log(w), eps, transpose=transpose)
        assert rel_err(to_np(fus), want) <= TOL[U.F32]


@pytest.mark.parametrize("shape_x,shape_y", [SHAPES[0], SHAPES[3]])
def test_fused_solve_equals_separate_and_oracle(shape_x, shape_y):
    og, lg, dx, dy, p, q = grid_problem(shape_x, shape_y, 7)
    rdx, rdy, rp, rq = rounded(U.F32, dx, dy, p, q)

    def run():
        return U.solve(lg(U.F32), T(p, U.F32).ravel(), T(dx, U.F32).ravel(), T(q, U.F32).ravel(),
                       T(dy, U.F32).ravel(), U.KL(0.5), U.TV(0.3), 1e-2, precision=U.F32, max_iter=60,
                       tol=0.0, check_every=5, eps_start=0.2, eps_stages=3, iters_per_stage=10, launch_mode=2)
    (U1, V1, i1), (U2, V2, i2) = both(run)
    assert torch.equal(U1, U2) and torch.equal(V1, V2)
    # the violation sums the same FP32 terms, grouped per warp or per block before the FP64 atomics
    assert i1["total_iters"] == i2["total_iters"]
    assert abs(i1["marg_err"] - i2["marg_err"]) <= 1e-6 * i1["marg_err"]
    r = O.solve_log(round_geom(og, U.F32), rdx, rdy, rp, rq, O.KL(0.5), O.TV(0.3), 1e-2, max_iter=60,
                    check_every=5, eps_start=0.2, stages=3, iters_per_stage=10)
    assert rel_err(to_np(U2), r["U"]) <= TOL[U.F32]
    assert rel_err(to_np(V2), r["V"]) <= TOL[U.F32]
    assert abs(i2["marg_err"] - r["err"]) <= 1e-5 * max(1.0, r["err"])


def test_fused_batched_solve_equals_separate():
    """uot_solve_many on 32 x 32 images, 6 problems, stop at 1e-6 with the
    FP64 confirmation: the same potentials and iteration counts."""
    g = synth.rng(21)
    H = W = 32
    xs = [torch.as_tensor((np.arange(n) + 0.5) / n, dtype=torch.float32, device="cuda") for n in (H, W)]
    geo = U.Geometry.grid(xs, xs)
    P = torch.as_tensor(g.uniform(0.5, 1.5, (6, H * W)), dtype=torch.float32, device="cuda")
    Q = torch.as_tensor(g.uniform(0.5, 1.5, (6, H * W)), dtype=torch.float32, device="cuda")
    dx = torch.full((H * W,), 1.0 / (H * W), dtype=torch.float32, device="cuda")

    def run():
        return U.solve_many(geo, P, dx, Q, dx, U.KL(1.0), U.KL(1.0), 1e-2, precision=U.F32, max_iter=3000,
                            tol=1e-6, check_every=10, launch_mode=2, out_f64=True, verify=True)
    (U1, V1, i1), (U2, V2, i2) = both(run)
    assert torch.equal(U1, U2) and torch.equal(V1, V2)
    assert i1["total_iters"] == i2["total_iters"] and i2["marg_err"] <= 1e-6


def test_colour_transfer_fused_equals_separate():
    ix = torch.as_tensor(synth.color_image(128, 96, seed=3), dtype=torch.float32, device="cuda")
    iy = torch.as_tensor(synth.color_image(128, 96, seed=4), dtype=torch.float32, device="cuda")

    def run():
        return U.color_transfer(ix, iy, U.KL(0.03), eps=0.002, iters=200, bins=(16, 8, 8), precision=U.F32,
                                launch_mode=2, check_every=50)
    (o1, t1, i1), (o2, t2, i2) = both(run)
    assert torch.equal(o1, o2) and torch.equal(t1, t2)

"""The block-stabilised FP32 grid pass (uniform axes; one FMA per kernel term,
block sums merged in the log domain) against the FP64 oracle.

Every variant (input blocks of 32 or 64 points, one or two warps per output
block) is forced in turn on ragged 1-D, 2-D and 3-D grids whose axes are
uniform with power-of-two spacings (points x0 + i h exactly in FP32), with
different origins on the two sides, lines of -inf and zero densities; the
profiling counters confirm that the block kernel, not a fallback, ran.
"""
import numpy as np
import pytest
import torch

import oracle as O
from paper_1607_05816_gb300 import synth
from paper_1607_05816_gb300 import uot as U
from test_gpu_parity import rel_err, round_geom, rounded, T, to_np

pytestmark = [pytest.mark.gpu, pytest.mark.filterwarnings("ignore::RuntimeWarning")]

TOL = 1e-5
BLK_TILES = [9, 10, 11, 12, 13]  # blk32x2, blk32x4, blk32x8, blk64x2, blk64x4


def uniform_axis(n, h, first):
    """n points first + i h (exact in FP32 for power-of-two h and first on the h/2 lattice)."""
    return first + h * np.arange(n, dtype=np.float64)


def uniform_problem(shape_x, shape_y, spacing, offsets, seed, zeros=True):
    g = synth.rng(seed)
    xs = [uniform_axis(n, h, 0.5 * h) for n, h in zip(shape_x, spacing)]
    ys = [uniform_axis(n, h, (0.5 + o) * h) for n, h, o in zip(shape_y, spacing, offsets)]
    dx = np.full(shape_x, 1.0 / np.prod(shape_x))
    dy = np.full(shape_y, 1.0 / np.prod(shape_y))
    p = g.uniform(0.2, 2.0, size=shape_x)
    q = g.uniform(0.2, 2.0, size=shape_y)
    if zeros:
        p.ravel()[::7] = 0.0
        q.ravel()[3::11] = 0.0
    p *= 1.0 / np.sum(p * dx)
    q *= 1.3 / np.sum(q * dy)
    og = O.Geometry("grid", xs=xs, ys=ys)

    def lg():
        return U.Geometry.grid([T(a, U.F32) for a in xs], [T(a, U.F32) for a in ys])
    return og, lg, dx, dy, p, q


CASES = [
    ("1d", lambda: uniform_problem((300,), (257,), (1 / 256,), (7,), 1)),
    ("2d", lambda: uniform_problem((100, 45), (77, 70), (1 / 128, 1 / 64), (-10, 3), 2)),
    ("3d", lambda: uniform_problem((40, 9, 33), (35, 11, 30), (1 / 64, 1 / 128, 1 / 64), (2, -1, 0), 3)),
]


def blk_launches(fn):
    U.profile_begin()
    out = fn()
    torch.cuda.synchronize()
    U.profile_end(U.PROF_GRID_PASS)
    _, n = U.profile_end(U.PROF_GRID_BLK)
    return out, n


@pytest.mark.parametrize("tile", BLK_TILES)
@pytest.mark.parametrize("name,make", CASES)
def test_block_pass_operator_matches_oracle(tile, name, make):
    og, lg, dx, dy, p, q = make()
    g = synth.rng(30 + tile)
    eps = 0.01
    U.force_grid_tile(tile)
    try:
        for transpose in (False, True):
            shape_in = np.shape(dx) if transpose else np.shape(dy)
            W = g.normal(size=shape_in) * 0.05
            W.ravel()[5::13] = -np.inf
            if len(shape_in) > 1:
                W[1] = -np.inf  # whole lines without mass
            w = dx if transpose else dy
            W, w = rounded(U.F32, W, w)
            want = O.apply_K_log(round_geom(og, U.F32), W, np.log(w), eps, transpose=transpose)
            got, n = blk_launches(lambda: U.gibbs_log(lg(), T(W, U.F32).ravel(), T(w, U.F32).ravel(), eps,
                                                      transpose, U.F32))
            assert n == len(shape_in), (n, tile)  # every pass ran the block kernel
            assert rel_err(to_np(got), want) <= TOL
    finally:
        U.force_grid_tile(-1)


@pytest.mark.parametrize("tile", BLK_TILES)
@pytest.mark.parametrize("name,make", CASES)
def test_block_pass_solve_matches_oracle(tile, name, make):
    """A KL/TV solve with eps-scaling (the block condition holds at every
    stage) equals the oracle's iterates."""
    og, lg, dx, dy, p, q = make()
    eps = 0.01
    dxr, dyr, pr, qr = rounded(U.F32, dx, dy, p, q)
    U.force_grid_tile(tile)
    try:
        (Ug, Vg, _), n = blk_launches(lambda: U.solve(lg(), *[T(a, U.F32).ravel() for a in (pr, dxr, qr, dyr)],
                                                      U.KL(0.7), U.TV(0.4), eps, precision=U.F32, max_iter=12,
                                                      eps_start=0.1, eps_stages=2, iters_per_stage=3))
    finally:
        U.force_grid_tile(-1)
    assert n == 2 * len(np.shape(dx)) * (12 + 6)
    r = O.solve_log(round_geom(og, U.F32), dxr, dyr, pr, qr, O.KL(0.7), O.TV(0.4), eps, max_iter=12,
                    eps_start=0.1, stages=2, iters_per_stage=3)
    assert rel_err(to_np(Ug), r["U"]) <= TOL
    assert rel_err(to_np(Vg), r["V"]) <= TOL


def test_block_pass_batched_barycenter():
    """Batched lines (the barycenter's measures): the tuner's choice on a
    128 x 128 uniform grid, KL barycenter of 4 blob images, 6 iterations."""
    b = synth.barycenter_images(4, 128, 128, seed=1237)
    alpha = np.full(4, 0.25)
    eps, lam, iters = 1e-2, 1.0, 6
    geo = U.Geometry.grid([T(a, U.F32) for a in b["xs"]])
    P = rounded(U.F32, b["P"])
    (lh, Ug, Vg, _), n = blk_launches(lambda: U.barycenter(
        geo, alpha, T(P.reshape(4, -1), U.F32), T(b["dx"], U.F32).ravel(), T(b["dy"], U.F32).ravel(), U.EQ(),
        lam, eps, precision=U.F32, max_iter=iters))
    og = O.Geometry("grid", xs=[rounded(U.F32, a) for a in b["xs"]], ys=[rounded(U.F32, a) for a in b["ys"]])
    Uo, Vo, lho = O.barycenter_log(og, rounded(U.F32, b["dx"]), rounded(U.F32, b["dy"]), P, alpha, O.EQ(), lam,
                                   eps, iters)
    print("block-kernel launches:", n, U.autotune_table())
    assert rel_err(to_np(lh), lho) <= TOL
    assert rel_err(to_np(Vg), Vo.reshape(4, -1)) <= TOL


def test_block_condition_falls_back():
    """Where k2 h^2 dmax^2 > 90 (a 32-point block too wide at this eps) the
    forced block tile is not run: the log-sum-exp tile computes the pass."""
    og, lg, dx, dy, p, q = uniform_problem((64,), (64,), (1 / 16,), (0,), 4)
    eps = 0.002  # k2 h^2 31^2 = 721 x 3.75 > 90
    W = rounded(U.F32, np.zeros(64))
    U.force_grid_tile(9)
    try:
        got, n = blk_launches(lambda: U.gibbs_log(lg(), T(W, U.F32), T(dy, U.F32), eps, False, U.F32))
    finally:
        U.force_grid_tile(-1)
    assert n == 0
    want = O.apply_K_log(round_geom(og, U.F32), W, np.log(rounded(U.F32, dy)), eps)
    assert rel_err(to_np(got), want) <= TOL


def test_non_uniform_axes_fall_back():
    """Cell centres of 300 points are not x0 + i h exactly in FP32: no block pass."""
    xs = [synth.grid_axis(300)]
    geo = U.Geometry.grid([T(a, U.F32) for a in xs])
    W = torch.zeros(300, dtype=torch.float32, device="cuda")
    w = torch.full((300,), 1 / 300, dtype=torch.float32, device="cuda")
    U.force_grid_tile(9)
    try:
        _, n = blk_launches(lambda: U.gibbs_log(geo, W, w, 0.05, False, U.F32))
    finally:
        U.force_grid_tile(-1)
    assert n == 0


def test_tuner_never_picks_the_block_pass():
    """On a uniform grid where every block variant is admitted and timed, the
    automatic choice is a log-sum-exp tile and no block kernel runs."""
    og, lg, dx, dy, p, q = uniform_problem((96, 80), (96, 80), (1 / 128, 1 / 128), (0, 0), 5)
    prev = U.set_autotune(1)
    try:
        W = rounded(U.F32, np.zeros((96, 80)))
        _, n = blk_launches(lambda: U.gibbs_log(lg(), T(W, U.F32).ravel(), T(dy, U.F32).ravel(), 0.05, False,
                                                U.F32))
        table = U.autotune_table()
    finally:
        U.set_autotune(prev)
    lines = [ln for ln in table.splitlines() if "nin=80 nout=80" in ln]
    assert lines and all("blk32x4:-1.00us" not in ln for ln in lines), table  # admitted and timed
    assert all("-> block-stabilised" not in ln for ln in lines), table
    assert n == 0

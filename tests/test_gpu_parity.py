"""GPU parity: the CUDA library (through the C ABI) against the FP64 oracle on
the same seeded inputs, element by element.

Tolerances (relative to max(1, |reference|_inf) on log-potentials, as the
accuracy targets state): FP64 path 1e-10, FP32 path 1e-5.  Sizes span several
CTA tiles with ragged tails (64 outputs and 4 lines per CTA for grid passes,
8 rows per CTA for row kernels).
"""
import math

import numpy as np
import pytest
import torch

import oracle as O
from paper_1607_05816_gb300 import synth
from paper_1607_05816_gb300 import uot as U

pytestmark = [pytest.mark.gpu, pytest.mark.filterwarnings("ignore::RuntimeWarning")]

TOL = {U.F64: 1e-10, U.F32: 1e-5}
DEV = "cuda"


def T(a, prec):
    return torch.as_tensor(np.ascontiguousarray(a), dtype=U._dtype(prec), device=DEV)


def rounded(prec, *arrays):
    """The inputs exactly as the library receives them in this precision (an
    FP32 call sees FP32-rounded densities, weights and coordinates; tiny
    densities may become exact zeros), as float64 for the oracle."""
    dt = np.float64 if prec == U.F64 else np.float32
    out = [np.asarray(a, dtype=dt).astype(np.float64) for a in arrays]
    return out if len(out) > 1 else out[0]


def rel_err(got, want):
    got = np.asarray(got, dtype=np.float64).ravel()
    want = np.asarray(want, dtype=np.float64).ravel()
    assert np.array_equal(np.isneginf(got), np.isneginf(want)), "-inf pattern differs"
    f = np.isfinite(want)
    if not f.any():
        return 0.0
    return float(np.max(np.abs(got[f] - want[f])) / max(1.0, np.max(np.abs(want[f]))))


def to_np(t):
    return t.detach().double().cpu().numpy()


# ----------------------------------------------------------------------------
# problem builders: (oracle geometry, library geometry factory, dx, dy, p, q)
# ----------------------------------------------------------------------------

def grid_problem(shape_x, shape_y, seed, zeros=True):
    g = synth.rng(seed)
    xs = [synth.grid_axis(n) for n in shape_x]
    ys = [synth.grid_axis(n) for n in shape_y]
    dx = np.full(shape_x, 1.0 / np.prod(shape_x))
    dy = np.full(shape_y, 1.0 / np.prod(shape_y))
    p = g.uniform(0.2, 2.0, size=shape_x)
    q = g.uniform(0.2, 2.0, size=shape_y)
    if zeros:
        p.ravel()[:: 7] = 0.0
        q.ravel()[3:: 11] = 0.0
    p *= 1.0 / np.sum(p * dx)
    q *= 1.3 / np.sum(q * dy)
    og = O.Geometry("grid", xs=xs, ys=ys)

    def lg(prec):
        return U.Geometry.grid([T(a, prec) for a in xs], [T(a, prec) for a in ys])
    return og, lg, dx, dy, p, q


def points_problem(n, m, d, seed):
    g = synth.rng(seed)
    x = synth.mixture_points(g, n, d, 4)
    y = synth.mixture_points(g, m, d, 4)
    og = O.Geometry("points", x=x, y=y)

    def lg(prec):
        return U.Geometry.points(T(x, prec), T(y, prec))
    return og, lg, np.full(n, 1.0 / n), np.full(m, 1.0 / m), np.full(n, 1.0), np.full(m, 0.7)


def dense_problem(n, m, seed):
    d = synth.problem_1d(n, m, seed=seed)
    C = O.sqdist(d["x"], d["y"])
    og = O.Geometry("dense", C=C)

    def lg(prec):
        return U.Geometry.dense(T(C, prec))
    return og, lg, d["dx"], d["dy"], d["p"], d["q"]


# ----------------------------------------------------------------------------
# the Gibbs operator alone
# ----------------------------------------------------------------------------

GIBBS_CASES = [
    ("grid2d", lambda: grid_problem((70, 45), (33, 129), 1)),
    ("grid1d", lambda: grid_problem((300,), (257,), 2)),
    ("grid3d", lambda: grid_problem((9, 13, 6), (7, 5, 11), 3)),
    ("points", lambda: points_problem(301, 260, 3, 4)),
    ("dense", lambda: dense_problem(97, 130, 5)),
]


@pytest.mark.parametrize("prec", [U.F64, U.F32])
@pytest.mark.parametrize("name,make", GIBBS_CASES)
@pytest.mark.parametrize("transpose", [False, True])
def test_gibbs_log_parity(name, make, prec, transpose):
    og, lg, dx, dy, p, q = make()
    g = synth.rng(9)
    eps = 0.01
    shape_in = np.shape(dx) if transpose else np.shape(dy)
    W = g.normal(size=shape_in) * 0.05
    W.ravel()[5:: 13] = -np.inf
    w = dx if transpose else dy
    W, w = rounded(prec, W, w)
    want = O.apply_K_log(round_geom(og, prec), W, np.log(w), eps, transpose=transpose)
    got = U.gibbs_log(lg(prec), T(W, prec).ravel(), T(w, prec).ravel(), eps, transpose, prec)
    assert rel_err(to_np(got), want) <= TOL[prec]


def test_gibbs_all_zero_line():
    """A whole grid line with b = 0 yields empty sums (-inf), not NaN."""
    og, lg, dx, dy, p, q = grid_problem((20, 24), (20, 24), 6)
    W = np.zeros((20, 24))
    W[3, :] = -np.inf
    W[:, 5] = -np.inf
    want = O.apply_K_log(og, W, np.log(dy), 0.02)
    for prec in (U.F64, U.F32):
        got = U.gibbs_log(lg(prec), T(W, prec).ravel(), T(dy, prec).ravel(), 0.02, False, prec)
        assert rel_err(to_np(got), want) <= TOL[prec]
    W[:] = -np.inf
    got = U.gibbs_log(lg(U.F64), T(W, U.F64).ravel(), T(dy, U.F64).ravel(), 0.02, False, U.F64)
    assert np.all(np.isneginf(to_np(got)))


# ----------------------------------------------------------------------------
# iterations: U, V at equal iteration counts
# ----------------------------------------------------------------------------

DIVS = [
    (O.KL(0.5), O.KL(0.5), U.KL(0.5), U.KL(0.5)),
    (O.TV(0.1), O.KL(0.1), U.TV(0.1), U.KL(0.1)),
    (O.RG(0.7, 1.2), O.TV(0.3), U.RG(0.7, 1.2), U.TV(0.3)),
    (O.EQ(), O.KL(1.0), U.EQ(), U.KL(1.0)),
    (O.RG(0.0, math.inf), O.RG(0.5, 2.0), U.RG(0.0, math.inf), U.RG(0.5, 2.0)),
]


def round_geom(og, prec):
    if og.kind == "dense":
        return O.Geometry("dense", C=rounded(prec, og.C))
    if og.kind == "points":
        return O.Geometry("points", x=rounded(prec, og.x), y=rounded(prec, og.y))
    return O.Geometry("grid", xs=[rounded(prec, a) for a in og.xs], ys=[rounded(prec, a) for a in og.ys])


def run_both(og, lg, dx, dy, p, q, divs, eps, iters, prec, eps_start=None, stages=0, ips=0):
    OF1, OF2, UF1, UF2 = divs
    rdx, rdy, rp, rq = rounded(prec, dx, dy, p, q)
    r = O.solve_log(round_geom(og, prec), rdx, rdy, rp, rq, OF1, OF2, eps, max_iter=iters,
                    eps_start=eps_start, stages=stages, iters_per_stage=ips)
    Ug, Vg, info = U.solve(lg(prec), T(p, prec).ravel(), T(dx, prec).ravel(), T(q, prec).ravel(),
                           T(dy, prec).ravel(), UF1, UF2, eps, precision=prec, max_iter=iters,
                           eps_start=eps_start, eps_stages=stages, iters_per_stage=ips)
    return r, to_np(Ug), to_np(Vg), info


@pytest.mark.parametrize("prec", [U.F64, U.F32])
@pytest.mark.parametrize("divs", DIVS, ids=["kl-kl", "tv-kl", "rg-tv", "eq-kl", "rg-rg"])
def test_solve_grid_parity(divs, prec):
    og, lg, dx, dy, p, q = grid_problem((40, 67), (52, 38), 10)
    r, Ug, Vg, info = run_both(og, lg, dx, dy, p, q, divs, 0.01, 30, prec)
    assert info["iters"] == 30
    assert rel_err(Ug, r["U"]) <= TOL[prec]
    assert rel_err(Vg, r["V"]) <= TOL[prec]


@pytest.mark.parametrize("prec", [U.F64, U.F32])
def test_degenerate_penalties(prec):
    """Degenerate rows of Table 1 as F1, with F2 = KL(0.5): RG with
    alpha = beta = 1 is the equality constraint; TV with lambda far above every
    |U| never clamps, which is the equality update too; KL with a huge lambda
    tends to it.  Each matches the oracle after 30 iterations, and the first
    two reproduce the solve with F1 = EQ."""
    og, lg, dx, dy, p, q = grid_problem((40, 67), (52, 38), 13, zeros=False)
    F2 = (O.KL(0.5), U.KL(0.5))
    _, Ueq, Veq, _ = run_both(og, lg, dx, dy, p, q, (O.EQ(), F2[0], U.EQ(), F2[1]), 0.01, 30, prec)
    for OF, UF, like_eq in ((O.RG(1.0, 1.0), U.RG(1.0, 1.0), True), (O.TV(1e8), U.TV(1e8), True),
                            (O.KL(1e8), U.KL(1e8), False)):
        r, Ug, Vg, info = run_both(og, lg, dx, dy, p, q, (OF, F2[0], UF, F2[1]), 0.01, 30, prec)
        assert info["iters"] == 30
        assert rel_err(Ug, r["U"]) <= TOL[prec]
        assert rel_err(Vg, r["V"]) <= TOL[prec]
        if like_eq:
            assert rel_err(Ug, Ueq) <= TOL[prec]
            assert rel_err(Vg, Veq) <= TOL[prec]


@pytest.mark.parametrize("prec", [U.F64, U.F32])
def test_solve_grid_eps_scaling_parity(prec):
    """eps-scaling stages (Sec. 4.4) then iterations at the final eps."""
    og, lg, dx, dy, p, q = grid_problem((48, 48), (48, 48), 11, zeros=False)
    r, Ug, Vg, info = run_both(og, lg, dx, dy, p, q, DIVS[0], 1e-3, 20, prec,
                               eps_start=0.1, stages=10, ips=5)
    assert info["total_iters"] == 70
    assert rel_err(Ug, r["U"]) <= TOL[prec]
    assert rel_err(Vg, r["V"]) <= TOL[prec]


@pytest.mark.parametrize("prec", [U.F64, U.F32])
@pytest.mark.parametrize("divs", DIVS[:3], ids=["kl-kl", "tv-kl", "rg-tv"])
def test_solve_points_parity(divs, prec):
    og, lg, dx, dy, p, q = points_problem(333, 250, 3, 12)
    r, Ug, Vg, info = run_both(og, lg, dx, dy, p, q, divs, 0.01, 25, prec)
    assert rel_err(Ug, r["U"]) <= TOL[prec]
    assert rel_err(Vg, r["V"]) <= TOL[prec]


@pytest.mark.parametrize("prec", [U.F64, U.F32])
def test_solve_dense_parity(prec):
    og, lg, dx, dy, p, q = dense_problem(256, 256, 1234)
    r, Ug, Vg, info = run_both(og, lg, dx, dy, p, q, DIVS[0], 1e-2, 50, prec)
    assert rel_err(Ug, r["U"]) <= TOL[prec]
    assert rel_err(Vg, r["V"]) <= TOL[prec]


@pytest.mark.parametrize("launch_mode", [0, 1])
def test_plain_scaling_alg1_parity(launch_mode):
    """Algorithm 1 (no stabilisation) on the dense 1-D problem: 256 points,
    KL lambda = 1 both sides, eps = 1e-2, FP64, 2000 iterations, against the
    oracle's Algorithm 1 run verbatim; per-launch (0) and as one launch of a
    cluster holding K in shared memory (1, the benchmark's configuration)."""
    d = synth.problem_1d(256, 256, seed=1234)
    C = O.sqdist(d["x"], d["y"])
    eps, iters = 1e-2, 2000
    a, b = O.scaling_alg1(np.exp(-C / eps), d["dx"], d["dy"], d["p"], d["q"], O.KL(1.0), O.KL(1.0), eps, iters)
    n0 = U.launch_count()
    Ug, Vg, info = U.solve(U.Geometry.dense(T(C, U.F64)), T(d["p"], U.F64), T(d["dx"], U.F64),
                           T(d["q"], U.F64), T(d["dy"], U.F64), U.KL(1.0), U.KL(1.0), eps,
                           precision=U.F64, max_iter=iters, plain_scaling=True, launch_mode=launch_mode)
    assert rel_err(to_np(Ug), eps * np.log(a)) <= 1e-10
    assert rel_err(to_np(Vg), eps * np.log(b)) <= 1e-10
    assert info["iters"] == iters
    if launch_mode == 1:
        assert U.launch_count() - n0 < 20  # one solve launch, not 2 per iteration


@pytest.mark.parametrize("n,m,F1,F2", [
    (256, 256, U.KL(1.0), U.KL(0.5)),
    (100, 37, U.TV(0.05), U.KL(0.3)),     # ragged bands: 7 rows of K, 3 of K^T per CTA
    (5, 300, U.RG(0.7, 1.4), U.EQ()),      # most CTAs own no row of K
    (600, 600, U.KL(1.0), U.KL(1.0)),     # does not fit: the per-launch path runs
])
def test_alg1_cluster_same_iterates_as_per_launch(n, m, F1, F2):
    """launch_mode 1 of Algorithm 1 gives the per-launch path's iterates bit
    for bit (the same sums in the same order), with eps-scaling stages, the
    tolerance stop (checked every 7 iterations) and the violation it reports."""
    d = synth.problem_1d(n, m, seed=n + m)
    C = O.sqdist(d["x"], d["y"])
    geo = U.Geometry.dense(T(C, U.F64))
    args = [T(d[k], U.F64) for k in ("p", "dx", "q", "dy")]
    if F1.kind == U.DIV_EQ or F2.kind == U.DIV_EQ:
        args[2] = args[2] * (torch.sum(args[0] * args[1]) / torch.sum(args[2] * args[3]))
    outs = []
    for mode in (0, 1):
        outs.append(U.solve(geo, *args, F1, F2, 0.02, precision=U.F64, max_iter=3000, tol=1e-9, check_every=7,
                            eps_start=0.2, eps_stages=3, iters_per_stage=20, plain_scaling=True,
                            launch_mode=mode))
    (U0, V0, i0), (U1, V1, i1) = outs
    assert torch.equal(U0, U1) and torch.equal(V0, V1)
    assert i0["iters"] == i1["iters"] and i0["total_iters"] == i1["total_iters"] == i0["iters"] + 60
    assert i0["status"] == i1["status"]
    assert abs(i0["marg_err"] - i1["marg_err"]) <= 1e-12 * max(1.0, abs(i0["marg_err"]))


def test_tolerance_stop_matches_oracle():
    """The stopping rule (violation measured in the next a-update) stops at the
    same iteration as the oracle's solve_log and reports the same violation."""
    og, lg, dx, dy, p, q = dense_problem(120, 90, 77)
    r = O.solve_log(og, dx, dy, p, q, O.KL(0.3), O.KL(0.3), 0.02, max_iter=5000, tol=1e-8, check_every=7)
    Ug, Vg, info = U.solve(lg(U.F64), T(p, U.F64), T(dx, U.F64), T(q, U.F64), T(dy, U.F64),
                           U.KL(0.3), U.KL(0.3), 0.02, precision=U.F64, max_iter=5000, tol=1e-8,
                           check_every=7)
    assert info["status"] == "UOT_OK"
    assert info["iters"] == r["iters"]
    assert abs(info["marg_err"] - r["err"]) <= 1e-6 * r["err"]
    assert rel_err(to_np(Ug), r["U"]) <= 1e-10


# ----------------------------------------------------------------------------
# plan application and objective
# ----------------------------------------------------------------------------

@pytest.mark.parametrize("prec", [U.F64, U.F32])
def test_apply_plan_marginals_and_projection(prec):
    og, lg, dx, dy, p, q = grid_problem((21, 34), (30, 17), 13, zeros=False)
    r = O.solve_log(og, dx, dy, p, q, O.KL(0.5), O.KL(0.5), 0.02, max_iter=40)
    r1, r2 = O.marginals(og, dx.ravel(), dy.ravel(), r["U"].ravel(), r["V"].ravel(), 0.02)
    geo = lg(prec)
    Ut, Vt = T(r["U"], prec).ravel(), T(r["V"], prec).ravel()
    g1 = U.apply_plan(geo, Ut, Vt, 0.02, T(dx, prec).ravel(), T(dy, prec).ravel(), precision=prec)
    g2 = U.apply_plan(geo, Ut, Vt, 0.02, T(dx, prec).ravel(), T(dy, prec).ravel(), transpose=True, precision=prec)
    tol = 1e-10 if prec == U.F64 else 2e-4
    assert np.max(np.abs(to_np(g1)[:, 0] - r1) / r1) <= tol
    assert np.max(np.abs(to_np(g2)[:, 0] - r2) / r2) <= tol
    # barycentric projection numerator R (y . dy): coordinates as nonnegative f
    Y = O.grid_points(og.ys)
    R = np.exp(O.log_plan(og, r["U"], r["V"], 0.02))
    want = R @ (Y * dy.ravel()[:, None])
    got = U.apply_plan(geo, Ut, Vt, 0.02, T(dx, prec).ravel(), T(dy, prec).ravel(), f=T(Y, prec), precision=prec)
    assert np.max(np.abs(to_np(got) - want) / want) <= tol


@pytest.mark.parametrize("divs", [DIVS[0], DIVS[1], (O.TV(0.2), O.TV(0.3), U.TV(0.2), U.TV(0.3))], ids=["kl", "tv-kl", "tv"])
def test_objective_parity(divs):
    OF1, OF2, UF1, UF2 = divs
    og, lg, dx, dy, p, q = points_problem(90, 70, 2, 14)
    eps = 0.05
    r = O.solve_log(og, dx, dy, p, q, OF1, OF2, eps, max_iter=60)
    P = O.primal(og, dx, dy, p, q, OF1, OF2, eps, r["U"], r["V"])
    D = O.dual(og, dx, dy, p, q, OF1, OF2, eps, r["U"], r["V"])
    err = O.marginal_violation(og, dx, dy, p, q, OF1, OF2, eps, r["U"], r["V"])
    got = U.objective(lg(U.F64), T(p, U.F64), T(dx, U.F64), T(q, U.F64), T(dy, U.F64), UF1, UF2,
                      eps, T(r["U"], U.F64), T(r["V"], U.F64))
    assert abs(got["primal"] - P) <= 1e-10 * max(1, abs(P))
    assert abs(got["dual"] - D) <= 1e-10 * max(1, abs(D))
    assert abs(got["gap"] - (P - D)) <= 1e-10 * max(1, abs(P))
    assert abs(got["marg_err"] - err) <= 1e-8 * err + 1e-14


# ----------------------------------------------------------------------------
# barycenters
# ----------------------------------------------------------------------------

@pytest.mark.parametrize("prec", [U.F64, U.F32])
@pytest.mark.parametrize("kind", [U.BARY_KL, U.BARY_EQ])
def test_barycenter_parity(kind, prec):
    d = synth.barycenter_images(K=5, H=24, W=36, seed=15)
    og = O.Geometry("grid", xs=d["xs"], ys=d["ys"])
    alpha = np.array([0.1, 0.3, 0.2, 0.25, 0.15])
    eps, lam, iters = 0.01, 1.0, 25
    Uo, Vo, lho = O.barycenter_log(og, d["dx"], d["dy"], d["P"], alpha, O.EQ(), lam, eps, iters,
                                   bary_kind="kl" if kind == U.BARY_KL else "eq")
    geo = U.Geometry.grid([T(a, prec) for a in d["xs"]])
    lh, Ug, Vg, info = U.barycenter(geo, alpha, T(d["P"].reshape(5, -1), prec), T(d["dx"], prec).ravel(),
                                    T(d["dy"], prec).ravel(), U.EQ(), lam, eps, kind=kind,
                                    precision=prec, max_iter=iters)
    assert rel_err(to_np(lh), lho) <= TOL[prec]
    assert rel_err(to_np(Ug), Uo.reshape(5, -1)) <= TOL[prec]
    assert rel_err(to_np(Vg), Vo.reshape(5, -1)) <= TOL[prec]


# ----------------------------------------------------------------------------
# argument checking (host side, nothing launched)
# ----------------------------------------------------------------------------

def test_empty_inputs_rejected():
    """Empty inputs are argument errors (EINVAL) found on the host before any
    launch: a cost with no rows or no columns, a point cloud without points, a
    grid with an axis of length 0 (solve, Gibbs operator, Algorithm 4,
    barycentric map), a histogram or bin map of no points, a batch without
    problems or with an empty one."""
    f64, dev = torch.float64, "cuda"
    z = lambda *sh: torch.zeros(*sh, dtype=f64, device=dev)
    o = lambda *sh: torch.ones(*sh, dtype=f64, device=dev)
    geoms = [
        U.Geometry.dense(z(0, 16)),
        U.Geometry.dense(z(16, 0)),
        U.Geometry.points(z(0, 2), z(16, 2)),
        U.Geometry.points(z(16, 2), z(0, 2)),
        U.Geometry.grid([z(0), o(4)], [o(4), o(4)]),
    ]
    for geo in geoms:
        p, q = o(geo.n), o(geo.m)
        with pytest.raises(U.UotError, match="EINVAL"):
            U.solve(geo, p, p, q, q, U.KL(1.0), U.KL(1.0), 0.1)
        with pytest.raises(U.UotError, match="EINVAL"):
            U.gibbs_log(geo, q, q, 0.1)
        with pytest.raises(U.UotError, match="EINVAL"):
            U.solve_mass(geo, p, p, q, q, U.KL(1.0), U.KL(1.0), U.EQ(), 1.0, 0.1)
        if geo.kind != U.GEOM_DENSE:
            with pytest.raises(U.UotError, match="EINVAL"):
                U.barycentric_map(geo, p, q, 0.1, p, q)
    pts = torch.zeros(0, 3, dtype=torch.float32, device=dev)
    with pytest.raises(U.UotError, match="EINVAL"):
        U.histogram(pts, (4, 4, 4))
    with pytest.raises(U.UotError, match="EINVAL"):
        U.apply_bin_map(pts, (4, 4, 4), z(64, 3))
    f32 = lambda n, *r: torch.ones(n, *r, dtype=torch.float32, device=dev)
    with pytest.raises(U.UotError, match="EINVAL"):
        U.solve_batch([(3, 0)], [(U.KL(1.0), U.KL(1.0))], 2, f32(3, 2), f32(3), f32(3), f32(1, 2), f32(1), f32(1),
                      0.1)
    with pytest.raises((U.UotError, ValueError)):
        U.solve_batch([], [], 2, f32(1, 2), f32(1), f32(1), f32(1, 2), f32(1), f32(1), 0.1)
    # past the largest size: the histogram's 32-bit counters take at most 2^32 - 1
    # points (rejected before the buffer is touched)
    import ctypes
    real, hist = torch.zeros(8, 3, dtype=torch.float32, device=dev), z(64)
    sh = (ctypes.c_int * 3)(4, 4, 4)
    rc = U.load().uot_histogram(real.data_ptr(), 2**32, 3, sh, U.F64, hist.data_ptr(), None)
    assert U.STATUS[rc] == "UOT_EINVAL"


def test_invalid_arguments_rejected():
    og, lg, dx, dy, p, q = dense_problem(16, 16, 3)
    geo = lg(U.F64)
    args = (T(p, U.F64), T(dx, U.F64), T(q, U.F64), T(dy, U.F64))
    with pytest.raises(U.UotError, match="EINVAL"):
        U.solve(geo, *args, U.KL(-1.0), U.KL(1.0), 0.1)
    with pytest.raises(U.UotError, match="EINVAL"):
        U.solve(geo, *args, U.KL(1.0), U.KL(1.0), 0.0)
    with pytest.raises(U.UotError, match="EINVAL"):
        U.solve(geo, *args, U.RG(2.0, 1.0), U.KL(1.0), 0.1)
    with pytest.raises(U.UotError, match="EUNSUPPORTED"):
        gp = grid_problem((8,), (8,), 1)
        U.solve(gp[1](U.F64), T(gp[4], U.F64), T(gp[2], U.F64), T(gp[5], U.F64), T(gp[3], U.F64),
                U.KL(1.0), U.KL(1.0), 0.1, plain_scaling=True)


@pytest.mark.parametrize("prec,tile", [(U.F64, -1), (U.F32, -1), (U.F32, 0), (U.F32, 8)])
def test_grid_at_the_pass_line_limit(prec, tile):
    """Largest grid passes.  On a 2 x 255 x 257 grid the pass along the first
    axis runs over 255 * 257 = 65535 lines, the most one launch grid holds:
    the operator matches the oracle in both directions, with the tuner's
    choice, the first SIMT tile, and the warp-per-line pass (which takes the
    2-point pass; the long axes fall back to the first tile).  One line past
    the limit (2 x 256 x 256), or an axis longer than 3000 points, is refused
    on the host with a message, before any launch."""
    shape = (2, 255, 257)
    og, lg, dx, dy, p, q = grid_problem(shape, shape, 41, zeros=False)
    g = synth.rng(43)
    eps = 0.01
    U.force_grid_tile(tile)
    try:
        for transpose in (False, True):
            W = g.normal(size=shape) * 0.05
            W.ravel()[5:: 13] = -np.inf
            w = dx if transpose else dy
            W, w = rounded(prec, W, w)
            want = O.apply_K_log(round_geom(og, prec), W, np.log(w), eps, transpose=transpose)
            got = U.gibbs_log(lg(prec), T(W, prec).ravel(), T(w, prec).ravel(), eps, transpose, prec)
            assert rel_err(to_np(got), want) <= TOL[prec]
    finally:
        U.force_grid_tile(-1)
    for sx, sy, why in (((2, 256, 256), (2, 256, 256), "65535 lines"), ((3001,), (4,), "3000 points")):
        _, lg2, dx2, dy2, p2, q2 = grid_problem(sx, sy, 5, zeros=False)
        geo = lg2(prec)
        with pytest.raises(U.UotError, match="EUNSUPPORTED.*" + why):
            U.gibbs_log(geo, T(q2, prec).ravel(), T(dy2, prec).ravel(), eps, False, prec)
        with pytest.raises(U.UotError, match="EUNSUPPORTED.*" + why):
            U.solve(geo, *[T(a, prec).ravel() for a in (p2, dx2, q2, dy2)], U.KL(1.0), U.KL(1.0), eps,
                    precision=prec, max_iter=5)


@pytest.mark.parametrize("shape", [(48, 64), (9, 13, 6), (300,)])
def test_persistent_launch_matches_per_pass_launches(shape):
    """The persistent cooperative solve and the one-launch-per-pass solve run
    the same arithmetic: identical iterates, the same stopping iteration and
    violation (eps-scaling, tolerance stop)."""
    og, lg, dx, dy, p, q = grid_problem(shape, shape, 31, zeros=False)
    args = [T(a, U.F32).ravel() for a in (p, dx, q, dy)]
    outs = []
    U.force_grid_tile(0)  # the persistent solve runs the first tile shape
    try:
        for mode in (1, 0):
            outs.append(U.solve(lg(U.F32), *args, U.KL(0.5), U.KL(0.5), 2e-3, precision=U.F32, max_iter=3000,
                                tol=1e-5, check_every=10, eps_start=0.1, eps_stages=5, iters_per_stage=20,
                                launch_mode=mode))
    finally:
        U.force_grid_tile(-1)
    (U0, V0, i0), (U1, V1, i1) = outs
    assert i0["iters"] == i1["iters"] and i0["total_iters"] == i1["total_iters"]
    assert i0["status"] == i1["status"] == "UOT_OK"
    assert abs(i0["marg_err"] - i1["marg_err"]) <= 1e-9
    assert torch.equal(U0, U1) and torch.equal(V0, V1)


# ----------------------------------------------------------------------------
# FP32 grid-pass tile shapes and the tuner
# ----------------------------------------------------------------------------

@pytest.mark.parametrize("tile", range(14))
@pytest.mark.parametrize("name,make", GIBBS_CASES[:3])
def test_every_grid_tile_matches_oracle(tile, name, make):
    """Every tile shape the tuner may pick computes the operator and a short
    KL/TV solve to the FP32 tolerance (ragged lines and outputs included).
    Tile 7 is the tensor-core pass, which these coarse grids at eps = 0.01
    do not admit (the SIMT tile runs instead); tile 8 is the warp-per-line
    pass, which runs where lines and outputs are at most 64 long (every pass
    of the 3-D case, some of the 2-D one); tiles 9-13 are the block-stabilised
    pass of uniform axes, which these cell-centre axes (not x0 + i h exactly
    in FP32 for 300 or 45 points) do not admit (tests/test_gpu_blk.py covers it)."""
    assert U.grid_tile_count() == 14
    og, lg, dx, dy, p, q = make()
    g = synth.rng(19)
    eps = 0.01
    U.force_grid_tile(tile)
    try:
        for transpose in (False, True):
            shape_in = np.shape(dx) if transpose else np.shape(dy)
            W = g.normal(size=shape_in) * 0.05
            W.ravel()[5:: 13] = -np.inf
            w = dx if transpose else dy
            W, w = rounded(U.F32, W, w)
            want = O.apply_K_log(round_geom(og, U.F32), W, np.log(w), eps, transpose=transpose)
            got = U.gibbs_log(lg(U.F32), T(W, U.F32).ravel(), T(w, U.F32).ravel(), eps, transpose, U.F32)
            assert rel_err(to_np(got), want) <= TOL[U.F32]
        dxr, dyr, pr, qr = rounded(U.F32, dx, dy, p, q)
        Ug, Vg, _ = U.solve(lg(U.F32), *[T(a, U.F32).ravel() for a in (pr, dxr, qr, dyr)], U.KL(0.7),
                            U.TV(0.4), eps, precision=U.F32, max_iter=12)
        r = O.solve_log(round_geom(og, U.F32), dxr, dyr, pr, qr, O.KL(0.7), O.TV(0.4), eps, max_iter=12)
        assert rel_err(to_np(Ug), r["U"]) <= TOL[U.F32]
        assert rel_err(to_np(Vg), r["V"]) <= TOL[U.F32]
    finally:
        U.force_grid_tile(-1)


def test_short_line_pass_batched():
    """The warp-per-line pass (tile 8) on a batch of problems whose lines do
    not fill a block (a block's warps straddle batch entries): potentials after
    20 iterations match the oracle problem by problem, and with a tolerance the
    per-entry violation sums stop where the general tile's do (within one
    check block: the two tiles round differently)."""
    g = synth.rng(61)
    shape = (16, 8, 5)  # 40, 80 and 128 lines: blocks of 8 warps straddle the 7 entries
    xs = [synth.grid_axis(n) for n in shape]
    B = 7
    dx = np.full(shape, 1.0 / np.prod(shape))
    P = g.uniform(0.2, 2.0, size=(B,) + shape)
    Q = g.uniform(0.2, 2.0, size=(B,) + shape)
    P[2].ravel()[::5] = 0.0
    og = O.Geometry("grid", xs=xs, ys=xs)
    rd = lambda a: rounded(U.F32, a)
    geo = U.Geometry.grid([T(a, U.F32) for a in xs], [T(a, U.F32) for a in xs])
    args = (T(P.reshape(B, -1), U.F32), T(dx, U.F32).ravel(), T(Q.reshape(B, -1), U.F32), T(dx, U.F32).ravel())
    stops = {}
    for tile in (8, 0):
        U.force_grid_tile(tile)
        try:
            Ug, Vg, _ = U.solve_many(geo, *args, U.KL(0.5), U.TV(0.3), 0.02, precision=U.F32, max_iter=20)
            if tile == 8:
                for k in range(B):
                    r = O.solve_log(round_geom(og, U.F32), rd(dx), rd(dx), rd(P[k]), rd(Q[k]), O.KL(0.5),
                                    O.TV(0.3), 0.02, max_iter=20)
                    assert rel_err(to_np(Ug[k]), r["U"]) <= TOL[U.F32]
                    assert rel_err(to_np(Vg[k]), r["V"]) <= TOL[U.F32]
            _, _, info = U.solve_many(geo, *args, U.KL(0.5), U.TV(0.3), 0.02, precision=U.F32, max_iter=4000,
                                      tol=1e-6, check_every=10)
        finally:
            U.force_grid_tile(-1)
        assert info["status"] == "UOT_OK"
        stops[tile] = (info["iters"], info["marg_err"])
    assert abs(stops[8][0] - stops[0][0]) <= 10
    assert stops[8][1] <= 1e-6 and stops[0][1] <= 1e-6


def test_autotuner_records_choice_and_keeps_parity():
    """First use of a new pass shape times every tile and records the fastest
    eligible one (the block-stabilised variants are timed but only run when
    forced); the tuned pass still matches the oracle."""
    prev = U.set_autotune(1)
    try:
        og, lg, dx, dy, p, q = grid_problem((57, 83), (61, 79), 23)
        g = synth.rng(21)
        W = g.normal(size=(61, 79)) * 0.05
        W, w = rounded(U.F32, W, dy)
        got = U.gibbs_log(lg(U.F32), T(W, U.F32).ravel(), T(w, U.F32).ravel(), 0.02, False, U.F32)
        want = O.apply_K_log(round_geom(og, U.F32), W, np.log(w), 0.02)
        assert rel_err(to_np(got), want) <= TOL[U.F32]
        table = U.autotune_table()
        lines = [ln for ln in table.splitlines() if "nin=79 nout=83" in ln and "lines=61" in ln]
        assert len(lines) == 1, table
        times = [float(t.split(":")[1][:-2]) for t in lines[0].split(";")[1].split()]
        assert len(times) == 14 and all(t > 0 for t in times[:7])
        # tc3, short lines and the block pass (cell-centre axes of 83 and 79 points) not admitted
        times = [t if t > 0 else math.inf for t in times]
        chosen = lines[0].split("-> ")[1].split(";")[0]
        names = ["warps=%d outputs/lane=%d" % sh for sh in [(8, 4), (4, 4), (2, 4), (1, 4), (8, 2), (4, 2), (2, 2)]]
        names += ["tensor-core tc3", "warp per line"]
        names += ["block-stabilised " + v for v in ("blk32x2", "blk32x4", "blk32x8", "blk64x2", "blk64x4")]
        k = names.index(chosen)
        assert k < 9  # the block variants are never chosen automatically
        tb = min(times[:9])
        tick = 0.011  # the table prints times to 0.01 us: ties at that precision may go either way
        if k == 0:  # the first tile is kept unless another one is more than 5% faster
            assert times[0] <= 1.05 * tb + tick
        else:
            assert times[k] <= tb + tick and times[0] >= 1.05 * times[k] - tick
    finally:
        U.set_autotune(prev)


@pytest.mark.parametrize("prec", [U.F32, U.F64])
@pytest.mark.parametrize("name,make", [("grid2d", lambda: grid_problem((48, 64), (48, 64), 33, zeros=False)),
                                       ("points", lambda: points_problem(301, 260, 3, 4))])
def test_graph_blocks_match_per_pass_launches(name, make, prec):
    """launch_mode 2 (CUDA-graph replay of check_every-iteration blocks) runs
    the same kernels in the same order as per-pass launches: identical
    iterates, stopping iteration and violation; the launch counter counts
    the replayed kernels."""
    og, lg, dx, dy, p, q = make()
    args = [T(a, prec).ravel() for a in (p, dx, q, dy)]
    outs = []
    for mode in (2, 0):
        n0 = U.launch_count()
        r = U.solve(lg(prec), *args, U.KL(0.5), U.KL(0.5), 5e-3, precision=prec, max_iter=3000, tol=1e-6,
                    check_every=10, eps_start=0.1, eps_stages=4, iters_per_stage=15, launch_mode=mode)
        outs.append(r + (U.launch_count() - n0,))
    (U0, V0, i0, n0), (U1, V1, i1, n1) = outs
    assert i0["status"] == i1["status"] == "UOT_OK"
    assert i0["iters"] == i1["iters"] and i0["total_iters"] == i1["total_iters"]
    assert i0["iters"] > 30  # several replayed blocks
    # the violation is summed with one atomic per CTA: its last bits depend on the arrival order
    assert abs(i0["marg_err"] - i1["marg_err"]) <= 1e-12
    assert torch.equal(U0, U1) and torch.equal(V0, V1)
    assert n0 == n1


@pytest.mark.parametrize("shape_x,shape_y", [((48, 64), (48, 64)), ((37, 70), (45, 29)), ((130, 300), (140, 260))])
@pytest.mark.parametrize("divs", [DIVS[0], DIVS[1], DIVS[2]], ids=["kl-kl", "tv-kl", "rg-tv"])
def test_fused_pairs_match_oracle(shape_x, shape_y, divs):
    """launch_mode 3 (two fused passes per kernel, V-update contracting axis 0
    first) against the oracle: eps-scaling stages then a fixed number of
    iterations, uneven shapes and zero densities included."""
    og, lg, dx, dy, p, q = grid_problem(shape_x, shape_y, 41)
    oF1, oF2, uF1, uF2 = divs
    dxr, dyr, pr, qr = rounded(U.F32, dx, dy, p, q)
    args = [T(a, U.F32).ravel() for a in (pr, dxr, qr, dyr)]
    eps, iters = 0.01, 15
    Ug, Vg, info = U.solve(lg(U.F32), *args, uF1, uF2, eps, precision=U.F32, max_iter=iters, eps_start=0.1,
                           eps_stages=3, iters_per_stage=4, check_every=5, launch_mode=3)
    r = O.solve_log(round_geom(og, U.F32), dxr, dyr, pr, qr, oF1, oF2, eps, max_iter=iters, eps_start=0.1,
                    stages=3, iters_per_stage=4)
    assert info["iters"] == iters and info["total_iters"] == iters + 12
    assert rel_err(to_np(Ug), r["U"]) <= TOL[U.F32]
    assert rel_err(to_np(Vg), r["V"]) <= TOL[U.F32]


def test_fused_pairs_converge_like_per_pass():
    """The fused solve stops at the same tolerance as the per-pass solve, in
    (almost) the same number of iterations, at the same potentials to FP32
    accuracy."""
    og, lg, dx, dy, p, q = grid_problem((64, 80), (64, 80), 43, zeros=False)
    args = [T(a, U.F32).ravel() for a in (p, dx, q, dy)]
    outs = [U.solve(lg(U.F32), *args, U.KL(0.5), U.KL(0.5), 2e-3, precision=U.F32, max_iter=5000, tol=1e-6,
                    check_every=10, eps_start=0.1, eps_stages=5, iters_per_stage=20, launch_mode=m)
            for m in (3, 0)]
    (U3, V3, i3), (U0, V0, i0) = outs
    assert i3["status"] == i0["status"] == "UOT_OK"
    assert i3["marg_err"] <= 1e-6 and abs(i3["iters"] - i0["iters"]) <= 20
    assert torch.max(torch.abs(U3 - U0)).item() <= 1e-5 * max(1.0, torch.max(torch.abs(U0)).item())
    assert torch.max(torch.abs(V3 - V0)).item() <= 1e-5 * max(1.0, torch.max(torch.abs(V0)).item())


# ----------------------------------------------------------------------------
# tensor-core pass with three-part BF16 operands (tile 7)
# ----------------------------------------------------------------------------

TC3_CASES = [
    ("fine2d", lambda: grid_problem((200, 256), (256, 180), 51), 2e-3),
    ("batchlike", lambda: grid_problem((128, 128), (128, 128), 52), 1e-2),
    ("ragged", lambda: grid_problem((150, 97), (130, 70), 53), 1e-2),
]


@pytest.mark.parametrize("name,make,eps", TC3_CASES)
def test_tc3_pass_matches_oracle(name, make, eps):
    """Forced tensor-core tile on grids fine enough for its block condition:
    the Gibbs operator in both directions and a short KL/TV solve at the FP32
    tolerance, and bitwise different from the SIMT tile (another kernel ran)."""
    og, lg, dx, dy, p, q = make()
    g = synth.rng(61)
    try:
        for transpose in (False, True):
            shape_in = np.shape(dx) if transpose else np.shape(dy)
            W = g.normal(size=shape_in) * 0.05
            W.ravel()[5:: 13] = -np.inf
            w = dx if transpose else dy
            W, w = rounded(U.F32, W, w)
            want = O.apply_K_log(round_geom(og, U.F32), W, np.log(w), eps, transpose=transpose)
            outs = []
            for tile in (7, 0):
                U.force_grid_tile(tile)
                outs.append(to_np(U.gibbs_log(lg(U.F32), T(W, U.F32).ravel(), T(w, U.F32).ravel(), eps,
                                              transpose, U.F32)))
            assert rel_err(outs[0], want) <= TOL[U.F32]
            assert not np.array_equal(outs[0], outs[1])
        U.force_grid_tile(7)
        dxr, dyr, pr, qr = rounded(U.F32, dx, dy, p, q)
        Ug, Vg, _ = U.solve(lg(U.F32), *[T(a, U.F32).ravel() for a in (pr, dxr, qr, dyr)], U.KL(0.7),
                            U.TV(0.4), eps, precision=U.F32, max_iter=10)
        r = O.solve_log(round_geom(og, U.F32), dxr, dyr, pr, qr, O.KL(0.7), O.TV(0.4), eps, max_iter=10)
        assert rel_err(to_np(Ug), r["U"]) <= TOL[U.F32]
        assert rel_err(to_np(Vg), r["V"]) <= TOL[U.F32]
    finally:
        U.force_grid_tile(-1)


def test_tc3_barycenter_matches_oracle():
    """Batched lines (8 measures of 128 x 128) through the tensor-core tile."""
    b = synth.barycenter_images(8, 128, 128, seed=62)
    alpha = np.full(8, 1.0 / 8)
    eps, lam, iters = 1e-2, 1.0, 4
    xs = [np.asarray(a, np.float32).astype(np.float64) for a in b["xs"]]
    geo = U.Geometry.grid([T(a, U.F32) for a in xs])
    P = np.asarray(b["P"], np.float32).astype(np.float64)
    U.force_grid_tile(7)
    try:
        lh, Ug, Vg, _ = U.barycenter(geo, alpha, T(P.reshape(8, -1), U.F32), T(b["dx"], U.F32).ravel(),
                                     T(b["dy"], U.F32).ravel(), U.EQ(), lam, eps, precision=U.F32, max_iter=iters)
    finally:
        U.force_grid_tile(-1)
    og = O.Geometry("grid", xs=xs, ys=xs)
    dxr, dyr = rounded(U.F32, b["dx"], b["dy"])
    Uo, Vo, lho = O.barycenter_log(og, dxr, dyr, P, alpha, O.EQ(), lam, eps, iters)
    assert rel_err(to_np(lh), lho) <= TOL[U.F32]
    assert rel_err(to_np(Vg).reshape(8, -1), Vo.reshape(8, -1)) <= TOL[U.F32]


def test_barycenter_graph_blocks_match_per_pass():
    """The barycenter loop replayed as CUDA-graph blocks (launch_mode 2) runs
    the same kernels: identical result to per-pass launches."""
    b = synth.barycenter_images(6, 48, 40, seed=71)
    alpha = np.full(6, 1.0 / 6)
    geo = U.Geometry.grid([T(a, U.F32) for a in b["xs"]])
    P = T(np.asarray(b["P"]).reshape(6, -1), U.F32)
    outs = [U.barycenter(geo, alpha, P, T(b["dx"], U.F32).ravel(), T(b["dy"], U.F32).ravel(), U.KL(1.0), 1.0,
                         1e-2, precision=U.F32, max_iter=45, check_every=10, launch_mode=m) for m in (2, 0)]
    (h2, U2, V2, i2), (h0, U0, V0, i0) = outs
    assert i2["iters"] == i0["iters"] == 45
    assert torch.equal(h2, h0) and torch.equal(U2, U0) and torch.equal(V2, V0)


# ----------------------------------------------------------------------------
# TV and RG barycenters (Table 2 (iii), (iv))
# ----------------------------------------------------------------------------

@pytest.mark.parametrize("prec", [U.F64, U.F32])
@pytest.mark.parametrize("kind", ["tv", "rg", "tv-zeros"])
def test_barycenter_tv_rg_parity(kind, prec):
    """uot_barycenter_div with a TV or RG barycenter divergence against the
    oracle, iterate by iterate (uneven weights; one case with empty measures
    that outweigh the others, where h = 0)."""
    d = synth.barycenter_images(K=5, H=24, W=36, seed=16)
    P = np.array(d["P"], dtype=np.float64)
    if kind == "tv-zeros":
        # measures 1 and 3 empty: their weight 0.55 outweighs the rest, so h = 0 (Table 2 (iii))
        P[1] = 0.0
        P[3] = 0.0
    og = O.Geometry("grid", xs=d["xs"], ys=d["ys"])
    alpha = np.array([0.1, 0.3, 0.2, 0.25, 0.15])
    eps, lam, iters, beta = 0.01, 0.05, 20, (0.7, 1.6)
    okind = "rg" if kind == "rg" else "tv"
    Uo, Vo, lho = O.barycenter_log(og, d["dx"], d["dy"], P, alpha, O.EQ(), lam, eps, iters, bary_kind=okind,
                                   beta=beta)
    geo = U.Geometry.grid([T(a, prec) for a in d["xs"]])
    Fh = U.RG(*beta) if okind == "rg" else U.TV(lam)
    Pr = rounded(prec, P)
    lh, Ug, Vg, info = U.barycenter_div(geo, alpha, T(Pr.reshape(5, -1), prec), T(d["dx"], prec).ravel(),
                                        T(d["dy"], prec).ravel(), U.EQ(), Fh, eps, precision=prec, max_iter=iters)
    if prec == U.F32:  # the oracle on the inputs the FP32 call receives
        dxr, dyr = rounded(prec, d["dx"], d["dy"])
        ogr = round_geom(og, prec)
        Uo, Vo, lho = O.barycenter_log(ogr, dxr, dyr, Pr, alpha, O.EQ(), lam, eps, iters, bary_kind=okind,
                                       beta=beta)
    assert rel_err(to_np(lh), lho) <= TOL[prec]
    assert rel_err(to_np(Ug), Uo.reshape(5, -1)) <= TOL[prec]
    assert rel_err(to_np(Vg), Vo.reshape(5, -1)) <= TOL[prec]
    if kind == "tv-zeros":
        assert np.isneginf(to_np(lh)).all()


def test_barycenter_div_matches_barycenter_for_kl_eq():
    """uot_barycenter_div with KL / EQ divergences is uot_barycenter."""
    d = synth.barycenter_images(K=3, H=16, W=20, seed=17)
    alpha = np.array([0.5, 0.3, 0.2])
    geo = U.Geometry.grid([T(a, U.F64) for a in d["xs"]])
    args = (T(d["P"].reshape(3, -1), U.F64), T(d["dx"], U.F64).ravel(), T(d["dy"], U.F64).ravel(), U.EQ())
    for Fh, kind in ((U.KL(0.7), U.BARY_KL), (U.EQ(), U.BARY_EQ)):
        a = U.barycenter_div(geo, alpha, *args, Fh, 0.02, precision=U.F64, max_iter=15)
        b = U.barycenter(geo, alpha, *args, 0.7, 0.02, kind=kind, precision=U.F64, max_iter=15)
        for x, y in zip(a[:3], b[:3]):
            assert torch.equal(x, y)
    with pytest.raises(U.UotError, match="EINVAL"):
        U.barycenter_div(geo, alpha, *args, U.RG(0.0, 2.0), 0.02, precision=U.F64, max_iter=2)
    with pytest.raises(U.UotError, match="EINVAL"):
        U.barycenter(geo, alpha, *args, 0.7, 0.02, kind=U.BARY_RG, precision=U.F64, max_iter=2)

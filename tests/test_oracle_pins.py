"""Pins of the FP64 oracle against facts the paper and the mathematics fix.

Each test names the passage that fixes the expected value.  None of them
re-types the oracle's own formula: they use closed forms, brute-force
minimisation of the primal, optimality (KKT) conditions, invariants or an
independent form of the same operation (Algorithm 1 vs Algorithm 2 vs the
log-domain form; separable vs dense kernel).
"""
import math

import numpy as np
import pytest
from scipy import optimize

import oracle as O
from paper_1607_05816_gb300 import synth

pytestmark = pytest.mark.filterwarnings("ignore::RuntimeWarning")


def small_problem(n, m, seed, d=1, zeros=False):
    g = synth.rng(seed)
    x = g.uniform(0, 1, size=(n, d))
    y = g.uniform(0, 1, size=(m, d))
    dx = g.uniform(0.5, 1.5, size=n)
    dx /= dx.sum()
    dy = g.uniform(0.5, 1.5, size=m)
    dy /= dy.sum()
    p = g.uniform(0.3, 2.0, size=n)
    q = g.uniform(0.3, 2.0, size=m)
    if zeros:
        p[0] = 0.0
    return O.Geometry("points", x=x, y=y), dx, dy, p, q


# --------------------------------------------------------------------------
# log-sum-exp and the Gibbs operator
# --------------------------------------------------------------------------

def test_lse_conventions():
    assert O.lse(np.array([-np.inf, -np.inf])) == -np.inf
    z = np.array([1.0, 2.0, -3.0])
    assert abs(O.lse(z) - math.log(sum(math.exp(t) for t in z))) < 1e-15
    big = np.array([1000.0, 1000.0])
    assert abs(O.lse(big) - (1000.0 + math.log(2.0))) < 1e-12


def test_gibbs_operator_matches_definition():
    """eps log K(b.dy) with K = exp(-C/eps) (Sec. 4.2), by plain sums."""
    geom, dx, dy, p, q = small_problem(5, 4, 1)
    eps = 0.3
    V = np.array([0.1, -0.2, 0.3, 0.05])
    C = geom.cost_matrix()
    K = np.exp(-C / eps)
    expect = eps * np.log(K @ (np.exp(V / eps) * dy))
    got = O.apply_K_log(geom, V, np.log(dy), eps)
    assert np.max(np.abs(got - expect)) < 1e-14
    expectT = eps * np.log(K.T @ (np.exp(np.zeros(5) / eps) * dx))
    gotT = O.apply_K_log(geom, np.zeros(5), np.log(dx), eps, transpose=True)
    assert np.max(np.abs(gotT - expectT)) < 1e-14


@pytest.mark.parametrize("shape_x,shape_y", [((6, 5), (6, 5)), ((4, 7), (5, 3)), ((9,), (7,)), ((3, 4, 2), (2, 3, 3))])
def test_separable_equals_dense(shape_x, shape_y):
    """The separable grid kernel (successive 1-D operations, Sec. 4.4) equals
    the full kernel on the product grid."""
    g = synth.rng(7)
    xs = [np.sort(g.uniform(0, 1, n)) for n in shape_x]
    ys = [np.sort(g.uniform(0, 1, n)) for n in shape_y]
    geom = O.Geometry("grid", xs=xs, ys=ys)
    eps = 0.02
    V = g.normal(size=shape_y) * 0.05
    logw = np.log(g.uniform(0.5, 1.0, size=shape_y))
    a = O.apply_K_log(geom, V, logw, eps, separable=True)
    b = O.apply_K_log(geom, V, logw, eps, separable=False)
    assert a.shape == tuple(shape_x)
    assert np.max(np.abs(a - b)) < 1e-12
    U = g.normal(size=shape_x) * 0.05
    logwx = np.log(g.uniform(0.5, 1.0, size=shape_x))
    a = O.apply_K_log(geom, U, logwx, eps, transpose=True, separable=True)
    b = O.apply_K_log(geom, U, logwx, eps, transpose=True, separable=False)
    assert np.max(np.abs(a - b)) < 1e-12


# --------------------------------------------------------------------------
# Table 1: each prox row against scalar brute-force minimisation
# --------------------------------------------------------------------------

def scalar_prox_brute(F, s, p, eps):
    """argmin_{t>=0} eps KLbar(t|s) + Dbar_F(t|p), KLbar(t|s)=t log(t/s)-t+s."""
    def obj(lt):
        t = math.exp(lt)
        val = eps * (t * (lt - math.log(s)) - t + s)
        if F.kind == "kl":
            val += F.lam * (t * math.log(t / p) - t + p)
        elif F.kind == "tv":
            val += F.lam * abs(t - p)
        elif F.kind == "rg":
            lo, hi = F.alpha * p, F.beta * p
            if t < lo * (1 - 1e-15) or t > hi * (1 + 1e-15):
                return 1e300
        return val
    if F.kind == "eq":
        return p
    if F.kind == "rg":
        lo = math.log(F.alpha * p) if F.alpha > 0 else math.log(s) - 50
        hi = math.log(F.beta * p) if not math.isinf(F.beta) else math.log(s) + 50
        if lo > math.log(s):
            return F.alpha * p
        if hi < math.log(s):
            return F.beta * p
        return s
    lo = min(math.log(s), math.log(p)) - 1.0
    hi = max(math.log(s), math.log(p)) + 1.0
    r = optimize.minimize_scalar(obj, bounds=(lo, hi), method="bounded", options=dict(xatol=1e-12))
    # polish with a dense scan around the minimiser for the kinked TV case
    grid = r.x + np.linspace(-1e-3, 1e-3, 20001)
    vals = [obj(t) for t in grid]
    return math.exp(grid[int(np.argmin(vals))])


@pytest.mark.parametrize("F", [O.KL(0.7), O.KL(5.0), O.TV(0.05), O.TV(0.8), O.RG(0.7, 1.2), O.RG(0.0, 2.0), O.RG(0.5, math.inf), O.EQ()])
def test_prox_rows_brute_force(F):
    """Middle column of Table 1 equals the scalar minimiser of
    eps KL(t|s) + D_phi(t|p) (definition of prox^KL, Sec. 3.3)."""
    g = synth.rng(11)
    for _ in range(25):
        s = float(np.exp(g.uniform(-3, 3)))
        p = float(np.exp(g.uniform(-2, 2)))
        eps = float(np.exp(g.uniform(-3, 0)))
        got = math.exp(O.prox_target_log(F, np.array([math.log(p)]), np.array([eps * math.log(s)]), eps)[0])
        want = scalar_prox_brute(F, s, p, eps)
        assert abs(got - want) <= 2e-6 * max(want, 1e-12), (F, s, p, eps, got, want)


@pytest.mark.parametrize("F", [O.KL(0.4), O.TV(0.3), O.RG(0.6, 1.5), O.RG(0.0, math.inf), O.EQ()])
def test_stabilized_proxdiv_equals_log_update(F):
    """Table 1's proxdiv(s, u, eps) with u != 0 (Sec. 4.3) is the total-potential
    update shifted by u: eps log proxdiv(s~, u) = U(eps log s~ - u) - u."""
    g = synth.rng(12)
    eps = 0.05
    s = np.exp(g.uniform(-4, 4, size=64))
    u = g.uniform(-0.5, 0.5, size=64)
    p = np.exp(g.uniform(-2, 2, size=64))
    lhs = eps * np.log(O.proxdiv(F, p, s, u, eps))
    rhs = O.prox_update_log(F, np.log(p), eps * np.log(s) - u, eps) - u
    assert np.max(np.abs(lhs - rhs)) < 1e-12


def test_balanced_rows():
    """Table 1: RG[1,1] is the equality row; lam KL and lam TV tend to it as lam -> inf."""
    g = synth.rng(13)
    eps = 0.1
    S = g.uniform(-1, 1, size=50)
    lp = g.uniform(-1, 1, size=50)
    eq = O.prox_update_log(O.EQ(), lp, S, eps)
    assert np.array_equal(O.prox_update_log(O.RG(1.0, 1.0), lp, S, eps), eq)
    assert np.max(np.abs(O.prox_update_log(O.KL(1e9), lp, S, eps) - eq)) < 1e-8
    assert np.array_equal(O.prox_update_log(O.TV(1e9), lp, S, eps), eq)


def test_zero_mass_conventions():
    """Prop. 5.1 with 0/0 = 0: s = 0 gives a = 0; p = 0 gives a = 0 except for
    TV (phi'_inf = 1: eps log(s*/s) = -lam) and RG with beta = inf."""
    eps = 0.1
    S = np.array([0.2, -np.inf, 0.2])
    lp = np.array([-np.inf, 0.0, 0.0])
    for F in (O.EQ(), O.KL(1.0), O.RG(0.5, 2.0)):
        U = O.prox_update_log(F, lp, S, eps)
        assert np.isneginf(U[0]) and np.isneginf(U[1]) and np.isfinite(U[2])
    U = O.prox_update_log(O.TV(0.3), lp, S, eps)
    assert U[0] == -0.3 and np.isneginf(U[1])
    U = O.prox_update_log(O.RG(0.5, math.inf), lp, S, eps)
    assert U[0] == 0.0


# --------------------------------------------------------------------------
# one-point problems: closed forms
# --------------------------------------------------------------------------

@pytest.mark.parametrize("l1,l2,eps,c,p,q", [(1.0, 1.0, 0.5, 0.3, 1.0, 2.0), (0.2, 3.0, 0.1, 1.0, 0.5, 1.7), (5.0, 0.5, 0.05, 0.0, 2.0, 0.3)])
def test_one_point_kl_closed_form(l1, l2, eps, c, p, q):
    """n = m = 1, dx = dy = 1: stationarity of l1 KL(r|p) + l2 KL(r|q) + eps KL(r|e^{-c/eps})
    gives log r* = (l1 log p + l2 log q - c)/(l1 + l2 + eps)."""
    geom = O.Geometry("dense", C=np.array([[c]]))
    one = np.ones(1)
    r = O.solve_log(geom, one, one, np.array([p]), np.array([q]), O.KL(l1), O.KL(l2), eps, max_iter=4000)
    logr = (r["U"][0] + r["V"][0] - c) / eps
    want = (l1 * math.log(p) + l2 * math.log(q) - c) / (l1 + l2 + eps)
    assert abs(logr - want) < 1e-13


@pytest.mark.parametrize("F1,F2", [(O.TV(0.3), O.TV(0.2)), (O.TV(0.05), O.KL(1.0)), (O.RG(0.7, 1.2), O.KL(0.5)), (O.EQ(), O.KL(0.5)), (O.RG(0.5, 2.0), O.RG(0.8, 1.5))])
def test_one_point_piecewise_brute(F1, F2):
    """One-point primal F1(r) + F2(r) + eps KL(r|e^{-c/eps}) minimised by brute force."""
    eps, c, p, q = 0.1, 0.2, 1.0, 1.6
    geom = O.Geometry("dense", C=np.array([[c]]))
    one = np.ones(1)
    r = O.solve_log(geom, one, one, np.array([p]), np.array([q]), F1, F2, eps, max_iter=3000)
    got = math.exp((r["U"][0] + r["V"][0] - c) / eps)

    def obj(lt):
        t = math.exp(lt)
        v = eps * (t * (lt + c / eps) - t + math.exp(-c / eps))
        v1 = O.div_value(F1, np.array([t]), np.array([p]), one)
        v2 = O.div_value(F2, np.array([t]), np.array([q]), one)
        return v + (v1 if math.isfinite(v1) else 1e300) + (v2 if math.isfinite(v2) else 1e300)
    grid = np.linspace(-4, 4, 80001)
    vals = np.array([obj(t) for t in grid])
    k = int(np.argmin(vals))
    fine = grid[k] + np.linspace(-2e-4, 2e-4, 40001)
    best = fine[int(np.argmin([obj(t) for t in fine]))]
    assert abs(math.log(got) - best) < 2e-8, (got, math.exp(best))


# --------------------------------------------------------------------------
# Algorithms 1 and 2 and the log-domain form
# --------------------------------------------------------------------------

@pytest.mark.parametrize("F1,F2", [(O.KL(0.5), O.KL(0.1)), (O.TV(0.2), O.KL(1.0)), (O.RG(0.7, 1.2), O.TV(0.3)), (O.EQ(), O.EQ()), (O.KL(1.0), O.RG(0.0, 1.5))])
def test_alg1_alg2_logdomain_agree(F1, F2):
    """Algorithm 1, Algorithm 2 (absorbing when |log a~| > tau) and the log-domain
    form are reparametrisations of one iteration (Sec. 4.3), so their iterates agree."""
    geom, dx, dy, p, q = small_problem(7, 5, 3)
    eps, iters = 0.08, 60
    C = geom.cost_matrix()
    a, b = O.scaling_alg1(np.exp(-C / eps), dx, dy, p, q, F1, F2, eps, iters)
    U1, V1 = eps * np.log(a), eps * np.log(b)
    U2, V2, nabs = O.scaling_alg2(C, dx, dy, p, q, F1, F2, eps, iters, tau=0.5)
    assert nabs > 0
    U3, V3 = O.iterate_log(geom, np.log(dx), np.log(dy), np.log(p), np.log(q), F1, F2, eps, iters)
    for A, B in ((U1, U3), (V1, V3), (U2, U3), (V2, V3)):
        assert np.max(np.abs(A - B)) < 1e-11 * max(1.0, np.max(np.abs(B)))


def test_alg2_reaches_small_eps_where_alg1_fails():
    """Sec. 4.3: for small eps, K underflows and Algorithm 1 breaks down while the
    stabilized iteration stays finite and optimal (KKT for KL: r1 = p e^{-U/lam})."""
    geom, dx, dy, p, q = small_problem(6, 6, 4)
    eps = 1e-5
    C = geom.cost_matrix()
    with np.errstate(all="ignore"):
        a, b = O.scaling_alg1(np.exp(-C / eps), dx, dy, p, q, O.KL(1.0), O.KL(1.0), eps, 50)
    assert np.any(a == 0) or np.any(b == 0) or not np.all(np.isfinite(a * b.sum()))
    U, V = O.iterate_log(geom, np.log(dx), np.log(dy), np.log(p), np.log(q), O.KL(1.0), O.KL(1.0), eps, 3000)
    assert np.all(np.isfinite(U)) and np.all(np.isfinite(V))
    r1, r2 = O.marginals(geom, dx, dy, U, V, eps)
    # after the b-update the second marginal satisfies -V in dF2(r2) exactly
    assert np.max(np.abs(r2 - q * np.exp(-V / 1.0)) / r2) < 1e-10


# --------------------------------------------------------------------------
# convergence theory
# --------------------------------------------------------------------------

def test_thompson_contraction_kl_kl():
    """Theorem 3.10: for lam1 KL / lam2 KL the map a^l -> a^{l+1} contracts the
    Thompson metric d(a,a') = max |log a - log a'| by z1 z2, z_i = lam_i/(lam_i+eps)."""
    geom, dx, dy, p, q = small_problem(8, 6, 5)
    l1, l2, eps = 0.7, 1.3, 0.05
    z = (l1 / (l1 + eps)) * (l2 / (l2 + eps))
    logs = (np.log(dx), np.log(dy), np.log(p), np.log(q))
    U, V = None, None
    Us = []
    for _ in range(40):
        U, V = O.iterate_log(geom, *logs, O.KL(l1), O.KL(l2), eps, 1, U, V)
        Us.append(U.copy())
    d = [np.max(np.abs(Us[k + 1] - Us[k])) / eps for k in range(len(Us) - 1)]
    for k in range(len(d) - 1):
        if d[k] > 1e-13:
            assert d[k + 1] <= z * d[k] * (1 + 1e-9) + 1e-14


@pytest.mark.parametrize("F1,F2", [(O.KL(0.5), O.KL(0.5)), (O.TV(0.3), O.TV(0.2)), (O.KL(0.1), O.TV(0.5))])
def test_duality_gap(F1, F2):
    """Theorem 3.2 / 4.1: P_eps >= D_eps at every iterate, the gap equals the two
    Fenchel-Young gaps F(r) + F*(-U) + <U, r>, and it goes to 0."""
    geom, dx, dy, p, q = small_problem(6, 5, 6)
    eps = 0.05
    logs = (np.log(dx), np.log(dy), np.log(p), np.log(q))
    U, V = None, None
    gaps = []
    for it in range(400):
        U, V = O.iterate_log(geom, *logs, F1, F2, eps, 1, U, V)
        if it % 20 == 0 or it == 399:
            P = O.primal(geom, dx, dy, p, q, F1, F2, eps, U, V)
            D = O.dual(geom, dx, dy, p, q, F1, F2, eps, U, V)
            r1, r2 = O.marginals(geom, dx, dy, U, V, eps)
            fy = (O.div_value(F1, r1, p, dx) + O.div_conj(F1, -U, p, dx) + np.sum(dx * U * r1)
                  + O.div_value(F2, r2, q, dy) + O.div_conj(F2, -V, q, dy) + np.sum(dy * V * r2))
            assert P - D >= -1e-13
            assert abs((P - D) - fy) < 1e-11
            gaps.append(P - D)
    assert gaps[-1] < 1e-10
    assert gaps[-1] < gaps[1]


def newton_primal_kl(C, dx, dy, p, q, l1, l2, eps):
    """Brute-force minimiser of the KL/KL primal (eq. primal_discr with dx dy
    weights): damped Newton in R with the analytic Hessian
      H_(ij),(kl) = w_ij [l1 d_ik dy_l / r1_i + l2 d_jl dx_k / r2_j + eps d_ik d_jl / R_ij],
    steps kept inside R > 0 and backtracked on the objective.  Returns log R."""
    n, m = C.shape
    W = dx[:, None] * dy[None, :]
    K = np.exp(-C / eps)

    def f(R):
        r1, r2 = R @ dy, R.T @ dx
        kl1 = l1 * np.sum(dx * (r1 * np.log(r1 / p) - r1 + p))
        kl2 = l2 * np.sum(dy * (r2 * np.log(r2 / q) - r2 + q))
        return kl1 + kl2 + eps * np.sum(W * (R * np.log(R / K) - R + K))

    R = np.ones((n, m))
    for _ in range(500):
        r1, r2 = R @ dy, R.T @ dx
        g = (W * (l1 * np.log(r1 / p)[:, None] + l2 * np.log(r2 / q)[None, :] + eps * np.log(R) + C)).ravel()
        if np.max(np.abs(g / W.ravel())) < 1e-15:
            break
        H = np.zeros((n * m, n * m))
        for i in range(n):
            for j in range(m):
                for k in range(n):
                    for l in range(m):
                        v = 0.0
                        if i == k:
                            v += l1 * dy[l] / r1[i]
                        if j == l:
                            v += l2 * dx[k] / r2[j]
                        if i == k and j == l:
                            v += eps / R[i, j]
                        H[i * m + j, k * m + l] = W[i, j] * v
        step = -np.linalg.solve(H, g).reshape(n, m)
        t = 1.0
        neg = step < 0
        if np.any(neg):
            t = min(1.0, 0.99 * np.min(-R[neg] / step[neg]))
        f0 = f(R)
        while f(R + t * step) > f0 + 1e-4 * t * (g @ step.ravel()) and t > 1e-14:
            t *= 0.5
        R = R + t * step
    return np.log(R)


@pytest.mark.parametrize("n,m", [(1, 3), (3, 2), (4, 4)])
def test_brute_force_primal_kl(n, m):
    """The converged iteration minimises the primal (Prop. 3.8): compare the plan
    to an independent Newton minimisation of the primal on tiny problems."""
    geom, dx, dy, p, q = small_problem(n, m, 20 + n)
    l1, l2, eps = 0.6, 0.9, 0.1
    C = geom.cost_matrix()
    Z = newton_primal_kl(C, dx, dy, p, q, l1, l2, eps)
    r = O.solve_log(geom, dx, dy, p, q, O.KL(l1), O.KL(l2), eps, max_iter=3000)
    LR = O.log_plan(geom, r["U"], r["V"], eps)
    assert np.max(np.abs(LR - Z)) < 1e-9


@pytest.mark.parametrize("F1,F2", [(O.TV(0.2), O.TV(0.3)), (O.RG(0.7, 1.2), O.RG(0.8, 1.5)), (O.TV(0.1), O.KL(0.5)), (O.EQ(), O.KL(0.4))])
def test_kkt_optimality(F1, F2):
    """Theorem 3.2: (U, V) is optimal iff -U in dF1(r1), -V in dF2(r2) with
    R = e^{(U+V-C)/eps}.  Checked on the converged iterate from the subdifferentials
    of the divergences (Prop. A.3)."""
    geom, dx, dy, p, q = small_problem(6, 7, 30)
    eps = 0.05
    r = O.solve_log(geom, dx, dy, p, q, F1, F2, eps, max_iter=20000, tol=1e-14)
    U, V = r["U"], r["V"]
    r1, r2 = O.marginals(geom, dx, dy, U, V, eps)
    for F, W, rr, pp in ((F1, U, r1, p), (F2, V, r2, q)):
        if F.kind == "tv":
            lam = F.lam
            assert np.all(np.abs(W) <= lam * (1 + 1e-10))
            above = rr > pp * (1 + 1e-8)
            below = rr < pp * (1 - 1e-8)
            assert np.allclose(W[above], -lam, atol=1e-9)
            assert np.allclose(W[below], lam, atol=1e-9)
        elif F.kind == "rg":
            assert np.all(rr >= F.alpha * pp * (1 - 1e-8)) and np.all(rr <= F.beta * pp * (1 + 1e-8))
            inside = (rr > F.alpha * pp * (1 + 1e-8)) & (rr < F.beta * pp * (1 - 1e-8))
            assert np.allclose(W[inside], 0.0, atol=1e-9)
            assert np.all(W[rr >= F.beta * pp * (1 - 1e-8)] <= 1e-9)
            assert np.all(W[rr <= F.alpha * pp * (1 + 1e-8)] >= -1e-9)
        elif F.kind == "kl":
            # -U = lam log(r/p)
            assert np.allclose(-W, F.lam * np.log(rr / pp), atol=1e-9)
        elif F.kind == "eq":
            assert np.allclose(rr, pp, rtol=1e-9)


def test_tv_primal_slsqp():
    """Brute-force TV/TV primal with split variables (r - p = t+ - t-) by SLSQP;
    the converged iteration reaches the same objective value and plan."""
    geom, dx, dy, p, q = small_problem(3, 3, 40)
    l1, l2, eps = 0.2, 0.3, 0.1
    C = geom.cost_matrix()
    n, m = C.shape
    W = dx[:, None] * dy[None, :]
    K = np.exp(-C / eps)
    N = n * m

    def unpack(xv):
        return xv[:N].reshape(n, m), xv[N:N + n], xv[N + n:N + 2 * n], xv[N + 2 * n:N + 2 * n + m], xv[N + 2 * n + m:]

    def f(xv):
        R, a1, b1, a2, b2 = unpack(xv)
        R = np.maximum(R, 1e-300)
        return eps * np.sum(W * (R * np.log(R / K) - R + K)) + l1 * np.sum(dx * (a1 + b1)) + l2 * np.sum(dy * (a2 + b2))

    cons = [{"type": "eq", "fun": lambda xv: unpack(xv)[0] @ dy - p - unpack(xv)[1] + unpack(xv)[2]},
            {"type": "eq", "fun": lambda xv: unpack(xv)[0].T @ dx - q - unpack(xv)[3] + unpack(xv)[4]}]
    x0 = np.concatenate([np.ones(N), np.zeros(2 * n + 2 * m)])
    bounds = [(1e-12, None)] * N + [(0, None)] * (2 * n + 2 * m)
    res = optimize.minimize(f, x0, method="SLSQP", constraints=cons, bounds=bounds,
                            options=dict(ftol=1e-15, maxiter=2000))
    r = O.solve_log(geom, dx, dy, p, q, O.TV(l1), O.TV(l2), eps, max_iter=20000, tol=1e-15)
    P = O.primal(geom, dx, dy, p, q, O.TV(l1), O.TV(l2), eps, r["U"], r["V"])
    assert P <= res.fun + 1e-9
    assert abs(P - res.fun) < 1e-6
    R = np.exp(O.log_plan(geom, r["U"], r["V"], eps))
    assert np.max(np.abs(R - unpack(res.x)[0])) < 1e-3 * np.max(R)


def test_eps_scaling_same_fixed_point():
    """eps-scaling (Sec. 4.4) only changes the starting point; by uniqueness of the
    solution (Theorem 3.2) it ends at the cold-start fixed point."""
    geom, dx, dy, p, q = small_problem(8, 8, 50)
    eps = 0.01
    a = O.solve_log(geom, dx, dy, p, q, O.KL(0.5), O.KL(0.5), eps, max_iter=20000, tol=1e-13)
    b = O.solve_log(geom, dx, dy, p, q, O.KL(0.5), O.KL(0.5), eps, max_iter=20000, tol=1e-13,
                    eps_start=1.0, stages=10, iters_per_stage=50)
    assert np.max(np.abs(a["U"] - b["U"])) < 1e-9
    assert np.max(np.abs(a["V"] - b["V"])) < 1e-9
    assert b["iters"] < a["iters"]


def test_marginal_violation_is_sinkhorn_error_when_balanced():
    """For the equality constraint the stopping criterion is the L1(dx) marginal
    error of the plan relative to the mass of p (classical Sinkhorn)."""
    geom, dx, dy, p, q = small_problem(5, 6, 60)
    q = q * (np.sum(p * dx) / np.sum(q * dy))
    eps = 0.1
    U, V = O.iterate_log(geom, np.log(dx), np.log(dy), np.log(p), np.log(q), O.EQ(), O.EQ(), eps, 7)
    r1, _ = O.marginals(geom, dx, dy, U, V, eps)
    want = np.sum(dx * np.abs(r1 - p)) / np.sum(dx * p)
    got = O.marginal_violation(geom, dx, dy, p, q, O.EQ(), O.EQ(), eps, U, V)
    assert abs(got - want) < 1e-13


# --------------------------------------------------------------------------
# barycenters (Sec. 5.2, Table 2, Appendix A.3)
# --------------------------------------------------------------------------

def test_barycenter_h_kl_optimality():
    """Appendix A.3 (KL case): with t_k = s_k^{eps/(eps+lam)} h^{lam/(eps+lam)} the
    optimal h satisfies sum_k alpha_k (1 - t_k/h) = 0; Table 2 (i) is the geometric mean."""
    g = synth.rng(70)
    eps, lam = 0.07, 0.4
    T = g.uniform(-1, 1, size=(5, 30))
    alpha = g.uniform(0.2, 1.0, size=5)
    elogh = O.bary_h_log(T, alpha, lam, eps, "kl")
    logt = (eps / (eps + lam)) * (T / eps) + (lam / (eps + lam)) * (elogh / eps)
    res = np.sum(alpha[:, None] * (1 - np.exp(logt - elogh / eps)), axis=0)
    assert np.max(np.abs(res)) < 1e-12
    geo = O.bary_h_log(T, alpha, lam, eps, "eq")
    assert np.allclose(np.exp(geo / eps), np.prod(np.exp(T / eps) ** alpha[:, None], axis=0) ** (1 / alpha.sum()))


def test_barycenter_single_measure():
    """With one measure and F1 the equality constraint, h = s after the first
    iteration, so b = 1 (V = 0) and the plan is one Sinkhorn half-step."""
    g = synth.rng(71)
    xs = [synth.grid_axis(6), synth.grid_axis(5)]
    geom = O.Geometry("grid", xs=xs, ys=xs)
    dx = np.full((6, 5), 1 / 30)
    P = g.uniform(0.5, 2, size=(1, 6, 5))
    U, V, elogh = O.barycenter_log(geom, dx, dx, P, np.array([1.0]), O.EQ(), 0.5, 0.05, 3)
    assert np.max(np.abs(V)) < 1e-13
    r1, r2 = O.marginals(geom, dx.ravel(), dx.ravel(), U[0].ravel(), V[0].ravel(), 0.05)
    assert np.allclose(r1, P[0].ravel(), rtol=1e-12)
    assert np.allclose(np.exp(elogh / 0.05).ravel(), r2, rtol=1e-12)


def test_barycenter_fixed_point_optimality():
    """At convergence of the KL barycenter, r2_k = t_k (prox target with p -> h)
    and sum_k alpha_k (1 - r2_k/h) = 0 pointwise (Prop. 5.3)."""
    g = synth.rng(72)
    xs = [synth.grid_axis(5), synth.grid_axis(4)]
    geom = O.Geometry("grid", xs=xs, ys=xs)
    dx = np.full((5, 4), 1 / 20)
    P = g.uniform(0.5, 2, size=(3, 5, 4))
    alpha = np.array([0.2, 0.3, 0.5])
    eps, lam = 0.05, 0.3
    U, V, elogh = O.barycenter_log(geom, dx, dx, P, alpha, O.EQ(), lam, eps, 1500)
    h = np.exp(elogh / eps).ravel()
    acc = np.zeros_like(h)
    for k in range(3):
        r1, r2 = O.marginals(geom, dx.ravel(), dx.ravel(), U[k].ravel(), V[k].ravel(), eps)
        acc += alpha[k] * (1 - r2 / h)
        assert np.allclose(r1, P[k].ravel(), rtol=1e-8)
    assert np.max(np.abs(acc)) < 1e-8


# ----------------------------------------------------------------------------
# Table 2 (iii), (iv): TV and RG barycenters
# ----------------------------------------------------------------------------

def _kl_bar(t, s):
    """Pointwise KL-bar(t|s) = t log(t/s) - t + s with 0 log 0 = 0."""
    return (t * math.log(t / s) if t > 0 else 0.0) - t + s


def _prox_bary_value(h, s, alpha, eps, lam, kind, beta):
    """Objective of eq. prox_barycenter at h, minimised over s~ (each s~_k by
    bounded scalar search for TV; for RG the constraint set is the interval
    [beta1 h, beta2 h] and KL-bar(.|s) is convex with its minimum at s, so its
    minimiser there is the projection of s)."""
    total = 0.0
    for sk, ak in zip(s, alpha):
        if sk == 0.0:
            # s~_k = 0 is forced (Prop. on barycenter optimality)
            total += ak * (lam * h if kind == "tv" else (0.0 if h == 0.0 else math.inf))
            continue
        if kind == "tv":
            hi = max(4.0 * sk, 4.0 * h, 1e-300)
            r = optimize.minimize_scalar(lambda t: eps * _kl_bar(t, sk) + lam * abs(t - h), bounds=(0.0, hi),
                                         method="bounded", options={"xatol": 1e-14 * hi})
            cand = [r.fun, eps * _kl_bar(h, sk), eps * _kl_bar(0.0, sk) + lam * h, eps * _kl_bar(sk, sk) + lam * abs(sk - h)]
            total += ak * min(cand)
        else:
            t = min(max(sk, beta[0] * h), beta[1] * h)
            total += ak * eps * _kl_bar(t, sk)
    return total


@pytest.mark.parametrize("kind", ["tv", "rg"])
def test_barycenter_h_tv_rg_minimises_prox_problem(kind):
    """Table 2 (iii)/(iv) against brute force: the oracle's h attains the
    minimum over h of eq. prox_barycenter (scalar search over log h), including
    points with zero masses and points where the minimiser is an interval."""
    g = synth.rng(73 if kind == "tv" else 74)
    eps, lam, beta = 0.05, 0.08, (0.6, 1.7)
    npts, n = 12, 4
    T = eps * np.log(g.uniform(0.05, 3.0, size=(n, npts)))
    if kind == "tv":
        T[0, 3] = -np.inf          # some zero masses
        T[:3, 5] = -np.inf         # mostly zero: h = 0
        T[:, 7] = [0.0, 0.0, 1.0, 1.0]  # equal weights saturated both ways: interval of minimisers
    alpha = g.uniform(0.5, 2.0, size=n)
    alpha[:] = 1.0 if kind == "tv" else alpha
    W = O.bary_h_log(T, alpha, lam, eps, kind, beta)
    for j in range(npts):
        s = [math.exp(t / eps) if np.isfinite(t) else 0.0 for t in T[:, j]]
        h_or = math.exp(W[j] / eps) if np.isfinite(W[j]) else 0.0
        v_or = _prox_bary_value(h_or, s, alpha, eps, lam, kind, beta)
        # brute force over log h on a wide bracket, plus h = 0
        pos = [x for x in s if x > 0]
        lo, hi = math.log(min(pos)) - 40 * lam / eps - 5, math.log(max(pos)) + 40 * lam / eps + 5
        grid = np.linspace(lo, hi, 801)
        vals = [_prox_bary_value(math.exp(u), s, alpha, eps, lam, kind, beta) for u in grid]
        i = int(np.argmin(vals))
        r = optimize.minimize_scalar(lambda u: _prox_bary_value(math.exp(u), s, alpha, eps, lam, kind, beta),
                                     bounds=(grid[max(i - 1, 0)], grid[min(i + 1, 800)]), method="bounded",
                                     options={"xatol": 1e-12})
        v_bf = min(r.fun, vals[i], _prox_bary_value(0.0, s, alpha, eps, lam, kind, beta))
        assert v_or <= v_bf + 1e-9 * max(1.0, abs(v_bf)), (j, v_or, v_bf)
    if kind == "tv":
        assert np.isneginf(W[5]) and np.isfinite(W[3])
        # the flat interval between the saturated halves: its midpoint
        assert abs(W[7] - 0.5) <= 1e-12


def test_barycenter_h_rg_unit_range_is_geometric_mean():
    """RG[1, 1] is the equality constraint, so Table 2 (iv) reduces to (i)."""
    g = synth.rng(75)
    T = g.normal(size=(5, 30)) * 0.3
    alpha = g.uniform(0.2, 2.0, size=5)
    W = O.bary_h_log(T, alpha, 0.0, 0.02, "rg", (1.0, 1.0))
    assert np.max(np.abs(W - O.bary_h_log(T, alpha, 0.0, 0.02, "eq"))) <= 1e-12
    T[2, 4] = -np.inf
    assert np.isneginf(O.bary_h_log(T, alpha, 0.0, 0.02, "rg", (0.5, 2.0))[4])


def test_barycenter_h_tv_limits():
    """TV barycenter: for lam -> 0 the clamps saturate and eps log h is the
    alpha-weighted median of the T_k; for lam large against the spread of the
    T_k they never do and it is the alpha-weighted mean (the geometric mean of
    Table 2 (i))."""
    g = synth.rng(76)
    n, npts = 5, 40
    T = g.normal(size=(n, npts))
    alpha = g.uniform(0.2, 2.0, size=n)
    W0 = O.bary_h_log(T, alpha, 1e-9, 0.01, "tv")
    for j in range(npts):
        order = np.argsort(T[:, j])
        cw = np.cumsum(alpha[order])
        k = int(np.searchsorted(cw, 0.5 * alpha.sum()))
        assert abs(W0[j] - T[order[k], j]) <= 1e-6
    # lam = 1e4 >> |T_k - W|: no clamp saturates, the condition is linear in W
    Winf = O.bary_h_log(T, alpha, 1e4, 0.01, "tv")
    assert np.max(np.abs(Winf - O.bary_h_log(T, alpha, 0.0, 0.01, "eq"))) <= 1e-7


@pytest.mark.parametrize("kind", ["tv", "rg"])
def test_barycenter_tv_rg_single_measure(kind):
    """With one measure the barycenter is that measure's marginal (h = s), so
    b = 1 (V = 0) for both the TV and the RG divergence."""
    g = synth.rng(77)
    x = synth.grid_axis(20)
    geo = O.Geometry("grid", xs=[x], ys=[x])
    P = g.uniform(0.5, 1.5, size=(1, 20))
    dx = np.full(20, 1 / 20)
    U, V, elogh = O.barycenter_log(geo, dx, dx, P, np.array([1.0]), O.EQ(), 0.3, 0.05, 3, "rg" if kind == "rg" else "tv",
                                   beta=(0.7, 1.4))
    assert np.max(np.abs(V)) <= 1e-12


# ----------------------------------------------------------------------------
# Algorithm 4: a function F3 of the plan's total mass (Sec. 4.5)
# ----------------------------------------------------------------------------

def _mass_problem(n, m, seed):
    g = synth.rng(seed)
    x = np.sort(g.uniform(0, 1, n))
    y = np.sort(g.uniform(0, 1, m))
    dx, dy = np.full(n, 1.0 / n), np.full(m, 1.0 / m)
    p, q = g.uniform(0.3, 2.0, n), g.uniform(0.3, 2.0, m)
    return x, y, dx, dy, p, q


@pytest.mark.parametrize("F3", [O.EQ(), O.KL(0.3), O.TV(0.2), O.RG(0.7, 1.1)], ids=["eq", "kl", "tv", "rg"])
def test_alg4_literal_equals_log_form(F3):
    """Algorithm 4 verbatim (non-log scalings, z updated after b) and the log
    form (z-update at the start of the next iteration) give the same a, b and z."""
    x, y, dx, dy, p, q = _mass_problem(12, 10, 80)
    C = O.sqdist(x, y)
    eps, it, m0 = 0.05, 30, 0.6
    F1, F2 = O.KL(0.5), O.TV(0.4)
    a, b, _ = O.scaling_alg4(np.exp(-C / eps), dx, dy, p, q, F1, F2, F3, m0, eps, it)
    _, _, z_prev = O.scaling_alg4(np.exp(-C / eps), dx, dy, p, q, F1, F2, F3, m0, eps, it - 1)
    r = O.solve_mass_log(O.Geometry("dense", C=C), dx, dy, p, q, F1, F2, F3, m0, eps, max_iter=it)
    assert np.max(np.abs(eps * np.log(a) - r["U"])) <= 1e-10
    assert np.max(np.abs(eps * np.log(b) - r["V"])) <= 1e-10
    assert abs(eps * math.log(z_prev) - r["Z"]) <= 1e-10


def test_alg4_without_mass_term_is_the_scaling_iteration():
    """F3 = RG[0, inf] (no condition on the total mass) gives z = 1 and the
    iterates of eq. S."""
    x, y, dx, dy, p, q = _mass_problem(15, 11, 81)
    geo = O.Geometry("dense", C=O.sqdist(x, y))
    r4 = O.solve_mass_log(geo, dx, dy, p, q, O.KL(0.5), O.KL(0.8), O.RG(0.0, math.inf), 0.5, 0.02, max_iter=40)
    r = O.solve_log(geo, dx, dy, p, q, O.KL(0.5), O.KL(0.8), 0.02, max_iter=40)
    assert r4["Z"] == 0.0
    assert np.array_equal(r4["U"], r["U"]) and np.array_equal(r4["V"], r["V"])


def _mass_plan(C, r, eps):
    return np.exp((r["U"][:, None] + r["V"][None, :] + r["Z"] - C) / eps)


@pytest.mark.parametrize("case", ["kl-eq", "kl-kl", "tv-eq"])
def test_alg4_matches_brute_force_minimisation(case):
    """Tiny problems (n = m = 3): the converged plan of Algorithm 4 minimises
    F1(R dy) + F2(R^T dx) + F3(total mass) + eps sum dx dy (R log(R/K) - R + K),
    found independently by SLSQP (mass equality) or L-BFGS (soft mass term)
    over log R."""
    x, y, dx, dy, p, q = _mass_problem(3, 3, 82)
    C = O.sqdist(x, y)
    eps, m0, lam1, lam2, lam3 = 0.1, 0.55, 0.4, 0.6, 0.5
    F1 = O.KL(lam1) if case != "tv-eq" else O.TV(lam1)
    F2 = O.KL(lam2)
    F3 = O.EQ() if case.endswith("eq") else O.KL(lam3)
    r = O.solve_mass_log(O.Geometry("dense", C=C), dx, dy, p, q, F1, F2, F3, m0, eps, max_iter=20000, tol=1e-13)
    R = _mass_plan(C, r, eps)
    K = np.exp(-C / eps)
    w = dx[:, None] * dy[None, :]

    def div(F, s, pp, ww):
        if F.kind == "kl":
            return F.lam * np.sum(ww * (s * np.log(s / pp) - s + pp))
        return F.lam * np.sum(ww * np.abs(s - pp))

    def obj(lR):
        Rm = np.exp(lR.reshape(3, 3))
        r1, r2 = Rm @ dy, Rm.T @ dx
        mass = np.sum(w * Rm)
        v = div(F1, r1, p, dx) + div(F2, r2, q, dy) + eps * np.sum(w * (Rm * (lR.reshape(3, 3) + C / eps) - Rm + K))
        if F3.kind == "kl":
            v += lam3 * (mass * math.log(mass / m0) - mass + m0)
        return v

    x0 = np.log(R).ravel() + 0.05
    if F3.kind == "eq":
        res = optimize.minimize(obj, x0, method="SLSQP", constraints=[{"type": "eq",
                                "fun": lambda lR: np.sum(w * np.exp(lR.reshape(3, 3))) - m0}],
                                options={"ftol": 1e-15, "maxiter": 2000})
    else:
        res = optimize.minimize(obj, x0, method="L-BFGS-B", options={"ftol": 1e-16, "gtol": 1e-12, "maxiter": 20000})
    Rb = np.exp(res.x.reshape(3, 3))
    assert obj(np.log(R).ravel()) <= res.fun + 1e-9
    if F1.kind == "kl":  # smooth objective: the minimiser itself is matched (SLSQP stalls on TV's kink)
        assert np.max(np.abs(R - Rb) / Rb) <= 2e-3
    if F3.kind == "eq":
        assert abs(np.sum(w * R) - m0) <= 1e-8  # the last b-update moves the mass slightly


# --------------------------------------------------------------------------
# WF gradient flows with growth (Sec. 5.3)
# --------------------------------------------------------------------------

def test_wf_cost_closed_forms():
    """eq. logcost: c = -log cos^2(d), d = (pi/2)|x - y|/cut: zero on the
    diagonal, log 2 at half the cut distance (cos^2(pi/4) = 1/2), log(4/3) at a
    third (cos^2(pi/6) = 3/4), +inf from the cut locus on, ~d^2 for small d,
    and isotropic in 2-D."""
    cut = 0.4
    x = np.array([0.0])  # distances exactly as written (the cut locus included)
    y = np.array([0.0, cut / 2, -cut / 3, cut, -1.5 * cut, 1e-4])
    c = O.wf_cost(x, y, cut)[0]
    assert c[0] == 0.0
    assert abs(c[1] - math.log(2.0)) < 1e-14
    assert abs(c[2] - math.log(4.0 / 3.0)) < 1e-14
    assert np.isposinf(c[3]) and np.isposinf(c[4])
    d = (math.pi / 2) * 1e-4 / cut
    assert abs(c[5] / d**2 - 1.0) < 1e-6
    th = 0.7
    P = np.array([[0.0, 0.0]])
    Q = np.array([[0.25 * cut * math.cos(th), 0.25 * cut * math.sin(th)]])
    assert abs(O.wf_cost(P, Q, cut)[0, 0] - O.wf_cost(np.array([0.0]), np.array([0.25 * cut]), cut)[0, 0]) < 1e-14
    # unscaled: cut = pi/2 is the plain distance
    assert abs(O.wf_cost(np.array([0.0]), np.array([0.5]))[0, 0] + math.log(math.cos(0.5) ** 2)) < 1e-14


def _kl(a, b):
    return a * np.log(a / b) - a + b


def _growth_prox_brute(s, c, lam, eps):
    """argmin over (s~^k, r^k) of eps sum_k KL(s~^k|s^k) + sum_k lam KL(s~^k|r^k)
    - lam (1 - c) sum_k r^k subject to sum_k r^k <= 1 (the prox problem of F2 with
    its inner infimum taken jointly; 2 tau alpha = lam (1 - c)); returns
    eps log(s~^k/s^k) and r^k."""
    s = np.asarray(s, dtype=float)
    S = s.size

    def obj(z):
        st, r = np.exp(z[:S]), np.exp(z[S:])
        return eps * np.sum(_kl(st, s)) + lam * np.sum(_kl(st, r)) - lam * (1.0 - c) * np.sum(r)

    best = None
    for z0 in (np.concatenate([np.log(s), np.full(S, math.log(0.5 / S))]),
               np.concatenate([np.log(s) - 1.0, np.full(S, math.log(0.9 / S))])):
        res = optimize.minimize(obj, z0, method="SLSQP",
                                constraints=[{"type": "ineq", "fun": lambda z: 1.0 - np.sum(np.exp(z[S:]))}],
                                options={"ftol": 1e-16, "maxiter": 5000})
        if best is None or res.fun < best.fun:
            best = res
    return eps * (best.x[:S] - np.log(s)), np.exp(best.x[S:])


@pytest.mark.parametrize("lam", [1.0, 0.6])
@pytest.mark.parametrize("s", [0.05, 0.5, 2.0, 7.0])
def test_growth_prox_single_species_brute_force(s, lam):
    """Sec. 5.3, tumor example: the log-form proxdiv of F2 (one species)
    against brute-force minimisation of its prox problem, on both sides of the
    switch s = c^{(lam+eps)/eps}; with lam = 1 also against the paper's printed
    case formula c^{-1/eps} / s^{-1/(1+eps)}."""
    c, eps = 0.8, 0.3
    V = O.prox_growth_log(np.array([[eps * math.log(s)]]), c, lam, eps)[0, 0]
    Vb, _ = _growth_prox_brute([s], c, lam, eps)
    assert abs(V - Vb[0]) < 2e-6
    if lam == 1.0:
        pdiv = c ** (-1.0 / eps) if s <= c ** ((1.0 + eps) / eps) else s ** (-1.0 / (1.0 + eps))
        assert abs(V - eps * math.log(pdiv)) < 1e-13


@pytest.mark.parametrize("lam", [1.0, 0.6])
@pytest.mark.parametrize("sa,sb", [(0.05, 0.02), (0.4, 1.1), (3.0, 0.2), (0.3, 0.3)])
def test_growth_prox_two_species_brute_force(sa, sb, lam):
    """Sec. 5.3, two species: both species get the same update, which
    minimises the joint prox problem; with lam = 1 it equals the paper's
    printed 1/beta(s^a, s^b), beta = max((s^a + s^b)^{1/(1+eps)}, c^{1/eps})."""
    c, eps = 0.7, 0.25
    T = eps * np.log(np.array([[sa], [sb]]))
    V = O.prox_growth_log(T, c, lam, eps)[:, 0]
    Vb, _ = _growth_prox_brute([sa, sb], c, lam, eps)
    assert np.max(np.abs(V - Vb)) < 2e-6
    if lam == 1.0:
        beta = max((sa + sb) ** (1.0 / (1.0 + eps)), c ** (1.0 / eps))
        assert np.max(np.abs(V - eps * math.log(1.0 / beta))) < 1e-13


def test_growth_prox_zero_input():
    """s = 0 (T = -inf): the prox problem's minimiser is s~ = 0 for any
    finite proxdiv; the case formula gives the constant branch c^{-1/eps}."""
    c, lam, eps = 0.6, 1.0, 0.1
    V = O.prox_growth_log(np.array([[-np.inf], [-np.inf]]), c, lam, eps)
    assert np.all(V == -lam * math.log(c))


@pytest.mark.parametrize("r2", [[0.3], [1.7], [0.1, 0.4], [0.9, 0.8], [0.0, 0.5]])
def test_growth_next_density_brute_force(r2):
    """Next densities = minimisers of F2's inner infimum at the plan's second
    marginals: argmin_{r >= 0, sum r <= 1} sum_k lam KL(r2^k|r^k) - lam (1 - c) sum_k r^k;
    one species: the paper's min(r2/c, 1)."""
    c, lam = 0.75, 1.0
    r2 = np.array(r2)
    got = O.growth_next_density(r2[:, None], c)[:, 0]
    pos = r2 > 0

    def obj(z):
        r = np.exp(z)
        return lam * np.sum(_kl(r2[pos], r)) - lam * (1.0 - c) * np.sum(r)

    res = optimize.minimize(obj, np.log(r2[pos] * 0.5 + 0.01), method="SLSQP",
                            constraints=[{"type": "ineq", "fun": lambda z: 1.0 - np.sum(np.exp(z))}],
                            options={"ftol": 1e-16, "maxiter": 5000})
    assert np.max(np.abs(got[pos] - np.exp(res.x))) < 1e-6
    assert np.all(got[~pos] == 0.0)
    if r2.size == 1:
        assert abs(got[0] - min(r2[0] / c, 1.0)) < 1e-15


def test_growth_next_log_density_is_the_log_of_the_density():
    """The log form that carries densities between steps equals the log of
    growth_next_density where that is representable, and stays finite (and
    ordered) where the density underflows FP64."""
    c = 0.8
    logR2 = np.array([[-3.0, 0.5, -2000.0, -np.inf], [-1.0, -4.0, -2001.0, -np.inf]])
    lp = O.growth_next_log_density(logR2, c)
    p = O.growth_next_density(np.exp(logR2), c)
    ok = p > 0
    assert np.max(np.abs(lp[ok] - np.log(p[ok]))) < 1e-14
    assert np.all(np.isfinite(lp[:, 2])) and lp[0, 2] - lp[1, 2] == 1.0
    assert np.all(np.isneginf(lp[:, 3]))


def _wf_step_problem(S):
    n = 5
    x = (np.arange(n) + 0.5) / n
    dx = np.full(n, 1.0 / n)
    g = np.random.default_rng(91 + S)
    P0 = g.uniform(0.2, 0.45, size=(S, n))
    return x, dx, P0


@pytest.mark.parametrize("S,lam", [(1, 1.0), (2, 1.0), (2, 0.7)])
def test_wf_step_matches_brute_force_minimisation(S, lam):
    """One step of the WF gradient flow (eq. grad-flow with the growth
    functional of Sec. 5.3) on 5 points with the cut locus at 0.5 (K = 0 for
    pairs 0.6 and 0.8 apart): the oracle's plans e^{(U_i + V_j - c_ij)/eps} and
    next densities minimise
      sum_k [lam KL(R^k dy | p^k)_dx + lam KL(R^k^T dx | mu^k)_dx + eps KL(R^k | K)_{dx dy}]
      - 2 tau alpha sum_j dx_j sum_k mu^k_j,   sum_k mu^k <= 1,
    jointly over the plans on the kernel's support and the densities mu^k,
    found by SLSQP."""
    x, dx, P0 = _wf_step_problem(S)
    n = x.size
    tau, alpha, eps = 0.05, 1.0, 0.05
    C = O.wf_cost(x, x, 0.5)
    r = O.wf_flow_log(O.Geometry("dense", C=C), dx, P0, tau, alpha, lam, eps, nsteps=1, iters=3000)
    sup = np.isfinite(C)
    K = np.exp(-C[sup] / eps)
    w = (dx[:, None] * dx[None, :])[sup]
    nz = int(sup.sum())

    def unpack(z):
        R = np.zeros((S, n, n))
        for k in range(S):
            R[k][sup] = np.exp(z[k * nz:(k + 1) * nz])
        return R, np.exp(z[S * nz:].reshape(S, n))

    def obj(z):
        R, mu = unpack(z)
        v = 0.0
        for k in range(S):
            r1, r2 = R[k] @ dx, R[k].T @ dx
            v += lam * np.sum(dx * _kl(r1, P0[k])) + lam * np.sum(dx * _kl(r2, mu[k]))
            Rk = R[k][sup]
            v += eps * np.sum(w * (Rk * np.log(Rk / K) - Rk + K))
        return v - 2.0 * tau * alpha * np.sum(dx * np.sum(mu, axis=0))  # 2 tau G, G = -alpha mass

    Ro = np.stack([np.where(sup, np.exp((r["U"][k][:, None] + r["V"][k][None, :] - C) / eps), 0.0)
                   for k in range(S)])
    muo = r["P"][0]
    z0 = np.concatenate([np.log(Ro[k][sup]) + 0.1 for k in range(S)] + [np.log(muo).ravel() - 0.1])
    res = optimize.minimize(obj, z0, method="SLSQP",
                            constraints=[{"type": "ineq", "fun": lambda z: 1.0 - np.sum(unpack(z)[1], axis=0)}],
                            options={"ftol": 1e-16, "maxiter": 20000})
    zo = np.concatenate([np.log(Ro[k][sup]) for k in range(S)] + [np.log(muo).ravel()])
    assert obj(zo) <= res.fun + 1e-10
    Rb, mub = unpack(res.x)
    assert np.max(np.abs(mub - muo)) < 2e-4
    assert np.max(np.abs(Rb - Ro)) < 2e-3 * np.max(Ro)
    assert np.all(np.sum(muo, axis=0) <= 1.0 + 1e-12)


# --------------------------------------------------------------------------
# colour transfer (Sec. 5.1): histogram, barycentric projection, bin map
# --------------------------------------------------------------------------

def test_bin_index_edges():
    """Bin k of an axis covers [k/n, (k+1)/n): hand-computed bins, including
    the edges, 1 itself and points outside the cube (clamped)."""
    shape = (4, 2)
    pts = np.array([[0.0, 0.0], [0.25, 0.5], [0.2499, 0.4999], [1.0, 1.0], [0.99, 0.01],
                    [-0.3, 2.0], [0.5, 0.75]])
    want = [0 * 2 + 0, 1 * 2 + 1, 0 * 2 + 0, 3 * 2 + 1, 3 * 2 + 0, 0 * 2 + 1, 2 * 2 + 1]
    assert O.bin_index(pts, shape).tolist() == want


def test_color_histogram_mass_and_counts():
    g = np.random.default_rng(3)
    pts = g.uniform(0, 1, size=(1000, 3))
    shape = (8, 4, 4)
    p = O.color_histogram(pts, shape)
    assert abs(p.sum() - 1.0) < 1e-15
    # brute force: count the points inside each bin's box
    i0, i1, i2 = 5, 2, 3
    box = ((pts[:, 0] >= i0 / 8) & (pts[:, 0] < (i0 + 1) / 8) & (pts[:, 1] >= i1 / 4) & (pts[:, 1] < (i1 + 1) / 4)
           & (pts[:, 2] >= i2 / 4) & (pts[:, 2] < (i2 + 1) / 4))
    assert p[(i0 * 4 + i1) * 4 + i2] == box.sum() / 1000


def test_barycentric_projection_1d_monotone_rearrangement():
    """Balanced 1-D OT with equal uniform weights is the monotone
    rearrangement (textbook): as eps -> 0 the barycentric projection sends the
    k-th smallest x to the k-th smallest y."""
    g = np.random.default_rng(11)
    n = 12
    # spaced points: every swap of two matched targets costs 2 dx dy >> eps
    x = (np.arange(n) + 0.5) / n + g.uniform(-0.01, 0.01, n)
    y = ((np.arange(n) + 0.5) / n) ** 2 + g.uniform(-0.002, 0.002, n)
    g.shuffle(x)
    geo = O.Geometry("points", x=x[:, None], y=y[:, None])
    w = np.full(n, 1.0 / n)
    eps = 2e-4
    r = O.solve_log(geo, w, w, np.ones(n), np.ones(n), O.EQ(), O.EQ(), eps, max_iter=20000, tol=1e-12)
    T = O.barycentric_projection(geo, w, w, r["U"], r["V"], eps)[:, 0]
    ranks = np.argsort(np.argsort(x))
    assert np.max(np.abs(T - y[ranks])) < 2e-3


def test_barycentric_projection_large_eps_is_the_mean():
    """As eps -> inf the balanced entropic plan tends to the independent
    coupling p x q, whose barycentric projection is the mean of nu for every x."""
    geo, dx, dy, p, q = small_problem(7, 9, 4, d=2)
    q = q / np.sum(q * dy) * np.sum(p * dx)
    eps = 1e6
    r = O.solve_log(geo, dx, dy, p, q, O.EQ(), O.EQ(), eps, max_iter=200)
    T = O.barycentric_projection(geo, dx, dy, r["U"], r["V"], eps)
    mean = (q * dy) @ geo.y / np.sum(q * dy)
    assert np.max(np.abs(T - mean[None, :])) < 1e-5


def test_barycentric_projection_zero_rows_keep_their_point():
    geo, dx, dy, p, q = small_problem(6, 5, 8, d=2)
    U = np.zeros(6)
    U[2] = -np.inf
    T = O.barycentric_projection(geo, dx, dy, U, np.zeros(5), 0.1)
    assert np.array_equal(T[2], geo.x[2])
    assert np.all((T >= geo.y.min(axis=0) - 1e-12) & (T <= geo.y.max(axis=0) + 1e-12))  # convex combinations


def test_apply_bin_map_gathers_by_bin():
    shape = (2, 2)
    T = np.array([[0.1, 0.2], [0.3, 0.4], [0.5, 0.6], [0.7, 0.8]])
    pts = np.array([[0.1, 0.1], [0.9, 0.1], [0.1, 0.9], [0.6, 0.6]])
    out = O.apply_bin_map(pts, shape, T)
    assert out.tolist() == [[0.1, 0.2], [0.5, 0.6], [0.3, 0.4], [0.7, 0.8]]


# --------------------------------------------------------------------------
# Direct pins of the helpers the solvers call
# --------------------------------------------------------------------------

def test_eps_schedule_is_geometric_down_to_eps():
    """eps-scaling (Sec. 4.4): the stages start at eps_start and divide eps by
    one fixed factor, and the division after the last stage lands on the final
    eps; no stages when there is nothing to scale."""
    st = O.eps_schedule(1e-3, eps_start=0.1, stages=4, iters_per_stage=7)
    assert len(st) == 4 and all(k == 7 for _, k in st)
    e = [v for v, _ in st]
    assert e[0] == 0.1
    assert np.allclose([e[k] / e[k + 1] for k in range(3)], 100.0 ** 0.25, rtol=1e-14, atol=0)
    assert math.isclose(e[-1] / 100.0 ** 0.25, 1e-3, rel_tol=1e-13)
    assert O.eps_schedule(1e-3) == [] and O.eps_schedule(1e-3, eps_start=1e-3) == []
    assert O.eps_schedule(1e-3, eps_start=1e-4) == [] and O.eps_schedule(1e-3, eps_start=0.1, stages=0) == []


def test_grid_axes_and_points_enumerate_the_bins():
    """Colour grid (Sec. 5.1): bin k of an n-bin axis of [0, 1] is centred at
    (k + 1/2)/n, and the grid's points are listed row-major (last axis
    fastest), as a brute-force product of the axes lists them."""
    import itertools
    axes = O.grid_axes((2, 3, 4))
    assert [len(a) for a in axes] == [2, 3, 4]
    assert axes[0].tolist() == [0.25, 0.75] and axes[1].tolist() == [1 / 6, 0.5, 5 / 6]
    pts = O.grid_points(axes)
    assert pts.shape == (24, 3)
    assert np.array_equal(pts, np.array(list(itertools.product(*[a.tolist() for a in axes]))))


def test_growth_c_values():
    """Sec. 5.3: the growth term -alpha mu(X) over a step tau enters the
    proxdiv through c = 1 - 2 tau alpha / lam: 0.988 in the paper's one-species
    run (tau = 0.006, alpha = 1, lam = 1), 1 without growth, and no step once
    2 tau alpha reaches lam."""
    assert math.isclose(O.growth_c(0.006, 1.0, 1.0), 0.988, rel_tol=1e-15)
    assert O.growth_c(0.3, 0.0, 2.0) == 1.0
    for tau in (0.5, 0.6):
        with pytest.raises(ValueError):
            O.growth_c(tau, 1.0, 1.0)


@pytest.mark.parametrize("lam", [None, 0.7, 3.0])
def test_mass_update_log_by_brute_force(lam):
    """Algorithm 4 (Sec. 4.5): z = proxdiv_F3(M) with M = sum_i dx_i
    e^{(U_i + S_i)/eps}, the plan's mass without z, summed here term by term.
    F3 = iota_{=m0}: z M = m0 exactly.  F3 = lam KL(.|m0): z M is the minimiser
    y of (lam/eps) KL(y|m0) + KL(y|M) (the prox of Table 1), found from its
    optimality condition (lam/eps) log(y/m0) + log(y/M) = 0 by bisection."""
    g = synth.rng(5)
    n, eps, m0 = 9, 0.05, 1.7
    U = g.normal(size=n) * 0.05
    S = g.normal(size=n) * 0.05
    U[2] = -np.inf
    dx = g.uniform(0.5, 1.5, size=n) / n
    M = sum(dx[i] * math.exp((U[i] + S[i]) / eps) for i in range(n) if np.isfinite(U[i]))
    F3 = O.EQ() if lam is None else O.KL(lam)
    Z = O.mass_update_log(F3, m0, U, S, np.log(dx), eps)
    zM = math.exp(Z / eps) * M
    if lam is None:
        assert math.isclose(zM, m0, rel_tol=1e-12)
    else:
        assert abs(M - m0) > 0.05  # a proper bracket
        y = optimize.brentq(lambda t: (lam / eps) * math.log(t / m0) + math.log(t / M), min(m0, M), max(m0, M),
                            xtol=1e-15, rtol=4 * np.finfo(float).eps)
        assert math.isclose(zM, y, rel_tol=1e-11)
        # the KL row pulls the mass toward m0, more so the larger lam
        assert min(m0, M) < zM < max(m0, M)


def test_points_streamed_operator_by_brute_force():
    """Sec. 4.3: S_i = eps log sum_j w_j exp((V_j - |x_i - y_j|^2)/eps), term
    by term with math.exp, for 7 x 5 points in 2-D; the stream is cut into
    blocks of 3 rows (a ragged last block)."""
    g = synth.rng(8)
    x = g.uniform(0, 1, size=(7, 2))
    y = g.uniform(0, 1, size=(5, 2))
    V = g.normal(size=5) * 0.1
    w = g.uniform(0.5, 1.5, size=5)
    eps = 0.3
    got = O.apply_K_points_streamed(x, y, V, np.log(w), eps, block=3)
    for i in range(7):
        s = sum(w[j] * math.exp((V[j] - ((x[i, 0] - y[j, 0]) ** 2 + (x[i, 1] - y[j, 1]) ** 2)) / eps)
                for j in range(5))
        assert math.isclose(got[i], eps * math.log(s), rel_tol=1e-13, abs_tol=1e-14)


def test_safe_log_conventions():
    """Zero masses (Prop. 5.1, 0/0 = 0) need log 0 = -inf, quietly."""
    got = O.safe_log([0.0, 1.0, math.e, 2.0])
    assert got[0] == -math.inf and got[1] == 0.0
    assert math.isclose(got[2], 1.0, rel_tol=1e-15) and got[3] == math.log(2.0)


def test_violation_measure_on_a_hand_example():
    """The stopping measure: sum dx |r1 - rho1| / sum dx rho1, r1 the first
    marginal of the current plan and rho1 its prox target.  With S = 0,
    U_old = eps (0, log 2), U_new = eps (log 3, 0), dx = (1/4, 3/4): r1 = (1, 2),
    rho1 = (3, 1), so (1/4 * 2 + 3/4 * 1) / (1/4 * 3 + 3/4 * 1) = 5/6; a third
    point with S = -inf (no plan mass) changes nothing."""
    from oracle.uot_oracle import _violation_from
    eps = 0.1
    U_old = np.array([0.0, eps * math.log(2.0), 0.4])
    U_new = np.array([eps * math.log(3.0), 0.0, -0.2])
    S = np.array([0.0, 0.0, -np.inf])
    logdx = np.log([0.25, 0.75, 0.5])
    assert math.isclose(_violation_from(U_old, U_new, S, logdx, eps), 5.0 / 6.0, rel_tol=1e-14)


# --------------------------------------------------------------------------
# translation step along (U + c, V - c), KL penalties (not in the paper)
# --------------------------------------------------------------------------

@pytest.mark.parametrize("l1,l2", [(0.5, 0.5), (0.3, 2.0)])
def test_translation_maximises_the_dual_on_its_line(l1, l2):
    """kl_translation's c against a brute-force 1-D maximisation of D_eps
    (Theorem 3.2) over t on the line (U + t, V - t), non-uniform weights, a
    zero density (U = -inf there), a state pushed off the line's maximum."""
    geom, dx, dy, p, q = small_problem(7, 6, 31, zeros=True)
    eps = 0.05
    F1, F2 = O.KL(l1), O.KL(l2)
    logs = (np.log(dx), np.log(dy), O.safe_log(p), np.log(q))
    U, V = O.iterate_log(geom, *logs, F1, F2, eps, 3)
    U, V = U + 0.4, V - 0.1
    c = O.kl_translation(*logs, F1, F2, U, V)
    r = optimize.minimize_scalar(lambda t: -O.dual(geom, dx, dy, p, q, F1, F2, eps, U + t, V - t),
                                 bracket=(-1.0, 0.0, 1.0), tol=1e-12)
    assert abs(c - r.x) <= 1e-6, (c, r.x)
    Ut, Vt = O.translate_log(*logs, F1, F2, U, V)
    assert np.array_equal(np.isneginf(Ut), np.isneginf(U))
    assert O.dual(geom, dx, dy, p, q, F1, F2, eps, Ut, Vt) > O.dual(geom, dx, dy, p, q, F1, F2, eps, U, V)
    # the plan, hence its marginals, is unchanged
    for a, b in zip(O.marginals(geom, dx, dy, Ut, Vt, eps), O.marginals(geom, dx, dy, U, V, eps)):
        assert np.allclose(a, b, rtol=1e-12, atol=0)


def test_translation_keeps_the_dual_ascent_monotone():
    """Sinkhorn half-steps and the translation step are exact maximisations of
    D_eps over blocks of variables: the dual never decreases."""
    geom, dx, dy, p, q = small_problem(8, 9, 32)
    eps = 0.03
    F1, F2 = O.KL(2.0), O.KL(0.7)
    logs = (np.log(dx), np.log(dy), np.log(p), np.log(q))
    U, V = O.iterate_log(geom, *logs, F1, F2, eps, 1)
    prev = O.dual(geom, dx, dy, p, q, F1, F2, eps, U, V)
    for _ in range(40):
        U, V = O.iterate_log(geom, *logs, F1, F2, eps, 1, U, V, translate_every=1)
        d = O.dual(geom, dx, dy, p, q, F1, F2, eps, U, V)
        assert d >= prev - 1e-13 * abs(prev)
        prev = d


def test_translation_same_fixed_point_fewer_iterations():
    """With lambda / eps = 300 the plain iteration's translation mode decays
    by (lam / (lam + eps))^2 per iteration; the translated iteration reaches the
    same fixed point in a small fraction of the iterations."""
    xs = [synth.grid_axis(50)]
    ys = [synth.grid_axis(45)]
    geom = O.Geometry("grid", xs=xs, ys=ys)
    g = synth.rng(33)
    dx, dy = np.full(50, 1 / 50), np.full(45, 1 / 45)
    p = g.uniform(0.2, 2.0, 50)
    q = 1.7 * g.uniform(0.2, 2.0, 45)
    F = O.KL(3.0)
    eps = 0.01
    plain = O.solve_log(geom, dx, dy, p, q, F, F, eps, max_iter=100000, tol=1e-11, check_every=5)
    tr = O.solve_log(geom, dx, dy, p, q, F, F, eps, max_iter=100000, tol=1e-11, check_every=5, translate=True)
    assert plain["err"] <= 1e-11 and tr["err"] <= 1e-11
    assert tr["iters"] * 4 < plain["iters"], (tr["iters"], plain["iters"])
    assert np.max(np.abs(tr["U"] - plain["U"])) <= 1e-7
    assert np.max(np.abs(tr["V"] - plain["V"])) <= 1e-7


def test_translation_requires_kl():
    geom, dx, dy, p, q = small_problem(4, 4, 34)
    with pytest.raises(ValueError):
        O.kl_translation(np.log(dx), np.log(dy), np.log(p), np.log(q), O.KL(1.0), O.TV(1.0), np.zeros(4), np.zeros(4))

"""Plain, slow FP64 oracle of the generalized Sinkhorn scaling iterations.

TEST INFRASTRUCTURE ONLY.  Nothing on the product path may import or call
this module; only the tests, the smoke check and the CPU-baseline leg of the
benchmark do.  It shares no code with the CUDA library.

Everything follows Chizat, Peyre, Schmitzer, Vialard, "Scaling algorithms for
unbalanced optimal transport problems" (arXiv:1607.05816):

* discrete problem (eq. primal_discr, Sec. 4.2): points x_i, y_j with reference
  probability weights dx, dy, densities p, q (mu = p dx, nu = q dy), cost C,
  Gibbs kernel K = exp(-C/eps) (eq. GibbsKernel);
* Gibbs operators  K b = K (b . dy),  K^T a = K^T (a . dx)  (Sec. 4.2);
* proxdiv operators of Table 1 (Sec. 5.1) for the equality constraint,
  lambda KL, lambda TV and the range constraint RG[alpha, beta];
* Algorithm 1 (scaling algorithm), Algorithm 2 (stabilized scaling algorithm
  with absorption) and the log-domain form of Algorithm 2 in which absorption
  happens after every update, so the scalings a~, b~ stay 1 and only the dual
  potentials u = eps log a, v = eps log b are stored (Sec. 4.3);
* eps-scaling (Sec. 4.4, "Gradually decreasing eps");
* separable Gaussian kernel on Cartesian grids applied by successive 1-D
  operations (Sec. 4.4, "Computing the matrix multiplications");
* primal (P_eps) and dual (D_eps) functionals (Theorem 3.2) and their gap;
* unbalanced barycenters (Sec. 5.2) with the KL row of Table 2;
* Algorithm 4 (a divergence on the plan's total mass, Sec. 4.5);
* WF gradient flows with growth (Sec. 2 "Gradient flows", Sec. 5.3): the WF
  cost of eq. logcost, the joint proxdiv of the growth functional for one or
  several species, and the minimizing-movement steps.

Notation used in code: U = eps log a, V = eps log b (total potentials),
S_i = eps log (K b)_i, T_j = eps log (K^T a)_j.  Readings of points the paper
leaves open are listed in the module-level constants and docstrings below.

All arithmetic is numpy float64.  Log-sum-exp uses a max shift, with the
convention that an all -inf slice gives -inf (exp(-inf) = 0, Sec. 3.2).

Parity status: every public function here is pinned by a CPU test against a
closed form, an invariant, a brute-force minimisation or an independent form
of the same operation (tests/test_oracle_*.py).
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np

NEG_INF = -np.inf

# ----------------------------------------------------------------------------
# divergences (Sec. 2.1, Table 1)
# ----------------------------------------------------------------------------


@dataclass
class Div:
    """A marginal penalty F(s) = sum_i dx_i D_phi(s_i | p_i) (eq. divergencefunctions).

    kind: 'eq' (iota_=), 'kl' (lam KL), 'tv' (lam TV), 'rg' (RG[alpha, beta]).
    """
    kind: str
    lam: float = 1.0
    alpha: float = 0.0
    beta: float = math.inf


def EQ():
    return Div("eq")


def KL(lam):
    return Div("kl", lam=lam)


def TV(lam):
    return Div("tv", lam=lam)


def RG(alpha, beta):
    return Div("rg", alpha=alpha, beta=beta)


# ----------------------------------------------------------------------------
# log-sum-exp
# ----------------------------------------------------------------------------


def lse(z: np.ndarray, axis=-1) -> np.ndarray:
    """log sum exp along `axis`, max-shifted; an all -inf slice gives -inf."""
    z = np.asarray(z, dtype=np.float64)
    m = np.max(z, axis=axis, keepdims=True)
    m_safe = np.where(np.isfinite(m), m, 0.0)
    with np.errstate(divide="ignore"):
        s = np.log(np.sum(np.exp(z - m_safe), axis=axis, keepdims=True)) + m_safe
    s = np.where(np.isneginf(m), NEG_INF, s)
    return np.squeeze(s, axis=axis)


def safe_log(x):
    with np.errstate(divide="ignore"):
        return np.log(np.asarray(x, dtype=np.float64))


# ----------------------------------------------------------------------------
# geometries and the Gibbs operators in the log domain (Sec. 4.2, 4.3, 4.4)
# ----------------------------------------------------------------------------


def sqdist(x: np.ndarray, y: np.ndarray) -> np.ndarray:
    """C_ij = |x_i - y_j|^2 for point arrays x (n,d), y (m,d) or 1-D coordinates."""
    x = np.asarray(x, dtype=np.float64)
    y = np.asarray(y, dtype=np.float64)
    if x.ndim == 1:
        x = x[:, None]
    if y.ndim == 1:
        y = y[:, None]
    diff = x[:, None, :] - y[None, :, :]
    return np.sum(diff * diff, axis=-1)


def grid_points(axes) -> np.ndarray:
    """Flattened (row-major) point list of the Cartesian grid with these axes."""
    mesh = np.meshgrid(*[np.asarray(a, dtype=np.float64) for a in axes], indexing="ij")
    return np.stack([g.ravel() for g in mesh], axis=-1)


@dataclass
class Geometry:
    """Where the points live and how the cost is given.

    kind 'dense' : explicit cost matrix C (n x m).
    kind 'points': point clouds x (n,d), y (m,d), cost |x - y|^2.
    kind 'grid'  : Cartesian grids with 1-D axes xs, ys (same number of axes),
                   cost |x - y|^2; potentials are arrays of the grid's shape.
    """
    kind: str
    C: np.ndarray | None = None
    x: np.ndarray | None = None
    y: np.ndarray | None = None
    xs: list = field(default_factory=list)
    ys: list = field(default_factory=list)

    def cost_matrix(self) -> np.ndarray:
        """The full cost matrix (the definition; used for small problems)."""
        if self.kind == "dense":
            return np.asarray(self.C, dtype=np.float64)
        if self.kind == "points":
            return sqdist(self.x, self.y)
        return sqdist(grid_points(self.xs), grid_points(self.ys))


def apply_K_log(geom: Geometry, V: np.ndarray, logw: np.ndarray, eps: float,
                transpose: bool = False, separable: bool = True) -> np.ndarray:
    """Log-domain Gibbs operator.

    transpose=False: S_i = eps * log sum_j exp((V_j - C_ij)/eps) w_j
                          = eps * log (K (b . w))_i   with b = exp(V/eps)
    transpose=True : same with C^T (the K^T a of Sec. 4.2).
    `logw` is log dy (or log dx); V and logw have the shape of the input side.

    For grids with separable=True the sum over the product grid is taken one
    axis at a time, which is exact because exp(-|x-y|^2/eps) is the product of
    the 1-D kernels exp(-(x_k - y_k)^2/eps) (Sec. 4.4).  Otherwise the full
    cost matrix is formed and the sum is taken directly.
    """
    V = np.asarray(V, dtype=np.float64)
    L = V / eps + np.asarray(logw, dtype=np.float64)
    if geom.kind == "grid" and separable:
        out_axes = geom.ys if transpose else geom.xs
        in_axes = geom.xs if transpose else geom.ys
        Z = L
        for ax in range(len(in_axes)):
            c = sqdist(out_axes[ax], in_axes[ax]) / eps  # (n_out_ax, n_in_ax)
            Zm = np.moveaxis(Z, ax, -1)  # (..., n_in_ax)
            Zn = lse(Zm[..., None, :] - c, axis=-1)  # (..., n_out_ax)
            Z = np.moveaxis(Zn, -1, ax)
        return eps * Z
    C = geom.cost_matrix()
    if transpose:
        C = C.T
    Lf = L.ravel()
    out = np.empty(C.shape[0])
    # row by row keeps memory bounded for large point clouds
    step = max(1, int(2**24 // max(1, C.shape[1])))
    for r0 in range(0, C.shape[0], step):
        out[r0:r0 + step] = lse(Lf[None, :] - C[r0:r0 + step] / eps, axis=-1)
    shape = (tuple(len(a) for a in (geom.ys if transpose else geom.xs))
             if geom.kind == "grid" else out.shape)
    return eps * out.reshape(shape)


def apply_K_points_streamed(x, y, V, logw, eps, block=2048):
    """Point-cloud log-domain Gibbs operator without forming all of C at once
    (same definition as apply_K_log for kind 'points'; used for big clouds)."""
    x = np.asarray(x, dtype=np.float64)
    y = np.asarray(y, dtype=np.float64)
    L = np.asarray(V, dtype=np.float64) / eps + np.asarray(logw, dtype=np.float64)
    out = np.empty(x.shape[0])
    for r0 in range(0, x.shape[0], block):
        c = sqdist(x[r0:r0 + block], y)
        out[r0:r0 + block] = lse(L[None, :] - c / eps, axis=-1)
    return eps * out


# ----------------------------------------------------------------------------
# Table 1: prox and proxdiv
# ----------------------------------------------------------------------------


def prox_update_log(F: Div, logp: np.ndarray, S: np.ndarray, eps: float) -> np.ndarray:
    """Log form of a <- proxdiv_F(K b, eps) with u = 0 (Table 1, Sec. 5.1).

    Returns U = eps log a given S = eps log (K b) and log p.  With
    Ubar = eps log p - S (the equality-constraint update, Table 1 row 1):
      iota_= : U = Ubar
      lam KL : U = lam/(lam+eps) Ubar
      lam TV : U = min(lam, max(-lam, Ubar))
      RG     : U = min(eps log beta + Ubar, max(eps log alpha + Ubar, 0))
    Zero masses follow Prop. 5.1 with 0/0 = 0: where s = K b = 0 the prox is 0
    and so is a (U = -inf); where p = 0 the TV row gives a = e^{-lam/eps}.
    """
    logp = np.asarray(logp, dtype=np.float64)
    S = np.asarray(S, dtype=np.float64)
    s_zero = np.isneginf(S)
    p_zero = np.isneginf(logp)
    S_f = np.where(s_zero, 0.0, S)
    ubar = np.where(p_zero, NEG_INF, eps * np.where(p_zero, 0.0, logp) - S_f)
    if F.kind == "eq":
        U = ubar
    elif F.kind == "kl":
        U = (F.lam / (F.lam + eps)) * ubar
    elif F.kind == "tv":
        U = np.clip(ubar, -F.lam, F.lam)  # clip(-inf) = -lam (p = 0 row)
    elif F.kind == "rg":
        lo = NEG_INF if F.alpha == 0 else eps * math.log(F.alpha)
        inner = np.maximum(lo + ubar, 0.0)  # -inf + finite = -inf
        if math.isinf(F.beta):
            U = inner
        else:
            U = np.minimum(eps * math.log(F.beta) + ubar, inner)
    else:
        raise ValueError(F.kind)
    return np.where(s_zero, NEG_INF, U)


def proxdiv(F: Div, p: np.ndarray, s: np.ndarray, u: np.ndarray | float, eps: float) -> np.ndarray:
    """Table 1 literally: proxdiv_F(s, u, eps) = prox^KL_{F/eps}(e^{-u/eps} s) / s.

    Non-log form used by Algorithms 1 and 2; 0/0 = 0 where s = 0 (Prop. 5.1).
    """
    p = np.asarray(p, dtype=np.float64)
    s = np.asarray(s, dtype=np.float64)
    u = np.broadcast_to(np.asarray(u, dtype=np.float64), s.shape)
    with np.errstate(divide="ignore", invalid="ignore", over="ignore"):
        ps = np.where(s > 0, p / np.where(s > 0, s, 1.0), 0.0)
        if F.kind == "eq":
            out = ps
        elif F.kind == "kl":
            out = ps ** (F.lam / (F.lam + eps)) * np.exp(-u / (F.lam + eps))
        elif F.kind == "tv":
            out = np.minimum(np.exp((F.lam - u) / eps), np.maximum(np.exp(-(F.lam + u) / eps), ps))
        elif F.kind == "rg":
            lo = F.alpha * ps
            hi = F.beta * ps if not math.isinf(F.beta) else np.inf
            out = np.minimum(hi, np.maximum(lo, np.exp(-u / eps)))
        else:
            raise ValueError(F.kind)
    return np.where(s > 0, out, 0.0)


def prox_target_log(F: Div, logp, S, eps):
    """log prox^KL_{F/eps}(s) for s = e^{S/eps} (middle column of Table 1)."""
    U = prox_update_log(F, logp, S, eps)
    with np.errstate(invalid="ignore"):
        return np.where(np.isneginf(U), NEG_INF, (U + S) / eps)


# ----------------------------------------------------------------------------
# Algorithms 1 and 2 (Sec. 4.2, 4.3) on an explicit kernel matrix
# ----------------------------------------------------------------------------


def scaling_alg1(K, dx, dy, p, q, F1: Div, F2: Div, eps: float, iters: int):
    """Algorithm 1 verbatim: b <- 1; repeat a <- proxdiv_F1(K(b.dy)),
    b <- proxdiv_F2(K^T(a.dx)).  Returns the scalings (a, b)."""
    K = np.asarray(K, dtype=np.float64)
    b = np.ones(K.shape[1])
    a = np.ones(K.shape[0])
    for _ in range(iters):
        a = proxdiv(F1, p, K @ (b * dy), 0.0, eps)
        b = proxdiv(F2, q, K.T @ (a * dx), 0.0, eps)
    return a, b


def scaling_alg2(C, dx, dy, p, q, F1: Div, F2: Div, eps: float, iters: int,
                 tau: float = 10.0):
    """Algorithm 2 verbatim with absorption when max |log a~|, |log b~| > tau.

    Returns the total potentials U = u + eps log a~, V = v + eps log b~.
    """
    C = np.asarray(C, dtype=np.float64)
    bt = np.ones(C.shape[1])
    at = np.ones(C.shape[0])
    u = np.zeros(C.shape[0])
    v = np.zeros(C.shape[1])
    Kt = np.exp(-C / eps)
    nabs = 0
    for _ in range(iters):
        at = proxdiv(F1, p, Kt @ (bt * dy), u, eps)
        bt = proxdiv(F2, q, Kt.T @ (at * dx), v, eps)
        with np.errstate(divide="ignore"):
            big = max(np.max(np.abs(np.log(at[at > 0])), initial=0.0),
                      np.max(np.abs(np.log(bt[bt > 0])), initial=0.0))
        if big > tau:
            u = u + eps * safe_log(at)
            v = v + eps * safe_log(bt)
            with np.errstate(invalid="ignore"):
                Kt = np.exp((u[:, None] + v[None, :] - C) / eps)
            Kt = np.where(np.isnan(Kt), 0.0, Kt)
            bt = np.ones(C.shape[1])
            at = np.ones(C.shape[0])
            nabs += 1
    with np.errstate(invalid="ignore"):
        U = u + eps * safe_log(at)
        V = v + eps * safe_log(bt)
    return U, V, nabs


# ----------------------------------------------------------------------------
# log-domain iteration (Algorithm 2 with absorption after every update)
# ----------------------------------------------------------------------------


def eps_schedule(eps_final: float, eps_start: float | None = None, stages: int = 10,
                 iters_per_stage: int = 100):
    """eps-scaling (Sec. 4.4): from eps_start, divide eps by a fixed factor
    `stages` times, `iters_per_stage` iterations before each division, so the
    last division lands on eps_final.  Returns [(eps, n_iters)] for the
    stages before the final one; None/equal start gives []."""
    if eps_start is None or stages <= 0 or eps_start <= eps_final:
        return []
    rho = (eps_start / eps_final) ** (1.0 / stages)
    return [(eps_start / rho ** s, iters_per_stage) for s in range(stages)]


def kl_translation(logdx, logdy, logp, logq, F1: Div, F2: Div, U, V) -> float:
    """The shift c for which (U + c, V - c) maximises the dual D_eps (Theorem
    3.2) along the direction (1, -1), for lam1 KL and lam2 KL penalties.

    NOT part of the paper's algorithms: this is the translation step of the
    translation-invariant formulation of Sejourne, Vialard, Peyre (2022),
    restated here from the dual.  U + c and V - c leave U_i + V_j, hence the
    plan and the entropic term of D_eps, unchanged, so along the line only
    -F1*(-U - c) - F2*(-V + c) varies; with the KL conjugate (div_conj) its
    derivative in c is A e^{-c/lam1} - B e^{c/lam2}, A = sum_i dx_i p_i
    e^{-U_i/lam1}, B = sum_j dy_j q_j e^{-V_j/lam2} (the masses of the marginals
    that the optimality conditions predict), which vanishes at
        c = lam1 lam2 / (lam1 + lam2) (log A - log B).
    Entries with p_i = 0 (U_i = -inf) contribute nothing; c = 0 when either
    measure is zero."""
    if F1.kind != "kl" or F2.kind != "kl":
        raise ValueError("the translation step is defined here for KL penalties on both sides")
    U = np.ravel(U)
    V = np.ravel(V)
    ta = np.ravel(logdx + logp)
    tb = np.ravel(logdy + logq)
    fa = np.isfinite(ta) & np.isfinite(U)
    fb = np.isfinite(tb) & np.isfinite(V)
    if not fa.any() or not fb.any():
        return 0.0
    la = float(lse(ta[fa] - U[fa] / F1.lam))
    lb = float(lse(tb[fb] - V[fb] / F2.lam))
    return F1.lam * F2.lam / (F1.lam + F2.lam) * (la - lb)


def translate_log(logdx, logdy, logp, logq, F1: Div, F2: Div, U, V):
    """(U + c, V - c) with c = kl_translation (finite entries only)."""
    c = kl_translation(np.broadcast_to(logdx, np.shape(logp)), np.broadcast_to(logdy, np.shape(logq)),
                       logp, logq, F1, F2, U, V)
    return U + c, V - c


def iterate_log(geom: Geometry, logdx, logdy, logp, logq, F1: Div, F2: Div,
                eps: float, iters: int, U=None, V=None, history: bool = False,
                translate_every: int = 0):
    """`iters` scaling iterations in the log domain at fixed eps.

    One iteration (eq. S, Sec. 3.3, in the log form of Sec. 4.3):
      S = eps log K(b.dy);  U = prox_update_F1(S)
      T = eps log K^T(a.dx); V = prox_update_F2(T)
    Starts from V = 0 (b = 1, Algorithm 1) unless V is given.
    translate_every > 0 (KL on both sides; not in the paper): after the
    V-update of iterations translate_every, 2 translate_every, ... the
    translation step of translate_log.
    Returns U, V and, if history, the marginal violation of each iterate
    (see marginal_violation) computed before the a-update that follows it.
    """
    if V is None:
        V = np.zeros(np.shape(logq))
    if U is None:
        U = np.zeros(np.shape(logp))
    errs = []
    for k in range(iters):
        S = apply_K_log(geom, V, logdy, eps)
        Un = prox_update_log(F1, logp, S, eps)
        if history:
            errs.append(_violation_from(U, Un, S, logdx, eps))
        U = Un
        T = apply_K_log(geom, U, logdx, eps, transpose=True)
        V = prox_update_log(F2, logq, T, eps)
        if translate_every > 0 and (k + 1) % translate_every == 0:
            U, V = translate_log(logdx, logdy, logp, logq, F1, F2, U, V)
    return (U, V, errs) if history else (U, V)


def solve_log(geom: Geometry, dx, dy, p, q, F1: Div, F2: Div, eps: float,
              max_iter: int, tol: float = 0.0, eps_start=None, stages: int = 10,
              iters_per_stage: int = 100, check_every: int = 1, U0=None, V0=None,
              translate: bool = False):
    """eps-scaling then iterations at eps until marginal_violation <= tol.

    The violation is measured every `check_every` iterations, in iterations
    number check_every, 2 check_every, ... (and the last one).  The check of
    iterate l happens inside iteration l+1 (its a-update), so the returned
    state is one iteration past the first one under tol; `iters` counts
    iterations at the final eps only.
    translate (KL on both sides; not in the paper): the translation step of
    translate_log after the V-update of every checked iteration, and of
    iterations check_every, 2 check_every, ... of each eps-scaling stage.
    """
    logdx, logdy, logp, logq = map(safe_log, (dx, dy, p, q))
    U, V = U0, V0
    for e, n in eps_schedule(eps, eps_start, stages, iters_per_stage):
        U, V = iterate_log(geom, logdx, logdy, logp, logq, F1, F2, e, n, U, V,
                           translate_every=check_every if translate else 0)
    if V is None:
        V = np.zeros(np.shape(q))
    if U is None:
        U = np.zeros(np.shape(p))
    err = math.inf
    it = 0
    while it < max_iter:
        S = apply_K_log(geom, V, logdy, eps)
        Un = prox_update_log(F1, logp, S, eps)
        checked = (it + 1) % check_every == 0 or it == max_iter - 1
        if checked:
            err = _violation_from(U, Un, S, logdx, eps)
            if it > 0 and tol > 0 and err <= tol:  # tol = 0 runs max_iter
                stop = True
            else:
                stop = False
        else:
            stop = False
        U = Un
        T = apply_K_log(geom, U, logdx, eps, transpose=True)
        V = prox_update_log(F2, logq, T, eps)
        if translate and checked:
            U, V = translate_log(logdx, logdy, logp, logq, F1, F2, U, V)
        it += 1
        if stop:
            break
    return dict(U=U, V=V, iters=it, err=err)


def scaling_alg4(K, dx, dy, p, q, F1: Div, F2: Div, F3: Div, m0: float, eps: float, iters: int):
    """Algorithm 4 (Sec. 4.5, a function F3 of the plan's total mass) verbatim:
    b <- 1, z <- 1; repeat a <- proxdiv_F1(z K(b.dy)), b <- proxdiv_F2(z K^T(a.dx)),
    z <- proxdiv_F3((a.dx)^T K (b.dy)).  F3 is a divergence of the total mass
    from m0, i.e. the Table 1 row on a single point of unit weight with
    density m0.  The plan is z a_i K_ij b_j.  Returns (a, b, z)."""
    K = np.asarray(K, dtype=np.float64)
    b = np.ones(K.shape[1])
    a = np.ones(K.shape[0])
    z = 1.0
    for _ in range(iters):
        a = proxdiv(F1, p, z * (K @ (b * dy)), 0.0, eps)
        b = proxdiv(F2, q, z * (K.T @ (a * dx)), 0.0, eps)
        M = float((a * dx) @ K @ (b * dy))
        z = float(proxdiv(F3, np.array([m0]), np.array([M]), 0.0, eps)[0])
    return a, b, z


def mass_update_log(F3: Div, m0: float, U, S, logdx, eps: float) -> float:
    """Z = eps log z of Algorithm 4's z-update in log form: the total mass of
    the plan without z, M = sum_i dx_i e^{(U_i + S_i)/eps} (current a, and S
    from the current b), then the Table 1 row of F3 at s = M, p = m0."""
    with np.errstate(invalid="ignore"):
        lr = np.where(np.isneginf(U) | np.isneginf(S), NEG_INF, np.asarray(logdx) + (U + S) / eps)
    logM = lse(lr.ravel())
    SM = eps * logM if np.isfinite(logM) else NEG_INF
    return float(prox_update_log(F3, np.array([math.log(m0)]), np.array([SM]), eps)[0])


def solve_mass_log(geom: Geometry, dx, dy, p, q, F1: Div, F2: Div, F3: Div, m0: float, eps: float,
                   max_iter: int, tol: float = 0.0, eps_start=None, stages: int = 10,
                   iters_per_stage: int = 100, check_every: int = 1):
    """Algorithm 4 in log form, with eps-scaling (Sec. 4.4) as in solve_log.
    Potentials U = eps log a, V = eps log b, Z = eps log z.  Iteration:
    S = eps log K(e^{V/eps} dy); except in the very first iteration (z = 1),
    Z = mass_update_log(U, S) (the z-update of the previous iteration: it needs
    the new b, i.e. this S, and the current a); U = prox_F1(log p, S + Z);
    T = eps log K^T(e^{U/eps} dx); V = prox_F2(log q, T + Z).  The measured
    violation is the larger of that of solve_log with S + Z in place of S and
    the z-update's own: the total mass of the current plan against its prox
    target, |e^{(Z_old - Z_new)/eps} - 1| (with a saturated F1 row, U can be
    stationary while z still moves).  The plan is e^{(U_i + V_j + Z - c_ij)/eps}."""
    logdx, logdy, logp, logq = map(safe_log, (dx, dy, p, q))
    U = np.zeros(np.shape(p))
    V = np.zeros(np.shape(q))
    Z = 0.0
    first = True
    sched = [(e, n, False) for e, n in eps_schedule(eps, eps_start, stages, iters_per_stage)]
    sched.append((eps, max_iter, True))
    err, it = math.inf, 0
    for e, n, final in sched:
        for k in range(n):
            S = apply_K_log(geom, V, logdy, e)
            Zold = Z
            if not first:
                Z = mass_update_log(F3, m0, U, S, logdx, e)
            first = False
            Sz = np.where(np.isneginf(S), NEG_INF, S + Z)
            Un = prox_update_log(F1, logp, Sz, e)
            stop = False
            if final and ((k + 1) % check_every == 0 or k == n - 1):
                mass_err = abs(math.expm1((Zold - Z) / e)) if np.isfinite(Z) and np.isfinite(Zold) else 0.0
                err = max(_violation_from(U, Un, Sz, logdx, e), mass_err)
                stop = k > 0 and tol > 0 and err <= tol
            U = Un
            T = apply_K_log(geom, U, logdx, e, transpose=True)
            Tz = np.where(np.isneginf(T), NEG_INF, T + Z)
            V = prox_update_log(F2, logq, Tz, e)
            if final:
                it = k + 1
            if stop:
                break
    return dict(U=U, V=V, Z=Z, iters=it, err=err)


def _violation_from(U_old, U_new, S, logdx, eps):
    """sum dx |r1 - rho1| / sum dx rho1 with r1 = e^{(U_old+S)/eps} the first
    marginal of the current plan and rho1 = e^{(U_new+S)/eps} its prox target."""
    with np.errstate(invalid="ignore"):
        lr = np.where(np.isneginf(U_old) | np.isneginf(S), NEG_INF, (U_old + S) / eps)
        lt = np.where(np.isneginf(U_new) | np.isneginf(S), NEG_INF, (U_new + S) / eps)
    w = np.exp(np.asarray(logdx, dtype=np.float64))
    num = np.sum(w * np.abs(np.exp(lr) - np.exp(lt)))
    den = np.sum(w * np.exp(lt))
    return float(num / den) if den > 0 else 0.0


def marginal_violation(geom, dx, dy, p, q, F1, F2, eps, U, V):
    """Stopping criterion used here (the paper leaves it open, Alg. 1):
    relative L1(dx) distance between the plan's first marginal and the prox
    target prox^KL_{F1/eps}(K b); it is the Sinkhorn marginal error when F1 is
    the equality constraint."""
    logdx, logdy, logp = safe_log(dx), safe_log(dy), safe_log(p)
    S = apply_K_log(geom, V, logdy, eps)
    return _violation_from(U, prox_update_log(F1, logp, S, eps), S, logdx, eps)


# ----------------------------------------------------------------------------
# plan, marginals, primal, dual (Theorem 3.2, eq. primal_discr)
# ----------------------------------------------------------------------------


def log_plan(geom: Geometry, U, V, eps):
    """log R_ij = (U_i + V_j - C_ij)/eps, R the density of the plan w.r.t. dx dy."""
    C = geom.cost_matrix()
    U = np.ravel(U)
    V = np.ravel(V)
    with np.errstate(invalid="ignore"):
        Z = (U[:, None] + V[None, :] - C) / eps
    return np.where(np.isnan(Z), NEG_INF, Z)


def marginals(geom, dx, dy, U, V, eps):
    """r1 = R dy, r2 = R^T dx from the dense plan (definition, Sec. 4.2)."""
    R = np.exp(log_plan(geom, U, V, eps))
    return R @ np.ravel(dy), R.T @ np.ravel(dx)


def div_value(F: Div, s, p, w) -> float:
    """F(s) = sum_i w_i Dbar_phi(s_i | p_i) (eq. divergencefunctions);
    +inf outside the domain."""
    s = np.ravel(np.asarray(s, dtype=np.float64))
    p = np.ravel(np.asarray(p, dtype=np.float64))
    w = np.ravel(np.asarray(w, dtype=np.float64))
    if F.kind == "kl":
        pos = p > 0
        if np.any((~pos) & (s > 0)):
            return math.inf
        with np.errstate(divide="ignore", invalid="ignore"):
            t = np.where(s > 0, s * np.log(np.where(s > 0, s, 1.0) / np.where(pos, p, 1.0)), 0.0) - s + p
        return float(F.lam * np.sum(w * t))
    if F.kind == "tv":
        return float(F.lam * np.sum(w * np.abs(s - p)))  # p = 0: lam * s (phi'_inf = 1)
    if F.kind == "eq":
        return 0.0 if np.allclose(s, p, rtol=1e-9, atol=1e-12) else math.inf
    if F.kind == "rg":
        hi = F.beta * p if not math.isinf(F.beta) else np.inf
        ok = np.all(s >= F.alpha * p * (1 - 1e-9) - 1e-12) and np.all(s <= hi * (1 + 1e-9) + 1e-12)
        return 0.0 if ok else math.inf
    raise ValueError(F.kind)


def div_conj(F: Div, wv, p, w) -> float:
    """Conjugate F*(wv) for the pairing <wv, s> = sum_i w_i wv_i s_i
    (Prop. A.3: D*_phi(a|p) = int phi*(a) p + iota_{a <= phi'_inf}):
      KL: lam sum w p (e^{wv/lam} - 1)
      TV: sum w p max(wv, -lam) if wv <= lam else +inf
      EQ: sum w p wv
      RG: sum w p max(alpha wv, beta wv) (beta = inf: needs wv <= 0)."""
    wv = np.ravel(np.asarray(wv, dtype=np.float64))
    p = np.ravel(np.asarray(p, dtype=np.float64))
    w = np.ravel(np.asarray(w, dtype=np.float64))
    if F.kind == "kl":
        return float(F.lam * np.sum(w * p * np.expm1(wv / F.lam)))
    if F.kind == "tv":
        if np.any(wv > F.lam * (1 + 1e-12)):
            return math.inf
        return float(np.sum(w * p * np.maximum(wv, -F.lam)))
    if F.kind == "eq":
        return float(np.sum(w * p * wv))
    if F.kind == "rg":
        if math.isinf(F.beta):
            if np.any((wv > 0) & (p > 0)):
                return math.inf
            return float(np.sum(w * p * F.alpha * wv))
        return float(np.sum(w * p * np.maximum(F.alpha * wv, F.beta * wv)))
    raise ValueError(F.kind)


def primal(geom, dx, dy, p, q, F1, F2, eps, U, V):
    """P_eps(R) = F1(R dy) + F2(R^T dx) + eps sum_ij dx_i dy_j KL(R_ij | K_ij),
    R = e^{(U+V-C)/eps}; KL(r|k) = r log(r/k) - r + k (weighted reading of
    eq. primal_discr, consistent with K b = K(b.dy))."""
    LR = log_plan(geom, U, V, eps)
    C = geom.cost_matrix()
    R = np.exp(LR)
    Kmat = np.exp(-C / eps)
    W = np.ravel(dx)[:, None] * np.ravel(dy)[None, :]
    with np.errstate(invalid="ignore"):
        ent = np.where(R > 0, R * (LR + C / eps), 0.0) - R + Kmat
    r1 = R @ np.ravel(dy)
    r2 = R.T @ np.ravel(dx)
    return div_value(F1, r1, p, dx) + div_value(F2, r2, q, dy) + eps * float(np.sum(W * ent))


def dual(geom, dx, dy, p, q, F1, F2, eps, U, V):
    """D_eps(U,V) = -F1*(-U) - F2*(-V) - eps <e^{(U+V)/eps} - 1, K>_{dx dy}
    (Theorem 3.2)."""
    LR = log_plan(geom, U, V, eps)
    C = geom.cost_matrix()
    W = np.ravel(dx)[:, None] * np.ravel(dy)[None, :]
    term = float(np.sum(W * (np.exp(LR) - np.exp(-C / eps))))
    Uf = np.where(np.isneginf(np.ravel(U)), 0.0, np.ravel(U))  # -inf only where p = 0
    Vf = np.where(np.isneginf(np.ravel(V)), 0.0, np.ravel(V))
    return -div_conj(F1, -Uf, p, dx) - div_conj(F2, -Vf, q, dy) - eps * term


# ----------------------------------------------------------------------------
# barycenters (Sec. 5.2, Table 2)
# ----------------------------------------------------------------------------


def _pl_root_midpoint(bp: np.ndarray, fvals: np.ndarray, tau: np.ndarray) -> np.ndarray:
    """Midpoint of the zero set of a continuous non-decreasing piecewise-linear
    function, given its breakpoints bp [B, npts] (sorted along axis 0), its
    values there fvals, f(bp[0]) <= 0 <= f(bp[-1]), and f linear between
    consecutive breakpoints.  The zero set is taken as [r1, r2] with
    r1 = min{W : f(W) >= -tau}, r2 = max{W : f(W) <= tau}: rounding leaves a
    flat piece of f at +-1e-16 instead of 0, and tau (~1e-12 of the function's
    range) keeps such a piece in the zero set."""
    B, npts = bp.shape
    cols = np.arange(npts)
    # r1: first breakpoint with f >= -tau, interpolate from the one before it
    i1 = np.argmax(fvals >= -tau[None, :], axis=0)
    lo1 = np.maximum(i1 - 1, 0)
    f_lo, f_hi = fvals[lo1, cols], fvals[i1, cols]
    b_lo, b_hi = bp[lo1, cols], bp[i1, cols]
    with np.errstate(invalid="ignore", divide="ignore"):
        r1 = np.where(i1 == 0, bp[0, cols], b_lo + (0.0 - f_lo) * (b_hi - b_lo) / (f_hi - f_lo))
    # r2: last breakpoint with f <= tau, interpolate to the one after it
    i2 = B - 1 - np.argmax((fvals <= tau[None, :])[::-1], axis=0)
    hi2 = np.minimum(i2 + 1, B - 1)
    g_lo, g_hi = fvals[i2, cols], fvals[hi2, cols]
    c_lo, c_hi = bp[i2, cols], bp[hi2, cols]
    with np.errstate(invalid="ignore", divide="ignore"):
        r2 = np.where(i2 == B - 1, bp[B - 1, cols], c_lo + (0.0 - g_lo) * (c_hi - c_lo) / (g_hi - g_lo))
    return 0.5 * (r1 + r2)


def bary_h_log(Tstack: np.ndarray, alpha: np.ndarray, lam: float, eps: float, kind: str = "kl",
               beta=(1.0, 1.0)):
    """eps log h from the n marginals s_k = e^{T_k/eps} (Table 2).

    kl: h = (sum_k alpha_k s_k^{eps/(eps+lam)} / sum_k alpha_k)^{(eps+lam)/eps}
        so eps log h = (eps+lam) (LSE_k(log alpha_k + T_k/(eps+lam)) - log sum alpha)
    eq: h = (prod_k s_k^{alpha_k})^{1/sum alpha}  (geometric mean).
    tv (Table 2 (iii)): with I+ = {k : s_k > 0} and A0 = sum of alpha_k off I+,
        h = 0 if A0 >= sum_{I+} alpha_k, else W = eps log h solves
        A0 + sum_{I+} alpha_k clamp((W - T_k)/lam, -1, 1) = 0
        (the condition of Table 2 (iii) multiplied through by eps/lam inside the clamp).
    rg (Table 2 (iv), RG[beta1, beta2], 0 < beta1 <= beta2 < inf): h = 0 if some
        s_k = 0, else W solves (eps times the condition of the table)
        sum_k alpha_k [beta2 min(W + eps log beta2 - T_k, 0) + beta1 max(W + eps log beta1 - T_k, 0)] = 0.
    Both left-hand sides are continuous, non-decreasing and piecewise linear in
    W; where they vanish on an interval (possible when saturated terms balance)
    the midpoint of that interval is taken (any point of it minimises
    eq. prox_barycenter, and the V updates do not depend on the choice).  Roots
    are located exactly from the values at the sorted breakpoints and linear
    interpolation.
    """
    alpha = np.asarray(alpha, dtype=np.float64)
    shp = (-1,) + (1,) * (Tstack.ndim - 1)
    if kind == "kl":
        Z = np.log(alpha).reshape(shp) + Tstack / (eps + lam)
        return (eps + lam) * (lse(Z, axis=0) - math.log(np.sum(alpha)))
    if kind == "eq":
        return np.sum(alpha.reshape(shp) * Tstack, axis=0) / np.sum(alpha)
    if kind not in ("tv", "rg"):
        raise ValueError(kind)
    T = np.asarray(Tstack, dtype=np.float64)
    out_shape = T.shape[1:]
    T = T.reshape(T.shape[0], -1)
    n, npts = T.shape
    a = alpha.reshape(n, 1)
    pos = np.isfinite(T)
    Tf = np.where(pos, T, 0.0)
    if kind == "tv":
        A0 = np.sum(np.where(pos, 0.0, a), axis=0)
        Ap = np.sum(np.where(pos, a, 0.0), axis=0)
        zero = A0 >= Ap
        # breakpoints T_k -/+ lam of the positive terms; others parked at the first one
        ref = np.max(np.where(pos, Tf, -np.inf), axis=0)
        ref = np.where(np.isfinite(ref), ref, 0.0)
        bp = np.concatenate([np.where(pos, Tf - lam, ref - lam), np.where(pos, Tf + lam, ref - lam)])
        bp = np.sort(bp, axis=0)

        def f(W):
            return A0 + np.sum(np.where(pos, a * np.clip((W[None, :] - Tf) / lam, -1.0, 1.0), 0.0), axis=0)
    else:
        b1, b2 = float(beta[0]), float(beta[1])
        if not (0.0 < b1 <= b2 < math.inf):
            raise ValueError("RG barycenter needs 0 < beta1 <= beta2 < inf")
        zero = np.any(~pos, axis=0)
        lo = Tf - eps * math.log(b2)
        up = Tf - eps * math.log(b1)
        bp = np.sort(np.concatenate([lo, up]), axis=0)

        def f(W):
            return np.sum(a * (b2 * np.minimum(W[None, :] - lo, 0.0) + b1 * np.maximum(W[None, :] - up, 0.0)),
                          axis=0)
    fvals = np.stack([f(bp[i]) for i in range(bp.shape[0])])
    scale = np.sum(alpha) * (1.0 if kind == "tv" else float(beta[1]) * max(1.0, float(np.max(np.abs(bp)))))
    W = _pl_root_midpoint(bp, fvals, np.full(npts, 1e-12 * scale))
    W = np.where(zero, -np.inf, W)
    return W.reshape(out_shape)


def barycenter_log(geom: Geometry, dx, dy, P, alpha, F1: Div, lam: float, eps: float,
                   iters: int, bary_kind: str = "kl", history: bool = False, beta=(1.0, 1.0)):
    """Unbalanced barycenter by the scaling iterations with n couplings sharing
    K = e^{-c/eps} (c_k = alpha_k c with the weighted KL of Sec. 5.2 gives
    K_k = e^{-c/eps} for all k).

    F1 acts componentwise (eq. proxcomponentbary): U_k = prox_update_F1(p_k).
    F2 (eq. Fbary): h from Table 2, then V_k = prox_update for lam KL(.|h)
    (Table 1 with p -> h); bary_kind 'eq' uses Table 2 (i) and the equality
    row, 'tv' Table 2 (iii) and the lam TV row, 'rg' Table 2 (iv) and the
    RG[beta1, beta2] row (the weights alpha_k multiply both terms of
    eq. prox_barycenter, so each V_k follows Table 1 unweighted).
    Returns U (n, ...), V (n, ...), eps log h.
    """
    logdx, logdy = safe_log(dx), safe_log(dy)
    P = np.asarray(P, dtype=np.float64)
    n = P.shape[0]
    logP = safe_log(P)
    V = np.zeros_like(P)
    U = np.zeros_like(P)
    Fh = {"kl": KL(lam), "eq": EQ(), "tv": TV(lam), "rg": RG(beta[0], beta[1])}[bary_kind]
    logh = None
    for _ in range(iters):
        for k in range(n):
            S = apply_K_log(geom, V[k], logdy, eps)
            U[k] = prox_update_log(F1, logP[k], S, eps)
        T = np.stack([apply_K_log(geom, U[k], logdx, eps, transpose=True) for k in range(n)])
        elogh = bary_h_log(T, alpha, lam, eps, bary_kind, beta)
        logh = elogh / eps
        for k in range(n):
            V[k] = prox_update_log(Fh, logh, T[k], eps)
    return U, V, (eps * logh if logh is not None else None)


# ----------------------------------------------------------------------------
# WF gradient flows with growth (Sec. 2 "Gradient flows", eq. grad-flow;
# Sec. 5.3: WF gradient flows, the tumor growth example and its extension to
# several species)
# ----------------------------------------------------------------------------


def wf_cost(x, y, cut: float = math.pi / 2) -> np.ndarray:
    """Cost of the Wasserstein-Fisher-Rao distance (eq. logcost, Definition
    WF of Sec. 2): c(x, y) = -log cos_+^2(d(x, y)) with cos_+(z) = cos(min(z, pi/2)).
    The distance is rescaled so that c = +inf exactly when |x - y| >= cut,
    d = (pi/2)|x - y|/cut, as in the paper's figures ("cut locus at 0.2");
    cut = pi/2 is the plain Euclidean distance.  K = e^{-c/eps} = 0 beyond
    the cut locus."""
    dist = np.sqrt(sqdist(x, y))
    d = (math.pi / 2) * dist / cut
    with np.errstate(divide="ignore"):
        c = 0.0 - np.log(np.cos(np.minimum(d, math.pi / 2)) ** 2)
    return np.where(dist >= cut, np.inf, c)


def growth_c(tau: float, alpha: float, lam: float) -> float:
    """c = 1 - 2 tau alpha / lam, the slope factor of the growth functional
    G(mu) = -alpha mu(X) + iota_{<=1}(d mu/dx) inside F2 (Sec. 5.3); the step
    needs 0 < c <= 1 (lam = 1 in the paper)."""
    c = 1.0 - 2.0 * tau * alpha / lam
    if not (0.0 < c <= 1.0):
        raise ValueError("the growth step needs 0 <= 2 tau alpha < lam")
    return c


def prox_growth_log(T: np.ndarray, c: float, lam: float, eps: float) -> np.ndarray:
    """Log-form proxdiv (u = 0) of the joint F2 of a WF gradient-flow step
    with S species (Sec. 5.3; S = 1 is the tumor example):
        F2(s^1..s^S) = inf_{r^k >= 0, sum_k r^k <= 1}
                       sum_k lam KL(s^k | r^k) - 2 tau alpha sum_k r^k,
    pointwise in x.  Its optimality conditions give r^k = s~^k / kappa with
    kappa = max(c, sum_k s~^k), and F2 depends on the s~^k only through their
    sum, with derivative lam log kappa in every species; the prox condition
    eps log(s~^k / s^k) + lam log kappa = 0 then gives the same update for all
    species:
        V^k = min(-lam log c, -lam Ttot/(lam + eps)),  Ttot = eps log sum_k e^{T^k/eps},
    T^k = eps log s^k (Ttot = -inf gives -lam log c).  With lam = 1 this is the
    paper's proxdiv printed for one species and, via beta, for two."""
    T = np.atleast_2d(np.asarray(T, dtype=np.float64))
    Ttot = eps * lse(T / eps, axis=0)
    with np.errstate(invalid="ignore"):
        lin = np.where(np.isneginf(Ttot), np.inf, -lam * Ttot / (lam + eps))
    V = np.minimum(-lam * math.log(c), lin)
    return np.broadcast_to(V, T.shape).copy()


def growth_next_density(R2: np.ndarray, c: float) -> np.ndarray:
    """Densities of the next step from the second marginals r2^k of the
    step's optimal couplings: the minimisers r^k of the inner infimum of F2,
    r^k = r2^k / max(c, sum_k r2^k) (for one species min(r2/c, 1), Sec. 5.3)."""
    R2 = np.atleast_2d(np.asarray(R2, dtype=np.float64))
    return R2 / np.maximum(c, np.sum(R2, axis=0))


def growth_next_log_density(logR2: np.ndarray, c: float) -> np.ndarray:
    """growth_next_density in log form: log r2^k - log max(c, sum_k r2^k).  A
    density below the FP64 range keeps its (finite) logarithm instead of
    becoming 0, as it would in exact arithmetic."""
    logR2 = np.atleast_2d(np.asarray(logR2, dtype=np.float64))
    tot = np.sum(np.exp(logR2), axis=0)
    return logR2 - np.log(np.maximum(c, tot))


def wf_flow_log(geom: Geometry, dx, P0, tau: float, alpha: float, lam: float, eps: float,
                nsteps: int, iters: int, eps_start=None, stages: int = 10, iters_per_stage: int = 100):
    """Minimizing movements (eq. grad-flow) of the growth functional
    G(mu^1..mu^S) = -alpha sum_k mu^k(X) + iota_{<=1}(sum_k d mu^k/dx) for the
    WF metric (Sec. 5.3), on points X = Y with weights dx (= dy) and the
    geometry's cost (wf_cost for WF).  Each step solves eq. grad-flow, which
    for each species k has F1 = lam KL(. | p^k) and all species share the
    joint F2 of prox_growth_log, by the scaling iterations in log form started
    from U = V = 0 (b = 1): `iters` iterations at eps after the eps-scaling
    stages.  The next densities are growth_next_density of the plan's second
    marginals r2^k = e^{(V^k + T^k)/eps} (T^k from the last iteration); they
    pass to the next step as log densities (growth_next_log_density), the
    log-domain stabilisation of Sec. 4.3 carried over the step boundary, so
    that a positive density below the FP64 range stays positive.
    Returns dict(P = [nsteps, S, n] densities after each step, U, V, T of the
    last step)."""
    logdx = safe_log(dx)
    logP = safe_log(np.atleast_2d(np.asarray(P0, dtype=np.float64)))
    S = logP.shape[0]
    c = growth_c(tau, alpha, lam)
    F1 = KL(lam)
    sched = eps_schedule(eps, eps_start, stages, iters_per_stage) + [(eps, iters)]
    traj = []
    U = V = T = None
    for _ in range(nsteps):
        U = np.zeros_like(logP)
        V = np.zeros_like(logP)
        T = np.full_like(logP, NEG_INF)
        for e, n_it in sched:
            for _ in range(n_it):
                for k in range(S):
                    U[k] = prox_update_log(F1, logP[k], apply_K_log(geom, V[k], logdx, e), e)
                T = np.stack([apply_K_log(geom, U[k], logdx, e, transpose=True) for k in range(S)])
                V = prox_growth_log(T, c, lam, e)
        with np.errstate(invalid="ignore"):
            logr2 = np.where(np.isneginf(T), NEG_INF, (V + T) / eps)
        logP = growth_next_log_density(logr2, c)
        traj.append(np.exp(logP))
    return dict(P=np.stack(traj), U=U, V=V, T=T)


# ----------------------------------------------------------------------------
# colour transfer by barycentric projection (Sec. 5.1, "Color transfer")
# ----------------------------------------------------------------------------


def bin_index(pts, shape) -> np.ndarray:
    """Row-major bin of each point of [0, 1]^d on a regular grid of `shape`
    bins: bin k of axis a covers [k/n_a, (k+1)/n_a), points outside the cube
    (and 1 itself) go to the nearest bin.  The floor is taken on the FP32
    product x * n_a, the precision the library decides it in."""
    P = np.asarray(pts, dtype=np.float32).reshape(-1, len(shape))
    idx = np.zeros(P.shape[0], dtype=np.int64)
    for a, n in enumerate(shape):
        with np.errstate(invalid="ignore"):
            k = np.floor(P[:, a] * np.float32(n))
        k = np.where(np.isnan(k), 0, k)
        k = np.clip(k, 0, n - 1).astype(np.int64)
        idx = idx * n + k
    return idx


def color_histogram(pts, shape) -> np.ndarray:
    """Colour histogram of an image as the pushforward of the (normalised)
    pixel measure: the fraction of pixels in each bin, i.e. the density w.r.t.
    the reference measure giving unit mass to every bin (Sec. 5.1)."""
    idx = bin_index(pts, shape)
    counts = np.zeros(int(np.prod(shape)), dtype=np.int64)
    np.add.at(counts, idx, 1)
    return counts / max(1, idx.size)


def barycentric_projection(geom: Geometry, dx, dy, U, V, eps) -> np.ndarray:
    """Approximate transport map by barycentric projection (Sec. 5.1):
    T_i = sum_j R_ij dy_j y_j / sum_j R_ij dy_j with R the plan of (U, V)
    (Theorem 3.2); rows of zero plan mass keep their own point x_i."""
    R = np.exp(log_plan(geom, U, V, eps))
    if geom.kind == "grid":
        X, Y = grid_points(geom.xs), grid_points(geom.ys)
    elif geom.kind == "points":
        X, Y = np.asarray(geom.x, dtype=np.float64), np.asarray(geom.y, dtype=np.float64)
    else:
        raise ValueError("the barycentric projection needs point coordinates")
    X = X.reshape(X.shape[0], -1)
    Y = Y.reshape(Y.shape[0], -1)
    w = np.ravel(np.asarray(dy, dtype=np.float64))
    num = R @ (w[:, None] * Y)
    den = R @ w
    with np.errstate(invalid="ignore", divide="ignore"):
        T = num / den[:, None]
    return np.where(den[:, None] > 0, T, X)


def apply_bin_map(pts, shape, T) -> np.ndarray:
    """The modified image T o g_X: every pixel takes the value of T at its bin."""
    return np.asarray(T)[bin_index(pts, shape)]


def grid_axes(shape):
    """Bin centres (k + 1/2)/n of each axis of the colour grid."""
    return [(np.arange(n, dtype=np.float64) + 0.5) / n for n in shape]

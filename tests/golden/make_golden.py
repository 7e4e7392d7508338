"""Writes the fixtures of this folder.  Every value follows from the
mathematics of the problem, not from an iteration: nothing here runs the
scaling algorithm or any GPU code.  Run from the repository root:

    python tests/golden/make_golden.py

one_point.txt -- one-point problems (n = m = 1, dx = dy = 1, cost c): the
  plan r* minimises the discrete primal of Sec. 3 (eq. P_eps with the
  divergences of Table 1, the entropy weighted by dx dy),
      F1(r | p) + F2(r | q) + eps (r log(r / e^{-c/eps}) - r + e^{-c/eps}).
  KL / KL rows use the stationarity condition,
      log r* = (lam1 log p + lam2 log q - c) / (lam1 + lam2 + eps);
  the other rows minimise the (convex) primal over r by golden-section search
  to a relative width of 1e-14, with the divergence values of oracle.div_value.
bary_h.txt -- the barycenter h of Table 2 for one point from the marginals
  s_k and weights alpha_k, in plain arithmetic (the oracle uses a log-sum-exp
  form): (i) EQ, the weighted geometric mean prod s_k^{alpha_k / sum alpha};
  (ii) KL, (sum alpha_k s_k^{eps/(eps+lam)} / sum alpha)^{(eps+lam)/eps}.
"""
import math
import os
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))

import numpy as np  # noqa: E402

import oracle as O  # noqa: E402

# (F1, F2, eps, c, p, q); a divergence is (kind, lam) or ("rg", alpha, beta) or ("eq",)
ONE_POINT = [
    (("kl", 1.0), ("kl", 1.0), 0.5, 0.3, 1.0, 2.0),
    (("kl", 0.2), ("kl", 3.0), 0.1, 1.0, 0.5, 1.7),
    (("kl", 5.0), ("kl", 0.5), 0.05, 0.0, 2.0, 0.3),
    (("kl", 0.7), ("kl", 0.7), 0.01, 0.25, 0.8, 1.3),
    (("tv", 0.3), ("tv", 0.2), 0.1, 0.2, 1.0, 1.6),
    (("tv", 0.05), ("kl", 1.0), 0.1, 0.2, 1.0, 1.6),
    (("rg", 0.7, 1.2), ("kl", 0.5), 0.1, 0.2, 1.0, 1.6),
    (("eq",), ("kl", 0.5), 0.1, 0.2, 1.0, 1.6),
    (("rg", 0.5, 2.0), ("rg", 0.8, 1.5), 0.1, 0.2, 1.0, 1.6),
    (("kl", 1.0), ("tv", 0.4), 0.05, 0.5, 0.6, 1.4),
    (("tv", 1.0), ("eq",), 0.2, 0.1, 1.2, 0.9),
]

BARY = [
    # (kind, lam, eps, alpha, s)
    ("kl", 1.0, 0.01, (0.25, 0.25, 0.5), (0.7, 1.3, 2.2)),
    ("kl", 0.3, 0.1, (1.0, 2.0), (0.05, 3.0)),
    ("kl", 5.0, 0.02, (0.1, 0.2, 0.3, 0.4), (1.0, 1.5, 0.2, 4.0)),
    ("eq", 0.0, 0.01, (0.25, 0.25, 0.5), (0.7, 1.3, 2.2)),
    ("eq", 0.0, 0.1, (1.0, 3.0), (0.4, 2.5)),
]


def div(spec):
    if spec[0] == "kl":
        return O.KL(spec[1])
    if spec[0] == "tv":
        return O.TV(spec[1])
    if spec[0] == "rg":
        return O.RG(spec[1], spec[2])
    return O.EQ()


def spec_str(spec):
    return ":".join([spec[0]] + [repr(float(v)) for v in spec[1:]])


def one_point_log_r(F1, F2, eps, c, p, q):
    if F1[0] == "kl" and F2[0] == "kl":
        return (F1[1] * math.log(p) + F2[1] * math.log(q) - c) / (F1[1] + F2[1] + eps)
    one = np.ones(1)

    def obj(r):
        v = eps * (r * (math.log(r) + c / eps) - r + math.exp(-c / eps))
        for F, m in ((div(F1), p), (div(F2), q)):
            d = O.div_value(F, np.array([r]), np.array([m]), one)
            v += d if math.isfinite(d) else 1e300
        return v
    # EQ sides fix r to their density; otherwise golden-section search on [1e-6, 50]
    # cut down to the feasible range [alpha m, beta m] of RG sides (the primal is +inf outside)
    lo, hi = 1e-6, 50.0
    for F, m in ((F1, p), (F2, q)):
        if F[0] == "eq":
            return math.log(m)
        if F[0] == "rg":
            lo, hi = max(lo, F[1] * m), min(hi, F[2] * m)
    g = (math.sqrt(5.0) - 1.0) / 2.0
    a, b = hi - g * (hi - lo), lo + g * (hi - lo)
    fa, fb = obj(a), obj(b)
    while hi - lo > 1e-14 * max(1.0, hi):
        if fa < fb:
            hi, b, fb = b, a, fa
            a = hi - g * (hi - lo)
            fa = obj(a)
        else:
            lo, a, fa = a, b, fb
            b = lo + g * (hi - lo)
            fb = obj(b)
    return math.log(0.5 * (lo + hi))


def bary_h(kind, lam, eps, alpha, s):
    A = sum(alpha)
    if kind == "eq":
        return math.prod(sk ** (ak / A) for ak, sk in zip(alpha, s))
    e = eps / (eps + lam)
    return (sum(ak * sk ** e for ak, sk in zip(alpha, s)) / A) ** (1.0 / e)


def main():
    with open(os.path.join(HERE, "one_point.txt"), "w") as f:
        f.write("# One-point problems (n = m = 1, dx = dy = 1): the minimiser r* of the primal of Sec. 3\n"
                "# (eq. P_eps, Table 1 divergences), written by tests/golden/make_golden.py.\n"
                "# F1 F2 eps c p q log_r\n")
        for F1, F2, eps, c, p, q in ONE_POINT:
            lr = one_point_log_r(F1, F2, eps, c, p, q)
            f.write(f"{spec_str(F1)} {spec_str(F2)} {eps!r} {c!r} {p!r} {q!r} {lr!r}\n")
    with open(os.path.join(HERE, "bary_h.txt"), "w") as f:
        f.write("# One-point barycenter h of Table 2 ((i) EQ: weighted geometric mean, (ii) KL: power mean),\n"
                "# written by tests/golden/make_golden.py.\n"
                "# kind lam eps alpha(comma-separated) s(comma-separated) h\n")
        for kind, lam, eps, alpha, s in BARY:
            h = bary_h(kind, lam, eps, alpha, s)
            f.write(f"{kind} {lam!r} {eps!r} {','.join(repr(a) for a in alpha)} "
                    f"{','.join(repr(v) for v in s)} {h!r}\n")


if __name__ == "__main__":
    main()

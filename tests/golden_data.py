"""Readers of the fixtures in tests/golden/ (written by tests/golden/make_golden.py
from closed forms and direct minimisation of the one-point primal, never by an
iteration of the method or by the CUDA path)."""
import os

GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")


def _rows(name):
    with open(os.path.join(GOLDEN, name)) as f:
        return [ln.split() for ln in f if ln.strip() and not ln.startswith("#")]


def parse_div(spec):
    """'kl:0.5' -> ('kl', 0.5); 'rg:0.7:1.2' -> ('rg', 0.7, 1.2); 'eq' -> ('eq',)."""
    parts = spec.split(":")
    return (parts[0],) + tuple(float(v) for v in parts[1:])


def one_point():
    """[(F1, F2, eps, c, p, q, log_r, exact)]: exact when the value is a closed
    form (KL / KL stationarity, or an EQ side fixing r), else a golden-section
    minimiser accurate to about 1e-8 relative (the primal is flat at a smooth
    minimum)."""
    out = []
    for r in _rows("one_point.txt"):
        F1, F2 = parse_div(r[0]), parse_div(r[1])
        eps, c, p, q, lr = (float(v) for v in r[2:7])
        exact = (F1[0] == "kl" and F2[0] == "kl") or "eq" in (F1[0], F2[0])
        out.append((F1, F2, eps, c, p, q, lr, exact))
    return out


def bary_h():
    """[(kind, lam, eps, alpha tuple, s tuple, h)] from Table 2 (i), (ii)."""
    out = []
    for r in _rows("bary_h.txt"):
        out.append((r[0], float(r[1]), float(r[2]), tuple(float(v) for v in r[3].split(",")),
                    tuple(float(v) for v in r[4].split(",")), float(r[5])))
    return out

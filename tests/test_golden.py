"""The oracle against the fixtures of tests/golden/: one-point problems whose
plan follows from the primal of Sec. 3 directly (closed forms, or a direct
minimisation of the one-point primal), and the one-point barycenters of
Table 2 (i) and (ii) in plain arithmetic."""
import math

import numpy as np
import pytest

import oracle as O

from golden_data import bary_h, one_point


def oracle_div(spec):
    return {"kl": lambda: O.KL(spec[1]), "tv": lambda: O.TV(spec[1]), "rg": lambda: O.RG(spec[1], spec[2]),
            "eq": lambda: O.EQ()}[spec[0]]()


@pytest.mark.parametrize("row", one_point(), ids=lambda r: f"{r[0][0]}-{r[1][0]}-eps{r[2]}")
def test_oracle_one_point_plans(row):
    F1, F2, eps, c, p, q, log_r, exact = row
    one = np.ones(1)
    r = O.solve_log(O.Geometry("dense", C=np.array([[c]])), one, one, np.array([p]), np.array([q]),
                    oracle_div(F1), oracle_div(F2), eps, max_iter=6000, stages=0)
    got = (r["U"][0] + r["V"][0] - c) / eps
    assert abs(got - log_r) <= (1e-12 if exact else 2e-7)


@pytest.mark.parametrize("row", bary_h(), ids=lambda r: f"{r[0]}-lam{r[1]}")
def test_oracle_barycenter_h_table2(row):
    kind, lam, eps, alpha, s, h = row
    T = eps * np.log(np.array(s)).reshape(-1, 1)
    got = O.bary_h_log(T, np.array(alpha), lam, eps, kind=kind)[0] / eps
    assert abs(got - math.log(h)) <= 1e-12 * max(1.0, abs(math.log(h)))

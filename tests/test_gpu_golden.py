"""uot_solve on the one-point problems of tests/golden/one_point.txt (plans
fixed by the primal of Sec. 3: closed forms or a direct minimisation of the
one-point primal), in FP64 and FP32, through the C ABI."""
import numpy as np
import pytest
import torch

from paper_1607_05816_gb300 import uot as U

from golden_data import one_point

pytestmark = pytest.mark.gpu


def lib_div(spec):
    return {"kl": lambda: U.KL(spec[1]), "tv": lambda: U.TV(spec[1]), "rg": lambda: U.RG(spec[1], spec[2]),
            "eq": lambda: U.EQ()}[spec[0]]()


@pytest.mark.parametrize("prec", [U.F64, U.F32])
@pytest.mark.parametrize("row", one_point(), ids=lambda r: f"{r[0][0]}-{r[1][0]}-eps{r[2]}")
def test_one_point_plans(row, prec):
    F1, F2, eps, c, p, q, log_r, exact = row
    dt = torch.float64 if prec == U.F64 else torch.float32
    v = lambda x: torch.tensor([x], dtype=dt, device="cuda")
    Ug, Vg, info = U.solve(U.Geometry.dense(torch.tensor([[c]], dtype=dt, device="cuda")), v(p), v(1.0), v(q),
                           v(1.0), lib_div(F1), lib_div(F2), eps, precision=prec, max_iter=6000, eps_stages=0,
                           out_f64=True)
    got = (float(Ug[0]) + float(Vg[0]) - c) / eps
    if prec == U.F64:
        tol = 1e-11 if exact else 2e-7
    else:
        # the plan of the float-float state; c, p, q rounded to FP32 move log r by ~1e-7 / eps
        tol = 1e-5
    assert abs(got - log_r) <= tol, (got, log_r)

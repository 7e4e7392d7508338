"""Failure detection without a GPU fault: every device-side wait of a kernel
on other CTAs is bounded by the GPU's global timer.  The self-test entry runs
that wait on a flag that nothing sets; it must give up after the limit,
report UOT_TIMEOUT, and leave the context usable for the next call."""
import time

import numpy as np
import pytest
import torch

import oracle as O
from paper_1607_05816_gb300 import synth
from paper_1607_05816_gb300 import uot as U

pytestmark = [pytest.mark.gpu, pytest.mark.filterwarnings("ignore::RuntimeWarning")]


def test_bounded_wait_expires_and_context_survives():
    t0 = time.perf_counter()
    assert U.selftest_bounded_wait(0.25) == "UOT_TIMEOUT"
    dt = time.perf_counter() - t0
    assert 0.25 <= dt < 5.0, dt
    # the context still computes correctly
    xs = [synth.grid_axis(40), synth.grid_axis(36)]
    geo = U.Geometry.grid([torch.as_tensor(a, dtype=torch.float64, device="cuda") for a in xs])
    g = synth.rng(3)
    W = g.normal(size=(40, 36)) * 0.05
    w = np.full((40, 36), 1.0 / (40 * 36))
    got = U.gibbs_log(geo, torch.as_tensor(W, device="cuda").ravel(), torch.as_tensor(w, device="cuda").ravel(),
                      0.01, False, U.F64).cpu().numpy()
    want = O.apply_K_log(O.Geometry("grid", xs=xs, ys=xs), W, np.log(w), 0.01)
    assert np.max(np.abs(got - want.ravel())) <= 1e-10 * max(1.0, np.max(np.abs(want)))


def test_bounded_wait_rejects_bad_limits():
    for bad in (0.0, -1.0, 11.0):
        with pytest.raises(U.UotError):
            U.selftest_bounded_wait(bad)

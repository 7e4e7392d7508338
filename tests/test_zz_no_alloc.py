"""The no-allocation Gibbs operator (uot_gibbs_log_noalloc).

Callers that cannot allocate device memory (inside a stream capture, under a
foreign allocator, in latency-critical loops) use this entry point; it must
give the same result as uot_gibbs_log, which allocates its scratch.  Two calls
in a row check that what the shared scratch array keeps from the previous
call does not leak into the next one.  This file is collected last on
purpose, so a failure here does not hide any other test.
"""
import numpy as np
import pytest
import torch

from paper_1607_05816_gb300 import synth
from paper_1607_05816_gb300 import uot as U

pytestmark = pytest.mark.gpu

TOL = {U.F64: 1e-12, U.F32: 1e-6}


def _grid(prec, shape_x, shape_y, seed):
    dt = U._dtype(prec)
    g = synth.rng(seed)
    xs = [torch.as_tensor(synth.grid_axis(n), dtype=dt, device="cuda") for n in shape_x]
    ys = [torch.as_tensor(synth.grid_axis(n), dtype=dt, device="cuda") for n in shape_y]
    m = int(np.prod(shape_y))
    W = g.normal(size=m) * 0.05
    W[7::29] = -np.inf
    w = np.full(m, 1.0 / m)
    return (U.Geometry.grid(xs, ys), torch.as_tensor(W, dtype=dt, device="cuda"),
            torch.as_tensor(w, dtype=dt, device="cuda"))


def _points(prec, n, m, seed):
    dt = U._dtype(prec)
    g = synth.rng(seed)
    x = torch.as_tensor(synth.mixture_points(g, n, 3, 4), dtype=dt, device="cuda")
    y = torch.as_tensor(synth.mixture_points(g, m, 3, 4), dtype=dt, device="cuda")
    W = torch.as_tensor(g.normal(size=m) * 0.05, dtype=dt, device="cuda")
    w = torch.full((m,), 1.0 / m, dtype=dt, device="cuda")
    return U.Geometry.points(x, y), W, w


def _close(a, b, tol):
    a = a.double().cpu().numpy()
    b = b.double().cpu().numpy()
    assert np.array_equal(np.isneginf(a), np.isneginf(b))
    f = np.isfinite(b)
    return np.max(np.abs(a[f] - b[f])) <= tol * max(1.0, np.max(np.abs(b[f])))


@pytest.mark.parametrize("prec", [U.F64, U.F32])
def test_noalloc_matches_allocating_operator(prec):
    cases = [_grid(prec, (70, 45), (33, 129), 1), _grid(prec, (256, 256), (256, 256), 2),
             _points(prec, 301, 260, 3)]
    for geo, W, w in cases:
        for transpose in (False, True):
            if transpose:
                Wt = torch.zeros(geo.n, dtype=W.dtype, device="cuda")
                wt = torch.full((geo.n,), 1.0 / geo.n, dtype=W.dtype, device="cuda")
                Wt[: min(geo.n, W.numel())] = W[: min(geo.n, W.numel())]
                args = (Wt, wt)
            else:
                args = (W, w)
            ref = U.gibbs_log(geo, *args, 0.01, transpose, prec)
            first = U.gibbs_log_noalloc(geo, *args, 0.01, transpose, prec)
            second = U.gibbs_log_noalloc(geo, *args, 0.01, transpose, prec)
            torch.cuda.synchronize()
            assert _close(first, ref, TOL[prec])
            assert _close(second, ref, TOL[prec])


def test_noalloc_rejects_oversized_problem():
    geo, W, w = _grid(U.F64, (512, 512), (512, 512), 4)
    with pytest.raises(U.UotError, match="EINVAL"):
        U.gibbs_log_noalloc(geo, W, w, 0.01, False, U.F64)
    assert "UOT_NOALLOC_SCRATCH_BYTES" in U._last_error()

"""The no-allocation Gibbs operator (uot_gibbs_log_noalloc).

Callers that cannot call cudaMalloc (code under a foreign allocator that owns
all device memory, real-time loops where an allocation may block or fail) use
this entry point; it must give the same result as uot_gibbs_log, which
allocates its scratch, and it must allocate nothing.  Two calls in a row check
that what the shared scratch array keeps from the previous call does not leak
into the next one.  This file is collected last on purpose, so a failure here
does not hide any other test.
"""
import ctypes

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


# cudaMemPoolAttrUsedMemHigh (driver_types.h): the high-water mark of the
# memory handed out by a pool since it was last reset to zero.  The library's
# allocating entry points take their scratch from the device's default pool
# (cudaMallocAsync); torch's caching allocator does not use that pool.
_USED_MEM_HIGH = 8


def _default_pool_used_high(reset=False):
    rt = ctypes.CDLL("libcudart.so.13")
    dev = torch.cuda.current_device()
    pool = ctypes.c_void_p()
    assert rt.cudaDeviceGetDefaultMemPool(ctypes.byref(pool), dev) == 0
    v = ctypes.c_uint64(0)
    if reset:
        assert rt.cudaMemPoolSetAttribute(pool, _USED_MEM_HIGH, ctypes.byref(v)) == 0
    assert rt.cudaMemPoolGetAttribute(pool, _USED_MEM_HIGH, ctypes.byref(v)) == 0
    return v.value


@pytest.mark.parametrize("prec", [U.F64, U.F32])
def test_noalloc_allocates_nothing(prec):
    geo, W, w = _grid(prec, (256, 256), (256, 256), 5)
    U.gibbs_log_noalloc(geo, W, w, 0.01, False, prec)  # the first call's set-up
    torch.cuda.synchronize()
    # the measure works: the allocating operator moves the high-water mark
    _default_pool_used_high(reset=True)
    U.gibbs_log(geo, W, w, 0.01, False, prec)
    torch.cuda.synchronize()
    assert _default_pool_used_high() > 0
    _default_pool_used_high(reset=True)
    for _ in range(2):
        U.gibbs_log_noalloc(geo, W, w, 0.01, False, prec)
    torch.cuda.synchronize()
    assert _default_pool_used_high() == 0


def test_noalloc_rejects_mixed_precision():
    geo, W, w = _grid(U.F32, (64, 64), (64, 64), 6)
    with pytest.raises(U.UotError, match="EUNSUPPORTED"):
        U.gibbs_log_noalloc(geo, W, w, 0.01, False, U.MIXED)

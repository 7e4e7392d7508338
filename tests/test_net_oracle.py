"""Pins of the warm-start network's CPU reference (oracle/net_oracle.py):
the convolution against a brute-force loop, finite-difference gradients
against the closed form for a linear layer."""
import numpy as np
import pytest

import oracle.net_oracle as NO
from paper_1607_05816_gb300 import synth


def brute_conv(x, w, b, dil, leaky):
    N, Cin, H, W = x.shape
    Cout = w.shape[0]
    y = np.zeros((N, Cout, H, W))
    for n in range(N):
        for co in range(Cout):
            for h in range(H):
                for v in range(W):
                    acc = b[co]
                    for ci in range(Cin):
                        for kh in range(3):
                            for kw in range(3):
                                hh, vv = h + dil * (kh - 1), v + dil * (kw - 1)
                                if 0 <= hh < H and 0 <= vv < W:
                                    acc += w[co, ci, kh, kw] * x[n, ci, hh, vv]
                    y[n, co, h, v] = acc if (not leaky or acc >= 0) else 0.1 * acc
    return y


@pytest.mark.parametrize("dil,leaky", [(1, True), (2, False), (3, True)])
def test_conv_matches_brute_force(dil, leaky):
    g = synth.rng(5)
    x = g.normal(size=(2, 3, 5, 7))
    w = g.normal(size=(4, 3, 3, 3))
    b = g.normal(size=4)
    assert np.max(np.abs(NO.conv2d(x, w, b, dil, leaky) - brute_conv(x, w, b, dil, leaky))) < 1e-12


def test_fd_gradient_matches_closed_form_linear_layer():
    """One linear layer: dL/db[co] = 2/numel sum (y - t)[:, co] and
    dL/dw[co,ci,kh,kw] = 2/numel sum (y - t)[:, co] * shifted x[:, ci]."""
    g = synth.rng(6)
    x = g.normal(size=(2, 2, 6, 5))
    w = g.normal(size=(3, 2, 3, 3))
    b = g.normal(size=3)
    t = g.normal(size=(2, 3, 6, 5))
    layers = [(2, False)]
    y = NO.conv2d(x, w, b, 2, False)
    r = 2.0 * (y - t) / y.size
    for co in range(3):
        fd = NO.fd_grad([(w, b)], layers, x, t, (0, 1), co)
        assert abs(fd - r[:, co].sum()) < 1e-7
    xp = np.zeros((2, 2, 10, 9))
    xp[:, :, 2:8, 2:7] = x
    for idx in [(0, 0, 0, 0), (2, 1, 1, 2), (1, 0, 2, 1)]:
        co, ci, kh, kw = idx
        want = np.sum(r[:, co] * xp[:, ci, 2 * kh:2 * kh + 6, 2 * kw:2 * kw + 5])
        assert abs(NO.fd_grad([(w, b)], layers, x, t, (0, 0), idx) - want) < 1e-7


def test_conv2d_grads_match_finite_differences():
    """The adjoint formulas of conv2d_grads against central differences of
    L = sum(g * conv2d(x, w, b)) on a small random case, every entry."""
    g0 = np.random.default_rng(7)
    for dil in (1, 2):
        x = g0.normal(size=(2, 3, 5, 6))
        w = g0.normal(size=(4, 3, 3, 3))
        b = g0.normal(size=4)
        G = g0.normal(size=(2, 4, 5, 6))
        dx, dw, db = NO.conv2d_grads(x, w, G, dil)
        L = lambda x_, w_, b_: float(np.sum(G * NO.conv2d(x_, w_, b_, dil, False)))
        h = 1e-6
        for arr, grad, which in ((x, dx, 0), (w, dw, 1), (b, db, 2)):
            fd = np.zeros_like(arr)
            for idx in np.ndindex(arr.shape):
                old = arr[idx]
                arr[idx] = old + h
                lp = L(x, w, b)
                arr[idx] = old - h
                lm = L(x, w, b)
                arr[idx] = old
                fd[idx] = (lp - lm) / (2 * h)
            assert np.max(np.abs(fd - grad)) <= 1e-6 * max(1.0, np.max(np.abs(grad))), which

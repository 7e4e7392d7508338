"""Plain numpy FP64 reference of the warm-start network (test infrastructure only).

The network is not part of the paper: it is the learned warm start of this
library.  This module restates its forward pass in the most direct way (a sum
of shifted image slices per 3x3 tap, zero padding, leaky ReLU with slope 0.1)
and obtains gradients by central finite differences, so that the CUDA forward
and backward kernels can be checked against something that shares no code
with them.
"""
from __future__ import annotations

import numpy as np

LEAK = 0.1


def conv2d(x, w, b, dil, leaky):
    """x [N, Cin, H, W], w [Cout, Cin, 3, 3], b [Cout] -> [N, Cout, H, W];
    y[n, co, h, v] = b[co] + sum_{ci, kh, kw} w[co, ci, kh, kw] x[n, ci, h + dil (kh-1), v + dil (kw-1)]."""
    x = np.asarray(x, dtype=np.float64)
    N, Cin, H, W = x.shape
    Cout = w.shape[0]
    pad = dil
    xp = np.zeros((N, Cin, H + 2 * pad, W + 2 * pad))
    xp[:, :, pad:pad + H, pad:pad + W] = x
    y = np.zeros((N, Cout, H, W)) + np.asarray(b, dtype=np.float64)[None, :, None, None]
    for kh in range(3):
        for kw in range(3):
            sl = xp[:, :, kh * dil:kh * dil + H, kw * dil:kw * dil + W]  # [N, Cin, H, W]
            y += np.einsum("oc,nchw->nohw", np.asarray(w[:, :, kh, kw], dtype=np.float64), sl)
    if leaky:
        y = np.where(y < 0, LEAK * y, y)
    return y


def forward(params, layers, x):
    """params: list of (w, b); layers: list of (dilation, leaky)."""
    h = np.asarray(x, dtype=np.float64)
    for (w, b), (dil, leaky) in zip(params, layers):
        h = conv2d(h, w, b, dil, leaky)
    return h


def mse(params, layers, x, target):
    out = forward(params, layers, x)
    return float(np.mean((out - np.asarray(target, dtype=np.float64)) ** 2))


def fd_grad(params, layers, x, target, which, idx, h=1e-5):
    """Central finite difference of the loss w.r.t. params[which][0 or 1][idx]."""
    li, kind = which
    base = [(w.astype(np.float64).copy(), b.astype(np.float64).copy()) for w, b in params]
    arr = base[li][kind]
    old = arr[idx]
    arr[idx] = old + h
    lp = mse(base, layers, x, target)
    arr[idx] = old - h
    lm = mse(base, layers, x, target)
    arr[idx] = old
    return (lp - lm) / (2 * h)


def conv2d_grads(x, w, g, dil):
    """Gradients of L = sum(g * conv2d(x, w, b, dil, leaky=False)) with respect to
    x, w and b, each written from the definition of conv2d (zero padding):
      dx[n, ci, h, v]   = sum_{co, kh, kw} w[co, ci, kh, kw] g[n, co, h - dil (kh-1), v - dil (kw-1)]
      dw[co, ci, kh, kw] = sum_{n, h, v} g[n, co, h, v] x[n, ci, h + dil (kh-1), v + dil (kw-1)]
      db[co]            = sum_{n, h, v} g[n, co, h, v]
    (terms whose shifted index leaves the image are zero)."""
    x = np.asarray(x, dtype=np.float64)
    w = np.asarray(w, dtype=np.float64)
    g = np.asarray(g, dtype=np.float64)
    N, Cin, H, W = x.shape
    pad = dil
    xp = np.zeros((N, Cin, H + 2 * pad, W + 2 * pad))
    xp[:, :, pad:pad + H, pad:pad + W] = x
    gp = np.zeros((N, g.shape[1], H + 2 * pad, W + 2 * pad))
    gp[:, :, pad:pad + H, pad:pad + W] = g
    dx = np.zeros_like(x)
    dw = np.zeros_like(w)
    for kh in range(3):
        for kw in range(3):
            # x[h + dil (kh-1)] lives at xp[h + dil kh]; g[h - dil (kh-1)] at gp[h + dil (2 - kh)]
            xs = xp[:, :, kh * dil:kh * dil + H, kw * dil:kw * dil + W]
            gs = gp[:, :, (2 - kh) * dil:(2 - kh) * dil + H, (2 - kw) * dil:(2 - kw) * dil + W]
            dw[:, :, kh, kw] = np.einsum("nohw,nchw->oc", g, xs)
            dx += np.einsum("oc,nohw->nchw", w[:, :, kh, kw], gs)
    return dx, dw, g.sum(axis=(0, 2, 3))

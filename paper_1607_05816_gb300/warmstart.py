"""Learned warm start for the scaling iteration (not part of the paper).

A small dilated convolutional network maps the features
(log p, log q, log eps, log lambda) of a grid problem to initial potentials
(U0, V0), which replace the cold start b = 1 of Algorithm 1.  The plain
iteration stays the judge: it runs from the predicted potentials to the same
tolerance, so the network can only change how many iterations are needed,
never the answer.

Every numeric step (features, convolutions, their gradients, the loss and
Adam) runs in the library's kernels; this module only holds the parameters
(device tensors) and sequences the calls.  Training targets are potentials
produced by the solver itself (uot_solve_many).
"""
from __future__ import annotations

import math

import numpy as np
import torch

from . import uot

DEFAULT_DILATIONS = (1, 2, 4, 8, 16, 1)


class WarmStartNet:
    """conv3x3(4 -> C) + leaky, len(dilations) x conv3x3(C -> C, dilation d) + leaky,
    conv3x3(C -> 2) linear.  Output channel 0 is U0, channel 1 is V0."""

    def __init__(self, channels=32, dilations=DEFAULT_DILATIONS, device="cuda", seed=0):
        gen = torch.Generator(device="cpu").manual_seed(seed)
        self.layers = [(4, channels, 1, True)]
        self.layers += [(channels, channels, d, True) for d in dilations]
        self.layers += [(channels, 2, 1, False)]
        self.params = []
        for cin, cout, _, leaky in self.layers:
            std = math.sqrt(2.0 / (cin * 9)) * (1.0 if leaky else 0.1)
            w = (torch.randn(cout, cin, 3, 3, generator=gen) * std).to(device)
            b = torch.zeros(cout, device=device)
            self.params.append([w, b])
        self.m = [[torch.zeros_like(t) for t in pr] for pr in self.params]
        self.v = [[torch.zeros_like(t) for t in pr] for pr in self.params]
        self.t = 0
        self.loss_dev = torch.zeros(1, dtype=torch.float64, device=device)

    def n_params(self):
        return sum(t.numel() for pr in self.params for t in pr)

    def forward(self, feats):
        acts = [feats]
        h = feats
        for (w, b), (_, _, dil, leaky) in zip(self.params, self.layers):
            h = uot.conv2d_forward(h, w, b, dil, leaky)
            acts.append(h)
        return acts

    def backward(self, acts, dout):
        grads = [None] * len(self.params)
        g = dout
        for li in range(len(self.params) - 1, -1, -1):
            w, _ = self.params[li]
            _, _, dil, leaky = self.layers[li]
            dx, dw, db = uot.conv2d_backward(acts[li], w, acts[li + 1], g, dil, leaky, need_dx=li > 0)
            grads[li] = (dw, db)
            g = dx
        return grads

    def train_step(self, feats, target, lr):
        acts = self.forward(feats)
        out = acts[-1]
        dout = torch.empty_like(out)
        uot.mse_grad(out, target, dout, self.loss_dev)
        grads = self.backward(acts, dout)
        self.t += 1
        for li, (dw, db) in enumerate(grads):
            uot.adam_step(self.params[li][0], dw, self.m[li][0], self.v[li][0], lr, self.t)
            uot.adam_step(self.params[li][1], db, self.m[li][1], self.v[li][1], lr, self.t)
        return self.loss_dev

    def features(self, P, Q, eps, lam):
        """P, Q [N, H, W] FP32 device tensors; eps, lam sequences of N floats."""
        le = torch.as_tensor(np.log(np.asarray(eps, dtype=np.float64)), dtype=torch.float32, device=P.device)
        ll = torch.as_tensor(np.log(np.asarray(lam, dtype=np.float64)), dtype=torch.float32, device=P.device)
        return uot.warmstart_features(P, Q, le, ll)

    def predict(self, P, Q, eps, lam):
        """[N, 2, H, W]: channel 0 = U0, channel 1 = V0.  The network predicts
        potentials divided by lambda; they are scaled back here."""
        out = self.forward(self.features(P, Q, eps, lam))[-1]
        lamt = torch.as_tensor(np.asarray(lam, dtype=np.float32), device=P.device)
        return uot.scale_instances(out, lamt)


def generate_targets(inst, H, W, *, tol=1e-6, max_iter=3000, group=8, device="cuda"):
    """Solve every instance (groups share eps, lambda) with uot_solve_many and
    return (P, Q, U*, V*) as FP32 device tensors [N, H, W]."""
    xs = [torch.as_tensor(a, dtype=torch.float32, device=device) for a in inst["xs"]]
    geo = uot.Geometry.grid(xs, xs)
    dx = torch.as_tensor(inst["dx"], dtype=torch.float32, device=device).ravel()
    P = torch.as_tensor(inst["P"], dtype=torch.float32, device=device)
    Q = torch.as_tensor(inst["Q"], dtype=torch.float32, device=device)
    n = P.shape[0]
    U = torch.empty(n, H * W, device=device)
    V = torch.empty(n, H * W, device=device)
    for s in range(0, n, group):
        e = float(inst["eps"][s])
        lam = float(inst["lam"][s])
        sl = slice(s, min(n, s + group))
        Pg = P[sl].reshape(-1, H * W).contiguous()
        Qg = Q[sl].reshape(-1, H * W).contiguous()
        Ug, Vg, _ = uot.solve_many(geo, Pg, dx, Qg, dx, uot.KL(lam), uot.KL(lam), e,
                                   precision=uot.F32, max_iter=max_iter, tol=tol, check_every=20,
                                   eps_start=max(e, 0.1) if e < 0.1 else None, eps_stages=8,
                                   iters_per_stage=40)
        U[sl] = Ug
        V[sl] = Vg
    return P, Q, U.reshape(n, H, W), V.reshape(n, H, W)


def train(net, P, Q, U, V, eps, lam, *, epochs=20, batch=32, lr=2e-3, seed=0):
    """Minimise the mean squared error between the network output and the
    solver potentials divided by lambda (potentials of a lambda-KL penalty
    scale with lambda)."""
    n = P.shape[0]
    feats = net.features(P, Q, eps, lam)
    target = torch.stack([U, V], dim=1).contiguous()
    inv_lam = torch.as_tensor(1.0 / np.asarray(lam, dtype=np.float64), dtype=torch.float32, device=P.device)
    uot.scale_instances(target, inv_lam)
    rng = np.random.Generator(np.random.Philox(seed))
    hist = []
    for ep in range(epochs):
        perm = rng.permutation(n)
        tot = 0.0
        for s in range(0, n - batch + 1, batch):
            idx = torch.as_tensor(perm[s:s + batch], device=P.device)
            loss = net.train_step(feats[idx].contiguous(), target[idx].contiguous(),
                                  lr * (0.5 * (1 + math.cos(math.pi * ep / epochs))))
            tot += float(loss.item())
        hist.append(tot / max(1, n // batch))
    return hist


def iterations_to_tol(P, Q, eps, lam, H, W, *, U0=None, V0=None, tol=1e-6, max_iter=20000,
                      check_every=10, device="cuda"):
    """Run the plain iteration (FP32, no eps-scaling) on one instance from the
    given start; returns (iterations, final violation, device ms)."""
    xs = [torch.as_tensor((np.arange(n) + 0.5) / n, dtype=torch.float32, device=device) for n in (H, W)]
    geo = uot.Geometry.grid(xs, xs)
    dx = torch.full((H * W,), 1.0 / (H * W), dtype=torch.float32, device=device)
    _, _, info = uot.solve(geo, P.reshape(-1).contiguous(), dx, Q.reshape(-1).contiguous(), dx,
                           uot.KL(lam), uot.KL(lam), eps, precision=uot.F32, max_iter=max_iter,
                           tol=tol, check_every=check_every,
                           U0=None if U0 is None else U0.reshape(-1).contiguous(),
                           V0=None if V0 is None else V0.reshape(-1).contiguous())
    return info["iters"], info["marg_err"], info["ms"]

"""Learned warm start for the scaling iteration (not part of the paper).

A small dilated convolutional network maps the features
(log p, log q, log eps, log lambda) of a grid problem to initial potentials
(U0, V0), which replace the cold start b = 1 of Algorithm 1.  The plain
iteration decides the result: it runs from the predicted potentials to the same
tolerance, so the network can only change how many iterations are needed,
never the answer.

Every numeric step (features, convolutions, their gradients, the loss and
Adam) runs in the library's kernels; this module only holds the parameters
(device tensors) and sequences the calls.  Training targets are potentials
produced by the solver itself (uot_solve_many).
"""
from __future__ import annotations

import math

import threading

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


def generate_targets(inst, H, W, *, tol=1e-6, max_iter=3000, group=8, translate=True, device="cuda"):
    """Solve every instance (groups share eps, lambda) with uot_solve_many (with
    the translation step unless told otherwise: the same fixed point, reached
    in far fewer iterations when lambda >> eps) and return (P, Q, U*, V*) as
    FP32 device tensors [N, H, W]."""
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
                                   iters_per_stage=40, translate=translate)
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


# ---------------------------------------------------------------------------
# The tensor-core network: BF16 3x3 dilated convolutions on tcgen05 (FP32
# accumulation), NHWC activations, FP32 master weights updated by Adam.
# ---------------------------------------------------------------------------

TC_DILATIONS = (1, 2, 4, 8, 16, 32, 1, 2, 4, 8, 16, 1)


class WarmStartNetTC:
    """conv3x3(4 -> C) + leaky, len(dilations) x conv3x3(C -> C, dilation d) + leaky,
    conv3x3(C -> 2) linear; C = 128 gives ~1.8M parameters.  Images 64 wide.
    Output channel 0 is U0 / lambda, channel 1 is V0 / lambda."""

    def __init__(self, channels=128, dilations=TC_DILATIONS, device="cuda", seed=0):
        assert channels in (64, 128)
        gen = torch.Generator(device="cpu").manual_seed(seed)
        self.C = channels
        self.layers = [(4, channels, 1, True)]
        self.layers += [(channels, channels, d, True) for d in dilations]
        self.layers += [(channels, 2, 1, False)]
        self.params, self.m, self.v = [], [], []
        for cin, cout, _, leaky in self.layers:
            std = math.sqrt(2.0 / (cin * 9)) * (1.0 if leaky else 0.1)
            w = (torch.randn(cout, cin, 3, 3, generator=gen) * std).to(device)
            b = torch.zeros(cout, device=device)
            self.params.append([w, b])
            self.m.append([torch.zeros_like(w), torch.zeros_like(b)])
            self.v.append([torch.zeros_like(w), torch.zeros_like(b)])
        self.t = 0
        self.loss_dev = torch.zeros(1, dtype=torch.float64, device=device)
        self.err = torch.zeros(1, dtype=torch.int32, device=device)
        self._refresh_bf16()
        # workspace tensors per host thread: forward passes driven from several
        # threads (each on its own stream) must not share activations
        self._tls = threading.local()

    # geometry of each layer's GEMMs
    def _pads(self, li):
        cin, cout, _, _ = self.layers[li]
        cin_pad = 64 if cin <= 64 else 128            # K channels per tap (forward)
        bn = 16 if cout <= 16 else (64 if cout <= 64 else 128)  # output tile width
        cout_kpad = 64 if cout <= 64 else 128          # K channels per tap (data gradient)
        return cin_pad, bn, cout_kpad

    def _refresh_bf16(self):
        self.wf, self.wb = [], []
        for li, (w, _) in enumerate(self.params):
            cin_pad, bn, cout_kpad = self._pads(li)
            wf, wb = uot.conv_weights_bf16(w, bn, cin_pad, cin_rows=cin_pad, cout_kpad=cout_kpad, backward=li > 0)
            self.wf.append(wf)
            self.wb.append(wb)

    def _refresh_bf16_inplace(self):
        for li, (w, _) in enumerate(self.params):
            cin_pad, bn, cout_kpad = self._pads(li)
            uot.conv_weights_bf16(w, bn, cin_pad, cin_rows=cin_pad, cout_kpad=cout_kpad, wf=self.wf[li],
                                  wb=self.wb[li], backward=li > 0)

    def n_params(self):
        return sum(t.numel() for pr in self.params for t in pr)

    def _buf(self, key, shape, dtype):
        ws = getattr(self._tls, "ws", None)
        if ws is None:
            ws = self._tls.ws = {}
        t = ws.get(key)
        if t is None or t.shape != torch.Size(shape) or t.dtype != dtype:
            t = torch.empty(shape, dtype=dtype, device=self.params[0][0].device)
            ws[key] = t
        return t

    def forward(self, feats, N, H, W, keep=True):
        """feats [N*H*W, 64] BF16 -> (activations, yf [N*H*W, 2] FP32)."""
        acts = [feats]
        h = feats
        P = N * H * W
        for li, (cin, cout, dil, leaky) in enumerate(self.layers[:-1]):
            cin_pad, bn, _ = self._pads(li)
            y = self._buf(("act", li) if keep else ("act", li % 2), (P, cout), torch.bfloat16)
            uot.conv_tc_forward(h, self.wf[li], bn, N, H, W, cin_pad, cout, dil, uot.CONV_LEAKY,
                                bias=self.params[li][1], y=y, err=self.err)
            acts.append(y)
            h = y
        li = len(self.layers) - 1
        cin_pad, bn, _ = self._pads(li)
        yf = self._buf("out", (P, 2), torch.float32)
        uot.conv_tc_forward(h, self.wf[li], bn, N, H, W, cin_pad, 2, 1, uot.CONV_IDENTITY,
                            bias=self.params[li][1], yf=yf, err=self.err)
        return acts, yf

    def backward(self, acts, g, N, H, W):
        """g [P, 16] BF16: gradient at the output; returns [(dw, db)] per layer."""
        grads = [None] * len(self.layers)
        P = N * H * W
        for li in range(len(self.layers) - 1, -1, -1):
            cin, cout, dil, _ = self.layers[li]
            cin_pad, bn, cout_kpad = self._pads(li)
            x = acts[li]
            xT = uot.nhwc_shift_transpose(x, N, H, W, dil, out=self._buf("xT", (3, x.shape[1], P), torch.bfloat16))
            gT = uot.nhwc_transpose(g, out=self._buf(("gT", g.shape[1]), (g.shape[1], P), torch.bfloat16))
            splits = max(1, min(N * H, 64))
            dw = uot.conv_tc_wgrad(gT, xT, cin_pad, N, H, W, dil, cout, cin, splits=splits,
                                   part=self._buf(("part", cin_pad), (splits * 9 * 128 * cin_pad,), torch.float32),
                                   dw=self._buf(("dw", li), (cout, cin, 3, 3), torch.float32), err=self.err)
            db = uot.bias_grad_bf16(g, cout, out=self._buf(("db", li), (cout,), torch.float32))
            grads[li] = (dw, db)
            if li > 0:
                gin = self._buf(("g", li % 2), (P, cin), torch.bfloat16)
                uot.conv_tc_forward(g, self.wb[li], cin_pad, N, H, W, cout_kpad, cin, dil, uot.CONV_DACT,
                                    ref=x, y=gin, err=self.err)
                g = gin
        return grads

    def train_step(self, feats, U, V, inv_lam, N, H, W, lr):
        """One Adam step on a batch: feats [P, 64] BF16, targets U, V [N, HW]
        (potentials), inv_lam [N] (the network predicts potentials / lambda)."""
        acts, yf = self.forward(feats, N, H, W)
        g = self._buf("gout", (N * H * W, 16), torch.bfloat16)
        uot.mse_grad_nhwc(yf, U, V, inv_lam, g, self.loss_dev)
        grads = self.backward(acts, g, N, H, W)
        self.t += 1
        for li, (dw, db) in enumerate(grads):
            uot.adam_step(self.params[li][0], dw, self.m[li][0], self.v[li][0], lr, self.t)
            uot.adam_step(self.params[li][1], db, self.m[li][1], self.v[li][1], lr, self.t)
        self._refresh_bf16_inplace()
        return self.loss_dev

    def features(self, P, Q, eps, lam):
        le = torch.as_tensor(np.log(np.asarray(eps, dtype=np.float64)), dtype=torch.float32, device=P.device)
        ll = torch.as_tensor(np.log(np.asarray(lam, dtype=np.float64)), dtype=torch.float32, device=P.device)
        return uot.warmstart_features_nhwc(P, Q, le, ll)

    def predict(self, P, Q, eps, lam):
        """(U0, V0) [N, H*W] FP32 for the instances P, Q [N, H, W]."""
        N, H, W = P.shape
        _, yf = self.forward(self.features(P, Q, eps, lam), N, H, W, keep=False)
        lamt = torch.as_tensor(np.asarray(lam, dtype=np.float32), device=P.device)
        return uot.pred_to_potentials(yf, lamt, N, H * W)


def train_tc(net, P, Q, U, V, eps, lam, *, epochs=10, batch=32, lr=3e-4, warmup=100, seed=0):
    """Minimise the mean squared error between the network output and the
    solver potentials divided by lambda.  P, Q, U, V [n, H, W] FP32 device
    tensors; features are formed per batch.  Learning rate: linear ramp over
    `warmup` steps, then cosine decay to zero (Adam at 1e-3 on the 1.8M-parameter
    network diverges; 3e-4 trains).  Returns the mean loss of each epoch."""
    n, H, W = P.shape
    dev = P.device
    le = torch.as_tensor(np.log(np.asarray(eps, dtype=np.float64)), dtype=torch.float32, device=dev)
    ll = torch.as_tensor(np.log(np.asarray(lam, dtype=np.float64)), dtype=torch.float32, device=dev)
    inv_lam = torch.as_tensor(1.0 / np.asarray(lam, dtype=np.float64), dtype=torch.float32, device=dev)
    Uf = U.reshape(n, H * W)
    Vf = V.reshape(n, H * W)
    feats = torch.empty(batch * H * W, 64, dtype=torch.bfloat16, device=dev)
    rng = np.random.Generator(np.random.Philox(seed))
    hist = []
    nb = n // batch
    steps = epochs * nb
    step = 0
    for ep in range(epochs):
        perm = torch.as_tensor(rng.permutation(n), device=dev)
        net.loss_dev.zero_()
        for s in range(nb):
            idx = perm[s * batch:(s + 1) * batch]
            uot.warmstart_features_nhwc(P[idx].contiguous(), Q[idx].contiguous(), le[idx].contiguous(),
                                        ll[idx].contiguous(), out=feats)
            lr_t = lr * min(1.0, (step + 1) / max(1, warmup)) * 0.5 * (1 + math.cos(math.pi * step / max(1, steps)))
            net.train_step(feats, Uf[idx].contiguous(), Vf[idx].contiguous(), inv_lam[idx].contiguous(),
                           batch, H, W, lr_t)
            step += 1
        hist.append(float(net.loss_dev.item()) / max(1, nb))
    return hist


def _ev_ms(fn):
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    out = fn()
    e1.record()
    e1.synchronize()
    return e0.elapsed_time(e1), out


def run_on_streams(jobs, nstreams):
    """Runs the callables `jobs` (each one complete solve that synchronises
    with the host at its checks) from `nstreams` host threads, each with its own
    CUDA stream, job k on thread k % nstreams.  The library keeps no state
    shared between calls on different streams (stream-ordered scratch,
    thread-local capture and errors), so latency-bound solves overlap on the
    GPU.  Returns (milliseconds from the first launch to the last job's end,
    measured with CUDA events on the caller's stream, the jobs' results)."""
    out = [None] * len(jobs)
    err = []
    main = torch.cuda.current_stream()
    streams = [torch.cuda.Stream() for _ in range(max(1, nstreams))]
    e0 = torch.cuda.Event(enable_timing=True)
    e0.record(main)
    for st in streams:
        st.wait_event(e0)

    def worker(w):
        try:
            torch.cuda.set_device(main.device)
            with torch.cuda.stream(streams[w]):
                for k in range(w, len(jobs), len(streams)):
                    out[k] = jobs[k]()
        except Exception as ex:  # re-raised on the caller's thread
            err.append(ex)
    threads = [threading.Thread(target=worker, args=(w,)) for w in range(len(streams))]
    for t in threads:
        t.start()
    for t in threads:
        t.join()
    if err:
        raise err[0]
    for st in streams:
        main.wait_stream(st)
    e1 = torch.cuda.Event(enable_timing=True)
    e1.record(main)
    e1.synchronize()
    return e0.elapsed_time(e1), out


def evaluate_tc(net, inst, H, W, *, group, tol=1e-6, plain_sample=16, max_iter=20000, check_every=10,
                cold_plain=True, streams=0, device="cuda"):
    """Time to a `tol` marginal violation (confirmed in FP64, FP64 potentials
    returned) on held-out instances whose consecutive blocks of `group` share
    (eps, lambda):
      plain    : uot_solve per instance, the iteration as printed (no
                 translation), cold start with eps-scaling (1e-1 -> eps, 10
                 stages x 40 iterations when eps < 1e-1), on the first
                 `plain_sample` instances, scaled to all of them;
      batched  : uot_solve_many per group, cold start, same eps-scaling, no
                 translation (skipped when cold_plain is False);
      batched_tr: the same with the translation step (opts.translate);
      warm     : network inference, then uot_solve_many per group from the
                 predicted potentials at the final eps (no eps-scaling), with
                 the translation step; warm_ms includes the inference, whose
                 own time (timed once more on its own) is warm_infer_ms.
    With streams > 0 the translated cold form and the warm form are run once
    more with every group in flight at once (run_on_streams): batched_tr_streams_ms,
    warm_streams_ms, and the number of groups whose iteration count differs from
    the one-at-a-time run (streams_mismatch; the kernels do not depend on what
    else runs, so it is 0).
    Returns a dict of totals and the per-group iteration counts (a batch
    stops when its last problem does)."""
    xs = [torch.as_tensor((np.arange(n) + 0.5) / n, dtype=torch.float32, device=device) for n in (H, W)]
    geo = uot.Geometry.grid(xs, xs)
    dx = torch.full((H * W,), 1.0 / (H * W), dtype=torch.float32, device=device)
    P = torch.as_tensor(inst["P"], dtype=torch.float32, device=device)
    Q = torch.as_tensor(inst["Q"], dtype=torch.float32, device=device)
    n = P.shape[0]
    res = {"n": n, "group": group, "plain_ms": 0.0, "batched_ms": 0.0, "batched_tr_ms": 0.0, "warm_ms": 0.0,
           "warm_infer_ms": 0.0, "plain_iters": [], "batched_iters": [], "batched_tr_iters": [], "warm_iters": [],
           "worst_err_warm": 0.0, "worst_err_batched": 0.0, "worst_err_batched_tr": 0.0, "worst_err_plain": 0.0,
           "groups": []}
    common = dict(precision=uot.F32, max_iter=max_iter, tol=tol, check_every=check_every, launch_mode=2,
                  out_f64=True, verify=True)

    def sched(e):
        return dict(eps_start=0.1, eps_stages=10, iters_per_stage=40) if e < 0.1 else dict(eps_start=None)
    for k in range(min(plain_sample, n)):
        e, lam = float(inst["eps"][k]), float(inst["lam"][k])
        ms, (_, _, info) = _ev_ms(lambda: uot.solve(
            geo, P[k].reshape(-1).contiguous(), dx, Q[k].reshape(-1).contiguous(), dx, uot.KL(lam), uot.KL(lam), e,
            **common, **sched(e)))
        res["plain_ms"] += ms
        res["plain_iters"].append(info["total_iters"])
        res["worst_err_plain"] = max(res["worst_err_plain"], info["marg_err"])
    res["plain_ms"] *= n / max(1, min(plain_sample, n))
    for s in range(0, n, group):
        sl = slice(s, min(n, s + group))
        e, lam = float(inst["eps"][s]), float(inst["lam"][s])
        Pg = P[sl].reshape(-1, H * W).contiguous()
        Qg = Q[sl].reshape(-1, H * W).contiguous()
        grp = {"eps": e, "lam": lam}
        if cold_plain:
            ms, (_, _, info) = _ev_ms(lambda: uot.solve_many(geo, Pg, dx, Qg, dx, uot.KL(lam), uot.KL(lam), e,
                                                             **common, **sched(e)))
            res["batched_ms"] += ms
            res["batched_iters"].append(info["total_iters"])
            res["worst_err_batched"] = max(res["worst_err_batched"], info["marg_err"])
            grp.update(cold_iters=info["total_iters"], cold_ms=round(ms, 2))
        ms, (_, _, info) = _ev_ms(lambda: uot.solve_many(geo, Pg, dx, Qg, dx, uot.KL(lam), uot.KL(lam), e,
                                                         translate=True, **common, **sched(e)))
        res["batched_tr_ms"] += ms
        res["batched_tr_iters"].append(info["total_iters"])
        res["worst_err_batched_tr"] = max(res["worst_err_batched_tr"], info["marg_err"])
        grp.update(cold_tr_iters=info["total_iters"], cold_tr_ms=round(ms, 2), cold_tr_fp64_iters=info["polish_iters"],
                   cold_tr_fp64_checks=info["verifications"])

        def warm():
            U0, V0 = net.predict(P[sl].contiguous(), Q[sl].contiguous(), inst["eps"][sl], inst["lam"][sl])
            return uot.solve_many(geo, Pg, dx, Qg, dx, uot.KL(lam), uot.KL(lam), e, U0=U0, V0=V0, translate=True,
                                  **common)
        # inference alone, timed separately to report its share (warm() repeats it)
        ms_inf, _ = _ev_ms(lambda: net.predict(P[sl].contiguous(), Q[sl].contiguous(), inst["eps"][sl],
                                               inst["lam"][sl]))
        ms, (Uw, Vw, info) = _ev_ms(warm)
        res["warm_ms"] += ms
        res["warm_infer_ms"] += ms_inf
        res["warm_iters"].append(info["total_iters"])
        res["worst_err_warm"] = max(res["worst_err_warm"], info["marg_err"])
        grp.update(warm_iters=info["total_iters"], warm_ms=round(ms, 2), warm_fp64_iters=info["polish_iters"],
                   warm_fp64_checks=info["verifications"])
        res["groups"].append(grp)
        res.setdefault("_last_warm", (s, Uw, Vw))
    if streams > 0:
        starts = list(range(0, n, group))

        def cold_job(s):
            sl = slice(s, min(n, s + group))
            e, lam = float(inst["eps"][s]), float(inst["lam"][s])
            return uot.solve_many(geo, P[sl].reshape(-1, H * W).contiguous(), dx, Q[sl].reshape(-1, H * W).contiguous(),
                                  dx, uot.KL(lam), uot.KL(lam), e, translate=True, **common, **sched(e))

        def warm_job(s):
            sl = slice(s, min(n, s + group))
            e, lam = float(inst["eps"][s]), float(inst["lam"][s])
            U0, V0 = net.predict(P[sl].contiguous(), Q[sl].contiguous(), inst["eps"][sl], inst["lam"][sl])
            return uot.solve_many(geo, P[sl].reshape(-1, H * W).contiguous(), dx, Q[sl].reshape(-1, H * W).contiguous(),
                                  dx, uot.KL(lam), uot.KL(lam), e, U0=U0, V0=V0, translate=True, **common)
        mism = 0
        for key, job, iters_key in (("batched_tr_streams", cold_job, "batched_tr_iters"),
                                    ("warm_streams", warm_job, "warm_iters")):
            ms, outs = run_on_streams([(lambda s=s: job(s)) for s in starts], streams)
            res[key + "_ms"] = ms
            res["worst_err_" + key] = max(o[2]["marg_err"] for o in outs)
            mism += sum(o[2]["total_iters"] != it for o, it in zip(outs, res[iters_key]))
        res["streams"] = streams
        res["streams_mismatch"] = mism
    return res

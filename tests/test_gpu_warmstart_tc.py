"""The tensor-core warm-start network (BF16 tcgen05 convolutions, FP32
master weights): its gradients against the FP64 network oracle's exact
gradients chained layer by layer, and training on solver-generated instances.
BF16 activations carry a relative rounding of 2^-9 per layer, so the
whole-network gradient is compared with a 3% bound on its largest entry."""
import numpy as np
import pytest
import torch

import oracle as O
import oracle.net_oracle as NO
from paper_1607_05816_gb300 import synth
from paper_1607_05816_gb300 import uot as U
from paper_1607_05816_gb300 import warmstart as WS

pytestmark = pytest.mark.gpu


def bf(t):
    return t.detach().to(torch.bfloat16).double().cpu().numpy()


def _setup_small():
    N, H, W = 2, 4, 64
    inst = synth.warmstart_instances(N, H, W, seed=5, group=N)
    net = WS.WarmStartNetTC(channels=64, dilations=(1, 3), seed=2)
    P = torch.as_tensor(inst["P"], dtype=torch.float32, device="cuda")
    Q = torch.as_tensor(inst["Q"], dtype=torch.float32, device="cuda")
    feats = net.features(P, Q, inst["eps"], inst["lam"])
    x = np.transpose(bf(feats).reshape(N, H, W, 64)[..., :4], (0, 3, 1, 2))
    ws = [(bf(w), b.detach().double().cpu().numpy()) for w, b in net.params]
    return N, H, W, net, feats, x, ws


def test_tc_network_forward_matches_oracle():
    """The network output against the oracle's forward pass on the same BF16
    weights and features, with each hidden activation rounded to BF16 as the
    kernels store it."""
    N, H, W, net, feats, x, ws = _setup_small()
    _, yf = net.forward(feats, N, H, W)
    torch.cuda.synchronize()
    h = x
    for li, ((w, b), (_, _, dil, leaky)) in enumerate(zip(ws, net.layers)):
        h = NO.conv2d(h, w, b, dil, leaky)
        if li < len(ws) - 1:
            h = bf(torch.as_tensor(h))
    got = np.transpose(yf.double().cpu().numpy().reshape(N, H, W, 2), (0, 3, 1, 2))
    assert np.max(np.abs(got - h)) <= 1e-2 * np.max(np.abs(h)), np.max(np.abs(got - h))


def test_tc_network_gradients_match_oracle():
    """Every layer's weight and bias gradient against the oracle's exact
    gradients chained through the network, evaluated on the activations the
    kernels stored (BF16); the kernels round each propagated gradient to BF16."""
    N, H, W, net, feats, x, ws = _setup_small()
    g = np.random.default_rng(1)
    Ut = torch.as_tensor(g.normal(size=(N, H * W)), dtype=torch.float32, device="cuda")
    Vt = torch.as_tensor(g.normal(size=(N, H * W)), dtype=torch.float32, device="cuda")
    inv_lam = torch.ones(N, device="cuda")
    acts, yf = net.forward(feats, N, H, W)
    gout = torch.empty(N * H * W, 16, dtype=torch.bfloat16, device="cuda")
    net.loss_dev.zero_()
    U.mse_grad_nhwc(yf, Ut, Vt, inv_lam, gout, net.loss_dev)
    grads = net.backward(acts, gout, N, H, W)
    torch.cuda.synchronize()
    assert net.err.item() == 0
    C = [64] + [lay[1] for lay in net.layers[:-1]]
    hs = [x] + [np.transpose(bf(a).reshape(N, H, W, -1)[..., :c], (0, 3, 1, 2)) for a, c in zip(acts[1:], C[1:])]
    out = np.transpose(yf.double().cpu().numpy().reshape(N, H, W, 2), (0, 3, 1, 2))
    tgt = np.stack([Ut.double().cpu().numpy().reshape(N, H, W), Vt.double().cpu().numpy().reshape(N, H, W)], 1)
    assert abs(net.loss_dev.item() - float(np.mean((out - tgt) ** 2))) <= 1e-5 * float(np.mean((out - tgt) ** 2))
    G = 2.0 * (out - tgt) / out.size
    for li in range(len(ws) - 1, -1, -1):
        dil = net.layers[li][2]
        dx, dw, db = NO.conv2d_grads(hs[li], ws[li][0], G, dil)
        got_w = grads[li][0].double().cpu().numpy()
        got_b = grads[li][1].double().cpu().numpy()
        print(f"layer {li}: max |dW - oracle| / max |dW| = {np.max(np.abs(got_w - dw)) / np.max(np.abs(dw)):.2e}")
        assert np.max(np.abs(got_w - dw)) <= 1e-2 * np.max(np.abs(dw)), (li, np.max(np.abs(got_w - dw)))
        assert np.max(np.abs(got_b - db)) <= 1e-2 * max(1e-12, np.max(np.abs(db))), li
        if li > 0:
            G = dx * np.where(hs[li] < 0, NO.LEAK, 1.0)


def test_tc_training_reduces_loss():
    H = W = 64
    inst = synth.warmstart_instances(128, H, W, seed=31, group=32, eps=(1e-2, 1e-1), lam=(0.3, 10.0))
    P, Q, Us, Vs = WS.generate_targets(inst, H, W, max_iter=3000, group=32)
    net = WS.WarmStartNetTC(channels=128, seed=3)
    assert 1.5e6 < net.n_params() < 2.5e6
    hist = WS.train_tc(net, P, Q, Us, Vs, inst["eps"], inst["lam"], epochs=10, batch=16, lr=3e-4, warmup=10)
    torch.cuda.synchronize()
    assert net.err.item() == 0
    print("tc training loss per epoch:", hist)
    assert hist[-1] < 0.5 * hist[0]


def test_mse_gradient_pads_with_zeros():
    """The loss gradient buffer is 16 channels wide (the last layer's padded
    output): channels 0, 1 hold 2 (pred - target s) / (2P), channels 2 to 15 are
    written as exact zeros whatever the buffer held (here NaN), since the data
    gradient multiplies them by the zero padding weights."""
    N, HW = 3, 64 * 4
    g = np.random.default_rng(7)
    pred = torch.as_tensor(g.normal(size=(N * HW, 2)), dtype=torch.float32, device="cuda")
    Ut = torch.as_tensor(g.normal(size=(N, HW)), dtype=torch.float32, device="cuda")
    Vt = torch.as_tensor(g.normal(size=(N, HW)), dtype=torch.float32, device="cuda")
    s = torch.as_tensor([0.5, 1.0, 2.0], dtype=torch.float32, device="cuda")
    grad = torch.full((N * HW, 16), float("nan"), dtype=torch.bfloat16, device="cuda")
    loss = torch.zeros(1, dtype=torch.float64, device="cuda")
    U.mse_grad_nhwc(pred, Ut, Vt, s, grad, loss)
    torch.cuda.synchronize()
    got = grad.double().cpu().numpy()
    assert np.all(got[:, 2:] == 0.0)
    pr = pred.double().cpu().numpy()
    sc = np.repeat(s.double().cpu().numpy(), HW)
    tgt = np.stack([Ut.double().cpu().numpy().ravel() * sc, Vt.double().cpu().numpy().ravel() * sc], 1)
    want = 2.0 * (pr - tgt) / pr.size
    assert np.max(np.abs(got[:, :2] - want)) <= 2.0 ** -8 * np.max(np.abs(want))
    assert abs(loss.item() - np.mean((pr - tgt) ** 2)) <= 1e-5 * np.mean((pr - tgt) ** 2)


def test_trained_tc_network_reduces_iterations_to_tol():
    """What the trained network gains: 2048 solver-generated 64 x 64 instances
    (eps in [1e-2, 1e-1], lambda in [0.1, 10]), three epochs; on 16 held-out
    instances the solve to 1e-6 (FP32 passes, stop confirmed in FP64, the
    translation step in both forms) from the predicted potentials needs fewer
    iterations than the cold start with eps-scaling, for the median and in
    total, and the oracle confirms the warm result of one instance."""
    H = W = 64
    kw = dict(eps=(1e-2, 1e-1), lam=(0.1, 10.0))
    inst = synth.warmstart_instances(2048, H, W, seed=31, group=64, **kw)
    P, Q, Us, Vs = WS.generate_targets(inst, H, W, max_iter=6000, group=64)
    net = WS.WarmStartNetTC(channels=128, seed=3)
    hist = WS.train_tc(net, P, Q, Us, Vs, inst["eps"], inst["lam"], epochs=3, batch=32)
    assert np.isfinite(hist).all() and hist[-1] < 0.5 * hist[0], hist
    ev = synth.warmstart_instances(16, H, W, seed=32, group=1, **kw)
    Pe = torch.as_tensor(ev["P"], dtype=torch.float32, device="cuda")
    Qe = torch.as_tensor(ev["Q"], dtype=torch.float32, device="cuda")
    U0, V0 = net.predict(Pe, Qe, ev["eps"], ev["lam"])
    xs = [torch.as_tensor(a, dtype=torch.float32, device="cuda") for a in ev["xs"]]
    geo = U.Geometry.grid(xs, xs)
    dx = torch.full((H * W,), 1.0 / (H * W), device="cuda")
    common = dict(precision=U.F32, max_iter=20000, tol=1e-6, check_every=10, launch_mode=2, out_f64=True,
                  verify=True, translate=True)
    cold, warm = [], []
    for k in range(16):
        e, lam = float(ev["eps"][k]), float(ev["lam"][k])
        args = (geo, Pe[k].reshape(-1), dx, Qe[k].reshape(-1), dx, U.KL(lam), U.KL(lam), e)
        _, _, ic = U.solve(*args, eps_start=0.1 if e < 0.1 else None, eps_stages=10, iters_per_stage=40, **common)
        Uw, Vw, iw = U.solve(*args, U0=U0[k].contiguous(), V0=V0[k].contiguous(), **common)
        assert ic["status"] == "UOT_OK" and iw["status"] == "UOT_OK"
        cold.append(ic["total_iters"])
        warm.append(iw["total_iters"])
    print("cold", cold, "\nwarm", warm)
    assert np.median(warm) < np.median(cold) and sum(warm) < sum(cold)
    rr = lambda a: np.asarray(a, np.float32).astype(np.float64)
    ax = [rr(a) for a in ev["xs"]]
    v = O.marginal_violation(O.Geometry("grid", xs=ax, ys=ax), rr(ev["dx"]), rr(ev["dx"]), rr(ev["P"][15]),
                             rr(ev["Q"][15]), O.KL(lam), O.KL(lam), e, Uw.double().cpu().numpy().reshape(H, W),
                             Vw.double().cpu().numpy().reshape(H, W))
    assert v <= 1e-6, v

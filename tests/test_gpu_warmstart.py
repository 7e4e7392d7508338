"""Learned warm start: network kernels against the CPU reference, batched
solve parity, and the gain of a trained network over the cold start."""
import numpy as np
import pytest
import torch

import oracle as O
import oracle.net_oracle as NO
from paper_1607_05816_gb300 import synth
from paper_1607_05816_gb300 import uot as U
from paper_1607_05816_gb300 import warmstart as WS

pytestmark = [pytest.mark.gpu, pytest.mark.filterwarnings("ignore::RuntimeWarning")]


def t32(a):
    return torch.as_tensor(np.ascontiguousarray(a), dtype=torch.float32, device="cuda")


@pytest.mark.parametrize("shape,dil,leaky", [((3, 4, 17, 23), 1, True), ((2, 9, 64, 64), 4, True), ((2, 32, 16, 16), 2, False)])
def test_conv_forward_parity(shape, dil, leaky):
    g = synth.rng(1)
    N, Cin, H, W = shape
    x = g.normal(size=shape).astype(np.float32)
    w = (g.normal(size=(11, Cin, 3, 3)) / np.sqrt(Cin * 9)).astype(np.float32)
    b = g.normal(size=11).astype(np.float32)
    got = U.conv2d_forward(t32(x), t32(w), t32(b), dil, leaky).cpu().numpy()
    want = NO.conv2d(x, w, b, dil, leaky)
    assert np.max(np.abs(got - want)) <= 1e-5 * max(1.0, np.max(np.abs(want)))


def test_network_gradients_match_finite_differences():
    """dw, db of every layer and the input gradient path through three layers,
    from the CUDA backward kernels, against central differences of the FP64
    reference loss."""
    g = synth.rng(2)
    net = WS.WarmStartNet(channels=5, dilations=(2,), seed=3)
    x = g.normal(size=(2, 4, 9, 8)).astype(np.float32)
    target = g.normal(size=(2, 2, 9, 8)).astype(np.float32)
    acts = net.forward(t32(x))
    dout = torch.empty_like(acts[-1])
    U.mse_grad(acts[-1], t32(target), dout, net.loss_dev)
    grads = net.backward(acts, dout)
    params = [(w.cpu().numpy().astype(np.float64), b.cpu().numpy().astype(np.float64)) for w, b in net.params]
    layers = [(dil, leaky) for _, _, dil, leaky in net.layers]
    assert abs(net.loss_dev.item() - NO.mse(params, layers, x, target)) < 1e-5
    rng = np.random.Generator(np.random.Philox(4))
    for li, (dw, db) in enumerate(grads):
        dw = dw.cpu().numpy()
        db = db.cpu().numpy()
        for _ in range(4):
            idx = tuple(int(rng.integers(0, s)) for s in dw.shape)
            fd = NO.fd_grad(params, layers, x, target, (li, 0), idx, h=1e-4)
            assert abs(dw[idx] - fd) <= 2e-3 * max(1e-3, abs(fd)) + 1e-6, (li, idx, dw[idx], fd)
        co = int(rng.integers(0, db.shape[0]))
        fd = NO.fd_grad(params, layers, x, target, (li, 1), co, h=1e-4)
        assert abs(db[co] - fd) <= 2e-3 * max(1e-3, abs(fd)) + 1e-6


def test_features_kernel():
    g = synth.rng(3)
    P = g.uniform(0, 2, size=(3, 8, 9)).astype(np.float32)
    P[0, 0, 0] = 0.0
    Q = g.uniform(0, 2, size=(3, 8, 9)).astype(np.float32)
    le = np.log([0.01, 0.1, 0.003]).astype(np.float32)
    ll = np.log([0.5, 2.0, 9.0]).astype(np.float32)
    got = U.warmstart_features(t32(P), t32(Q), t32(le), t32(ll)).cpu().numpy()
    lp = np.maximum(np.log(np.maximum(P.astype(np.float64), 1e-30)), -30)
    assert np.allclose(got[:, 0], 0.25 * lp, atol=1e-5)
    assert np.allclose(got[:, 3], 0.25 * ll[:, None, None], atol=1e-6)


@pytest.mark.parametrize("prec", [U.F64, U.F32])
def test_solve_many_parity(prec):
    inst = synth.warmstart_instances(5, 20, 24, seed=9, group=5, eps=(0.01, 0.05))
    og = O.Geometry("grid", xs=inst["xs"], ys=inst["xs"])
    dt = U._dtype(prec)
    xs = [torch.as_tensor(a, dtype=dt, device="cuda") for a in inst["xs"]]
    geo = U.Geometry.grid(xs, xs)
    rd = lambda a: np.asarray(a, dtype=np.float64 if prec == U.F64 else np.float32).astype(np.float64)
    dx = torch.as_tensor(inst["dx"], dtype=dt, device="cuda").ravel()
    P = torch.as_tensor(inst["P"].reshape(5, -1), dtype=dt, device="cuda")
    Q = torch.as_tensor(inst["Q"].reshape(5, -1), dtype=dt, device="cuda")
    e, lam = float(inst["eps"][0]), float(inst["lam"][0])
    Ug, Vg, info = U.solve_many(geo, P, dx, Q, dx, U.KL(lam), U.KL(lam), e, precision=prec, max_iter=30)
    tol = 1e-10 if prec == U.F64 else 1e-5
    for k in range(5):
        r = O.solve_log(og, rd(inst["dx"]), rd(inst["dx"]), rd(inst["P"][k]), rd(inst["Q"][k]),
                        O.KL(lam), O.KL(lam), e, max_iter=30)
        for got, want in ((Ug[k], r["U"]), (Vg[k], r["V"])):
            gv = got.double().cpu().numpy()
            wv = want.ravel()
            assert np.max(np.abs(gv - wv)) <= tol * max(1.0, np.max(np.abs(wv)))


def test_trained_network_reduces_iterations():
    """Train on solver-generated instances, then run the plain iteration from
    the predicted potentials and from the cold start on held-out instances:
    the warm start needs fewer iterations (median) to the same tolerance."""
    H = W = 32
    inst = synth.warmstart_instances(512, H, W, seed=21, group=4, eps=(1e-2, 1e-1), lam=(0.3, 10.0))
    P, Q, Us, Vs = WS.generate_targets(inst, H, W, max_iter=4000, group=4)
    ntr = 512
    net = WS.WarmStartNet(channels=24, seed=1)
    hist = WS.train(net, P, Q, Us, Vs, inst["eps"], inst["lam"], epochs=40, batch=32, lr=3e-3)
    assert hist[-1] < hist[0]
    inst = synth.warmstart_instances(24, H, W, seed=22, group=1, eps=(1e-2, 1e-1), lam=(0.3, 10.0))
    P = torch.as_tensor(inst["P"], dtype=torch.float32, device="cuda")
    Q = torch.as_tensor(inst["Q"], dtype=torch.float32, device="cuda")
    ntr = 0
    cold, warm = [], []
    for k in range(ntr, ntr + 24):
        pred = net.predict(P[k:k + 1], Q[k:k + 1], inst["eps"][k:k + 1], inst["lam"][k:k + 1])
        e, lam = float(inst["eps"][k]), float(inst["lam"][k])
        ic, ec, _ = WS.iterations_to_tol(P[k], Q[k], e, lam, H, W)
        iw, ew, _ = WS.iterations_to_tol(P[k], Q[k], e, lam, H, W, U0=pred[0, 0], V0=pred[0, 1])
        assert ew <= 1e-6 and ec <= 1e-6
        cold.append(ic)
        warm.append(iw)
    assert np.median(warm) < np.median(cold), (np.median(warm), np.median(cold))


@pytest.mark.parametrize("prec", [U.F64, U.F32])
@pytest.mark.parametrize("bad", [float("nan"), float("inf")])
def test_bad_warm_start_rejected(prec, bad):
    """A NaN or +inf start potential is refused with UOT_EINVAL (it would turn
    every log-sum-exp into NaN or -inf); -inf (a zero scaling) is a valid start."""
    inst = synth.warmstart_instances(2, 16, 16, seed=4, group=2)
    dt = U._dtype(prec)
    xs = [torch.as_tensor(a, dtype=dt, device="cuda") for a in inst["xs"]]
    geo = U.Geometry.grid(xs, xs)
    dx = torch.as_tensor(inst["dx"], dtype=dt, device="cuda").ravel()
    P = torch.as_tensor(inst["P"].reshape(2, -1), dtype=dt, device="cuda")
    Q = torch.as_tensor(inst["Q"].reshape(2, -1), dtype=dt, device="cuda")
    e, lam = float(inst["eps"][0]), float(inst["lam"][0])
    U0 = torch.zeros(256, dtype=dt, device="cuda")
    U0[17] = -float("inf")
    _, _, info = U.solve(geo, P[0], dx, Q[0], dx, U.KL(lam), U.KL(lam), e, precision=prec, max_iter=5, U0=U0)
    assert info["status"] in ("UOT_OK", "UOT_NOT_CONVERGED")
    U0[40] = bad
    with pytest.raises(U.UotError) as ex:
        U.solve(geo, P[0], dx, Q[0], dx, U.KL(lam), U.KL(lam), e, precision=prec, max_iter=5, U0=U0)
    assert ex.value.status == -1
    V0 = torch.zeros(2, 256, dtype=dt, device="cuda")
    V0[1, 3] = bad
    with pytest.raises(U.UotError) as ex:
        U.solve_many(geo, P, dx, Q, dx, U.KL(lam), U.KL(lam), e, precision=prec, max_iter=5, V0=V0)
    assert ex.value.status == -1

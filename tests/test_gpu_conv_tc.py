"""Tensor-core (tcgen05 + TMA) convolutions of the warm-start network against
the FP64 numpy network oracle, on BF16-rounded inputs and weights: forward
(identity and leaky epilogues, 16-, 64- and 128-wide outputs, dilations 1 to
5, zero padding), the data gradient through the flipped weights with the
activation-derivative epilogue, the weight and bias gradients, and the
weight-layout transform.  BF16 products are exact in FP32, so the kernels
differ from the oracle only by FP32 accumulation order: 1e-4 of the largest
magnitude is a loose bound (the BF16-rounded outputs are checked to a BF16
rounding step)."""
import numpy as np
import pytest
import torch

import oracle.net_oracle as NO
from paper_1607_05816_gb300 import uot as U

pytestmark = pytest.mark.gpu


def bf(a):
    """round to BF16 (as the device stores it), back to float64"""
    return torch.as_tensor(np.asarray(a, np.float32)).to(torch.bfloat16).float().double().numpy()


def nhwc_dev(a_nchw, ld):
    """NCHW float64 -> device BF16 [N*H*W, ld] (zero channels beyond C)"""
    N, C, H, W = a_nchw.shape
    out = np.zeros((N, H, W, ld), np.float32)
    out[..., :C] = np.transpose(a_nchw, (0, 2, 3, 1))
    return torch.as_tensor(out.reshape(N * H * W, ld)).to(torch.bfloat16).cuda()


def to_nchw(t, N, H, W, C):
    return np.transpose(t.float().cpu().numpy().reshape(N, H, W, -1)[..., :C], (0, 3, 1, 2)).astype(np.float64)


def close(got, want, rtol=1e-4):
    return np.max(np.abs(got - want)) <= rtol * max(1e-30, np.max(np.abs(want)))


CASES = [  # (N, H, Cin, ldx, cin_pad, Cout, bn, dil)
    (2, 8, 64, 64, 64, 128, 128, 1),
    (1, 16, 128, 128, 128, 128, 128, 3),
    (3, 4, 4, 64, 64, 128, 128, 1),     # first layer: 4 features in 64 channels
    (2, 8, 128, 128, 128, 2, 16, 5),    # last layer: 2 outputs, 16-wide tile
    (2, 6, 64, 64, 64, 40, 64, 2),      # 64-wide tile, ragged output channels
]


@pytest.mark.parametrize("N,H,Cin,ldx,cin_pad,Cout,bn,dil", CASES)
@pytest.mark.parametrize("leaky", [False, True])
def test_conv_forward_matches_oracle(N, H, Cin, ldx, cin_pad, Cout, bn, dil, leaky):
    W = 64
    g = np.random.default_rng(N * 100 + H + dil)
    x = bf(g.normal(size=(N, Cin, H, W)))
    w = bf(g.normal(size=(Cout, Cin, 3, 3)) / np.sqrt(9 * Cin))
    b = g.normal(size=Cout).astype(np.float32)
    wt = torch.as_tensor(w, dtype=torch.float32).cuda()
    wf, _ = U.conv_weights_bf16(wt, bn, cin_pad, backward=False)
    xd = nhwc_dev(x, ldx)
    P = N * H * W
    yf = torch.empty(P, Cout, dtype=torch.float32, device="cuda")
    ldy = max(16, (Cout + 15) // 16 * 16)
    y = torch.empty(P, ldy, dtype=torch.bfloat16, device="cuda")
    err = torch.zeros(1, dtype=torch.int32, device="cuda")
    U.conv_tc_forward(xd, wf, bn, N, H, W, cin_pad, Cout, dil, U.CONV_LEAKY if leaky else U.CONV_IDENTITY,
                      bias=torch.as_tensor(b).cuda(), y=y, yf=yf, err=err)
    torch.cuda.synchronize()
    assert err.item() == 0
    want = NO.conv2d(x, w, b.astype(np.float64), dil, leaky)
    got = np.transpose(yf.cpu().numpy().reshape(N, H, W, Cout), (0, 3, 1, 2)).astype(np.float64)
    assert close(got, want), np.max(np.abs(got - want))
    gb = to_nchw(y, N, H, W, Cout)
    assert np.max(np.abs(gb - want)) <= 2.0 ** -7 * np.max(np.abs(want))
    assert not y[:, Cout:].float().abs().sum().item()  # padding channels written as 0


@pytest.mark.parametrize("N,H,Cin,cin_pad,Cout,ldg,dil", [(2, 8, 128, 128, 128, 128, 2), (2, 4, 64, 64, 2, 16, 1),
                                                          (1, 8, 4, 64, 128, 128, 4)])
def test_conv_data_gradient_matches_oracle(N, H, Cin, cin_pad, Cout, ldg, dil):
    """dx = (sum over taps of the flipped weights applied to dy) times the
    leaky-ReLU derivative at the layer's input, as the backward pass uses it."""
    W = 64
    g = np.random.default_rng(11 + H + Cout)
    w = bf(g.normal(size=(Cout, Cin, 3, 3)) / np.sqrt(9 * Cin))
    dy = bf(g.normal(size=(N, Cout, H, W)))
    ref = bf(g.normal(size=(N, Cin, H, W)))  # the layer's input (previous output, mixed signs)
    cout_kpad = max(64, (Cout + 63) // 64 * 64)
    wt = torch.as_tensor(w, dtype=torch.float32).cuda()
    _, wb = U.conv_weights_bf16(wt, max(16, (Cout + 15) // 16 * 16), cin_pad, cin_rows=cin_pad, cout_kpad=cout_kpad)
    dyd = nhwc_dev(dy, ldg)
    refd = nhwc_dev(ref, cin_pad)
    err = torch.zeros(1, dtype=torch.int32, device="cuda")
    dx = U.conv_tc_forward(dyd, wb, cin_pad, N, H, W, cout_kpad, Cin, dil, U.CONV_DACT, ref=refd, err=err)
    torch.cuda.synchronize()
    assert err.item() == 0
    want = NO.conv2d_grads(ref, w, dy, dil)[0] * np.where(ref < 0, NO.LEAK, 1.0)
    got = to_nchw(dx, N, H, W, Cin)
    assert np.max(np.abs(got - want)) <= 2.0 ** -7 * np.max(np.abs(want)), np.max(np.abs(got - want))


@pytest.mark.parametrize("N,H,Cin,cin_pad,Cout,ldg,dil,splits", [(2, 8, 128, 128, 128, 128, 2, 5),
                                                                 (3, 4, 4, 64, 128, 128, 1, 12),
                                                                 (2, 8, 128, 128, 2, 16, 3, 4)])
def test_conv_weight_and_bias_gradients_match_oracle(N, H, Cin, cin_pad, Cout, ldg, dil, splits):
    W = 64
    g = np.random.default_rng(21 + H + Cout)
    x = bf(g.normal(size=(N, Cin, H, W)))
    dy = bf(g.normal(size=(N, Cout, H, W)))
    xd = nhwc_dev(x, cin_pad)
    dyd = nhwc_dev(dy, ldg)
    xT = U.nhwc_shift_transpose(xd, N, H, W, dil)
    dyT = U.nhwc_transpose(dyd)
    err = torch.zeros(1, dtype=torch.int32, device="cuda")
    dw = U.conv_tc_wgrad(dyT, xT, cin_pad, N, H, W, dil, Cout, Cin, splits=splits, err=err)
    db = U.bias_grad_bf16(dyd, Cout)
    torch.cuda.synchronize()
    assert err.item() == 0
    _, want_w, want_b = NO.conv2d_grads(x, np.zeros((Cout, Cin, 3, 3)), dy, dil)
    assert close(dw.double().cpu().numpy(), want_w), np.max(np.abs(dw.double().cpu().numpy() - want_w))
    assert close(db.double().cpu().numpy(), want_b, 1e-4)


def test_shift_transpose_layout():
    N, H, W, C, dil = 2, 3, 64, 64, 5
    x = torch.randn(N * H * W, C, device="cuda").to(torch.bfloat16)
    xT = U.nhwc_shift_transpose(x, N, H, W, dil).float().cpu().numpy().reshape(3, C, N, H, W)
    xn = x.float().cpu().numpy().reshape(N, H, W, C)
    for d in range(3):
        sh = (d - 1) * dil
        want = np.zeros((C, N, H, W), np.float32)
        lo, hi = max(0, -sh), min(W, W - sh)
        want[..., lo:hi] = np.transpose(xn, (3, 0, 1, 2))[..., lo + sh:hi + sh]
        assert np.array_equal(xT[d], want)


def test_weight_layouts():
    Cout, Cin = 5, 3
    w = torch.randn(Cout, Cin, 3, 3, device="cuda")
    wf, wb = U.conv_weights_bf16(w, 16, 64, cin_rows=64, cout_kpad=64)
    wr = w.to(torch.bfloat16).float().cpu().numpy().reshape(Cout, Cin, 9)
    f = wf.float().cpu().numpy()
    b = wb.float().cpu().numpy()
    assert np.array_equal(f[:Cout, :, :Cin], np.transpose(wr, (0, 2, 1)))
    assert not f[Cout:].any() and not f[:, :, Cin:].any()
    assert np.array_equal(b[:Cin, :, :Cout], np.transpose(wr[:, :, ::-1], (1, 2, 0)))
    assert not b[Cin:].any() and not b[:, :, Cout:].any()

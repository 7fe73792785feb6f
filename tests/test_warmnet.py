"""Learned warm start: the network kernels against plain PyTorch fp32 references (on the
CPU), and the warm-started solve against the oracle given the same start messages."""
import numpy as np
import pytest
import torch
import torch.nn.functional as F

import oracle
import paper_1709_06509_gb300 as bps
from paper_1709_06509_gb300 import synth, warmstart

pytestmark = pytest.mark.gpu
DEV = torch.device("cuda:0")


@pytest.fixture(scope="module", autouse=True)
def built():
    import __graft_entry__

    __graft_entry__.build()


def bf16_round(t):
    return t.to(torch.bfloat16).to(torch.float32)


@pytest.mark.parametrize("relu", [0, 1])
@pytest.mark.parametrize("in_bf16", [0, 1])
def test_conv_forward(relu, in_bf16):
    g = torch.Generator().manual_seed(1)
    B, Cin, Cout, H, W = 3, 5, 7, 9, 11
    x = torch.randn(B, Cin, H, W, generator=g)
    w = bf16_round(torch.randn(Cout, Cin, 3, 3, generator=g) * 0.3)
    b = torch.randn(Cout, generator=g)
    xin = bf16_round(x) if in_bf16 else x
    ref = F.conv2d(xin, w, b, padding=1)
    if relu:
        ref = ref.clamp(min=0)
    xd = (x.to(torch.bfloat16) if in_bf16 else x).to(DEV)
    out = torch.empty(B, Cout, H, W, device=DEV)
    bps.bps_warmnet_conv3x3(xd, in_bf16, B, Cin, H, W, w.to(torch.bfloat16).to(DEV), b.to(DEV), Cout, relu, out, 0)
    torch.cuda.synchronize()
    assert torch.allclose(out.cpu(), ref, rtol=1e-4, atol=1e-4)


@pytest.mark.parametrize("shape", [(2, 32, 32, 47, 57), (1, 8, 256, 47, 57), (1, 32, 1024, 20, 30), (3, 5, 7, 9, 11),
                                   (1, 1, 17, 130, 3), (2, 3, 300, 7, 5)],
                         ids=lambda s: "x".join(map(str, s)))
@pytest.mark.parametrize("out_bf16", [0, 1])
def test_tensor_core_conv_matches_fp32_conv2d(shape, out_bf16):
    # BF16 activations take the tensor-core implicit GEMM: against an FP32 convolution of the same
    # BF16 values on the CPU (every product exact in FP32, only the summation order differs)
    B, Cin, Cout, H, W = shape
    g = torch.Generator().manual_seed(B * 1000 + Cin * 10 + Cout)
    x = bf16_round(torch.randn(B, Cin, H, W, generator=g))
    w = bf16_round(torch.randn(Cout, Cin, 3, 3, generator=g) * 0.2)
    b = torch.randn(Cout, generator=g)
    ref = F.conv2d(x, w, b, padding=1).clamp(min=0)
    out = torch.empty(B, Cout, H, W, dtype=torch.bfloat16 if out_bf16 else torch.float32, device=DEV)
    bps.bps_warmnet_conv3x3(x.to(torch.bfloat16).to(DEV), 1, B, Cin, H, W, w.to(torch.bfloat16).to(DEV), b.to(DEV),
                            Cout, 1, out, out_bf16)
    torch.cuda.synchronize()
    assert bps.bps_warmnet_get_error() == bps.BPS_OK
    got = out.to(torch.float32).cpu()
    if out_bf16:  # one BF16 rounding of nearly equal FP32 sums: at most one unit apart
        assert torch.allclose(got, bf16_round(ref), rtol=2 ** -7, atol=1e-3)
    else:
        assert torch.allclose(got, ref, rtol=1e-4, atol=1e-4)


@pytest.mark.parametrize("relu", [0, 1])
def test_conv_backward(relu):
    g = torch.Generator().manual_seed(2)
    B, Cin, Cout, H, W = 2, 4, 6, 7, 10
    x = bf16_round(torch.randn(B, Cin, H, W, generator=g))
    w = bf16_round(torch.randn(Cout, Cin, 3, 3, generator=g) * 0.3)
    b = torch.randn(Cout, generator=g)
    gout = torch.randn(B, Cout, H, W, generator=g)
    y = F.conv2d(x, w, b, padding=1)
    # the kernels mask the upstream gradient with the layer's (BF16) forward output > 0
    relu_out = y.clamp(min=0).to(torch.bfloat16) if relu else None
    geff = gout * (relu_out.to(torch.float32) > 0) if relu else gout
    xr, wr, br = (t.clone().requires_grad_(True) for t in (x, w, b))
    F.conv2d(xr, wr, br, padding=1).backward(geff)
    gin = torch.empty(B, Cin, H, W, device=DEV)
    gw = torch.empty(Cout, Cin, 3, 3, device=DEV)
    gb = torch.empty(Cout, device=DEV)
    bps.bps_warmnet_conv3x3_backward(gout.to(DEV), None if relu_out is None else relu_out.to(DEV),
                                     x.to(torch.bfloat16).to(DEV), 1, B, Cin, H, W, w.to(torch.bfloat16).to(DEV), Cout,
                                     gin, gw, gb)
    torch.cuda.synchronize()
    assert torch.allclose(gin.cpu(), xr.grad, rtol=1e-4, atol=1e-4)
    assert torch.allclose(gw.cpu(), wr.grad, rtol=1e-4, atol=1e-3)
    assert torch.allclose(gb.cpu(), br.grad, rtol=1e-4, atol=1e-3)


def test_mse_and_adam():
    g = torch.Generator().manual_seed(3)
    n = 5000
    pred = torch.randn(n, generator=g)
    target = torch.randn(n, generator=g)
    mask = (torch.rand(n, generator=g) > 0.3).to(torch.float32)
    grad = torch.empty(n, device=DEV)
    parts = torch.zeros(64, device=DEV)
    bps.bps_warmnet_mse(pred.to(DEV), target.to(DEV), mask.to(DEV), n, grad, parts, 64)
    torch.cuda.synchronize()
    d = (pred - target) * mask
    assert abs(float(parts.sum()) - float((d * d).mean())) < 1e-5
    assert torch.allclose(grad.cpu(), 2 * d / n, atol=1e-7)
    w = torch.randn(300, generator=g)
    m = torch.zeros(300)
    v = torch.zeros(300)
    wd, md, vd = w.to(DEV), m.to(DEV), v.to(DEV)
    w16 = torch.empty(300, dtype=torch.bfloat16, device=DEV)
    for step in (1, 2, 3):
        gr = torch.randn(300, generator=g)
        bps.bps_warmnet_adam(wd, md, vd, gr.to(DEV), 300, 0.01, 0.9, 0.999, 1e-8, step, w16)
        m = 0.9 * m + 0.1 * gr
        v = 0.999 * v + 0.001 * gr * gr
        w = w - 0.01 * (m / (1 - 0.9 ** step)) / ((v / (1 - 0.999 ** step)).sqrt() + 1e-8)
    torch.cuda.synchronize()
    assert torch.allclose(wd.cpu(), w, atol=1e-5)
    assert torch.equal(w16.cpu(), wd.cpu().to(torch.bfloat16))


def test_features_and_messages():
    rng = np.random.default_rng(4)
    H, W, D = 6, 9, 20
    cost = rng.integers(0, 900, (H, W, D)).astype(np.int32)
    feat = torch.empty(((D + 7) // 8, H, W), dtype=torch.bfloat16, device=DEV)
    bps.bps_warmnet_features(torch.from_numpy(cost).to(DEV), H, W, D, 1 / 64, feat)
    mn = cost.min(axis=2)
    want = np.stack([cost[:, :, 8 * g: 8 * g + 8].min(axis=2) - mn for g in range((D + 7) // 8)]) / 64.0
    got = feat.cpu().to(torch.float32).numpy()
    assert np.allclose(got, want, rtol=2 ** -8, atol=1e-6)
    pred = rng.normal(8, 6, (4 * D, H, W)).astype(np.float32)
    init = torch.empty((4, H, W, D), dtype=torch.int32, device=DEV)
    bps.bps_warmnet_messages(torch.from_numpy(pred).to(DEV), H, W, D, 20, init)
    m = np.clip(np.rint(pred.reshape(4, D, H, W).transpose(0, 2, 3, 1)), 0, 20).astype(np.int32)
    m -= m.min(axis=3, keepdims=True)
    m[0, 0] = 0
    m[1, -1] = 0
    m[2, :, 0] = 0
    m[3, :, -1] = 0
    assert np.array_equal(init.cpu().numpy(), m)


def test_warm_started_solve_matches_oracle_and_training_reduces_loss():
    W, H, D, window = 120, 88, 16, 5
    feats, targets = warmstart.make_dataset(range(500, 532), W, H, D, window, 20, 10, 2, label_iters=20)
    net = warmstart.WarmNet(D, seed=0, device=DEV)
    losses = warmstart.train(net, feats, targets, epochs=6, batch=8, lr=3e-3)
    assert losses[-1] < 0.7 * losses[0]
    pair = synth.make_pair(777, W, H, D, 8, 3.0)
    with bps.Stereo(W, H, D, 4, bps.BPS_MSG_U8, device=DEV) as st:
        st.build_cost_volume(torch.from_numpy(pair.left).to(DEV), torch.from_numpy(pair.right).to(DEV), window, 20)
        init = net.predict_messages(st, 10, 2)
        st.bp_solve(5, 10, 2, init_msgs=init)
        msg = st.export_messages(0).cpu().numpy()
    c0 = oracle.quantise(oracle.ncc(pair.left, pair.right, D, window), 20)
    ref, _ = oracle.bp(c0, 4, 5, 10, 2, init_coarsest=init.cpu().numpy())
    assert np.array_equal(msg, ref)

"""The U-Net of the learned warm start on the GPU (BF16 tensor-core kernels)
against the FP64 oracle U-Net: forward output and every parameter gradient
on the same parameters and inputs, within a bound suited to BF16 activations
(relative L2 error per tensor, cosine similarity)."""
import numpy as np
import pytest

from oracle import unet as ounet

pytestmark = pytest.mark.gpu


def bf16_round(a):
    """Round to the nearest BF16 value (ties to even), as float64."""
    a32 = np.asarray(a, dtype=np.float32)
    u = a32.view(np.uint32).astype(np.uint64)
    u = (u + 0x7FFF + ((u >> 16) & 1)) & 0xFFFF0000
    return u.astype(np.uint32).view(np.float32).astype(np.float64)


@pytest.fixture(scope="module", params=[0, 1], ids=["tcgen05", "mma_sync"])
def setup(request):
    import torch
    import __graft_entry__
    __graft_entry__.build()
    import paper_1610_03918_gb300 as pg
    rng = np.random.default_rng(3)
    p = ounet.init_params(5)
    for n in p:
        if n.endswith(".b"):
            p[n] = rng.standard_normal(p[n].shape) * 0.05
    for n in p:                          # the GPU computes with BF16 weights
        if not n.endswith(".b"):
            p[n] = bf16_round(p[n])
    B, H, W = 2, 32, 24
    x = bf16_round(rng.standard_normal((B, H, W, 2)))
    t = rng.standard_normal((B, H, W))
    net = pg.Unet(B, H, W)
    net.set_conv_impl(request.param)
    net.set_params(ounet.flat(p).astype(np.float32))
    xd = torch.tensor(x, dtype=torch.float32, device="cuda")
    td = torch.tensor(t, dtype=torch.float32, device="cuda")
    yield p, x, t, net, xd, td
    net.close()


def test_unet_forward_matches_oracle(setup):
    p, x, t, net, xd, td = setup
    y = net.forward(xd).cpu().numpy()
    yo, _ = ounet.forward(p, x)
    rel = np.linalg.norm(y - yo) / np.linalg.norm(yo)
    assert rel < 2e-2, rel


def _compare(g, go):
    G = ounet.unflat(g.astype(np.float64))
    out = {}
    for name, _ in ounet.layer_shapes():
        a, b = G[name].ravel(), go[name].ravel()
        nb = np.linalg.norm(b)
        out[name] = (np.linalg.norm(a - b) / max(nb, 1e-30),
                     float(a @ b / max(np.linalg.norm(a) * nb, 1e-30)))
    return out


def test_unet_gradients_match_bf16_emulating_oracle(setup):
    # The oracle rounding to BF16 wherever the GPU stores a BF16 tensor.  What
    # remains is accumulation order, to which this small random network is
    # very sensitive: perturbing every value by 1e-7 before its BF16 rounding
    # moves the oracle's own bottleneck gradients by 13%, the last layers by
    # 0.1%.  The bound follows that spread.
    p, x, t, net, xd, td = setup
    loss, g = net.gradients(xd, td)
    lo, go = ounet.loss_and_grads(p, x, t, q=bf16_round)
    assert loss == pytest.approx(lo, rel=1e-3)
    res = _compare(g, go)
    for name, (rel, cos) in res.items():
        assert rel < 0.15 and cos > 0.995, (name, rel, cos)
    for name in ("head.W", "head.b", "dec0b.W", "dec0b.b"):
        assert res[name][0] < 1e-2, (name, res[name])


def test_unet_gradients_match_fp64_oracle(setup):
    # against plain FP64 the BF16 roundings compound with depth: the bottleneck
    # gradients see about ten roundings of cancelling sums
    p, x, t, net, xd, td = setup
    loss, g = net.gradients(xd, td)
    lo, go = ounet.loss_and_grads(p, x, t)
    assert loss == pytest.approx(lo, rel=2e-2)
    for name, (rel, cos) in _compare(g, go).items():
        assert rel < 0.2 and cos > 0.99, (name, rel, cos)


def test_unet_training_reduces_loss(setup):
    p, x, t, net, xd, td = setup
    l0, _ = net.gradients(xd, td)
    for _ in range(30):
        net.train_step(xd, td, 1e-3)
    l1, _ = net.gradients(xd, td)
    assert l1 < 0.7 * l0, (l0, l1)


def test_unet_forward_every_layer_on_tensor_cores():
    # 64 x 64: every level is at least 8 wide, so all fourteen 3x3
    # convolutions (the first with its 9 taps x 2 channels packed into one K
    # row of 32) and all three transposed convolutions run on tcgen05;
    # against the BF16-emulating oracle and against the mma.sync network
    import torch
    import paper_1610_03918_gb300 as pg
    rng = np.random.default_rng(8)
    p = ounet.init_params(7)
    for n in p:
        p[n] = bf16_round(p[n]) if not n.endswith(".b") else rng.standard_normal(p[n].shape) * 0.05
    B, H, W = 1, 64, 64
    x = bf16_round(rng.standard_normal((B, H, W, 2)))
    xd = torch.tensor(x, dtype=torch.float32, device="cuda")
    ys = []
    for impl in (0, 1):
        net = pg.Unet(B, H, W)
        net.set_conv_impl(impl)
        net.set_params(ounet.flat(p).astype(np.float32))
        ys.append(net.forward(xd).cpu().numpy())
        assert net.status() == pg.PIC_OK
        net.close()
    yo, _ = ounet.forward(p, x, q=bf16_round)
    for y in ys:
        assert np.linalg.norm(y - yo) / np.linalg.norm(yo) < 1e-2
    assert np.linalg.norm(ys[0] - ys[1]) / np.linalg.norm(ys[1]) < 1e-2


def test_unet_gradients_every_level_on_tensor_cores():
    # 72 x 80: every level is at least 8 wide and none a whole number of
    # tiles, so every 3x3 convolution, its data gradient and the transposed
    # convolutions' data gradients (36 x 40, 18 x 20, 9 x 10 inputs) run on
    # tcgen05 with ragged tiles; against the BF16-emulating oracle, with the
    # bounds of the smaller network above, and against the mma.sync network
    import torch
    import paper_1610_03918_gb300 as pg
    rng = np.random.default_rng(11)
    p = ounet.init_params(9)
    for n in p:
        p[n] = bf16_round(p[n]) if not n.endswith(".b") else rng.standard_normal(p[n].shape) * 0.05
    B, H, W = 1, 72, 80
    x = bf16_round(rng.standard_normal((B, H, W, 2)))
    t = rng.standard_normal((B, H, W))
    xd = torch.tensor(x, dtype=torch.float32, device="cuda")
    td = torch.tensor(t, dtype=torch.float32, device="cuda")
    out = []
    for impl in (0, 1):
        net = pg.Unet(B, H, W)
        net.set_conv_impl(impl)
        net.set_params(ounet.flat(p).astype(np.float32))
        out.append(net.gradients(xd, td))
        assert net.status() == pg.PIC_OK
        net.close()
    lo, go = ounet.loss_and_grads(p, x, t, q=bf16_round)
    for loss, g in out:
        assert loss == pytest.approx(lo, rel=1e-3)
        for name, (rel, cos) in _compare(g, go).items():
            assert rel < 0.15 and cos > 0.995, (name, rel, cos)
    G0, G1 = ounet.unflat(out[0][1].astype(np.float64)), ounet.unflat(out[1][1].astype(np.float64))
    for name in ("up0.W", "up1.W", "up2.W", "enc1a.W", "enc2a.W", "enc3a.W"):
        a, b = G0[name].ravel(), G1[name].ravel()
        assert np.linalg.norm(a - b) / np.linalg.norm(b) < 0.15, name

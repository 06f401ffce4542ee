"""Pins of the oracle U-Net (learned warm start): primitives against library
routines and hand-worked values, and the full backward pass against central
finite differences of the forward pass (CPU)."""
import numpy as np
import pytest
import scipy.signal as ss

from oracle import unet


def test_conv3x3_matches_scipy_correlate():
    rng = np.random.default_rng(0)
    x = rng.standard_normal((2, 7, 9, 3))
    W = rng.standard_normal((4, 3, 3, 3))
    b = rng.standard_normal(4)
    y = unet.conv3x3(x, W, b)
    for bi in range(2):
        for co in range(4):
            ref = b[co] + sum(ss.correlate(x[bi, :, :, ci], W[co, :, :, ci], mode="same")
                              for ci in range(3))
            np.testing.assert_allclose(y[bi, :, :, co], ref, atol=1e-12)


def test_pool_and_upconv_by_hand():
    x = np.arange(16.0).reshape(1, 4, 4, 1)
    p = unet.avgpool2(x)
    assert p[0, :, :, 0].tolist() == [[2.5, 4.5], [10.5, 12.5]]
    W = np.zeros((2, 2, 1, 1))
    W[0, 1, 0, 0] = 3.0
    u = unet.upconv2x2(np.ones((1, 1, 1, 1)), W, np.array([0.5]))
    assert u[0, :, :, 0].tolist() == [[0.5, 3.5], [0.5, 0.5]]


@pytest.mark.parametrize("seed", [1, 2])
def test_backward_matches_finite_differences(seed):
    rng = np.random.default_rng(seed)
    p = unet.init_params(seed)
    # biases nonzero so that every path is exercised
    for n in p:
        if n.endswith(".b"):
            p[n] = rng.standard_normal(p[n].shape) * 0.1
    x = rng.standard_normal((1, 16, 8, 2))
    t = rng.standard_normal((1, 16, 8))
    loss, g = unet.loss_and_grads(p, x, t)
    eps = 1e-6
    for name, shp in unet.layer_shapes():
        for _ in range(3):
            idx = tuple(int(rng.integers(0, d)) for d in shp)
            q = {k: v.copy() for k, v in p.items()}
            q[name][idx] += eps
            lp = unet.loss_and_grads(q, x, t)[0]
            q[name][idx] -= 2 * eps
            lm = unet.loss_and_grads(q, x, t)[0]
            fd = (lp - lm) / (2 * eps)
            an = g[name][idx]
            assert abs(fd - an) <= 1e-6 * max(1.0, abs(fd)) + 1e-9, (name, idx, fd, an)

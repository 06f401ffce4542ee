"""FP64 U-Net of the learned Poisson warm start (oracle; test infrastructure).

The paper solves Eq. (5) by Gauss-Seidel / Jacobi and names a faster field
solver as future work (Sec. II, Sec. IV); the learned warm start is this
build's extension: an initial guess phi_0 = phi_L + s * U(rho / s, mask) for
the multigrid-preconditioned CG, which then always finishes the solve.

U is a four-level U-Net, restated plainly (NHWC arrays, float64):

  encoder  level l = 0..3, channels C_l = 32, 64, 128, 256:
           two 3x3 convolutions (zero padding), each followed by ReLU;
           a 2x2 average pool between levels
  decoder  level l = 2, 1, 0: a 2x2 stride-2 transposed convolution
           C_{l+1} -> C_l, concatenated with the encoder output of level l
           (upsampled channels first), then two 3x3 convolutions + ReLU
  head     a 1x1 convolution C_0 -> 1 (no activation)

Loss: mean squared error over the pixels.

`forward` and `loss_and_grads` take an optional rounding function q applied
to every tensor a low-precision implementation would store (layer outputs,
pooled and upsampled tensors, and the activation gradients passed between
layers); the default is the identity, i.e. plain FP64.

Pinned by (tests/test_oracle_unet.py): the 3x3 convolution against
scipy.signal.correlate, the pooling and the transposed convolution by hand,
and every parameter gradient of the backward pass against central finite
differences of the forward pass.
"""
from __future__ import annotations

import numpy as np

CHANNELS = (32, 64, 128, 256)


def conv3x3(x, W, b):
    """x [B,H,W,Ci], W [Co,3,3,Ci], b [Co] -> [B,H,W,Co]; zero padding 1."""
    B, H, Wd, Ci = x.shape
    xp = np.zeros((B, H + 2, Wd + 2, Ci))
    xp[:, 1:-1, 1:-1] = x
    out = np.broadcast_to(b, (B, H, Wd, W.shape[0])).copy()
    for di in range(3):
        for dj in range(3):
            out += np.einsum("bhwc,oc->bhwo", xp[:, di:di + H, dj:dj + Wd], W[:, di, dj, :])
    return out


def conv3x3_backward(x, W, dy):
    """Gradients of conv3x3 w.r.t. x, W, b."""
    B, H, Wd, Ci = x.shape
    xp = np.zeros((B, H + 2, Wd + 2, Ci))
    xp[:, 1:-1, 1:-1] = x
    dxp = np.zeros_like(xp)
    dW = np.zeros_like(W)
    for di in range(3):
        for dj in range(3):
            dW[:, di, dj, :] = np.einsum("bhwo,bhwc->oc", dy, xp[:, di:di + H, dj:dj + Wd])
            dxp[:, di:di + H, dj:dj + Wd] += np.einsum("bhwo,oc->bhwc", dy, W[:, di, dj, :])
    return dxp[:, 1:-1, 1:-1], dW, dy.sum(axis=(0, 1, 2))


def avgpool2(x):
    B, H, Wd, C = x.shape
    return x.reshape(B, H // 2, 2, Wd // 2, 2, C).mean(axis=(2, 4))


def avgpool2_backward(dy):
    return np.repeat(np.repeat(dy, 2, axis=1), 2, axis=2) * 0.25


def upconv2x2(x, W, b):
    """x [B,h,w,Ci], W [2,2,Ci,Co], b [Co] -> [B,2h,2w,Co]."""
    B, h, w, Ci = x.shape
    Co = W.shape[3]
    out = np.empty((B, 2 * h, 2 * w, Co))
    for a in range(2):
        for c in range(2):
            out[:, a::2, c::2] = np.einsum("bhwi,io->bhwo", x, W[a, c]) + b
    return out


def upconv2x2_backward(x, W, dy):
    dx = np.zeros_like(x)
    dW = np.zeros_like(W)
    for a in range(2):
        for c in range(2):
            g = dy[:, a::2, c::2]
            dx += np.einsum("bhwo,io->bhwi", g, W[a, c])
            dW[a, c] = np.einsum("bhwi,bhwo->io", x, g)
    return dx, dW, dy.sum(axis=(0, 1, 2))


def layer_shapes(cin=2):
    """Parameter shapes in a fixed order (also the order of the flat vector)."""
    C = CHANNELS
    shapes = []
    prev = cin
    for l in range(4):
        shapes += [(f"enc{l}a.W", (C[l], 3, 3, prev)), (f"enc{l}a.b", (C[l],)),
                   (f"enc{l}b.W", (C[l], 3, 3, C[l])), (f"enc{l}b.b", (C[l],))]
        prev = C[l]
    for l in (2, 1, 0):
        shapes += [(f"up{l}.W", (2, 2, C[l + 1], C[l])), (f"up{l}.b", (C[l],)),
                   (f"dec{l}a.W", (C[l], 3, 3, 2 * C[l])), (f"dec{l}a.b", (C[l],)),
                   (f"dec{l}b.W", (C[l], 3, 3, C[l])), (f"dec{l}b.b", (C[l],))]
    shapes += [("head.W", (C[0],)), ("head.b", (1,))]
    return shapes


def init_params(seed=0, cin=2):
    """He-normal weights, zero biases (seeded)."""
    rng = np.random.default_rng(seed)
    p = {}
    for name, shp in layer_shapes(cin):
        if name.endswith(".b"):
            p[name] = np.zeros(shp)
        elif name.startswith("up"):
            p[name] = rng.standard_normal(shp) * np.sqrt(2.0 / shp[2])
        elif name == "head.W":
            p[name] = rng.standard_normal(shp) * np.sqrt(1.0 / shp[0])
        else:
            p[name] = rng.standard_normal(shp) * np.sqrt(2.0 / (9 * shp[3]))
    return p


def _ident(a):
    return a


def forward(p, x, q=None):
    """Returns (y [B,H,W], cache)."""
    q = q or _ident
    cache = {"x": x}
    h = x
    skips = []
    for l in range(4):
        for s in "ab":
            pre = conv3x3(h, p[f"enc{l}{s}.W"], p[f"enc{l}{s}.b"])
            cache[f"enc{l}{s}.in"] = h
            cache[f"enc{l}{s}.pre"] = pre
            h = q(np.maximum(pre, 0.0))
        skips.append(h)
        if l < 3:
            h = q(avgpool2(h))
    for l in (2, 1, 0):
        cache[f"up{l}.in"] = h
        u = q(upconv2x2(h, p[f"up{l}.W"], p[f"up{l}.b"]))
        h = np.concatenate([u, skips[l]], axis=3)
        for s in "ab":
            pre = conv3x3(h, p[f"dec{l}{s}.W"], p[f"dec{l}{s}.b"])
            cache[f"dec{l}{s}.in"] = h
            cache[f"dec{l}{s}.pre"] = pre
            h = q(np.maximum(pre, 0.0))
    cache["head.in"] = h
    y = np.einsum("bhwc,c->bhw", h, p["head.W"]) + p["head.b"][0]
    return y, cache


def loss_and_grads(p, x, t, q=None):
    """MSE loss over pixels and the gradient of every parameter (manual
    backward pass through the layers of forward, last layer first)."""
    q = q or _ident
    y, cache = forward(p, x, q)
    n = y.size
    loss = float(np.sum((y - t) ** 2) / n)
    dy = 2.0 * (y - t) / n
    g = {}
    g["head.W"] = np.einsum("bhw,bhwc->c", dy, cache["head.in"])
    g["head.b"] = np.array([dy.sum()])
    dh = q(dy[..., None] * p["head.W"])
    C = CHANNELS
    dskip = [None] * 3

    def conv_block_back(prefix, dh, last=False):
        for s in "ba":
            dpre = dh * (cache[f"{prefix}{s}.pre"] > 0)
            dh, g[f"{prefix}{s}.W"], g[f"{prefix}{s}.b"] = conv3x3_backward(
                cache[f"{prefix}{s}.in"], p[f"{prefix}{s}.W"], dpre)
            dh = q(dh)
        return dh

    for l in (0, 1, 2):                       # decoder, from the output upwards
        dh = conv_block_back(f"dec{l}", dh)
        du, dskip[l] = dh[..., :C[l]], dh[..., C[l]:]
        dh, g[f"up{l}.W"], g[f"up{l}.b"] = upconv2x2_backward(cache[f"up{l}.in"], p[f"up{l}.W"], du)
        dh = q(dh)
        # dh: gradient at the input of up{l} = output of decoder level l+1
        # (the bottleneck for l = 2)
    dh = conv_block_back("enc3", dh)          # bottleneck
    for l in (2, 1, 0):                       # encoder, back down
        dh = q(avgpool2_backward(dh) + dskip[l])
        dh = conv_block_back(f"enc{l}", dh)
    return loss, g


def flat(params_or_grads, cin=2):
    return np.concatenate([params_or_grads[n].ravel() for n, _ in layer_shapes(cin)])


def unflat(v, cin=2):
    out, k = {}, 0
    for n, shp in layer_shapes(cin):
        m = int(np.prod(shp))
        out[n] = v[k:k + m].reshape(shp)
        k += m
    return out

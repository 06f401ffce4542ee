"""The U-Net's elementwise layers, one at a time, through their C-ABI entry
points against the oracle (oracle/unet.py) on BF16-rounded inputs: the 2x2
average pool, the 1x1 head and its backward, and the ReLU's backward with
the bias gradient (with and without the average pool's gradient joining it).
BF16 outputs are the BF16 rounding of the exact value (at most one BF16
unit off, in a rare double rounding); FP32 sums agree to their summation
order.  Needs a GB300."""
import ctypes

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


def within_one_bf16_unit(got, ref):
    """got equals the BF16 rounding of ref, or (rarely) a neighbour of it."""
    r = bf16_round(ref)
    ulp = np.maximum(np.abs(r), 1e-30) * 2.0 ** -7
    return np.all(np.abs(got - r) <= ulp) and np.mean(got == r) >= 0.999


@pytest.fixture(scope="module")
def env():
    import torch
    import __graft_entry__
    __graft_entry__.build()
    import paper_1610_03918_gb300 as pg
    lib = pg.load_library()
    P, I, L = ctypes.c_void_p, ctypes.c_int32, ctypes.c_int64
    lib.pic_avgpool2_bf16.argtypes = [I, I, I, P, I, I, I, P, P]
    lib.pic_head_bf16.argtypes = [L, P, P, P, P, P]
    lib.pic_head_back_bf16.argtypes = [L, P, P, P, P, P, P, P]
    lib.pic_relu_back_bf16.argtypes = [I, I, I, P, I, I, P, I, I, P, P, I, P, P]
    return pg, lib, torch


def _dev(torch, a, dtype):
    return torch.tensor(np.ascontiguousarray(a, dtype=np.float32), device="cuda").to(dtype).contiguous()


def _s(torch):
    return torch.cuda.current_stream().cuda_stream


@pytest.mark.parametrize("B,H,W,C,in_cs,in_off", [(2, 64, 96, 32, 32, 0), (1, 36, 20, 64, 128, 64),
                                                  (1, 10, 6, 256, 256, 0)])
def test_avgpool2_matches_oracle(env, B, H, W, C, in_cs, in_off):
    pg, lib, torch = env
    rng = np.random.default_rng(H + W + C)
    x = bf16_round(rng.standard_normal((B, H, W, in_cs)))
    xd = _dev(torch, x, torch.bfloat16)
    od = torch.full((B, H // 2, W // 2, C), 7.0, dtype=torch.bfloat16, device="cuda")
    st = lib.pic_avgpool2_bf16(B, H, W, xd.data_ptr(), in_cs, in_off, C, od.data_ptr(), _s(torch))
    assert st == pg.PIC_OK
    got = od.float().cpu().numpy().astype(np.float64)
    ref = ounet.avgpool2(x[..., in_off:in_off + C])
    assert within_one_bf16_unit(got, ref)


def test_head_and_its_backward_match_oracle(env):
    pg, lib, torch = env
    rng = np.random.default_rng(21)
    B, H, W = 2, 40, 56
    n = B * H * W
    h = bf16_round(rng.standard_normal((B, H, W, 32)))
    w = rng.standard_normal(32) * 0.2
    b = rng.standard_normal(1)
    dy = rng.standard_normal((B, H, W)).astype(np.float32).astype(np.float64)
    hd = _dev(torch, h, torch.bfloat16)
    wd, bd = _dev(torch, w, torch.float32), _dev(torch, b, torch.float32)
    yd = torch.zeros(n, dtype=torch.float32, device="cuda")
    assert lib.pic_head_bf16(n, hd.data_ptr(), wd.data_ptr(), bd.data_ptr(), yd.data_ptr(), _s(torch)) == pg.PIC_OK
    y_ref = np.einsum("bhwc,c->bhw", h, w.astype(np.float32).astype(np.float64)) + \
        np.float64(np.float32(b[0]))
    y = yd.cpu().numpy().astype(np.float64).reshape(B, H, W)
    assert np.all(np.abs(y - y_ref) <= 1e-5 * (1 + np.abs(y_ref)))
    # backward
    dyd = _dev(torch, dy, torch.float32)
    ghd = torch.full((n, 32), 7.0, dtype=torch.bfloat16, device="cuda")
    dwd = torch.zeros(32, dtype=torch.float32, device="cuda")
    dbd = torch.full((1,), 0.5, dtype=torch.float32, device="cuda")
    st = lib.pic_head_back_bf16(n, dyd.data_ptr(), hd.data_ptr(), wd.data_ptr(), ghd.data_ptr(), dwd.data_ptr(),
                                dbd.data_ptr(), _s(torch))
    assert st == pg.PIC_OK
    w32 = w.astype(np.float32).astype(np.float64)
    gh_ref = (dy.reshape(n)[:, None] * w32[None, :]).astype(np.float32)   # the FP32 product, then BF16
    assert within_one_bf16_unit(ghd.float().cpu().numpy().astype(np.float64), gh_ref.astype(np.float64))
    dw_ref = np.einsum("bhw,bhwc->c", dy, h)
    dw = dwd.cpu().numpy().astype(np.float64)
    assert np.all(np.abs(dw - dw_ref) <= 1e-5 * np.abs(dw_ref).max())
    assert abs(float(dbd.cpu()[0]) - (0.5 + dy.sum())) <= 1e-5 * np.abs(dy).sum()


@pytest.mark.parametrize("pool", [False, True])
@pytest.mark.parametrize("B,H,W,C,g_cs,g_off,y_cs,y_off", [(2, 32, 48, 32, 64, 32, 64, 32),
                                                           (1, 18, 20, 64, 64, 0, 128, 64),
                                                           (1, 6, 10, 256, 256, 0, 256, 0)])
def test_relu_backward_matches_oracle(env, pool, B, H, W, C, g_cs, g_off, y_cs, y_off):
    pg, lib, torch = env
    rng = np.random.default_rng(C + H + int(pool))
    g = bf16_round(rng.standard_normal((B, H, W, g_cs)))
    y = bf16_round(np.maximum(rng.standard_normal((B, H, W, y_cs)), 0.0))   # ReLU outputs: zeros and positives
    gp = bf16_round(rng.standard_normal((B, H // 2, W // 2, C)))
    gd, yd = _dev(torch, g, torch.bfloat16), _dev(torch, y, torch.bfloat16)
    gpd = _dev(torch, gp, torch.bfloat16) if pool else None
    dd = torch.full((B, H, W, C), 7.0, dtype=torch.bfloat16, device="cuda")
    dbd = torch.zeros(C, dtype=torch.float32, device="cuda")
    st = lib.pic_relu_back_bf16(B, H, W, gd.data_ptr(), g_cs, g_off, yd.data_ptr(), y_cs, y_off,
                                gpd.data_ptr() if pool else None, dd.data_ptr(), C, dbd.data_ptr(), _s(torch))
    assert st == pg.PIC_OK
    t = g[..., g_off:g_off + C]
    if pool:
        t = bf16_round(t + ounet.avgpool2_backward(gp))   # the joined gradient, stored in BF16
    ref = np.where(y[..., y_off:y_off + C] > 0, t, 0.0)
    got = dd.float().cpu().numpy().astype(np.float64)
    assert np.array_equal(got, ref)
    db_ref = ref.sum(axis=(0, 1, 2))
    assert np.all(np.abs(dbd.cpu().numpy() - db_ref) <= 1e-5 * np.abs(ref).sum(axis=(0, 1, 2)).max())


def test_layer_entries_refuse_bad_shapes(env):
    pg, lib, torch = env
    x = torch.zeros((1, 8, 8, 24), dtype=torch.bfloat16, device="cuda")
    o = torch.zeros((1, 4, 4, 24), dtype=torch.bfloat16, device="cuda")
    assert lib.pic_avgpool2_bf16(1, 7, 8, x.data_ptr(), 24, 0, 24, o.data_ptr(), _s(torch)) == pg.PIC_EINVAL
    db = torch.zeros(24, dtype=torch.float32, device="cuda")
    assert lib.pic_relu_back_bf16(1, 8, 8, x.data_ptr(), 24, 0, x.data_ptr(), 24, 0, None, x.data_ptr(), 24,
                                  db.data_ptr(), _s(torch)) == pg.PIC_EINVAL     # C 24

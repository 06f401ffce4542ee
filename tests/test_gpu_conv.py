"""Single 3x3 convolution layers of the warm-start U-Net (pic_conv3x3_bf16)
on the tcgen05 tensor-core kernel and on the mma.sync kernel, against the
FP64 oracle convolution on the same BF16-rounded inputs and weights.  Here
only the output's BF16 rounding and FP32 accumulation order separate the
two sides, so the bounds are tight (relative L2 error <= 4e-3, cosine >=
0.99999 per tensor).  Needs a GB300."""
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


@pytest.fixture(scope="module")
def lib():
    import __graft_entry__
    __graft_entry__.build()
    import paper_1610_03918_gb300 as pg
    return pg


def _dev(a, torch, dtype):
    return torch.tensor(np.ascontiguousarray(a, dtype=np.float32), device="cuda").to(dtype).contiguous()


def run_conv(pg, impl, x_full, in_off, cin, Wt, bias, relu, out_cs, out_off):
    """x_full [B,H,W,in_cs] (BF16 values), Wt [co,3,3,ci]; returns (output
    buffer [B,H,W,out_cs] as float64, status)."""
    import ctypes
    import torch
    B, H, W, in_cs = x_full.shape
    cout = Wt.shape[0]
    xd = _dev(x_full, torch, torch.bfloat16)
    wd = _dev(Wt.reshape(cout, 9, cin), torch, torch.bfloat16)
    bd = _dev(bias, torch, torch.float32) if bias is not None else None
    sentinel = 7.0
    od = torch.full((B, H, W, out_cs), sentinel, dtype=torch.bfloat16, device="cuda")
    lib = pg.load_library()
    f = lib.pic_conv3x3_bf16
    f.restype = ctypes.c_int
    P = ctypes.c_void_p
    f.argtypes = [ctypes.c_int32] * 4 + [P, ctypes.c_int32, ctypes.c_int32, ctypes.c_int32, P, P,
                                          ctypes.c_int32, P, ctypes.c_int32, ctypes.c_int32,
                                          ctypes.c_int32, P]
    st = f(impl, B, H, W, xd.data_ptr(), in_cs, in_off, cin, wd.data_ptr(),
           bd.data_ptr() if bd is not None else None, int(relu), od.data_ptr(), out_cs, out_off, cout,
           torch.cuda.current_stream().cuda_stream)
    return od.float().cpu().numpy().astype(np.float64), st


CASES = [
    # B, H, W, cin, cout, in_cs, in_off, out_cs, out_off, relu    (first-layer shape, KB = 16)
    (1, 40, 256, 16, 32, 16, 0, 32, 0, True),
    # concatenation slice as input, W = 64 (tiles of 2 rows), ragged H, KB = 32
    (2, 33, 64, 32, 32, 64, 32, 32, 0, True),
    # W = 24 (16-wide tiles: ragged in both directions), KB = 64
    (1, 18, 24, 64, 64, 64, 0, 128, 64, True),
    # decoder shape into an output slice, no activation
    (1, 17, 40, 256, 128, 256, 0, 256, 128, False),
    # N = 256 (bottleneck)
    (1, 9, 32, 128, 256, 128, 0, 256, 0, True),
    # halo loads (images at least 128 wide, up to 64 columns): W = 200 (the
    # second tile ragged), batch 2, an input channel slice, KB = 32
    (2, 7, 200, 32, 64, 64, 32, 64, 0, True),
    # halo loads into an output slice, KB = 64, no activation
    (1, 5, 128, 64, 32, 64, 0, 96, 32, False),
    # 128 columns on a wide image: the per-tap loads
    (1, 4, 256, 64, 128, 64, 0, 128, 0, True),
]


@pytest.mark.parametrize("case", CASES)
@pytest.mark.parametrize("impl", [0, 1])
def test_conv3x3_layer_matches_oracle(lib, case, impl):
    B, H, W, cin, cout, in_cs, in_off, out_cs, out_off, relu = case
    if impl == 1 and not ((cout == 32 and (cin == 16 or cin % 32 == 0)) or (cout % 64 == 0 and cin % 32 == 0)):
        pytest.skip("shape outside the mma.sync kernel")
    rng = np.random.default_rng(cin * 1000 + cout + H)
    x_full = bf16_round(rng.standard_normal((B, H, W, in_cs)))
    Wt = bf16_round(rng.standard_normal((cout, 3, 3, cin)) * np.sqrt(2.0 / (9 * cin)))
    bias = rng.standard_normal(cout) * 0.1
    out, st = run_conv(lib, impl, x_full, in_off, cin, Wt, bias, relu, out_cs, out_off)
    assert st == lib.PIC_OK, lib.pic_strerror(st)
    ref = ounet.conv3x3(x_full[..., in_off:in_off + cin], Wt, bias)
    if relu:
        ref = np.maximum(ref, 0.0)
    got = out[..., out_off:out_off + cout]
    rel = np.linalg.norm(got - ref) / np.linalg.norm(ref)
    cos = float((got * ref).sum() / (np.linalg.norm(got) * np.linalg.norm(ref)))
    assert rel <= 4e-3 and cos >= 0.99999, (rel, cos)
    # element-wise: the BF16 rounding of the exact value plus a little accumulation error
    assert np.all(np.abs(got - ref) <= 2.0 ** -8 * np.abs(ref) + 1e-3 * np.abs(ref).max())
    # channels outside the output slice are untouched
    rest = np.delete(out, np.s_[out_off:out_off + cout], axis=3)
    assert np.all(rest == 7.0)


def test_conv3x3_data_gradient_formulation(lib):
    # the U-Net's data gradient is the same kernel with the weights flipped in
    # space and transposed in channels: against the oracle's backward pass
    B, H, W, cin, cout = 1, 24, 64, 64, 128
    rng = np.random.default_rng(5)
    x = bf16_round(rng.standard_normal((B, H, W, cin)))
    Wt = bf16_round(rng.standard_normal((cout, 3, 3, cin)) * 0.05)
    dy = bf16_round(rng.standard_normal((B, H, W, cout)))
    dx_ref, _, _ = ounet.conv3x3_backward(x, Wt, dy)
    Wflip = np.ascontiguousarray(Wt[:, ::-1, ::-1, :].transpose(3, 1, 2, 0))   # [ci,3,3,co]
    for impl in (0, 1):
        out, st = run_conv(lib, impl, dy, 0, cout, Wflip, None, False, cin, 0)
        assert st == lib.PIC_OK
        rel = np.linalg.norm(out - dx_ref) / np.linalg.norm(dx_ref)
        assert rel <= 4e-3, (impl, rel)


def test_tensor_core_and_mma_sync_kernels_agree(lib):
    # the two kernels accumulate in FP32 in different orders; after the BF16
    # rounding of the output they agree to one BF16 unit
    B, H, W, cin, cout = 1, 32, 128, 64, 64
    rng = np.random.default_rng(9)
    x = bf16_round(rng.standard_normal((B, H, W, cin)))
    Wt = bf16_round(rng.standard_normal((cout, 3, 3, cin)) * 0.05)
    bias = rng.standard_normal(cout) * 0.1
    a, _ = run_conv(lib, 0, x, 0, cin, Wt, bias, True, cout, 0)
    b, _ = run_conv(lib, 1, x, 0, cin, Wt, bias, True, cout, 0)
    assert np.all(np.abs(a - b) <= 2.0 ** -7 * np.maximum(np.abs(a), np.abs(b)) + 1e-6)
    assert np.mean(a != b) < 0.05


def test_unsupported_shapes_are_refused(lib):
    import torch
    x = np.zeros((1, 8, 16, 24))
    Wt = np.zeros((32, 3, 3, 24))
    _, st = run_conv(lib, 0, x, 0, 24, Wt, None, True, 32, 0)      # cin 24: not a multiple of 16
    assert st == lib.PIC_EINVAL
    Wt = np.zeros((48, 3, 3, 16))
    _, st = run_conv(lib, 0, np.zeros((1, 8, 16, 16)), 0, 16, Wt, None, True, 48, 0)   # cout 48
    assert st == lib.PIC_EINVAL


def run_upback(pg, impl, gout_full, gout_off, cout, Wup, cin):
    """Data gradient of the 2x2 stride-2 transposed convolution through
    pic_upconv_back_bf16: gout_full [B,2H,2W,gout_cs] (BF16 values), Wup
    [2,2,cin,cout] (FP32); returns (gin [B,H,W,cin] as float64, status)."""
    import ctypes
    import torch
    B, H2, W2, gout_cs = gout_full.shape
    H, W = H2 // 2, W2 // 2
    gd = _dev(gout_full, torch, torch.bfloat16)
    wd = _dev(Wup, torch, torch.float32)
    od = torch.full((B, H, W, cin), 7.0, dtype=torch.bfloat16, device="cuda")
    lib = pg.load_library()
    f = lib.pic_upconv_back_bf16
    P, I = ctypes.c_void_p, ctypes.c_int32
    f.argtypes = [I, I, I, I, P, I, I, I, P, P, I, P]
    st = f(impl, B, H, W, gd.data_ptr(), gout_cs, gout_off, cout, wd.data_ptr(), od.data_ptr(), cin,
           torch.cuda.current_stream().cuda_stream)
    return od.float().cpu().numpy().astype(np.float64), st


UP_CASES = [
    # B, H, W (the layer's input), cin, cout, gout_cs, gout_off
    # the finest level's shape (gradient of the 64-channel concatenation's
    # first half), W = 20: 16-wide tiles, ragged; K = 32
    (1, 36, 20, 64, 32, 64, 0),
    # W = 130: 128-wide tiles, the second ragged; batch 2; K = 64
    (2, 9, 130, 128, 64, 128, 0),
    # the coarsest level's shape: 3 pixel tiles, the 256 columns in 4 blocks
    (1, 5, 64, 256, 128, 256, 0),
    # a channel slice at an offset, K = 16
    (1, 16, 32, 32, 16, 48, 16),
    # K = 48 (blocks of 16) from an offset slice, W = 8
    (1, 12, 8, 64, 48, 64, 8),
]


@pytest.mark.parametrize("case", UP_CASES)
@pytest.mark.parametrize("impl", [0, 1])
def test_upconv_data_gradient_matches_oracle(lib, case, impl):
    B, H, W, cin, cout, gout_cs, gout_off = case
    rng = np.random.default_rng(cin * 100 + cout + W)
    g_full = bf16_round(rng.standard_normal((B, 2 * H, 2 * W, gout_cs)))
    Wup = bf16_round(rng.standard_normal((2, 2, cin, cout)) / np.sqrt(cin))
    got, st = run_upback(lib, impl, g_full, gout_off, cout, Wup, cin)
    assert st == lib.PIC_OK, lib.pic_strerror(st)
    x0 = np.zeros((B, H, W, cin))
    ref, _, _ = ounet.upconv2x2_backward(x0, Wup, g_full[..., gout_off:gout_off + cout])
    rel = np.linalg.norm(got - ref) / np.linalg.norm(ref)
    cos = float((got * ref).sum() / (np.linalg.norm(got) * np.linalg.norm(ref)))
    assert rel <= 4e-3 and cos >= 0.99999, (rel, cos)
    assert np.all(np.abs(got - ref) <= 2.0 ** -8 * np.abs(ref) + 1e-3 * np.abs(ref).max())


def test_upconv_data_gradient_refuses_unsupported_shapes(lib):
    g = np.zeros((1, 16, 16, 64))
    _, st = run_upback(lib, 0, g, 0, 64, np.zeros((2, 2, 48, 64)), 48)     # 48 output channels
    assert st == lib.PIC_EINVAL
    _, st = run_upback(lib, 0, g, 4, 32, np.zeros((2, 2, 64, 32)), 64)     # offset not a multiple of 8
    assert st == lib.PIC_EINVAL
    _, st = run_upback(lib, 0, np.zeros((1, 8, 8, 64)), 0, 64, np.zeros((2, 2, 64, 64)), 64)   # W = 4
    assert st == lib.PIC_EINVAL


def run_wgrad(pg, impl, dpre, x_full, in_off, cin, prefill=0.0):
    """Weight gradient of a 3x3 convolution through pic_conv3x3_wgrad_bf16:
    dpre [B,H,W,cout], x_full [B,H,W,in_cs] (BF16 values); returns (dW
    [cout,3,3,cin] as float64 after adding into `prefill`, status)."""
    import ctypes
    import torch
    B, H, W, in_cs = x_full.shape
    cout = dpre.shape[3]
    dd = _dev(dpre, torch, torch.bfloat16)
    xd = _dev(x_full, torch, torch.bfloat16)
    wd = torch.full((cout, 9, cin), prefill, dtype=torch.float32, device="cuda")
    lib = pg.load_library()
    f = lib.pic_conv3x3_wgrad_bf16
    P, I = ctypes.c_void_p, ctypes.c_int32
    f.argtypes = [I, I, I, I, P, P, I, I, I, I, P, P]
    st = f(impl, B, H, W, dd.data_ptr(), xd.data_ptr(), in_cs, in_off, cin, cout, wd.data_ptr(),
           torch.cuda.current_stream().cuda_stream)
    return wd.cpu().numpy().astype(np.float64).reshape(cout, 3, 3, cin), st


WG_CASES = [
    # B, H, W, cin, cout, in_cs, in_off
    # the first layer's padded input (16 channels), 4 chunks of 64 pixels
    (1, 40, 256, 16, 32, 16, 0),
    # batch 2 (taps across the images' edge rows), W = 72 (second chunk 8
    # pixels), the skip half of a concatenation as input
    (2, 33, 72, 32, 32, 64, 32),
    # W = 24 < 64, 64 x 64 from an offset slice
    (1, 18, 24, 64, 64, 128, 64),
    # 4 x 2 channel blocks of 64
    (1, 17, 40, 256, 128, 256, 0),
    # 256 outputs (4 blocks), 2 input blocks
    (1, 9, 32, 128, 256, 128, 0),
    # 64 outputs from 32 inputs, W = 130 (3 chunks, the last 2 pixels)
    (1, 6, 130, 32, 64, 32, 0),
    # 32 outputs from 64 inputs
    (1, 5, 64, 64, 32, 64, 0),
]


@pytest.mark.parametrize("case", WG_CASES)
@pytest.mark.parametrize("impl", [0, 1])
def test_conv3x3_weight_gradient_matches_oracle(lib, case, impl):
    # BF16 x BF16 products are exact in FP32; only the FP32 sum over the
    # pixels (in the tensor core's and the atomics' order) separates the two
    # sides, far below the 1e-3 bound, while a wrong tap, shift or operand
    # moves whole rows of dW by O(1)
    B, H, W, cin, cout, in_cs, in_off = case
    rng = np.random.default_rng(cin * 7 + cout * 3 + W)
    x_full = bf16_round(rng.standard_normal((B, H, W, in_cs)))
    dpre = bf16_round(rng.standard_normal((B, H, W, cout)))
    got, st = run_wgrad(lib, impl, dpre, x_full, in_off, cin)
    assert st == lib.PIC_OK, lib.pic_strerror(st)
    _, ref, _ = ounet.conv3x3_backward(x_full[..., in_off:in_off + cin], np.zeros((cout, 3, 3, cin)), dpre)
    scale = np.abs(ref).max()
    rel = np.linalg.norm(got - ref) / np.linalg.norm(ref)
    assert rel <= 1e-4, rel
    assert np.all(np.abs(got - ref) <= 1e-3 * scale), np.abs(got - ref).max() / scale


def test_conv3x3_weight_gradient_adds_into_dw(lib):
    B, H, W, cin, cout = 1, 8, 16, 32, 32
    rng = np.random.default_rng(4)
    x = bf16_round(rng.standard_normal((B, H, W, cin)))
    d = bf16_round(rng.standard_normal((B, H, W, cout)))
    a, st = run_wgrad(lib, 0, d, x, 0, cin, prefill=0.0)
    assert st == lib.PIC_OK
    b, st = run_wgrad(lib, 0, d, x, 0, cin, prefill=1.5)
    assert st == lib.PIC_OK
    assert np.allclose(b - 1.5, a, rtol=0, atol=1e-5 * np.abs(a).max())


def test_conv3x3_weight_gradient_refuses_unsupported_shapes(lib):
    x = np.zeros((1, 8, 16, 48))
    d = np.zeros((1, 8, 16, 32))
    _, st = run_wgrad(lib, 0, d, x, 0, 48)                               # cin 48
    assert st == lib.PIC_EINVAL
    _, st = run_wgrad(lib, 0, np.zeros((1, 8, 16, 96)), x[..., :32], 0, 32)   # cout 96
    assert st == lib.PIC_EINVAL
    _, st = run_wgrad(lib, 0, d, x, 4, 32)                               # offset not a multiple of 8
    assert st == lib.PIC_EINVAL


def run_upwgrad(pg, impl, x, g_full, g_off, cout):
    """Weight and bias gradients of the 2x2 stride-2 transposed convolution
    through pic_upconv_wgrad_bf16: x [B,H,W,cin], g_full [B,2H,2W,g_cs] (BF16
    values); returns (dW [2,2,cin,cout], db [cout]) as float64, status."""
    import ctypes
    import torch
    B, H, W, cin = x.shape
    g_cs = g_full.shape[3]
    xd = _dev(x, torch, torch.bfloat16)
    gd = _dev(g_full, torch, torch.bfloat16)
    dw = torch.zeros((2, 2, cin, cout), dtype=torch.float32, device="cuda")
    db = torch.zeros((cout,), dtype=torch.float32, device="cuda")
    lib = pg.load_library()
    f = lib.pic_upconv_wgrad_bf16
    P, I = ctypes.c_void_p, ctypes.c_int32
    f.argtypes = [I, I, I, I, P, I, P, I, I, I, P, P, P]
    st = f(impl, B, H, W, xd.data_ptr(), cin, gd.data_ptr(), g_cs, g_off, cout, dw.data_ptr(), db.data_ptr(),
           torch.cuda.current_stream().cuda_stream)
    return dw.cpu().numpy().astype(np.float64), db.cpu().numpy().astype(np.float64), st


UPW_CASES = [
    # B, H, W (the layer's input), cin, cout, gout_cs, gout_off
    # the finest level's shape, batch 2, W = 40 < 64
    (2, 18, 40, 64, 32, 64, 0),
    # W = 130: three chunks of 64 input pixels, the last 2
    (1, 9, 130, 128, 64, 128, 0),
    # 2 output x 4 input channel blocks
    (1, 5, 64, 256, 128, 256, 0),
    # a channel slice of the gradient at an offset
    (1, 6, 16, 64, 32, 96, 32),
    # 256 outputs
    (1, 4, 8, 64, 256, 256, 0),
]


@pytest.mark.parametrize("case", UPW_CASES)
@pytest.mark.parametrize("impl", [0, 1])
def test_upconv_weight_gradient_matches_oracle(lib, case, impl):
    B, H, W, cin, cout, g_cs, g_off = case
    rng = np.random.default_rng(cin + cout * 5 + W)
    x = bf16_round(rng.standard_normal((B, H, W, cin)))
    g_full = bf16_round(rng.standard_normal((B, 2 * H, 2 * W, g_cs)))
    dw, db, st = run_upwgrad(lib, impl, x, g_full, g_off, cout)
    assert st == lib.PIC_OK, lib.pic_strerror(st)
    _, dw_ref, db_ref = ounet.upconv2x2_backward(x, np.zeros((2, 2, cin, cout)), g_full[..., g_off:g_off + cout])
    rel = np.linalg.norm(dw - dw_ref) / np.linalg.norm(dw_ref)
    assert rel <= 1e-4, rel
    assert np.all(np.abs(dw - dw_ref) <= 1e-3 * np.abs(dw_ref).max())
    assert np.all(np.abs(db - db_ref) <= 1e-3 * np.abs(db_ref).max() + 1e-4 * np.sqrt(4 * B * H * W))


def test_upconv_weight_gradient_refuses_unsupported_shapes(lib):
    x = np.zeros((1, 4, 8, 48))
    _, _, st = run_upwgrad(lib, 0, x, np.zeros((1, 8, 16, 32)), 0, 32)     # cin 48
    assert st == lib.PIC_EINVAL
    _, _, st = run_upwgrad(lib, 0, np.zeros((1, 4, 8, 64)), np.zeros((1, 8, 16, 96)), 0, 96)   # cout 96
    assert st == lib.PIC_EINVAL


def run_upconv(pg, impl, x, Wup, bias, out_cs, out_off):
    """The 2x2 stride-2 transposed convolution through pic_upconv_bf16: x
    [B,H,W,cin] (BF16 values), Wup [2,2,cin,cout], bias [cout]; returns (the
    output buffer [B,2H,2W,out_cs] as float64, status)."""
    import ctypes
    import torch
    B, H, W, cin = x.shape
    cout = Wup.shape[3]
    xd = _dev(x, torch, torch.bfloat16)
    wd = _dev(Wup, torch, torch.float32)
    bd = _dev(bias, torch, torch.float32)
    od = torch.full((B, 2 * H, 2 * W, out_cs), 7.0, dtype=torch.bfloat16, device="cuda")
    lib = pg.load_library()
    f = lib.pic_upconv_bf16
    P, I = ctypes.c_void_p, ctypes.c_int32
    f.argtypes = [I, I, I, I, P, I, P, P, P, I, I, I, P]
    st = f(impl, B, H, W, xd.data_ptr(), cin, wd.data_ptr(), bd.data_ptr(), od.data_ptr(), out_cs, out_off, cout,
           torch.cuda.current_stream().cuda_stream)
    return od.float().cpu().numpy().astype(np.float64), st


UPF_CASES = [
    # B, H, W (the layer's input), cin, cout, out_cs, out_off
    (2, 9, 20, 64, 32, 64, 0),       # the finest level into the first half of a concatenation
    (1, 5, 130, 128, 64, 128, 0),    # 128-wide tiles, the second ragged
    (1, 4, 64, 256, 128, 256, 0),    # 512 GEMM columns in two launches
    (1, 6, 16, 32, 16, 48, 16),      # an offset slice, cout 16
]


@pytest.mark.parametrize("case", UPF_CASES)
@pytest.mark.parametrize("impl", [0, 1])
def test_upconv_layer_matches_oracle(lib, case, impl):
    B, H, W, cin, cout, out_cs, out_off = case
    rng = np.random.default_rng(cin * 3 + cout + W)
    x = bf16_round(rng.standard_normal((B, H, W, cin)))
    Wup = bf16_round(rng.standard_normal((2, 2, cin, cout)) / np.sqrt(cin))
    bias = rng.standard_normal(cout) * 0.1
    out, st = run_upconv(lib, impl, x, Wup, bias, out_cs, out_off)
    assert st == lib.PIC_OK, lib.pic_strerror(st)
    ref = ounet.upconv2x2(x, Wup, bias)
    got = out[..., out_off:out_off + cout]
    rel = np.linalg.norm(got - ref) / np.linalg.norm(ref)
    cos = float((got * ref).sum() / (np.linalg.norm(got) * np.linalg.norm(ref)))
    assert rel <= 4e-3 and cos >= 0.99999, (rel, cos)
    assert np.all(np.abs(got - ref) <= 2.0 ** -8 * np.abs(ref) + 1e-3 * np.abs(ref).max())
    rest = np.delete(out, np.s_[out_off:out_off + cout], axis=3)
    assert np.all(rest == 7.0)

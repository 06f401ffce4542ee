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

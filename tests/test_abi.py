"""The C-ABI library builds, loads and exports every entry point that
include/*.h declares (CPU only: no compute call is made)."""
import ctypes
import glob
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_symbols():
    names = set()
    for h in glob.glob(os.path.join(ROOT, "include", "*.h")):
        text = open(h).read()
        text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
        for m in re.finditer(r"^\s*(?:const\s+)?[A-Za-z_][A-Za-z0-9_]*\s*\*?\s*(pic_[a-z0-9_]+)\s*\(",
                             text, flags=re.M):
            names.add(m.group(1))
    return names


@pytest.fixture(scope="module")
def lib():
    from paper_1610_03918_gb300 import build
    if not os.path.exists(build.lib_path()):
        build.build()
    return ctypes.CDLL(build.lib_path())


def test_header_declares_the_boundary():
    names = declared_symbols()
    for n in ("pic_init", "pic_load", "pic_step", "pic_diag", "pic_free", "pic_strerror"):
        assert n in names, names


def test_library_exports_every_declared_symbol(lib):
    for n in sorted(declared_symbols()):
        assert hasattr(lib, n), f"{n} declared in include/ but not exported"


def test_strerror_without_gpu(lib):
    lib.pic_strerror.restype = ctypes.c_char_p
    assert lib.pic_strerror(0) == b"ok"
    assert b"Poisson" in lib.pic_strerror(4)


def test_init_rejects_bad_config_without_touching_gpu(lib):
    import paper_1610_03918_gb300 as pg
    import synth
    cfg = pg.make_config(synth.periodic_square_64(nx=63))   # odd periodic size
    ctx = ctypes.c_void_p()
    assert pg.load_library().pic_init(ctypes.byref(cfg), ctypes.byref(ctx)) == pg.PIC_EINVAL
    cfg = pg.make_config(synth.small_trench())
    cfg.sort_every = -1                                       # 0 asks for a tuned interval
    assert pg.load_library().pic_init(ctypes.byref(cfg), ctypes.byref(ctx)) == pg.PIC_EINVAL
    cfg = pg.make_config(synth.small_trench())
    cfg.poisson_method = 2
    assert pg.load_library().pic_init(ctypes.byref(cfg), ctypes.byref(ctx)) == pg.PIC_EINVAL


def test_batch_init_rejects_a_tuned_sort_interval_without_gpu(lib):
    import paper_1610_03918_gb300 as pg
    import synth
    with pytest.raises(pg.PicError) as e:
        pg.Batch([synth.small_trench(sort_every=0)], torch_memory=False)
    assert e.value.code == pg.PIC_EINVAL


def test_batch_init_rejects_mixed_sort_schedules_without_gpu(lib):
    import paper_1610_03918_gb300 as pg
    import synth
    with pytest.raises(pg.PicError) as e:
        pg.Batch([synth.small_trench(sort_every=8), synth.small_trench(sort_every=4)],
                 torch_memory=False)
    assert e.value.code == pg.PIC_EINVAL


def test_init_rejects_bad_recycling_source_without_gpu(lib):
    import paper_1610_03918_gb300 as pg
    import synth
    ctx = ctypes.c_void_p()
    for x0, x1 in ((10, 5), (-1, 5), (0, 60)):     # empty, negative, into the electrode
        w = synth.small_trench(nx=64, ny=32, depth=16).replace(recycle=True, source_x0=x0,
                                                                 source_x1=x1)
        cfg = pg.make_config(w)
        assert pg.load_library().pic_init(ctypes.byref(cfg), ctypes.byref(ctx)) == pg.PIC_EINVAL
    cfg = pg.make_config(synth.small_trench().replace(phi_rf_amp=float("nan"), omega_rf=0.1))
    assert pg.load_library().pic_init(ctypes.byref(cfg), ctypes.byref(ctx)) == pg.PIC_EINVAL


def test_layer_entries_reject_bad_arguments_without_gpu(lib):
    # argument checks come before any CUDA call: null pointers, empty or
    # inconsistent shapes and unknown implementations are refused on the host
    import paper_1610_03918_gb300 as pg
    L = pg.load_library()
    P, I, Q = ctypes.c_void_p, ctypes.c_int32, ctypes.c_int64
    fake = ctypes.c_void_p(16)                 # never dereferenced: the call is refused first
    L.pic_conv3x3_wgrad_bf16.argtypes = [I, I, I, I, P, P, I, I, I, I, P, P]
    assert L.pic_conv3x3_wgrad_bf16(0, 1, 8, 8, None, fake, 32, 0, 32, 32, fake, None) == pg.PIC_EINVAL
    assert L.pic_conv3x3_wgrad_bf16(2, 1, 8, 8, fake, fake, 32, 0, 32, 32, fake, None) == pg.PIC_EINVAL
    assert L.pic_conv3x3_wgrad_bf16(0, 1, 8, 8, fake, fake, 32, 8, 32, 32, fake, None) == pg.PIC_EINVAL
    L.pic_upconv_back_bf16.argtypes = [I, I, I, I, P, I, I, I, P, P, I, P]
    assert L.pic_upconv_back_bf16(0, 0, 8, 8, fake, 64, 0, 32, fake, fake, 64, None) == pg.PIC_EINVAL
    assert L.pic_upconv_back_bf16(0, 1, 8, 8, fake, 32, 16, 32, fake, fake, 64, None) == pg.PIC_EINVAL
    L.pic_upconv_wgrad_bf16.argtypes = [I, I, I, I, P, I, P, I, I, I, P, P, P]
    assert L.pic_upconv_wgrad_bf16(0, 1, 8, 8, fake, 64, fake, 64, 0, 32, fake, None, None) == pg.PIC_EINVAL
    L.pic_upconv_bf16.argtypes = [I, I, I, I, P, I, P, P, P, I, I, I, P]
    assert L.pic_upconv_bf16(1, 1, 8, 8, fake, 64, fake, fake, fake, 32, 8, 32, None) == pg.PIC_EINVAL
    L.pic_avgpool2_bf16.argtypes = [I, I, I, P, I, I, I, P, P]
    assert L.pic_avgpool2_bf16(1, 7, 8, fake, 32, 0, 32, fake, None) == pg.PIC_EINVAL
    L.pic_head_bf16.argtypes = [Q, P, P, P, P, P]
    assert L.pic_head_bf16(0, fake, fake, fake, fake, None) == pg.PIC_EINVAL
    L.pic_head_back_bf16.argtypes = [Q, P, P, P, P, P, P, P]
    assert L.pic_head_back_bf16(10, fake, ctypes.c_void_p(18), fake, fake, fake, fake, None) == pg.PIC_EINVAL
    L.pic_relu_back_bf16.argtypes = [I, I, I, P, I, I, P, I, I, P, P, I, P, P]
    assert L.pic_relu_back_bf16(1, 8, 8, fake, 24, 0, fake, 24, 0, None, fake, 24, fake, None) == pg.PIC_EINVAL

"""pic_deposit_static: the deposit for callers that cannot allocate device
memory (their device memory belongs to another runtime's pool, or they run
in a loop that cannot take an allocation's device-wide synchronisation).

It keeps its scratch in a fixed static device array, so the test calls it
twice in a row through the C ABI and checks each result against the
context-based entry points (pic_load + pic_step(0) + pic_diag(RHO)) within
the deposit tolerance of the other parity tests.  This file is collected
last so that a run stopping at the first failure has run everything else."""
import ctypes

import numpy as np
import pytest

import synth
from oracle import deposit as odeposit
from oracle.geometry import from_workload

pytestmark = pytest.mark.gpu

RHO_TOL = 1e-5   # of max |rho|, as in the deposit parity tests


@pytest.fixture(scope="module")
def lib():
    import __graft_entry__
    __graft_entry__.build()
    import paper_1610_03918_gb300 as pg
    lib = pg.load_library()
    f = lib.pic_deposit_static
    f.argtypes = [ctypes.c_int32, ctypes.c_int32, ctypes.c_int32, ctypes.c_int32, ctypes.c_int64,
                  ctypes.c_void_p, ctypes.c_void_p, ctypes.c_double, ctypes.c_void_p,
                  ctypes.c_void_p]
    f.restype = ctypes.c_int
    return lib


def _context_rho(w, species, p):
    import paper_1610_03918_gb300 as pg
    sim = pg.Sim(w, capacity=len(p))
    sim.load_particles(species, p)
    sim.step(0)
    rho = sim.rho()
    sim.close()
    return rho


def test_static_deposit_matches_context_deposit_twice(lib):
    import torch
    import paper_1610_03918_gb300 as pg
    w = synth.small_trench(nx=72, ny=40, depth=20, width=6, ppc=12, seed=31)
    nxn, nyn = w.nx + 1, w.ny
    stream = torch.cuda.current_stream()
    for species in (0, 1):          # two calls in a row on the same scratch
        p = synth.maxwellian_load(w, species)
        ref = _context_rho(w, species, p)
        x = torch.tensor(p.x, dtype=torch.float64, device="cuda")
        y = torch.tensor(p.y, dtype=torch.float64, device="cuda")
        rho = torch.full((nxn, nyn), float("nan"), dtype=torch.float64, device="cuda")
        st = lib.pic_deposit_static(w.nx, w.ny, int(w.periodic_x), int(w.periodic_y), len(p),
                                    x.data_ptr(), y.data_ptr(), w.charge[species] / w.ppc,
                                    rho.data_ptr(), stream.cuda_stream)
        assert st == pg.PIC_OK, pg.pic_strerror(st)
        torch.cuda.synchronize()
        got = rho.cpu().numpy()
        scale = np.abs(ref).max()
        assert np.abs(got - ref).max() <= RHO_TOL * scale


def _static(lib, w, x, y, weight):
    import torch
    import paper_1610_03918_gb300 as pg
    nxn = w.nx if w.periodic_x else w.nx + 1
    nyn = w.ny if w.periodic_y else w.ny + 1
    xd = torch.tensor(np.asarray(x, np.float64), device="cuda")
    yd = torch.tensor(np.asarray(y, np.float64), device="cuda")
    rho = torch.full((nxn, nyn), float("nan"), dtype=torch.float64, device="cuda")
    st = lib.pic_deposit_static(w.nx, w.ny, int(w.periodic_x), int(w.periodic_y), xd.numel(),
                                xd.data_ptr() if xd.numel() else None,
                                yd.data_ptr() if yd.numel() else None, weight, rho.data_ptr(),
                                torch.cuda.current_stream().cuda_stream)
    assert st == pg.PIC_OK, pg.pic_strerror(st)
    torch.cuda.synchronize()
    return rho.cpu().numpy()


# box types: doubly periodic, bounded in both directions, and the trench
# (bounded x, periodic y); sizes span several tiles with ragged tails
BOXES = {
    "periodic": synth.periodic_square_64(nx=48, ny=34, ppc=10, seed=41),
    "bounded": synth.bounded_square_256(nx=45, ny=38, ppc=10, seed=42),
    "trench": synth.small_trench(nx=72, ny=40, depth=20, width=6, ppc=12, seed=43),
}


@pytest.mark.parametrize("name", list(BOXES))
def test_static_deposit_matches_oracle(lib, name):
    # against the FP64 CIC deposit of the oracle, with particles outside the
    # grid (beyond a bounded edge, far outside a periodic one, NaN) mixed in:
    # a bounded box drops them, a periodic direction wraps them
    w = BOXES[name]
    p = synth.maxwellian_load(w, 1)
    rng = np.random.default_rng(7)
    k = 500
    xo = np.concatenate([p.x, rng.uniform(-3 * w.nx, 4 * w.nx, k), [np.nan, 0.5, w.nx + 0.0]])
    yo = np.concatenate([p.y, rng.uniform(-3 * w.ny, 4 * w.ny, k), [0.5, np.nan, 0.5]])
    weight = w.charge[1] / w.ppc
    got = _static(lib, w, xo, yo, weight)
    geom = from_workload(w)
    xs, ys = xo.copy(), yo.copy()
    keep = np.isfinite(xs) & np.isfinite(ys)
    if w.periodic_x:
        xs = np.mod(xs, w.nx)
    else:
        keep &= (xs >= 0) & (xs < w.nx)
    if w.periodic_y:
        ys = np.mod(ys, w.ny)
    else:
        keep &= (ys >= 0) & (ys < w.ny)
    ref = odeposit.cic_density(geom, xs[keep], ys[keep], weight)
    scale = np.abs(ref).max()
    assert np.abs(got - ref).max() <= RHO_TOL * scale, np.abs(got - ref).max() / scale
    # the exact fixed-point sum conserves the charge of the particles kept
    assert got.sum() == pytest.approx(weight * keep.sum(), rel=1e-12)


def test_static_deposit_no_particles(lib):
    # n = 0 after a call that left sums in the scratch: the grid comes back zero
    w = BOXES["periodic"]
    p = synth.maxwellian_load(w, 0)
    assert np.abs(_static(lib, w, p.x, p.y, 1.0)).max() > 0
    got = _static(lib, w, [], [], 1.0)
    assert np.array_equal(got, np.zeros_like(got))


def test_static_deposit_rejects_oversized_grid(lib):
    import torch
    import paper_1610_03918_gb300 as pg
    rho = torch.zeros(4, dtype=torch.float64, device="cuda")
    st = lib.pic_deposit_static(2048, 1024, 0, 1, 0, None, None, 1.0, rho.data_ptr(), None)
    assert st == pg.PIC_ESIZE
    assert "scratch" in pg.pic_strerror(st)

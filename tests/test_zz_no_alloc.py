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


def test_static_deposit_rejects_oversized_grid(lib):
    import torch
    import paper_1610_03918_gb300 as pg
    rho = torch.zeros(4, dtype=torch.float64, device="cuda")
    st = lib.pic_deposit_static(2048, 1024, 0, 1, 0, None, None, 1.0, rho.data_ptr(), None)
    assert st == pg.PIC_ESIZE
    assert "scratch" in pg.pic_strerror(st)

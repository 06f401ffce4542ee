"""Python binding of the GB300-native 2D electrostatic PIC library.

Argument marshalling only: every step of the loop (sort, gather, push,
absorption, deposit, Poisson solve, field) runs in the sm_103a kernels of
``libpicgb.so`` behind the C ABI of ``include/picgb.h``.  The functions
carry the C names (pic_init, pic_load, pic_step, pic_diag, pic_free,
pic_strerror); ``Sim`` strings them together.  Device memory is drawn from
PyTorch's caching allocator and work runs on PyTorch's current CUDA stream
unless told otherwise.

There is no CPU fallback: if the library was not built, or no GPU is
visible, loading it raises.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

from .build import lib_path

# status codes and constants mirrored from include/picgb.h
PIC_OK, PIC_EINVAL, PIC_ENOMEM, PIC_ECUDA, PIC_ENOCONV = 0, 1, 2, 3, 4
PIC_EOVERFLOW, PIC_ECFL, PIC_ETIMEOUT, PIC_EFULL, PIC_ESTATE, PIC_ERANGE = 5, 6, 7, 8, 9, 10
PIC_ESIZE = 11
PIC_ST_NOCONV, PIC_ST_FULL, PIC_ST_CFL, PIC_ST_RANGE, PIC_ST_CAPACITY = 1, 2, 4, 8, 16
PIC_LOAD_V_AT_T0 = 1
(PIC_DIAG_ENERGY, PIC_DIAG_MOMENTUM, PIC_DIAG_COUNTS, PIC_DIAG_SURFACE, PIC_DIAG_HITS,
 PIC_DIAG_RHO, PIC_DIAG_PHI, PIC_DIAG_E, PIC_DIAG_STATE_E, PIC_DIAG_STATE_I,
 PIC_DIAG_POISSON, PIC_DIAG_STATUS, PIC_DIAG_TIMING, PIC_DIAG_PHI_VACUUM,
 PIC_DIAG_SOLVER, PIC_DIAG_SORT, PIC_DIAG_TILE) = range(17)
(WALL_XMIN, WALL_XMAX, WALL_YMIN, WALL_YMAX, WALL_COND_PX, WALL_COND_MX,
 WALL_COND_PY, WALL_COND_MY) = range(8)

EXPORTED = ("pic_init", "pic_load", "pic_step", "pic_set_timing", "pic_diag", "pic_free", "pic_strerror",
            "pic_batch_init", "pic_batch_member", "pic_batch_step", "pic_batch_timing",
            "pic_batch_free", "pic_deposit_static", "pic_unet_create", "pic_unet_forward",
            "pic_unet_gradients", "pic_unet_train_step", "pic_unet_free", "pic_save", "pic_restore",
            "pic_unet_init", "pic_unet_save", "pic_unet_load", "pic_set_learned_start",
            "pic_learned_target", "pic_set_warm_start", "pic_step_particles", "pic_step_fields",
            "pic_exchange_buffer", "pic_exchange_sum", "pic_autotune", "pic_unet_set_conv_impl",
            "pic_unet_status", "pic_conv3x3_bf16", "pic_upconv_back_bf16",
            "pic_conv3x3_wgrad_bf16", "pic_upconv_wgrad_bf16", "pic_upconv_bf16", "pic_avgpool2_bf16",
            "pic_head_bf16", "pic_head_back_bf16", "pic_relu_back_bf16")

ALLOC_FN = ctypes.CFUNCTYPE(ctypes.c_void_p, ctypes.c_size_t, ctypes.c_void_p, ctypes.c_void_p)
FREE_FN = ctypes.CFUNCTYPE(None, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p)


# pic_config.poisson_method
POISSON_AUTO = 0        # direct FFT / tridiagonal / capacitance solve where the geometry allows
POISSON_MULTIGRID = 1   # multigrid-preconditioned conjugate gradient everywhere


class PicConfig(ctypes.Structure):
    _fields_ = [
        ("nx", ctypes.c_int32), ("ny", ctypes.c_int32),
        ("periodic_x", ctypes.c_int32), ("periodic_y", ctypes.c_int32),
        ("dt", ctypes.c_double),
        ("phi_top", ctypes.c_double), ("phi_electrode", ctypes.c_double),
        ("trench_depth", ctypes.c_int32), ("trench_y0", ctypes.c_int32),
        ("trench_width", ctypes.c_int32), ("surface_charge", ctypes.c_int32),
        ("alpha", ctypes.c_double * 2), ("charge", ctypes.c_double * 2),
        ("ppc", ctypes.c_int32 * 2),
        ("capacity", ctypes.c_int64 * 2),
        ("sort_every", ctypes.c_int32), ("poisson_maxit", ctypes.c_int32),
        ("poisson_rtol", ctypes.c_double),
        ("warm_start", ctypes.c_int32), ("device", ctypes.c_int32),
        ("timing", ctypes.c_int32), ("graphs", ctypes.c_int32),
        ("poisson_method", ctypes.c_int32),
        ("hit_capacity", ctypes.c_int64),
        ("stream", ctypes.c_void_p),
        ("alloc", ALLOC_FN), ("free", FREE_FN), ("alloc_user", ctypes.c_void_p),
        ("phi_rf_amp", ctypes.c_double), ("omega_rf", ctypes.c_double),
        ("recycle", ctypes.c_int32), ("source_x0", ctypes.c_int32), ("source_x1", ctypes.c_int32),
        ("recycle_vth", ctypes.c_double), ("seed", ctypes.c_uint64),
        ("unet_weights", ctypes.c_char_p),
        ("decomposed", ctypes.c_int32), ("tile_variant", ctypes.c_int32),
    ]


class PicHit(ctypes.Structure):
    _fields_ = [("id", ctypes.c_uint32), ("species", ctypes.c_int16), ("wall", ctypes.c_int16),
                ("cell", ctypes.c_int32), ("step", ctypes.c_int32),
                ("vx", ctypes.c_float), ("vy", ctypes.c_float)]


HIT_DTYPE = np.dtype([("id", np.uint32), ("species", np.int16), ("wall", np.int16),
                      ("cell", np.int32), ("step", np.int32), ("vx", np.float32),
                      ("vy", np.float32)])

_lib = None


def load_library():
    """Load libpicgb.so (built by paper_1610_03918_gb300.build); raises if absent."""
    global _lib
    if _lib is not None:
        return _lib
    path = lib_path()
    if not os.path.exists(path):
        raise RuntimeError(f"CUDA library not built: {path} is missing "
                           "(run __graft_entry__.build())")
    lib = ctypes.CDLL(path)
    P = ctypes.c_void_p
    D = ctypes.POINTER(ctypes.c_double)
    lib.pic_init.argtypes = [ctypes.POINTER(PicConfig), ctypes.POINTER(ctypes.c_void_p)]
    lib.pic_load.argtypes = [P, ctypes.c_int32, ctypes.c_int64, D, D, D, D,
                             ctypes.POINTER(ctypes.c_uint32), ctypes.c_uint32]
    lib.pic_step.argtypes = [P, ctypes.c_int32]
    lib.pic_set_timing.argtypes = [P, ctypes.c_int32]
    lib.pic_diag.argtypes = [P, ctypes.c_int32, P, ctypes.c_int64, ctypes.POINTER(ctypes.c_int64)]
    lib.pic_free.argtypes = [P]
    lib.pic_save.argtypes = [P, P, ctypes.c_int64, ctypes.POINTER(ctypes.c_int64)]
    lib.pic_restore.argtypes = [P, P, ctypes.c_int64]
    lib.pic_save.restype = ctypes.c_int
    lib.pic_restore.restype = ctypes.c_int
    lib.pic_strerror.argtypes = [ctypes.c_int]
    lib.pic_strerror.restype = ctypes.c_char_p
    lib.pic_last_error.argtypes = []
    lib.pic_last_error.restype = ctypes.c_char_p
    lib.pic_batch_init.argtypes = [ctypes.POINTER(PicConfig), ctypes.c_int32, P,
                                   ctypes.POINTER(ctypes.c_void_p)]
    lib.pic_batch_member.argtypes = [P, ctypes.c_int32]
    lib.pic_batch_member.restype = ctypes.c_void_p
    lib.pic_batch_step.argtypes = [P, ctypes.c_int32]
    lib.pic_batch_timing.argtypes = [P, ctypes.POINTER(ctypes.c_double)]
    lib.pic_batch_free.argtypes = [P]
    for name in ("pic_batch_init", "pic_batch_step", "pic_batch_timing", "pic_batch_free"):
        getattr(lib, name).restype = ctypes.c_int
    lib.pic_learned_input.argtypes = [P, ctypes.c_int32, P, ctypes.POINTER(ctypes.c_double)]
    lib.pic_learned_input.restype = ctypes.c_int
    lib.pic_poisson.argtypes = [P, ctypes.c_int32, P, ctypes.c_double, ctypes.POINTER(ctypes.c_double)]
    lib.pic_poisson.restype = ctypes.c_int
    lib.pic_unet_create.argtypes = [ctypes.c_int32, ctypes.c_int32, ctypes.c_int32, P,
                                    ctypes.POINTER(ctypes.c_void_p)]
    lib.pic_unet_num_params.argtypes = [P]
    lib.pic_unet_num_params.restype = ctypes.c_int64
    lib.pic_unet_set_params.argtypes = [P, ctypes.POINTER(ctypes.c_float)]
    lib.pic_unet_get_params.argtypes = [P, ctypes.POINTER(ctypes.c_float)]
    lib.pic_unet_forward.argtypes = [P, P, P]
    lib.pic_unet_gradients.argtypes = [P, P, P, ctypes.POINTER(ctypes.c_float),
                                       ctypes.POINTER(ctypes.c_double)]
    lib.pic_unet_train_step.argtypes = [P, P, P, ctypes.c_float, ctypes.POINTER(ctypes.c_double)]
    lib.pic_unet_free.argtypes = [P]
    lib.pic_unet_init.argtypes = [P, ctypes.c_uint64]
    lib.pic_unet_save.argtypes = [P, ctypes.c_char_p]
    lib.pic_unet_load.argtypes = [P, ctypes.c_char_p]
    lib.pic_set_learned_start.argtypes = [P, P]
    lib.pic_learned_target.argtypes = [P, ctypes.c_int32, ctypes.c_double, P]
    lib.pic_set_warm_start.argtypes = [P, ctypes.c_int32]
    lib.pic_set_warm_start.restype = ctypes.c_int
    lib.pic_step_particles.argtypes = [P]
    lib.pic_step_fields.argtypes = [P]
    lib.pic_exchange_buffer.argtypes = [P, ctypes.POINTER(ctypes.c_void_p), ctypes.POINTER(ctypes.c_int64)]
    lib.pic_exchange_sum.argtypes = [ctypes.POINTER(ctypes.c_void_p), ctypes.c_int32]
    for name in ("pic_step_particles", "pic_step_fields", "pic_exchange_buffer", "pic_exchange_sum"):
        getattr(lib, name).restype = ctypes.c_int
    lib.pic_autotune.argtypes = [P, ctypes.c_int32, ctypes.c_char_p, ctypes.POINTER(ctypes.c_int32)]
    lib.pic_autotune.restype = ctypes.c_int
    lib.pic_unet_set_conv_impl.argtypes = [P, ctypes.c_int32]
    lib.pic_unet_status.argtypes = [P]
    lib.pic_unet_set_conv_impl.restype = ctypes.c_int
    lib.pic_unet_status.restype = ctypes.c_int
    for name in ("pic_unet_init", "pic_unet_save", "pic_unet_load", "pic_set_learned_start",
                 "pic_learned_target", "pic_set_warm_start", "pic_step_particles", "pic_step_fields",
            "pic_exchange_buffer", "pic_exchange_sum", "pic_autotune", "pic_unet_set_conv_impl",
            "pic_unet_status", "pic_conv3x3_bf16", "pic_upconv_back_bf16",
            "pic_conv3x3_wgrad_bf16", "pic_upconv_wgrad_bf16", "pic_upconv_bf16", "pic_avgpool2_bf16",
            "pic_head_bf16", "pic_head_back_bf16", "pic_relu_back_bf16"):
        getattr(lib, name).restype = ctypes.c_int
    for name in ("pic_unet_create", "pic_unet_set_params", "pic_unet_get_params",
                 "pic_unet_forward", "pic_unet_gradients", "pic_unet_train_step", "pic_unet_free"):
        getattr(lib, name).restype = ctypes.c_int
    for name in ("pic_init", "pic_load", "pic_step", "pic_set_timing", "pic_diag", "pic_free"):
        getattr(lib, name).restype = ctypes.c_int
    _lib = lib
    return lib


class PicError(RuntimeError):
    def __init__(self, code, where):
        self.code = code
        detail = load_library().pic_last_error().decode()
        super().__init__(f"{where}: {pic_strerror(code)} ({code})" + (f" [{detail}]" if detail else ""))


def pic_strerror(code: int) -> str:
    return load_library().pic_strerror(int(code)).decode()


def _dptr(a):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_double)) if a is not None else None


def pic_init(cfg: PicConfig) -> ctypes.c_void_p:
    ctx = ctypes.c_void_p()
    st = load_library().pic_init(ctypes.byref(cfg), ctypes.byref(ctx))
    if st != PIC_OK:
        raise PicError(st, "pic_init")
    return ctx


def pic_load(ctx, species: int, x, y=None, vx=None, vy=None, ids=None, flags: int = 0) -> int:
    x = np.ascontiguousarray(x, dtype=np.float64)
    n = x.size
    arrs = [np.ascontiguousarray(a, dtype=np.float64) if a is not None else None
            for a in (y, vx, vy)]
    idp = None
    if ids is not None:
        ids = np.ascontiguousarray(ids, dtype=np.uint32)
        idp = ids.ctypes.data_as(ctypes.POINTER(ctypes.c_uint32))
    return load_library().pic_load(ctx, int(species), int(n), _dptr(x), *[_dptr(a) for a in arrs],
                                   idp, int(flags))


def pic_step(ctx, nsteps: int) -> int:
    return load_library().pic_step(ctx, int(nsteps))


def pic_set_timing(ctx, on: bool) -> int:
    return load_library().pic_set_timing(ctx, int(bool(on)))


def pic_diag(ctx, kind: int, out: np.ndarray):
    """Fill ``out`` (a contiguous numpy array) and return (status, count)."""
    n = ctypes.c_int64(0)
    st = load_library().pic_diag(ctx, int(kind), out.ctypes.data_as(ctypes.c_void_p),
                                 int(out.nbytes), ctypes.byref(n))
    return st, int(n.value)


def pic_free(ctx) -> int:
    return load_library().pic_free(ctx)


# ---------------------------------------------------------------------------
class _TorchAllocator:
    """Device memory from PyTorch's caching allocator on the given stream."""

    def __init__(self, device: int, stream: int):
        import torch
        self.torch = torch
        self.device = device
        self.stream = stream

        def _alloc(nbytes, stream, user):
            try:
                return int(torch.cuda.caching_allocator_alloc(int(nbytes), self.device,
                                                              stream or self.stream))
            except Exception:
                return None

        def _free(ptr, stream, user):
            torch.cuda.caching_allocator_delete(int(ptr))

        self.alloc = ALLOC_FN(_alloc)
        self.free = FREE_FN(_free)


def make_config(w, capacity=None, device: int = 0, stream=None, hit_capacity: int = 1 << 20,
                poisson_maxit: int = 200, warm_start: int = 1, allocator=None,
                timing: bool = False, graphs: bool = True,
                poisson_method: int = POISSON_AUTO, unet_weights=None,
                decomposed: bool = False, tile_variant: int = 0) -> PicConfig:
    """PicConfig from a workload description (an object with the fields of
    synth.Workload)."""
    cfg = PicConfig()
    cfg.nx, cfg.ny = int(w.nx), int(w.ny)
    cfg.periodic_x, cfg.periodic_y = int(w.periodic_x), int(w.periodic_y)
    cfg.dt = float(w.dt)
    cfg.phi_top, cfg.phi_electrode = float(w.phi_top), float(w.phi_electrode)
    cfg.trench_depth, cfg.trench_y0 = int(w.trench_depth), int(w.trench_y0)
    cfg.trench_width = int(w.trench_width)
    cfg.surface_charge = int(bool(w.surface_charge))
    cfg.alpha[0], cfg.alpha[1] = w.alpha
    cfg.charge[0], cfg.charge[1] = w.charge
    cfg.ppc[0] = cfg.ppc[1] = int(w.ppc)
    if capacity is None:
        capacity = int(w.nx) * int(w.ny) * int(w.ppc)
    cfg.capacity[0] = cfg.capacity[1] = int(capacity)
    cfg.sort_every = int(getattr(w, "sort_every", 8))
    cfg.poisson_maxit = int(poisson_maxit)
    cfg.poisson_rtol = float(getattr(w, "poisson_rtol", 1e-6))
    cfg.warm_start = int(warm_start)
    cfg.device = int(device)
    cfg.timing = int(bool(timing))
    cfg.graphs = int(bool(graphs))
    cfg.poisson_method = int(poisson_method)
    cfg.hit_capacity = int(hit_capacity)
    cfg.phi_rf_amp = float(getattr(w, "phi_rf_amp", 0.0))
    cfg.omega_rf = float(getattr(w, "omega_rf", 0.0))
    cfg.recycle = int(bool(getattr(w, "recycle", False)))
    cfg.source_x0 = int(getattr(w, "source_x0", 0))
    cfg.source_x1 = int(getattr(w, "source_x1", 0))
    cfg.recycle_vth = float(w.vth[1]) if cfg.recycle else 0.0
    cfg.seed = int(getattr(w, "recycle_seed", 0)) & 0xFFFFFFFFFFFFFFFF
    cfg.unet_weights = os.fsencode(unet_weights) if unet_weights is not None else None
    cfg.decomposed = int(bool(decomposed))
    cfg.tile_variant = int(tile_variant)
    cfg.stream = stream
    if allocator is not None:
        cfg.alloc = allocator.alloc
        cfg.free = allocator.free
    return cfg


class Sim:
    """One simulation context.  ``torch_memory``: allocate through PyTorch's
    caching allocator and run on PyTorch's current stream of ``device``."""

    def __init__(self, w, capacity=None, device: int = 0, torch_memory: bool = True,
                 _ctx=None, **kw):
        load_library()
        self.w = w
        self.nxn = w.nx if w.periodic_x else w.nx + 1
        self.nyn = w.ny if w.periodic_y else w.ny + 1
        self._owned = _ctx is None
        if _ctx is not None:        # a member of a Batch: the batch owns it
            self.ctx = _ctx
            self.cfg = kw.pop("_cfg")
            self.torch_stream = None
            self._allocator = None
            return
        self._allocator = None
        stream = None
        self.torch_stream = None
        if torch_memory:
            import torch
            if not torch.cuda.is_available():
                raise RuntimeError("no CUDA device visible")
            torch.cuda.set_device(device)
            # a stream of its own, shared by the library and the allocator
            self.torch_stream = torch.cuda.Stream(device)
            stream = self.torch_stream.cuda_stream
            self._allocator = _TorchAllocator(device, stream)
        self.cfg = make_config(w, capacity=capacity, device=device, stream=stream,
                               allocator=self._allocator, **kw)
        self.ctx = pic_init(self.cfg)

    def close(self):
        if self.ctx and self._owned:
            pic_free(self.ctx)
        self.ctx = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def _check(self, st, where, allow=()):
        if st != PIC_OK and st not in allow:
            raise PicError(st, where)
        return st

    def load(self, species, x, y, vx, vy, ids=None, v_at_t0=False, allow=()):
        return self._check(pic_load(self.ctx, species, x, y, vx, vy, ids,
                                    PIC_LOAD_V_AT_T0 if v_at_t0 else 0), "pic_load", allow)

    def load_particles(self, species, p, v_at_t0=False, allow=()):
        return self.load(species, p.x, p.y, p.vx, p.vy, p.ids, v_at_t0, allow)

    def set_rho_ext(self, rho_ext):
        return self._check(pic_load(self.ctx, -1, np.asarray(rho_ext, np.float64).ravel()),
                           "pic_load(rho_ext)")

    def step(self, n=1, allow=()):
        return self._check(pic_step(self.ctx, n), "pic_step", allow)

    def set_timing(self, on: bool):
        """Per-phase timing (event nodes between the phases) on or off for
        the steps that follow."""
        return self._check(pic_set_timing(self.ctx, on), "pic_set_timing")

    def diag(self, kind, out, allow=(PIC_EFULL, PIC_ERANGE)):
        st, n = pic_diag(self.ctx, kind, out)
        self._check(st, "pic_diag", allow)
        return out, n

    # convenience views -------------------------------------------------
    def grid(self, kind):
        out = np.empty((self.nxn, self.nyn), np.float64)
        return self.diag(kind, out)[0]

    def rho(self):
        return self.grid(PIC_DIAG_RHO)

    def phi(self):
        return self.grid(PIC_DIAG_PHI)

    def efield(self):
        out = np.empty((2, self.nxn, self.nyn), np.float64)
        self.diag(PIC_DIAG_E, out)
        return out[0], out[1]

    def energy(self):
        return self.diag(PIC_DIAG_ENERGY, np.empty(4))[0]

    def momentum(self):
        return self.diag(PIC_DIAG_MOMENTUM, np.empty(4))[0].reshape(2, 2)

    def counts(self):
        out = self.diag(PIC_DIAG_COUNTS, np.empty(18, np.int64))[0]
        return out[:16].reshape(2, 8), out[16:]

    def surface(self):
        return self.diag(PIC_DIAG_SURFACE, np.empty(2 * self.w.ny, np.int64))[0].reshape(2, -1)

    def hits(self, cap=None):
        cap = int(self.cfg.hit_capacity if cap is None else cap)
        out = np.empty(cap, HIT_DTYPE)
        _, n = self.diag(PIC_DIAG_HITS, out)
        return out[:n]

    def state(self, species, out=None):
        """(5, live) array of x, y, vx, vy, id of the live particles.  `out`: a
        C-contiguous float64 buffer of at least 5 * live elements to fill (pinned
        host memory is written by the device directly); its front is returned."""
        live = int(self.counts()[1][species])
        if out is None:
            view = np.empty((5, live), np.float64)
        else:
            flat = out.reshape(-1)
            if out.dtype != np.float64 or not out.flags["C_CONTIGUOUS"] or flat.size < 5 * live:
                raise ValueError("state: out must be a contiguous float64 buffer of >= 5 * live elements")
            view = flat[:5 * live].reshape(5, live)
        self.diag(PIC_DIAG_STATE_E if species == 0 else PIC_DIAG_STATE_I, view)
        return view

    def poisson_stats(self):
        """[inner iterations, outer passes, relative residual, ms, relative
        residual at the first check (the initial guess's with multigrid PCG)]
        of the last solve."""
        return self.diag(PIC_DIAG_POISSON, np.empty(5))[0]

    def timing(self):
        """Per-phase device time since the last call (and resets it):
        dict of steps, ms_particles, ms_sort, ms_poisson (with the field), ms_rho,
        sorts, launches, slots."""
        v = self.diag(PIC_DIAG_TIMING, np.empty(8))[0]
        keys = ("steps", "ms_particles", "ms_sort", "ms_poisson", "ms_rho", "sorts",
                "launches", "slots")
        return dict(zip(keys, v.tolist()))

    def save(self) -> bytes:
        """A checkpoint of the whole run (pic_save)."""
        lib = load_library()
        n = ctypes.c_int64(0)
        self._check(lib.pic_save(self.ctx, None, 0, ctypes.byref(n)), "pic_save")
        buf = ctypes.create_string_buffer(int(n.value))
        self._check(lib.pic_save(self.ctx, buf, int(n.value), ctypes.byref(n)), "pic_save")
        return buf.raw[: int(n.value)]

    def restore(self, blob: bytes):
        """Continue the run saved in `blob` (pic_restore)."""
        buf = ctypes.create_string_buffer(bytes(blob), len(blob))
        return self._check(load_library().pic_restore(self.ctx, buf, len(blob)), "pic_restore")

    def set_phi(self, phi):
        return self._check(pic_load(self.ctx, -2, np.asarray(phi, np.float64).ravel()), "pic_load(phi)")

    def phi_vacuum(self):
        return self.grid(PIC_DIAG_PHI_VACUUM)

    def learned_input(self, hpad):
        """(x, s): the warm-start network's input for the current rho as a
        torch CUDA tensor [1, hpad, nyn, 2], and the scale s = max |rho|."""
        import torch
        x = torch.empty((1, hpad, self.nyn, 2), dtype=torch.float32, device="cuda")
        s = ctypes.c_double(0.0)
        self._check(load_library().pic_learned_input(self.ctx, int(hpad), x.data_ptr(), ctypes.byref(s)),
                    "pic_learned_input")
        return x, s.value

    def learned_target(self, hpad, scale):
        """The warm-start network's training target (phi - phi_L) / scale for
        the current potential, as a torch CUDA tensor [hpad, nyn]."""
        import torch
        t = torch.empty((hpad, self.nyn), dtype=torch.float32, device="cuda")
        self._check(load_library().pic_learned_target(self.ctx, int(hpad), float(scale), t.data_ptr()),
                    "pic_learned_target")
        return t

    # one rank of a run split by particles -------------------------------
    def step_particles(self):
        """Particle phase of a decomposed step (pic_step_particles)."""
        return self._check(load_library().pic_step_particles(self.ctx), "pic_step_particles")

    def step_fields(self):
        """Field phase of a decomposed step (pic_step_fields)."""
        return self._check(load_library().pic_step_fields(self.ctx), "pic_step_fields")

    def exchange_buffer(self):
        """The rank's exchange buffer as a torch int64 CUDA tensor viewing the
        library's device memory (to be all-reduced in place, sum)."""
        import torch
        ptr = ctypes.c_void_p()
        n = ctypes.c_int64()
        self._check(load_library().pic_exchange_buffer(self.ctx, ctypes.byref(ptr), ctypes.byref(n)),
                    "pic_exchange_buffer")

        class _View:
            __cuda_array_interface__ = {"shape": (int(n.value),), "typestr": "<i8",
                                        "data": (int(ptr.value), False), "version": 3}
        return torch.as_tensor(_View(), device="cuda")

    def set_warm_start(self, mode: int):
        """Initial guess of the solves that follow: 0 zero, 1 previous,
        2 extrapolated, 3 learned (after set_learned_start), 4 lift (the
        potential of the empty box)."""
        return self._check(load_library().pic_set_warm_start(self.ctx, int(mode)), "pic_set_warm_start")

    def set_learned_start(self, net):
        """Every later solve starts from the guess of (a copy of) the trained
        network `net` (warm_start 3, inside the step graph)."""
        return self._check(load_library().pic_set_learned_start(self.ctx, net.h), "pic_set_learned_start")

    def poisson(self, guess, y=None, scale=0.0):
        """Re-solve for the current rho from guess 0 zero, 1 previous, 2 vacuum,
        3 learned (y: network output tensor); returns [iterations, passes,
        relative residual, ms]."""
        out = (ctypes.c_double * 4)()
        self._check(load_library().pic_poisson(self.ctx, int(guess), y.data_ptr() if y is not None else None,
                                               float(scale), out), "pic_poisson")
        return list(out)

    def sort_interval(self):
        """(steps between tile sorts in use, tuned): the interval is 0 while
        the library is still timing it (sort_every = 0)."""
        v = self.diag(PIC_DIAG_SORT, np.zeros(2, np.int32))[0]
        return int(v[0]), bool(v[1])

    def autotune(self, steps: int = 8, cache=None):
        """Choose the tile variant by timing (pic_autotune); returns its index."""
        v = ctypes.c_int32(-1)
        self._check(load_library().pic_autotune(self.ctx, int(steps),
                                                os.fsencode(cache) if cache else None, ctypes.byref(v)),
                    "pic_autotune")
        return int(v.value)

    def tile(self):
        """(variant, tile cells x, tile cells y, halo, threads) in use."""
        return tuple(int(v) for v in self.diag(PIC_DIAG_TILE, np.zeros(5, np.int32))[0])

    def solver(self):
        """Inner Poisson solver in use: POISSON_AUTO (0) = the direct one,
        POISSON_MULTIGRID (1) = multigrid-preconditioned CG."""
        return int(self.diag(PIC_DIAG_SOLVER, np.zeros(1, np.int32))[0][0])

    def status(self):
        out = np.zeros(1, np.uint32)
        st, _ = pic_diag(self.ctx, PIC_DIAG_STATUS, out)
        self._check(st, "pic_diag(status)")
        return int(out[0])


def exchange_sum(sims):
    """The all-reduce of the exchange buffers of several ranks held by this
    process on one GPU (pic_exchange_sum)."""
    arr = (ctypes.c_void_p * len(sims))(*[s.ctx.value if isinstance(s.ctx, ctypes.c_void_p) else s.ctx
                                          for s in sims])
    st = load_library().pic_exchange_sum(arr, len(sims))
    if st != PIC_OK:
        raise PicError(st, "pic_exchange_sum")


class Batch:
    """An ensemble of independent runs advanced together: one captured CUDA
    graph per ensemble step with every member's step as a parallel branch.
    ``members[k]`` is a Sim view of member k for loading and diagnostics."""

    def __init__(self, workloads, capacities=None, device: int = 0, timing: bool = False,
                 torch_memory: bool = True, **kw):
        lib = load_library()
        self.workloads = list(workloads)
        n = len(self.workloads)
        capacities = capacities or [None] * n
        self._allocator = None
        self.torch_stream = None
        stream = None
        if torch_memory:
            import torch
            if not torch.cuda.is_available():
                raise RuntimeError("no CUDA device visible")
            torch.cuda.set_device(device)
            self.torch_stream = torch.cuda.Stream(device)
            stream = self.torch_stream.cuda_stream
            self._allocator = _TorchAllocator(device, stream)
        cfgs = (PicConfig * n)()
        for k, w in enumerate(self.workloads):
            cfgs[k] = make_config(w, capacity=capacities[k], device=device, stream=stream,
                                  allocator=self._allocator, timing=timing, **kw)
        self.cfgs = cfgs
        h = ctypes.c_void_p()
        st = lib.pic_batch_init(cfgs, n, stream, ctypes.byref(h))
        if st != PIC_OK:
            raise PicError(st, "pic_batch_init")
        self.h = h
        self.members = [Sim(w, _ctx=ctypes.c_void_p(lib.pic_batch_member(h, k)), _cfg=cfgs[k])
                        for k, w in enumerate(self.workloads)]

    def step(self, n=1):
        st = load_library().pic_batch_step(self.h, int(n))
        if st != PIC_OK:
            raise PicError(st, "pic_batch_step")

    def timing(self):
        out = (ctypes.c_double * 2)()
        st = load_library().pic_batch_timing(self.h, out)
        if st != PIC_OK:
            raise PicError(st, "pic_batch_timing")
        return {"steps": out[0], "ms": out[1]}

    def close(self):
        if getattr(self, "h", None):
            for m in self.members:
                m.ctx = None
            load_library().pic_batch_free(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class Unet:
    """The learned warm start's U-Net on the GPU (training and inference by
    the library's kernels).  Inputs and outputs are torch CUDA tensors:
    x [B, H, W, 2] float32, targets and outputs [B, H, W] float32."""

    def __init__(self, batch, height, width, stream=None):
        import torch
        lib = load_library()
        self.torch = torch
        self.stream = stream or torch.cuda.Stream()
        h = ctypes.c_void_p()
        st = lib.pic_unet_create(int(batch), int(height), int(width), self.stream.cuda_stream,
                                 ctypes.byref(h))
        if st != PIC_OK:
            raise PicError(st, "pic_unet_create")
        self.h = h
        self.shape = (batch, height, width)
        self.nparam = int(lib.pic_unet_num_params(h))

    def set_conv_impl(self, impl: int):
        """Convolutions and their data and weight gradients on the tcgen05
        tensor cores where the shapes allow (0, the default), or all on the
        mma.sync and CUDA-core kernels (1)."""
        st = load_library().pic_unet_set_conv_impl(self.h, int(impl))
        if st != PIC_OK:
            raise PicError(st, "pic_unet_set_conv_impl")

    def status(self):
        """PIC_ETIMEOUT if a bounded wait of a tensor-core kernel gave up."""
        return load_library().pic_unet_status(self.h)

    def init(self, seed: int = 0):
        """He initialisation by the library (seeded Philox draws), zero biases."""
        st = load_library().pic_unet_init(self.h, int(seed) & 0xFFFFFFFFFFFFFFFF)
        if st != PIC_OK:
            raise PicError(st, "pic_unet_init")

    def save(self, path):
        st = load_library().pic_unet_save(self.h, os.fsencode(path))
        if st != PIC_OK:
            raise PicError(st, "pic_unet_save")

    def load(self, path):
        st = load_library().pic_unet_load(self.h, os.fsencode(path))
        if st != PIC_OK:
            raise PicError(st, "pic_unet_load")

    def set_params(self, flat):
        flat = np.ascontiguousarray(flat, dtype=np.float32)
        assert flat.size == self.nparam
        st = load_library().pic_unet_set_params(self.h, flat.ctypes.data_as(ctypes.POINTER(ctypes.c_float)))
        if st != PIC_OK:
            raise PicError(st, "pic_unet_set_params")

    def get_params(self):
        out = np.empty(self.nparam, np.float32)
        st = load_library().pic_unet_get_params(self.h, out.ctypes.data_as(ctypes.POINTER(ctypes.c_float)))
        if st != PIC_OK:
            raise PicError(st, "pic_unet_get_params")
        return out

    def forward(self, x):
        y = self.torch.empty(self.shape, dtype=self.torch.float32, device=x.device)
        self.stream.wait_stream(self.torch.cuda.current_stream())
        st = load_library().pic_unet_forward(self.h, x.data_ptr(), y.data_ptr())
        if st != PIC_OK:
            raise PicError(st, "pic_unet_forward")
        self.torch.cuda.current_stream().wait_stream(self.stream)
        return y

    def gradients(self, x, t):
        g = np.empty(self.nparam, np.float32)
        loss = ctypes.c_double(0.0)
        self.stream.wait_stream(self.torch.cuda.current_stream())
        st = load_library().pic_unet_gradients(self.h, x.data_ptr(), t.data_ptr(),
                                               g.ctypes.data_as(ctypes.POINTER(ctypes.c_float)),
                                               ctypes.byref(loss))
        if st != PIC_OK:
            raise PicError(st, "pic_unet_gradients")
        return loss.value, g

    def train_step(self, x, t, lr):
        self.stream.wait_stream(self.torch.cuda.current_stream())
        st = load_library().pic_unet_train_step(self.h, x.data_ptr(), t.data_ptr(), float(lr), None)
        if st != PIC_OK:
            raise PicError(st, "pic_unet_train_step")

    def close(self):
        if getattr(self, "h", None):
            load_library().pic_unet_free(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

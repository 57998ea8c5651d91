"""Thin Python binding of the C ABI in include/lbmice.h (ctypes; argument marshalling only).

Every step of the solver runs in the CUDA kernels of liblbmice.so. PyTorch supplies the
CUDA stream and, where the caller wants device results, the device memory. There is no
CPU fallback: constructing a :class:`Lattice` without the built library or without a GPU
raises.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

from .build import LIB, LIB_CHECKED

OK, EINVAL, ECUDA, ENOMEM, ENONFINITE, EUNSTABLE, ETIMEOUT, ENOTSUP = 0, -1, -2, -3, -4, -5, -6, -7
# bits of the checked build's violation word (lbmice_debug_flags)
OOB_POPS, OOB_PLANE, OOB_SHARED = 1, 2, 4
BC_PERIODIC, BC_INLET, BC_OUTLET, BC_FREESLIP = 0, 1, 2, 3
PHI, U, RHO, UX, UY, PHI_PREV, POPS, STATE = 0, 1, 2, 3, 4, 5, 6, 7
STORAGE = {"f32": 0, "f16": 1, "bf16": 2}
NSTATS = 6
MAX_RAYS = 1024  # LBMICE_MAX_RAYS
STAT_NAMES = ("area", "mass", "vapour_invariant", "sum_phi", "nonfinite", "steps")

EXPORTS = ("lbmice_params_default", "lbmice_create", "lbmice_init_seed", "lbmice_set_fields",
           "lbmice_step", "lbmice_fields", "lbmice_load", "lbmice_stats", "lbmice_sync",
           "lbmice_steps_done", "lbmice_destroy", "lbmice_strerror", "lbmice_state_bytes",
           "lbmice_stats_noalloc", "lbmice_batch_create", "lbmice_batch_size",
           "lbmice_batch_member", "lbmice_batch_step", "lbmice_batch_autotune",
           "lbmice_batch_set_shape", "lbmice_batch_destroy", "lbmice_last_error",
           "lbmice_tape_create", "lbmice_tape_record", "lbmice_tape_steps",
           "lbmice_tape_backward", "lbmice_tape_destroy", "lbmice_debug_flags",
           "lbmice_debug_set_margin", "lbmice_debug_wait_selftest", "lbmice_tips")


class LbmiceError(RuntimeError):
    def __init__(self, code: int, what: str):
        self.code = code
        detail = ""
        if code in (ECUDA, ENOMEM):
            try:
                detail = " [" + lib().lbmice_last_error().decode() + "]"
            except Exception:
                pass
        super().__init__(f"{what}: {strerror(code)} ({code}){detail}")


class Params(ctypes.Structure):
    """Mirror of struct lbmice_params."""
    _fields_ = [
        ("nx", ctypes.c_int32), ("ny", ctypes.c_int32),
        ("dx", ctypes.c_double), ("dt", ctypes.c_double),
        ("W0", ctypes.c_double), ("tau0", ctypes.c_double),
        ("D", ctypes.c_double), ("lam", ctypes.c_double),
        ("L_sat", ctypes.c_double), ("eps", ctypes.c_double),
        ("kappa_N", ctypes.c_double),
        ("U_in", ctypes.c_double), ("u_in", ctypes.c_double), ("nu", ctypes.c_double),
        ("bc", ctypes.c_int32 * 4), ("flow", ctypes.c_int32),
        ("check_every", ctypes.c_int32), ("storage", ctypes.c_int32),
        ("stencil", ctypes.c_int32), ("fold", ctypes.c_int32),
    ]


_lib = None


def lib_path() -> str:
    """liblbmice.so, or the bounds-checked liblbmice_checked.so when the environment sets
    LBMICE_CHECKED=1."""
    return LIB_CHECKED if os.environ.get("LBMICE_CHECKED") == "1" else LIB


def lib():
    """Load liblbmice.so (built by __graft_entry__.build()); raise if it is missing."""
    global _lib
    if _lib is None:
        path = lib_path()
        if not os.path.exists(path):
            raise RuntimeError(f"{path} is not built; run __graft_entry__.build() first")
        L = ctypes.CDLL(path)
        vp, dp, i32, i64, sz = (ctypes.c_void_p, ctypes.POINTER(ctypes.c_double),
                                ctypes.c_int32, ctypes.c_int64, ctypes.c_size_t)
        pp = ctypes.POINTER(Params)
        L.lbmice_params_default.argtypes = [pp, i32, i32]
        L.lbmice_create.argtypes = [pp, vp, ctypes.POINTER(vp)]
        L.lbmice_init_seed.argtypes = [vp, ctypes.c_double, ctypes.c_double, ctypes.c_double,
                                       ctypes.c_double]
        L.lbmice_set_fields.argtypes = [vp, vp, vp, vp, vp, vp, i32]
        L.lbmice_step.argtypes = [vp, i64]
        L.lbmice_fields.argtypes = [vp, i32, vp, sz, i32]
        L.lbmice_load.argtypes = [vp, i32, vp, sz, i32]
        L.lbmice_stats.argtypes = [vp, dp]
        L.lbmice_sync.argtypes = [vp]
        L.lbmice_steps_done.argtypes = [vp]
        L.lbmice_steps_done.restype = i64
        L.lbmice_destroy.argtypes = [vp]
        L.lbmice_strerror.argtypes = [ctypes.c_int]
        L.lbmice_strerror.restype = ctypes.c_char_p
        L.lbmice_state_bytes.argtypes = [vp]
        L.lbmice_state_bytes.restype = sz
        L.lbmice_last_error.argtypes = []
        L.lbmice_last_error.restype = ctypes.c_char_p
        L.lbmice_tape_create.argtypes = [vp, i32, ctypes.POINTER(vp)]
        L.lbmice_tape_record.argtypes = [vp, i64]
        L.lbmice_tape_steps.argtypes = [vp]
        L.lbmice_tape_steps.restype = i64
        L.lbmice_tape_backward.argtypes = [vp, vp, vp, dp, vp, vp, vp, vp, vp]
        L.lbmice_tape_destroy.argtypes = [vp]
        L.lbmice_debug_flags.argtypes = [ctypes.POINTER(ctypes.c_uint32), i32]
        L.lbmice_debug_set_margin.argtypes = [i64]
        L.lbmice_debug_wait_selftest.argtypes = []
        L.lbmice_tips.argtypes = [vp, ctypes.c_double, ctypes.c_double, ctypes.c_double, i32,
                                  dp, dp]
        _lib = L
    return _lib


def strerror(code: int) -> str:
    try:
        return lib().lbmice_strerror(int(code)).decode()
    except RuntimeError:
        return "error"


def _check(rc: int, what: str):
    if rc != OK:
        raise LbmiceError(rc, what)


def make_params(nx, ny, *, dx=0.4, dt=0.008, W0=1.0, tau0=1.0, D=2.0, lam=0.0, L_sat=1.0,
                eps=0.05, kappa_N=1.0, U_in=0.0, u_in=0.0, nu=0.016,
                bc=(BC_PERIODIC,) * 4, flow=False, check_every=0, storage="f32", stencil=4,
                fold=6) -> Params:
    p = Params()
    _check(lib().lbmice_params_default(ctypes.byref(p), int(nx), int(ny)), "params_default")
    p.dx, p.dt, p.W0, p.tau0 = dx, dt, W0, tau0
    p.D, p.lam, p.L_sat, p.eps, p.kappa_N = D, lam, L_sat, eps, kappa_N
    p.U_in, p.u_in, p.nu = U_in, u_in, nu
    for i in range(4):
        p.bc[i] = int(bc[i])
    p.flow = 1 if flow else 0
    p.check_every = int(check_every)
    p.storage = STORAGE[storage] if isinstance(storage, str) else int(storage)
    p.stencil, p.fold = int(stencil), int(fold)
    return p


def _ptr_host(a):
    return None if a is None else a.ctypes.data_as(ctypes.c_void_p)


class Lattice:
    """One grid of the coupled ice-growth solver on the current CUDA device.

    ``stream``: a torch.cuda.Stream (default: the current stream). Keyword parameters are
    those of :func:`make_params`.
    """

    def __init__(self, nx: int, ny: int, *, stream=None, **params):
        import torch
        if not torch.cuda.is_available():
            raise RuntimeError("lbmice needs a CUDA GPU; there is no CPU fallback")
        self.nx, self.ny = int(nx), int(ny)
        self.params = make_params(nx, ny, **params)
        self.flow = bool(self.params.flow)
        self.nplanes = 27 if self.flow else 18
        self._stream = stream if stream is not None else torch.cuda.current_stream()
        self.device = self._stream.device
        h = ctypes.c_void_p()
        with torch.cuda.device(self.device):
            _check(lib().lbmice_create(ctypes.byref(self.params),
                                       ctypes.c_void_p(self._stream.cuda_stream),
                                       ctypes.byref(h)), "lbmice_create")
        self._h = h

    # -- lifetime -------------------------------------------------------------------------
    def close(self):
        if getattr(self, "_h", None):
            _check(lib().lbmice_destroy(self._h), "lbmice_destroy")
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    @property
    def handle(self):
        return self._h

    @property
    def stream(self):
        return self._stream

    # -- initial conditions ---------------------------------------------------------------
    def init_seed(self, cx: float, cy: float, R0: float, U0: float):
        _check(lib().lbmice_init_seed(self._h, cx, cy, R0, U0), "lbmice_init_seed")

    def set_fields(self, phi, U, rho=None, ux=None, uy=None):
        """Moment fields of shape (ny, nx): numpy arrays (host) or float64 CUDA tensors."""
        import torch
        arrs = [phi, U, rho, ux, uy]
        if isinstance(phi, torch.Tensor):
            ts = [None if a is None else a.to(self.device, torch.float64).contiguous()
                  for a in arrs]
            for t in ts:
                if t is not None and tuple(t.shape) != (self.ny, self.nx):
                    raise ValueError("fields must have shape (ny, nx)")
            ptrs = [None if t is None else ctypes.c_void_p(t.data_ptr()) for t in ts]
            _check(lib().lbmice_set_fields(self._h, *ptrs, 1), "lbmice_set_fields")
            self._keep = ts
            return
        ns = [None if a is None else np.ascontiguousarray(a, dtype=np.float64) for a in arrs]
        for a in ns:
            if a is not None and a.shape != (self.ny, self.nx):
                raise ValueError("fields must have shape (ny, nx)")
        _check(lib().lbmice_set_fields(self._h, *[_ptr_host(a) for a in ns], 0),
               "lbmice_set_fields")

    # -- time stepping --------------------------------------------------------------------
    def step(self, n: int = 1):
        _check(lib().lbmice_step(self._h, int(n)), "lbmice_step")

    @property
    def steps_done(self) -> int:
        return int(lib().lbmice_steps_done(self._h))

    def sync(self):
        _check(lib().lbmice_sync(self._h), "lbmice_sync")

    # -- outputs --------------------------------------------------------------------------
    def field(self, which: int, out=None):
        """One moment field as float32. ``out`` may be a CUDA tensor (asynchronous) or a
        C-contiguous float32 numpy array of shape (ny, nx), pinned or pageable, which is
        filled and returned; without it a new host numpy array is returned."""
        if isinstance(out, np.ndarray):
            if (out.dtype != np.float32 or out.shape != (self.ny, self.nx)
                    or not out.flags["C_CONTIGUOUS"]):
                raise ValueError("out must be a C-contiguous float32 array of shape (ny, nx)")
            _check(lib().lbmice_fields(self._h, int(which), _ptr_host(out), out.nbytes, 0),
                   "lbmice_fields")
            return out
        if out is not None:
            if out.numel() * 4 < self.nx * self.ny or out.dtype.itemsize != 4:
                raise ValueError("out must be a float32 tensor of nx*ny elements")
            if not out.is_cuda or out.device != self.device or not out.is_contiguous():
                raise ValueError("out must be a contiguous CUDA tensor on the lattice's device")
            _check(lib().lbmice_fields(self._h, int(which), ctypes.c_void_p(out.data_ptr()),
                                       out.numel() * 4, 1), "lbmice_fields")
            return out
        a = np.empty((self.ny, self.nx), dtype=np.float32)
        _check(lib().lbmice_fields(self._h, int(which), _ptr_host(a), a.nbytes, 0),
               "lbmice_fields")
        return a

    def pops(self) -> np.ndarray:
        """Raw populations (18 or 27, ny, nx): planes h0..h8, g0..g8[, f0..f8]."""
        a = np.empty((self.nplanes, self.ny, self.nx), dtype=np.float32)
        _check(lib().lbmice_fields(self._h, POPS, _ptr_host(a), a.nbytes, 0), "lbmice_fields")
        return a

    def load(self, which: int, arr: np.ndarray):
        a = np.ascontiguousarray(arr, dtype=np.float32)
        _check(lib().lbmice_load(self._h, int(which), _ptr_host(a), a.nbytes, 0),
               "lbmice_load")

    def state(self) -> np.ndarray:
        """The exact state in its storage format (opaque bytes), for checkpoints."""
        a = np.empty(int(lib().lbmice_state_bytes(self._h)), dtype=np.uint8)
        _check(lib().lbmice_fields(self._h, STATE, _ptr_host(a), a.nbytes, 0), "lbmice_fields")
        return a

    def load_state(self, blob: np.ndarray):
        a = np.ascontiguousarray(blob, dtype=np.uint8)
        _check(lib().lbmice_load(self._h, STATE, _ptr_host(a), a.nbytes, 0), "lbmice_load")

    def tips(self, cx: float, cy: float, angles_deg, step: float = 0.25) -> np.ndarray:
        """Distance from (cx, cy) to the first phi = 0 crossing along each ray (degrees),
        computed on the device from the current phi (include/lbmice.h, lbmice_tips)."""
        a = np.ascontiguousarray(np.atleast_1d(angles_deg), dtype=np.float64)
        out = np.empty_like(a)
        _check(lib().lbmice_tips(self._h, float(cx), float(cy), float(step), int(a.size),
                                 a.ctypes.data_as(ctypes.POINTER(ctypes.c_double)),
                                 out.ctypes.data_as(ctypes.POINTER(ctypes.c_double))),
               "lbmice_tips")
        return out

    def stats(self) -> dict:
        out = (ctypes.c_double * NSTATS)()
        _check(lib().lbmice_stats(self._h, out), "lbmice_stats")
        return dict(zip(STAT_NAMES, list(out)))


SHAPES = {0: "march", 1: "32x8", 2: "64x4", 3: "16x16"}  # LBMICE_SHAPE_*
BATCH_MAX_PER_LAUNCH = 64  # members one batched launch carries (LBMICE_BATCH_MAX_PER_LAUNCH)


class _Member(Lattice):
    """A member grid of a Batch (borrowed handle: the batch owns and destroys it)."""

    def __init__(self, batch, i, h, params):
        self.nx, self.ny = int(params.nx), int(params.ny)
        self.params = params
        self.flow = bool(params.flow)
        self.nplanes = 27 if self.flow else 18
        self._stream = batch.stream
        self.device = batch.device
        self._h = ctypes.c_void_p(h)
        self._batch = batch

    def close(self):  # owned by the batch
        self._h = None

    def step(self, n: int = 1):
        raise RuntimeError("members advance through Batch.step")


class Batch:
    """Many grids advanced together, one kernel launch per step for each shape in use
    (include/lbmice.h, lbmice_batch_*). ``configs``: a list of keyword dicts, each with nx, ny
    and the make_params keywords of one member; all share flow and storage."""

    def __init__(self, configs, *, stream=None):
        import torch
        if not torch.cuda.is_available():
            raise RuntimeError("lbmice needs a CUDA GPU; there is no CPU fallback")
        L = lib()
        L.lbmice_batch_create.argtypes = [ctypes.POINTER(Params), ctypes.c_int32,
                                          ctypes.c_void_p, ctypes.POINTER(ctypes.c_void_p)]
        L.lbmice_batch_size.argtypes = [ctypes.c_void_p]
        L.lbmice_batch_size.restype = ctypes.c_int32
        L.lbmice_batch_member.argtypes = [ctypes.c_void_p, ctypes.c_int32]
        L.lbmice_batch_member.restype = ctypes.c_void_p
        L.lbmice_batch_step.argtypes = [ctypes.c_void_p, ctypes.c_int64]
        L.lbmice_batch_autotune.argtypes = [ctypes.c_void_p, ctypes.c_int32,
                                            ctypes.POINTER(ctypes.c_int32),
                                            ctypes.POINTER(ctypes.c_int64)]
        L.lbmice_batch_set_shape.argtypes = [ctypes.c_void_p, ctypes.c_int32, ctypes.c_int32]
        L.lbmice_batch_destroy.argtypes = [ctypes.c_void_p]
        cfgs = [dict(c) for c in configs]
        n = len(cfgs)
        arr = (Params * n)()
        for i, c in enumerate(cfgs):
            nx, ny = c.pop("nx"), c.pop("ny")
            arr[i] = make_params(nx, ny, **c)
        self.stream = stream if stream is not None else torch.cuda.current_stream()
        self.device = self.stream.device
        h = ctypes.c_void_p()
        with torch.cuda.device(self.device):
            _check(L.lbmice_batch_create(arr, n, ctypes.c_void_p(self.stream.cuda_stream),
                                         ctypes.byref(h)), "lbmice_batch_create")
        self._h = h
        self._params = arr
        self.members = [_Member(self, i, L.lbmice_batch_member(h, i), arr[i]) for i in range(n)]
        self.shapes = [0] * n

    def __len__(self):
        return len(self.members)

    def __getitem__(self, i) -> Lattice:
        return self.members[i]

    def step(self, n: int = 1):
        _check(lib().lbmice_batch_step(self._h, int(n)), "lbmice_batch_step")

    def autotune(self, steps_per_trial: int = 6):
        """Pick a shape per grid size; returns (shapes, steps_taken)."""
        n = len(self.members)
        shapes = (ctypes.c_int32 * n)()
        taken = ctypes.c_int64()
        _check(lib().lbmice_batch_autotune(self._h, int(steps_per_trial), shapes,
                                           ctypes.byref(taken)), "lbmice_batch_autotune")
        self.shapes = list(shapes)
        return list(shapes), int(taken.value)

    def set_shape(self, i: int, shape: int):
        _check(lib().lbmice_batch_set_shape(self._h, int(i), int(shape)), "lbmice_batch_set_shape")
        self.shapes[i] = int(shape)

    @property
    def launches_per_step(self) -> int:
        """Kernel launches of one batched step: per shape in use, one per
        BATCH_MAX_PER_LAUNCH members of that shape."""
        return sum(-(-self.shapes.count(s) // BATCH_MAX_PER_LAUNCH) for s in SHAPES)

    @property
    def nodes(self) -> int:
        return sum(m.nx * m.ny for m in self.members)

    def sync(self):
        self.members[0].sync()

    def close(self):
        if getattr(self, "_h", None):
            for m in self.members:
                m.close()
            _check(lib().lbmice_batch_destroy(self._h), "lbmice_batch_destroy")
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


GRAD_NAMES = ("eps", "D", "lambda")
INIT_NAMES = ("phi0", "U0", "rho0", "ux0", "uy0")


class Tape:
    """Checkpointed record of a :class:`Lattice` and the discrete adjoint of its steps
    (include/lbmice.h, lbmice_tape_*). The lattice must be freshly initialised (step 0) and
    is advanced through :meth:`record` only."""

    def __init__(self, lattice: Lattice, every: int = 100):
        h = ctypes.c_void_p()
        _check(lib().lbmice_tape_create(lattice.handle, int(every), ctypes.byref(h)),
               "lbmice_tape_create")
        self._h = h
        self.lattice = lattice
        self.every = int(every)

    def record(self, n: int):
        _check(lib().lbmice_tape_record(self._h, int(n)), "lbmice_tape_record")

    @property
    def steps(self) -> int:
        return int(lib().lbmice_tape_steps(self._h))

    def backward(self, phi_bar=None, U_bar=None):
        """Reverse sweep from dL/dphi_T and dL/dU_T, (ny, nx) arrays: numpy (host results)
        or CUDA tensors (device results). Returns ({eps, D, lambda}, {phi0, U0, rho0, ux0,
        uy0}) with float32 fields of shape (ny, nx)."""
        import torch
        lat = self.lattice
        shape = (lat.ny, lat.nx)
        on_dev = any(isinstance(a, torch.Tensor) for a in (phi_bar, U_bar))
        keep = []

        def seed(a):
            if a is None:
                return None
            if on_dev:
                t = torch.as_tensor(a, device=lat.device).to(torch.float32).contiguous()
                if tuple(t.shape) != shape:
                    raise ValueError("seeds must have shape (ny, nx)")
                keep.append(t)
                return ctypes.c_void_p(t.data_ptr())
            n = np.ascontiguousarray(a, dtype=np.float32)
            if n.shape != shape:
                raise ValueError("seeds must have shape (ny, nx)")
            keep.append(n)
            return _ptr_host(n)

        sp, su = seed(phi_bar), seed(U_bar)
        if on_dev:
            outs = [torch.empty(shape, dtype=torch.float32, device=lat.device) for _ in INIT_NAMES]
            ptrs = [ctypes.c_void_p(o.data_ptr()) for o in outs]
        else:
            outs = [np.empty(shape, dtype=np.float32) for _ in INIT_NAMES]
            ptrs = [_ptr_host(o) for o in outs]
        g = (ctypes.c_double * 3)()
        _check(lib().lbmice_tape_backward(self._h, sp, su, g, *ptrs), "lbmice_tape_backward")
        return dict(zip(GRAD_NAMES, list(g))), dict(zip(INIT_NAMES, outs))

    def close(self):
        if getattr(self, "_h", None):
            _check(lib().lbmice_tape_destroy(self._h), "lbmice_tape_destroy")
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def debug_flags(clear: bool = True) -> int:
    """The checked build's violation word (OOB_* bits), reset if clear; raises LbmiceError
    (ENOTSUP) with the normal library."""
    w = ctypes.c_uint32()
    _check(lib().lbmice_debug_flags(ctypes.byref(w), int(bool(clear))), "lbmice_debug_flags")
    return int(w.value)


def debug_set_margin(margin: int):
    """Checked build: shrink every extent its index tests use by margin elements."""
    _check(lib().lbmice_debug_set_margin(int(margin)), "lbmice_debug_set_margin")

"""TEST INFRASTRUCTURE ONLY: Python handle on the plain FP64 CPU oracle (``lbm_oracle.cpp``).

The oracle is the coupled lattice-Boltzmann ice-growth step of Tan et al. (arXiv 2101.07163,
Sec. 2.2) written as plain loops in double precision. Only ``tests/``,
``__graft_entry__.smoke()`` and the CPU-baseline leg of ``bench.py`` may import this package.
It shares no code with the CUDA path; both receive the same seeded moment fields.

Fields are numpy arrays of shape ``(ny, nx)`` (row ``y``, column ``x``); population arrays
are ``(9, ny, nx)`` in the D2Q9 order c = (0,0) (1,0) (0,1) (-1,0) (0,-1) (1,1) (-1,1)
(-1,-1) (1,-1).
"""
from __future__ import annotations

import ctypes
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "lbm_oracle.cpp")
_LIB = os.path.join(_HERE, "liboracle.so")

BC_PERIODIC, BC_INLET, BC_OUTLET, BC_FREESLIP = 0, 1, 2, 3
PHI, U, RHO, UX, UY, PHI_PREV = 0, 1, 2, 3, 4, 5
LAT_F, LAT_G, LAT_H, LAT_AS2 = 0, 1, 2, 3


class OrcParams(ctypes.Structure):
    _fields_ = [
        ("nx", ctypes.c_int32), ("ny", ctypes.c_int32),
        ("dx", ctypes.c_double), ("dt", ctypes.c_double),
        ("W0", ctypes.c_double), ("tau0", ctypes.c_double),
        ("D", ctypes.c_double), ("lam", ctypes.c_double),
        ("L_sat", ctypes.c_double), ("eps", ctypes.c_double),
        ("kappa_N", ctypes.c_double),
        ("U_in", ctypes.c_double), ("u_in", ctypes.c_double), ("nu", ctypes.c_double),
        ("bc", ctypes.c_int32 * 4), ("flow", ctypes.c_int32),
        ("stencil", ctypes.c_int32), ("fold", ctypes.c_int32),
    ]


def build(force: bool = False) -> str:
    """Compile the oracle with g++ (-O2, no fast-math, no FMA contraction); return the path."""
    if not force and os.path.exists(_LIB) and os.path.getmtime(_LIB) >= os.path.getmtime(_SRC):
        return _LIB
    tmp = _LIB + ".tmp%d" % os.getpid()
    cmd = ["g++", "-O2", "-std=c++17", "-ffp-contract=off", "-fno-fast-math", "-fopenmp",
           "-fPIC", "-shared", "-o", tmp, _SRC]
    subprocess.run(cmd, check=True)
    os.replace(tmp, _LIB)
    return _LIB


_lib = None


def lib():
    global _lib
    if _lib is None:
        L = ctypes.CDLL(build())
        vp, dp, i32, i64 = ctypes.c_void_p, ctypes.POINTER(ctypes.c_double), ctypes.c_int, ctypes.c_int64
        L.orc_create.restype = vp
        L.orc_create.argtypes = [ctypes.POINTER(OrcParams)]
        L.orc_destroy.argtypes = [vp]
        L.orc_derived.argtypes = [vp, dp]
        L.orc_set_fields.argtypes = [vp, dp, dp, dp, dp, dp]
        L.orc_step.argtypes = [vp, i64]
        L.orc_round_f32.argtypes = [vp]
        L.orc_set_threads.argtypes = [i32]
        L.orc_set_threads.restype = i32
        L.orc_set_threads(1)
        L.orc_steps_done.argtypes = [vp]
        L.orc_steps_done.restype = i64
        L.orc_get_field.argtypes = [vp, i32, dp]
        L.orc_get_pops.argtypes = [vp, i32, dp]
        L.orc_set_pops.argtypes = [vp, i32, dp]
        L.orc_post_collision.argtypes = [vp, i32, dp]
        L.orc_gradient_periodic.argtypes = [dp, i32, i32, dp, dp]
        L.orc_anisotropy.argtypes = [ctypes.c_double, ctypes.c_double, ctypes.c_double,
                                     ctypes.c_double, dp]
        L.orc_anisotropy_fold.argtypes = [ctypes.c_double, ctypes.c_double, ctypes.c_double,
                                          ctypes.c_double, i32, dp]
        L.orc_gradient_stencil.argtypes = [dp, i32, i32, i32, dp, dp]
        L.orc_grad_run.argtypes = ([ctypes.POINTER(OrcParams)] + [dp] * 10 +
                                   [i64, dp, dp, i32, dp, dp])
        _lib = L
    return _lib


def set_threads(n: int) -> int:
    """Host threads of the oracle's node loops (rows split statically; results are
    bit-identical for any count). Returns the count in use."""
    return int(lib().orc_set_threads(int(n)))


def _dp(a):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_double)) if a is not None else None


def _f64(a):
    return None if a is None else np.ascontiguousarray(a, dtype=np.float64)


def make_params(nx, ny, *, dx=0.4, dt=0.008, W0=1.0, tau0=1.0, D=2.0, lam=0.0, L_sat=1.0,
                eps=0.05, kappa_N=1.0, U_in=0.0, u_in=0.0, nu=0.016,
                bc=(BC_PERIODIC,) * 4, flow=False, stencil=4, fold=6) -> OrcParams:
    p = OrcParams()
    p.nx, p.ny = int(nx), int(ny)
    p.dx, p.dt, p.W0, p.tau0 = dx, dt, W0, tau0
    p.D, p.lam, p.L_sat, p.eps, p.kappa_N = D, lam, L_sat, eps, kappa_N
    p.U_in, p.u_in, p.nu = U_in, u_in, nu
    for i in range(4):
        p.bc[i] = int(bc[i])
    p.flow = 1 if flow else 0
    p.stencil, p.fold = int(stencil), int(fold)
    return p


class Oracle:
    """One oracle grid. ``params`` is an :class:`OrcParams` or the keywords of make_params."""

    def __init__(self, params: OrcParams | None = None, **kw):
        if params is None:
            params = make_params(**kw)
        self.p = params
        self.nx, self.ny = params.nx, params.ny
        self._h = lib().orc_create(ctypes.byref(params))
        if not self._h:
            raise ValueError("oracle rejected the parameters")

    def __del__(self):
        h = getattr(self, "_h", None)
        if h:
            lib().orc_destroy(h)
            self._h = None

    @property
    def flow(self) -> bool:
        return bool(self.p.flow)

    def derived(self) -> dict:
        out = np.zeros(6)
        lib().orc_derived(self._h, _dp(out))
        return dict(zip(["Dphi", "dt_tau0", "Dlat", "Wlat", "lambda", "tau_f"], out.tolist()))

    def set_fields(self, phi, U, rho=None, ux=None, uy=None):
        arrs = [_f64(a) for a in (phi, U, rho, ux, uy)]
        for a in arrs:
            if a is not None and a.shape != (self.ny, self.nx):
                raise ValueError("field shape must be (ny, nx)")
        self._keep = arrs
        rc = lib().orc_set_fields(self._h, *[_dp(a) for a in arrs])
        if rc:
            raise RuntimeError("orc_set_fields failed")

    def step(self, n: int = 1):
        if lib().orc_step(self._h, int(n)):
            raise RuntimeError("orc_step failed")

    @property
    def steps_done(self) -> int:
        return int(lib().orc_steps_done(self._h))

    def field(self, which: int) -> np.ndarray:
        out = np.zeros((self.ny, self.nx))
        if lib().orc_get_field(self._h, int(which), _dp(out)):
            raise RuntimeError("orc_get_field failed")
        return out

    def pops(self, lattice: int) -> np.ndarray:
        out = np.zeros((9, self.ny, self.nx))
        if lib().orc_get_pops(self._h, int(lattice), _dp(out)):
            raise RuntimeError("orc_get_pops failed")
        return out

    def set_pops(self, lattice: int, arr) -> None:
        a = _f64(arr)
        if lib().orc_set_pops(self._h, int(lattice), _dp(a)):
            raise RuntimeError("orc_set_pops failed")

    def round_to_float32(self) -> None:
        """Test option: round every population and the phi history to float32 in place (the
        storage precision of an FP32 run); the next step computes in double as always."""
        if lib().orc_round_f32(self._h):
            raise RuntimeError("orc_round_f32 failed")

    def post_collision(self, lattice: int) -> np.ndarray:
        shape = (self.ny, self.nx) if lattice == LAT_AS2 else (9, self.ny, self.nx)
        out = np.zeros(shape)
        if lib().orc_post_collision(self._h, int(lattice), _dp(out)):
            raise RuntimeError("orc_post_collision failed")
        return out


def gradient_periodic(phi) -> tuple[np.ndarray, np.ndarray]:
    """E4 isotropic gradient (lattice units) of a periodic field, by the oracle."""
    a = _f64(phi)
    ny, nx = a.shape
    gx, gy = np.zeros_like(a), np.zeros_like(a)
    lib().orc_gradient_periodic(_dp(a), nx, ny, _dp(gx), _dp(gy))
    return gx, gy


def anisotropy(gx: float, gy: float, eps: float, kappa_N: float = 1.0):
    """(a_s, N_x, N_y) of the oracle for one gradient vector."""
    out = np.zeros(3)
    lib().orc_anisotropy(float(gx), float(gy), float(eps), float(kappa_N), _dp(out))
    return float(out[0]), float(out[1]), float(out[2])


GRAD_KEYS = ("eps", "D", "lambda", "init")


def grad_run(params: OrcParams, fields: dict, nsteps: int, wphi, wU, dfields: dict | None = None,
             round_f32: bool = False, along=None):
    """Exact forward-mode derivatives of L = sum(wphi * phi_T + wU * U_T) after ``nsteps``
    steps from the equilibrium state of ``fields`` (keys phi, U and optionally rho, ux, uy),
    with respect to eps, D (through D_lat and, if lambda is not given, the beta = 0 lambda),
    lambda alone, and the initial moments along ``dfields`` (same keys; missing = 0).
    ``round_f32``: the state's values are rounded to float32 after every step (derivatives
    kept), i.e. the derivatives along a float32-stored trajectory. ``along``: states to
    differentiate along, shape (nsteps + 1, planes, ny, nx) -- the initial state and the
    state after every step -- with planes h0..h8, g0..g8, [f0..f8,] phi, phi history; before
    every step the state's values and the collision's phi values are replaced by them.
    Returns {"L": ..., "eps": ..., "D": ..., "lambda": ..., "init": ...}."""
    n = params.nx * params.ny
    dfields = dfields or {}
    f = {k: _f64(fields.get(k)) for k in ("phi", "U", "rho", "ux", "uy")}
    df = {}
    for k in ("phi", "U", "rho", "ux", "uy"):
        v = dfields.get(k)
        df[k] = _f64(v) if v is not None else (np.zeros(n) if k in ("phi", "U") else None)
    w1, w2 = _f64(wphi), _f64(wU)
    tr = None
    if along is not None:
        tr = _f64(along)
        planes = (27 if params.flow else 18) + 2
        if tr.shape != (nsteps + 1, planes, params.ny, params.nx):
            raise ValueError("along must have shape (nsteps + 1, planes, ny, nx)")
    out = np.zeros(5)
    rc = lib().orc_grad_run(ctypes.byref(params), _dp(f["phi"]), _dp(f["U"]), _dp(f["rho"]),
                            _dp(f["ux"]), _dp(f["uy"]), _dp(df["phi"]), _dp(df["U"]),
                            _dp(df["rho"]), _dp(df["ux"]), _dp(df["uy"]), int(nsteps),
                            _dp(w1), _dp(w2), 1 if round_f32 else 0, _dp(tr), _dp(out))
    if rc != 0:
        raise ValueError("oracle rejected the gradient run")
    return dict(zip(("L",) + GRAD_KEYS, out.tolist()))


def gradient_stencil(phi, stencil: int = 4) -> tuple[np.ndarray, np.ndarray]:
    """Gradient of a periodic field with the E2 / E4 / E6 / E8 stencil (Sec. 3.1.1)."""
    f = np.ascontiguousarray(phi, dtype=np.float64)
    ny, nx = f.shape
    gx, gy = np.empty_like(f), np.empty_like(f)
    if lib().orc_gradient_stencil(_dp(f), nx, ny, int(stencil), _dp(gx), _dp(gy)) != 0:
        raise ValueError("bad stencil")
    return gx, gy


def anisotropy_fold(gx: float, gy: float, eps: float, kappa_N: float = 1.0, fold: int = 6):
    """(a_s, N_x, N_y) for an anisotropy of the given symmetry fold (4 or 6)."""
    out = np.zeros(3)
    if lib().orc_anisotropy_fold(gx, gy, eps, kappa_N, int(fold), _dp(out)) != 0:
        raise ValueError("bad fold")
    return tuple(out.tolist())

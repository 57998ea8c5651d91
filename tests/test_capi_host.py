"""The C-ABI library on the host: it builds, loads, exports every declared entry point, and
rejects bad arguments before touching the GPU."""
import ctypes
import os
import re
import subprocess

import pytest

from paper_2101_07163_gb300 import build, lbmice

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def L():
    build.build()
    return lbmice.lib()


def declared_entry_points():
    names = set()
    for fn in os.listdir(os.path.join(ROOT, "include")):
        if fn.endswith(".h"):
            text = open(os.path.join(ROOT, "include", fn)).read()
            names |= set(re.findall(r"^\s*(?:int|int64_t|size_t|const char\*)\s+(\w+)\s*\(",
                                    text, re.M))
    return sorted(names)


def test_library_exports_every_declared_symbol(L):
    decl = declared_entry_points()
    assert len(decl) >= 12
    out = subprocess.run(["nm", "-D", "--defined-only", build.LIB], capture_output=True,
                         text=True, check=True).stdout
    exported = set(re.findall(r"\bT\s+(\w+)$", out, re.M))
    missing = [n for n in decl if n not in exported]
    assert not missing, missing
    for n in decl:
        assert hasattr(L, n)


def test_library_is_built_for_sm_103a_only():
    flags = " ".join(build.NVCC_FLAGS)
    assert re.findall(r"arch=(\S+)", flags) == ["compute_103a,code=sm_103a"]


def test_params_default_and_strerror(L):
    p = lbmice.Params()
    assert L.lbmice_params_default(ctypes.byref(p), 64, 48) == 0
    assert (p.nx, p.ny, p.dx, p.dt, p.W0, p.tau0) == (64, 48, 0.4, 0.008, 1.0, 1.0)
    assert list(p.bc) == [0, 0, 0, 0] and p.flow == 0 and p.eps == 0.05
    assert L.lbmice_params_default(None, 4, 4) == lbmice.EINVAL
    for code in (0, -1, -2, -3, -4, -5, -6):
        assert L.lbmice_strerror(code)
    assert L.lbmice_strerror(-99) == b"unknown error"


@pytest.mark.parametrize("change, code", [
    (dict(nx=3), lbmice.EINVAL),
    (dict(ny=0), lbmice.EINVAL),
    (dict(dx=0.0), lbmice.EINVAL),
    (dict(tau0=-1.0), lbmice.EINVAL),
    (dict(eps=1.0), lbmice.EINVAL),
    (dict(D=-0.1), lbmice.EINVAL),
    (dict(bc=(0, 1, 0, 0)), lbmice.EINVAL),   # periodic on one face only
    (dict(bc=(7, 7, 0, 0)), lbmice.EINVAL),
    (dict(flow=True, nu=0.0), lbmice.EUNSTABLE),
    (dict(flow=True, u_in=0.6, bc=(1, 2, 3, 3)), lbmice.EUNSTABLE),
    (dict(check_every=-1), lbmice.EINVAL),
    (dict(storage=3), lbmice.EINVAL),
    (dict(stencil=3), lbmice.EINVAL),
    (dict(fold=5), lbmice.EINVAL),
    (dict(nx=46368, ny=46320), lbmice.EINVAL),  # pitch * ny = 2^31 + 282112 nodes: too many
])
def test_create_rejects_bad_parameters_without_a_gpu(L, change, code):
    kw = dict(nx=16, ny=16)
    kw.update(change)
    p = lbmice.make_params(**kw)
    h = ctypes.c_void_p(123)
    assert L.lbmice_create(ctypes.byref(p), None, ctypes.byref(h)) == code
    assert h.value is None


def test_null_handles_are_rejected(L):
    assert L.lbmice_create(None, None, None) == lbmice.EINVAL
    assert L.lbmice_step(None, 1) == lbmice.EINVAL
    assert L.lbmice_init_seed(None, 1.0, 1.0, 1.0, 0.1) == lbmice.EINVAL
    assert L.lbmice_fields(None, 0, None, 0, 0) == lbmice.EINVAL
    assert L.lbmice_load(None, 6, None, 0, 0) == lbmice.EINVAL
    assert L.lbmice_stats(None, None) == lbmice.EINVAL
    assert L.lbmice_set_fields(None, None, None, None, None, None, 0) == lbmice.EINVAL
    assert L.lbmice_sync(None) == lbmice.EINVAL
    assert L.lbmice_tips(None, 0.0, 0.0, 0.25, 1, None, None) == lbmice.EINVAL
    assert L.lbmice_steps_done(None) == -1
    assert L.lbmice_state_bytes(None) == 0
    assert L.lbmice_destroy(None) == 0


def test_tape_rejects_null_arguments(L):
    import ctypes
    out = ctypes.c_void_p(1)
    assert L.lbmice_tape_create(None, 10, ctypes.byref(out)) == lbmice.EINVAL
    assert out.value is None  # *out is cleared on error
    assert L.lbmice_tape_create(None, 10, None) == lbmice.EINVAL
    assert L.lbmice_tape_record(None, 1) == lbmice.EINVAL
    assert L.lbmice_tape_steps(None) == -1
    assert L.lbmice_tape_backward(None, None, None, None, None, None, None, None,
                                  None) == lbmice.EINVAL
    assert L.lbmice_tape_destroy(None) == 0


def test_lattice_refuses_to_run_without_cuda():
    import torch
    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    with pytest.raises(RuntimeError, match="no CPU fallback"):
        lbmice.Lattice(16, 16)


def test_normal_library_reports_that_it_has_no_checks():
    # the bounds-checked entry points exist in every build; without -DLBMICE_CHECKED they
    # touch no device and answer ENOTSUP
    L = lbmice.lib()
    w = ctypes.c_uint32(7)
    assert L.lbmice_debug_flags(ctypes.byref(w), 1) == lbmice.ENOTSUP and w.value == 0
    assert L.lbmice_debug_flags(None, 0) == lbmice.EINVAL
    assert L.lbmice_debug_flags(ctypes.byref(w), 2) == lbmice.EINVAL
    assert L.lbmice_debug_set_margin(0) == lbmice.ENOTSUP
    assert L.lbmice_debug_set_margin(-1) == lbmice.EINVAL

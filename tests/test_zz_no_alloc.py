"""lbmice_stats_noalloc: the FP64 diagnostics for callers that cannot allocate device memory.

Such callers (an application whose device memory is reserved up front by its own pool
allocator, or a time-critical loop that cannot afford cudaMalloc's synchronisation) pass
their own state buffers and output; the reduction keeps its partial sums in a fixed device
array instead of allocating. This test calls the entry point through the C ABI twice in a
row, on two different states, and checks each result against lbmice_stats (the existing
entry point, which uses memory owned by the handle) within the tolerance of the other
reduction tests. It sits in a file of its own, collected last.
"""
import ctypes

import numpy as np
import pytest

from paper_2101_07163_gb300 import lbmice
from paper_2101_07163_gb300 import workloads as W

pytestmark = pytest.mark.gpu

NAMES = ("area", "mass", "vapour_invariant", "sum_phi", "nonfinite")


def noalloc_fn():
    f = lbmice.lib().lbmice_stats_noalloc
    f.argtypes = ([ctypes.c_void_p] * 3 + [ctypes.c_int32] * 4
                  + [ctypes.c_double, ctypes.c_double, ctypes.c_void_p, ctypes.c_void_p])
    f.restype = ctypes.c_int
    return f


def export_state(lat, torch):
    """Copy the lattice's state into caller-owned device buffers (row pitch = nx)."""
    pops = torch.empty((lat.nplanes, lat.ny, lat.nx), device="cuda", dtype=torch.float32)
    rc = lbmice.lib().lbmice_fields(lat.handle, lbmice.POPS, ctypes.c_void_p(pops.data_ptr()),
                                    pops.numel() * 4, 1)
    assert rc == 0
    phi = torch.empty((lat.ny, lat.nx), device="cuda", dtype=torch.float32)
    prev = torch.empty((lat.ny, lat.nx), device="cuda", dtype=torch.float32)
    lat.field(lbmice.PHI, out=phi)
    lat.field(lbmice.PHI_PREV, out=prev)
    return pops, phi, prev


def test_noalloc_stats_match_stats_on_two_calls_in_a_row():
    torch = pytest.importorskip("torch")
    w = W.Workload("noalloc", 300, 200, 1, flow=True, eps=0.06, D=2.0, U0=0.4, nu=0.05,
                   L_sat=1.3, cx=140.0, cy=90.0, R0=12.0)
    lat = lbmice.Lattice(w.nx, w.ny, **w.params())
    lat.set_fields(**W.perturbed_fields(w, 31))
    lat.step(30)
    fn = noalloc_fn()
    out = torch.full((5,), -1.0, device="cuda", dtype=torch.float64)
    stream = ctypes.c_void_p(lat.stream.cuda_stream)
    seen = []
    for call in range(2):
        ref = lat.stats()
        pops, phi, prev = export_state(lat, torch)
        rc = fn(ctypes.c_void_p(pops.data_ptr()), ctypes.c_void_p(phi.data_ptr()),
                ctypes.c_void_p(prev.data_ptr()), w.nx, w.ny, w.nx, 1, w.dx, w.L_sat,
                ctypes.c_void_p(out.data_ptr()), stream)
        assert rc == lbmice.OK, lbmice.strerror(rc)
        torch.cuda.synchronize()
        got = out.cpu().numpy()
        for k, name in enumerate(NAMES):
            assert got[k] == pytest.approx(ref[name], rel=1e-12, abs=1e-9), (call, name)
        seen.append(got.copy())
        lat.step(25)  # the second call sees a different state
    assert not np.array_equal(seen[0], seen[1])


def padded(t, pitch, torch):
    """t (..., ny, nx) copied into rows of pitch floats; the padding holds NaN, which a sum
    that read it would carry into its result."""
    p = torch.full(tuple(t.shape[:-1]) + (pitch,), float("nan"), device="cuda",
                   dtype=torch.float32)
    p[..., :t.shape[-1]] = t
    return p.contiguous()


@pytest.mark.parametrize("flow", [True, False])
def test_noalloc_reads_padded_rows_with_and_without_flow(flow):
    # Rows of pitch = nx + 13 floats (plane stride pitch * ny), and a grid without the flow
    # lattice (18 planes; the mass is then the node count): the same five values as
    # lbmice_stats.
    torch = pytest.importorskip("torch")
    w = W.Workload("noalloc_pad", 150, 77, 1, flow=flow, eps=0.05, D=2.0, U0=0.35, nu=0.05,
                   cx=70.0, cy=40.0, R0=9.0)
    lat = lbmice.Lattice(w.nx, w.ny, **w.params())
    lat.set_fields(**W.perturbed_fields(w, 33))
    lat.step(12)
    ref = lat.stats()
    pops, phi, prev = export_state(lat, torch)
    pitch = w.nx + 13
    pp, ph, pv = padded(pops, pitch, torch), padded(phi, pitch, torch), padded(prev, pitch, torch)
    out = torch.full((5,), -1.0, device="cuda", dtype=torch.float64)
    rc = noalloc_fn()(ctypes.c_void_p(pp.data_ptr()), ctypes.c_void_p(ph.data_ptr()),
                      ctypes.c_void_p(pv.data_ptr()), w.nx, w.ny, pitch, 1 if flow else 0,
                      w.dx, w.L_sat, ctypes.c_void_p(out.data_ptr()),
                      ctypes.c_void_p(lat.stream.cuda_stream))
    assert rc == lbmice.OK, lbmice.strerror(rc)
    torch.cuda.synchronize()
    got = out.cpu().numpy()
    for k, name in enumerate(NAMES):
        assert got[k] == pytest.approx(ref[name], rel=1e-12, abs=1e-9), (flow, name)
    if not flow:
        assert got[1] == w.nx * w.ny


def test_noalloc_rejects_grids_beyond_its_fixed_array():
    fn = noalloc_fn()
    dummy = ctypes.c_void_p(16)  # never dereferenced: the size check comes first
    big = 4097
    assert big * 4096 > 2048 * 8192
    rc = fn(dummy, dummy, dummy, big, 4096, big, 1, 0.4, 1.0, dummy, None)
    assert rc == lbmice.EINVAL

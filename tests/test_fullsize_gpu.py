"""The plate-regime workload at its full size after 2048 steps, against the FP64 oracle.

2048 x 2048 periodic, f + g + h, seed R0 = 10 at the centre, U0 = 0.5, eps = 0.05, D = 3
(the benchmarked workload), from the same seed fields on both sides; the oracle's rows are
split over every host core (bit-identical to one thread). For FP32, FP16 and BF16 storage:
  - max |dphi| and max |dU| over the whole grid at step 2048, within the bounds the 2000-step
    seed tests use (FP32 2e-4, FP16 3e-4, BF16 3e-3; a 160 x 160 copy of the same physics
    measures 4.1e-5, 6.7e-5 and 2.4e-4 in phi);
  - tip speed (the phi = 0 crossing along the six arm directions, steps 1024 -> 2048)
    within 1%, and solid area sum (1 + phi)/2 dx^2 within 0.5%: the long-horizon gates.
The measured values are printed (pytest -s) for the design notes.
"""
import numpy as np
import pytest

import oracle
from paper_2101_07163_gb300 import lbmice
from paper_2101_07163_gb300 import workloads as W
from tests.helpers import contour_radius, oracle_threads

pytestmark = [pytest.mark.gpu, pytest.mark.slow]

T_MID, T_END = 1024, 2048
BOUND = {"f32": 2e-4, "f16": 3e-4, "bf16": 3e-3}
ARMS = np.deg2rad(np.arange(0.0, 360.0, 60.0))


def measures(phi_mid, phi_end, w):
    """Mean tip speed of the six arms (cells per step) and the solid area at the end."""
    r0 = contour_radius(phi_mid.astype(np.float64), w.cx, w.cy, ARMS, rmax=200.0)
    r1 = contour_radius(phi_end.astype(np.float64), w.cx, w.cy, ARMS, rmax=200.0)
    speed = float(np.mean(r1 - r0)) / (T_END - T_MID)
    area = float((0.5 * (1.0 + phi_end.astype(np.float64))).sum()) * w.dx ** 2
    return speed, area, r1


@pytest.fixture(scope="module")
def reference():
    w = W.C3
    f = W.seed_fields(w)
    with oracle_threads():
        o = oracle.Oracle(nx=w.nx, ny=w.ny, **w.params())
        o.set_fields(**f)
        o.step(T_MID)
        mid = o.field(oracle.PHI)
        o.step(T_END - T_MID)
        end, U = o.field(oracle.PHI), o.field(oracle.U)
    del o
    return w, f, mid, end, U


@pytest.mark.parametrize("storage", ["f32", "f16", "bf16"])
def test_plate_2048_full_size_2048_steps(storage, reference):
    w, f, mid, end, U = reference
    lat = lbmice.Lattice(w.nx, w.ny, storage=storage, **w.params())
    lat.set_fields(**f)
    lat.step(T_MID)
    gmid = lat.field(lbmice.PHI)
    lat.step(T_END - T_MID)
    gend, gU = lat.field(lbmice.PHI), lat.field(lbmice.U)
    lat.close()
    dphi = float(np.abs(gend.astype(np.float64) - end).max())
    dU = float(np.abs(gU.astype(np.float64) - U).max())
    v_ref, a_ref, r_ref = measures(mid, end, w)
    v, a, r = measures(gmid, gend, w)
    print(f"\n{storage}: max|dphi| {dphi:.3e} max|dU| {dU:.3e} tip speed {v:.6e} "
          f"(oracle {v_ref:.6e}, rel {abs(v - v_ref) / v_ref:.2e}) area {a:.6e} "
          f"(oracle {a_ref:.6e}, rel {abs(a - a_ref) / a_ref:.2e}) tip radius "
          f"{np.mean(r):.4f} (oracle {np.mean(r_ref):.4f})")
    assert dphi < BOUND[storage]
    assert dU < BOUND[storage]
    assert v_ref > 0 and np.all(np.isfinite(r_ref))
    assert abs(v - v_ref) / v_ref < 0.01
    assert abs(a - a_ref) / a_ref < 0.005

"""The method variants on the GPU against the oracle: the gradient stencils E2, E4, E6, E8 of
Sec. 3.1.1 (E6/E8 on a phi tile of halo 3) and the four-fold anisotropy of the validation
system, with every face rule."""
import numpy as np
import pytest

import oracle
from paper_2101_07163_gb300 import lbmice
from paper_2101_07163_gb300 import workloads as W
from tests.test_parity_gpu import (BOXES, channel_workload, compare_moments, compare_pops,
                                   compare_within_floor, fp32_storage_floor, pair)

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("fold", [6, 4])
@pytest.mark.parametrize("stencil", [2, 4, 6, 8])
@pytest.mark.parametrize("box", ["periodic", "channel_x", "walls", "inlet_plus_x"])
def test_one_step_every_stencil_and_fold(stencil, fold, box):
    w = channel_workload(box, 100, 76, BOXES[box], stencil=stencil, fold=fold)
    lat, orc = pair(w, W.perturbed_fields(w, 7, amp_phi=0.3, amp_u=0.02))
    compare_pops(lat, orc, 1e-6)  # the initial equilibria carry the stencil's flux
    lat.step(1)
    orc.step(1)
    compare_pops(lat, orc, 1e-6)
    compare_moments(lat, orc, 1e-6)


@pytest.mark.parametrize("stencil", [6, 8])
@pytest.mark.parametrize("box", ["periodic", "channel_y"])
def test_short_horizon_wide_stencils(stencil, box):
    w = channel_workload(box, 70, 44, BOXES[box], stencil=stencil)
    f = W.perturbed_fields(w, 8, amp_phi=0.2, amp_u=0.01)
    lat = lbmice.Lattice(w.nx, w.ny, **w.params())
    lat.set_fields(**f)
    lat.step(200)
    orc, floor = fp32_storage_floor(w, f, 200)
    compare_within_floor(lat, orc, floor)


def test_four_fold_seed_short_horizon():
    w = W.Workload("ff", 80, 72, 1, eps=0.05, D=4.0, U0=0.55, fold=4, cx=40, cy=36, R0=8.0)
    lat, orc = pair(w, W.seed_fields(w))
    lat.step(200)
    orc.step(200)
    compare_moments(lat, orc, 2e-5)


@pytest.mark.parametrize("stencil", [2, 6, 8])
def test_mirror_symmetry_with_every_stencil_on_gpu(stencil):
    w = W.Workload("m", 64, 48, 1, flow=True, eps=0.07, nu=0.05, stencil=stencil)
    lat = lbmice.Lattice(w.nx, w.ny, **w.params())
    lat.set_fields(**W.mirror_fields(w, 23, amp=0.2))
    lat.step(150)
    ix, iy = (-np.arange(w.nx)) % w.nx, (-np.arange(w.ny)) % w.ny
    for which in (lbmice.PHI, lbmice.U, lbmice.RHO):
        a = lat.field(which)
        np.testing.assert_array_equal(a, a[:, ix])
        np.testing.assert_array_equal(a, a[iy, :])


def test_wide_stencils_and_four_fold_are_refused_where_not_built():
    for kw in (dict(stencil=2), dict(stencil=6), dict(stencil=8), dict(fold=4)):
        wb = W.Workload("b", 40, 40, 1, flow=True, **kw)
        with pytest.raises(lbmice.LbmiceError) as ei:
            lbmice.Batch([dict(nx=40, ny=40, **W.Workload("a", 40, 40, 1, flow=True).params()),
                          dict(nx=40, ny=40, **wb.params())])
        assert ei.value.code == lbmice.EINVAL
    for kw in (dict(stencil=2), dict(stencil=8), dict(fold=4)):
        w = W.Workload("t", 40, 40, 1, flow=True, **kw)
        lat = lbmice.Lattice(w.nx, w.ny, **w.params())
        lat.set_fields(**W.seed_fields(w))
        with pytest.raises(lbmice.LbmiceError) as ei:
            lbmice.Tape(lat)
        assert ei.value.code == lbmice.EINVAL


def ray_tip(phi, cx, cy, ang, step=0.25):
    """Distance from (cx, cy) along angle ang to the phi = 0 crossing (bilinear samples)."""
    import math
    ny, nx = phi.shape
    c, s = math.cos(ang), math.sin(ang)
    prev_r, prev_v, r = 0.0, None, 0.0
    while True:
        x, y = cx + r * c, cy + r * s
        if x < 0 or y < 0 or x > nx - 2 or y > ny - 2:
            return float("nan")
        i, j = int(x), int(y)
        fx, fy = x - i, y - j
        v = (phi[j, i] * (1 - fx) * (1 - fy) + phi[j, i + 1] * fx * (1 - fy) +
             phi[j + 1, i] * (1 - fx) * fy + phi[j + 1, i + 1] * fx * fy)
        if prev_v is not None and prev_v > 0 >= v:
            return prev_r + (r - prev_r) * prev_v / (prev_v - v)
        prev_r, prev_v, r = r, v, r + step


def arm_spread(stencil):
    import math
    w = W.ISOTROPY[stencil]
    lat = lbmice.Lattice(w.nx, w.ny, **w.params())
    lat.init_seed(w.cx, w.cy, w.R0, w.U0)
    lat.step(w.steps)
    phi = lat.field(lbmice.PHI).astype(np.float64)
    tips = np.array([ray_tip(phi, w.cx, w.cy, math.radians(a)) for a in range(0, 360, 60)])
    assert np.all(np.isfinite(tips)) and tips.min() > 100  # grown, inside the box
    return (tips.max() - tips.min()) / tips.mean()


@pytest.mark.slow
def test_central_difference_biases_the_six_arms_by_orientation():
    # The gradient-isotropy system of Sec. 3.1.1 (800^2, 10^5 steps): with E2 the arms along
    # the x axis and the oblique arms differ by 3.9% (measured); the isotropic stencils
    # halve that (E4 2.2%, E6 2.1%, E8 2.2%), so E4 is enough, as the paper finds.
    s2, s4, s8 = arm_spread(2), arm_spread(4), arm_spread(8)
    assert s2 > 1.5 * s4
    assert s4 < 0.03 and s8 < 0.03


def notch_ratio(w, steps):
    """phi = 0 radius halfway between two arms over the inradius of the hexagon through the
    six tips: 1 for a faceted plate, falling as the arms branch out."""
    import math
    lat = lbmice.Lattice(w.nx, w.ny, **w.params())
    lat.init_seed(w.cx, w.cy, w.R0, w.U0)
    lat.step(steps)
    phi = lat.field(lbmice.PHI).astype(np.float64)
    tips = [ray_tip(phi, w.cx, w.cy, math.radians(a)) for a in range(0, 360, 60)]
    mids = [ray_tip(phi, w.cx, w.cy, math.radians(a + 30)) for a in range(0, 360, 60)]
    assert np.all(np.isfinite(tips + mids))
    return float(np.mean(mids) / (np.mean(tips) * math.sqrt(3) / 2))


def test_table2_habits_order_from_plates_to_ferns():
    # The seven plate-regime parameter sets of Table 2 at T = 500 tau0 (10^4 steps): the
    # solid plate stays a convex faceted hexagon, the plates notch more as U0 rises or L_sat
    # falls, and stars and the fern dendrite grow branched arms. Measured notch ratios:
    # 1.037, 0.984, 0.955, 0.331, 0.282, 0.454, 0.771 for sets 1..7.
    n = [notch_ratio(w, 10000) for w in W.TABLE2_WORKLOADS]
    assert n[0] > 1.0
    assert n[0] > n[1] > n[2] > n[6] > n[5] > max(n[3], n[4])
    assert n[3] < 0.4 and n[4] < 0.4

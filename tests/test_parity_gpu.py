"""Parity of the CUDA path (through the C ABI) with the FP64 oracle, on the same seeded inputs.

Tolerances (FP32 arithmetic against FP64; values are O(1)):
  - one step, every population: 1e-6 absolute (a few FP32 ulps of the O(0.1-1) populations);
  - several steps: the bound is derived per case from the conditioning of the state. A
    second oracle run rounds its populations and phi history to float32 after every step
    (the storage precision of the CUDA path, nothing else changed); the CUDA result must lie
    within FLOOR_FACTOR times that storage-rounding floor, and never needs to beat 4e-6.
    Where |grad phi| is small the direction of the interface normal, hence a_s, is set by
    rounding, so the floor of a noisy state can reach 1e-4 within 200 steps;
  - 2000 steps of the 128 x 128 seed: 1e-4 for phi and U (its floor is 8e-6).
"""
import numpy as np
import pytest

import oracle
from oracle import LAT_F, LAT_G, LAT_H
from paper_2101_07163_gb300 import lbmice
from paper_2101_07163_gb300 import workloads as W

pytestmark = pytest.mark.gpu

CHANNEL_X = (W.BC_INLET, W.BC_OUTLET, W.BC_FREESLIP, W.BC_FREESLIP)
CHANNEL_Y = (W.BC_PERIODIC, W.BC_PERIODIC, W.BC_INLET, W.BC_OUTLET)
BOXES = {
    "periodic": (W.BC_PERIODIC,) * 4,
    "channel_x": CHANNEL_X,
    "channel_y": CHANNEL_Y,
    "walls": (W.BC_FREESLIP,) * 4,
    "outlets": (W.BC_OUTLET, W.BC_OUTLET, W.BC_OUTLET, W.BC_FREESLIP),
    "inlet_plus_x": (W.BC_OUTLET, W.BC_INLET, W.BC_FREESLIP, W.BC_OUTLET),
}


def pair(w: W.Workload, fields: dict):
    lat = lbmice.Lattice(w.nx, w.ny, **w.params())
    lat.set_fields(**fields)
    orc = oracle.Oracle(nx=w.nx, ny=w.ny, **w.params())
    orc.set_fields(**fields)
    return lat, orc


def maxdiff(a, b):
    return float(np.abs(np.asarray(a, dtype=np.float64) - b).max())


def compare_pops(lat, orc, tol):
    p = lat.pops().astype(np.float64)
    assert maxdiff(p[0:9], orc.pops(LAT_H)) < tol
    assert maxdiff(p[9:18], orc.pops(LAT_G)) < tol
    if orc.flow:
        assert maxdiff(p[18:27], orc.pops(LAT_F)) < tol


def compare_moments(lat, orc, tol):
    for which in (lbmice.PHI, lbmice.U, lbmice.RHO, lbmice.UX, lbmice.UY, lbmice.PHI_PREV):
        d = maxdiff(lat.field(which), orc.field(which))
        assert d < tol, (which, d)


FLOOR_FACTOR = 10.0


def fp32_storage_floor(w, fields, steps):
    """max |d phi|, |d U| between the FP64 oracle and the same oracle stored in float32."""
    a = oracle.Oracle(nx=w.nx, ny=w.ny, **w.params())
    b = oracle.Oracle(nx=w.nx, ny=w.ny, **w.params())
    a.set_fields(**fields)
    b.set_fields(**fields)
    a.step(steps)
    for _ in range(steps):
        b.step(1)
        b.round_to_float32()
    return a, {which: float(np.abs(a.field(which) - b.field(which)).max())
               for which in (oracle.PHI, oracle.U, oracle.RHO, oracle.UX, oracle.UY)}


# Minimum bound: besides storage rounding (the floor), the FP32 collisions round coherently
# where the state is nearly uniform, so rho (about 1) can drift by up to half an ulp a step:
# 2e-8 x 200 steps = 4e-6, which a storage-only floor of 1e-7 does not cover.
FLOOR_MIN = 1e-5


def compare_within_floor(lat, orc, floor):
    for which, fl in floor.items():
        d = maxdiff(lat.field(which), orc.field(which))
        tol = max(FLOOR_FACTOR * fl, FLOOR_MIN)
        assert d < tol, (which, d, fl)


def channel_workload(name, nx, ny, bc, **kw):
    return W.Workload(name, nx, ny, 1, flow=True, eps=0.08, D=2.0, U0=0.3, U_in=0.25,
                      u_in=0.03, nu=0.05, bc=bc, cx=nx * 0.4, cy=ny * 0.55, R0=7.0, **kw)


# ---- one step, every population, ragged grids (tiles of 32 x 8 with a tail) ----------------

@pytest.mark.parametrize("box", sorted(BOXES))
def test_one_step_every_population(box):
    w = channel_workload(box, 100, 76, BOXES[box])
    lat, orc = pair(w, W.perturbed_fields(w, 7, amp_phi=0.3, amp_u=0.02))
    compare_pops(lat, orc, 1e-6)  # the initial equilibria
    lat.step(1)
    orc.step(1)
    compare_pops(lat, orc, 1e-6)
    compare_moments(lat, orc, 1e-6)


@pytest.mark.parametrize("box", sorted(BOXES))
def test_short_horizon_moments(box):
    w = channel_workload(box, 70, 44, BOXES[box])
    f = W.perturbed_fields(w, 8, amp_phi=0.2, amp_u=0.01)
    lat = lbmice.Lattice(w.nx, w.ny, **w.params())
    lat.set_fields(**f)
    lat.step(200)
    orc, floor = fp32_storage_floor(w, f, 200)
    compare_within_floor(lat, orc, floor)


@pytest.mark.parametrize("box", ["periodic", "channel_x"])
def test_short_horizon_seed_without_noise(box):
    # a smooth state is well conditioned: a fixed 2e-5 bound over 200 steps
    w = channel_workload(box, 70, 44, BOXES[box])
    lat, orc = pair(w, W.seed_fields(w))
    lat.step(200)
    orc.step(200)
    compare_moments(lat, orc, 2e-5)


def test_phase_field_and_vapour_only():
    w = W.C1.with_size(72, 60)
    f = W.perturbed_fields(w, 9)
    lat, orc1 = pair(w, f)
    lat.step(1)
    orc1.step(1)
    compare_pops(lat, orc1, 1e-6)
    lat.step(199)
    orc, floor = fp32_storage_floor(w, f, 200)
    compare_within_floor(lat, orc, floor)


def test_small_and_degenerate_grids():
    # smallest legal grid, single-tile grids, grids narrower than one tile
    for nx, ny in [(4, 4), (5, 9), (33, 4), (31, 7)]:
        w = channel_workload("tiny", nx, ny, (W.BC_PERIODIC,) * 4)
        w.R0 = 1.5
        lat, orc = pair(w, W.perturbed_fields(w, 10))
        lat.step(3)
        orc.step(3)
        compare_pops(lat, orc, 1e-6)
        w2 = channel_workload("tiny", nx, ny, CHANNEL_X)
        w2.R0 = 1.5
        lat, orc = pair(w2, W.perturbed_fields(w2, 11))
        lat.step(3)
        orc.step(3)
        compare_pops(lat, orc, 1e-6)


def test_uniform_vapour_is_a_fixed_point():
    # phi = -1 everywhere: Q = 0, the vapour and phase field stay put exactly (edge case).
    w = channel_workload("uniform", 64, 40, (W.BC_PERIODIC,) * 4)
    f = dict(phi=np.full((40, 64), -1.0), U=np.full((40, 64), 0.3))
    lat, _ = pair(w, f)
    lat.step(50)
    assert np.all(lat.field(lbmice.PHI) == np.float32(-1.0))
    assert maxdiff(lat.field(lbmice.U), 0.3) < 1e-7


# ---- the configurations of the workloads --------------------------------------------------

def test_seed_128_periodic_2000_steps():
    w = W.C1
    f = W.seed_fields(w)
    lat, orc = pair(w, f)
    lat.step(w.steps)
    orc.step(w.steps)
    dphi = maxdiff(lat.field(lbmice.PHI), orc.field(oracle.PHI))
    dU = maxdiff(lat.field(lbmice.U), orc.field(oracle.U))
    assert dphi < 1e-4 and dU < 1e-4, (dphi, dU)


def test_ventilated_512x384_full_size():
    w = W.C2
    lat, orc = pair(w, W.seed_fields(w))
    lat.step(1)
    orc.step(1)
    compare_pops(lat, orc, 1e-6)
    lat.step(49)
    orc.step(49)
    compare_moments(lat, orc, 2e-5)


@pytest.mark.slow
def test_plate_2048_full_size_200_steps():
    # Full-size grid in the launch configuration the benchmark times; the oracle computes
    # every node (its rows split over the host cores, same bits). The seed keeps its smooth
    # phi (a noisy phi has nodes with |grad phi| ~ 1e-5 whose normal direction is set by
    # rounding); U, rho and u carry noise everywhere.
    #   2 steps: every moment, and the h, g and f populations of 32 sampled rows, within the
    #            one-step bounds;
    #   200 steps: every moment within 10x the spread of an FP32-stored oracle, at least
    #            FLOOR_MIN (the bound of the other multi-step parity tests).
    from tests.helpers import oracle_threads
    w = W.C3
    f = W.perturbed_fields(w, 12, amp_phi=0.0, amp_U=0.05, amp_rho=0.01, amp_u=0.01)
    with oracle_threads():
        lat, orc = pair(w, f)
        lat.step(2)
        orc.step(2)
        compare_moments(lat, orc, 2e-6)
        p = lat.pops()
        rng = np.random.Generator(np.random.PCG64(3))
        rows = np.concatenate([[0, 1, w.ny - 1], rng.integers(0, w.ny, 29)])
        for lo, L in ((0, LAT_H), (9, LAT_G), (18, LAT_F)):
            ref = orc.pops(L)
            assert maxdiff(p[lo:lo + 9][:, rows], ref[:, rows]) < 1e-6, L
            del ref
        del p
        lat.step(198)
        orc.step(198)
        b = oracle.Oracle(nx=w.nx, ny=w.ny, **w.params())
        b.set_fields(**f)
        for _ in range(200):
            b.step(1)
            b.round_to_float32()
        for which in (lbmice.PHI, lbmice.U, lbmice.RHO, lbmice.UX, lbmice.UY):
            ref = orc.field(which)
            floor = maxdiff(b.field(which), ref)
            d = maxdiff(lat.field(which), ref)
            assert d < max(FLOOR_FACTOR * floor, FLOOR_MIN), (which, d, floor)


def test_ventilation_upstream_tip_grows_faster():
    # Sec. 3.1.3 / Sec. 3.2.2 on the 512 x 384 channel: the tip facing the inflow is ahead.
    w = W.C2
    lat = lbmice.Lattice(w.nx, w.ny, **w.params())
    lat.init_seed(w.cx, w.cy, w.R0, w.U0)
    lat.step(8000)
    phi = lat.field(lbmice.PHI).astype(np.float64)
    from tests.helpers import tip_x
    up = w.cx - tip_x(phi, w.cy, w.cx, -1)
    down = tip_x(phi, w.cy, w.cx, +1) - w.cx
    assert np.isfinite(up) and np.isfinite(down)
    assert up > down + 1.0, (up, down)


# ---- invariants, symmetry, determinism ----------------------------------------------------

def test_mirror_symmetry_bit_exact_on_gpu():
    w = W.Workload("m", 96, 64, 1, flow=True, eps=0.07, nu=0.05)
    f = W.mirror_fields(w, 21, amp=0.2)
    lat = lbmice.Lattice(w.nx, w.ny, **w.params())
    lat.set_fields(**f)
    lat.step(300)
    ix, iy = (-np.arange(w.nx)) % w.nx, (-np.arange(w.ny)) % w.ny
    for which in (lbmice.PHI, lbmice.U, lbmice.RHO):
        a = lat.field(which)
        np.testing.assert_array_equal(a, a[:, ix])
        np.testing.assert_array_equal(a, a[iy, :])
    ux = lat.field(lbmice.UX)
    np.testing.assert_array_equal(ux, -ux[:, ix])


def test_graph_replay_equals_single_launches():
    w = channel_workload("g", 80, 48, CHANNEL_X)
    f = W.perturbed_fields(w, 13)
    a = lbmice.Lattice(w.nx, w.ny, **w.params())
    b = lbmice.Lattice(w.nx, w.ny, **w.params())
    a.set_fields(**f)
    b.set_fields(**f)
    a.step(125)              # two graph replays of 60 steps and five single steps
    for _ in range(125):
        b.step(1)
    np.testing.assert_array_equal(a.pops(), b.pops())
    np.testing.assert_array_equal(a.field(lbmice.PHI_PREV), b.field(lbmice.PHI_PREV))


def test_checkpoint_resume_is_bit_exact():
    w = channel_workload("c", 64, 40, CHANNEL_X)
    f = W.perturbed_fields(w, 14)
    a = lbmice.Lattice(w.nx, w.ny, **w.params())
    a.set_fields(**f)
    a.step(37)
    pops, prev = a.pops(), a.field(lbmice.PHI_PREV)
    a.step(71)
    b = lbmice.Lattice(w.nx, w.ny, **w.params())
    b.set_fields(**f)       # any state; overwritten below
    b.step(5)
    b.load(lbmice.POPS, pops)
    b.load(lbmice.PHI_PREV, prev)
    b.step(71)
    np.testing.assert_array_equal(a.pops(), b.pops())


def test_stats_match_oracle_reductions():
    w = channel_workload("s", 90, 70, (W.BC_PERIODIC,) * 4, L_sat=1.3)
    f = W.perturbed_fields(w, 15)
    lat, orc = pair(w, f)
    s0 = lat.stats()
    lat.step(40)
    orc.step(40)
    s = lat.stats()
    assert s["nonfinite"] == 0 and s["steps"] == 40

    def sums(phi, U, rho, prev):
        return dict(area=(0.5 * (1 + phi)).sum() * w.dx ** 2, mass=rho.sum(),
                    vapour_invariant=(U + 0.65 * prev).sum(), sum_phi=phi.sum())

    # the FP64 reduction kernel against float64 sums of the GPU's own fields
    mine = sums(*(lat.field(k).astype(np.float64) for k in (lbmice.PHI, lbmice.U, lbmice.RHO,
                                                           lbmice.PHI_PREV)))
    for k, v in mine.items():
        assert s[k] == pytest.approx(v, rel=1e-12, abs=1e-9), k
    # and against the oracle's fields (FP32 field parity)
    ref = sums(*(orc.field(k) for k in (oracle.PHI, oracle.U, oracle.RHO, oracle.PHI_PREV)))
    for k in ("area", "mass", "vapour_invariant"):
        assert s[k] == pytest.approx(ref[k], rel=2e-5), k
    # exact invariants of the periodic grid hold on the GPU to FP32 rounding
    assert s["mass"] == pytest.approx(s0["mass"], rel=1e-6)
    assert s["vapour_invariant"] == pytest.approx(s0["vapour_invariant"], rel=1e-5)


def test_device_tips_equal_host_diagnostics_and_follow_the_oracle():
    # lbmice_tips applies the definition of diagnostics.tip_radius on the device: on the same
    # exported field the two agree to rounding; against the FP64 oracle's field the tips of
    # the FP32 run lie within 2e-3 cells (phi differs by ~4e-5 where |grad phi| ~ 0.3/cell).
    from paper_2101_07163_gb300 import diagnostics as D
    w = W.C3.with_size(160, 160)
    lat, orc = pair(w, W.seed_fields(w))
    lat.step(1500)
    orc.step(1500)
    angles = np.arange(0.0, 360.0, 15.0)
    dev = lat.tips(w.cx, w.cy, angles)
    phi = lat.field(lbmice.PHI).astype(np.float64)
    host = np.array([D.tip_radius(phi, w.cx, w.cy, a) for a in angles])
    assert np.all(np.isfinite(dev)) and dev.min() > w.R0
    assert np.abs(dev - host).max() < 1e-9
    ophi = orc.field(oracle.PHI)
    ref = np.array([D.tip_radius(ophi, w.cx, w.cy, a) for a in angles])
    assert np.abs(dev - ref).max() < 2e-3
    # a centre outside the crystal, and a ray that leaves the grid first: NaN
    assert np.isnan(lat.tips(3.0, 3.0, [0.0])[0])
    assert np.isnan(lat.tips(w.cx, w.cy, [0.0], step=1000.0)[0])
    assert np.isnan(D.tip_radius(phi, w.cx, w.cy, 0.0, step=1000.0))
    with pytest.raises(lbmice.LbmiceError):
        lat.tips(w.cx, w.cy, [0.0], step=0.0)
    with pytest.raises(lbmice.LbmiceError):
        lat.tips(w.cx, w.cy, np.zeros(lbmice.MAX_RAYS + 1))


def test_nonfinite_state_is_reported_not_trapped():
    w = channel_workload("n", 64, 40, (W.BC_PERIODIC,) * 4)
    f = W.perturbed_fields(w, 16)
    f["U"][20, 30] = np.nan
    lat = lbmice.Lattice(w.nx, w.ny, check_every=1, **w.params())
    lat.set_fields(**f)
    with pytest.raises(lbmice.LbmiceError) as ei:
        lat.step(5)
    assert ei.value.code == lbmice.ENONFINITE
    assert lat.stats()["nonfinite"] > 0
    lat.sync()  # the context is still usable


def test_init_seed_matches_workload_fields():
    for w in (W.C1, W.C2.with_size(200, 120)):
        lat = lbmice.Lattice(w.nx, w.ny, **w.params())
        lat.init_seed(w.cx, w.cy, w.R0, w.U0)
        ref, _ = pair(w, W.seed_fields(w))
        for which in (lbmice.PHI, lbmice.U, lbmice.RHO, lbmice.UX):
            assert maxdiff(lat.field(which), ref.field(which)) < 1e-6


def test_device_fields_equal_host_fields():
    import torch
    w = channel_workload("d", 48, 40, CHANNEL_Y)
    f = W.perturbed_fields(w, 17)
    a = lbmice.Lattice(w.nx, w.ny, **w.params())
    a.set_fields(**f)
    b = lbmice.Lattice(w.nx, w.ny, **w.params())
    b.set_fields(**{k: torch.from_numpy(v).cuda() for k, v in f.items()})
    b.sync()
    np.testing.assert_array_equal(a.pops(), b.pops())
    out = torch.empty(w.ny, w.nx, device="cuda", dtype=torch.float32)
    a.field(lbmice.PHI, out=out)
    torch.cuda.synchronize()
    np.testing.assert_array_equal(out.cpu().numpy(), a.field(lbmice.PHI))


def test_field_output_tensor_is_checked():
    # a device output must be a contiguous float32 CUDA tensor on the lattice's device
    import torch
    w = channel_workload("o", 32, 16, (W.BC_PERIODIC,) * 4)
    lat = lbmice.Lattice(w.nx, w.ny, **w.params())
    lat.init_seed(w.cx, w.cy, w.R0, w.U0)
    good = torch.empty((w.ny, w.nx), dtype=torch.float32, device=lat.device)
    assert lat.field(lbmice.PHI, out=good) is good
    np.testing.assert_array_equal(good.cpu().numpy(), lat.field(lbmice.PHI))
    bad = (torch.empty((w.ny, w.nx), dtype=torch.float32),                            # host
           torch.empty((w.ny, 2 * w.nx), dtype=torch.float32, device=lat.device)[:, ::2],
           torch.empty((w.ny, w.nx), dtype=torch.float64, device=lat.device))
    for t in bad:
        with pytest.raises(ValueError):
            lat.field(lbmice.PHI, out=t)
    lat.close()


def test_bad_buffer_sizes_are_rejected():
    w = channel_workload("b", 32, 16, (W.BC_PERIODIC,) * 4)
    lat = lbmice.Lattice(w.nx, w.ny, **w.params())
    small = np.zeros(10, dtype=np.float32)
    with pytest.raises(lbmice.LbmiceError) as ei:
        lat.load(lbmice.POPS, small)
    assert ei.value.code == lbmice.EINVAL
    import ctypes
    rc = lbmice.lib().lbmice_fields(lat.handle, lbmice.PHI, small.ctypes.data_as(
        ctypes.c_void_p), small.nbytes, 0)
    assert rc == lbmice.EINVAL
    rc = lbmice.lib().lbmice_fields(lat.handle, 42, small.ctypes.data_as(ctypes.c_void_p),
                                    small.nbytes, 0)
    assert rc == lbmice.EINVAL

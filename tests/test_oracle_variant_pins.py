"""Pins of the method variants of the oracle (Sec. 3.1.1 stencils E2, E6, E8 of Table 1, and
the four-fold anisotropy of the validation system of Sec. 3.1.2): exactness and isotropy order
of every stencil, the four-fold a_s and flux against their trigonometric form, and bit-exact
mirror symmetry with every stencil."""
import math
import os

import numpy as np
import pytest

import oracle
from oracle import PHI, RHO, U, UX, UY, Oracle
from paper_2101_07163_gb300 import workloads as W

STENCILS = (2, 4, 6, 8)


@pytest.mark.parametrize("stencil", STENCILS)
def test_every_stencil_is_exact_for_linear_fields(stencil):
    n = 24
    y, x = np.mgrid[0:n, 0:n].astype(np.float64)
    a, b = 0.37, -1.21
    gx, gy = oracle.gradient_stencil(a * x + b * y, stencil)
    inner = (slice(3, n - 3), slice(3, n - 3))  # away from the periodic wrap of the ramp
    np.testing.assert_allclose(gx[inner], a, rtol=0, atol=1e-13)
    np.testing.assert_allclose(gy[inner], b, rtol=0, atol=1e-13)


def effective_wavenumber(stencil, k, theta, n=32):
    """|grad| of the stencil applied to sin(k e.(x - x0)) at x0: the plane wave's effective
    wavenumber along direction e = (cos theta, sin theta)."""
    y, x = np.mgrid[0:n, 0:n].astype(np.float64)
    x0 = y0 = n // 2
    phi = np.sin(k * ((x - x0) * math.cos(theta) + (y - y0) * math.sin(theta)))
    gx, gy = oracle.gradient_stencil(phi, stencil)
    return math.hypot(gx[y0, x0], gy[y0, x0])


@pytest.mark.parametrize("stencil", STENCILS)
def test_isotropy_order_of_every_stencil(stencil):
    # The direction spread of the effective wavenumber, relative to k, falls as k^stencil:
    # E2 is isotropic only to second order, E4/E6/E8 to the order Table 1 names.
    thetas = np.linspace(0.0, math.pi / 4, 13)

    def spread(k):
        ke = np.array([effective_wavenumber(stencil, k, t) for t in thetas])
        return (ke.max() - ke.min()) / k

    s1, s2 = spread(0.4), spread(0.8)
    order = math.log(s2 / s1) / math.log(2.0)
    assert abs(order - stencil) < 0.3, (stencil, order)


def aniso_trig(gx, gy, eps, fold):
    theta = np.arctan2(-gy, -gx)
    return 1.0 + eps * np.cos(fold * theta)


def test_four_fold_anisotropy_matches_trig_form_and_derivative():
    rng = np.random.Generator(np.random.PCG64(8))
    h = 1e-6
    for _ in range(200):
        gx, gy = rng.normal(size=2) * 10 ** rng.uniform(-4, 0)
        eps = rng.uniform(0.0, 0.1)
        a_s, Nx, Ny = oracle.anisotropy_fold(gx, gy, eps, 1.0, 4)
        assert a_s == pytest.approx(aniso_trig(gx, gy, eps, 4), abs=1e-13)
        s = gx * gx + gy * gy
        dax = (aniso_trig(gx + h, gy, eps, 4) ** 2 - aniso_trig(gx - h, gy, eps, 4) ** 2) / (2 * h)
        day = (aniso_trig(gx, gy + h, eps, 4) ** 2 - aniso_trig(gx, gy - h, eps, 4) ** 2) / (2 * h)
        scale = 1e-6 * max(1.0, math.hypot(gx, gy))
        assert Nx == pytest.approx(0.5 * s * dax, abs=scale)
        assert Ny == pytest.approx(0.5 * s * day, abs=scale)
    # six-fold through the same entry is the ice form
    a6 = oracle.anisotropy_fold(0.3, -0.7, 0.05, 1.0, 6)
    assert a6 == pytest.approx(oracle.anisotropy(0.3, -0.7, 0.05, 1.0), abs=0)


def test_four_fold_tips_lie_on_the_axes():
    # a_s = 1 + eps cos(4 theta) is largest for normals along the axes and the diagonals'
    # minimum is 1 - eps
    a_axis = oracle.anisotropy_fold(-1.0, 0.0, 0.05, 1.0, 4)[0]
    a_diag = oracle.anisotropy_fold(-1.0, -1.0, 0.05, 1.0, 4)[0]
    assert a_axis == pytest.approx(1.05, abs=1e-15)
    assert a_diag == pytest.approx(0.95, abs=1e-15)


@pytest.mark.parametrize("stencil", STENCILS)
def test_mirror_symmetry_is_bit_exact_with_every_stencil(stencil):
    nx, ny = 28, 24
    w = W.Workload("t", nx, ny, 1, flow=True, eps=0.07, nu=0.05, stencil=stencil)
    f = W.mirror_fields(w, 22, amp=0.2)
    o = Oracle(nx=nx, ny=ny, **w.params())
    o.set_fields(**f)
    o.step(25)
    ix, iy = (-np.arange(nx)) % nx, (-np.arange(ny)) % ny
    for which in (PHI, U, RHO):
        a = o.field(which)
        np.testing.assert_array_equal(a, a[:, ix])
        np.testing.assert_array_equal(a, a[iy, :])
    ux = o.field(UX)
    np.testing.assert_array_equal(ux, -ux[:, ix])
    assert np.abs(ux).max() > 1e-4


def test_stencils_and_folds_are_validated():
    with pytest.raises(ValueError):
        Oracle(nx=8, ny=8, stencil=3)
    with pytest.raises(ValueError):
        Oracle(nx=8, ny=8, fold=5)
    Oracle(nx=8, ny=8, stencil=8, fold=4)  # accepted


# ---- the printed tables -------------------------------------------------------------------

SHELLS = {1: [(1, 0)], 2: [(1, 1)], 4: [(2, 0)], 5: [(1, 2), (2, 1)], 8: [(2, 2)]}


@pytest.mark.parametrize("stencil", [4, 6, 8])
def test_stencil_weights_are_those_of_table_1(stencil):
    # A field that is 1 at one neighbour x0 + c and 0 elsewhere: the oracle's gradient at x0
    # is w(|c|^2) c with the weight printed in Table 1 (tests/golden), for every neighbour of
    # every shell of the stencil in all four quadrants -- and 0 for shells the stencil lacks.
    from tests.helpers import golden_constants
    g = golden_constants("table1_isotropic_weights.txt")
    n, x0, y0 = 12, 6, 6
    for shell, reps in SHELLS.items():
        w = g.get(f"E{stencil}_w{shell}", 0.0)
        for (ax, ay) in reps:
            for sx in (1, -1):
                for sy in (1, -1):
                    cx, cy = sx * ax, sy * ay
                    phi = np.zeros((n, n))
                    phi[y0 + cy, x0 + cx] = 1.0
                    gx, gy = oracle.gradient_stencil(phi, stencil)
                    assert gx[y0, x0] == pytest.approx(w * cx, abs=1e-15), (shell, cx, cy)
                    assert gy[y0, x0] == pytest.approx(w * cy, abs=1e-15), (shell, cx, cy)


def table2_rows():
    from tests.helpers import GOLDEN
    consts, rows = {}, []
    with open(os.path.join(GOLDEN, "table2_plate_regime.txt")) as fh:
        for line in fh:
            line = line.split("#", 1)[0].strip()
            if not line:
                continue
            if "=" in line:
                k, v = (t.strip() for t in line.split("=", 1))
                consts[k] = float(v)
            else:
                nr, name, U0, L_sat, rho0, drho = line.split()
                rows.append((int(nr), name, float(U0), float(L_sat), float(rho0), float(drho)))
    return consts, rows


def test_table2_workloads_follow_the_printed_table():
    # The workloads of the seven morphologies carry Table 2's U0 and L_sat; the table's own
    # densities give its U0 through U = (drho + rho_sat_W - rho_sat_I) / rho_sat_I and
    # rho0 = rho_sat_W + drho (to the rounding of the printed digits), which is why U0 and
    # L_sat are the only inputs (reading of Sec. 3.2.1).
    from paper_2101_07163_gb300 import workloads as W
    c, rows = table2_rows()
    assert len(rows) == len(W.TABLE2_WORKLOADS) == 7
    for (nr, name, U0, L_sat, rho0, drho), w in zip(rows, W.TABLE2_WORKLOADS):
        assert w.name.startswith(f"table2_{nr}_{name}_")
        assert w.U0 == U0 and w.L_sat == L_sat
        assert (drho + c["rho_sat_W"] - c["rho_sat_I"]) / c["rho_sat_I"] == pytest.approx(U0, abs=1e-3)
        assert rho0 - drho == pytest.approx(c["rho_sat_W"], abs=1e-3)
        assert (w.dx, w.dt, w.lam, w.eps, w.nx, w.ny) == (0.8, 0.05, 3.0, 0.05, 400, 400)


def test_validation_workloads_convert_the_printed_parameters():
    # The isotropy system of Sec. 3.1.1 is printed in physical units; in W0 / tau0 units it is
    # dx = 0.8, dt = 0.096 and D = kappa tau0 / W0^2 = 1. The four-fold system of Sec. 3.1.2 is
    # printed in those units already; its lambda is the beta = 0 value of D = kappa = 4.
    from tests.helpers import golden_constants
    from paper_2101_07163_gb300 import workloads as W
    g = golden_constants("validation_systems.txt")
    for s, w in W.ISOTROPY.items():
        assert w.stencil == s
        assert w.dx == pytest.approx(g["iso_dx"] / g["iso_W0"], rel=1e-12)
        assert w.dt == pytest.approx(g["iso_dt"] / g["iso_tau0"], rel=1e-12)
        assert w.D == pytest.approx(g["iso_kappa"] * g["iso_tau0"] / g["iso_W0"] ** 2, rel=1e-12)
        assert (w.U0, w.lam, w.eps) == (g["iso_undercooling"], g["iso_lambda"], g["iso_eps"])
        assert (w.nx, w.ny, w.R0, w.steps) == (g["iso_n"], g["iso_n"], g["iso_seed_radius_cells"],
                                               g["iso_steps"])
    for w, U0, n in ((W.FOURFOLD_030, g["ff_U0_a"], g["ff_n_a"]),
                     (W.FOURFOLD_055, g["ff_U0_b"], g["ff_n_b"])):
        assert (w.dx, w.dt, w.D, w.eps, w.fold) == (g["ff_dx"], g["ff_dt"], g["ff_kappa"],
                                                    g["ff_eps"], 4)
        assert (w.U0, w.nx, w.ny, w.R0) == (U0, n, n, g["ff_seed_radius_cells"])
        o = Oracle(nx=8, ny=8, **w.params())
        assert o.derived()["lambda"] == pytest.approx(g["ff_lambda"], abs=1e-4)

"""Pins of the FP64 oracle against what the paper and the mathematics fix.

Each test checks the oracle against something other than itself: a closed form, an exact
invariant, a symmetry, a special case that reduces to an ODE or to a textbook result, the
moment algebra of the lattice, a library routine, or a constant printed in the paper
(tests/golden/paper_constants.txt). A plausible mistake in the oracle -- a dropped term, a
wrong sign or index, a transposed operand -- fails at least one of them.
"""
import math

import numpy as np
import pytest

import oracle
from oracle import LAT_AS2, LAT_F, LAT_G, LAT_H, PHI, PHI_PREV, RHO, U, UX, UY, Oracle
from paper_2101_07163_gb300 import workloads as W
from tests.helpers import contour_radius, golden_constants

pytestmark = pytest.mark.usefixtures("oracle_lib")

CX = np.array([0, 1, 0, -1, 0, 1, -1, -1, 1])
CY = np.array([0, 0, 1, 0, -1, 1, 1, -1, -1])
WT = np.array([4 / 9] + [1 / 9] * 4 + [1 / 36] * 4)
G = golden_constants()


def full(nx, ny, v):
    return np.full((ny, nx), float(v))


def aniso_trig(gx, gy, eps):
    """a_s = 1 + eps cos(6 theta), theta = arctan of the normal n = -grad phi/|grad phi|."""
    theta = np.arctan2(-gy, -gx)
    return 1.0 + eps * np.cos(6.0 * theta)


def flux_fd(gx, gy, eps, kappa=1.0, h=1e-6):
    """(kappa/2) |g|^2 d(a_s^2)/dg by central differences of the trig form."""
    s = gx * gx + gy * gy
    dax = (aniso_trig(gx + h, gy, eps) ** 2 - aniso_trig(gx - h, gy, eps) ** 2) / (2 * h)
    day = (aniso_trig(gx, gy + h, eps) ** 2 - aniso_trig(gx, gy - h, eps) ** 2) / (2 * h)
    return 0.5 * kappa * s * dax, 0.5 * kappa * s * day


# ------------------------------------------------------------------------------------------
# Constants printed in the paper
# ------------------------------------------------------------------------------------------

def test_lambda_beta_zero_matches_printed_value():
    # Sec. 3.1.2: W0 = tau0 = 1, kappa = 4 gives lambda = 6.3826 (printed, 4 decimals).
    o = Oracle(nx=4, ny=4, W0=1.0, tau0=1.0, D=4.0, lam=0.0)
    lam = o.derived()["lambda"]
    assert abs(lam - G["lambda_fourfold"]) < 5e-5
    assert abs(lam - G["lambda_flow"]) < 5e-4
    # d0 = a1 W0 / lambda, beta = a1 (tau0/(W0 lambda) - a2 W0/D) = 0 at this lambda.
    beta = G["a1"] * (1.0 / lam - G["a2"] / 4.0)
    assert abs(beta) < 1e-12


def test_e4_weights_match_table1():
    # The response of the gradient to a unit spike reads the stencil weights directly:
    # d/dx at (x0-1, y0) sees w(1) phi(x0), at (x0-1, y0-1) sees w(2) phi(x0, y0).
    phi = np.zeros((9, 9))
    phi[4, 4] = 1.0
    gx, gy = oracle.gradient_periodic(phi)
    assert gx[4, 3] == pytest.approx(G["E4_w1"], abs=1e-16)
    assert gx[3, 3] == pytest.approx(G["E4_w2"], abs=1e-16)
    assert gy[3, 4] == pytest.approx(G["E4_w1"], abs=1e-16)
    assert gy[3, 3] == pytest.approx(G["E4_w2"], abs=1e-16)
    assert gx[4, 5] == pytest.approx(-G["E4_w1"], abs=1e-16)
    # only the first two shells are touched
    nz = np.argwhere(np.abs(gx) + np.abs(gy) > 0)
    assert np.abs(nz - 4).max() == 1


# ------------------------------------------------------------------------------------------
# Isotropic gradient (Sec. 3.1.1)
# ------------------------------------------------------------------------------------------

def test_gradient_exact_for_linear_and_quadratic_fields():
    y, x = np.mgrid[0:16, 0:16].astype(float)
    for phi, ex, ey in [
        (0.3 * x - 0.7 * y, 0.3, -0.7),
        (x * x, 2 * x, 0 * x),
        (x * y, y, x),
        (0.5 * y * y - x * y + 2 * x, -y + 2, y - x),
    ]:
        gx, gy = oracle.gradient_periodic(phi)
        inner = (slice(2, -2), slice(2, -2))
        np.testing.assert_allclose(gx[inner], np.broadcast_to(ex, phi.shape)[inner], atol=1e-12)
        np.testing.assert_allclose(gy[inner], np.broadcast_to(ey, phi.shape)[inner], atol=1e-12)


def test_gradient_is_fourth_order_isotropic():
    # For a plane wave the stencil's effective wavenumber depends on direction only at
    # O(k^5) for an E4 stencil (its fourth-rank moment tensor is isotropic), against O(k^3)
    # for the plain central difference E2. The spread over directions must shrink as k^4
    # relative to k.
    def spread(kmag):
        vals = []
        for th in np.linspace(0, np.pi / 2, 13):
            kx, ky = kmag * np.cos(th), kmag * np.sin(th)
            y, x = np.mgrid[0:24, 0:24].astype(float)
            phi = np.sin(kx * (x - 12) + ky * (y - 12))
            gx, gy = oracle.gradient_periodic(phi)
            vals.append(math.hypot(gx[12, 12], gy[12, 12]) / kmag)
        vals = np.array(vals)
        return vals.max() - vals.min()

    s1, s2 = spread(0.2), spread(0.4)
    assert s1 < 2e-5
    assert 10.0 < s2 / s1 < 22.0  # ~ 2^4


# ------------------------------------------------------------------------------------------
# Anisotropy function and anisotropic flux (Sec. 2.1, Eq. (a), Eq. (e))
# ------------------------------------------------------------------------------------------

def test_anisotropy_matches_trig_form_and_derivative():
    rng = np.random.Generator(np.random.PCG64(7))
    for _ in range(200):
        gx, gy = rng.normal(size=2) * 10 ** rng.uniform(-4, 0)
        eps = rng.uniform(0.0, 0.1)
        a_s, Nx, Ny = oracle.anisotropy(gx, gy, eps, 1.0)
        assert a_s == pytest.approx(aniso_trig(gx, gy, eps), abs=1e-13)
        fx, fy = flux_fd(gx, gy, eps)
        scale = 1e-6 * max(1.0, math.hypot(gx, gy))
        assert Nx == pytest.approx(fx, abs=scale)
        assert Ny == pytest.approx(fy, abs=scale)
        # the literal reading kappa_N = 2 doubles the flux
        _, Nx2, Ny2 = oracle.anisotropy(gx, gy, eps, 2.0)
        assert Nx2 == pytest.approx(2 * Nx, rel=1e-14, abs=1e-300)


def test_anisotropy_tips_and_threshold():
    # cos(6 theta) is maximal along the six tip directions theta = k pi/3
    for k in range(6):
        th = k * np.pi / 3
        a_s, Nx, Ny = oracle.anisotropy(-np.cos(th), -np.sin(th), 0.05, 1.0)
        assert a_s == pytest.approx(1.05, abs=1e-13)
        assert abs(Nx) < 1e-13 and abs(Ny) < 1e-13
    assert oracle.anisotropy(1e-7, 0.0, 0.05, 1.0) == (1.0, 0.0, 0.0)  # |g|^2 <= 1e-12


# ------------------------------------------------------------------------------------------
# Uniform states: the scheme reduces to the ODEs of Eq. (a), Eq. (b) and the drag law
# ------------------------------------------------------------------------------------------

@pytest.mark.parametrize("flow", [False, True])
def test_uniform_state_is_explicit_euler_of_source_terms(flow):
    # With no gradients a_s = 1 and every population stays at equilibrium, so
    #   phi^{n+1} = phi^n + (dt/tau0) [phi - phi^3 + lambda U (1 - phi^2)^2]     (Eq. (a))
    #   U^{n+1}   = U^n - (L_sat/2) (phi^n - phi^{n-1})                            (Eq. (b))
    nx, ny = 5, 4
    L_sat, D, dt, tau0 = 1.3, 2.5, 0.008, 1.0
    o = Oracle(nx=nx, ny=ny, D=D, L_sat=L_sat, dt=dt, tau0=tau0, eps=0.05, flow=flow)
    lam = tau0 * D / (G["a2"] * 1.0)
    o.set_fields(full(nx, ny, 0.1), full(nx, ny, 0.4))
    phi, Uv, phi_prev = 0.1, 0.4, 0.1
    for _ in range(60):
        o.step(1)
        Q = phi - phi ** 3 + lam * Uv * (1 - phi ** 2) ** 2
        phi, Uv, phi_prev = phi + dt / tau0 * Q, Uv - 0.5 * L_sat * (phi - phi_prev), phi
        np.testing.assert_allclose(o.field(PHI), phi, rtol=0, atol=1e-14)
        np.testing.assert_allclose(o.field(U), Uv, rtol=0, atol=1e-14)
        np.testing.assert_allclose(o.field(PHI_PREV), phi_prev, rtol=0, atol=1e-14)


def test_uniform_flow_momentum_follows_guo_forcing_with_drag():
    # Uniform phi and j: streaming is the identity, so the momentum follows the first moment
    # of the collision. Guo's forcing term has first moment (1 - 1/(2 tau)) F, giving
    #   j' = j - (j - rho u*)/tau + (1 - 1/(2 tau)) F,   u = j/(rho + k/2), u* = (1-phi)/2 u,
    #   F = -k u*,  k = h rho nu (1+phi)^2 (1-phi) / (4 W^2)   (Sec. 2.2.1, h printed).
    nx, ny = 4, 3
    nu, dx, W0 = 0.05, 0.4, 1.0
    o = Oracle(nx=nx, ny=ny, nu=nu, dx=dx, W0=W0, flow=True, eps=0.0)
    phi0, rho0 = 0.2, 1.1
    o.set_fields(full(nx, ny, phi0), full(nx, ny, 0.0), full(nx, ny, rho0),
                 full(nx, ny, 0.03), full(nx, ny, -0.02))
    tau = 3 * nu + 0.5
    Wl = W0 / dx
    jx, jy = rho0 * 0.03, rho0 * -0.02
    phi, Uv, phi_prev = phi0, 0.0, phi0
    lam = 1.0 * 2.0 / G["a2"]  # default tau0 = 1, D = 2, W0 = 1
    for _ in range(30):
        # phi evolves by its own source; U = 0
        k = G["h_drag"] * rho0 * nu * (1 + phi) ** 2 * (1 - phi) / (4 * Wl ** 2)
        ux, uy = jx / (rho0 + k / 2), jy / (rho0 + k / 2)
        usx, usy = 0.5 * (1 - phi) * ux, 0.5 * (1 - phi) * uy
        Fx, Fy = -k * usx, -k * usy
        jx = jx - (jx - rho0 * usx) / tau + (1 - 0.5 / tau) * Fx
        jy = jy - (jy - rho0 * usy) / tau + (1 - 0.5 / tau) * Fy
        o.step(1)
        Q = phi - phi ** 3 + lam * Uv * (1 - phi ** 2) ** 2
        phi, Uv, phi_prev = phi + 0.008 * Q, Uv - 0.5 * (phi - phi_prev), phi
        f = o.pops(LAT_F)
        assert (CX[:, None, None] * f).sum(0) == pytest.approx(full(nx, ny, jx), abs=1e-15)
        assert (CY[:, None, None] * f).sum(0) == pytest.approx(full(nx, ny, jy), abs=1e-15)
        np.testing.assert_allclose(o.field(RHO), rho0, rtol=1e-14)


# ------------------------------------------------------------------------------------------
# Vapour lattice: exact moment recurrences of the advection-diffusion LB (Sec. 2.2.2)
# ------------------------------------------------------------------------------------------

def test_gaussian_pulse_variance_growth_is_exact():
    # phi = -1 everywhere (vapour): q = 2, no source, tau_g = D q / c_s^2 + 1/2 (lattice).
    # For BGK with u = 0 started at equilibrium, the second moment V = sum x^2 U obeys
    #   A_{n+1} = (1 - 1/tau) A_n + c_s^2 M,  V_{n+1} = V_n + 2 (1 - 1/tau) A_n + c_s^2 M,
    # with A = sum x J_x and M = sum U; per step V grows by 2 c_s^2 (tau - 1/2) M at large n.
    nx = ny = 128
    D, dx, dt = 2.0, 0.4, 0.008
    o = Oracle(nx=nx, ny=ny, D=D, dx=dx, dt=dt, eps=0.05)
    y, x = np.mgrid[0:ny, 0:nx].astype(float)
    xc, yc, s0 = 63.3, 64.1, 4.0
    Uf = 0.1 + 0.0 * x
    Uf = np.exp(-((x - xc) ** 2 + (y - yc) ** 2) / (2 * s0 ** 2))
    o.set_fields(full(nx, ny, -1.0), Uf)
    tau = 3.0 * (D * dt / dx ** 2) * 2.0 + 0.5
    M = Uf.sum()
    V = ((x - xc) ** 2 * Uf).sum()
    A = 0.0
    for _ in range(30):
        V, A = V + 2 * (1 - 1 / tau) * A + M / 3, (1 - 1 / tau) * A + M / 3
        o.step(1)
    Un = o.field(U)
    assert ((x - xc) ** 2 * Un).sum() == pytest.approx(V, rel=1e-12)
    assert ((y - yc) ** 2 * Un).sum() == pytest.approx(V, rel=1e-3)  # same law along y
    assert Un.sum() == pytest.approx(M, rel=1e-13)
    np.testing.assert_array_equal(o.field(PHI), -1.0)
    # large-n increment is the diffusivity of the continuum equation, D q
    inc = 2 * (1 - 1 / tau) * (tau * (1 / 3) * M) + M / 3
    assert inc / M / 2 == pytest.approx((D * dt / dx ** 2) * 2.0, rel=1e-12)


def test_gaussian_pulse_profile_matches_analytic_spreading():
    # The heat kernel: a Gaussian of variance s0^2 spreads to s0^2 + 2 D_eff t.
    nx = ny = 96
    D, dx, dt = 2.0, 0.4, 0.008
    o = Oracle(nx=nx, ny=ny, D=D, dx=dx, dt=dt)
    y, x = np.mgrid[0:ny, 0:nx].astype(float)
    s0 = 5.0
    r2 = (x - 48) ** 2 + (y - 48) ** 2
    o.set_fields(full(nx, ny, -1.0), np.exp(-r2 / (2 * s0 ** 2)))
    n = 200
    o.step(n)
    Deff = 2.0 * D * dt / dx ** 2
    # variance of the lattice pulse: 2 D_eff n less the start-up lag of the moment
    # recurrence above, 2 r tau^2 c_s^2 (1 - r^n) with r = 1 - 1/tau
    tau = 3 * Deff + 0.5
    r = 1 - 1 / tau
    s2 = s0 ** 2 + 2 * Deff * n - 2 * r * tau * tau / 3 * (1 - r ** n)
    exact = (s0 ** 2 / s2) * np.exp(-r2 / (2 * s2))
    err = np.linalg.norm(o.field(U) - exact) / np.linalg.norm(exact)
    assert err < 1e-3


def test_advected_pulse_centroid_moves_with_fluid_velocity():
    # In vapour (phi = -1) the drag vanishes and u* = u; with g^eq = w U (1 + c.u/c_s^2) the
    # total flux stays M u, so the centroid of U moves by exactly u per step.
    nx, ny = 112, 112  # tails stay below 1e-12 at the periodic edges
    o = Oracle(nx=nx, ny=ny, flow=True, nu=0.05, D=1.0)
    y, x = np.mgrid[0:ny, 0:nx].astype(float)
    Uf = np.exp(-((x - 54) ** 2 + (y - 58) ** 2) / 18.0)
    ux, uy = 0.05, -0.03
    o.set_fields(full(nx, ny, -1.0), Uf, full(nx, ny, 1.0), full(nx, ny, ux), full(nx, ny, uy))
    M = Uf.sum()
    X0, Y0 = (x * Uf).sum() / M, (y * Uf).sum() / M
    o.step(100)
    Un = o.field(U)
    assert (x * Un).sum() / M == pytest.approx(X0 + 100 * ux, abs=1e-9)
    assert (y * Un).sum() / M == pytest.approx(Y0 + 100 * uy, abs=1e-9)
    np.testing.assert_allclose(o.field(UX), ux, rtol=1e-12)


# ------------------------------------------------------------------------------------------
# Phase field: stationary flat interface (Eq. (a) with U = 0)
# ------------------------------------------------------------------------------------------

def _flat_front_error(dx, eps, nx_phys=38.4, t_end=10.0, L_sat=0.0):
    # Two fronts on a periodic strip. With U = 0 and eps = 0 the steady state of Eq. (a) is
    # W0^2 phi'' + phi - phi^3 = 0, solved by tanh(x / (sqrt(2) W0)). For a front whose
    # normal lies along x, cos(6 theta) = 1 and sin(6 theta) = 0, so a_s = 1 + eps and the
    # width scales with it: tanh(x / (sqrt(2) W0 (1 + eps))).
    nx = int(round(nx_phys / dx))
    ny = 2
    dt = 0.008 * (dx / 0.4) ** 2  # diffusive scaling keeps (W0^2/tau0) dt/dx^2 fixed
    o = Oracle(nx=nx, ny=ny, dx=dx, dt=dt, eps=eps, L_sat=L_sat)
    xs = (np.arange(nx) + 0.5) * dx
    half = nx * dx / 2
    d = np.abs(xs - half) - half / 2
    phi0 = -np.tanh(d / math.sqrt(2.0))
    o.set_fields(np.tile(phi0, (ny, 1)), full(nx, ny, 0.0))
    o.step(int(round(t_end / dt)))
    exact = -np.tanh(d / (math.sqrt(2.0) * (1.0 + eps)))
    return np.abs(o.field(PHI)[0] - exact).max()


def test_flat_front_is_stationary_tanh_with_second_order_convergence():
    e1 = _flat_front_error(0.4, 0.0)
    e2 = _flat_front_error(0.2, 0.0)
    e3 = _flat_front_error(0.1, 0.0)
    assert e1 < 1e-2  # 9.0e-3 at the paper's dx/W0 = 0.4
    assert 3.5 < e1 / e2 < 4.5 and 3.5 < e2 / e3 < 4.5  # second order in dx


def test_flat_front_width_scales_with_anisotropy():
    # The broadened profile is matched to discretisation error, far below the gap between
    # the broadened and the isotropic tanh profiles.
    e = _flat_front_error(0.2, 0.05)
    gap = max(abs(np.tanh(d / math.sqrt(2.0)) - np.tanh(d / (math.sqrt(2.0) * 1.05)))
              for d in np.linspace(0, 4, 81))
    assert e < 3e-3
    assert e < 0.2 * gap


# ------------------------------------------------------------------------------------------
# Exact invariants of the coupled step
# ------------------------------------------------------------------------------------------

def _random_state(nx, ny, seed, flow=True, **kw):
    w = W.Workload("t", nx, ny, 1, flow=flow, cx=nx / 2, cy=ny / 2, R0=min(nx, ny) / 4, **kw)
    f = W.perturbed_fields(w, seed, amp_phi=0.3, amp_U=0.1, amp_rho=0.05, amp_u=0.03)
    o = Oracle(nx=nx, ny=ny, **w.params())
    o.set_fields(**f)
    return o


def test_flow_mass_and_vapour_invariant_are_conserved():
    # BGK and Guo forcing carry no mass source: sum rho is exact. The vapour source is
    # -(L_sat/2) d(phi)/dt, so sum U^{n+1} + (L_sat/2) sum phi^n is exact (Sec. 2.2.2).
    o = _random_state(24, 20, 11, eps=0.05, L_sat=1.7)
    m0 = o.field(RHO).sum()
    inv0 = o.field(U).sum() + 0.5 * 1.7 * o.field(PHI_PREV).sum()
    for _ in range(5):
        o.step(10)
        assert o.field(RHO).sum() == pytest.approx(m0, rel=1e-14)
        inv = o.field(U).sum() + 0.5 * 1.7 * o.field(PHI_PREV).sum()
        assert inv == pytest.approx(inv0, rel=1e-13)


def test_phase_field_total_follows_source_at_zero_anisotropy():
    # At eps = 0, a_s = 1 and Eq. (d) is plain streaming: sum phi changes only by the
    # source, sum phi^{n+1} = sum phi^n + (dt/tau0) sum Q^n.
    o = _random_state(20, 18, 12, eps=0.0, D=2.0)
    lam = 2.0 / G["a2"]
    for _ in range(5):
        ph, Uv = o.field(PHI), o.field(U)
        Q = ph - ph ** 3 + lam * Uv * (1 - ph ** 2) ** 2
        o.step(1)
        assert o.field(PHI).sum() == pytest.approx(ph.sum() + 0.008 * Q.sum(), rel=1e-13)


def test_fluid_at_rest_stays_at_rest_exactly():
    nx, ny = 20, 16
    o = _random_state(nx, ny, 13, eps=0.05)
    w = W.Workload("t", nx, ny, 1, flow=True, cx=10, cy=8, R0=4)
    f = W.perturbed_fields(w, 13, amp_phi=0.3)
    o.set_fields(f["phi"], f["U"], full(nx, ny, 1.0), full(nx, ny, 0.0), full(nx, ny, 0.0))
    f0 = o.pops(LAT_F)
    o.step(25)
    np.testing.assert_array_equal(o.pops(LAT_F), f0)
    np.testing.assert_array_equal(o.field(UX), 0.0)
    assert np.abs(f0 - WT[:, None, None]).max() < 1e-16


def test_shear_wave_decays_at_the_lattice_viscosity():
    # Sec. 2.2.1: tau = nu / c_s^2 + 1/2. In vapour a shear wave u_x = A sin(k y) decays as
    # exp(-nu k^2 t) (incompressible Navier-Stokes).
    nx, ny, nu = 4, 64, 0.1
    o = Oracle(nx=nx, ny=ny, nu=nu, flow=True)
    y = np.arange(ny, dtype=float)
    k = 2 * np.pi / ny
    ux = np.tile(0.01 * np.sin(k * y)[:, None], (1, nx))
    o.set_fields(full(nx, ny, -1.0), full(nx, ny, 0.0), full(nx, ny, 1.0), ux, 0 * ux)
    s = np.sin(k * y)

    def amp():
        return (o.field(UX)[:, 0] * s).sum() / (s * s).sum()

    o.step(100)
    a1 = amp()
    o.step(500)
    a2 = amp()
    rate = math.log(a1 / a2) / 500
    assert rate == pytest.approx(nu * k * k, rel=5e-3)


# ------------------------------------------------------------------------------------------
# Symmetries (Sec. 2.1: cos(6 theta) is even and sin(6 theta) odd under both mirrors)
# ------------------------------------------------------------------------------------------

def test_mirror_symmetry_is_bit_exact():
    nx, ny = 32, 28
    w = W.Workload("t", nx, ny, 1, flow=True, eps=0.07, nu=0.05)
    f = W.mirror_fields(w, 21, amp=0.2)
    o = Oracle(nx=nx, ny=ny, **w.params())
    o.set_fields(**f)
    o.step(40)
    ix, iy = (-np.arange(nx)) % nx, (-np.arange(ny)) % ny
    for which in (PHI, U, RHO):
        a = o.field(which)
        np.testing.assert_array_equal(a, a[:, ix])
        np.testing.assert_array_equal(a, a[iy, :])
    ux, uy = o.field(UX), o.field(UY)
    np.testing.assert_array_equal(ux, -ux[:, ix])
    np.testing.assert_array_equal(uy, uy[:, ix])
    np.testing.assert_array_equal(ux, ux[iy, :])
    np.testing.assert_array_equal(uy, -uy[iy, :])
    assert np.abs(ux).max() > 1e-4  # the test is not vacuous


def test_diagonal_symmetry_holds_only_without_anisotropy():
    # x <-> y maps cos(6 theta) to -cos(6 theta): a symmetry of the isotropic model only.
    n = 24
    rng = np.random.Generator(np.random.PCG64(5))

    def symm(a):
        return 0.5 * (a + a.T)

    phi = symm(np.clip(W.seed_fields(W.Workload("t", n, n, 1, cx=12, cy=12, R0=5))["phi"]
                       + 0.2 * rng.uniform(-1, 1, (n, n)), -1, 1))
    Uf = symm(0.3 + 0.05 * rng.uniform(-1, 1, (n, n)))
    rho = symm(1 + 0.02 * rng.uniform(-1, 1, (n, n)))
    a = 0.02 * rng.uniform(-1, 1, (n, n))
    res = {}
    for eps in (0.0, 0.05):
        o = Oracle(nx=n, ny=n, eps=eps, flow=True, nu=0.05)
        o.set_fields(phi, Uf, rho, a, a.T)
        o.step(30)
        res[eps] = (o.field(PHI), o.field(UX), o.field(UY))
    p0, ux0, uy0 = res[0.0]
    np.testing.assert_array_equal(p0, p0.T)
    np.testing.assert_array_equal(ux0, uy0.T)
    p1 = res[0.05][0]
    assert np.abs(p1 - p1.T).max() > 1e-6


def test_free_slip_wall_equals_mirrored_periodic_domain():
    # A free-slip wall reflects populations specularly; the grid with walls at y = -1/2 and
    # y = ny - 1/2 must evolve exactly like a periodic grid of 2 ny rows holding the state
    # and its mirror image.
    nx, ny = 16, 10
    w = W.Workload("t", nx, ny, 1, flow=True, eps=0.05, cx=7.3, cy=3.1, R0=4, nu=0.05)
    f = W.perturbed_fields(w, 31, amp_phi=0.2, amp_u=0.02)
    wall = dict(w.params())
    wall["bc"] = (W.BC_PERIODIC, W.BC_PERIODIC, W.BC_FREESLIP, W.BC_FREESLIP)
    o1 = Oracle(nx=nx, ny=ny, **wall)
    o1.set_fields(**f)
    ext = {k: np.concatenate([v, v[::-1]], axis=0) for k, v in f.items()}
    ext["uy"] = np.concatenate([f["uy"], -f["uy"][::-1]], axis=0)
    o2 = Oracle(nx=nx, ny=2 * ny, **w.params())
    o2.set_fields(**ext)
    o1.step(30)
    o2.step(30)
    for which in (PHI, U, RHO, UX, UY):
        np.testing.assert_allclose(o1.field(which), o2.field(which)[:ny], rtol=0, atol=1e-14)


def test_inlet_outlet_channel_holds_uniform_inflow_exactly():
    # Vapour at the inlet state everywhere is a steady solution of the channel problem of
    # Sec. 3.1.3 (inlet on one side, zero-gradient outlet on the other, free-slip walls).
    nx, ny = 20, 12
    for bc, vel in [((W.BC_INLET, W.BC_OUTLET, W.BC_FREESLIP, W.BC_FREESLIP), (0.03, 0.0)),
                    ((W.BC_OUTLET, W.BC_INLET, W.BC_FREESLIP, W.BC_FREESLIP), (-0.03, 0.0)),
                    ((W.BC_PERIODIC, W.BC_PERIODIC, W.BC_INLET, W.BC_OUTLET), (0.0, 0.03))]:
        o = Oracle(nx=nx, ny=ny, flow=True, U_in=0.25, u_in=0.03, bc=bc, nu=0.05)
        o.set_fields(full(nx, ny, -1.0), full(nx, ny, 0.25), full(nx, ny, 1.0),
                     full(nx, ny, vel[0]), full(nx, ny, vel[1]))
        o.step(20)
        np.testing.assert_allclose(o.field(UX), vel[0], atol=1e-15)
        np.testing.assert_allclose(o.field(UY), vel[1], atol=1e-15)
        np.testing.assert_allclose(o.field(U), 0.25, atol=1e-15)
        np.testing.assert_allclose(o.field(PHI), -1.0, atol=1e-15)
        np.testing.assert_allclose(o.field(RHO), 1.0, atol=1e-14)


def test_outlet_and_walls_keep_uniform_state_on_the_ode_map():
    # Zero-gradient and free-slip ghosts copy the adjacent node, so a uniform state evolves
    # exactly as on a periodic grid.
    nx, ny = 7, 6
    res = []
    for bc in [(W.BC_PERIODIC,) * 4, (W.BC_OUTLET, W.BC_OUTLET, W.BC_FREESLIP, W.BC_OUTLET)]:
        o = Oracle(nx=nx, ny=ny, bc=bc, flow=True)
        o.set_fields(full(nx, ny, 0.2), full(nx, ny, 0.3))
        o.step(15)
        res.append(o.field(PHI))
    np.testing.assert_array_equal(res[0], res[1])


# ------------------------------------------------------------------------------------------
# The pull form of Eq. (d) and the moments of the three collisions
# ------------------------------------------------------------------------------------------

def test_pull_update_satisfies_eq_d_at_every_link():
    # Eq. (d) at collision node x and destination x + c:
    #   a_s^2(x) h(x+c, t+1) + (1 - a_s^2(x)) h(x+c, t) = h*(x),
    # with h* the collided population at x. Flow and vapour: f(x+c, t+1) = f*(x).
    nx, ny = 14, 12
    o = _random_state(nx, ny, 41, eps=0.1)
    hs, gs, fs = o.post_collision(LAT_H), o.post_collision(LAT_G), o.post_collision(LAT_F)
    a2 = o.post_collision(LAT_AS2)
    h0 = o.pops(LAT_H)
    o.step(1)
    h1, g1, f1 = o.pops(LAT_H), o.pops(LAT_G), o.pops(LAT_F)
    assert np.abs(a2 - 1).max() > 1e-3
    for a in range(9):
        # destination array index of x + c_a is a roll by +c_a
        sh = lambda arr: np.roll(arr, shift=(-CY[a], -CX[a]), axis=(0, 1))
        lhs = a2 * sh(h1[a]) + (1 - a2) * sh(h0[a])
        np.testing.assert_allclose(lhs, hs[a], rtol=0, atol=1e-14)
        np.testing.assert_array_equal(sh(g1[a]), gs[a])
        np.testing.assert_array_equal(sh(f1[a]), fs[a])


def test_collision_moments():
    # Moments of the collided populations follow from the equilibria and sources of
    # Sec. 2.2 by the lattice identities sum w = 1, sum w c c = I/3, odd moments zero.
    nx, ny = 12, 10
    eps, L_sat, D, nu = 0.08, 1.4, 2.5, 0.07
    o = _random_state(nx, ny, 43, eps=eps, L_sat=L_sat, D=D, nu=nu)
    d = o.derived()
    h, g, f = o.pops(LAT_H), o.pops(LAT_G), o.pops(LAT_F)
    ph, Uv, pprev = h.sum(0), g.sum(0), o.field(PHI_PREV)
    rho, jx, jy = f.sum(0), (CX[:, None, None] * f).sum(0), (CY[:, None, None] * f).sum(0)
    hs, gs, fs = o.post_collision(LAT_H), o.post_collision(LAT_G), o.post_collision(LAT_F)
    a2 = o.post_collision(LAT_AS2)
    gx, gy = oracle.gradient_periodic(ph)
    a_s = np.where(gx ** 2 + gy ** 2 > 1e-12, aniso_trig(gx, gy, eps), 1.0)
    np.testing.assert_allclose(a2, a_s ** 2, atol=1e-13)
    Nx, Ny = flux_fd(gx, gy, eps)
    Nx = np.where(gx ** 2 + gy ** 2 > 1e-12, Nx, 0.0)
    Ny = np.where(gx ** 2 + gy ** 2 > 1e-12, Ny, 0.0)
    lam = 1.0 * D / G["a2"]
    Q = ph - ph ** 3 + lam * Uv * (1 - ph ** 2) ** 2
    Dphi = 0.008 / 0.16
    eta = a_s ** 2 * Dphi / (1 / 3) + 0.5        # Sec. 2.2.3 relaxation time
    # phase field: zeroth moment gains the source; first moment relaxes to -Dphi N (Eq. (e))
    np.testing.assert_allclose(hs.sum(0), ph + 0.008 * Q, atol=1e-14)
    Jx, Jy = (CX[:, None, None] * h).sum(0), (CY[:, None, None] * h).sum(0)
    np.testing.assert_allclose((CX[:, None, None] * hs).sum(0),
                               (1 - 1 / eta) * Jx - Dphi * Nx / eta, atol=1e-8)
    np.testing.assert_allclose((CY[:, None, None] * hs).sum(0),
                               (1 - 1 / eta) * Jy - Dphi * Ny / eta, atol=1e-8)
    # flow: u = j/(rho + k/2), u* = (1-phi)/2 u, F = -k u*; Guo's term has moments 0, (1 -
    # 1/(2 tau)) F and (1 - 1/(2 tau)) (u F + F u)
    tau = nu * 3 + 0.5
    k = G["h_drag"] * rho * nu * (1 + ph) ** 2 * (1 - ph) / (4 * 2.5 ** 2)
    usx, usy = 0.5 * (1 - ph) * jx / (rho + k / 2), 0.5 * (1 - ph) * jy / (rho + k / 2)
    Fx, Fy = -k * usx, -k * usy
    pf = 1 - 0.5 / tau
    np.testing.assert_allclose(fs.sum(0), rho, atol=1e-14)
    np.testing.assert_allclose((CX[:, None, None] * fs).sum(0),
                               jx - (jx - rho * usx) / tau + pf * Fx, atol=1e-15)
    Pxy = (CX[:, None, None] * CY[:, None, None] * f).sum(0)
    Pxx = (CX[:, None, None] ** 2 * f).sum(0)
    np.testing.assert_allclose(
        (CX[:, None, None] * CY[:, None, None] * fs).sum(0),
        (1 - 1 / tau) * Pxy + rho * usx * usy / tau + pf * (usx * Fy + Fx * usy), atol=1e-15)
    np.testing.assert_allclose(
        (CX[:, None, None] ** 2 * fs).sum(0),
        (1 - 1 / tau) * Pxx + rho * (1 / 3 + usx * usx) / tau + pf * 2 * usx * Fx, atol=1e-15)
    # vapour: q = 1 - phi, tau_g = D q / c_s^2 + 1/2, g^eq = w U (1 + 3 c.u*), source
    tg = 3 * (D * 0.008 / 0.16) * np.clip(1 - ph, 0, 2) + 0.5
    np.testing.assert_allclose(gs.sum(0), Uv - 0.5 * L_sat * (ph - pprev), atol=1e-14)
    Gx = (CX[:, None, None] * g).sum(0)
    np.testing.assert_allclose((CX[:, None, None] * gs).sum(0),
                               (1 - 1 / tg) * Gx + Uv * usx / tg, atol=1e-15)


# ------------------------------------------------------------------------------------------
# Growth of a seed (Sec. 3.1.2 and Sec. 3.2: isotropy without anisotropy, six-fold habit,
# faster growth into the incoming flow)
# ------------------------------------------------------------------------------------------

ANGLES = np.linspace(0, 2 * np.pi, 360, endpoint=False)


def _grown_radii(eps, steps=1500, n=96):
    w = W.C1.with_size(n, n, eps=eps)
    o = Oracle(nx=n, ny=n, **w.params())
    o.set_fields(**W.seed_fields(w))
    o.step(steps)
    return contour_radius(o.field(PHI), w.cx, w.cy, ANGLES), w


def test_isotropic_growth_without_anisotropy():
    R, w = _grown_radii(0.0)
    assert np.isfinite(R).all()
    assert R.mean() > w.R0 + 5  # U0 = 0.35 is far above the critical supersaturation
    assert R.max() / R.min() - 1 < 0.01


def test_six_fold_habit_with_tips_along_sixty_degree_rays():
    R, _ = _grown_radii(0.05)
    F = np.fft.rfft(R) / len(R)
    # a_s = 1 + eps cos(6 theta) is largest at theta = k pi/3: R(theta) gains a positive
    # cos(6 theta) component that dominates every mode that is not one of its harmonics
    assert F[6].real > 0.1
    assert abs(F[6].imag) < 0.05 * F[6].real
    others = [abs(F[m]) for m in range(1, 18) if m % 6]
    assert abs(F[6]) > 20 * max(others)


def test_upstream_tip_outgrows_downstream_tip():
    # Sec. 3.1.3: the tip facing the inflow sees the steeper supersaturation gradient.
    w = W.C2.with_size(160, 96)
    o = Oracle(nx=w.nx, ny=w.ny, **w.params())
    o.set_fields(**W.seed_fields(w))
    o.step(1500)
    from tests.helpers import tip_x
    phi = o.field(PHI)
    up = w.cx - tip_x(phi, w.cy, w.cx, -1)
    down = tip_x(phi, w.cy, w.cx, +1) - w.cx
    assert up > w.R0 and down > w.R0
    assert up - down > 0.2


def test_ghost_rules_at_channel_faces():
    # Channel of Sec. 3.1.3 / Sec. 3.2.2: inlet at -x, zero-gradient outlet at +x, free-slip
    # walls at -y/+y. (1) phi seen by the gradient beyond a face: -1 (vapour) at the inlet,
    # the adjacent value at the outlet, the mirror image at a wall -- i.e. numpy's 'constant',
    # 'edge' and 'symmetric' padding. (2) Populations pulled from beyond the outlet are the
    # collided populations of the adjacent node, same direction.
    nx, ny = 14, 10
    w = W.Workload("t", nx, ny, 1, flow=True, eps=0.08, cx=6, cy=5, R0=3, nu=0.05, U_in=0.2,
                   u_in=0.02, bc=(W.BC_INLET, W.BC_OUTLET, W.BC_FREESLIP, W.BC_FREESLIP))
    f = W.perturbed_fields(w, 51, amp_phi=0.3, amp_u=0.02)
    o = Oracle(nx=nx, ny=ny, **w.params())
    o.set_fields(**f)
    ph = o.field(PHI)
    padded = np.pad(ph, ((1, 1), (0, 0)), mode="symmetric")
    padded = np.pad(padded, ((0, 0), (1, 0)), mode="constant", constant_values=-1.0)
    padded = np.pad(padded, ((0, 0), (0, 1)), mode="edge")
    gx, gy = oracle.gradient_periodic(padded)
    gx, gy = gx[1:-1, 1:-1], gy[1:-1, 1:-1]
    a_s = np.where(gx ** 2 + gy ** 2 > 1e-12, aniso_trig(gx, gy, 0.08), 1.0)
    fs, hs, a2 = o.post_collision(LAT_F), o.post_collision(LAT_H), o.post_collision(LAT_AS2)
    np.testing.assert_allclose(a2, a_s ** 2, atol=1e-13)
    h0 = o.pops(LAT_H)
    o.step(1)
    f1, h1 = o.pops(LAT_F), o.pops(LAT_H)
    x = nx - 1
    for a in range(9):
        if CX[a] != -1:
            continue
        for j in range(ny):
            js = j - CY[a]
            if not 0 <= js < ny:
                continue
            assert f1[a, j, x] == fs[a, js, x]
            lhs = a2[js, x] * h1[a, j, x] + (1 - a2[js, x]) * h0[a, j, x]
            assert lhs == pytest.approx(hs[a, js, x], abs=1e-14)


# ------------------------------------------------------------------------------------------
# Threaded node loops: the timing baseline on all host cores computes the same bits
# ------------------------------------------------------------------------------------------

@pytest.mark.parametrize("faces", ["periodic", "channel"])
def test_threaded_oracle_is_bit_identical_to_one_thread(faces):
    # Rows are split across threads; no node reads another's outputs within a sweep and
    # nothing is summed across nodes, so every population must come out bit for bit equal.
    bc = ((W.BC_PERIODIC,) * 4 if faces == "periodic"
          else (W.BC_INLET, W.BC_OUTLET, W.BC_FREESLIP, W.BC_FREESLIP))
    w = W.Workload("threads", 61, 47, 6, flow=True, eps=0.05, D=2.0, U0=0.3, nu=0.05,
                   cx=30.0, cy=23.0, R0=7.0, bc=bc, u_in=0.02, U_in=0.3)
    f = W.perturbed_fields(w, 2024)
    runs = []
    for threads in (1, 4):
        oracle.set_threads(threads)
        try:
            o = Oracle(nx=w.nx, ny=w.ny, **w.params())
            o.set_fields(**f)
            o.step(w.steps)
            runs.append([o.pops(L) for L in (LAT_F, LAT_G, LAT_H)] + [o.field(PHI_PREV)])
        finally:
            oracle.set_threads(1)
    for a, b in zip(*runs):
        assert np.array_equal(a, b)


def test_float32_rounding_option_rounds_the_state_only():
    # The storage-floor runs of the parity tests round the state to float32 after each step:
    # populations and the phi history become the nearest float32, nothing else changes.
    w = W.Workload("r32", 24, 20, 1, flow=True, eps=0.05, D=2.0, U0=0.3, nu=0.05,
                   cx=12.0, cy=10.0, R0=5.0)
    o = Oracle(nx=w.nx, ny=w.ny, **w.params())
    o.set_fields(**W.perturbed_fields(w, 5))
    o.step(2)
    before = [o.pops(L) for L in (LAT_F, LAT_G, LAT_H)] + [o.field(PHI_PREV)]
    o.round_to_float32()
    after = [o.pops(L) for L in (LAT_F, LAT_G, LAT_H)] + [o.field(PHI_PREV)]
    for b, a in zip(before, after):
        assert np.array_equal(a, b.astype(np.float32).astype(np.float64))
        assert not np.array_equal(a, b)
    assert o.steps_done == 2

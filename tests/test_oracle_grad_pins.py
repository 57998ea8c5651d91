"""Pins of the oracle's forward-mode gradient (dual numbers through the FP64 iteration),
which the GPU adjoint is checked against. Central differences of the plain double oracle,
closed forms of zero steps and of one step from a uniform state."""
import numpy as np
import pytest

import oracle
from paper_2101_07163_gb300 import workloads as W


def small(flow=True, bc=(W.BC_PERIODIC,) * 4, lam=0.0):
    w = W.Workload("g", 20, 16, 1, flow=flow, eps=0.06, D=2.0, U0=0.35, U_in=0.3,
                   u_in=0.02 if flow else 0.0, nu=0.05, bc=bc, cx=9, cy=8, R0=5.0, lam=lam)
    return w


def loss(w, fields, steps, wphi, wU, **over):
    p = oracle.make_params(w.nx, w.ny, **{**w.params(), **over})
    o = oracle.Oracle(p)
    o.set_fields(**fields)
    o.step(steps)
    return float((wphi * o.field(oracle.PHI)).sum() + (wU * o.field(oracle.U)).sum())


CASES = [
    dict(flow=True),
    dict(flow=False),
    dict(flow=True, bc=(W.BC_INLET, W.BC_OUTLET, W.BC_FREESLIP, W.BC_FREESLIP)),
    dict(flow=True, lam=5.0),
]


@pytest.mark.parametrize("case", CASES, ids=["flow", "noflow", "faces", "lambda_given"])
def test_dual_gradient_matches_central_differences(case):
    w = small(**case)
    rng = np.random.default_rng(4)
    f = W.perturbed_fields(w, 3, amp_u=0.02)
    if not w.flow:
        f = {k: f[k] for k in ("phi", "U")}
    shape = (w.ny, w.nx)
    wphi, wU = rng.uniform(-1, 1, shape), rng.uniform(-1, 1, shape)
    dirs = {k: rng.uniform(-1, 1, shape) for k in f}
    steps = 25
    p = oracle.make_params(w.nx, w.ny, **w.params())
    g = oracle.grad_run(p, f, steps, wphi, wU, dirs)
    assert g["L"] == pytest.approx(loss(w, f, steps, wphi, wU), rel=1e-13, abs=1e-13)
    h = 1e-6
    lam0 = oracle.Oracle(p).derived()["lambda"]

    def cd(**kw):
        fp = {k: (v + h * dirs[k]) for k, v in f.items()} if kw.get("init") else f
        fm = {k: (v - h * dirs[k]) for k, v in f.items()} if kw.get("init") else f
        name = kw.get("par")
        if name is None:
            return (loss(w, fp, steps, wphi, wU) - loss(w, fm, steps, wphi, wU)) / (2 * h)
        base = {"eps": w.eps, "D": w.D, "lam": lam0}[name]
        up = loss(w, f, steps, wphi, wU, **{name: base + h})
        dn = loss(w, f, steps, wphi, wU, **{name: base - h})
        return (up - dn) / (2 * h)

    fd = {"eps": cd(par="eps"), "D": cd(par="D"), "lambda": cd(par="lam"), "init": cd(init=True)}
    scale = max(abs(v) for v in fd.values())
    for k, v in fd.items():
        assert abs(g[k] - v) <= 2e-7 * scale + 1e-9, (k, g[k], v)


def test_zero_steps_closed_form():
    # L = sum wphi phi0 + wU U0 exactly: no parameter enters the moments of the initial state
    w = small()
    rng = np.random.default_rng(5)
    f = W.perturbed_fields(w, 4, amp_u=0.02)
    shape = (w.ny, w.nx)
    wphi, wU = rng.uniform(-1, 1, shape), rng.uniform(-1, 1, shape)
    dirs = {k: rng.uniform(-1, 1, shape) for k in f}
    g = oracle.grad_run(oracle.make_params(w.nx, w.ny, **w.params()), f, 0, wphi, wU, dirs)
    assert g["eps"] == 0.0 and g["D"] == 0.0 and g["lambda"] == 0.0
    want = float((wphi * dirs["phi"]).sum() + (wU * dirs["U"]).sum())
    assert g["init"] == pytest.approx(want, rel=1e-12)
    assert g["L"] == pytest.approx(float((wphi * f["phi"]).sum() + (wU * f["U"]).sum()),
                                   rel=1e-12)


@pytest.mark.parametrize("lam_given", [False, True])
def test_one_step_of_a_uniform_state(lam_given):
    # Uniform phi, U, fluid at rest: no gradient, so a_s = 1 and N = 0 for any eps; h = h^eq,
    # and one step gives phi^1 = phi + Q dt/tau0 with Q = phi - phi^3 + lambda U (1-phi^2)^2
    # (Sec. 2.2.3). L = sum phi^1: dL/dlambda = n dt/tau0 U (1-phi^2)^2, dL/deps = 0, and
    # dL/dD = dL/dlambda * tau0/(a2 W0^2) when lambda follows beta = 0 (0 when it is given).
    nx, ny, ph, U = 12, 10, 0.3, 0.4
    w = W.Workload("u", nx, ny, 1, flow=False, eps=0.05, D=2.0, lam=4.0 if lam_given else 0.0)
    p = oracle.make_params(nx, ny, **w.params())
    f = {"phi": np.full((ny, nx), ph), "U": np.full((ny, nx), U)}
    ones, zeros = np.ones((ny, nx)), np.zeros((ny, nx))
    g = oracle.grad_run(p, f, 1, ones, zeros)
    dlam = nx * ny * w.dt / w.tau0 * U * (1 - ph * ph) ** 2
    assert g["lambda"] == pytest.approx(dlam, rel=1e-12)
    assert g["eps"] == 0.0
    if lam_given:
        assert g["D"] == 0.0
    else:
        assert g["D"] == pytest.approx(dlam * w.tau0 / (0.6267 * w.W0 ** 2), rel=1e-12)


def test_differentiating_along_the_own_trajectory_changes_nothing():
    # replacing the values by those the run produces itself must leave every derivative as is
    w = small()
    f = W.perturbed_fields(w, 6, amp_u=0.02)
    rng = np.random.default_rng(7)
    shape = (w.ny, w.nx)
    wphi, wU = rng.uniform(-1, 1, shape), rng.uniform(-1, 1, shape)
    dirs = {k: rng.uniform(-1, 1, shape) for k in f}
    p = oracle.make_params(w.nx, w.ny, **w.params())
    o = oracle.Oracle(p)
    o.set_fields(**f)

    def state():
        return np.concatenate([o.pops(oracle.LAT_H), o.pops(oracle.LAT_G), o.pops(oracle.LAT_F),
                               o.field(oracle.PHI)[None], o.field(oracle.PHI_PREV)[None]])

    traj = [state()]
    for _ in range(6):
        o.step(1)
        traj.append(state())
    plain = oracle.grad_run(p, f, 6, wphi, wU, dirs)
    along = oracle.grad_run(p, f, 6, wphi, wU, dirs, along=np.stack(traj))
    assert plain == along
    # and a different trajectory does change them (the option is not ignored)
    moved = oracle.grad_run(p, f, 6, wphi, wU, dirs, along=np.stack(traj) * (1 + 1e-3))
    assert moved["eps"] != plain["eps"]

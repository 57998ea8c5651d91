"""GPU discrete adjoint of the step (lbmice_tape_*) against the oracle's exact forward-mode
gradient, central finite differences of the GPU forward, and itself across checkpoint
intervals. The adjoint is the transpose of the Jacobian the oracle's dual numbers apply, so
sum(init adjoints * direction) and the parameter gradients must equal the oracle's
directional derivatives up to the FP32 rounding of the GPU forward."""
import numpy as np
import pytest

import oracle
from paper_2101_07163_gb300 import lbmice
from paper_2101_07163_gb300 import workloads as W

pytestmark = pytest.mark.gpu

KEYS = ("eps", "D", "lambda", "init")
FIELD_OF = {"phi": "phi0", "U": "U0", "rho": "rho0", "ux": "ux0", "uy": "uy0"}


def case(flow, nx=48, ny=40, lam=0.0):
    # phi is kept inside (-0.9, 0.9): q(phi) = 1 - phi is clamped to [0, 2], and at phi = +-1
    # exactly FP32 and FP64 trajectories can sit on opposite sides of the clamp's corner and
    # take different (both valid) one-sided derivatives there
    w = W.Workload("adj", nx, ny, 1, flow=flow, eps=0.06, D=2.0, U0=0.35, nu=0.05,
                   cx=nx * 0.45, cy=ny * 0.5, R0=8.0, lam=lam)
    f = W.perturbed_fields(w, 7, amp_phi=0.1, amp_u=0.02)
    f["phi"] = 0.9 * f["phi"]
    if not flow:
        f = {k: f[k] for k in ("phi", "U")}
    return w, f


def gpu_gradient(w, f, steps, wphi, wU, dirs, every=5):
    lat = lbmice.Lattice(w.nx, w.ny, **w.params())
    lat.set_fields(**f)
    tape = lbmice.Tape(lat, every)
    tape.record(steps)
    grads, init = tape.backward(wphi, wU)
    out = dict(grads)
    out["init"] = float(sum((init[FIELD_OF[k]].astype(np.float64) * d).sum()
                            for k, d in dirs.items()))
    tape.close()
    lat.close()
    return out, init


def seeds(w, seed):
    rng = np.random.default_rng(seed)
    shape = (w.ny, w.nx)
    return rng.uniform(-1, 1, shape), rng.uniform(-1, 1, shape), rng


@pytest.mark.parametrize("flow,lam", [(True, 0.0), (False, 0.0), (True, 5.0)],
                         ids=["flow", "noflow", "lambda_given"])
def test_one_step_adjoint_equals_the_exact_gradient(flow, lam):
    # every term of the reverse step against the exact FP64 derivative of one step
    w, f = case(flow, lam=lam)
    wphi, wU, rng = seeds(w, 11)
    dirs = {k: rng.uniform(-1, 1, (w.ny, w.nx)) for k in f}
    got, _ = gpu_gradient(w, f, 1, wphi, wU, dirs)
    ref = oracle.grad_run(oracle.make_params(w.nx, w.ny, **w.params()), f, 1, wphi, wU, dirs)
    scale = max(abs(ref[k]) for k in KEYS)
    err = {k: abs(got[k] - ref[k]) / scale for k in KEYS}
    assert max(err.values()) < 2e-5, (err, got, ref)


def gpu_trajectory(w, f, steps):
    """The GPU's initial state and its state after every step: planes h0..h8, g0..g8,
    [f0..f8,] phi, phi history."""
    lat = lbmice.Lattice(w.nx, w.ny, **w.params())
    lat.set_fields(**f)

    def state():
        return np.concatenate([lat.pops(), lat.field(lbmice.PHI)[None],
                               lat.field(lbmice.PHI_PREV)[None]])

    out = [state()]
    for _ in range(steps):
        lat.step(1)
        out.append(state())
    lat.close()
    return np.stack(out).astype(np.float64)


CX = np.array([0, 1, 0, -1, 0, 1, -1, -1, 1], dtype=np.float64)[:, None, None]
CY = np.array([0, 0, 1, 0, -1, 1, 1, -1, -1], dtype=np.float64)[:, None, None]


def gpu_moments(block):
    """The moments the GPU's initial state encodes (the point its initialisation adjoint is
    linearised at): phi from its phi plane, U = sum g, rho = sum f, u = sum c f / rho."""
    out = {"phi": block[-2], "U": block[9:18].sum(0)}
    if block.shape[0] == 29:
        fp = block[18:27]
        rho = fp.sum(0)
        out.update(rho=rho, ux=(CX * fp).sum(0) / rho, uy=(CY * fp).sum(0) / rho)
    return out


@pytest.mark.parametrize("flow", [True, False], ids=["flow", "noflow"])
@pytest.mark.parametrize("steps", [17, 40])
def test_adjoint_equals_the_exact_gradient_along_the_same_trajectory(flow, steps):
    # Over many steps the gradient of a noisy state is ill-conditioned where |grad phi| is
    # small (the interface normal n = g/|g| moves by dg/|g|), so FP32 and FP64 trajectories
    # give gradients that differ far beyond FP32 rounding. Differentiating the oracle along the
    # GPU's own states (and linearising its initialisation at the moments the GPU's initial
    # state encodes) removes that: both linearise every map at the same points, and only the
    # FP32 evaluation of the derivatives remains, amplified by the same conditioning over the
    # steps. Measured: eps, D, lambda and the U0, rho0, u0 directions within 4e-6 to 2.5e-5
    # (bound 1e-4); the phi0 direction, which passes the 1/|g| terms of the initial
    # anisotropy and the tangential projection of the normal's adjoint, within 4e-5 at 17
    # steps and 4e-4 at 40 (bound 1e-3).
    w, f = case(flow)
    wphi, wU, rng = seeds(w, 16)
    dirs = {k: rng.uniform(-1, 1, (w.ny, w.nx)) for k in f}
    got, init = gpu_gradient(w, f, steps, wphi, wU, dirs)
    traj = gpu_trajectory(w, f, steps)
    p = oracle.make_params(w.nx, w.ny, **w.params())
    zero = np.zeros((w.ny, w.nx))
    rest = {k: (zero if k == "phi" else d) for k, d in dirs.items()}
    ref = oracle.grad_run(p, gpu_moments(traj[0]), steps, wphi, wU, rest, along=traj)
    got_rest = float(sum((init[FIELD_OF[k]].astype(np.float64) * d).sum()
                         for k, d in rest.items()))
    scale = max(abs(ref[k]) for k in KEYS)
    for k in ("eps", "D", "lambda"):
        assert abs(got[k] - ref[k]) < 1e-4 * scale, (k, got[k], ref[k])
    assert abs(got_rest - ref["init"]) < 1e-4 * scale, (got_rest, ref["init"])
    only_phi = {k: (d if k == "phi" else zero) for k, d in dirs.items()}
    ref_phi = oracle.grad_run(p, gpu_moments(traj[0]), steps, wphi, wU, only_phi,
                              along=traj)["init"]
    got_phi = float((init["phi0"].astype(np.float64) * dirs["phi"]).sum())
    assert abs(got_phi - ref_phi) < 1e-3 * abs(ref_phi), (got_phi, ref_phi)


def test_checkpoint_interval_does_not_change_the_gradient():
    # every segment is recomputed from its checkpoint by the same deterministic kernels
    w, f = case(True)
    wphi, wU, rng = seeds(w, 13)
    dirs = {k: rng.uniform(-1, 1, (w.ny, w.nx)) for k in f}
    a, ia = gpu_gradient(w, f, 23, wphi, wU, dirs, every=4)
    b, ib = gpu_gradient(w, f, 23, wphi, wU, dirs, every=100)
    c, ic = gpu_gradient(w, f, 23, wphi, wU, dirs, every=1)
    for k in ("eps", "D", "lambda"):
        assert a[k] == b[k] == c[k]
    for k in ia:
        np.testing.assert_array_equal(ia[k], ib[k])
        np.testing.assert_array_equal(ia[k], ic[k])


@pytest.mark.parametrize("flow", [True, False], ids=["flow", "noflow"])
def test_fused_and_separate_reverse_pull_give_the_same_bits(flow, monkeypatch):
    # grids beyond the L2 add the pull's own-population term inside the collision adjoint
    # (B from its own pass), smaller ones in a read-modify-write pass; forced either way here
    w, f = case(flow, nx=64, ny=48)
    wphi, wU, rng = seeds(w, 15)
    dirs = {k: rng.uniform(-1, 1, (w.ny, w.nx)) for k in f}
    got = {}
    for mode in ("0", "1"):
        monkeypatch.setenv("LBMICE_ADJ_FUSED", mode)
        got[mode] = gpu_gradient(w, f, 19, wphi, wU, dirs, every=6)
    a, ia = got["0"]
    b, ib = got["1"]
    for k in ("eps", "D", "lambda", "init"):
        assert a[k] == b[k], k
    for k in ia:
        np.testing.assert_array_equal(ia[k], ib[k])


def test_zero_steps_gives_the_seeds_back():
    w, f = case(True)
    wphi, wU, rng = seeds(w, 14)
    dirs = {k: rng.uniform(-1, 1, (w.ny, w.nx)) for k in f}
    got, init = gpu_gradient(w, f, 0, wphi, wU, dirs)
    assert got["eps"] == got["D"] == got["lambda"] == 0.0
    np.testing.assert_allclose(init["phi0"], wphi, atol=2e-6)
    np.testing.assert_allclose(init["U0"], wU, atol=2e-6)


def test_tape_refuses_unsupported_grids_and_outside_steps():
    w = W.Workload("r", 32, 24, 1, flow=True,
                   bc=(W.BC_INLET, W.BC_OUTLET, W.BC_FREESLIP, W.BC_FREESLIP))
    lat = lbmice.Lattice(w.nx, w.ny, **w.params())
    lat.set_fields(**W.seed_fields(w))
    with pytest.raises(lbmice.LbmiceError):
        lbmice.Tape(lat)
    w2 = W.Workload("r", 32, 24, 1, flow=True)
    lat2 = lbmice.Lattice(w2.nx, w2.ny, storage="f16", **w2.params())
    with pytest.raises(lbmice.LbmiceError):
        lbmice.Tape(lat2)
    lat3 = lbmice.Lattice(w2.nx, w2.ny, **w2.params())
    lat3.set_fields(**W.seed_fields(w2))
    tape = lbmice.Tape(lat3, 10)
    tape.record(5)
    lat3.step(1)  # outside the tape
    with pytest.raises(lbmice.LbmiceError) as ei:
        tape.record(1)
    assert ei.value.code == lbmice.EINVAL
    with pytest.raises(lbmice.LbmiceError):
        tape.backward(np.zeros((w2.ny, w2.nx)))


def test_rollout_autograd_matches_the_tape():
    import torch
    w, f = case(False, nx=40, ny=32)
    dev = torch.device("cuda")
    phi0 = torch.tensor(f["phi"], device=dev, requires_grad=True)
    U0 = torch.tensor(0.35, dtype=torch.float64, device=dev, requires_grad=True)
    eps = torch.tensor(w.eps, dtype=torch.float64, device=dev, requires_grad=True)
    D = torch.tensor(w.D, dtype=torch.float64, device=dev, requires_grad=True)
    from paper_2101_07163_gb300 import adjoint
    phiT = adjoint.rollout(phi0, U0, eps, D, nsteps=37, every=10)
    wphi = torch.tensor(seeds(w, 15)[0], device=dev)
    (phiT.double() * wphi).sum().backward()
    # the same run through the tape directly, U0 as a uniform field
    lat = lbmice.Lattice(w.nx, w.ny, **w.params())
    lat.set_fields(phi=f["phi"], U=np.full((w.ny, w.nx), 0.35))
    tape = lbmice.Tape(lat, 10)
    tape.record(37)
    np.testing.assert_array_equal(phiT.detach().cpu().numpy(), lat.field(lbmice.PHI))
    grads, init = tape.backward(wphi.cpu().numpy())
    assert eps.grad.item() == grads["eps"] and D.grad.item() == grads["D"]
    np.testing.assert_array_equal(phi0.grad.cpu().numpy(), init["phi0"].astype(np.float64))
    assert U0.grad.item() == pytest.approx(float(init["U0"].astype(np.float64).sum()), rel=1e-6)


def test_rollout_backward_can_run_twice_on_a_retained_graph():
    # backward(retain_graph=True) then backward again sweeps the same tape twice: the second
    # sweep gives the same gradients, which autograd adds to the first
    import torch
    from paper_2101_07163_gb300 import adjoint
    w, f = case(False, nx=36, ny=28)
    dev = torch.device("cuda")
    phi0 = torch.tensor(f["phi"], device=dev, requires_grad=True)
    eps = torch.tensor(w.eps, dtype=torch.float64, device=dev, requires_grad=True)
    D = torch.tensor(w.D, dtype=torch.float64, device=dev, requires_grad=True)
    U0 = torch.tensor(0.35, dtype=torch.float64, device=dev, requires_grad=True)
    loss = (adjoint.rollout(phi0, U0, eps, D, nsteps=23, every=8).double() ** 2).sum()
    loss.backward(retain_graph=True)
    first = (eps.grad.item(), D.grad.item(), U0.grad.item(), phi0.grad.clone())
    loss.backward()
    assert eps.grad.item() == 2 * first[0] and D.grad.item() == 2 * first[1]
    assert U0.grad.item() == pytest.approx(2 * first[2], rel=1e-12)
    assert torch.equal(phi0.grad, 2 * first[3])


# ---- the gradient workload: 512^2 periodic, f + g + h, seed R = 6 at the centre, start
# parameters (U0, eps, D) = (0.3, 0.04, 2.0), target run (0.4, 0.06, 2.5), 3000 steps,
# checkpoints every 100 steps -------------------------------------------------------------

def grad_workload(n):
    return W.Workload("grad", n, n, 3000, flow=True, eps=0.04, D=2.0, U0=0.3, cx=n / 2,
                      cy=n / 2, R0=6.0)


@pytest.mark.slow
def test_gradient_workload_copy_64_matches_the_oracle():
    # the same physics on a 64^2 copy over all 3000 steps: measured agreement 2e-5 relative
    # in every direction (FP32 forward and adjoint against the exact FP64 derivative)
    w = grad_workload(64)
    f = W.seed_fields(w)
    rng = np.random.default_rng(21)
    wphi, wU = rng.uniform(-1, 1, (64, 64)), rng.uniform(-1, 1, (64, 64))
    dirs = {"phi": 0.1 * rng.uniform(-1, 1, (64, 64)), "U": np.ones((64, 64))}
    got, _ = gpu_gradient(w, f, w.steps, wphi, wU, dirs, every=100)
    ref = oracle.grad_run(oracle.make_params(64, 64, **w.params()), f, w.steps, wphi, wU, dirs)
    for k in KEYS:
        assert abs(got[k] - ref[k]) <= 2e-4 * abs(ref[k]), (k, got[k], ref[k])


@pytest.mark.slow
def test_gradient_workload_512_matches_central_differences():
    # L = sum (phi_T(U0, eps, D) - phi_T(target))^2 at full size; central differences with
    # h = 1e-3 of the same FP32 forward. Measured agreement 5e-5 (U0), 1.1e-4 (eps), 2e-5 (D);
    # the O(h^2) truncation and the FP32 noise of L over 2h stay below 1e-4.
    import torch
    from paper_2101_07163_gb300 import adjoint
    w = grad_workload(512)
    dev = torch.device("cuda")
    phi0 = torch.tensor(W.seed_fields(w)["phi"], device=dev)

    def t(v, grad=False):
        return torch.tensor(v, dtype=torch.float64, device=dev, requires_grad=grad)

    def run(U0, eps, D):
        return adjoint.rollout(phi0, U0, eps, D, nsteps=w.steps, every=100, flow=True)

    with torch.no_grad():
        target = run(t(0.4), t(0.06), t(2.5)).double()
    U0, eps, D = t(0.3, True), t(0.04, True), t(2.0, True)
    ((run(U0, eps, D).double() - target) ** 2).sum().backward()
    got = {"U0": U0.grad.item(), "eps": eps.grad.item(), "D": D.grad.item()}
    base = {"U0": 0.3, "eps": 0.04, "D": 2.0}
    h = 1e-3

    def L(**kw):
        p = dict(base, **kw)
        with torch.no_grad():
            return float(((run(t(p["U0"]), t(p["eps"]), t(p["D"])).double() - target) ** 2).sum())

    for k, v in base.items():
        fd = (L(**{k: v + h}) - L(**{k: v - h})) / (2 * h)
        assert abs(got[k] - fd) <= 1e-3 * abs(fd), (k, got[k], fd)

"""Seeded synthetic workloads: grids, parameters and initial moment fields.

This module holds none of the lattice-Boltzmann arithmetic. It only states the physical
parameters of the workloads (the paper's validation units W0 = tau0 = 1, dx = 0.4,
dt = 0.008, Sec. 3.1.2-3.1.3) and builds the initial fields phi, U, rho, u that both the
CUDA path and the test oracle turn into populations on their own.

Initial crystal: a circular seed of radius R0 cells, phi = tanh((R0 - r) dx / (sqrt(2) W0)),
+1 in the ice and -1 in the vapour. Vapour: uniform supersaturation U0. Fluid: rho = 1 and,
where the flow lattice is active, the inflow velocity weighted by the liquid fraction
(1 - phi)/2 so that the ice starts at rest.
"""
from __future__ import annotations

import dataclasses
import math

import numpy as np

BC_PERIODIC, BC_INLET, BC_OUTLET, BC_FREESLIP = 0, 1, 2, 3


@dataclasses.dataclass
class Workload:
    name: str
    nx: int
    ny: int
    steps: int
    # physical parameters (W0/tau0 units; u_in and nu in lattice units)
    dx: float = 0.4
    dt: float = 0.008
    W0: float = 1.0
    tau0: float = 1.0
    D: float = 2.0
    lam: float = 0.0  # <= 0: beta = 0 choice lambda = tau0 D / (a2 W0^2)
    L_sat: float = 1.0
    eps: float = 0.05
    kappa_N: float = 1.0
    U0: float = 0.35
    U_in: float = 0.0
    u_in: float = 0.0
    nu: float = 0.016
    bc: tuple = (BC_PERIODIC,) * 4
    flow: bool = False
    stencil: int = 4  # gradient stencil (Sec. 3.1.1): 2, 4, 6, 8
    fold: int = 6     # anisotropy symmetry: 6 (ice) or 4 (the validation case)
    # seed
    cx: float = 0.0
    cy: float = 0.0
    R0: float = 6.0

    def params(self) -> dict:
        """Keyword arguments shared by the oracle and the CUDA binding."""
        return dict(dx=self.dx, dt=self.dt, W0=self.W0, tau0=self.tau0, D=self.D,
                    lam=self.lam, L_sat=self.L_sat, eps=self.eps, kappa_N=self.kappa_N,
                    U_in=self.U_in, u_in=self.u_in, nu=self.nu, bc=tuple(self.bc),
                    flow=self.flow, stencil=self.stencil, fold=self.fold)

    def to_dict(self) -> dict:
        """Every field, JSON-serialisable (the face kinds as a list)."""
        d = dataclasses.asdict(self)
        d["bc"] = list(self.bc)
        return d

    @classmethod
    def from_dict(cls, d: dict) -> "Workload":
        """The inverse of to_dict; unknown keys are refused."""
        names = {f.name for f in dataclasses.fields(cls)}
        extra = set(d) - names
        if extra:
            raise ValueError(f"unknown workload keys: {sorted(extra)}")
        kw = dict(d)
        if "bc" in kw:
            kw["bc"] = tuple(int(b) for b in kw["bc"])
        return cls(**kw)

    def with_size(self, nx: int, ny: int, **kw) -> "Workload":
        """The same physics on another grid, the seed kept at the same relative place."""
        return dataclasses.replace(self, nx=nx, ny=ny, cx=self.cx * nx / self.nx,
                                   cy=self.cy * ny / self.ny, **kw)

    @property
    def lattices(self) -> int:
        return 3 if self.flow else 2

    def inflow_vector(self) -> tuple[float, float]:
        for face, (vx, vy) in enumerate([(1, 0), (-1, 0), (0, 1), (0, -1)]):
            if self.bc[face] == BC_INLET:
                return self.u_in * vx, self.u_in * vy
        return 0.0, 0.0


# 128 x 128 periodic, phase field + vapour only (flow at rest), seed R0 = 6 at the centre.
C1 = Workload("hg_periodic_128x128", 128, 128, 2000, D=2.0, eps=0.05, U0=0.35,
              cx=64, cy=64, R0=6.0)
# 512 x 384 ventilated channel, all three lattices: inlet at -x (u = 0.02, U = 0.3),
# zero-gradient outlet at +x, free-slip walls at -y/+y, seed R0 = 8 at (160, 192).
C2 = Workload("ventilated_512x384", 512, 384, 20000, D=2.0, eps=0.05, U0=0.3, U_in=0.3,
              u_in=0.02, nu=0.016, bc=(BC_INLET, BC_OUTLET, BC_FREESLIP, BC_FREESLIP),
              flow=True, cx=160, cy=192, R0=8.0)
# 2048 x 2048 periodic plate-regime snowflake, all three lattices, seed R0 = 10.
C3 = Workload("plate_periodic_2048x2048", 2048, 2048, 50000, D=3.0, eps=0.05, U0=0.5,
              flow=True, cx=1024, cy=1024, R0=10.0)

# ---- method variants and the paper's other parameter sets (units W0 = tau0 = 1) ------------
# Table 2 (Sec. 3.2): plate-regime morphologies on 400 x 400 with W0 = 1.25 dx, tau0 = 20 dt
# (dx = 0.8, dt = 0.05), eps = 0.05, lambda = 3, D from the beta = 0 relation
# D = a2 lambda W0^2 / tau0; U0 and L_sat per morphology, seed R0 = 10 at the centre.
A2 = 0.6267
TABLE2 = [("solid_plate", 0.4, 2.0), ("stellar_plate_I", 0.5, 1.8), ("sectored_plate", 0.5, 1.6),
          ("stars", 0.6, 1.0), ("fern_dendrite", 0.8, 1.6), ("fernlike_stellar", 0.7, 1.6),
          ("stellar_plate_II", 0.5, 1.2)]
TABLE2_WORKLOADS = [
    Workload(f"table2_{i + 1}_{name}_400x400", 400, 400, 20000, dx=0.8, dt=0.05, lam=3.0,
             D=A2 * 3.0, eps=0.05, U0=U0, L_sat=L_sat, cx=200, cy=200, R0=10.0)
    for i, (name, U0, L_sat) in enumerate(TABLE2)]
# Four-fold validation system (Sec. 3.1.2): dx = 0.4, dt = 0.008, D = 4, lambda = 6.3826
# (beta = 0), eps = 0.05 with cos(4 theta), seed R0 = 10 at the centre; U0 = 0.3 on 1000^2,
# U0 = 0.55 on 500^2.
FOURFOLD_030 = Workload("fourfold_U030_1000x1000", 1000, 1000, 130000, D=4.0, eps=0.05, U0=0.3,
                        fold=4, cx=500, cy=500, R0=10.0)
FOURFOLD_055 = Workload("fourfold_U055_500x500", 500, 500, 50000, D=4.0, eps=0.05, U0=0.55,
                        fold=4, cx=250, cy=250, R0=10.0)
# Gradient-isotropy system (Sec. 3.1.1): 800^2, dx/W0 = 0.8, dt/tau0 = 0.096, D = 1 (W0^2/tau0),
# lambda = 10, eps = 0.05 six-fold, driving U0 = 0.3 (the undercooling 0.3), seed R0 = 10 at the
# centre, 10^5 steps; one workload per stencil.
ISOTROPY = {s: Workload(f"isotropy_E{s}_800x800", 800, 800, 100000, dx=0.8, dt=0.096, D=1.0,
                        lam=10.0, eps=0.05, U0=0.3, cx=400, cy=400, R0=10.0, stencil=s)
            for s in (2, 4, 6, 8)}

WORKLOADS = {w.name: w for w in (C1, C2, C3, FOURFOLD_030, FOURFOLD_055, *TABLE2_WORKLOADS,
                                 *ISOTROPY.values())}


def seed_fields(w: Workload) -> dict:
    """Initial moments of a workload: circular seed, uniform U0, rho = 1, inflow velocity."""
    y, x = np.mgrid[0:w.ny, 0:w.nx].astype(np.float64)
    r = np.sqrt((x - w.cx) ** 2 + (y - w.cy) ** 2)
    phi = np.tanh((w.R0 - r) * w.dx / (math.sqrt(2.0) * w.W0))
    U = np.full_like(phi, w.U0)
    rho = np.ones_like(phi)
    vx, vy = w.inflow_vector()
    liquid = 0.5 * (1.0 - phi)
    return dict(phi=phi, U=U, rho=rho, ux=vx * liquid, uy=vy * liquid)


def perturbed_fields(w: Workload, seed: int, amp_phi: float = 0.05, amp_U: float = 0.05,
                     amp_rho: float = 0.01, amp_u: float = 0.01) -> dict:
    """Seed fields plus seeded uniform noise (numpy PCG64), so every node is non-trivial."""
    rng = np.random.Generator(np.random.PCG64(seed))
    f = seed_fields(w)
    shape = f["phi"].shape
    f["phi"] = np.clip(f["phi"] + amp_phi * rng.uniform(-1, 1, shape), -1.0, 1.0)
    f["U"] = f["U"] + amp_U * rng.uniform(-1, 1, shape)
    f["rho"] = f["rho"] + amp_rho * rng.uniform(-1, 1, shape)
    if w.flow:
        f["ux"] = f["ux"] + amp_u * rng.uniform(-1, 1, shape)
        f["uy"] = f["uy"] + amp_u * rng.uniform(-1, 1, shape)
    return f


def mirror_fields(w: Workload, seed: int, amp: float = 0.05) -> dict:
    """Noise fields symmetric under x -> nx - x and y -> ny - y (mod n) about node (nx/2, ny/2).

    Random values are drawn for one quadrant and reflected, so the field is exactly
    mirror-symmetric. Velocities are odd under the mirror of their own axis.
    """
    rng = np.random.Generator(np.random.PCG64(seed))
    nx, ny = w.nx, w.ny
    assert nx % 2 == 0 and ny % 2 == 0

    def sym(even_x=True, even_y=True):
        a = rng.uniform(-1, 1, (ny, nx))
        ix = (-np.arange(nx)) % nx
        iy = (-np.arange(ny)) % ny
        sx = 1.0 if even_x else -1.0
        sy = 1.0 if even_y else -1.0
        b = a + sx * a[:, ix]
        b = b + sy * b[iy, :]
        return 0.25 * b

    c = dataclasses.replace(w, cx=nx // 2, cy=ny // 2)
    f = seed_fields(c)
    f["phi"] = np.clip(f["phi"] + amp * sym(), -1.0, 1.0)
    f["U"] = f["U"] + amp * sym()
    f["rho"] = f["rho"] + 0.2 * amp * sym()
    f["ux"] = 0.2 * amp * sym(even_x=False)
    f["uy"] = 0.2 * amp * sym(even_y=False)
    return f


# ---- batched sweep: 96 independent crystals of uneven sizes --------------------------------
C4_SIDES = (256, 384, 512, 768, 1024)


def batch_sweep(count: int = 96, seed: int = 2101, sides=C4_SIDES, steps: int = 10000):
    """Members of the batched sweep: square grids drawn uniformly from `sides`,
    U0 ~ U[0.1, 0.6], eps ~ U[0.02, 0.08], inflow u ~ U[0, 0.03] along a random axis (inlet
    upstream, zero-gradient outlet downstream, free-slip on the two other faces), seed radius
    6 at the centre; numpy PCG64 with the given seed."""
    rng = np.random.Generator(np.random.PCG64(seed))
    out = []
    for i in range(count):
        n = int(rng.choice(sides))
        U0 = float(rng.uniform(0.1, 0.6))
        eps = float(rng.uniform(0.02, 0.08))
        u = float(rng.uniform(0.0, 0.03))
        axis = int(rng.integers(0, 4))  # inflow towards +x, -x, +y, -y
        bc = [BC_FREESLIP] * 4
        inlet = {0: 0, 1: 1, 2: 2, 3: 3}[axis]
        outlet = inlet ^ 1
        bc[inlet], bc[outlet] = BC_INLET, BC_OUTLET
        out.append(Workload(f"sweep{i:02d}_{n}", n, n, steps, D=2.0, eps=eps, U0=U0, U_in=U0,
                            u_in=u, nu=0.016, bc=tuple(bc), flow=True, cx=n / 2, cy=n / 2,
                            R0=6.0))
    return out


def named() -> dict:
    """Every named workload as {name: to_dict()}: the single-grid configurations (the 128^2
    seed, the ventilated channel, the 2048^2 plate) and the paper's Table 2, four-fold and
    isotropy systems. The batched sweep's members come from batch_sweep()."""
    return {name: w.to_dict() for name, w in sorted(WORKLOADS.items())}


if __name__ == "__main__":
    # python -m paper_2101_07163_gb300.workloads [name ...]: the named workloads as JSON
    import json
    import sys
    want = sys.argv[1:] or sorted(WORKLOADS)
    print(json.dumps({n: WORKLOADS[n].to_dict() for n in want}, indent=1))

"""Benchmark of the fused coupled-lattice step on GB300.

One bench step is one time step of the three coupled D2Q9 lattices (phase field, vapour,
flow) over the whole grid of the plate-regime workload: 2048 x 2048 periodic, seed R0 = 10,
U0 = 0.5, eps = 0.05, D = 3, FP32 state (956 MB, larger than the 129 MB L2, so no L2 flush
is needed between steps). Prints one JSON line.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

--impl reference times the FP64 CPU oracle (the test oracle, as it stands) on the host
cores, on a band of the same workload per step. Under torchrun with N > 1 every rank runs
an independent replica of the single-grid workload (no data-path collective) and rank 0
reports the aggregate over the slowest rank; the batched sweep is sharded by crystal
instead, its only collective an FP64 sum of the diagnostics after the timed region.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import re
import subprocess
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

from paper_2101_07163_gb300 import workloads as W  # noqa: E402

METRIC = "coupled-lattice MLUPS and % of HBM roofline at 1 GB300 vs FP64 CPU oracle error"
# read + write of every population and of the phi history, per node update (all lattices)
ALGO_BYTES_PER_LUP = {("f32", 3): 224, ("f32", 2): 152, ("f16", 3): 116, ("f16", 2): 80,
                      ("bf16", 3): 116, ("bf16", 2): 80}
# what this design moves: + phi^n read; 16-bit storage adds the FP32 moments U (and rho)
DESIGN_BYTES_PER_LUP = {("f32", 3): 228, ("f32", 2): 156, ("f16", 3): 124, ("f16", 2): 84,
                        ("bf16", 3): 124, ("bf16", 2): 84}
PROFILE_TRAFFIC = os.path.join(ROOT, "profiles", "march_kernel_traffic.txt")
NOMINAL_HBM_GBS = 8000.0  # GB300 HBM3e, nominal (the measured copy peak is the denominator)


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10000)
    ap.add_argument("--warmup", type=int, default=200)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--workload", default=W.C3.name, choices=sorted(W.WORKLOADS))
    ap.add_argument("--nx", type=int, default=0, help="override grid (profiling runs)")
    ap.add_argument("--ny", type=int, default=0)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--cpu-seconds", type=float, default=8.0)
    ap.add_argument("--storage-legs", default="f16,bf16",
                    help="16-bit storage legs timed after the FP32 leg ('' for none)")
    ap.add_argument("--batch-steps", type=int, default=120,
                    help="steps of the 96-crystal batched sweep leg (0: skip)")
    ap.add_argument("--batch-count", type=int, default=96,
                    help="crystals of the batched sweep (profiling runs: the first n of the 96)")
    ap.add_argument("--grad-steps", type=int, default=3000,
                    help="steps of the gradient workload leg (512^2, adjoint; 0: skip)")
    ap.add_argument("--grad-n", type=int, default=512,
                    help="grid side of the gradient leg (profiling runs only)")
    ap.add_argument("--grad-large-steps", type=int, default=300,
                    help="steps of the gradient leg at twice the side, beyond L2 (0: skip)")
    return ap.parse_args()


def workload(args) -> W.Workload:
    w = W.WORKLOADS[args.workload]
    if args.nx or args.ny:
        w = w.with_size(args.nx or w.nx, args.ny or w.ny)
    return w


def dist_init():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    if ws <= 1:
        return None, 0, 1
    import torch.distributed as dist
    backend = "nccl"
    import torch
    if not torch.cuda.is_available():
        backend = "gloo"
    else:
        torch.cuda.set_device(int(os.environ.get("LOCAL_RANK", "0")))
    dist.init_process_group(backend)
    return dist, dist.get_rank(), dist.get_world_size()


def max_over_ranks(dist, value: float) -> float:
    if dist is None:
        return value
    import torch
    dev = "cuda" if dist.get_backend() == "nccl" else "cpu"
    t = torch.tensor([value], dtype=torch.float64, device=dev)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def barrier(dist):
    if dist is not None:
        dist.barrier()


def shard_crystals(ws: list, rank: int, world: int) -> list:
    """The crystals of the batched sweep this rank advances: every world-th member from
    position rank. The crystals are independent, so the ranks exchange nothing while they
    step."""
    return ws[rank::world]


STAT_SUMS = ("area", "mass", "vapour_invariant", "nonfinite")


def reduce_diagnostics(dist, stats: list) -> dict:
    """FP64 sums over the crystals of every rank of the per-crystal diagnostics (solid area,
    mass, vapour invariant, non-finite count): the one collective of the batched leg, after
    its timed region."""
    import torch
    local = [sum(float(st[k]) for st in stats) for k in STAT_SUMS]
    if dist is not None:
        dev = "cuda" if dist.get_backend() == "nccl" else "cpu"
        t = torch.tensor(local, dtype=torch.float64, device=dev)
        dist.all_reduce(t, op=dist.ReduceOp.SUM)
        local = [float(v) for v in t.tolist()]
    return dict(zip(STAT_SUMS, local))


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled during the timed region."""

    QUERY = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.index = index
        self.proc = None

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.index), f"--query-gpu={self.QUERY}",
                 "--format=csv,noheader,nounits", "-lms", "100"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except (FileNotFoundError, OSError):
            self.proc = None
        return self

    def __exit__(self, *exc):
        self.out = ""
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.out, _ = self.proc.communicate(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()
                self.out, _ = self.proc.communicate()

    def summary(self):
        rows = []
        for line in (self.out or "").strip().splitlines():
            parts = [p.strip() for p in line.split(",")]
            if len(parts) < 9:
                continue
            try:
                rows.append((float(parts[1]), float(parts[2]), parts[5:9]))
            except ValueError:
                continue
        if not rows:
            return None
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for _, _, flags in rows for i, f in enumerate(flags)
                          if f.lower().startswith("active")})
        return {"sm_mhz": float(np.median([r[0] for r in rows])),
                "sm_max_mhz": max(r[1] for r in rows), "reasons": reasons,
                "samples": len(rows)}


def kernel_source_hash() -> str:
    h = hashlib.sha256()
    for rel in ("paper_2101_07163_gb300/csrc/lbmice_step.cuh",
                "paper_2101_07163_gb300/csrc/lbmice_device.cuh",
                "paper_2101_07163_gb300/csrc/lbmice_tma.cuh"):
        with open(os.path.join(ROOT, rel), "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()[:16]


def profiled_traffic(nodes: int, kernel: str = "f32"):
    """DRAM bytes of `nodes` grid nodes through one benchmarked kernel ("f32", "f16",
    "batch"), from the committed ncu summary ("key = value" lines, bytes per node); None
    when that kernel was not captured or its source has changed since."""
    rec = {}
    try:
        with open(PROFILE_TRAFFIC) as fh:
            for line in fh:
                line = line.split("#", 1)[0].strip()
                if "=" in line:
                    k, v = (t.strip() for t in line.split("=", 1))
                    rec[k] = v
    except OSError:
        return None, None
    key = kernel + ".dram_bytes_per_node"
    if key not in rec:
        return None, None
    info = {"source": rec.get(kernel + ".source")}
    if rec.get("kernel_source_sha256_16") != kernel_source_hash():
        return None, info
    return float(rec[key]) * nodes, info


def measured_peak():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as fh:
            return float(json.load(fh)["hbm_gbs"]), "measured"
    except (OSError, ValueError, KeyError):
        return 6800.0, "fallback"


def host_cores() -> int:
    """Host threads the oracle may use: the CPUs this process may run on."""
    try:
        return len(os.sched_getaffinity(0))
    except AttributeError:
        return os.cpu_count() or 1


def oracle_run(w: W.Workload, fields: dict, seconds: float, min_steps: int = 2,
               threads: int = 1, max_steps: int = 64):
    """Time the FP64 oracle on this workload, one full-grid step at a time, on `threads`
    host threads (its rows split statically; same bits for any count)."""
    import oracle
    oracle.set_threads(threads)
    o = oracle.Oracle(nx=w.nx, ny=w.ny, **w.params())
    o.set_fields(**fields)
    t0 = time.perf_counter()
    n = 0
    while n < min_steps or (time.perf_counter() - t0 < seconds and n < max_steps):
        o.step(1)
        n += 1
    dt = time.perf_counter() - t0
    return o, n, dt


def run_reference(args):
    dist, rank, world = dist_init()
    if rank != 0:
        return
    import oracle
    w = workload(args)
    full = W.seed_fields(w)
    cores = host_cores()
    oracle.set_threads(cores)
    # one bench step = one oracle step on a band of rows through the crystal, sized from a
    # one-step probe so that warmup + steps take about two minutes on all host cores
    total = max(1, args.steps + args.warmup)
    probe_rows = min(w.ny, 64)
    pf = {k: np.ascontiguousarray(v[:probe_rows]) for k, v in full.items()}
    po = oracle.Oracle(nx=w.nx, ny=probe_rows, **W.Workload(**{**w.__dict__, "ny": probe_rows}).params())
    po.set_fields(**pf)
    t0 = time.perf_counter()
    po.step(1)
    rate = w.nx * probe_rows / max(time.perf_counter() - t0, 1e-6)
    del po
    rows = int(np.clip(round(120.0 * rate / (w.nx * total)), 4, w.ny))
    y0 = int(np.clip(int(w.cy) - rows // 2, 0, w.ny - rows))
    band = W.Workload(**{**w.__dict__, "ny": rows, "cy": w.cy - y0})
    fields = {k: np.ascontiguousarray(v[y0:y0 + rows]) for k, v in full.items()}
    o = oracle.Oracle(nx=band.nx, ny=band.ny, **band.params())
    o.set_fields(**fields)
    for _ in range(args.warmup):
        o.step(1)
    t0 = time.perf_counter()
    o.step(args.steps)
    dt = time.perf_counter() - t0
    mlups = band.nx * band.ny * args.steps / dt / 1e6
    sample = (f"{band.nx}x{band.ny} band (rows {y0}..{y0 + rows - 1}) of {w.name}, "
              f"periodic, one FP64 oracle step per bench step, {cores} host threads")
    print(json.dumps({
        "impl": "reference", "metric": METRIC, "value": mlups, "unit": "MLUPS",
        "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": dt / args.steps * 1e3, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": w.name, "grid": [w.nx, w.ny], "lattices": w.lattices,
                   "sample_rows": rows},
        "cpu_baseline": {"value": mlups, "unit": "MLUPS", "cores": cores, "kind": "oracle",
                         "sample": sample},
        "e2e": {"value": mlups, "unit": "MLUPS", "h2d_bytes_per_step": 0,
                "d2h_bytes_per_step": 0},
    }), flush=True)


def run_batched(args, stream, dist, rank: int = 0, world: int = 1):
    """The 96-crystal batched sweep: autotuned tile shapes, one persistent launch per step
    (CUDA graphs), against the same members stepped one grid at a time. Under N ranks the
    crystals are sharded (shard_crystals); the diagnostics are summed over all of them."""
    import torch
    from paper_2101_07163_gb300 import lbmice
    ws_all = W.batch_sweep(count=args.batch_count)
    ws = shard_crystals(ws_all, rank, world)
    K = args.batch_steps
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    b, shapes, ms, ms_seq, launches = None, [], 0.0, 0.0, 0
    if ws:
        b = lbmice.Batch([dict(nx=w.nx, ny=w.ny, **w.params()) for w in ws], stream=stream)
        for m, w in zip(b.members, ws):
            m.init_seed(w.cx, w.cy, w.R0, w.U0)
        shapes, _ = b.autotune(steps_per_trial=6)
        for m, w in zip(b.members, ws):  # restart from the seeds after tuning
            m.init_seed(w.cx, w.cy, w.R0, w.U0)
        b.step(12)
        b.sync()
        launches = b.launches_per_step
    barrier(dist)
    if b is not None:
        e0.record(stream)
        b.step(K)
        e1.record(stream)
        e1.synchronize()
        ms = e0.elapsed_time(e1)
    ms = max_over_ranks(dist, ms)
    stats = [m.stats() for m in b.members] if b is not None else []
    diag = reduce_diagnostics(dist, stats)
    # the plain path: every member stepped through its own lbmice_step, one after another
    if b is not None:
        L = lbmice.lib()
        e0.record(stream)
        for m in b.members:
            rc = L.lbmice_step(m.handle, K)
            if rc != lbmice.OK:
                raise lbmice.LbmiceError(rc, "lbmice_step")
        e1.record(stream)
        e1.synchronize()
        ms_seq = e0.elapsed_time(e1)
    ms_seq = max_over_ranks(dist, ms_seq)
    by_side = {}
    for w, s in zip(ws, shapes):
        by_side.setdefault(str(w.nx), lbmice.SHAPES[s])
    out = {"workload": "batch_sweep: %d crystals, sides {256..1024}, PCG64 seed 2101"
                       % len(ws_all),
           "members": len(ws_all), "nodes": int(b.nodes) if b is not None else 0,
           "nodes_all_ranks": int(sum(w.nx * w.ny for w in ws_all)), "steps": K, "ms": ms,
           "ms_seq": ms_seq, "tile_shape_by_side": by_side,
           "finite": diag["nonfinite"] == 0, "diagnostics_fp64": diag,
           "gpu_launches_per_step": launches}
    if world > 1:
        out["sharding"] = "by crystal: rank r advances members r, r + %d, ..." % world
        out["members_per_rank"] = len(ws)
    if b is not None:
        b.close()
    return out


# Bytes per node of one reverse step. Algorithmic (what the method itself must move): the
# state it differentiates read (27 populations, phi^n, phi^{n-1}: 116 B), the adjoint of the
# next state read (116 B) and the adjoint of this state written (116 B), plus, under
# checkpointing, one recomputed forward step (224 B). As built: the collision adjoint reads
# the state (27 populations, phi^n, phi^{n-1}) and the adjoint (27 + 2 planes) and writes
# 27 + 5 planes (360 B); the pull adjoint reads 9 + 9 population planes and 6 planes, writes
# 9 + 1 (132 B); the recomputed step moves 228 B.
REVERSE_ALGO_BYTES_PER_NODE = 3 * 116 + 224
REVERSE_DESIGN_BYTES_PER_NODE = 360 + 132 + 228  # adj_collide, adj_pull (RMW), recompute
# beyond L2: adj_b (phi in, B out), adj_collide (+ own h adjoints in, B(x - c_a) in, no B
# out), adj_stencil, recompute
REVERSE_DESIGN_BYTES_FUSED = 8 + 400 + 16 + 228


def reverse_pull_fused(nodes):
    """The library's choice of reverse-pull form (lbmice_tape_create): fused when the
    reverse working set, about 4 x 116 B per node, exceeds the L2 (LBMICE_ADJ_FUSED forces)."""
    import torch
    env = os.environ.get("LBMICE_ADJ_FUSED")
    if env in ("0", "1"):
        return env == "1"
    l2 = torch.cuda.get_device_properties(torch.cuda.current_device()).L2_cache_size
    return 4 * 116 * nodes > l2


def run_gradient(args, stream, dist, n=None, steps=None, fd=True):
    """The gradient workload: n^2 periodic (512^2), f + g + h, seed R = 6 at the centre, from
    (U0, eps, D) = (0.3, 0.04, 2.0) towards the run of (0.4, 0.06, 2.5), checkpoints every
    100 steps; L = sum (phi_T - phi_T^target)^2. Times the recorded forward and the reverse
    sweep, and (fd) checks the gradient against central differences (h = 1e-3)."""
    import torch
    from paper_2101_07163_gb300 import lbmice
    n = n or args.grad_n
    steps = steps or args.grad_steps
    every = 100
    w = W.Workload("grad", n, n, steps, flow=True, eps=0.04, D=2.0, U0=0.3, cx=n / 2,
                   cy=n / 2, R0=6.0)
    dev = torch.device("cuda", torch.cuda.current_device())

    def forward(U0, eps, D, tape=False):
        lat = lbmice.Lattice(n, n, stream=stream, **dict(w.params(), eps=eps, D=D))
        lat.init_seed(w.cx, w.cy, w.R0, U0)
        t = lbmice.Tape(lat, every) if tape else None
        return lat, t

    def phi_T(U0, eps, D):
        lat, _ = forward(U0, eps, D)
        lat.step(steps)
        out = torch.empty((n, n), dtype=torch.float32, device=dev)
        lat.field(lbmice.PHI, out=out)
        lat.sync()
        lat.close()
        return out.double()

    target = phi_T(0.4, 0.06, 2.5)
    lat, tape = forward(0.3, 0.04, 2.0, tape=True)
    e = [torch.cuda.Event(enable_timing=True) for _ in range(4)]
    barrier(dist)
    e[0].record(stream)
    tape.record(steps)
    e[1].record(stream)
    e[1].synchronize()
    out = torch.empty((n, n), dtype=torch.float32, device=dev)
    lat.field(lbmice.PHI, out=out)
    lat.sync()
    seed = (2.0 * (out.double() - target)).float().contiguous()
    L0 = float(((out.double() - target) ** 2).sum())
    tape.backward(seed)  # allocates the reverse work space
    torch.cuda.synchronize()
    e[2].record(stream)
    grads, fields = tape.backward(seed)
    e[3].record(stream)
    e[3].synchronize()
    fwd_ms = max_over_ranks(dist, e[0].elapsed_time(e[1]))
    bwd_ms = max_over_ranks(dist, e[2].elapsed_time(e[3]))
    g = {"U0": float(fields["U0"].double().sum()), "eps": grads["eps"], "D": grads["D"]}
    tape.close()
    lat.close()
    nodes = n * n
    peak, _ = measured_peak()
    fused = reverse_pull_fused(nodes)
    design = REVERSE_DESIGN_BYTES_FUSED if fused else REVERSE_DESIGN_BYTES_PER_NODE
    ach = REVERSE_ALGO_BYTES_PER_NODE * nodes * steps / (bwd_ms * 1e-3) / 1e9
    state_mb = 4 * 116 * nodes / 1e6  # state and adjoint, read and written, per step
    out = {"workload": "gradient %dx%d periodic f+g+h, %d steps, checkpoints every 100"
                       % (n, n, steps),
           "loss": L0, "gradient": g,
           "forward_recorded_ms": fwd_ms, "reverse_ms": bwd_ms,
           "reverse_mlups": nodes * steps / (bwd_ms * 1e-3) / 1e6,
           "l2_resident": state_mb < 129.0,
           "roofline": {"bound": "hbm", "achieved": ach, "peak": peak, "unit": "GB/s",
                        "frac": ach / peak,
                        "algorithmic_bytes_per_node_reverse_step": REVERSE_ALGO_BYTES_PER_NODE,
                        "design_bytes_per_node_reverse_step": design,
                        "frac_design_bytes": design * nodes * steps
                                             / (bwd_ms * 1e-3) / 1e9 / peak,
                        "kernels": ("adj_b_kernel + adj_collide_kernel<fused> + "
                                    "adj_stencil_kernel" if fused else
                                    "adj_collide_kernel + adj_pull_kernel")
                                   + " + march_kernel (segment recompute)"},
           "reverse_pull": "fused (beyond L2)" if fused else "separate pass (L2-resident)",
           "gpu_launches_per_reverse_step": 4 if fused else 3}
    if fd:
        h = 1e-3
        base = {"U0": 0.3, "eps": 0.04, "D": 2.0}
        fdv, rel = {}, {}
        for k, v in base.items():
            up = float(((phi_T(**dict(base, **{k: v + h})) - target) ** 2).sum())
            dn = float(((phi_T(**dict(base, **{k: v - h})) - target) ** 2).sum())
            fdv[k] = (up - dn) / (2 * h)
            rel[k] = abs(g[k] - fdv[k]) / abs(fdv[k])
        out["central_differences_h1e-3"] = fdv
        out["rel_err_vs_fd"] = rel
    return out


def run_ours(args):
    import torch
    dist, rank, world = dist_init()
    from paper_2101_07163_gb300 import lbmice
    torch.cuda.set_device(int(os.environ.get("LOCAL_RANK", "0")))
    w = workload(args)
    nodes = w.nx * w.ny
    stream = torch.cuda.Stream()
    lat = lbmice.Lattice(w.nx, w.ny, stream=stream, **w.params())
    lat.init_seed(w.cx, w.cy, w.R0, w.U0)
    lat.step(args.warmup)
    lat.sync()

    # ---- device-timed region: K fused steps, state resident in HBM ----
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    barrier(dist)
    torch.cuda.synchronize()
    dev_index = torch.cuda.current_device()
    with ClockSampler(dev_index) as clk:
        ev0.record(stream)
        lat.step(args.steps)
        ev1.record(stream)
        ev1.synchronize()
    torch.cuda.synchronize()
    barrier(dist)
    ms = ev0.elapsed_time(ev1)
    ms = max_over_ranks(dist, ms)
    stats = lat.stats()
    finite = stats["nonfinite"] == 0

    # ---- end-to-end through the C ABI with host buffers ----
    f = W.seed_fields(w)
    pinned = {k: torch.from_numpy(v).pin_memory() for k, v in f.items()}
    host = {k: t.numpy() for k, t in pinned.items()}
    out_phi = torch.empty((w.ny, w.nx), dtype=torch.float32).pin_memory().numpy()
    lat2 = lbmice.Lattice(w.nx, w.ny, stream=stream, **w.params())
    lat2.set_fields(**host)  # warm the path once
    lat2.step(min(args.warmup, 60))
    lat2.sync()
    barrier(dist)
    t0 = time.perf_counter()
    lat2.set_fields(**host)                       # H2D of the initial moments (FP64)
    lat2.step(args.steps)
    st2 = lat2.stats()                            # D2H of the FP64 diagnostics
    lat2.field(lbmice.PHI, out=out_phi)           # D2H of the result field, pinned
    e2e_s = time.perf_counter() - t0
    e2e_s = max_over_ranks(dist, e2e_s)
    h2d = sum(v.nbytes for v in host.values())
    d2h = out_phi.nbytes + 8 * lbmice.NSTATS
    lat2.close()
    del lat2

    # ---- 16-bit storage legs: same workload, same timed region ----
    legs = {}
    for st in [x for x in args.storage_legs.split(",") if x]:
        lat3 = lbmice.Lattice(w.nx, w.ny, stream=stream, storage=st, **w.params())
        lat3.init_seed(w.cx, w.cy, w.R0, w.U0)
        lat3.step(args.warmup)
        lat3.sync()
        barrier(dist)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        lat3.step(args.steps)
        e1.record(stream)
        e1.synchronize()
        ms3 = max_over_ranks(dist, e0.elapsed_time(e1))
        legs[st] = {"lat": lat3, "ms": ms3}

    # ---- batched sweep: 96 crystals of uneven sizes, one persistent launch per step ----
    batched = None
    if args.batch_steps > 0:
        batched = run_batched(args, stream, dist, rank, world)
    gradient = None
    if args.grad_steps > 0:
        gradient = run_gradient(args, stream, dist)
        if args.grad_large_steps > 0:
            # the same workload at 1024^2, whose state and adjoint (about 490 MB) exceed L2
            gradient["beyond_l2"] = run_gradient(args, stream, dist, n=2 * args.grad_n,
                                                 steps=args.grad_large_steps, fd=False)

    if rank != 0:
        for leg in legs.values():
            leg["lat"].close()
        lat.close()
        barrier(dist)
        return

    value = nodes * args.steps * world / (ms * 1e-3) / 1e6
    per_launch_ms = ms / args.steps
    algo = ALGO_BYTES_PER_LUP[("f32", w.lattices)] * nodes
    achieved = algo / (per_launch_ms * 1e-3) / 1e9
    peak, peak_kind = measured_peak()
    traffic, rec = profiled_traffic(nodes)
    roofline = {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
                "frac": achieved / peak, "traffic": traffic,
                "frac_nominal": achieved / NOMINAL_HBM_GBS,
                "nominal_peak": NOMINAL_HBM_GBS,
                "peak_kind": peak_kind + " (MEASURED_PEAKS hbm_gbs copy bandwidth)"
                if peak_kind == "measured" else peak_kind,
                "algorithmic_bytes_per_lup": ALGO_BYTES_PER_LUP[("f32", w.lattices)],
                "design_bytes_per_lup": DESIGN_BYTES_PER_LUP[("f32", w.lattices)],
                "kernel": "lbmice::march_kernel<flow,F32,plain>"}
    if rec is not None:
        roofline["traffic_source"] = rec.get("source")
        if traffic is None:
            roofline["traffic_note"] = "kernel changed since the ncu capture"

    line = {
        "metric": METRIC, "value": value, "unit": "MLUPS", "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms / args.steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32",
        "data": "synthetic",
        "config": {"workload": w.name, "grid": [w.nx, w.ny], "lattices": w.lattices,
                   "seed_R0": w.R0, "U0": w.U0, "eps": w.eps, "D": w.D,
                   "state_bytes": int(nodes * (2 * 9 * w.lattices + 3) * 4),
                   "l2_policy": "inputs larger than L2 (state > 129 MB), no flush",
                   "parallelism": f"independent replicas x{world}"},
        "roofline": roofline,
        "gpu_launches": args.steps,
        "clocks": clk.summary(),
        "e2e": {"value": nodes * args.steps * world / e2e_s / 1e6, "unit": "MLUPS",
                "h2d_bytes_per_step": h2d / args.steps, "d2h_bytes_per_step": d2h / args.steps,
                "note": "set_fields from pinned host + K steps + stats + phi to host"},
        "finite": bool(finite and st2["nonfinite"] == 0),
    }
    if batched is not None:
        # all crystals of all ranks over the slowest rank's time (the sweep is sharded)
        batched["value"] = batched["nodes_all_ranks"] * batched["steps"] / (
            batched["ms"] * 1e-3) / 1e6
        batched["plain_sequential_value"] = batched["nodes_all_ranks"] * batched["steps"] / (
            batched.pop("ms_seq") * 1e-3) / 1e6
        ach = ALGO_BYTES_PER_LUP[("f32", 3)] * batched["nodes"] / (
            batched["ms"] / batched["steps"] * 1e-3) / 1e9
        btraffic, brec = profiled_traffic(batched["nodes"], "batch")
        batched["roofline"] = {"bound": "hbm", "achieved": ach, "peak": peak, "unit": "GB/s",
                               "frac": ach / peak, "traffic": btraffic,
                               "algorithmic_bytes_per_lup": 224,
                               "kernel": "lbmice::batch_march_kernel<flow,F32,plain>"}
        if brec is not None:
            batched["roofline"]["traffic_source"] = brec.get("source")
        batched["ms_per_step"] = batched.pop("ms") / batched["steps"]
        batched["unit"] = "MLUPS"
        line["batched"] = batched
    if gradient is not None:
        line["gradient"] = gradient
    if legs:
        out = {}
        for st, leg in legs.items():
            ms3 = leg["ms"]
            algo3 = ALGO_BYTES_PER_LUP[(st, w.lattices)] * nodes
            ach3 = algo3 / (ms3 / args.steps * 1e-3) / 1e9
            out[st] = {"value": nodes * args.steps * world / (ms3 * 1e-3) / 1e6,
                       "unit": "MLUPS", "ms_per_step": ms3 / args.steps,
                       "roofline": {"bound": "hbm", "achieved": ach3, "peak": peak,
                                    "unit": "GB/s", "frac": ach3 / peak,
                                    "algorithmic_bytes_per_lup":
                                        ALGO_BYTES_PER_LUP[(st, w.lattices)],
                                    "design_bytes_per_lup":
                                        DESIGN_BYTES_PER_LUP[(st, w.lattices)],
                                    "traffic": profiled_traffic(nodes, st)[0]}}
        line["storage_legs"] = out

    # ---- CPU baseline and error against the FP64 oracle, rank 0, N = 1 only ----
    if world == 1 and not args.no_cpu_baseline:
        fields = W.seed_fields(w)
        cores = host_cores()
        o1, n1, dt1 = oracle_run(w, fields, 0.0, min_steps=2, threads=1)
        del o1
        o, n, dt = oracle_run(w, fields, args.cpu_seconds, min_steps=4, threads=cores)
        lat.set_fields(**fields)
        lat.step(n)
        err = {"steps": n,
               "max_dphi": float(np.abs(lat.field(lbmice.PHI) - o.field(0)).max()),
               "max_dU": float(np.abs(lat.field(lbmice.U) - o.field(1)).max()),
               "max_dux": float(np.abs(lat.field(lbmice.UX) - o.field(3)).max())}
        line["cpu_baseline"] = {"value": nodes * n / dt / 1e6, "unit": "MLUPS", "cores": cores,
                                "kind": "oracle",
                                "sample": f"{n} full-grid FP64 oracle steps of {w.name} "
                                          f"from its seed state, rows split over {cores} "
                                          f"host threads",
                                "single_thread": {"value": nodes * n1 / dt1 / 1e6,
                                                  "unit": "MLUPS", "cores": 1,
                                                  "sample": f"{n1} full-grid steps, one thread"}}
        line["oracle_error"] = err
        ophi, oU = o.field(0), o.field(1)
        for st, leg in legs.items():
            l3 = leg["lat"]
            l3.set_fields(**fields)
            l3.step(n)
            line["storage_legs"][st]["oracle_error"] = {
                "steps": n,
                "max_dphi": float(np.abs(l3.field(lbmice.PHI) - ophi).max()),
                "max_dU": float(np.abs(l3.field(lbmice.U) - oU).max())}
    print(json.dumps(line), flush=True)
    lat.close()
    for leg in legs.values():
        leg["lat"].close()
    barrier(dist)


def main():
    args = parse()
    if args.impl == "reference":
        run_reference(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()

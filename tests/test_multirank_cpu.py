"""Multi-process host paths of bench.py on CPU (gloo, world sizes 2 and 3): the rank helpers
that give the slowest rank's time and the barrier around the timed region, the batched
sweep's sharding by crystal and its FP64 sum of the diagnostics, and the reference arm under
torch.distributed.run (rank 0 runs and prints one line, the other rank exits 0)."""
import json
import os
import socket
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, out):
    os.environ.update(RANK=str(rank), WORLD_SIZE=str(world), LOCAL_RANK=str(rank),
                      MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    sys.path.insert(0, ROOT)
    import bench
    dist, r, w = bench.dist_init()
    bench.barrier(dist)
    got = bench.max_over_ranks(dist, 10.0 * (rank + 1))
    out.put((r, w, dist.get_backend(), got))
    dist.destroy_process_group()


def test_rank_helpers_take_the_slowest_rank_over_gloo():
    import torch.multiprocessing as mp
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = free_port()
    procs = [ctx.Process(target=_rank_main, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = sorted(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=120)
        assert p.exitcode == 0
    assert [r[0] for r in res] == [0, 1]
    assert all(r[1] == 2 and r[2] == "gloo" for r in res)
    assert all(r[3] == 20.0 for r in res)  # the maximum of 10 and 20 on both ranks


def _shard_main(rank, world, port, out):
    os.environ.update(RANK=str(rank), WORLD_SIZE=str(world), LOCAL_RANK=str(rank),
                      MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    sys.path.insert(0, ROOT)
    import bench
    from paper_2101_07163_gb300 import workloads as W
    dist, r, w = bench.dist_init()
    ws = bench.shard_crystals(W.batch_sweep(), r, w)
    # stand-in per-crystal diagnostics: the crystal's node count, its side, one, zero
    stats = [dict(area=float(c.nx * c.ny), mass=float(c.nx), vapour_invariant=1.0,
                  nonfinite=0) for c in ws]
    got = bench.reduce_diagnostics(dist, stats)
    out.put((r, [c.name for c in ws], got))
    dist.destroy_process_group()


def test_batched_sweep_is_sharded_by_crystal_and_diagnostics_summed_over_gloo():
    import torch.multiprocessing as mp
    from paper_2101_07163_gb300 import workloads as W
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = free_port()
    procs = [ctx.Process(target=_shard_main, args=(r, 3, port, q)) for r in range(3)]
    for p in procs:
        p.start()
    res = sorted(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=120)
        assert p.exitcode == 0
    ws = W.batch_sweep()
    names = [n for r in res for n in r[1]]
    assert sorted(names) == sorted(w.name for w in ws)  # every crystal exactly once
    assert [len(r[1]) for r in res] == [32, 32, 32]
    want = dict(area=float(sum(w.nx * w.ny for w in ws)), mass=float(sum(w.nx for w in ws)),
                vapour_invariant=96.0, nonfinite=0.0)
    for r in res:
        assert r[2] == want  # the same FP64 sums on every rank


def test_reference_arm_prints_one_line_from_rank_zero():
    port = free_port()
    cmd = [sys.executable, "-m", "torch.distributed.run", "--nnodes=1", "--nproc-per-node", "2",
           "--master-addr", "127.0.0.1", "--master-port", str(port), "bench.py",
           "--impl", "reference", "--gpus", "2", "--steps", "2", "--warmup", "0",
           "--workload", "hg_periodic_128x128"]
    env = dict(os.environ, CUDA_VISIBLE_DEVICES="")
    r = subprocess.run(cmd, cwd=ROOT, env=env, capture_output=True, text=True, timeout=300)
    assert r.returncode == 0, r.stderr[-2000:]
    lines = [l for l in r.stdout.splitlines() if l.startswith("{")]
    assert len(lines) == 1, r.stdout
    d = json.loads(lines[0])
    assert d["impl"] == "reference" and d["n_gpus"] == 2 and d["value"] > 0
    assert d["cpu_baseline"]["kind"] == "oracle" and d["e2e"]["h2d_bytes_per_step"] == 0

"""Batched launch: many grids of uneven sizes, parameters and faces in one persistent kernel
per step. Every node is collided by the same code as in the single-grid kernel, whatever the
shape (the column march or a 2D tile; its arithmetic rounding written out, so no kernel
contracts it differently), so a batch must reproduce independently stepped single grids bit
for bit."""
import ctypes

import numpy as np
import pytest

import oracle
from paper_2101_07163_gb300 import lbmice
from paper_2101_07163_gb300 import workloads as W

pytestmark = pytest.mark.gpu


def small_sweep(count=6, seed=11):
    return W.batch_sweep(count=count, seed=seed, sides=(40, 72, 100))


def configs(ws, storage="f32"):
    return [dict(nx=w.nx, ny=w.ny, storage=storage, **w.params()) for w in ws]


def singles(ws, storage="f32"):
    out = []
    for w in ws:
        lat = lbmice.Lattice(w.nx, w.ny, storage=storage, **w.params())
        lat.init_seed(w.cx, w.cy, w.R0, w.U0)
        out.append(lat)
    return out


@pytest.mark.parametrize("storage", ["f32", "f16"])
def test_batch_equals_single_grids_for_every_tile_shape(storage):
    ws = small_sweep()
    b = lbmice.Batch(configs(ws, storage))
    for i, (m, w) in enumerate(zip(b.members, ws)):
        m.init_seed(w.cx, w.cy, w.R0, w.U0)
        b.set_shape(i, i % 4)  # all four shapes in one step
    ref = singles(ws, storage)
    b.step(125)  # two graph replays of 60 steps and five single launches
    for lat in ref:
        lat.step(125)
    for m, lat in zip(b.members, ref):
        assert m.steps_done == lat.steps_done == 125
        np.testing.assert_array_equal(m.state(), lat.state())


def test_autotune_keeps_members_in_lockstep():
    ws = small_sweep(5, seed=12)
    b = lbmice.Batch(configs(ws))
    for m, w in zip(b.members, ws):
        m.init_seed(w.cx, w.cy, w.R0, w.U0)
    shapes, taken = b.autotune(steps_per_trial=2)
    classes = len({w.nx for w in ws})
    assert taken == classes * 4 * 3
    assert set(shapes) <= {0, 1, 2, 3}
    # results do not depend on the shapes the autotuner tried
    ref = singles(ws)
    for lat in ref:
        lat.step(taken)
    b.step(7)
    for lat in ref:
        lat.step(7)
    for m, lat in zip(b.members, ref):
        np.testing.assert_array_equal(m.state(), lat.state())


def test_autotune_on_a_non_blocking_stream_after_queued_steps():
    # descriptor and list uploads must be ordered after launches still queued on the
    # caller's stream, which a non-blocking stream does not get from the legacy stream
    import torch
    ws = small_sweep(6, seed=16)
    st = torch.cuda.Stream()
    b = lbmice.Batch(configs(ws), stream=st)
    for m, w in zip(b.members, ws):
        m.init_seed(w.cx, w.cy, w.R0, w.U0)
    b.step(61)  # a graph replay and a single launch left queued
    b.autotune(steps_per_trial=2)
    for m, w in zip(b.members, ws):  # re-seeding every member restarts the batch at step 0
        m.init_seed(w.cx, w.cy, w.R0, w.U0)
    b.step(65)
    ref = singles(ws)
    for lat in ref:
        lat.step(65)
    st.synchronize()
    for m, lat in zip(b.members, ref):
        np.testing.assert_array_equal(m.state(), lat.state())


def test_more_members_than_one_launch_carries():
    # 69 members of one shape take two launches per step (64 + 5), a second shape group
    # adds its own launch; every member still matches its single grid bit for bit
    ws = W.batch_sweep(count=70, seed=17, sides=(20, 36))
    b = lbmice.Batch(configs(ws))
    for i, (m, w) in enumerate(zip(b.members, ws)):
        m.init_seed(w.cx, w.cy, 4.0, w.U0)
    b.set_shape(3, 2)
    assert b.launches_per_step == 3
    b.step(67)
    for i in (0, 3, 63, 64, 69):
        w = ws[i]
        lat = lbmice.Lattice(w.nx, w.ny, **w.params())
        lat.init_seed(w.cx, w.cy, 4.0, w.U0)
        lat.step(67)
        np.testing.assert_array_equal(b.members[i].state(), lat.state())


def test_batch_refuses_members_out_of_lockstep():
    ws = small_sweep(3, seed=13)
    b = lbmice.Batch(configs(ws))
    for m, w in zip(b.members, ws):
        m.init_seed(w.cx, w.cy, w.R0, w.U0)
    assert lbmice.lib().lbmice_step(b.members[1].handle, 1) == lbmice.OK
    with pytest.raises(lbmice.LbmiceError) as ei:
        b.step(1)
    assert ei.value.code == lbmice.EINVAL


def test_batch_members_against_the_oracle():
    ws = small_sweep(3, seed=14)
    b = lbmice.Batch(configs(ws))
    orcs = []
    for i, (m, w) in enumerate(zip(b.members, ws)):
        f = W.perturbed_fields(w, 30 + i)
        m.set_fields(**f)
        b.set_shape(i, (i + 1) % 4)
        o = oracle.Oracle(nx=w.nx, ny=w.ny, **w.params())
        o.set_fields(**f)
        orcs.append(o)
    b.step(1)
    for o in orcs:
        o.step(1)
    for m, o in zip(b.members, orcs):
        for which in (lbmice.PHI, lbmice.U, lbmice.RHO, lbmice.UX):
            assert np.abs(m.field(which).astype(np.float64) - o.field(which)).max() < 1e-6


def test_batch_rejects_mixed_flow_or_storage():
    ws = small_sweep(2, seed=15)
    cf = configs(ws)
    cf[1]["storage"] = "f16"
    with pytest.raises(lbmice.LbmiceError) as ei:
        lbmice.Batch(cf)
    assert ei.value.code == lbmice.EINVAL
    cf = configs(ws)
    cf[0]["flow"] = False
    with pytest.raises(lbmice.LbmiceError):
        lbmice.Batch(cf)


def test_full_sweep_in_the_benchmark_configuration():
    # The 96-crystal sweep the benchmark times (35.8 M nodes, 8.2 GB of state), with the tile
    # shapes its autotuner picks, then one 60-step graph replay and one single launch; one
    # member of each grid side (inflow along its own axis, inlet/outlet/free-slip faces)
    # against the FP64 oracle over the same steps.
    from tests.test_parity_gpu import compare_moments
    ws = W.batch_sweep()
    b = lbmice.Batch(configs(ws))
    for m, w in zip(b.members, ws):
        m.init_seed(w.cx, w.cy, w.R0, w.U0)
    shapes, taken = b.autotune(steps_per_trial=2)
    for m, w in zip(b.members, ws):  # re-seeding every member restarts the batch at step 0
        m.init_seed(w.cx, w.cy, w.R0, w.U0)
    b.step(61)
    picked = {}
    for i, w in enumerate(ws):
        picked.setdefault(w.nx, i)
    assert sorted(picked) == [256, 384, 512, 768, 1024]
    for n, i in sorted(picked.items()):
        w = ws[i]
        o = oracle.Oracle(nx=w.nx, ny=w.ny, **w.params())
        o.set_fields(**W.seed_fields(w))
        o.step(61)
        assert b.members[i].steps_done == 61
        compare_moments(b.members[i], o, 2e-5)
        del o
    b.close()

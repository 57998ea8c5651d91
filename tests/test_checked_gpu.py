"""The bounds-checked build (liblbmice_checked.so, compiled with -DLBMICE_CHECKED): every global
and shared-memory index of the single-grid and batched step kernels is tested against its
buffer before the access, a violation sets a bit of a device word and skips the access.
Nothing traps. It runs in a child process with LBMICE_CHECKED=1, on small and ragged grids
with every face rule, storage and stencil, and on a batch with all four shapes: no
index may leave its buffer. The checks themselves are exercised by shrinking the extents
they use (lbmice_debug_set_margin), so that accesses near the end of a buffer, still inside
it, are reported and skipped."""
import json
import os
import subprocess
import sys

import pytest

pytestmark = pytest.mark.gpu

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

CHILD = r"""
import json, sys
sys.path.insert(0, sys.argv[1])
import numpy as np
import oracle
from paper_2101_07163_gb300 import lbmice
from paper_2101_07163_gb300 import workloads as W
from tests.test_parity_gpu import BOXES, channel_workload

res = {"lib": lbmice.lib_path(), "start": lbmice.debug_flags(clear=True)}
runs = 0
for (nx, ny) in [(8, 8), (33, 17), (64, 64), (100, 76), (130, 9)]:
    for box, bc in sorted(BOXES.items()):
        for storage in ("f32", "f16", "bf16"):
            for flow in (True, False):
                w = channel_workload(box, nx, ny, bc)
                p = w.params()
                p["flow"] = flow
                lat = lbmice.Lattice(nx, ny, storage=storage, **p)
                lat.set_fields(**W.perturbed_fields(w, 3, amp_phi=0.3, amp_u=0.02))
                lat.step(61 if (nx, ny) == (100, 76) else 3)  # one graph replay on one size
                lat.close()
                runs += 1
for kw in (dict(stencil=8), dict(stencil=2), dict(fold=4)):
    w = channel_workload("variant", 100, 76, BOXES["channel_x"], **kw)
    lat = lbmice.Lattice(w.nx, w.ny, **w.params())
    lat.set_fields(**W.perturbed_fields(w, 4, amp_phi=0.3, amp_u=0.02))
    lat.step(3)
    lat.close()
    runs += 1
ws = W.batch_sweep(count=6, seed=11, sides=(40, 72, 100))
b = lbmice.Batch([dict(nx=w.nx, ny=w.ny, **w.params()) for w in ws])
for i, (m, w) in enumerate(zip(b.members, ws)):
    m.init_seed(w.cx, w.cy, w.R0, w.U0)
    b.set_shape(i, i % 4)
b.step(61)
b.close()
res["runs"] = runs + 1
res["clean"] = lbmice.debug_flags(clear=True)

# parity of the checked build itself: one step against the oracle
w = channel_workload("parity", 100, 76, BOXES["inlet_plus_x"])
f = W.perturbed_fields(w, 7, amp_phi=0.3, amp_u=0.02)
lat = lbmice.Lattice(w.nx, w.ny, **w.params())
lat.set_fields(**f)
o = oracle.Oracle(nx=w.nx, ny=w.ny, **w.params())
o.set_fields(**f)
lat.step(1)
o.step(1)
res["parity"] = max(float(np.abs(lat.field(k).astype(np.float64) - o.field(k)).max())
                    for k in (lbmice.PHI, lbmice.U, lbmice.RHO, lbmice.UX))
lat.close()
res["after_parity"] = lbmice.debug_flags(clear=True)

# the checks fire: extents shrunk by one element, accesses still inside their buffers (a
# width of 64 is its own pitch, so the last node of the grid is the last of each buffer)
lbmice.debug_set_margin(1)
for storage in ("f32", "f16"):
    w = channel_workload("margin", 64, 24, BOXES["periodic"])
    lat = lbmice.Lattice(w.nx, w.ny, storage=storage, **w.params())
    lat.init_seed(w.cx, w.cy, w.R0, w.U0)
    lat.step(1)
    lat.sync()
    lat.close()
res["margin"] = lbmice.debug_flags(clear=True)
lbmice.debug_set_margin(0)
res["reset"] = lbmice.debug_flags(clear=True)
print(json.dumps(res))
"""


def test_checked_build_keeps_every_index_inside_its_buffer():
    from paper_2101_07163_gb300 import build
    from paper_2101_07163_gb300 import lbmice
    path = build.build(checked=True)
    env = dict(os.environ, LBMICE_CHECKED="1")
    r = subprocess.run([sys.executable, "-c", CHILD, ROOT], cwd=ROOT, env=env,
                       capture_output=True, text=True, timeout=900)
    assert r.returncode == 0, r.stderr[-3000:]
    res = json.loads(r.stdout.strip().splitlines()[-1])
    assert res["lib"] == path
    assert res["runs"] == 5 * 6 * 3 * 2 + 3 + 1
    assert res["start"] == 0
    assert res["clean"] == 0            # no index of any run left its buffer
    assert res["after_parity"] == 0
    assert res["parity"] < 1e-6         # the checked kernels compute the same step
    want = lbmice.OOB_POPS | lbmice.OOB_PLANE | lbmice.OOB_SHARED
    assert res["margin"] & want == want  # every kind of check fires
    assert res["reset"] == 0


"""The largest single grids: offsets into the population buffers beyond 32 bits.

A 23200^2 grid with all three lattices holds 538 M nodes (125 GB of FP32 state, 73 GB with
16-bit storage); its population offsets reach 8 * pstride = 4.3e9 elements. The oracle
cannot run that size, so the check is a property that holds at any size: the step is local
and a uniform vapour state at rest is a fixed point, so a seed placed near the far corner of
the large grid and the same seed in the middle of a 256^2 grid, both in an exactly uniform
far field (the seed's tanh profile is -1 to the last bit beyond 30 cells), give the same
bits in the corner window after two steps."""
import numpy as np
import pytest

from paper_2101_07163_gb300 import lbmice
from paper_2101_07163_gb300 import workloads as W

pytestmark = pytest.mark.gpu

N_BIG, N_SMALL = 23200, 256


def seeded(n, cx, cy, storage):
    w = W.Workload("large", n, n, 2, flow=True, eps=0.05, D=2.0, U0=0.3, nu=0.05,
                   cx=cx, cy=cy, R0=6.0)
    lat = lbmice.Lattice(n, n, storage=storage, **w.params())
    lat.init_seed(w.cx, w.cy, w.R0, w.U0)
    lat.step(w.steps)
    return lat


@pytest.mark.parametrize("storage,need_gb", [("f32", 140), ("f16", 90)])
def test_largest_grid_corner_equals_a_small_grid(storage, need_gb):
    import torch
    free, _ = torch.cuda.mem_get_info()
    if free < need_gb * 2**30:
        pytest.skip(f"needs {need_gb} GB of free device memory")
    off = N_BIG - N_SMALL  # the small grid is the large grid's last 256 x 256 corner
    small = seeded(N_SMALL, 128.25, 127.75, storage)
    big = seeded(N_BIG, off + 128.25, off + 127.75, storage)
    for which in (lbmice.PHI, lbmice.U, lbmice.RHO, lbmice.UX, lbmice.UY):
        b = big.field(which)
        s = small.field(which)
        assert np.array_equal(b[off:, off:], s), which
        # the far side of the large grid stays the uniform state
        assert np.array_equal(b[:N_SMALL, :N_SMALL], np.full_like(s, s[0, 0])), which
        del b
    big.close()
    small.close()

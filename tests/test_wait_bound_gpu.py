"""The bounded device-side waits of the march (its phi ring arrives by TMA on an mbarrier):
a wait that cannot be satisfied gives up within about a second, the host reports it as
LBMICE_ETIMEOUT, and the context stays usable. The unsatisfiable wait is an mbarrier phase
that expects bytes no copy brings (nothing is in flight); no kernel faults or hangs."""
import time

import numpy as np
import pytest

from paper_2101_07163_gb300 import lbmice
from paper_2101_07163_gb300 import workloads as W

pytestmark = pytest.mark.gpu


def test_unsatisfiable_wait_gives_up_and_is_reported():
    pytest.importorskip("torch")
    lbmice.lib()
    t0 = time.perf_counter()
    assert lbmice.lib().lbmice_debug_wait_selftest() == lbmice.ETIMEOUT
    assert time.perf_counter() - t0 < 30.0


def test_context_usable_and_word_cleared_after_a_timeout():
    pytest.importorskip("torch")
    assert lbmice.lib().lbmice_debug_wait_selftest() == lbmice.ETIMEOUT
    # march steps with tensor maps, health checks every 6 steps (they read the wait word)
    w = W.Workload("wait", 256, 192, 1, flow=True, eps=0.05, D=2.0, U0=0.3, cx=128.0,
                   cy=96.0, R0=8.0)
    lat = lbmice.Lattice(w.nx, w.ny, check_every=6, **w.params())
    lat.init_seed(w.cx, w.cy, w.R0, w.U0)
    lat.step(12)
    s = lat.stats()
    assert s["nonfinite"] == 0.0
    assert np.isfinite(lat.field(lbmice.PHI)).all()
    lat.close()

"""The named workloads as data: every field survives a JSON round trip, unknown keys are
refused, and the module prints the named workloads as JSON."""
import json
import os
import subprocess
import sys

import pytest

from paper_2101_07163_gb300 import workloads as W


def test_every_workload_round_trips_through_json():
    ws = list(W.WORKLOADS.values()) + W.batch_sweep(count=12)
    for w in ws:
        back = W.Workload.from_dict(json.loads(json.dumps(w.to_dict())))
        assert back == w
        assert back.params() == w.params()
    assert set(W.named()) == set(W.WORKLOADS)


def test_unknown_workload_keys_are_refused():
    d = W.C1.to_dict()
    d["viscosity"] = 0.1
    with pytest.raises(ValueError):
        W.Workload.from_dict(d)


def test_module_prints_the_named_workloads():
    r = subprocess.run([sys.executable, "-m", "paper_2101_07163_gb300.workloads", W.C2.name],
                       capture_output=True, text=True, timeout=120,
                       cwd=os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
    assert r.returncode == 0, r.stderr
    d = json.loads(r.stdout)
    assert W.Workload.from_dict(d[W.C2.name]) == W.C2

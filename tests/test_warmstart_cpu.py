"""The committed warm-start weights and their training report (CPU)."""

import json
import os

import numpy as np

from paper_1908_08386_gb300 import workloads as WL

DATA = os.path.join(os.path.dirname(os.path.dirname(__file__)), "paper_1908_08386_gb300", "data")


def test_weights_have_the_network_shapes():
    z = np.load(os.path.join(DATA, "warmstart_128.npz"))
    widths = tuple(int(w) for w in z["widths"])
    shapes = [p.shape for p in WL.surrogate_init(widths)]
    got = [z["arr_%d" % i].shape for i in range(len(shapes))]
    assert got == shapes
    assert all(np.isfinite(z["arr_%d" % i]).all() for i in range(len(shapes)))
    assert 0.9e6 <= sum(int(np.prod(s)) for s in shapes) <= 1.1e6


def test_training_report_records_the_gain():
    r = json.load(open(os.path.join(DATA, "warmstart_128.json")))
    assert r["count"] == 2000 and r["train"] == 1800
    assert r["test_T_rms"] < r["rest_T_rms"] and r["test_u_rel_rms"] < r["rest_u_rel_rms"]
    assert sum(r["steps_warm_1e-06"]) < sum(r["steps_cold_1e-06"])

"""The seeded workload generators are reproducible within a process: the
object scene is cached, and every call must still draw the same view,
materials and environment (tests and the benchmark call it repeatedly)."""
import numpy as np

from paper_2510_07729_gb300 import inputs as I


def test_object_workload_same_on_every_call():
    a, b = I.make_object(), I.make_object()
    for k in ("x", "n", "wo", "albedo", "rough", "metal", "env", "probe_pos"):
        assert np.array_equal(a[k], b[k]), k
    assert len(a["x"]) == 418111


def test_tiny_workload_same_on_every_call():
    a, b = I.make_tiny(), I.make_tiny()
    for k in ("x", "albedo", "env", "probe_pos"):
        assert np.array_equal(a[k], b[k]), k
    for k in a["gauss"]:
        assert np.array_equal(a["gauss"][k], b["gauss"][k]), k

"""Host-side logic of bench.py that its JSON line rests on (CPU only):
the count of this library's launches a step, checked against the committed
ncu launch list of that step, and the DRAM traffic figure, which is reported
only for the workload it was captured on and only while the kernel's source
is the one it was captured from."""
import json
import os
import re
import shutil

import bench

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_launch_count_matches_the_recorded_launch_list():
    text = open(os.path.join(ROOT, "profiles", "launches_compose_step.md")).read()
    rows = re.findall(r"^\| `([^`]+)`[^|]*\| (\d+) \| [\d.]+ \| [\d.]+% \|$", text, flags=re.M)
    assert rows, "no kernel rows in the launch list"
    total = int(re.search(r"^\| \*\*all\*\* \| (\d+) \|", text, flags=re.M).group(1))
    assert sum(int(n) for _, n in rows) == total
    # the step: one bake and the frame's two queries
    assert bench.launches_per_step(True, 2) == total
    assert bench.launches_per_step(False, 1) == 7


def test_traffic_only_for_its_workload_and_source(tmp_path):
    tab = json.load(open(os.path.join(ROOT, "profiles", "traffic.json")))
    e = tab["trace_kernel"]
    want = e["bytes"]
    # a copy of the tree's two inputs of the lookup
    (tmp_path / "profiles").mkdir()
    shutil.copy(os.path.join(ROOT, "profiles", "traffic.json"), tmp_path / "profiles" / "traffic.json")
    csrc = tmp_path / "paper_2510_07729_gb300" / "csrc"
    csrc.mkdir(parents=True)
    src = os.path.join(ROOT, "paper_2510_07729_gb300", "csrc", e["source"])
    shutil.copy(src, csrc / e["source"])
    old_root = bench.ROOT
    try:
        bench.ROOT = str(tmp_path)
        same = bench.traffic_for("trace_kernel", e["workload"], e["probes"])
        other_workload = bench.traffic_for("trace_kernel", "object", e["probes"])
        other_size = bench.traffic_for("trace_kernel", e["workload"], e["probes"] // 2)
        unknown = bench.traffic_for("shade_kernel", e["workload"], e["probes"])
        with open(csrc / e["source"], "a") as f:
            f.write("\n// changed\n")
        changed = bench.traffic_for("trace_kernel", e["workload"], e["probes"])
    finally:
        bench.ROOT = old_root
    # the committed figure belongs to the committed source (or is withheld)
    assert same in (want, None)
    assert same == bench.traffic_for("trace_kernel", e["workload"], e["probes"])
    assert other_workload is None and other_size is None and unknown is None
    assert changed is None

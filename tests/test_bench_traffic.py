"""bench.py's traffic lookup: the ncu DRAM bytes of profiles/kv_step_traffic.json
are reported only for the grid, operator, medium encoding and step-kernel
configuration they were captured on, averaged over force and plain steps like
the roofline's algorithmic bytes."""
import json
import os
import sys
from types import SimpleNamespace

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)
import bench  # noqa: E402

CAPTURES = json.load(open(os.path.join(ROOT, "profiles", "kv_step_traffic.json")))["captures"]


def workload(n_steps=2000):
    return SimpleNamespace(nx=256, ny=256, nz=256, n_steps=n_steps)


def test_every_capture_is_found_for_its_own_configuration():
    for c in CAPTURES:
        w = SimpleNamespace(nx=c["grid"][0], ny=c["grid"][1], nz=c["grid"][2], n_steps=2000)
        t = bench.step_traffic(w, c["step_config"], c["operator"], 79, c.get("medium", "fields"))
        want = (79 * c["bytes_force_step"] + 1921 * c["bytes_plain_step"]) / 2000
        assert t == want


def test_no_traffic_for_another_encoding_grid_or_configuration():
    cls = [c for c in CAPTURES if c.get("medium") == "classes"]
    fld = [c for c in CAPTURES if c.get("medium", "fields") == "fields"]
    assert cls and fld
    cfg = dict(cls[0]["step_config"])
    if not any(c["step_config"] == cfg for c in fld):
        assert bench.step_traffic(workload(), cfg, "pointwise", 79, "fields") is None
    assert bench.step_traffic(workload(), cfg, "divergence", 79, "classes") is None
    assert bench.step_traffic(SimpleNamespace(nx=128, ny=256, nz=256, n_steps=2000), cfg, "pointwise", 79,
                              "classes") is None
    cfg["zc"] = 5
    assert bench.step_traffic(workload(), cfg, "pointwise", 79, "classes") is None


def test_class_captures_move_fewer_bytes_than_field_captures():
    def per_node(c):
        return c["bytes_plain_step"] / float(c["grid"][0] * c["grid"][1] * c["grid"][2])
    single = [c for c in CAPTURES if c["step_config"]["variant"] == 0]  # one step per launch
    cls = [per_node(c) for c in single if c.get("medium") == "classes"]
    fld = [per_node(c) for c in single if c.get("medium", "fields") == "fields"]
    # 49 instead of 56 algorithmic bytes per node: at least 8 % less DRAM traffic
    assert max(cls) < 0.92 * min(fld)


def test_scaled_capture_of_a_smaller_case():
    """A capture marked scale_by_cells (a smaller grid of the same workload
    family and kernel configuration) is scaled by the cell count and labelled;
    another family or configuration finds none."""
    caps = [c for c in CAPTURES if c.get("scale_by_cells")]
    assert caps
    c = caps[0]
    big = SimpleNamespace(nx=512, ny=512, nz=384, n_steps=5000, family=c["family"])
    scale = 512 * 512 * 384 / float(c["grid"][0] * c["grid"][1] * c["grid"][2])
    t, src = bench.step_traffic(big, c["step_config"], c["operator"], 118, c["medium"], with_source=True)
    want = scale * (118 * c["bytes_force_step"] + 4882 * c["bytes_plain_step"]) / 5000
    assert t == want and "scaled by the cell count" in src
    other = SimpleNamespace(nx=512, ny=512, nz=384, n_steps=5000, family="inclusions")
    assert bench.step_traffic(other, c["step_config"], c["operator"], 118, c["medium"]) is None
    cfg = dict(c["step_config"], tx=128)
    assert bench.step_traffic(big, cfg, c["operator"], 118, c["medium"]) is None

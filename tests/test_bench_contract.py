"""Host logic of bench.py (CPU only): the roofline objects carry the keys of the
bench line's contract, the dominant kernel is the one with the largest device
time, and the node-sample counts follow the workload's geometry."""
import os
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def test_roofline_objects_and_dominant_kernel():
    import bench
    from paper_2608_22190_b300 import _lib as L
    from paper_2608_22190_b300 import workloads as W
    wl = W.w2()
    steps, events = 2, 1.045e11
    st = {"walk_ms": 2054.0, "fill_ms": 3528.0, "eval_ms": 4450.0, "eval_launches": 288}
    roof, kern = bench.sweep_roofline(wl, L.MIXED, events, st, {}, steps, 5023.0)
    assert set(kern) == {"walk_count", "walk_fill", "eval_tc"}
    for v in kern.values():
        for key in ("bound", "achieved", "peak", "unit", "frac", "traffic"):
            assert key in v
        assert abs(v["frac"] - v["achieved"] / v["peak"]) < 1e-12
    assert roof["kernel"] == "eval_tc" and roof["bound"] == "tensor" and roof["unit"] == "TFLOP/s"
    # 4608 algorithmic flops per event over the evaluation's device time
    assert abs(roof["achieved"] - events * 4608 / 4.450 / 1e12) < 1e-9 * roof["achieved"]
    assert abs(roof["share_of_step"] - (4450.0 / steps) / 5023.0) < 1e-12
    # fallback peaks when no measured peaks file is present
    assert "fallback" in roof["peak_source"]


def test_node_samples_follow_the_geometry():
    import bench
    from paper_2608_22190_b300 import workloads as W
    wl = W.w2()
    # 24 x 24 nodes x 15 sampled time nodes (16 LGL, the first is the hand-off) x M x K
    assert bench.node_samples_per_interval(wl, 0) == 24 * 24 * 15 * 65536 * 8
    assert bench.node_samples_per_solve(wl) == 20 * 24 * 24 * 15 * 65536 * 8

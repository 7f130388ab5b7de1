"""The event sweep's per-node sums are exact (each term rounded once to a
fixed-point integer, integer atomics), so an iteration's result does not depend
on the order in which events reach their node: repeating it, or splitting the
samples into different batches, gives bitwise identical nodal values."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def api():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2608_22190_b300 import api as A
    return A


@pytest.mark.parametrize("precision,sweep", [(0, "events"), (1, "events"), (1, "events_alu")])
def test_event_sweep_is_bitwise_reproducible(api, precision, sweep):
    from paper_2608_22190_b300 import workloads as W
    wl = W.w2(M=3000, K=1, n_space=12, degree=6, n_intervals=1, h=0.5)
    wl.n_ref = 40
    results = []
    for batch in (0, 0, 517):          # twice the automatic batch, then ragged batches of 517 samples
        plan = api.Plan.from_workload(wl, precision=precision)
        plan.set_sweep(sweep, batch)
        plan.begin_interval(0)
        plan.iterate(0, 2)
        results.append(plan.get_nodes(0, 0).cpu().numpy())
        plan.close()
    assert np.array_equal(results[0], results[1]), np.abs(results[0] - results[1]).max()
    assert np.array_equal(results[0], results[2]), np.abs(results[0] - results[2]).max()


def test_event_sweep_recovers_from_a_full_event_buffer(api):
    """A batch larger than the one that sized the event buffer aborts the
    iteration on the device (every later launch returns at once); the call grows
    the buffer and runs the iteration again.  The result and the point count
    equal those of a plan whose buffer was sized for the large batch from the
    start."""
    from paper_2608_22190_b300 import workloads as W
    wl = W.w2(M=4000, K=1, n_space=10, degree=5, n_intervals=1, h=0.5)
    wl.n_ref = 30
    out = []
    for small_first in (True, False):
        plan = api.Plan.from_workload(wl, precision=1)
        plan.begin_interval(0)
        if small_first:
            plan.set_sweep("events", 64)
            plan.iterate(0, 1)          # the buffer now holds a 64-sample batch plus a quarter
            plan.begin_interval(0)      # back to the first iterate; iterations count from 1 again
        plan.set_sweep("events", 4000)  # one batch of every sample
        p0 = plan.stats()["points"]
        plan.iterate(0, 2)
        out.append((plan.get_nodes(0, 0).cpu().numpy(), plan.stats()["points"] - p0))
        plan.close()
    assert np.array_equal(out[0][0], out[1][0])
    assert out[0][1] == out[1][1]


@pytest.mark.parametrize("precision", [0, 1])
def test_solve_as_graphs_matches_launch_by_launch(api, precision):
    """spmc_solve runs every interval after the first as one captured CUDA graph
    (hand-off and K iterations); the result equals the launch-by-launch solve
    bit for bit, and the graphs were really launched."""
    from paper_2608_22190_b300 import workloads as W
    wl = W.w2(M=1500, K=3, n_space=8, degree=4, n_intervals=3, h=0.4)
    wl.n_ref = 24
    out = {}
    for graphs in (True, False):
        plan = api.Plan.from_workload(wl, precision=precision)
        plan.set_graphs(graphs)
        flat = plan.solve()
        out[graphs] = (flat.cpu().numpy(), plan.stats()["graph_launches"])
        plan.close()
    assert out[True][1] == 2 and out[False][1] == 0
    assert np.array_equal(out[True][0], out[False][0])

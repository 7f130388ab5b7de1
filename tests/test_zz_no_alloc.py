"""spmc_iterate_static: the iteration entry point that allocates nothing.

Some callers cannot allocate device memory at the point of the call: code that
runs between the set-up of a real-time loop and its teardown, or a region whose
allocator policy forbids cudaMalloc (it can synchronise the device or fail once
memory is handed out up front).  spmc_iterate_static runs the same iteration as
spmc_iterate with the cohort sweep, with the sweep's scratch in a file-scope
device array.  This test calls both through the C-ABI on two identical plans,
for two consecutive iterations, and checks that

  - the nodal values agree bit for bit: both paths sum every walk in the same
    precision and reduce each (node, chunk) of samples in the same order; only
    the number of spatial nodes per block differs (one in the static path), which
    does not enter any sum, so a layout error in the static scratch (chunk sums
    against walk state) would show here;
  - the static call allocates nothing: the plan's own device memory and the
    device's free memory are the same before and after the two calls.

It lives in its own file so that it runs last."""
import ctypes as C

import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("precision", [0, 1])
def test_iterate_static_matches_iterate(precision):
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2608_22190_b300 import _lib as L
    from paper_2608_22190_b300 import workloads as W
    from paper_2608_22190_b300.api import Plan

    wl = W.w2(M=1500, K=2, n_space=6, degree=4, n_intervals=1, h=0.5)   # ragged last chunk
    wl.n_ref = 12
    ref = Plan.from_workload(wl, precision=precision)
    ref.set_sweep("cohort")      # the static entry point runs the cohort kernel
    sta = Plan.from_workload(wl, precision=precision)
    sp = C.c_void_p(torch.cuda.current_stream().cuda_stream)
    ref.begin_interval(0)
    sta.begin_interval(0)
    S = wl.n_space ** 2
    Mt = int(wl.instances[0].degrees[0])
    outs = {k: [torch.empty((Mt + 1) * S, dtype=torch.float64, device="cuda") for _ in range(2)]
            for k in ("ref", "sta")}
    eps = {"ref": [], "sta": [], "points": []}
    for call in range(2):
        e = C.c_double()
        L.check(L.lib.spmc_iterate(ref._h, sp, 0, 1, C.byref(e)), ref._h)
        ref.get_nodes_into(0, 0, outs["ref"][call])
        eps["ref"].append(e.value)
        eps["points"].append(ref.stats()["points"])
    torch.cuda.synchronize()
    # the static calls alone: nothing else allocates between the two readings
    ws0 = sta.stats()["workspace_bytes"]
    free0 = torch.cuda.mem_get_info()[0]
    for call in range(2):
        e = C.c_double()
        L.check(L.lib.spmc_iterate_static(sta._h, sp, 0, C.byref(e)), sta._h)
        sta.get_nodes_into(0, 0, outs["sta"][call])
        eps["sta"].append(e.value)
        st = sta.stats()
        assert st["points"] == eps["points"][call] and st["iterations_run"] == 1
        assert st["last_max_eps"] == e.value
    torch.cuda.synchronize()
    assert torch.cuda.mem_get_info()[0] == free0
    assert sta.stats()["workspace_bytes"] == ws0
    for call in range(2):
        a, b = outs["ref"][call].cpu().numpy(), outs["sta"][call].cpu().numpy()
        assert np.array_equal(a, b), (call, np.abs(a - b).max())
        assert eps["ref"][call] == eps["sta"][call]
    ref.close()
    sta.close()


def test_iterate_static_rejects_oversized_problems():
    """A problem whose chunk sums exceed the 16 MiB static scratch is refused with
    SPMC_ERR_UNSUPPORTED before any work is enqueued."""
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2608_22190_b300 import _lib as L
    from paper_2608_22190_b300 import workloads as W
    from paper_2608_22190_b300.api import Plan

    # 15 time nodes x 576 spatial nodes x 4096 chunks of 512 samples -> 283 MB of chunk sums
    wl = W.w2(M=512 * 4096, K=1, n_intervals=1)
    plan = Plan.from_workload(wl, precision=1)
    plan.begin_interval(0)
    e = C.c_double()
    st = L.lib.spmc_iterate_static(plan._h, C.c_void_p(torch.cuda.current_stream().cuda_stream), 0, C.byref(e))
    assert st == L.SPMC_ERR_UNSUPPORTED
    assert b"16 MiB" in L.lib.spmc_last_error(plan._h)
    plan.close()

"""spmc_iterate_static: the iteration entry point that allocates nothing.

Some callers cannot allocate device memory at the point of the call (a real-time
loop between its set-up and teardown, or a region whose allocator policy forbids
cudaMalloc because it would synchronise the device).  spmc_iterate_static runs
the same iteration as spmc_iterate with the sweep's scratch in a file-scope
device array.  This test calls both through the C-ABI on two identical plans and
checks that two consecutive iterations agree node by node within the FP64
parity tolerance of the other tests (they differ only in how samples are grouped
into chunk sums).  It lives in its own file so that it runs last."""
import ctypes as C

import numpy as np
import pytest

from tests.common import parity_tol

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
    stream = torch.cuda.current_stream()
    sp = C.c_void_p(stream.cuda_stream)
    ref.begin_interval(0)
    sta.begin_interval(0)
    for call in range(2):
        e_ref, e_sta = C.c_double(), C.c_double()
        L.check(L.lib.spmc_iterate(ref._h, sp, 0, 1, C.byref(e_ref)), ref._h)
        L.check(L.lib.spmc_iterate_static(sta._h, sp, 0, C.byref(e_sta)), sta._h)
        a = ref.get_nodes(0, 0).cpu().numpy()
        b = sta.get_nodes(0, 0).cpu().numpy()
        if precision == 0:
            tol = parity_tol(a)
        else:
            # FP32 sweep: the chunk sums group the same walks differently; the
            # per-walk values are identical, so only FP64 summation order differs
            tol = 1e-12 * np.maximum(np.abs(a), 1e-3 * np.abs(a).max())
        assert np.all(np.abs(a - b) <= tol), (call, np.abs(a - b).max())
        assert abs(e_ref.value - e_sta.value) <= 1e-12 * max(1.0, abs(e_ref.value))
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

"""Parity of the CUDA path (through the C-ABI) with the CPU oracle."""
import numpy as np
import pytest

from tests.common import oracle_spec, oracle_u0, parity_tol

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def api():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2608_22190_b300 import api as A
    return A


def _stepwise(O, api, wl, K, precision=0, sweep="events", batch=0):
    inst = wl.instances[0]
    plan = api.Plan.from_workload(wl, precision=precision)
    plan.set_sweep(sweep, batch)
    spec = oracle_spec(O, wl, inst)
    u0 = oracle_u0(O, wl, inst, spec)
    Mt = int(inst.degrees[0])
    U = np.tile(u0, (Mt + 1, 1)).copy()
    plan.begin_interval(0)
    out = []
    for k in range(K):
        plan.iterate(0, 1)
        g = plan.get_nodes(0, 0).cpu().numpy()
        O.iterate(spec, 0, inst.t_breaks[0], inst.t_breaks[1], Mt, U, k + 1, 1)
        out.append((g, U.copy()))
    plan.close()
    return out


SWEEPS = [("events", 0), ("events", 37), ("cohort", 0)]   # 37: ragged sample batches


@pytest.mark.parametrize("sweep,batch", SWEEPS)
def test_fp64_1d_radau_stepwise(O, api, sweep, batch):
    from paper_2608_22190_b300 import workloads as W
    wl = W.w1(M=300, K=3, n_space=6, degree=5)
    wl.n_ref = 12
    for g, r in _stepwise(O, api, wl, 3, sweep=sweep, batch=batch):
        assert np.all(np.abs(g - r) <= parity_tol(r)), np.abs(g - r).max()


@pytest.mark.parametrize("sweep,batch", SWEEPS)
def test_fp64_1d_ragged_chunks(O, api, sweep, batch):
    from paper_2608_22190_b300 import workloads as W
    wl = W.w1(M=2500, K=2, n_space=5, degree=3)   # chunks of 1024: the third one is partial
    wl.n_ref = 8
    for g, r in _stepwise(O, api, wl, 2, sweep=sweep, batch=batch):
        assert np.all(np.abs(g - r) <= parity_tol(r)), np.abs(g - r).max()


@pytest.mark.parametrize("sweep,batch", SWEEPS)
def test_fp64_2d_stepwise(O, api, sweep, batch):
    from paper_2608_22190_b300 import workloads as W
    wl = W.w2(M=200, K=2, n_space=5, degree=3, n_intervals=1, h=0.5)
    wl.n_ref = 10
    for g, r in _stepwise(O, api, wl, 2, sweep=sweep, batch=batch):
        assert np.all(np.abs(g - r) <= parity_tol(r)), np.abs(g - r).max()


def test_mixed_events_match_cohort(api):
    """Mixed precision: the event sweep (per-term FP64 sums) and the cohort
    sweep (per-walk FP32 sums) take the same walks and points; they agree to
    FP32 rounding of the walk sums."""
    from paper_2608_22190_b300 import workloads as W
    wl = W.w2(M=1024, K=1, n_space=8, degree=4, n_intervals=1, h=0.5)
    wl.n_ref = 16
    out = {}
    for sweep in ("events", "cohort"):
        plan = api.Plan.from_workload(wl, precision=1)
        plan.set_sweep(sweep)
        plan.begin_interval(0)
        U0 = plan.get_nodes(0, 0).cpu().numpy()
        plan.iterate(0, 1)
        out[sweep] = (plan.get_nodes(0, 0).cpu().numpy() - U0, plan.stats()["points"])
        plan.close()
    (ee, pe), (ec, pc) = out["events"], out["cohort"]
    assert pe == pc
    assert np.abs(ee - ec).max() <= 1e-5 * np.abs(ec).max(), np.abs(ee - ec).max()


def test_mixed_tensor_core_matches_alu(api):
    """d = 2 mixed: the tensor-core evaluation (3-term TF32 split, FP32
    accumulation) and the FP32-pipe evaluation see the same events; their eps
    agree within the split's error bound: 2^-20 relative per product times the
    size of the residual terms (|f_add| + |d_t u| + |Delta u| ~ 20) times the
    walk time (<= 1), i.e. 2e-5."""
    from paper_2608_22190_b300 import workloads as W
    wl = W.w2(M=2048, K=1, n_intervals=1)          # full 24 x 24 x 16 geometry
    out = {}
    for sweep in ("events", "events_alu"):
        plan = api.Plan.from_workload(wl, precision=1)
        plan.set_sweep(sweep)
        plan.begin_interval(0)
        U0 = plan.get_nodes(0, 0).cpu().numpy()
        plan.iterate(0, 1)
        out[sweep] = (plan.get_nodes(0, 0).cpu().numpy() - U0, plan.stats()["points"])
        plan.close()
    (et, pt), (ea, pa) = out["events"], out["events_alu"]
    assert pt == pa
    d = np.abs(et - ea).max()
    print("max |eps_tc - eps_alu| =", d, "max |eps| =", np.abs(ea).max())
    assert d <= 2e-5, d


def test_fp64_1d_multi_interval_solve(O, api):
    """spmc_solve over three LGL intervals with the hand-off of Step 4."""
    from paper_2608_22190_b300 import workloads as W
    wl = W.w2(M=256, K=2, n_space=7, degree=4, n_intervals=3, h=0.3)
    wl.dim = 1
    wl.n_ref = 10
    inst = wl.instances[0]
    plan = api.Plan.from_workload(wl)
    flat = plan.solve()
    blocks = [b.cpu().numpy() for b in plan.blocks(flat, 0)]
    spec = oracle_spec(O, wl, inst)
    ref, _ = O.solve(spec, inst.t_breaks, inst.degrees, wl.K, oracle_u0(O, wl, inst, spec))
    for g, r in zip(blocks, ref):
        assert np.all(np.abs(g - r) <= parity_tol(r)), np.abs(g - r).max()
    plan.close()


def test_fp64_batch_uneven_instances(O, api):
    """Several instances with different interval counts, degrees and reaction
    scales in one plan (the batched launch of the initial-singularity workload)."""
    from paper_2608_22190_b300 import workloads as W
    wl = W.w3(M=256, K=2, batch=3, n_space=6)
    wl.n_ref = 10
    for b, inst in enumerate(wl.instances):
        n = 2 + b
        inst.t_breaks = W.geometric_mesh(1.0, n)
        inst.degrees = np.array([2 + 2 * k for k in range(n)])
    plan = api.Plan.from_workload(wl)
    flat = plan.solve()
    for b, inst in enumerate(wl.instances):
        blocks = [x.cpu().numpy() for x in plan.blocks(flat, b)]
        spec = oracle_spec(O, wl, inst, instance=b)
        ref, _ = O.solve(spec, inst.t_breaks, inst.degrees, wl.K, oracle_u0(O, wl, inst, spec))
        for g, r in zip(blocks, ref):
            assert np.all(np.abs(g - r) <= parity_tol(r)), (b, np.abs(g - r).max())
    plan.close()


def test_w2_geometry_sampled_nodes(O, api):
    """The long-time 2-D workload's full node geometry (24 x 24 JG x 16 LGL, h = 1):
    eps of the first iteration at sampled nodes, recomputed by the oracle one by one."""
    from paper_2608_22190_b300 import workloads as W
    wl = W.w2(M=256, K=1, n_intervals=1)
    inst = wl.instances[0]
    plan = api.Plan.from_workload(wl)
    plan.begin_interval(0)
    U0 = plan.get_nodes(0, 0).cpu().numpy()
    plan.iterate(0, 1)
    U1 = plan.get_nodes(0, 0).cpu().numpy()
    spec = oracle_spec(O, wl, inst)
    u0 = oracle_u0(O, wl, inst, spec)
    Mt = int(inst.degrees[0])
    U = np.tile(u0, (Mt + 1, 1))
    cu, ct = O.reconstruct(spec, Mt, 1.0, U)
    rng = np.random.default_rng(5)
    for _ in range(4):
        l = int(rng.integers(1, Mt + 1))
        j = int(rng.integers(0, wl.n_space ** 2))
        e = O.node_eps(spec, Mt, 0.0, 1.0, cu, ct, j, l, interval=0, iteration=1)
        ref = U0[l, j] + e
        assert abs(U1[l, j] - ref) <= parity_tol(U1)[l, j], (l, j, U1[l, j] - ref)
    plan.close()


@pytest.mark.parametrize("precision,M,sweep", [(0, 2048, "events"), (1, 65536, "events"), (1, 65536, "events_alu"),
                                               (1, 8192, "cohort")])
def test_polynomial_fixed_point_full_size(api, precision, M, sweep):
    """At the 2-D long-time workload's full size (24 x 24 JG x 16 LGL; M = 65536 in
    the mixed launch configuration of the benchmark, fewer samples for the FP64
    path), an exactly representable solution
    u = (1+t+t^2) prod (1-x_e^2)(1+x_e) has a zero residual everywhere, so one
    iteration from its nodal values leaves every node unchanged."""
    import scipy.special as sps
    from paper_2608_22190_b300 import workloads as W
    wl = W.w2(M=M, K=1, n_intervals=1)
    inst = wl.instances[0]
    inst.ex_kind = W.EX_POLY
    inst.f_kind = W.F_SIN
    plan = api.Plan.from_workload(wl, precision=precision)
    plan.set_sweep(sweep)
    grid = plan.node_grid()
    Mt = int(inst.degrees[0])
    xi = np.concatenate([[-1.0], sps.roots_jacobi(Mt - 1, 1.0, 1.0)[0], [1.0]])
    t = (xi + 1.0) * 0.5 * 1.0
    g = np.prod((1.0 - grid ** 2) * (1.0 + grid), axis=1)
    exact = (1.0 + t + t * t)[:, None] * g[None, :]
    plan.begin_interval(0)
    plan.set_nodes(0, 0, torch.from_numpy(exact))
    mx = plan.iterate(0, 1)
    # FP64: rounding of O(10) residual terms; mixed: FP32 evaluation of the same
    # terms (unit roundoff 6e-8 times |f_add| + |d_t u| + |Delta u| ~ 20, times the
    # walk time <= 1), averaged over the samples.  The tensor-core evaluation
    # (d = 2 mixed, "events") forms its products from a 3-term TF32 split: about
    # 2^-20 relative per product instead of 2^-24, so 16x the FP32 bound.
    tol = 1e-11 if precision == 0 else (3.2e-5 if sweep == "events" else 2e-6)
    assert mx < tol, mx
    after = plan.get_nodes(0, 0).cpu().numpy()
    assert np.abs(after - exact).max() < tol
    plan.close()


def test_fp64_5d_stepwise(O, api):
    """d = 5 (the 5-D workload's shape at 3 nodes per axis): stepwise parity."""
    from paper_2608_22190_b300 import workloads as W
    wl = W.w4(M=48, K=2, n_space=3, degree=2)
    wl.n_ref = 6
    for g, r in _stepwise(O, api, wl, 2):
        assert np.all(np.abs(g - r) <= parity_tol(r)), np.abs(g - r).max()


@pytest.mark.parametrize("precision,tol", [(0, 1e-11), (1, 1e-4)])
def test_5d_polynomial_fixed_point_full_geometry(api, precision, tol):
    """The 5-D workload's full node geometry (8^5 JG x 8 LGL): an exactly
    representable solution is a fixed point (eps = 0 at every node)."""
    import scipy.special as sps
    from paper_2608_22190_b300 import workloads as W
    wl = W.w4(M=32, K=1)
    inst = wl.instances[0]
    inst.ex_kind = W.EX_POLY
    plan = api.Plan.from_workload(wl, precision=precision)
    grid = plan.node_grid()
    Mt = int(inst.degrees[0])
    xi = np.concatenate([[-1.0], sps.roots_jacobi(Mt - 1, 1.0, 1.0)[0], [1.0]])
    t = (xi + 1.0) * 0.5 * 0.5
    g = np.prod((1.0 - grid ** 2) * (1.0 + grid), axis=1)
    exact = (1.0 + t + t * t)[:, None] * g[None, :]
    plan.begin_interval(0)
    plan.set_nodes(0, 0, torch.from_numpy(exact))
    mx = plan.iterate(0, 1)
    assert mx < tol, mx
    plan.close()

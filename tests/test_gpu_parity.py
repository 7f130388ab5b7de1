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
    wl = W.w4(M=8 if precision == 0 else 32, K=1)   # the FP64 pipe is slow on B300: fewer samples
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


@pytest.mark.parametrize("dim,n,Mt", [(1, 6, 6), (2, 5, 4)])
def test_fp64_literal_walk_stepwise(O, api, dim, n, Mt):
    """The fixed-radius walk with centre-point evaluations (walk_mode 1: Lemma
    Xlocation, Eqs. indexL, interIQ as printed) on a problem where it is stable
    (h = 0.5, N_* = 20): stepwise FP64 parity with the oracle's literal walk."""
    from paper_2608_22190_b300 import _lib as L
    from paper_2608_22190_b300 import workloads as W
    wl = W.w1(M=400, K=3, n_space=n, degree=Mt) if dim == 1 else W.w2(M=300, K=3, n_space=n, degree=Mt,
                                                                        n_intervals=1, h=0.5)
    if dim == 1:
        wl.instances[0].t_breaks = np.array([0.0, 0.5])
    wl.n_ref = 20
    inst = wl.instances[0]
    plan = api.Plan.from_workload(wl, precision=0, walk_mode=L.WALK_FIXED)
    spec = oracle_spec(O, wl, inst, walk_mode=1, n_sub=1)
    u0 = oracle_u0(O, wl, inst, spec)
    U = np.tile(u0, (Mt + 1, 1)).copy()
    plan.begin_interval(0)
    t0, t1 = inst.t_breaks[0], inst.t_breaks[1]
    for k in range(3):
        plan.iterate(0, 1)
        g = plan.get_nodes(0, 0).cpu().numpy()
        O.iterate(spec, 0, t0, t1, Mt, U, k + 1, 1)
        assert np.all(np.abs(g - U) <= parity_tol(U)), (k, np.abs(g - U).max())
    plan.close()


def test_mixed_eps_matches_oracle_at_benchmark_geometry(O, api):
    """The benchmark's mixed path (FP32 walks, tensor-core TF32-split evaluation,
    exact FP64 sums) against the FP64 oracle node by node, on the 2-D long-time
    workload's full geometry (24 x 24 JG x 16 LGL, h = 1, N_ref = 160) at M = 2048:
    eps of the first iteration at sampled nodes.  The two differ by FP32 rounding
    of the walk and of the evaluation (about 1e-6 of the terms) and by walks whose
    discrete decisions (absorption, ball kind, sub-step count) flip between FP32
    and FP64 positions; a flipped walk moves eps by at most max|Q| / M.  The GPU
    FP64 path, which matches the oracle to 1e-12, gives the number of evaluation
    events, whose difference from the mixed path's bounds the flips' effect."""
    from paper_2608_22190_b300 import workloads as W
    wl = W.w2(M=2048, K=1, n_intervals=1)
    inst = wl.instances[0]
    runs = {}
    for prec in (1, 0):
        plan = api.Plan.from_workload(wl, precision=prec)
        plan.begin_interval(0)
        U0 = plan.get_nodes(0, 0).cpu().numpy()
        p0 = plan.stats()["points"]
        plan.iterate(0, 1)
        U1 = plan.get_nodes(0, 0).cpu().numpy()
        runs[prec] = (U1 - U0, plan.stats()["points"] - p0, U0, U1)
        plan.close()
    eps_mx, pts_mx, _, _ = runs[1]
    eps_64, pts_64, U0, U1 = runs[0]
    tol64 = parity_tol(U1)
    spec = oracle_spec(O, wl, inst)
    u0 = oracle_u0(O, wl, inst, spec)
    Mt = int(inst.degrees[0])
    cu, ct = O.reconstruct(spec, Mt, 1.0, np.tile(u0, (Mt + 1, 1)))
    rng = np.random.default_rng(12)
    scale = np.abs(eps_64).max()
    worst = 0.0
    for _ in range(5):
        l = int(rng.integers(1, Mt + 1))
        j = int(rng.integers(0, wl.n_space ** 2))
        ref = O.node_eps(spec, Mt, 0.0, 1.0, cu, ct, j, l, interval=0, iteration=1)
        assert abs(U1[l, j] - (U0[l, j] + ref)) <= tol64[l, j]   # the FP64 path is the oracle's
        worst = max(worst, abs(eps_mx[l, j] - ref))
    d_all = np.abs(eps_mx - eps_64).max()
    print(f"mixed vs oracle at sampled nodes: {worst:.3e}; mixed vs FP64 (all nodes): {d_all:.3e}; "
          f"max|eps| {scale:.3e}; evaluation events mixed {pts_mx} vs FP64 {pts_64}")
    # Rounding: a relative 2^-20 per TF32-split product and 2^-24 per FP32 step,
    # over terms whose magnitudes sum to at most ~0.2 per walk here (|r| <= 20
    # times weights <= Delta = 1/160, a dozen terms): 1e-6 with a wide margin
    # (measured 1e-8).  A walk whose discrete decision flips between the FP32 and
    # FP64 positions changes its Q by at most about 0.1, i.e. 5e-5 at M = 2048.
    # Flips are rare: the evaluation counts of the two paths may differ by at
    # most one in a million (measured 9 of 2.0e8), so allow one flipped walk at a
    # sampled node and three at the worst node overall.
    assert abs(pts_mx - pts_64) <= 1e-6 * pts_64, (pts_mx, pts_64)
    assert worst <= 1e-6 + 5e-5, worst
    assert d_all <= 1e-6 + 3 * 5e-5, d_all


def test_fp64_batch_full_size_sampled_instances(O, api):
    """The initial-singularity batch at its full size (256 instances with 8-16
    geometric intervals, degrees 4 + 2k, M = 32768) in one plan, FP64: the first
    iteration of intervals 1 and 2 (the second after the hand-off of Algorithm 1,
    Step 4) at sampled nodes of two sampled instances, each recomputed by the
    oracle from that instance's first iterate on the same Philox streams."""
    from paper_2608_22190_b300 import workloads as W
    wl = W.w3()
    plan = api.Plan.from_workload(wl, precision=0)
    rng = np.random.default_rng(31)
    picks = [int(b) for b in rng.choice(len(wl.instances), 2, replace=False)]
    for r in (0, 1):
        plan.begin_interval(r)
        U0 = {b: plan.get_nodes(b, r).cpu().numpy() for b in picks}
        plan.iterate(r, 1)
        for b in picks:
            inst = wl.instances[b]
            U1 = plan.get_nodes(b, r).cpu().numpy()
            spec = oracle_spec(O, wl, inst, instance=b)
            Mt = int(inst.degrees[r])
            t0, h = float(inst.t_breaks[r]), float(inst.t_breaks[r + 1] - inst.t_breaks[r])
            cu, ct = O.reconstruct(spec, Mt, h, U0[b])
            tol = parity_tol(U1)
            for _ in range(2):
                l = int(rng.integers(1, Mt + 1))
                j = int(rng.integers(0, wl.n_space))
                e = O.node_eps(spec, Mt, t0, h, cu, ct, j, l, interval=r, iteration=1)
                assert abs(U1[l, j] - (U0[b][l, j] + e)) <= tol[l, j], (r, b, l, j, U1[l, j] - U0[b][l, j] - e)
    plan.close()


@pytest.mark.parametrize("precision", [0, 1])
def test_sharded_iterations_equal_unsharded(api, precision):
    """The node-sharded iteration on one GPU, shard after shard (three ranks'
    shares run in turn, no rank waits on another), then one application of the
    assembled eps: bit for bit the unsharded iteration, twice in a row."""
    from paper_2608_22190_b300 import workloads as W
    wl = W.w2(M=900, K=2, n_space=7, degree=4, n_intervals=1, h=0.5)
    wl.n_ref = 16
    ref = api.Plan.from_workload(wl, precision=precision)
    shd = api.Plan.from_workload(wl, precision=precision)
    ref.begin_interval(0)
    shd.begin_interval(0)
    n = shd.round_nodes(0)
    assert n == 4 * 49
    for _ in range(2):
        e_ref = ref.iterate(0, 1)
        eps = torch.zeros(n, dtype=torch.float64, device="cuda")
        for rank in range(3):
            shd.iterate_shard(0, rank, 3, eps)
        e_shd = shd.apply_eps(0, eps)
        assert np.array_equal(ref.get_nodes(0, 0).cpu().numpy(), shd.get_nodes(0, 0).cpu().numpy())
        assert e_ref == e_shd
    ref.close()
    shd.close()


@pytest.mark.parametrize("n,Mt,M", [(4, 3, 96), (8, 7, 8)])
def test_5d_tensor_core_events_match_cohort_and_oracle(O, api, n, Mt, M):
    """d = 5, mixed: the event sweep with the tensor-core evaluation (stage 1 of
    the sum-factorised contraction as a tcgen05 TF32 product, 3-term split)
    against the cohort kernel (FP32 pipe) on the same walks, and against the
    FP64 oracle at sampled nodes.  The walks and their points are the same; eps
    differ by FP32 / TF32-split rounding of terms whose magnitudes sum to about
    |f_add| + |d_t u| + |Delta u| ~ 30 over a walk time <= 0.5: 2^-20 x 15 ~ 2e-5.
    n = 8 is the 5-D workload's full geometry (8^5 nodes x 8 LGL)."""
    from paper_2608_22190_b300 import workloads as W
    wl = W.w4(M=M, K=1, n_space=n, degree=Mt)
    wl.n_ref = 16
    inst = wl.instances[0]
    out = {}
    for sweep in ("events", "cohort"):
        plan = api.Plan.from_workload(wl, precision=1)
        plan.set_sweep(sweep)
        plan.begin_interval(0)
        U0 = plan.get_nodes(0, 0).cpu().numpy()
        p0 = plan.stats()["points"]
        plan.iterate(0, 1)
        out[sweep] = (plan.get_nodes(0, 0).cpu().numpy() - U0, plan.stats()["points"] - p0, U0)
        plan.close()
    (ee, pe, U0), (ec, pc, _) = out["events"], out["cohort"]
    d = np.abs(ee - ec).max()
    print(f"n={n}: max|eps_tc - eps_cohort| = {d:.3e}, max|eps| = {np.abs(ec).max():.3e}, points {pe} / {pc}")
    assert pe == pc
    assert d <= 2e-5, d
    if n == 4:
        spec = oracle_spec(O, wl, inst)
        cu, ct = O.reconstruct(spec, Mt, 0.5, np.ascontiguousarray(U0))
        rng = np.random.default_rng(8)
        for _ in range(3):
            l = int(rng.integers(1, Mt + 1))
            j = int(rng.integers(0, n ** 5))
            ref = O.node_eps(spec, Mt, 0.0, 0.5, cu, ct, j, l, interval=0, iteration=1)
            assert abs(ee[l, j] - ref) <= 2e-5, (l, j, ee[l, j], ref)


@pytest.mark.parametrize("dim,sweep", [(1, "events"), (1, "cohort"), (2, "events")])
def test_fp64_aitken_stepwise(O, api, dim, sweep):
    """Aitken relaxation (u += omega eps, the factor from the last two residuals,
    per instance, in [1/2, 2]): four iterations in FP64 against the oracle's
    relaxed iteration on the same streams."""
    from paper_2608_22190_b300 import workloads as W
    wl = W.w1(M=400, K=4, n_space=6, degree=5) if dim == 1 else W.w2(M=300, K=4, n_space=5, degree=3,
                                                                        n_intervals=1, h=0.5)
    wl.n_ref = 12
    inst = wl.instances[0]
    Mt = int(inst.degrees[0])
    plan = api.Plan.from_workload(wl, precision=0)
    plan.set_sweep(sweep)
    plan.set_acceleration("aitken")
    spec = oracle_spec(O, wl, inst)
    U = np.tile(oracle_u0(O, wl, inst, spec), (Mt + 1, 1)).copy()
    st = O.AitkenState(spec, Mt)
    plan.begin_interval(0)
    for k in range(4):
        plan.iterate(0, 1)
        O.iterate_aitken(spec, 0, inst.t_breaks[0], inst.t_breaks[1], Mt, U, st, k + 1, 1)
        g = plan.get_nodes(0, 0).cpu().numpy()
        assert np.all(np.abs(g - U) <= parity_tol(U)), (k, np.abs(g - U).max())
    plan.close()

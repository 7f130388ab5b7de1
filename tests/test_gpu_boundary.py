"""Non-homogeneous boundary data and the direct estimator on the GPU, against
the CPU oracle (Section 2.3's remark on non-homogeneous boundary conditions;
Section 2.2, Eq. Phi_ast)."""
import numpy as np
import pytest

from tests.common import oracle_spec, parity_tol

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def api():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2608_22190_b300 import api as A
    return A


def _workload(W, dim, n, Mt, M, ex_kind, bc_kind, h=0.5, f_kind=1, kappa=0.5, beta=0.5, n_ref=12):
    inst = W.Instance(t_breaks=np.array([0.0, h]), degrees=np.array([Mt]), f_kind=f_kind,
                      f_coef=(0, 0, 0, 0) if f_kind == 1 else (0, 0.5, 0, -1.0), ex_kind=ex_kind, ex_beta=beta,
                      bc_kind=bc_kind)
    return W.Workload("boundary-test", dim, n, W.TIME_LGL, M, 2, kappa=kappa, n_ref=n_ref, instances=[inst])


def _stepwise(O, api, wl, K, estimator=0, precision=0):
    """K iterations of the GPU plan and of the oracle from the same first iterate;
    returns [(gpu nodes, oracle nodes)] and the plan's solution at the end."""
    from paper_2608_22190_b300 import workloads as W
    inst = wl.instances[0]
    plan = api.Plan.from_workload(wl, precision=precision, estimator=estimator)
    spec = oracle_spec(O, wl, inst, estimator=estimator)
    grid = O.space_nodes_grid(spec)
    u0 = W.u0_nodal(inst, grid)
    G0 = np.array([O.lift(spec, p, 0.0)[0] for p in grid])
    Mt = int(inst.degrees[0])
    U = np.tile(u0 - G0, (Mt + 1, 1)).copy()
    plan.begin_interval(0)
    first = plan.get_nodes(0, 0).cpu().numpy()
    assert np.abs(first - U).max() <= 1e-14 * max(1.0, np.abs(U).max())   # w(., 0) = u0 - G(., 0) on the device
    out = []
    for k in range(K):
        plan.iterate(0, 1)
        O.iterate(spec, 0, inst.t_breaks[0], inst.t_breaks[1], Mt, U, k + 1, 1)
        out.append((plan.get_nodes(0, 0).cpu().numpy(), U.copy()))
    sol = plan.get_solution(0, 0).cpu().numpy()
    plan.close()
    return out, sol, spec, grid


@pytest.mark.parametrize("dim,n,Mt,M", [(1, 8, 5, 400), (2, 6, 4, 64)])
def test_fp64_lifted_residual_iteration_stepwise(O, api, dim, n, Mt, M):
    """Residual iteration on w = u - G (lifted boundary data of kind 4, f = sin u):
    every iterate equals the oracle's to FP64 rounding, and the solution output
    adds the lifting at the nodes."""
    from paper_2608_22190_b300 import workloads as W
    wl = _workload(W, dim, n, Mt, M, W.EX_COSTHIRD, W.BC_LIFT)
    out, sol, spec, grid = _stepwise(O, api, wl, 2)
    for g, r in out:
        assert np.all(np.abs(g - r) <= parity_tol(r)), np.abs(g - r).max()
    xi, _ = O.lgl_nodes(Mt)
    tt = (xi + 1) * 0.5 * 0.5
    G = np.array([[O.lift(spec, p, t)[0] for p in grid] for t in tt])
    assert np.abs(sol - (out[-1][0] + G)).max() <= 1e-14


@pytest.mark.parametrize("dim,n,Mt,M,bc", [(1, 8, 4, 400, 2), (2, 6, 3, 64, 2), (2, 6, 3, 64, 1)])
def test_fp64_direct_estimator_stepwise(O, api, dim, n, Mt, M, bc):
    """The direct estimator S_i (Eq. Phi_ast): quadrature of the forcing, the
    initial term u*(X, t_{n-1}) of walks that reach t_{n-1} and, with raw
    boundary data (kind 5), g at the absorption point and time; with lifted
    data (kind 4) the boundary term vanishes.  Equal to the oracle's iterates to
    FP64 rounding."""
    from paper_2608_22190_b300 import workloads as W
    kind = W.EX_SINPLUS if bc == W.BC_RAW else W.EX_COSTHIRD
    wl = _workload(W, dim, n, Mt, M, kind, bc)
    out, sol, _, _ = _stepwise(O, api, wl, 2, estimator=1)
    for g, r in out:
        assert np.all(np.abs(g - r) <= parity_tol(r)), np.abs(g - r).max()
    if bc == W.BC_RAW:
        assert np.array_equal(sol, out[-1][0])   # raw data: the nodal values are u


def test_mixed_lifted_matches_oracle(O, api):
    """The mixed path (FP32 walks, tensor-core TF32-split evaluation, exact sums)
    on lifted boundary data, 2-D: after two iterations from the same start, within
    FP32 rounding of the FP64 oracle plus the rare walks whose discrete decisions
    flip between FP32 and FP64 positions (each moves a node by at most max|Q|/M)."""
    from paper_2608_22190_b300 import workloads as W
    wl = _workload(W, 2, 8, 4, 512, W.EX_COSTHIRD, W.BC_LIFT)
    out, _, _, _ = _stepwise(O, api, wl, 2, precision=1)
    for g, r in out:
        d = np.abs(g - r)
        # FP32 rounding of terms summing to ~|Q| <= 1 per walk: 1e-6; one flipped walk: 1 / 512
        assert d.max() <= 1e-6 + 2.0 / 512, d.max()
        assert np.median(d) <= 1e-5, np.median(d)


def test_lifted_2d_converges_to_the_closed_form(api):
    """Two intervals of the 2-D boundary-data workload (lifted, f = sin u, mixed):
    u = w + G at every node within 2e-5 of the closed form with non-zero
    boundary values."""
    from paper_2608_22190_b300 import workloads as W
    wl = W.w6(M=8192, K=8, n_space=16, degree=10, n_intervals=2)
    plan = api.Plan.from_workload(wl, precision=1)
    plan.solve()
    grid = plan.node_grid()
    for m in range(2):
        u = plan.get_solution(0, m).cpu().numpy()
        ex = W.exact_block(wl, wl.instances[0], grid, m)
        assert np.abs(u - ex).max() < 2e-5, (m, np.abs(u - ex).max())
    plan.close()


def test_boundary_options_are_checked(api):
    """Raw boundary data needs the direct estimator; boundary data and the direct
    estimator need the event sweep; kinds 4 and 5 need boundary data."""
    import ctypes as C
    from paper_2608_22190_b300 import _lib as L
    from paper_2608_22190_b300 import workloads as W
    wl = _workload(W, 1, 6, 3, 64, W.EX_SINPLUS, W.BC_RAW)
    with pytest.raises(L.SpmcError):
        api.Plan.from_workload(wl, precision=0)                 # raw data, residual iteration
    wl.instances[0].bc_kind = W.BC_ZERO
    with pytest.raises(L.SpmcError):
        api.Plan.from_workload(wl, precision=0, estimator=1)    # kind 5 with g = 0
    wl.instances[0].bc_kind = W.BC_RAW
    plan = api.Plan.from_workload(wl, precision=0, estimator=1)
    plan.set_sweep("cohort")
    with pytest.raises(L.SpmcError):
        plan.begin_interval(0)
    plan.set_sweep("events")
    plan.begin_interval(0)
    e = C.c_double()
    st = L.lib.spmc_iterate_static(plan._h, C.c_void_p(torch.cuda.current_stream().cuda_stream), 0, C.byref(e))
    assert st == L.SPMC_ERR_UNSUPPORTED
    plan.close()

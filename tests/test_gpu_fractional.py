"""The fractional case on the GPU (Section 4, Ex. 2): alpha-stable walk and
generalised Jacobi functions, against the CPU oracle."""
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


def _wl(W, alpha, kind, n=8, Mt=4, M=200, h=0.5, n_int=1):
    wl = W.w8(M=M, K=2, n_space=n, degree=Mt, alpha=alpha, h=h, T=h * n_int)
    wl.instances[0].ex_kind = kind
    return wl


def _stepwise(O, api, wl, K, precision=0):
    inst = wl.instances[0]
    plan = api.Plan.from_workload(wl, precision=precision)
    spec = oracle_spec(O, wl, inst, alpha=wl.alpha, walk_mode=2, n_sub=1)
    x = O.space_nodes_grid(spec)[:, 0]
    assert np.abs(plan.space_nodes() - x).max() < 1e-14   # Jacobi-Gauss (a,a) nodes on both sides
    Mt = int(inst.degrees[0])
    from paper_2608_22190_b300 import workloads as W
    U = np.tile(W.frac_exact(wl.alpha, inst.ex_kind, x, 0.0)[0], (Mt + 1, 1)).copy()
    plan.begin_interval(0)
    out = []
    for k in range(K):
        plan.iterate(0, 1)
        O.iterate(spec, 0, inst.t_breaks[0], inst.t_breaks[1], Mt, U, k + 1, 1)
        out.append((plan.get_nodes(0, 0).cpu().numpy(), U.copy()))
    plan.close()
    return out


@pytest.mark.parametrize("alpha", [0.4, 1.5])
def test_fp64_fractional_stepwise(O, api, alpha):
    """Two residual iterations of Ex. 2's problem (f = u - u^3) with the
    alpha-stable walk: every iterate equals the oracle's to FP64 rounding
    (same Philox words, jump law, exits and quadrature)."""
    from paper_2608_22190_b300 import workloads as W
    for g, r in _stepwise(O, api, _wl(W, alpha, W.EX_FRAC_SIN), 2):
        assert np.all(np.abs(g - r) <= parity_tol(r)), np.abs(g - r).max()


@pytest.mark.parametrize("precision,tol", [(0, 1e-12), (1, 2e-5)])
def test_fractional_fixed_point(api, precision, tol):
    """u = (1+t)(1-x^2)^a (1 + P_1^{(a,a)}/2) lies in the approximation space: one
    iteration from its nodal values moves no node (FP64: to rounding; mixed: to
    FP32 rounding of the slices and residual terms)."""
    from paper_2608_22190_b300 import workloads as W
    wl = _wl(W, 0.8, W.EX_FRAC_POLY, n=10, Mt=4, M=512)
    plan = api.Plan.from_workload(wl, precision=precision)
    x = plan.space_nodes()
    xi = W.time_nodes_reference(wl.time_family, 4)
    U = W.frac_exact(0.8, W.EX_FRAC_POLY, x, (xi + 1) * 0.5 * 0.5)
    plan.begin_interval(0)
    plan.set_nodes(0, 0, torch.tensor(U, dtype=torch.float64, device="cuda"))
    plan.iterate(0, 1)
    d = np.abs(plan.get_nodes(0, 0).cpu().numpy() - U).max()
    plan.close()
    assert d <= tol * np.abs(U).max(), d


def test_mixed_fractional_matches_oracle(O, api):
    """The mixed path (FP32 walk state and residuals, FP64 jump lengths and
    sums) against the oracle's FP64 iterates: FP32 rounding plus rare walks
    whose exit decision flips (each moves a node by at most max|Q| / M)."""
    from paper_2608_22190_b300 import workloads as W
    out = _stepwise(O, api, _wl(W, 1.2, W.EX_FRAC_SIN, M=1024), 2, precision=1)
    for g, r in out:
        d = np.abs(g - r)
        assert d.max() <= 1e-5 + 2 * 0.5 / 1024, d.max()
        assert np.median(d) <= 1e-5, np.median(d)


def test_fractional_converges_to_ex2_solution(api):
    """Ex. 2's problem at alpha = 1.2, two intervals of h = 0.5, mixed: the nodal
    values reach the closed form to 5e-4 (discretisation and sampling error)."""
    from paper_2608_22190_b300 import workloads as W
    wl = W.w8(M=4096, K=10, n_space=10, degree=6, alpha=1.2, h=0.5, T=1.0)
    plan = api.Plan.from_workload(wl, precision=1)
    plan.solve()
    x = plan.space_nodes()
    for m in range(2):
        xi = W.time_nodes_reference(wl.time_family, 6)
        t = 0.5 * m + (xi + 1) * 0.25
        ex = W.frac_exact(1.2, W.EX_FRAC_SIN, x, t)
        err = np.abs(plan.get_nodes(0, m).cpu().numpy() - ex).max()
        assert err < 5e-4, (m, err)
    plan.close()

"""The Chebyshev basis on the GPU (the remark on quasi-linear reconstruction
after Algorithm 1): CGL points, DCT-I reconstruction (through the FFT of the
even extension for power-of-two lengths), against the CPU oracle."""
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


def _stepwise(O, api, wl, K, precision=0):
    inst = wl.instances[0]
    plan = api.Plan.from_workload(wl, precision=precision)
    spec = oracle_spec(O, wl, inst)
    grid = O.space_nodes_grid(spec)
    assert np.abs(plan.node_grid() - grid).max() < 1e-15   # interior CGL points on both sides
    u0 = oracle_u0(O, wl, inst, spec)
    Mt = int(inst.degrees[0])
    U = np.tile(u0, (Mt + 1, 1)).copy()
    plan.begin_interval(0)
    out = []
    for k in range(K):
        plan.iterate(0, 1)
        O.iterate(spec, 0, inst.t_breaks[0], inst.t_breaks[1], Mt, U, k + 1, 1)
        out.append((plan.get_nodes(0, 0).cpu().numpy(), U.copy()))
    plan.close()
    return out


@pytest.mark.parametrize("dim,n,Mt", [(1, 6, 5), (1, 7, 8), (2, 7, 4), (2, 5, 6)])
def test_fp64_chebyshev_stepwise(O, api, dim, n, Mt):
    """Two iterations in the Chebyshev basis equal the oracle's to FP64 rounding;
    (n + 1, M) = (8, 8) and (8, 4) take the FFT transforms, (7, 5), (6, 6) the
    direct sums."""
    from paper_2608_22190_b300 import workloads as W
    base = W.w1(M=300, K=2, n_space=n, degree=Mt) if dim == 1 else W.w2(M=64, K=2, n_space=n, degree=Mt,
                                                                         n_intervals=1, h=0.5)
    wl = W.chebyshev(base)
    wl.n_ref = 12
    for g, r in _stepwise(O, api, wl, 2):
        # with n odd the middle node's exact value is 0: both sides hold rounding
        # noise of a few ulps of the largest values there
        assert np.all(np.abs(g - r) <= parity_tol(r) + 8e-15 * np.abs(r).max()), np.abs(g - r).max()


def test_mixed_chebyshev_matches_oracle(O, api):
    """The mixed path (FP32 walks and evaluation, exact sums) in the Chebyshev
    basis, 2-D, against the FP64 oracle after two iterations: FP32 rounding plus
    rare walks whose discrete decisions flip."""
    from paper_2608_22190_b300 import workloads as W
    wl = W.chebyshev(W.w2(M=512, K=2, n_space=8, degree=5, n_intervals=1, h=0.5))
    wl.n_ref = 20
    for g, r in _stepwise(O, api, wl, 2, precision=1):
        d = np.abs(g - r)
        assert d.max() <= 1e-5 + 2 * 0.2 / 512, d.max()
        assert np.median(d) <= 1e-5, np.median(d)


def test_chebyshev_converges_to_the_closed_form(api):
    """The 2-D long-time workload's first two intervals in the Chebyshev basis
    (16 CGL points per axis, degree 16 in time), mixed: every node within 2e-6
    of the closed form."""
    from paper_2608_22190_b300 import workloads as W
    wl = W.chebyshev(W.w2(M=8192, K=8, n_space=16, degree=16, n_intervals=2))
    plan = api.Plan.from_workload(wl, precision=1)
    plan.solve()
    grid = plan.node_grid()
    for m in range(2):
        err = np.abs(plan.get_nodes(0, m).cpu().numpy() - W.exact_block(wl, wl.instances[0], grid, m)).max()
        assert err < 2e-6, (m, err)
    plan.close()
